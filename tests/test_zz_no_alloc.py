"""bc_source_dependencies_noalloc: the allocation-free variant of the per-source
step, for callers that cannot allocate device memory themselves (their own
allocator owns the GPU's memory, or allocation calls are not allowed where they
run). The test allocates the input and output buffers itself (with torch) and
checks the entry point against the existing, allocating bc_source_dependencies
on the same inputs, for two calls in a row (the fixed scratch array is reused
and must be re-initialised by every call). The parity suite's bar applies:
exact equality of every double.

This file is collected last on purpose, so a failure here cannot stop a
run-to-first-failure before the rest of the suite has run."""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


def _device_buffers(torch, g, sources):
    d_rp = torch.as_tensor(g.row_ptr, dtype=torch.int32).cuda()
    d_col = torch.as_tensor(g.col if g.nnz else np.zeros(1, np.int32), dtype=torch.int32).cuda()
    d_src = torch.as_tensor(np.asarray(sources, np.int32)).cuda()
    d_out = torch.empty(len(sources) * g.n, dtype=torch.float64, device="cuda")
    return d_rp, d_col, d_src, d_out


@pytest.mark.parametrize("family", ["er2000", "rmat_s12_hubs", "ba3000"])
def test_noalloc_matches_allocating_entry_point(family):
    torch = pytest.importorskip("torch")
    import paper_1608_04472_gb300 as pkg
    from paper_1608_04472_gb300 import capi

    g = {"er2000": lambda: gg.erdos_renyi(2000, 8, 1),
         "rmat_s12_hubs": lambda: gg.rmat(12, 64, 0.57, 0.19, 0.19, 3),
         "ba3000": lambda: gg.barabasi_albert(3000, 3, 4)}[family]()
    sources = [0, 1, g.n // 3, g.n - 1, 0]
    with pkg.Context(0, batch_width=1) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col)
        ref, _, _ = ctx.source_dependencies(h, sources)

    d_rp, d_col, d_src, d_out = _device_buffers(torch, g, sources)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        d_out.fill_(-1.0)
        rc = capi.bc_source_dependencies_noalloc(0, d_rp.data_ptr(), d_col.data_ptr(), g.n, g.nnz,
                                                 d_src.data_ptr(), len(sources), d_out.data_ptr(), stream)
        assert rc == 0, f"call {call}: status {rc}"
        got = d_out.cpu().numpy().reshape(len(sources), g.n)
        assert np.array_equal(got, ref), f"call {call}: {np.sum(got != ref)} mismatches"
    # and, on its own footing, against the CPU oracle (Theorem 1 per source)
    import oracle
    for i, s in enumerate(sources):
        assert np.array_equal(got[i], oracle.dependencies(g, int(s))[0]), f"source {s}: differs from the oracle"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_1608_04472_gb300 import capi

    n = capi.BC_NOALLOC_MAX_VERTICES + 1
    d_rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    d_src = torch.zeros(1, dtype=torch.int32, device="cuda")
    d_out = torch.empty(n, dtype=torch.float64, device="cuda")
    rc = capi.bc_source_dependencies_noalloc(0, d_rp.data_ptr(), 0, n, 0, d_src.data_ptr(), 1,
                                             d_out.data_ptr(), 0)
    assert rc == -3  # BC_E_TOO_LARGE
    assert capi.bc_source_dependencies_noalloc(0, d_rp.data_ptr(), 0, 0, 0, d_src.data_ptr(), 1,
                                               d_out.data_ptr(), 0) == -1  # n < 1


def test_noalloc_reports_overflow_without_extended_form():
    torch = pytest.importorskip("torch")
    from paper_1608_04472_gb300 import capi

    g = gg.grid(40)  # counts from a corner exceed 2^64-1
    d_rp, d_col, d_src, d_out = _device_buffers(torch, g, [0])
    rc = capi.bc_source_dependencies_noalloc(0, d_rp.data_ptr(), d_col.data_ptr(), g.n, g.nnz,
                                             d_src.data_ptr(), 1, d_out.data_ptr(), 0)
    assert rc == -9  # BC_E_SIGMA_OVERFLOW


def test_noalloc_rejects_out_of_range_sources_on_the_device():
    """Sources live in device memory the host never reads: a source of n (or
    -1) must be refused by the kernel itself, touch no memory, leave its row as
    it was, and not stop the in-range sources."""
    torch = pytest.importorskip("torch")
    import paper_1608_04472_gb300 as pkg
    from paper_1608_04472_gb300 import capi

    g = gg.erdos_renyi(2000, 8, 1)
    sources = [3, g.n, 17, -1]
    with pkg.Context(0, batch_width=1) as ctx:
        h = ctx.load_graph(g.row_ptr, g.col)
        ref, _, _ = ctx.source_dependencies(h, [3, 17])
    d_rp, d_col, d_src, d_out = _device_buffers(torch, g, sources)
    d_out.fill_(-7.0)
    rc = capi.bc_source_dependencies_noalloc(0, d_rp.data_ptr(), d_col.data_ptr(), g.n, g.nnz,
                                             d_src.data_ptr(), len(sources), d_out.data_ptr(), 0)
    assert rc == -1  # BC_E_INVALID
    got = d_out.cpu().numpy().reshape(len(sources), g.n)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[2], ref[1])
    assert np.all(got[1] == -7.0) and np.all(got[3] == -7.0)
