"""GB300-native sampled betweenness centrality (Ji & Yan, arXiv 1608.04472).

The computation lives in ``libbcgb300.so`` (hand-written CUDA for sm_103a behind
the C ABI declared in ``include/bc.h``). This package is a thin ctypes binding:
it marshals numpy arrays and checks status codes, nothing else. Using any
binding name when the library has not been built raises ``ImportError``; there
is no CPU fallback. ``paper_1608_04472_gb300.build`` compiles the library.

Two layers are exported:

* ``capi`` -- one Python function per C entry point, same names
  (``bc_create``, ``bc_graph_load_csr``, ``bc_exact``, ...).
* ``Context`` -- a small object wrapper that owns a ``bc_ctx*`` and graph handles.
"""
import importlib

_EXPORTS = ("Context", "BCError", "capi", "BC_STOPPED", "BC_CAPPED", "BC_UNDIRECTED",
            "BC_VALIDATE", "BC_DIRECTED", "BC_NORMALIZE", "LIB_PATH", "BC_OK", "BC_PENDING", "BC_QUERY_SOURCES", "BC_QUERY_PAIRS",
            "BC_QUERY_UNIFORM")
__all__ = list(_EXPORTS)


def __getattr__(name):
    if name in _EXPORTS:
        mod = importlib.import_module(".capi", __name__)
        return getattr(mod, name)
    raise AttributeError(name)
