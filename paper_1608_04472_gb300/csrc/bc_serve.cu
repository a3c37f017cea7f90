// bc_serve.cu -- continuous-batching query server behind bc_submit / bc_poll /
// bc_cancel. One worker thread per context:
//   * admits queued queries FIFO while the active-slot limit and the device
//     memory budget allow (a pair query holds d(v,.) and sigma_v. for each of
//     its targets, n*T*12 bytes);
//   * picks a (graph, kind) group round-robin and fills one 64-lane batch with
//     the next draws of the group's active queries (each query's lanes
//     contiguous and in its own draw order);
//   * runs the batched Brandes step (sources; the weighted or lane-major
//     engine for graphs with lengths or direction) or the bidirectional pair
//     search (pairs), routes each lane's per-target values to its query, and runs each
//     query's sequential stop scan on the device (Sec. 4 step 3; Algorithm 1);
//   * writes a finished query's outputs into the caller's buffers.
// Because every query keeps its own draw stream and every sum is exact, a query's
// result is bit-identical whether it runs alone or mixed with others.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bc_internal.h"
#include "bc_xf.cuh"

namespace bcg {

void run_source_batch(bc_ctx *ctx, const Graph &g, int count, const Sink &sink);

namespace {

using Clock = std::chrono::steady_clock;

enum QState { Q_QUEUED = 0, Q_ACTIVE, Q_DONE, Q_CANCELLED, Q_FAILED };

struct SQuery {
  bc_ticket id = 0;
  int kind = 0;
  bc_graph gh = 0;
  Graph g;
  std::vector<int32_t> targets;
  double c = 1.0, scale = 1.0;
  int64_t cap = 0, kuni = 0;
  uint64_t seed = 0, qid = 0;
  double *est = nullptr;
  int64_t *k_out = nullptr;
  double *S_out = nullptr;
  int32_t *status_out = nullptr;
  bc_query_stats *stats_out = nullptr;
  // progress
  int64_t issued = 0;
  int32_t remaining = 0;
  int state = Q_QUEUED;
  bc_status result = BC_OK;
  std::string err;
  bool cancel = false;
  bool prepared = false;
  size_t mem = 0;
  DevBuf dstate;      // S[T] f64 | k[T] i64 | done[T] i32 | remaining i32
  DevBuf tdist, tsig; // pairs: [n][T]
  DevBuf dtarg, texp, dtx;  // pairs: targets on the device; extended-form exponents [n][T] and flags [T]
  std::vector<int32_t> tx;
  DevBuf acc;         // uniform: [n] Acc
  Clock::time_point t_submit, t_admit;
  int64_t samples = 0, batches = 0;

  int T() const { return (int)targets.size(); }
  double *S() const { return dstate.as<double>(); }
  int64_t *K() const { return reinterpret_cast<int64_t *>(dstate.as<char>() + 8 * (size_t)std::max(T(), 1)); }
  int32_t *Done() const { return reinterpret_cast<int32_t *>(dstate.as<char>() + 16 * (size_t)std::max(T(), 1)); }
  int32_t *Rem() const {
    return reinterpret_cast<int32_t *>(dstate.as<char>() + (20 * (size_t)std::max(T(), 1) + 15) / 16 * 16);
  }
  bool needs_draws() const {
    if (state != Q_ACTIVE || cancel) return false;
    if (kind == BC_QUERY_UNIFORM) return issued < kuni;
    return remaining > 0 && issued < cap;
  }
};

}  // namespace

struct LaneDraw {
  uint64_t seed, qid, i;
};

struct ScanEntry {
  double *S;
  int64_t *k;
  int32_t *done;
  int32_t *rem;
  int32_t j, a, c, pad;
  int64_t i0;
  double cn, scale;
};

struct PairEntry {
  const int32_t *tdist;
  const uint64_t *tsig;
  const int32_t *texp;  // null unless some target of the query is in the extended form
  const int32_t *tx;
  int32_t v, j, T, a, c, pad;
};

__global__ void k_draw_lanes(int count, const LaneDraw *__restrict__ ld, int32_t n, bool pairs,
                             int32_t *__restrict__ s_out, int32_t *__restrict__ t_out) {
  const int i = threadIdx.x;
  if (i >= count) return;
  if (pairs) {
    int32_t u, t;
    draw_pair(ld[i].seed, ld[i].qid, ld[i].i, n, u, t);
    s_out[i] = u;
    t_out[i] = t;
  } else {
    s_out[i] = draw_source(ld[i].seed, ld[i].qid, ld[i].i, n);
  }
}

__global__ void k_set_heads(int nh, const int32_t *__restrict__ hv, const int32_t *__restrict__ he,
                            int32_t *__restrict__ tslot) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nh) tslot[hv[i]] = he[i];
}

// Per-entry sequential stop scan over the entry's query lanes, in draw order.
__global__ void k_stop_scan_multi(int E, const ScanEntry *__restrict__ ent, const double *__restrict__ vals) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const ScanEntry d = ent[e];
  if (d.done[d.j]) return;
  double S = d.S[d.j];
  int64_t k = d.k[d.j];
  bool stop = false;
  for (int t = 0; t < d.c; ++t) {
    S = __dadd_rn(S, vals[(size_t)e * 64 + d.a + t]);
    k = d.i0 + t + 1;
    if (__dmul_rn(S, d.scale) > d.cn) {
      stop = true;
      break;
    }
  }
  d.S[d.j] = S;
  d.k[d.j] = k;
  if (stop) {
    d.done[d.j] = 1;
    atomicSub(d.rem, 1);
  }
}

__global__ void k_pair_values_multi(int E, const PairEntry *__restrict__ ent, const int32_t *__restrict__ ps,
                                    const int32_t *__restrict__ pt, const int32_t *__restrict__ pd,
                                    const uint64_t *__restrict__ psig, const int32_t *__restrict__ pexp,
                                    uint64_t pxmask, double *__restrict__ vals) {
  const int e = blockIdx.x, i = threadIdx.x;
  if (e >= E || i >= 64) return;
  const PairEntry d = ent[e];
  double y = 0.0;
  if (i >= d.a && i < d.a + d.c) {
    const int32_t v = d.v, s = ps[i], t = pt[i], dst = pd[i];
    const uint64_t sst = psig[i];
    if (v != s && v != t && sst != 0ull && dst >= 0) {
      const size_t is = (size_t)s * d.T + d.j, it = (size_t)t * d.T + d.j;
      const int32_t ds = d.tdist[is], dt = d.tdist[it];
      if (ds >= 0 && dt >= 0 && ds + dt == dst) {
        const bool vx = d.tx && d.tx[d.j], px = (pxmask >> i) & 1ull;
        if (vx || px) {
          y = pair_y(vx, d.tsig[is], vx ? d.texp[is] : 0, d.tsig[it], vx ? d.texp[it] : 0, px, sst, px ? pexp[i] : 0);
        } else {
          const double a = sigma_to_double(d.tsig[is]);
          const double b = sigma_to_double(d.tsig[it]);
          y = __ddiv_rn(__dmul_rn(a, b), sigma_to_double(sst));
        }
      }
    }
  }
  vals[(size_t)e * 64 + i] = y;
}

__global__ void k_gather_rem(int P, int32_t *const *__restrict__ rem, int32_t *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) out[i] = *rem[i];
}

__global__ void k_serve_finalize(int T, const double *__restrict__ S, const int64_t *__restrict__ k,
                                 const int32_t *__restrict__ done, double scale_n, double *__restrict__ est,
                                 int32_t *__restrict__ status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= T) return;
  est[j] = __ddiv_rn(__dmul_rn(scale_n, S[j]), (double)k[j]);
  status[j] = done[j] ? BC_STOPPED : BC_CAPPED;
}

__global__ void k_serve_finalize_uniform(int32_t n, const Acc *__restrict__ acc, double nd, double kd,
                                         double *__restrict__ out) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) out[v] = __ddiv_rn(__dmul_rn(nd, acc_round(acc[v])), kd);
}

struct Server {
  bc_ctx *ctx = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  std::unordered_map<bc_ticket, std::shared_ptr<SQuery>> queries;
  std::deque<std::shared_ptr<SQuery>> queued;
  std::vector<std::shared_ptr<SQuery>> active;
  bc_ticket next_ticket = 1;
  size_t rr = 0;
  int32_t max_active = 64;
  int64_t mem_budget = 0;
  int64_t mem_used = 0;
  // batch staging (worker only)
  DevBuf d_lane, d_laneq, d_enext, d_eq, d_heads, d_scan, d_pair, d_rem, d_tdelta, d_tslot, d_misc;

  void loop();
  void admit_locked();
  void yield_to_api();
  bool prepare(SQuery &q);                    // device state; pairs: per-target BFS
  void run_group(std::vector<std::shared_ptr<SQuery>> &part, std::vector<int> &lanes);
  void finish(SQuery &q);
  void fail_query(SQuery &q, bc_status code, const std::string &msg);
};

static size_t query_mem(const SQuery &q) {
  const size_t T = (size_t)std::max(q.T(), 1), n = (size_t)q.g.n;
  if (q.kind == BC_QUERY_PAIRS) return T * n * 12 + T * 64;
  if (q.kind == BC_QUERY_UNIFORM) return n * sizeof(Acc);
  return T * 64;
}

void Server::fail_query(SQuery &q, bc_status code, const std::string &msg) {
  q.state = Q_FAILED;
  q.result = code;
  q.err = msg;
}

// API calls waiting for the context go first (at most 2 ms per batch), so a
// submit or poll never waits for more than about one batch of the worker.
void Server::yield_to_api() {
  const auto t0 = Clock::now();
  while (ctx->api_waiting.load() > 0 && Clock::now() - t0 < std::chrono::milliseconds(2)) std::this_thread::yield();
}

void Server::admit_locked() {
  while (!queued.empty() && (int32_t)active.size() < max_active) {
    auto q = queued.front();
    if (q->cancel) {
      queued.pop_front();
      q->state = Q_CANCELLED;
      q->result = BC_E_CANCELLED;
      cv_done.notify_all();
      continue;
    }
    if (mem_used + (int64_t)q->mem > mem_budget && !active.empty()) break;
    queued.pop_front();
    q->state = Q_ACTIVE;
    q->t_admit = Clock::now();
    mem_used += (int64_t)q->mem;
    active.push_back(q);
  }
}

bool Server::prepare(SQuery &q) {
  // called by the worker with ctx->mu held; allocates device state
  const size_t T = (size_t)std::max(q.T(), 1);
  q.dstate.ensure((20 * T + 15) / 16 * 16 + 16);
  BCG_CUDA(cudaMemsetAsync(q.dstate.p, 0, q.dstate.bytes, ctx->stream));
  const int32_t rem = q.T();
  BCG_CUDA(cudaMemcpyAsync(q.Rem(), &rem, 4, cudaMemcpyHostToDevice, ctx->stream));
  q.remaining = rem;
  if (q.kind == BC_QUERY_UNIFORM) {
    q.acc.ensure((size_t)q.g.n * sizeof(Acc));
    BCG_CUDA(cudaMemsetAsync(q.acc.p, 0, (size_t)q.g.n * sizeof(Acc), ctx->stream));
    q.remaining = 1;
  } else if (q.kind == BC_QUERY_PAIRS) {
    const size_t n = (size_t)q.g.n;
    q.tdist.ensure(n * T * 4);
    q.tsig.ensure(n * T * 8);
    q.dtarg.ensure((size_t)T * 4);
    BCG_CUDA(cudaMemcpyAsync(q.dtarg.p, q.targets.data(), (size_t)q.T() * 4, cudaMemcpyHostToDevice, ctx->stream));
    target_bfs(ctx, q.g, q.dtarg.as<int32_t>(), q.T(), T, q.tdist.as<int32_t>(), q.tsig.as<uint64_t>(), q.texp, q.tx);
    if (q.texp.p) {
      q.dtx.ensure((size_t)T * 4);
      BCG_CUDA(cudaMemcpyAsync(q.dtx.p, q.tx.data(), (size_t)T * 4, cudaMemcpyHostToDevice, ctx->stream));
    }
  }
  sync(ctx);
  return true;
}

void Server::finish(SQuery &q) {
  // called by the worker with ctx->mu held: write the caller's outputs
  cudaStream_t st = ctx->stream;
  if (q.kind == BC_QUERY_UNIFORM) {
    d_misc.ensure((size_t)q.g.n * 8);
    {
      LaunchScope ls(ctx, F_SCAN);
      k_serve_finalize_uniform<<<(q.g.n + 255) / 256, 256, 0, st>>>(q.g.n, q.acc.as<Acc>(), (double)q.g.n,
                                                                     (double)q.kuni, d_misc.as<double>());
    }
    sync(ctx);
    BCG_CUDA(cudaMemcpy(q.est, d_misc.p, (size_t)q.g.n * 8, cudaMemcpyDeviceToHost));
  } else {
    const int T = q.T();
    d_misc.ensure((size_t)std::max(T, 1) * 12 + 64);
    double *d_est = d_misc.as<double>();
    int32_t *d_st = reinterpret_cast<int32_t *>(d_est + std::max(T, 1));
    const double scale_n = q.kind == BC_QUERY_PAIRS ? (double)q.g.n * (double)(q.g.n - 1) : (double)q.g.n;
    if (T > 0) {
      LaunchScope ls(ctx, F_SCAN);
      k_serve_finalize<<<(T + 127) / 128, 128, 0, st>>>(T, q.S(), q.K(), q.Done(), scale_n, d_est, d_st);
    }
    sync(ctx);
    if (T > 0) {
      BCG_CUDA(cudaMemcpy(q.est, d_est, (size_t)T * 8, cudaMemcpyDeviceToHost));
      if (q.k_out) BCG_CUDA(cudaMemcpy(q.k_out, q.K(), (size_t)T * 8, cudaMemcpyDeviceToHost));
      if (q.S_out) BCG_CUDA(cudaMemcpy(q.S_out, q.S(), (size_t)T * 8, cudaMemcpyDeviceToHost));
      if (q.status_out) BCG_CUDA(cudaMemcpy(q.status_out, d_st, (size_t)T * 4, cudaMemcpyDeviceToHost));
    }
  }
}

// One batch for `part` (same graph and kind), lanes[i] draws for part[i].
void Server::run_group(std::vector<std::shared_ptr<SQuery>> &part, std::vector<int> &lanes) {
  Workspace &ws = ctx->ws;
  cudaStream_t st = ctx->stream;
  const Graph &g = part[0]->g;
  KnobScope ks(ctx, g);  // the graph's tuning as of the queries' submission
  const int kind = part[0]->kind;
  const int P = (int)part.size();
  std::vector<LaneDraw> ld;
  std::vector<int32_t> laneq, a(P);
  for (int b = 0; b < P; ++b) {
    a[b] = (int)ld.size();
    for (int i = 0; i < lanes[b]; ++i) {
      ld.push_back(LaneDraw{part[b]->seed, part[b]->qid, (uint64_t)(part[b]->issued + i)});
      laneq.push_back(b);
    }
  }
  const int L = (int)ld.size();
  d_lane.ensure(64 * sizeof(LaneDraw));
  BCG_CUDA(cudaMemcpyAsync(d_lane.p, ld.data(), L * sizeof(LaneDraw), cudaMemcpyHostToDevice, st));
  {
    LaunchScope ls(ctx, F_DRAW);
    k_draw_lanes<<<1, 64, 0, st>>>(L, d_lane.as<LaneDraw>(), g.n, kind == BC_QUERY_PAIRS, ws.sources.as<int32_t>(),
                                   ws.targets.as<int32_t>());
  }
  if (kind == BC_QUERY_UNIFORM) {
    Sink sink;
    sink.acc = part[0]->acc.as<Acc>();
    run_source_batch(ctx, g, L, sink);
  } else {
    // target entries: one per (query in batch, target)
    std::vector<int32_t> enext, eq;
    std::unordered_map<int32_t, int32_t> head;
    std::vector<ScanEntry> se;
    std::vector<PairEntry> pe;
    for (int b = 0; b < P; ++b) {
      SQuery &q = *part[b];
      for (int j = 0; j < q.T(); ++j) {
        const int32_t v = q.targets[j];
        const int32_t e = (int32_t)enext.size();
        auto it = head.find(v);
        enext.push_back(it == head.end() ? -1 : it->second);
        head[v] = e;
        eq.push_back(b);
        se.push_back(ScanEntry{q.S(), q.K(), q.Done(), q.Rem(), j, a[b], lanes[b], 0, q.issued,
                               q.c * (double)g.n, kind == BC_QUERY_PAIRS ? q.scale : 1.0});
        if (kind == BC_QUERY_PAIRS)
          pe.push_back(PairEntry{q.tdist.as<int32_t>(), q.tsig.as<uint64_t>(), q.texp.as<int32_t>(),
                                 q.texp.p ? q.dtx.as<int32_t>() : nullptr, v, j, std::max(q.T(), 1), a[b], lanes[b],
                                 0});
      }
    }
    const int E = (int)enext.size();
    d_tdelta.ensure((size_t)std::max(E, 1) * 64 * 8);
    BCG_CUDA(cudaMemsetAsync(d_tdelta.p, 0, (size_t)std::max(E, 1) * 64 * 8, st));
    if (kind == BC_QUERY_SOURCES) {
      std::vector<int32_t> hv, he;
      for (auto &kv : head) {
        hv.push_back(kv.first);
        he.push_back(kv.second);
      }
      const int nh = (int)hv.size();
      d_enext.ensure((size_t)std::max(E, 1) * 4);
      d_eq.ensure((size_t)std::max(E, 1) * 4);
      d_laneq.ensure(64 * 4);
      d_heads.ensure((size_t)std::max(nh, 1) * 8);
      d_tslot.ensure((size_t)g.n * 4);
      BCG_CUDA(cudaMemcpyAsync(d_enext.p, enext.data(), (size_t)E * 4, cudaMemcpyHostToDevice, st));
      BCG_CUDA(cudaMemcpyAsync(d_eq.p, eq.data(), (size_t)E * 4, cudaMemcpyHostToDevice, st));
      BCG_CUDA(cudaMemcpyAsync(d_laneq.p, laneq.data(), (size_t)L * 4, cudaMemcpyHostToDevice, st));
      BCG_CUDA(cudaMemcpyAsync(d_heads.p, hv.data(), (size_t)nh * 4, cudaMemcpyHostToDevice, st));
      BCG_CUDA(cudaMemcpyAsync(d_heads.as<int32_t>() + nh, he.data(), (size_t)nh * 4, cudaMemcpyHostToDevice, st));
      BCG_CUDA(cudaMemsetAsync(d_tslot.p, 0xFF, (size_t)g.n * 4, st));
      {
        LaunchScope ls(ctx, F_MISC);
        k_set_heads<<<(nh + 127) / 128, 128, 0, st>>>(nh, d_heads.as<int32_t>(), d_heads.as<int32_t>() + nh,
                                                      d_tslot.as<int32_t>());
      }
      Sink sink;
      sink.tslot = d_tslot.as<int32_t>();
      sink.tnext = d_enext.as<int32_t>();
      sink.eq = d_eq.as<int32_t>();
      sink.lane_q = d_laneq.as<int32_t>();
      sink.tdelta = d_tdelta.as<double>();
      run_source_batch(ctx, g, L, sink);
    } else {
      // (the plain pair path handles one lane; batches are of one in that mode)
      const uint64_t px = pair_batch(ctx, g, L);
      d_pair.ensure((size_t)std::max(E, 1) * sizeof(PairEntry));
      BCG_CUDA(cudaMemcpyAsync(d_pair.p, pe.data(), (size_t)E * sizeof(PairEntry), cudaMemcpyHostToDevice, st));
      LaunchScope ls(ctx, F_PAIR);
      k_pair_values_multi<<<E, 64, 0, st>>>(E, d_pair.as<PairEntry>(), ws.sources.as<int32_t>(),
                                            ws.targets.as<int32_t>(), ws.pair_d.as<int32_t>(),
                                            ws.pair_sig.as<uint64_t>(), ws.pair_exp.as<int32_t>(), px,
                                            d_tdelta.as<double>());
    }
    d_scan.ensure((size_t)std::max(E, 1) * sizeof(ScanEntry));
    BCG_CUDA(cudaMemcpyAsync(d_scan.p, se.data(), (size_t)E * sizeof(ScanEntry), cudaMemcpyHostToDevice, st));
    {
      LaunchScope ls(ctx, F_SCAN);
      k_stop_scan_multi<<<(E + 127) / 128, 128, 0, st>>>(E, d_scan.as<ScanEntry>(), d_tdelta.as<double>());
    }
    // remaining targets per query
    std::vector<int32_t *> rp(P);
    for (int b = 0; b < P; ++b) rp[b] = part[b]->Rem();
    d_rem.ensure(64 * 8 + 64 * 4);
    BCG_CUDA(cudaMemcpyAsync(d_rem.p, rp.data(), (size_t)P * 8, cudaMemcpyHostToDevice, st));
    int32_t *d_out = reinterpret_cast<int32_t *>(d_rem.as<char>() + 64 * 8);
    {
      LaunchScope ls(ctx, F_MISC);
      k_gather_rem<<<1, 64, 0, st>>>(P, d_rem.as<int32_t *>(), d_out);
    }
    int32_t *h = static_cast<int32_t *>(ws.pinned);
    BCG_CUDA(cudaMemcpyAsync(h, d_out, (size_t)P * 4, cudaMemcpyDeviceToHost, st));
    sync(ctx);
    for (int b = 0; b < P; ++b) part[b]->remaining = h[b];
  }
  sync(ctx);
  for (int b = 0; b < P; ++b) {
    part[b]->issued += lanes[b];
    part[b]->samples += lanes[b];
    part[b]->batches += 1;
  }
}

void Server::loop() {
  cudaSetDevice(ctx->device);
  for (;;) {
    std::vector<std::shared_ptr<SQuery>> to_prepare, done, part;
    std::vector<int> lanes;
    // 1. wait for work and admit
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !queued.empty() || !active.empty(); });
      if (stop) return;
      admit_locked();
      for (auto &q : active)
        if (!q->prepared && !q->cancel && q->state == Q_ACTIVE) to_prepare.push_back(q);
    }
    // 2. device state for newly admitted queries (pairs: one BFS per target)
    for (auto &q : to_prepare) {
      yield_to_api();
      std::lock_guard<std::recursive_mutex> g(ctx->mu);
      try {
        prepare(*q);
        q->prepared = true;
      } catch (const Error &e) {
        std::lock_guard<std::mutex> lk(mu);
        fail_query(*q, e.code, e.msg);
      }
    }
    // 3. retire cancelled, failed and finished queries
    {
      std::lock_guard<std::mutex> lk(mu);
      std::vector<std::shared_ptr<SQuery>> keep;
      for (auto &q : active) {
        if (q->cancel) {
          q->state = Q_CANCELLED;
          q->result = BC_E_CANCELLED;
          mem_used -= (int64_t)q->mem;
        } else if (q->state == Q_FAILED) {
          mem_used -= (int64_t)q->mem;
        } else if (q->prepared && !q->needs_draws()) {
          done.push_back(q);
        } else {
          keep.push_back(q);
        }
      }
      active.swap(keep);
    }
    for (auto &q : done) {
      bc_status fcode = BC_OK;
      std::string fmsg;
      {
        yield_to_api();
        std::lock_guard<std::recursive_mutex> g(ctx->mu);
        try {
          finish(*q);
        } catch (const Error &e) {
          fcode = e.code;
          fmsg = e.msg;
        }
      }
      if (q->stats_out) {
        const auto now = Clock::now();
        q->stats_out->queue_ms = std::chrono::duration<double, std::milli>(q->t_admit - q->t_submit).count();
        q->stats_out->run_ms = std::chrono::duration<double, std::milli>(now - q->t_admit).count();
        q->stats_out->samples = q->samples;
        q->stats_out->batches = q->batches;
      }
      q->dstate.release();
      q->tdist.release();
      q->tsig.release();
      q->dtarg.release();
      q->texp.release();
      q->dtx.release();
      q->acc.release();
      std::lock_guard<std::mutex> lk(mu);
      if (fcode == BC_OK) {
        q->state = Q_DONE;
        q->result = BC_OK;
      } else {
        fail_query(*q, fcode, fmsg);
      }
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      for (auto &q : done) mem_used -= (int64_t)q->mem;
      // 4. next group, round-robin over active queries
      const size_t na = active.size();
      int lead = -1;
      for (size_t s = 0; s < na; ++s) {
        const size_t i = (rr + s) % na;
        if (active[i]->prepared && active[i]->needs_draws()) {
          lead = (int)i;
          break;
        }
      }
      if (lead >= 0) {
        rr = (size_t)lead + 1;
        const SQuery &L0 = *active[lead];
        const int width = batch_width_is_plain(ctx) ? 1 : 64;
        std::vector<int> idx;
        for (size_t s = 0; s < na && (int)idx.size() < width; ++s) {
          const size_t i = ((size_t)lead + s) % na;
          SQuery &q = *active[i];
          if (q.gh == L0.gh && q.kind == L0.kind && q.prepared && q.needs_draws()) {
            idx.push_back((int)i);
            if (q.kind == BC_QUERY_UNIFORM) break;  // a uniform query fills its batches alone
          }
        }
        const int P = (int)idx.size();
        std::vector<int64_t> need(P);
        for (int b = 0; b < P; ++b) {
          const SQuery &q = *active[idx[b]];
          need[b] = (q.kind == BC_QUERY_UNIFORM ? q.kuni : q.cap) - q.issued;
        }
        std::vector<int> take(P, 0);
        int left = width;
        const int quota = std::max(1, width / std::max(P, 1));
        for (int b = 0; b < P && left > 0; ++b) {
          const int t = (int)std::min<int64_t>(std::min<int64_t>(quota, need[b]), left);
          take[b] = t;
          left -= t;
        }
        for (int b = 0; b < P && left > 0; ++b) {
          const int t = (int)std::min<int64_t>(need[b] - take[b], left);
          take[b] += t;
          left -= t;
        }
        for (int b = 0; b < P; ++b)
          if (take[b] > 0) {
            part.push_back(active[idx[b]]);
            lanes.push_back(take[b]);
          }
      }
    }
    cv_done.notify_all();
    if (part.empty()) continue;
    // 5. one shared batch
    yield_to_api();
    std::lock_guard<std::recursive_mutex> g(ctx->mu);
    try {
      run_group(part, lanes);
      const unsigned eb = read_and_clear_err(ctx);
      if (eb) {
        std::lock_guard<std::mutex> lk(mu);
        const bc_status code = (eb & ERR_SIGMA_OVERFLOW) ? BC_E_SIGMA_OVERFLOW : BC_E_RANGE;
        for (auto &q : part) fail_query(*q, code, "device arithmetic error in a batch of this query");
      }
    } catch (const Error &e) {
      std::lock_guard<std::mutex> lk(mu);
      for (auto &q : part) fail_query(*q, e.code, e.msg);
    }
  }
}

Server *server_of(bc_ctx *ctx) {
  if (!ctx->server) {
    Server *s = new Server();
    s->ctx = ctx;
    size_t fr = 0, tot = 0;
    cudaSetDevice(ctx->device);
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      tot = (size_t)16 << 30;
    }
    s->mem_budget = (int64_t)(tot / 4);
    s->worker = std::thread([s] { s->loop(); });
    ctx->server = s;
  }
  return ctx->server;
}

void server_shutdown(bc_ctx *ctx) {
  Server *s = ctx->server;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (DevBuf *b : {&s->d_lane, &s->d_laneq, &s->d_enext, &s->d_eq, &s->d_heads, &s->d_scan, &s->d_pair, &s->d_rem,
                    &s->d_tdelta, &s->d_tslot, &s->d_misc})
    b->release();
  for (auto &kv : s->queries) {
    kv.second->dstate.release();
    kv.second->tdist.release();
    kv.second->tsig.release();
    kv.second->dtarg.release();
    kv.second->texp.release();
    kv.second->dtx.release();
    kv.second->acc.release();
  }
  delete s;
  ctx->server = nullptr;
}

bool server_uses_graph(bc_ctx *ctx, bc_graph g) {
  Server *s = ctx->server;
  if (!s) return false;
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto &kv : s->queries) {
    const SQuery &q = *kv.second;
    if (q.gh == g && (q.state == Q_QUEUED || q.state == Q_ACTIVE)) return true;
  }
  return false;
}

}  // namespace bcg

using namespace bcg;

extern "C" {

bc_status bc_submit(bc_ctx *ctx, const bc_query *q, bc_ticket *out) {
  if (!ctx || !q || !out) return BC_E_INVALID;
  auto sq = std::make_shared<SQuery>();
  {
    ApiLock lk(ctx);
    try {
      const Graph &g = get_graph(ctx, q->graph);
      if (q->kind != BC_QUERY_SOURCES && q->kind != BC_QUERY_PAIRS && q->kind != BC_QUERY_UNIFORM)
        fail(BC_E_INVALID, "unknown query kind");
      if (!q->est) fail(BC_E_INVALID, "est is NULL");
      if (q->kind == BC_QUERY_UNIFORM) {
        if (q->k < 1 || q->k > ((int64_t)1 << 32)) fail(BC_E_INVALID, "k must be in [1, 2^32]");
      } else {
        if (q->T < 1 || !q->targets) fail(BC_E_INVALID, "a query needs T >= 1 targets");
        if (!(q->c >= 1.0) || !(q->c < 1e300)) fail(BC_E_INVALID, "c must be >= 1 and finite");
        if (q->cap < 1 || q->cap > ((int64_t)1 << 32)) fail(BC_E_INVALID, "cap must be in [1, 2^32]");
        if (q->kind == BC_QUERY_PAIRS && g.n < 2) fail(BC_E_INVALID, "pair sampling needs n >= 2");
        if (q->kind == BC_QUERY_PAIRS && g.directed) fail(BC_E_INVALID, "pair sampling needs an undirected graph");
        if (q->kind == BC_QUERY_PAIRS && g.w) fail(BC_E_INVALID, "pair sampling needs an unweighted graph");
        const double sc = q->threshold_scale == 0.0 ? 1.0 : q->threshold_scale;
        if (!(sc > 0.0) || !(sc < 1e300)) fail(BC_E_INVALID, "threshold_scale must be > 0");
        std::vector<int32_t> t(q->targets, q->targets + q->T);
        for (int32_t v : t)
          if (v < 0 || v >= g.n) fail(BC_E_INVALID, "target out of range");
        std::vector<int32_t> srt = t;
        std::sort(srt.begin(), srt.end());
        for (size_t i = 1; i < srt.size(); ++i)
          if (srt[i] == srt[i - 1]) fail(BC_E_INVALID, "targets must be distinct");
        sq->targets = t;
        sq->scale = sc;
      }
      sq->kind = q->kind;
      sq->gh = q->graph;
      sq->g = g;
      sq->c = q->c;
      sq->cap = q->cap;
      sq->kuni = q->k;
      sq->seed = q->seed;
      sq->qid = q->qid;
      sq->est = q->est;
      sq->k_out = q->k_out;
      sq->S_out = q->S_out;
      sq->status_out = q->stop_status;
      sq->stats_out = q->stats;
      sq->mem = query_mem(*sq);
      server_of(ctx);
      ctx->err = "no error";
    } catch (const Error &e) {
      ctx->err = e.msg;
      return e.code;
    }
  }
  Server *s = ctx->server;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int64_t)sq->mem > s->mem_budget) {
      ApiLock g(ctx);
      ctx->err = "query needs more device memory than the server budget";
      return BC_E_NOMEM;
    }
    sq->id = s->next_ticket++;
    sq->t_submit = Clock::now();
    s->queries[sq->id] = sq;
    s->queued.push_back(sq);
    *out = sq->id;
  }
  s->cv_work.notify_all();
  return BC_OK;
}

bc_status bc_poll(bc_ctx *ctx, bc_ticket t, int64_t timeout_us) {
  if (!ctx) return BC_E_INVALID;
  Server *s = ctx->server;
  if (!s) return BC_E_UNKNOWN_HANDLE;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->queries.find(t);
  if (it == s->queries.end()) return BC_E_UNKNOWN_HANDLE;
  auto q = it->second;
  auto finished = [&] { return q->state == Q_DONE || q->state == Q_CANCELLED || q->state == Q_FAILED; };
  if (!finished()) {
    if (timeout_us < 0) s->cv_done.wait(lk, finished);
    else if (timeout_us > 0) s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), finished);
  }
  if (!finished()) return BC_PENDING;
  const bc_status r = q->result;
  const std::string msg = q->err;
  s->queries.erase(it);
  lk.unlock();
  if (r != BC_OK) {
    ApiLock g(ctx);
    ctx->err = msg.empty() ? "query cancelled" : msg;
  }
  return r;
}

bc_status bc_cancel(bc_ctx *ctx, bc_ticket t) {
  if (!ctx) return BC_E_INVALID;
  Server *s = ctx->server;
  if (!s) return BC_E_UNKNOWN_HANDLE;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->queries.find(t);
    if (it == s->queries.end()) return BC_E_UNKNOWN_HANDLE;
    auto &q = *it->second;
    if (q.state == Q_QUEUED || q.state == Q_ACTIVE) q.cancel = true;
    if (q.state == Q_QUEUED) {
      // drop it from the queue right away
      for (auto qi = s->queued.begin(); qi != s->queued.end(); ++qi)
        if ((*qi)->id == t) {
          s->queued.erase(qi);
          break;
        }
      q.state = Q_CANCELLED;
      q.result = BC_E_CANCELLED;
    }
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  return BC_OK;
}

bc_status bc_server_limits(bc_ctx *ctx, int32_t max_active, int64_t mem_budget_bytes) {
  if (!ctx) return BC_E_INVALID;
  Server *s;
  {
    ApiLock lk(ctx);
    s = server_of(ctx);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (max_active > 0) s->max_active = max_active;
    if (mem_budget_bytes > 0) s->mem_budget = mem_budget_bytes;
  }
  s->cv_work.notify_all();
  return BC_OK;
}

}  // extern "C"
