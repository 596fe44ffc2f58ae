// The batched serving form: many netlists' initializers at once.  Algorithm 1
// runs per design, so the designs of a batch are independent.
//
// Union form: A0 and each round's hint build run per design on worker
// threads, each driving one of the caller's CUDA streams and taking the next
// design (largest first, so the long ones start early); each round's filter
// then runs as one launch per kernel and power over all designs
// (run_filter_batch: a block-diagonal union of the designs' matrices).
// Per-design form: each worker runs whole initializers.  A design's result
// does not depend on the form, the stream or the worker: every kernel of the
// path adds in a fixed order, and a design's units in a union launch compute
// what its own launch computes.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "pl_internal.h"

namespace pl {
namespace {

__global__ void k_cells_out(int32_t C, const float2 *g, float2 *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x)
    out[i] = g[i];
}

// fn(i, stream) for every design i of `order` (in that order) on nw worker
// threads, worker k driving streams[k].  Returns the first failing design's
// status (by position in order), with its message.
template <typename F>
pl_status for_designs(const std::vector<int32_t> &order, int nw, const pl_stream *streams, int dev,
                      F fn) {
  const int n = (int)order.size();
  std::atomic<int32_t> next{0};
  std::vector<pl_status> st(n, PL_OK);
  std::vector<std::string> msg(n);
  std::atomic<bool> devok{true};
  auto work = [&](int k) {
    if (cudaSetDevice(dev) != cudaSuccess) {
      devok = false;
      return;
    }
    for (;;) {
      const int32_t q = next.fetch_add(1);
      if (q >= n) break;
      const int32_t i = order[q];
      clear_error();
      st[q] = fn(i, reinterpret_cast<cudaStream_t>(streams[k]));
      if (st[q] != PL_OK) msg[q] = pl_last_error();
    }
  };
  const int w = std::max(1, std::min(nw, n));
  std::vector<std::thread> th;
  th.reserve(w);
  for (int k = 0; k < w; ++k) th.emplace_back(work, k);
  for (auto &t : th) t.join();
  for (int q = 0; q < n; ++q)
    if (st[q] != PL_OK) {
      set_error("design %d: %s", order[q], msg[q].c_str());
      return st[q];
    }
  if (!devok || next.load() < n) {
    set_error("a worker could not select the device");
    return PL_ERR_CUDA;
  }
  return PL_OK;
}

// The union form in two groups of designs (alternate designs of the
// largest-first order), pipelined: while one group's filter runs on the GPU,
// the other group's hint builds run on the workers' streams.  Each group's
// filter runs on its first two graphs' second streams (its own copy of the
// launch arguments in its half of ws).
pl_status union_batch(int32_t n, pl_graph *const *graphs, const pl_params *p, const uint64_t *seeds,
                      float *const *xy_out_cells, int nw, const pl_stream *streams, int rows_ctas,
                      void *ws, size_t ws_bytes, const std::vector<int32_t> &order, int dev) {
  std::vector<float *> cur(n), nxt(n);
  for (int i = 0; i < n; ++i) {
    cur[i] = P<float>(graphs[i]->xc);
    nxt[i] = P<float>(graphs[i]->g0);
  }
  // A0 per design
  pl_status st = for_designs(order, nw, streams, dev, [&](int i, cudaStream_t s) -> pl_status {
    pl_graph *g = graphs[i];
    ArenaScope scope(&g->arena);
    g->arena.short_need = 0;
    g->stream = s;
    cudaError_t e = cudaMemsetAsync(g->status.p, 0, 32, s);
    if (e != cudaSuccess) return cuda_fail(e, "status reset");
    pl_status r = run_init_signal(g, seeds[i], nullptr, cur[i], s);
    if (r == PL_OK) r = p->gift_enable ? run_gift(g, p, cur[i], nxt[i], s) : clamp_nodes(g, p, cur[i], nxt[i], s);
    if (r == PL_OK) r = read_status(g, s);
    return r;
  });
  if (st != PL_OK) return st;
  std::swap(cur, nxt);
  const int ngr = n >= 2 ? 2 : 1;
  struct Group {
    std::vector<int32_t> order;  // its designs, largest first
    std::vector<pl_graph *> gs;
    std::vector<const float *> in;
    std::vector<float *> out;
    cudaStream_t s = nullptr, sh = nullptr;
    bool pending = false;
  } grp[2];
  for (int q = 0; q < n; ++q) grp[q % ngr].order.push_back(order[q]);
  const size_t half = (ws_bytes / 2) & ~(size_t)255;  // each half 256-byte aligned
  for (int k = 0; k < ngr; ++k) {
    Group &G = grp[k];
    for (int32_t i : G.order) G.gs.push_back(graphs[i]);
    pl_graph *a = G.gs[0], *b = G.gs[G.gs.size() > 1 ? 1 : 0];
    cudaError_t e = ensure_side(a);
    if (e == cudaSuccess) e = ensure_side(b);
    if (e != cudaSuccess) return cuda_fail(e, "batch streams");
    G.s = a->side;
    G.sh = b->side;
  }
  for (int t = 0; t < p->t_hint; ++t) {
    for (int k = 0; k < ngr; ++k) {
      Group &G = grp[k];
      if (G.pending) {  // the group's previous filter ends before its next hint build
        const cudaError_t e = cudaStreamSynchronize(G.s);
        if (e != cudaSuccess) return cuda_fail(e, "batched filter");
        G.pending = false;
      }
      st = for_designs(G.order, nw, streams, dev, [&](int i, cudaStream_t s) -> pl_status {
        pl_graph *g = graphs[i];
        ArenaScope scope(&g->arena);
        g->arena.short_need = 0;
        g->stream = s;
        pl_status r = t ? read_status(g, s) : PL_OK;
        if (r == PL_OK) r = build_hints(g, p, cur[i], s);
        if (r == PL_OK) {
          const cudaError_t e = cudaStreamSynchronize(s);
          if (e != cudaSuccess) r = cuda_fail(e, "hint build");
        }
        return r;
      });
      if (st != PL_OK) return st;
      G.in.clear();
      G.out.clear();
      for (int32_t i : G.order) {
        G.in.push_back(cur[i]);
        G.out.push_back(nxt[i]);
      }
      st = run_filter_batch(G.gs.data(), (int)G.gs.size(), p, G.in.data(), G.out.data(),
                            static_cast<char *>(ws) + k * half, half, rows_ctas, G.s, G.sh);
      if (st != PL_OK) return st;
      G.pending = true;
      for (int32_t i : G.order) std::swap(cur[i], nxt[i]);
    }
  }
  for (int k = 0; k < ngr; ++k)
    if (grp[k].pending) {
      const cudaError_t e = cudaStreamSynchronize(grp[k].s);
      if (e != cudaSuccess) return cuda_fail(e, "batched filter");
    }
  return for_designs(order, nw, streams, dev, [&](int i, cudaStream_t s) -> pl_status {
    pl_graph *g = graphs[i];
    g->stream = s;
    k_cells_out<<<grid_for(g->C, 256), 256, 0, s>>>(g->C, reinterpret_cast<const float2 *>(cur[i]),
                                                    reinterpret_cast<float2 *>(xy_out_cells[i]));
    note_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "copy out");
    return read_status(g, s);
  });
}

}  // namespace
}  // namespace pl

using namespace pl;

extern "C" void pl_batch_opts_default(pl_batch_opts *o) {
  if (!o) return;
  o->union_products = 1;
  o->streams = 0;
  o->rows_ctas_per_sm = 5;
}

extern "C" size_t pl_batch_workspace_size(int32_t n, const pl_params *p) {
  if (n < 1 || !p || p->ntaps < 1 || p->ntaps > 4) return 0;
  return 2 * batch_ws_bytes(n, p);  // a half for each of the two pipelined groups
}

extern "C" pl_status pl_filter_init_batch(int32_t n, pl_graph *const *graphs, const pl_params *p,
                                          const uint64_t *seeds, float *const *xy_out_cells,
                                          int32_t nstreams, const pl_stream *streams,
                                          const pl_batch_opts *opts, void *ws, size_t ws_bytes) {
  clear_error();
  if (n < 0 || (n && (!graphs || !p || !seeds || !xy_out_cells)) || nstreams < 1 || !streams) {
    set_error("bad batch arguments");
    return PL_ERR_INVALID_ARG;
  }
  pl_batch_opts o;
  pl_batch_opts_default(&o);
  if (opts) o = *opts;
  if (o.streams < 0 || o.streams > nstreams || o.rows_ctas_per_sm < 0 || o.rows_ctas_per_sm > 5) {
    set_error("bad batch options");
    return PL_ERR_INVALID_ARG;
  }
  const int nw = o.streams ? o.streams : nstreams;
  for (int32_t i = 0; i < n; ++i)
    if (!graphs[i] || !xy_out_cells[i]) {
      set_error("design %d: NULL graph or output", i);
      return PL_ERR_INVALID_ARG;
    }
  if (n == 0) return PL_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "pl_filter_init_batch");
  std::vector<int32_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return graphs[a]->N > graphs[b]->N; });
  if (!o.union_products) {
    return for_designs(order, nw, streams, dev, [&](int i, cudaStream_t s) -> pl_status {
      return pl_filter_init(graphs[i], p, seeds[i], nullptr, xy_out_cells[i], s);
    });
  }
  pl_status st = check_params(p);
  for (int32_t i = 0; st == PL_OK && i < n; ++i) {
    st = same_layout(graphs[i], p);
    if (st == PL_OK && graphs[i]->wdtype != graphs[0]->wdtype) {
      set_error("the union form needs one weight type for all designs");
      st = PL_ERR_INVALID_ARG;
    }
  }
  if (st != PL_OK) return st;
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) {
    set_error("the union form needs a 256-byte aligned workspace");
    return PL_ERR_INVALID_ARG;
  }
  if (ws_bytes < 2 * batch_ws_bytes(n, p)) {
    set_error("batch workspace too small: need %zu bytes", 2 * batch_ws_bytes(n, p));
    return PL_ERR_WORKSPACE;
  }
  return union_batch(n, graphs, p, seeds, xy_out_cells, nw, streams,
                     o.rows_ctas_per_sm ? o.rows_ctas_per_sm : 5, ws, ws_bytes, order, dev);
}

extern "C" pl_status pl_batch_autotune(int32_t n, pl_graph *const *graphs, const pl_params *p,
                                       const uint64_t *seeds, float *const *xy_out_cells,
                                       int32_t nstreams, const pl_stream *streams, void *ws,
                                       size_t ws_bytes, pl_batch_opts *best, double *best_ms) {
  clear_error();
  if (!best || nstreams < 1) {
    set_error("bad autotune arguments");
    return PL_ERR_INVALID_ARG;
  }
  std::vector<pl_batch_opts> cand;
  for (int S : {1, 2, 4, 8, 16})
    if (S <= nstreams) cand.push_back({0, S, 5});
  if (ws)
    for (int S : {4, 8, 16})
      if (S <= nstreams)
        for (int rc : {3, 4, 5}) cand.push_back({1, S, rc});
  if (cand.empty()) cand.push_back({0, nstreams, 5});
  double bt = -1.0;
  for (const pl_batch_opts &c : cand) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "pl_batch_autotune");
    const auto t0 = std::chrono::steady_clock::now();
    const pl_status st = pl_filter_init_batch(n, graphs, p, seeds, xy_out_cells, nstreams, streams,
                                              &c, ws, ws_bytes);
    if (st != PL_OK) return st;
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "pl_batch_autotune");
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (bt < 0.0 || ms < bt) {
      bt = ms;
      *best = c;
    }
  }
  if (best_ms) *best_ms = bt;
  return PL_OK;
}
