// The batched serving form: many netlists' initializers at once.  Algorithm 1
// runs per design, so the designs of a batch are independent.  Each worker
// thread drives one of the caller's CUDA streams and takes the next design
// (largest first, so the long ones start early) until none is left; the
// designs' kernels then overlap on the GPU, which a single small design
// cannot fill.  A design's result does not depend on the stream or the
// worker that ran it: every kernel of the path adds in a fixed order.
#include <algorithm>
#include <atomic>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "pl_internal.h"

extern "C" pl_status pl_filter_init_batch(int32_t n, pl_graph *const *graphs, const pl_params *p,
                                          const uint64_t *seeds, float *const *xy_out_cells,
                                          int32_t nstreams, const pl_stream *streams) {
  using namespace pl;
  clear_error();
  if (n < 0 || (n && (!graphs || !p || !seeds || !xy_out_cells)) || nstreams < 1 || !streams) {
    set_error("bad batch arguments");
    return PL_ERR_INVALID_ARG;
  }
  for (int32_t i = 0; i < n; ++i)
    if (!graphs[i] || !xy_out_cells[i]) {
      set_error("design %d: NULL graph or output", i);
      return PL_ERR_INVALID_ARG;
    }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "pl_filter_init_batch");
  std::vector<int32_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return graphs[a]->N > graphs[b]->N; });
  std::atomic<int32_t> next{0};
  std::vector<pl_status> st(n, PL_OK);
  std::vector<std::string> msg(n);
  auto work = [&](int k) {
    if (cudaSetDevice(dev) != cudaSuccess) return;
    for (;;) {
      const int32_t q = next.fetch_add(1);
      if (q >= n) break;
      const int32_t i = order[q];
      st[i] = pl_filter_init(graphs[i], p, seeds[i], nullptr, xy_out_cells[i], streams[k]);
      if (st[i] != PL_OK) msg[i] = pl_last_error();
    }
  };
  const int nw = std::min<int32_t>(nstreams, std::max<int32_t>(n, 1));
  std::vector<std::thread> th;
  th.reserve(nw);
  for (int k = 0; k < nw; ++k) th.emplace_back(work, k);
  for (auto &t : th) t.join();
  for (int32_t i = 0; i < n; ++i)
    if (st[i] != PL_OK) {
      set_error("design %d: %s", i, msg[i].c_str());
      return st[i];
    }
  if (next.load() < n) {
    set_error("a worker could not select the device");
    return PL_ERR_CUDA;
  }
  return PL_OK;
}
