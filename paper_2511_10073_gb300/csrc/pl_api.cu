// C ABI entry points of libpl (see include/pl.h): argument checks, error
// reporting, graph lifetime and host copies for exact comparison.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "pl_internal.h"

namespace pl {

// ---------------------------------------------------------- benchmark hooks
static std::atomic<long long> g_launches{0};
static std::atomic<bool> g_prof{false};
static std::mutex g_prof_mu;
struct ProfRec {
  cudaEvent_t a, b;
  int kind;
  double bytes;
};
static std::vector<ProfRec> g_recs;
static std::vector<cudaEvent_t> g_pool;
static long long g_launch0 = 0, g_launch1 = -1;

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
bool prof_on() { return g_prof.load(std::memory_order_relaxed); }

static cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_begin(cudaStream_t s, int kind, double bytes) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfRec r{take_event(), take_event(), kind, bytes};
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
}

void prof_end(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_recs.empty()) cudaEventRecord(g_recs.back().b, s);
}

static thread_local char g_err[512] = "";

void clear_error() { g_err[0] = 0; }

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

pl_status cuda_fail(cudaError_t e, const char *what) {
  const Arena *a = current_arena();
  if (e == cudaErrorMemoryAllocation && a && a->short_need) {
    set_error("workspace too small: %zu bytes needed so far, %zu given (%s)", a->short_need,
              a->cap, what);
    return PL_ERR_WORKSPACE;
  }
  set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  return e == cudaErrorMemoryAllocation ? PL_ERR_OOM : PL_ERR_CUDA;
}

// An entry point's use of a graph's workspace: the arena becomes the calling
// thread's current one, with no shortfall recorded yet.
struct GraphScope {
  ArenaScope scope;
  explicit GraphScope(pl_graph *g) : scope(&g->arena) { g->arena.short_need = 0; }
};

int hpwl_blocks(int32_t M);
size_t hpwl_ws_bytes(int32_t M);
cudaError_t launch_hpwl(const pl_netlist *nl, const float *xy, double *out, void *ws,
                        cudaStream_t s);

static bool finite(double v) { return std::isfinite(v); }

pl_status check_params(const pl_params *p) {
  if (!p) { set_error("params is NULL"); return PL_ERR_INVALID_ARG; }
  if (p->clique_max < 2 || p->clique_max > 16) { set_error("clique_max must be in 2..16"); return PL_ERR_INVALID_ARG; }
  if (p->wdtype != PL_W_FP32 && p->wdtype != PL_W_BF16) { set_error("wdtype must be PL_W_FP32 or PL_W_BF16"); return PL_ERR_INVALID_ARG; }
  for (int b = 0; b < 3; ++b) {
    if (p->gift_k[b] < 0 || p->gift_k[b] > 64) { set_error("gift_k must be in 0..64"); return PL_ERR_INVALID_ARG; }
    if (!(p->gift_sigma[b] > 0.0) || !finite(p->gift_sigma[b])) { set_error("gift_sigma must be > 0"); return PL_ERR_INVALID_ARG; }
    if (!finite(p->gift_alpha[b])) { set_error("gift_alpha must be finite"); return PL_ERR_INVALID_ARG; }
  }
  if (p->t_hint < 0 || p->t_hint > 1000) { set_error("t_hint must be in 0..1000"); return PL_ERR_INVALID_ARG; }
  if (p->nbx < 1 || p->nby < 1 || (long long)p->nbx * p->nby > (1LL << 22)) { set_error("bins must be >= 1 and at most 2^22 in total"); return PL_ERR_INVALID_ARG; }
  if (!(p->gamma >= 0.0 && p->gamma <= 1.0)) { set_error("gamma must be in [0, 1]"); return PL_ERR_INVALID_ARG; }
  if (!(p->det_ratio >= 0.0) || !finite(p->det_ratio)) { set_error("det_ratio must be >= 0"); return PL_ERR_INVALID_ARG; }
  if (!finite(p->capacity) || !finite(p->mu)) { set_error("capacity and mu must be finite"); return PL_ERR_INVALID_ARG; }
  if (p->ntaps < 1 || p->ntaps > 4) { set_error("ntaps must be in 1..4"); return PL_ERR_INVALID_ARG; }
  for (int j = 0; j < p->ntaps; ++j) {
    if (p->tap_k[j] < 1 || p->tap_k[j] > 64 || (j && p->tap_k[j] <= p->tap_k[j - 1])) { set_error("tap_k must be strictly increasing in 1..64"); return PL_ERR_INVALID_ARG; }
    if (!finite(p->tap_alpha[j])) { set_error("tap_alpha must be finite"); return PL_ERR_INVALID_ARG; }
  }
  return PL_OK;
}

static pl_status check_netlist(const pl_netlist *nl) {
  if (!nl) { set_error("netlist is NULL"); return PL_ERR_INVALID_ARG; }
  if (nl->num_cells < 0 || nl->num_nets < 0 || nl->num_pins < 0) { set_error("negative netlist size"); return PL_ERR_INVALID_ARG; }
  if (!nl->net_ptr || (nl->num_pins && !nl->pin_cell)) { set_error("net_ptr / pin_cell is NULL"); return PL_ERR_INVALID_ARG; }
  if (nl->num_cells && (!nl->cell_w || !nl->cell_h || !nl->cell_kind || !nl->fixed_x || !nl->fixed_y)) { set_error("a cell array is NULL"); return PL_ERR_INVALID_ARG; }
  if (!finite(nl->xl) || !finite(nl->yl) || !finite(nl->xh) || !finite(nl->yh) || !(nl->xh > nl->xl) || !(nl->yh > nl->yl)) { set_error("placement region must be finite with xh > xl, yh > yl"); return PL_ERR_INVALID_ARG; }
  return PL_OK;
}

pl_status same_layout(const pl_graph *g, const pl_params *p) {
  if (p->nbx != g->nbx || p->nby != g->nby || p->det_ratio != g->det_ratio ||
      p->wdtype != g->wdtype || p->clique_max != g->clique_max) {
    set_error("bins, detection ratio, weight type and clique_max must match the graph build");
    return PL_ERR_INVALID_ARG;
  }
  return PL_OK;
}

static void destroy(pl_graph *g) {
  if (!g) return;
  if (g->side) {  // the side stream's work ends before its buffers go
    cudaStreamSynchronize(g->side);
    cudaStreamDestroy(g->side);
  }
  if (g->side2) {
    cudaStreamSynchronize(g->side2);
    cudaStreamDestroy(g->side2);
  }
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  if (g->ev_join2) cudaEventDestroy(g->ev_join2);
  delete g;  // its device memory is the caller's workspace
}

pl_status read_status(pl_graph *g, cudaStream_t s) {
  int st[8];
  cudaError_t e = cudaMemcpyAsync(st, g->status.p, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (st[0] & ST_SPECTRUM) { set_error("lambda_up <= 0 or not finite"); return PL_ERR_SPECTRUM; }
  if (st[0] & ST_NONFINITE) { set_error("non-finite coordinate"); return PL_ERR_NONFINITE; }
  if (st[0] & ST_TIMEOUT) { set_error("a bounded device-side wait gave up"); return PL_ERR_TIMEOUT; }
  return PL_OK;
}

pl_status clamp_nodes(pl_graph *g, const pl_params *p, const float *in, float *out,
                      cudaStream_t s);

}  // namespace pl

using namespace pl;

extern "C" {

void pl_params_default(pl_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->clique_max = 16;
  p->wdtype = PL_W_FP32;
  p->gift_enable = 1;
  p->gift_center = 0;
  p->gift_k[0] = 4; p->gift_k[1] = 2; p->gift_k[2] = 2;
  p->gift_sigma[0] = 4.0; p->gift_sigma[1] = 4.0; p->gift_sigma[2] = 2.0;
  p->gift_alpha[0] = 0.7; p->gift_alpha[1] = 0.2; p->gift_alpha[2] = 0.1;
  p->t_hint = 3;
  p->nbx = 32;
  p->nby = 32;
  p->gamma = 0.5;
  p->det_ratio = 0.1;
  p->capacity = 1.0;
  p->mu = 4.0;
  p->ntaps = 1;
  p->tap_k[0] = 8;
  p->tap_alpha[0] = 1.0;
  p->pin_every_step = 0;
  p->clamp = 1;
}

const char *pl_last_error(void) { return pl::g_err; }

pl_status pl_build_graph(const pl_netlist *nl, const pl_params *p, const float *xy_nodes,
                         void *ws, size_t ws_bytes, pl_stream stream, pl_graph **gp) {
  pl::g_err[0] = 0;
  if (!gp) { set_error("graph out-pointer is NULL"); return PL_ERR_INVALID_ARG; }
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) { set_error("workspace must be a 256-byte aligned device pointer"); return PL_ERR_INVALID_ARG; }
  pl_status st = check_netlist(nl);
  if (st == PL_OK) st = check_params(p);
  if (st != PL_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  bool created = false;
  if (!*gp) {
    *gp = new (std::nothrow) pl_graph();
    if (!*gp) { set_error("host allocation failed"); return PL_ERR_OOM; }
    created = true;
  } else if ((*gp)->stream) {
    // the previous build's work on its streams ends before its memory is reused
    cudaStreamSynchronize((*gp)->stream);
    if ((*gp)->side) cudaStreamSynchronize((*gp)->side);
  }
  pl_graph *g = *gp;
  for_each_buf(g, 0, [](Buf &b) { release(b); });
  g->arena = Arena{};
  g->arena.base = static_cast<char *>(ws);
  g->arena.cap = ws_bytes;
  g->hint_mark = 0;
  g->star_w_ok = false;
  GraphScope scope(g);
  {
    // the static build's merge sort reads a process-wide constant (the merge
    // context), so static builds on different threads take turns
    static std::mutex build_mu;
    std::lock_guard<std::mutex> lk(build_mu);
    st = build_static(g, nl, p, s);
  }
  if (st == PL_OK && xy_nodes) st = build_hints(g, p, xy_nodes, s);
  if (st == PL_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "pl_build_graph");
  }
  if (st != PL_OK && created) {
    destroy(*gp);
    *gp = nullptr;
  }
  return st;
}

pl_status pl_graph_info(const pl_graph *g, int64_t *out) {
  if (!g || !out) { set_error("NULL argument"); return PL_ERR_INVALID_ARG; }
  for (int k = 0; k < 16; ++k) out[k] = 0;
  out[0] = g->C; out[1] = g->Pm; out[2] = g->S; out[3] = g->Mm; out[4] = g->NB;
  out[5] = g->Nst; out[6] = g->N; out[7] = (int64_t)g->nnz_static;
  out[8] = g->have_hints
               ? (int64_t)(g->st.nnz_s + g->st.nnz_l + g->hm.nnz_s + g->hm.nnz_l) + 2 * g->nslot
               : 0;
  out[9] = g->hx; out[10] = g->hy; out[11] = g->have_hints ? g->hm.nlong : 0;
  out[12] = g->nmov;
  out[13] = (int64_t)g->arena.peak;
  out[14] = (int64_t)g->arena.cap;
  out[15] = (int64_t)g->hint_mark;
  return PL_OK;
}

pl_status pl_build_hints(pl_graph *g, const pl_params *p, const float *xy_nodes,
                         pl_stream stream) {
  pl::g_err[0] = 0;
  if (!g || !xy_nodes) { set_error("NULL argument"); return PL_ERR_INVALID_ARG; }
  pl_status st = check_params(p);
  if (st == PL_OK) st = same_layout(g, p);
  if (st != PL_OK) return st;
  GraphScope scope(g);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  g->stream = s;
  return build_hints(g, p, xy_nodes, s);
}

pl_status pl_filter_apply(pl_graph *g, const pl_params *p, const float *xy_in, float *xy_out,
                          pl_stream stream) {
  pl::g_err[0] = 0;
  if (!g || !xy_in || !xy_out || xy_in == xy_out) { set_error("bad arguments (NULL or in == out)"); return PL_ERR_INVALID_ARG; }
  pl_status st = check_params(p);
  if (st == PL_OK) st = same_layout(g, p);
  if (st != PL_OK) return st;
  if (!g->have_hints) { set_error("no augmented graph: call pl_build_hints first"); return PL_ERR_INVALID_ARG; }
  GraphScope scope(g);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  g->stream = s;
  cudaError_t e = cudaMemsetAsync(g->status.p, 0, 32, s);
  if (e != cudaSuccess) return cuda_fail(e, "status reset");
  st = run_filter(g, p, xy_in, xy_out, s);
  return st != PL_OK ? st : read_status(g, s);
}

pl_status pl_gift(pl_graph *g, const pl_params *p, const float *xy_in, float *xy_out,
                  pl_stream stream) {
  pl::g_err[0] = 0;
  if (!g || !xy_in || !xy_out || xy_in == xy_out) { set_error("bad arguments (NULL or in == out)"); return PL_ERR_INVALID_ARG; }
  pl_status st = check_params(p);
  if (st == PL_OK) st = same_layout(g, p);
  if (st != PL_OK) return st;
  GraphScope scope(g);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  g->stream = s;
  cudaError_t e = cudaMemsetAsync(g->status.p, 0, 32, s);
  if (e != cudaSuccess) return cuda_fail(e, "status reset");
  st = run_gift(g, p, xy_in, xy_out, s);
  return st != PL_OK ? st : read_status(g, s);
}

pl_status pl_init_signal(pl_graph *g, uint64_t seed, const float *xy0_cells, float *xy_nodes,
                         pl_stream stream) {
  pl::g_err[0] = 0;
  if (!g || !xy_nodes) { set_error("NULL argument"); return PL_ERR_INVALID_ARG; }
  GraphScope scope(g);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  g->stream = s;
  return run_init_signal(g, seed, xy0_cells, xy_nodes, s);
}

__global__ void k_copy_cells(int32_t C, const float2 *g, float2 *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x)
    out[i] = g[i];
}

}  // extern "C"

namespace pl {
// The whole initializer (A0, then T_hint rounds of A2-A4), with the plain
// filter (m == NULL) or the learned one in every round; a learned round whose
// output is not finite is run again with the plain filter.
static pl_status init_run(pl_graph *g, const pl_params *p, const pl_learned *m, uint64_t seed,
                          const float *xy0_cells, float *xy_out_cells, int32_t *fallbacks,
                          cudaStream_t s) {
  g->stream = s;
  const int64_t N = g->N;
  cudaError_t e = ensure(g->xc, (size_t)N * 8 + 64);
  if (e == cudaSuccess) e = ensure(g->g0, (size_t)N * 8 + 64);
  if (e != cudaSuccess) return cuda_fail(e, "filter buffers");
  float *cur = P<float>(g->xc), *nxt = P<float>(g->g0);
  e = cudaMemsetAsync(g->status.p, 0, 32, s);
  if (e != cudaSuccess) return cuda_fail(e, "status reset");
  pl_status st = run_init_signal(g, seed, xy0_cells, cur, s);
  if (st != PL_OK) return st;
  if (p->gift_enable) {
    st = run_gift(g, p, cur, nxt, s);
  } else {
    st = clamp_nodes(g, p, cur, nxt, s);
  }
  if (st == PL_OK) st = read_status(g, s);
  if (st != PL_OK) return st;
  std::swap(cur, nxt);
  int32_t nfall = 0;
  for (int t = 0; t < p->t_hint; ++t) {
    if (t && !m) {
      st = read_status(g, s);
      if (st != PL_OK) return st;
    }
    st = build_hints(g, p, cur, s);
    if (st != PL_OK) return st;
    if (m) {
      st = run_learned(g, p, m, t, cur, nxt, s);
      int w0 = 0;
      if (st == PL_OK) {
        e = cudaMemcpyAsync(&w0, g->status.p, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "status read");
      }
      if (st == PL_OK && (w0 & ST_LEARNED_NF) && !(w0 & ~ST_LEARNED_NF)) {
        e = cudaMemsetAsync(g->status.p, 0, sizeof(int), s);  // the fallback: the plain round
        if (e != cudaSuccess) return cuda_fail(e, "status reset");
        st = run_filter(g, p, cur, nxt, s);
        ++nfall;
      }
      if (st == PL_OK) st = read_status(g, s);
    } else {
      st = run_filter(g, p, cur, nxt, s);
    }
    if (st != PL_OK) return st;
    std::swap(cur, nxt);
  }
  if (fallbacks) *fallbacks = nfall;
  k_copy_cells<<<grid_for(g->C, 256), 256, 0, s>>>(g->C, reinterpret_cast<const float2 *>(cur),
                                                   reinterpret_cast<float2 *>(xy_out_cells));
  note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "copy out");
  return read_status(g, s);
}
}  // namespace pl

extern "C" {

pl_status pl_filter_init(pl_graph *g, const pl_params *p, uint64_t seed, const float *xy0_cells,
                         float *xy_out_cells, pl_stream stream) {
  pl::g_err[0] = 0;
  if (!g || !xy_out_cells) { set_error("NULL argument"); return PL_ERR_INVALID_ARG; }
  pl_status st = check_params(p);
  if (st == PL_OK) st = same_layout(g, p);
  if (st != PL_OK) return st;
  GraphScope scope(g);
  return init_run(g, p, nullptr, seed, xy0_cells, xy_out_cells, nullptr,
                  reinterpret_cast<cudaStream_t>(stream));
}

pl_status pl_filter_init_learned(pl_graph *g, const pl_params *p, const pl_learned *m,
                                 uint64_t seed, const float *xy0_cells, float *xy_out_cells,
                                 int32_t *fallbacks, pl_stream stream) {
  pl::g_err[0] = 0;
  if (fallbacks) *fallbacks = 0;
  if (!g || !xy_out_cells) { set_error("NULL argument"); return PL_ERR_INVALID_ARG; }
  pl_status st = check_params(p);
  if (st == PL_OK) st = same_layout(g, p);
  if (st == PL_OK && m) st = check_model(m);
  if (st != PL_OK) return st;
  GraphScope scope(g);
  return init_run(g, p, m, seed, xy0_cells, xy_out_cells, fallbacks,
                  reinterpret_cast<cudaStream_t>(stream));
}

size_t pl_hpwl_workspace_size(int32_t num_nets) { return hpwl_ws_bytes(num_nets < 0 ? 0 : num_nets); }

pl_status pl_hpwl(const pl_netlist *nl, const float *xy_cells, double *hpwl, void *ws,
                  size_t ws_bytes, pl_stream stream) {
  pl::g_err[0] = 0;
  if (!nl || !xy_cells || !hpwl || !ws) { set_error("NULL argument"); return PL_ERR_INVALID_ARG; }
  if (nl->num_nets < 0 || nl->num_cells < 0 || !nl->net_ptr || (nl->num_pins && !nl->pin_cell)) { set_error("bad netlist"); return PL_ERR_INVALID_ARG; }
  if (reinterpret_cast<uintptr_t>(ws) % 256) { set_error("workspace must be 256-byte aligned"); return PL_ERR_INVALID_ARG; }
  if (ws_bytes < hpwl_ws_bytes(nl->num_nets)) { set_error("workspace too small: need %zu bytes", hpwl_ws_bytes(nl->num_nets)); return PL_ERR_WORKSPACE; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(ws, 0, 8, s);
  if (e == cudaSuccess) e = launch_hpwl(nl, xy_cells, hpwl, ws, s);
  if (e != cudaSuccess) return cuda_fail(e, "pl_hpwl");
  return PL_OK;
}

// Host copy of one split matrix.
struct HostSplit {
  std::vector<uint32_t> rp;
  std::vector<int32_t> lidx, col;
  std::vector<uint64_t> lptr;
  std::vector<float> w;
  bool ok = false;
};

static cudaError_t fetch_split(const pl_graph *g, const SpMat &m, HostSplit &h, cudaStream_t s) {
  const int64_t N = m.N;
  const uint64_t tot = m.nnz_s + m.nnz_l;
  h.rp.resize(N + 1);
  h.lidx.resize(N);
  h.lptr.resize(m.nlong + 1);
  h.col.resize(tot + 1);
  h.w.resize(tot + 1);
  cudaError_t e = cudaMemcpyAsync(h.rp.data(), m.rp_s.p, (N + 1) * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.lidx.data(), m.longidx.p, N * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.lptr.data(), m.lptr.p, (m.nlong + 1) * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && tot) e = cudaMemcpyAsync(h.col.data(), m.col.p, tot * 4, cudaMemcpyDeviceToHost, s);
  if (g->wdtype == PL_W_BF16) {
    std::vector<uint16_t> wb(tot + 1);
    if (e == cudaSuccess && tot) e = cudaMemcpyAsync(wb.data(), m.w.p, tot * 2, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (uint64_t k = 0; k < tot; ++k) {
      uint32_t u = (uint32_t)wb[k] << 16;
      memcpy(&h.w[k], &u, 4);
    }
  } else {
    if (e == cudaSuccess && tot) e = cudaMemcpyAsync(h.w.data(), m.w.p, tot * 4, cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  h.ok = e == cudaSuccess;
  return e;
}

static void row_range(const HostSplit &h, int64_t v, uint64_t *a, uint64_t *b) {
  if (h.lidx[v] >= 0) {
    *a = h.lptr[h.lidx[v]];
    *b = h.lptr[h.lidx[v] + 1];
  } else {
    *a = h.rp[v] & kOffMask;
    *b = h.rp[v + 1] & kOffMask;
  }
}

// Rows in canonical order: the st piece, then (augmented graph) the hm piece;
// a row kept in another order on the device (bin rows are the concatenation
// of their window bins' lists) is sorted by column.
// The augmented graph's bin entries are stored without columns: each hint
// cell's window block of W slots (slot s = (dy + hy)(2 hx + 1) + (dx + hx)
// for the bin at offset (dx, dy) from the cell's bin), and the bin rows are
// its transpose.  The export writes them out as explicit entries.
struct HostWindows {
  std::vector<int32_t> hbin;            // bin of each hint cell, -1 otherwise
  std::vector<float> w;                 // [C * W] slot weights
  std::vector<std::vector<std::pair<int32_t, float>>> bins;  // bin rows, ascending cell
};

static cudaError_t fetch_windows(const pl_graph *g, HostWindows &hw) {
  const size_t C = (size_t)g->C, W = (size_t)g->W;
  hw.hbin.resize(C);
  hw.w.assign(C * W, 0.f);
  cudaError_t e = C ? cudaMemcpy(hw.hbin.data(), g->hbin.p, C * 4, cudaMemcpyDeviceToHost)
                    : cudaSuccess;
  if (e != cudaSuccess || !C || !W) return e;
  if (g->wdtype == PL_W_BF16) {
    std::vector<uint16_t> b(C * W);
    e = cudaMemcpy(b.data(), g->hbw.p, C * W * 2, cudaMemcpyDeviceToHost);
    for (size_t k = 0; k < C * W; ++k) {
      const uint32_t u = (uint32_t)b[k] << 16;
      memcpy(&hw.w[k], &u, 4);
    }
  } else {
    e = cudaMemcpy(hw.w.data(), g->hbw.p, C * W * 4, cudaMemcpyDeviceToHost);
  }
  hw.bins.assign((size_t)g->NB, {});
  for (size_t i = 0; i < C; ++i) {
    const int hb = hw.hbin[i];
    if (hb < 0) continue;
    const int bx = hb % g->nbx, by = hb / g->nbx, wx = 2 * g->hx + 1;
    for (size_t sl = 0; sl < W; ++sl) {
      const int xx = bx + (int)(sl % wx) - g->hx, yy = by + (int)(sl / wx) - g->hy;
      if (xx < 0 || yy < 0 || xx >= g->nbx || yy >= g->nby) continue;
      hw.bins[(size_t)yy * g->nbx + xx].emplace_back((int32_t)i, hw.w[i * W + sl]);
    }
  }
  return e;
}

static pl_status export_matrix(const pl_graph *g, const SpMat &st, const SpMat *hm, int64_t rows,
                               int64_t *rp, int32_t *col, double *w, double *deg) {
  cudaStream_t s = g->stream;
  HostSplit hs, hh;
  HostWindows hw;
  cudaError_t e = fetch_split(g, st, hs, s);
  if (e == cudaSuccess && hm) e = fetch_split(g, *hm, hh, s);
  if (e == cudaSuccess && hm) e = fetch_windows(g, hw);
  std::vector<dfl> ds(st.N);
  if (e == cudaSuccess && deg)
    e = cudaMemcpy(ds.data(), (hm ? hm->dsum : st.dsum).p, st.N * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "export");
  const int64_t bn0 = g->Nst + g->Mm;
  std::vector<std::pair<int32_t, float>> ent;
  int64_t o = 0;
  for (int64_t v = 0; v < rows; ++v) {
    ent.clear();
    uint64_t a, b;
    row_range(hs, v, &a, &b);
    for (uint64_t k = a; k < b; ++k) ent.emplace_back(hs.col[k], hs.w[k]);
    if (hm) {
      row_range(hh, v, &a, &b);
      for (uint64_t k = a; k < b; ++k) ent.emplace_back(hh.col[k], hh.w[k]);
      if (v < g->C && hw.hbin[v] >= 0) {
        const int hb = hw.hbin[v], bx = hb % g->nbx, by = hb / g->nbx, wx = 2 * g->hx + 1;
        for (int sl = 0; sl < g->W; ++sl) {
          const int xx = bx + sl % wx - g->hx, yy = by + sl / wx - g->hy;
          if (xx < 0 || yy < 0 || xx >= g->nbx || yy >= g->nby) continue;
          ent.emplace_back((int32_t)(bn0 + (int64_t)yy * g->nbx + xx), hw.w[(size_t)v * g->W + sl]);
        }
      } else if (v >= bn0 && v < bn0 + g->NB) {
        for (auto &pr : hw.bins[v - bn0]) ent.push_back(pr);
      }
    }
    auto by_col = [](const std::pair<int32_t, float> &x, const std::pair<int32_t, float> &y) {
      return x.first < y.first;
    };
    if (!std::is_sorted(ent.begin(), ent.end(), by_col)) std::sort(ent.begin(), ent.end(), by_col);
    if (rp) rp[v] = o;
    for (auto &pr : ent) {
      if (col) col[o] = pr.first;
      if (w) w[o] = pr.second;
      ++o;
    }
    if (deg) deg[v] = (double)ds[v].hi + (double)ds[v].lo;
  }
  if (rp) rp[rows] = o;
  return PL_OK;
}

pl_status pl_graph_export_static(const pl_graph *g, int64_t *rp, int32_t *col, double *w,
                                 double *base_w) {
  pl::g_err[0] = 0;
  if (!g) { set_error("NULL graph"); return PL_ERR_INVALID_ARG; }
  pl_status st = export_matrix(g, g->st, nullptr, g->Nst, rp, col, w, nullptr);
  if (st != PL_OK) return st;
  if (base_w && g->C) {
    cudaError_t e = cudaMemcpy(base_w, g->base_w.p, (size_t)g->C * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "export base_w");
  }
  return PL_OK;
}

pl_status pl_graph_export(const pl_graph *g, int64_t *rp, int32_t *col, double *w, double *deg,
                          double *lam_up, double *Db, double *Cb, double *phi,
                          int32_t *cell_bin) {
  pl::g_err[0] = 0;
  if (!g) { set_error("NULL graph"); return PL_ERR_INVALID_ARG; }
  if (!g->have_hints) { set_error("no augmented graph built yet"); return PL_ERR_INVALID_ARG; }
  pl_status st = export_matrix(g, g->st, &g->hm, g->N, rp, col, w, deg);
  if (st != PL_OK) return st;
  cudaError_t e = cudaSuccess;
  if (lam_up) e = cudaMemcpy(lam_up, g->hm.lam.p, 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && Db) e = cudaMemcpy(Db, g->Db.p, (size_t)g->NB * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && Cb) e = cudaMemcpy(Cb, g->Cb.p, (size_t)g->NB * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && phi) e = cudaMemcpy(phi, g->phi.p, (size_t)g->NB * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && cell_bin && g->C) e = cudaMemcpy(cell_bin, g->cell_bin.p, (size_t)g->C * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "export");
  return PL_OK;
}

void pl_prof_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (on) {
    for (ProfRec &r : g_recs) {
      g_pool.push_back(r.a);
      g_pool.push_back(r.b);
    }
    g_recs.clear();
    g_launch0 = g_launches.load();
    g_launch1 = -1;
  } else if (g_prof.load()) {
    g_launch1 = g_launches.load();
  }
  g_prof.store(on != 0);
}

pl_status pl_prof_read(double *out) {
  pl::g_err[0] = 0;
  if (!out) { set_error("NULL argument"); return PL_ERR_INVALID_ARG; }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int k = 0; k < 8; ++k) out[k] = 0.0;
  out[0] = (double)((g_launch1 >= 0 ? g_launch1 : g_launches.load()) - g_launch0);
  for (ProfRec &r : g_recs) {
    cudaError_t e = cudaEventSynchronize(r.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "pl_prof_read");
    int base = r.kind == PROF_HR ? 1 : 4;
    out[base] += 1.0;
    out[base + 1] += ms;
    out[base + 2] += r.bytes;
  }
  return PL_OK;
}

void pl_graph_destroy(pl_graph *g) {
  if (g) cudaStreamSynchronize(g->stream);
  destroy(g);
}

}  // extern "C"

namespace pl {
__global__ void k_clamp_nodes(int64_t N, const uint8_t *nkind, const float2 *fixedp,
                              const float4 *bounds, const float2 *in, float2 *out, int clamp) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    float2 p = in[v];
    if (nkind[v] == 2) p = fixedp[v];
    else if (clamp) {
      float4 bd = bounds[v];
      p.x = fminf(fmaxf(p.x, bd.x), bd.z);
      p.y = fminf(fmaxf(p.y, bd.y), bd.w);
    }
    out[v] = p;
  }
}

pl_status clamp_nodes(pl_graph *g, const pl_params *p, const float *in, float *out,
                      cudaStream_t s) {
  pl::k_clamp_nodes<<<pl::grid_for(g->N, 256), 256, 0, s>>>(
      g->N, pl::P<uint8_t>(g->nkind), pl::P<float2>(g->fixedp), pl::P<float4>(g->bounds),
      reinterpret_cast<const float2 *>(in), reinterpret_cast<float2 *>(out), p->clamp);
  note_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PL_OK : pl::cuda_fail(e, "clamp");
}

}  // namespace pl
