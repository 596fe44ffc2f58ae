// A0 and A4: graph filters as repeated sparse products, GPU-side.
//
// One launch computes, for every node v,  y_v = a_v x_v + b_v sum_j w_vj x_j
// on interleaved (x, y) coordinate pairs:
//   refinement filter  (Sec. V):  a_v = 1 - D_vv / lambda_up, b = 1/lambda_up,
//                                 i.e. y = ((lambda_up I - L_hint)/lambda_up) x;
//   GiFt band filter   (Sec. IV): with u = D_sigma^{-1/2} g carried between
//                                 steps, a_v = sigma / d_v, b_v = 1 / d_v,
//                                 d_v = D_vv + sigma, i.e. u' = D_sigma^{-1}(A + sigma I) u.
// Short rows (<= kLong entries): a CTA stages the products of an nnz tile in
// shared memory (coalesced 16-byte index/weight loads, gathered x), then sums
// each row with a warp.  Hub rows (virtual nodes, very long rows): chunks of
// kChunk entries accumulate exact products in double-float; the last chunk of
// a row to finish (ticket) adds the partials in chunk order in FP64 and does
// the combine in FP64, since those rows amplify rounding error by up to
// a_v^k when D_vv < 0.
// The epilogue also applies the taps (FP64 accumulation), the re-pinning of
// fixed nodes, the relaxation of Algorithm 1 (FP64) and the clamping.
#include <cmath>
#include <type_traits>

#include "pl_internal.h"

namespace pl {

#define TRY(x)                                       \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

enum { MODE_HR = 0, MODE_GIFT = 1 };

struct StepArgs {
  const uint32_t *rp_s;
  const int32_t *col;
  const void *w;
  const int32_t *tile_row;
  int32_t ntiles;
  const int32_t *lrow;
  const uint64_t *lptr;
  const int32_t *lchunk;
  const int32_t *chunk_lr;
  int32_t nchunks;
  const int32_t *longidx;
  double *part;
  int32_t *tick;
  const float2 *x;
  float2 *y;
  // coefficients
  const float *a;        // per row a_v (FP32)
  const float *b;        // per row b_v (GIFT) or nullptr (HR: lam[1])
  const double *c64l;    // HR hub rows: a_v in FP64
  const double *lam;     // HR: lambda_up, 1/lambda_up
  const float *tscale;   // GIFT: band value = u * tscale (sqrt(d_v)); nullptr: 1
  // epilogue
  int pin, tap, fin, relax, clamp;
  double alpha, gamma, cx, cy;
  int single;            // final value is y itself (one tap, alpha 1)
  double2 *acc;
  const float2 *g0;
  float2 *gnext;
  const uint8_t *nkind;
  const float2 *fixedp;
  const float4 *bounds;
  int *status;
};

template <typename T>
__device__ __forceinline__ void epilogue(const StepArgs &A, int64_t v, T yx, T yy) {
  const uint8_t kd = A.nkind[v];
  if (A.pin && kd == 2) {
    float2 f = A.fixedp[v];
    yx = (T)f.x;
    yy = (T)f.y;
  }
  if (!A.fin) A.y[v] = make_float2((float)yx, (float)yy);
  double tx = 0.0, ty = 0.0;
  if (A.tap) {
    double sc = A.tscale ? (double)A.tscale[v] : 1.0;
    double2 ac = A.acc[v];
    ac.x += A.alpha * ((double)yx * sc);
    ac.y += A.alpha * ((double)yy * sc);
    A.acc[v] = ac;
    tx = ac.x;
    ty = ac.y;
  }
  if (A.fin) {
    double gx, gy;
    if (A.single) {
      gx = (double)yx;
      gy = (double)yy;
    } else {
      gx = tx;
      gy = ty;
    }
    gx += A.cx;
    gy += A.cy;
    float ox, oy;
    if (kd == 2) {
      float2 f = A.fixedp[v];
      ox = f.x;
      oy = f.y;
    } else {
      if (A.relax) {
        float2 g = A.g0[v];
        gx = (1.0 - A.gamma) * (double)g.x + A.gamma * gx;
        gy = (1.0 - A.gamma) * (double)g.y + A.gamma * gy;
      }
      ox = __double2float_rn(gx);
      oy = __double2float_rn(gy);
      if (A.clamp) {
        float4 bd = A.bounds[v];
        ox = fminf(fmaxf(ox, bd.x), bd.z);
        oy = fminf(fmaxf(oy, bd.y), bd.w);
      }
    }
    A.gnext[v] = make_float2(ox, oy);
  }
}

// ------------------------------------------------------- warp work units
// Units: hub chunks [0, nchunks) of kChunk entries, then short tiles of at
// most kTile keys (rows + entries; rows <= kLong entries).  Each warp takes
// units gw, gw + nwarps, ...; a unit needs no block-wide barrier.
//  * tile: the lanes load the unit's indices and weights (all loads issued
//    before the gathers), write w * x[col] to the warp's shared-memory slice,
//    then each lane sums whole rows (lane per row) and runs their epilogue;
//  * hub chunk: exact products accumulated in double-float, reduced over the
//    warp, written as an FP64 partial; the last warp to finish a row (ticket,
//    no waiting) adds the row's partials in chunk order (lane-strided, then a
//    fixed tree) and combines in FP64.
constexpr int kEntWarp = kTile + kLong;  // entries of one tile < kTile + kLong
constexpr int kBatch = 4;                // loads in flight per lane and batch

template <int WT>
__device__ __forceinline__ float wload(const void *w, uint64_t k) {
  if (WT == 0) return __ldcs(reinterpret_cast<const float *>(w) + k);
  return __uint_as_float((uint32_t)__ldcs(reinterpret_cast<const unsigned short *>(w) + k) << 16);
}

template <int WT, int MODE>
__device__ void warp_tile(const StepArgs &A, int t, float2 *sp) {
  const int lane = threadIdx.x & 31;
  const int r0 = A.tile_row[t], r1 = A.tile_row[t + 1];
  const uint32_t e0 = A.rp_s[r0] & kOffMask, e1 = A.rp_s[r1] & kOffMask;
  const uint32_t n = e1 - e0;
  for (uint32_t k0 = 0; k0 < n; k0 += 32 * kBatch) {
    int c[kBatch];
    float wv[kBatch];
#pragma unroll
    for (int q = 0; q < kBatch; ++q) {
      const uint32_t k = k0 + q * 32 + lane;
      c[q] = k < n ? __ldcs(A.col + e0 + k) : 0;
      wv[q] = k < n ? wload<WT>(A.w, e0 + k) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kBatch; ++q) {
      const uint32_t k = k0 + q * 32 + lane;
      if (k < n) {
        const float2 xv = __ldg(A.x + c[q]);
        sp[k] = make_float2(wv[q] * xv.x, wv[q] * xv.y);
      }
    }
  }
  __syncwarp();
  const float bconst = MODE == MODE_HR ? (float)A.lam[1] : 0.f;
  for (int r = r0 + lane; r < r1; r += 32) {
    const uint32_t raw = A.rp_s[r];
    if (raw & kHubFlag) continue;
    const uint32_t a = (raw & kOffMask) - e0, b = (A.rp_s[r + 1] & kOffMask) - e0;
    float sx = 0.f, sy = 0.f;
    for (uint32_t k = a; k < b; ++k) {
      const float2 q = sp[k];
      sx += q.x;
      sy += q.y;
    }
    const float av = A.a[r];
    const float bv = MODE == MODE_HR ? bconst : A.b[r];
    const float2 xv = A.x[r];
    epilogue<float>(A, r, av * xv.x + bv * sx, av * xv.y + bv * sy);
  }
  __syncwarp();
}

template <int WT, int MODE>
__device__ void warp_chunk(const StepArgs &A, int c) {
  const int lane = threadIdx.x & 31;
  const int l = A.chunk_lr[c];
  const int64_t v = A.lrow[l];
  const uint64_t beg = A.lptr[l], end = A.lptr[l + 1];
  const int c0 = A.lchunk[l], nch = A.lchunk[l + 1] - c0;
  const uint64_t cb = beg + (uint64_t)(c - c0) * kChunk;
  const uint64_t ce = cb + kChunk < end ? cb + kChunk : end;
  dfl sx{0.f, 0.f}, sy{0.f, 0.f};
  for (uint64_t k0 = cb; k0 < ce; k0 += 32 * kBatch) {
    int cc[kBatch];
    float wv[kBatch];
#pragma unroll
    for (int q = 0; q < kBatch; ++q) {
      const uint64_t k = k0 + q * 32 + lane;
      cc[q] = k < ce ? __ldcs(A.col + k) : 0;
      wv[q] = k < ce ? wload<WT>(A.w, k) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kBatch; ++q) {
      const uint64_t k = k0 + q * 32 + lane;
      if (k < ce) {
        const float2 xv = __ldg(A.x + cc[q]);
        df_add_prod(sx, wv[q], xv.x);
        df_add_prod(sy, wv[q], xv.y);
      }
    }
  }
  sx = warp_sum_df(sx);
  sy = warp_sum_df(sy);
  int last = 0;
  if (lane == 0) {
    A.part[2 * (int64_t)c] = df_to_d(sx);
    A.part[2 * (int64_t)c + 1] = df_to_d(sy);
    __threadfence();
    last = atomicAdd(&A.tick[l], 1) == nch - 1;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  double tx = 0.0, ty = 0.0;
  for (int k = lane; k < nch; k += 32) {
    tx += __ldcg(&A.part[2 * (int64_t)(c0 + k)]);
    ty += __ldcg(&A.part[2 * (int64_t)(c0 + k) + 1]);
  }
  tx = warp_sum(tx);
  ty = warp_sum(ty);
  if (lane == 0) {
    double av, bv;
    if (MODE == MODE_HR) {
      av = A.c64l[l];
      bv = A.lam[1];
    } else {
      av = (double)A.a[v];
      bv = (double)A.b[v];
    }
    const float2 xv = A.x[v];
    epilogue<double>(A, v, av * (double)xv.x + bv * tx, av * (double)xv.y + bv * ty);
    A.tick[l] = 0;
  }
}

constexpr int kSpmmThreads = 256;

template <int WT, int MODE>
__global__ void __launch_bounds__(kSpmmThreads) k_spmm(StepArgs A) {
  __shared__ float2 sp_all[kSpmmThreads / 32][kEntWarp];
  float2 *sp = sp_all[threadIdx.x >> 5];
  const long long nunits = (long long)A.nchunks + A.ntiles;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long u = gw; u < nunits; u += nw) {
    if (u < A.nchunks) warp_chunk<WT, MODE>(A, (int)u);
    else warp_tile<WT, MODE>(A, (int)(u - A.nchunks), sp);
  }
}

// ------------------------------------------------------------- helpers
__global__ void k_init_signal(int64_t N, int32_t C, uint64_t seed, const float2 *xy0,
                              const uint8_t *nkind, const float2 *fixedp, double xl, double yl,
                              double xh, double yh, float2 *g) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    uint8_t k = nkind[v];
    float2 o = make_float2(0.f, 0.f);
    if (k == 2) {
      o = fixedp[v];
    } else if (v < C) {
      if (xy0) {
        o = xy0[v];
      } else {
        double ux = u01(seed, 2ull * (uint64_t)v), uy = u01(seed, 2ull * (uint64_t)v + 1ull);
        o = make_float2(__double2float_rn(__dadd_rn(xl, __dmul_rn(ux, xh - xl))),
                        __double2float_rn(__dadd_rn(yl, __dmul_rn(uy, yh - yl))));
      }
    }
    g[v] = o;
  }
}

// Star node = mean of its net's distinct nodes (warp per star, FP64).
__global__ void k_star_init(int32_t S, int64_t star0, const int32_t *star_net,
                            const int64_t *net_ptr, const uint32_t *nd, const int32_t *net_p,
                            float2 *g) {
  const int lane = threadIdx.x & 31;
  for (long long s = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; s < S;
       s += ((long long)gridDim.x * blockDim.x) >> 5) {
    int e = star_net[s];
    long long b = net_ptr[e];
    int p = net_p[e];
    double sx = 0.0, sy = 0.0;
    for (int k = lane; k < p; k += 32) {
      float2 q = g[nd[b + k]];
      sx += q.x;
      sy += q.y;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) g[star0 + s] = make_float2(__double2float_rn(sx / p), __double2float_rn(sy / p));
  }
}

__global__ void k_clamp(int64_t N, const uint8_t *nkind, const float2 *fixedp,
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

// GiFt per-node coefficients of one sigma: a = sigma/d, b = 1/d, band scale
// sqrt(d), and u0 = (g - centre)/sqrt(d), d = D_vv + sigma.
__global__ void k_gift_prep(int64_t N, int64_t Nst, const double *sdeg, double sigma,
                            const float2 *g, double cx, double cy, float *a, float *b,
                            float *sq, float2 *u0) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    double d = (v < Nst ? sdeg[v] : 0.0) + sigma;
    double r = sqrt(d);
    a[v] = (float)(sigma / d);
    b[v] = (float)(1.0 / d);
    sq[v] = (float)r;
    float2 q = g[v];
    u0[v] = make_float2((float)(((double)q.x - cx) / r), (float)(((double)q.y - cy) / r));
  }
}

__global__ void k_acc_add(int64_t N, const float2 *u, const float *sq, double alpha,
                          double2 *acc) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    double2 a = acc[v];
    a.x += alpha * ((double)u[v].x * (double)sq[v]);
    a.y += alpha * ((double)u[v].y * (double)sq[v]);
    acc[v] = a;
  }
}

__global__ void k_acc_final(int64_t N, const double2 *acc, double cx, double cy,
                            const uint8_t *nkind, const float2 *fixedp, const float4 *bounds,
                            int clamp, float2 *out) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    float2 o;
    if (nkind[v] == 2) {
      o = fixedp[v];
    } else {
      o = make_float2(__double2float_rn(acc[v].x + cx), __double2float_rn(acc[v].y + cy));
      if (clamp) {
        float4 bd = bounds[v];
        o.x = fminf(fmaxf(o.x, bd.x), bd.z);
        o.y = fminf(fmaxf(o.y, bd.y), bd.w);
      }
    }
    out[v] = o;
  }
}

// --------------------------------------------------------------- drivers
static void fill_matrix(StepArgs &A, const SpMat &m) {
  A.rp_s = P<uint32_t>(m.rp_s);
  A.col = P<int32_t>(m.col);
  A.w = m.w.p;
  A.tile_row = P<int32_t>(m.tile_row);
  A.ntiles = m.ntiles;
  A.lrow = P<int32_t>(m.lrow);
  A.lptr = P<uint64_t>(m.lptr);
  A.lchunk = P<int32_t>(m.lchunk);
  A.chunk_lr = P<int32_t>(m.chunk_lr);
  A.nchunks = m.nchunks;
  A.longidx = P<int32_t>(m.longidx);
  A.part = const_cast<double *>(P<double>(m.part));
  A.tick = const_cast<int32_t *>(P<int32_t>(m.tick));
}

// Algorithmic bytes of one sparse product over (x, y) pairs: indices and
// weights once, row pointers, x read, y written, one coefficient per row.
static double spmm_bytes(const SpMat &m, int wdtype) {
  const double nnz = (double)(m.nnz_s + m.nnz_l), N = (double)m.N;
  return nnz * (4.0 + (wdtype == PL_W_BF16 ? 2.0 : 4.0)) + (N + 1.0) * 4.0 + N * (8.0 + 8.0 + 4.0);
}

template <int MODE>
static cudaError_t launch_step(const StepArgs &A, const SpMat &m, int wdtype, cudaStream_t s) {
  const long long nunits = (long long)A.nchunks + A.ntiles;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 152;
  }
  const long long want = (nunits + kSpmmThreads / 32 - 1) / (kSpmmThreads / 32);
  const int grid = (int)(want < 8LL * nsm ? (want > 0 ? want : 1) : 8LL * nsm);
  const bool prof = prof_on();
  if (prof) prof_begin(s, MODE == MODE_HR ? PROF_HR : PROF_GIFT, spmm_bytes(m, wdtype));
  if (wdtype == PL_W_BF16) k_spmm<1, MODE><<<grid, kSpmmThreads, 0, s>>>(A);
  else k_spmm<0, MODE><<<grid, kSpmmThreads, 0, s>>>(A);
  note_launch();
  if (prof) prof_end(s);
  return cudaGetLastError();
}

static void fill_nodes(StepArgs &A, pl_graph *g) {
  A.status = P<int>(g->status);
  A.nkind = P<uint8_t>(g->nkind);
  A.fixedp = P<float2>(g->fixedp);
  A.bounds = P<float4>(g->bounds);
}

pl_status run_init_signal(pl_graph *g, uint64_t seed, const float *xy0, float *xy,
                          cudaStream_t s) {
  float2 *out = reinterpret_cast<float2 *>(xy);
  k_init_signal<<<grid_for(g->N, 256), 256, 0, s>>>(
      g->N, g->C, seed, reinterpret_cast<const float2 *>(xy0), P<uint8_t>(g->nkind),
      P<float2>(g->fixedp), g->xl, g->yl, g->xh, g->yh, out);
  note_launch();
  if (g->S) {
    k_star_init<<<grid_for((long long)g->S * 32, 256), 256, 0, s>>>(
        g->S, (int64_t)g->C + g->Pm, P<int32_t>(g->star_net), P<int64_t>(g->net_ptr),
        P<uint32_t>(g->nd), P<int32_t>(g->net_p), out);
    note_launch();
  }
  TRY(cudaGetLastError());
  return PL_OK;
}

pl_status run_gift(pl_graph *g, const pl_params *p, const float *in, float *out, cudaStream_t s) {
  const int64_t N = g->N;
  const float2 *gin = reinterpret_cast<const float2 *>(in);
  float2 *gout = reinterpret_cast<float2 *>(out);
  const double cx = p->gift_center ? 0.5 * (g->xl + g->xh) : 0.0;
  const double cy = p->gift_center ? 0.5 * (g->yl + g->yh) : 0.0;
  // chains of equal sigma, in order of first appearance
  double sig[3];
  int kmax[3], nch = 0, chain_of[3];
  for (int bnd = 0; bnd < 3; ++bnd) {
    int q = -1;
    for (int k = 0; k < nch; ++k)
      if (sig[k] == p->gift_sigma[bnd]) q = k;
    if (q < 0) {
      q = nch++;
      sig[q] = p->gift_sigma[bnd];
      kmax[q] = 0;
    }
    chain_of[bnd] = q;
    if (p->gift_k[bnd] > kmax[q]) kmax[q] = p->gift_k[bnd];
  }
  TRY(ensure(g->acc, (size_t)N * 16 + 16));
  TRY(cudaMemsetAsync(g->acc.p, 0, (size_t)N * 16, s));
  TRY(ensure(g->gsc, (size_t)N * 12 + 64));
  TRY(ensure(g->ua, (size_t)N * 8 + 64));
  TRY(ensure(g->ub, (size_t)N * 8 + 64));
  TRY(ensure(g->xa, (size_t)N * 8 + 64));
  float *ga = P<float>(g->gsc), *gb = ga + N, *gq = gb + N;
  StepArgs A{};
  fill_matrix(A, g->st);
  fill_nodes(A, g);
  A.acc = P<double2>(g->acc);
  A.tscale = gq;
  A.a = ga;
  A.b = gb;
  A.relax = 0;
  A.clamp = p->clamp;
  A.gnext = gout;
  A.single = 0;
  // find the chain that finishes last (the final step)
  int last_chain = -1;
  for (int q = 0; q < nch; ++q)
    if (kmax[q] > 0) last_chain = q;
  bool any = false;
  for (int q = 0; q < nch; ++q) {
    k_gift_prep<<<grid_for(N, 256), 256, 0, s>>>(N, g->Nst, P<double>(g->sdeg), sig[q], gin, cx,
                                                 cy, ga, gb, gq, P<float2>(g->ua));
    note_launch();
    // bands with k = 0 contribute alpha * (g - centre)
    for (int bnd = 0; bnd < 3; ++bnd) {
      if (chain_of[bnd] != q || p->gift_k[bnd] != 0) continue;
      k_acc_add<<<grid_for(N, 256), 256, 0, s>>>(N, P<float2>(g->ua), gq, p->gift_alpha[bnd],
                                                 P<double2>(g->acc));
      note_launch();
    }
    float2 *x = P<float2>(g->ua), *y = P<float2>(g->ub);
    for (int t = 1; t <= kmax[q]; ++t) {
      A.x = x;
      A.y = y;
      A.tap = 0;
      A.alpha = 0.0;
      for (int bnd = 0; bnd < 3; ++bnd)
        if (chain_of[bnd] == q && p->gift_k[bnd] == t) {
          A.tap = 1;
          A.alpha += p->gift_alpha[bnd];
        }
      A.fin = (q == last_chain && t == kmax[q]) ? 1 : 0;
      A.cx = A.fin ? cx : 0.0;
      A.cy = A.fin ? cy : 0.0;
      A.pin = 0;
      TRY(launch_step<MODE_GIFT>(A, g->st, g->wdtype, s));
      any = true;
      float2 *tt = x;
      x = y;
      y = tt;
    }
  }
  if (!any) {
    // every band has k = 0: the filter is sum(alpha) * g
    k_acc_final<<<grid_for(N, 256), 256, 0, s>>>(N, P<double2>(g->acc), cx, cy, P<uint8_t>(g->nkind),
                                                 P<float2>(g->fixedp), P<float4>(g->bounds),
                                                 p->clamp, gout);
    note_launch();
  }
  TRY(cudaGetLastError());
  return PL_OK;
}

pl_status run_filter(pl_graph *g, const pl_params *p, const float *in, float *out,
                     cudaStream_t s) {
  const int64_t N = g->N;
  const float2 *gin = reinterpret_cast<const float2 *>(in);
  float2 *gout = reinterpret_cast<float2 *>(out);
  if (p->gamma == 0.0) {
    k_clamp<<<grid_for(N, 256), 256, 0, s>>>(N, P<uint8_t>(g->nkind), P<float2>(g->fixedp),
                                             P<float4>(g->bounds), gin, gout, p->clamp);
    note_launch();
    TRY(cudaGetLastError());
    return PL_OK;
  }
  const int kmax = p->tap_k[p->ntaps - 1];
  const bool single = p->ntaps == 1 && p->tap_alpha[0] == 1.0;
  TRY(ensure(g->xa, (size_t)N * 8 + 64));
  TRY(ensure(g->xb, (size_t)N * 8 + 64));
  if (!single) {
    TRY(ensure(g->acc, (size_t)N * 16 + 16));
    TRY(cudaMemsetAsync(g->acc.p, 0, (size_t)N * 16, s));
  }
  const SpMat &m = g->hm;
  StepArgs A{};
  fill_matrix(A, m);
  fill_nodes(A, g);
  A.a = P<float>(m.c32);
  A.b = nullptr;
  A.c64l = P<double>(m.c64l);
  A.lam = P<double>(m.lam);
  A.tscale = nullptr;
  A.acc = P<double2>(g->acc);
  A.g0 = gin;
  A.gnext = gout;
  A.gamma = p->gamma;
  A.relax = 1;
  A.clamp = p->clamp;
  A.single = single ? 1 : 0;
  A.pin = p->pin_every_step;
  A.cx = A.cy = 0.0;
  const float2 *x = gin;
  float2 *bufs[2] = {P<float2>(g->xa), P<float2>(g->xb)};
  for (int t = 1; t <= kmax; ++t) {
    A.x = x;
    A.y = bufs[t & 1];
    A.tap = 0;
    A.alpha = 0.0;
    if (!single)
      for (int j = 0; j < p->ntaps; ++j)
        if (p->tap_k[j] == t) {
          A.tap = 1;
          A.alpha = p->tap_alpha[j];
        }
    A.fin = t == kmax;
    TRY(launch_step<MODE_HR>(A, m, g->wdtype, s));
    x = bufs[t & 1];
  }
  return PL_OK;
}

}  // namespace pl
