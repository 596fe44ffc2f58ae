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

// ------------------------------------------------ TMA pipeline (bulk copies)
// Work items: hub chunks [0, nchunks), then short tiles.  A persistent CTA
// takes items blockIdx.x, blockIdx.x + gridDim.x, ...; thread 0 keeps the
// index/weight range of the next items (and a tile's row pointers) in flight
// in shared-memory stages with cp.async.bulk on an mbarrier per stage, so the
// DRAM stream does not wait for the gathers and reductions of the current item.
// Every wait on an mbarrier is bounded; on expiry the CTA raises ST_TIMEOUT,
// waits (bounded) for its own copies in flight and returns.
constexpr int kThreadRow = 32;
constexpr int kEntCap = kTile + kLong + 16;  // aligned entries of one item
constexpr int kRowCap = kTile + 8;           // aligned row pointers of one tile
constexpr long long kWaitLimit = 1LL << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_arrive(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kWaitLimit; ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(policy)
      : "memory");
}

template <int WT>
struct StageT {
  int32_t col[kEntCap];
  typename std::conditional<WT == 0, float, uint16_t>::type w[kEntCap];
  uint32_t rp[kRowCap];
};

struct ItemDesc {
  uint64_t e0, e1, ea;  // entries [e0, e1) of the item; stage holds [ea, ea + count)
  int32_t r0, r1, ra;   // tile rows [r0, r1); stage row pointers start at ra
  int32_t chunk;        // >= 0 for a hub chunk
};

// Decode item `it` and issue its copies into stage `st` (thread 0 only).
template <int WT>
__device__ void issue_item(const StepArgs &A, long long it, StageT<WT> &st, ItemDesc &d,
                           uint32_t bar, uint64_t policy) {
  uint64_t e0, e1;
  if (it < A.nchunks) {
    const int c = (int)it, l = A.chunk_lr[c];
    const uint64_t beg = A.lptr[l], end = A.lptr[l + 1];
    e0 = beg + (uint64_t)(c - A.lchunk[l]) * kChunk;
    e1 = e0 + kChunk < end ? e0 + kChunk : end;
    d.chunk = c;
    d.r0 = d.r1 = d.ra = 0;
  } else {
    const int t = (int)(it - A.nchunks);
    d.r0 = A.tile_row[t];
    d.r1 = A.tile_row[t + 1];
    e0 = A.rp_s[d.r0] & kOffMask;
    e1 = A.rp_s[d.r1] & kOffMask;
    d.chunk = -1;
  }
  d.e0 = e0;
  d.e1 = e1;
  const uint64_t ea = e0 & ~uint64_t(7), eb = (e1 + 7) & ~uint64_t(7);
  d.ea = ea;
  const uint32_t ne = (uint32_t)(eb - ea);
  uint32_t nr = 0;
  if (d.chunk < 0) {
    d.ra = d.r0 & ~3;
    nr = (uint32_t)((((d.r1 + 1) + 3) & ~3) - d.ra);
  }
  const uint32_t bytes = ne * 4u + ne * (uint32_t)sizeof(st.w[0]) + nr * 4u;
  mbar_expect_arrive(bar, bytes);
  if (ne) {
    bulk_g2s(smem_u32(st.col), A.col + ea, ne * 4u, bar, policy);
    using WTy = typename std::conditional<WT == 0, float, uint16_t>::type;
    static_assert(sizeof(st.w[0]) == sizeof(WTy), "weight element size");
    bulk_g2s(smem_u32(st.w), reinterpret_cast<const WTy *>(A.w) + ea,
             ne * (uint32_t)sizeof(WTy), bar, policy);
  }
  if (nr) bulk_g2s(smem_u32(st.rp), A.rp_s + d.ra, nr * 4u, bar, policy);
}

template <int WT>
__device__ __forceinline__ float wval(const StageT<WT> &st, uint32_t k) {
  if (WT == 0) return (float)st.w[k];
  return __uint_as_float((uint32_t)st.w[k] << 16);
}

template <int WT, int MODE>
__device__ void tile_item(const StepArgs &A, const StageT<WT> &st, const ItemDesc &d, float2 *sp,
                          int *wide, int *nwide) {
  const int nrows = d.r1 - d.r0;
  const uint32_t n = (uint32_t)(d.e1 - d.e0), off = (uint32_t)(d.e0 - d.ea);
  for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
    const int c = st.col[off + k];
    const float wv = wval<WT>(st, off + k);
    const float2 xv = __ldg(A.x + c);
    sp[k] = make_float2(wv * xv.x, wv * xv.y);
  }
  __syncthreads();
  const float bconst = MODE == MODE_HR ? (float)A.lam[1] : 0.f;
  const uint32_t base = (uint32_t)d.e0;
  const int rb = d.r0 - d.ra;
  for (int j = threadIdx.x; j < nrows; j += blockDim.x) {
    const uint32_t raw = st.rp[rb + j];
    if (raw & kHubFlag) continue;
    const uint32_t a = (raw & kOffMask) - base, b = (st.rp[rb + j + 1] & kOffMask) - base;
    if (b - a > (uint32_t)kThreadRow) {
      wide[atomicAdd(nwide, 1)] = j;
      continue;
    }
    float sx = 0.f, sy = 0.f;
    for (uint32_t k = a; k < b; ++k) {
      const float2 q = sp[k];
      sx += q.x;
      sy += q.y;
    }
    const int r = d.r0 + j;
    const float av = A.a[r];
    const float bv = MODE == MODE_HR ? bconst : A.b[r];
    const float2 xv = A.x[r];
    epilogue<float>(A, r, av * xv.x + bv * sx, av * xv.y + bv * sy);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = wid; q < *nwide; q += nw) {
    const int j = wide[q], r = d.r0 + j;
    const uint32_t a = (st.rp[rb + j] & kOffMask) - base, b = (st.rp[rb + j + 1] & kOffMask) - base;
    float sx = 0.f, sy = 0.f;
    for (uint32_t k = a + lane; k < b; k += 32) {
      const float2 v = sp[k];
      sx += v.x;
      sy += v.y;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) {
      const float av = A.a[r];
      const float bv = MODE == MODE_HR ? bconst : A.b[r];
      const float2 xv = A.x[r];
      epilogue<float>(A, r, av * xv.x + bv * sx, av * xv.y + bv * sy);
    }
  }
}

template <int WT, int MODE>
__device__ void chunk_item(const StepArgs &A, const StageT<WT> &st, const ItemDesc &d,
                           dfl (*red)[32], double (*fin)[32], int *last) {
  const int c = d.chunk, l = A.chunk_lr[c];
  const int64_t v = A.lrow[l];
  const int c0 = A.lchunk[l], nch = A.lchunk[l + 1] - c0;
  const uint32_t n = (uint32_t)(d.e1 - d.e0), off = (uint32_t)(d.e0 - d.ea);
  dfl sx{0.f, 0.f}, sy{0.f, 0.f};
  for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
    const int cc = st.col[off + k];
    const float wv = wval<WT>(st, off + k);
    const float2 xv = __ldg(A.x + cc);
    df_add_prod(sx, wv, xv.x);
    df_add_prod(sy, wv, xv.y);
  }
  sx = warp_sum_df(sx);
  sy = warp_sum_df(sy);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    red[0][wid] = sx;
    red[1][wid] = sy;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double px = 0.0, py = 0.0;
    for (int k = 0; k < nw; ++k) {
      px += df_to_d(red[0][k]);
      py += df_to_d(red[1][k]);
    }
    A.part[2 * (int64_t)c] = px;
    A.part[2 * (int64_t)c + 1] = py;
    __threadfence();
    *last = atomicAdd(&A.tick[l], 1) == nch - 1;
  }
  __syncthreads();
  if (*last) {
    // the row's partials in chunk order: thread k adds chunks k, k + blockDim,
    // ..., then a fixed tree over threads (deterministic)
    __threadfence();
    double tx = 0.0, ty = 0.0;
    for (int k = threadIdx.x; k < nch; k += blockDim.x) {
      tx += __ldcg(&A.part[2 * (int64_t)(c0 + k)]);
      ty += __ldcg(&A.part[2 * (int64_t)(c0 + k) + 1]);
    }
    tx = warp_sum(tx);
    ty = warp_sum(ty);
    if (lane == 0) {
      fin[0][wid] = tx;
      fin[1][wid] = ty;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      tx = 0.0;
      ty = 0.0;
      for (int k = 0; k < nw; ++k) {
        tx += fin[0][k];
        ty += fin[1][k];
      }
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
}

template <int WT>
constexpr int stages_for() { return WT == 0 ? 2 : 3; }

template <int WT, int MODE>
__global__ void __launch_bounds__(256) k_spmm(StepArgs A) {
  constexpr int S = stages_for<WT>();
  extern __shared__ __align__(128) unsigned char smem[];
  StageT<WT> *stage = reinterpret_cast<StageT<WT> *>(smem);
  float2 *sp = reinterpret_cast<float2 *>(smem + S * sizeof(StageT<WT>));
  __shared__ __align__(8) uint64_t bars[S];
  __shared__ ItemDesc desc[S];
  __shared__ int wide[(kTile + kLong) / (kThreadRow + 1) + 1];
  __shared__ int nwide, last, abort_;
  __shared__ dfl red[2][32];
  __shared__ double fin[2][32];
  const long long nitems = (long long)A.nchunks + A.ntiles;
  uint64_t policy = 0;
  if (threadIdx.x == 0) {
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    for (int k = 0; k < S; ++k) mbar_init(smem_u32(&bars[k]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_ = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < S; ++k) {
      const long long it = blockIdx.x + (long long)k * gridDim.x;
      if (it < nitems) issue_item<WT>(A, it, stage[k], desc[k], smem_u32(&bars[k]), policy);
    }
  uint32_t phase = 0;  // bit k: parity to wait for on stage k
  int k = 0;
  for (long long it = blockIdx.x; it < nitems; it += gridDim.x, k = (k + 1 == S) ? 0 : k + 1) {
    if (!mbar_wait(smem_u32(&bars[k]), (phase >> k) & 1u)) abort_ = 1;
    phase ^= 1u << k;
    if (threadIdx.x == 0) nwide = 0;
    __syncthreads();
    if (abort_) break;
    if (desc[k].chunk >= 0) chunk_item<WT, MODE>(A, stage[k], desc[k], red, fin, &last);
    else tile_item<WT, MODE>(A, stage[k], desc[k], sp, wide, &nwide);
    __syncthreads();
    if (threadIdx.x == 0) {
      const long long nx = it + (long long)S * gridDim.x;
      if (nx < nitems) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_item<WT>(A, nx, stage[k], desc[k], smem_u32(&bars[k]), policy);
      }
    }
  }
  if (abort_ && threadIdx.x == 0) {
    flag(A.status, ST_TIMEOUT);
    // copies possibly still in flight into this CTA's stages: wait (bounded)
    for (int q = 0; q < S; ++q) mbar_wait(smem_u32(&bars[q]), (phase >> q) & 1u);
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

template <int WT, int MODE>
static size_t step_smem() {
  return (size_t)stages_for<WT>() * sizeof(StageT<WT>) + (size_t)(kTile + kLong) * sizeof(float2);
}

template <int MODE>
static cudaError_t launch_step(const StepArgs &A, const SpMat &m, int wdtype, cudaStream_t s) {
  const long long nitems = (long long)A.nchunks + A.ntiles;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 152;
  }
  const int grid = (int)(nitems < 2LL * nsm ? nitems : 2LL * nsm);
  const bool prof = prof_on();
  if (prof) prof_begin(s, MODE == MODE_HR ? PROF_HR : PROF_GIFT, spmm_bytes(m, wdtype));
  if (wdtype == PL_W_BF16) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_spmm<1, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)step_smem<1, MODE>());
      attr = true;
    }
    k_spmm<1, MODE><<<grid, 256, step_smem<1, MODE>(), s>>>(A);
  } else {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_spmm<0, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)step_smem<0, MODE>());
      attr = true;
    }
    k_spmm<0, MODE><<<grid, 256, step_smem<0, MODE>(), s>>>(A);
  }
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
