// A0 and A4: graph filters as repeated sparse products, GPU-side.
//
// One launch computes, for every node v,  y_v = a_v x_v + b_v sum_j w_vj x_j
// on interleaved (x, y) coordinate pairs:
//   refinement filter  (Sec. V):  a_v = 1 - D_vv / lambda_up, b = 1/lambda_up,
//                                 i.e. y = ((lambda_up I - L_hint)/lambda_up) x;
//   GiFt band filter   (Sec. IV): with u = D_sigma^{-1/2} g carried between
//                                 steps, a_v = sigma / d_v, b_v = 1 / d_v,
//                                 d_v = D_vv + sigma, i.e. u' = D_sigma^{-1}(A + sigma I) u.
// Short rows (<= kLong entries): a group of two lanes per row reads the row's
// indices and weights from global memory with several loads in flight per
// lane, gathers x and sums in FP32.  Hub rows (virtual nodes, very long rows): chunks of
// kChunk entries accumulate exact products in double-float (one launch); the
// next launch adds each hub row's partials in a fixed order and does the
// combine in FP64, since those rows amplify rounding error by up to a_v^k when
// D_vv < 0.
// The epilogue also applies the taps (FP64 accumulation), the re-pinning of
// fixed nodes, the relaxation of Algorithm 1 (FP64) and the clamping.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "pl_bins.cuh"
#include "pl_internal.h"

namespace pl {

#define TRY(x)                                       \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

enum { MODE_HR = 0, MODE_GIFT = 1 };

struct StepArgs {
  // static part of every row (st) and, for the refinement filter, the hint
  // part (hm; hrp == nullptr for the GiFt filter, which uses st alone)
  const uint32_t *srp;
  const int32_t *scol;
  const void *sw;
  const uint32_t *hrp;
  const int32_t *hcol;
  const void *hw;
  // work units of the applied matrix
  int64_t nrows;  // rows of the applied matrix
  const int32_t *lrow;
  const uint64_t *lsb, *lhb;
  const uint32_t *lsl, *lhl;
  const int32_t *lchunk;
  const int32_t *chunk_lr;
  int32_t nchunks;
  int32_t nlong;
  float4 *part;  // per hub chunk: (sx.hi, sx.lo, sy.hi, sy.lo)
  const float2 *x;
  float2 *y;
  // coefficients
  const float *a;        // per row a_v (FP32)
  const float *b;        // per row b_v (GIFT) or nullptr (HR: binv)
  const double *c64l;    // HR hub rows: a_v in FP64
  double binv;           // HR: 1 / lambda_up
  float binvf;           // the same, rounded to FP32
  const float *tscale;   // GIFT: band value = u * tscale (sqrt(d_v)); nullptr: 1
  // epilogue
  int pin, tap, fin, relax, clamp;
  double alpha, gamma, omg, cx, cy;  // omg = 1 - gamma
  int addc;                          // cx or cy is not zero
  int single;            // final value is y itself (one tap, alpha 1)
  double2 *acc;
  const float2 *g0;
  float2 *gnext;
  const uint8_t *nkind;
  const float2 *fixedp;
  const float4 *bounds;
  int *status;
  // GiFt hub passes: stride of x and y in float2 units (2 for one chain's
  // half of an interleaved chain pair, else 1)
  int xs;
  // GiFt chain pair (k_spmm_rows4): the second chain's coefficients and tap,
  // and x and y of both chains interleaved as (x1, y1, x2, y2) per node
  const float *a2, *b2, *tscale2;
  int tap2;
  double alpha2;
  const float4 *x4;
  float4 *y4;
  // refinement filter: bin hints without stored columns.  A hint cell v
  // (hbin[v] >= 0) has W window-slot weights hbw[v W + s] towards the bin
  // nodes bn0 + hbin[v] + offset(s); bin rows are the transposes, summed from
  // chunk partials (bpart) of the bins' hint buckets.
  const void *hbw;
  const void *hbwq;  // the same blocks in bucket-list order
  const int32_t *hbin;
  int32_t C;
  int64_t bn0;
  BinGeo B;
  const int32_t *bchunk;
  const int32_t *cown;
  const int64_t *boff;
  const uint32_t *blist;
  float4 *bpart;
  // windows of at most kSlotUnroll * kRowLanes slots: lane m's slot
  // m + u kRowLanes is at bin offset soff[m][u] from the cell's bin
  int sfast;
  int soff[2][5];
};

// Epilogue of node v with its kind kd and (tap steps) accumulator ac loaded
// by the caller.
template <typename T>
__device__ __forceinline__ void epilogue_k(const StepArgs &A, int64_t v, uint8_t kd, double2 ac,
                                           T yx, T yy, int64_t yi) {
  if (A.pin && kd == 2) {
    float2 f = A.fixedp[v];
    yx = (T)f.x;
    yy = (T)f.y;
  }
  if (!A.fin) A.y[yi] = make_float2((float)yx, (float)yy);
  double tx = 0.0, ty = 0.0;
  if (A.tap) {
    double sc = A.tscale ? (double)A.tscale[v] : 1.0;
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

// Final value of coordinate c (0: x, 1: y) of node v from its filter sum gv:
// centre, relaxation, FP32 rounding, clamping; fixed nodes keep their place.
__device__ __forceinline__ void finish_c(const StepArgs &A, int64_t v, uint8_t kd, int c,
                                         double gv) {
  if (A.addc) gv += c ? A.cy : A.cx;
  float o;
  if (kd == 2) {
    o = reinterpret_cast<const float *>(A.fixedp)[2 * v + c];
  } else {
    if (A.relax) {
      const float g = reinterpret_cast<const float *>(A.g0)[2 * v + c];
      gv = A.omg * (double)g + A.gamma * gv;
    }
    o = __double2float_rn(gv);
    if (A.clamp) {
      const float4 bd = A.bounds[v];
      o = c ? fminf(fmaxf(o, bd.y), bd.w) : fminf(fmaxf(o, bd.x), bd.z);
    }
  }
  reinterpret_cast<float *>(A.gnext)[2 * v + c] = o;
}

// The same epilogue for one coordinate c of node v, so that the two lanes of
// a row share its FP64 work.
__device__ __forceinline__ void epilogue_c(const StepArgs &A, int64_t v, uint8_t kd, int c,
                                           double acv, float yv) {
  if (A.pin && kd == 2) yv = reinterpret_cast<const float *>(A.fixedp)[2 * v + c];
  if (!A.fin) reinterpret_cast<float *>(A.y)[2 * v + c] = yv;
  // (FP64 is slow: no product by a unit scale, no sum with a zero centre,
  // 1 - gamma from the host, no store of the last tap sum)
  double t = 0.0;
  if (A.tap) {
    double pv = (double)yv;
    if (A.tscale) pv *= (double)A.tscale[v];
    acv += A.alpha * pv;
    if (!A.fin) reinterpret_cast<double *>(A.acc)[2 * v + c] = acv;
    t = acv;
  }
  if (A.fin) finish_c(A, v, kd, c, A.single ? (double)yv : t);
}

// Epilogue of coordinate c of node v for a GiFt chain pair: both chains'
// values (y1, y2) are stored interleaved and their taps added to the one
// band sum, the first chain's first.
__device__ __forceinline__ void epilogue_c2(const StepArgs &A, int64_t v, uint8_t kd, int c,
                                            double acv, float y1, float y2) {
  if (A.pin && kd == 2) y1 = y2 = reinterpret_cast<const float *>(A.fixedp)[2 * v + c];
  if (!A.fin) {
    float *yp = reinterpret_cast<float *>(A.y4) + 4 * v + c;
    yp[0] = y1;
    yp[2] = y2;
  }
  if (A.tap) {
    double pv = (double)y1;
    if (A.tscale) pv *= (double)A.tscale[v];
    acv += A.alpha * pv;
  }
  if (A.tap2) {
    double pv = (double)y2;
    if (A.tscale2) pv *= (double)A.tscale2[v];
    acv += A.alpha2 * pv;
  }
  if ((A.tap || A.tap2) && !A.fin) reinterpret_cast<double *>(A.acc)[2 * v + c] = acv;
  if (A.fin) finish_c(A, v, kd, c, acv);
}

template <typename T>
__device__ __forceinline__ void epilogue(const StepArgs &A, int64_t v, T yx, T yy, int64_t yi) {
  epilogue_k<T>(A, v, A.nkind[v], A.tap ? A.acc[v] : make_double2(0.0, 0.0), yx, yy, yi);
}

// ------------------------------------------------------- work units
// Hub chunks [0, nchunks) of kChunk entries (first launch), hub rows (second
// launch), then the short rows (third launch); warps take units gw,
// gw + nwarps, ... and no unit needs a block-wide barrier.
//  * hub chunk: exact products accumulated in double-float, reduced over the
//    warp, written as a double-float partial;
//  * hub row: the row's partials added by a warp in a fixed order, then
//    combined in FP64 by a lane per row;
//  * short rows: a group of lanes per row (below).
constexpr int kChunkBatch = 8;  // loads in flight per lane (hub chunks)

template <int WT>
__device__ __forceinline__ float wload(const void *w, uint64_t k) {
  if (WT == 0) return __ldcs(reinterpret_cast<const float *>(w) + k);
  return __uint_as_float((uint32_t)__ldcs(reinterpret_cast<const unsigned short *>(w) + k) << 16);
}

template <int WT>
__device__ __forceinline__ void chunk_piece(const int32_t *colp, const void *wp, uint64_t b,
                                            uint64_t e, const float2 *x, int xs, dfl &sx,
                                            dfl &sy) {
  const int lane = threadIdx.x & 31;
  for (uint64_t k0 = b; k0 < e; k0 += 32 * kChunkBatch) {
    int cc[kChunkBatch];
    float wv[kChunkBatch];
#pragma unroll
    for (int q = 0; q < kChunkBatch; ++q) {
      const uint64_t k = k0 + q * 32 + lane;
      cc[q] = k < e ? __ldcs(colp + k) : 0;
      wv[q] = k < e ? wload<WT>(wp, k) : 0.f;
    }
    float2 xv[kChunkBatch];
#pragma unroll
    for (int q = 0; q < kChunkBatch; ++q) {
      const uint64_t k = k0 + q * 32 + lane;
      xv[q] = k < e ? __ldg(x + (size_t)cc[q] * xs) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < kChunkBatch; ++q) {
      df_add_prod(sx, wv[q], xv[q].x);
      df_add_prod(sy, wv[q], xv[q].y);
    }
  }
}

// A hub chunk covers positions [q0, q1) of the row's st piece followed by its
// hm piece; its double-float sums over the warp are the chunk's partial.
template <int WT, int MODE>
__device__ void warp_chunk(const StepArgs &A, int c) {
  const int lane = threadIdx.x & 31;
  const int xs = MODE == MODE_GIFT ? A.xs : 1;
  const int l = A.chunk_lr[c];
  const int c0 = A.lchunk[l];
  const uint64_t sl = A.lsl[l], hl = A.lhl[l];
  const uint64_t q0 = (uint64_t)(c - c0) * kChunk;
  const uint64_t q1 = q0 + kChunk < sl + hl ? q0 + kChunk : sl + hl;
  dfl sx{0.f, 0.f}, sy{0.f, 0.f};
  if (q0 < sl)
    chunk_piece<WT>(A.scol, A.sw, A.lsb[l] + q0, A.lsb[l] + (q1 < sl ? q1 : sl), A.x, xs, sx, sy);
  if (q1 > sl) {
    const uint64_t hb = A.lhb[l];
    chunk_piece<WT>(A.hcol, A.hw, hb + (q0 > sl ? q0 - sl : 0), hb + (q1 - sl), A.x, xs, sx, sy);
  }
  sx = warp_sum_df(sx);
  sy = warp_sum_df(sy);
  if (lane == 0) A.part[c] = make_float4(sx.hi, sx.lo, sy.hi, sy.lo);
}

// Hub chunks: warp w of the grid takes chunks w, w + nwarps, ...
template <int WT, int MODE>
__global__ void __launch_bounds__(256) k_spmm_hub(StepArgs A) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long c = gw; c < A.nchunks; c += nw) warp_chunk<WT, MODE>(A, (int)c);
}

// Short rows, row-split: a group of kRowLanes lanes per row reads the row's
// st and hm pieces straight from global memory (lane m takes entries m,
// m + kRowLanes, ...; several index and weight loads in flight, then their
// gathers of x), a butterfly over the group sums them, and the group's first
// lane applies the epilogue.  Hub rows are skipped (their own launches).
constexpr int kRowLanes = 2;  // the epilogue takes one coordinate per lane
static_assert(kRowLanes == 2, "the row epilogue splits x and y over the row's two lanes");
constexpr int kRowUnroll = 8;  // entries per lane and pass of a GiFt pair's static row
// A short row's hm piece holds only its macro entries (the bin hints have no
// stored columns), in nearly every warp pass but rarely more than one per
// row: kHmUnroll entries per lane and pass keep that piece to a few
// instructions.
constexpr int kHmUnroll = 2;
constexpr int kRowThreads = 256;
constexpr int kRowCtasSide = 5;  // short-row CTAs per SM beside the hub and bin-row kernels

template <int WT, int L, int U>
__device__ __forceinline__ void row_piece(const int32_t *col, const void *w, uint32_t k,
                                          uint32_t e, const float2 *x, float &sx, float &sy) {
  for (; k < e; k += U * L) {
    int c[U];
    float wv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t kk = k + u * L;
      c[u] = kk < e ? __ldcs(col + kk) : -1;
      wv[u] = kk < e ? wload<WT>(w, kk) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (c[u] >= 0) {
        const float2 xv = __ldg(x + c[u]);
        sx = fmaf(wv[u], xv.x, sx);
        sy = fmaf(wv[u], xv.y, sy);
      }
    }
  }
}

// Window slots of hint cell v (refinement filter): lane m of the row's group
// takes slots m, m + L, ...; the column of a slot is the bin node at the
// cell's bin plus the slot's offset.  Slots outside the bin grid hold weight
// 0, so their bin index is clamped into the grid instead of tested (a finite
// coordinate times 0).  The weights are loaded before their gathers of x.
constexpr int kSlotUnroll = 5;  // slots a lane loads at once (a 3 x 3 window over 2 lanes)
static_assert(kRowLanes == 2 && kSlotUnroll == 5, "StepArgs::soff is [kRowLanes][kSlotUnroll]");
template <int WT, int L>
__device__ __forceinline__ void slot_piece(const StepArgs &A, long long v, int hb, int m, float &sx,
                                           float &sy) {
  if (hb < 0) return;
  const int nbx = A.B.nbx, nby = A.B.nby, wx = 2 * A.B.hx + 1, W = A.B.W;
  const int bx = hb % nbx, by = hb / nbx;
  const float iwx = 1.0f / (float)wx;  // row of a slot: (s + 1/2) / wx, exact below 2^12
  const float *wf = reinterpret_cast<const float *>(A.hbw) + (size_t)v * W;
  const unsigned short *wh = reinterpret_cast<const unsigned short *>(A.hbw) + (size_t)v * W;
  const float2 *xb = A.x + A.bn0;
  for (int s0 = m; s0 < W; s0 += kSlotUnroll * L) {
    float wv[kSlotUnroll];
    int cb[kSlotUnroll];
#pragma unroll
    for (int u = 0; u < kSlotUnroll; ++u) {
      const int sl = s0 + u * L;
      const bool ok = sl < W;
      wv[u] = ok ? (WT == 0 ? __ldcs(wf + sl) : __uint_as_float((uint32_t)__ldcs(wh + sl) << 16)) : 0.f;
      const int iy = (int)(((float)sl + 0.5f) * iwx);
      const int xx = min(max(bx + sl - iy * wx - A.B.hx, 0), nbx - 1);
      const int yy = min(max(by + iy - A.B.hy, 0), nby - 1);
      cb[u] = ok ? yy * nbx + xx : -1;
    }
#pragma unroll
    for (int u = 0; u < kSlotUnroll; ++u) {
      if (cb[u] >= 0) {
        const float2 xv = __ldg(xb + cb[u]);
        sx = fmaf(wv[u], xv.x, sx);
        sy = fmaf(wv[u], xv.y, sy);
      }
    }
  }
}

// The same slots as slot_piece when the window has at most
// kSlotUnroll * kRowLanes of them (the 3 x 3 window of 32 x 32 bins has 9):
// lane m's slots m + u kRowLanes have the bin offsets A.soff[m][u] (dy nbx +
// dx, computed on the host), and the bin of a slot is the cell's bin plus its
// offset, clamped into the grid as a linear index (slots outside the grid
// hold weight 0, so any bin there adds 0).
template <int WT>
__device__ __forceinline__ void slot_piece_fast(const StepArgs &A, long long v, int hb, int m,
                                                float &sx, float &sy) {
  if (hb < 0) return;
  const float *wf = reinterpret_cast<const float *>(A.hbw) + (size_t)v * A.B.W;
  const unsigned short *wh = reinterpret_cast<const unsigned short *>(A.hbw) + (size_t)v * A.B.W;
  const float2 *xb = A.x + A.bn0;
  const int nb1 = A.B.NB - 1;
  float wv[kSlotUnroll];
  int cb[kSlotUnroll];
#pragma unroll
  for (int u = 0; u < kSlotUnroll; ++u) {
    const int sl = m + u * kRowLanes;
    const bool on = sl < A.B.W;
    wv[u] = on ? (WT == 0 ? __ldcs(wf + sl) : __uint_as_float((uint32_t)__ldcs(wh + sl) << 16)) : 0.f;
    cb[u] = on ? min(max(hb + (m ? A.soff[1][u] : A.soff[0][u]), 0), nb1) : -1;
  }
#pragma unroll
  for (int u = 0; u < kSlotUnroll; ++u) {
    if (cb[u] >= 0) {
      const float2 xv = __ldg(xb + cb[u]);
      sx = fmaf(wv[u], xv.x, sx);
      sy = fmaf(wv[u], xv.y, sy);
    }
  }
}

// A short row's st piece [k, e) by the row's pair of lanes in aligned groups
// of 4 entries: lane m takes groups m, m + 2, ... from the group holding k,
// one 16-byte index load and one 8-byte (BF16) or 16-byte (FP32) weight load
// per group, entries outside [k, e) masked.  kGroupUnroll groups' loads are in
// flight before their gathers.
constexpr int kGroupUnroll = 2;
template <int WT>
__device__ __forceinline__ void row_groups(const int32_t *col, const void *w, uint32_t k,
                                           uint32_t e, int m, const float2 *x, float &sx,
                                           float &sy) {
  if (k >= e) return;
  for (uint32_t g = (k & ~3u) + 4u * m; g < e; g += 8u * kGroupUnroll) {
    int4 cc[kGroupUnroll];
    float wv[kGroupUnroll][4];
#pragma unroll
    for (int u = 0; u < kGroupUnroll; ++u) {
      const uint32_t gg = g + 8u * u;
      if (gg < e) {
        cc[u] = __ldcs(reinterpret_cast<const int4 *>(col + gg));
        if (WT == 0) {
          const float4 q = __ldcs(reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(w) + gg));
          wv[u][0] = q.x; wv[u][1] = q.y; wv[u][2] = q.z; wv[u][3] = q.w;
        } else {
          const uint2 q = __ldcs(reinterpret_cast<const uint2 *>(reinterpret_cast<const unsigned short *>(w) + gg));
          wv[u][0] = __uint_as_float(q.x << 16);
          wv[u][1] = __uint_as_float(q.x & 0xffff0000u);
          wv[u][2] = __uint_as_float(q.y << 16);
          wv[u][3] = __uint_as_float(q.y & 0xffff0000u);
        }
      } else {
        cc[u] = make_int4(0, 0, 0, 0);
        wv[u][0] = wv[u][1] = wv[u][2] = wv[u][3] = 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < kGroupUnroll; ++u) {
      const uint32_t gg = g + 8u * u;
      const int ci[4] = {cc[u].x, cc[u].y, cc[u].z, cc[u].w};
      float2 xv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool in = gg + q >= k && gg + q < e;
        xv[q] = in ? __ldg(x + ci[q]) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sx = fmaf(wv[u][q], xv[q].x, sx);
        sy = fmaf(wv[u][q], xv[q].y, sy);
      }
    }
  }
}

// One pass of a warp over 32 / kRowLanes consecutive short rows from `base`.
template <int WT, int MODE>
__device__ __forceinline__ void rows_group(const StepArgs &A, long long base) {
  const int64_t N = A.nrows;
  constexpr int L = kRowLanes;
  const int lane = threadIdx.x & 31, m = lane & (L - 1);
  const bool two = A.hrp != nullptr;
  const long long v = base + lane / L;
  bool live = false;
  uint32_t sa = 0, sb = 0, ha = 0, hb = 0;
  int hbv = -1;
  if (v < N) {
    const uint32_t f0 = A.srp[v], f1 = A.srp[v + 1];
    if (MODE == MODE_HR && two && v < A.C) hbv = A.hbin[v];  // in flight with the row pointers
    sa = f0 & kOffMask;
    sb = f1 & kOffMask;
    if (two) {
      const uint32_t h0 = A.hrp[v];
      ha = h0 & kOffMask;
      hb = A.hrp[v + 1] & kOffMask;
      live = !(h0 & kHubFlag);
    } else {
      live = !(f0 & kHubFlag);
    }
  }
  float sx = 0.f, sy = 0.f;
  if (live) {
    row_groups<WT>(A.scol, A.sw, sa, sb, m, A.x, sx, sy);
    if (two) {
      row_piece<WT, L, kHmUnroll>(A.hcol, A.hw, ha + m, hb, A.x, sx, sy);
      if (MODE == MODE_HR) {
        if (A.sfast) slot_piece_fast<WT>(A, v, hbv, m, sx, sy);
        else slot_piece<WT, L>(A, v, hbv, m, sx, sy);
      }
    }
  }
#pragma unroll
  for (int d = 1; d < L; d <<= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, d);
    sy += __shfl_xor_sync(0xffffffffu, sy, d);
  }
  if (live) {
    // lane m of the pair finishes coordinate m
    const float av = A.a[v];
    const float bv = MODE == MODE_GIFT ? A.b[v] : A.binvf;
    const float xr = reinterpret_cast<const float *>(A.x)[2 * v + m];
    const double acv = A.tap ? reinterpret_cast<const double *>(A.acc)[2 * v + m] : 0.0;
    epilogue_c(A, v, A.nkind[v], m, acv, av * xr + bv * (m ? sy : sx));
  }
}

template <int WT, int MODE>
__global__ void __launch_bounds__(kRowThreads, 6) k_spmm_rows(StepArgs A) {
  constexpr int RPW = 32 / kRowLanes;
  const long long gw = ((long long)blockIdx.x * kRowThreads + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * kRowThreads) >> 5;
  for (long long base = gw * RPW; base < A.nrows; base += nw * RPW) rows_group<WT, MODE>(A, base);
}

// A GiFt chain pair over the short rows of the static matrix: the same
// row-split walk, one gather of (x1, y1, x2, y2) per entry for both chains
// (the indices, weights and gathers of one product serve two).
template <int WT>
__device__ __forceinline__ void row_piece4(const int32_t *col, const void *w, uint32_t k,
                                           uint32_t e, const float4 *x, float4 &s) {
  for (; k < e; k += kRowUnroll * kRowLanes) {
    int c[kRowUnroll];
    float wv[kRowUnroll];
#pragma unroll
    for (int u = 0; u < kRowUnroll; ++u) {
      const uint32_t kk = k + u * kRowLanes;
      c[u] = kk < e ? __ldcs(col + kk) : -1;
      wv[u] = kk < e ? wload<WT>(w, kk) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kRowUnroll; ++u) {
      if (c[u] >= 0) {
        const float4 xv = __ldg(x + c[u]);
        s.x = fmaf(wv[u], xv.x, s.x);
        s.y = fmaf(wv[u], xv.y, s.y);
        s.z = fmaf(wv[u], xv.z, s.z);
        s.w = fmaf(wv[u], xv.w, s.w);
      }
    }
  }
}

template <int WT>
__global__ void __launch_bounds__(kRowThreads) k_spmm_rows4(StepArgs A) {
  const int64_t N = A.nrows;
  constexpr int L = kRowLanes, RPW = 32 / L;
  const int lane = threadIdx.x & 31, m = lane & (L - 1);
  const long long gw = ((long long)blockIdx.x * kRowThreads + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * kRowThreads) >> 5;
  for (long long base = gw * RPW; base < N; base += nw * RPW) {
    const long long v = base + lane / L;
    bool live = false;
    uint32_t sa = 0, sb = 0;
    if (v < N) {
      const uint32_t f0 = A.srp[v];
      sa = f0 & kOffMask;
      sb = A.srp[v + 1] & kOffMask;
      live = !(f0 & kHubFlag);
    }
    float4 sm = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) row_piece4<WT>(A.scol, A.sw, sa + m, sb, A.x4, sm);
    sm.x += __shfl_xor_sync(0xffffffffu, sm.x, 1);
    sm.y += __shfl_xor_sync(0xffffffffu, sm.y, 1);
    sm.z += __shfl_xor_sync(0xffffffffu, sm.z, 1);
    sm.w += __shfl_xor_sync(0xffffffffu, sm.w, 1);
    if (live) {
      // lane m of the pair finishes coordinate m of both chains
      const float *xr = reinterpret_cast<const float *>(A.x4) + 4 * v + m;
      const float y1 = A.a[v] * xr[0] + A.b[v] * (m ? sm.y : sm.x);
      const float y2 = A.a2[v] * xr[2] + A.b2[v] * (m ? sm.w : sm.z);
      const double acv = (A.tap || A.tap2 || A.fin)
                             ? reinterpret_cast<const double *>(A.acc)[2 * v + m]
                             : 0.0;
      epilogue_c2(A, v, A.nkind[v], m, acv, y1, y2);
    }
  }
}

// Hub rows, after the chunk launch: a block takes kHubRows rows, a warp per
// row adding the row's partials in a fixed order (lane-strided over the
// chunks, then a fixed tree); one warp then does the combines in FP64, a lane
// per row, so the FP64 work of kHubRows rows shares its instructions.
constexpr int kHubRows = 8;
// Row block `blk` (kHubRows rows) by a block of kHubRows warps; sums: the
// block's shared scratch of kHubRows float4.
template <int WT, int MODE>
__device__ __forceinline__ void hub_rows_block(const StepArgs &A, long long blk, float4 *sums) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long l = blk * kHubRows + w;
  if (l < A.nlong) {
    const int c0 = A.lchunk[l], nch = A.lchunk[l + 1] - c0;
    dfl px{0.f, 0.f}, py{0.f, 0.f};
    for (int k = lane; k < nch; k += 32) {
      const float4 q = __ldcg(&A.part[c0 + k]);
      df_add_df(px, dfl{q.x, q.y});
      df_add_df(py, dfl{q.z, q.w});
    }
    px = warp_sum_df(px);
    py = warp_sum_df(py);
    if (MODE == MODE_HR) {
      const int64_t v = A.lrow[l];
      if (v >= A.bn0) {
        // a bin row: its window-slot partials over the source buckets
        dfl bx, by;
        bin_row_chunks(A.B, (int)(v - A.bn0), A.bchunk, A.bpart, &bx, &by);
        df_add_df(px, bx);
        df_add_df(py, by);
      } else if (v < A.C && A.hbin[v] >= 0) {
        // a hint cell with a hub row: its window slots, exact products
        const int hb = A.hbin[v], bxc = hb % A.B.nbx, byc = hb / A.B.nbx;
        dfl qx{0.f, 0.f}, qy{0.f, 0.f};
        for (int sl = lane; sl < A.B.W; sl += 32) {
          int dx, dy;
          slot_off(A.B, sl, &dx, &dy);
          const int xx = bxc + dx, yy = byc + dy;
          if (xx < 0 || yy < 0 || xx >= A.B.nbx || yy >= A.B.nby) continue;
          const float wv = bw_load<WT>(A.hbw, (size_t)v * A.B.W + sl);
          const float2 xv = A.x[A.bn0 + yy * A.B.nbx + xx];
          df_add_prod(qx, wv, xv.x);
          df_add_prod(qy, wv, xv.y);
        }
        df_add_df(px, warp_sum_df(qx));
        df_add_df(py, warp_sum_df(qy));
      }
    }
    if (lane == 0) sums[w] = make_float4(px.hi, px.lo, py.hi, py.lo);
  }
  __syncthreads();
  const long long lr = blk * kHubRows + lane;
  if (w != 0 || lane >= kHubRows || lr >= A.nlong) return;
  const float4 q = sums[lane];
  const int64_t v = A.lrow[lr];
  const double tx = df_to_d(dfl{q.x, q.y}), ty = df_to_d(dfl{q.z, q.w});
  double av, bv;
  if (MODE == MODE_HR) {
    av = A.c64l[lr];
    bv = A.binv;
  } else {
    av = (double)A.a[v];
    bv = (double)A.b[v];
  }
  const int64_t xi = MODE == MODE_GIFT ? v * A.xs : v;
  const float2 xv = A.x[xi];
  epilogue<double>(A, v, av * (double)xv.x + bv * tx, av * (double)xv.y + bv * ty, xi);
}

template <int WT, int MODE>
__global__ void __launch_bounds__(kHubRows * 32) k_hub_rows(StepArgs A) {
  __shared__ float4 sums[kHubRows];
  hub_rows_block<WT, MODE>(A, blockIdx.x, sums);
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

// Star node = mean of its net's distinct nodes (warp per star): double-float
// sums (about 48 bits) over the lanes and a fixed butterfly, then the
// quotient by p as a double-float in FP32 operations (the remainder of the
// leading quotient is exact), rounded once to FP32.
__device__ __forceinline__ float df_div_int(dfl s, int p) {
  const float fp = (float)p;
  const float q = __fdiv_rn(s.hi, fp);
  const float r = __fmaf_rn(-q, fp, s.hi);
  return __fadd_rn(q, __fdiv_rn(__fadd_rn(r, s.lo), fp));
}
__global__ void k_star_init(int32_t S, int64_t star0, const int32_t *star_net,
                            const int64_t *net_ptr, const uint32_t *nd, const int32_t *net_p,
                            float2 *g) {
  const int lane = threadIdx.x & 31;
  for (long long s = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; s < S;
       s += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int e = star_net[s];
    const long long b = net_ptr[e];
    const int p = net_p[e];
    dfl sx{0.f, 0.f}, sy{0.f, 0.f};
    for (int k = lane; k < p; k += 32) {
      const float2 q = g[nd[b + k]];
      df_add(sx, q.x);
      df_add(sy, q.y);
    }
    sx = warp_sum_df(sx);
    sy = warp_sum_df(sy);
    if (lane == 0) g[star0 + s] = make_float2(df_div_int(sx, p), df_div_int(sy, p));
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
// sqrt(d), and u0 = (g - centre)/sqrt(d), d = D_vv + sigma.  d is the static
// degree (double-float) plus sigma, rounded once to FP32; the rest is FP32,
// the precision the sparse products run in (a centre is subtracted in FP64).
__global__ void k_gift_prep(int64_t N, const dfl *deg, double sigma, const float2 *g,
                            int center, double cx, double cy, float *a, float *b, float *sq,
                            float2 *u0) {
  const float sh = (float)sigma, sl = (float)(sigma - (double)sh);  // sigma as a double-float
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    dfl t = deg[v];
    df_add(t, sh);
    df_add(t, sl);
    const float d = df_norm(t).hi;
    const float r = sqrtf(d);
    a[v] = sh / d;
    b[v] = 1.0f / d;
    sq[v] = r;
    const float2 q = g[v];
    if (center)
      u0[v] = make_float2((float)((double)q.x - cx) / r, (float)((double)q.y - cy) / r);
    else
      u0[v] = make_float2(q.x / r, q.y / r);
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
// st gives every row's static part; units and hub rows come from the applied
// matrix (hm with hint parts for the refinement filter, st for GiFt).
static void fill_matrix(StepArgs &A, const SpMat &st, const SpMat *hm) {
  const SpMat &m = hm ? *hm : st;
  A.srp = P<uint32_t>(st.rp_s);
  A.scol = P<int32_t>(st.col);
  A.sw = st.w.p;
  A.hrp = hm ? P<uint32_t>(hm->rp_s) : nullptr;
  A.hcol = hm ? P<int32_t>(hm->col) : nullptr;
  A.hw = hm ? hm->w.p : nullptr;
  A.nrows = m.N;
  A.lrow = P<int32_t>(m.lrow);
  A.lsb = P<uint64_t>(m.lsb);
  A.lhb = P<uint64_t>(m.lhb);
  A.lsl = P<uint32_t>(m.lsl);
  A.lhl = P<uint32_t>(m.lhl);
  A.lchunk = P<int32_t>(m.lchunk);
  A.chunk_lr = P<int32_t>(m.chunk_lr);
  A.nchunks = m.nchunks;
  A.nlong = m.nlong;
  A.part = const_cast<float4 *>(P<float4>(m.part));
}

// Algorithmic bytes of one sparse product over (x, y) pairs: indices and
// weights once, row pointers, x read, y written, one coefficient per row.
static double spmm_bytes(double nnz, double N, int wdtype) {
  return nnz * (4.0 + (wdtype == PL_W_BF16 ? 2.0 : 4.0)) + (N + 1.0) * 4.0 + N * (8.0 + 8.0 + 4.0);
}

// Algorithmic bytes of one refinement product with column-free bin hints:
// the stored entries (static, macro) once, each hint cell's window block
// twice (its own row, and the bin rows' pass over the buckets) with the
// bucket list once, row pointers, x read, y written, one coefficient per row.
static double spmm_bytes_hint(const pl_graph *g) {
  const double sw = g->wdtype == PL_W_BF16 ? 2.0 : 4.0;
  const double stored = (double)(g->st.nnz_s + g->st.nnz_l + g->hm.nnz_s + g->hm.nnz_l);
  const double nh = (double)g->nhint;
  return stored * (4.0 + sw) + nh * (2.0 * g->W * sw + 4.0) + ((double)g->N + 1.0) * 4.0 +
         (double)g->N * (8.0 + 8.0 + 4.0);
}

// One sparse product: the hub chunks and then the hub rows on the graph's
// side stream, the short rows on the caller's stream at the same time (they
// write disjoint rows of y); the caller's stream waits for both.
// SM count of the graph's device, looked up once per graph (a graph is used
// from one host thread at a time and stays on the device it was built on).
static int graph_nsm(pl_graph *g) {
  if (!g->nsm) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 152;
    g->nsm = n;
  }
  return g->nsm;
}

template <int MODE>
static cudaError_t launch_step(const StepArgs &A, double bytes, int wdtype, cudaStream_t s,
                               pl_graph *g) {
  const int nsm = graph_nsm(g);
  // short rows: one wave of resident blocks, row groups dealt round robin
  int *occ = g->occ_rows[MODE];
  const int wi = wdtype == PL_W_BF16 ? 1 : 0;
  if (!occ[wi]) {
    int b = 0;
    cudaError_t e = wi ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_spmm_rows<1, MODE>, kRowThreads, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_spmm_rows<0, MODE>, kRowThreads, 0);
    occ[wi] = (e == cudaSuccess && b > 0) ? b : 1;
  }
  const bool prof = prof_on();
  if (prof) prof_begin(s, MODE == MODE_HR ? PROF_HR : PROF_GIFT, bytes);
  const bool fork = A.nchunks > 0;
  if (fork) {
    cudaError_t e = ensure_side(g);
    if (e == cudaSuccess) e = cudaEventRecord(g->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->side, g->ev_fork, 0);
    if (e != cudaSuccess) return e;
    cudaStream_t sh = g->side;
    const long long want = ((long long)A.nchunks + 7) / 8;
    const int hgrid = (int)(want < 8LL * nsm ? want : 8LL * nsm);
    if (wi) k_spmm_hub<1, MODE><<<hgrid, 256, 0, sh>>>(A);
    else k_spmm_hub<0, MODE><<<hgrid, 256, 0, sh>>>(A);
    note_launch();
    if (MODE == MODE_HR && A.bpart) {
      // bin rows: chunk partials of the window blocks times the cells' x
      const long long bwant = (g->nbc_max + kBinThreads / 32 - 1) / (kBinThreads / 32);
      const int bgrid = (int)(bwant < 152LL * 16 ? bwant : 152LL * 16);
      e = launch_bin_partials<false>(wi ? PL_W_BF16 : PL_W_FP32, bgrid, sh, A.B, A.bchunk, A.cown,
                                     A.boff, A.blist, A.hbwq, A.x, A.bpart);
      if (e != cudaSuccess) return e;
      note_launch();
    }
    const int rgrid = (int)(((long long)A.nlong + kHubRows - 1) / kHubRows);
    if (wi) k_hub_rows<1, MODE><<<rgrid, kHubRows * 32, 0, sh>>>(A);
    else k_hub_rows<0, MODE><<<rgrid, kHubRows * 32, 0, sh>>>(A);
    note_launch();
    e = cudaEventRecord(g->ev_join, sh);
    if (e != cudaSuccess) return e;
  }
  const long long rows_per_block = (long long)(kRowThreads / 32) * (32 / kRowLanes);
  const long long want = (A.nrows + rows_per_block - 1) / rows_per_block;
  // refinement products with a second stream: at most kRowCtasSide CTAs per
  // SM, so the registers they leave free hold the second stream's CTAs, which
  // then run beside the short rows rather than after them
  const int per_sm = MODE == MODE_HR && fork && occ[wi] > kRowCtasSide ? kRowCtasSide : occ[wi];
  const long long cap = (long long)per_sm * nsm;
  const int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
  if (wi) k_spmm_rows<1, MODE><<<grid, kRowThreads, 0, s>>>(A);
  else k_spmm_rows<0, MODE><<<grid, kRowThreads, 0, s>>>(A);
  note_launch();
  if (fork) {
    const cudaError_t e = cudaStreamWaitEvent(s, g->ev_join, 0);
    if (e != cudaSuccess) return e;
  }
  if (prof) prof_end(s);
  return cudaGetLastError();
}

// Algorithmic bytes of one product of a GiFt chain pair: indices and weights
// once, row pointers, the four signals read and written, two coefficients.
static double spmm_bytes_pair(double nnz, double N, int wdtype) {
  return nnz * (4.0 + (wdtype == PL_W_BF16 ? 2.0 : 4.0)) + (N + 1.0) * 4.0 +
         N * (16.0 + 16.0 + 8.0);
}

// One product of a GiFt chain pair: the hub rows of each chain in turn (its
// half of the interleaved signals, stride 2) on the side stream, the short
// rows of both chains in one launch on the caller's stream.
static cudaError_t launch_pair(const StepArgs &A, double bytes, int wdtype, cudaStream_t s,
                               pl_graph *g) {
  const int nsm = graph_nsm(g);
  int *occ = g->occ_rows4;
  const int wi = wdtype == PL_W_BF16 ? 1 : 0;
  if (!occ[wi]) {
    int b = 0;
    cudaError_t e = wi ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_spmm_rows4<1>, kRowThreads, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_spmm_rows4<0>, kRowThreads, 0);
    occ[wi] = (e == cudaSuccess && b > 0) ? b : 1;
  }
  const bool prof = prof_on();
  if (prof) prof_begin(s, PROF_GIFT, bytes);
  const bool fork = A.nchunks > 0;
  if (fork) {
    cudaError_t e = ensure_side(g);
    if (e == cudaSuccess) e = cudaEventRecord(g->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->side, g->ev_fork, 0);
    if (e != cudaSuccess) return e;
    cudaStream_t sh = g->side;
    const long long want = ((long long)A.nchunks + 7) / 8;
    const int hgrid = (int)(want < 8LL * nsm ? want : 8LL * nsm);
    const int rgrid = (int)(((long long)A.nlong + kHubRows - 1) / kHubRows);
    for (int h = 0; h < 2; ++h) {
      StepArgs H = A;
      H.x = reinterpret_cast<const float2 *>(A.x4) + h;
      H.y = reinterpret_cast<float2 *>(A.y4) + h;
      H.xs = 2;
      if (h == 0) {  // the first chain never finishes: its tap goes to the sum
        H.fin = 0;
        H.cx = H.cy = 0.0;
        H.addc = 0;
      } else {
        H.a = A.a2;
        H.b = A.b2;
        H.tscale = A.tscale2;
        H.tap = A.tap2;
        H.alpha = A.alpha2;
        if (H.fin && !H.tap) {  // the final value reads the sum
          H.tap = 1;
          H.alpha = 0.0;
        }
      }
      if (wi) k_spmm_hub<1, MODE_GIFT><<<hgrid, 256, 0, sh>>>(H);
      else k_spmm_hub<0, MODE_GIFT><<<hgrid, 256, 0, sh>>>(H);
      if (wi) k_hub_rows<1, MODE_GIFT><<<rgrid, kHubRows * 32, 0, sh>>>(H);
      else k_hub_rows<0, MODE_GIFT><<<rgrid, kHubRows * 32, 0, sh>>>(H);
      note_launch();
      note_launch();
    }
    e = cudaEventRecord(g->ev_join, sh);
    if (e != cudaSuccess) return e;
  }
  const long long rows_per_block = (long long)(kRowThreads / 32) * (32 / kRowLanes);
  const long long want = (A.nrows + rows_per_block - 1) / rows_per_block;
  const long long cap = (long long)occ[wi] * nsm;
  const int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
  if (wi) k_spmm_rows4<1><<<grid, kRowThreads, 0, s>>>(A);
  else k_spmm_rows4<0><<<grid, kRowThreads, 0, s>>>(A);
  note_launch();
  if (fork) {
    const cudaError_t e = cudaStreamWaitEvent(s, g->ev_join, 0);
    if (e != cudaSuccess) return e;
  }
  if (prof) prof_end(s);
  return cudaGetLastError();
}

// The pair's interleaved start: (x1, y1) of the first chain, (x2, y2) of the
// second.
__global__ void k_pack_pair(int64_t N, const float2 *a, const float2 *b, float4 *q) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    const float2 u = a[v], w = b[v];
    q[v] = make_float4(u.x, u.y, w.x, w.y);
  }
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
  TRY(ensure(g->gsc, (size_t)N * 24 + 64));
  TRY(ensure(g->ua, (size_t)N * 8 + 64));
  TRY(ensure(g->ub, (size_t)N * 8 + 64));
  TRY(ensure(g->xa, (size_t)N * 8 + 64));
  float *ga = P<float>(g->gsc), *gb = ga + N, *gq = gb + N;
  float *ga2 = gq + N, *gb2 = ga2 + N, *gq2 = gb2 + N;
  StepArgs A{};
  fill_matrix(A, g->st, nullptr);
  const double bytes = spmm_bytes((double)(g->st.nnz_s + g->st.nnz_l), (double)N, g->wdtype);
  fill_nodes(A, g);
  A.acc = P<double2>(g->acc);
  A.relax = 0;
  A.clamp = p->clamp;
  A.gnext = gout;
  A.single = 0;
  A.pin = 0;
  A.xs = 1;
  // tap of chain q at step t: the summed alpha of its bands with k = t
  auto tap_of = [&](int q, int t, double *alpha) {
    *alpha = 0.0;
    int tap = 0;
    for (int bnd = 0; bnd < 3; ++bnd)
      if (chain_of[bnd] == q && p->gift_k[bnd] == t) {
        tap = 1;
        *alpha += p->gift_alpha[bnd];
      }
    return tap;
  };
  // per-node coefficients of chain q, its start u0, and its bands with k = 0
  // (they contribute alpha * (g - centre))
  auto prep = [&](int q, float *a, float *b, float *sq, float2 *u0) -> cudaError_t {
    k_gift_prep<<<grid_for(N, 256), 256, 0, s>>>(N, P<dfl>(g->st.dsum), sig[q], gin,
                                                 p->gift_center ? 1 : 0, cx, cy, a, b, sq, u0);
    note_launch();
    for (int bnd = 0; bnd < 3; ++bnd) {
      if (chain_of[bnd] != q || p->gift_k[bnd] != 0) continue;
      k_acc_add<<<grid_for(N, 256), 256, 0, s>>>(N, u0, sq, p->gift_alpha[bnd],
                                                 P<double2>(g->acc));
      note_launch();
    }
    return cudaGetLastError();
  };
  auto set_final = [&](bool fin) {
    A.fin = fin ? 1 : 0;
    A.cx = fin ? cx : 0.0;
    A.cy = fin ? cy : 0.0;
    A.addc = (A.cx != 0.0 || A.cy != 0.0) ? 1 : 0;
  };
  // Chains without steps first (their bands only add to the sum that the
  // final step reads), then the chains with steps: all but the last two
  // alone, the last two as a pair.  The longer chain of the pair runs alone
  // until the two have equal steps left, then both advance in one product
  // per step (interleaved signals); the pair's last step is the final one.
  int qs[3], ns = 0;
  for (int q = 0; q < nch; ++q)
    if (kmax[q] == 0) TRY(prep(q, ga, gb, gq, P<float2>(g->ua)));
  for (int q = 0; q < nch; ++q)
    if (kmax[q] > 0) qs[ns++] = q;
  const bool pair = ns >= 2;
  const int nsolo = pair ? ns - 2 : ns;
  // one chain alone from x for steps t0 + 1 .. t1 (ping-pong x, y)
  auto run_chain = [&](int q, float2 *&x, float2 *&y, int t0, int t1, bool last) -> cudaError_t {
    A.a = ga;
    A.b = gb;
    A.tscale = gq;
    for (int t = t0 + 1; t <= t1; ++t) {
      A.x = x;
      A.y = y;
      A.tap = tap_of(q, t, &A.alpha);
      set_final(last && t == t1);
      const cudaError_t e = launch_step<MODE_GIFT>(A, bytes, g->wdtype, s, g);
      if (e != cudaSuccess) return e;
      float2 *tt = x;
      x = y;
      y = tt;
    }
    return cudaSuccess;
  };
  for (int i = 0; i < nsolo; ++i) {
    const int q = qs[i];
    TRY(prep(q, ga, gb, gq, P<float2>(g->ua)));
    float2 *x = P<float2>(g->ua), *y = P<float2>(g->ub);
    TRY(run_chain(q, x, y, 0, kmax[q], i == ns - 1));
  }
  if (pair) {
    const int q1 = qs[ns - 2], q2 = qs[ns - 1];
    const int qL = kmax[q1] >= kmax[q2] ? q1 : q2, qS = qL == q1 ? q2 : q1;
    const int d = kmax[qL] - kmax[qS];
    TRY(prep(qL, ga, gb, gq, P<float2>(g->ua)));
    TRY(prep(qS, ga2, gb2, gq2, P<float2>(g->xa)));
    float2 *x = P<float2>(g->ua), *y = P<float2>(g->ub);
    TRY(run_chain(qL, x, y, 0, d, false));
    TRY(ensure(g->q4a, (size_t)N * 16 + 64));
    TRY(ensure(g->q4b, (size_t)N * 16 + 64));
    float4 *x4 = P<float4>(g->q4a), *y4 = P<float4>(g->q4b);
    k_pack_pair<<<grid_for(N, 256), 256, 0, s>>>(N, x, P<float2>(g->xa), x4);
    note_launch();
    const double bytes4 = spmm_bytes_pair((double)(g->st.nnz_s + g->st.nnz_l), (double)N,
                                          g->wdtype);
    A.a = ga;
    A.b = gb;
    A.tscale = gq;
    A.a2 = ga2;
    A.b2 = gb2;
    A.tscale2 = gq2;
    for (int t = 1; t <= kmax[qS]; ++t) {
      A.tap = tap_of(qL, d + t, &A.alpha);
      A.tap2 = tap_of(qS, t, &A.alpha2);
      A.x4 = x4;
      A.y4 = y4;
      set_final(t == kmax[qS]);
      TRY(launch_pair(A, bytes4, g->wdtype, s, g));
      float4 *tt = x4;
      x4 = y4;
      y4 = tt;
    }
  }
  const bool any = ns > 0;
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

// The refinement product's arguments on the current augmented graph (A4):
// matrix, column-free bin hints, coefficients and node tables.
static void hr_args(pl_graph *g, StepArgs &A) {
  const SpMat &m = g->hm;
  fill_matrix(A, g->st, &m);
  A.hbw = g->hbw.p;
  A.hbwq = g->hbwq.p;
  A.hbin = P<int32_t>(g->hbin);
  A.C = g->C;
  A.bn0 = g->Nst + g->Mm;
  A.B.nbx = g->nbx;
  A.B.nby = g->nby;
  A.B.hx = g->hx;
  A.B.hy = g->hy;
  A.B.W = g->W;
  A.B.NB = g->NB;
  A.sfast = g->W <= kSlotUnroll * kRowLanes ? 1 : 0;
  for (int mm = 0; mm < kRowLanes; ++mm)
    for (int u = 0; u < kSlotUnroll; ++u) {
      const int sl = mm + u * kRowLanes, wx = 2 * g->hx + 1;
      A.soff[mm][u] = (sl / wx - g->hy) * g->nbx + (sl % wx - g->hx);
    }
  A.bchunk = P<int32_t>(g->bchunk);
  A.cown = P<int32_t>(g->cown);
  A.boff = P<int64_t>(g->boff);
  A.blist = P<uint32_t>(g->blist);
  A.bpart = P<float4>(g->bpart);
  fill_nodes(A, g);
  A.a = P<float>(m.c32);
  A.b = nullptr;
  A.c64l = P<double>(m.c64l);
  A.binv = g->lam_h[1];
  A.binvf = (float)g->lam_h[1];
  A.tscale = nullptr;
  A.acc = P<double2>(g->acc);
  A.cx = A.cy = 0.0;
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
  StepArgs A{};
  hr_args(g, A);
  const double bytes = spmm_bytes_hint(g);
  A.g0 = gin;
  A.gnext = gout;
  A.gamma = p->gamma;
  A.omg = 1.0 - p->gamma;
  A.relax = 1;
  A.clamp = p->clamp;
  A.single = single ? 1 : 0;
  A.pin = p->pin_every_step;
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
    TRY(launch_step<MODE_HR>(A, bytes, g->wdtype, s, g));
    x = bufs[t & 1];
  }
  return PL_OK;
}

// Powers H_r^k g for the learned filter's taps k[0] < k[1] < k[2]: one
// refinement product per power up to k[2], each stored in FP32 and re-pinned
// when p asks for it (as the plain filter's powers).  out[i] points at
// H_r^{k[i]} g: the input itself for k = 0, else ua (k[0]), ub (k[1]) or one
// of xa / xb (k[2]).
pl_status run_powers(pl_graph *g, const pl_params *p, const float *in, const int32_t k[3],
                     const float2 *out[3], cudaStream_t s) {
  const float2 *gin = reinterpret_cast<const float2 *>(in);
  StepArgs A{};
  hr_args(g, A);
  const double bytes = spmm_bytes_hint(g);
  A.pin = p->pin_every_step;
  A.fin = 0;
  A.tap = 0;
  const float2 *x = gin;
  float2 *bufs[2] = {P<float2>(g->xa), P<float2>(g->xb)};
  for (int i = 0; i < 3; ++i)
    if (k[i] == 0) out[i] = gin;
  for (int t = 1; t <= k[2]; ++t) {
    float2 *y = t == k[0] ? P<float2>(g->ua) : t == k[1] ? P<float2>(g->ub) : bufs[t & 1];
    A.x = x;
    A.y = y;
    TRY(launch_step<MODE_HR>(A, bytes, g->wdtype, s, g));
    for (int i = 0; i < 3; ++i)
      if (k[i] == t) out[i] = y;
    x = y;
  }
  return PL_OK;
}

}  // namespace pl

// ------------------------------------------------ the batched product (NEXT-1)
// One launch per kernel of a refinement product covers every design of a
// batch: the designs' work units (short-row groups, hub chunks, bin chunks,
// hub-row blocks) are concatenated, a block-diagonal
// union of the designs' matrices with each design's own lambda_up and
// per-node coefficients.  Unit u belongs to the design d with
// pre[d] <= u < pre[d + 1]; a warp takes a run of consecutive units and
// keeps its design's arguments in shared memory.  A design's units compute
// exactly what its own launch computes, so every result keeps its bits.
namespace pl {

enum { BK_ROWS = 0, BK_HUB = 1, BK_BINC = 2, BK_HROW = 3, BK_KINDS = 4 };

__device__ __forceinline__ int unit_design(const long long *pre, int nd, long long u) {
  int lo = 0, hi = nd - 1;  // the largest d with pre[d] <= u
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void warp_copy_args(StepArgs *dst, const StepArgs *src) {
  const int lane = threadIdx.x & 31;
  const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
  uint32_t *d = reinterpret_cast<uint32_t *>(dst);
  for (int i = lane; i < (int)(sizeof(StepArgs) / 4); i += 32) d[i] = s[i];
  __syncwarp();
}

// Warp-level units of kind K: the warp's run [u, u1) of pre's units.
template <int K, int WT, int MODE>
__device__ __forceinline__ void batch_units(const StepArgs *As, const long long *pre, int nd,
                                            long long per, StepArgs *sa) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long total = pre[nd];
  long long u = gw * per;
  const long long u1 = u + per < total ? u + per : total;
  if (u >= u1) return;
  int d = unit_design(pre, nd, u);
  warp_copy_args(sa, &As[d]);
  for (; u < u1; ++u) {
    if (u >= pre[d + 1]) {
      __syncwarp();
      d = unit_design(pre, nd, u);
      warp_copy_args(sa, &As[d]);
    }
    const StepArgs &A = *sa;
    const long long k = u - pre[d];
    if (K == BK_ROWS) {
      rows_group<WT, MODE>(A, k * (32 / kRowLanes));
    } else if (K == BK_HUB) {
      warp_chunk<WT, MODE>(A, (int)k);
    } else {
      if (k < A.bchunk[A.B.NB])
        bin_chunk<WT, false>(A.B, A.bchunk, A.cown, A.boff, A.blist, A.hbwq, A.x, A.bpart, k);
    }
  }
}

template <int WT>
__global__ void __launch_bounds__(kRowThreads, 5) k_rows_batch(const StepArgs *As,
                                                              const long long *pre, int nd,
                                                              long long per) {
  __shared__ StepArgs sa[kRowThreads / 32];
  batch_units<BK_ROWS, WT, MODE_HR>(As, pre, nd, per, &sa[threadIdx.x >> 5]);
}

template <int K, int WT>
__global__ void __launch_bounds__(256) k_side_batch(const StepArgs *As, const long long *pre,
                                                     int nd, long long per) {
  __shared__ StepArgs sa[8];
  batch_units<K, WT, MODE_HR>(As, pre, nd, per, &sa[threadIdx.x >> 5]);
}

template <int WT>
__global__ void __launch_bounds__(kHubRows * 32) k_hub_rows_batch(const StepArgs *As,
                                                                  const long long *pre, int nd) {
  __shared__ StepArgs sa;
  __shared__ float4 sums[kHubRows];
  const int d = unit_design(pre, nd, blockIdx.x);
  {
    const uint32_t *s = reinterpret_cast<const uint32_t *>(&As[d]);
    uint32_t *t = reinterpret_cast<uint32_t *>(&sa);
    for (int i = threadIdx.x; i < (int)(sizeof(StepArgs) / 4); i += blockDim.x) t[i] = s[i];
  }
  __syncthreads();
  hub_rows_block<WT, MODE_HR>(sa, blockIdx.x - pre[d], sums);
}

size_t batch_ws_bytes(int nd, const pl_params *p) {
  const int kmax = p->ntaps >= 1 ? p->tap_k[p->ntaps - 1] : 1;
  return ((size_t)kmax * nd * sizeof(StepArgs) + 255) / 256 * 256 +
         ((size_t)BK_KINDS * (nd + 1) * sizeof(long long) + 255) / 256 * 256 + 256;
}

// One round's filter (A4) for every design of a batch, each from in[d] into
// out[d]: the plain filter's products and epilogues, one launch per kernel
// and power over all designs (short rows on s, the hub and bin-row kernels on
// sh, forked and joined with the first graph's events).  rows_ctas: CTAs per
// SM of the short-row kernel.  ws: batch_ws_bytes(nd, p) device bytes, not in
// use by another launch.  Does not synchronize.
pl_status run_filter_batch(pl_graph *const *gs, int nd, const pl_params *p, const float *const *in,
                           float *const *out, void *ws, size_t ws_bytes, int rows_ctas,
                           cudaStream_t s, cudaStream_t sh) {
  if (nd < 1) return PL_OK;
  if (ws_bytes < batch_ws_bytes(nd, p)) {
    set_error("batch workspace too small: need %zu bytes", batch_ws_bytes(nd, p));
    return PL_ERR_WORKSPACE;
  }
  if (p->gamma == 0.0) {
    for (int d = 0; d < nd; ++d) {
      pl_graph *g = gs[d];
      k_clamp<<<grid_for(g->N, 256), 256, 0, s>>>(g->N, P<uint8_t>(g->nkind), P<float2>(g->fixedp),
                                                   P<float4>(g->bounds),
                                                   reinterpret_cast<const float2 *>(in[d]),
                                                   reinterpret_cast<float2 *>(out[d]), p->clamp);
      note_launch();
    }
    TRY(cudaGetLastError());
    return PL_OK;
  }
  const int kmax = p->tap_k[p->ntaps - 1];
  const bool single = p->ntaps == 1 && p->tap_alpha[0] == 1.0;
  const int wd = gs[0]->wdtype;
  std::vector<StepArgs> hA((size_t)kmax * nd);
  std::vector<long long> pre((size_t)BK_KINDS * (nd + 1), 0);
  for (int d = 0; d < nd; ++d) {
    pl_graph *g = gs[d];
    if (g->wdtype != wd) {
      set_error("designs of a batch need one weight type");
      return PL_ERR_INVALID_ARG;
    }
    if (!single) TRY(cudaMemsetAsync(g->acc.p, 0, (size_t)g->N * 16, s));
    StepArgs A{};
    hr_args(g, A);
    A.g0 = reinterpret_cast<const float2 *>(in[d]);
    A.gnext = reinterpret_cast<float2 *>(out[d]);
    A.gamma = p->gamma;
    A.omg = 1.0 - p->gamma;
    A.relax = 1;
    A.clamp = p->clamp;
    A.single = single ? 1 : 0;
    A.pin = p->pin_every_step;
    float2 *bufs[2] = {P<float2>(g->xa), P<float2>(g->xb)};
    for (int t = 1; t <= kmax; ++t) {
      StepArgs &B = hA[(size_t)(t - 1) * nd + d];
      B = A;
      B.x = t == 1 ? reinterpret_cast<const float2 *>(in[d]) : bufs[(t - 1) & 1];
      B.y = bufs[t & 1];
      B.tap = 0;
      B.alpha = 0.0;
      if (!single)
        for (int j = 0; j < p->ntaps; ++j)
          if (p->tap_k[j] == t) {
            B.tap = 1;
            B.alpha = p->tap_alpha[j];
          }
      B.fin = t == kmax;
    }
    const long long units[BK_KINDS] = {
        (g->N + 32 / kRowLanes - 1) / (32 / kRowLanes), (long long)A.nchunks,
        A.bpart ? (long long)g->nbc_max : 0LL, ((long long)A.nlong + kHubRows - 1) / kHubRows};
    for (int k = 0; k < BK_KINDS; ++k) pre[(size_t)k * (nd + 1) + d + 1] = units[k];
  }
  for (int k = 0; k < BK_KINDS; ++k)
    for (int d = 0; d < nd; ++d) pre[(size_t)k * (nd + 1) + d + 1] += pre[(size_t)k * (nd + 1) + d];
  StepArgs *dA = static_cast<StepArgs *>(ws);
  long long *dpre = reinterpret_cast<long long *>(
      static_cast<char *>(ws) + ((size_t)kmax * nd * sizeof(StepArgs) + 255) / 256 * 256);
  TRY(cudaMemcpyAsync(dA, hA.data(), hA.size() * sizeof(StepArgs), cudaMemcpyHostToDevice, s));
  TRY(cudaMemcpyAsync(dpre, pre.data(), pre.size() * sizeof(long long), cudaMemcpyHostToDevice, s));
  pl_graph *g0 = gs[0];
  TRY(ensure_side(g0));  // its fork and join events
  const int nsm = graph_nsm(g0);
  auto total = [&](int k) { return pre[(size_t)k * (nd + 1) + nd]; };
  auto per_for = [&](long long U, long long warps) {
    return std::max(1LL, (U + warps - 1) / warps);
  };
  const int rc = std::min(std::max(rows_ctas, 1), 5);
  const long long rows_per = per_for(total(BK_ROWS), (long long)rc * nsm * (kRowThreads / 32));
  const int rows_grid = (int)std::max(1LL, (total(BK_ROWS) + rows_per * (kRowThreads / 32) - 1) /
                                                 (rows_per * (kRowThreads / 32)));
  long long side_per[BK_KINDS] = {0, 0, 0, 0};
  int side_grid[BK_KINDS] = {0, 0, 0, 0};
  for (int k = BK_HUB; k <= BK_BINC; ++k) {
    const long long U = total(k);
    if (!U) continue;
    side_per[k] = per_for(U, 8LL * nsm * 8);
    side_grid[k] = (int)((U + side_per[k] * 8 - 1) / (side_per[k] * 8));
  }
  const int hrow_grid = (int)total(BK_HROW);
  for (int t = 1; t <= kmax; ++t) {
    const StepArgs *dAt = dA + (size_t)(t - 1) * nd;
    TRY(cudaEventRecord(g0->ev_fork, s));
    TRY(cudaStreamWaitEvent(sh, g0->ev_fork, 0));
    if (side_grid[BK_HUB]) {
      if (wd == PL_W_BF16) k_side_batch<BK_HUB, 1><<<side_grid[BK_HUB], 256, 0, sh>>>(dAt, dpre + 1 * (nd + 1), nd, side_per[BK_HUB]);
      else k_side_batch<BK_HUB, 0><<<side_grid[BK_HUB], 256, 0, sh>>>(dAt, dpre + 1 * (nd + 1), nd, side_per[BK_HUB]);
      note_launch();
    }
    if (side_grid[BK_BINC]) {
      if (wd == PL_W_BF16) k_side_batch<BK_BINC, 1><<<side_grid[BK_BINC], 256, 0, sh>>>(dAt, dpre + 2 * (nd + 1), nd, side_per[BK_BINC]);
      else k_side_batch<BK_BINC, 0><<<side_grid[BK_BINC], 256, 0, sh>>>(dAt, dpre + 2 * (nd + 1), nd, side_per[BK_BINC]);
      note_launch();
    }
    if (hrow_grid) {
      if (wd == PL_W_BF16) k_hub_rows_batch<1><<<hrow_grid, kHubRows * 32, 0, sh>>>(dAt, dpre + 3 * (nd + 1), nd);
      else k_hub_rows_batch<0><<<hrow_grid, kHubRows * 32, 0, sh>>>(dAt, dpre + 3 * (nd + 1), nd);
      note_launch();
    }
    TRY(cudaEventRecord(g0->ev_join, sh));
    if (wd == PL_W_BF16) k_rows_batch<1><<<rows_grid, kRowThreads, 0, s>>>(dAt, dpre, nd, rows_per);
    else k_rows_batch<0><<<rows_grid, kRowThreads, 0, s>>>(dAt, dpre, nd, rows_per);
    note_launch();
    TRY(cudaStreamWaitEvent(s, g0->ev_join, 0));
  }
  TRY(cudaGetLastError());
  return PL_OK;
}

}  // namespace pl
