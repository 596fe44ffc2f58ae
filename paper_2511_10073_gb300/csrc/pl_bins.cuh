// Bin rows of the augmented graph as the transpose of the cells' window
// blocks (Sec. V, bin virtual nodes; the column-free storage of the bin
// hints follows the Laplacian-sparsification outlook of Sec. IX).
//
// A hint cell i in bin b' stores the weights of its detection window as W
// slots, slot s = (dy + hy) (2 hx + 1) + (dx + hx) for the window bin
// b' + (dx, dy).  The row of bin node b therefore holds, for every slot s whose
// source bin b' = b - (dx_s, dy_s) lies in the grid, the cells of b''s hint
// bucket with weight w_s(i).  No entry of a bin row is stored: its sums are
// formed from the bucket lists and the window blocks.
//
// The hint cells of each bucket (ascending id) are cut into chunks of
// kBinChunk; a warp per chunk forms, for every slot, the chunk's double-float
// sum (exact products for the filter, weights and positive weights for the
// degrees), each lane over its cells in order and then a fixed tree over the
// lanes, so every partial is a fixed function of the inputs.  The row of bin b adds, slot by slot, the
// partials of that slot's source-bucket chunks (bin_row_chunks).
#pragma once

#include "pl_common.cuh"

namespace pl {

// 4 warps a CTA, each on its own chunks: a CTA of 8 K registers fits beside
// the refinement product's short-row kernel held to 5 CTAs per SM, so the bin
// rows run beside the short rows instead of after them
constexpr int kBinThreads = 128;
constexpr int kBinPer = 8;         // hint cells per lane
constexpr int kBinChunk = 32 * kBinPer;  // hint cells per chunk (one warp)

struct BinGeo {
  int nbx, nby, hx, hy, W;  // bin grid, window half widths, slots per window
  int NB;
};

// Offset (dx, dy) of slot s of a window.
__device__ __forceinline__ void slot_off(const BinGeo &B, int s, int *dx, int *dy) {
  const int wx = 2 * B.hx + 1;
  *dy = s / wx - B.hy;
  *dx = s % wx - B.hx;
}


template <int WT>
__device__ __forceinline__ float bw_load(const void *bw, size_t k) {
  if (WT == 0) return reinterpret_cast<const float *>(bw)[k];
  return __uint_as_float((uint32_t)reinterpret_cast<const unsigned short *>(bw)[k] << 16);
}

// Per chunk and slot, a float4 partial: with DEG, (sum w, sum of positive w)
// as two double-floats; otherwise (sum w x_i, sum w y_i) with exact products.
// A warp per chunk: lane j takes the chunk's cells j, j + 32, ... (all their
// loads in flight together); per slot, each lane adds its cells in order and
// a fixed tree adds the lanes, so every partial is a fixed function of the
// inputs.  bwq: the chunks' window blocks, slot-major within a chunk (slot t
// of the chunk's i-th cell at (c W + t) kBinChunk + i), so each slot is read
// as consecutive weights; x: coordinates of every node (the cells' ones are
// gathered).  The chunk count is bchunk[NB];
// the grid may be any size.
// Slots T0 .. T0 + NT - 1 of chunk c with the partials of all of them
// reduced over the warp at once (warp_rs_df): value 2 t of the slot group is
// the first double-float of slot T0 + t, value 2 t + 1 the second.  The same
// sums, bit for bit, as a warp_sum_df per slot and value.
template <int WT, bool DEG, int T0, int NT>
__device__ __forceinline__ void bin_slot_group(const void *bwq, size_t wbase, const bool *cv,
                                               const float2 *xi, float4 *part, size_t pbase) {
  const int lane = threadIdx.x & 31;
  dfl v[2 * NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    float w[kBinPer];
#pragma unroll
    for (int u = 0; u < kBinPer; ++u)
      w[u] = cv[u] ? bw_load<WT>(bwq, wbase + (size_t)(T0 + t) * kBinChunk + lane + 32 * u) : 0.f;
    dfl a{0.f, 0.f}, e{0.f, 0.f};
#pragma unroll
    for (int u = 0; u < kBinPer; ++u) {
      if (DEG) {
        df_add(a, w[u]);
        if (w[u] > 0.f) df_add(e, w[u]);
      } else {
        df_add_prod(a, w[u], xi[u].x);
        df_add_prod(e, w[u], xi[u].y);
      }
    }
    v[2 * t] = a;
    v[2 * t + 1] = e;
  }
  int pos = 0, cnt = 2 * NT;
  warp_rs_df<2 * NT, 16>(v, pos, cnt);
  if (cnt == 1) {
    const dfl r = df_norm(v[0]);
    reinterpret_cast<float2 *>(part)[(pbase + T0 + (pos >> 1)) * 2 + (pos & 1)] = make_float2(r.hi, r.lo);
  }
}

// Chunk c's partials (a warp).
template <int WT, bool DEG>
__device__ __forceinline__ void bin_chunk(const BinGeo &B, const int32_t *bchunk,
                                          const int32_t *cown, const int64_t *boff,
                                          const uint32_t *blist, const void *bwq,
                                          const float2 *x, float4 *part, long long c) {
  const int lane = threadIdx.x & 31;
  const int b = cown[c];
  const long long k0 = boff[2 * b] + (long long)(c - bchunk[b]) * kBinChunk;
  const long long k1 = boff[2 * b + 1];
  uint32_t kp[kBinPer];  // list positions (below 2^31: movable cells)
  bool cv[kBinPer];
  uint32_t ci[kBinPer];
#pragma unroll
  for (int u = 0; u < kBinPer; ++u) {
    kp[u] = (uint32_t)(k0 + lane + 32LL * u);
    cv[u] = k0 + lane + 32LL * u < k1;
    ci[u] = (!DEG && cv[u]) ? blist[kp[u]] : 0u;
  }
  float2 xi[kBinPer];
#pragma unroll
  for (int u = 0; u < kBinPer; ++u) xi[u] = (!DEG && cv[u]) ? x[ci[u]] : make_float2(0.f, 0.f);
  const size_t wbase = (size_t)c * B.W * kBinChunk;
  if (B.W == 9) {  // the 3 x 3 window: two slot groups, each reduced at once
    bin_slot_group<WT, DEG, 0, 5>(bwq, wbase, cv, xi, part, (size_t)c * 9);
    bin_slot_group<WT, DEG, 5, 4>(bwq, wbase, cv, xi, part, (size_t)c * 9);
    return;
  }
  for (int t = 0; t < B.W; ++t) {
    float w[kBinPer];
#pragma unroll
    for (int u = 0; u < kBinPer; ++u)
      w[u] = cv[u] ? bw_load<WT>(bwq, wbase + (size_t)t * kBinChunk + lane + 32 * u) : 0.f;
    dfl a{0.f, 0.f}, e{0.f, 0.f};
#pragma unroll
    for (int u = 0; u < kBinPer; ++u) {
      if (DEG) {
        df_add(a, w[u]);
        if (w[u] > 0.f) df_add(e, w[u]);
      } else {
        df_add_prod(a, w[u], xi[u].x);
        df_add_prod(e, w[u], xi[u].y);
      }
    }
    a = warp_sum_df(a);
    e = warp_sum_df(e);
    if (lane == 0) part[(size_t)c * B.W + t] = make_float4(a.hi, a.lo, e.hi, e.lo);
  }
}

template <int WT, bool DEG>
__global__ void __launch_bounds__(kBinThreads, 8) k_bin_partials(BinGeo B, const int32_t *bchunk,
                                                              const int32_t *cown,
                                                              const int64_t *boff,
                                                              const uint32_t *blist,
                                                              const void *bwq, const float2 *x,
                                                              float4 *part) {
  const int nchunk = bchunk[B.NB];
  for (long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; c < nchunk;
       c += ((long long)gridDim.x * blockDim.x) >> 5)
    bin_chunk<WT, DEG>(B, bchunk, cown, boff, blist, bwq, x, part, c);
}

template <bool DEG>
inline cudaError_t launch_bin_partials(int wt, int grid, cudaStream_t s, const BinGeo &B,
                                       const int32_t *bchunk, const int32_t *cown,
                                       const int64_t *boff, const uint32_t *blist,
                                       const void *bwq, const float2 *x, float4 *part) {
  if (wt == 2) k_bin_partials<1, DEG><<<grid, kBinThreads, 0, s>>>(B, bchunk, cown, boff, blist, bwq, x, part);
  else k_bin_partials<0, DEG><<<grid, kBinThreads, 0, s>>>(B, bchunk, cown, boff, blist, bwq, x, part);
  return cudaGetLastError();
}

// Sums of bin b's row by the lanes of one warp, straight from the chunk
// partials: for every slot s whose source bucket b - offset(s) lies in the
// grid, the partials of slot s of that bucket's chunks.  The items (slot by
// slot, each bucket's chunks in order; slots in groups of 32) are dealt to
// the lanes in turn, then a fixed tree adds the lanes, so the sums are a fixed
// function of the partials.  Returns the two double-floats of the partials'
// layout.
__device__ __forceinline__ void bin_row_chunks(const BinGeo &B, int b, const int32_t *bchunk,
                                               const float4 *part, dfl *a, dfl *e) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int bx = b % B.nbx, by = b / B.nbx, wx = 2 * B.hx + 1;
  dfl sa{0.f, 0.f}, se{0.f, 0.f};
  for (int s0 = 0; s0 < B.W; s0 += 32) {
    // lane j: the chunk range of slot s0 + j's source bucket
    const int s = s0 + lane;
    int c0 = 0, n = 0;
    if (s < B.W) {
      const int sx = bx - (s % wx - B.hx), sy = by - (s / wx - B.hy);
      if (sx >= 0 && sy >= 0 && sx < B.nbx && sy < B.nby) {
        const int bb = sy * B.nbx + sx;
        c0 = bchunk[bb];
        n = bchunk[bb + 1] - c0;
      }
    }
    int inc = n;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(full, inc, d);
      if (lane >= d) inc += t;
    }
    const int exc = inc - n, tot = __shfl_sync(full, inc, 31);
    constexpr int kU = 4;  // items a lane loads at once
    for (int i0 = 0; i0 < tot; i0 += 32 * kU) {
      float4 q[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int i = i0 + 32 * u + lane;
        // the lane whose range holds item i: the last one starting at or before it
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (__shfl_sync(full, exc, lo + step) <= i) lo += step;
        const int cj = __shfl_sync(full, c0, lo), ej = __shfl_sync(full, exc, lo);
        q[u] = i < tot ? __ldcg(&part[(size_t)(cj + i - ej) * B.W + s0 + lo])
                       : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        if (i0 + 32 * u + lane < tot) {
          df_add_df(sa, dfl{q[u].x, q[u].y});
          df_add_df(se, dfl{q[u].z, q[u].w});
        }
      }
    }
  }
  *a = warp_sum_df(sa);
  *e = warp_sum_df(se);
}

// Chunks of each bin's hint bucket: counts, to be scanned into bchunk.
static __global__ void k_bin_chunk_count(int NB, const int64_t *boff, int32_t *cnt) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < NB; b += gridDim.x * blockDim.x) {
    const long long n = boff[2 * b + 1] - boff[2 * b];
    cnt[b] = (int32_t)((n + kBinChunk - 1) / kBinChunk);
  }
}

// Bucket of each chunk: a thread per chunk finds the last bucket whose first
// chunk is at or before it (bchunk is nondecreasing).
static __global__ void k_chunk_bins(int NB, long long ncmax, const int32_t *bchunk, int32_t *cown) {
  const int nchunk = bchunk[NB];
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncmax && c < nchunk;
       c += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = NB - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (bchunk[mid] <= c) lo = mid;
      else hi = mid - 1;
    }
    cown[c] = lo;
  }
}

}  // namespace pl
