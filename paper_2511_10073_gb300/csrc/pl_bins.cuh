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
// kBinChunk; a CTA per chunk forms, for every slot, the chunk's double-float
// sum (exact products for the filter, weights and positive weights for the
// degrees), warps first and then the warps in order, so every partial is a
// fixed function of the inputs.  The row of bin b adds its slots' chunk
// partials in slot order, each slot's chunks in order.
#pragma once

#include "pl_common.cuh"

namespace pl {

constexpr int kBinThreads = 256;   // one CTA per chunk
constexpr int kBinPer = 4;         // hint cells per thread
constexpr int kBinChunk = kBinThreads * kBinPer;  // hint cells per chunk
constexpr int kBinSlotTile = 10;   // slots per round of a chunk (a warp sums each)

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
// bwq: the window blocks in bucket-list order (the block of the cell at list
// position k at k W), so a warp reads consecutive blocks; x: coordinates of
// every node (the cells' ones are gathered).  The chunk count is bchunk[NB];
// the grid may be any size.  Slots go in rounds of kBinSlotTile:
// each thread forms its cells' sums for the round's slots (every weight load
// of the round in flight at once) and leaves them in shared memory; warp j
// then adds slot j's 256 thread sums, lane q taking threads q, q + 32, ...
// in order, and a fixed tree over the lanes.
template <int WT, bool DEG>
__global__ void __launch_bounds__(kBinThreads) k_bin_partials(BinGeo B, const int32_t *bchunk,
                                                              const int32_t *cown,
                                                              const int64_t *boff,
                                                              const uint32_t *blist,
                                                              const void *bwq, const float2 *x,
                                                              float4 *part) {
  __shared__ float4 red[kBinSlotTile][kBinThreads];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nchunk = bchunk[B.NB];
  for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
    const int b = cown[c];
    const long long k0 = boff[2 * b] + (long long)(c - bchunk[b]) * kBinChunk;
    const long long k1 = boff[2 * b + 1];
    // thread t takes the chunk's cells t, t + kBinThreads, ...
    uint32_t ci[kBinPer];
    long long kp[kBinPer];
    bool cv[kBinPer];
#pragma unroll
    for (int u = 0; u < kBinPer; ++u) {
      kp[u] = k0 + threadIdx.x + (long long)u * kBinThreads;
      cv[u] = kp[u] < k1;
      ci[u] = (!DEG && cv[u]) ? blist[kp[u]] : 0u;
    }
    float2 xi[kBinPer];
#pragma unroll
    for (int u = 0; u < kBinPer; ++u) xi[u] = (!DEG && cv[u]) ? x[ci[u]] : make_float2(0.f, 0.f);
    for (int s0 = 0; s0 < B.W; s0 += kBinSlotTile) {
      const int ns = B.W - s0 < kBinSlotTile ? B.W - s0 : kBinSlotTile;
      float w[kBinPer][kBinSlotTile];
#pragma unroll
      for (int u = 0; u < kBinPer; ++u)
#pragma unroll
        for (int t = 0; t < kBinSlotTile; ++t)
          w[u][t] = (cv[u] && t < ns) ? bw_load<WT>(bwq, (size_t)kp[u] * B.W + s0 + t) : 0.f;
#pragma unroll
      for (int t = 0; t < kBinSlotTile; ++t) {
        if (t >= ns) break;
        dfl a{0.f, 0.f}, e{0.f, 0.f};
#pragma unroll
        for (int u = 0; u < kBinPer; ++u) {
          if (DEG) {
            df_add(a, w[u][t]);
            if (w[u][t] > 0.f) df_add(e, w[u][t]);
          } else {
            df_add_prod(a, w[u][t], xi[u].x);
            df_add_prod(e, w[u][t], xi[u].y);
          }
        }
        red[t][threadIdx.x] = make_float4(a.hi, a.lo, e.hi, e.lo);
      }
      __syncthreads();
      for (int t = wid; t < ns; t += kBinThreads / 32) {
        dfl a{0.f, 0.f}, e{0.f, 0.f};
#pragma unroll
        for (int q = lane; q < kBinThreads; q += 32) {
          const float4 v = red[t][q];
          df_add_df(a, dfl{v.x, v.y});
          df_add_df(e, dfl{v.z, v.w});
        }
        a = warp_sum_df(a);
        e = warp_sum_df(e);
        if (lane == 0) part[(size_t)c * B.W + s0 + t] = make_float4(a.hi, a.lo, e.hi, e.lo);
      }
      __syncthreads();
    }
  }
}

// Sums of bin b's row by the lanes of one warp.  Its (slot, chunk) pairs are
// taken in slot order, each slot's chunks of its source bucket in order, and
// dealt round robin to the lanes (a hot bucket's chunks spread over the
// warp); each lane adds its pairs in that order, then a fixed tree.  Returns
// the two double-floats of the partials' layout.
__device__ __forceinline__ void bin_row_sums(const BinGeo &B, int b, const int32_t *bchunk,
                                             const float4 *part, dfl *a, dfl *e) {
  const int lane = threadIdx.x & 31;
  const int bx = b % B.nbx, by = b / B.nbx, wx = 2 * B.hx + 1;
  dfl sa{0.f, 0.f}, se{0.f, 0.f};
  int flat = 0;  // pairs dealt before this slot
  for (int s = 0; s < B.W; ++s) {
    const int sx = bx - (s % wx - B.hx), sy = by - (s / wx - B.hy);
    if (sx < 0 || sy < 0 || sx >= B.nbx || sy >= B.nby) continue;
    const int src = sy * B.nbx + sx;
    const int c0 = bchunk[src], n = bchunk[src + 1] - c0;
    for (int k = (lane - flat % 32 + 32) % 32; k < n; k += 32) {
      const float4 q = __ldcg(&part[(size_t)(c0 + k) * B.W + s]);
      df_add_df(sa, dfl{q.x, q.y});
      df_add_df(se, dfl{q.z, q.w});
    }
    flat += n;
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

// Bucket of each chunk.
static __global__ void k_chunk_bins(int NB, const int32_t *bchunk, int32_t *cown) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < NB; b += gridDim.x * blockDim.x)
    for (int c = bchunk[b]; c < bchunk[b + 1]; ++c) cown[c] = b;
}

// Place of each movable cell in the bucket lists (the bucket-order copies of
// the window blocks are written at it).
static __global__ void k_bucket_rank(long long n, const uint32_t *blist, int32_t *crank) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    crank[blist[k]] = (int32_t)k;
}

}  // namespace pl
