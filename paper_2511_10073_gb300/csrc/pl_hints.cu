// A2 + A3: area hints and the signed Laplacian, GPU-side (Sec. V).
//
//  * macro virtual node v_m joined to every movable cell overlapping macro m
//    by w = -exp(-maxRatio_{i,m}) * baseWeight_i;
//  * bin virtual node v_b joined to every movable cell whose centre bin lies
//    in the detection window of b by w = -exp(-maxRatio_{i,b}) phi_b
//    baseWeight_i, phi_b = 2 sigmoid(mu (D_b - C_b)) - 1;
//  * L_hint = D - A with signed D_ii; lambda_up = max_i (D_ii + sum_j |w_ij|)
//    (Gershgorin), which equals max_i 2 * (sum of positive w_ij).
// Decisions (bin of a centre, overlap) are FP32 with one stated operation
// sequence; D_b and phi_b are FP64; degree sums are double-float.  Edge
// weights are the FP64 value of the definition rounded once to the storage
// type: for BF16 storage an FP32 value (exponent argument carried in FP64)
// rounds to the same bf16 except within a few FP32 ulps of a bf16 rounding
// midpoint, where the FP64 value is computed; FP32 storage, whose rounding
// step an FP32 estimate cannot decide, always takes the FP64 value.
#include <cmath>
#include <cstring>
#include <mutex>

#include "pl_bins.cuh"
#include "pl_internal.h"

namespace pl {

#define TRY(x)                                       \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

constexpr int kMaxWin = 31;  // detection window at most 31 x 31 bins (a window row fits a warp)

struct HintGeo {
  float xlf, ylf, sxf, syf;      // bin decision: floor((x - xl) * sx)
  float gxf, gyf, gsxf, gsyf;    // macro grid bucket of a centre
  double xl, yl, wb, hb, iwb2, ihb2;  // bin centres; 2 / w_b, 2 / h_b
  float xlh, xll, ylh, yll;          // x_l, y_l as double-floats
  float iwh, iwl, ihh, ihl;          // 2 / w_b, 2 / h_b as double-floats
  int nbx, nby, hx, hy, gnx, gny;
  int32_t C, Pm, S, Mm;
  int64_t Nst, mv0, bn0, N;
};

__device__ __forceinline__ int bin_of(float x, float xl, float sc, int nb) {
  float t = __fmul_rn(__fadd_rn(x, -xl), sc);
  float f = floorf(t);
  if (!(f >= 0.f)) return 0;
  if (f > (float)(nb - 1)) return nb - 1;
  return (int)f;
}
__device__ __forceinline__ bool overlaps(float x, float y, float w, float h, float xm, float ym,
                                         float wm, float hm) {
  float dx = fabsf(__fadd_rn(x, -xm)), dy = fabsf(__fadd_rn(y, -ym));
  return dx < __fmul_rn(0.5f, __fadd_rn(w, wm)) && dy < __fmul_rn(0.5f, __fadd_rn(h, hm));
}
__device__ __forceinline__ int grid_of(float x, float x0, float sc, int n) { return bin_of(x, x0, sc, n); }

// e^{-r} for r >= 0 carried in FP64: FP32 exp of the rounded argument times
// the first-order correction for the rounding residue.
__device__ __forceinline__ float exp_neg(double r) {
  float rh = __double2float_rn(r);
  float rl = __double2float_rn(r - (double)rh);
  return expf(-rh) * (1.0f - rl);
}

// BF16 storage rounds the FP64 weight of the definition once.  The fast FP32
// value is within a few FP32 ulps of it (FP32 exp: 2 ulps, three roundings),
// so it rounds to the same bf16 unless it lies within kNearTie FP32 ulps of a
// bf16 rounding midpoint (low 16 bits near 0x8000); only then the weight is
// recomputed in FP64 with the exact operation sequence of the definition.
constexpr int kNearTie = 8;
__device__ __forceinline__ bool near_bf16_tie(float v) {
  int d = (int)(__float_as_uint(v) & 0xffffu) - 0x8000;
  return d >= -kNearTie && d <= kNearTie;
}
// -((e^{-maxRatio} * phi) * bw) for cell centre (x, y) and bin (xx, yy), FP64.
// Kept out of line: the fast path must not carry any of its FP64 work.
__device__ __noinline__ double bin_w_exact(float x, float y, int xx, int yy, const HintGeo &G, double phi,
                              double bw) {
  double xb = __dadd_rn(G.xl, __dmul_rn((double)xx + 0.5, G.wb));
  double yb = __dadd_rn(G.yl, __dmul_rn((double)yy + 0.5, G.hb));
  double dx = fabs(__dadd_rn((double)x, -xb)), dy = fabs(__dadd_rn((double)y, -yb));
  double r = fmax(__ddiv_rn(dx, __dmul_rn(G.wb, 0.5)), __ddiv_rn(dy, __dmul_rn(G.hb, 0.5)));
  double t = __dmul_rn(__dmul_rn(exp_cw(-r), phi), bw);
  return -t;
}
// -(e^{-maxRatio} * bw) for a cell centre and a macro (centre xm, ym; size wm, hm).
__device__ __noinline__ double macro_w_exact(float x, float y, float xm, float ym, float wm, float hm,
                                double bw) {
  double dx = fabs(__dadd_rn((double)x, -(double)xm)), dy = fabs(__dadd_rn((double)y, -(double)ym));
  double r = fmax(__ddiv_rn(dx, __dmul_rn((double)wm, 0.5)), __ddiv_rn(dy, __dmul_rn((double)hm, 0.5)));
  return -__dmul_rn(exp_cw(-r), bw);
}

// Writes the stored form of v and returns the value it stores.
__device__ __forceinline__ float store_w(void *wbuf, int wdtype, uint64_t k, float v) {
  if (wdtype == PL_W_BF16) {
    uint16_t h = f2bf16(v);
    reinterpret_cast<uint16_t *>(wbuf)[k] = h;
    return bf16_to_f(h);
  }
  reinterpret_cast<float *>(wbuf)[k] = v;
  return v;
}
// BF16 store of an exactly rounded FP64 weight.
__device__ __forceinline__ float store_bits(void *wbuf, uint64_t k, uint16_t h) {
  reinterpret_cast<uint16_t *>(wbuf)[k] = h;
  return bf16_to_f(h);
}
__device__ __forceinline__ float load_w(const void *wbuf, int wdtype, uint64_t k) {
  if (wdtype == PL_W_BF16) return bf16_to_f(reinterpret_cast<const uint16_t *>(wbuf)[k]);
  return reinterpret_cast<const float *>(wbuf)[k];
}
__device__ __forceinline__ void copy_w(void *dst, const void *src, int wdtype, uint64_t kd,
                                       uint64_t ks) {
  if (wdtype == PL_W_BF16)
    reinterpret_cast<uint16_t *>(dst)[kd] = reinterpret_cast<const uint16_t *>(src)[ks];
  else
    reinterpret_cast<float *>(dst)[kd] = reinterpret_cast<const float *>(src)[ks];
}

// Stores the stored form of v at k and, when k2 is not ~0, at k2 (the
// transposed entry of a symmetric pair); returns the value it stores.
__device__ __forceinline__ float store_w2(void *wbuf, int wdtype, uint64_t k, uint64_t k2, float v) {
  if (wdtype == PL_W_BF16) {
    const uint16_t h = f2bf16(v);
    reinterpret_cast<uint16_t *>(wbuf)[k] = h;
    if (k2 != ~0ull) reinterpret_cast<uint16_t *>(wbuf)[k2] = h;
    return bf16_to_f(h);
  }
  reinterpret_cast<float *>(wbuf)[k] = v;
  if (k2 != ~0ull) reinterpret_cast<float *>(wbuf)[k2] = v;
  return v;
}
__device__ __forceinline__ float store_bits2(void *wbuf, uint64_t k, uint64_t k2, uint16_t h) {
  reinterpret_cast<uint16_t *>(wbuf)[k] = h;
  if (k2 != ~0ull) reinterpret_cast<uint16_t *>(wbuf)[k2] = h;
  return bf16_to_f(h);
}

// Cells are taken in tiles of kBinTile consecutive ids by the stable counting
// sorts (bin buckets, macro lists).
constexpr int kBinTile = 4096;
constexpr int kMaxSmemBuckets = 12288;
constexpr int kMacroSlots = 8;        // macros one cell may overlap in the tiled macro lists
constexpr int kMaxSmemMacros = 12288;  // macros of the tiled macro lists (runs and masks in smem)

// --------------------------------------------------------- H1: cells
__global__ void k_hint_cells(HintGeo G, const float2 *xy, const uint8_t *ckind,
                             const uint8_t *hflag, const float *cw, const float *ch,
                             const int64_t *gptr, const uint32_t *glist, const float4 *ggeo,
                             int32_t *cell_bin, int32_t *n_ovl, int32_t *bcnt, int32_t *mcnt,
                             int32_t *mtc, int ntile, int32_t *cmem, int *status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.C; i += gridDim.x * blockDim.x) {
    // the cell's inputs in flight together, before the kind test
    const uint8_t kd = ckind[i];
    float2 p = xy[i];
    const bool hint = hflag[i] != 0;
    const float cwi = cw[i], chi = ch[i];
    if (kd != 0) {
      cell_bin[i] = -1;
      n_ovl[i] = 0;
      continue;
    }
    if (!isfinite(p.x) || !isfinite(p.y)) {
      flag(status, ST_NONFINITE);
      p = make_float2(0.f, 0.f);
    }
    int bx = bin_of(p.x, G.xlf, G.sxf, G.nbx), by = bin_of(p.y, G.ylf, G.syf, G.nby);
    int b = by * G.nbx + bx;
    cell_bin[i] = b;
    if (bcnt) atomicAdd(&bcnt[2 * b + (hint ? 0 : 1)], 1);
    int n = 0;
    if (hint) {
      int kx = grid_of(p.x, G.gxf, G.gsxf, G.gnx), ky = grid_of(p.y, G.gyf, G.gsyf, G.gny);
      long long k = (long long)ky * G.gnx + kx;
      for (long long q = gptr[k]; q < gptr[k + 1]; ++q) {
        const float4 mg = ggeo[q];
        if (overlaps(p.x, p.y, cwi, chi, mg.x, mg.y, mg.z, mg.w)) {
          const uint32_t m = glist[q];
          if (mtc) {
            atomicAdd(&mtc[(long long)m * ntile + i / kBinTile], 1);
            if (n < kMacroSlots) cmem[(long long)i * kMacroSlots + n] = (int32_t)m;
          } else {
            atomicAdd(&mcnt[m], 1);
          }
          ++n;
        }
      }
      if (mtc && n > kMacroSlots) flag(status, ST_MANY_OVL);
    }
    n_ovl[i] = n;
  }
}

// Cells overlapping each macro (the macro virtual rows), unordered here and
// sorted by cell id afterwards.
__global__ void k_macro_scatter(HintGeo G, const float2 *xy, const uint8_t *ckind,
                                const uint8_t *hflag, const float *cw, const float *ch,
                                const int64_t *gptr, const uint32_t *glist, const float4 *ggeo,
                                int32_t *mcur, uint32_t *mlist) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.C; i += gridDim.x * blockDim.x) {
    if (ckind[i] != 0 || !hflag[i]) continue;
    float2 p = xy[i];
    if (!isfinite(p.x) || !isfinite(p.y)) p = make_float2(0.f, 0.f);
    int kx = grid_of(p.x, G.gxf, G.gsxf, G.gnx), ky = grid_of(p.y, G.gyf, G.gsyf, G.gny);
    long long k = (long long)ky * G.gnx + kx;
    const float cwi = cw[i], chi = ch[i];
    for (long long q = gptr[k]; q < gptr[k + 1]; ++q) {
      const float4 mg = ggeo[q];
      if (overlaps(p.x, p.y, cwi, chi, mg.x, mg.y, mg.z, mg.w))
        mlist[atomicAdd(&mcur[glist[q]], 1)] = (uint32_t)i;
    }
  }
}

// Macro lists in ascending cell id without a sort: a CTA per tile of kBinTile
// cells, counts per (macro, tile) macro-major and each cell's macros (at most
// kMacroSlots) from k_hint_cells.  In rounds of blockDim cells the warps take
// turns; inside a turn the lanes mark their macros in a per-macro lane mask,
// and a membership's place is its macro's tile start (loaded before the
// turns), the macro's run so far and the number of lower lanes marked.
__global__ void __launch_bounds__(256, 4) k_macro_tile_scatter(int32_t C, const int32_t *n_ovl,
                                                            const int32_t *cmem, int Mm,
                                                            int ntile, const int64_t *off,
                                                            uint32_t *mlist) {
  extern __shared__ uint32_t lmask[];  // [Mm] lane masks, then [Mm] runs (at most kBinTile)
  uint16_t *run = reinterpret_cast<uint16_t *>(lmask + Mm);
  for (int k = threadIdx.x; k < Mm; k += blockDim.x) {
    run[k] = 0;
    lmask[k] = 0u;
  }
  __syncthreads();
  const int t = blockIdx.x, i0 = t * kBinTile, i1 = min(C, i0 + kBinTile);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  // a round's cell memberships are loaded during the round before
  int nn = i0 + (int)threadIdx.x < i1 ? min(n_ovl[i0 + threadIdx.x], kMacroSlots) : 0;
  int32_t mn[kMacroSlots];
#pragma unroll
  for (int j = 0; j < kMacroSlots; ++j)
    mn[j] = j < nn ? cmem[(long long)(i0 + threadIdx.x) * kMacroSlots + j] : 0;
  for (int base = i0; base < i1; base += blockDim.x) {
    const int i = base + threadIdx.x;
    // n_ovl is 0 for cells other than movable hint cells
    const int n = nn;
    int32_t mk[kMacroSlots];
    long long tst[kMacroSlots];
#pragma unroll
    for (int j = 0; j < kMacroSlots; ++j) {
      mk[j] = mn[j];
      tst[j] = j < n ? off[(long long)mk[j] * ntile + t] : 0;
    }
    const int inext = i + (int)blockDim.x;
    nn = inext < i1 ? min(n_ovl[inext], kMacroSlots) : 0;
#pragma unroll
    for (int j = 0; j < kMacroSlots; ++j)
      mn[j] = j < nn ? cmem[(long long)inext * kMacroSlots + j] : 0;
    // places within the tile's runs, by turns in shared memory; the stores
    // wait for the tile starts only after the turns
    int rel[kMacroSlots];
    for (int w = 0; w < nw; ++w) {
      if (wid == w) {
#pragma unroll
        for (int j = 0; j < kMacroSlots; ++j)
          if (j < n) atomicOr(&lmask[mk[j]], 1u << lane);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kMacroSlots; ++j)
          rel[j] = j < n ? (int)run[mk[j]] + __popc(lmask[mk[j]] & lt) : 0;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kMacroSlots; ++j) {
          if (j < n) {
            const uint32_t msk = lmask[mk[j]];
            if (msk && lane == __ffs(msk) - 1) {
              run[mk[j]] = (uint16_t)(run[mk[j]] + __popc(msk));
              lmask[mk[j]] = 0u;
            }
          }
        }
        __syncwarp();
      }
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < kMacroSlots; ++j)
      if (j < n) mlist[tst[j] + rel[j]] = (uint32_t)i;
  }
}

// Bin buckets: key 2*bin + (baseWeight == 0).  A stable counting sort over
// tiles of kBinTile consecutive cells writes every bucket in ascending cell id
// directly (no sort).  Counts per (bucket, tile), bucket-major.

__device__ __forceinline__ int bucket_of(const uint8_t *hflag, const int32_t *cell_bin, int i) {
  return 2 * cell_bin[i] + (hflag[i] ? 0 : 1);
}

__global__ void __launch_bounds__(256) k_bin_tile_count(int32_t C, int nbk, int ntile,
                                                        const uint8_t *ckind,
                                                        const uint8_t *hflag,
                                                        const int32_t *cell_bin, int32_t *cnt) {
  extern __shared__ int32_t sc[];
  for (int k = threadIdx.x; k < nbk; k += blockDim.x) sc[k] = 0;
  __syncthreads();
  const int t = blockIdx.x, i0 = t * kBinTile, i1 = min(C, i0 + kBinTile);
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x)
    if (ckind[i] == 0) atomicAdd(&sc[bucket_of(hflag, cell_bin, i)], 1);
  __syncthreads();
  for (int k = threadIdx.x; k < nbk; k += blockDim.x) cnt[(long long)k * ntile + t] = sc[k];
}

// Rounds of blockDim cells; inside a round the warps take turns (so equal
// buckets keep cell order), lanes of a warp rank themselves with match_any.
__global__ void __launch_bounds__(256) k_bin_tile_scatter(int32_t C, int nbk, int ntile,
                                                          const uint8_t *ckind,
                                                          const uint8_t *hflag,
                                                          const int32_t *cell_bin,
                                                          const int64_t *off, uint32_t *blist) {
  extern __shared__ int32_t run[];
  for (int k = threadIdx.x; k < nbk; k += blockDim.x) run[k] = 0;
  __syncthreads();
  const int t = blockIdx.x, i0 = t * kBinTile, i1 = min(C, i0 + kBinTile);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int base = i0; base < i1; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const bool mv = i < i1 && ckind[i] == 0;
    const int key = mv ? bucket_of(hflag, cell_bin, i) : -1 - lane;
    const long long tst = mv ? off[(long long)key * ntile + t] : 0;  // loaded before the turns
    int rel = 0;  // place within the tile's run of the bucket (the store waits for tst after the turns)
    for (int w = 0; w < nw; ++w) {
      if (wid == w) {
        unsigned grp = __match_any_sync(0xffffffffu, key);
        int leader = __ffs(grp) - 1;
        int before = 0;
        if (mv && lane == leader) {
          before = run[key];
          run[key] = before + __popc(grp);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        rel = before + __popc(grp & lt);
      }
      __syncthreads();
    }
    if (mv) blist[tst + rel] = (uint32_t)i;
  }
}

// The same lists without turns, for grids whose per-warp counters fit shared
// memory (20 nbk bytes): in each round every warp ranks its lanes by key with
// match_any and writes its group sizes to its own row of counters; after a
// barrier a cell's place is the key's run so far, plus the same key's cells in
// the round's lower warps, plus its lower lanes of the same key, which is its
// place in cell order.  Two barriers per round instead of one per warp.
__global__ void __launch_bounds__(256) k_bin_tile_scatter_wc(int32_t C, int nbk, int ntile,
                                                             const uint8_t *ckind,
                                                             const uint8_t *hflag,
                                                             const int32_t *cell_bin,
                                                             const int64_t *off, uint32_t *blist) {
  extern __shared__ int32_t run[];  // [nbk] runs, then uint16 [8][nbk] counts of the round
  uint16_t *wc = reinterpret_cast<uint16_t *>(run + nbk);
  for (int k = threadIdx.x; k < nbk; k += blockDim.x) run[k] = 0;
  for (int k = threadIdx.x; k < 8 * nbk; k += blockDim.x) wc[k] = 0;
  __syncthreads();
  const int t = blockIdx.x, i0 = t * kBinTile, i1 = min(C, i0 + kBinTile);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int base = i0; base < i1; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const bool mv = i < i1 && ckind[i] == 0;
    const int key = mv ? bucket_of(hflag, cell_bin, i) : -1 - lane;
    const long long tst = mv ? off[(long long)key * ntile + t] : 0;
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const bool lead = mv && lane == __ffs(grp) - 1;
    if (lead) wc[wid * nbk + key] = (uint16_t)__popc(grp);
    __syncthreads();
    int rel = 0;
    if (mv) {
      rel = run[key] + __popc(grp & lt);
      for (int w = 0; w < wid; ++w) rel += wc[w * nbk + key];
    }
    __syncthreads();  // the round's counters are read
    if (lead) {
      atomicAdd(&run[key], __popc(grp));  // warps of the round may share a key
      wc[wid * nbk + key] = 0;
    }
    __syncwarp();
    if (mv) blist[tst + rel] = (uint32_t)i;
  }
}

__global__ void k_bucket_starts(int nbk, int ntile, const int64_t *off, int64_t *boff) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= nbk; k += gridDim.x * blockDim.x)
    boff[k] = off[(long long)k * ntile];
}

// Fallback for bin grids too large for the shared-memory counters: atomic
// scatter, then the buckets are sorted.
__global__ void k_bin_scatter_atomic(int32_t C, const uint8_t *ckind, const uint8_t *hflag,
                                     const int32_t *cell_bin, int32_t *bcur, uint32_t *blist) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x)
    if (ckind[i] == 0) blist[atomicAdd(&bcur[bucket_of(hflag, cell_bin, i)], 1)] = (uint32_t)i;
}

// ------------------------------------------------ H5: bin density and phi
// D_b: FP64 sum of the cell areas w*h of bin b's sequence (its hint bucket
// then its other bucket, each ascending), in the blocked order: blocks of 64
// added left to right, block sums summed the same way, recursively.  A CTA per
// bin forms every level in parallel; level l of bin b lives at offset
// floor(start_{l-1}/64) + b of that level's region, so bins never overlap.
constexpr int kMaxLevels = 8;
struct LevelBufs {
  double *base[kMaxLevels];
};

// Cell areas w h in FP64 (exact: a product of two floats fits a double), once
// per netlist, so that the density sums take one FP64 operation per cell.
__global__ void k_cell_area(int32_t C, const float *cw, const float *ch, double *area) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x)
    area[i] = __dmul_rn((double)cw[i], (double)ch[i]);
}

// A_mov(b) as a blocked FP64 sum: the bin's cells (hint cells ascending,
// then the others ascending) in blocks of 64 added left to right, the block
// sums blocked again, until at most 64 values remain, which are added left to
// right.  Level L of bin b reads len_L(b) values starting at st_L(b) (level
// 0: cell areas through the bucket list) and writes its block sums to
// out_L(b) = st_L(b) / 64 + b onwards; these ranges are disjoint and
// increasing in b, so every block of every bin is one thread of one launch.
struct DensLevel {
  int64_t st, len, out;
};
__device__ __forceinline__ DensLevel dens_level(const int64_t *boff, int b, int L) {
  DensLevel d;
  d.st = boff[2 * b];
  d.len = boff[2 * b + 2] - d.st;
  d.out = d.st / 64 + b;
  for (int l = 0; l < L; ++l) {
    d.st = d.out;
    d.len = (d.len + 63) / 64;
    d.out = d.st / 64 + b;
  }
  return d;
}

__global__ void __launch_bounds__(256) k_dens_level(int NB, int L, const int64_t *boff,
                                                    const uint32_t *blist, const double *area,
                                                    const double *prev, double *out,
                                                    long long nidx) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nidx;
       idx += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = NB - 1;  // last bin with out_L(b) <= idx
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (dens_level(boff, mid, L).out <= idx) lo = mid; else hi = mid - 1;
    }
    const DensLevel d = dens_level(boff, lo, L);
    const int64_t j = idx - d.out;
    if (d.len <= 64 || j < 0 || j >= (d.len + 63) / 64) continue;
    const int64_t k0 = d.st + 64 * j, k1 = min(d.st + d.len, k0 + 64);
    double acc = 0.0;
    if (L == 0) {
      for (int64_t k = k0; k < k1; k += 16) {
        double a[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) a[q] = k + q < k1 ? area[blist[k + q]] : 0.0;
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (k + q < k1) acc = __dadd_rn(acc, a[q]);
      }
    } else {
      for (int64_t k = k0; k < k1; ++k) acc = __dadd_rn(acc, prev[k]);
    }
    out[idx] = acc;
  }
}

// Per bin: the last (at most 64-value) sum, D_b, C_b, phi_b and the hub row
// length (hint cells of the window bins).
__global__ void k_dens_final(HintGeo G, int nlev, const int64_t *boff, const uint32_t *blist,
                             const double *area, LevelBufs lv, const double *amac,
                             double abin, double cap, double mu, double *Db, double *Cb,
                             double *phi, float *phif) {
  const int NB = G.nbx * G.nby;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < NB; b += gridDim.x * blockDim.x) {
    int L = 0;
    DensLevel d = dens_level(boff, b, 0);
    while (d.len > 64 && L < nlev) {
      ++L;
      d = dens_level(boff, b, L);
    }
    const double *src = L ? lv.base[L - 1] : nullptr;
    double acc = 0.0;
    for (int64_t k = 0; k < d.len; k += 16) {
      double a[16];
#pragma unroll
      for (int q = 0; q < 16; ++q)
        a[q] = k + q < d.len ? (L == 0 ? area[blist[d.st + k + q]] : src[d.st + k + q])
                             : 0.0;
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (k + q < d.len) acc = __dadd_rn(acc, a[q]);
    }
    const double dd = __ddiv_rn(acc, abin);
    const double c = __ddiv_rn(__dmul_rn(cap, __dadd_rn(abin, -amac[b])), abin);
    const double t = __dmul_rn(mu, __dadd_rn(dd, -c));
    const double ph = __dadd_rn(__ddiv_rn(2.0, __dadd_rn(1.0, exp_cw(-t))), -1.0);
    Db[b] = dd;
    Cb[b] = c;
    phi[b] = ph;
    phif[b] = __double2float_rn(ph);
  }
}

// ------------------------------------------------------- H6: row lengths
__device__ __forceinline__ int win_count(int bx, int by, const HintGeo &G) {
  int nx = min(G.nbx - 1, bx + G.hx) - max(0, bx - G.hx) + 1;
  int ny = min(G.nby - 1, by + G.hy) - max(0, by - G.hy) + 1;
  return nx * ny;
}

// Per-row lengths of a split matrix.  Static mode: the st rows (hub when
// longer than kLong).  Hint mode: the stored hm part of each row (a hint
// cell's macro entries, a macro row's cells; bin rows store nothing, their
// sums come from the window blocks); a row is a hub row when it is a virtual
// node or its static entries, macro entries and window slots exceed kLong.
// clen is the stored length the hub chunks cover (st part + hm part).
__global__ void k_row_len(HintGeo G, int with_hints, const int64_t *srp, const uint8_t *hflag,
                          const int32_t *cell_bin, const int32_t *n_ovl, const int64_t *moff,
                          uint32_t *slen, uint64_t *llen, uint8_t *lflag, uint64_t *clen) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < G.N;
       v += (long long)gridDim.x * blockDim.x) {
    const long long sl = v < G.Nst ? srp[v + 1] - srp[v] : 0;
    if (!with_hints) {
      const bool hub = sl > kLong;
      slen[v] = hub ? 0u : (uint32_t)sl;
      llen[v] = hub ? (uint64_t)sl : 0ull;
      lflag[v] = hub ? 1 : 0;
      clen[v] = hub ? (uint64_t)sl : 0ull;
      continue;
    }
    long long hl = 0, ws = 0;
    bool virt = false;
    if (v < G.C && hflag[v]) {
      int b = cell_bin[v];
      hl = n_ovl[v];
      ws = win_count(b % G.nbx, b / G.nbx, G);
    } else if (v >= G.mv0 && v < G.bn0) {
      hl = moff[v - G.mv0 + 1] - moff[v - G.mv0];
      virt = true;
    } else if (v >= G.bn0) {
      virt = true;
    }
    const bool hub = virt || sl + hl + ws > kLong;
    slen[v] = hub ? 0u : (uint32_t)hl;
    llen[v] = hub ? (uint64_t)hl : 0ull;
    lflag[v] = hub ? 1 : 0;
    clen[v] = hub ? (uint64_t)(sl + hl) : 0ull;
  }
}

__global__ void k_layout_long(int64_t N, const uint8_t *lflag, const int32_t *lscan,
                              const uint64_t *lpos, const uint64_t *clen, uint64_t nnz_s,
                              int32_t *lrow, uint64_t *lptr, int32_t *longidx,
                              int32_t *nchunk_of) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    if (lflag[v]) {
      int li = lscan[v];
      lrow[li] = (int32_t)v;
      lptr[li] = nnz_s + lpos[v];
      longidx[v] = li;
      const uint64_t len = clen[v];
      nchunk_of[li] = len == 0 ? 1 : (int32_t)((len + kChunk - 1) / kChunk);
    } else {
      longidx[v] = -1;
    }
    if (v == N - 1) {
      int nl = lscan[N];
      lptr[nl] = nnz_s + lpos[N];
    }
  }
}

__global__ void k_chunk_owner(int32_t nlong, const int32_t *lchunk, int32_t *chunk_lr) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlong; l += gridDim.x * blockDim.x)
    for (int c = lchunk[l]; c < lchunk[l + 1]; ++c) chunk_lr[c] = l;
}

// Short-row pointers with the hub flag of each row in bit 31; padded with the
// end offset so that aligned bulk copies may read a few entries past N.
__global__ void k_rp_pack(const uint64_t *s64, const uint8_t *lflag, int64_t N, uint32_t *rp) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v <= N + kRpPad;
       v += (long long)gridDim.x * blockDim.x) {
    if (v < N) rp[v] = (uint32_t)s64[v] | (lflag[v] ? kHubFlag : 0u);
    else rp[v] = (uint32_t)s64[N];
  }
}

__global__ void k_u64_to_u32(const uint64_t *a, uint32_t *b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (uint32_t)a[i];
}

// st and hm pieces of every hub row (see SpMat).  Static matrix: its own hub
// region only.  Hint matrix: the row's st part (short or hub region of st) and
// its hm hub part.
__global__ void k_hub_desc(int32_t nlong, int with_hints, const int32_t *lrow,
                           const uint64_t *lptr, const int64_t *srp, int64_t Nst,
                           const uint32_t *st_rp, const int32_t *st_longidx,
                           const uint64_t *st_lptr, uint64_t *lsb, uint32_t *lsl, uint64_t *lhb,
                           uint32_t *lhl) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlong; l += gridDim.x * blockDim.x) {
    if (!with_hints) {
      lsb[l] = lptr[l];
      lsl[l] = (uint32_t)(lptr[l + 1] - lptr[l]);
      lhb[l] = 0;
      lhl[l] = 0;
      continue;
    }
    const int64_t v = lrow[l];
    const long long sl = v < Nst ? srp[v + 1] - srp[v] : 0;
    const int sli = v < Nst ? st_longidx[v] : -1;
    lsb[l] = sli >= 0 ? st_lptr[sli] : (uint64_t)(st_rp[v] & kOffMask);
    lsl[l] = (uint32_t)sl;
    lhb[l] = lptr[l];
    lhl[l] = (uint32_t)(lptr[l + 1] - lptr[l]);
  }
}

// ------------------------------------------------------- H9: row assembly
__device__ __forceinline__ void acc_deg(dfl &D, dfl &Pp, float w) {
  df_add(D, w);
  if (w > 0.f) df_add(Pp, w);
}

// |u - c| as a normalized double-float, for u = uh + ul (ul the rounding
// residue of uh) and an exactly representable c: TwoSum of uh and -c, then
// the low parts.
__device__ __forceinline__ dfl df_absdiff(float uh, float ul, float c) {
  dfl s{uh, 0.f};
  df_add(s, -c);
  s.lo = __fadd_rn(s.lo, ul);
  s = df_norm(s);
  if (s.hi < 0.f) s = dfl{-s.hi, -s.lo};
  return s;
}
__device__ __forceinline__ bool df_ge(dfl a, dfl b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo);
}
// e^{-r} for r = hi + lo >= 0, the form of exp_neg.
__device__ __forceinline__ float exp_neg_df(dfl r) { return expf(-r.hi) * (1.0f - r.lo); }

// (x - o) * s for a float x, o = oh + ol and s = sh + sl (double-floats), to
// about 44 bits with FP32 operations only.
__device__ __forceinline__ dfl df_offset_scale(float x, float oh, float ol, float sh, float sl) {
  dfl d{x, 0.f};
  df_add(d, -oh);
  d.lo = __fadd_rn(d.lo, -ol);
  d = df_norm(d);
  const float ph = __fmul_rn(d.hi, sh);
  float pl = __fmaf_rn(d.hi, sh, -ph);
  pl = __fmaf_rn(d.hi, sl, pl);
  pl = __fmaf_rn(d.lo, sh, pl);
  return df_norm(dfl{ph, pl});
}
// |x - c| / h for floats x, c and h > 0 as a double-float: the difference
// is exact (TwoSum), the quotient carries its FMA remainder.
__device__ __forceinline__ dfl df_ratio(float x, float c, float h) {
  if (!(h > 0.f)) return dfl{__int_as_float(0x7f800000), 0.f};
  dfl d{x, 0.f};
  df_add(d, -c);
  d = df_norm(d);
  if (d.hi < 0.f) d = dfl{-d.hi, -d.lo};
  const float q = __fdiv_rn(d.hi, h);
  const float r = __fmaf_rn(-q, h, d.hi);
  return df_norm(dfl{q, __fdiv_rn(__fadd_rn(r, d.lo), h)});
}

// Hint part of the rows of cells, macro pins and stars (thread per row): for a
// hint cell its macro entries (ascending macro), written to the row's hm
// place, and the weights of its detection-window bins as a dense block of W
// slots, slot s = (yy - by + hy) (2 hx + 1) + (xx - bx + hx) for window bin
// (xx, yy) around the cell's bin (bx, by); slots outside the bin grid hold 0.
// The column of a slot is implicit (the bin node of that window position), and
// the bin rows are the transpose of these blocks (k_bin_partials).  The degree
// sums of the whole augmented row are the static ones plus the hint entries.
// The window ratios |x - x_b| / (w_b / 2) = |u - (2 xx + 1)|, u = 2 (x - x_l) /
// w_b, come from u (double-float, once per cell) as exact double-float
// differences; macro ratios are double-float quotients.  With BF16 storage FP64
// only recomputes weights near a bf16 rounding midpoint; with FP32 storage
// every weight is the FP64 value of the definition rounded once.
constexpr int kAsmStage = 768;  // own entries of a warp's 32 rows staged in shared memory
__global__ void __launch_bounds__(256, 3) k_assemble_hints(
    HintGeo G, int wdtype, const uint32_t *hrp, const int32_t *longidx, const uint64_t *lptr,
    const dfl *sdsum, const dfl *spsum, const uint8_t *hflag, const int32_t *cell_bin,
    const int32_t *n_ovl, const float2 *xy, const float *cw, const float *ch,
    const int64_t *gptr, const uint32_t *glist, const float4 *ggeo, const double *base_w,
    const float *phif, const double *phid, int W, const int32_t *cmem, const float4 *mgeo,
    int32_t *col, void *w, void *bwin, int32_t *hbin, dfl *dsum, dfl *psum, uint64_t *mac_base,
    unsigned long long *counts) {
  __shared__ int32_t stage_col[8][kAsmStage];
  __shared__ uint32_t stage_w[8][kAsmStage];
  const bool bf = wdtype == PL_W_BF16;
  const int lane = threadIdx.x & 31;
  int32_t *scol = stage_col[threadIdx.x >> 5];
  uint32_t *sw = stage_w[threadIdx.x >> 5];
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long slots = 0, hints = 0;  // this thread's window slots in the grid, hint cells
  for (long long v0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); v0 < G.Nst;
       v0 += stride) {
    const long long v = v0 + lane;
    // the warp's rows own a contiguous short-region range [rb, re)
    const uint64_t rb = hrp[v0] & kOffMask;
    const uint64_t re = hrp[v0 + 32 < G.Nst ? v0 + 32 : G.Nst] & kOffMask;
    const bool staged = re - rb <= (uint64_t)kAsmStage;  // warp-uniform
    if (v >= G.Nst) goto flush;
    {
    dfl Dl = sdsum[v], Pl = spsum[v];
    // a cell's inputs, loaded before its hint test so that they are in flight
    // together rather than one dependent round after another
    uint8_t hf = 0;
    int li = -1, cb = 0, nov = 0;
    uint32_t hr = 0;
    float2 p = make_float2(0.f, 0.f);
    double bw = 0.0;
    if (v < G.C) {
      hf = hflag[v];
      li = longidx[v];
      hr = hrp[v];
      p = xy[v];
      bw = base_w[v];
      cb = cell_bin[v];
      nov = n_ovl[v];
    }
    if (v < G.C) hbin[v] = hf ? cb : -1;
    if (hf) {
      ++hints;
      const uint64_t mb = li >= 0 ? lptr[li] : (uint64_t)(hr & kOffMask);
      const bool use_s = staged && li < 0;
      // an own entry: to the warp's stage (short rows) or straight to memory
      auto put = [&](uint64_t kk, int32_t c, uint32_t bits) {
        if (use_s) {
          scol[kk - rb] = c;
          sw[kk - rb] = bits;
        } else {
          col[kk] = c;
          if (bf) reinterpret_cast<uint16_t *>(w)[kk] = (uint16_t)bits;
          else reinterpret_cast<uint32_t *>(w)[kk] = bits;
        }
      };
      if (!isfinite(p.x) || !isfinite(p.y)) p = make_float2(0.f, 0.f);
      const float bwf = __double2float_rn(bw);
      // macro entries, ascending macro id (grid bucket lists are sorted)
      uint64_t k = mb;
      auto mac_entry = [&](int m, float4 mg) {
        uint32_t bits;
        float sv;
        if (bf) {
          const dfl rx = df_ratio(p.x, mg.x, __fmul_rn(0.5f, mg.z));
          const dfl ry = df_ratio(p.y, mg.y, __fmul_rn(0.5f, mg.w));
          const float wv = -(exp_neg_df(df_ge(rx, ry) ? rx : ry) * bwf);
          const uint16_t h = near_bf16_tie(wv)
                                 ? d2bf16(macro_w_exact(p.x, p.y, mg.x, mg.y, mg.z, mg.w, bw))
                                 : f2bf16(wv);
          bits = h;
          sv = bf16_to_f(h);
        } else {
          sv = __double2float_rn(macro_w_exact(p.x, p.y, mg.x, mg.y, mg.z, mg.w, bw));
          bits = __float_as_uint(sv);
        }
        put(k, (int32_t)(G.mv0 + m), bits);
        acc_deg(Dl, Pl, sv);
        ++k;
      };
      if (cmem) {
        // the cell's macros as the cell pass found them (same geometry values)
        for (int j = 0; j < nov; ++j) {
          const int m = cmem[(long long)v * kMacroSlots + j];
          mac_entry(m, mgeo[m]);
        }
      } else {
        const int kx = grid_of(p.x, G.gxf, G.gsxf, G.gnx), ky = grid_of(p.y, G.gyf, G.gsyf, G.gny);
        const long long gk = (long long)ky * G.gnx + kx;
        const float cwv = cw[v], chv = ch[v];
        const long long qa = gptr[gk], qb = gptr[gk + 1];
        for (long long q0 = qa; q0 < qb; q0 += 4) {
          float4 mgs[4];  // four grid entries' geometry loaded at once
#pragma unroll
          for (int u = 0; u < 4; ++u) mgs[u] = q0 + u < qb ? ggeo[q0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const long long q = q0 + u;
            const float4 mg = mgs[u];
            if (q >= qb || !overlaps(p.x, p.y, cwv, chv, mg.x, mg.y, mg.z, mg.w)) continue;
            mac_entry((int)glist[q], mg);
          }
        }
      }
      // window slots, row-major over the full window
      const int b = cb, bx = b % G.nbx, by = b / G.nbx, wx = 2 * G.hx + 1;
      const dfl ux = df_offset_scale(p.x, G.xlh, G.xll, G.iwh, G.iwl);
      const dfl uy = df_offset_scale(p.y, G.ylh, G.yll, G.ihh, G.ihl);
      uint16_t *wb16 = reinterpret_cast<uint16_t *>(bwin) + (size_t)v * W;
      uint32_t *wb32 = reinterpret_cast<uint32_t *>(bwin) + (size_t)v * W;
      int sidx = 0;
      if (bf && G.hx == 1) {
        // three window columns: their ratios and e^{-rx} once per cell, not
        // once per window row (the same values, so the same weights)
        dfl rxs[3];
        float exs[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int xx = bx - 1 + c;
          rxs[c] = df_absdiff(ux.hi, ux.lo, (float)(2 * xx + 1));
          exs[c] = (xx >= 0 && xx < G.nbx) ? exp_neg_df(rxs[c]) : 0.f;
        }
        for (int yy = by - G.hy; yy <= by + G.hy; ++yy) {
          const bool yin = yy >= 0 && yy < G.nby;
          const dfl ry = df_absdiff(uy.hi, uy.lo, (float)(2 * yy + 1));
          const float ey = yin ? exp_neg_df(ry) : 0.f;
          float ph[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int xx = bx - 1 + c;
            ph[c] = (yin && xx >= 0 && xx < G.nbx) ? phif[yy * G.nbx + xx] : 0.f;
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int xx = bx - 1 + c;
            uint16_t h = 0;
            if (yin && xx >= 0 && xx < G.nbx) {
              const float e = df_ge(rxs[c], ry) ? exs[c] : ey;
              const float wv = -((e * ph[c]) * bwf);
              h = near_bf16_tie(wv)
                      ? d2bf16(bin_w_exact(p.x, p.y, xx, yy, G, phid[yy * G.nbx + xx], bw))
                      : f2bf16(wv);
              acc_deg(Dl, Pl, bf16_to_f(h));
              ++slots;
            }
            wb16[sidx++] = h;
          }
        }
      } else
      for (int yy = by - G.hy; yy <= by + G.hy; ++yy) {
        const bool yin = yy >= 0 && yy < G.nby;
        // e^{-max(rx, ry)} is e^{-rx} or e^{-ry}
        const dfl ry = df_absdiff(uy.hi, uy.lo, (float)(2 * yy + 1));
        const float ey = (bf && yin) ? exp_neg_df(ry) : 0.f;
        for (int xc = bx - G.hx; xc <= bx + G.hx; xc += 4) {
          float ph[4];  // four window bins' phi loaded at once
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int xx = xc + u;
            ph[u] = (yin && xx >= 0 && xx < G.nbx && xx <= bx + G.hx) ? phif[yy * G.nbx + xx] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int xx = xc + u;
            if (xx > bx + G.hx) break;
            uint32_t bits = 0;
            if (yin && xx >= 0 && xx < G.nbx) {
              const int bb = yy * G.nbx + xx;
              float sv;
              if (bf) {
                const dfl rx = df_absdiff(ux.hi, ux.lo, (float)(2 * xx + 1));
                const float e = df_ge(rx, ry) ? exp_neg_df(rx) : ey;
                const float wv = -((e * ph[u]) * bwf);
                const uint16_t h = near_bf16_tie(wv)
                                       ? d2bf16(bin_w_exact(p.x, p.y, xx, yy, G, phid[bb], bw))
                                       : f2bf16(wv);
                bits = h;
                sv = bf16_to_f(h);
              } else {
                sv = __double2float_rn(bin_w_exact(p.x, p.y, xx, yy, G, phid[bb], bw));
                bits = __float_as_uint(sv);
              }
              acc_deg(Dl, Pl, sv);
              ++slots;
            }
            if (bf) wb16[sidx] = (uint16_t)bits;
            else wb32[sidx] = bits;
            ++sidx;
          }
        }
      }
      (void)wx;
      mac_base[v] = mb;
    }
    dsum[v] = df_norm(Dl);
    psum[v] = df_norm(Pl);
    }
  flush:
    // the staged range, written with coalesced stores
    if (staged) {
      __syncwarp();
      for (uint64_t i = lane; i < re - rb; i += 32) {
        col[rb + i] = scol[i];
        if (bf) reinterpret_cast<uint16_t *>(w)[rb + i] = (uint16_t)sw[i];
        else reinterpret_cast<uint32_t *>(w)[rb + i] = sw[i];
      }
      __syncwarp();
    }
  }
  slots = warp_sum(slots);
  hints = warp_sum(hints);
  if (lane == 0 && slots) atomicAdd(counts, slots);
  if (lane == 0 && hints) atomicAdd(counts + 1, hints);
}

// The window blocks of the bin rows' chunks, slot-major within a chunk: the
// weight of slot t of the i-th hint cell of chunk c (the cell at list
// position boff[2b] + (c - bchunk[b]) kBinChunk + i of its bin b) goes to
// out[(c W + t) kBinChunk + i], so the bin rows read each slot of a chunk as
// consecutive weights.  A thread per (chunk, cell) gathers the cell's block
// and writes its W weights; places past a bucket's last hint cell get 0.
template <typename T>
__global__ void k_blocks_to_chunks(long long nthreads, int W, const int32_t *bchunk, int NB,
                                   const int32_t *cown, const int64_t *boff,
                                   const uint32_t *blist, const T *blk, T *out) {
  const int nchunk = bchunk[NB];
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nthreads;
       q += (long long)gridDim.x * blockDim.x) {
    const long long c = q / kBinChunk;
    if (c >= nchunk) break;
    const int i = (int)(q - c * kBinChunk), b = cown[c];
    const long long k = boff[2 * b] + (long long)(c - bchunk[b]) * kBinChunk + i;
    T *dst = out + (size_t)c * W * kBinChunk + i;
    if (k < boff[2 * b + 1]) {
      const T *src = blk + (size_t)blist[k] * W;
      for (int t = 0; t < W; ++t) dst[(size_t)t * kBinChunk] = src[t];
    } else {
      for (int t = 0; t < W; ++t) dst[(size_t)t * kBinChunk] = (T)0;
    }
  }
}

// Macro rows, in the hub chunks of the sparse-product layout (one CTA per
// chunk of kChunk entries): a macro row lists the cells overlapping it
// (sorted by id), with the weights copied from the cells' own entries, so the
// matrix is exactly symmetric.  Degree partials per chunk.
__global__ void __launch_bounds__(256) k_hub_chunks(
    HintGeo G, int wdtype, int32_t nchunks, const int32_t *chunk_lr, const int32_t *lrow,
    const uint64_t *lptr, const int32_t *lchunk, const int64_t *moff, const uint32_t *mlist,
    const int32_t *n_ovl, const uint64_t *mac_base, int32_t *col, void *w, dfl *cpart) {
  __shared__ dfl red[2][8];
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int l = chunk_lr[c];
    const int64_t v = lrow[l];
    if (v < G.mv0 || v >= G.bn0) continue;  // macro rows only
    const uint64_t base = lptr[l];
    const long long len = (long long)(lptr[l + 1] - base);
    const long long q0 = (long long)(c - lchunk[l]) * kChunk;
    const long long q1 = min(len, q0 + (long long)kChunk);
    const int m = (int)(v - G.mv0);
    dfl D{0.f, 0.f}, Pp{0.f, 0.f};
    for (long long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
      const int i = (int)mlist[moff[m] + q];
      const uint64_t mb = mac_base[i];
      const int n = n_ovl[i];
      int j = 0;
      while (j < n - 1 && col[mb + j] != (int32_t)v) ++j;
      const uint64_t src = mb + j;
      col[base + q] = i;
      copy_w(w, w, wdtype, base + q, src);
      acc_deg(D, Pp, load_w(w, wdtype, src));
    }
    D = warp_sum_df(D);
    Pp = warp_sum_df(Pp);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
      red[0][wid] = D;
      red[1][wid] = Pp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      dfl a = red[0][0], e = red[1][0];
      for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
        df_add_df(a, red[0][k]);
        df_add_df(e, red[1][k]);
      }
      cpart[2 * (long long)c] = df_norm(a);
      cpart[2 * (long long)c + 1] = df_norm(e);
    }
    __syncthreads();
  }
}

// Degrees of virtual rows (warp per row): a macro row from its chunk
// partials, a bin row from the window blocks' degree partials per chunk.
__global__ void k_hub_finalize(HintGeo G, BinGeo B, int32_t nlong, const int32_t *lrow,
                               const int32_t *lchunk, const dfl *cpart, const int32_t *bchunk,
                               const float4 *bdeg,
                               dfl *dsum, dfl *psum) {
  const int lane = threadIdx.x & 31;
  for (long long l = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; l < nlong;
       l += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int64_t v = lrow[l];
    if (v < G.mv0) continue;
    dfl D{0.f, 0.f}, Pp{0.f, 0.f};
    if (v >= G.bn0) {
      bin_row_chunks(B, (int)(v - G.bn0), bchunk, bdeg, &D, &Pp);
    } else {
      for (int c = lchunk[l] + lane; c < lchunk[l + 1]; c += 32) {
        df_add_df(D, cpart[2 * (long long)c]);
        df_add_df(Pp, cpart[2 * (long long)c + 1]);
      }
      D = warp_sum_df(D);
      Pp = warp_sum_df(Pp);
    }
    if (lane == 0) {
      dsum[v] = D;
      psum[v] = Pp;
    }
  }
}

// ------------------------------------------------- H11: lambda_up, c_i
__global__ void k_lambda_max(int64_t N, const dfl *psum, unsigned long long *key) {
  unsigned long long best = 0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    dfl p = psum[v];
    dfl two = df_norm(dfl{__fmul_rn(2.f, p.hi), __fmul_rn(2.f, p.lo)});
    unsigned long long k = df_maxkey(two);
    if (k > best) best = k;
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    unsigned long long o = __shfl_xor_sync(0xffffffffu, best, m);
    best = o > best ? o : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(key, best);
}

// lambda_up and 1 / lambda_up, also copied to status words 4..7 so that the
// host reads them with the status.
__global__ void k_lambda_final(double *lam, const unsigned long long *key, int *status) {
  double l = df_from_maxkey(*key);
  double il = 0.0;
  if (!(l > 0.0) || isinf(l)) {
    flag(status, ST_SPECTRUM);
  } else {
    il = __ddiv_rn(1.0, l);
  }
  lam[0] = l;
  lam[1] = il;
  reinterpret_cast<double *>(status + 4)[0] = l;
  reinterpret_cast<double *>(status + 4)[1] = il;
}

__global__ void k_coef(int64_t N, const dfl *dsum, const double *lam, float *c32) {
  const float il = __double2float_rn(lam[1]);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    dfl d = dsum[v];
    c32[v] = __fadd_rn(1.f, -__fmaf_rn(d.hi, il, __fmul_rn(d.lo, il)));
  }
}

__global__ void k_coef_long(int32_t nlong, const int32_t *lrow, const dfl *dsum,
                            const double *lam, double *c64) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlong; l += gridDim.x * blockDim.x) {
    double d = df_to_d(dsum[lrow[l]]);
    c64[l] = 1.0 - d * lam[1];
  }
}

// --------------------------------------------------------------- driver
template <typename T>
static cudaError_t d2h(T *h, const void *d, size_t n, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(h, d, n * sizeof(T), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

static HintGeo make_geo(const pl_graph *g) {
  HintGeo G;
  G.xlf = (float)g->xl;
  G.ylf = (float)g->yl;
  G.sxf = (float)((double)g->nbx / (g->xh - g->xl));
  G.syf = (float)((double)g->nby / (g->yh - g->yl));
  G.gxf = (float)g->xl;
  G.gyf = (float)g->yl;
  G.gsxf = (float)g->gsx;
  G.gsyf = (float)g->gsy;
  G.xl = g->xl;
  G.yl = g->yl;
  G.wb = g->wb;
  G.hb = g->hb;
  G.iwb2 = 2.0 / g->wb;
  G.ihb2 = 2.0 / g->hb;
  auto split = [](double d, float *h, float *l) {
    *h = (float)d;
    *l = (float)(d - (double)*h);
  };
  split(G.xl, &G.xlh, &G.xll);
  split(G.yl, &G.ylh, &G.yll);
  split(G.iwb2, &G.iwh, &G.iwl);
  split(G.ihb2, &G.ihh, &G.ihl);
  G.nbx = g->nbx;
  G.nby = g->nby;
  G.hx = g->hx;
  G.hy = g->hy;
  G.gnx = g->gnx;
  G.gny = g->gny;
  G.C = g->C;
  G.Pm = g->Pm;
  G.S = g->S;
  G.Mm = g->Mm;
  G.Nst = g->Nst;
  G.mv0 = g->Nst;
  G.bn0 = g->Nst + g->Mm;
  G.N = g->N;
  return G;
}

static BinGeo make_bingeo(const pl_graph *g) {
  BinGeo B;
  B.nbx = g->nbx;
  B.nby = g->nby;
  B.hx = g->hx;
  B.hy = g->hy;
  B.W = (2 * g->hx + 1) * (2 * g->hy + 1);
  B.NB = g->NB;
  return B;
}

// Layout of a split matrix from per-row lengths already in g->slen/llen/lflag.
// Layout of a split matrix from per-row lengths in g->slen/llen/clen and
// hub flags in g->hubf.
static pl_status layout(pl_graph *g, SpMat &m, int with_hints, cudaStream_t s) {
  const int64_t N = g->N;
  m.N = N;
  void *stmp;
  TRY(ensure(g->tmp[7], scan_tmp_bytes(N + 1) + 4096));
  stmp = g->tmp[7].p;
  TRY(ensure(g->lay[0], (size_t)(N + 1) * 8 + 256));
  uint64_t *s64 = P<uint64_t>(g->lay[0]);
  TRY((exclusive_scan<uint32_t, uint64_t>(P<uint32_t>(g->slen), s64, N, stmp, s)));
  TRY(ensure(g->lay[1], (size_t)(N + 1) * 8 + 256));
  uint64_t *lpos = P<uint64_t>(g->lay[1]);
  TRY((exclusive_scan<uint64_t, uint64_t>(P<uint64_t>(g->llen), lpos, N, stmp, s)));
  TRY(ensure(g->lflag, (size_t)(N + 1) * 4 + 256));
  int32_t *lscan = P<int32_t>(g->lflag);
  TRY((exclusive_scan<uint8_t, int32_t>(P<uint8_t>(g->hubf), lscan, N, stmp, s)));
  uint64_t tot[2];
  int32_t nl;
  {
    const D2H it[3] = {{&tot[0], s64 + N, 8}, {&tot[1], lpos + N, 8}, {&nl, lscan + N, 4}};
    TRY(d2h_many(g->stage, it, 3, s));
  }
  if (tot[0] + kPad >= (uint64_t)kOffMask || tot[0] + tot[1] >= (1ull << 40)) {
    set_error("graph too large for the 31-bit short-row layout (%llu entries)",
              (unsigned long long)tot[0]);
    return PL_ERR_UNSUPPORTED;
  }
  m.nnz_s = tot[0];
  m.nnz_l = tot[1];
  m.nlong = nl;
  m.wbytes = g->wdtype == PL_W_BF16 ? 2 : 4;
  TRY(ensure(m.rp_s, (size_t)(N + 1 + kRpPad) * 4));
  k_rp_pack<<<grid_for(N + 1 + kRpPad, 256), 256, 0, s>>>(s64, P<uint8_t>(g->hubf), N,
                                                         P<uint32_t>(m.rp_s));
  note_launch();
  const uint64_t cap = m.nnz_s + m.nnz_l + kPad;
  TRY(ensure(m.col, cap * 4));
  TRY(ensure(m.w, cap * m.wbytes));
  TRY(ensure(m.lrow, (size_t)nl * 4 + 16));
  TRY(ensure(m.lptr, (size_t)(nl + 1) * 8));
  TRY(ensure(m.lsb, (size_t)nl * 8 + 16));
  TRY(ensure(m.lhb, (size_t)nl * 8 + 16));
  TRY(ensure(m.lsl, (size_t)nl * 4 + 16));
  TRY(ensure(m.lhl, (size_t)nl * 4 + 16));
  TRY(ensure(m.longidx, (size_t)N * 4 + 16));
  TRY(ensure(m.lchunk, (size_t)(nl + 1) * 4));
  TRY(ensure(g->lay[3], (size_t)(nl + 1) * 4 + 256));
  int32_t *nch = P<int32_t>(g->lay[3]);
  k_layout_long<<<grid_for(N, 256), 256, 0, s>>>(N, P<uint8_t>(g->hubf), lscan, lpos,
                                                 P<uint64_t>(g->clen), m.nnz_s,
                                                 P<int32_t>(m.lrow), P<uint64_t>(m.lptr),
                                                 P<int32_t>(m.longidx), nch);
  note_launch();
  if (nl == 0) {
    TRY(cudaMemsetAsync(m.lchunk.p, 0, 4, s));
    m.nchunks = 0;
  } else {
    TRY((exclusive_scan<int32_t, int32_t>(nch, P<int32_t>(m.lchunk), nl, stmp, s)));
    int32_t nc;
    TRY(d2h(&nc, P<int32_t>(m.lchunk) + nl, 1, s));
    m.nchunks = nc;
    k_hub_desc<<<grid_for(nl, 256), 256, 0, s>>>(
        nl, with_hints, P<int32_t>(m.lrow), P<uint64_t>(m.lptr), P<int64_t>(g->srp), g->Nst,
        P<uint32_t>(g->st.rp_s), P<int32_t>(g->st.longidx), P<uint64_t>(g->st.lptr),
        P<uint64_t>(m.lsb), P<uint32_t>(m.lsl), P<uint64_t>(m.lhb), P<uint32_t>(m.lhl));
    note_launch();
  }
  TRY(ensure(m.chunk_lr, (size_t)m.nchunks * 4 + 16));
  if (nl) {
    k_chunk_owner<<<grid_for(nl, 256), 256, 0, s>>>(nl, P<int32_t>(m.lchunk), P<int32_t>(m.chunk_lr));
    note_launch();
  }
  TRY(ensure(m.dsum, (size_t)N * 8 + 16));
  TRY(ensure(m.psum, (size_t)N * 8 + 16));
  TRY(ensure(m.c32, (size_t)N * 4 + 16));
  TRY(ensure(m.c64l, (size_t)nl * 8 + 16));
  TRY(ensure(m.lam, 64));
  size_t pbytes = (size_t)(m.nchunks + 1) * 6 * 8;
  TRY(ensure(m.part, pbytes));
  TRY(cudaMemsetAsync(P<char>(m.col) + (m.nnz_s + m.nnz_l) * 4, 0, kPad * 4, s));
  TRY(cudaMemsetAsync(P<char>(m.w) + (m.nnz_s + m.nnz_l) * m.wbytes, 0, kPad * m.wbytes, s));
  return PL_OK;
}

static pl_status ensure_row_arrays(pl_graph *g) {
  const int64_t N = g->N;
  TRY(ensure(g->slen, (size_t)N * 4 + 16));
  TRY(ensure(g->llen, (size_t)N * 8 + 16));
  TRY(ensure(g->clen, (size_t)N * 8 + 16));
  TRY(ensure(g->hubf, (size_t)N + 256));
  return PL_OK;
}

// Layout of the static split matrix from the static row pointers; the
// entries and degree sums are written by the static compaction.
pl_status prepare_static_layout(pl_graph *g, cudaStream_t s) {
  const int64_t N = g->N;
  HintGeo G{};
  G.N = N;
  G.Nst = g->Nst;
  pl_status st = ensure_row_arrays(g);
  if (st != PL_OK) return st;
  k_row_len<<<grid_for(N, 256), 256, 0, s>>>(G, 0, P<int64_t>(g->srp), nullptr, nullptr, nullptr,
                                             nullptr, P<uint32_t>(g->slen),
                                             P<uint64_t>(g->llen), P<uint8_t>(g->hubf),
                                             P<uint64_t>(g->clen));
  note_launch();
  return layout(g, g->st, 0, s);
}

pl_status build_hints(pl_graph *g, const pl_params *p, const float *xy_in, cudaStream_t s) {
  const int64_t N = g->N;
  const int32_t C = g->C, NB = g->NB, Mm = g->Mm;
  const float2 *xy = reinterpret_cast<const float2 *>(xy_in);
  HintGeo G = make_geo(g);
  g->have_hints = false;
  // a hint build takes its buffers anew, above the static build's part of
  // the workspace
  for_each_buf(g, 1, [](Buf &b) { release(b); });
  g->arena.used = g->hint_mark;
  if (g->hx * 2 + 1 > kMaxWin || g->hy * 2 + 1 > kMaxWin) {
    set_error("detection window larger than 31 x 31 bins");
    return PL_ERR_UNSUPPORTED;
  }
  TRY(cudaMemsetAsync(g->status.p, 0, 32, s));
  int *status = P<int>(g->status);
  void *stmp;
  TRY(ensure(g->tmp[7], scan_tmp_bytes(N + 1) + 4096));
  stmp = g->tmp[7].p;

  // H1: bins and macro overlaps of movable cells (bucket counts by atomics
  // only when the buckets do not fit the tiled counting sort)
  const int nbk = 2 * NB;
  const bool tiled = nbk <= kMaxSmemBuckets;
  TRY(ensure(g->cell_bin, (size_t)C * 4 + 16));
  TRY(ensure(g->n_ovl, (size_t)C * 4 + 16));
  TRY(ensure(g->bcnt, (size_t)(nbk + 1) * 4));
  TRY(ensure(g->mcnt, (size_t)(Mm + 1) * 4));
  if (!tiled) TRY(cudaMemsetAsync(g->bcnt.p, 0, (size_t)(nbk + 1) * 4, s));
  const int ntile = (int)((C + kBinTile - 1) / kBinTile) > 0 ? (int)((C + kBinTile - 1) / kBinTile) : 1;
  // macro lists by a tiled counting sort when the macros' run counters fit
  // shared memory (else: scatter by atomics, then a segmented sort)
  const bool tiledm = Mm > 0 && Mm <= kMaxSmemMacros;
  const long long nmt = (long long)Mm * ntile;
  if (tiledm) {
    TRY(ensure(g->mtc, (size_t)nmt * 4 + 16));
    TRY(ensure(g->cmem, (size_t)C * kMacroSlots * 4 + 16));
    TRY(cudaMemsetAsync(g->mtc.p, 0, (size_t)nmt * 4, s));
  } else {
    TRY(cudaMemsetAsync(g->mcnt.p, 0, (size_t)(Mm + 1) * 4, s));
  }
  k_hint_cells<<<grid_for(C, 256), 256, 0, s>>>(
      G, xy, P<uint8_t>(g->ckind), P<uint8_t>(g->hflag), P<float>(g->cw), P<float>(g->ch),
      P<int64_t>(g->gptr), P<uint32_t>(g->glist), P<float4>(g->ggeo), P<int32_t>(g->cell_bin),
      P<int32_t>(g->n_ovl), tiled ? nullptr : P<int32_t>(g->bcnt), P<int32_t>(g->mcnt),
      tiledm ? P<int32_t>(g->mtc) : nullptr, ntile, tiledm ? P<int32_t>(g->cmem) : nullptr,
      status);
  note_launch();
  // H2: bucket offsets
  TRY(ensure(g->boff, (size_t)(nbk + 1) * 8));
  TRY(ensure(g->moff, (size_t)(Mm + 1) * 8));
  if (tiledm) {
    TRY(ensure(g->mtoff, (size_t)(nmt + 1) * 8 + 256));
    TRY(ensure(g->tmp[7], scan_tmp_bytes(nmt + 1) + 4096));
    stmp = g->tmp[7].p;
    TRY((exclusive_scan<int32_t, int64_t>(P<int32_t>(g->mtc), P<int64_t>(g->mtoff), nmt, stmp, s)));
    k_bucket_starts<<<grid_for(Mm + 1, 256), 256, 0, s>>>(Mm, ntile, P<int64_t>(g->mtoff),
                                                         P<int64_t>(g->moff));
    note_launch();
  } else {
    TRY((exclusive_scan<int32_t, int64_t>(P<int32_t>(g->mcnt), P<int64_t>(g->moff), Mm, stmp, s)));
  }
  int32_t *cm = nullptr;
  int64_t *cmo = nullptr;
  if (tiled) {
    const long long ncm = (long long)nbk * ntile;
    TRY(ensure(g->tmp[5], (size_t)ncm * 4 + 256));
    TRY(ensure(g->tmp[6], (size_t)(ncm + 1) * 8 + 256));
    TRY(ensure(g->tmp[7], scan_tmp_bytes(ncm + 1) + 4096));
    stmp = g->tmp[7].p;
    cm = P<int32_t>(g->tmp[5]);
    cmo = P<int64_t>(g->tmp[6]);
    k_bin_tile_count<<<ntile, 256, (size_t)nbk * 4, s>>>(C, nbk, ntile, P<uint8_t>(g->ckind),
                                                        P<uint8_t>(g->hflag),
                                                        P<int32_t>(g->cell_bin), cm);
    note_launch();
    TRY((exclusive_scan<int32_t, int64_t>(cm, cmo, ncm, stmp, s)));
    k_bucket_starts<<<grid_for(nbk + 1, 256), 256, 0, s>>>(nbk, ntile, cmo, P<int64_t>(g->boff));
    note_launch();
  } else {
    TRY((exclusive_scan<int32_t, int64_t>(P<int32_t>(g->bcnt), P<int64_t>(g->boff), nbk, stmp, s)));
  }
  int hst[8];
  int64_t nbl, nml;
  {
    const D2H it[3] = {{hst, g->status.p, 32}, {&nbl, P<int64_t>(g->boff) + nbk, 8},
                       {&nml, P<int64_t>(g->moff) + Mm, 8}};
    TRY(d2h_many(g->stage, it, 3, s));
  }
  if (hst[0] & ST_NONFINITE) {
    set_error("non-finite movable cell coordinate");
    return PL_ERR_NONFINITE;
  }
  if (nml > (int64_t)g->nmov * kMaxCellMacros) {
    set_error("%lld macro-cell overlaps, more than %d per movable cell", (long long)nml,
              kMaxCellMacros);
    return PL_ERR_UNSUPPORTED;
  }
  // H3-H4: bin buckets (ascending cell id) and macro lists (sorted)
  TRY(ensure(g->blist, (size_t)nbl * 4 + 16));
  TRY(ensure(g->mlist, (size_t)nml * 4 + 16));
  if (tiled) {
    if ((size_t)nbk * 20 <= 48 * 1024)
      k_bin_tile_scatter_wc<<<ntile, 256, (size_t)nbk * 20, s>>>(
          C, nbk, ntile, P<uint8_t>(g->ckind), P<uint8_t>(g->hflag), P<int32_t>(g->cell_bin), cmo,
          P<uint32_t>(g->blist));
    else
      k_bin_tile_scatter<<<ntile, 256, (size_t)nbk * 4, s>>>(C, nbk, ntile, P<uint8_t>(g->ckind),
                                                            P<uint8_t>(g->hflag),
                                                            P<int32_t>(g->cell_bin), cmo,
                                                            P<uint32_t>(g->blist));
    note_launch();
  } else {
    TRY(ensure(g->bcur, (size_t)(nbk + 1) * 4));
    k_u64_to_u32<<<grid_for(nbk, 256), 256, 0, s>>>(P<uint64_t>(g->boff), P<uint32_t>(g->bcur), nbk);
    note_launch();
    k_bin_scatter_atomic<<<grid_for(C, 256), 256, 0, s>>>(C, P<uint8_t>(g->ckind), P<uint8_t>(g->hflag),
                                                          P<int32_t>(g->cell_bin),
                                                          P<int32_t>(g->bcur), P<uint32_t>(g->blist));
    note_launch();
    TRY(ensure(g->tmp[3], segsort_tmp_bytes(nbk, nbl, 4)));
    TRY((segmented_sort<uint32_t, MODE_SORT>(P<uint32_t>(g->blist), P<int64_t>(g->boff), nbk,
                                             nbl, nullptr, nullptr, nullptr, g->tmp[3].p, s)));
  }
  const bool cmem_ok = tiledm && !(hst[0] & ST_MANY_OVL);  // every hint cell's macros recorded
  if (!cmem_ok && Mm) {
    TRY(ensure(g->mcur, (size_t)(Mm + 1) * 4));
    k_u64_to_u32<<<grid_for(Mm, 256), 256, 0, s>>>(P<uint64_t>(g->moff), P<uint32_t>(g->mcur), Mm);
    note_launch();
    k_macro_scatter<<<grid_for(C, 256), 256, 0, s>>>(
        G, xy, P<uint8_t>(g->ckind), P<uint8_t>(g->hflag), P<float>(g->cw), P<float>(g->ch),
        P<int64_t>(g->gptr), P<uint32_t>(g->glist), P<float4>(g->ggeo), P<int32_t>(g->mcur),
        P<uint32_t>(g->mlist));
    note_launch();
    TRY(ensure(g->tmp[3], segsort_tmp_bytes(Mm, nml, 4)));
    TRY((segmented_sort<uint32_t, MODE_SORT>(P<uint32_t>(g->mlist), P<int64_t>(g->moff), Mm, nml,
                                             nullptr, nullptr, nullptr, g->tmp[3].p, s)));
  }
  // H5: densities and phi on the side stream, the tiled macro lists on a
  // third one, while the row lengths and the layout go on (both joined
  // before the assembly)
  TRY(ensure_side2(g));
  cudaStream_t s2 = g->side, s3 = g->side2;
  TRY(ensure(g->Db, (size_t)NB * 8 + 16));
  TRY(ensure(g->phi, (size_t)NB * 8 + 16));
  TRY(ensure(g->tmp[4], (size_t)NB * 4 + 256));
  float *phif = P<float>(g->tmp[4]);
  TRY(cudaEventRecord(g->ev_fork, s));
  TRY(cudaStreamWaitEvent(s2, g->ev_fork, 0));
  TRY(cudaStreamWaitEvent(s3, g->ev_fork, 0));
  if (cmem_ok) {
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
      cudaFuncSetAttribute(k_macro_tile_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kMaxSmemMacros * 6);
    });
    k_macro_tile_scatter<<<ntile, 256, (size_t)Mm * 6, s3>>>(C, P<int32_t>(g->n_ovl),
                                                            P<int32_t>(g->cmem), Mm, ntile,
                                                            P<int64_t>(g->mtoff),
                                                            P<uint32_t>(g->mlist));
    note_launch();
  }
  LevelBufs lv;
  int nlev = 0;  // launches: level L exists while 64^(L+1) < the longest bin
  {
    size_t sizes[kMaxLevels], tot = 0;
    size_t prev = (size_t)nbl;
    for (int k = 0; k < kMaxLevels; ++k) {
      sizes[k] = prev / 64 + (size_t)NB + 2;
      tot += sizes[k];
      prev = sizes[k];
    }
    TRY(ensure(g->hubtmp, tot * 8 + 256));
    double *q = P<double>(g->hubtmp);
    for (int k = 0; k < kMaxLevels; ++k) {
      lv.base[k] = q;
      q += sizes[k];
    }
    double span = 64.0;
    while (nlev < kMaxLevels && (double)nbl > span) {
      ++nlev;
      span *= 64.0;
    }
    for (int L = 0; L < nlev; ++L) {
      // blocks of 64 threads, so that the first level's FP64 sums spread over every SM
      k_dens_level<<<grid_for((long long)sizes[L], 64, 152 * 64), 64, 0, s2>>>(
          NB, L, P<int64_t>(g->boff), P<uint32_t>(g->blist), P<double>(g->carea),
          L ? lv.base[L - 1] : nullptr, lv.base[L], (long long)sizes[L]);
      note_launch();
    }
  }
  k_dens_final<<<grid_for(NB, 32), 32, 0, s2>>>(  // a warp per 32 bins: spread over the SMs
      G, nlev, P<int64_t>(g->boff), P<uint32_t>(g->blist), P<double>(g->carea), lv,
      P<double>(g->amac), g->abin, p->capacity, p->mu, P<double>(g->Db), P<double>(g->Cb),
      P<double>(g->phi), phif);
  note_launch();
  TRY(cudaEventRecord(g->ev_join, s2));
  TRY(cudaEventRecord(g->ev_join2, s3));
  // H6-H7: row lengths and layout
  pl_status st = ensure_row_arrays(g);
  if (st != PL_OK) return st;
  k_row_len<<<grid_for(N, 256), 256, 0, s>>>(G, 1, P<int64_t>(g->srp), P<uint8_t>(g->hflag),
                                             P<int32_t>(g->cell_bin), P<int32_t>(g->n_ovl),
                                             P<int64_t>(g->moff), P<uint32_t>(g->slen),
                                             P<uint64_t>(g->llen), P<uint8_t>(g->hubf),
                                             P<uint64_t>(g->clen));
  note_launch();
  st = layout(g, g->hm, 1, s);
  if (st != PL_OK) return st;
  SpMat &m = g->hm;
  // H9: hint parts of cells (macro entries, window blocks) and degrees of
  // every real node
  TRY(ensure(g->mac_base, (size_t)C * 8 + 16));
  const int W = (2 * g->hx + 1) * (2 * g->hy + 1);
  g->W = W;
  TRY(ensure(g->hbw, (size_t)C * W * m.wbytes + 64));
  TRY(ensure(g->hbin, (size_t)C * 4 + 16));
  unsigned long long *counts = reinterpret_cast<unsigned long long *>(P<double>(m.lam) + 3);
  TRY(cudaMemsetAsync(counts, 0, 16, s));
  TRY(cudaStreamWaitEvent(s, g->ev_join, 0));   // phi
  TRY(cudaStreamWaitEvent(s, g->ev_join2, 0));  // the macro lists
  k_assemble_hints<<<grid_for(g->Nst, 256), 256, 0, s>>>(
      G, g->wdtype, P<uint32_t>(m.rp_s), P<int32_t>(m.longidx), P<uint64_t>(m.lptr),
      P<dfl>(g->st.dsum), P<dfl>(g->st.psum), P<uint8_t>(g->hflag), P<int32_t>(g->cell_bin),
      P<int32_t>(g->n_ovl), xy, P<float>(g->cw), P<float>(g->ch), P<int64_t>(g->gptr),
      P<uint32_t>(g->glist), P<float4>(g->ggeo), P<double>(g->base_w), phif, P<double>(g->phi),
      W, cmem_ok ? P<int32_t>(g->cmem) : nullptr, P<float4>(g->mgeo), P<int32_t>(m.col), m.w.p,
      g->hbw.p, P<int32_t>(g->hbin), P<dfl>(m.dsum), P<dfl>(m.psum), P<uint64_t>(g->mac_base),
      counts);
  note_launch();
  // H10: bin rows (degree partials of the window blocks, chunk by chunk) and
  // macro rows (their entries and degree partials)
  const BinGeo B = make_bingeo(g);
  TRY(ensure(g->bchunk, (size_t)(NB + 1) * 4 + 256));
  TRY(ensure(g->tmp[6], (size_t)(NB + 1) * 4 + 256));
  k_bin_chunk_count<<<grid_for(NB, 256), 256, 0, s>>>(NB, P<int64_t>(g->boff), P<int32_t>(g->tmp[6]));
  note_launch();
  TRY((exclusive_scan<int32_t, int32_t>(P<int32_t>(g->tmp[6]), P<int32_t>(g->bchunk), NB, stmp, s)));
  const long long nbc_max = nbl / kBinChunk + NB + 1;  // chunks at most (the grid size)
  g->nbc_max = nbc_max;
  TRY(ensure(g->cown, (size_t)nbc_max * 4 + 256));
  k_chunk_bins<<<grid_for(nbc_max, 256), 256, 0, s>>>(NB, nbc_max, P<int32_t>(g->bchunk), P<int32_t>(g->cown));
  note_launch();
  // the chunks' copy of the window blocks (read slot by slot by the bin rows)
  TRY(ensure(g->hbwq, (size_t)nbc_max * kBinChunk * W * m.wbytes + 64));
  {
    const long long nth = nbc_max * kBinChunk;
    if (g->wdtype == PL_W_BF16)
      k_blocks_to_chunks<uint16_t><<<grid_for(nth, 256), 256, 0, s>>>(
          nth, W, P<int32_t>(g->bchunk), NB, P<int32_t>(g->cown), P<int64_t>(g->boff),
          P<uint32_t>(g->blist), P<uint16_t>(g->hbw), P<uint16_t>(g->hbwq));
    else
      k_blocks_to_chunks<uint32_t><<<grid_for(nth, 256), 256, 0, s>>>(
          nth, W, P<int32_t>(g->bchunk), NB, P<int32_t>(g->cown), P<int64_t>(g->boff),
          P<uint32_t>(g->blist), P<uint32_t>(g->hbw), P<uint32_t>(g->hbwq));
    note_launch();
  }
  TRY(ensure(g->bdeg, (size_t)nbc_max * W * 16 + 256));
  TRY(ensure(g->bpart, (size_t)nbc_max * W * 16 + 256));
  const long long bwant = (nbc_max + kBinThreads / 32 - 1) / (kBinThreads / 32);
  const int bgrid = (int)(bwant < 152 * 16 ? bwant : 152 * 16);
  TRY(launch_bin_partials<true>(g->wdtype, bgrid, s, B, P<int32_t>(g->bchunk), P<int32_t>(g->cown),
                                 P<int64_t>(g->boff), P<uint32_t>(g->blist), g->hbwq.p, nullptr,
                                 P<float4>(g->bdeg)));
  note_launch();
  TRY(ensure(g->tmp[5], (size_t)(m.nchunks + 1) * 2 * sizeof(dfl) + 256));
  dfl *cpart = P<dfl>(g->tmp[5]);
  if (m.nchunks) {
    k_hub_chunks<<<m.nchunks < 152 * 32 ? m.nchunks : 152 * 32, 256, 0, s>>>(
        G, g->wdtype, m.nchunks, P<int32_t>(m.chunk_lr), P<int32_t>(m.lrow), P<uint64_t>(m.lptr),
        P<int32_t>(m.lchunk), P<int64_t>(g->moff), P<uint32_t>(g->mlist), P<int32_t>(g->n_ovl),
        P<uint64_t>(g->mac_base), P<int32_t>(m.col), m.w.p, cpart);
    note_launch();
    k_hub_finalize<<<grid_for((long long)m.nlong * 32, 256), 256, 0, s>>>(
        G, B, m.nlong, P<int32_t>(m.lrow), P<int32_t>(m.lchunk), cpart, P<int32_t>(g->bchunk),
        P<float4>(g->bdeg),
        P<dfl>(m.dsum), P<dfl>(m.psum));
    note_launch();
  }
  // H11: lambda_up and coefficients
  unsigned long long *key = reinterpret_cast<unsigned long long *>(P<double>(m.lam) + 2);
  TRY(cudaMemsetAsync(key, 0, 8, s));
  k_lambda_max<<<grid_for(N, 256, 152 * 8), 256, 0, s>>>(N, P<dfl>(m.psum), key);
  note_launch();
  k_lambda_final<<<1, 1, 0, s>>>(P<double>(m.lam), key, status);
  note_launch();
  k_coef<<<grid_for(N, 256), 256, 0, s>>>(N, P<dfl>(m.dsum), P<double>(m.lam), P<float>(m.c32));
  note_launch();
  if (m.nlong) {
    k_coef_long<<<grid_for(m.nlong, 256), 256, 0, s>>>(m.nlong, P<int32_t>(m.lrow), P<dfl>(m.dsum),
                                                        P<double>(m.lam), P<double>(m.c64l));
    note_launch();
  }
  TRY(cudaGetLastError());
  {
    unsigned long long ns[2] = {0, 0};
    const D2H it[2] = {{hst, g->status.p, 32}, {ns, counts, 16}};
    TRY(d2h_many(g->stage, it, 2, s));
    g->nslot = (int64_t)ns[0];
    g->nhint = (int64_t)ns[1];
  }
  memcpy(g->lam_h, hst + 4, sizeof(g->lam_h));
  g->have_hints = true;
  if (hst[0] & ST_SPECTRUM) {
    set_error("lambda_up <= 0 or not finite: the refinement filter is undefined");
    return PL_ERR_SPECTRUM;
  }
  return PL_OK;
}

}  // namespace pl
