// Device helpers and device-wide primitives shared by the libpl kernels.
// Nothing here is shared with any other implementation; the arithmetic each helper implements is
// stated at the helper.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>

namespace pl {

constexpr int kWarp = 32;

// ------------------------------------------------------------------ errors
enum : int { ST_BAD_INDEX = 1, ST_NONFINITE = 2, ST_SPECTRUM = 4, ST_TOO_BIG = 8, ST_BAD_NET = 16,
             ST_BAD_CELL = 32, ST_TIMEOUT = 64, ST_MANY_OVL = 128,
             ST_LEARNED_NF = 256 /* a free node's learned g~ is not finite */ };

__device__ __forceinline__ void flag(int *status, int bit) { atomicOr(status, bit); }

// ------------------------------------------------------------ FP64 helpers
// exp(x): Cody & Waite reduction x = n ln2 + r with ln2 split into a head of
// 32 significant bits (n * head exact) and a tail, the degree-13 Taylor
// polynomial of e^r in Horner form, then scaling by 2^n.  Every operation is
// an explicitly rounded IEEE double operation (no contraction), so the result
// is a fixed function of x.  Used for the bin logistic phi_b.
__device__ __forceinline__ double pow2_d(int k) {  // 2^k for -1022 <= k <= 1023
  return __longlong_as_double((long long)(k + 1023) << 52);
}
__device__ inline double exp_cw(double x) {
  const double inv_ln2 = 0x1.71547652b82fep+0;
  const double ln2_hi = 0x1.62e42fee00000p-1;
  const double ln2_lo = 0x1.a39ef35793c76p-33;
  if (x != x) return x;
  if (x > 709.78) return __longlong_as_double(0x7ff0000000000000LL);
  if (x < -745.2) return 0.0;
  double n = floor(__dadd_rn(__dmul_rn(x, inv_ln2), 0.5));
  double r = __dadd_rn(__dadd_rn(x, -__dmul_rn(n, ln2_hi)), -__dmul_rn(n, ln2_lo));
  const double c[14] = {0x1.6124613a86d09p-33, 0x1.1eed8eff8d898p-29, 0x1.ae64567f544e4p-26,
                        0x1.27e4fb7789f5cp-22, 0x1.71de3a556c734p-19, 0x1.a01a01a01a01ap-16,
                        0x1.a01a01a01a01ap-13, 0x1.6c16c16c16c17p-10, 0x1.1111111111111p-7,
                        0x1.5555555555555p-5,  0x1.5555555555555p-3,  0x1.0000000000000p-1,
                        1.0, 1.0};
  double p = c[0];
#pragma unroll
  for (int j = 1; j < 14; ++j) p = __dadd_rn(__dmul_rn(p, r), c[j]);
  int ni = (int)n;
  if (ni < -1020) return __dmul_rn(__dmul_rn(p, pow2_d(ni + 1020)), pow2_d(-1020));
  if (ni > 1023) return __dmul_rn(__dmul_rn(p, pow2_d(1023)), pow2_d(ni - 1023));
  return __dmul_rn(p, pow2_d(ni));
}

// Round a double to bfloat16 (8 significant bits, FP32 exponent range,
// subnormal quantum 2^-133) to nearest, ties to even, directly from the double
// bits.  Returns the 16-bit pattern.
__device__ __forceinline__ uint16_t d2bf16(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  uint16_t sign = (uint16_t)((b >> 48) & 0x8000u);
  unsigned long long a = b & 0x7fffffffffffffffULL;
  if (a == 0) return sign;
  if (a > 0x7ff0000000000000ULL) return (uint16_t)(sign | 0x7fc0u);
  if (a == 0x7ff0000000000000ULL) return (uint16_t)(sign | 0x7f80u);
  int e = (int)(a >> 52);
  if (e == 0) return sign;  // |d| < 2^-1022: far below half the bf16 quantum
  int E = e - 1023;
  unsigned long long m = a & 0x000fffffffffffffULL;
  if (E >= -126) {  // normal bf16
    unsigned long long keep = m >> 45, rem = m & ((1ULL << 45) - 1), half = 1ULL << 44;
    if (rem > half || (rem == half && (keep & 1))) ++keep;
    if (keep == 128) { keep = 0; ++E; }
    if (E > 127) return (uint16_t)(sign | 0x7f80u);
    return (uint16_t)(sign | (uint16_t)((E + 127) << 7) | (uint16_t)keep);
  }
  // subnormal bf16: q = round(full * 2^(E - 52 + 133))
  unsigned long long full = m | (1ULL << 52);
  int s = -81 - E;  // right shift, >= 47 here
  if (s > 54) return sign;
  unsigned long long q = full >> s, rem = full & ((1ULL << s) - 1), half = 1ULL << (s - 1);
  if (rem > half || (rem == half && (q & 1))) ++q;
  return (uint16_t)(sign | (uint16_t)q);
}
__device__ __forceinline__ float bf16_to_f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
// Nearest-even bf16 of a float.
__device__ __forceinline__ uint16_t f2bf16(float f) {
  uint32_t u = __float_as_uint(f);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
  uint32_t lsb = (u >> 16) & 1u;
  return (uint16_t)((u + 0x7fffu + lsb) >> 16);
}

// splitmix64 (Steele, Lea & Flood 2014) at counter ctr of stream `seed`; the
// top 53 bits mapped to [0, 1).
__device__ __forceinline__ double u01(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return __dmul_rn((double)(z >> 11), 0x1.0p-53);
}

// --------------------------------------------------------- double-float
// Unevaluated sums hi + lo of two floats (about 48 significant bits) with
// Knuth's TwoSum and an FMA-based exact product; all operations explicitly
// rounded so the compiler cannot contract them.
struct dfl {
  float hi, lo;
};
__device__ __forceinline__ void df_add(dfl &s, float a) {
  float t = __fadd_rn(s.hi, a);
  float bp = __fadd_rn(t, -s.hi);
  float e = __fadd_rn(__fadd_rn(s.hi, -__fadd_rn(t, -bp)), __fadd_rn(a, -bp));
  s.hi = t;
  s.lo = __fadd_rn(s.lo, e);
}
__device__ __forceinline__ void df_add_prod(dfl &s, float w, float x) {
  float ph = __fmul_rn(w, x);
  float pl = __fmaf_rn(w, x, -ph);
  df_add(s, ph);
  s.lo = __fadd_rn(s.lo, pl);
}
__device__ __forceinline__ void df_add_df(dfl &s, dfl b) {
  df_add(s, b.hi);
  s.lo = __fadd_rn(s.lo, b.lo);
}
__device__ __forceinline__ dfl df_norm(dfl s) {
  float t = __fadd_rn(s.hi, s.lo);
  float e = __fadd_rn(s.lo, -__fadd_rn(t, -s.hi));
  return dfl{t, e};
}
__device__ __forceinline__ double df_to_d(dfl s) { return __dadd_rn((double)s.hi, (double)s.lo); }
__device__ __forceinline__ dfl df_shfl_xor(dfl s, int m) {
  return dfl{__shfl_xor_sync(0xffffffffu, s.hi, m), __shfl_xor_sync(0xffffffffu, s.lo, m)};
}
__device__ __forceinline__ dfl warp_sum_df(dfl s) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) df_add_df(s, df_shfl_xor(s, m));
  return df_norm(s);
}

// Reduce-scatter of the N double-floats v over the warp (level M = 16, 8, ...,
// 1): at each level a lane keeps one half of its values (the upper half when
// its bit M is set), sends the other half to lane ^ M and adds what it
// receives, the lower lane's partial first.  On return exactly one lane holds
// the warp sum of value j, in v[0], with pos = j and cnt = 1; the others have
// cnt = 0.  Every sum follows the tree of warp_sum_df's lane 0 (the group of
// lanes with the bit clear plus the group with it set, level by level), so
// before df_norm it is bit-identical to it, for far fewer shuffles and adds
// when N is large.  Call with pos = 0, cnt = N.
template <int N, int M>
__device__ __forceinline__ void warp_rs_df(dfl *v, int &pos, int &cnt) {
  constexpr int H = (N + 1) / 2;
  const bool hi = (threadIdx.x & M) != 0;
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const dfl a = v[i];
    const dfl b = i + H < N ? v[i + H] : dfl{0.f, 0.f};
    const dfl r = df_shfl_xor(hi ? a : b, M);
    dfl s = hi ? r : a;
    df_add_df(s, hi ? b : r);
    v[i] = s;
  }
  if (hi) {
    pos += H;
    cnt = cnt > H ? cnt - H : 0;
  } else {
    cnt = cnt < H ? cnt : H;
  }
  if constexpr (M > 1) warp_rs_df<H, M / 2>(v, pos, cnt);
}

// Monotone 64-bit key of a non-negative double-float value (hi >= 0), for
// atomicMax: hi's bits above lo's order-preserving bits.
__device__ __forceinline__ unsigned long long df_maxkey(dfl s) {
  uint32_t lo = __float_as_uint(s.lo);
  lo = (lo & 0x80000000u) ? ~lo : (lo | 0x80000000u);
  return ((unsigned long long)__float_as_uint(s.hi) << 32) | lo;
}
__host__ __device__ inline double df_from_maxkey(unsigned long long k) {
  uint32_t hi = (uint32_t)(k >> 32), lo = (uint32_t)k;
  lo = (lo & 0x80000000u) ? (lo & 0x7fffffffu) : ~lo;
  float fh, fl;
  memcpy(&fh, &hi, 4);
  memcpy(&fl, &lo, 4);
  return (double)fh + (double)fl;
}

// ------------------------------------------------------------ warp helpers
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// Ascending bitonic sort of one key per lane across a warp.
template <typename K>
__device__ __forceinline__ K warp_bitonic(K key, int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      K other = __shfl_xor_sync(0xffffffffu, key, j);
      bool up = (lane & k) == 0;
      bool lower = (lane & j) == 0;
      key = (lower == up) ? (other < key ? other : key) : (other > key ? other : key);
    }
  }
  return key;
}

// Ascending bitonic sort of n (power of two) keys in shared memory by a CTA.
template <typename K>
__device__ void cta_bitonic(K *a, int n) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
        int i = 2 * j * (t / j) + (t % j);
        int p = i + j;
        K x = a[i], y = a[p];
        bool up = (i & k) == 0;
        if ((x > y) == up) { a[i] = y; a[p] = x; }
      }
      __syncthreads();
    }
  }
}

// Merge path: number of elements of A among the first d outputs of the
// stable merge of sorted A (na) and B (nb).
template <typename K>
__device__ __forceinline__ long long co_rank(const K *A, long long na, const K *B, long long nb,
                                             long long d) {
  long long lo = d - nb > 0 ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    long long mid = (lo + hi) >> 1;
    if (A[mid] <= B[d - mid - 1]) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// CTA-cooperative stable merge of sorted A and B into C (all global).
template <typename K>
__device__ void cta_merge(const K *A, long long na, const K *B, long long nb, K *C) {
  const long long n = na + nb;
  const int E = 16;
  for (long long base = 0; base < n; base += (long long)blockDim.x * E) {
    long long d0 = base + (long long)threadIdx.x * E;
    if (d0 >= n) continue;
    long long d1 = d0 + E < n ? d0 + E : n;
    long long i = co_rank(A, na, B, nb, d0);
    long long j = d0 - i;
    for (long long d = d0; d < d1; ++d) {
      bool takeA = j >= nb || (i < na && A[i] <= B[j]);
      C[d] = takeA ? A[i++] : B[j++];
    }
  }
}

// Merge adjacent sorted runs of `src` pairwise until one run is left.
// run_off[0..nruns] are run boundaries relative to src (modified).  Uses
// `tmp` (same length) as ping-pong space; the result ends in src.
template <typename K>
__device__ void cta_merge_runs(K *src, K *tmp, long long *run_off, int nruns) {
  K *a = src, *b = tmp;
  while (nruns > 1) {
    for (int r = 0; r + 1 < nruns; r += 2)
      cta_merge(a + run_off[r], run_off[r + 1] - run_off[r], a + run_off[r + 1],
                run_off[r + 2] - run_off[r + 1], b + run_off[r]);
    if (nruns & 1)
      for (long long q = run_off[nruns - 1] + threadIdx.x; q < run_off[nruns]; q += blockDim.x)
        b[q] = a[q];
    __syncthreads();
    if (threadIdx.x == 0) {
      int w = 0;
      for (int r = 0; r < nruns; r += 2) run_off[w++] = run_off[r];
      run_off[w] = run_off[nruns];
    }
    __syncthreads();
    nruns = (nruns + 1) >> 1;
    K *t = a; a = b; b = t;
  }
  if (a != src) {
    for (long long q = run_off[0] + threadIdx.x; q < run_off[1]; q += blockDim.x) src[q] = a[q];
    __syncthreads();
  }
}

// ------------------------------------------------------- host utilities
// Benchmark hooks: every kernel launch is counted; while profiling is on, the
// sparse-product launches are bracketed by CUDA events on their stream.
void note_launch();
enum { PROF_HR = 0, PROF_GIFT = 1 };
bool prof_on();
void prof_begin(cudaStream_t s, int kind, double bytes);
void prof_end(cudaStream_t s);

// Device memory of a graph comes from the caller's workspace: an arena that
// hands out 256-byte aligned pieces in order and never frees one.  A Buf
// grows by taking a new piece (its old piece is abandoned until the arena is
// reset).  The arena in use is the calling thread's current one, set by
// ArenaScope for the duration of an entry point.
struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
};
struct Arena {
  char *base = nullptr;
  size_t cap = 0, used = 0, peak = 0;
  size_t short_need = 0;  // offset + bytes of a request that did not fit (0: none)
};
Arena *&current_arena();
struct ArenaScope {
  Arena *prev;
  explicit ArenaScope(Arena *a) : prev(current_arena()) { current_arena() = a; }
  ~ArenaScope() { current_arena() = prev; }
};
// Gives b at least `bytes` (contents not kept when it grows).  Fails with
// cudaErrorMemoryAllocation, and records the shortfall in the arena, when the
// workspace is too small.
cudaError_t ensure(Buf &b, size_t bytes);

// Several small device values to the host with one synchronisation: each is
// copied device to device (asynchronously) into the staging buffer, then one
// copy brings them all back.
struct D2H {
  void *h;
  const void *d;
  size_t n;  // bytes, at most 64 each
};
cudaError_t d2h_many(Buf &stage, const D2H *items, int count, cudaStream_t s);
void release(Buf &b);  // forgets the piece (the arena's memory is the caller's)
template <typename T>
inline T *P(Buf &b) { return reinterpret_cast<T *>(b.p); }
template <typename T>
inline const T *P(const Buf &b) { return reinterpret_cast<const T *>(b.p); }


inline int grid_for(long long n, int per_block, int cap = 152 * 64) {
  long long g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// Exclusive scan: out[0..n] with out[n] = total.  Tin is widened to Tout.
// tmp must hold scan_tmp_bytes(n) bytes.
size_t scan_tmp_bytes(long long n);
template <typename Tin, typename Tout>
cudaError_t exclusive_scan(const Tin *in, Tout *out, long long n, void *tmp, cudaStream_t s);

// Segmented sort of keys in place, segments [off[s], off[s+1]).
//   MODE_SORT   : sort only (keys unique or order of equal keys irrelevant)
//   MODE_UNIQUE : sort, then move the distinct keys to the segment start and
//                 write their count to cnt[s]
//   MODE_MERGE  : keys are (col << 32 | uint32 value) (64-bit keys) or
//                 (col << 4 | code) (32-bit keys, values decoded by the merge
//                 context below); sort, then for each distinct col write
//                 (col, sum of values as int64; a negative value is kept as
//                 is) to mcol/mval at the segment start and the count to cnt[s]
enum { MODE_SORT = 0, MODE_UNIQUE = 1, MODE_MERGE = 2 };
// Value of a 32-bit merge key's code in segment (row) s: code c >= 1 is a
// clique pair of weight 1/c in lattice units (lattice / c); code 0 is a star
// edge, value -p for the star's net of p nodes, the star node being the row
// when the row is one, else the column.
struct MergeCtx {
  long long lattice, star0;
  int32_t nstar;
  int32_t latq[16];  // lattice / c for c = 1..15 (no integer division per key)
  const int32_t *star_p;  // node count of each star's net
};
cudaError_t set_merge_ctx(const MergeCtx &c, cudaStream_t s);
size_t segsort_tmp_bytes(long long nseg, long long nkeys, int key_bytes);
// maxlen: a bound on the longest segment when the caller knows one (< 0:
// nkeys), which bounds the merge passes of segments beyond shared memory.
template <typename K, int MODE>
cudaError_t segmented_sort(K *keys, const int64_t *off, long long nseg, long long nkeys,
                           int32_t *cnt, int32_t *mcol, int64_t *mval, void *tmp,
                           cudaStream_t s, long long maxlen = -1);
// Largest of n int32 values, combined into *out with atomicMax (*out >= 0).
cudaError_t max_i32(const int32_t *a, long long n, int *out, cudaStream_t s);

}  // namespace pl
