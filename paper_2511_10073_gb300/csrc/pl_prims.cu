// Device-wide primitives: exclusive scan and segmented sort (+ unique / merge).
#include <cstring>
#include <mutex>

#include "pl_common.cuh"

namespace pl {

Arena *&current_arena() {
  static thread_local Arena *a = nullptr;
  return a;
}

cudaError_t ensure(Buf &b, size_t bytes) {
  if (bytes <= b.bytes && b.p) return cudaSuccess;
  Arena *a = current_arena();
  if (!a || !a->base) return cudaErrorInvalidValue;
  const size_t off = (a->used + 255) & ~size_t(255);
  if (off > a->cap || bytes > a->cap - off) {
    if (off + bytes > a->short_need) a->short_need = off + bytes;
    return cudaErrorMemoryAllocation;
  }
  b.p = a->base + off;
  b.bytes = bytes;
  a->used = off + bytes;
  if (a->used > a->peak) a->peak = a->used;
  return cudaSuccess;
}

// The device values of a d2h_many call: item i's n[i] bytes (at most 64) go
// to slot i of the staging buffer.
struct GatherItems {
  const unsigned char *src[8];
  int n[8];
};
__global__ void k_gather_items(GatherItems it, int count, unsigned char *stage) {
  const int i = threadIdx.x >> 6, b = threadIdx.x & 63;  // a thread per byte of a slot
  if (i < count && b < it.n[i]) stage[i * 64 + b] = it.src[i][b];
}

cudaError_t d2h_many(Buf &stage, const D2H *items, int count, cudaStream_t s) {
  constexpr int kMax = 8, kSlot = 64;
  if (count < 1 || count > kMax) return cudaErrorInvalidValue;
  cudaError_t e = ensure(stage, (size_t)kMax * kSlot);
  if (e != cudaSuccess) return e;
  GatherItems g{};
  for (int i = 0; i < count; ++i) {
    if (items[i].n > (size_t)kSlot) return cudaErrorInvalidValue;
    g.src[i] = static_cast<const unsigned char *>(items[i].d);
    g.n[i] = (int)items[i].n;
  }
  // one gather kernel instead of a copy per item
  k_gather_items<<<1, kMax * kSlot, 0, s>>>(g, count, static_cast<unsigned char *>(stage.p));
  note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  unsigned char host[kMax * kSlot];
  e = cudaMemcpyAsync(host, stage.p, (size_t)count * kSlot, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < count; ++i) memcpy(items[i].h, host + i * kSlot, items[i].n);
  return cudaSuccess;
}

void release(Buf &b) {
  b.p = nullptr;
  b.bytes = 0;
}

// ------------------------------------------------------------------- scan
constexpr int SCAN_T = 256, SCAN_V = 8, SCAN_B = SCAN_T * SCAN_V;

template <typename Tout>
__device__ Tout block_excl_scan(Tout v, Tout *total) {
  __shared__ Tout wsum[SCAN_T / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  Tout x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    Tout y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    Tout t = lane < SCAN_T / 32 ? wsum[lane] : Tout(0);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      Tout y = __shfl_up_sync(0xffffffffu, t, d);
      if (lane >= d) t += y;
    }
    if (lane < SCAN_T / 32) wsum[lane] = t;
  }
  __syncthreads();
  Tout before = w ? wsum[w - 1] : Tout(0);
  *total = wsum[SCAN_T / 32 - 1];
  __syncthreads();
  return before + x - v;
}

template <typename Tin, typename Tout>
__global__ void k_scan_reduce(const Tin *in, Tout *bsum, long long n) {
  long long base = (long long)blockIdx.x * SCAN_B;
  Tout s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_V; ++k) {
    long long i = base + k * SCAN_T + threadIdx.x;
    if (i < n) s += (Tout)in[i];
  }
  Tout tot;
  block_excl_scan<Tout>(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <typename Tin, typename Tout>
__global__ void k_scan_apply(const Tin *in, Tout *out, long long n, const Tout *boff) {
  __shared__ Tout sm[SCAN_B];
  long long base = (long long)blockIdx.x * SCAN_B;
#pragma unroll
  for (int k = 0; k < SCAN_V; ++k) {
    long long i = base + k * SCAN_T + threadIdx.x;
    sm[k * SCAN_T + threadIdx.x] = i < n ? (Tout)in[i] : Tout(0);
  }
  __syncthreads();
  Tout v[SCAN_V];
  Tout s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_V; ++k) {
    v[k] = s;
    s += sm[threadIdx.x * SCAN_V + k];
  }
  Tout tot;
  Tout pre = block_excl_scan<Tout>(s, &tot);
  Tout off = boff ? boff[blockIdx.x] : Tout(0);
#pragma unroll
  for (int k = 0; k < SCAN_V; ++k) sm[threadIdx.x * SCAN_V + k] = v[k] + pre + off;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < SCAN_V; ++k) {
    long long i = base + k * SCAN_T + threadIdx.x;
    if (i < n) out[i] = sm[k * SCAN_T + threadIdx.x];
  }
  if (threadIdx.x == 0 && base + SCAN_B >= n) out[n] = off + tot;
}

size_t scan_tmp_bytes(long long n) {
  size_t b = 0;
  while (n > SCAN_B) {
    long long nb = (n + SCAN_B - 1) / SCAN_B;
    b += (size_t)(2 * nb + 2) * sizeof(int64_t) + 512;
    n = nb;
  }
  return b + 512;
}

template <typename Tin, typename Tout>
cudaError_t exclusive_scan(const Tin *in, Tout *out, long long n, void *tmp, cudaStream_t s) {
  if (n <= 0) {
    return cudaMemsetAsync(out, 0, sizeof(Tout), s);
  }
  long long nb = (n + SCAN_B - 1) / SCAN_B;
  if (nb == 1) {
    k_scan_apply<Tin, Tout><<<1, SCAN_T, 0, s>>>(in, out, n, nullptr);
    note_launch();
    return cudaGetLastError();
  }
  char *t = static_cast<char *>(tmp);
  Tout *bsum = reinterpret_cast<Tout *>(t);
  Tout *boff = reinterpret_cast<Tout *>(t + (((size_t)nb * sizeof(Tout) + 255) & ~size_t(255)));
  char *rest = reinterpret_cast<char *>(boff) + (((size_t)(nb + 1) * sizeof(Tout) + 255) & ~size_t(255));
  k_scan_reduce<Tin, Tout><<<(unsigned)nb, SCAN_T, 0, s>>>(in, bsum, n);
  note_launch();
  cudaError_t e = exclusive_scan<Tout, Tout>(bsum, boff, nb, rest, s);
  if (e != cudaSuccess) return e;
  k_scan_apply<Tin, Tout><<<(unsigned)nb, SCAN_T, 0, s>>>(in, out, n, boff);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t exclusive_scan<int32_t, int32_t>(const int32_t *, int32_t *, long long, void *, cudaStream_t);
template cudaError_t exclusive_scan<int32_t, int64_t>(const int32_t *, int64_t *, long long, void *, cudaStream_t);
template cudaError_t exclusive_scan<int64_t, int64_t>(const int64_t *, int64_t *, long long, void *, cudaStream_t);
template cudaError_t exclusive_scan<uint32_t, uint64_t>(const uint32_t *, uint64_t *, long long, void *, cudaStream_t);
template cudaError_t exclusive_scan<uint64_t, uint64_t>(const uint64_t *, uint64_t *, long long, void *, cudaStream_t);
template cudaError_t exclusive_scan<uint8_t, int32_t>(const uint8_t *, int32_t *, long long, void *, cudaStream_t);

// --------------------------------------------------------- segmented sort
constexpr int SEG_T = 256;
constexpr int SEG_CAP = 4096;  // keys sorted in shared memory at once

template <typename K>
__device__ __forceinline__ K key_max() { return ~K(0); }
// Merge keys: (col << 32 | value) for 64-bit keys, (col << 4 | code) for
// 32-bit keys with the value decoded from the merge context.
__constant__ MergeCtx c_merge;
static MergeCtx h_merge;  // source of the asynchronous copy (kept alive)

cudaError_t set_merge_ctx(const MergeCtx &c, cudaStream_t s) {
  h_merge = c;
  return cudaMemcpyToSymbolAsync(c_merge, &h_merge, sizeof(MergeCtx), 0, cudaMemcpyHostToDevice, s);
}

template <typename K>
__device__ __forceinline__ int32_t key_col(K k) {
  if (sizeof(K) == 8) return (int32_t)((uint64_t)k >> 32);
  return (int32_t)((uint32_t)k >> 4);
}
template <typename K>
__device__ __forceinline__ long long key_val(K k, long long s) {
  if (sizeof(K) == 8) return (long long)(int32_t)(uint32_t)((uint64_t)k & 0xffffffffu);
  const uint32_t code = (uint32_t)k & 15u;
  if (code) return c_merge.latq[code];
  const long long col = (long long)((uint32_t)k >> 4);
  const long long st = (s >= c_merge.star0 && s < c_merge.star0 + c_merge.nstar) ? s : col;
  return -(long long)c_merge.star_p[st - c_merge.star0];
}

// Segments are sorted by size class: up to 8, 16 and 32 keys by groups of 8,
// 16 or 32 lanes (several segments per warp); up to 64..512 keys by one warp
// holding 2..16 keys per lane; up to SEG_CAP by a CTA in shared memory; the
// rest by a CTA merge sort in global memory.
constexpr int kSegClasses = 9;  // <=8, <=16, <=32, <=64, <=128, <=256, <=512, <=SEG_CAP, more
struct SegLists {
  int32_t n[kSegClasses];
  int32_t maxbig;  // keys of the longest segment above SEG_CAP
};
__device__ __forceinline__ int seg_class(long long n) {
  if (n <= 8) return 0;
  if (n <= 16) return 1;
  if (n <= 32) return 2;
  if (n <= 64) return 3;
  if (n <= 128) return 4;
  if (n <= 256) return 5;
  if (n <= 512) return 6;
  if (n <= SEG_CAP) return 7;
  return 8;
}

template <typename K, int MODE>
__device__ __forceinline__ void write_single(K key, long long o, int32_t *cnt, long long s,
                                             int32_t *mcol, int64_t *mval) {
  if (MODE == MODE_MERGE) {
    mcol[o] = key_col<K>(key);
    mval[o] = key_val<K>(key, s);
  }
  if (MODE != MODE_SORT) cnt[s] = 1;
}

// Segment lists per class (warp-aggregated appends); segments of 0 or 1 key
// are finished here.
template <typename K, int MODE>
__global__ void k_seg_classify(K *keys, const int64_t *off, long long nseg, int32_t *cnt,
                               int32_t *mcol, int64_t *mval, int32_t *lists,
                               SegLists *ln) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (long long s0 = (blockIdx.x * (long long)blockDim.x) + (threadIdx.x & ~31); s0 < nseg;
       s0 += (long long)gridDim.x * blockDim.x) {
    const long long s = s0 + lane;
    int cls = -1;
    if (s < nseg) {
      const long long o = off[s], n = off[s + 1] - o;
      if (n <= 0) {
        if (MODE != MODE_SORT) cnt[s] = 0;
      } else if (n == 1) {
        write_single<K, MODE>(keys[o], o, cnt, s, mcol, mval);
      } else {
        cls = seg_class(n);
      }
    }
    const unsigned grp = __match_any_sync(0xffffffffu, cls);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (cls >= 0 && lane == leader) base = atomicAdd(&ln->n[cls], __popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (cls >= 0) lists[(long long)cls * nseg + base + __popc(grp & lt)] = (int32_t)s;
    if (cls == kSegClasses - 1) atomicMax(&ln->maxbig, (int32_t)(off[s + 1] - off[s]));
  }
}

// Bitonic sort of 32*R keys held R per lane (element r*32 + lane), ascending.
template <typename K, int R>
__device__ __forceinline__ void warp_bitonic_regs(K (&key)[R], int lane) {
#pragma unroll
  for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        const int jr = j >> 5;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (r & jr) continue;
          const bool up = (((r << 5) | lane) & k) == 0;
          const K a = key[r], b = key[r + jr];
          const bool sw = up ? (b < a) : (a < b);
          key[r] = sw ? b : a;
          key[r + jr] = sw ? a : b;
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const K other = __shfl_xor_sync(0xffffffffu, key[r], j);
          const bool up = (((r << 5) | lane) & k) == 0;
          const bool lower = (lane & j) == 0;
          key[r] = (lower == up) ? (other < key[r] ? other : key[r])
                                 : (other > key[r] ? other : key[r]);
        }
      }
    }
  }
}

// Groups of W lanes (W = 8, 16, 32) each sort one segment of at most W keys.
template <typename K, int MODE, int W>
__global__ void __launch_bounds__(256) k_seg_group(K *keys, const int64_t *off, int32_t *cnt,
                                                   int32_t *mcol, int64_t *mval,
                                                   const int32_t *list, const SegLists *ln,
                                                   int cls) {
  const int lane = threadIdx.x & 31, sub = lane & (W - 1);
  const unsigned gmask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << (lane & ~(W - 1)));
  const unsigned lt = (1u << lane) - 1u;
  const int nl = ln->n[cls];
  const long long per = 32 / W;
  for (long long i0 = ((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5) * per; i0 < nl;
       i0 += (((long long)gridDim.x * blockDim.x) >> 5) * per) {
    const long long it = i0 + lane / W;
    long long o = 0, s = 0;
    int n = 0;
    if (it < nl) {
      s = list[it];
      o = off[s];
      n = (int)(off[s + 1] - o);
    }
    K key = sub < n ? keys[o + sub] : key_max<K>();
#pragma unroll
    for (int k = 2; k <= W; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const K other = __shfl_xor_sync(0xffffffffu, key, j);
        const bool up = (sub & k) == 0;
        const bool lower = (sub & j) == 0;
        key = (lower == up) ? (other < key ? other : key) : (other > key ? other : key);
      }
    }
    if (MODE == MODE_SORT) {
      if (sub < n) keys[o + sub] = key;
      continue;
    }
    if (MODE == MODE_UNIQUE) {
      const K prev = __shfl_up_sync(0xffffffffu, key, 1);
      const bool head = sub < n && (sub == 0 || prev != key);
      const unsigned hm = __ballot_sync(0xffffffffu, head) & gmask;
      if (head) keys[o + __popc(hm & lt)] = key;
      if (sub == 0 && it < nl) cnt[s] = __popc(hm);
      continue;
    }
    // MODE_MERGE: sum the values of equal columns
    const int32_t col = key_col<K>(key);
    long long val = sub < n ? key_val<K>(key, s) : 0;
    const int32_t pcol = __shfl_up_sync(0xffffffffu, col, 1);
    const bool head = sub < n && (sub == 0 || pcol != col);
    const unsigned hm = __ballot_sync(0xffffffffu, head) & gmask;
    const int seg = 31 - __clz(hm & (lt | (1u << lane)));
#pragma unroll
    for (int d = 1; d < W; d <<= 1) {
      const long long ov = __shfl_up_sync(0xffffffffu, val, d);
      const int os = __shfl_up_sync(0xffffffffu, seg, d);
      if (sub >= d && os == seg) val += ov;
    }
    const bool tail = sub < n && (sub + 1 >= n || ((hm >> (lane + 1)) & 1u));
    if (tail) {
      const int idx = __popc(hm & (lt | (1u << lane))) - 1;
      mcol[o + idx] = col;
      mval[o + idx] = val;
    }
    if (sub == 0 && it < nl) cnt[s] = __popc(hm);
  }
}

// One warp per segment of 33..32*R keys, R keys per lane; the sorted keys go
// through the warp's shared-memory slice for the compaction (each lane a
// contiguous run of R positions).
template <typename K, int MODE, int R>
__global__ void __launch_bounds__(256) k_seg_regs(K *keys, const int64_t *off, int32_t *cnt,
                                                  int32_t *mcol, int64_t *mval,
                                                  const int32_t *list, const SegLists *ln,
                                                  int cls) {
  __shared__ K sk[8][32 * R];
  const int lane = threadIdx.x & 31;
  K *a = sk[threadIdx.x >> 5];
  const int nl = ln->n[cls];
  for (long long it = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; it < nl;
       it += ((long long)gridDim.x * blockDim.x) >> 5) {
    const long long s = list[it];
    const long long o = off[s];
    const int n = (int)(off[s + 1] - o);
    K key[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = (r << 5) | lane;
      key[r] = e < n ? keys[o + e] : key_max<K>();
    }
    warp_bitonic_regs<K, R>(key, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) a[(r << 5) | lane] = key[r];
    __syncwarp();
    const int e0 = lane * R, e1 = min(n, e0 + R);
    if (MODE == MODE_SORT) {
      for (int e = e0; e < e1; ++e) keys[o + e] = a[e];
      __syncwarp();
      continue;
    }
    int nh = 0;
    for (int e = e0; e < e1; ++e) {
      const bool head = MODE == MODE_MERGE ? (e == 0 || key_col<K>(a[e]) != key_col<K>(a[e - 1]))
                                           : (e == 0 || a[e] != a[e - 1]);
      nh += head;
    }
    int x = nh;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    int w = x - nh;
    for (int e = e0; e < e1; ++e) {
      if (MODE == MODE_MERGE) {
        if (!(e == 0 || key_col<K>(a[e]) != key_col<K>(a[e - 1]))) continue;
        const int32_t col = key_col<K>(a[e]);
        long long v = 0;
        for (int q = e; q < n && key_col<K>(a[q]) == col; ++q) v += key_val<K>(a[q], s);
        mcol[o + w] = col;
        mval[o + w] = v;
      } else {
        if (!(e == 0 || a[e] != a[e - 1])) continue;
        keys[o + w] = a[e];
      }
      ++w;
    }
    if (lane == 31) cnt[s] = x;
    __syncwarp();
  }
}

// After a segment of n keys (at `a`, shared or global) is sorted: compaction
// for the UNIQUE / MERGE modes by a CTA.  Each thread owns a contiguous
// sub-range; heads are counted, block-scanned and written.
template <typename K, int MODE>
__device__ void cta_compact(K *a, long long n, long long o, long long s, int32_t *cnt,
                            int32_t *mcol, int64_t *mval, K *gkeys) {
  __shared__ long long s_base;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  const long long chunk = (long long)SEG_T * 16;
  for (long long c0 = 0; c0 < n; c0 += chunk) {
    long long c1 = c0 + chunk < n ? c0 + chunk : n;
    long long per = (c1 - c0 + SEG_T - 1) / SEG_T;
    long long b = c0 + threadIdx.x * per, e = b + per < c1 ? b + per : c1;
    int nh = 0;
    for (long long q = b; q < e; ++q) {
      bool head;
      if (MODE == MODE_MERGE) head = q == 0 || key_col<K>(a[q]) != key_col<K>(a[q - 1]);
      else head = q == 0 || a[q] != a[q - 1];
      nh += head;
    }
    int64_t tot;
    int64_t pre = block_excl_scan<int64_t>((int64_t)nh, &tot);
    long long w = s_base + pre;
    // all threads must read a[] before anyone writes the compacted output when
    // a aliases the output (UNIQUE mode in global memory): collect first.
    for (long long q = b; q < e; ++q) {
      bool head;
      if (MODE == MODE_MERGE) head = q == 0 || key_col<K>(a[q]) != key_col<K>(a[q - 1]);
      else head = q == 0 || a[q] != a[q - 1];
      if (!head) continue;
      if (MODE == MODE_MERGE) {
        int32_t col = key_col<K>(a[q]);
        long long v = 0;
        for (long long r = q; r < n && key_col<K>(a[r]) == col; ++r) v += key_val<K>(a[r], s);
        mcol[o + w] = col;
        mval[o + w] = v;
      } else {
        gkeys[o + w] = a[q];
      }
      ++w;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) cnt[s] = (int32_t)s_base;
  __syncthreads();
}

template <typename K, int MODE>
__global__ void __launch_bounds__(SEG_T) k_seg_cta(K *keys, const int64_t *off, int32_t *cnt,
                                                   int32_t *mcol, int64_t *mval,
                                                   const int32_t *med, const SegLists *lists) {
  extern __shared__ __align__(16) unsigned char smraw[];
  K *a = reinterpret_cast<K *>(smraw);
  const int nmed = lists->n[7];
  for (int it = blockIdx.x; it < nmed; it += gridDim.x) {
    long long s = med[it];
    long long o = off[s];
    int n = (int)(off[s + 1] - o);
    int p2 = 64;
    while (p2 < n) p2 <<= 1;
    for (int q = threadIdx.x; q < p2; q += SEG_T) a[q] = q < n ? keys[o + q] : key_max<K>();
    __syncthreads();
    cta_bitonic<K>(a, p2);
    if (MODE == MODE_SORT) {
      for (int q = threadIdx.x; q < n; q += SEG_T) keys[o + q] = a[q];
      __syncthreads();
    } else {
      cta_compact<K, MODE>(a, n, o, s, cnt, mcol, mval, keys);
    }
  }
}

// Segments longer than SEG_CAP, spread over all CTAs: each is cut into units
// of SEG_CAP keys; bpre[i] is the first unit of the i-th listed segment.  The
// units are sorted in shared memory, then runs of doubling length are merged
// pass by pass (one launch per pass, every CTA merging one unit of output),
// between the key array and a scratch copy.
__global__ void __launch_bounds__(SEG_T) k_big_prefix(const int32_t *big, const SegLists *lists,
                                                      const int64_t *off, long long *bpre) {
  const int nbig = lists->n[kSegClasses - 1];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int i0 = 0; i0 <= nbig; i0 += SEG_T) {
    const int i = i0 + threadIdx.x;
    long long u = 0;
    if (i < nbig) {
      const long long sgm = big[i];
      u = (off[sgm + 1] - off[sgm] + SEG_CAP - 1) / SEG_CAP;
    }
    long long tot;
    const long long ex = block_excl_scan<long long>(u, &tot);
    if (i <= nbig) bpre[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

// The listed segment holding unit u (binary search over bpre): its key
// offset and length, and u's index inside it; false past the last unit.
__device__ __forceinline__ bool big_unit(const int32_t *big, int nbig, const long long *bpre,
                                         const int64_t *off, long long u, long long *o,
                                         long long *n, long long *c) {
  if (u >= bpre[nbig]) return false;
  int lo = 0, hi = nbig - 1;  // last i with bpre[i] <= u
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bpre[mid] <= u) lo = mid; else hi = mid - 1;
  }
  const long long sgm = big[lo];
  *o = off[sgm];
  *n = off[sgm + 1] - *o;
  *c = u - bpre[lo];
  return true;
}

template <typename K>
__global__ void __launch_bounds__(SEG_T) k_big_units(K *keys, const int32_t *big,
                                                     const SegLists *lists,
                                                     const long long *bpre, const int64_t *off) {
  extern __shared__ __align__(16) unsigned char smraw[];
  K *a = reinterpret_cast<K *>(smraw);
  const int nbig = lists->n[kSegClasses - 1];
  long long o, n, c;
  for (long long u = blockIdx.x; big_unit(big, nbig, bpre, off, u, &o, &n, &c); u += gridDim.x) {
    const long long c0 = c * SEG_CAP;
    const int m = (int)(n - c0 < SEG_CAP ? n - c0 : SEG_CAP);
    for (int q = threadIdx.x; q < SEG_CAP; q += SEG_T) a[q] = q < m ? keys[o + c0 + q] : key_max<K>();
    __syncthreads();
    cta_bitonic<K>(a, SEG_CAP);
    for (int q = threadIdx.x; q < m; q += SEG_T) keys[o + c0 + q] = a[q];
    __syncthreads();
  }
}

// One merge pass over runs of R keys: output unit c of a segment lies inside
// one pair of runs (2R is a multiple of SEG_CAP); each thread merges 16
// consecutive outputs from its merge-path split.  A segment of at most R keys
// (one run) is copied.
template <typename K>
__global__ void __launch_bounds__(SEG_T) k_big_merge(const K *src, K *dst, const int32_t *big,
                                                     const SegLists *lists,
                                                     const long long *bpre, const int64_t *off,
                                                     long long R) {
  const int nbig = lists->n[kSegClasses - 1];
  if (R >= lists->maxbig) return;
  long long o, n, c;
  for (long long u = blockIdx.x; big_unit(big, nbig, bpre, off, u, &o, &n, &c); u += gridDim.x) {
    const long long t0 = c * SEG_CAP, t1 = t0 + SEG_CAP < n ? t0 + SEG_CAP : n;
    const long long base = (t0 / (2 * R)) * (2 * R);
    const long long na = n - base < R ? n - base : R;
    const long long nb = n - base - na < R ? n - base - na : R;
    const K *A = src + o + base, *B = A + na;
    if (nb <= 0) {
      for (long long q = t0 + threadIdx.x; q < t1; q += SEG_T) dst[o + q] = src[o + q];
      continue;
    }
    const int E = 16;
    for (long long d0 = t0 - base + (long long)threadIdx.x * E; d0 < t1 - base;
         d0 += (long long)SEG_T * E) {
      const long long d1 = d0 + E < t1 - base ? d0 + E : t1 - base;
      long long i = co_rank(A, na, B, nb, d0);
      long long j = d0 - i;
      for (long long d = d0; d < d1; ++d) {
        const bool takeA = j >= nb || (i < na && A[i] <= B[j]);
        dst[o + base + d] = takeA ? A[i++] : B[j++];
      }
    }
  }
}

// After the merge passes: the keys are in the scratch copy when the number of
// passes that ran (runs of SEG_CAP doubling while below the longest segment)
// is odd.
template <typename K>
__global__ void __launch_bounds__(SEG_T) k_big_copy(const K *src, K *dst, const int32_t *big,
                                                    const SegLists *lists, const long long *bpre,
                                                    const int64_t *off) {
  const int nbig = lists->n[kSegClasses - 1];
  int passes = 0;
  for (long long R = SEG_CAP; R < lists->maxbig; R <<= 1) ++passes;
  if (!(passes & 1)) return;
  long long o, n, c;
  for (long long u = blockIdx.x; big_unit(big, nbig, bpre, off, u, &o, &n, &c); u += gridDim.x) {
    const long long t0 = c * SEG_CAP, t1 = t0 + SEG_CAP < n ? t0 + SEG_CAP : n;
    for (long long q = t0 + threadIdx.x; q < t1; q += SEG_T) dst[o + q] = src[o + q];
  }
}

// Compaction of the sorted big segments (UNIQUE / MERGE), a CTA each.
template <typename K, int MODE>
__global__ void __launch_bounds__(SEG_T) k_big_compact(K *keys, K *scratch, const int64_t *off,
                                                       int32_t *cnt, int32_t *mcol, int64_t *mval,
                                                       const int32_t *big, const SegLists *lists) {
  const int nbig = lists->n[kSegClasses - 1];
  for (int it = blockIdx.x; it < nbig; it += gridDim.x) {
    const long long sgm = big[it];
    const long long o = off[sgm], n = off[sgm + 1] - o;
    // UNIQUE output goes to scratch first (the input would be overwritten
    // while read), then back
    if (MODE == MODE_UNIQUE) {
      cta_compact<K, MODE>(keys + o, n, 0, sgm, cnt, mcol, mval, scratch + o);
      const int m = cnt[sgm];
      __syncthreads();
      for (long long q = threadIdx.x; q < m; q += SEG_T) keys[o + q] = scratch[o + q];
      __syncthreads();
    } else {
      cta_compact<K, MODE>(keys + o, n, o, sgm, cnt, mcol, mval, keys);
    }
  }
}

size_t segsort_tmp_bytes(long long nseg, long long nkeys, int key_bytes) {
  return 1024 + (size_t)kSegClasses * (size_t)(nseg + 1) * sizeof(int32_t) +
         (size_t)nkeys * key_bytes + 512;
}

__global__ void k_max_i32(const int32_t *a, long long n, int *out) {
  int m = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = max(m, a[i]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}

cudaError_t max_i32(const int32_t *a, long long n, int *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_max_i32<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(a, n, out);
  note_launch();
  return cudaGetLastError();
}

template <typename K, int MODE>
cudaError_t segmented_sort(K *keys, const int64_t *off, long long nseg, long long nkeys,
                           int32_t *cnt, int32_t *mcol, int64_t *mval, void *tmp,
                           cudaStream_t s, long long maxlen) {
  if (nseg <= 0) return cudaSuccess;
  char *t = static_cast<char *>(tmp);
  SegLists *lists = reinterpret_cast<SegLists *>(t);
  int32_t *cl = reinterpret_cast<int32_t *>(t + 256);
  size_t kb = ((256 + (size_t)kSegClasses * (size_t)(nseg + 1) * sizeof(int32_t)) + 255) & ~size_t(255);
  K *scratch = reinterpret_cast<K *>(t + kb);
  cudaError_t e = cudaMemsetAsync(lists, 0, sizeof(SegLists), s);
  if (e != cudaSuccess) return e;
  k_seg_classify<K, MODE><<<grid_for(nseg, 256), 256, 0, s>>>(keys, off, nseg, cnt, mcol, mval,
                                                              cl, lists);
  note_launch();
  // every class kernel reads its list length on the device (no host round
  // trip); an empty class costs one launch that returns at once
  const int gb = 152 * 8;
  k_seg_group<K, MODE, 8><<<gb, 256, 0, s>>>(keys, off, cnt, mcol, mval, cl, lists, 0);
  k_seg_group<K, MODE, 16><<<gb, 256, 0, s>>>(keys, off, cnt, mcol, mval, cl + nseg, lists, 1);
  k_seg_group<K, MODE, 32><<<gb, 256, 0, s>>>(keys, off, cnt, mcol, mval, cl + 2 * nseg, lists, 2);
  k_seg_regs<K, MODE, 2><<<gb, 256, 0, s>>>(keys, off, cnt, mcol, mval, cl + 3 * nseg, lists, 3);
  k_seg_regs<K, MODE, 4><<<gb, 256, 0, s>>>(keys, off, cnt, mcol, mval, cl + 4 * nseg, lists, 4);
  k_seg_regs<K, MODE, 8><<<gb, 256, 0, s>>>(keys, off, cnt, mcol, mval, cl + 5 * nseg, lists, 5);
  k_seg_regs<K, MODE, 16><<<gb, 256, 0, s>>>(keys, off, cnt, mcol, mval, cl + 6 * nseg, lists, 6);
  for (int q = 0; q < 7; ++q) note_launch();
  size_t sm = SEG_CAP * sizeof(K);
  static std::once_flag attr_once;
  std::call_once(attr_once, [sm] {
    cudaFuncSetAttribute(k_seg_cta<K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_big_units<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  });
  k_seg_cta<K, MODE><<<152 * 4, SEG_T, sm, s>>>(keys, off, cnt, mcol, mval, cl + 7 * nseg, lists);
  note_launch();
  if (nkeys > SEG_CAP && (maxlen < 0 || maxlen > SEG_CAP)) {
    // The unit prefix overwrites the lists of the small classes (consumed by
    // the launches above): (nbig + 1) 8-byte entries fit below the list of
    // class 8 at byte 32 * nseg, since nbig <= nseg.
    const int32_t *big = cl + 8 * nseg;
    long long *bpre = reinterpret_cast<long long *>(t + 256);
    k_big_prefix<<<1, SEG_T, 0, s>>>(big, lists, off, bpre);
    k_big_units<K><<<152 * 4, SEG_T, sm, s>>>(keys, big, lists, bpre, off);
    note_launch();
    note_launch();
    // passes while R < the longest segment (a pass past it returns at once);
    // maxlen, else nkeys, bounds that length
    const long long bound = maxlen >= 0 && maxlen < nkeys ? maxlen : nkeys;
    int npass = 0;
    for (long long R = SEG_CAP; R < bound; R <<= 1) {
      k_big_merge<K><<<152 * 4, SEG_T, 0, s>>>(npass & 1 ? scratch : keys, npass & 1 ? keys : scratch,
                                               big, lists, bpre, off, R);
      note_launch();
      ++npass;
    }
    if (npass) {
      k_big_copy<K><<<152 * 4, SEG_T, 0, s>>>(scratch, keys, big, lists, bpre, off);
      note_launch();
    }
    if (MODE != MODE_SORT) {
      k_big_compact<K, MODE><<<152, SEG_T, 0, s>>>(keys, scratch, off, cnt, mcol, mval, big, lists);
      note_launch();
    }
  }
  (void)nkeys;
  return cudaGetLastError();
}

template cudaError_t segmented_sort<uint32_t, MODE_SORT>(uint32_t *, const int64_t *, long long, long long, int32_t *, int32_t *, int64_t *, void *, cudaStream_t, long long);
template cudaError_t segmented_sort<uint32_t, MODE_UNIQUE>(uint32_t *, const int64_t *, long long, long long, int32_t *, int32_t *, int64_t *, void *, cudaStream_t, long long);
template cudaError_t segmented_sort<uint64_t, MODE_MERGE>(uint64_t *, const int64_t *, long long, long long, int32_t *, int32_t *, int64_t *, void *, cudaStream_t, long long);
template cudaError_t segmented_sort<uint32_t, MODE_MERGE>(uint32_t *, const int64_t *, long long, long long, int32_t *, int32_t *, int64_t *, void *, cudaStream_t, long long);

}  // namespace pl
