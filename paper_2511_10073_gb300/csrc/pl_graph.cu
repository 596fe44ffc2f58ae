// A1: the static instance graph of a netlist hypergraph, GPU-side.
//
// Sec. V "Macro pin expansion": every pin on a macro is its own fixed node at
// macro centre + pin offset; other pins map to their cell.  Net model (a
// reading; the paper gives none): a net with p distinct nodes is a clique of
// weight 1/(p-1) when 2 <= p <= clique_max, else a star of weight p/(p-1) to
// a new movable star node.  Parallel edges add exactly on the integer lattice
// 1/360360 = 1/lcm(1..15) and are divided once (IEEE correctly rounded).
#include <cmath>
#include <cstring>

#include "pl_internal.h"

namespace pl {

constexpr long long kLattice = 360360;
constexpr long long kMaxNetPins = 32768;

#define TRY(x)                                   \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

// ----------------------------------------------------------- validation
__global__ void k_validate_cells(const float *w, const float *h, const uint8_t *kind,
                                 const float *fx, const float *fy, int32_t C, int *status,
                                 uint8_t *is_macro, unsigned *maxdims) {
  // per-thread counts and maxima (a grid of a few blocks per SM, each thread
  // many cells), combined over the warp
  const int lane = threadIdx.x & 31;
  int nmov = 0;
  unsigned mx[4] = {0u, 0u, 0u, 0u};
  bool bad = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
    uint8_t k = kind[i];
    float wi = w[i], hi = h[i];
    bool ok = k <= 2 && isfinite(wi) && isfinite(hi) && wi >= 0.f && hi >= 0.f;
    if (k == 1) ok = ok && wi > 0.f && hi > 0.f;
    if (k != 0) ok = ok && isfinite(fx[i]) && isfinite(fy[i]);
    bad |= !ok;
    is_macro[i] = k == 1;
    if (k == 0) ++nmov;
    if (ok) {
      if (k == 0) {
        mx[0] = max(mx[0], __float_as_uint(wi));
        mx[1] = max(mx[1], __float_as_uint(hi));
      } else if (k == 1) {
        mx[2] = max(mx[2], __float_as_uint(wi));
        mx[3] = max(mx[3], __float_as_uint(hi));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nmov += __shfl_xor_sync(0xffffffffu, nmov, o);
#pragma unroll
    for (int q = 0; q < 4; ++q) mx[q] = max(mx[q], __shfl_xor_sync(0xffffffffu, mx[q], o));
  }
  // then over the block (one atomic per block and counter)
  __shared__ int s_n[32], s_bad[32];
  __shared__ unsigned s_mx[32][4];
  const int wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const bool anybad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    s_n[wid] = nmov;
    s_bad[wid] = anybad;
#pragma unroll
    for (int q = 0; q < 4; ++q) s_mx[wid][q] = mx[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0, b = 0;
    unsigned m[4] = {0u, 0u, 0u, 0u};
    for (int k = 0; k < nw; ++k) {
      n += s_n[k];
      b |= s_bad[k];
#pragma unroll
      for (int q = 0; q < 4; ++q) m[q] = max(m[q], s_mx[k][q]);
    }
    if (b) flag(status, ST_BAD_CELL);
    if (n) atomicAdd(&status[12], n);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (m[q]) atomicMax(&maxdims[q], m[q]);
  }
}

__global__ void k_validate_nets(const int64_t *ptr, int32_t M, int64_t P, int *status) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= M; e += gridDim.x * blockDim.x) {
    if (e == 0 && ptr[0] != 0) flag(status, ST_BAD_NET);
    if (e == M && ptr[M] != P) flag(status, ST_BAD_NET);
    if (e < M) {
      long long d = ptr[e + 1] - ptr[e];
      if (d < 0) flag(status, ST_BAD_NET);
      if (d > kMaxNetPins) flag(status, ST_TOO_BIG);
    }
    // the largest net beyond 1024 pins (status[13], else 0) bounds the merge
    // passes of the net sort
    if (e < M) {
      const long long d = ptr[e + 1] - ptr[e];
      if (d > 1024) atomicMax(&status[13], (int)min(d, (long long)INT32_MAX));
    }
  }
}

__global__ void k_validate_pins(const int32_t *pin_cell, const float *dx, const float *dy,
                                int64_t P, int32_t C, int *status) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    int32_t c = pin_cell[p];
    if (c < 0 || c >= C) flag(status, ST_BAD_INDEX);
    if ((dx && !isfinite(dx[p])) || (dy && !isfinite(dy[p]))) flag(status, ST_BAD_CELL);
  }
}

// ------------------------------------------------------- node numbering
__global__ void k_macro_list(const uint8_t *is_macro, const int32_t *scan, int32_t C,
                             int32_t *macro_cell) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x)
    if (is_macro[i]) macro_cell[scan[i]] = i;
}

__global__ void k_pin_macro_flag(const int32_t *pin_cell, const uint8_t *is_macro, int64_t P,
                                 int32_t C, uint8_t *f) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x)
  {
    const int32_t c = pin_cell[p];  // checked by the validation, read before its result
    f[p] = (c >= 0 && c < C) ? is_macro[c] : (uint8_t)0;
  }
}

__global__ void k_pin_node(const int32_t *pin_cell, const uint8_t *f, const int32_t *scan,
                           int64_t P, int32_t C, int32_t *pin_node, uint32_t *keys) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    int32_t v = f[p] ? C + scan[p] : pin_cell[p];
    pin_node[p] = v;
    keys[p] = (uint32_t)v;
  }
}

__global__ void k_star_flag(const int32_t *net_p, int32_t M, int32_t cmax, uint8_t *f) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M; e += gridDim.x * blockDim.x)
    f[e] = net_p[e] > cmax;
}

__global__ void k_star_p(int32_t S, const int32_t *star_net, const int32_t *net_p,
                         int32_t *star_p) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < S; q += gridDim.x * blockDim.x)
    star_p[q] = net_p[star_net[q]];
}

__global__ void k_star_list(const uint8_t *f, const int32_t *scan, int32_t M, int32_t *star_net) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M; e += gridDim.x * blockDim.x)
    if (f[e]) star_net[scan[e]] = e;
}

// ---------------------------------------------------- edge expansion
// Row counts of the unmerged edge list: warp per net.
// Unmerged row lengths: a clique net adds p - 1 to each of its nodes' rows, a
// star net 1 (and p to its star's row).  A thread takes a net of up to 32
// distinct nodes; larger nets are taken by the whole warp in turn.
__global__ void k_row_count(const int64_t *ptr, const uint32_t *nd, const int32_t *net_p,
                            const int32_t *star_of, int32_t M, int32_t cmax, int64_t star0,
                            int32_t *cnt) {
  const int lane = threadIdx.x & 31;
  for (long long e0 = (blockIdx.x * (long long)blockDim.x) + (threadIdx.x & ~31); e0 < M;
       e0 += (long long)gridDim.x * blockDim.x) {
    const long long e = e0 + lane;
    int p = 0;
    long long b = 0;
    if (e < M) {
      p = net_p[e];
      b = ptr[e];
    }
    const bool big = p > 32;
    if (!big && p >= 2) {
      const int add = p <= cmax ? p - 1 : 1;
      for (int k = 0; k < p; ++k) atomicAdd(&cnt[nd[b + k]], add);
      if (p > cmax) cnt[star0 + star_of[e]] = p;
    }
    unsigned bm = __ballot_sync(0xffffffffu, big);
    while (bm) {
      const int src = __ffs(bm) - 1;
      bm &= bm - 1;
      const long long ee = e0 + src;
      const int pp = __shfl_sync(0xffffffffu, p, src);
      const long long bb = __shfl_sync(0xffffffffu, b, src);
      const int add = pp <= cmax ? pp - 1 : 1;
      for (int k = lane; k < pp; k += 32) atomicAdd(&cnt[nd[bb + k]], add);
      if (pp > cmax && lane == 0) cnt[star0 + star_of[ee]] = pp;
    }
  }
}

constexpr int kScatterRegs = 4;  // clique nets up to this size kept in registers

// Unmerged entries as 32-bit keys (col << 4 | code): code p - 1 (1..15) for a
// clique pair of a p-node net (value 360360/(p-1) in lattice units), code 0
// for a star edge (value -p, p taken from the star node when merging).  Star
// rows are written in node order directly.
// A thread takes a clique net of up to kScatterRegs nodes (each node reserves
// its p - 1 slots with one atomic, all of the net's reservations in flight at
// once); larger clique nets and star nets are taken by the whole warp in turn.
__global__ void k_scatter(const int64_t *ptr, const uint32_t *nd, const int32_t *net_p,
                          const int32_t *star_of, int32_t M, int32_t cmax, int64_t star0,
                          const int64_t *row_off, unsigned long long *cursor, uint32_t *keys) {
  const int lane = threadIdx.x & 31;
  for (long long e0 = (blockIdx.x * (long long)blockDim.x) + (threadIdx.x & ~31); e0 < M;
       e0 += (long long)gridDim.x * blockDim.x) {
    const long long e = e0 + lane;
    int p = 0;
    long long b = 0;
    if (e < M) {
      p = net_p[e];
      b = ptr[e];
    }
    if (p >= 2 && p <= cmax) {
      const uint32_t lat = (uint32_t)(p - 1);  // code
      if (p <= kScatterRegs) {
        uint32_t node[kScatterRegs];
        unsigned long long slot[kScatterRegs];
#pragma unroll
        for (int a = 0; a < kScatterRegs; ++a)
          if (a < p) node[a] = nd[b + a];
#pragma unroll
        for (int a = 0; a < kScatterRegs; ++a)
          if (a < p) slot[a] = atomicAdd(&cursor[node[a]], (unsigned long long)(p - 1));
#pragma unroll
        for (int a = 0; a < kScatterRegs; ++a) {
          if (a >= p) break;
          unsigned long long k = slot[a];
#pragma unroll
          for (int c = 0; c < kScatterRegs; ++c) {
            if (c >= p) break;
            if (c != a) keys[k++] = (node[c] << 4) | lat;
          }
        }
      }
    }
    // larger clique nets (up to 16 nodes) by the whole warp in turn: lane a
    // holds node a and its slots, lanes then write the p (p - 1) keys
    unsigned bc = __ballot_sync(0xffffffffu, p > kScatterRegs && p <= cmax);
    while (bc) {
      const int src = __ffs(bc) - 1;
      bc &= bc - 1;
      const int pp = __shfl_sync(0xffffffffu, p, src);
      const long long bb = __shfl_sync(0xffffffffu, b, src);
      uint32_t node = 0;
      unsigned long long slot = 0;
      if (lane < pp) {
        node = nd[bb + lane];
        slot = atomicAdd(&cursor[node], (unsigned long long)(pp - 1));
      }
      const uint32_t lat = (uint32_t)(pp - 1);
      const int tot = pp * (pp - 1);
      for (int t0 = 0; t0 < tot; t0 += 32) {
        const int t = t0 + lane;
        const int a = t / (pp - 1), cq = t - a * (pp - 1);  // key cq of node a's run
        const int c = cq + (cq >= a ? 1 : 0);                // the other node (a skipped)
        const uint32_t nc = __shfl_sync(0xffffffffu, node, c & 31);
        const unsigned long long sa = __shfl_sync(0xffffffffu, slot, a & 31);
        if (t < tot) keys[sa + cq] = (nc << 4) | lat;
      }
    }
    unsigned bm = __ballot_sync(0xffffffffu, p > cmax);
    while (bm) {
      const int src = __ffs(bm) - 1;
      bm &= bm - 1;
      const long long ee = e0 + src;
      const int pp = __shfl_sync(0xffffffffu, p, src);
      const long long bb = __shfl_sync(0xffffffffu, b, src);
      const long long st = star0 + star_of[ee];
      const long long so = row_off[st];
      for (int k = lane; k < pp; k += 32) {
        const uint32_t v = nd[bb + k];
        const unsigned long long slot = atomicAdd(&cursor[v], 1ull);
        keys[slot] = (uint32_t)st << 4;
        keys[so + k] = v << 4;
      }
    }
  }
}

// 1/d correctly rounded for d = 1..15 (the weight of a pair seen by one
// clique net of d+1 nodes), filled from the host's IEEE division.
__constant__ double c_recip[16];

// Weight of a merged entry from its lattice value: val > 0 is a sum of clique
// lattice units (weight val / kLattice), val < 0 is -p for a star edge of a
// p-node net (weight p / (p - 1)).  A single clique edge (val = kLattice / d,
// d <= 15) takes the table; every other value needs an IEEE division.
__device__ __forceinline__ bool lattice_easy(long long val, const double *star_w, double *w) {
  if (val < 0 && -val <= kMaxNetPins) {  // star edge of a (-val)-node net
    *w = star_w[-val];
    return true;
  }
  if (val >= kLattice / 15 && val <= kLattice) {
    // 32-bit conversions (a 64-bit integer conversion would take the FP64 pipe)
    // d = kLattice / val to within 2 ulp: exact d is recovered for val =
    // kLattice / d, and every candidate is confirmed in integers
    const int d = (int)(__fdividef((float)kLattice, (float)(int)val) + 0.5f);
    if (d >= 1 && d <= 15 && (long long)d * val == kLattice) {
      *w = c_recip[d];
      return true;
    }
  }
  return false;
}
__device__ __forceinline__ double lattice_div(long long val) {
  if (val > 0) return __ddiv_rn((double)val, (double)kLattice);
  const long long p = -val;
  return __ddiv_rn((double)p, (double)(p - 1));
}

// p / (p - 1) for p = 2..kMaxNetPins, the weight of a star edge of a p-node
// net, each an IEEE division (filled once per graph).
__global__ void k_star_weights(double *star_w) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p <= kMaxNetPins;
       p += (long long)gridDim.x * blockDim.x)
    star_w[p] = p >= 2 ? __ddiv_rn((double)p, (double)(p - 1)) : 0.0;
}

// Table weights in place of the merged values.  A warp takes 32 rows and
// walks their entries as one flat sequence, a lane per entry (the row of an
// entry is found from the rows' length prefix sums), so that short rows keep
// every lane busy; entries that need a division are listed, so that the
// divisions run together in k_static_div instead of stalling whole warps.
constexpr int kDivBuf = 256;  // listed entries a warp buffers before one global append

__global__ void __launch_bounds__(256) k_static_weights(const int64_t *row_off, int64_t *mval,
                                                        const int64_t *srp, int64_t Nst,
                                                        const double *star_w, uint32_t *list,
                                                        unsigned long long *nlist) {
  __shared__ uint32_t wbuf[8][kDivBuf];
  const int lane = threadIdx.x & 31;
  uint32_t *buf = wbuf[threadIdx.x >> 5];
  int nb = 0;  // warp-uniform
  auto flush = [&]() {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(nlist, (unsigned long long)nb);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int i = lane; i < nb; i += 32) list[base + i] = buf[i];
    __syncwarp();
    nb = 0;
  };
  const long long wg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long v0 = wg * 32; v0 < Nst; v0 += nwarp * 32) {
    const long long v = v0 + lane;
    long long src = 0;
    uint32_t m = 0;
    if (v < Nst) {
      src = row_off[v];
      m = (uint32_t)(srp[v + 1] - srp[v]);
    }
    uint32_t incl = m;  // inclusive prefix sum of the lengths (< 2^32 entries in all)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const long long rb = src - (long long)(incl - m);  // entry e of the warp is at rb_j + e
    const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
    for (uint32_t e0 = 0; e0 < T; e0 += 32) {
      const uint32_t e = e0 + lane;
      int j = 0;  // the row holding entry e: rows whose prefix ends at or before e
#pragma unroll
      for (int st = 16; st > 0; st >>= 1)
        if (__shfl_sync(0xffffffffu, incl, j + st - 1) <= e) j += st;
      const long long q = __shfl_sync(0xffffffffu, rb, j) + e;
      bool hard = false;
      if (e < T) {
        double w;
        if (lattice_easy(mval[q], star_w, &w)) reinterpret_cast<double *>(mval)[q] = w;
        else hard = true;
      }
      const unsigned hm = __ballot_sync(0xffffffffu, hard);
      if (nb + 32 > kDivBuf) flush();
      if (hard) buf[nb + __popc(hm & ((1u << lane) - 1u))] = (uint32_t)q;
      nb += __popc(hm);
      __syncwarp();
    }
  }
  if (nb) flush();
}

__global__ void k_static_div(const uint32_t *list, const unsigned long long *nlist,
                             int64_t *mval) {
  const unsigned long long n = *nlist;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t k = list[i];
    reinterpret_cast<double *>(mval)[k] = lattice_div(mval[k]);
  }
}

// BF16 bits of a double, rounded to nearest even, from the double's high word
// with 32-bit integer operations when the result is a normal number (the
// exponent rebias and the mantissa carry are one integer addition); other
// values take d2bf16.
__device__ __forceinline__ uint16_t d2bf16_normal(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t ah = hi & 0x7fffffffu;
  if ((ah >> 20) - 897u < 254u) {  // unbiased exponent in [-126, 127]
    const uint32_t t = ah >> 13;    // double exponent and the 7 kept mantissa bits
    const uint32_t r = ah & 0x1fffu;  // the next 13 mantissa bits; 0x1000 is half
    const uint32_t inc = (r > 0x1000u || (r == 0x1000u && (lo != 0u || (t & 1u)))) ? 1u : 0u;
    return (uint16_t)(((hi >> 16) & 0x8000u) | (t - (896u << 7) + inc));
  }
  return d2bf16(d);
}

// A positive double of at least 2^-15 in 128-bit fixed point with 2^-67
// resolution (exact: its last mantissa bit is worth at least 2^-67), as four
// 32-bit limbs, least significant first.
struct Fix128 {
  uint32_t a0, a1, a2, a3;
};
__device__ __forceinline__ void fix_add_double(Fix128 &a, double w) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(w);
  const uint32_t hi = (uint32_t)(b >> 32), Ml = (uint32_t)b;
  const uint32_t Mh = (hi & 0xfffffu) | 0x100000u;  // w = M 2^(e - 52), M = Mh:Ml
  const int sh = (int)((hi >> 20) & 0x7ffu) - 1008;  // w 2^67 = M << (e + 15), 0 <= sh < 75
  const int q = sh >> 5, r = sh & 31;
  // M << r as three limbs, then moved up by q limbs
  const uint32_t c0 = Ml << r, c1 = __funnelshift_l(Ml, Mh, r), c2 = __funnelshift_l(Mh, 0u, r);
  const bool q0 = q == 0, q1 = q == 1;
  const uint32_t A0 = q0 ? c0 : 0u;
  const uint32_t A1 = q0 ? c1 : (q1 ? c0 : 0u);
  const uint32_t A2 = q0 ? c2 : (q1 ? c1 : c0);
  const uint32_t A3 = q0 ? 0u : (q1 ? c2 : c1);
  asm("add.cc.u32 %0, %0, %4;\n\t"
      "addc.cc.u32 %1, %1, %5;\n\t"
      "addc.cc.u32 %2, %2, %6;\n\t"
      "addc.u32 %3, %3, %7;"
      : "+r"(a.a0), "+r"(a.a1), "+r"(a.a2), "+r"(a.a3)
      : "r"(A0), "r"(A1), "r"(A2), "r"(A3));
}
// RN(x) * 2^e for x > 0 with a normal result, in integer arithmetic (the
// conversion and scaling instructions of FP64 would take the slow FP64 pipe):
// round the top 53 bits to nearest, ties to even, and assemble the bits.
__device__ __forceinline__ double u64_rn_scaled(unsigned long long x, int e) {
  int nb = 64 - __clzll((long long)x);
  unsigned long long m;
  if (nb <= 53) {
    m = x << (53 - nb);
  } else {
    const int sh = nb - 53;
    m = x >> sh;
    const unsigned long long rem = x & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) ++m;
    if (m >> 53) {
      m >>= 1;
      ++nb;
    }
  }
  const unsigned long long bits =
      ((unsigned long long)(nb - 1 + e + 1023) << 52) | (m & 0xfffffffffffffull);
  return __longlong_as_double((long long)bits);
}

// The fixed-point value rounded once to the nearest double (ties to even):
// the top 64 bits with a sticky bit, then one correctly rounded conversion.
__device__ __forceinline__ double fix_to_double(const Fix128 &f) {
  const unsigned long long lo = ((unsigned long long)f.a1 << 32) | f.a0;
  const unsigned long long hi = ((unsigned long long)f.a3 << 32) | f.a2;
  if (hi == 0) return lo ? u64_rn_scaled(lo, -67) : 0.0;
  const int sh = 64 - __clzll((long long)hi);  // bits of hi, 1..64
  unsigned long long top, rest;
  if (sh == 64) {
    top = hi;
    rest = lo;
  } else {
    top = (hi << (64 - sh)) | (lo >> sh);
    rest = lo & ((1ull << sh) - 1ull);
  }
  if (rest) top |= 1ull;
  return u64_rn_scaled(top, sh - 67);
}

// Final static matrix, written straight into its split layout, from the FP64
// weights (in place of the merged values): each row's columns and stored
// weights go to the row's place (short region or hub region); its static
// degree is summed in double-float over the stored weights (every static
// weight is positive, so it is also the positive sum) and, for a cell, the
// FP64 weights are summed exactly (128-bit fixed point, order-free) for
// baseWeight = RN(sum) / count.  A thread takes a short row (entry order);
// the warp takes each of its hub rows in turn (lanes over the entries, then
// a fixed butterfly), so that a row of thousands of entries is no serial tail.
struct CompactRow {
  dfl dl{0.f, 0.f};
  Fix128 fl{0u, 0u, 0u, 0u};
};
// One entry: its stored bits (BF16 or FP32), added to the degree (stored
// value) and, for a cell, to the exact sum (FP64 value).
template <bool BF>
__device__ __forceinline__ uint32_t compact_entry(CompactRow &r, double w, bool cell) {
  float f;
  uint32_t bits;
  if (BF) {
    const uint16_t h = d2bf16_normal(w);
    f = bf16_to_f(h);
    bits = h;
  } else {
    f = __double2float_rn(w);
    bits = __float_as_uint(f);
  }
  df_add(r.dl, f);
  if (cell) fix_add_double(r.fl, w);
  return bits;
}
// Exact sum of the lanes' fixed-point values (a butterfly; every lane gets it).
__device__ __forceinline__ Fix128 warp_sum_fix(Fix128 a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t b0 = __shfl_xor_sync(0xffffffffu, a.a0, o);
    const uint32_t b1 = __shfl_xor_sync(0xffffffffu, a.a1, o);
    const uint32_t b2 = __shfl_xor_sync(0xffffffffu, a.a2, o);
    const uint32_t b3 = __shfl_xor_sync(0xffffffffu, a.a3, o);
    asm("add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, %5;\n\t"
        "addc.cc.u32 %2, %2, %6;\n\t"
        "addc.u32 %3, %3, %7;"
        : "+r"(a.a0), "+r"(a.a1), "+r"(a.a2), "+r"(a.a3)
        : "r"(b0), "r"(b1), "r"(b2), "r"(b3));
  }
  return a;
}

constexpr int kCompactUnroll = 4;  // entries of a short row loaded at once

template <bool BF>
__global__ void __launch_bounds__(256) k_static_compact(
    const int64_t *row_off, const int32_t *mcol, const int64_t *mval, const int64_t *srp,
    int64_t Nst, int32_t C, const uint8_t *ckind, const uint32_t *rp_s, const int32_t *longidx,
    const uint64_t *lptr, int32_t *scol, void *sw, dfl *dsum, dfl *psum, double *base_w,
    uint8_t *hflag) {
  const int lane = threadIdx.x & 31;
  const double *w64 = reinterpret_cast<const double *>(mval);
  auto put = [&](long long k, uint32_t b) {
    if (BF) reinterpret_cast<uint16_t *>(sw)[k] = (uint16_t)b;
    else reinterpret_cast<uint32_t *>(sw)[k] = b;
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); v0 < Nst;
       v0 += stride) {
    const long long v = v0 + lane;
    long long src = 0, dst = 0;
    int m = 0, li = -1;
    if (v < Nst) {
      src = row_off[v];
      m = (int)(srp[v + 1] - srp[v]);
      li = longidx[v];
      dst = li >= 0 ? (long long)lptr[li] : (long long)(rp_s[v] & kOffMask);
    }
    const bool cell = v < C;
    CompactRow r;
    if (v < Nst && li < 0) {
      int k = 0;
      for (; k + kCompactUnroll <= m; k += kCompactUnroll) {  // loads in flight, then the entries
        double wv[kCompactUnroll];
        int32_t cv[kCompactUnroll];
#pragma unroll
        for (int u = 0; u < kCompactUnroll; ++u) {
          wv[u] = w64[src + k + u];
          cv[u] = mcol[src + k + u];
        }
#pragma unroll
        for (int u = 0; u < kCompactUnroll; ++u) {
          put(dst + k + u, compact_entry<BF>(r, wv[u], cell));
          scol[dst + k + u] = cv[u];
        }
      }
      for (; k < m; ++k) {
        put(dst + k, compact_entry<BF>(r, w64[src + k], cell));
        scol[dst + k] = mcol[src + k];
      }
    }
    unsigned hubs = __ballot_sync(0xffffffffu, v < Nst && li >= 0);
    while (hubs) {
      const int j = __ffs(hubs) - 1;
      hubs &= hubs - 1;
      const long long sj = __shfl_sync(0xffffffffu, src, j);
      const long long dj = __shfl_sync(0xffffffffu, dst, j);
      const int mj = __shfl_sync(0xffffffffu, m, j);
      const bool cj = v0 + j < C;
      CompactRow h;
      for (int k = lane; k < mj; k += 32) {
        put(dj + k, compact_entry<BF>(h, w64[sj + k], cj));
        scol[dj + k] = mcol[sj + k];
      }
      const dfl d = warp_sum_df(h.dl);
      const Fix128 f = warp_sum_fix(h.fl);
      if (lane == j) {
        r.dl = d;
        r.fl = f;
      }
    }
    if (v >= Nst) continue;
    const dfl dl = df_norm(r.dl);
    dsum[v] = dl;
    psum[v] = dl;
    if (cell) {
      const double bw = m > 0 ? __ddiv_rn(fix_to_double(r.fl), (double)m) : 0.0;
      base_w[v] = bw;
      hflag[v] = (ckind[v] == 0 && __double_as_longlong(bw) > 0) ? 1 : 0;  // bw > 0 (integer test)
    }
  }
}

// ---------------------------------------------------------- node tables
__global__ void k_nodes(int64_t N, int32_t C, int32_t Pm, int32_t S, int32_t Mm, int32_t nbx,
                        const uint8_t *ckind, const float *cw, const float *ch, const float *fx,
                        const float *fy, const int32_t *macro_cell, double xl, double yl,
                        double xh, double yh, double wb, double hb, uint8_t *nkind,
                        float2 *fixedp, float4 *bounds) {
  const int64_t st0 = (int64_t)C + Pm, mv0 = st0 + S, bn0 = mv0 + Mm;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    uint8_t k = 2;
    float2 f = make_float2(0.f, 0.f);
    float4 bd = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v < C) {
      if (ckind[v] == 0) {
        k = 0;
        double hw = (double)cw[v] * 0.5, hh = (double)ch[v] * 0.5;
        bd = make_float4(__double2float_rn(xl + hw), __double2float_rn(yl + hh),
                         __double2float_rn(xh - hw), __double2float_rn(yh - hh));
      } else {
        f = make_float2(fx[v], fy[v]);
      }
    } else if (v < st0) {
      // macro pins: filled by k_pin_fixed
    } else if (v < mv0) {
      k = 1;
      bd = make_float4(__double2float_rn(xl), __double2float_rn(yl), __double2float_rn(xh),
                       __double2float_rn(yh));
    } else if (v < bn0) {
      int32_t c = macro_cell[v - mv0];
      f = make_float2(fx[c], fy[c]);
    } else {
      long long b = v - bn0;
      int bx = (int)(b % nbx), by = (int)(b / nbx);
      f = make_float2(__double2float_rn(xl + ((double)bx + 0.5) * wb),
                      __double2float_rn(yl + ((double)by + 0.5) * hb));
    }
    nkind[v] = k;
    if (v < C || v >= st0) fixedp[v] = f;
    bounds[v] = bd;
  }
}

__global__ void k_pin_fixed(const int32_t *pin_node, const int32_t *pin_cell, const float *dx,
                            const float *dy, const float *fx, const float *fy, int64_t P,
                            int32_t C, float2 *fixedp) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    int32_t v = pin_node[p];
    if (v < C) continue;
    int32_t c = pin_cell[p];
    double x = (double)fx[c] + (dx ? (double)dx[p] : 0.0);
    double y = (double)fy[c] + (dy ? (double)dy[p] : 0.0);
    fixedp[v] = make_float2(__double2float_rn(x), __double2float_rn(y));
  }
}

// Macro area inside each bin, summed over macros in macro order (FP64).  Warp
// per bin: lanes test 32 macros at a time (FP32 box reject, then the FP64
// overlap), lane 0 adds the overlapping ones in macro order.
// Centre and size of every macro (float4), read by the area and grid kernels.
__global__ void k_macro_geo(int32_t Mm, const int32_t *macro_cell, const float *fx,
                            const float *fy, const float *cw, const float *ch, float4 *geo) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < Mm; m += gridDim.x * blockDim.x) {
    const int c = macro_cell[m];
    geo[m] = make_float4(fx[c], fy[c], cw[c], ch[c]);
  }
}

// Macro area inside each bin (warp per bin): lanes test 32 macros at a time,
// four such groups loaded at once; the overlaps are added in macro order.
__global__ void k_bin_macro_area(int32_t NB, int32_t nbx, int32_t Mm, const float4 *mgeo,
                                 double xl, double yl, double wb, double hb, double *amac) {
  const int lane = threadIdx.x & 31;
  for (long long b = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; b < NB;
       b += ((long long)gridDim.x * blockDim.x) >> 5) {
    int bx = (int)(b % nbx), by = (int)(b / nbx);
    double bxl = xl + (double)bx * wb, bxh = xl + (double)(bx + 1) * wb;
    double byl = yl + (double)by * hb, byh = yl + (double)(by + 1) * hb;
    float fxl = (float)bxl, fxh = (float)bxh, fyl = (float)byl, fyh = (float)byh;
    double a = 0.0;
    for (int m0 = 0; m0 < Mm; m0 += 4 * 32) {
      float4 g4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int m = m0 + u * 32 + lane;
        g4[u] = m < Mm ? mgeo[m] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int m = m0 + u * 32 + lane;
        const float4 g = g4[u];
        double ov = 0.0;
        if (m < Mm) {
          float hwf = g.z * 0.5f, hhf = g.w * 0.5f;
          if (!(g.x - hwf > fxh + 1.f || g.x + hwf < fxl - 1.f || g.y - hhf > fyh + 1.f ||
                g.y + hhf < fyl - 1.f)) {
            double hwm = __dmul_rn((double)g.z, 0.5), hhm = __dmul_rn((double)g.w, 0.5);
            double ox = __dadd_rn(fmin(bxh, __dadd_rn((double)g.x, hwm)),
                                  -fmax(bxl, __dadd_rn((double)g.x, -hwm)));
            double oy = __dadd_rn(fmin(byh, __dadd_rn((double)g.y, hhm)),
                                  -fmax(byl, __dadd_rn((double)g.y, -hhm)));
            if (ox > 0.0 && oy > 0.0) ov = __dmul_rn(ox, oy);
          }
        }
        unsigned hit = __ballot_sync(0xffffffffu, ov != 0.0);
        while (hit) {
          int src = __ffs(hit) - 1;
          hit &= hit - 1;
          double t = __shfl_sync(0xffffffffu, ov, src);
          a = __dadd_rn(a, t);
        }
      }
    }
    if (lane == 0) amac[b] = a;
  }
}

// Macro lookup grid: every macro is listed in the grid buckets its rectangle,
// grown by half the largest movable cell, touches, widened by mgx / mgy bucket
// units: more than the FP32 error of a cell centre's bucket coordinate, so the
// bucket of every overlapping cell lists the macro.
__device__ __forceinline__ void macro_bucket_range(int m, const int32_t *macro_cell,
                                                   const float *cw, const float *ch,
                                                   const float *fx, const float *fy, float wmax,
                                                   float hmax, double xl, double yl, double sx,
                                                   double sy, double mgx, double mgy, int gnx,
                                                   int gny, int *k) {
  int c = macro_cell[m];
  double ex = 0.5 * ((double)cw[c] + (double)wmax) * (1.0 + 1e-6) + 1e-6;
  double ey = 0.5 * ((double)ch[c] + (double)hmax) * (1.0 + 1e-6) + 1e-6;
  double a0 = floor(((double)fx[c] - ex - xl) * sx - mgx), a1 = floor(((double)fx[c] + ex - xl) * sx + mgx);
  double b0 = floor(((double)fy[c] - ey - yl) * sy - mgy), b1 = floor(((double)fy[c] + ey - yl) * sy + mgy);
  k[0] = (int)fmin(fmax(a0, 0.0), (double)(gnx - 1));
  k[1] = (int)fmin(fmax(a1, 0.0), (double)(gnx - 1));
  k[2] = (int)fmin(fmax(b0, 0.0), (double)(gny - 1));
  k[3] = (int)fmin(fmax(b1, 0.0), (double)(gny - 1));
}

__global__ void k_grid_count(int32_t Mm, const int32_t *macro_cell, const float *cw,
                             const float *ch, const float *fx, const float *fy, float wmax,
                             float hmax, double xl, double yl, double sx, double sy, double mgx,
                             double mgy, int gnx, int gny, int32_t *cnt) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < Mm; m += gridDim.x * blockDim.x) {
    int k[4];
    macro_bucket_range(m, macro_cell, cw, ch, fx, fy, wmax, hmax, xl, yl, sx, sy, mgx, mgy, gnx,
                       gny, k);
    for (int y = k[2]; y <= k[3]; ++y)
      for (int x = k[0]; x <= k[1]; ++x) atomicAdd(&cnt[(long long)y * gnx + x], 1);
  }
}

__global__ void k_grid_fill(int32_t Mm, const int32_t *macro_cell, const float *cw,
                            const float *ch, const float *fx, const float *fy, float wmax,
                            float hmax, double xl, double yl, double sx, double sy, double mgx,
                            double mgy, int gnx, int gny, int32_t *cur, uint32_t *list) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < Mm; m += gridDim.x * blockDim.x) {
    int k[4];
    macro_bucket_range(m, macro_cell, cw, ch, fx, fy, wmax, hmax, xl, yl, sx, sy, mgx, mgy, gnx,
                       gny, k);
    for (int y = k[2]; y <= k[3]; ++y)
      for (int x = k[0]; x <= k[1]; ++x) list[atomicAdd(&cur[(long long)y * gnx + x], 1)] = m;
  }
}

// Centre and size of each macro listed in the lookup grid, beside its id, so
// that a lookup reads the list and the geometry in one step.
__global__ void k_grid_geo(long long n, const uint32_t *list, const int32_t *macro_cell,
                           const float *fx, const float *fy, const float *cw, const float *ch,
                           float4 *geo) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = macro_cell[list[i]];
    geo[i] = make_float4(fx[c], fy[c], cw[c], ch[c]);
  }
}

__global__ void k_i32_to_i64(const int32_t *a, int64_t *b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = a[i];
}

__global__ void k_i64_to_i32(const int64_t *a, int32_t *b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (int32_t)a[i];
}

// ------------------------------------------------------------- driver
template <typename T>
static cudaError_t d2h(T *h, const void *d, size_t n, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(h, d, n * sizeof(T), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

static cudaError_t scan_tmp(pl_graph *g, long long n, void **t) {
  cudaError_t e = ensure(g->tmp[7], scan_tmp_bytes(n) + 4096);
  *t = g->tmp[7].p;
  return e;
}

pl_status build_static(pl_graph *g, const pl_netlist *nl, const pl_params *p, cudaStream_t s) {
  const int32_t C = nl->num_cells, M = nl->num_nets;
  const int64_t NP = nl->num_pins;
  g->C = C;
  g->M = M;
  g->P = NP;
  g->xl = nl->xl; g->yl = nl->yl; g->xh = nl->xh; g->yh = nl->yh;
  g->wdtype = p->wdtype;
  g->clique_max = p->clique_max;
  g->det_ratio = p->det_ratio;
  g->nbx = p->nbx;
  g->nby = p->nby;
  g->NB = p->nbx * p->nby;
  g->have_hints = false;
  g->stream = s;

  // copies of the netlist arrays
  TRY(ensure(g->cw, (size_t)C * 4 + 16));
  TRY(ensure(g->ch, (size_t)C * 4 + 16));
  TRY(ensure(g->ckind, (size_t)C + 16));
  TRY(ensure(g->cfx, (size_t)C * 4 + 16));
  TRY(ensure(g->cfy, (size_t)C * 4 + 16));
  TRY(ensure(g->net_ptr, (size_t)(M + 1) * 8));
  if (C) {
    TRY(cudaMemcpyAsync(g->cw.p, nl->cell_w, (size_t)C * 4, cudaMemcpyDeviceToDevice, s));
    TRY(cudaMemcpyAsync(g->ch.p, nl->cell_h, (size_t)C * 4, cudaMemcpyDeviceToDevice, s));
    TRY(cudaMemcpyAsync(g->ckind.p, nl->cell_kind, (size_t)C, cudaMemcpyDeviceToDevice, s));
    TRY(cudaMemcpyAsync(g->cfx.p, nl->fixed_x, (size_t)C * 4, cudaMemcpyDeviceToDevice, s));
    TRY(cudaMemcpyAsync(g->cfy.p, nl->fixed_y, (size_t)C * 4, cudaMemcpyDeviceToDevice, s));
  }
  TRY(cudaMemcpyAsync(g->net_ptr.p, nl->net_ptr, (size_t)(M + 1) * 8, cudaMemcpyDeviceToDevice, s));

  TRY(ensure(g->status, 64));
  TRY(cudaMemsetAsync(g->status.p, 0, 64, s));
  int *status = P<int>(g->status);
  unsigned *maxdims = reinterpret_cast<unsigned *>(status + 8);
  uint8_t *is_macro;
  TRY(ensure(g->tmp[0], (size_t)C + 256));
  is_macro = P<uint8_t>(g->tmp[0]);
  k_validate_cells<<<grid_for(C, 256, 152 * 4), 256, 0, s>>>(P<float>(g->cw), P<float>(g->ch),
                                                    P<uint8_t>(g->ckind), P<float>(g->cfx),
                                                    P<float>(g->cfy), C, status, is_macro, maxdims);
  note_launch();
  k_validate_nets<<<grid_for(M + 1, 256), 256, 0, s>>>(P<int64_t>(g->net_ptr), M, NP, status);
  note_launch();
  if (NP) {
    k_validate_pins<<<grid_for(NP, 256), 256, 0, s>>>(nl->pin_cell, nl->pin_dx, nl->pin_dy, NP, C,
                                                     status);
    note_launch();
  }
  TRY(cudaGetLastError());

  // macros and macro pin nodes (their counts read with the validation's
  // result: the pin flags skip pins out of range)
  void *stmp;
  TRY(ensure(g->cell_macro, (size_t)(C + 1) * 4));
  TRY(scan_tmp(g, C > NP ? C : NP, &stmp));
  TRY((exclusive_scan<uint8_t, int32_t>(is_macro, P<int32_t>(g->cell_macro), C, stmp, s)));
  TRY(ensure(g->tmp[1], (size_t)(NP > M ? NP : M) + 256));  // pin flags, later net flags
  uint8_t *pflag = P<uint8_t>(g->tmp[1]);
  TRY(ensure(g->tmp[2], (size_t)(NP + 1) * 4 + 256));
  int32_t *pscan = P<int32_t>(g->tmp[2]);
  if (NP) {
    k_pin_macro_flag<<<grid_for(NP, 256), 256, 0, s>>>(nl->pin_cell, is_macro, NP, C, pflag);
    note_launch();
  }
  TRY((exclusive_scan<uint8_t, int32_t>(pflag, pscan, NP, stmp, s)));
  int hst[16];
  int32_t sizes2[2];
  {
    const D2H it[3] = {{hst, g->status.p, 64},
                       {&sizes2[0], P<int32_t>(g->cell_macro) + C, 4},
                       {&sizes2[1], pscan + NP, 4}};
    TRY(d2h_many(g->stage, it, 3, s));
  }
  if (hst[0] & (ST_BAD_CELL | ST_BAD_NET | ST_BAD_INDEX)) {
    set_error("invalid netlist:%s%s%s", (hst[0] & ST_BAD_CELL) ? " cell size/kind/position" : "",
              (hst[0] & ST_BAD_NET) ? " net_ptr" : "",
              (hst[0] & ST_BAD_INDEX) ? " pin_cell out of range" : "");
    return PL_ERR_INVALID_ARG;
  }
  if (hst[0] & ST_TOO_BIG) {
    set_error("a net has more than %lld pins", (long long)kMaxNetPins);
    return PL_ERR_UNSUPPORTED;
  }
  g->nmov = hst[12];
  const int maxnet = hst[13];  // 0: no net above 1024 pins
  float wmax, hmax, mwmax, mhmax;
  memcpy(&wmax, &hst[8], 4);
  memcpy(&hmax, &hst[9], 4);
  memcpy(&mwmax, &hst[10], 4);
  memcpy(&mhmax, &hst[11], 4);
  g->Mm = sizes2[0];
  g->Pm = sizes2[1];
  TRY(ensure(g->macro_cell, (size_t)g->Mm * 4 + 16));
  k_macro_list<<<grid_for(C, 256), 256, 0, s>>>(is_macro, P<int32_t>(g->cell_macro), C,
                                                P<int32_t>(g->macro_cell));
  note_launch();
  TRY(ensure(g->pin_node, (size_t)NP * 4 + 16));
  TRY(ensure(g->nd, (size_t)NP * 4 + 16));
  if (NP) {
    k_pin_node<<<grid_for(NP, 256), 256, 0, s>>>(nl->pin_cell, pflag, pscan, NP, C,
                                                P<int32_t>(g->pin_node), P<uint32_t>(g->nd));
    note_launch();
  }

  // distinct nodes of each net
  TRY(ensure(g->net_p, (size_t)M * 4 + 16));
  TRY(ensure(g->tmp[3], segsort_tmp_bytes(M, NP, 4)));
  TRY((segmented_sort<uint32_t, MODE_UNIQUE>(P<uint32_t>(g->nd), P<int64_t>(g->net_ptr), M, NP,
                                             P<int32_t>(g->net_p), nullptr, nullptr,
                                             g->tmp[3].p, s, maxnet > 0 ? maxnet : 1024)));
  // star nodes
  TRY(ensure(g->star_of, (size_t)(M + 1) * 4));
  k_star_flag<<<grid_for(M, 256), 256, 0, s>>>(P<int32_t>(g->net_p), M, p->clique_max, pflag);
  note_launch();
  TRY(scan_tmp(g, M, &stmp));
  TRY((exclusive_scan<uint8_t, int32_t>(pflag, P<int32_t>(g->star_of), M, stmp, s)));
  int32_t S;
  TRY(d2h(&S, P<int32_t>(g->star_of) + M, 1, s));
  g->S = S;
  TRY(ensure(g->star_net, (size_t)S * 4 + 16));
  k_star_list<<<grid_for(M, 256), 256, 0, s>>>(pflag, P<int32_t>(g->star_of), M,
                                               P<int32_t>(g->star_net));
  note_launch();
  TRY(ensure(g->star_p, (size_t)S * 4 + 16));
  if (S) {
    k_star_p<<<grid_for(S, 256), 256, 0, s>>>(S, P<int32_t>(g->star_net), P<int32_t>(g->net_p),
                                             P<int32_t>(g->star_p));
    note_launch();
  }
  g->Nst = (int64_t)C + g->Pm + S;
  g->N = g->Nst + g->Mm + g->NB;
  if (g->N >= (1LL << 31) - 1) {
    set_error("too many nodes (%lld)", (long long)g->N);
    return PL_ERR_UNSUPPORTED;
  }
  const int64_t Nst = g->Nst, star0 = (int64_t)C + g->Pm;

  // unmerged row counts and offsets
  TRY(ensure(g->tmp[4], (size_t)(Nst + 1) * 4 + 256));
  int32_t *cnt = P<int32_t>(g->tmp[4]);
  TRY(cudaMemsetAsync(cnt, 0, (size_t)(Nst + 1) * 4, s));
  k_row_count<<<grid_for((long long)M, 256), 256, 0, s>>>(
      P<int64_t>(g->net_ptr), P<uint32_t>(g->nd), P<int32_t>(g->net_p), P<int32_t>(g->star_of),
      M, p->clique_max, star0, cnt);
  note_launch();
  TRY(ensure(g->tmp[5], (size_t)(Nst + 1) * 8 + 256));
  int64_t *row_off = P<int64_t>(g->tmp[5]);
  TRY(scan_tmp(g, Nst, &stmp));
  TRY((exclusive_scan<int32_t, int64_t>(cnt, row_off, Nst, stmp, s)));
  // the longest unmerged row bounds the merge passes of the row sort
  int *rowmax = P<int>(g->status) + 14;
  TRY(cudaMemsetAsync(rowmax, 0, 4, s));
  TRY(max_i32(cnt, Nst, rowmax, s));
  int64_t npre;
  int32_t maxrow = 0;
  {
    const D2H it[2] = {{&npre, row_off + Nst, 8}, {&maxrow, rowmax, 4}};
    TRY(d2h_many(g->stage, it, 2, s));
  }

  // scatter, sort, merge (32-bit keys: node ids below 2^28)
  if (Nst >= (1LL << 28)) {
    set_error("too many static nodes (%lld) for the expansion's 28-bit columns", (long long)Nst);
    return PL_ERR_UNSUPPORTED;
  }
  const size_t kbytes = ((size_t)(npre + 4) * 4 + 15) & ~size_t(15);
  TRY(ensure(g->tmp[6], kbytes + (size_t)(Nst + 1) * 8 + 512));
  uint32_t *keys = P<uint32_t>(g->tmp[6]);
  unsigned long long *cursor = reinterpret_cast<unsigned long long *>(P<char>(g->tmp[6]) + kbytes);
  TRY(cudaMemcpyAsync(cursor, row_off, (size_t)Nst * 8, cudaMemcpyDeviceToDevice, s));
  k_scatter<<<grid_for((long long)M, 256), 256, 0, s>>>(
      P<int64_t>(g->net_ptr), P<uint32_t>(g->nd), P<int32_t>(g->net_p), P<int32_t>(g->star_of),
      M, p->clique_max, star0, row_off, cursor, keys);
  note_launch();
  TRY(ensure(g->tmp[1], (size_t)npre * 12 + 512));  // merged col (int32) + value (int64)
  int64_t *mval = P<int64_t>(g->tmp[1]);
  int32_t *mcol = reinterpret_cast<int32_t *>(mval + npre + 1);
  TRY(ensure(g->tmp[3], segsort_tmp_bytes(Nst, npre, 4)));
  {
    MergeCtx mc;
    mc.lattice = kLattice;
    mc.latq[0] = 0;
    for (int c = 1; c < 16; ++c) mc.latq[c] = (int32_t)(kLattice / c);
    mc.star0 = star0;
    mc.nstar = g->S;
    mc.star_p = P<int32_t>(g->star_p);
    TRY(set_merge_ctx(mc, s));
  }
  TRY((segmented_sort<uint32_t, MODE_MERGE>(keys, row_off, Nst, npre, cnt, mcol, mval,
                                            g->tmp[3].p, s, maxrow)));
  TRY(ensure(g->srp, (size_t)(Nst + 1) * 8));
  TRY((exclusive_scan<int32_t, int64_t>(cnt, P<int64_t>(g->srp), Nst, stmp, s)));
  {
    pl_status ls = prepare_static_layout(g, s);
    if (ls != PL_OK) return ls;
  }
  TRY(ensure(g->base_w, (size_t)C * 8 + 16));
  TRY(ensure(g->hflag, (size_t)C + 16));
  if (!g->star_w_ok) {
    // weight tables, once per graph: 1/d (host IEEE division) and p / (p - 1)
    double rc[16];
    rc[0] = 0.0;
    for (int d = 1; d < 16; ++d) rc[d] = 1.0 / (double)d;
    TRY(cudaMemcpyToSymbolAsync(c_recip, rc, sizeof(rc), 0, cudaMemcpyHostToDevice, s));
    TRY(ensure(g->star_w, (size_t)(kMaxNetPins + 1) * 8));
    k_star_weights<<<grid_for(kMaxNetPins + 1, 256), 256, 0, s>>>(P<double>(g->star_w));
    note_launch();
    TRY(cudaStreamSynchronize(s));  // rc lives on this stack frame
    g->star_w_ok = true;
  }
  TRY(ensure_side(g));
  TRY(cudaEventRecord(g->ev_fork, s));
  TRY(cudaStreamWaitEvent(g->side, g->ev_fork, 0));
  {
    // keys are consumed by the merge: their buffer holds the division list
    if ((unsigned long long)npre >= (1ull << 32)) {
      set_error("static graph too large (%lld entries before merging)", (long long)npre);
      return PL_ERR_UNSUPPORTED;
    }
    unsigned long long *nlist = reinterpret_cast<unsigned long long *>(keys);
    uint32_t *list = keys + 4;
    TRY(cudaMemsetAsync(nlist, 0, 8, s));
    k_static_weights<<<grid_for(Nst * 32, 256), 256, 0, s>>>(row_off, mval, P<int64_t>(g->srp),
                                                            Nst, P<double>(g->star_w), list,
                                                            nlist);
    note_launch();
    k_static_div<<<152 * 8, 256, 0, s>>>(list, nlist, mval);
    note_launch();
  }
  SpMat &sm = g->st;
  (p->wdtype == PL_W_BF16 ? k_static_compact<true> : k_static_compact<false>)
      <<<grid_for(Nst, 256), 256, 0, s>>>(
          row_off, mcol, mval, P<int64_t>(g->srp), Nst, C, P<uint8_t>(g->ckind),
          P<uint32_t>(sm.rp_s), P<int32_t>(sm.longidx), P<uint64_t>(sm.lptr),
          P<int32_t>(sm.col), sm.w.p, P<dfl>(sm.dsum), P<dfl>(sm.psum), P<double>(g->base_w),
          P<uint8_t>(g->hflag));
  note_launch();
  if (g->N > Nst) {
    TRY(cudaMemsetAsync(P<dfl>(sm.dsum) + Nst, 0, (size_t)(g->N - Nst) * sizeof(dfl), s));
    TRY(cudaMemsetAsync(P<dfl>(sm.psum) + Nst, 0, (size_t)(g->N - Nst) * sizeof(dfl), s));
  }
  TRY(cudaGetLastError());

  // node tables and the macro lookup grid, on the side stream (forked before
  // the weights) while the weights and the compaction run
  cudaStream_t s2 = g->side;
  // node tables
  const int64_t N = g->N;
  g->wb = (g->xh - g->xl) / (double)g->nbx;
  g->hb = (g->yh - g->yl) / (double)g->nby;
  g->abin = g->wb * g->hb;
  int nx = (int)floor(p->det_ratio * (double)g->nbx), ny = (int)floor(p->det_ratio * (double)g->nby);
  if (nx < 1) nx = 1;
  if (ny < 1) ny = 1;
  g->hx = (nx - 1) / 2;
  g->hy = (ny - 1) / 2;
  TRY(ensure(g->nkind, (size_t)N + 16));
  TRY(ensure(g->fixedp, (size_t)N * 8 + 16));
  TRY(ensure(g->bounds, (size_t)N * 16 + 16));
  k_nodes<<<grid_for(N, 256), 256, 0, s2>>>(N, C, g->Pm, S, g->Mm, g->nbx, P<uint8_t>(g->ckind),
                                           P<float>(g->cw), P<float>(g->ch), P<float>(g->cfx),
                                           P<float>(g->cfy), P<int32_t>(g->macro_cell), g->xl,
                                           g->yl, g->xh, g->yh, g->wb, g->hb, P<uint8_t>(g->nkind),
                                           P<float2>(g->fixedp), P<float4>(g->bounds));
  note_launch();
  if (NP) {
    k_pin_fixed<<<grid_for(NP, 256), 256, 0, s2>>>(P<int32_t>(g->pin_node), nl->pin_cell, nl->pin_dx,
                                                 nl->pin_dy, P<float>(g->cfx), P<float>(g->cfy), NP,
                                                 C, P<float2>(g->fixedp));
    note_launch();
  }
  TRY(ensure(g->carea, (size_t)C * 8 + 16));
  if (C) {
    k_cell_area<<<grid_for(C, 256), 256, 0, s2>>>(C, P<float>(g->cw), P<float>(g->ch),
                                                  P<double>(g->carea));
    note_launch();
  }
  TRY(ensure(g->amac, (size_t)g->NB * 8 + 16));
  TRY(ensure(g->Cb, (size_t)g->NB * 8 + 16));
  TRY(ensure(g->mgeo, (size_t)g->Mm * 16 + 16));
  if (g->Mm) {
    k_macro_geo<<<grid_for(g->Mm, 256), 256, 0, s2>>>(g->Mm, P<int32_t>(g->macro_cell),
                                                     P<float>(g->cfx), P<float>(g->cfy),
                                                     P<float>(g->cw), P<float>(g->ch),
                                                     P<float4>(g->mgeo));
    note_launch();
  }
  k_bin_macro_area<<<grid_for((long long)g->NB * 32, 256), 256, 0, s2>>>(
      g->NB, g->nbx, g->Mm, P<float4>(g->mgeo), g->xl, g->yl, g->wb, g->hb, P<double>(g->amac));
  note_launch();

  // macro lookup grid
  // buckets at least as large as any macro or movable cell side, so a macro
  // is listed in at most 6 x 6 buckets (the workspace bound counts on it)
  double gs = fmax(1.0, fmax(fmax((double)mwmax, (double)mhmax), fmax((double)wmax, (double)hmax)));
  g->gnx = (int)fmin(2048.0, fmax(1.0, ceil((g->xh - g->xl) / gs)));
  g->gny = (int)fmin(2048.0, fmax(1.0, ceil((g->yh - g->yl) / gs)));
  const long long ng = (long long)g->gnx * g->gny;
  const double sx = (double)g->gnx / (g->xh - g->xl), sy = (double)g->gny / (g->yh - g->yl);
  // FP32 bucket coordinate of a centre: a few half-ulps of the coordinate and
  // of the bucket index, far below these margins
  const double u24 = 1.0 / 16777216.0;
  const double mgx = 0.01 + 8.0 * u24 * (fmax(fabs(g->xl), fabs(g->xh)) * sx + g->gnx);
  const double mgy = 0.01 + 8.0 * u24 * (fmax(fabs(g->yl), fabs(g->yh)) * sy + g->gny);
  TRY(ensure(g->gptr, (size_t)(ng + 1) * 8 + 16));
  TRY(ensure(g->tmp[4], (size_t)(ng + 1) * 4 + 256));
  int32_t *gcnt = P<int32_t>(g->tmp[4]);
  TRY(cudaMemsetAsync(gcnt, 0, (size_t)(ng + 1) * 4, s2));
  k_grid_count<<<grid_for(g->Mm, 128), 128, 0, s2>>>(
      g->Mm, P<int32_t>(g->macro_cell), P<float>(g->cw), P<float>(g->ch), P<float>(g->cfx),
      P<float>(g->cfy), wmax, hmax, g->xl, g->yl, sx, sy, mgx, mgy, g->gnx, g->gny, gcnt);
  note_launch();
  int64_t *gptr = P<int64_t>(g->gptr);
  TRY(scan_tmp(g, ng, &stmp));
  TRY((exclusive_scan<int32_t, int64_t>(gcnt, gptr, ng, stmp, s2)));
  int64_t nreg;
  TRY(d2h(&nreg, gptr + ng, 1, s2));
  if (nreg > 36LL * g->Mm) {
    set_error("macro lookup grid: %lld entries for %d macros", (long long)nreg, g->Mm);
    return PL_ERR_UNSUPPORTED;
  }
  TRY(ensure(g->glist, (size_t)nreg * 4 + 16));
  if (nreg >= (1LL << 31)) {
    set_error("macro lookup grid too large");
    return PL_ERR_UNSUPPORTED;
  }
  TRY(ensure(g->tmp[2], (size_t)(ng + 1) * 4 + 256));
  int32_t *gcur = P<int32_t>(g->tmp[2]);
  k_i64_to_i32<<<grid_for(ng, 256), 256, 0, s2>>>(gptr, gcur, ng);
  note_launch();
  k_grid_fill<<<grid_for(g->Mm, 128), 128, 0, s2>>>(
      g->Mm, P<int32_t>(g->macro_cell), P<float>(g->cw), P<float>(g->ch), P<float>(g->cfx),
      P<float>(g->cfy), wmax, hmax, g->xl, g->yl, sx, sy, mgx, mgy, g->gnx, g->gny, gcur,
      P<uint32_t>(g->glist));
  note_launch();
  TRY(ensure(g->tmp[3], segsort_tmp_bytes(ng, nreg, 4)));
  TRY((segmented_sort<uint32_t, MODE_SORT>(P<uint32_t>(g->glist), gptr, ng, nreg, nullptr,
                                           nullptr, nullptr, g->tmp[3].p, s2)));
  TRY(ensure(g->ggeo, (size_t)nreg * 16 + 16));
  if (nreg) {
    k_grid_geo<<<grid_for(nreg, 256), 256, 0, s2>>>(nreg, P<uint32_t>(g->glist),
                                                   P<int32_t>(g->macro_cell), P<float>(g->cfx),
                                                   P<float>(g->cfy), P<float>(g->cw),
                                                   P<float>(g->ch), P<float4>(g->ggeo));
    note_launch();
  }
  g->gsz = gs;
  g->gsx = sx;
  g->gsy = sy;
  TRY(cudaEventRecord(g->ev_join, s2));
  TRY(cudaStreamWaitEvent(s, g->ev_join, 0));
  TRY(cudaGetLastError());
  {
    int64_t nnz;  // read with the build's final synchronisation
    TRY(d2h(&nnz, P<int64_t>(g->srp) + Nst, 1, s));
    g->nnz_static = (uint64_t)nnz;
  }
  (void)kMaxNetPins;
  {
    pl_status fs = take_filter_buffers(g);
    if (fs != PL_OK) return fs;
  }
  g->hint_mark = g->arena.used;
  return PL_OK;
}

}  // namespace pl
