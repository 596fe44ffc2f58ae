// The learned refinement filter (declared in pl.h): three taps at powers
// k0 < k1 < k2 of the refinement filter H_r (Sec. V) plus a per-node MLP
// correction, standing in for the plain filter's high-order polynomial in
// Algorithm 1's filter step with k2 sparse products instead of the plain
// filter's highest power.
//
// The MLP (16 -> 64 ReLU -> 4) runs on the tensor cores: a CTA of 128
// threads takes tiles of 128 nodes (the MMA's M), one thread per node.
//   1. each thread writes its node's 16 normalised BF16 inputs into the A
//      tile in shared memory (no swizzle, K-major 8 x 16-byte core matrices);
//   2. one elected thread issues tcgen05.mma kind::f16 (BF16 x BF16 -> FP32)
//      D1[128 x 64] = X W1^T into tensor memory and commits to an mbarrier;
//   3. each warp reads its 32 rows of D1 back (tcgen05.ld 32x32b), adds b1,
//      applies ReLU, rounds to BF16 and writes the hidden tile (the A operand
//      of layer 2, K = 64 as four K = 16 slabs);
//   4. four MMAs D2[128 x 16] = H W2^T (W2's 4 rows padded to N = 16);
//   5. each thread reads its 4 outputs and finishes its node.
// Every mbarrier wait is bounded (about 2 s of clocks); a CTA that gives up
// flags ST_TIMEOUT, frees its tensor memory and returns.
//
// Training runs the same tile forward and a backward pass on CUDA cores
// (FP32; BF16 roundings passed straight through), one tile per CTA, with the
// tile's gradient summed over its 128 records in a fixed order into a
// per-block row, the rows added in block order and Adam applied per weight.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pl_internal.h"

namespace pl {

#define TRY(x)                                       \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

namespace {

constexpr int kNF = PL_LEARNED_NF, kHid = PL_LEARNED_HID, kNOut = PL_LEARNED_NOUT;
constexpr int kLW = PL_LEARNED_SIZE, kRec = PL_LEARNED_REC;
constexpr int kMU = PL_LW_MU, kISD = PL_LW_ISD, kTH = PL_LW_THETA, kW1 = PL_LW_W1,
              kB1 = PL_LW_B1, kW2 = PL_LW_W2, kB2 = PL_LW_B2;
static_assert(kW1 == kTH + 3 && kB1 == kW1 + kHid * kNF && kW2 == kB1 + kHid &&
                  kB2 == kW2 + kNOut * kHid && kLW == kB2 + kNOut,
              "parameter layout");
constexpr int kTile = 128;      // nodes per tile (MMA M), threads per CTA
constexpr int kTmemCols = 64;   // D1 in columns 0..63; D2 reuses 0..15 once D1 is read
constexpr int kN2 = 16;         // layer 2's N (4 outputs padded)
constexpr int kPart = kLW + 1;  // per-block row: gradient at its weight's index, loss last
constexpr int kMaxBatch = 1024; // tiles per training step at most
constexpr int kStats = 41;      // sum f, sum f^2 (16 each), normal equations (6 + 3)
constexpr long long kWaitCycles = 4000000000LL;

// shared memory (byte offsets from a 1024-aligned base)
constexpr int SM_XA = 0;         // A of layer 1: 128 x 16 BF16
constexpr int SM_HA = 4096;      // A of layer 2: 128 x 64 BF16 (four 4 KB slabs)
constexpr int SM_W1 = 20480;     // B of layer 1: 64 x 16 BF16
constexpr int SM_W2 = 22528;     // B of layer 2: 16 x 64 BF16 (four 512 B slabs)
constexpr int SM_B1 = 24576;     // float [64]
constexpr int SM_PRM = 24832;    // float mu[16], isd[16], theta[4], b2[4]
constexpr int SM_W2F = 25088;    // float [4][64]: W2 as BF16 values (backward)
constexpr int SM_BAR = 26112;    // mbarrier
constexpr int SM_TMEM = 26120;   // tensor memory base address
constexpr int SM_TC = 26240;     // end of the forward's part
// training's part (floats, padded strides)
constexpr int kDhS = kHid + 1, kXsS = kNF + 1;
constexpr int SM_DH = SM_TC;                        // [128][65]
constexpr int SM_XS = SM_DH + kTile * kDhS * 4;      // [128][17]
constexpr int SM_DO = SM_XS + kTile * kXsS * 4;      // [128][4]
constexpr int SM_GT = SM_DO + kTile * 4 * 4;         // [128][4]: theta terms, loss
constexpr int SM_TR = SM_GT + kTile * 4 * 4;
// Shared memory per CTA also bounds the CTAs per SM, so that their tensor
// memory (64 columns each) never exceeds the SM's 512 columns: at most 8
// forward CTAs, at most 3 training CTAs, and no mix above 8 in total.
constexpr int kSmemFwd = SM_TC + 1024;
constexpr int kSmemTrain = SM_TR + 1024;
static_assert(9 * (kSmemFwd + 1024) > 233472 && 8 * (kSmemFwd + 1024) <= 233472, "forward smem");
static_assert(4 * (kSmemTrain + 1024) > 233472, "training: at most 3 CTAs per SM");

// instruction descriptors (kind::f16): D FP32 (bit 4), A and B BF16 (bits 7,
// 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t kIdesc1 = idesc(kTile, kHid);
constexpr uint32_t kIdesc2 = idesc(kTile, kN2);

// byte offset of element (row, k) in a K-major no-swizzle operand with 8-row
// groups 256 bytes apart and the two 8-element K halves 128 bytes apart, K in
// slabs of 16 (slab stride `slab`)
__host__ __device__ constexpr int opnd_off(int row, int k, int slab) {
  return (k >> 4) * slab + (row >> 3) * 256 + ((k >> 3) & 1) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// shared memory descriptor: start, leading byte offset 128 (K direction),
// stride byte offset 256 (8-row groups), version 1 (bit 46), no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(256 >> 4) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Waits for phase `parity` of the mbarrier, for at most `limit` clocks.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity,
                                         long long limit = kWaitCycles) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_ld4(uint32_t addr, float *v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Two floats rounded to BF16 (nearest even) in one conversion: lo in the low
// half; with RELU, negative values become 0.
template <bool RELU>
__device__ __forceinline__ uint32_t cvt_bf16x2(float lo, float hi) {
  uint32_t r;
  if (RELU)
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  else
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ uint8_t *smem_base() {
  extern __shared__ __align__(1024) uint8_t dyn_smem[];
  const uint32_t a = su32(dyn_smem);
  return dyn_smem + ((1024u - (a & 1023u)) & 1023u);
}

// Weights into shared memory, the mbarrier, and 128 tensor-memory columns.
// Called by all 128 threads; returns the tensor memory base.
__device__ uint32_t tc_setup(uint8_t *sm, const float *w) {
  const int t = threadIdx.x;
  for (int i = t; i < kHid * kNF; i += kTile)
    *reinterpret_cast<uint16_t *>(sm + SM_W1 + opnd_off(i / kNF, i % kNF, 0)) = f2bf16(w[kW1 + i]);
  float *w2f = reinterpret_cast<float *>(sm + SM_W2F);
  for (int i = t; i < kN2 * kHid; i += kTile) {
    const int n = i / kHid, j = i % kHid;
    const uint16_t b = n < kNOut ? f2bf16(w[kW2 + n * kHid + j]) : (uint16_t)0;
    *reinterpret_cast<uint16_t *>(sm + SM_W2 + opnd_off(n, j, 512)) = b;
    if (n < kNOut) w2f[n * kHid + j] = bf16_to_f(b);
  }
  float *b1 = reinterpret_cast<float *>(sm + SM_B1);
  float *prm = reinterpret_cast<float *>(sm + SM_PRM);
  if (t < kHid) b1[t] = w[kB1 + t];
  if (t < kNF) {
    prm[t] = w[kMU + t];
    prm[16 + t] = w[kISD + t];
  }
  if (t < 3) prm[32 + t] = w[kTH + t];
  if (t < kNOut) prm[36 + t] = w[kB2 + t];
  const uint32_t bar = su32(sm + SM_BAR);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async();
  __syncthreads();
  if (t < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(sm + SM_TMEM)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_before();
  __syncthreads();
  tc_after();
  return *reinterpret_cast<volatile uint32_t *>(sm + SM_TMEM);
}

__device__ void tc_teardown(uint32_t tmem) {
  tc_before();
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// The bounded wait's own check: set up as the learned kernels do, wait on
// an mbarrier phase that nothing completes, for at most `limit` clocks, then
// free the tensor memory and report.
__global__ void __launch_bounds__(kTile) k_wait_check(long long limit, const float *w, int *status) {
  uint8_t *sm = smem_base();
  const uint32_t tmem = tc_setup(sm, w);
  const bool ok = bar_wait(su32(sm + SM_BAR), 0u, limit);
  if (!__syncthreads_and(ok) && threadIdx.x == 0) flag(status, ST_TIMEOUT);
  tc_teardown(tmem);
}

// Normalised BF16 inputs of one node from its raw features.
__device__ __forceinline__ void normalise(const uint8_t *sm, const float *f, uint32_t *xw) {
  const float *prm = reinterpret_cast<const float *>(sm + SM_PRM);
#pragma unroll
  for (int k = 0; k < kNF; k += 2)
    xw[k / 2] = cvt_bf16x2<false>((f[k] - prm[k]) * prm[16 + k],
                                  (f[k + 1] - prm[k + 1]) * prm[16 + k + 1]);
}

// One tile through both layers.  xw: this thread's row (8 words of BF16
// pairs).  out: the 4 outputs (with b2).  With MASK, *mask gets bit j set
// where pre-activation j (with b1) is positive (the ReLU's derivative).  ph:
// the mbarrier's next phase parity.  False (the same in every thread) when a
// wait gave up.
template <bool MASK>
__device__ bool tc_tile(uint8_t *sm, uint32_t tmem, uint32_t &ph, const uint32_t *xw, float *out,
                        uint64_t *mask) {
  const int r = threadIdx.x, warp = r >> 5;
  *reinterpret_cast<uint4 *>(sm + SM_XA + opnd_off(r, 0, 0)) = make_uint4(xw[0], xw[1], xw[2], xw[3]);
  *reinterpret_cast<uint4 *>(sm + SM_XA + opnd_off(r, 8, 0)) = make_uint4(xw[4], xw[5], xw[6], xw[7]);
  fence_async();
  tc_before();
  __syncthreads();
  const uint32_t bar = su32(sm + SM_BAR);
  if (r == 0) {
    tc_after();
    mma(tmem, sdesc(su32(sm + SM_XA)), sdesc(su32(sm + SM_W1)), kIdesc1, 0);
    commit(bar);
  }
  bool ok = bar_wait(bar, ph);
  ph ^= 1u;
  if (!__syncthreads_and(ok)) return false;
  tc_after();
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
  const float *b1 = reinterpret_cast<const float *>(sm + SM_B1);
  uint64_t msk = 0;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float d[32];
    tmem_ld32(lane_base + 32 * half, d);
    tmem_wait_ld();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t h[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int jj = 8 * q + 2 * u, j = 32 * half + jj;
        const float a = d[jj] + b1[j], b = d[jj + 1] + b1[j + 1];
        if (MASK) msk |= (uint64_t)(a > 0.f) << j | (uint64_t)(b > 0.f) << (j + 1);
        h[u] = cvt_bf16x2<true>(a, b);
      }
      *reinterpret_cast<uint4 *>(sm + SM_HA + opnd_off(r, 32 * half + 8 * q, 4096)) =
          make_uint4(h[0], h[1], h[2], h[3]);
    }
  }
  if (MASK) *mask = msk;
  fence_async();
  tc_before();
  __syncthreads();
  if (r == 0) {
    tc_after();
#pragma unroll
    for (int c = 0; c < kHid / 16; ++c)
      mma(tmem, sdesc(su32(sm + SM_HA + c * 4096)), sdesc(su32(sm + SM_W2 + c * 512)), kIdesc2,
          c > 0 ? 1u : 0u);
    commit(bar);
  }
  ok = bar_wait(bar, ph);
  ph ^= 1u;
  if (!__syncthreads_and(ok)) return false;
  tc_after();
  tmem_ld4(lane_base, out);
  tmem_wait_ld();
  const float *b2 = reinterpret_cast<const float *>(sm + SM_PRM) + 36;
#pragma unroll
  for (int m = 0; m < kNOut; ++m) out[m] += b2[m];
  return true;
}

// ------------------------------------------------------------ node side
struct NodeArgs {
  int64_t N;
  int32_t C;
  const float2 *g, *t0, *t1, *t2;  // input and the three taps
  const dfl *dsum, *psum;
  const int32_t *hbin;
  const double *phi;
  const float *cw, *ch;
  const uint8_t *nkind;
  const float2 *fixedp;
  const float4 *bounds;
  float sx, sy, cx, cy, rnd, gamma, omg;
  float isx, isy, ilam, iba;  // 1 / bin width, 1 / bin height, 1 / lambda_up, 1 / bin area
  int clamp;
  const float *w;
  float2 *out;
  int *status;
  // records
  const float2 *tgt;
  float *rec;
  const int32_t *boff;
};

struct NodeIn {
  float G[3][2];  // taps in bin units about the centre
  float f[kNF];   // raw features
};

// The taps in bin units and the raw features of node v (FP32).
__device__ __forceinline__ void node_in(const NodeArgs &A, int64_t v, NodeIn &q) {
  const float2 t[3] = {A.t0[v], A.t1[v], A.t2[v]};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    q.G[i][0] = (t[i].x - A.cx) * A.isx;
    q.G[i][1] = (t[i].y - A.cy) * A.isy;
  }
  const uint8_t kd = A.nkind[v];
  const dfl D = A.dsum[v], Pp = A.psum[v];
  const float d = D.hi + D.lo, p = Pp.hi + Pp.lo;
  int hb = -1;
  float area = 0.f;
  if (v < A.C) {
    hb = A.hbin[v];
    if (kd == 0) area = (A.cw[v] * A.ch[v]) * A.iba;
  }
  q.f[0] = q.G[1][0] - q.G[0][0];
  q.f[1] = q.G[1][1] - q.G[0][1];
  q.f[2] = q.G[2][0] - q.G[0][0];
  q.f[3] = q.G[2][1] - q.G[0][1];
  q.f[4] = d * A.ilam;
  q.f[5] = (2.f * p - d) * A.ilam;
  q.f[6] = (d - p) * A.ilam;
  q.f[7] = hb >= 0 ? (float)A.phi[hb] : 0.f;
  q.f[8] = hb >= 0 ? 1.f : 0.f;
  q.f[9] = kd == 1 ? 1.f : 0.f;
  q.f[10] = area;
  q.f[11] = A.rnd;
#pragma unroll
  for (int k = 12; k < kNF; ++k) q.f[k] = 0.f;
}

// Persistent: CTA b takes tiles b, b + grid, ...
__global__ void __launch_bounds__(kTile, 8) k_learned_apply(NodeArgs A) {
  uint8_t *sm = smem_base();
  const uint32_t tmem = tc_setup(sm, A.w);
  const float *prm = reinterpret_cast<const float *>(sm + SM_PRM);
  uint32_t ph = 0;
  const long long ntiles = (A.N + kTile - 1) / kTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t v = tile * kTile + threadIdx.x;
    const bool live = v < A.N;
    NodeIn q;
    uint8_t kd = 2;
    float2 g = make_float2(0.f, 0.f);
    float4 bd = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
      node_in(A, v, q);
      // the round's end reads these: loaded now, in flight during the MMAs
      kd = A.nkind[v];
      g = A.g[v];
      if (A.clamp) bd = A.bounds[v];
    } else {
#pragma unroll
      for (int k = 0; k < kNF; ++k) q.f[k] = 0.f;
    }
    uint32_t xw[8];
    normalise(sm, q.f, xw);
    float o[kNOut];
    if (!tc_tile<false>(sm, tmem, ph, xw, o, nullptr)) {
      if (threadIdx.x == 0) flag(A.status, ST_TIMEOUT);
      break;
    }
    if (!live) continue;
    float gt[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float G0 = q.G[0][c], G1 = q.G[1][c], G2 = q.G[2][c];
      float P = prm[32] * G0 + prm[33] * G1;
      P += prm[34] * G2;
      P += o[0] * (G1 - G0);
      P += o[1] * (G2 - G0);
      P += o[2 + c];
      gt[c] = c ? A.cy + A.sy * P : A.cx + A.sx * P;
    }
    float2 r;
    if (kd == 2) {
      r = A.fixedp[v];
    } else {
      if (!isfinite(gt[0]) || !isfinite(gt[1])) flag(A.status, ST_LEARNED_NF);
      r.x = A.omg * g.x + A.gamma * gt[0];
      r.y = A.omg * g.y + A.gamma * gt[1];
      if (A.clamp) {
        r.x = fminf(fmaxf(r.x, bd.x), bd.z);
        r.y = fminf(fmaxf(r.y, bd.y), bd.w);
      }
    }
    A.out[v] = r;
  }
  tc_teardown(tmem);
}

// The MLP alone on given raw features (n x 16 floats) -> n x 4 floats.
__global__ void __launch_bounds__(kTile, 8) k_learned_forward(const float *w, const float *feat,
                                                              int64_t n, float *out) {
  uint8_t *sm = smem_base();
  const uint32_t tmem = tc_setup(sm, w);
  uint32_t ph = 0;
  const long long ntiles = (n + kTile - 1) / kTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i = tile * kTile + threadIdx.x;
    float f[kNF];
    if (i < n) {
      const float4 *fp = reinterpret_cast<const float4 *>(feat + i * kNF);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 a = fp[u];
        f[4 * u] = a.x;
        f[4 * u + 1] = a.y;
        f[4 * u + 2] = a.z;
        f[4 * u + 3] = a.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kNF; ++k) f[k] = 0.f;
    }
    uint32_t xw[8];
    normalise(sm, f, xw);
    float o[kNOut];
    const bool ok = tc_tile<false>(sm, tmem, ph, xw, o, nullptr);
    if (!ok) o[0] = o[1] = o[2] = o[3] = __int_as_float(0x7fc00000);
    if (i < n) reinterpret_cast<float4 *>(out)[i] = make_float4(o[0], o[1], o[2], o[3]);
    if (!ok) break;
  }
  tc_teardown(tmem);
}

// ------------------------------------------------------------- records
// Free nodes (kind != 2) per block of 1024 nodes.
__global__ void k_free_count(int64_t N, const uint8_t *nkind, int32_t *cnt) {
  __shared__ int ws[8];
  const int64_t base = (int64_t)blockIdx.x * 1024;
  int c = 0;
  for (int u = 0; u < 4; ++u) {
    const int64_t v = base + threadIdx.x + 256 * u;
    c += (v < N && nkind[v] != 2) ? 1 : 0;
  }
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int k = 0; k < 8; ++k) s += ws[k];
    cnt[blockIdx.x] = s;
  }
}

// Exclusive scan of nb counts in place, total at [nb] (one block).
__global__ void k_free_scan(int32_t nb, int32_t *cnt) {
  __shared__ int32_t sh[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int32_t b0 = 0; b0 < nb; b0 += 1024) {
    const int32_t i = b0 + threadIdx.x;
    const int32_t x = i < nb ? cnt[i] : 0;
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
      const int32_t y = threadIdx.x >= d ? sh[threadIdx.x - d] : 0;
      __syncthreads();
      sh[threadIdx.x] += y;
      __syncthreads();
    }
    const int32_t incl = sh[threadIdx.x];
    if (i < nb) cnt[i] = carry + incl - x;
    __syncthreads();
    if (threadIdx.x == 1023) carry += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) cnt[nb] = carry;
}

// One record per free node, in node order: block b (1024 nodes) writes from
// boff[b].
__global__ void __launch_bounds__(1024) k_collect(NodeArgs A) {
  __shared__ int32_t wsum[32];
  const int64_t v = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  const bool fr = v < A.N && A.nkind[v] != 2;
  const unsigned bal = __ballot_sync(0xffffffffu, fr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wsum[warp] = __popc(bal);
  __syncthreads();
  int off = 0;
  for (int k = 0; k < warp; ++k) off += wsum[k];
  if (!fr) return;
  const int64_t idx = (int64_t)A.boff[blockIdx.x] + off + __popc(bal & ((1u << lane) - 1u));
  NodeIn q;
  node_in(A, v, q);
  const float2 t = A.tgt[v];
  float *r = A.rec + idx * kRec;
  float4 *r4 = reinterpret_cast<float4 *>(r);
  r4[0] = make_float4(q.f[0], q.f[1], q.f[2], q.f[3]);
  r4[1] = make_float4(q.f[4], q.f[5], q.f[6], q.f[7]);
  r4[2] = make_float4(q.f[8], q.f[9], q.f[10], q.f[11]);
  r4[3] = make_float4(q.f[12], q.f[13], q.f[14], q.f[15]);
  r4[4] = make_float4(q.G[0][0], q.G[0][1], q.G[1][0], q.G[1][1]);
  // the target: the filter output that the relaxation maps to the plain
  // round's result g' (clamping included), (g' - (1 - gamma) g) / gamma
  const float2 g = A.g[v];
  const float tx = (t.x - A.omg * g.x) / A.gamma, ty = (t.y - A.omg * g.y) / A.gamma;
  r4[5] = make_float4(q.G[2][0], q.G[2][1], (tx - A.cx) / A.sx, (ty - A.cy) / A.sy);
}

// ------------------------------------------------------------- training
struct RecIn {
  float f[kNF];
  float G[3][2];
  float T[2];
};

__device__ __forceinline__ void load_rec(const float *rec, int64_t i, RecIn &q) {
  const float4 *r4 = reinterpret_cast<const float4 *>(rec + i * kRec);
  float a[kRec];
#pragma unroll
  for (int u = 0; u < kRec / 4; ++u) {
    const float4 x = r4[u];
    a[4 * u] = x.x;
    a[4 * u + 1] = x.y;
    a[4 * u + 2] = x.z;
    a[4 * u + 3] = x.w;
  }
#pragma unroll
  for (int k = 0; k < kNF; ++k) q.f[k] = a[k];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    q.G[i][0] = a[16 + 2 * i];
    q.G[i][1] = a[17 + 2 * i];
  }
  q.T[0] = a[22];
  q.T[1] = a[23];
}

// One tile of records per CTA: the loss and its gradient over the tile,
// summed in thread order into part[blockIdx.x] (gradient of weight i at
// index i, the loss at kLW).  Tile: tiles[blockIdx.x], or tile0 + blockIdx.x
// when tiles is NULL.  inv_n: 1 / (records the loss is averaged over).
__global__ void __launch_bounds__(kTile) k_train_tile(const float *rec, int64_t nrec,
                                                      const int32_t *tiles, int64_t tile0,
                                                      float inv_n, const float *w, float *part,
                                                      int *status) {
  uint8_t *sm = smem_base();
  const uint32_t tmem = tc_setup(sm, w);
  const float *prm = reinterpret_cast<const float *>(sm + SM_PRM);
  const int t = threadIdx.x;
  const int64_t tile = tiles ? (int64_t)tiles[blockIdx.x] : tile0 + blockIdx.x;
  const int64_t i = tile * kTile + t;
  const bool live = i < nrec;
  RecIn q;
  if (live) {
    load_rec(rec, i, q);
  } else {
#pragma unroll
    for (int k = 0; k < kNF; ++k) q.f[k] = 0.f;
    q.G[0][0] = q.G[0][1] = q.G[1][0] = q.G[1][1] = q.G[2][0] = q.G[2][1] = q.T[0] = q.T[1] = 0.f;
  }
  uint32_t xw[8];
  normalise(sm, q.f, xw);
  float o[kNOut];
  uint64_t pos = 0;
  uint32_t ph = 0;
  const bool ok = tc_tile<true>(sm, tmem, ph, xw, o, &pos);
  if (!ok) {
    if (t == 0) flag(status, ST_TIMEOUT);
    tc_teardown(tmem);
    return;
  }
  float *dh = reinterpret_cast<float *>(sm + SM_DH);
  float *xs = reinterpret_cast<float *>(sm + SM_XS);
  float *dout = reinterpret_cast<float *>(sm + SM_DO);
  float *gth = reinterpret_cast<float *>(sm + SM_GT);
  const float *w2f = reinterpret_cast<const float *>(sm + SM_W2F);
  float dP[2] = {0.f, 0.f}, l = 0.f;
  if (live) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float G0 = q.G[0][c], G1 = q.G[1][c], G2 = q.G[2][c];
      float P = prm[32] * G0 + prm[33] * G1;
      P += prm[34] * G2;
      P += o[0] * (G1 - G0);
      P += o[1] * (G2 - G0);
      P += o[2 + c];
      const float e = P - q.T[c];
      l += e * e;
      dP[c] = 2.f * e * inv_n;
    }
  }
  float d[kNOut];
  d[0] = dP[0] * (q.G[1][0] - q.G[0][0]) + dP[1] * (q.G[1][1] - q.G[0][1]);
  d[1] = dP[0] * (q.G[2][0] - q.G[0][0]) + dP[1] * (q.G[2][1] - q.G[0][1]);
  d[2] = dP[0];
  d[3] = dP[1];
#pragma unroll
  for (int m = 0; m < kNOut; ++m) dout[t * 4 + m] = d[m];
  gth[t * 4 + 0] = dP[0] * q.G[0][0] + dP[1] * q.G[0][1];
  gth[t * 4 + 1] = dP[0] * q.G[1][0] + dP[1] * q.G[1][1];
  gth[t * 4 + 2] = dP[0] * q.G[2][0] + dP[1] * q.G[2][1];
  gth[t * 4 + 3] = l * inv_n;
#pragma unroll
  for (int j = 0; j < kHid; ++j) {
    float s = d[0] * w2f[j];
    s += d[1] * w2f[kHid + j];
    s += d[2] * w2f[2 * kHid + j];
    s += d[3] * w2f[3 * kHid + j];
    dh[t * kDhS + j] = (pos >> j) & 1u ? s : 0.f;
  }
#pragma unroll
  for (int k = 0; k < kNF; k += 2) {
    xs[t * kXsS + k] = bf16_to_f((uint16_t)(xw[k / 2] & 0xffffu));
    xs[t * kXsS + k + 1] = bf16_to_f((uint16_t)(xw[k / 2] >> 16));
  }
  __syncthreads();
  float *row = part + (int64_t)blockIdx.x * kPart;
  constexpr int nout = kHid * kNF + kHid + kNOut * kHid + kNOut + 3 + 1;
  for (int oi = t; oi < nout; oi += kTile) {
    float s = 0.f;
    int dst;
    if (oi < kHid * kNF) {
      const int j = oi / kNF, k = oi % kNF;
      for (int r = 0; r < kTile; ++r) s += dh[r * kDhS + j] * xs[r * kXsS + k];
      dst = kW1 + oi;
    } else if (oi < kHid * kNF + kHid) {
      const int j = oi - kHid * kNF;
      for (int r = 0; r < kTile; ++r) s += dh[r * kDhS + j];
      dst = kB1 + j;
    } else if (oi < kHid * kNF + kHid + kNOut * kHid) {
      const int u = oi - kHid * kNF - kHid, m = u / kHid, j = u % kHid;
      for (int r = 0; r < kTile; ++r)
        s += dout[r * 4 + m] * bf16_to_f(*reinterpret_cast<const uint16_t *>(sm + SM_HA + opnd_off(r, j, 4096)));
      dst = kW2 + u;
    } else if (oi < kHid * kNF + kHid + kNOut * kHid + kNOut) {
      const int m = oi - (kHid * kNF + kHid + kNOut * kHid);
      for (int r = 0; r < kTile; ++r) s += dout[r * 4 + m];
      dst = kB2 + m;
    } else {
      const int m = oi - (kHid * kNF + kHid + kNOut * kHid + kNOut);  // 0..2 theta, 3 loss
      for (int r = 0; r < kTile; ++r) s += gth[r * 4 + m];
      dst = m < 3 ? kTH + m : kLW;
    }
    row[dst] = s;
  }
  tc_teardown(tmem);
}

// acc[i] (+)= sum over blocks b (in order) of part[b][i], for the trained
// weights and the loss (i >= kTH).
__global__ void k_reduce_parts(const float *part, int nblk, double *acc, int first) {
  const int i = kTH + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kPart) return;
  double s = first ? 0.0 : acc[i];
  for (int b = 0; b < nblk; ++b) s += (double)part[(int64_t)b * kPart + i];
  acc[i] = s;
}

// One Adam step on every trained weight from the summed gradient; the
// minibatch loss is added to *loss.
__global__ void k_adam(const double *acc, float *w, float *m, float *v, float lr, float b1,
                       float b2, float eps, float bc1, float bc2, double *loss) {
  const int i = kTH + blockIdx.x * blockDim.x + threadIdx.x;
  if (i == kLW) *loss += acc[kLW];
  if (i >= kLW) return;
  const float g = (float)acc[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void k_acc_to_grad(const double *acc, float *grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kLW) grad[i] = i < kTH ? 0.f : (float)acc[i];
}

// Per-block FP64 sums over records: sum f_k, sum f_k^2, and the normal
// equations of the taps (A = sum G G^T over both axes, 6 entries; b = sum G T).
__global__ void k_rec_stats(const float *rec, int64_t nrec, double *part) {
  double s[kStats];
#pragma unroll
  for (int k = 0; k < kStats; ++k) s[k] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrec;
       i += (int64_t)gridDim.x * blockDim.x) {
    RecIn q;
    load_rec(rec, i, q);
#pragma unroll
    for (int k = 0; k < kNF; ++k) {
      const double f = q.f[k];
      s[k] += f;
      s[16 + k] += f * f;
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const double a = q.G[0][c], b = q.G[1][c], d = q.G[2][c], T = q.T[c];
      s[32] += a * a;
      s[33] += a * b;
      s[34] += a * d;
      s[35] += b * b;
      s[36] += b * d;
      s[37] += d * d;
      s[38] += a * T;
      s[39] += b * T;
      s[40] += d * T;
    }
  }
  __shared__ double sh[256];
#pragma unroll
  for (int k = 0; k < kStats; ++k) {
    sh[threadIdx.x] = s[k];
    __syncthreads();
    for (int d = 128; d > 0; d >>= 1) {
      if (threadIdx.x < d) sh[threadIdx.x] += sh[threadIdx.x + d];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * kStats + k] = sh[0];
    __syncthreads();
  }
}

__global__ void k_stats_final(const double *part, int nblk, double *out) {
  const int k = threadIdx.x;
  if (k >= kStats) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * kStats + k];
  out[k] = s;
}

// ------------------------------------------------------------- host side
uint64_t splitmix(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int device_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
    n = 152;
  return n;
}

cudaError_t smem_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_learned_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFwd);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_learned_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFwd);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_train_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTrain);
  return e;
}

// Node-side arguments of the current round on graph g.
NodeArgs node_args(pl_graph *g, const pl_params *p, int32_t round) {
  NodeArgs A{};
  A.N = g->N;
  A.C = g->C;
  A.dsum = P<dfl>(g->hm.dsum);
  A.psum = P<dfl>(g->hm.psum);
  A.hbin = P<int32_t>(g->hbin);
  A.phi = P<double>(g->phi);
  A.cw = P<float>(g->cw);
  A.ch = P<float>(g->ch);
  A.nkind = P<uint8_t>(g->nkind);
  A.fixedp = P<float2>(g->fixedp);
  A.bounds = P<float4>(g->bounds);
  A.sx = (float)g->wb;
  A.sy = (float)g->hb;
  A.cx = (float)(0.5 * (g->xl + g->xh));
  A.cy = (float)(0.5 * (g->yl + g->yh));
  A.isx = (float)(1.0 / g->wb);
  A.isy = (float)(1.0 / g->hb);
  A.iba = (float)(1.0 / ((double)A.sx * (double)A.sy));
  A.ilam = (float)g->lam_h[1];
  A.rnd = p->t_hint > 0 ? (float)round / (float)p->t_hint : 0.f;
  A.gamma = (float)p->gamma;
  A.omg = (float)(1.0 - p->gamma);
  A.clamp = p->clamp;
  A.status = P<int>(g->status);
  return A;
}

pl_status status_word(pl_graph *g, cudaStream_t s, int *w0) {
  TRY(cudaMemcpyAsync(w0, g->status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  return PL_OK;
}

}  // namespace

pl_status check_model(const pl_learned *m) {
  if (!m || !m->w) { set_error("learned model or its weights are NULL"); return PL_ERR_INVALID_ARG; }
  if (m->k[0] < 0 || m->k[1] <= m->k[0] || m->k[2] <= m->k[1] || m->k[2] > 64) {
    set_error("learned tap powers must satisfy 0 <= k0 < k1 < k2 <= 64");
    return PL_ERR_INVALID_ARG;
  }
  return PL_OK;
}

// One learned round (powers, then the fused kernel).  Does not read the status.
pl_status run_learned(pl_graph *g, const pl_params *p, const pl_learned *m, int32_t round,
                      const float *in, float *out, cudaStream_t s) {
  if (p->gamma == 0.0) return clamp_nodes(g, p, in, out, s);
  const float2 *t[3];
  pl_status st = run_powers(g, p, in, m->k, t, s);
  if (st != PL_OK) return st;
  NodeArgs A = node_args(g, p, round);
  A.g = reinterpret_cast<const float2 *>(in);
  A.t0 = t[0];
  A.t1 = t[1];
  A.t2 = t[2];
  A.w = m->w;
  A.out = reinterpret_cast<float2 *>(out);
  TRY(smem_attrs());
  const long long ntiles = (g->N + kTile - 1) / kTile;
  const long long cap = 8LL * device_sms();
  const int grid = (int)std::max(1LL, std::min(ntiles, cap));
  k_learned_apply<<<grid, kTile, kSmemFwd, s>>>(A);
  note_launch();
  TRY(cudaGetLastError());
  return PL_OK;
}

}  // namespace pl

using namespace pl;

extern "C" {

pl_status pl_learned_apply(pl_graph *g, const pl_params *p, const pl_learned *m, int32_t round,
                           const float *xy_in, float *xy_out, pl_stream stream) {
  clear_error();
  if (!g || !p || !xy_in || !xy_out || xy_in == xy_out) { set_error("bad arguments (NULL or in == out)"); return PL_ERR_INVALID_ARG; }
  pl_status st = check_model(m);
  if (st != PL_OK) return st;
  if (!g->have_hints) { set_error("no augmented graph: call pl_build_hints first"); return PL_ERR_INVALID_ARG; }
  if (p->nbx != g->nbx || p->nby != g->nby || p->wdtype != g->wdtype) { set_error("bins and weight type must match the graph build"); return PL_ERR_INVALID_ARG; }
  if (p->gamma < 0.0 || p->gamma > 1.0) { set_error("gamma must be in [0, 1]"); return PL_ERR_INVALID_ARG; }
  ArenaScope scope(&g->arena);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  g->stream = s;
  cudaError_t e = cudaMemsetAsync(g->status.p, 0, 4, s);
  if (e != cudaSuccess) return cuda_fail(e, "status reset");
  st = run_learned(g, p, m, round, xy_in, xy_out, s);
  if (st != PL_OK) return st;
  int w0 = 0;
  st = status_word(g, s, &w0);
  if (st != PL_OK) return st;
  if (w0 & ST_TIMEOUT) { set_error("a bounded device-side wait gave up"); return PL_ERR_TIMEOUT; }
  if (w0 & (ST_LEARNED_NF | ST_NONFINITE)) { set_error("the learned filter's output is not finite"); return PL_ERR_NONFINITE; }
  return PL_OK;
}

pl_status pl_learned_wait_check(int64_t cycles, void *ws, size_t ws_bytes, pl_stream stream) {
  clear_error();
  if (cycles < 1 || cycles > kWaitCycles) { set_error("cycles must be in 1..4e9"); return PL_ERR_INVALID_ARG; }
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) { set_error("workspace must be non-NULL and 256-byte aligned"); return PL_ERR_INVALID_ARG; }
  if (ws_bytes < 8192) { set_error("workspace too small: need 8192 bytes"); return PL_ERR_WORKSPACE; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TRY(cudaFuncSetAttribute(k_wait_check, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFwd));
  // the workspace: a zero parameter vector, then the status word
  float *w = static_cast<float *>(ws);
  int *status = reinterpret_cast<int *>(static_cast<char *>(ws) + 6144);
  TRY(cudaMemsetAsync(ws, 0, 8192, s));
  k_wait_check<<<1, kTile, kSmemFwd, s>>>((long long)cycles, w, status);
  note_launch();
  TRY(cudaGetLastError());
  int sw = 0;
  TRY(cudaMemcpyAsync(&sw, status, 4, cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (sw & ST_TIMEOUT) { set_error("a bounded device-side wait gave up"); return PL_ERR_TIMEOUT; }
  return PL_OK;
}

pl_status pl_learned_forward(const float *w, const float *feat, int64_t n, float *out,
                             pl_stream stream) {
  clear_error();
  if (!w || n < 0 || (n && (!feat || !out))) { set_error("bad arguments"); return PL_ERR_INVALID_ARG; }
  if (n == 0) return PL_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TRY(smem_attrs());
  const long long ntiles = (n + kTile - 1) / kTile;
  const int grid = (int)std::min(ntiles, 8LL * device_sms());
  k_learned_forward<<<grid, kTile, kSmemFwd, s>>>(w, feat, n, out);
  note_launch();
  TRY(cudaGetLastError());
  return PL_OK;
}

pl_status pl_learned_collect(pl_graph *g, const pl_params *p, const int32_t k[3], int32_t round,
                             const float *xy_in, float *rec, int64_t cap, int64_t *count,
                             pl_stream stream) {
  clear_error();
  if (!g || !p || !k || !xy_in || !count || cap < 0 || (cap && !rec)) { set_error("bad arguments"); return PL_ERR_INVALID_ARG; }
  pl_learned m{{k[0], k[1], k[2]}, reinterpret_cast<const float *>(rec ? rec : xy_in)};
  pl_status st = check_model(&m);
  if (st != PL_OK) return st;
  if (!g->have_hints) { set_error("no augmented graph: call pl_build_hints first"); return PL_ERR_INVALID_ARG; }
  if (p->nbx != g->nbx || p->nby != g->nby || p->wdtype != g->wdtype) { set_error("bins and weight type must match the graph build"); return PL_ERR_INVALID_ARG; }
  if (!(p->gamma > 0.0 && p->gamma <= 1.0)) { set_error("records need a relaxation gamma in (0, 1]"); return PL_ERR_INVALID_ARG; }
  ArenaScope scope(&g->arena);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  g->stream = s;
  const int64_t N = g->N;
  const int32_t nb = (int32_t)((N + 1023) / 1024);
  int32_t *cnt = P<int32_t>(g->lscr);
  k_free_count<<<std::max(nb, 1), 256, 0, s>>>(N, P<uint8_t>(g->nkind), cnt);
  k_free_scan<<<1, 1024, 0, s>>>(nb, cnt);
  note_launch();
  note_launch();
  int32_t total = 0;
  TRY(cudaMemcpyAsync(&total, cnt + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  *count = total;
  if (total > cap) { set_error("record buffer too small: %d records needed", (int)total); return PL_ERR_WORKSPACE; }
  // the plain round's result g' (relaxation, re-pinning, clamping) into q4a
  float *tgt = P<float>(g->q4a);
  TRY(cudaMemsetAsync(g->status.p, 0, 4, s));
  st = run_filter(g, p, xy_in, tgt, s);
  if (st != PL_OK) return st;
  const float2 *t[3];
  st = run_powers(g, p, xy_in, k, t, s);
  if (st != PL_OK) return st;
  NodeArgs A = node_args(g, p, round);
  A.t0 = t[0];
  A.t1 = t[1];
  A.t2 = t[2];
  A.g = reinterpret_cast<const float2 *>(xy_in);
  A.tgt = reinterpret_cast<const float2 *>(tgt);
  A.rec = rec;
  A.boff = cnt;
  if (total) {
    k_collect<<<nb, 1024, 0, s>>>(A);
    note_launch();
  }
  TRY(cudaGetLastError());
  int w0 = 0;
  st = status_word(g, s, &w0);
  if (st != PL_OK) return st;
  if (w0 & ST_NONFINITE) { set_error("non-finite coordinate"); return PL_ERR_NONFINITE; }
  return PL_OK;
}

void pl_train_opts_default(pl_train_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->epochs = 20;
  o->batch_tiles = 128;
  o->lr = 2e-3;
  o->lr_min = 1e-4;
  o->beta1 = 0.9;
  o->beta2 = 0.999;
  o->eps = 1e-8;
  o->seed = 1;
  o->fit_norm = 1;
  o->fit_taps = 1;
}

namespace {
struct TrainWs {
  float *part;
  double *acc;
  float *m, *v;
  int32_t *tiles;
  double *spart, *sout, *loss;
};
size_t rup(size_t b) { return (b + 255) / 256 * 256; }
size_t train_ws(int64_t nrec, TrainWs *w, uint8_t *base) {
  const int64_t ntiles = (nrec + kTile - 1) / kTile;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    uint8_t *p = base ? base + off : nullptr;
    off += rup(bytes);
    return p;
  };
  TrainWs t;
  t.part = reinterpret_cast<float *>(take((size_t)kMaxBatch * kPart * 4));
  t.acc = reinterpret_cast<double *>(take((size_t)kPart * 8));
  t.m = reinterpret_cast<float *>(take((size_t)kLW * 4));
  t.v = reinterpret_cast<float *>(take((size_t)kLW * 4));
  t.tiles = reinterpret_cast<int32_t *>(take((size_t)std::max<int64_t>(ntiles, 1) * 4));
  t.spart = reinterpret_cast<double *>(take((size_t)kMaxBatch * kStats * 8));
  t.sout = reinterpret_cast<double *>(take((size_t)kStats * 8));
  t.loss = reinterpret_cast<double *>(take(8));
  if (w) *w = t;
  return off;
}

pl_status check_ws(int64_t nrec, void *ws, size_t ws_bytes, TrainWs *w) {
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) { set_error("workspace must be non-NULL and 256-byte aligned"); return PL_ERR_INVALID_ARG; }
  const size_t need = train_ws(nrec, w, reinterpret_cast<uint8_t *>(ws));
  if (ws_bytes < need) { set_error("workspace too small: need %zu bytes", need); return PL_ERR_WORKSPACE; }
  return PL_OK;
}

// mu, isd and / or theta from the records (FP64 sums on the device, the 3 x 3
// normal equations solved here by Gaussian elimination with partial pivoting).
pl_status fit_start(const float *rec, int64_t nrec, float *w, const pl_train_opts *o,
                    const TrainWs &W, cudaStream_t s) {
  const int nblk = (int)std::min<int64_t>(kMaxBatch, std::max<int64_t>(1, (nrec + 255) / 256));
  k_rec_stats<<<nblk, 256, 0, s>>>(rec, nrec, W.spart);
  k_stats_final<<<1, 64, 0, s>>>(W.spart, nblk, W.sout);
  note_launch();
  note_launch();
  double S[kStats];
  TRY(cudaMemcpyAsync(S, W.sout, sizeof(S), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (o->fit_norm) {
    float mu[kNF], isd[kNF];
    for (int k = 0; k < kNF; ++k) {
      const double m = S[k] / (double)nrec;
      const double sd = std::sqrt(std::max(S[16 + k] / (double)nrec - m * m, 0.0));
      mu[k] = (float)m;
      isd[k] = sd > 1e-12 * (1.0 + std::fabs(m)) ? (float)(1.0 / sd) : 1.f;
    }
    TRY(cudaMemcpyAsync(w + kMU, mu, sizeof(mu), cudaMemcpyHostToDevice, s));
    TRY(cudaMemcpyAsync(w + kISD, isd, sizeof(isd), cudaMemcpyHostToDevice, s));
    TRY(cudaStreamSynchronize(s));
  }
  if (o->fit_taps) {
    double a[3][4] = {{S[32], S[33], S[34], S[38]},
                      {S[33], S[35], S[36], S[39]},
                      {S[34], S[36], S[37], S[40]}};
    for (int c = 0; c < 3; ++c) {
      int piv = c;
      for (int r = c + 1; r < 3; ++r)
        if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
      if (!(std::fabs(a[piv][c]) > 0.0)) { set_error("the taps' normal equations are singular"); return PL_ERR_INVALID_ARG; }
      for (int k = 0; k < 4; ++k) std::swap(a[c][k], a[piv][k]);
      for (int r = c + 1; r < 3; ++r) {
        const double f = a[r][c] / a[c][c];
        for (int k = c; k < 4; ++k) a[r][k] -= f * a[c][k];
      }
    }
    double th[3];
    for (int c = 2; c >= 0; --c) {
      double v = a[c][3];
      for (int k = c + 1; k < 3; ++k) v -= a[c][k] * th[k];
      th[c] = v / a[c][c];
    }
    const float thf[3] = {(float)th[0], (float)th[1], (float)th[2]};
    TRY(cudaMemcpyAsync(w + kTH, thf, sizeof(thf), cudaMemcpyHostToDevice, s));
    TRY(cudaStreamSynchronize(s));
  }
  return PL_OK;
}
}  // namespace

size_t pl_learned_train_ws(int64_t nrec) {
  if (nrec < 0) return 0;
  return train_ws(nrec, nullptr, nullptr);
}

pl_status pl_learned_train(const float *rec, int64_t nrec, float *w, const pl_train_opts *o,
                           void *ws, size_t ws_bytes, double *epoch_loss, pl_stream stream) {
  clear_error();
  if (!rec || !w || !o || nrec < kTile) { set_error("bad arguments (NULL, or fewer than 128 records)"); return PL_ERR_INVALID_ARG; }
  if (o->epochs < 1 || o->batch_tiles < 1 || o->batch_tiles > kMaxBatch || !(o->lr > 0.0) ||
      !(o->lr_min >= 0.0) || !(o->beta1 >= 0.0 && o->beta1 < 1.0) ||
      !(o->beta2 >= 0.0 && o->beta2 < 1.0) || !(o->eps > 0.0)) {
    set_error("bad training options");
    return PL_ERR_INVALID_ARG;
  }
  TrainWs W;
  pl_status st = check_ws(nrec, ws, ws_bytes, &W);
  if (st != PL_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TRY(smem_attrs());
  TRY(cudaMemsetAsync(W.part, 0, (size_t)kMaxBatch * kPart * 4, s));
  if (o->fit_norm || o->fit_taps) {
    st = fit_start(rec, nrec, w, o, W, s);
    if (st != PL_OK) return st;
  }
  TRY(cudaMemsetAsync(W.m, 0, kLW * 4, s));
  TRY(cudaMemsetAsync(W.v, 0, kLW * 4, s));
  int *status = reinterpret_cast<int *>(W.spart);  // a word of scratch for the status
  TRY(cudaMemsetAsync(status, 0, 4, s));
  const int64_t nfull = nrec / kTile;
  const int bt = (int)std::min<int64_t>(o->batch_tiles, nfull);
  const int64_t spe = nfull / bt;
  const int64_t total = (int64_t)o->epochs * spe;
  std::vector<int32_t> order((size_t)nfull);
  const int rgrid = (kPart - kTH + 127) / 128;
  int64_t step = 0;
  for (int ep = 0; ep < o->epochs; ++ep) {
    for (int64_t i = 0; i < nfull; ++i) order[(size_t)i] = (int32_t)i;
    for (int64_t i = nfull - 1; i > 0; --i) {
      const uint64_t j = splitmix(o->seed, ((uint64_t)ep << 40) + (uint64_t)i) % (uint64_t)(i + 1);
      std::swap(order[(size_t)i], order[(size_t)j]);
    }
    TRY(cudaMemcpyAsync(W.tiles, order.data(), (size_t)nfull * 4, cudaMemcpyHostToDevice, s));
    TRY(cudaMemsetAsync(W.loss, 0, 8, s));
    for (int64_t k = 0; k < spe; ++k, ++step) {
      const double lr = o->lr_min + 0.5 * (o->lr - o->lr_min) *
                                        (1.0 + std::cos(3.14159265358979323846 * (double)step / (double)total));
      const double t = (double)(step + 1);
      k_train_tile<<<bt, kTile, kSmemTrain, s>>>(rec, nrec, W.tiles + k * bt, 0,
                                                1.f / (float)(bt * kTile), w, W.part, status);
      k_reduce_parts<<<rgrid, 128, 0, s>>>(W.part, bt, W.acc, 1);
      k_adam<<<rgrid, 128, 0, s>>>(W.acc, w, W.m, W.v, (float)lr, (float)o->beta1,
                                   (float)o->beta2, (float)o->eps,
                                   (float)(1.0 - std::pow(o->beta1, t)),
                                   (float)(1.0 - std::pow(o->beta2, t)), W.loss);
      note_launch();
      note_launch();
      note_launch();
    }
    TRY(cudaGetLastError());
    double l = 0.0;
    int sw = 0;
    TRY(cudaMemcpyAsync(&l, W.loss, 8, cudaMemcpyDeviceToHost, s));
    TRY(cudaMemcpyAsync(&sw, status, 4, cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    if (sw & ST_TIMEOUT) { set_error("a bounded device-side wait gave up"); return PL_ERR_TIMEOUT; }
    if (epoch_loss) epoch_loss[ep] = l / (double)spe;
  }
  return PL_OK;
}

pl_status pl_learned_loss(const float *rec, int64_t nrec, const float *w, void *ws,
                          size_t ws_bytes, double *loss, float *grad, pl_stream stream) {
  clear_error();
  if (!rec || !w || !loss || nrec < 1) { set_error("bad arguments"); return PL_ERR_INVALID_ARG; }
  TrainWs W;
  pl_status st = check_ws(nrec, ws, ws_bytes, &W);
  if (st != PL_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TRY(smem_attrs());
  int *status = reinterpret_cast<int *>(W.spart);
  TRY(cudaMemsetAsync(status, 0, 4, s));
  const int64_t ntiles = (nrec + kTile - 1) / kTile;
  const int rgrid = (kPart - kTH + 127) / 128;
  for (int64_t t0 = 0; t0 < ntiles; t0 += kMaxBatch) {
    const int nb = (int)std::min<int64_t>(kMaxBatch, ntiles - t0);
    k_train_tile<<<nb, kTile, kSmemTrain, s>>>(rec, nrec, nullptr, t0, (float)(1.0 / (double)nrec), w,
                                               W.part, status);
    k_reduce_parts<<<rgrid, 128, 0, s>>>(W.part, nb, W.acc, t0 == 0);
    note_launch();
    note_launch();
  }
  if (grad) {
    k_acc_to_grad<<<(kLW + 127) / 128, 128, 0, s>>>(W.acc, grad);
    note_launch();
  }
  TRY(cudaGetLastError());
  double l = 0.0;
  int sw = 0;
  TRY(cudaMemcpyAsync(&l, W.acc + kLW, 8, cudaMemcpyDeviceToHost, s));
  TRY(cudaMemcpyAsync(&sw, status, 4, cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (sw & ST_TIMEOUT) { set_error("a bounded device-side wait gave up"); return PL_ERR_TIMEOUT; }
  *loss = l;
  return PL_OK;
}

}  // extern "C"
