// A5: half-perimeter wirelength (the quality metric of Sec. VII-VIII):
// sum over nets of (max - min) pin x + (max - min) pin y, pin = cell centre +
// offset.  A thread takes a net of up to 32 pins (a warp stages the pins of 32
// consecutive nets when they fit), a warp a net of up to 1024; each block then
// spans the larger nets of its own range of nets, one at a time with all its
// threads.  Pin positions and extrema are FP32 (min/max are exact); each net's
// span is formed exactly and summed in double-float per thread, the threads'
// sums in FP64.  Per-block sums go to the caller's workspace; the last block
// to finish (ticket) adds them in a fixed order (strided over its threads,
// then a fixed tree), so the result does not depend on scheduling.  A pin
// whose cell index is out of range makes the result NaN (it is not
// dereferenced).
#include <mutex>

#include "pl_internal.h"

namespace pl {

constexpr int kHpwlThreads = 256;
constexpr int kHpwlBlocks = 152 * 8;
constexpr int kHpwlStage = 512;  // pins of one batch of 32 nets staged per warp
constexpr int kHpwlWarpMax = 1024;  // longer nets are spanned by a whole block

// Pin position; a pin_cell outside [0, C) is counted in *bad and reads cell 0
// instead (the call then reports NaN).
__device__ __forceinline__ float2 pin_pos(const float2 *xy, const int32_t *pin_cell,
                                          const float *dx, const float *dy, long long k,
                                          int32_t C, int *bad) {
  int32_t i = pin_cell[k];
  if ((uint32_t)i >= (uint32_t)C) {
    atomicAdd(bad, 1);
    i = 0;
  }
  float2 c = xy[i];
  if (dx) c.x += dx[k];
  if (dy) c.y += dy[k];
  return c;
}

// A net's span (x1 - x0) + (y1 - y0) added to a double-float sum: each
// difference is exact as a TwoSum pair (FP32 arithmetic only).
__device__ __forceinline__ void span_add(dfl &acc, float x0, float x1, float y0, float y1) {
  dfl dx{x1, 0.f}, dy{y1, 0.f};
  df_add(dx, -x0);
  df_add(dy, -y0);
  df_add_df(acc, dx);
  df_add_df(acc, dy);
}

__global__ void __launch_bounds__(kHpwlThreads) k_hpwl(const int64_t *net_ptr,
                                                       const int32_t *pin_cell, const float *dx,
                                                       const float *dy, const float2 *xy,
                                                       int32_t M, int32_t C, double *part,
                                                       int *ticket, double *out) {
  __shared__ double red[kHpwlThreads / 32];
  __shared__ int last;
  __shared__ float2 stage_all[kHpwlThreads / 32][kHpwlStage];
  __shared__ int32_t bigs[kHpwlThreads];
  __shared__ int wcnt[kHpwlThreads / 32];
  __shared__ float4 mm[kHpwlThreads / 32];
  float2 *stg = stage_all[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  dfl acc{0.f, 0.f};
  // each warp takes batches of 32 consecutive nets (warp-uniform loop): a
  // staged batch spans every net in it from shared memory; otherwise a lane
  // spans each net of at most 32 pins and the warp each one of at most
  // kHpwlWarpMax; longer nets are left to the block pass below
  const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = wg * 32; base < M; base += nwarp * 32) {
    const long long e = base + lane;
    const long long p0 = net_ptr[base], p1 = net_ptr[base + 32 < M ? base + 32 : M];
    if (p1 - p0 <= kHpwlStage) {
      // the batch's pins fit the warp's stage: lanes load all of them (all
      // gathers in flight), then each lane spans its own net from the stage
      for (long long k0 = p0; k0 < p1; k0 += 4 * 32) {
        float2 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long long k = k0 + u * 32 + lane;
          if (k < p1) q[u] = pin_pos(xy, pin_cell, dx, dy, k, C, ticket + 1);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long long k = k0 + u * 32 + lane;
          if (k < p1) stg[k - p0] = q[u];
        }
      }
      __syncwarp();
      if (e < M) {
        const long long b = net_ptr[e] - p0, n = net_ptr[e + 1] - net_ptr[e];
        if (n > 0 && n <= kHpwlWarpMax) {
          float2 p = stg[b];
          float x0 = p.x, x1 = p.x, y0 = p.y, y1 = p.y;
          for (long long k = b + 1; k < b + n; ++k) {
            p = stg[k];
            x0 = fminf(x0, p.x); x1 = fmaxf(x1, p.x);
            y0 = fminf(y0, p.y); y1 = fmaxf(y1, p.y);
          }
          span_add(acc, x0, x1, y0, y1);
        }
      }
      __syncwarp();
      continue;
    }
    bool mid = false;
    if (e < M) {
      const long long b = net_ptr[e], n = net_ptr[e + 1] - b;
      if (n > 0 && n <= 32) {
        float2 p = pin_pos(xy, pin_cell, dx, dy, b, C, ticket + 1);
        float x0 = p.x, x1 = p.x, y0 = p.y, y1 = p.y;
        for (long long k = b + 1; k < b + n; ++k) {
          p = pin_pos(xy, pin_cell, dx, dy, k, C, ticket + 1);
          x0 = fminf(x0, p.x); x1 = fmaxf(x1, p.x);
          y0 = fminf(y0, p.y); y1 = fmaxf(y1, p.y);
        }
        span_add(acc, x0, x1, y0, y1);
      }
      mid = n > 32 && n <= kHpwlWarpMax;
    }
    // nets of 33..kHpwlWarpMax pins: the whole warp, one net at a time
    unsigned bm = __ballot_sync(0xffffffffu, mid);
    while (bm) {
      const int src = __ffs(bm) - 1;
      bm &= bm - 1;
      const long long b = net_ptr[base + src], n = net_ptr[base + src + 1] - b;
      float x0 = 3.4e38f, x1 = -3.4e38f, y0 = 3.4e38f, y1 = -3.4e38f;
      for (long long k = b + lane; k < b + n; k += 32) {
        const float2 p = pin_pos(xy, pin_cell, dx, dy, k, C, ticket + 1);
        x0 = fminf(x0, p.x); x1 = fmaxf(x1, p.x);
        y0 = fminf(y0, p.y); y1 = fmaxf(y1, p.y);
      }
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, m));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, m));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, m));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, m));
      }
      if (lane == src) span_add(acc, x0, x1, y0, y1);
    }
  }
  // nets of more than kHpwlWarpMax pins in this block's range of nets, in
  // net order, each spanned by the whole block (strided pins, then a fixed
  // tree)
  double bigacc = 0.0;  // thread 0
  const long long R = ((long long)M + gridDim.x - 1) / gridDim.x;
  const long long r0 = (long long)blockIdx.x * R, r1 = r0 + R < M ? r0 + R : M;
  for (long long c0 = r0; c0 < r1; c0 += kHpwlThreads) {
    const long long e = c0 + threadIdx.x;
    const bool big = e < r1 && net_ptr[e + 1] - net_ptr[e] > kHpwlWarpMax;
    const unsigned bal = __ballot_sync(0xffffffffu, big);
    if (lane == 0) wcnt[wid] = __popc(bal);
    __syncthreads();
    int before = 0, nbig = 0;
    for (int w = 0; w < kHpwlThreads / 32; ++w) {
      before += w < wid ? wcnt[w] : 0;
      nbig += wcnt[w];
    }
    if (big) bigs[before + __popc(bal & ((1u << lane) - 1u))] = (int32_t)e;
    __syncthreads();
    for (int i = 0; i < nbig; ++i) {
      const long long ee = bigs[i], b = net_ptr[ee], n = net_ptr[ee + 1] - b;
      float x0 = 3.4e38f, x1 = -3.4e38f, y0 = 3.4e38f, y1 = -3.4e38f;
      for (long long k = b + threadIdx.x; k < b + n; k += kHpwlThreads) {
        const float2 p = pin_pos(xy, pin_cell, dx, dy, k, C, ticket + 1);
        x0 = fminf(x0, p.x); x1 = fmaxf(x1, p.x);
        y0 = fminf(y0, p.y); y1 = fmaxf(y1, p.y);
      }
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, m));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, m));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, m));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, m));
      }
      if (lane == 0) mm[wid] = make_float4(x0, x1, y0, y1);
      __syncthreads();
      if (threadIdx.x == 0) {
        float4 t = mm[0];
        for (int w = 1; w < kHpwlThreads / 32; ++w) {
          t.x = fminf(t.x, mm[w].x); t.y = fmaxf(t.y, mm[w].y);
          t.z = fminf(t.z, mm[w].z); t.w = fmaxf(t.w, mm[w].w);
        }
        bigacc += ((double)t.y - (double)t.x) + ((double)t.w - (double)t.z);
      }
      __syncthreads();
    }
  }
  const double accd = warp_sum(df_to_d(df_norm(acc)));
  if (lane == 0) red[wid] = accd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kHpwlThreads / 32; ++k) s += red[k];
    part[blockIdx.x] = s + bigacc;
    __threadfence();
    last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  // the last block: thread t adds partials t, t + 256, ... in order, then a
  // fixed tree over the threads
  __threadfence();
  double s = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += kHpwlThreads) s += __ldcg(&part[k]);
  s = warp_sum(s);
  if (lane == 0) red[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kHpwlThreads / 32; ++k) t += red[k];
    *out = __ldcg(ticket + 1) ? __longlong_as_double(0x7ff8000000000000LL) : t;
    ticket[0] = 0;
    ticket[1] = 0;
  }
}

int hpwl_blocks(int32_t M) { return grid_for((long long)M, kHpwlThreads, kHpwlBlocks); }

size_t hpwl_ws_bytes(int32_t M) { return 256 + (size_t)hpwl_blocks(M) * sizeof(double); }

cudaError_t launch_hpwl(const pl_netlist *nl, const float *xy, double *out, void *ws,
                        cudaStream_t s) {
  int nb = hpwl_blocks(nl->num_nets);
  int *ticket = reinterpret_cast<int *>(ws);
  double *part = reinterpret_cast<double *>(static_cast<char *>(ws) + 256);
  k_hpwl<<<nb, kHpwlThreads, 0, s>>>(nl->net_ptr, nl->pin_cell, nl->pin_dx, nl->pin_dy,
                                     reinterpret_cast<const float2 *>(xy), nl->num_nets,
                                     nl->num_cells, part, ticket, out);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------- allocation-free variant
// Scratch of pl_hpwl_noalloc: the ticket words and one FP64 partial per block
// of the largest grid k_hpwl is ever launched with (kHpwlBlocks), in a
// file-scope device array of about 10 KB.  Every GPU that loads the library
// holds it until the process exits, and every call shares it.
constexpr int kNoAllocBlocks = kHpwlBlocks;
constexpr size_t kNoAllocBytes = 256 + (size_t)kNoAllocBlocks * sizeof(double);
static __device__ __align__(256) unsigned char g_hpwl_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device.  Host code cannot use
// the symbol itself (it names a host-side stand-in), so the address is looked
// up once per device, with that device current, and cached.
static cudaError_t noalloc_scratch(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_hpwl_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace pl

extern "C" pl_status pl_hpwl_noalloc(const pl_netlist *nl, const float *xy_cells, double *hpwl,
                                     pl_stream stream) {
  using namespace pl;
  clear_error();
  if (!nl || !xy_cells || !hpwl) {
    set_error("NULL argument");
    return PL_ERR_INVALID_ARG;
  }
  if (nl->num_nets < 0 || nl->num_cells < 0 || !nl->net_ptr || (nl->num_pins && !nl->pin_cell)) {
    set_error("bad netlist");
    return PL_ERR_INVALID_ARG;
  }
  const int nb = hpwl_blocks(nl->num_nets);
  if (nb > kNoAllocBlocks || hpwl_ws_bytes(nl->num_nets) > kNoAllocBytes) {
    set_error("pl_hpwl_noalloc: %d blocks exceed its fixed scratch of %d blocks", nb,
              kNoAllocBlocks);
    return PL_ERR_UNSUPPORTED;
  }
  void *scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return cuda_fail(e, "pl_hpwl_noalloc scratch lookup");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  e = cudaMemsetAsync(scratch, 0, 8, s);  // ticket and error count start at zero
  if (e == cudaSuccess) e = launch_hpwl(nl, xy_cells, hpwl, scratch, s);
  if (e != cudaSuccess) return cuda_fail(e, "pl_hpwl_noalloc");
  return PL_OK;
}
