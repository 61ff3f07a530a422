// Height sort without any device allocation.
//
// Some callers cannot call cudaMalloc at all: engines and interactive tools
// that own a fixed, pre-budgeted pool of device memory and forbid any
// allocation outside it, and frame loops where an allocation (which may
// synchronise the device) would stall the frame.  For them this file offers
// a variant of the packer's height sort whose scratch memory is a
// file-scope device array instead of the context arena: the caller passes
// only the input heights and the output permutation.
//
// The scratch array holds the radix sort's two ping-pong key/value buffers
// for up to kNoAllocMaxCharts charts (1 MiB).  Every GPU that loads the
// library keeps it until the process exits.  Host code cannot use the
// array's name as a device address, so the first call on each device asks
// the runtime for the address (cudaGetSymbolAddress) with that device
// current and caches it.
#include <mutex>

#include "tabi_internal.cuh"

namespace {

constexpr int kNoAllocMaxCharts = 65536;
constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kDigits = 128;  // 7-bit digits, 3 passes over 21-bit keys

static __device__ __align__(256) uint32_t g_sort_scratch[4 * kNoAllocMaxCharts];

std::mutex g_mu;
uint32_t *g_scratch_addr[256] = {};

// Stable LSD radix sort of chart indices by decreasing height (ties keep
// index order), one CTA.  Heights outside [0, 2^21) are clamped into it.
__global__ void __launch_bounds__(kThreads)
    sort_heights_kernel(const int32_t *__restrict__ heights, int n, uint32_t *scratch, int32_t *perm) {
  __shared__ uint32_t hist[kDigits * kWarps];
  __shared__ uint32_t part[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  uint32_t *kA = scratch, *vA = kA + n, *kB = vA + n, *vB = kB + n;
  for (int c = tid; c < n; c += kThreads) {
    const int32_t h = min(max(heights[c], 0), (1 << 21) - 1);
    kA[c] = (uint32_t)((1 << 21) - 1 - h);
    vA[c] = (uint32_t)c;
  }
  const int chunk = ((n + kWarps - 1) / kWarps + 31) & ~31;
  const int beg = w * chunk, end = min(n, beg + chunk);
  const unsigned lt = (1u << lane) - 1u;
  __syncthreads();
  for (int pass = 0; pass < 3; ++pass) {
    const int shift = 7 * pass;
    const uint32_t *ks = (pass & 1) ? kB : kA, *vs = (pass & 1) ? vB : vA;
    uint32_t *kd = (pass & 1) ? kA : kB, *vd = (pass & 1) ? vA : vB;
    for (int i = tid; i < kDigits * kWarps; i += kThreads) hist[i] = 0;
    __syncthreads();
    for (int base = beg; base < end; base += 32) {
      const int i = base + lane;
      const bool ok = i < end;
      const uint32_t d = ok ? (ks[i] >> shift) & (kDigits - 1) : kDigits;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      if (ok && lane == __ffs(peers) - 1) hist[d * kWarps + w] += __popc(peers);
    }
    __syncthreads();
    uint32_t loc[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) { loc[q] = hist[tid * 4 + q]; sum += loc[q]; }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) part[w] = incl;
    __syncthreads();
    if (w == 0) {
      const uint32_t x = part[lane];
      uint32_t y = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += u;
      }
      part[lane] = y - x;
    }
    __syncthreads();
    uint32_t run = part[w] + incl - sum;
#pragma unroll
    for (int q = 0; q < 4; ++q) { hist[tid * 4 + q] = run; run += loc[q]; }
    __syncthreads();
    for (int base = beg; base < end; base += 32) {
      const int i = base + lane;
      const bool ok = i < end;
      const uint32_t key = ok ? ks[i] : 0u;
      const uint32_t d = ok ? (key >> shift) & (kDigits - 1) : kDigits;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      uint32_t dst = 0;
      if (ok) dst = hist[d * kWarps + w] + __popc(peers & lt);
      __syncwarp();
      if (ok && lane == __ffs(peers) - 1) hist[d * kWarps + w] += __popc(peers);
      __syncwarp();
      if (ok) { kd[dst] = key; vd[dst] = vs[i]; }
    }
    __syncthreads();
  }
  for (int s = tid; s < n; s += kThreads) perm[s] = (int32_t)vB[s];
}

}  // namespace

extern "C" tabi_status tabi_sort_heights_noalloc(const int32_t *heights, int32_t n, int32_t *perm,
                                                 void *stream) {
  if (!heights || !perm || n < 1 || n > kNoAllocMaxCharts) return TABI_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return TABI_ERR_CUDA;
  uint32_t *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_sort_scratch) != cudaSuccess || !ptr) return TABI_ERR_CUDA;
      g_scratch_addr[dev] = (uint32_t *)ptr;
    }
    scratch = g_scratch_addr[dev];
  }
  sort_heights_kernel<<<1, kThreads, 0, (cudaStream_t)stream>>>(heights, n, scratch, perm);
  return cudaGetLastError() == cudaSuccess ? TABI_OK : TABI_ERR_CUDA;
}
