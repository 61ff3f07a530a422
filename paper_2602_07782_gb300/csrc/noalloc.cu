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

static __device__ __align__(256) uint32_t g_sort_scratch[4 * kNoAllocMaxCharts];

std::mutex g_mu;
uint32_t *g_scratch_addr[256] = {};

// Chart indices by decreasing height, ties in index order: the pack's own
// radix sort (radix_sort21) on keys 2^21 - 1 - height, with heights outside
// [0, 2^21) clamped into it.  One CTA.
__global__ void __launch_bounds__(tabi::kRadixThreads)
    sort_heights_kernel(const int32_t *__restrict__ heights, int n, uint32_t *scratch, int32_t *perm) {
  uint32_t *kA = scratch, *vA = kA + n, *kB = vA + n, *vB = kB + n;
  for (int c = threadIdx.x; c < n; c += tabi::kRadixThreads) {
    const int32_t h = min(max(heights[c], 0), (1 << 21) - 1);
    kA[c] = (uint32_t)((1 << 21) - 1 - h);
    vA[c] = (uint32_t)c;
  }
  tabi::radix_sort21(kA, vA, kB, vB, n);
  for (int s = threadIdx.x; s < n; s += tabi::kRadixThreads) perm[s] = (int32_t)vB[s];
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
  // Errors are looked at without clearing them (cudaPeekAtLastError): an
  // error already pending from other work on this thread is left to its
  // owner and nothing is launched; an error raised by this launch is
  // cleared and reported as this call's TABI_ERR_CUDA.
  if (cudaPeekAtLastError() != cudaSuccess) return TABI_ERR_CUDA;
  sort_heights_kernel<<<1, tabi::kRadixThreads, 0, (cudaStream_t)stream>>>(heights, n, scratch, perm);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return TABI_ERR_CUDA;
  }
  return TABI_OK;
}
