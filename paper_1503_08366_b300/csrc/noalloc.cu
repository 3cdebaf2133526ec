// pogs_gram_noalloc: the Gram formation of pogs_gram without any device allocation.
//
// Some callers cannot allocate device memory when they need this step: a process whose
// device memory is entirely owned by another allocator (a caching allocator, or a server
// that admits work against a fixed memory budget), or a latency-critical path where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.  For them the
// scratch this step needs -- the packed tensor-core operands and a status word -- lives in
// one file-scope device array of fixed size, reserved when the library is loaded and held by
// every device that loads it until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"

namespace {

// 32 MiB of scratch.  Layout: [0, 256) status word; [256, ...) packed operands.
constexpr size_t kNoAllocBytes = size_t(32) << 20;
constexpr size_t kStatusBytes = 256;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device, looked up once with that device current
// (in host code the symbol is only a host-side stand-in for the device array).
constexpr int kMaxDevices = 64;
void* g_dev_ptr[kMaxDevices] = {};
std::mutex g_mu;

int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return POGS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return POGS_ERR_CUDA;
    }
    g_dev_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_dev_ptr[dev]);
  return 0;
}

}  // namespace

extern "C" int pogs_gram_noalloc(const float* A, int64_t m, int64_t n, int64_t lda, int gram_prec, float* G,
                                 void* stream) {
  if (!A || !G || m < 1 || n < 1 || lda < n || gram_prec < POGS_GRAM_BF16 || gram_prec > POGS_GRAM_FP32)
    return POGS_ERR_ARG;
  for (const void* p : {static_cast<const void*>(A), static_cast<const void*>(G)}) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return POGS_ERR_ARG;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool tall = m >= n;
  const int64_t q = tall ? n : m;
  // size check first: no device work for a request that does not fit
  size_t need = 0;
  if (gram_prec != POGS_GRAM_FP32) {
    if (pogs::gram_tensor(gram_prec, A, lda, m, n, tall, G, q, nullptr, 0, &need, nullptr, s) != 0)
      return POGS_ERR_CUDA;
    if (need > kNoAllocBytes - kStatusBytes) return POGS_ERR_CAPACITY;
  }
  unsigned char* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc != 0) return rc;
  int* status = reinterpret_cast<int*>(base);
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return POGS_ERR_CUDA;
  }
  if (gram_prec == POGS_GRAM_FP32) {
    if (tall) pogs::gemm_f32(true, false, q, q, m, 1.0f, A, lda, A, lda, 0.0f, G, q, true, s);
    else pogs::gemm_f32(false, true, q, q, n, 1.0f, A, lda, A, lda, 0.0f, G, q, true, s);
  } else if (pogs::gram_tensor(gram_prec, A, lda, m, n, tall, G, q, base + kStatusBytes,
                               kNoAllocBytes - kStatusBytes, &need, status, s) != 0) {
    return POGS_ERR_CUDA;
  }
  int host_status = 0;
  if (cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return POGS_ERR_CUDA;
  }
  if (host_status != 0) return host_status;
  return cudaGetLastError() == cudaSuccess ? 0 : POGS_ERR_CUDA;
}
