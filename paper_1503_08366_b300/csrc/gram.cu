// Tensor-core Gram formation (placeholder until the tcgen05 path lands): reports
// "unsupported" so the caller falls back to the FP32 SIMT GEMM.
#include "kernels.h"

namespace pogs {

int gram_tensor(int prec, const float* A, int64_t lda, int64_t m, int64_t n, bool tall, float* G, int64_t ldg,
                void* scratch, size_t scratch_bytes, size_t* need_bytes, int* err, cudaStream_t s) {
  (void)prec; (void)A; (void)lda; (void)m; (void)n; (void)tall; (void)G; (void)ldg; (void)scratch;
  (void)scratch_bytes; (void)err; (void)s;
  if (need_bytes) *need_bytes = 0;
  return -1;
}

}  // namespace pogs
