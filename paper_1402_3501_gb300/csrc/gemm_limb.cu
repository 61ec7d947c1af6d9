// fgemm, limb form (tcgen05 tensor cores): placeholder until the kernel lands.
#include "common.cuh"

int limb_form_supported(uint32_t p) {
  (void)p;
  return 0;
}

int fgemm_sub_limb(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A, int64_t lda,
                   const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc) {
  (void)c; (void)M; (void)N; (void)K; (void)A; (void)lda; (void)B; (void)ldb; (void)C; (void)ldc;
  return PLUQ_ERR_UNSUPPORTED_FORM;
}
