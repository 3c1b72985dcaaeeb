// Low-precision preconditioner sweeps with BF16 storage and FP32 arithmetic (kernels in
// sweep_lp.cuh).
#include "sweep_lp.cuh"

cudaError_t launch_site_inverse_bf16(const Op& op, const double* u, void* u_lp, void* g_lp,
                                     double* g64, int L, cudaStream_t st) {
  return lp::launch_site_inverse<lp::bf16x2>(op, u, static_cast<lp::bf16x2*>(u_lp),
                                             static_cast<lp::bf16x2*>(g_lp), g64, L, st);
}

cudaError_t launch_jacobi_bf16_tiled(const Op& op, const void* g_in, const void* u_lp, void* g_lp,
                                     double* g64, int L, int rhs_per_thread, int block,
                                     int min_blocks, int staged, cudaStream_t st) {
  return lp::launch_sweep_tiled<lp::bf16x2>(op, static_cast<const lp::bf16x2*>(g_in),
                                            static_cast<const lp::bf16x2*>(u_lp),
                                            static_cast<lp::bf16x2*>(g_lp), g64, L,
                                            rhs_per_thread, block, min_blocks, staged, st);
}
