// Internal interfaces between the translation units of the library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

#ifndef WD_LMAX
#define WD_LMAX 16
#endif

// The operator A on the device.  FP64 fields are always present; FP32 copies serve the
// FP32 preconditioner.
struct Op {
  Geom g;
  double kappa, csw;
  double* links;     // [V][4][3][3] complex
  double* clov;      // [V][2][36]  A_D blocks, packed Hermitian
  double* clov_inv;  // [V][2][36]  A_D^{-1} blocks
  float* links32;     // [4 mu][9 entries][V] complex, FP32 (component-major)
  float* clov_inv32;  // [2 chirality][36][V], FP32 (component-major)
};

// ---- dslash.cu (FP64)
cudaError_t launch_apply_f64(const Op& op, const double* x, double* y, int L, cudaStream_t st);
cudaError_t launch_resid_f64(const Op& op, const double* x, const double* b, double* y, int L,
                             cudaStream_t st);
cudaError_t launch_jacobi_f64(const Op& op, const double* g_in, const double* u, double* g_out,
                              int L, cudaStream_t st);
cudaError_t launch_site_inverse_f64(const Op& op, const double* u, double* g_out, int L,
                                    cudaStream_t st);

// ---- dslash.cu: the FP32 preconditioner.  Its blocks (u32, g32) are component-major,
// [spin*3+colour][site][rhs]; FP64 blocks are site-major.  Exactly one of g32 / g64 is non-null.
cudaError_t launch_fp32_operator_copies(const Op& op, cudaStream_t st);
cudaError_t launch_site_inverse_mixed(const Op& op, const double* u, float* u32, float* g32,
                                      double* g64, int L, cudaStream_t st);

// FP32 sweep with `rhs_per_thread` (1 or 2; divides L) RHS per thread and `block` threads (64,
// 128, 256) per CTA -- with min_blocks 8 and block 64 compiled for at most 128 registers -- or,
// rhs_per_thread 0, the stencil of each pair split over two warps (block 128); exactly one of
// g32 / g64 is non-null.
cudaError_t launch_jacobi_f32_tiled(const Op& op, const float* g_in, const float* u32, float* g32,
                                    double* g64, int L, int rhs_per_thread, int block,
                                    int min_blocks, cudaStream_t st);

// ---- clover.cu
// Builds clov and clov_inv from links; *singular_dev receives 1 if some 6x6 block is singular.
cudaError_t launch_clover_build(const Op& op, int* singular_dev, cudaStream_t st);

// ---- blas.cu: tall-skinny N x L operations with deterministic reductions
struct SolverState {
  double2 rtv[WD_LMAX * WD_LMAX];      // R~_0^H V_k
  double2 rtr[WD_LMAX * WD_LMAX];      // R~_0^H R_k
  double2 rtr_new[WD_LMAX * WD_LMAX];  // R~_0^H R_{k+1}
  double2 alpha[WD_LMAX * WD_LMAX];
  double2 gamma[WD_LMAX * WD_LMAX];
  double2 zeta;
  double2 trwr;                          // Tr[W^H R]
  double trww;                           // Tr[W^H W]
  double rnorm2[WD_LMAX];                // ||r_i||^2 of the latest R
  int status;                            // 0, or ST_* below
};
enum { ST_OK = 0, ST_ALPHA_SINGULAR = 1, ST_GAMMA_SINGULAR = 2, ST_ZETA_BAD = 3 };

// Partial-sum slots per block of the reduction kernels.
constexpr int PART_STRIDE = WD_LMAX * WD_LMAX + WD_LMAX;
int ts_blocks(long long rows);   // grid size of the tall-skinny kernels for `rows` rows

// Which L x L result a gram pass writes.
enum { GRAM_RTR = 0, GRAM_RTR_NEW = 1, GRAM_RTV = 2 };

cudaError_t launch_gram(const double* A, const double* B, int L, long long rows, double2* part,
                        SolverState* st, int which, bool norms_of_b, cudaStream_t s);
cudaError_t launch_colnorms(const double* A, int L, long long rows, double2* part,
                            double* out_norm2, cudaStream_t s);
cudaError_t launch_traces(const double* W, const double* R, int L, long long rows,
                          double2* part, SolverState* st, cudaStream_t s);
cudaError_t launch_solve_alpha(SolverState* st, int L, cudaStream_t s);
cudaError_t launch_solve_gamma(SolverState* st, int L, cudaStream_t s);
// df: the products with L x L matrices and the Gram products in double-float arithmetic.
cudaError_t launch_update_u(const double* P, const double* V, double* U, int L, long long rows,
                            const SolverState* st, cudaStream_t s, bool df);
cudaError_t launch_update_xr(double* X, const double* F, const double* G, double* R,
                             const double* W, const double* Y, const double* Rt, int L,
                             long long rows, double2* part, SolverState* st, cudaStream_t s,
                             bool df);
cudaError_t launch_update_pv(double* P, double* V, const double* R, const double* W,
                             const double* U, const double* Y, const double* Rt, int L,
                             long long rows, double2* part, SolverState* st, cudaStream_t s,
                             bool df);

// ---- abi.cu helpers for other translation units
struct wd_ctx;
const Op* wd_ctx_op(const wd_ctx* ctx);
void wd_set_error(const char* fmt, ...);

// ---- net.cu: the learned preconditioner (activations FP32, component-major per channel)
cudaError_t net_launch_layer(const Op& op, const float* in, float* out, const float2* W, int cin,
                             int cout, int L, cudaStream_t st);
cudaError_t net_launch_wgrad(const Op& op, const float* in, const float* delta, int cin, int cout,
                             int L, double2* part, int nblocks, double2* grad, cudaStream_t st);
cudaError_t net_launch_adjoint_weights(const float2* W, float2* Wa, int cin, int cout,
                                       cudaStream_t st);
cudaError_t net_launch_to_cm(const double* x, float* y, int V, int L, cudaStream_t st);
cudaError_t net_launch_from_cm(const float* y, double* x, int V, int L, cudaStream_t st);
cudaError_t net_launch_loss_delta(const float* y, const double* E, const double* wcol,
                                  float* delta, double* part, int nblocks, double* loss, int V,
                                  int L, cudaStream_t st);
cudaError_t net_launch_adam(float2* W, const double2* G, float2* m, float2* v, int n, float lr,
                            float b1, float b2, float eps, int t, cudaStream_t st);
// ---- net_abi.cu
struct wd_net;
int wd_net_precondition(wd_ctx* ctx, wd_net* net, const double* R, double* G, int L,
                        cudaStream_t s);
int wd_net_prepare(wd_ctx* ctx, wd_net* net, int L);
