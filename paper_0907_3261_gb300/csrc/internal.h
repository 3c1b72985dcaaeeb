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
  // 1: the low-precision sweeps read rows 0 and 1 of each FP32 link and rebuild row 2 (the links
  // are special unitary to LINK12_TOL); 0: they read all three rows.
  int link12;
  // 1: every link's rows and columns have norm at most 1 + LINK12_TOL (unitary links), which the
  // grid-biased double-float sweep relies on; 0: that sweep is not used.
  int links_unitary;
  // [2 chirality][V]: for each site's inverse block D, max over rows i of
  // max(sum_j |Re D_ij|, sum_j |Im D_ij|), rounded up -- a bound on the partial sums of a row
  // times a vector in units of the vector's largest real part.
  float* clov_bound32;
  // Site-major FP32 copies for the grid-sum double-float sweep, read in 16-byte loads: the links
  // [site][mu][20 floats] (9 entries (re, im) row by row, two zeros) and A_D^{-1}
  // [site][chirality][36 floats] (the packed blocks of clov_inv32).
  float4* links32s;
  float4* clov_inv32s;
  // The FP32-lane form of the FP64 stencil (dslash_x3.cu): the links cut into three FP32 levels,
  // [site][mu][level][entry] as (re, re, im, im) (null when the links are not unitary), a scratch
  // of V * WD_LMAX exponents, and the form in use (1: this one, 0: the FP64-pipe kernel).
  float4* links_x3;
  int* xexp;
  int apply_form;
};

// Largest entry error |row2 - conj(row0 x row1)| of a link that still counts as special unitary.
constexpr double LINK12_TOL = 1e-6;

// ---- dslash.cu (FP64)
cudaError_t launch_apply_f64(const Op& op, const double* x, double* y, int L, cudaStream_t st);
cudaError_t launch_resid_f64(const Op& op, const double* x, const double* b, double* y, int L,
                             cudaStream_t st);
cudaError_t launch_jacobi_f64(const Op& op, const double* g_in, const double* u, double* g_out,
                              int L, cudaStream_t st);
cudaError_t launch_site_inverse_f64(const Op& op, const double* u, double* g_out, int L,
                                    cudaStream_t st);

// ---- dslash_x3.cu (the same FP64 operations with the hopping sums on the FP32 lanes)
cudaError_t launch_link_split(const Op& op, cudaStream_t st);
cudaError_t launch_apply_x3(const Op& op, const double* x, double* y, int L, cudaStream_t st);
cudaError_t launch_resid_x3(const Op& op, const double* x, const double* b, double* y, int L,
                            cudaStream_t st);
cudaError_t launch_jacobi_x3(const Op& op, const double* g_in, const double* u, double* g_out,
                             int L, cudaStream_t st);
// Kernels one FP64 stencil launch takes (the x3 form adds its exponent pre-pass).
inline int stencil_kernels(const Op& op) { return op.apply_form == 1 ? 2 : 1; }

// ---- sweep_lp.cu, sweep_f32.cu, sweep_bf16.cu: the low-precision preconditioner.  Its private
// blocks (u_lp, g_lp) are component-major, [spin*3+colour][site][rhs], one complex number per
// element: float2 (LP_F32) or two packed BF16 numbers (LP_BF16); FP64 blocks are site-major.
// Exactly one of g_lp / g64 is non-null.
enum { LP_F32 = 0, LP_BF16 = 1, LP_DF = 2 };   // LP_DF: the double-float sweep's tile table
constexpr size_t lp_elem_bytes(int storage) { return storage == LP_BF16 ? 4 : 8; }

// FP32 component-major links and A_D^{-1} and the row bounds of A_D^{-1}; sets flags[0] (device)
// when some link is not special unitary to LINK12_TOL and flags[1] when some link has a row or a
// column of norm above 1 + LINK12_TOL.
cudaError_t launch_lp_operator_copies(const Op& op, int* flags, cudaStream_t st);
// First sweep from G = 0: G = A_D^{-1} U, with the low-precision copy of U stored in u_lp.
cudaError_t launch_site_inverse_lp(const Op& op, int storage, const double* u, void* u_lp,
                                   void* g_lp, double* g64, int L, cudaStream_t st);
// One sweep with `rhs_per_thread` (1 or 2; divides L) RHS per thread and `block` threads (64,
// 128, 256) per CTA -- with min_blocks 8 and block 64 compiled for at most 128 registers -- or,
// rhs_per_thread 0, the stencil of each pair split over two warps (block 128); staged 1 (with 2
// RHS per thread and block 64) stages each direction's neighbour data in shared memory with
// cp.async while the previous direction is computed.
cudaError_t launch_jacobi_lp_tiled(const Op& op, int storage, const void* g_in, const void* u_lp,
                                   void* g_lp, double* g64, int L, int rhs_per_thread, int block,
                                   int min_blocks, int staged, cudaStream_t st);
// The same per storage type.
cudaError_t launch_site_inverse_f32(const Op& op, const double* u, void* u_lp, void* g_lp,
                                    double* g64, int L, cudaStream_t st);
cudaError_t launch_site_inverse_bf16(const Op& op, const double* u, void* u_lp, void* g_lp,
                                     double* g64, int L, cudaStream_t st);
cudaError_t launch_jacobi_f32_tiled(const Op& op, const void* g_in, const void* u_lp, void* g_lp,
                                    double* g64, int L, int rhs_per_thread, int block,
                                    int min_blocks, int staged, cudaStream_t st);
cudaError_t launch_jacobi_bf16_tiled(const Op& op, const void* g_in, const void* u_lp, void* g_lp,
                                     double* g64, int L, int rhs_per_thread, int block,
                                     int min_blocks, int staged, cudaStream_t st);

// ---- sweep_df.cu: the double-float preconditioner (FP32 operator, spinors as FP32 pairs).  Its
// blocks are component-major with one float4 (re.hi, im.hi, re.lo, im.lo) per complex number.
cudaError_t launch_site_inverse_df(const Op& op, const double* u, void* u_df, void* g_df,
                                   double* g64, int L, cudaStream_t st);
// One sweep with 1 or 2 RHS per thread (dividing L) and `block` (64 or 128) threads per CTA;
// packed 1 (with 1 RHS per thread) runs the FP32x2 (real, imaginary lanes) variant, packed 2 the
// FP32x2 variant whose link and clover products are summed on a fixed grid (needs
// op.links_unitary).
cudaError_t launch_jacobi_df(const Op& op, const void* g_in, const void* u_df, void* g_df,
                             double* g64, int L, int rhs_per_thread, int block, int packed,
                             cudaStream_t st);

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
int ts_max_blocks();             // largest such grid on the current device (4 x its SM count)

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
int wd_ctx_device(const wd_ctx* ctx);   // the device the context was created on
// Counts `nkernels` launches of class `cls` (WD_K_*) in the context's instrumentation.
void wd_ctx_count_launches(wd_ctx* ctx, int cls, int nkernels);
void wd_set_error(const char* fmt, ...);

// ---- noalloc.cu
// Loads the static scratch array of jacobi_precond_noalloc on the current device (resolving its
// address forces the module, and with it the array, to be loaded); WD_OK or an error code.
int noalloc_reserve(void);

// ---- net.cu: the learned preconditioner (activations component-major per channel)
cudaError_t net_launch_layer(const Op& op, const float* in, float* out, const float2* W, int cin,
                             int cout, int L, cudaStream_t st);
cudaError_t net_launch_wgrad(const Op& op, const float* in, const float* delta, int cin, int cout,
                             int L, double2* part, int nblocks, double2* grad, cudaStream_t st);
cudaError_t net_launch_adjoint_weights(const float2* W, float2* Wa, int cin, int cout,
                                       cudaStream_t st);
// FP64 site-major <-> component-major channel of FP32 (bf16 false) or BF16 elements.
cudaError_t net_launch_to_cm(const double* x, void* y, int V, int L, bool bf16, cudaStream_t st);
cudaError_t net_launch_from_cm(const void* y, double* x, int V, int L, bool bf16, cudaStream_t st);
// One layer on BF16-stored activations (inference).
cudaError_t net_launch_layer_bf16(const Op& op, const void* in, void* out, const float2* W,
                                  int cin, int cout, int L, cudaStream_t st);
cudaError_t net_launch_loss_delta(const float* y, const double* E, const double* wcol,
                                  float* delta, double* part, int nblocks, double* loss, int V,
                                  int L, cudaStream_t st);
cudaError_t net_launch_adam(float2* W, const double2* G, float2* m, float2* v, int n, float lr,
                            float b1, float b2, float eps, int t, cudaStream_t st);
// ---- net_abi.cu
struct wd_net;
// G = N(R); bf16: activations stored in BF16.
int wd_net_precondition(wd_ctx* ctx, wd_net* net, const double* R, double* G, int L, bool bf16,
                        cudaStream_t s);
int wd_net_prepare(wd_ctx* ctx, wd_net* net, int L);
