// The low-precision preconditioner's operator copies (FP32, component-major) and the dispatch of
// its sweeps by storage type.
#include "common.cuh"
#include "internal.h"

namespace {

__global__ void links_to_cm_kernel(const double* __restrict__ links, float* __restrict__ out, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  for (int mu = 0; mu < 4; ++mu)
    for (int e = 0; e < 9; ++e) {
      const double* p = links + 18 * ((size_t)s * 4 + mu) + 2 * e;
      float* q = out + 2 * ((size_t)(mu * 9 + e) * V + s);
      q[0] = (float)p[0];
      q[1] = (float)p[1];
    }
}

__global__ void clover_to_cm_kernel(const double* __restrict__ cl, float* __restrict__ out, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  for (int ch = 0; ch < 2; ++ch)
    for (int t = 0; t < CLOV_REALS; ++t)
      out[(size_t)(ch * CLOV_REALS + t) * V + s] = (float)cl[((size_t)s * 2 + ch) * CLOV_REALS + t];
}

// The site-major copies of the double-float sweep (same FP32 values as links32 and clov_inv32).
__global__ void operator_to_sm_kernel(const double* __restrict__ links, const double* __restrict__ cl,
                                      float* __restrict__ lsm, float* __restrict__ csm, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  for (int mu = 0; mu < 4; ++mu) {
    const double* p = links + 18 * ((size_t)s * 4 + mu);
    float* q = lsm + 20 * ((size_t)s * 4 + mu);
    for (int k = 0; k < 18; ++k) q[k] = (float)p[k];
    q[18] = 0.f;
    q[19] = 0.f;
  }
  for (int k = 0; k < 2 * CLOV_REALS; ++k) csm[(size_t)s * 2 * CLOV_REALS + k] = (float)cl[(size_t)s * 2 * CLOV_REALS + k];
}

// Sets flags[0] when some link's third row differs from conj(row0 x row1) by more than tol in
// some entry, and flags[1] when some row or column has norm above 1 + tol (checked in FP64 on the
// caller's links).
__global__ void su3_check_kernel(const double* __restrict__ links, int V, double tol,
                                 int* __restrict__ flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * V) return;
  const double* p = links + 18 * (size_t)i;
  Cx<double> m[3][3];
  for (int e = 0; e < 9; ++e) m[e / 3][e % 3] = cmake<double>(p[2 * e], p[2 * e + 1]);
  const Cx<double> r[3] = {conj(cmul(m[0][1], m[1][2]) - cmul(m[0][2], m[1][1])),
                           conj(cmul(m[0][2], m[1][0]) - cmul(m[0][0], m[1][2])),
                           conj(cmul(m[0][0], m[1][1]) - cmul(m[0][1], m[1][0]))};
  double err = 0.0;
  for (int b = 0; b < 3; ++b) err = fmax(err, sqrt(cnorm2(r[b] - m[2][b])));
  if (!(err <= tol)) flags[0] = 1;   // NaN counts as a violation
  double nmax = 0.0;
  for (int a = 0; a < 3; ++a) {
    double row = 0.0, col = 0.0;
    for (int b = 0; b < 3; ++b) { row += cnorm2(m[a][b]); col += cnorm2(m[b][a]); }
    nmax = fmax(nmax, fmax(row, col));
  }
  if (!(sqrt(nmax) <= 1.0 + tol)) flags[1] = 1;
}

// Per site and chirality: max over rows i of max(sum_j |Re D_ij|, sum_j |Im D_ij|) of the packed
// Hermitian inverse block (the upper entries are conjugates of the lower ones), times 1 + 2^-20,
// which covers the FP32 rounding of the stored entries and of this sum.
__global__ void clover_bound_kernel(const double* __restrict__ cl, float* __restrict__ out, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  for (int ch = 0; ch < 2; ++ch) {
    const double* b = cl + ((size_t)s * 2 + ch) * CLOV_REALS;
    double worst = 0.0;
    for (int i = 0; i < 6; ++i) {
      double re = fabs(b[i]), im = 0.0;
      for (int j = 0; j < 6; ++j) {
        if (j == i) continue;
        const int t = i > j ? tri_index(i, j) : tri_index(j, i);
        re += fabs(b[t]);
        im += fabs(b[t + 1]);
      }
      worst = fmax(worst, fmax(re, im));
    }
    out[(size_t)ch * V + s] = (float)(worst * (1.0 + 0x1p-20));
  }
}

}  // namespace

cudaError_t launch_lp_operator_copies(const Op& op, int* flags, cudaStream_t st) {
  const int threads = 128;
  const unsigned grid = (unsigned)((op.g.V + threads - 1) / threads);
  links_to_cm_kernel<<<grid, threads, 0, st>>>(op.links, op.links32, op.g.V);
  clover_to_cm_kernel<<<grid, threads, 0, st>>>(op.clov_inv, op.clov_inv32, op.g.V);
  operator_to_sm_kernel<<<grid, threads, 0, st>>>(op.links, op.clov_inv,
                                                  reinterpret_cast<float*>(op.links32s),
                                                  reinterpret_cast<float*>(op.clov_inv32s), op.g.V);
  clover_bound_kernel<<<grid, threads, 0, st>>>(op.clov_inv, op.clov_bound32, op.g.V);
  const unsigned grid4 = (unsigned)((4LL * op.g.V + threads - 1) / threads);
  su3_check_kernel<<<grid4, threads, 0, st>>>(op.links, op.g.V, LINK12_TOL, flags);
  return cudaGetLastError();
}

cudaError_t launch_site_inverse_lp(const Op& op, int storage, const double* u, void* u_lp,
                                   void* g_lp, double* g64, int L, cudaStream_t st) {
  return storage == LP_BF16 ? launch_site_inverse_bf16(op, u, u_lp, g_lp, g64, L, st)
                            : launch_site_inverse_f32(op, u, u_lp, g_lp, g64, L, st);
}

cudaError_t launch_jacobi_lp_tiled(const Op& op, int storage, const void* g_in, const void* u_lp,
                                   void* g_lp, double* g64, int L, int rhs_per_thread, int block,
                                   int min_blocks, int staged, cudaStream_t st) {
  return storage == LP_BF16
             ? launch_jacobi_bf16_tiled(op, g_in, u_lp, g_lp, g64, L, rhs_per_thread, block,
                                        min_blocks, staged, st)
             : launch_jacobi_f32_tiled(op, g_in, u_lp, g_lp, g64, L, rhs_per_thread, block,
                                       min_blocks, staged, st);
}
