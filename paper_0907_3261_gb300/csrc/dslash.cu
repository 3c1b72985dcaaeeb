// Multi-RHS clover Wilson-Dirac stencil: Y = A X, the residual B - A X, and the Jacobi sweep
// G <- A_D^{-1}(U + kappa H G) of the preconditioner (arXiv:0907.3261, Sec. 2, Eq. (1) and the
// Jacobi polynomial for G_k).
//
// One thread owns one (site, right-hand side) pair.  Block vectors are [site][spin][colour][rhs],
// so the L threads of a site read consecutive addresses of every spinor component and share the
// site's links and clover blocks through L1.  The hopping term uses the rank-2 spin projectors of
// the chiral basis: (1 -/+ g_mu) psi = (h, -/+ G_mu^H h) with h = psi_up -/+ G_mu psi_down, where
// g_mu = [[0, G_mu], [G_mu^H, 0]], G_k = -i sigma_k, G_t = 1; only the 2-spinor h is multiplied
// by the link.  The site term is two packed Hermitian 6x6 blocks (chirality +: spins 0,1;
// chirality -: spins 2,3).
#include "common.cuh"
#include "internal.h"
#include "spin.cuh"

namespace {

enum { MODE_APPLY = 0, MODE_RESID = 1, MODE_JACOBI = 2 };

template <typename T, typename TS>
WD_DEV void load_spinor(const TS* __restrict__ p, int L, Cx<T> up[2][3], Cx<T> dn[2][3]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      auto a = ldc(p + 2 * (size_t)((s * 3 + c) * L));
      auto b = ldc(p + 2 * (size_t)(((s + 2) * 3 + c) * L));
      up[s][c] = cmake<T>(T(a.re), T(a.im));
      dn[s][c] = cmake<T>(T(b.re), T(b.im));
    }
}

// Adds (1 - DIR g_mu) W psi(x + DIR mu) to (au, ad), W = U_mu(x) for DIR = +1 and
// U_mu(x - mu)^H for DIR = -1.
template <int MU, int DIR, typename T, typename TS>
WD_DEV void hop(const TS* __restrict__ x, const T* __restrict__ links, const Geom& g, int s,
                const int c[4], int r, int L, Cx<T> au[2][3], Cx<T> ad[2][3]) {
  const int sn = neighbour(g, s, c, MU, DIR);
  Cx<T> up[2][3], dn[2][3];
  load_spinor<T>(x + 2 * ((size_t)sn * 12 * L + r), L, up, dn);
  Cx<T> h0[3], h1[3];
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    Cx<T> g0, g1;
    gamma_down<MU>(dn[0][col], dn[1][col], g0, g1);
    if constexpr (DIR > 0) { h0[col] = up[0][col] - g0; h1[col] = up[1][col] - g1; }
    else { h0[col] = up[0][col] + g0; h1[col] = up[1][col] + g1; }
  }
  const T* U = links + 18 * ((size_t)(DIR > 0 ? s : sn) * 4 + MU);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cx<T> w0 = czero<T>(), w1 = czero<T>();
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if constexpr (DIR > 0) {
        Cx<T> u = ldc(U + 2 * (a * 3 + b));
        w0 = cfma(u, h0[b], w0);
        w1 = cfma(u, h1[b], w1);
      } else {
        Cx<T> u = ldc(U + 2 * (b * 3 + a));
        w0 = cfmaj(u, h0[b], w0);
        w1 = cfmaj(u, h1[b], w1);
      }
    }
    Cx<T> g0, g1;
    gamma_up<MU>(w0, w1, g0, g1);
    au[0][a] = au[0][a] + w0;
    au[1][a] = au[1][a] + w1;
    if constexpr (DIR > 0) { ad[0][a] = ad[0][a] - g0; ad[1][a] = ad[1][a] - g1; }
    else { ad[0][a] = ad[0][a] + g0; ad[1][a] = ad[1][a] + g1; }
  }
}

// out = M v for a packed Hermitian 6x6 block M.
template <typename T>
WD_DEV void herm6(const T* __restrict__ m, const Cx<T> v[6], Cx<T> out[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) out[i] = __ldg(m + i) * v[i];
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      Cx<T> l = ldc(m + tri_index(i, j));
      out[i] = cfma(l, v[j], out[i]);
      out[j] = cfmaj(l, v[i], out[j]);
    }
}

template <typename T, typename TX, typename TY, typename TU, int MODE>
__global__ void __launch_bounds__(128)
dslash_kernel(const TX* __restrict__ x, TY* __restrict__ y, const TU* __restrict__ u,
              const T* __restrict__ links, const T* __restrict__ clov, Geom g, int L, T kappa) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.V * L) return;
  const int s = tid / L;
  const int r = tid - s * L;
  int c[4];
  site_coords(g, s, c);
  Cx<T> au[2][3], ad[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) { au[a][b] = czero<T>(); ad[a][b] = czero<T>(); }
  hop<0, +1>(x, links, g, s, c, r, L, au, ad);
  hop<0, -1>(x, links, g, s, c, r, L, au, ad);
  hop<1, +1>(x, links, g, s, c, r, L, au, ad);
  hop<1, -1>(x, links, g, s, c, r, L, au, ad);
  hop<2, +1>(x, links, g, s, c, r, L, au, ad);
  hop<2, -1>(x, links, g, s, c, r, L, au, ad);
  hop<3, +1>(x, links, g, s, c, r, L, au, ad);
  hop<3, -1>(x, links, g, s, c, r, L, au, ad);

  const size_t base = 2 * ((size_t)s * 12 * L + r);
  Cx<T> vin[2][6];   // chirality +: (spin0, spin1) x colour; chirality -: (spin2, spin3) x colour
  if constexpr (MODE == MODE_JACOBI) {
    Cx<T> up[2][3], dn[2][3];
    load_spinor<T>(u + base, L, up, dn);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int col = 0; col < 3; ++col) {
        vin[0][sp * 3 + col] = up[sp][col] + kappa * au[sp][col];
        vin[1][sp * 3 + col] = dn[sp][col] + kappa * ad[sp][col];
      }
  } else {
    Cx<T> up[2][3], dn[2][3];
    load_spinor<T>(x + base, L, up, dn);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int col = 0; col < 3; ++col) {
        vin[0][sp * 3 + col] = up[sp][col];
        vin[1][sp * 3 + col] = dn[sp][col];
      }
  }
  Cx<T> out[2][6];
  herm6(clov + (size_t)s * 2 * CLOV_REALS, vin[0], out[0]);
  herm6(clov + (size_t)s * 2 * CLOV_REALS + CLOV_REALS, vin[1], out[1]);

  Cx<T> bin[2][6];
  if constexpr (MODE == MODE_RESID) {
    Cx<T> up[2][3], dn[2][3];
    load_spinor<T>(u + base, L, up, dn);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int col = 0; col < 3; ++col) {
        bin[0][sp * 3 + col] = up[sp][col];
        bin[1][sp * 3 + col] = dn[sp][col];
      }
  }
#pragma unroll
  for (int ch = 0; ch < 2; ++ch)
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int col = 0; col < 3; ++col) {
        const int i = sp * 3 + col;
        Cx<T> v = out[ch][i];
        if constexpr (MODE != MODE_JACOBI) {
          const Cx<T> hsum = ch == 0 ? au[sp][col] : ad[sp][col];
          v = v - kappa * hsum;
          if constexpr (MODE == MODE_RESID) v = bin[ch][i] - v;
        }
        const size_t off = base + 2 * (size_t)(((ch * 2 + sp) * 3 + col) * L);
        Cx<TY> o = cmake<TY>(TY(v.re), TY(v.im));
        stc(y + off, o);
      }
}

// G = A_D^{-1} U: the first Jacobi sweep from G = 0, site-local.
template <typename T, typename TU, typename TY>
__global__ void __launch_bounds__(128)
site_inverse_kernel(const TU* __restrict__ u, TY* __restrict__ y, const T* __restrict__ clov_inv,
                    int V, int L) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= V * L) return;
  const int s = tid / L;
  const int r = tid - s * L;
  const size_t base = 2 * ((size_t)s * 12 * L + r);
  Cx<T> up[2][3], dn[2][3];
  load_spinor<T>(u + base, L, up, dn);
  Cx<T> vin[2][6], out[2][6];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      vin[0][sp * 3 + col] = up[sp][col];
      vin[1][sp * 3 + col] = dn[sp][col];
    }
  herm6(clov_inv + (size_t)s * 2 * CLOV_REALS, vin[0], out[0]);
  herm6(clov_inv + (size_t)s * 2 * CLOV_REALS + CLOV_REALS, vin[1], out[1]);
#pragma unroll
  for (int ch = 0; ch < 2; ++ch)
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const size_t off = base + 2 * (size_t)((ch * 6 + i) * L);
      stc(y + off, cmake<TY>(TY(out[ch][i].re), TY(out[ch][i].im)));
    }
}

constexpr int DS_THREADS = 128;
inline unsigned grid_for(long long n) { return (unsigned)((n + DS_THREADS - 1) / DS_THREADS); }

}  // namespace

// ------------------------------------------------------------------ launchers (FP64)
// With op.apply_form 1 the stencils run in their FP32-lane form (dslash_x3.cu).
cudaError_t launch_apply_f64(const Op& op, const double* x, double* y, int L, cudaStream_t st) {
  if (op.apply_form == 1) return launch_apply_x3(op, x, y, L, st);
  dslash_kernel<double, double, double, double, MODE_APPLY>
      <<<grid_for((long long)op.g.V * L), DS_THREADS, 0, st>>>(x, y, nullptr, op.links, op.clov,
                                                               op.g, L, op.kappa);
  return cudaGetLastError();
}

cudaError_t launch_resid_f64(const Op& op, const double* x, const double* b, double* y, int L,
                             cudaStream_t st) {
  if (op.apply_form == 1) return launch_resid_x3(op, x, b, y, L, st);
  dslash_kernel<double, double, double, double, MODE_RESID>
      <<<grid_for((long long)op.g.V * L), DS_THREADS, 0, st>>>(x, y, b, op.links, op.clov, op.g,
                                                               L, op.kappa);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_f64(const Op& op, const double* g_in, const double* u, double* g_out,
                              int L, cudaStream_t st) {
  if (op.apply_form == 1) return launch_jacobi_x3(op, g_in, u, g_out, L, st);
  dslash_kernel<double, double, double, double, MODE_JACOBI>
      <<<grid_for((long long)op.g.V * L), DS_THREADS, 0, st>>>(g_in, g_out, u, op.links,
                                                               op.clov_inv, op.g, L, op.kappa);
  return cudaGetLastError();
}

cudaError_t launch_site_inverse_f64(const Op& op, const double* u, double* g_out, int L,
                                    cudaStream_t st) {
  site_inverse_kernel<double, double, double>
      <<<grid_for((long long)op.g.V * L), DS_THREADS, 0, st>>>(u, g_out, op.clov_inv, op.g.V, L);
  return cudaGetLastError();
}
