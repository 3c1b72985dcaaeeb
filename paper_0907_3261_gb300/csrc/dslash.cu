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

namespace {

enum { MODE_APPLY = 0, MODE_RESID = 1, MODE_JACOBI = 2 };

// G_mu d for the lower 2-spinor d = (d0, d1), one colour component.
template <int MU, typename T>
WD_DEV void gamma_down(Cx<T> d0, Cx<T> d1, Cx<T>& g0, Cx<T>& g1) {
  if constexpr (MU == 0) { g0 = tmi(d1); g1 = tmi(d0); }
  else if constexpr (MU == 1) { g0 = -d1; g1 = d0; }
  else if constexpr (MU == 2) { g0 = tmi(d0); g1 = ti(d1); }
  else { g0 = d0; g1 = d1; }
}
// G_mu^H w.
template <int MU, typename T>
WD_DEV void gamma_up(Cx<T> w0, Cx<T> w1, Cx<T>& g0, Cx<T>& g1) {
  if constexpr (MU == 0) { g0 = ti(w1); g1 = ti(w0); }
  else if constexpr (MU == 1) { g0 = w1; g1 = -w0; }
  else if constexpr (MU == 2) { g0 = ti(w0); g1 = tmi(w1); }
  else { g0 = w0; g1 = w1; }
}

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

// Packed Hermitian 6x6 times a vector, block entries `stride` apart (component-major storage).
template <typename T>
WD_DEV void herm6s(const T* __restrict__ m, size_t stride, const Cx<T> v[6], Cx<T> out[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) out[i] = __ldg(m + i * stride) * v[i];
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      const int t = tri_index(i, j);
      const Cx<T> l = cmake<T>(__ldg(m + t * stride), __ldg(m + (t + 1) * stride));
      out[i] = cfma(l, v[j], out[i]);
      out[j] = cfmaj(l, v[i], out[j]);
    }
}

// First sweep of the FP32 preconditioner: reads the FP64 right-hand side U (site-major), stores
// its FP32 copy in u32 (component-major, when not null) for the later sweeps, and writes
// G = A_D^{-1} U computed in FP32 -- component-major FP32 or site-major FP64.
template <typename TY>
__global__ void __launch_bounds__(128)
site_inverse_mixed_kernel(const double* __restrict__ u, float* __restrict__ u32,
                          TY* __restrict__ y, const float* __restrict__ clov_inv_cm, int V, int L) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= V * L) return;
  const int s = tid / L;
  const int r = tid - s * L;
  const size_t base = 2 * ((size_t)s * 12 * L + r);
  Cx<float> vin[2][6], out[2][6];
#pragma unroll
  for (int ch = 0; ch < 2; ++ch)
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int k = ch * 6 + i;
      const Cx<double> a = ldc(u + base + 2 * (size_t)(k * L));
      vin[ch][i] = cmake<float>((float)a.re, (float)a.im);
      if (u32) stc(u32 + 2 * (((size_t)k * V + s) * L + r), vin[ch][i]);
    }
  herm6s(clov_inv_cm + s, (size_t)V, vin[0], out[0]);
  herm6s(clov_inv_cm + (size_t)CLOV_REALS * V + s, (size_t)V, vin[1], out[1]);
#pragma unroll
  for (int ch = 0; ch < 2; ++ch)
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int k = ch * 6 + i;
      TY* p = sizeof(TY) == 4 ? y + 2 * (((size_t)k * V + s) * L + r) : y + base + 2 * (size_t)(k * L);
      stc(p, cmake<TY>(TY(out[ch][i].re), TY(out[ch][i].im)));
    }
}

constexpr int DS_THREADS = 128;
inline unsigned grid_for(long long n) { return (unsigned)((n + DS_THREADS - 1) / DS_THREADS); }

}  // namespace

// ------------------------------------------------------------------ launchers (FP64)
cudaError_t launch_apply_f64(const Op& op, const double* x, double* y, int L, cudaStream_t st) {
  dslash_kernel<double, double, double, double, MODE_APPLY>
      <<<grid_for((long long)op.g.V * L), DS_THREADS, 0, st>>>(x, y, nullptr, op.links, op.clov,
                                                               op.g, L, op.kappa);
  return cudaGetLastError();
}

cudaError_t launch_resid_f64(const Op& op, const double* x, const double* b, double* y, int L,
                             cudaStream_t st) {
  dslash_kernel<double, double, double, double, MODE_RESID>
      <<<grid_for((long long)op.g.V * L), DS_THREADS, 0, st>>>(x, y, b, op.links, op.clov, op.g,
                                                               L, op.kappa);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_f64(const Op& op, const double* g_in, const double* u, double* g_out,
                              int L, cudaStream_t st) {
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

// ------------------------------------------------------------------ launchers (FP32 sweeps)
cudaError_t launch_site_inverse_mixed(const Op& op, const double* u, float* u32, float* g32,
                                      double* g64, int L, cudaStream_t st) {
  const unsigned grid = grid_for((long long)op.g.V * L);
  if (g32)
    site_inverse_mixed_kernel<float><<<grid, DS_THREADS, 0, st>>>(u, u32, g32, op.clov_inv32,
                                                                  op.g.V, L);
  else
    site_inverse_mixed_kernel<double><<<grid, DS_THREADS, 0, st>>>(u, u32, g64, op.clov_inv32,
                                                                   op.g.V, L);
  return cudaGetLastError();
}


// ------------------------------------------------------------------ FP32 sweep, R RHS per thread
// The FP32 Jacobi sweep G' = A_D^{-1}(U + kappa H G) on the preconditioner's private FP32 blocks,
// which are stored component-major, [spin*3+colour][site][rhs]: the threads of a warp take
// consecutive (site, rhs) pairs, so every component of every neighbour spinor is one contiguous
// run of 8*32 bytes per warp instruction.  The FP32 links ([mu][3x3 entry][site]) and A_D^{-1}
// blocks ([chirality][36][site]) are component-major too.  Each thread owns R consecutive
// right-hand sides (R = 1 or 2 dividing L); links and clover entries serve all R.  The last sweep
// writes FP64 in the caller's site-major layout.
namespace {

template <int R>
WD_DEV void ld_row(const float* __restrict__ p, Cx<float> v[R]) {
  if constexpr (R == 1) {
    v[0] = ldc(p);
  } else {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = {a.x, a.y};
    v[1] = {a.z, a.w};
  }
}

template <int R, typename TY>
WD_DEV void st_row(TY* __restrict__ p, const Cx<float> v[R]) {
  if constexpr (sizeof(TY) == 4 && R == 2) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
  } else {
#pragma unroll
    for (int q = 0; q < R; ++q) stc(p + 2 * q, cmake<TY>(TY(v[q].re), TY(v[q].im)));
  }
}

template <int MU, int DIR, int R>
WD_DEV void hop_cm(const float* __restrict__ x, const float* __restrict__ links, const Geom& g,
                   int s, const int c[4], int r0, int L, Cx<float> au[R][2][3],
                   Cx<float> ad[R][2][3]) {
  const int sn = neighbour(g, s, c, MU, DIR);
  const size_t V = (size_t)g.V;
  const float* base = x + 2 * ((size_t)sn * L + r0);
  const size_t cstride = 2 * V * L;            // floats between components
  Cx<float> h0[R][3], h1[R][3];
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    Cx<float> u0[R], u1[R], d0[R], d1[R];
    ld_row<R>(base + (0 * 3 + col) * cstride, u0);
    ld_row<R>(base + (1 * 3 + col) * cstride, u1);
    ld_row<R>(base + (2 * 3 + col) * cstride, d0);
    ld_row<R>(base + (3 * 3 + col) * cstride, d1);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      Cx<float> g0, g1;
      gamma_down<MU>(d0[q], d1[q], g0, g1);
      if constexpr (DIR > 0) { h0[q][col] = u0[q] - g0; h1[q][col] = u1[q] - g1; }
      else { h0[q][col] = u0[q] + g0; h1[q][col] = u1[q] + g1; }
    }
  }
  const float* U = links + 2 * ((size_t)MU * 9 * V + (DIR > 0 ? s : sn));
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cx<float> ua[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) ua[b] = ldc(U + 2 * (size_t)(DIR > 0 ? a * 3 + b : b * 3 + a) * V);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      Cx<float> w0 = czero<float>(), w1 = czero<float>();
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if constexpr (DIR > 0) { w0 = cfma(ua[b], h0[q][b], w0); w1 = cfma(ua[b], h1[q][b], w1); }
        else { w0 = cfmaj(ua[b], h0[q][b], w0); w1 = cfmaj(ua[b], h1[q][b], w1); }
      }
      Cx<float> g0, g1;
      gamma_up<MU>(w0, w1, g0, g1);
      au[q][0][a] = au[q][0][a] + w0;
      au[q][1][a] = au[q][1][a] + w1;
      if constexpr (DIR > 0) { ad[q][0][a] = ad[q][0][a] - g0; ad[q][1][a] = ad[q][1][a] - g1; }
      else { ad[q][0][a] = ad[q][0][a] + g0; ad[q][1][a] = ad[q][1][a] + g1; }
    }
  }
}

template <int R, typename TY, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
jacobi_f32_kernel(const float* __restrict__ x, TY* __restrict__ y, const float* __restrict__ u,
                  const float* __restrict__ links, const float* __restrict__ clov_inv, Geom g,
                  int L, float kappa) {
  const int groups = L / R;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.V * groups) return;
  const int s = tid / groups;
  const int r0 = (tid - s * groups) * R;
  const size_t V = (size_t)g.V;
  int c[4];
  site_coords(g, s, c);
  Cx<float> au[R][2][3], ad[R][2][3];
#pragma unroll
  for (int q = 0; q < R; ++q)
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) { au[q][a][b] = czero<float>(); ad[q][a][b] = czero<float>(); }
  hop_cm<0, +1, R>(x, links, g, s, c, r0, L, au, ad);
  hop_cm<0, -1, R>(x, links, g, s, c, r0, L, au, ad);
  hop_cm<1, +1, R>(x, links, g, s, c, r0, L, au, ad);
  hop_cm<1, -1, R>(x, links, g, s, c, r0, L, au, ad);
  hop_cm<2, +1, R>(x, links, g, s, c, r0, L, au, ad);
  hop_cm<2, -1, R>(x, links, g, s, c, r0, L, au, ad);
  hop_cm<3, +1, R>(x, links, g, s, c, r0, L, au, ad);
  hop_cm<3, -1, R>(x, links, g, s, c, r0, L, au, ad);
#pragma unroll
  for (int ch = 0; ch < 2; ++ch) {
    Cx<float> vin[R][6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int k = ch * 6 + i;
      Cx<float> uu[R];
      ld_row<R>(u + 2 * (((size_t)k * V + s) * L + r0), uu);
#pragma unroll
      for (int q = 0; q < R; ++q)
        vin[q][i] = uu[q] + kappa * (ch == 0 ? au[q][i / 3][i % 3] : ad[q][i / 3][i % 3]);
    }
    Cx<float> out[R][6];
#pragma unroll
    for (int q = 0; q < R; ++q) herm6s(clov_inv + (size_t)ch * CLOV_REALS * V + s, V, vin[q], out[q]);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int k = ch * 6 + i;
      Cx<float> o[R];
#pragma unroll
      for (int q = 0; q < R; ++q) o[q] = out[q][i];
      TY* p = sizeof(TY) == 4 ? y + 2 * (((size_t)k * V + s) * L + r0)
                              : y + 2 * (((size_t)s * 12 + k) * L + r0);
      st_row<R, TY>(p, o);
    }
  }
}

template <int R, typename TY>
cudaError_t launch_jacobi_f32_r(const Op& op, const float* g_in, const float* u32, TY* out, int L,
                                int block, int min_blocks, cudaStream_t st) {
  const long long n = (long long)op.g.V * (L / R);
  const unsigned grid = (unsigned)((n + block - 1) / block);
  if (min_blocks == 8 && block == 64)    // at most 128 registers: 16 warps per SM
    jacobi_f32_kernel<R, TY, 64, 8><<<grid, block, 0, st>>>(
        g_in, out, u32, op.links32, op.clov_inv32, op.g, L, (float)op.kappa);
  else
    jacobi_f32_kernel<R, TY, 256, 1><<<grid, block, 0, st>>>(
        g_in, out, u32, op.links32, op.clov_inv32, op.g, L, (float)op.kappa);
  return cudaGetLastError();
}

// FP32 component-major copies of the links and of the A_D^{-1} blocks.
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

}  // namespace

cudaError_t launch_jacobi_f32_split(const Op& op, const float* g_in, const float* u32, float* g32,
                                    double* g64, int L, cudaStream_t st);

cudaError_t launch_jacobi_f32_tiled(const Op& op, const float* g_in, const float* u32, float* g32,
                                    double* g64, int L, int rhs_per_thread, int block,
                                    int min_blocks, cudaStream_t st) {
  if (rhs_per_thread == 0) return launch_jacobi_f32_split(op, g_in, u32, g32, g64, L, st);
  if (L % rhs_per_thread != 0 || (block != 64 && block != 128 && block != 256))
    return cudaErrorInvalidValue;
  switch (rhs_per_thread) {
    case 1: return g32 ? launch_jacobi_f32_r<1>(op, g_in, u32, g32, L, block, min_blocks, st)
                       : launch_jacobi_f32_r<1>(op, g_in, u32, g64, L, block, min_blocks, st);
    case 2: return g32 ? launch_jacobi_f32_r<2>(op, g_in, u32, g32, L, block, min_blocks, st)
                       : launch_jacobi_f32_r<2>(op, g_in, u32, g64, L, block, min_blocks, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fp32_operator_copies(const Op& op, cudaStream_t st) {
  const int threads = 128;
  const unsigned grid = (unsigned)((op.g.V + threads - 1) / threads);
  links_to_cm_kernel<<<grid, threads, 0, st>>>(op.links, op.links32, op.g.V);
  clover_to_cm_kernel<<<grid, threads, 0, st>>>(op.clov_inv, op.clov_inv32, op.g.V);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ FP32 sweep, split stencil
// The same sweep with the stencil of one (site, rhs) pair split over two warps: in every group of
// 64 threads, warp 0 takes the x and y hops and warp 1 the z and t hops of the same 32 pairs; the
// partial sums meet in shared memory, and warp 0 then applies the chirality + block of A_D^{-1}
// while warp 1 applies the chirality - block.  Twice as many warps cover the same pairs.
namespace {

template <typename TY>
__global__ void __launch_bounds__(128)
jacobi_f32_split_kernel(const float* __restrict__ x, TY* __restrict__ y, const float* __restrict__ u,
                        const float* __restrict__ links, const float* __restrict__ clov_inv, Geom g,
                        int L, float kappa) {
  __shared__ float xch[2][2][12][2][32];   // [group][warp half][component][re/im][lane]
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;       // 0..3
  const int grp = warp >> 1, half = warp & 1;
  const long long pair = ((long long)blockIdx.x * 2 + grp) * 32 + lane;
  const bool valid = pair < (long long)g.V * L;
  const int s = valid ? (int)(pair / L) : 0;
  const int r = valid ? (int)(pair - (long long)s * L) : 0;
  const size_t V = (size_t)g.V;
  Cx<float> au[2][3], ad[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) { au[a][b] = czero<float>(); ad[a][b] = czero<float>(); }
  if (valid) {
    int c[4];
    site_coords(g, s, c);
    Cx<float> pu[1][2][3], pd[1][2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) { pu[0][a][b] = czero<float>(); pd[0][a][b] = czero<float>(); }
    if (half == 0) {
      hop_cm<0, +1, 1>(x, links, g, s, c, r, L, pu, pd);
      hop_cm<0, -1, 1>(x, links, g, s, c, r, L, pu, pd);
      hop_cm<1, +1, 1>(x, links, g, s, c, r, L, pu, pd);
      hop_cm<1, -1, 1>(x, links, g, s, c, r, L, pu, pd);
    } else {
      hop_cm<2, +1, 1>(x, links, g, s, c, r, L, pu, pd);
      hop_cm<2, -1, 1>(x, links, g, s, c, r, L, pu, pd);
      hop_cm<3, +1, 1>(x, links, g, s, c, r, L, pu, pd);
      hop_cm<3, -1, 1>(x, links, g, s, c, r, L, pu, pd);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) { au[a][b] = pu[0][a][b]; ad[a][b] = pd[0][a][b]; }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    xch[grp][half][k][0][lane] = au[k / 3][k % 3].re;
    xch[grp][half][k][1][lane] = au[k / 3][k % 3].im;
    xch[grp][half][6 + k][0][lane] = ad[k / 3][k % 3].re;
    xch[grp][half][6 + k][1][lane] = ad[k / 3][k % 3].im;
  }
  __syncthreads();
  if (!valid) return;
  // warp half 0: chirality + (components 0..5); half 1: chirality - (components 6..11)
  const int ch = half;
  Cx<float> vin[6], out[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const int k = ch * 6 + i;
    const Cx<float> hs = {xch[grp][0][k][0][lane] + xch[grp][1][k][0][lane],
                          xch[grp][0][k][1][lane] + xch[grp][1][k][1][lane]};
    vin[i] = ldc(u + 2 * (((size_t)k * V + s) * L + r)) + kappa * hs;
  }
  herm6s(clov_inv + (size_t)ch * CLOV_REALS * V + s, V, vin, out);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const int k = ch * 6 + i;
    TY* p = sizeof(TY) == 4 ? y + 2 * (((size_t)k * V + s) * L + r)
                            : y + 2 * (((size_t)s * 12 + k) * L + r);
    stc(p, cmake<TY>(TY(out[i].re), TY(out[i].im)));
  }
}

}  // namespace

cudaError_t launch_jacobi_f32_split(const Op& op, const float* g_in, const float* u32, float* g32,
                                    double* g64, int L, cudaStream_t st) {
  const long long pairs = (long long)op.g.V * L;
  const unsigned grid = (unsigned)((pairs + 63) / 64);   // 64 pairs per 128-thread CTA
  if (g32)
    jacobi_f32_split_kernel<float><<<grid, 128, 0, st>>>(g_in, g32, u32, op.links32,
                                                         op.clov_inv32, op.g, L, (float)op.kappa);
  else
    jacobi_f32_split_kernel<double><<<grid, 128, 0, st>>>(g_in, g64, u32, op.links32,
                                                          op.clov_inv32, op.g, L, (float)op.kappa);
  return cudaGetLastError();
}
