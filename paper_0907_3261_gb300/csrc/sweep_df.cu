// Double-float Jacobi sweeps of the preconditioner M (arXiv:0907.3261, Sec. 2: G^0 = 0,
// G^{i+1} = A_D^{-1}(U + kappa H G^i) for i < j) on the FP32 pipes.
//
// Block BiCGGR needs M to be a fixed linear operator.  Rounding the stored operator (links, A_D^{-1}
// and kappa in FP32) changes which linear operator M is, which the method tolerates; rounding in
// the arithmetic on the spinors makes M non-linear, which near the critical kappa stalls it when
// the rounding is FP32's.  So these sweeps keep the operator in FP32 and carry every spinor value
// as an unevaluated sum hi + lo of two FP32 numbers (about 48 significant bits): each product of
// an FP32 operator entry with a spinor value is split exactly into p + e with an FMA (Dekker), and
// sums use Knuth's two-sum, so M is linear to ~1e-14.  On GB300, where FP64 runs at 1/61 of the
// FP32 rate, this is several times faster than FP64 sweeps.
//
// Blocks are component-major, [spin*3+colour][site][rhs], one float4 (re.hi, re.lo, im.hi,
// im.lo) per complex number; one thread owns one (site, rhs) pair.  The first sweep converts the
// FP64 right-hand side and stores its double-float copy; the last writes FP64 site-major.
#include <type_traits>

#include "common.cuh"
#include "elem.cuh"
#include "internal.h"

namespace {

// ------------------------------------------------------------------ double-float helpers
WD_DEV DF dfz() { return {0.f, 0.f}; }
WD_DEV DF dneg(DF a) { return {-a.hi, -a.lo}; }
// a + b, result unnormalised (hi carries the sum, lo the accumulated errors)
WD_DEV DF dadd(DF a, DF b) {
  float s, t;
  two_sum(a.hi, b.hi, s, t);
  return {s, __fadd_rn(__fadd_rn(a.lo, b.lo), t)};
}
WD_DEV DF dsub(DF a, DF b) { return dadd(a, dneg(b)); }
// acc + a b for an FP32 operator entry a: a b.hi = p + e exactly, a b.lo in FP32
WD_DEV void dmac(DF& acc, float a, DF b) {
  const float p = __fmul_rn(a, b.hi);
  float e = __fmaf_rn(a, b.hi, -p);
  e = __fmaf_rn(a, b.lo, e);
  float s, t;
  two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}

using C = CDF;
WD_DEV C cz() { return {dfz(), dfz()}; }
WD_DEV C cadd(C a, C b) { return {dadd(a.re, b.re), dadd(a.im, b.im)}; }
WD_DEV C csub(C a, C b) { return {dsub(a.re, b.re), dsub(a.im, b.im)}; }
WD_DEV C cneg(C a) { return {dneg(a.re), dneg(a.im)}; }
WD_DEV C cti(C a) { return {dneg(a.im), a.re}; }    // i a
WD_DEV C ctmi(C a) { return {a.im, dneg(a.re)}; }   // -i a
// acc + a b and acc + conj(a) b for an FP32 complex a
WD_DEV void cmac(C& acc, Cx<float> a, C b) {
  dmac(acc.re, a.re, b.re);
  dmac(acc.re, -a.im, b.im);
  dmac(acc.im, a.re, b.im);
  dmac(acc.im, a.im, b.re);
}
WD_DEV void cmacj(C& acc, Cx<float> a, C b) {
  dmac(acc.re, a.re, b.re);
  dmac(acc.re, a.im, b.im);
  dmac(acc.im, a.re, b.im);
  dmac(acc.im, -a.im, b.re);
}

WD_DEV C ldq(const float4* p) {
  const float4 a = __ldg(p);
  return {{a.x, a.y}, {a.z, a.w}};
}
WD_DEV void stq(float4* p, C z) {
  const DF re = df_norm(z.re), im = df_norm(z.im);
  *p = make_float4(re.hi, re.lo, im.hi, im.lo);
}
WD_DEV void stq(double* p, C z) { stc(p, cdf_to(z)); }

// Address of component k of (site s, rhs r): component-major element, or site-major FP64.
template <typename TY>
WD_DEV TY* at(TY* y, size_t V, int L, int s, int k, int r) {
  if constexpr (std::is_same<TY, double>::value)
    return y + 2 * (((size_t)s * 12 + k) * L + r);
  else
    return y + ((size_t)k * V + s) * L + r;
}

// G_mu d and G_mu^H w of the chiral basis (see dslash.cu) on double-float values.
template <int MU>
WD_DEV void gdown(C d0, C d1, C& g0, C& g1) {
  if constexpr (MU == 0) { g0 = ctmi(d1); g1 = ctmi(d0); }
  else if constexpr (MU == 1) { g0 = cneg(d1); g1 = d0; }
  else if constexpr (MU == 2) { g0 = ctmi(d0); g1 = cti(d1); }
  else { g0 = d0; g1 = d1; }
}
template <int MU>
WD_DEV void gup(C w0, C w1, C& g0, C& g1) {
  if constexpr (MU == 0) { g0 = cti(w1); g1 = cti(w0); }
  else if constexpr (MU == 1) { g0 = w1; g1 = cneg(w0); }
  else if constexpr (MU == 2) { g0 = cti(w0); g1 = ctmi(w1); }
  else { g0 = w0; g1 = w1; }
}

// The 3x3 FP32 link with entry (a, b) at U[(3a + b) V]; row 2 read or rebuilt (SU(3)).
WD_DEV void link(const float2* __restrict__ U, size_t V, bool link12, Cx<float> m[3][3]) {
#pragma unroll
  for (int e = 0; e < 6; ++e) m[e / 3][e % 3] = lp::ld1(U + e * V);
  if (link12) {
    m[2][0] = conj(cmul(m[0][1], m[1][2]) - cmul(m[0][2], m[1][1]));
    m[2][1] = conj(cmul(m[0][2], m[1][0]) - cmul(m[0][0], m[1][2]));
    m[2][2] = conj(cmul(m[0][0], m[1][1]) - cmul(m[0][1], m[1][0]));
  } else {
#pragma unroll
    for (int b = 0; b < 3; ++b) m[2][b] = lp::ld1(U + (6 + b) * V);
  }
}

// Adds (1 - DIR g_mu) W x(s + DIR mu) to (au, ad); W = U_mu(s) (DIR = +1) or U_mu(s - mu)^H.
template <int MU, int DIR>
WD_DEV void hop(const float4* __restrict__ x, const float2* __restrict__ links, const Geom& g,
                int s, const int c[4], int r, int L, bool link12, C au[2][3], C ad[2][3]) {
  const int sn = neighbour(g, s, c, MU, DIR);
  const size_t V = (size_t)g.V;
  const float4* base = x + (size_t)sn * L + r;
  const size_t cs = V * L;
  C h0[3], h1[3];
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    const C u0 = ldq(base + (0 * 3 + col) * cs), u1 = ldq(base + (1 * 3 + col) * cs);
    const C d0 = ldq(base + (2 * 3 + col) * cs), d1 = ldq(base + (3 * 3 + col) * cs);
    C g0, g1;
    gdown<MU>(d0, d1, g0, g1);
    if constexpr (DIR > 0) { h0[col] = csub(u0, g0); h1[col] = csub(u1, g1); }
    else { h0[col] = cadd(u0, g0); h1[col] = cadd(u1, g1); }
  }
  Cx<float> m[3][3];
  link(links + (size_t)MU * 9 * V + (DIR > 0 ? s : sn), V, link12, m);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    C w0 = cz(), w1 = cz();
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if constexpr (DIR > 0) { cmac(w0, m[a][b], h0[b]); cmac(w1, m[a][b], h1[b]); }
      else { cmacj(w0, m[b][a], h0[b]); cmacj(w1, m[b][a], h1[b]); }
    }
    C g0, g1;
    gup<MU>(w0, w1, g0, g1);
    au[0][a] = cadd(au[0][a], w0);
    au[1][a] = cadd(au[1][a], w1);
    if constexpr (DIR > 0) { ad[0][a] = csub(ad[0][a], g0); ad[1][a] = csub(ad[1][a], g1); }
    else { ad[0][a] = cadd(ad[0][a], g0); ad[1][a] = cadd(ad[1][a], g1); }
  }
}

// out = M v for a packed Hermitian 6x6 FP32 block with entries `stride` apart.
WD_DEV void herm6(const float* __restrict__ m, size_t stride, const C v[6], C out[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float d = __ldg(m + i * stride);
    out[i] = cz();
    dmac(out[i].re, d, v[i].re);
    dmac(out[i].im, d, v[i].im);
  }
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      const int t = tri_index(i, j);
      const Cx<float> l = cmake<float>(__ldg(m + t * stride), __ldg(m + (t + 1) * stride));
      cmac(out[i], l, v[j]);
      cmacj(out[j], l, v[i]);
    }
}

// kappa h added to u (kappa an FP32 operator constant)
WD_DEV C axpy(float kappa, C h, C u) {
  dmac(u.re, kappa, h.re);
  dmac(u.im, kappa, h.im);
  return u;
}

template <typename TY>
__global__ void __launch_bounds__(128)
sweep_df_kernel(const float4* __restrict__ x, TY* __restrict__ y, const float4* __restrict__ u,
                const float2* __restrict__ links, const float* __restrict__ clov_inv, Geom g,
                int L, float kappa, int link12) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.V * L) return;
  const int s = tid / L;
  const int r = tid - s * L;
  const size_t V = (size_t)g.V;
  const bool l12 = link12 != 0;
  int c[4];
  site_coords(g, s, c);
  C au[2][3], ad[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) { au[a][b] = cz(); ad[a][b] = cz(); }
  hop<0, +1>(x, links, g, s, c, r, L, l12, au, ad);
  hop<0, -1>(x, links, g, s, c, r, L, l12, au, ad);
  hop<1, +1>(x, links, g, s, c, r, L, l12, au, ad);
  hop<1, -1>(x, links, g, s, c, r, L, l12, au, ad);
  hop<2, +1>(x, links, g, s, c, r, L, l12, au, ad);
  hop<2, -1>(x, links, g, s, c, r, L, l12, au, ad);
  hop<3, +1>(x, links, g, s, c, r, L, l12, au, ad);
  hop<3, -1>(x, links, g, s, c, r, L, l12, au, ad);
#pragma unroll
  for (int ch = 0; ch < 2; ++ch) {
    C vin[6], out[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int k = ch * 6 + i;
      vin[i] = axpy(kappa, ch == 0 ? au[i / 3][i % 3] : ad[i / 3][i % 3],
                    ldq(u + ((size_t)k * V + s) * L + r));
    }
    herm6(clov_inv + (size_t)ch * CLOV_REALS * V + s, V, vin, out);
#pragma unroll
    for (int i = 0; i < 6; ++i) stq(at(y, V, L, s, ch * 6 + i, r), out[i]);
  }
}

// First sweep from G = 0: stores the double-float copy of the FP64 right-hand side (when u_df is
// not null) and writes G = A_D^{-1} U.
template <typename TY>
__global__ void __launch_bounds__(128)
site_inverse_df_kernel(const double* __restrict__ u, float4* __restrict__ u_df, TY* __restrict__ y,
                       const float* __restrict__ clov_inv, int V, int L) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= V * L) return;
  const int s = tid / L;
  const int r = tid - s * L;
  const size_t base = 2 * ((size_t)s * 12 * L + r);
  C vin[2][6], out[2][6];
#pragma unroll
  for (int ch = 0; ch < 2; ++ch)
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int k = ch * 6 + i;
      vin[ch][i] = cdf_from(ldc(u + base + 2 * (size_t)(k * L)));
      if (u_df) stq(at(u_df, (size_t)V, L, s, k, r), vin[ch][i]);
    }
  herm6(clov_inv + s, (size_t)V, vin[0], out[0]);
  herm6(clov_inv + (size_t)CLOV_REALS * V + s, (size_t)V, vin[1], out[1]);
#pragma unroll
  for (int ch = 0; ch < 2; ++ch)
#pragma unroll
    for (int i = 0; i < 6; ++i) stq(at(y, (size_t)V, L, s, ch * 6 + i, r), out[ch][i]);
}

}  // namespace

cudaError_t launch_site_inverse_df(const Op& op, const double* u, void* u_df, void* g_df,
                                   double* g64, int L, cudaStream_t st) {
  const unsigned grid = (unsigned)(((long long)op.g.V * L + 127) / 128);
  float4* ud = static_cast<float4*>(u_df);
  if (g_df)
    site_inverse_df_kernel<float4><<<grid, 128, 0, st>>>(u, ud, static_cast<float4*>(g_df),
                                                         op.clov_inv32, op.g.V, L);
  else
    site_inverse_df_kernel<double><<<grid, 128, 0, st>>>(u, ud, g64, op.clov_inv32, op.g.V, L);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_df(const Op& op, const void* g_in, const void* u_df, void* g_df,
                             double* g64, int L, int block, cudaStream_t st) {
  if (block != 64 && block != 128) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)(((long long)op.g.V * L + block - 1) / block);
  const float4* x = static_cast<const float4*>(g_in);
  const float4* u = static_cast<const float4*>(u_df);
  const float2* links = reinterpret_cast<const float2*>(op.links32);
  if (g_df)
    sweep_df_kernel<float4><<<grid, block, 0, st>>>(x, static_cast<float4*>(g_df), u, links,
                                                    op.clov_inv32, op.g, L, (float)op.kappa,
                                                    op.link12);
  else
    sweep_df_kernel<double><<<grid, block, 0, st>>>(x, g64, u, links, op.clov_inv32, op.g, L,
                                                    (float)op.kappa, op.link12);
  return cudaGetLastError();
}
