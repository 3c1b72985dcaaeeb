// Double-float Jacobi sweeps of the preconditioner M (arXiv:0907.3261, Sec. 2: G^0 = 0,
// G^{i+1} = A_D^{-1}(U + kappa H G^i) for i < j) on the FP32 pipes.
//
// Block BiCGGR needs M to be a fixed linear operator.  Rounding the stored operator (links, A_D^{-1}
// and kappa in FP32) changes which linear operator M is, which the method tolerates; rounding in
// the arithmetic on the spinors makes M non-linear, which near the critical kappa stalls it when
// the rounding is FP32's.  So these sweeps keep the operator in FP32 and carry every spinor value
// as an unevaluated sum hi + lo of two FP32 numbers (about 48 significant bits): each product of
// an FP32 operator entry with a spinor value is split exactly into p + e with an FMA (Dekker), and
// sums use Knuth's two-sum, so M is linear to ~1e-13.  On GB300, where FP64 runs at 1/61 of the
// FP32 rate, this is several times faster than FP64 sweeps.  The scalar kernel does the FP32 work
// one operation per instruction; the packed one (below) puts the real and imaginary halves in the
// two lanes of FP32x2 instructions.
//
// Blocks are component-major, [spin*3+colour][site][rhs], one float4 (re.hi, im.hi, re.lo,
// im.lo) per complex number; one thread owns one site and 1 or 2 consecutive right-hand sides.
// The first sweep converts the FP64 right-hand side from its bit fields and stores its
// double-float copy; the last writes FP64 site-major.
#include <type_traits>

#include "common.cuh"
#include "elem.cuh"
#include "internal.h"

namespace {

// ------------------------------------------------------------------ double-float helpers
WD_DEV DF dfz() { return {0.f, 0.f}; }
// a + b, result unnormalised (hi carries the sum, lo the accumulated errors)
WD_DEV DF dadd(DF a, DF b) {
  float s, t;
  two_sum(a.hi, b.hi, s, t);
  return {s, __fadd_rn(__fadd_rn(a.lo, b.lo), t)};
}
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

// a b for an FP32 operator entry a, as the first term of a sum (no addition needed)
WD_DEV DF dmul(float a, DF b) {
  const float p = __fmul_rn(a, b.hi);
  float e = __fmaf_rn(a, b.hi, -p);
  return {p, __fmaf_rn(a, b.lo, e)};
}

using C = CDF;
WD_DEV C cz() { return {dfz(), dfz()}; }
WD_DEV C cadd(C a, C b) { return {dadd(a.re, b.re), dadd(a.im, b.im)}; }
// acc + a b and acc + conj(a) b for an FP32 complex a
WD_DEV C cmul1(Cx<float> a, C b) {   // a b, the first term of a sum
  C acc = {dmul(a.re, b.re), dmul(a.re, b.im)};
  dmac(acc.re, -a.im, b.im);
  dmac(acc.im, a.im, b.re);
  return acc;
}
WD_DEV void cmac(C& acc, Cx<float> a, C b) {
  dmac(acc.re, a.re, b.re);
  dmac(acc.re, -a.im, b.im);
  dmac(acc.im, a.re, b.im);
  dmac(acc.im, a.im, b.re);
}

// A stored element is (re.hi, im.hi, re.lo, im.lo): the two high words, then the two low words,
// so that the packed kernel gets its (re, im) lane pairs straight from one 16-byte load.
WD_DEV C ldq(const float4* p) {
  const float4 a = __ldg(p);
  return {{a.x, a.z}, {a.y, a.w}};
}
WD_DEV void stq(float4* p, C z) {
  const DF re = df_norm(z.re), im = df_norm(z.im);
  *p = make_float4(re.hi, im.hi, re.lo, im.lo);
}
WD_DEV void stq(double* p, C z) { stc(p, cdf_join(z)); }

// Address of component k of (site s, rhs r): component-major element, or site-major FP64.
template <typename TY>
WD_DEV TY* at(TY* y, size_t V, int L, int s, int k, int r) {
  if constexpr (std::is_same<TY, double>::value)
    return y + 2 * (((size_t)s * 12 + k) * L + r);
  else
    return y + ((size_t)k * V + s) * L + r;
}

// a + sg b for sg = +1 or -1, with the sign folded into FMAs: fma(sg, b, a) rounds a + sg b once,
// exactly as an addition would, so this is two-sum on (a, sg b) at no extra cost.
WD_DEV DF dadd_s(DF a, DF b, float sg) {
  const float s = __fmaf_rn(sg, b.hi, a.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fmaf_rn(sg, b.hi, -bb));
  return {s, __fadd_rn(__fmaf_rn(sg, b.lo, a.lo), t)};
}
// (re, im) or (im, re)
WD_DEV C cswap(C z, bool swap) { return {swap ? z.im : z.re, swap ? z.re : z.im}; }

// Spin structure of direction mu (chiral basis, see dslash.cu).  The hop multiplies
// h = x_up - dir G_mu x_down by the link and adds w to the upper and -dir G_mu^H w to the lower
// half.  Each G_mu is a signed, possibly re/im-swapped, diagonal or anti-diagonal of
// {1, -1, i, -i}:  G_0 d = (-i d1, -i d0), G_1 d = (-d1, d0), G_2 d = (-i d0, i d1),
// G_3 d = (d0, d1); G_0^H w = (i w1, i w0), G_1^H w = (w1, -w0), G_2^H w = (i w0, -i w1).
// `cross` picks the anti-diagonal, `swap` multiplication by +-i, and the signs are those of the
// (re, im) parts of slot 0 and slot 1, before the factor -dir.
// Per direction d = 2 mu + (0 forward, 1 backward): the signs of (re, im) of slot 0 and slot 1 of
// -dir G_mu x_down (dn) and of -dir G_mu^H w (up).  Read with a warp-uniform index.
__constant__ float c_spin_dn[8][4] = {
    {-1, 1, -1, 1}, {1, -1, 1, -1},     // mu 0: -i, -i
    {1, 1, -1, -1}, {-1, -1, 1, 1},     // mu 1: -1, +1
    {-1, 1, 1, -1}, {1, -1, -1, 1},     // mu 2: -i, +i
    {-1, -1, -1, -1}, {1, 1, 1, 1}};    // mu 3: +1, +1
__constant__ float c_spin_up[8][4] = {
    {1, -1, 1, -1}, {-1, 1, -1, 1},     // mu 0: +i, +i
    {-1, -1, 1, 1}, {1, 1, -1, -1},     // mu 1: +1, -1
    {1, -1, -1, 1}, {-1, 1, 1, -1},     // mu 2: +i, -i
    {-1, -1, -1, -1}, {1, 1, 1, 1}};    // mu 3: +1, +1
struct SpinDir {
  bool cross, swap;
  float dn[4], up[4];
};
WD_DEV SpinDir spin_dir(int d) {
  SpinDir t;
  t.cross = d < 4;
  t.swap = ((d >> 1) & 1) == 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) { t.dn[k] = c_spin_dn[d][k]; t.up[k] = c_spin_up[d][k]; }
  return t;
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

// The hopping term H x at (s, r), accumulated into (au, ad) over the 8 directions in one rolled,
// branch-free loop body: one copy of code serves every direction (which keeps the kernel inside
// the instruction cache), the spin structure enters through load addresses, selects and signs
// folded into the two-sum additions, and the backward link U_mu(s - mu)^H is conjugate-transposed
// in registers.
template <int R>
WD_DEV void hopping(const float4* __restrict__ x, const float2* __restrict__ links, const Geom& g,
                    int s, const int c[4], int r, int L, bool link12, C au[R][2][3],
                    C ad[R][2][3]) {
  const size_t V = (size_t)g.V;
  const size_t cs = V * L;
#pragma unroll 1
  for (int d = 0; d < 8; ++d) {
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    const int cm = mu == 0 ? c[0] : mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
    const int ext = g.d[mu], str = g.stride[mu];
    const int sn = fwd ? (cm == ext - 1 ? s - (ext - 1) * str : s + str)
                       : (cm == 0 ? s + (ext - 1) * str : s - str);
    const SpinDir sd = spin_dir(d);
    const float4* base = x + (size_t)sn * L + r;
    const int k0 = sd.cross ? 9 : 6, k1 = sd.cross ? 6 : 9;   // lower-spin rows feeding slots 0, 1
    C h0[R][3], h1[R][3];
#pragma unroll
    for (int col = 0; col < 3; ++col)
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const C u0 = ldq(base + (0 * 3 + col) * cs + q), u1 = ldq(base + (1 * 3 + col) * cs + q);
        const C x0 = cswap(ldq(base + (k0 + col) * cs + q), sd.swap);
        const C x1 = cswap(ldq(base + (k1 + col) * cs + q), sd.swap);
        h0[q][col] = {dadd_s(u0.re, x0.re, sd.dn[0]), dadd_s(u0.im, x0.im, sd.dn[1])};
        h1[q][col] = {dadd_s(u1.re, x1.re, sd.dn[2]), dadd_s(u1.im, x1.im, sd.dn[3])};
      }
    Cx<float> m[3][3];
    link(links + (size_t)mu * 9 * V + (fwd ? s : sn), V, link12, m);
    if (!fwd) {   // W = m^H
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a + 1; b < 3; ++b) {
          const Cx<float> t = m[a][b];
          m[a][b] = conj(m[b][a]);
          m[b][a] = conj(t);
        }
#pragma unroll
      for (int a = 0; a < 3; ++a) m[a][a] = conj(m[a][a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int q = 0; q < R; ++q) {
        C w0 = cmul1(m[a][0], h0[q][0]), w1 = cmul1(m[a][0], h1[q][0]);
#pragma unroll
        for (int b = 1; b < 3; ++b) { cmac(w0, m[a][b], h0[q][b]); cmac(w1, m[a][b], h1[q][b]); }
        au[q][0][a] = cadd(au[q][0][a], w0);
        au[q][1][a] = cadd(au[q][1][a], w1);
        const C y0 = cswap(sd.cross ? w1 : w0, sd.swap), y1 = cswap(sd.cross ? w0 : w1, sd.swap);
        ad[q][0][a] = {dadd_s(ad[q][0][a].re, y0.re, sd.up[0]), dadd_s(ad[q][0][a].im, y0.im, sd.up[1])};
        ad[q][1][a] = {dadd_s(ad[q][1][a].re, y1.re, sd.up[2]), dadd_s(ad[q][1][a].im, y1.im, sd.up[3])};
      }
  }
}

// Row i of a packed Hermitian 6x6 FP32 block (entries `stride` apart) times v: M_ij = l_ij below
// the diagonal, conj(l_ji) above it, the real d_i on it (taken as a complex entry with a zero
// imaginary part, which adds exact zeros and keeps the row branch-free).  Called in a rolled loop
// over i.
// Offset of the real part of M_ij in the packed block (the diagonal reals first, then the
// strictly-lower pairs), and the sign of the imaginary part: 0 on the diagonal (no imaginary part),
// +1 below it, -1 above it (conjugate of the lower entry).
__constant__ int c_h6_off[6][6] = {
    {0, 6, 8, 12, 18, 26}, {6, 1, 10, 14, 20, 28}, {8, 10, 2, 16, 22, 30},
    {12, 14, 16, 3, 24, 32}, {18, 20, 22, 24, 4, 34}, {26, 28, 30, 32, 34, 5}};
__constant__ float c_h6_sgn[6][6] = {
    {0, -1, -1, -1, -1, -1}, {1, 0, -1, -1, -1, -1}, {1, 1, 0, -1, -1, -1},
    {1, 1, 1, 0, -1, -1}, {1, 1, 1, 1, 0, -1}, {1, 1, 1, 1, 1, 0}};

template <int R>
WD_DEV void herm6_row(const float* __restrict__ m, size_t stride, int i, const C v[R][6],
                      C acc[R]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int t = c_h6_off[i][j];
    const float sg = c_h6_sgn[i][j];
    const float re = __ldg(m + t * stride);
    const float im = __ldg(m + (t + (sg != 0.f)) * stride);   // the diagonal reads itself twice
    const Cx<float> l = cmake<float>(re, sg * im);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (j == 0) acc[q] = cmul1(l, v[q][0]);
      else cmac(acc[q], l, v[q][j]);
    }
  }
}

// kappa h added to u (kappa an FP32 operator constant)
WD_DEV C axpy(float kappa, C h, C u) {
  dmac(u.re, kappa, h.re);
  dmac(u.im, kappa, h.im);
  return u;
}

// R consecutive right-hand sides per thread (R = 1 or 2 dividing L); the links, the spin
// constants and the clover entries serve all R.
template <int R, typename TY>
__global__ void __launch_bounds__(128, R == 1 ? 4 : 2)
sweep_df_kernel(const float4* __restrict__ x, TY* __restrict__ y, const float4* __restrict__ u,
                const float2* __restrict__ links, const float* __restrict__ clov_inv, Geom g,
                int L, float kappa, int link12) {
  const int groups = L / R;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.V * groups) return;
  const int s = tid / groups;
  const int r = (tid - s * groups) * R;
  const size_t V = (size_t)g.V;
  int c[4];
  site_coords(g, s, c);
  C au[R][2][3], ad[R][2][3];
#pragma unroll
  for (int q = 0; q < R; ++q)
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) { au[q][a][b] = cz(); ad[q][a][b] = cz(); }
  hopping<R>(x, links, g, s, c, r, L, link12 != 0, au, ad);
#pragma unroll 1
  for (int ch = 0; ch < 2; ++ch) {
    C vin[R][6];
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const int k = ch * 6 + i;
        vin[q][i] = axpy(kappa, ch == 0 ? au[q][i / 3][i % 3] : ad[q][i / 3][i % 3],
                         ldq(u + ((size_t)k * V + s) * L + r + q));
      }
    const float* m = clov_inv + (size_t)ch * CLOV_REALS * V + s;
#pragma unroll 1
    for (int i = 0; i < 6; ++i) {
      C out[R];
      herm6_row<R>(m, V, i, vin, out);
#pragma unroll
      for (int q = 0; q < R; ++q) stq(at(y, V, L, s, ch * 6 + i, r + q), out[q]);
    }
  }
}

// ------------------------------------------------------------------ packed variant
// The same sweep with the real and imaginary halves of every double-float value in the two lanes
// of FP32x2 instructions (FFMA2/FADD2/FMUL2, each lane an IEEE round-to-nearest operation), which
// cuts the instructions the scheduler issues by about a third (the FMA pipe then sets the pace).
// A value is hi = (re.hi, im.hi), lo = (re.lo, im.lo) (helpers in common.cuh).  Subtractions are FMAs with a (-1, -1) operand (negation is exact).  A complex product
// sum  sum_b a_b h_b  is accumulated as X = sum ar_b (h_b.re, h_b.im) and Y = sum ai_b (h_b.re,
// h_b.im) with broadcast operator lanes, and combined once: (re, im) = X + (-Y.im, Y.re).
WD_DEV P2 psel(bool c, P2 a, P2 b) { return c ? a : b; }

// acc + a b for an FP32 operator value a broadcast to both lanes (na = -a).
WD_DEV void pmac(P2& acc, float2 a, float2 na, P2 b, float2 m1) {
  const float2 np = __fmul2_rn(na, b.hi);   // -(a b.hi), rounded
  float2 e = __ffma2_rn(a, b.hi, np);       // the rounding error of a b.hi, exactly
  e = __ffma2_rn(a, b.lo, e);
  float2 s, t;
  two_sum2(acc.hi, np, m1, m1, s, t);       // acc.hi - np
  acc.hi = s;
  acc.lo = __fadd2_rn(acc.lo, __fadd2_rn(t, e));
}
WD_DEV P2 pmul(float2 a, float2 na, P2 b) {   // a b as the first term of a sum
  const float2 p = __fmul2_rn(a, b.hi);
  const float2 np = __fmul2_rn(na, b.hi);
  const float2 e = __ffma2_rn(a, b.hi, np);
  return {p, __ffma2_rn(a, b.lo, e)};
}

WD_DEV P2 ldq2(const float4* p) {
  const float4 a = __ldg(p);
  return {make_float2(a.x, a.y), make_float2(a.z, a.w)};
}
WD_DEV void stq2(float4* p, P2 z, float2 m1) {   // renormalise both lanes, then store
  const float2 s = __fadd2_rn(z.hi, z.lo);
  const float2 lo = __ffma2_rn(__ffma2_rn(z.hi, m1, s), m1, z.lo);   // lo - (s - hi)
  *p = make_float4(s.x, s.y, lo.x, lo.y);
}
WD_DEV void stq2(double* p, P2 z, float2) {
  stc(p, cmake<double>(f_widen(z.hi.x) + f_widen(z.lo.x), f_widen(z.hi.y) + f_widen(z.lo.y)));
}

// The hopping term H x at (s, r) in packed arithmetic (one rolled, branch-free loop body as in
// hopping<R>).
WD_DEV void hopping2(const float4* __restrict__ x, const float2* __restrict__ links, const Geom& g,
                     int s, const int c[4], int r, int L, bool link12, P2 au[2][3], P2 ad[2][3],
                     float2 m1) {
  const size_t V = (size_t)g.V;
  const size_t cs = V * L;
  const float2 one = make_float2(1.f, 1.f);
#pragma unroll 1
  for (int d = 0; d < 8; ++d) {
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    const int cm = mu == 0 ? c[0] : mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
    const int ext = g.d[mu], str = g.stride[mu];
    const int sn = fwd ? (cm == ext - 1 ? s - (ext - 1) * str : s + str)
                       : (cm == 0 ? s + (ext - 1) * str : s - str);
    const SpinDir sd = spin_dir(d);
    const float2 dn0 = make_float2(sd.dn[0], sd.dn[1]), dn1 = make_float2(sd.dn[2], sd.dn[3]);
    const float2 up0 = make_float2(sd.up[0], sd.up[1]), up1 = make_float2(sd.up[2], sd.up[3]);
    const float4* base = x + (size_t)sn * L + r;
    const int k0 = sd.cross ? 9 : 6, k1 = sd.cross ? 6 : 9;
    P2 h0[3], h1[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      const P2 u0 = ldq2(base + (0 * 3 + col) * cs), u1 = ldq2(base + (1 * 3 + col) * cs);
      const P2 x0 = ldq2(base + (k0 + col) * cs), x1 = ldq2(base + (k1 + col) * cs);
      h0[col] = padd(u0, psel(sd.swap, pswap(x0), x0), dn0, m1);
      h1[col] = padd(u1, psel(sd.swap, pswap(x1), x1), dn1, m1);
    }
    Cx<float> m[3][3];
    link(links + (size_t)mu * 9 * V + (fwd ? s : sn), V, link12, m);
    if (!fwd) {   // W = m^H
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a + 1; b < 3; ++b) {
          const Cx<float> t = m[a][b];
          m[a][b] = conj(m[b][a]);
          m[b][a] = conj(t);
        }
#pragma unroll
      for (int a = 0; a < 3; ++a) m[a][a] = conj(m[a][a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float2 r0 = dup(m[a][0].re), nr0 = dup(-m[a][0].re);
      const float2 i0 = dup(m[a][0].im), ni0 = dup(-m[a][0].im);
      P2 X0 = pmul(r0, nr0, h0[0]), Y0 = pmul(i0, ni0, h0[0]);
      P2 X1 = pmul(r0, nr0, h1[0]), Y1 = pmul(i0, ni0, h1[0]);
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        const float2 rb = dup(m[a][b].re), nrb = dup(-m[a][b].re);
        const float2 ib = dup(m[a][b].im), nib = dup(-m[a][b].im);
        pmac(X0, rb, nrb, h0[b], m1);
        pmac(Y0, ib, nib, h0[b], m1);
        pmac(X1, rb, nrb, h1[b], m1);
        pmac(Y1, ib, nib, h1[b], m1);
      }
      const P2 w0 = pcombine(X0, Y0, m1), w1 = pcombine(X1, Y1, m1);
      au[0][a] = padd(au[0][a], w0, one, m1);
      au[1][a] = padd(au[1][a], w1, one, m1);
      const P2 y0 = psel(sd.cross, w1, w0), y1 = psel(sd.cross, w0, w1);
      ad[0][a] = padd(ad[0][a], psel(sd.swap, pswap(y0), y0), up0, m1);
      ad[1][a] = padd(ad[1][a], psel(sd.swap, pswap(y1), y1), up1, m1);
    }
  }
}

// Row i of a packed Hermitian 6x6 FP32 block times v (as herm6_row), in packed arithmetic.
WD_DEV P2 herm6_row2(const float* __restrict__ m, size_t stride, int i, const P2 v[6], float2 m1) {
  P2 X, Y;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int t = c_h6_off[i][j];
    const float sg = c_h6_sgn[i][j];
    const float re = __ldg(m + t * stride);
    const float im = sg * __ldg(m + (t + (sg != 0.f)) * stride);
    if (j == 0) {
      X = pmul(dup(re), dup(-re), v[0]);
      Y = pmul(dup(im), dup(-im), v[0]);
    } else {
      pmac(X, dup(re), dup(-re), v[j], m1);
      pmac(Y, dup(im), dup(-im), v[j], m1);
    }
  }
  return pcombine(X, Y, m1);
}

template <typename TY>
__global__ void __launch_bounds__(128, 4)
sweep_df2_kernel(const float4* __restrict__ x, TY* __restrict__ y, const float4* __restrict__ u,
                 const float2* __restrict__ links, const float* __restrict__ clov_inv, Geom g,
                 int L, float kappa, int link12) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.V * L) return;
  const int s = tid / L;
  const int r = tid - s * L;
  const size_t V = (size_t)g.V;
  const float2 m1 = make_float2(-1.f, -1.f);
  int c[4];
  site_coords(g, s, c);
  P2 au[2][3], ad[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) { au[a][b] = pzero(); ad[a][b] = pzero(); }
  hopping2(x, links, g, s, c, r, L, link12 != 0, au, ad, m1);
  const float2 kap = dup(kappa), nkap = dup(-kappa);
#pragma unroll 1
  for (int ch = 0; ch < 2; ++ch) {
    P2 vin[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int k = ch * 6 + i;
      vin[i] = ldq2(u + ((size_t)k * V + s) * L + r);
      pmac(vin[i], kap, nkap, ch == 0 ? au[i / 3][i % 3] : ad[i / 3][i % 3], m1);
    }
    const float* mm = clov_inv + (size_t)ch * CLOV_REALS * V + s;
#pragma unroll 1
    for (int i = 0; i < 6; ++i) stq2(at(y, V, L, s, ch * 6 + i, r), herm6_row2(mm, V, i, vin, m1), m1);
  }
}

// ------------------------------------------------------------------ packed variant, grid sums
// The same sweep with the link and clover products summed on a fixed grid instead of by two-sum.
// Error-free extraction on a grid (Rump, Ogita and Oishi, "Accurate floating-point summation",
// SIAM J. Sci. Comput. 31, 2008): if the partial sums of  sum_k a_k b_k  stay below 2^(E-1) in
// magnitude, an FP32 accumulator S started at sigma = 1.5 * 2^E stays in [2^E, 2^(E+1)), where the
// FP32 numbers are exactly the multiples of g = 2^(E-23).  Then S' = fma(a, b.hi, S) is S plus the
// product rounded to the grid, with no other rounding, and fma(a, b.hi, S - S') -- S - S' is exact
// -- is the part of the product below the grid, |.| <= g/2, rounded to 24 bits of itself.  That
// part and a b.lo go into a plain FP32 sum.  Per product: 5 FP32x2 operations instead of 11, at an
// error of ~2^-24 g per product instead of an exact high part (see DESIGN: the sum's error stays
// ~2^-44 of the bound, the order of the two-sum form's low-word rounding).
//   Bounds.  A hop sums three products of a link row (norm <= 1: op.links_unitary) with the
// projected half-spinor h, so each partial sum is below sqrt(3) m, m = max |h.hi| over the hop's
// twelve reals: E = e(m) + 3 (2^e(m) <= m < 2^(e(m)+1)) gives 2^(E-1) = 4 2^e(m) > 2m.  A clover
// row sums six products; its bound is the stored row sum (op.clov_bound32) times m =
// max |v.hi| over the block's input, enlarged by 2^-16 to cover the grid roundings.

WD_DEV float habs_max(const P2& z, float m) { return fmaxf(m, fmaxf(fabsf(z.hi.x), fabsf(z.hi.y))); }

// A link from the site-major copy ([site][mu][20 floats]: the 9 entries (re, im) row by row, then
// two zeros), rows 0 and 1 in three 16-byte loads and row 2 rebuilt (link12) or loaded.
WD_DEV void link_sm(const float4* __restrict__ U, bool link12, Cx<float> m[3][3]) {
  const float4 a = __ldg(U), b = __ldg(U + 1), c = __ldg(U + 2);
  m[0][0] = cmake<float>(a.x, a.y);
  m[0][1] = cmake<float>(a.z, a.w);
  m[0][2] = cmake<float>(b.x, b.y);
  m[1][0] = cmake<float>(b.z, b.w);
  m[1][1] = cmake<float>(c.x, c.y);
  m[1][2] = cmake<float>(c.z, c.w);
  if (link12) {
    m[2][0] = conj(cmul(m[0][1], m[1][2]) - cmul(m[0][2], m[1][1]));
    m[2][1] = conj(cmul(m[0][2], m[1][0]) - cmul(m[0][0], m[1][2]));
    m[2][2] = conj(cmul(m[0][0], m[1][1]) - cmul(m[0][1], m[1][0]));
  } else {
    const float4 d = __ldg(U + 3), e = __ldg(U + 4);
    m[2][0] = cmake<float>(d.x, d.y);
    m[2][1] = cmake<float>(d.z, d.w);
    m[2][2] = cmake<float>(e.x, e.y);
  }
}

// The hopping term H x at (s, r) as hopping2, the link products summed on the hop's grid.
WD_DEV void hopping3(const float4* __restrict__ x, const float4* __restrict__ links, const Geom& g,
                     int s, const int c[4], int r, int L, bool link12, P2 au[2][3], P2 ad[2][3],
                     float2 m1) {
  const size_t V = (size_t)g.V;
  const size_t cs = V * L;
  const float2 one = make_float2(1.f, 1.f);
#pragma unroll 1
  for (int d = 0; d < 8; ++d) {
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    const int cm = mu == 0 ? c[0] : mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
    const int ext = g.d[mu], str = g.stride[mu];
    const int sn = fwd ? (cm == ext - 1 ? s - (ext - 1) * str : s + str)
                       : (cm == 0 ? s + (ext - 1) * str : s - str);
    const SpinDir sd = spin_dir(d);
    const float2 dn0 = make_float2(sd.dn[0], sd.dn[1]), dn1 = make_float2(sd.dn[2], sd.dn[3]);
    const float2 up0 = make_float2(sd.up[0], sd.up[1]), up1 = make_float2(sd.up[2], sd.up[3]);
    const float4* base = x + (size_t)sn * L + r;
    const int k0 = sd.cross ? 9 : 6, k1 = sd.cross ? 6 : 9;
    P2 h0[3], h1[3];
    float hm = 0.f;
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      const P2 u0 = ldq2(base + (0 * 3 + col) * cs), u1 = ldq2(base + (1 * 3 + col) * cs);
      const P2 x0 = ldq2(base + (k0 + col) * cs), x1 = ldq2(base + (k1 + col) * cs);
      h0[col] = padd(u0, psel(sd.swap, pswap(x0), x0), dn0, m1);
      h1[col] = padd(u1, psel(sd.swap, pswap(x1), x1), dn1, m1);
      hm = habs_max(h0[col], habs_max(h1[col], hm));
    }
    const float2 sigma = grid_bias(hm, 3);
    const float2 nsigma = make_float2(-sigma.x, -sigma.y);
    Cx<float> m[3][3];
    link_sm(links + (size_t)((fwd ? s : sn) * 4 + mu) * 5, link12, m);
    if (!fwd) {   // W = m^H
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a + 1; b < 3; ++b) {
          const Cx<float> t = m[a][b];
          m[a][b] = conj(m[b][a]);
          m[b][a] = conj(t);
        }
#pragma unroll
      for (int a = 0; a < 3; ++a) m[a][a] = conj(m[a][a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 SX0, LX0, SY0, LY0, SX1, LX1, SY1, LY1;
      gmul(SX0, LX0, dup(m[a][0].re), h0[0], sigma, m1);
      gmul(SY0, LY0, dup(m[a][0].im), h0[0], sigma, m1);
      gmul(SX1, LX1, dup(m[a][0].re), h1[0], sigma, m1);
      gmul(SY1, LY1, dup(m[a][0].im), h1[0], sigma, m1);
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        const float2 rb = dup(m[a][b].re), ib = dup(m[a][b].im);
        gmac(SX0, LX0, rb, h0[b], m1);
        gmac(SY0, LY0, ib, h0[b], m1);
        gmac(SX1, LX1, rb, h1[b], m1);
        gmac(SY1, LY1, ib, h1[b], m1);
      }
      const P2 w0 = gcombine(SX0, LX0, SY0, LY0, nsigma);
      const P2 w1 = gcombine(SX1, LX1, SY1, LY1, nsigma);
      au[0][a] = padd(au[0][a], w0, one, m1);
      au[1][a] = padd(au[1][a], w1, one, m1);
      const P2 y0 = psel(sd.cross, w1, w0), y1 = psel(sd.cross, w0, w1);
      ad[0][a] = padd(ad[0][a], psel(sd.swap, pswap(y0), y0), up0, m1);
      ad[1][a] = padd(ad[1][a], psel(sd.swap, pswap(y1), y1), up1, m1);
    }
  }
}


// Row i of a packed Hermitian 6x6 block held in registers (cl: the 36 reals of the packed block,
// the diagonal first, then the strictly-lower pairs) times v, summed on the grid sigma; the same
// products in the same order as herm6_row3, the entries indexed at compile time.
template <int I>
WD_DEV P2 herm6_row3r(const float cl[CLOV_REALS], const P2 v[6], float2 sigma, float2 nsigma,
                      float2 m1) {
  float2 SX, LX, SY, LY;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float re, im;
    if (j == I) {
      re = cl[I];
      im = 0.f * cl[I];
    } else if (j < I) {
      re = cl[tri_index(I, j)];
      im = cl[tri_index(I, j) + 1];
    } else {
      re = cl[tri_index(j, I)];
      im = -cl[tri_index(j, I) + 1];
    }
    if (j == 0) {
      gmul(SX, LX, dup(re), v[0], sigma, m1);
      gmul(SY, LY, dup(im), v[0], sigma, m1);
    } else {
      gmac(SX, LX, dup(re), v[j], m1);
      gmac(SY, LY, dup(im), v[j], m1);
    }
  }
  return gcombine(SX, LX, SY, LY, nsigma);
}

// One chirality block of the site-major inverse copy ([site][chirality][36 floats]) into registers.
WD_DEV void clover_block(const float4* __restrict__ p, float cl[CLOV_REALS]) {
#pragma unroll
  for (int q = 0; q < CLOV_REALS / 4; ++q) {
    const float4 t = __ldg(p + q);
    cl[4 * q] = t.x;
    cl[4 * q + 1] = t.y;
    cl[4 * q + 2] = t.z;
    cl[4 * q + 3] = t.w;
  }
}

// The six rows of one chirality block, stored as they are formed.
template <typename TY>
WD_DEV void herm6_rows3r(const float cl[CLOV_REALS], const P2 vin[6], float2 sigma, float2 nsigma,
                         float2 m1, TY* y, size_t V, int L, int s, int ch, int r) {
  stq2(at(y, V, L, s, ch * 6 + 0, r), herm6_row3r<0>(cl, vin, sigma, nsigma, m1), m1);
  stq2(at(y, V, L, s, ch * 6 + 1, r), herm6_row3r<1>(cl, vin, sigma, nsigma, m1), m1);
  stq2(at(y, V, L, s, ch * 6 + 2, r), herm6_row3r<2>(cl, vin, sigma, nsigma, m1), m1);
  stq2(at(y, V, L, s, ch * 6 + 3, r), herm6_row3r<3>(cl, vin, sigma, nsigma, m1), m1);
  stq2(at(y, V, L, s, ch * 6 + 4, r), herm6_row3r<4>(cl, vin, sigma, nsigma, m1), m1);
  stq2(at(y, V, L, s, ch * 6 + 5, r), herm6_row3r<5>(cl, vin, sigma, nsigma, m1), m1);
}

template <typename TY>
__global__ void __launch_bounds__(128, 4)
sweep_df3_kernel(const float4* __restrict__ x, TY* __restrict__ y, const float4* __restrict__ u,
                 const float4* __restrict__ links, const float4* __restrict__ clov_inv,
                 const float* __restrict__ clov_bound, Geom g, int L, float kappa, int link12) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.V * L) return;
  const int s = tid / L;
  const int r = tid - s * L;
  const size_t V = (size_t)g.V;
  const float2 m1 = make_float2(-1.f, -1.f);
  int c[4];
  site_coords(g, s, c);
  P2 au[2][3], ad[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) { au[a][b] = pzero(); ad[a][b] = pzero(); }
  hopping3(x, links, g, s, c, r, L, link12 != 0, au, ad, m1);
  const float2 kap = dup(kappa), nkap = dup(-kappa);
#pragma unroll 1
  for (int ch = 0; ch < 2; ++ch) {
    P2 vin[6];
    float vm = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int k = ch * 6 + i;
      vin[i] = ldq2(u + ((size_t)k * V + s) * L + r);
      pmac(vin[i], kap, nkap, ch == 0 ? au[i / 3][i % 3] : ad[i / 3][i % 3], m1);
      vm = habs_max(vin[i], vm);
    }
    const float bnd = __ldg(clov_bound + (size_t)ch * V + s) * vm * (1.f + 0x1p-16f);
    const float2 sigma = grid_bias(bnd, 2);
    const float2 nsigma = make_float2(-sigma.x, -sigma.y);
    float cl[CLOV_REALS];
    clover_block(clov_inv + ((size_t)s * 2 + ch) * (CLOV_REALS / 4), cl);
    herm6_rows3r(cl, vin, sigma, nsigma, m1, y, V, L, s, ch, r);
  }
}

// First sweep from G = 0: stores the double-float copy of the FP64 right-hand side (when u_df is
// not null) and writes G = A_D^{-1} U, the clover rows in packed grid sums (as sweep_df3_kernel;
// with links that are not unitary the clover row bound still holds, so this needs no check).
template <typename TY>
__global__ void __launch_bounds__(128)
site_inverse_df_kernel(const double* __restrict__ u, float4* __restrict__ u_df, TY* __restrict__ y,
                       const float4* __restrict__ clov_inv, const float* __restrict__ clov_bound,
                       int V, int L) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= V * L) return;
  const int s = tid / L;
  const int r = tid - s * L;
  const float2 m1 = make_float2(-1.f, -1.f);
  const size_t base = (size_t)s * 12 * L + r;    // complex index of (s, component 0, r)
  const double2* u2 = reinterpret_cast<const double2*>(u);
#pragma unroll 1
  for (int ch = 0; ch < 2; ++ch) {
    P2 vin[6];
    float vm = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int k = ch * 6 + i;
      vin[i] = p2_split(__ldg(u2 + base + (size_t)k * L));
      if (u_df)
        *at(u_df, (size_t)V, L, s, k, r) =
            make_float4(vin[i].hi.x, vin[i].hi.y, vin[i].lo.x, vin[i].lo.y);
      vm = habs_max(vin[i], vm);
    }
    const float bnd = __ldg(clov_bound + (size_t)ch * V + s) * vm * (1.f + 0x1p-16f);
    const float2 sigma = grid_bias(bnd, 2);
    const float2 nsigma = make_float2(-sigma.x, -sigma.y);
    float cl[CLOV_REALS];
    clover_block(clov_inv + ((size_t)s * 2 + ch) * (CLOV_REALS / 4), cl);
    herm6_rows3r(cl, vin, sigma, nsigma, m1, y, (size_t)V, L, s, ch, r);
  }
}

}  // namespace

cudaError_t launch_site_inverse_df(const Op& op, const double* u, void* u_df, void* g_df,
                                   double* g64, int L, cudaStream_t st) {
  const unsigned grid = (unsigned)(((long long)op.g.V * L + 127) / 128);
  float4* ud = static_cast<float4*>(u_df);
  if (g_df)
    site_inverse_df_kernel<float4><<<grid, 128, 0, st>>>(u, ud, static_cast<float4*>(g_df),
                                                         op.clov_inv32s, op.clov_bound32, op.g.V, L);
  else
    site_inverse_df_kernel<double><<<grid, 128, 0, st>>>(u, ud, g64, op.clov_inv32s,
                                                         op.clov_bound32, op.g.V, L);
  return cudaGetLastError();
}

namespace {
template <int R>
cudaError_t launch_df_r(const Op& op, const float4* x, const float4* u, float4* g_df, double* g64,
                        int L, int block, cudaStream_t st) {
  const unsigned grid = (unsigned)(((long long)op.g.V * (L / R) + block - 1) / block);
  const float2* links = reinterpret_cast<const float2*>(op.links32);
  if (g_df)
    sweep_df_kernel<R, float4><<<grid, block, 0, st>>>(x, g_df, u, links, op.clov_inv32, op.g, L,
                                                       (float)op.kappa, op.link12);
  else
    sweep_df_kernel<R, double><<<grid, block, 0, st>>>(x, g64, u, links, op.clov_inv32, op.g, L,
                                                       (float)op.kappa, op.link12);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_jacobi_df(const Op& op, const void* g_in, const void* u_df, void* g_df,
                             double* g64, int L, int rhs_per_thread, int block, int packed,
                             cudaStream_t st) {
  if ((block != 64 && block != 128) || (rhs_per_thread != 1 && rhs_per_thread != 2) ||
      L % rhs_per_thread != 0 || (packed && rhs_per_thread != 1) || packed < 0 || packed > 2 ||
      (packed == 2 && !op.links_unitary))
    return cudaErrorInvalidValue;
  const float4* x = static_cast<const float4*>(g_in);
  const float4* u = static_cast<const float4*>(u_df);
  float4* gd = static_cast<float4*>(g_df);
  if (packed == 2) {
    const unsigned grid = (unsigned)(((long long)op.g.V * L + block - 1) / block);
    if (gd)
      sweep_df3_kernel<float4><<<grid, block, 0, st>>>(x, gd, u, op.links32s, op.clov_inv32s,
                                                       op.clov_bound32, op.g, L, (float)op.kappa,
                                                       op.link12);
    else
      sweep_df3_kernel<double><<<grid, block, 0, st>>>(x, g64, u, op.links32s, op.clov_inv32s,
                                                       op.clov_bound32, op.g, L, (float)op.kappa,
                                                       op.link12);
    return cudaGetLastError();
  }
  if (packed) {
    const unsigned grid = (unsigned)(((long long)op.g.V * L + block - 1) / block);
    const float2* links = reinterpret_cast<const float2*>(op.links32);
    if (gd)
      sweep_df2_kernel<float4><<<grid, block, 0, st>>>(x, gd, u, links, op.clov_inv32, op.g, L,
                                                       (float)op.kappa, op.link12);
    else
      sweep_df2_kernel<double><<<grid, block, 0, st>>>(x, g64, u, links, op.clov_inv32, op.g, L,
                                                       (float)op.kappa, op.link12);
    return cudaGetLastError();
  }
  return rhs_per_thread == 2 ? launch_df_r<2>(op, x, u, gd, g64, L, block, st)
                             : launch_df_r<1>(op, x, u, gd, g64, L, block, st);
}
