// Shared device helpers: complex arithmetic on (re, im) pairs, double-float arithmetic (scalar and
// packed FP32x2) with its conversions, lattice geometry, launch checks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define WD_DEV __device__ __forceinline__

// ------------------------------------------------------------------ complex numbers
template <typename T>
struct Cx {
  T re, im;
};

template <typename T> WD_DEV Cx<T> cmake(T r, T i) { return Cx<T>{r, i}; }
template <typename T> WD_DEV Cx<T> czero() { return Cx<T>{T(0), T(0)}; }
template <typename T> WD_DEV Cx<T> operator+(Cx<T> a, Cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> WD_DEV Cx<T> operator-(Cx<T> a, Cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> WD_DEV Cx<T> operator-(Cx<T> a) { return {-a.re, -a.im}; }
template <typename T> WD_DEV Cx<T> operator*(T s, Cx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> WD_DEV Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> WD_DEV Cx<T> conj(Cx<T> a) { return {a.re, -a.im}; }
// i*a and -i*a
template <typename T> WD_DEV Cx<T> ti(Cx<T> a) { return {-a.im, a.re}; }
template <typename T> WD_DEV Cx<T> tmi(Cx<T> a) { return {a.im, -a.re}; }
// acc + a*b
template <typename T> WD_DEV Cx<T> cfma(Cx<T> a, Cx<T> b, Cx<T> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a)*b
template <typename T> WD_DEV Cx<T> cfmaj(Cx<T> a, Cx<T> b, Cx<T> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
template <typename T> WD_DEV T cnorm2(Cx<T> a) { return a.re * a.re + a.im * a.im; }

// Vector loads/stores of one complex number (16 B for double, 8 B for float).
WD_DEV Cx<double> ldc(const double* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}
WD_DEV Cx<float> ldc(const float* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}
WD_DEV void stc(double* p, Cx<double> a) { *reinterpret_cast<double2*>(p) = make_double2(a.re, a.im); }
WD_DEV void stc(float* p, Cx<float> a) { *reinterpret_cast<float2*>(p) = make_float2(a.re, a.im); }

// ------------------------------------------------------------------ lattice geometry
// Periodic Lx*Ly*Lz*Lt lattice, site = x + Lx*(y + Ly*(z + Lz*t)).
struct Geom {
  int d[4];        // Lx, Ly, Lz, Lt
  int stride[4];   // 1, Lx, Lx*Ly, Lx*Ly*Lz
  int V;
};

WD_DEV void site_coords(const Geom& g, int s, int c[4]) {
  c[0] = s % g.d[0];
  int r = s / g.d[0];
  c[1] = r % g.d[1];
  r /= g.d[1];
  c[2] = r % g.d[2];
  c[3] = r / g.d[2];
}
// Site of x + mu (dir = +1) or x - mu (dir = -1).
WD_DEV int neighbour(const Geom& g, int s, const int c[4], int mu, int dir) {
  if (dir > 0)
    return (c[mu] == g.d[mu] - 1) ? s - (g.d[mu] - 1) * g.stride[mu] : s + g.stride[mu];
  return (c[mu] == 0) ? s + (g.d[mu] - 1) * g.stride[mu] : s - g.stride[mu];
}

static inline Geom make_geom(const int dims[4]) {
  Geom g;
  int st = 1;
  for (int m = 0; m < 4; ++m) {
    g.d[m] = dims[m];
    g.stride[m] = st;
    st *= dims[m];
  }
  g.V = st;
  return g;
}

// Packed Hermitian 6x6: 6 real diagonal entries, then the 15 strictly-lower entries (i > j) as
// (re, im) pairs at 6 + 2*(i*(i-1)/2 + j).  36 reals per block, two blocks (chirality +, -) a site.
constexpr int CLOV_REALS = 36;
__host__ __device__ constexpr int tri_index(int i, int j) { return 6 + 2 * (i * (i - 1) / 2 + j); }

// ------------------------------------------------------------------ double-float (FP32 pairs)
// A value hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits, computed on the FP32 pipes
// with the error-free transformations of Knuth (two-sum) and Dekker (two-product via FMA).
struct DF {
  float hi, lo;
};
WD_DEV DF df_from(double d) {
  const float hi = __double2float_rn(d);
  return {hi, __double2float_rn(d - (double)hi)};
}
WD_DEV double df_to(DF a) { return (double)a.hi + (double)a.lo; }
// The same two conversions built from the IEEE-754 bit fields on the integer and FP32 pipes.  On
// GB300 the FP64 pipe issues two lanes per clock per SM, and the FP64 <-> FP32 conversions above
// run on it; the bulk conversions of whole blocks use these instead.
//   df_split: hi = d truncated to 24 significant bits; lo = d - hi rounded to nearest FP32.  The
//   remainder (29 fraction bits r) enters as two exact differences 2^E (1 + f) - 2^E, one for the
//   top 23 bits of r and one for its low 6, and their FP32 sum rounds once, so
//   |d - (hi + lo)| <= 2^-48 |d| for |d| >= 2^-79.  Below that lo keeps fewer bits, below 2^-103
//   none, and below 2^-126 hi is 0.  Values beyond the FP32 range become +-inf; NaN stays NaN.
WD_DEV DF df_split(double d) {
  const unsigned int h = (unsigned int)__double2hiint(d), l = (unsigned int)__double2loint(d);
  const unsigned int s = h & 0x80000000u;
  const int e = (int)((h >> 20) & 0x7FFu);                    // biased FP64 exponent
  const unsigned int m = __funnelshift_l(l, h, 3) & 0x7FFFFFu;  // top 23 fraction bits
  const unsigned int r = l & 0x1FFFFFFFu;                      // the other 29
  unsigned int hb = s | ((unsigned int)(e - 896) << 23) | m;
  const unsigned int b1 = s | ((unsigned int)(e - 919) << 23);   // 2^(e-1046): r >> 6 in units of 2^(e-1069)
  const unsigned int b2 = s | ((unsigned int)(e - 942) << 23);   // 2^(e-1069): r & 63 in units of 2^(e-1075)
  const float t1 = __fsub_rn(__uint_as_float(b1 | (r >> 6)), __uint_as_float(b1));
  const float t2 = __fsub_rn(__uint_as_float(b2 | ((r & 63u) << 17)), __uint_as_float(b2));
  float lo = __fadd_rn(t1, t2);
  if (e < 943) lo = e < 920 ? 0.f : t1;
  if (e < 897) hb = s;
  if (e > 1150) {
    hb = (e == 2047 && ((h & 0xFFFFFu) | l)) ? 0x7FC00000u : (s | 0x7F800000u);
    lo = 0.f;
  }
  return {__uint_as_float(hb), lo};
}
//   f_widen: the FP64 value of an FP32 number, exact for normal numbers, 0 for FP32 subnormals.
WD_DEV double f_widen(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int e = (b >> 23) & 0xFFu;
  unsigned int hw = (b & 0x80000000u) | ((e == 255u ? 2047u : e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
  unsigned int lw = b << 29;
  if (e == 0u) {
    hw = b & 0x80000000u;
    lw = 0u;
  }
  return __hiloint2double((int)hw, (int)lw);
}
WD_DEV double df_join(DF a) { return f_widen(a.hi) + f_widen(a.lo); }
// s + e = a + b exactly.  The __f*_rn intrinsics are never contracted into FMAs, which would
// break the exactness the transformation relies on.
WD_DEV void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// acc += a * b, accumulator left unnormalised (hi carries the sum, lo gathers the errors)
WD_DEV void df_mac(DF& acc, DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);      // the rounding error of p, exactly
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}
WD_DEV void df_msub(DF& acc, DF a, DF b) {   // acc -= a * b
  df_mac(acc, {-a.hi, -a.lo}, b);
}
WD_DEV DF df_norm(DF a) {
  const float s = __fadd_rn(a.hi, a.lo);
  return {s, __fsub_rn(a.lo, __fsub_rn(s, a.hi))};
}
struct CDF {
  DF re, im;
};
WD_DEV CDF cdf_from(Cx<double> z) { return {df_from(z.re), df_from(z.im)}; }
WD_DEV Cx<double> cdf_to(CDF z) { return {df_to(z.re), df_to(z.im)}; }
WD_DEV CDF cdf_split(Cx<double> z) { return {df_split(z.re), df_split(z.im)}; }
WD_DEV Cx<double> cdf_join(CDF z) { return {df_join(z.re), df_join(z.im)}; }
WD_DEV CDF cdf_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
// acc += a * b (complex)
WD_DEV void cdf_mac(CDF& acc, CDF a, CDF b) {
  df_mac(acc.re, a.re, b.re);
  df_msub(acc.re, a.im, b.im);
  df_mac(acc.im, a.re, b.im);
  df_mac(acc.im, a.im, b.re);
}
// acc += conj(a) * b
WD_DEV void cdf_macj(CDF& acc, CDF a, CDF b) {
  df_mac(acc.re, a.re, b.re);
  df_mac(acc.re, a.im, b.im);
  df_mac(acc.im, a.re, b.im);
  df_msub(acc.im, a.im, b.re);
}

// ------------------------------------------------------------------ packed double-float
// The real and imaginary halves of a double-float complex value in the two lanes of FP32x2
// instructions (FFMA2/FADD2/FMUL2, each lane an IEEE round-to-nearest operation), so that one
// instruction does the work of two: hi = (re.hi, im.hi), lo = (re.lo, im.lo).  Subtractions are FMAs with
// m1 = (-1, -1) (negation is exact).  A complex product sum  sum_k a_k b_k  is accumulated as
// X = sum a_k.re (b_k.re, b_k.im) and Y = sum a_k.im (b_k.re, b_k.im), the scalar factor in both
// lanes, and combined once.
struct P2 {
  float2 hi, lo;
};
WD_DEV float2 dup(float a) { return make_float2(a, a); }
WD_DEV P2 pzero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
WD_DEV P2 pswap(P2 z) { return {make_float2(z.hi.y, z.hi.x), make_float2(z.lo.y, z.lo.x)}; }

// s + e = a + sg b exactly in each lane (sg = +1 or -1 per lane); two-sum with the sign folded in.
WD_DEV void two_sum2(float2 a, float2 b, float2 sg, float2 m1, float2& s, float2& e) {
  s = __ffma2_rn(sg, b, a);
  const float2 nbb = __ffma2_rn(s, m1, a);   // a - s: minus the part of sg b that reached s
  const float2 t1 = __fadd2_rn(s, nbb);      // s - bb
  const float2 t2 = __ffma2_rn(t1, m1, a);   // a - (s - bb)
  const float2 t3 = __ffma2_rn(sg, b, nbb);  // sg b - bb
  e = __fadd2_rn(t2, t3);
}
WD_DEV P2 padd(P2 a, P2 b, float2 sg, float2 m1) {   // a + sg b
  float2 s, e;
  two_sum2(a.hi, b.hi, sg, m1, s, e);
  return {s, __fadd2_rn(__ffma2_rn(sg, b.lo, a.lo), e)};
}
// (re, im) = X + (-Y.im, Y.re): sum a_k b_k from its two accumulators.
WD_DEV P2 pcombine(P2 X, P2 Y, float2 m1) { return padd(X, pswap(Y), make_float2(-1.f, 1.f), m1); }
// (re, im) = X + (Y.im, -Y.re): sum conj(a_k) b_k from its two accumulators.
WD_DEV P2 pcombine_conj(P2 X, P2 Y, float2 m1) {
  return padd(X, pswap(Y), make_float2(1.f, -1.f), m1);
}
// hi + lo renormalised so that |lo| <= ulp(hi)/2, in both lanes.
WD_DEV P2 pnorm(P2 z, float2 m1) {
  const float2 s = __fadd2_rn(z.hi, z.lo);
  return {s, __ffma2_rn(__ffma2_rn(z.hi, m1, s), m1, z.lo)};   // lo - (s - hi)
}
// acc + a b for a double-float factor a = ahi + alo given per lane (nahi = -ahi), b packed.
WD_DEV void pmac_dd(P2& acc, float2 ahi, float2 nahi, float2 alo, P2 b, float2 m1) {
  const float2 np = __fmul2_rn(nahi, b.hi);   // -(ahi b.hi), rounded
  float2 e = __ffma2_rn(ahi, b.hi, np);       // its rounding error, exactly
  e = __ffma2_rn(ahi, b.lo, e);
  e = __ffma2_rn(alo, b.hi, e);
  float2 s, t;
  two_sum2(acc.hi, np, m1, m1, s, t);         // acc.hi - np
  acc.hi = s;
  acc.lo = __fadd2_rn(acc.lo, __fadd2_rn(t, e));
}
// FP64 (re, im) <-> packed double-float through the bit-field conversions.
WD_DEV P2 p2_split(double2 v) {
  const DF r = df_split(v.x), i = df_split(v.y);
  return {make_float2(r.hi, i.hi), make_float2(r.lo, i.lo)};
}
WD_DEV double2 p2_join(P2 z) {   // one FP64 rounding of hi + lo per lane
  return make_double2(f_widen(z.hi.x) + f_widen(z.lo.x), f_widen(z.hi.y) + f_widen(z.lo.y));
}

// ------------------------------------------------------------------ grid sums (packed)
// Error-free extraction on a fixed grid (Rump, Ogita and Oishi, "Accurate floating-point
// summation", SIAM J. Sci. Comput. 31, 2008): if every partial sum of  sum_k a_k b_k  stays below
// 2^(E-1) in magnitude, an FP32 accumulator S started at sigma = 1.5 * 2^E stays in [2^E, 2^(E+1)),
// where the FP32 numbers are exactly the multiples of g = 2^(E-23).  S' = fma(a, b.hi, S) is then S
// plus the product rounded to the grid, with no other rounding, and fma(a, b.hi, S - S') (S - S'
// is exact) is the part of the product below the grid, |.| <= g/2, rounded to 24 bits of itself.
// That part and the products with the low words go into a plain FP32 sum Lo.  Callers choose E
// from a bound on the partial sums.  Lo grows to a few g over a sum and rounds at 2^-24 of its size,
// so the sum's error is ~2^-43 of the bound for a handful of terms (the sweep's three- and six-term
// sums), and grows with the number of terms.
// dup(1.5 * 2^(e + k)) for 2^e <= m < 2^(e+1) (m >= 0; m = 0 gives 1.5 * 2^(k - 127)).
WD_DEV float2 grid_bias(float m, int k) {
  const unsigned eb = __float_as_uint(m) & 0x7F800000u;
  return dup(__uint_as_float((eb + ((unsigned)k << 23)) | 0x00400000u));
}
// (S, Lo) for the first product a b of a grid sum started at sigma.
WD_DEV void gmul(float2& S, float2& Lo, float2 a, const P2& b, float2 sigma, float2 m1) {
  S = __ffma2_rn(a, b.hi, sigma);
  const float2 d = __ffma2_rn(S, m1, sigma);   // sigma - S, exact
  Lo = __ffma2_rn(a, b.lo, __ffma2_rn(a, b.hi, d));
}
// (S, Lo) + a b.
WD_DEV void gmac(float2& S, float2& Lo, float2 a, const P2& b, float2 m1) {
  const float2 s = __ffma2_rn(a, b.hi, S);
  const float2 d = __ffma2_rn(s, m1, S);       // S - s, exact
  Lo = __ffma2_rn(a, b.lo, Lo);
  Lo = __fadd2_rn(Lo, __ffma2_rn(a, b.hi, d));
  S = s;
}
WD_DEV float2 fswap(float2 v) { return make_float2(v.y, v.x); }
// (re, im) = X + (-Y.im, Y.re) for grid sums X = (SX, LX), Y = (SY, LY) started at sigma: the high
// parts SX - sigma, SY - sigma and their combination are exact (multiples of g below 2^E).
WD_DEV P2 gcombine(float2 SX, float2 LX, float2 SY, float2 LY, float2 nsigma) {
  const float2 cs = make_float2(-1.f, 1.f);
  const float2 xh = __fadd2_rn(SX, nsigma), yh = __fadd2_rn(SY, nsigma);
  return {__ffma2_rn(cs, fswap(yh), xh), __ffma2_rn(cs, fswap(LY), LX)};
}
