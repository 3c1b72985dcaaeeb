// The FP64 stencil Y = A X, R = B - A X and the FP64 Jacobi sweep with the hopping term computed
// on the FP32 pipes, exactly up to a final rounding (arXiv:0907.3261, Eq. (1); the paper's method
// is FP64 throughout, Sec. 3.1).
//
// On GB300 the FP64 pipe issues two lanes per clock per SM, and the FP64 stencil is bound by it
// (the 576 multiply-adds of the link products, the 192 reconstruction adds and the clover block
// per site and right-hand side).  Here the link products and their sums run on the FP32 lanes
// instead, in packed FP32x2 instructions with (re, im) in the two lanes:
//   * every operand is cut into three FP32 numbers whose sum is the FP64 value exactly -- the
//     links once at creation, each projected half-spinor h when it is formed (x3_split);
//   * the sums of products are accumulated on fixed grids (Rump, Ogita and Oishi, "Accurate
//     floating-point summation", SIAM J. Sci. Comput. 31, 2008) in three levels: S1 on the grid
//     2^-15 around 1.5 * 2^8, S2 on the grid 2^-32 around 1.5 * 2^-9, and a plain FP32 sum S3.
//     The leading product a1 b1 is split exactly (Dekker's two-product via FMA) and both parts
//     are extracted into S1 and S2 with Fast2Sum; a1 b2 and a2 b1 are extracted into S2 by FMA;
//     the three terms of weight ~2^-48 go into S3; terms below ~2^-69 are dropped.  Everything
//     that reaches S1 and S2 is exact, so the only roundings are those of S3 (~2^-52 of the bound
//     in total) and the final one to FP64;
//   * the operands are scaled by 2^-k, 2^k above the largest entry of the eight neighbouring
//     spinors (read from a pre-pass that records every (site, rhs)'s largest exponent), which
//     bounds every partial sum by 2^7 for unitary links (|h| < 4, sum_b |U_ab|^2 = 1, 8 hops) and
//     makes the grids fixed constants.
// The projection h = psi_up -/+ G psi_down, the site term (two Hermitian 6x6 blocks) and the final
// combination y = A_D x - kappa H x stay in FP64.  The result carries FP64 accuracy: the hopping
// sum is exact to ~2^-52 of its bound before its one FP64 rounding, where the FP64 stencil rounds
// after every operation.  Requires links whose rows have norm <= 1 + LINK12_TOL.
#include "common.cuh"
#include "internal.h"
#include "spin.cuh"

namespace {

enum { MODE_APPLY = 0, MODE_RESID = 1, MODE_JACOBI = 2 };

constexpr float XS1 = 384.f;            // 1.5 * 2^8: S1's grid, step 2^-15, partial sums < 2^7
constexpr float XS2 = 0.0029296875f;    // 1.5 * 2^-9: S2's grid, step 2^-32, partial sums < 2^-10

// v 2^-k as f1 + f2 + f3 exactly: f1 = the top 24 significant bits (truncated), f2 the next 23,
// f3 the last 6, the lower two built as exact differences 2^E (1 + f) - 2^E from the IEEE-754 bit
// fields (integer and FP32 pipes only).  Parts below the FP32 normal range are dropped (|v 2^-k|
// below 2^-80 loses f3, below 2^-103 f2, below 2^-126 everything); zero and FP64 subnormals give 0.
WD_DEV void x3_split(double v, int k, float& f1, float& f2, float& f3) {
  const unsigned int h = (unsigned int)__double2hiint(v), l = (unsigned int)__double2loint(v);
  const unsigned int s = h & 0x80000000u;
  const int eraw = (int)((h >> 20) & 0x7FFu);
  const int e = eraw - k;
  const unsigned int m = __funnelshift_l(l, h, 3) & 0x7FFFFFu;   // fraction bits 51..29
  const unsigned int r = l & 0x1FFFFFFFu;                         // fraction bits 28..0
  const unsigned int b1 = s | ((unsigned int)(e - 919) << 23);    // 2^(e-1046)
  const unsigned int b2 = s | ((unsigned int)(e - 942) << 23);    // 2^(e-1069)
  float t1 = __fsub_rn(__uint_as_float(b1 | (r >> 6)), __uint_as_float(b1));
  float t2 = __fsub_rn(__uint_as_float(b2 | ((r & 63u) << 17)), __uint_as_float(b2));
  unsigned int hb = s | ((unsigned int)(e - 896) << 23) | m;
  if (e < 943) t2 = 0.f;
  if (e < 920) t1 = 0.f;
  if (e < 897 || eraw == 0) { hb = s; t1 = 0.f; t2 = 0.f; }
  f1 = __uint_as_float(hb);
  f2 = t1;
  f3 = t2;
}

// A three-level grid sum per lane: value = (s1 - XS1) + (s2 - XS2) + s3.
struct X3 {
  float2 s1, s2, s3;
};
WD_DEV X3 x3_zero() { return {dup(XS1), dup(XS2), dup(0.f)}; }

// acc += a b for a = a1 + a2 + a3 (the same real factor in both lanes) and b = b1 + b2 + b3
// (packed; nb1 = -b1).  24 packed operations.
WD_DEV void x3_mac(X3& acc, float2 a1, float2 a2, float2 a3, float2 b1, float2 nb1, float2 b2,
                   float2 b3, float2 m1) {
  const float2 np = __fmul2_rn(a1, nb1);            // -p, p = RN(a1 b1)
  const float2 e = __ffma2_rn(a1, b1, np);          // a1 b1 - p, exact
  const float2 t = __ffma2_rn(np, m1, acc.s1);      // s1 + p on the grid
  const float2 nq = __fadd2_rn(np, __ffma2_rn(acc.s1, m1, t));   // -(p - (t - s1)), exact
  acc.s1 = t;
  const float2 u = __ffma2_rn(nq, m1, acc.s2);      // s2 + q
  const float2 nq2 = __fadd2_rn(nq, __ffma2_rn(acc.s2, m1, u));  // -(q - (u - s2)), exact
  const float2 u2 = __fadd2_rn(u, e);               // + e
  const float2 re = __ffma2_rn(__ffma2_rn(u, m1, u2), m1, e);    // e - (u2 - u), exact
  const float2 u3 = __ffma2_rn(a1, b2, u2);         // + a1 b2
  const float2 r3 = __ffma2_rn(a1, b2, __ffma2_rn(u3, m1, u2));  // a1 b2 - (u3 - u2)
  const float2 u4 = __ffma2_rn(a2, b1, u3);         // + a2 b1
  const float2 r4 = __ffma2_rn(a2, b1, __ffma2_rn(u4, m1, u3));  // a2 b1 - (u4 - u3)
  acc.s2 = u4;
  float2 lo = __ffma2_rn(nq2, m1, re);              // q2 + e's remainder
  lo = __fadd2_rn(lo, __fadd2_rn(r3, r4));
  lo = __ffma2_rn(a1, b3, lo);
  lo = __ffma2_rn(a2, b2, lo);
  lo = __ffma2_rn(a3, b1, lo);
  acc.s3 = __fadd2_rn(acc.s3, lo);
}

// T += phase * w levelwise (w offset-free; T's grid levels stay exact).
template <int PH>
WD_DEV void x3_add(X3& T, const X3& w) {
  if constexpr (PH == 0) {
    T.s1 = __fadd2_rn(T.s1, w.s1);
    T.s2 = __fadd2_rn(T.s2, w.s2);
    T.s3 = __fadd2_rn(T.s3, w.s3);
  } else if constexpr (PH == 2) {
    const float2 m1 = dup(-1.f);
    T.s1 = __ffma2_rn(m1, w.s1, T.s1);
    T.s2 = __ffma2_rn(m1, w.s2, T.s2);
    T.s3 = __ffma2_rn(m1, w.s3, T.s3);
  } else {
    // +i (re, im) = (-im, re); -i (re, im) = (im, -re)
    const float2 cs = PH == 1 ? make_float2(-1.f, 1.f) : make_float2(1.f, -1.f);
    T.s1 = __ffma2_rn(cs, fswap(w.s1), T.s1);
    T.s2 = __ffma2_rn(cs, fswap(w.s2), T.s2);
    T.s3 = __ffma2_rn(cs, fswap(w.s3), T.s3);
  }
}

// The sums of the hopping term live in shared memory, one slot per thread and value:
// [level][12][threads] float2, value index ch * 6 + sp * 3 + a (chirality ch: upper spins 0, 1
// or lower spins 2, 3; spin sp within it; colour a).  Each thread touches only its own slots.
struct SumRef {
  float2* base;   // smem + threadIdx.x
  int stride;     // threads per CTA
};
template <int PH>
WD_DEV void x3_add_sm(SumRef t, int idx, const X3& w) {
  float2* p1 = t.base + (size_t)idx * t.stride;
  float2* p2 = p1 + (size_t)12 * t.stride;
  float2* p3 = p2 + (size_t)12 * t.stride;
  X3 T = {*p1, *p2, *p3};
  x3_add<PH>(T, w);
  *p1 = T.s1;
  *p2 = T.s2;
  *p3 = T.s3;
}

// w = W h for one upper spin SP of the hopping term of Eq. (1) in direction (mu, dir), with
// h = psi_up,SP -/+ (G_mu psi_down)_SP and W = U_mu(x) (dir = +1) or U_mu(x - mu)^H (dir = -1),
// added to the upper spin SP and, through G_mu^H, to one lower spin.  The spin tables of
// gamma_down / gamma_up (spin.cuh) enter at run time, so that one loop body serves all eight
// hops: (G_mu d)_SP = phase * d_pi and G_mu^H sends w_SP to lower spin t with another phase
// (phases 0 = +1, 1 = +i, 2 = -1, 3 = -i).  SP is a run-time value as well (the caller loops over
// the two upper spins): one spin's body is half the code, which keeps the hop loop out of
// instruction-fetch stalls and spills.  xp points at the neighbour's spinor, U at the link's
// three-level copy ([level][entry], each entry (re, re, im, im)).
WD_DEV void hop_x3_spin(int SP, const double* __restrict__ xp, const float4* __restrict__ U, int L,
                        int k, int mu, int dir, SumRef sums, float2 m1) {
  const int pi = mu <= 1 ? 1 - SP : SP;
  // 2-bit tables over mu = 0..3: gamma_down's phase (SP 0: 3, 2, 3, 0; SP 1: 3, 0, 1, 0) and
  // gamma_up's (SP 0: 1, 2, 1, 0; SP 1: 1, 0, 3, 0); gamma_up's target spin equals pi
  const int phd = ((SP == 0 ? 0x3B : 0x13) >> (2 * mu)) & 3;
  const int t = pi;
  const int phu = ((((SP == 0 ? 0x19 : 0x31) >> (2 * mu)) & 3) + (dir > 0 ? 2 : 0)) & 3;
  // (G_mu d)_SP: (a, b) = the lanes of d after the phase's swap, with signs sa, sb; h = up -dir G d
  const bool swd = phd & 1;
  const bool na = (phd == 1 || phd == 2) != (dir > 0), nb = (phd >= 2) != (dir > 0);
  const double sa = na ? -1.0 : 1.0, sb = nb ? -1.0 : 1.0;
  float2 b1[3], nb1[3], b2[3], b3[3];
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    const Cx<double> up = ldc(xp + 2 * (size_t)((SP * 3 + col) * L));
    const Cx<double> dn = ldc(xp + 2 * (size_t)(((pi + 2) * 3 + col) * L));
    const double hre = fma(sa, swd ? dn.im : dn.re, up.re);
    const double him = fma(sb, swd ? dn.re : dn.im, up.im);
    float r1, r2, r3, i1, i2, i3;
    x3_split(hre, k, r1, r2, r3);
    x3_split(him, k, i1, i2, i3);
    b1[col] = make_float2(r1, i1);
    nb1[col] = make_float2(-r1, -i1);
    b2[col] = make_float2(r2, i2);
    b3[col] = make_float2(r3, i3);
  }
  // w = X + i Y (W = U) or X - i Y (W = U^H): lanes (re, im) = X + cs (Y.im, Y.re)
  const float2 cs = dir > 0 ? make_float2(-1.f, 1.f) : make_float2(1.f, -1.f);
  // the lower spin takes phu * w: lanes swapped for +-i, signs csu
  const bool swu = phu & 1;
  const float2 csu = make_float2((phu == 1 || phu == 2) ? -1.f : 1.f, phu >= 2 ? -1.f : 1.f);
  const float2 ns1 = dup(-XS1), ns2 = dup(-XS2);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    X3 X = x3_zero(), Y = x3_zero();   // sum_b Re W_ab h_b and sum_b Im W_ab h_b
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int e = dir > 0 ? a * 3 + b : b * 3 + a;
      const float4 l1 = __ldg(U + e), l2 = __ldg(U + 9 + e), l3 = __ldg(U + 18 + e);
      x3_mac(X, make_float2(l1.x, l1.y), make_float2(l2.x, l2.y), make_float2(l3.x, l3.y), b1[b],
             nb1[b], b2[b], b3[b], m1);
      x3_mac(Y, make_float2(l1.z, l1.w), make_float2(l2.z, l2.w), make_float2(l3.z, l3.w), b1[b],
             nb1[b], b2[b], b3[b], m1);
    }
    X3 w;   // offset-free; exact on both grids
    w.s1 = __ffma2_rn(cs, fswap(__fadd2_rn(Y.s1, ns1)), __fadd2_rn(X.s1, ns1));
    w.s2 = __ffma2_rn(cs, fswap(__fadd2_rn(Y.s2, ns2)), __fadd2_rn(X.s2, ns2));
    w.s3 = __ffma2_rn(cs, fswap(Y.s3), X.s3);
    x3_add_sm<0>(sums, SP * 3 + a, w);
    X3 wl;
    wl.s1 = swu ? fswap(w.s1) : w.s1;
    wl.s2 = swu ? fswap(w.s2) : w.s2;
    wl.s3 = swu ? fswap(w.s3) : w.s3;
    float2* p1 = sums.base + (size_t)(6 + t * 3 + a) * sums.stride;
    float2* p2 = p1 + (size_t)12 * sums.stride;
    float2* p3 = p2 + (size_t)12 * sums.stride;
    *p1 = __ffma2_rn(csu, wl.s1, *p1);
    *p2 = __ffma2_rn(csu, wl.s2, *p2);
    *p3 = __ffma2_rn(csu, wl.s3, *p3);
  }
}

template <int MODE>
__global__ void __launch_bounds__(128, 4)
dslash_x3_kernel(const double* __restrict__ x, double* __restrict__ y,
                 const double* __restrict__ u, const float4* __restrict__ lx,
                 const int* __restrict__ xexp, const double* __restrict__ clov, Geom g, int L,
                 double kappa) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.V * L) return;
  const int s = tid / L;
  const int r = tid - s * L;
  int c[4];
  site_coords(g, s, c);
  // the scale 2^k: every entry of the eight neighbouring spinors is below 2^(k+1)
  int emax = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    emax = max(emax, __ldg(xexp + (size_t)neighbour(g, s, c, mu, +1) * L + r));
    emax = max(emax, __ldg(xexp + (size_t)neighbour(g, s, c, mu, -1) * L + r));
  }
  const bool finite = emax < 2047;
  const int k = max(emax, 24) - 1023;
  const float2 m1 = dup(-1.f);
  extern __shared__ float2 x3_smem[];
  const SumRef sums{x3_smem + threadIdx.x, (int)blockDim.x};
  {
    const X3 z = x3_zero();
#pragma unroll
    for (int v = 0; v < 12; ++v) {
      float2* p = sums.base + (size_t)v * sums.stride;
      p[0] = z.s1;
      p[(size_t)12 * sums.stride] = z.s2;
      p[(size_t)24 * sums.stride] = z.s3;
    }
  }
#pragma unroll 1
  for (int hop = 0; hop < 8; ++hop) {
    const int mu = hop >> 1;
    const int dir = (hop & 1) ? -1 : 1;
    const int cm = mu == 0 ? c[0] : mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
    const int dm = g.d[0] * (mu == 0) + g.d[1] * (mu == 1) + g.d[2] * (mu == 2) + g.d[3] * (mu == 3);
    const int st = mu == 0 ? 1 : mu == 1 ? g.stride[1] : mu == 2 ? g.stride[2] : g.stride[3];
    const int sn = dir > 0 ? (cm == dm - 1 ? s - (dm - 1) * st : s + st)
                           : (cm == 0 ? s + (dm - 1) * st : s - st);
    const double* xp = x + 2 * ((size_t)sn * 12 * L + r);
    const float4* U = lx + (size_t)((dir > 0 ? s : sn) * 4 + mu) * 27;
#pragma unroll 1
    for (int sp = 0; sp < 2; ++sp) hop_x3_spin(sp, xp, U, L, k, mu, dir, sums, m1);
  }

  // H x = 2^k ((S1 - XS1) + (S2 - XS2) + S3): the first two levels join exactly in FP64, S3 and
  // the scale enter through kappa 2^k (a power-of-two product, exact).  One chirality at a time:
  const double kk = finite ? kappa * __hiloint2double((k + 1023) << 20, 0)
                           : __longlong_as_double(0x7FF8000000000000LL);
  const size_t base = 2 * ((size_t)s * 12 * L + r);
  const double* src = MODE == MODE_JACOBI ? u : x;
#pragma unroll
  for (int ch = 0; ch < 2; ++ch) {
    Cx<double> hs[6], vin[6], out[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float2* p = sums.base + (size_t)(ch * 6 + i) * sums.stride;
      const X3 A = {p[0], p[(size_t)12 * sums.stride], p[(size_t)24 * sums.stride]};
      hs[i] = cmake<double>(
          f_widen(__fsub_rn(A.s1.x, XS1)) + f_widen(__fsub_rn(A.s2.x, XS2)) + f_widen(A.s3.x),
          f_widen(__fsub_rn(A.s1.y, XS1)) + f_widen(__fsub_rn(A.s2.y, XS2)) + f_widen(A.s3.y));
      const Cx<double> v = ldc(src + base + 2 * (size_t)((ch * 6 + i) * L));
      if constexpr (MODE == MODE_JACOBI)
        vin[i] = cmake<double>(fma(kk, hs[i].re, v.re), fma(kk, hs[i].im, v.im));
      else
        vin[i] = v;
    }
    herm6s(clov + (size_t)s * 2 * CLOV_REALS + ch * CLOV_REALS, 1, vin, out);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      Cx<double> v = out[i];
      if constexpr (MODE != MODE_JACOBI) {
        v = cmake<double>(fma(-kk, hs[i].re, v.re), fma(-kk, hs[i].im, v.im));
        if constexpr (MODE == MODE_RESID) v = ldc(u + base + 2 * (size_t)((ch * 6 + i) * L)) - v;
      }
      stc(y + base + 2 * (size_t)((ch * 6 + i) * L), v);
    }
  }
}

// The largest biased FP64 exponent among the 24 reals of every (site, rhs) of x.
__global__ void __launch_bounds__(256)
max_exponent_kernel(const double* __restrict__ x, int* __restrict__ xexp, int V, int L) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= V * L) return;
  const int s = tid / L;
  const int r = tid - s * L;
  const double* p = x + 2 * ((size_t)s * 12 * L + r);
  int e = 0;
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p + 2 * (size_t)i * L));
    e = max(e, (__double2hiint(v.x) >> 20) & 0x7FF);
    e = max(e, (__double2hiint(v.y) >> 20) & 0x7FF);
  }
  xexp[tid] = e;
}

// The three-level copy of the links: [site][mu][level][entry] as (re, re, im, im).
__global__ void link_split_kernel(const double* __restrict__ links, float4* __restrict__ lx, int V) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= V * 36) return;
  const int sm = tid / 9;          // site * 4 + mu
  const int e = tid - sm * 9;
  const double re = links[(size_t)sm * 18 + 2 * e], im = links[(size_t)sm * 18 + 2 * e + 1];
  float r[3], i[3];
  x3_split(re, 0, r[0], r[1], r[2]);
  x3_split(im, 0, i[0], i[1], i[2]);
#pragma unroll
  for (int lv = 0; lv < 3; ++lv)
    lx[(size_t)sm * 27 + lv * 9 + e] = make_float4(r[lv], r[lv], i[lv], i[lv]);
}

constexpr int X3_THREADS = 128;
inline unsigned x3_grid(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <int MODE>
cudaError_t launch_x3(const Op& op, const double* x, const double* u, double* y, const double* clov,
                      int L, cudaStream_t st) {
  const long long n = (long long)op.g.V * L;
  max_exponent_kernel<<<x3_grid(n, 256), 256, 0, st>>>(x, op.xexp, op.g.V, L);
  dslash_x3_kernel<MODE><<<x3_grid(n, X3_THREADS), X3_THREADS, X3_THREADS * 36 * sizeof(float2), st>>>(
      x, y, u, op.links_x3, op.xexp, clov, op.g, L, op.kappa);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_link_split(const Op& op, cudaStream_t st) {
  const long long n = (long long)op.g.V * 36;
  link_split_kernel<<<x3_grid(n, 256), 256, 0, st>>>(op.links, op.links_x3, op.g.V);
  return cudaGetLastError();
}

cudaError_t launch_apply_x3(const Op& op, const double* x, double* y, int L, cudaStream_t st) {
  return launch_x3<MODE_APPLY>(op, x, nullptr, y, op.clov, L, st);
}

cudaError_t launch_resid_x3(const Op& op, const double* x, const double* b, double* y, int L,
                            cudaStream_t st) {
  return launch_x3<MODE_RESID>(op, x, b, y, op.clov, L, st);
}

cudaError_t launch_jacobi_x3(const Op& op, const double* g_in, const double* u, double* g_out,
                             int L, cudaStream_t st) {
  return launch_x3<MODE_JACOBI>(op, g_in, u, g_out, op.clov_inv, L, st);
}
