// Low-precision Jacobi sweeps of the preconditioner M (arXiv:0907.3261, Sec. 2: G^0 = 0,
// G^{i+1} = A_D^{-1}(U + kappa H G^i) for i < j), computed in FP32 on blocks stored in FP32 or BF16.
//
// The preconditioner's private blocks are component-major, [spin*3+colour][site][rhs], one complex
// number per element: float2, or two BF16 halves packed in a 32-bit word (re in the low half).
// The threads of a warp take consecutive (site, rhs) pairs, so every component of every neighbour
// spinor is one contiguous run per warp instruction.  The FP32 links ([mu][3x3 entry][site]) and
// A_D^{-1} blocks ([chirality][36][site]) are component-major too.  When the links are special
// unitary (Op::link12), a sweep reads only the first two rows of each link (12 reals) and rebuilds
// the third as the complex conjugate of their cross product.  Each thread owns R consecutive
// right-hand sides (R = 1 or 2 dividing L), and the links and clover entries it loads serve all R.
// The first sweep (from G = 0) is site-local and also stores the low-precision copy of U; the last
// sweep writes FP64 in the caller's site-major layout.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "elem.cuh"
#include "spin.cuh"

namespace lp {

// R consecutive elements in one vector access.
template <int R>
WD_DEV void ldr(const float2* __restrict__ p, Cx<float> v[R]) {
  if constexpr (R == 1) {
    v[0] = ld1(p);
  } else {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = {a.x, a.y};
    v[1] = {a.z, a.w};
  }
}
template <int R>
WD_DEV void ldr(const bf16x2* __restrict__ p, Cx<float> v[R]) {
  if constexpr (R == 1) {
    v[0] = ld1(p);
  } else {
    const uint2 a = __ldg(reinterpret_cast<const uint2*>(p));
    v[0] = unpack(a.x);
    v[1] = unpack(a.y);
  }
}
template <int R>
WD_DEV void str(float2* __restrict__ p, const Cx<float> v[R]) {
  if constexpr (R == 1)
    *p = make_float2(v[0].re, v[0].im);
  else
    *reinterpret_cast<float4*>(p) = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
}
template <int R>
WD_DEV void str(bf16x2* __restrict__ p, const Cx<float> v[R]) {
  if constexpr (R == 1)
    p->w = pack(v[0]);
  else
    *reinterpret_cast<uint2*>(p) = make_uint2(pack(v[0]), pack(v[1]));
}
// FP64 site-major output (the last sweep): R consecutive complex doubles.
template <int R>
WD_DEV void str(double* __restrict__ p, const Cx<float> v[R]) {
#pragma unroll
  for (int q = 0; q < R; ++q) stc(p + 2 * q, cmake<double>(v[q].re, v[q].im));
}

// The value an element of type E holds after storing a.
template <typename E>
WD_DEV Cx<float> stored(Cx<float> a) {
  if constexpr (std::is_same<E, bf16x2>::value) return unpack(pack(a));
  else return a;
}

// Address of component k of (site s, rhs r): component-major element, or site-major FP64.
template <typename TY>
WD_DEV TY* at(TY* y, size_t V, int L, int s, int k, int r) {
  if constexpr (std::is_same<TY, double>::value)
    return y + 2 * (((size_t)s * 12 + k) * L + r);
  else
    return y + ((size_t)k * V + s) * L + r;
}

// ------------------------------------------------------------------ links
// The 3x3 link whose entry (a, b) sits at U[(3a + b) V].  Row 2 is read, or rebuilt from rows 0
// and 1: for a special unitary matrix it is conj(row0 x row1).
WD_DEV void load_link(const float2* __restrict__ U, size_t V, bool link12, Cx<float> m[3][3]) {
#pragma unroll
  for (int e = 0; e < 6; ++e) m[e / 3][e % 3] = ld1(U + e * V);
  if (link12) {
    m[2][0] = conj(cmul(m[0][1], m[1][2]) - cmul(m[0][2], m[1][1]));
    m[2][1] = conj(cmul(m[0][2], m[1][0]) - cmul(m[0][0], m[1][2]));
    m[2][2] = conj(cmul(m[0][0], m[1][1]) - cmul(m[0][1], m[1][0]));
  } else {
#pragma unroll
    for (int b = 0; b < 3; ++b) m[2][b] = ld1(U + (6 + b) * V);
  }
}

// ------------------------------------------------------------------ one hopping direction
// Direction mu, DIR = +1 (forward) or -1 (backward): adds (1 - DIR g_mu) W x_n to (au, ad) for R
// right-hand sides, where x_n is the neighbour spinor and W = U_mu(s) for DIR = +1 or
// U_mu(s - mu)^H for DIR = -1.  Only the projected 2-spinor h = x_up - DIR G_mu x_down is
// multiplied by the link.  hop_project forms h for one colour from the neighbour's four spin rows
// of that colour (so that only four rows are live at a time); hop_mult applies the link m.
template <int MU, int DIR, int R>
WD_DEV void hop_project(const Cx<float> u0[R], const Cx<float> u1[R], const Cx<float> d0[R],
                        const Cx<float> d1[R], int col, Cx<float> h0[R][3], Cx<float> h1[R][3]) {
#pragma unroll
  for (int q = 0; q < R; ++q) {
    Cx<float> g0, g1;
    gamma_down<MU>(d0[q], d1[q], g0, g1);
    if constexpr (DIR > 0) { h0[q][col] = u0[q] - g0; h1[q][col] = u1[q] - g1; }
    else { h0[q][col] = u0[q] + g0; h1[q][col] = u1[q] + g1; }
  }
}

template <int MU, int DIR, int R>
WD_DEV void hop_mult(const Cx<float> h0[R][3], const Cx<float> h1[R][3], const Cx<float> m[3][3],
                     Cx<float> au[R][2][3], Cx<float> ad[R][2][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int q = 0; q < R; ++q) {
      Cx<float> w0 = czero<float>(), w1 = czero<float>();
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if constexpr (DIR > 0) { w0 = cfma(m[a][b], h0[q][b], w0); w1 = cfma(m[a][b], h1[q][b], w1); }
        else { w0 = cfmaj(m[b][a], h0[q][b], w0); w1 = cfmaj(m[b][a], h1[q][b], w1); }
      }
      Cx<float> g0, g1;
      gamma_up<MU>(w0, w1, g0, g1);
      au[q][0][a] = au[q][0][a] + w0;
      au[q][1][a] = au[q][1][a] + w1;
      if constexpr (DIR > 0) { ad[q][0][a] = ad[q][0][a] - g0; ad[q][1][a] = ad[q][1][a] - g1; }
      else { ad[q][0][a] = ad[q][0][a] + g0; ad[q][1][a] = ad[q][1][a] + g1; }
    }
}

// The direction with the neighbour spinor and the link read from global memory.
template <int MU, int DIR, int R, typename E>
WD_DEV void hop(const E* __restrict__ x, const float2* __restrict__ links, const Geom& g, int s,
                const int c[4], int r0, int L, bool link12, Cx<float> au[R][2][3],
                Cx<float> ad[R][2][3]) {
  const int sn = neighbour(g, s, c, MU, DIR);
  const size_t V = (size_t)g.V;
  const E* base = x + (size_t)sn * L + r0;
  const size_t cs = V * L;   // elements between components
  Cx<float> h0[R][3], h1[R][3];
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    Cx<float> u0[R], u1[R], d0[R], d1[R];
    ldr<R>(base + (0 * 3 + col) * cs, u0);
    ldr<R>(base + (1 * 3 + col) * cs, u1);
    ldr<R>(base + (2 * 3 + col) * cs, d0);
    ldr<R>(base + (3 * 3 + col) * cs, d1);
    hop_project<MU, DIR, R>(u0, u1, d0, d1, col, h0, h1);
  }
  Cx<float> m[3][3];
  load_link(links + (size_t)MU * 9 * V + (DIR > 0 ? s : sn), V, link12, m);
  hop_mult<MU, DIR, R>(h0, h1, m, au, ad);
}

// ------------------------------------------------------------------ sweep, R RHS per thread
template <int R, typename E, typename TY, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
sweep_kernel(const E* __restrict__ x, TY* __restrict__ y, const E* __restrict__ u,
             const float2* __restrict__ links, const float* __restrict__ clov_inv, Geom g, int L,
             float kappa, int link12) {
  const int groups = L / R;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.V * groups) return;
  const int s = tid / groups;
  const int r0 = (tid - s * groups) * R;
  const size_t V = (size_t)g.V;
  const bool l12 = link12 != 0;
  int c[4];
  site_coords(g, s, c);
  Cx<float> au[R][2][3], ad[R][2][3];
#pragma unroll
  for (int q = 0; q < R; ++q)
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) { au[q][a][b] = czero<float>(); ad[q][a][b] = czero<float>(); }
  hop<0, +1, R>(x, links, g, s, c, r0, L, l12, au, ad);
  hop<0, -1, R>(x, links, g, s, c, r0, L, l12, au, ad);
  hop<1, +1, R>(x, links, g, s, c, r0, L, l12, au, ad);
  hop<1, -1, R>(x, links, g, s, c, r0, L, l12, au, ad);
  hop<2, +1, R>(x, links, g, s, c, r0, L, l12, au, ad);
  hop<2, -1, R>(x, links, g, s, c, r0, L, l12, au, ad);
  hop<3, +1, R>(x, links, g, s, c, r0, L, l12, au, ad);
  hop<3, -1, R>(x, links, g, s, c, r0, L, l12, au, ad);
#pragma unroll
  for (int ch = 0; ch < 2; ++ch) {
    Cx<float> vin[R][6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int k = ch * 6 + i;
      Cx<float> uu[R];
      ldr<R>(u + ((size_t)k * V + s) * L + r0, uu);
#pragma unroll
      for (int q = 0; q < R; ++q)
        vin[q][i] = uu[q] + kappa * (ch == 0 ? au[q][i / 3][i % 3] : ad[q][i / 3][i % 3]);
    }
    Cx<float> out[R][6];
#pragma unroll
    for (int q = 0; q < R; ++q) herm6s(clov_inv + (size_t)ch * CLOV_REALS * V + s, V, vin[q], out[q]);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      Cx<float> o[R];
#pragma unroll
      for (int q = 0; q < R; ++q) o[q] = out[q][i];
      str<R>(at(y, V, L, s, ch * 6 + i, r0), o);
    }
  }
}

// ------------------------------------------------------------------ sweep, split stencil
// The same sweep with the stencil of one (site, rhs) pair split over two warps: in every group of
// 64 threads, warp 0 takes the x and y hops and warp 1 the z and t hops of the same 32 pairs; the
// partial sums meet in shared memory, and warp 0 then applies the chirality + block of A_D^{-1}
// while warp 1 applies the chirality - block.  Twice as many warps cover the same pairs.
template <typename E, typename TY>
__global__ void __launch_bounds__(128)
sweep_split_kernel(const E* __restrict__ x, TY* __restrict__ y, const E* __restrict__ u,
                   const float2* __restrict__ links, const float* __restrict__ clov_inv, Geom g,
                   int L, float kappa, int link12) {
  __shared__ float xch[2][2][12][2][32];   // [group][warp half][component][re/im][lane]
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;       // 0..3
  const int grp = warp >> 1, half = warp & 1;
  const long long pair = ((long long)blockIdx.x * 2 + grp) * 32 + lane;
  const bool valid = pair < (long long)g.V * L;
  const int s = valid ? (int)(pair / L) : 0;
  const int r = valid ? (int)(pair - (long long)s * L) : 0;
  const size_t V = (size_t)g.V;
  const bool l12 = link12 != 0;
  Cx<float> au[1][2][3], ad[1][2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) { au[0][a][b] = czero<float>(); ad[0][a][b] = czero<float>(); }
  if (valid) {
    int c[4];
    site_coords(g, s, c);
    if (half == 0) {
      hop<0, +1, 1>(x, links, g, s, c, r, L, l12, au, ad);
      hop<0, -1, 1>(x, links, g, s, c, r, L, l12, au, ad);
      hop<1, +1, 1>(x, links, g, s, c, r, L, l12, au, ad);
      hop<1, -1, 1>(x, links, g, s, c, r, L, l12, au, ad);
    } else {
      hop<2, +1, 1>(x, links, g, s, c, r, L, l12, au, ad);
      hop<2, -1, 1>(x, links, g, s, c, r, L, l12, au, ad);
      hop<3, +1, 1>(x, links, g, s, c, r, L, l12, au, ad);
      hop<3, -1, 1>(x, links, g, s, c, r, L, l12, au, ad);
    }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    xch[grp][half][k][0][lane] = au[0][k / 3][k % 3].re;
    xch[grp][half][k][1][lane] = au[0][k / 3][k % 3].im;
    xch[grp][half][6 + k][0][lane] = ad[0][k / 3][k % 3].re;
    xch[grp][half][6 + k][1][lane] = ad[0][k / 3][k % 3].im;
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
    vin[i] = ld1(u + ((size_t)k * V + s) * L + r) + kappa * hs;
  }
  herm6s(clov_inv + (size_t)ch * CLOV_REALS * V + s, V, vin, out);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    Cx<float> o[1] = {out[i]};
    str<1>(at(y, V, L, s, ch * 6 + i, r), o);
  }
}

// ------------------------------------------------------------------ sweep, staged loads
// The sweep with 2 RHS per thread in 64-thread CTAs, where each thread copies the neighbour spinor
// rows and link entries of the next direction into shared memory with cp.async while it computes
// the current one (two stages), and prefetches its own U rows during the last direction.  Each
// thread reads back only what it copied itself, so no barrier is needed: cp.async.wait_group
// orders a thread's own copies before its reads.  The shared arrays are [stage][row][thread], so a
// warp's 32 accesses to one row are contiguous.
template <typename E> struct Row2;
template <> struct Row2<float2> { using T = float4; static constexpr int BYTES = 16; static constexpr int MINB = 6; };
template <> struct Row2<bf16x2> { using T = uint2; static constexpr int BYTES = 8; static constexpr int MINB = 8; };

WD_DEV void from_row(float4 a, Cx<float> v[2]) { v[0] = {a.x, a.y}; v[1] = {a.z, a.w}; }
WD_DEV void from_row(uint2 a, Cx<float> v[2]) { v[0] = unpack(a.x); v[1] = unpack(a.y); }

template <int BYTES>
WD_DEV void cp_async(void* smem, const void* gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gmem), "n"(BYTES)
                 : "memory");
}
WD_DEV void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
WD_DEV void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int ST_THREADS = 64;

// Issues the copies of direction H = 2 mu + (0: forward, 1: backward) into one stage.
template <int H, typename E>
WD_DEV void stage_hop(const E* __restrict__ x, const float2* __restrict__ links, const Geom& g,
                      int s, const int c[4], int r0, int L, bool link12,
                      typename Row2<E>::T (*sx)[ST_THREADS], float2 (*sl)[ST_THREADS], int t) {
  constexpr int MU = H / 2, DIR = (H % 2 == 0) ? 1 : -1;
  const int sn = neighbour(g, s, c, MU, DIR);
  const size_t V = (size_t)g.V;
  const E* base = x + (size_t)sn * L + r0;
#pragma unroll
  for (int k = 0; k < 12; ++k) cp_async<Row2<E>::BYTES>(&sx[k][t], base + (size_t)k * V * L);
  const float2* U = links + (size_t)MU * 9 * V + (DIR > 0 ? s : sn);
#pragma unroll
  for (int e = 0; e < 6; ++e) cp_async<8>(&sl[e][t], U + e * V);
  if (!link12) {
#pragma unroll
    for (int e = 6; e < 9; ++e) cp_async<8>(&sl[e][t], U + e * V);
  }
  cp_commit();
}

template <int H, typename E>
WD_DEV void hop_staged(const typename Row2<E>::T (*sx)[ST_THREADS], const float2 (*sl)[ST_THREADS],
                       int t, bool link12, Cx<float> au[2][2][3], Cx<float> ad[2][2][3]) {
  constexpr int MU = H / 2, DIR = (H % 2 == 0) ? 1 : -1;
  Cx<float> h0[2][3], h1[2][3];
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    Cx<float> u0[2], u1[2], d0[2], d1[2];
    from_row(sx[0 * 3 + col][t], u0);
    from_row(sx[1 * 3 + col][t], u1);
    from_row(sx[2 * 3 + col][t], d0);
    from_row(sx[3 * 3 + col][t], d1);
    hop_project<MU, DIR, 2>(u0, u1, d0, d1, col, h0, h1);
  }
  Cx<float> m[3][3];
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const float2 v = sl[e][t];
    m[e / 3][e % 3] = {v.x, v.y};
  }
  if (link12) {
    m[2][0] = conj(cmul(m[0][1], m[1][2]) - cmul(m[0][2], m[1][1]));
    m[2][1] = conj(cmul(m[0][2], m[1][0]) - cmul(m[0][0], m[1][2]));
    m[2][2] = conj(cmul(m[0][0], m[1][1]) - cmul(m[0][1], m[1][0]));
  } else {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float2 v = sl[6 + b][t];
      m[2][b] = {v.x, v.y};
    }
  }
  hop_mult<MU, DIR, 2>(h0, h1, m, au, ad);
}

template <typename E, typename TY>
__global__ void __launch_bounds__(ST_THREADS, Row2<E>::MINB)
sweep_staged_kernel(const E* __restrict__ x, TY* __restrict__ y, const E* __restrict__ u,
                    const float2* __restrict__ links, const float* __restrict__ clov_inv, Geom g,
                    int L, float kappa, int link12) {
  using Row = typename Row2<E>::T;
  __shared__ Row sx[2][12][ST_THREADS];
  __shared__ float2 sl[2][9][ST_THREADS];
  const int groups = L / 2;
  const int tid = blockIdx.x * ST_THREADS + threadIdx.x;
  if (tid >= g.V * groups) return;
  const int t = threadIdx.x;
  const int s = tid / groups;
  const int r0 = (tid - s * groups) * 2;
  const size_t V = (size_t)g.V;
  const bool l12 = link12 != 0;
  int c[4];
  site_coords(g, s, c);
  Cx<float> au[2][2][3], ad[2][2][3];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) { au[q][a][b] = czero<float>(); ad[q][a][b] = czero<float>(); }
  stage_hop<0>(x, links, g, s, c, r0, L, l12, sx[0], sl[0], t);
  stage_hop<1>(x, links, g, s, c, r0, L, l12, sx[1], sl[1], t);
  cp_wait<1>(); hop_staged<0, E>(sx[0], sl[0], t, l12, au, ad);
  stage_hop<2>(x, links, g, s, c, r0, L, l12, sx[0], sl[0], t);
  cp_wait<1>(); hop_staged<1, E>(sx[1], sl[1], t, l12, au, ad);
  stage_hop<3>(x, links, g, s, c, r0, L, l12, sx[1], sl[1], t);
  cp_wait<1>(); hop_staged<2, E>(sx[0], sl[0], t, l12, au, ad);
  stage_hop<4>(x, links, g, s, c, r0, L, l12, sx[0], sl[0], t);
  cp_wait<1>(); hop_staged<3, E>(sx[1], sl[1], t, l12, au, ad);
  stage_hop<5>(x, links, g, s, c, r0, L, l12, sx[1], sl[1], t);
  cp_wait<1>(); hop_staged<4, E>(sx[0], sl[0], t, l12, au, ad);
  stage_hop<6>(x, links, g, s, c, r0, L, l12, sx[0], sl[0], t);
  cp_wait<1>(); hop_staged<5, E>(sx[1], sl[1], t, l12, au, ad);
  stage_hop<7>(x, links, g, s, c, r0, L, l12, sx[1], sl[1], t);
  cp_wait<1>(); hop_staged<6, E>(sx[0], sl[0], t, l12, au, ad);
  // U rows of this site into stage 0
#pragma unroll
  for (int k = 0; k < 12; ++k)
    cp_async<Row2<E>::BYTES>(&sx[0][k][t], u + ((size_t)k * V + s) * L + r0);
  cp_commit();
  cp_wait<1>(); hop_staged<7, E>(sx[1], sl[1], t, l12, au, ad);
  cp_wait<0>();
#pragma unroll
  for (int ch = 0; ch < 2; ++ch) {
    Cx<float> vin[2][6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      Cx<float> uu[2];
      from_row(sx[0][ch * 6 + i][t], uu);
#pragma unroll
      for (int q = 0; q < 2; ++q)
        vin[q][i] = uu[q] + kappa * (ch == 0 ? au[q][i / 3][i % 3] : ad[q][i / 3][i % 3]);
    }
    Cx<float> out[2][6];
#pragma unroll
    for (int q = 0; q < 2; ++q) herm6s(clov_inv + (size_t)ch * CLOV_REALS * V + s, V, vin[q], out[q]);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      Cx<float> o[2] = {out[0][i], out[1][i]};
      str<2>(at(y, V, L, s, ch * 6 + i, r0), o);
    }
  }
}

// ------------------------------------------------------------------ first sweep (from G = 0)
// Reads the FP64 right-hand side U (site-major), stores its low-precision copy in u_lp (when not
// null) for the later sweeps, and writes G = A_D^{-1} U computed in FP32: component-major
// low-precision elements, or site-major FP64 when it is also the last sweep.
template <typename E, typename TY>
__global__ void __launch_bounds__(128)
site_inverse_kernel(const double* __restrict__ u, E* __restrict__ u_lp, TY* __restrict__ y,
                    const float* __restrict__ clov_inv, int V, int L) {
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
      Cx<float> v[1] = {cmake<float>((float)a.re, (float)a.im)};
      v[0] = stored<E>(v[0]);   // the later sweeps see U as stored
      if (u_lp) str<1>(at(u_lp, (size_t)V, L, s, k, r), v);
      vin[ch][i] = v[0];
    }
  herm6s(clov_inv + s, (size_t)V, vin[0], out[0]);
  herm6s(clov_inv + (size_t)CLOV_REALS * V + s, (size_t)V, vin[1], out[1]);
#pragma unroll
  for (int ch = 0; ch < 2; ++ch)
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      Cx<float> o[1] = {out[ch][i]};
      str<1>(at(y, (size_t)V, L, s, ch * 6 + i, r), o);
    }
}

// ------------------------------------------------------------------ launchers
constexpr int SI_THREADS = 128;

template <typename E>
cudaError_t launch_site_inverse(const Op& op, const double* u, E* u_lp, E* g_lp, double* g64,
                                int L, cudaStream_t st) {
  const unsigned grid = (unsigned)(((long long)op.g.V * L + SI_THREADS - 1) / SI_THREADS);
  if (g_lp)
    site_inverse_kernel<E, E><<<grid, SI_THREADS, 0, st>>>(u, u_lp, g_lp, op.clov_inv32, op.g.V, L);
  else
    site_inverse_kernel<E, double><<<grid, SI_THREADS, 0, st>>>(u, u_lp, g64, op.clov_inv32,
                                                                 op.g.V, L);
  return cudaGetLastError();
}

template <int R, typename E, typename TY>
cudaError_t launch_sweep_r(const Op& op, const E* g_in, const E* u_lp, TY* out, int L, int block,
                           int min_blocks, cudaStream_t st) {
  const long long n = (long long)op.g.V * (L / R);
  const unsigned grid = (unsigned)((n + block - 1) / block);
  const float2* links = reinterpret_cast<const float2*>(op.links32);
  if (min_blocks == 8 && block == 64)    // at most 128 registers: 16 warps per SM
    sweep_kernel<R, E, TY, 64, 8><<<grid, block, 0, st>>>(g_in, out, u_lp, links, op.clov_inv32,
                                                          op.g, L, (float)op.kappa, op.link12);
  else if (min_blocks == 12 && block == 64 && R == 1)   // at most 80 registers: 24 warps per SM
    sweep_kernel<1, E, TY, 64, 12><<<grid, block, 0, st>>>(g_in, out, u_lp, links, op.clov_inv32,
                                                           op.g, L, (float)op.kappa, op.link12);
  else
    sweep_kernel<R, E, TY, 256, 1><<<grid, block, 0, st>>>(g_in, out, u_lp, links, op.clov_inv32,
                                                           op.g, L, (float)op.kappa, op.link12);
  return cudaGetLastError();
}

template <typename E, typename TY>
cudaError_t launch_sweep_split(const Op& op, const E* g_in, const E* u_lp, TY* out, int L,
                               cudaStream_t st) {
  const long long pairs = (long long)op.g.V * L;
  const unsigned grid = (unsigned)((pairs + 63) / 64);   // 64 pairs per 128-thread CTA
  sweep_split_kernel<E, TY><<<grid, 128, 0, st>>>(g_in, out, u_lp,
                                                  reinterpret_cast<const float2*>(op.links32),
                                                  op.clov_inv32, op.g, L, (float)op.kappa,
                                                  op.link12);
  return cudaGetLastError();
}

template <typename E, typename TY>
cudaError_t launch_sweep_staged(const Op& op, const E* g_in, const E* u_lp, TY* out, int L,
                                cudaStream_t st) {
  const long long n = (long long)op.g.V * (L / 2);
  const unsigned grid = (unsigned)((n + ST_THREADS - 1) / ST_THREADS);
  sweep_staged_kernel<E, TY><<<grid, ST_THREADS, 0, st>>>(
      g_in, out, u_lp, reinterpret_cast<const float2*>(op.links32), op.clov_inv32, op.g, L,
      (float)op.kappa, op.link12);
  return cudaGetLastError();
}

// One sweep with the tile (rhs_per_thread, block, min_blocks, staged); rhs_per_thread 0 is the
// split stencil, staged the shared-memory pipeline (2 RHS per thread, 64 threads).  Exactly one of
// g_lp / g64 is non-null.
template <typename E>
cudaError_t launch_sweep_tiled(const Op& op, const E* g_in, const E* u_lp, E* g_lp, double* g64,
                               int L, int rhs_per_thread, int block, int min_blocks, int staged,
                               cudaStream_t st) {
  if (staged) {
    if (rhs_per_thread != 2 || block != ST_THREADS || L % 2 != 0) return cudaErrorInvalidValue;
    return g_lp ? launch_sweep_staged<E, E>(op, g_in, u_lp, g_lp, L, st)
                : launch_sweep_staged<E, double>(op, g_in, u_lp, g64, L, st);
  }
  if (rhs_per_thread == 0)
    return g_lp ? launch_sweep_split<E, E>(op, g_in, u_lp, g_lp, L, st)
                : launch_sweep_split<E, double>(op, g_in, u_lp, g64, L, st);
  if (L % rhs_per_thread != 0 || (block != 64 && block != 128 && block != 256))
    return cudaErrorInvalidValue;
  switch (rhs_per_thread) {
    case 1: return g_lp ? launch_sweep_r<1, E, E>(op, g_in, u_lp, g_lp, L, block, min_blocks, st)
                        : launch_sweep_r<1, E, double>(op, g_in, u_lp, g64, L, block, min_blocks, st);
    case 2: return g_lp ? launch_sweep_r<2, E, E>(op, g_in, u_lp, g_lp, L, block, min_blocks, st)
                        : launch_sweep_r<2, E, double>(op, g_in, u_lp, g64, L, block, min_blocks, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lp
