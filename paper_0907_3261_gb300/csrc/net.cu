// Learned gauge-covariant preconditioner: inference and training kernels.
//
// The paper names a better preconditioner than j-step Jacobi as future work (Sec. 4).  This network
// is linear in the spinor, so M_net is a fixed linear operator for block BiCGGR, and gauge
// covariant.  A layer maps C_in to C_out channels of spinor fields:
//     out_{c'}(x) = sum_{d=0..8} sum_c W[d][c'][c] (T_d psi_c)(x),
//     T_0 psi = psi,  T_{1+mu} psi(x) = U_mu(x) psi(x+mu),  T_{5+mu} psi(x) = U_mu(x-mu)^H psi(x-mu),
// W[d][c'][c] a complex 4x4 spin matrix.  Activations are component-major per channel,
// [channel][spin*3+colour][site][rhs], stored in FP32 (training and inference) or BF16 (inference
// only), with FP32 arithmetic; weights are complex64, [9][C_out][C_in][4][4] per layer.
// Training minimises (1/L) sum_i ||N(r_i) - e_i||^2 / ||e_i||^2 over pairs (r_i, e_i = A^{-1} r_i):
// the backward pass runs each layer's adjoint (T_d^H = T_{opposite d}, W -> W^H, channels swapped)
// with the same layer kernel, and the weight gradient d loss / d conj(W) is a deterministic
// two-level reduction of delta_{c'} (T_d a_c)^H over sites, RHS and colour.  Adam updates the
// real parameters (Re W, Im W) with the real gradient (2 Re G, 2 Im G).
#include <cstdint>
#include <vector>

#include "common.cuh"
#include "elem.cuh"
#include "internal.h"

namespace {

// 64-thread CTAs: the 4->4 layer's 168 registers a thread and 36.9 KB of staged weights fit six
// CTAs (12 warps) per SM, where 128-thread CTAs fit two or three.
constexpr int NET_THREADS = 64;
constexpr int WG_THREADS = 256;
constexpr int WG_PAIRS = 32;        // (site, rhs) pairs per chunk of the weight-gradient kernel

// v <- U v (DIR = +1) or U^H v (DIR = -1) on the colour index of a 4x3 spinor.
template <int DIR>
WD_DEV void colour_mult(const float* __restrict__ U, size_t V, Cx<float> v[12]) {
  Cx<float> u[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) u[a][b] = ldc(U + 2 * (size_t)(a * 3 + b) * V);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) {
    Cx<float> w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Cx<float> acc = czero<float>();
#pragma unroll
      for (int b = 0; b < 3; ++b)
        acc = DIR > 0 ? cfma(u[a][b], v[sp * 3 + b], acc) : cfmaj(u[b][a], v[sp * 3 + b], acc);
      w[a] = acc;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) v[sp * 3 + a] = w[a];
  }
}

// T_d psi at site s for one channel of a component-major block; x points at the channel.
template <int D, typename E>
WD_DEV void transport_at(const E* __restrict__ x, const float* __restrict__ links,
                         const Geom& g, int s, const int c[4], int r, int L, Cx<float> v[12]) {
  const size_t V = (size_t)g.V;
  int sn = s;
  if constexpr (D >= 1 && D <= 4) sn = neighbour(g, s, c, D - 1, +1);
  if constexpr (D >= 5) sn = neighbour(g, s, c, D - 5, -1);
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = lp::ld1(x + ((size_t)k * V + sn) * L + r);
  if constexpr (D >= 1 && D <= 4) colour_mult<+1>(links + 2 * ((size_t)(D - 1) * 9 * V + s), V, v);
  if constexpr (D >= 5) colour_mult<-1>(links + 2 * ((size_t)(D - 5) * 9 * V + sn), V, v);
}

// acc + a b for complex values held as (re, im) lane pairs, with a given as the pairs
// (a.re, a.re) and (-a.im, a.im) and b also as (b.im, b.re): two paired FMAs, rounded in the same
// order as cfma (re: (acc + a.re b.re) - a.im b.im; im: (acc + a.re b.im) + a.im b.re).
WD_DEV float2 cfma_pair(float2 arr, float2 nai, float2 b, float2 bsw, float2 acc) {
  return __ffma2_rn(nai, bsw, __ffma2_rn(arr, b, acc));
}

// T_d psi at site s for one channel, the direction d (0..8) given at run time, so that one rolled
// loop over d serves all nine (an unrolled body of nine directions takes every register and spills).
// The result is returned as lane pairs v and their swapped copies vs, ready for cfma_pair.
template <typename E>
WD_DEV void transport_rt(const E* __restrict__ x, const float* __restrict__ links, const Geom& g,
                         int s, const int c[4], int r, int L, int d, float2 v[12], float2 vs[12]) {
  const size_t V = (size_t)g.V;
  int sn = s;
  const int mu = (d - 1) & 3;
  const bool fwd = d <= 4;
  if (d > 0) {
    const int cm = mu == 0 ? c[0] : mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
    const int dm = mu == 0 ? g.d[0] : mu == 1 ? g.d[1] : mu == 2 ? g.d[2] : g.d[3];
    const int st = mu == 0 ? g.stride[0] : mu == 1 ? g.stride[1] : mu == 2 ? g.stride[2] : g.stride[3];
    sn = fwd ? (cm == dm - 1 ? s - (dm - 1) * st : s + st) : (cm == 0 ? s + (dm - 1) * st : s - st);
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const Cx<float> t = lp::ld1(x + ((size_t)k * V + sn) * L + r);
    v[k] = make_float2(t.re, t.im);
  }
  if (d > 0) {
    // W = U_mu(s) forward, U_mu(s - mu)^H backward: entry (a, b) = u[a][b] or conj(u[b][a])
    const float* U = links + 2 * ((size_t)mu * 9 * V + (fwd ? s : sn));
    float2 w[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = make_float2(0.f, 0.f);
    // each link entry is loaded, paired and used on the four spins before the next one
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const Cx<float> t = ldc(U + 2 * (size_t)((fwd ? a * 3 + b : b * 3 + a)) * V);
        const float im = fwd ? t.im : -t.im;
        const float2 mrr = make_float2(t.re, t.re), mni = make_float2(-im, im);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
          const float2 x2 = v[sp * 3 + b];
          w[sp * 3 + a] = cfma_pair(mrr, mni, x2, make_float2(x2.y, x2.x), w[sp * 3 + a]);
        }
      }
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = w[k];
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) vs[k] = make_float2(v[k].y, v[k].x);
}

// One gauge-covariant layer: out_co(x) = sum_d sum_ci W[d][co][ci] (T_d in_ci)(x), one thread per
// (site, RHS). The weights sit in shared memory as (w.re, w.re, -w.im, w.im), the direction and
// input-channel loops are rolled (an unrolled body overflows the instruction cache) and the output
// channels' accumulators stay in registers.
template <int CIN, int COUT, typename E>
__global__ void __launch_bounds__(NET_THREADS, 5)
net_layer_kernel(const E* __restrict__ in, E* __restrict__ out,
                 const float* __restrict__ links, const float2* __restrict__ W, Geom g, int L) {
  __shared__ float4 Ws[9 * COUT * CIN * 16];
  for (int e = threadIdx.x; e < 9 * COUT * CIN * 16; e += blockDim.x) {
    const float2 w = W[e];
    Ws[e] = make_float4(w.x, w.x, -w.y, w.y);
  }
  __syncthreads();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.V * L) return;
  const int s = tid / L;
  const int r = tid - s * L;
  int c[4];
  site_coords(g, s, c);
  float2 acc[COUT][12];
#pragma unroll
  for (int co = 0; co < COUT; ++co)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[co][k] = make_float2(0.f, 0.f);
  const size_t chan_in = (size_t)12 * g.V * L;
#pragma unroll 1
  for (int d = 0; d < 9; ++d) {
#pragma unroll 1
    for (int ci = 0; ci < CIN; ++ci) {
      float2 v[12], vs[12];
      transport_rt(in + ci * chan_in, links, g, s, c, r, L, d, v, vs);
#pragma unroll
      for (int co = 0; co < COUT; ++co) {
        const float4* w = Ws + ((d * COUT + co) * CIN + ci) * 16;
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const float4 wv = w[sp * 4 + t];
            const float2 wrr = make_float2(wv.x, wv.y), wni = make_float2(wv.z, wv.w);
#pragma unroll
            for (int a = 0; a < 3; ++a)
              acc[co][sp * 3 + a] = cfma_pair(wrr, wni, v[t * 3 + a], vs[t * 3 + a],
                                              acc[co][sp * 3 + a]);
          }
      }
    }
  }
  const size_t V = (size_t)g.V;
  const size_t chan = (size_t)12 * V * L;
#pragma unroll
  for (int co = 0; co < COUT; ++co)
#pragma unroll
    for (int k = 0; k < 12; ++k)
      lp::st1(out + co * chan + ((size_t)k * V + s) * L + r, Cx<float>{acc[co][k].x, acc[co][k].y});
}

// W^adj[d'][c][c'] = W[d][c'][c]^H with d' the opposite direction of d (0 stays 0).
__global__ void adjoint_weights_kernel(const float2* __restrict__ W, float2* __restrict__ Wa,
                                       int cin, int cout) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = 9 * cout * cin * 16;
  if (e >= n) return;
  // e indexes W: ((d*cout + co)*cin + ci)*16 + sp*4 + t
  const int t = e % 4, sp = (e / 4) % 4, ci = (e / 16) % cin, co = (e / (16 * cin)) % cout;
  const int d = e / (16 * cin * cout);
  const int da = d == 0 ? 0 : (d <= 4 ? d + 4 : d - 4);
  const float2 w = W[e];
  // adjoint layer maps cout -> cin channels: Wa[((da*cin + ci)*cout + co)*16 + t*4 + sp]
  Wa[((da * cin + ci) * cout + co) * 16 + t * 4 + sp] = make_float2(w.x, -w.y);
}

// FP64 site-major block -> component-major channel (FP32 or BF16 elements), and back.
template <typename E>
__global__ void to_cm_kernel(const double* __restrict__ x, E* __restrict__ y, int V, int L) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= V * L) return;
  const int s = tid / L, r = tid - (tid / L) * L;
  for (int k = 0; k < 12; ++k) {
    const Cx<double> a = ldc(x + 2 * (((size_t)s * 12 + k) * L + r));
    lp::st1(y + ((size_t)k * V + s) * L + r, cmake<float>((float)a.re, (float)a.im));
  }
}
template <typename E>
__global__ void from_cm_kernel(const E* __restrict__ y, double* __restrict__ x, int V, int L) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= V * L) return;
  const int s = tid / L, r = tid - (tid / L) * L;
  for (int k = 0; k < 12; ++k) {
    const Cx<float> a = lp::ld1(y + ((size_t)k * V + s) * L + r);
    stc(x + 2 * (((size_t)s * 12 + k) * L + r), cmake<double>(a.re, a.im));
  }
}

// delta = w_i (y - e) for column i, w_i = 1 / (L ||e_i||^2); per-block partial loss sums.
__global__ void __launch_bounds__(256)
loss_delta_kernel(const float* __restrict__ y, const double* __restrict__ E,
                  const double* __restrict__ wcol, float* __restrict__ delta,
                  double* __restrict__ part, int V, int L) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x; tid < (long long)V * L;
       tid += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(tid / L), r = (int)(tid - (tid / L) * L);
    const double w = wcol[r];
    for (int k = 0; k < 12; ++k) {
      const size_t cm = 2 * (((size_t)k * V + s) * L + r);
      const Cx<float> yv = ldc(y + cm);
      const Cx<double> ev = ldc(E + 2 * (((size_t)s * 12 + k) * L + r));
      const double dr = yv.re - ev.re, di = yv.im - ev.im;
      acc += w * (dr * dr + di * di);
      stc(delta + cm, cmake<float>((float)(w * dr), (float)(w * di)));
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Transported input of one channel at one (site, rhs) pair into shared memory.
template <int D>
WD_DEV void stage_transport(const float* __restrict__ in, const float* __restrict__ links,
                            const Geom& g, long long q, int L, float2* dst, int stride) {
  const int s = (int)(q / L), r = (int)(q - (q / L) * L);
  int c[4];
  site_coords(g, s, c);
  Cx<float> v[12];
  transport_at<D>(reinterpret_cast<const float2*>(in), links, g, s, c, r, L, v);
#pragma unroll
  for (int k = 0; k < 12; ++k) dst[k * stride] = make_float2(v[k].re, v[k].im);
}

template <int CIN, int COUT, int D>
WD_DEV void wgrad_dir(const float* __restrict__ in, const float* __restrict__ links,
                      const Geom& g, long long q0, int np, int L, float2* vs, const float2* ds,
                      Cx<float> acc[9][(COUT * CIN * 16 + WG_THREADS - 1) / WG_THREADS]) {
  constexpr int NE = COUT * CIN * 16;
  constexpr int PER = (NE + WG_THREADS - 1) / WG_THREADS;
  const size_t chan = (size_t)12 * g.V * L * 2;
  for (int task = threadIdx.x; task < CIN * WG_PAIRS; task += blockDim.x) {
    const int ci = task / WG_PAIRS, p = task - (task / WG_PAIRS) * WG_PAIRS;
    if (p < np) stage_transport<D>(in + ci * chan, links, g, q0 + p, L, vs + ci * 12 * WG_PAIRS + p, WG_PAIRS);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int e = threadIdx.x + j * WG_THREADS;
    if (e < NE) {
      const int t = e % 4, sp = (e / 4) % 4, ci = (e / 16) % CIN, co = e / (16 * CIN);
      Cx<float> a = acc[D][j];
      for (int p = 0; p < np; ++p)
#pragma unroll
        for (int col = 0; col < 3; ++col) {
          const float2 dv = ds[(co * 12 + sp * 3 + col) * WG_PAIRS + p];
          const float2 vv = vs[(ci * 12 + t * 3 + col) * WG_PAIRS + p];
          a = cfmaj(Cx<float>{vv.x, vv.y}, Cx<float>{dv.x, dv.y}, a);   // delta * conj(v)
        }
      acc[D][j] = a;
    }
  }
  __syncthreads();
}

// Partial sums of G[d][c'][c][sp][t] = sum_{site, rhs, colour} delta_c'[sp] conj((T_d a_c)[t]).
template <int CIN, int COUT>
__global__ void __launch_bounds__(WG_THREADS)
wgrad_kernel(const float* __restrict__ in, const float* __restrict__ delta,
             const float* __restrict__ links, Geom g, int L, double2* __restrict__ part) {
  constexpr int NE = COUT * CIN * 16;
  constexpr int PER = (NE + WG_THREADS - 1) / WG_THREADS;
  __shared__ float2 vs[CIN * 12 * WG_PAIRS];
  __shared__ float2 ds[COUT * 12 * WG_PAIRS];
  Cx<float> acc[9][PER];
#pragma unroll
  for (int d = 0; d < 9; ++d)
#pragma unroll
    for (int j = 0; j < PER; ++j) acc[d][j] = czero<float>();
  const long long pairs = (long long)g.V * L;
  const long long nchunks = (pairs + WG_PAIRS - 1) / WG_PAIRS;
  const size_t V = (size_t)g.V;
  const size_t chan = (size_t)12 * V * L * 2;
  for (long long ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
    const long long q0 = ck * WG_PAIRS;
    const int np = (int)min((long long)WG_PAIRS, pairs - q0);
    for (int task = threadIdx.x; task < COUT * 12 * WG_PAIRS; task += blockDim.x) {
      const int co = task / (12 * WG_PAIRS), k = (task / WG_PAIRS) % 12, p = task % WG_PAIRS;
      if (p < np) {
        const Cx<float> v = ldc(delta + co * chan + 2 * ((size_t)k * V * L + q0 + p));
        ds[(co * 12 + k) * WG_PAIRS + p] = make_float2(v.re, v.im);
      }
    }
    wgrad_dir<CIN, COUT, 0>(in, links, g, q0, np, L, vs, ds, acc);
    wgrad_dir<CIN, COUT, 1>(in, links, g, q0, np, L, vs, ds, acc);
    wgrad_dir<CIN, COUT, 2>(in, links, g, q0, np, L, vs, ds, acc);
    wgrad_dir<CIN, COUT, 3>(in, links, g, q0, np, L, vs, ds, acc);
    wgrad_dir<CIN, COUT, 4>(in, links, g, q0, np, L, vs, ds, acc);
    wgrad_dir<CIN, COUT, 5>(in, links, g, q0, np, L, vs, ds, acc);
    wgrad_dir<CIN, COUT, 6>(in, links, g, q0, np, L, vs, ds, acc);
    wgrad_dir<CIN, COUT, 7>(in, links, g, q0, np, L, vs, ds, acc);
    wgrad_dir<CIN, COUT, 8>(in, links, g, q0, np, L, vs, ds, acc);
  }
#pragma unroll
  for (int d = 0; d < 9; ++d)
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int e = threadIdx.x + j * WG_THREADS;
      if (e < NE) part[(size_t)blockIdx.x * 9 * NE + d * NE + e] = make_double2(acc[d][j].re, acc[d][j].im);
    }
}

// grad[d*NE + e] = sum over blocks of part, in block order.
__global__ void wgrad_finalize_kernel(const double2* __restrict__ part, int nblocks, int n,
                                      double2* __restrict__ grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nblocks; ++b) {
    const double2 v = part[(size_t)b * n + e];
    s.x += v.x;
    s.y += v.y;
  }
  grad[e] = s;
}

__global__ void loss_finalize_kernel(const double* __restrict__ part, int nblocks, double* loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += part[b];
  *loss = s;
}

// Adam on the real parameters (Re W, Im W) with real gradient (2 Re G, 2 Im G).
__global__ void adam_kernel(float2* __restrict__ W, const double2* __restrict__ G,
                            float2* __restrict__ m, float2* __restrict__ v, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gr = (float)(2.0 * G[e].x), gi = (float)(2.0 * G[e].y);
  float2 mm = m[e], vv = v[e], w = W[e];
  mm.x = b1 * mm.x + (1.f - b1) * gr;
  mm.y = b1 * mm.y + (1.f - b1) * gi;
  vv.x = b2 * vv.x + (1.f - b2) * gr * gr;
  vv.y = b2 * vv.y + (1.f - b2) * gi * gi;
  w.x -= lr * (mm.x / c1) / (sqrtf(vv.x / c2) + eps);
  w.y -= lr * (mm.y / c1) / (sqrtf(vv.y / c2) + eps);
  m[e] = mm;
  v[e] = vv;
  W[e] = w;
}

template <int CIN, int COUT, typename E>
cudaError_t run_layer(const Op& op, const E* in, E* out, const float2* W, int L, cudaStream_t st) {
  const long long n = (long long)op.g.V * L;
  net_layer_kernel<CIN, COUT, E><<<(unsigned)((n + NET_THREADS - 1) / NET_THREADS), NET_THREADS, 0, st>>>(
      in, out, op.links32, W, op.g, L);
  return cudaGetLastError();
}

template <typename E>
cudaError_t layer_by_channels(const Op& op, const E* in, E* out, const float2* W, int cin,
                              int cout, int L, cudaStream_t st) {
#define WD_LAYER(a, b) if (cin == a && cout == b) return run_layer<a, b, E>(op, in, out, W, L, st);
  WD_LAYER(1, 4) WD_LAYER(4, 4) WD_LAYER(4, 1) WD_LAYER(1, 2) WD_LAYER(2, 2) WD_LAYER(2, 1)
  WD_LAYER(1, 1)
#undef WD_LAYER
  return cudaErrorInvalidValue;
}

template <int CIN, int COUT>
cudaError_t run_wgrad(const Op& op, const float* in, const float* delta, int L, double2* part,
                      int nblocks, cudaStream_t st) {
  wgrad_kernel<CIN, COUT><<<nblocks, WG_THREADS, 0, st>>>(in, delta, op.links32, op.g, L, part);
  return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------------ launchers
cudaError_t net_launch_layer(const Op& op, const float* in, float* out, const float2* W, int cin,
                             int cout, int L, cudaStream_t st) {
  return layer_by_channels(op, reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out),
                           W, cin, cout, L, st);
}

cudaError_t net_launch_layer_bf16(const Op& op, const void* in, void* out, const float2* W,
                                  int cin, int cout, int L, cudaStream_t st) {
  return layer_by_channels(op, static_cast<const lp::bf16x2*>(in), static_cast<lp::bf16x2*>(out),
                           W, cin, cout, L, st);
}

cudaError_t net_launch_wgrad(const Op& op, const float* in, const float* delta, int cin, int cout,
                             int L, double2* part, int nblocks, double2* grad, cudaStream_t st) {
  cudaError_t e = cudaErrorInvalidValue;
#define WD_WG(a, b) if (cin == a && cout == b) e = run_wgrad<a, b>(op, in, delta, L, part, nblocks, st);
  WD_WG(1, 4) WD_WG(4, 4) WD_WG(4, 1) WD_WG(1, 2) WD_WG(2, 2) WD_WG(2, 1) WD_WG(1, 1)
#undef WD_WG
  if (e != cudaSuccess) return e;
  const int n = 9 * cout * cin * 16;
  wgrad_finalize_kernel<<<(n + 255) / 256, 256, 0, st>>>(part, nblocks, n, grad);
  return cudaGetLastError();
}

cudaError_t net_launch_adjoint_weights(const float2* W, float2* Wa, int cin, int cout,
                                       cudaStream_t st) {
  const int n = 9 * cout * cin * 16;
  adjoint_weights_kernel<<<(n + 255) / 256, 256, 0, st>>>(W, Wa, cin, cout);
  return cudaGetLastError();
}

cudaError_t net_launch_to_cm(const double* x, void* y, int V, int L, bool bf16, cudaStream_t st) {
  const unsigned grid = (unsigned)(((long long)V * L + 127) / 128);
  if (bf16)
    to_cm_kernel<<<grid, 128, 0, st>>>(x, static_cast<lp::bf16x2*>(y), V, L);
  else
    to_cm_kernel<<<grid, 128, 0, st>>>(x, static_cast<float2*>(y), V, L);
  return cudaGetLastError();
}

cudaError_t net_launch_from_cm(const void* y, double* x, int V, int L, bool bf16, cudaStream_t st) {
  const unsigned grid = (unsigned)(((long long)V * L + 127) / 128);
  if (bf16)
    from_cm_kernel<<<grid, 128, 0, st>>>(static_cast<const lp::bf16x2*>(y), x, V, L);
  else
    from_cm_kernel<<<grid, 128, 0, st>>>(static_cast<const float2*>(y), x, V, L);
  return cudaGetLastError();
}

cudaError_t net_launch_loss_delta(const float* y, const double* E, const double* wcol,
                                  float* delta, double* part, int nblocks, double* loss, int V,
                                  int L, cudaStream_t st) {
  loss_delta_kernel<<<nblocks, 256, 0, st>>>(y, E, wcol, delta, part, V, L);
  loss_finalize_kernel<<<1, 32, 0, st>>>(part, nblocks, loss);
  return cudaGetLastError();
}

cudaError_t net_launch_adam(float2* W, const double2* G, float2* m, float2* v, int n, float lr,
                            float b1, float b2, float eps, int t, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(W, G, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}
