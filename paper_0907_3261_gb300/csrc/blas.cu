// Tall-skinny block operations of preconditioned block BiCGGR (arXiv:0907.3261, Sec. 2, the
// algorithm box): the L x L Gram products R~_0^H V and R~_0^H R, the traces Tr[W^H R] and
// Tr[W^H W] that give zeta_k, the column norms of the stopping test, the L x L solves for alpha_k
// and gamma_k, and the block updates
//   U = (P - zeta V) alpha,  X += zeta F + G,  R -= zeta W + Y,  P = R + U gamma,  V = W + Y gamma.
//
// A block is N rows of L complex numbers (row n at n*L).  Every kernel walks rows in chunks of
// CH rows with a fixed chunk -> block assignment (block b takes chunks b, b + grid, ...), stages the
// chunk in shared memory, and accumulates its share of the reductions in a fixed order.  Each
// block writes its partial sums to a slot of `part`; a one-block finalize kernel adds the slots in
// block order.  Results are therefore bitwise reproducible from run to run (no float atomics).
#include "common.cuh"
#include "internal.h"

namespace {

constexpr int TS_THREADS = 256;
constexpr int CH = 32;                     // rows per chunk
constexpr int CHE = CH * WD_LMAX;          // complex entries per chunk at most
constexpr int CHU = 64;                    // rows per chunk of update_u (L = 12: 768 entries, 3 per thread)

WD_DEV Cx<double> ld2(const double* p, size_t e) {
  double2 v = *reinterpret_cast<const double2*>(p + 2 * e);
  return {v.x, v.y};
}
WD_DEV void st2(double* p, size_t e, Cx<double> a) {
  *reinterpret_cast<double2*>(p + 2 * e) = make_double2(a.re, a.im);
}
WD_DEV Cx<double> sm(const double2& v) { return {v.x, v.y}; }
WD_DEV double2 d2(Cx<double> a) { return make_double2(a.re, a.im); }

// Gram accumulation over one staged chunk: thread t < L*L owns entry (a, b) = (t / L, t % L) of
// A^H B; thread t < L also accumulates ||B_col t||^2 when `norms`.
WD_DEV void gram_chunk(const double2* As, const double2* Bs, int rows, int L, Cx<double>& acc,
                       double& nacc, bool norms) {
  const int t = threadIdx.x;
  if (t < L * L) {
    const int a = t / L, b = t - (t / L) * L;
    for (int n = 0; n < rows; ++n) acc = cfmaj(sm(As[n * L + a]), sm(Bs[n * L + b]), acc);
  }
  if (norms && t < L)
    for (int n = 0; n < rows; ++n) nacc += cnorm2(sm(Bs[n * L + t]));
}

WD_DEV void write_partial(double2* part, int L, Cx<double> acc, double nacc, bool norms) {
  const int t = threadIdx.x;
  double2* p = part + (size_t)blockIdx.x * PART_STRIDE;
  if (t < L * L) p[t] = d2(acc);
  if (norms && t < L) p[WD_LMAX * WD_LMAX + t] = make_double2(nacc, 0.0);
}

// ---------------------------------------------------------------- Gram A^H B (+ norms of B)
__global__ void __launch_bounds__(TS_THREADS)
gram_kernel(const double* __restrict__ A, const double* __restrict__ B, int L, long long rows,
            double2* __restrict__ part, bool norms) {
  __shared__ double2 As[CHE], Bs[CHE];
  Cx<double> acc = czero<double>();
  double nacc = 0.0;
  const long long nchunks = (rows + CH - 1) / CH;
  for (long long ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
    const long long r0 = ck * CH;
    const int nr = (int)min((long long)CH, rows - r0);
    const int cnt = nr * L;
    const size_t e0 = (size_t)r0 * L;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      As[e] = d2(ld2(A, e0 + e));
      Bs[e] = d2(ld2(B, e0 + e));
    }
    __syncthreads();
    gram_chunk(As, Bs, nr, L, acc, nacc, norms);
    __syncthreads();
  }
  write_partial(part, L, acc, nacc, norms);
}

// Column norms ||A_col||^2 only.
__global__ void __launch_bounds__(TS_THREADS)
colnorm_kernel(const double* __restrict__ A, int L, long long rows, double2* __restrict__ part) {
  __shared__ double red[TS_THREADS];
  // thread t handles column t % L of rows strided by (TS_THREADS / L) within a chunk
  const int per = TS_THREADS / L;
  const int col = threadIdx.x % L, lane_row = threadIdx.x / L;
  double acc = 0.0;
  if (lane_row < per) {
    const long long nchunks = (rows + CH - 1) / CH;
    for (long long ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
      const long long r0 = ck * CH;
      const int nr = (int)min((long long)CH, rows - r0);
      for (int n = lane_row; n < nr; n += per) acc += cnorm2(ld2(A, (size_t)(r0 + n) * L + col));
    }
  }
  red[threadIdx.x] = (lane_row < per) ? acc : 0.0;
  __syncthreads();
  if (threadIdx.x < L) {
    double s = 0.0;
    for (int k = 0; k < per; ++k) s += red[k * L + threadIdx.x];
    part[(size_t)blockIdx.x * PART_STRIDE + WD_LMAX * WD_LMAX + threadIdx.x] = make_double2(s, 0.0);
  }
}

// Tr[W^H R] and Tr[W^H W] over all N*L entries.
__global__ void __launch_bounds__(TS_THREADS)
trace_kernel(const double* __restrict__ W, const double* __restrict__ R, long long count,
             double2* __restrict__ part) {
  __shared__ double red[3][TS_THREADS];
  Cx<double> wr = czero<double>();
  double ww = 0.0;
  const long long per_block = (long long)CH * WD_LMAX;
  const long long nchunks = (count + per_block - 1) / per_block;
  for (long long ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
    const long long e0 = ck * per_block;
    const long long e1 = min(count, e0 + per_block);
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const Cx<double> w = ld2(W, e), r = ld2(R, e);
      wr = cfmaj(w, r, wr);
      ww += cnorm2(w);
    }
  }
  red[0][threadIdx.x] = wr.re;
  red[1][threadIdx.x] = wr.im;
  red[2][threadIdx.x] = ww;
  __syncthreads();
  for (int off = TS_THREADS / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double2* p = part + (size_t)blockIdx.x * PART_STRIDE;
    p[0] = make_double2(red[0][0], red[1][0]);
    p[1] = make_double2(red[2][0], 0.0);
  }
}

// Sum the per-block partials in block order.  which: GRAM_* target, -1 none; norms_out: where the
// column norms go (may be null); traces: finalize Tr[W^H R], Tr[W^H W] instead.
__global__ void finalize_kernel(const double2* __restrict__ part, int nblocks, int L,
                                SolverState* st, int which, double* norms_out, bool traces) {
  const int t = threadIdx.x;
  if (traces) {
    if (t < 2) {
      double2 s = make_double2(0.0, 0.0);
      for (int b = 0; b < nblocks; ++b) {
        const double2 v = part[(size_t)b * PART_STRIDE + t];
        s.x += v.x;
        s.y += v.y;
      }
      if (t == 0) st->trwr = s; else st->trww = s.x;
    }
    return;
  }
  if (which >= 0 && t < L * L) {
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < nblocks; ++b) {
      const double2 v = part[(size_t)b * PART_STRIDE + t];
      s.x += v.x;
      s.y += v.y;
    }
    double2* dst = which == GRAM_RTR ? st->rtr : which == GRAM_RTR_NEW ? st->rtr_new : st->rtv;
    dst[t] = s;
  }
  if (norms_out && t < L) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * PART_STRIDE + WD_LMAX * WD_LMAX + t].x;
    norms_out[t] = s;
  }
}

// ---------------------------------------------------------------- L x L solves (one warp)
// Solves C Z = Rhs in place: M is the augmented L x 2L matrix [C | Rhs] in shared memory,
// row-major with leading dimension 2*WD_LMAX.  Partial pivoting by the largest modulus.  Returns
// true when the system is singular in the sense of the oracle: a pivot that is not finite or whose
// modulus is below 1e-13 times the largest pivot modulus.
constexpr double PIVOT_RTOL = 1e-13;
constexpr int LD = 2 * WD_LMAX;

__device__ bool lu_solve_warp(Cx<double>* M, int L) {
  const int lane = threadIdx.x;
  double pmax = 0.0, pmin = 1e308;
  bool bad = false;
  for (int k = 0; k < L; ++k) {
    int p = k;
    double best = cnorm2(M[k * LD + k]);
    for (int i = k + 1; i < L; ++i) {
      const double v = cnorm2(M[i * LD + k]);
      if (v > best) { best = v; p = i; }
    }
    __syncwarp();
    if (p != k && lane < 2 * L) {
      const Cx<double> tmp = M[k * LD + lane];
      M[k * LD + lane] = M[p * LD + lane];
      M[p * LD + lane] = tmp;
    }
    __syncwarp();
    const Cx<double> piv = M[k * LD + k];
    const double pa = sqrt(cnorm2(piv));
    if (!isfinite(pa) || pa == 0.0) bad = true;
    pmax = fmax(pmax, pa);
    pmin = fmin(pmin, pa);
    const double pn = cnorm2(piv);
    const Cx<double> rp = cmake(piv.re / pn, -piv.im / pn);
    for (int i = k + 1; i < L; ++i) {
      const Cx<double> f = cmul(M[i * LD + k], rp);
      __syncwarp();
      if (lane > k && lane < 2 * L) M[i * LD + lane] = M[i * LD + lane] - cmul(f, M[k * LD + lane]);
      if (lane == k) M[i * LD + k] = f;
      __syncwarp();
    }
  }
  if (!(pmin >= PIVOT_RTOL * pmax)) bad = true;
  // back substitution, one right-hand-side column per lane
  if (lane >= L && lane < 2 * L) {
    for (int i = L - 1; i >= 0; --i) {
      Cx<double> v = M[i * LD + lane];
      for (int jj = i + 1; jj < L; ++jj) v = v - cmul(M[i * LD + jj], M[jj * LD + lane]);
      const Cx<double> d = M[i * LD + i];
      const double dn = cnorm2(d);
      M[i * LD + lane] = cmul(v, cmake(d.re / dn, -d.im / dn));
    }
  }
  __syncwarp();
  return bad;
}

// alpha_k from (R~_0^H V_k) alpha_k = R~_0^H R_k, and zeta_k = Tr[W^H R] / Tr[W^H W].
__global__ void solve_alpha_kernel(SolverState* st, int L) {
  __shared__ Cx<double> M[WD_LMAX * LD];
  if (st->status != ST_OK) return;
  const int lane = threadIdx.x;
  for (int i = 0; i < L; ++i)
    if (lane < L) {
      M[i * LD + lane] = sm(st->rtv[i * L + lane]);
      M[i * LD + L + lane] = sm(st->rtr[i * L + lane]);
    }
  __syncwarp();
  const bool bad = lu_solve_warp(M, L);
  if (lane < L)
    for (int i = 0; i < L; ++i) st->alpha[i * L + lane] = bad ? make_double2(0, 0) : d2(M[i * LD + L + lane]);
  if (lane == 0) {
    const double ww = st->trww;
    const Cx<double> wr = sm(st->trwr);
    Cx<double> z = cmake(wr.re / ww, wr.im / ww);
    bool zbad = !(ww > 0.0) || !isfinite(z.re) || !isfinite(z.im);
    st->zeta = zbad ? make_double2(0, 0) : d2(z);
    if (bad) st->status = ST_ALPHA_SINGULAR;
    else if (zbad) st->status = ST_ZETA_BAD;
  }
}

// gamma_k from (R~_0^H R_k) gamma_k = R~_0^H R_{k+1} / zeta_k; then R~_0^H R_k <- R~_0^H R_{k+1}.
__global__ void solve_gamma_kernel(SolverState* st, int L) {
  __shared__ Cx<double> M[WD_LMAX * LD];
  if (st->status != ST_OK) return;
  const int lane = threadIdx.x;
  const Cx<double> z = sm(st->zeta);
  const double zn = cnorm2(z);
  const Cx<double> rz = cmake(z.re / zn, -z.im / zn);
  for (int i = 0; i < L; ++i)
    if (lane < L) {
      M[i * LD + lane] = sm(st->rtr[i * L + lane]);
      M[i * LD + L + lane] = cmul(sm(st->rtr_new[i * L + lane]), rz);
    }
  __syncwarp();
  const bool bad = lu_solve_warp(M, L);
  if (lane < L)
    for (int i = 0; i < L; ++i) {
      st->gamma[i * L + lane] = bad ? make_double2(0, 0) : d2(M[i * LD + L + lane]);
      st->rtr[i * L + lane] = st->rtr_new[i * L + lane];
    }
  if (lane == 0 && bad) st->status = ST_GAMMA_SINGULAR;
}

// ---------------------------------------------------------------- block updates
// U = (P - zeta V) alpha  (S_k of the algorithm box is never stored).
__global__ void __launch_bounds__(TS_THREADS)
update_u_kernel(const double* __restrict__ P, const double* __restrict__ V, double* __restrict__ U,
                int L, long long rows, const SolverState* __restrict__ st) {
  __shared__ double2 Ss[CHE];
  __shared__ double2 al[WD_LMAX * WD_LMAX];
  if (st->status != ST_OK) return;
  const Cx<double> z = sm(st->zeta);
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) al[e] = st->alpha[e];
  const long long nchunks = (rows + CH - 1) / CH;
  for (long long ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
    const long long r0 = ck * CH;
    const int nr = (int)min((long long)CH, rows - r0);
    const int cnt = nr * L;
    const size_t e0 = (size_t)r0 * L;
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += blockDim.x)
      Ss[e] = d2(ld2(P, e0 + e) - cmul(z, ld2(V, e0 + e)));
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int n = e / L, b = e - (e / L) * L;
      Cx<double> acc = czero<double>();
      for (int a = 0; a < L; ++a) acc = cfma(sm(Ss[n * L + a]), sm(al[a * L + b]), acc);
      st2(U, e0 + e, acc);
    }
  }
}

// X += zeta F + G;  R -= zeta W + Y;  partial R~_0^H R_{k+1} and ||r_i||^2.
__global__ void __launch_bounds__(TS_THREADS)
update_xr_kernel(double* __restrict__ X, const double* __restrict__ F, const double* __restrict__ G,
                 double* __restrict__ R, const double* __restrict__ W, const double* __restrict__ Y,
                 const double* __restrict__ Rt, int L, long long rows, double2* __restrict__ part,
                 const SolverState* __restrict__ st) {
  __shared__ double2 As[CHE], Bs[CHE];
  if (st->status != ST_OK) return;
  const Cx<double> z = sm(st->zeta);
  Cx<double> acc = czero<double>();
  double nacc = 0.0;
  const long long nchunks = (rows + CH - 1) / CH;
  for (long long ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
    const long long r0 = ck * CH;
    const int nr = (int)min((long long)CH, rows - r0);
    const int cnt = nr * L;
    const size_t e0 = (size_t)r0 * L;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const size_t q = e0 + e;
      const Cx<double> x = ld2(X, q) + cmul(z, ld2(F, q)) + ld2(G, q);
      const Cx<double> r = ld2(R, q) - cmul(z, ld2(W, q)) - ld2(Y, q);
      st2(X, q, x);
      st2(R, q, r);
      Bs[e] = d2(r);
      As[e] = d2(ld2(Rt, q));
    }
    __syncthreads();
    gram_chunk(As, Bs, nr, L, acc, nacc, true);
    __syncthreads();
  }
  write_partial(part, L, acc, nacc, true);
}

// P = R + U gamma;  V = W + Y gamma;  partial R~_0^H V_{k+1}.
__global__ void __launch_bounds__(TS_THREADS)
update_pv_kernel(double* __restrict__ P, double* __restrict__ V, const double* __restrict__ R,
                 const double* __restrict__ W, const double* __restrict__ U,
                 const double* __restrict__ Y, const double* __restrict__ Rt, int L, long long rows,
                 double2* __restrict__ part, const SolverState* __restrict__ st) {
  __shared__ double2 Us[CHE], Ys[CHE], Vs[CHE], Rs[CHE];
  __shared__ double2 ga[WD_LMAX * WD_LMAX];
  if (st->status != ST_OK) return;
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) ga[e] = st->gamma[e];
  Cx<double> acc = czero<double>();
  double nacc = 0.0;
  const long long nchunks = (rows + CH - 1) / CH;
  for (long long ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
    const long long r0 = ck * CH;
    const int nr = (int)min((long long)CH, rows - r0);
    const int cnt = nr * L;
    const size_t e0 = (size_t)r0 * L;
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      Us[e] = d2(ld2(U, e0 + e));
      Ys[e] = d2(ld2(Y, e0 + e));
      Rs[e] = d2(ld2(Rt, e0 + e));
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int n = e / L, b = e - (e / L) * L;
      Cx<double> pu = czero<double>(), py = czero<double>();
      for (int a = 0; a < L; ++a) {
        const Cx<double> gm = sm(ga[a * L + b]);
        pu = cfma(sm(Us[n * L + a]), gm, pu);
        py = cfma(sm(Ys[n * L + a]), gm, py);
      }
      const size_t q = e0 + e;
      st2(P, q, ld2(R, q) + pu);
      const Cx<double> v = ld2(W, q) + py;
      st2(V, q, v);
      Vs[e] = d2(v);
    }
    __syncthreads();
    gram_chunk(Rs, Vs, nr, L, acc, nacc, false);
  }
  write_partial(part, L, acc, nacc, false);
}

// ---------------------------------------------------------------- double-float variants
// The same three updates with every product of an N x L block by an L x L matrix, and the Gram
// products, in double-float arithmetic (FP32 pairs, ~48 bits) on the FP32 pipes, packed two lanes
// per instruction: the (re, im) halves of a block element share one FP32x2 value, and the factor
// from the L x L matrix (or the other Gram operand) enters both lanes.  The X and R updates and the
// column norms stay FP64: X and R are updated with the F, G whose products with A are subtracted
// from R, so R = B - AX holds to FP64 rounding whatever precision the directions U, P, V and the
// coefficients alpha, gamma are computed in.  Block elements convert through the bit-field forms
// (no FP64 pipe); the L x L coefficients, a few hundred per launch, through the rounding ones.
WD_DEV CDF cdf_of(double2 v) { return cdf_from(Cx<double>{v.x, v.y}); }
WD_DEV P2 ldp2(const double* p, size_t e) { return p2_split(reinterpret_cast<const double2*>(p)[e]); }
// acc + g b for a double-float complex coefficient g: X and Y of the product sum (see pcombine).
WD_DEV void pmac_coef(P2& X, P2& Y, const CDF& g, P2 b, float2 m1) {
  pmac_dd(X, dup(g.re.hi), dup(-g.re.hi), dup(g.re.lo), b, m1);
  pmac_dd(Y, dup(g.im.hi), dup(-g.im.hi), dup(g.im.lo), b, m1);
}

__global__ void __launch_bounds__(TS_THREADS)
update_u_df_kernel(const double* __restrict__ P, const double* __restrict__ V, double* __restrict__ U,
                   int L, long long rows, const SolverState* __restrict__ st) {
  __shared__ P2 Ss[CHU * WD_LMAX];
  __shared__ CDF al[WD_LMAX * WD_LMAX];
  if (st->status != ST_OK) return;
  const float2 m1 = make_float2(-1.f, -1.f);
  const CDF z = cdf_of(st->zeta);
  // -zeta v = (-z.re) (v.re, v.im) + (z.im, -z.im) (v.im, v.re)
  const float2 a1 = dup(-z.re.hi), na1 = dup(z.re.hi), a1lo = dup(-z.re.lo);
  const float2 a2 = make_float2(z.im.hi, -z.im.hi), na2 = make_float2(-z.im.hi, z.im.hi);
  const float2 a2lo = make_float2(z.im.lo, -z.im.lo);
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) al[e] = cdf_of(st->alpha[e]);
  const long long nchunks = (rows + CHU - 1) / CHU;
  // The next chunk's P and V are loaded into registers while the current one is computed (a
  // thread holds at most CHU * WD_LMAX / TS_THREADS = 4 elements of a chunk).
  double2 pn[CHU * WD_LMAX / TS_THREADS], vn[CHU * WD_LMAX / TS_THREADS];
  auto fetch = [&](long long ck) {
    if (ck >= nchunks) return;
    const long long r0 = ck * CHU;
    const int cnt = (int)min((long long)CHU, rows - r0) * L;
    const size_t e0 = (size_t)r0 * L;
#pragma unroll
    for (int q = 0; q < CHU * WD_LMAX / TS_THREADS; ++q) {
      const int e = threadIdx.x + q * TS_THREADS;
      if (e < cnt) {
        pn[q] = reinterpret_cast<const double2*>(P)[e0 + e];
        vn[q] = reinterpret_cast<const double2*>(V)[e0 + e];
      }
    }
  };
  fetch(blockIdx.x);
  for (long long ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
    const long long r0 = ck * CHU;
    const int nr = (int)min((long long)CHU, rows - r0);
    const int cnt = nr * L;
    const size_t e0 = (size_t)r0 * L;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < CHU * WD_LMAX / TS_THREADS; ++q) {
      const int e = threadIdx.x + q * TS_THREADS;
      if (e < cnt) {
        P2 sv = p2_split(pn[q]);
        const P2 v = p2_split(vn[q]);
        pmac_dd(sv, a1, na1, a1lo, v, m1);          // P - zeta V
        pmac_dd(sv, a2, na2, a2lo, pswap(v), m1);
        Ss[e] = sv;
      }
    }
    fetch(ck + gridDim.x);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int n = e / L, b = e - (e / L) * L;
      P2 X = pzero(), Y = pzero();
      for (int a = 0; a < L; ++a) pmac_coef(X, Y, al[a * L + b], Ss[n * L + a], m1);
      reinterpret_cast<double2*>(U)[e0 + e] = p2_join(pcombine(X, Y, m1));
    }
  }
}

// t + z f with two FMAs per real part (the FP64 pipe is this kernel's bound).
WD_DEV Cx<double> xr_step(Cx<double> t, Cx<double> z, Cx<double> f) {
  return {fma(-z.im, f.im, fma(z.re, f.re, t.re)), fma(z.im, f.re, fma(z.re, f.im, t.im))};
}

// Gram entry (a, b) of a chunk: sum_n conj(A[n, a]) B[n, b] into X, Y (see pcombine_conj).  Long
// sums (thousands of rows per block): both accumulators are renormalised after every product, so
// their low words never outgrow ulp(hi) and keep ~48-bit accuracy.
WD_DEV void gram_chunk_p2(const P2* As, const P2* Bs, int rows, int L, P2& X, P2& Y, float2 m1) {
  const int t = threadIdx.x;
  if (t < L * L) {
    const int a = t / L, b = t - (t / L) * L;
    for (int n = 0; n < rows; ++n) {
      const P2 x = As[n * L + a];
      const P2 y = Bs[n * L + b];
      pmac_dd(X, dup(x.hi.x), dup(-x.hi.x), dup(x.lo.x), y, m1);
      pmac_dd(Y, dup(x.hi.y), dup(-x.hi.y), dup(x.lo.y), y, m1);
      X = pnorm(X, m1);
      Y = pnorm(Y, m1);
    }
  }
}

__global__ void __launch_bounds__(TS_THREADS)
update_xr_df_kernel(double* __restrict__ X, const double* __restrict__ F, const double* __restrict__ G,
                    double* __restrict__ R, const double* __restrict__ W, const double* __restrict__ Y,
                    const double* __restrict__ Rt, int L, long long rows, double2* __restrict__ part,
                    const SolverState* __restrict__ st) {
  __shared__ P2 As[CHE], Bs[CHE];
  __shared__ double nred[CHE];
  if (st->status != ST_OK) return;
  const float2 m1 = make_float2(-1.f, -1.f);
  const Cx<double> z = sm(st->zeta), mz = -z;
  P2 gx = pzero(), gy = pzero();
  double nacc = 0.0;
  const long long nchunks = (rows + CH - 1) / CH;
  for (long long ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
    const long long r0 = ck * CH;
    const int nr = (int)min((long long)CH, rows - r0);
    const int cnt = nr * L;
    const size_t e0 = (size_t)r0 * L;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const size_t q = e0 + e;
      const Cx<double> x = xr_step(ld2(X, q) + ld2(G, q), z, ld2(F, q));
      const Cx<double> r = xr_step(ld2(R, q) - ld2(Y, q), mz, ld2(W, q));
      st2(X, q, x);
      st2(R, q, r);
      Bs[e] = p2_split(make_double2(r.re, r.im));
      As[e] = ldp2(Rt, q);
      nred[e] = cnorm2(r);
    }
    __syncthreads();
    gram_chunk_p2(As, Bs, nr, L, gx, gy, m1);
    if (threadIdx.x < L)
      for (int n = 0; n < nr; ++n) nacc += nred[n * L + threadIdx.x];
    __syncthreads();
  }
  double2* p = part + (size_t)blockIdx.x * PART_STRIDE;
  if (threadIdx.x < L * L) p[threadIdx.x] = p2_join(pcombine_conj(gx, gy, m1));
  if (threadIdx.x < L) p[WD_LMAX * WD_LMAX + threadIdx.x] = make_double2(nacc, 0.0);
}

__global__ void __launch_bounds__(TS_THREADS)
update_pv_df_kernel(double* __restrict__ P, double* __restrict__ V, const double* __restrict__ R,
                    const double* __restrict__ W, const double* __restrict__ U,
                    const double* __restrict__ Y, const double* __restrict__ Rt, int L,
                    long long rows, double2* __restrict__ part, const SolverState* __restrict__ st) {
  __shared__ P2 Us[CHE], Ys[CHE], Vs[CHE], Rs[CHE];
  __shared__ CDF ga[WD_LMAX * WD_LMAX];
  if (st->status != ST_OK) return;
  const float2 m1 = make_float2(-1.f, -1.f);
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) ga[e] = cdf_of(st->gamma[e]);
  P2 gx = pzero(), gy = pzero();
  const long long nchunks = (rows + CH - 1) / CH;
  for (long long ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
    const long long r0 = ck * CH;
    const int nr = (int)min((long long)CH, rows - r0);
    const int cnt = nr * L;
    const size_t e0 = (size_t)r0 * L;
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      Us[e] = ldp2(U, e0 + e);
      Ys[e] = ldp2(Y, e0 + e);
      Rs[e] = ldp2(Rt, e0 + e);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int n = e / L, b = e - (e / L) * L;
      P2 ux = pzero(), uy = pzero(), yx = pzero(), yy = pzero();
      for (int a = 0; a < L; ++a) {
        const CDF& g = ga[a * L + b];
        pmac_coef(ux, uy, g, Us[n * L + a], m1);
        pmac_coef(yx, yy, g, Ys[n * L + a], m1);
      }
      const size_t q = e0 + e;
      const double2 pd = p2_join(pcombine(ux, uy, m1)), yd = p2_join(pcombine(yx, yy, m1));
      const Cx<double> pv = ld2(R, q) + Cx<double>{pd.x, pd.y};
      const Cx<double> v = ld2(W, q) + Cx<double>{yd.x, yd.y};
      st2(P, q, pv);
      st2(V, q, v);
      Vs[e] = p2_split(make_double2(v.re, v.im));
    }
    __syncthreads();
    gram_chunk_p2(Rs, Vs, nr, L, gx, gy, m1);
  }
  double2* p = part + (size_t)blockIdx.x * PART_STRIDE;
  if (threadIdx.x < L * L) p[threadIdx.x] = p2_join(pcombine_conj(gx, gy, m1));
}

// Four blocks of TS_THREADS per SM, for the current device (its SM count is read once per device).
constexpr int MAX_DEVICES = 64;
int g_sm_count[MAX_DEVICES] = {};

int max_blocks() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    cudaGetLastError();
    return 4 * 152;
  }
  if (!g_sm_count[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 152;
    }
    g_sm_count[dev] = n;
  }
  return 4 * g_sm_count[dev];
}

inline int blocks_for(long long rows) {
  const long long nchunks = (rows + CH - 1) / CH;
  const long long cap = max_blocks();
  return (int)(nchunks < cap ? (nchunks > 0 ? nchunks : 1) : cap);
}

}  // namespace

int ts_blocks(long long rows) { return blocks_for(rows); }
int ts_max_blocks() { return max_blocks(); }

cudaError_t launch_gram(const double* A, const double* B, int L, long long rows, double2* part,
                        SolverState* st, int which, bool norms_of_b, cudaStream_t s) {
  const int nb = blocks_for(rows);
  gram_kernel<<<nb, TS_THREADS, 0, s>>>(A, B, L, rows, part, norms_of_b);
  finalize_kernel<<<1, WD_LMAX * WD_LMAX, 0, s>>>(part, nb, L, st, which,
                                                  norms_of_b ? st->rnorm2 : nullptr, false);
  return cudaGetLastError();
}

cudaError_t launch_colnorms(const double* A, int L, long long rows, double2* part,
                            double* out_norm2, cudaStream_t s) {
  const int nb = blocks_for(rows);
  colnorm_kernel<<<nb, TS_THREADS, 0, s>>>(A, L, rows, part);
  finalize_kernel<<<1, WD_LMAX * WD_LMAX, 0, s>>>(part, nb, L, nullptr, -1, out_norm2, false);
  return cudaGetLastError();
}

cudaError_t launch_traces(const double* W, const double* R, int L, long long rows,
                          double2* part, SolverState* st, cudaStream_t s) {
  const int nb = blocks_for(rows);
  trace_kernel<<<nb, TS_THREADS, 0, s>>>(W, R, rows * L, part);
  finalize_kernel<<<1, WD_LMAX * WD_LMAX, 0, s>>>(part, nb, L, st, -1, nullptr, true);
  return cudaGetLastError();
}

cudaError_t launch_solve_alpha(SolverState* st, int L, cudaStream_t s) {
  solve_alpha_kernel<<<1, 32, 0, s>>>(st, L);
  return cudaGetLastError();
}

cudaError_t launch_solve_gamma(SolverState* st, int L, cudaStream_t s) {
  solve_gamma_kernel<<<1, 32, 0, s>>>(st, L);
  return cudaGetLastError();
}

cudaError_t launch_update_u(const double* P, const double* V, double* U, int L, long long rows,
                            const SolverState* st, cudaStream_t s, bool df) {
  if (df)
    update_u_df_kernel<<<blocks_for((rows + 1) / 2), TS_THREADS, 0, s>>>(P, V, U, L, rows, st);
  else
    update_u_kernel<<<blocks_for(rows), TS_THREADS, 0, s>>>(P, V, U, L, rows, st);
  return cudaGetLastError();
}

cudaError_t launch_update_xr(double* X, const double* F, const double* G, double* R,
                             const double* W, const double* Y, const double* Rt, int L,
                             long long rows, double2* part, SolverState* st, cudaStream_t s,
                             bool df) {
  const int nb = blocks_for(rows);
  if (df)
    update_xr_df_kernel<<<nb, TS_THREADS, 0, s>>>(X, F, G, R, W, Y, Rt, L, rows, part, st);
  else
    update_xr_kernel<<<nb, TS_THREADS, 0, s>>>(X, F, G, R, W, Y, Rt, L, rows, part, st);
  finalize_kernel<<<1, WD_LMAX * WD_LMAX, 0, s>>>(part, nb, L, st, GRAM_RTR_NEW, st->rnorm2, false);
  return cudaGetLastError();
}

cudaError_t launch_update_pv(double* P, double* V, const double* R, const double* W,
                             const double* U, const double* Y, const double* Rt, int L,
                             long long rows, double2* part, SolverState* st, cudaStream_t s,
                             bool df) {
  const int nb = blocks_for(rows);
  if (df)
    update_pv_df_kernel<<<nb, TS_THREADS, 0, s>>>(P, V, R, W, U, Y, Rt, L, rows, part, st);
  else
    update_pv_kernel<<<nb, TS_THREADS, 0, s>>>(P, V, R, W, U, Y, Rt, L, rows, part, st);
  finalize_kernel<<<1, WD_LMAX * WD_LMAX, 0, s>>>(part, nb, L, st, GRAM_RTV, nullptr, false);
  return cudaGetLastError();
}
