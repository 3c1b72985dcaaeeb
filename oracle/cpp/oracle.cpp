// Plain FP64 C++ oracle of the preconditioned block BiCGGR solve -- TEST INFRASTRUCTURE ONLY.
//
// Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg and reference arm load this
// library.  It shares no code with the CUDA path and none with the numpy oracle: it is a second,
// independent statement of the same definitions, written for speed on host cores (OpenMP over
// sites) so that the CPU baseline can be a measured solve rather than a model.
//
//   * The operator of Eq. (1) (Sec. 2), in the conventions the paper leaves to its Ref.
//     [blockbicggr_app] (kappa normalisation, chiral gamma basis, four-leaf clover):
//       (A psi)(x) = A_D(x) psi(x) - kappa sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu)
//                                                 + (1 + g_mu) U_mu(x-mu)^H psi(x-mu) ],
//       A_D(x) = 1 - kappa c_SW sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x)  (a full 12 x 12 block),
//       sigma_{mu nu} = (i/2)[g_mu, g_nu],  F = (Q - Q^H)/(8i),  Q the four plaquette leaves at x.
//     Full 4 x 4 spin matrices (no half-spinor projection); A_D^{-1} per site by Gauss-Jordan.
//   * The Jacobi preconditioner of Sec. 2 from G = 0: j sweeps G <- G + A_D^{-1}(U - A G).
//   * Block BiCGGR, the algorithm box of Sec. 2, with R~_0 = R_0 and X_0 from the caller
//     (Sec. 3.3).  Readings where the paper is silent: the stopping test on R_0 and after every
//     R_{k+1} update (the order that reproduces Table 1's #MVM); L x L systems by LU with partial
//     pivoting, singular when a pivot is not finite or below 1e-13 times the largest; divergence
//     above 1e2; at exit the true residual, with restarts from X while it is above tol.
//
// Layouts: links [V][4][3][3] complex, blocks [V][4 spin][3 colour][L] complex (row n = spin*3 +
// colour of a site, column = right-hand side), site = x + Lx(y + Ly(z + Lz t)), periodic.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cd = std::complex<double>;
const cd I1(0.0, 1.0);

struct Lattice {
  int d[4];
  long V;
  std::vector<long> fwd[4], bwd[4];
  explicit Lattice(const int* dims) {
    V = 1;
    for (int m = 0; m < 4; ++m) { d[m] = dims[m]; V *= dims[m]; }
    for (int m = 0; m < 4; ++m) { fwd[m].resize(V); bwd[m].resize(V); }
    for (long s = 0; s < V; ++s) {
      long c[4] = {s % d[0], (s / d[0]) % d[1], (s / ((long)d[0] * d[1])) % d[2],
                   s / ((long)d[0] * d[1] * d[2])};
      for (int m = 0; m < 4; ++m) {
        long cf[4] = {c[0], c[1], c[2], c[3]}, cb[4] = {c[0], c[1], c[2], c[3]};
        cf[m] = (c[m] + 1) % d[m];
        cb[m] = (c[m] - 1 + d[m]) % d[m];
        fwd[m][s] = cf[0] + d[0] * (cf[1] + (long)d[1] * (cf[2] + (long)d[2] * cf[3]));
        bwd[m][s] = cb[0] + d[0] * (cb[1] + (long)d[1] * (cb[2] + (long)d[2] * cb[3]));
      }
    }
  }
};

using M3 = cd[3][3];
using M4 = cd[4][4];

// Euclidean gamma matrices of the chiral basis: g_k = [[0, -i s_k], [i s_k, 0]] (k = x, y, z),
// g_t = [[0, 1], [1, 0]].
void gammas(M4 g[4]) {
  const cd s[3][2][2] = {{{0.0, 1.0}, {1.0, 0.0}},
                         {{0.0, -I1}, {I1, 0.0}},
                         {{1.0, 0.0}, {0.0, -1.0}}};
  for (int m = 0; m < 4; ++m)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) g[m][a][b] = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        g[k][a][2 + b] = -I1 * s[k][a][b];
        g[k][2 + a][b] = I1 * s[k][a][b];
      }
  for (int a = 0; a < 2; ++a) { g[3][a][2 + a] = 1.0; g[3][2 + a][a] = 1.0; }
}

void mul3(const M3 a, const M3 b, M3 out) {
  M3 t;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cd acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += a[i][k] * b[k][j];
      t[i][j] = acc;
    }
  std::memcpy(out, t, sizeof(M3));
}
void dag3(const M3 a, M3 out) {
  M3 t;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) t[i][j] = std::conj(a[j][i]);
  std::memcpy(out, t, sizeof(M3));
}

struct Op {
  Lattice lat;
  double kappa, csw;
  std::vector<cd> U;       // [V][4][3][3]
  std::vector<cd> AD;      // [V][12][12]
  std::vector<cd> ADinv;   // [V][12][12]
  M4 g[4];
  bool singular = false;

  const cd* link(long s, int mu) const { return &U[((size_t)s * 4 + mu) * 9]; }

  Op(const double* links, const int* dims, double k, double c) : lat(dims), kappa(k), csw(c) {
    const long V = lat.V;
    U.assign(reinterpret_cast<const cd*>(links), reinterpret_cast<const cd*>(links) + V * 36);
    gammas(g);
    AD.assign((size_t)V * 144, 0.0);
    ADinv.assign((size_t)V * 144, 0.0);
    // sigma_{mu nu} = (i/2)[g_mu, g_nu]
    M4 sig[4][4];
    for (int m = 0; m < 4; ++m)
      for (int n = 0; n < 4; ++n)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            cd c1 = 0.0;
            for (int e = 0; e < 4; ++e) c1 += g[m][a][e] * g[n][e][b] - g[n][a][e] * g[m][e][b];
            sig[m][n][a][b] = 0.5 * I1 * c1;
          }
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long s = 0; s < V; ++s) {
      cd* ad = &AD[(size_t)s * 144];
      for (int i = 0; i < 12; ++i) ad[i * 12 + i] = 1.0;
      for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu) {
          M3 F;
          field_strength(s, mu, nu, F);
          for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
              for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                  ad[(a * 3 + i) * 12 + b * 3 + j] -= kappa * csw * sig[mu][nu][a][b] * F[i][j];
        }
      if (!invert12(ad, &ADinv[(size_t)s * 144])) bad |= 1;
    }
    singular = bad != 0;
  }

  // F_{mu nu}(s) = (Q - Q^H) / (8i) with Q the sum of the four counter-clockwise leaves at s.
  void field_strength(long s, int mu, int nu, M3 F) const {
    const long xpm = lat.fwd[mu][s], xpn = lat.fwd[nu][s];
    const long xmm = lat.bwd[mu][s], xmn = lat.bwd[nu][s];
    const long xmm_pn = lat.fwd[nu][xmm], xmm_mn = lat.bwd[nu][xmm], xmn_pm = lat.fwd[mu][xmn];
    auto L = [&](long site, int d, M3 out) { std::memcpy(out, link(site, d), sizeof(M3)); };
    M3 a, b, c, d, t, Q;
    // x -> x+mu -> x+mu+nu -> x+nu -> x
    L(s, mu, a); L(xpm, nu, b); L(xpn, mu, c); dag3(c, c); L(s, nu, d); dag3(d, d);
    mul3(a, b, t); mul3(t, c, t); mul3(t, d, Q);
    // x -> x+nu -> x+nu-mu -> x-mu -> x
    L(s, nu, a); L(xmm_pn, mu, b); dag3(b, b); L(xmm, nu, c); dag3(c, c); L(xmm, mu, d);
    mul3(a, b, t); mul3(t, c, t); mul3(t, d, t);
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) Q[i][j] += t[i][j];
    // x -> x-mu -> x-mu-nu -> x-nu -> x
    L(xmm, mu, a); dag3(a, a); L(xmm_mn, nu, b); dag3(b, b); L(xmm_mn, mu, c); L(xmn, nu, d);
    mul3(a, b, t); mul3(t, c, t); mul3(t, d, t);
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) Q[i][j] += t[i][j];
    // x -> x-nu -> x-nu+mu -> x+mu -> x
    L(xmn, nu, a); dag3(a, a); L(xmn, mu, b); L(xmn_pm, nu, c); L(s, mu, d); dag3(d, d);
    mul3(a, b, t); mul3(t, c, t); mul3(t, d, t);
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) Q[i][j] += t[i][j];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) F[i][j] = (Q[i][j] - std::conj(Q[j][i])) / (8.0 * I1);
  }

  // Gauss-Jordan with partial pivoting on a 12 x 12 block; false if a pivot is tiny.
  static bool invert12(const cd* a_in, cd* inv) {
    cd a[12][12];
    for (int i = 0; i < 12; ++i)
      for (int j = 0; j < 12; ++j) { a[i][j] = a_in[i * 12 + j]; inv[i * 12 + j] = i == j ? 1.0 : 0.0; }
    for (int k = 0; k < 12; ++k) {
      int p = k;
      for (int i = k + 1; i < 12; ++i)
        if (std::abs(a[i][k]) > std::abs(a[p][k])) p = i;
      if (!(std::abs(a[p][k]) > 1e-14)) return false;
      if (p != k)
        for (int j = 0; j < 12; ++j) { std::swap(a[k][j], a[p][j]); std::swap(inv[k * 12 + j], inv[p * 12 + j]); }
      const cd r = 1.0 / a[k][k];
      for (int j = 0; j < 12; ++j) { a[k][j] *= r; inv[k * 12 + j] *= r; }
      for (int i = 0; i < 12; ++i) {
        if (i == k) continue;
        const cd f = a[i][k];
        if (f == 0.0) continue;
        for (int j = 0; j < 12; ++j) { a[i][j] -= f * a[k][j]; inv[i * 12 + j] -= f * inv[k * 12 + j]; }
      }
    }
    return true;
  }

  // y = A_D x (inverse = false) or A_D^{-1} x, site by site with the full 12 x 12 block.
  void site_diag(const cd* x, cd* y, int L, bool inverse) const {
    const std::vector<cd>& M = inverse ? ADinv : AD;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < lat.V; ++s) {
      const cd* m = &M[(size_t)s * 144];
      const cd* xs = x + (size_t)s * 12 * L;
      cd* ys = y + (size_t)s * 12 * L;
      for (int i = 0; i < 12; ++i)
        for (int l = 0; l < L; ++l) {
          cd acc = 0.0;
          for (int k = 0; k < 12; ++k) acc += m[i * 12 + k] * xs[k * L + l];
          ys[i * L + l] = acc;
        }
    }
  }

  // y = A x: the literal stencil with full 4 x 4 spin matrices (1 -+ g_mu).
  void apply(const cd* x, cd* y, int L) const {
    site_diag(x, y, L, false);
#pragma omp parallel
    {
    std::vector<cd> h(12 * (size_t)L), ux(12 * (size_t)L);
#pragma omp for schedule(static)
    for (long s = 0; s < lat.V; ++s) {
      std::fill(h.begin(), h.end(), cd(0.0));
      for (int mu = 0; mu < 4; ++mu)
        for (int dir = 0; dir < 2; ++dir) {
          const long n = dir == 0 ? lat.fwd[mu][s] : lat.bwd[mu][s];
          const cd* u = dir == 0 ? link(s, mu) : link(n, mu);
          const cd* xn = x + (size_t)n * 12 * L;
          // colour: U psi (forward) or U^H psi (backward), for every spin
          for (int sp = 0; sp < 4; ++sp)
            for (int a = 0; a < 3; ++a)
              for (int l = 0; l < L; ++l) {
                cd acc = 0.0;
                for (int b = 0; b < 3; ++b)
                  acc += (dir == 0 ? u[a * 3 + b] : std::conj(u[b * 3 + a])) * xn[(sp * 3 + b) * L + l];
                ux[(sp * 3 + a) * L + l] = acc;
              }
          // spin: (1 - g_mu) forward, (1 + g_mu) backward
          const double sg = dir == 0 ? -1.0 : 1.0;
          for (int sp = 0; sp < 4; ++sp)
            for (int t = 0; t < 4; ++t) {
              const cd p = (sp == t ? 1.0 : 0.0) + sg * g[mu][sp][t];
              if (p == 0.0) continue;
              for (int a = 0; a < 3; ++a)
                for (int l = 0; l < L; ++l) h[(sp * 3 + a) * L + l] += p * ux[(t * 3 + a) * L + l];
            }
        }
      cd* ys = y + (size_t)s * 12 * L;
      for (size_t e = 0; e < 12 * (size_t)L; ++e) ys[e] -= kappa * h[e];
    }
    }
  }
};

// ---- block operations on N x L blocks (row-major, N = 12 V).  Reductions give each thread a
// fixed, contiguous range of rows and add the threads' partial sums in thread order, so a result
// depends only on the thread count, not on scheduling.
int nthreads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
int thread_id() {
#ifdef _OPENMP
  return omp_get_thread_num();
#else
  return 0;
#endif
}

void herm(const cd* A, const cd* B, long N, int L, cd* out) {   // out = A^H B (L x L)
  const int nt = nthreads();
  std::vector<cd> part((size_t)nt * L * L, 0.0);
#pragma omp parallel num_threads(nt)
  {
    cd* loc = &part[(size_t)thread_id() * L * L];
#pragma omp for schedule(static)
    for (long n = 0; n < N; ++n)
      for (int a = 0; a < L; ++a) {
        const cd ca = std::conj(A[n * L + a]);
        for (int b = 0; b < L; ++b) loc[a * L + b] += ca * B[n * L + b];
      }
  }
  for (int e = 0; e < L * L; ++e) {
    cd acc = 0.0;
    for (int t = 0; t < nt; ++t) acc += part[(size_t)t * L * L + e];
    out[e] = acc;
  }
}
cd vdot(const cd* A, const cd* B, long n) {   // sum conj(A) B
  const int nt = nthreads();
  std::vector<cd> part(nt, 0.0);
#pragma omp parallel num_threads(nt)
  {
    cd acc = 0.0;
#pragma omp for schedule(static)
    for (long e = 0; e < n; ++e) acc += std::conj(A[e]) * B[e];
    part[thread_id()] = acc;
  }
  cd acc = 0.0;
  for (int t = 0; t < nt; ++t) acc += part[t];
  return acc;
}
void colnorms(const cd* A, long N, int L, double* out) {
  for (int l = 0; l < L; ++l) out[l] = 0.0;
  for (long n = 0; n < N; ++n)
    for (int l = 0; l < L; ++l) out[l] += std::norm(A[n * L + l]);
  for (int l = 0; l < L; ++l) out[l] = std::sqrt(out[l]);
}
void right_mul(const cd* X, const cd* C, long N, int L, cd* out) {   // out = X C
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; ++n)
    for (int b = 0; b < L; ++b) {
      cd acc = 0.0;
      for (int a = 0; a < L; ++a) acc += X[n * L + a] * C[a * L + b];
      out[n * L + b] = acc;
    }
}

// C Z = R (L x L) by LU with partial pivoting; false when singular (a pivot not finite or below
// 1e-13 times the largest).
bool solve_small(std::vector<cd> C, std::vector<cd> R, int L, cd* Z) {
  std::vector<int> piv(L);
  double pmax = 0.0, pmin = 1e308;
  for (int k = 0; k < L; ++k) {
    int p = k;
    for (int i = k + 1; i < L; ++i)
      if (std::abs(C[i * L + k]) > std::abs(C[p * L + k])) p = i;
    if (p != k)
      for (int j = 0; j < L; ++j) { std::swap(C[k * L + j], C[p * L + j]); std::swap(R[k * L + j], R[p * L + j]); }
    const double pa = std::abs(C[k * L + k]);
    if (!std::isfinite(pa) || pa == 0.0) return false;
    pmax = std::max(pmax, pa);
    pmin = std::min(pmin, pa);
    for (int i = k + 1; i < L; ++i) {
      const cd f = C[i * L + k] / C[k * L + k];
      for (int j = k; j < L; ++j) C[i * L + j] -= f * C[k * L + j];
      for (int j = 0; j < L; ++j) R[i * L + j] -= f * R[k * L + j];
    }
  }
  if (!(pmin >= 1e-13 * pmax)) return false;
  for (int col = 0; col < L; ++col)
    for (int i = L - 1; i >= 0; --i) {
      cd v = R[i * L + col];
      for (int j = i + 1; j < L; ++j) v -= C[i * L + j] * Z[j * L + col];
      Z[i * L + col] = v / C[i * L + i];
    }
  return true;
}

struct Counters {
  long long mvm = 0;
  std::vector<cd> T, D;   // work blocks of the Jacobi sweeps, kept between calls
};

void jacobi(const Op& op, const cd* U, cd* G, int L, int j, Counters& cnt) {
  const size_t n = (size_t)op.lat.V * 12 * L;
  if (j == 0) { std::memcpy(G, U, n * sizeof(cd)); return; }
  std::vector<cd>& T = cnt.T;
  std::vector<cd>& D = cnt.D;
  T.resize(n);
  D.resize(n);
  std::fill(G, G + n, cd(0.0));
  for (int it = 0; it < j; ++it) {
    op.apply(G, T.data(), L);                  // A G
#pragma omp parallel for schedule(static)
    for (long e = 0; e < (long)n; ++e) T[e] = U[e] - T[e];
    op.site_diag(T.data(), D.data(), L, true);   // A_D^{-1} (U - A G)
#pragma omp parallel for schedule(static)
    for (long e = 0; e < (long)n; ++e) G[e] += D[e];
    ++cnt.mvm;
  }
}

enum { OK = 0, NOT_CONVERGED = 4, DIVERGED = 5, BREAKDOWN = 6, RUNNING = -1 };

// The algorithm box of Sec. 2 as a state machine: start() computes R_0, P_0, R~_0 and, unless R_0
// already meets the tolerance, F_0 = M R_0 and V_0 = W_0 = A F_0; every step() is one outer
// iteration up to and including the stopping test after the R_{k+1} update and, if the run goes
// on, F_{k+1}, W_{k+1}, gamma_k, P_{k+1} and V_{k+1}.
struct BlockBiCGGR {
  const Op& op;
  int L, j;
  double eps;
  long N;
  size_t n;
  std::vector<cd> X, R, P, Rt, F, W, V, Uk, G, Y, S, T;
  std::vector<double> bn, rn, rec;
  std::vector<cd> rtv, rtr, rtr_new, alpha, gamma, rhs;
  Counters cnt;
  int k = 0;

  BlockBiCGGR(const Op& o, int L_, int j_, double eps_)
      : op(o), L(L_), j(j_), eps(eps_), N(o.lat.V * 12), n((size_t)o.lat.V * 12 * L_),
        bn(L_), rn(L_), rec(L_), rtv(L_ * L_), rtr(L_ * L_), rtr_new(L_ * L_), alpha(L_ * L_),
        gamma(L_ * L_), rhs(L_ * L_) {
    for (auto* v : {&X, &R, &P, &Rt, &F, &W, &V, &Uk, &G, &Y, &S, &T}) v->resize(n);
  }

  double rel_max(const std::vector<cd>& Rv) {
    colnorms(Rv.data(), N, L, rn.data());
    double m = 0.0;
    for (int l = 0; l < L; ++l) {
      rec[l] = rn[l] / bn[l];
      if (!(rec[l] <= m)) m = rec[l];
    }
    return m;
  }

  int start(const cd* B, const cd* X0) {
    std::memcpy(X.data(), X0, n * sizeof(cd));
    colnorms(B, N, L, bn.data());
    k = 0;
    op.apply(X.data(), T.data(), L);
    ++cnt.mvm;
    for (size_t e = 0; e < n; ++e) R[e] = B[e] - T[e];            // R_0 = B - A X_0
    P = R;                                                        // P_0 = R_0
    Rt = R;                                                       // R~_0 = R_0
    if (rel_max(R) <= eps) return OK;
    jacobi(op, R.data(), F.data(), L, j, cnt);                    // F_0 = M R_0
    op.apply(F.data(), W.data(), L);                              // V_0 = W_0 = A F_0
    ++cnt.mvm;
    V = W;
    return RUNNING;
  }

  int step() {
    herm(Rt.data(), V.data(), N, L, rtv.data());
    herm(Rt.data(), R.data(), N, L, rtr.data());
    if (!solve_small(rtv, rtr, L, alpha.data())) return BREAKDOWN;   // alpha_k
    const cd ww = vdot(W.data(), W.data(), (long)n);
    if (ww == 0.0) return BREAKDOWN;
    const cd zeta = vdot(W.data(), R.data(), (long)n) / ww;       // zeta_k
    for (size_t e = 0; e < n; ++e) S[e] = P[e] - zeta * V[e];     // S_k = P_k - zeta_k V_k
    right_mul(S.data(), alpha.data(), N, L, Uk.data());           // U_k = S_k alpha_k
    jacobi(op, Uk.data(), G.data(), L, j, cnt);                   // G_k = M U_k
    op.apply(G.data(), Y.data(), L);                              // Y_k = A G_k
    ++cnt.mvm;
    for (size_t e = 0; e < n; ++e) {
      X[e] += zeta * F[e] + G[e];                                 // X_{k+1}
      T[e] = R[e] - zeta * W[e] - Y[e];                           // R_{k+1}
    }
    ++k;
    const double m = rel_max(T);
    if (!std::isfinite(m)) { R.swap(T); return BREAKDOWN; }
    if (m <= eps) { R.swap(T); return OK; }
    if (m > 1e2) { R.swap(T); return DIVERGED; }
    jacobi(op, T.data(), F.data(), L, j, cnt);                    // F_{k+1} = M R_{k+1}
    op.apply(F.data(), W.data(), L);                              // W_{k+1} = A F_{k+1}
    ++cnt.mvm;
    herm(Rt.data(), T.data(), N, L, rtr_new.data());
    for (int e = 0; e < L * L; ++e) rhs[e] = rtr_new[e] / zeta;
    if (!solve_small(rtr, rhs, L, gamma.data())) { R.swap(T); return BREAKDOWN; }   // gamma_k
    right_mul(Uk.data(), gamma.data(), N, L, S.data());
    for (size_t e = 0; e < n; ++e) P[e] = T[e] + S[e];            // P_{k+1} = R_{k+1} + U_k gamma_k
    right_mul(Y.data(), gamma.data(), N, L, S.data());
    for (size_t e = 0; e < n; ++e) V[e] = W[e] + S[e];            // V_{k+1} = W_{k+1} + Y_k gamma_k
    R.swap(T);
    return RUNNING;
  }

  // ||b_i - A x_i|| / ||b_i|| per column; the largest.
  double true_residual(const cd* B, double* out) {
    op.apply(X.data(), T.data(), L);
    for (size_t e = 0; e < n; ++e) T[e] = B[e] - T[e];
    std::vector<double> tn(L);
    colnorms(T.data(), N, L, tn.data());
    double mt = 0.0;
    for (int l = 0; l < L; ++l) {
      out[l] = tn[l] / bn[l];
      mt = std::max(mt, out[l]);
    }
    return mt;
  }
};

struct Handle {
  Op op;
  std::vector<cd> B;
  BlockBiCGGR* run = nullptr;
  int L = 0, status = RUNNING;
  Handle(const double* links, const int* dims, double k, double c) : op(links, dims, k, c) {}
  ~Handle() { delete run; }
};

}  // namespace

extern "C" {

int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

// y = A x (Eq. (1)); returns 6 if a site block is singular.
int oracle_apply(const double* links, const int* dims, double kappa, double csw, const double* x,
                 double* y, int L) {
  Op op(links, dims, kappa, csw);
  op.apply(reinterpret_cast<const cd*>(x), reinterpret_cast<cd*>(y), L);
  return op.singular ? BREAKDOWN : OK;
}

// y = A_D x (inverse 0) or A_D^{-1} x (inverse 1).
int oracle_site_diag(const double* links, const int* dims, double kappa, double csw,
                     const double* x, double* y, int L, int inverse) {
  Op op(links, dims, kappa, csw);
  op.site_diag(reinterpret_cast<const cd*>(x), reinterpret_cast<cd*>(y), L, inverse != 0);
  return op.singular ? BREAKDOWN : OK;
}

// G = M U, j Jacobi sweeps from G = 0 (Sec. 2).
int oracle_jacobi(const double* links, const int* dims, double kappa, double csw, const double* u,
                  double* g, int L, int j) {
  Op op(links, dims, kappa, csw);
  Counters c;
  jacobi(op, reinterpret_cast<const cd*>(u), reinterpret_cast<cd*>(g), L, j, c);
  return op.singular ? BREAKDOWN : OK;
}

// A stepwise solve: oracle_create builds the operator (clover, inverse blocks); oracle_start
// begins the algorithm box for B, X_0 (returns -1 while running, 0 if R_0 already converged);
// oracle_step runs one outer iteration (-1 while running, else the final status); oracle_result
// copies X and the per-column recursive and true residuals (NULL to skip) and returns
// (iterations, MVMs per column) through out[2].
void* oracle_create(const double* links, const int* dims, double kappa, double csw) {
  Handle* h = new Handle(links, dims, kappa, csw);
  if (h->op.singular) { delete h; return nullptr; }
  return h;
}
void oracle_destroy(void* p) { delete static_cast<Handle*>(p); }

int oracle_start(void* p, const double* B, const double* X0, int L, int j, double tol) {
  Handle* h = static_cast<Handle*>(p);
  delete h->run;
  h->L = L;
  h->B.assign(reinterpret_cast<const cd*>(B),
              reinterpret_cast<const cd*>(B) + (size_t)h->op.lat.V * 12 * L);
  h->run = new BlockBiCGGR(h->op, L, j, tol);
  h->status = h->run->start(h->B.data(), reinterpret_cast<const cd*>(X0));
  return h->status;
}

int oracle_step(void* p) {
  Handle* h = static_cast<Handle*>(p);
  if (!h->run || h->status != RUNNING) return h->status;
  h->status = h->run->step();
  return h->status;
}

void oracle_result(void* p, double* X, double* rec, double* true_resid, long long* out) {
  Handle* h = static_cast<Handle*>(p);
  if (!h->run) return;
  if (X) std::memcpy(X, h->run->X.data(), h->run->n * sizeof(cd));
  if (rec) std::memcpy(rec, h->run->rec.data(), h->L * sizeof(double));
  if (true_resid) h->run->true_residual(h->B.data(), true_resid);
  if (out) { out[0] = h->run->k; out[1] = h->run->cnt.mvm; }
}

// The whole solve with restarts from X while the true residual is above tol (at most
// max_restarts).  X holds X_0 on entry and the solution on exit.  out[3]: outer iterations,
// restarts, MVMs per column (a Jacobi sweep counts as one, as in Table 1); true_resid[L] or NULL.
int oracle_solve(const double* links, const int* dims, double kappa, double csw, const double* B,
                 double* X, int L, int j, double tol, int maxit, int max_restarts,
                 long long* out, double* true_resid) {
  Handle* h = static_cast<Handle*>(oracle_create(links, dims, kappa, csw));
  if (!h) return BREAKDOWN;
  int iters = 0, restarts = 0, status = OK;
  long long mvm = 0;
  std::vector<double> tr(L);
  for (;;) {
    status = oracle_start(h, B, X, L, j, tol);
    while (status == RUNNING && h->run->k + iters < maxit) status = oracle_step(h);
    if (status == RUNNING) status = NOT_CONVERGED;
    long long o[2];
    oracle_result(h, X, nullptr, tr.data(), o);
    iters += (int)o[0];
    mvm += o[1];
    double mt = 0.0;
    for (int l = 0; l < L; ++l) mt = std::max(mt, tr[l]);
    if (status != OK || mt <= tol || restarts >= max_restarts) {
      if (status == OK && mt > tol) status = NOT_CONVERGED;
      break;
    }
    ++restarts;
  }
  if (out) { out[0] = iters; out[1] = restarts; out[2] = mvm; }
  if (true_resid) std::memcpy(true_resid, tr.data(), L * sizeof(double));
  delete h;
  return status;
}

}  // extern "C"
