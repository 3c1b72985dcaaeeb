// Site-diagonal part A_D of the clover Wilson-Dirac matrix and its inverse, built once per set of
// links.  A_D is "the diagonal part of the coefficient matrix" of the Jacobi preconditioner
// (arXiv:0907.3261, Sec. 2), read as the site-block diagonal 1 + clover term, with c_SW of
// Sec. 3.1:
//   A_D = 1 - kappa c_SW sum_{mu<nu} sigma_{mu nu} F_{mu nu},
//   F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^H) / (8i),  Q = the four plaquette leaves at x.
// In the chiral basis sigma_{jk} = -e_jkl (s_l (+) s_l) and sigma_{jt} = s_j (+) (-s_j), so A_D is
// block diagonal with one 6x6 block per chirality:
//   A_D^(+/-) = 1 - kappa c_SW sum_l s_l (x) M_l,   M_l = +/-E_l - B_l,
//   B_1 = F_yz, B_2 = F_zx, B_3 = F_xy, E_l = F_lt,
// which, with s_1..s_3 written out, is the 2x2 arrangement of 3x3 colour blocks
//   [[1 - k M_3, -k (M_1 - i M_2)], [-k (M_1 + i M_2), 1 + k M_3]],   k = kappa c_SW.
// Each block and its inverse (Gauss-Jordan with partial pivoting, FP64) are stored packed.
#include "common.cuh"
#include "internal.h"

namespace {

struct M3 {
  Cx<double> m[3][3];
};

__device__ M3 load_link(const double* links, int s, int mu) {
  M3 r;
  const double* p = links + 18 * ((size_t)s * 4 + mu);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) r.m[a][b] = cmake(p[2 * (a * 3 + b)], p[2 * (a * 3 + b) + 1]);
  return r;
}
__device__ M3 mul(const M3& a, const M3& b) {
  M3 r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Cx<double> acc = czero<double>();
      for (int k = 0; k < 3; ++k) acc = cfma(a.m[i][k], b.m[k][j], acc);
      r.m[i][j] = acc;
    }
  return r;
}
__device__ M3 dag(const M3& a) {
  M3 r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = conj(a.m[j][i]);
  return r;
}
__device__ int shift(const Geom& g, int s, int mu, int dir) {
  int c[4];
  site_coords(g, s, c);
  return neighbour(g, s, c, mu, dir);
}

// F_{mu nu}(s) (Hermitian) from the four counter-clockwise leaves.
__device__ M3 field_strength(const double* links, const Geom& g, int s, int mu, int nu) {
  const int xpm = shift(g, s, mu, +1), xpn = shift(g, s, nu, +1);
  const int xmm = shift(g, s, mu, -1), xmn = shift(g, s, nu, -1);
  const int xmm_pn = shift(g, xmm, nu, +1), xmm_mn = shift(g, xmm, nu, -1);
  const int xmn_pm = shift(g, xmn, mu, +1);
  const M3 Um = load_link(links, s, mu), Un = load_link(links, s, nu);
  // x -> x+mu -> x+mu+nu -> x+nu -> x
  M3 q = mul(mul(Um, load_link(links, xpm, nu)), dag(mul(Un, load_link(links, xpn, mu))));
  // x -> x+nu -> x-mu+nu -> x-mu -> x
  M3 l2 = mul(mul(Un, dag(mul(load_link(links, xmm, nu), load_link(links, xmm_pn, mu)))),
              load_link(links, xmm, mu));
  // x -> x-mu -> x-mu-nu -> x-nu -> x
  M3 l3 = mul(dag(mul(load_link(links, xmm_mn, nu), load_link(links, xmm, mu))),
              mul(load_link(links, xmm_mn, mu), load_link(links, xmn, nu)));
  // x -> x-nu -> x-nu+mu -> x+mu -> x
  M3 l4 = mul(mul(dag(load_link(links, xmn, nu)), load_link(links, xmn, mu)),
              mul(load_link(links, xmn_pm, nu), dag(Um)));
  M3 f;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) q.m[i][j] = q.m[i][j] + l2.m[i][j] + l3.m[i][j] + l4.m[i][j];
  // (Q - Q^H) / (8i) = -i (Q - Q^H) / 8
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) f.m[i][j] = 0.125 * tmi(q.m[i][j] - conj(q.m[j][i]));
  return f;
}

// In-place inverse of a 6x6 complex matrix; returns false if a pivot is tiny or not finite.
__device__ bool invert6(Cx<double> a[6][6], Cx<double> inv[6][6]) {
  double scale = 0.0;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      inv[i][j] = cmake(i == j ? 1.0 : 0.0, 0.0);
      scale = fmax(scale, sqrt(cnorm2(a[i][j])));
    }
  bool ok = isfinite(scale) && scale > 0.0;
  for (int k = 0; k < 6; ++k) {
    int p = k;
    double best = cnorm2(a[k][k]);
    for (int i = k + 1; i < 6; ++i)
      if (cnorm2(a[i][k]) > best) { best = cnorm2(a[i][k]); p = i; }
    if (!(sqrt(best) > 1e-14 * scale)) ok = false;
    if (p != k)
      for (int j = 0; j < 6; ++j) {
        Cx<double> t = a[k][j]; a[k][j] = a[p][j]; a[p][j] = t;
        t = inv[k][j]; inv[k][j] = inv[p][j]; inv[p][j] = t;
      }
    const Cx<double> piv = a[k][k];
    const double pn = cnorm2(piv);
    const Cx<double> rp = cmake(piv.re / pn, -piv.im / pn);
    for (int j = 0; j < 6; ++j) { a[k][j] = cmul(a[k][j], rp); inv[k][j] = cmul(inv[k][j], rp); }
    for (int i = 0; i < 6; ++i) {
      if (i == k) continue;
      const Cx<double> f = a[i][k];
      for (int j = 0; j < 6; ++j) {
        a[i][j] = a[i][j] - cmul(f, a[k][j]);
        inv[i][j] = inv[i][j] - cmul(f, inv[k][j]);
      }
    }
  }
  return ok;
}

__device__ void pack_herm6(const Cx<double> m[6][6], double* out) {
  for (int i = 0; i < 6; ++i) out[i] = m[i][i].re;
  for (int i = 1; i < 6; ++i)
    for (int j = 0; j < i; ++j) {
      // Hermitian part of the lower entry: (m_ij + conj(m_ji)) / 2
      out[tri_index(i, j)] = 0.5 * (m[i][j].re + m[j][i].re);
      out[tri_index(i, j) + 1] = 0.5 * (m[i][j].im - m[j][i].im);
    }
}

__global__ void clover_build_kernel(const double* __restrict__ links, double* __restrict__ clov,
                                    double* __restrict__ clov_inv, Geom g, double kappa,
                                    double csw, int* singular) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  // F_{mu nu} for (x,y) (x,z) (x,t) (y,z) (y,t) (z,t)
  const M3 Fxy = field_strength(links, g, s, 0, 1);
  const M3 Fxz = field_strength(links, g, s, 0, 2);
  const M3 Fxt = field_strength(links, g, s, 0, 3);
  const M3 Fyz = field_strength(links, g, s, 1, 2);
  const M3 Fyt = field_strength(links, g, s, 1, 3);
  const M3 Fzt = field_strength(links, g, s, 2, 3);
  const double k = kappa * csw;
  for (int ch = 0; ch < 2; ++ch) {
    const double e = ch == 0 ? 1.0 : -1.0;
    Cx<double> blk[6][6], inv[6][6];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        // M_1 = e F_xt - F_yz, M_2 = e F_yt - F_zx = e F_yt + F_xz, M_3 = e F_zt - F_xy
        const Cx<double> m1 = e * Fxt.m[a][b] - Fyz.m[a][b];
        const Cx<double> m2 = e * Fyt.m[a][b] + Fxz.m[a][b];
        const Cx<double> m3 = e * Fzt.m[a][b] - Fxy.m[a][b];
        const double d = a == b ? 1.0 : 0.0;
        blk[a][b] = cmake(d, 0.0) - k * m3;
        blk[a + 3][b + 3] = cmake(d, 0.0) + k * m3;
        blk[a][b + 3] = -k * (m1 - ti(m2));
        blk[a + 3][b] = -k * (m1 + ti(m2));
      }
    double* out = clov + ((size_t)s * 2 + ch) * CLOV_REALS;
    pack_herm6(blk, out);
    if (!invert6(blk, inv)) atomicExch(singular, 1);
    double* oi = clov_inv + ((size_t)s * 2 + ch) * CLOV_REALS;
    pack_herm6(inv, oi);
  }
}

}  // namespace

cudaError_t launch_clover_build(const Op& op, int* singular_dev, cudaStream_t st) {
  const int threads = 64;
  clover_build_kernel<<<(op.g.V + threads - 1) / threads, threads, 0, st>>>(
      op.links, op.clov, op.clov_inv, op.g, op.kappa, op.csw, singular_dev);
  return cudaGetLastError();
}
