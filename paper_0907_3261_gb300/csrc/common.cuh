// Shared device helpers: complex arithmetic on (re, im) pairs, lattice geometry, launch checks.
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
