// Spin algebra shared by the stencil kernels: the chiral-basis projector blocks of the hopping
// term and the packed Hermitian 6x6 site blocks of A_D and A_D^{-1}.
#pragma once

#include "common.cuh"

// G_mu d for the lower 2-spinor d = (d0, d1), one colour component.
template <int MU, typename T>
WD_DEV void gamma_down(Cx<T> d0, Cx<T> d1, Cx<T>& g0, Cx<T>& g1) {
  if constexpr (MU == 0) { g0 = tmi(d1); g1 = tmi(d0); }
  else if constexpr (MU == 1) { g0 = -d1; g1 = d0; }
  else if constexpr (MU == 2) { g0 = tmi(d0); g1 = ti(d1); }
  else { g0 = d0; g1 = d1; }
}
// G_mu^H w.
template <int MU, typename T>
WD_DEV void gamma_up(Cx<T> w0, Cx<T> w1, Cx<T>& g0, Cx<T>& g1) {
  if constexpr (MU == 0) { g0 = ti(w1); g1 = ti(w0); }
  else if constexpr (MU == 1) { g0 = w1; g1 = -w0; }
  else if constexpr (MU == 2) { g0 = ti(w0); g1 = tmi(w1); }
  else { g0 = w0; g1 = w1; }
}

// Packed Hermitian 6x6 times a vector, block entries `stride` apart (component-major storage).
template <typename T>
WD_DEV void herm6s(const T* __restrict__ m, size_t stride, const Cx<T> v[6], Cx<T> out[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) out[i] = __ldg(m + i * stride) * v[i];
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      const int t = tri_index(i, j);
      const Cx<T> l = cmake<T>(__ldg(m + t * stride), __ldg(m + (t + 1) * stride));
      out[i] = cfma(l, v[j], out[i]);
      out[j] = cfmaj(l, v[i], out[j]);
    }
}
