// Helpers shared by the sweep kernels: per-mode forcing weights and the
// compile-time dispatch over the number R of separable forcing terms (the
// weights P_{r,J} live in registers, so R must be a template parameter).
#pragma once
#include "pe_internal.h"

// P[r] = prod_a axisF[R*off[a] + r*n_a + j_a]
template <int R, typename T>
__device__ inline void load_P(const Geom& g, int64_t J, const T* __restrict__ axisF, T* P) {
  int j[PE_MAX_D];
  unflatten(g, J, j);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    T v = axisF[(int64_t)R * g.off[0] + (int64_t)r * g.n[0] + j[0]];
#pragma unroll
    for (int a = 1; a < PE_MAX_D; ++a) if (a < g.d) v *= axisF[(int64_t)R * g.off[a] + (int64_t)r * g.n[a] + j[a]];
    P[r] = v;
  }
}

#define PE_R_CASE(X) \
  case X:            \
    return L<X>::run(args...);

template <template <int> class L, typename... Args>
pe_status dispatch_R(int R, Args... args) {
  switch (R) {
    PE_R_CASE(1) PE_R_CASE(2) PE_R_CASE(3) PE_R_CASE(4) PE_R_CASE(5) PE_R_CASE(6) PE_R_CASE(7) PE_R_CASE(8)
    PE_R_CASE(9) PE_R_CASE(10) PE_R_CASE(11) PE_R_CASE(12) PE_R_CASE(13) PE_R_CASE(14) PE_R_CASE(15)
    PE_R_CASE(16) PE_R_CASE(17) PE_R_CASE(18) PE_R_CASE(19) PE_R_CASE(20) PE_R_CASE(21) PE_R_CASE(22)
    PE_R_CASE(23) PE_R_CASE(24) PE_R_CASE(25) PE_R_CASE(26) PE_R_CASE(27) PE_R_CASE(28) PE_R_CASE(29)
    PE_R_CASE(30) PE_R_CASE(31) PE_R_CASE(32)
    default:
      return pe_fail(PE_EINVAL, "number of forcing terms must be in 1..32");
  }
}
