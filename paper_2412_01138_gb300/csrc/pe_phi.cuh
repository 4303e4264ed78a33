// Device evaluation of phi_1..phi_s and of the weights b_i of Eq. (3-12).
//
// b_i(z) = sum_m a_{im} m! phi_{m+1}(z) with a_{im} the monomial coefficients of
// the Lagrange basis polynomial l_i.  phi_s is summed as a Taylor series for
// |z| < 2 and the lower phi_j follow by the backward recurrence
// phi_j = z phi_{j+1} + 1/j! (stable there); for |z| >= 2, phi_1 = expm1(z)/z
// and phi_{j+1} = (phi_j - 1/j!)/z.
#pragma once
#include "pe_internal.h"

constexpr double inv_factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= (double)i;
  return 1.0 / f;
}

// 1/k! for k = 0..47 (one copy per translation unit, initialised at compile time)
static __constant__ double c_inv_fact[48] = {
    inv_factorial(0),  inv_factorial(1),  inv_factorial(2),  inv_factorial(3),  inv_factorial(4),
    inv_factorial(5),  inv_factorial(6),  inv_factorial(7),  inv_factorial(8),  inv_factorial(9),
    inv_factorial(10), inv_factorial(11), inv_factorial(12), inv_factorial(13), inv_factorial(14),
    inv_factorial(15), inv_factorial(16), inv_factorial(17), inv_factorial(18), inv_factorial(19),
    inv_factorial(20), inv_factorial(21), inv_factorial(22), inv_factorial(23), inv_factorial(24),
    inv_factorial(25), inv_factorial(26), inv_factorial(27), inv_factorial(28), inv_factorial(29),
    inv_factorial(30), inv_factorial(31), inv_factorial(32), inv_factorial(33), inv_factorial(34),
    inv_factorial(35), inv_factorial(36), inv_factorial(37), inv_factorial(38), inv_factorial(39),
    inv_factorial(40), inv_factorial(41), inv_factorial(42), inv_factorial(43), inv_factorial(44),
    inv_factorial(45), inv_factorial(46), inv_factorial(47)};

// phi_1..phi_s at z into ph[0..s-1].
__device__ inline void phi_all(double z, int s, double* ph) {
  if (fabs(z) < 2.0) {
    const int K = 27;
    double acc = c_inv_fact[K + s];
    for (int k = K - 1; k >= 0; --k) acc = fma(acc, z, c_inv_fact[k + s]);
    ph[s - 1] = acc;
    for (int j = s - 1; j >= 1; --j) ph[j - 1] = fma(z, ph[j], c_inv_fact[j]);
  } else {
    ph[0] = expm1(z) / z;
    for (int j = 1; j < s; ++j) ph[j] = (ph[j - 1] - c_inv_fact[j]) / z;
  }
}

struct Lag {
  double a[PE_MAX_S][PE_MAX_S];  // a[i][m]: coefficient of theta^m in l_i
};

__device__ inline void b_weights(double z, int s, const Lag& L, double* b) {
  double ph[PE_MAX_S];
  phi_all(z, s, ph);
  for (int i = 0; i < s; ++i) {
    double acc = 0.0;
    double mf = 1.0;  // m!
    for (int m = 0; m < s; ++m) {
      acc = fma(L.a[i][m] * mf, ph[m], acc);
      mf *= (double)(m + 1);
    }
    b[i] = acc;
  }
}

