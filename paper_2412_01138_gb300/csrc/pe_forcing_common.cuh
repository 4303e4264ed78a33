// Descriptor evaluation shared by the forcing kernels: separable terms
// amp * time(t) * prod_a spatial_a(x_a) (kinds as in include/pe.h) and the
// Gauss-Legendre rule used for consistent loads.
#pragma once
#include <math.h>

#include "pe_internal.h"

// lk[r][a]: how the 1D "load" of term r along axis a is formed from its factor g:
// 0 consistent load int g phi_k (Gauss quadrature); for the Dirichlet lifting, from the
// factor's values at the full-grid nodes x_{k}, x_{k+1}, x_{k+2} around interior node k:
// 1 mass rows (h/6)(g_k + 4 g_{k+1} + g_{k+2}), 2 stiffness rows (1/h)(-g_k + 2 g_{k+1} - g_{k+2}),
// 3 the nodal value g_{k+1}.
struct TermsDev {
  int n;
  pe_term t[PE_MAX_TERMS];
  signed char lk[PE_MAX_TERMS][PE_MAX_D];
};

struct Nodes {
  double c[PE_MAX_S];
};

struct Gauss {
  int npts;
  double s[8];  // nodes in [0,1]
  double w[8];  // weights summing to 1
};

// Spatial factor at x; t is used only by factors that move (PE_S_MOVING_HAT:
// max(1 - |x - c(t)|/p3, 0) with c(t) = p0 + p1 sin(2 pi p2 t)).
__device__ inline double eval_space(int kind, const double* p, double x, double t = 0.0) {
  switch (kind) {
    case PE_S_SIN: return sin(p[0] * x + p[1]);
    case PE_S_GAUSS: { const double u = x - p[0]; return exp(-(u * u) / (2.0 * p[1] * p[1])); }
    case PE_S_POLY: return p[0] + x * (p[1] + x * (p[2] + x * p[3]));
    case PE_S_MOVING_HAT: {
      const double c = p[0] + p[1] * sinpi(2.0 * p[2] * t);
      return fmax(1.0 - fabs(x - c) / p[3], 0.0);
    }
    default: return 1.0;
  }
}

__device__ inline double eval_time(const pe_term& t, double tt) {
  if (t.tkind == PE_T_SIN) return sin(t.tp[0] * tt + t.tp[1]);
  return exp(t.tp[0] * tt);
}


// Gauss-Legendre rule on [0,1] by Newton iteration on the Legendre polynomial.
inline Gauss make_gauss(int npts) {
  Gauss G{};
  G.npts = npts;
  for (int i = 0; i < npts; ++i) {
    double x = cos(M_PI * (i + 0.75) / (npts + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= npts; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (npts == 1) { p1 = x; p0 = 1.0; }
      dp = npts * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    // recompute derivative at the converged root
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= npts; ++k) {
      const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (npts == 1) { p1 = x; p0 = 1.0; }
    dp = npts * (x * p1 - p0) / (x * x - 1.0);
    const double w = 2.0 / ((1.0 - x * x) * dp * dp);
    G.s[npts - 1 - i] = 0.5 * (x + 1.0);
    G.w[npts - 1 - i] = 0.5 * w;
  }
  return G;
}

inline TermsDev pack_terms(const pe_term* terms, int n, const signed char (*lk)[PE_MAX_D] = nullptr) {
  TermsDev T{};
  T.n = n;
  for (int i = 0; i < n; ++i) {
    T.t[i] = terms[i];
    for (int a = 0; a < PE_MAX_D; ++a) T.lk[i][a] = lk ? lk[i][a] : 0;
  }
  return T;
}

