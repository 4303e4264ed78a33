// Closed-form spectra of the Q1 matrices, lam_J, and the phi/b coefficient tables.
//
// Sec. 2.3 (closing paragraph): the Q1 mass and stiffness matrices are
// diagonalised at once by the tensor DST-I.  Per axis, with
// theta_j = j pi/(n+1):  mu^M_j = (h/3)(2 + cos theta_j),
// mu^K_j = (4/h) sin^2(theta_j/2), and lam_J = D sum_a mu^K_a/mu^M_a.
//
// Eq. (3-12): b_i(z) = int_0^1 e^{z(1-theta)} l_i(theta) dtheta.  Writing the
// Lagrange basis in monomials, l_i(theta) = sum_m a_{im} theta^m, gives
// b_i(z) = sum_m a_{im} m! phi_{m+1}(z) with phi_j as in Theorem 3.1's proof.
// phi_s is summed as a Taylor series for |z| < 2 and the lower phi_j follow by
// the backward recurrence phi_j = z phi_{j+1} + 1/j! (stable there); for
// |z| >= 2, phi_1 = expm1(z)/z and phi_{j+1} = (phi_j - 1/j!)/z.
#include <math.h>

#include "pe_internal.h"
#include "pe_phi.cuh"


namespace {

// 1D eigenvalue tables of every axis, concatenated.
__global__ void axis_tables_kernel(Geom g, double h0, double h1, double h2, double* muM, double* ratio) {
  const int a = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;  // 0-based mode index, mode number j+1
  if (a >= g.d || j >= g.n[a]) return;
  const double h = a == 0 ? h0 : (a == 1 ? h1 : h2);
  // theta = (j+1) pi/(n+1) (Dirichlet, DST-I) or 2 pi j/n (periodic, DHT)
  double cth, sh;
  if (g.per[a]) {
    cth = cospi(2.0 * (double)j / (double)g.n[a]);
    sh = sinpi((double)j / (double)g.n[a]);
  } else {
    const double np1 = (double)(g.n[a] + 1);
    cth = cospi((double)(j + 1) / np1);
    sh = sinpi((double)(j + 1) / (2.0 * np1));
  }
  const double mM = (h / 3.0) * (2.0 + cth);
  const double mK = (4.0 / h) * (sh * sh);
  muM[g.off[a] + j] = mM;
  ratio[g.off[a] + j] = mK / mM;
}

__global__ void coef_tables_kernel(Geom g, const double* __restrict__ ratio, double D, double dt, double dT,
                                   int M, int q, int p, Lag LF, Lag LG, double* __restrict__ lam_out,
                                   double* __restrict__ coefF, double* __restrict__ coefG,
                                   float* __restrict__ coefF32) {
  const int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= g.ndof) return;
  int j[PE_MAX_D];
  unflatten(g, J, j);
  double s = 0.0;
#pragma unroll
  for (int a = 0; a < PE_MAX_D; ++a) if (a < g.d) s += ratio[g.off[a] + j[a]];
  const double lam = D * s;
  lam_out[J] = lam;
  const int64_t nd = g.ndof;
  double b[PE_MAX_S];
  // fine step dt, q nodes
  {
    const double z = -lam * dt;
    const double E = exp(z);
    b_weights(z, q, LF, b);
    coefF[J] = E;
    for (int i = 0; i < q; ++i) coefF[(1 + i) * nd + J] = dt * b[i];
    const double EM = exp(-lam * ((double)M * dt));
    coefF[(q + 1) * nd + J] = EM;
    if (coefF32) {
      const float ehi = (float)E;
      coefF32[J] = ehi;
      coefF32[nd + J] = (float)(E - (double)ehi);
      for (int i = 0; i < q; ++i) coefF32[(2 + i) * nd + J] = (float)(dt * b[i]);
    }
  }
  // coarse step dT, p nodes
  {
    const double z = -lam * dT;
    b_weights(z, p, LG, b);
    coefG[J] = exp(z);
    for (int i = 0; i < p; ++i) coefG[(1 + i) * nd + J] = dT * b[i];
  }
}

// DST-I (Dirichlet) or, for a periodic axis, the DHT H[j][k] = (cos + sin)(2 pi j k/n)/sqrt(n)
// (j k reduced modulo the period in both cases)
__device__ inline double axis_transform_entry(int n, int j, int k, int periodic) {
  if (periodic) {
    const int64_t m = ((int64_t)j * k) % n;
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    return (c + s) / sqrt((double)n);
  }
  const int64_t period = 2 * (int64_t)(n + 1);
  const int64_t m = ((int64_t)(j + 1) * (k + 1)) % period;
  return sqrt(2.0 / (double)(n + 1)) * sinpi((double)m / (double)(n + 1));
}

__global__ void dst_matrix_kernel(int n, double* S, int periodic) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (k >= n || j >= n) return;
  S[(int64_t)j * n + k] = axis_transform_entry(n, j, k, periodic);
}

}  // namespace

// Per-axis eigenvalue tables of the modes this context owns (a sharded context: the whole
// axes first, then its rows).
__global__ void reciprocal_kernel(int n, const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = 1.0 / x[i];
}

pe_status launch_axis_tables(pe_ctx* c) {
  int nmax = 1;
  for (int a = 0; a < c->gn.d; ++a) nmax = c->gn.n[a] > nmax ? c->gn.n[a] : nmax;
  dim3 grid((nmax + 127) / 128, c->gn.d);
  double* mu = c->sharded ? c->muM_full : c->muM_axis;
  double* ratio = c->sharded ? c->ratio_full : c->ratio_axis;
  axis_tables_kernel<<<grid, 128, 0, c->stream>>>(c->gn, c->h[0], c->gn.d > 1 ? c->h[1] : 1.0,
                                                  c->gn.d > 2 ? c->h[2] : 1.0, mu, ratio);
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  if (c->muM_inv) {  // of the whole axes (the per-axis factors are made for the whole grid)
    const int nsum = c->gn.off[c->gn.d - 1] + c->gn.n[c->gn.d - 1];
    reciprocal_kernel<<<(nsum + 255) / 256, 256, 0, c->stream>>>(nsum, mu, c->muM_inv);
    c->launches += 1;
    PE_CUDA_TRY(cudaGetLastError());
  }
  if (c->sharded) {
    PE_TRY(compact_axis_tables(c, 1, c->muM_full, c->muM_axis, nullptr));
    PE_TRY(compact_axis_tables(c, 1, c->ratio_full, c->ratio_axis, nullptr));
  }
  return PE_OK;
}

pe_status launch_coef_tables(pe_ctx* c) {
  Lag LF{}, LG{};
  for (int i = 0; i < PE_MAX_S; ++i)
    for (int m = 0; m < PE_MAX_S; ++m) {
      LF.a[i][m] = c->lagF[i][m];
      LG.a[i][m] = c->lagG[i][m];
    }
  const int threads = 256;
  const int64_t blocks = (c->g.ndof + threads - 1) / threads;
  coef_tables_kernel<<<(unsigned)blocks, threads, 0, c->stream>>>(
      c->g, c->ratio_axis, c->D, c->dt, c->dT, c->M, c->q, c->p, LF, LG, c->lam, c->coefF, c->coefG,
      c->precision == PE_MIXED ? c->coefF32 : nullptr);
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

__global__ void dst_matrix_f32_kernel(int n, float* S, int periodic) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (k >= n || j >= n) return;
  S[(int64_t)j * n + k] = (float)axis_transform_entry(n, j, k, periodic);
}

pe_status build_dst_matrix_f32(int n, float* S, cudaStream_t st, int periodic) {
  dim3 grid((n + 127) / 128, n);
  dst_matrix_f32_kernel<<<grid, 128, 0, st>>>(n, S, periodic);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status build_dst_matrix(int n, double* S, cudaStream_t st, int periodic) {
  dim3 grid((n + 127) / 128, n);
  dst_matrix_kernel<<<grid, 128, 0, st>>>(n, S, periodic);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}
