// Batched Parareal EIFE-linear: many independent problems in one set of launches.
//
// Each array kind (slice arrays, tables, forcing factors) lives in one arena; a
// device table of per-problem records (BProb) holds offsets into the arenas.
// Work is cut into items:
//   mode items  (problem, 256 consecutive modes)          coefficient tables, U^0,
//                                                         coarse sweep, correction
//   fine items  (problem, slice n, threads*MPT modes)     fine propagator
// The fine kernel is persistent: every CTA pulls items from an atomic counter
// and dispatches on the problem's number of forcing terms R (each R has its own
// register-resident tile body).  One Parareal iteration (reset of the counter,
// fine sweep, correction, per-problem residual + stop flags, readback of the
// number of active problems) is captured once as a CUDA graph and replayed.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "pe_batch.h"
#include "pe_phi.cuh"

namespace {

__device__ __forceinline__ int find_prob(const int64_t* __restrict__ prefix, int P, int64_t idx) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= idx) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// setup kernels
// ---------------------------------------------------------------------------
__global__ void b_axis_tables_kernel(const BProb* __restrict__ probs, const int64_t* __restrict__ mu_prefix, int P,
                                     int64_t total, double* __restrict__ muM, double* __restrict__ ratio) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int p = find_prob(mu_prefix, P, idx);
  const BProb& B = probs[p];
  const int local = (int)(idx - B.oMu);
  int a = 0;
  while (a + 1 < B.g.d && local >= B.g.off[a + 1]) ++a;
  const int j = local - B.g.off[a];
  const double h = B.h[a];
  const double np1 = (double)(B.g.n[a] + 1);
  const double cth = cospi((double)(j + 1) / np1);
  const double sh = sinpi((double)(j + 1) / (2.0 * np1));
  const double mM = (h / 3.0) * (2.0 + cth);
  const double mK = (4.0 / h) * (sh * sh);
  muM[idx] = mM;
  ratio[idx] = mK / mM;
}

__global__ void b_coef_tables_kernel(const BProb* __restrict__ probs, const ModeItem* __restrict__ items,
                                     int n_items, const double* __restrict__ ratio, double* __restrict__ coefF,
                                     double* __restrict__ coefG, float* __restrict__ coefF32) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const ModeItem m = items[it];
    const BProb& B = probs[m.p];
    const int64_t J = m.J0 + threadIdx.x;
    if (J >= B.g.ndof) continue;
    const int64_t nd = B.g.ndof;
    int j[PE_MAX_D];
    unflatten(B.g, J, j);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < PE_MAX_D; ++a) if (a < B.g.d) s += ratio[B.oMu + B.g.off[a] + j[a]];
    const double lam = B.D * s;
    Lag LF, LG;
    for (int i = 0; i < PE_MAX_S; ++i)
      for (int k = 0; k < PE_MAX_S; ++k) {
        LF.a[i][k] = B.lagF[i][k];
        LG.a[i][k] = B.lagG[i][k];
      }
    double b[PE_MAX_S];
    {
      const double z = -lam * B.dt;
      const double E = exp(z);
      b_weights(z, B.q, LF, b);
      double* cf = coefF + B.oCF;
      cf[J] = E;
      for (int i = 0; i < B.q; ++i) cf[(1 + i) * nd + J] = B.dt * b[i];
      cf[(B.q + 1) * nd + J] = exp(-lam * ((double)B.M * B.dt));
      if (coefF32) {
        float* c32 = coefF32 + B.oCF;
        const float ehi = (float)E;
        c32[J] = ehi;
        c32[nd + J] = (float)(E - (double)ehi);
        for (int i = 0; i < B.q; ++i) c32[(2 + i) * nd + J] = (float)(B.dt * b[i]);
      }
    }
    {
      const double z = -lam * B.dT;
      b_weights(z, B.p, LG, b);
      double* cg = coefG + B.oCG;
      cg[J] = exp(z);
      for (int i = 0; i < B.p; ++i) cg[(1 + i) * nd + J] = B.dT * b[i];
    }
  }
}

// Time tables of every problem, one thread per entry (layout as in the single-problem
// solver): fine substep starts Y[(n*M + m)*K + k] (float copy: rows of KC = roundup(K, 4)),
// coarse stage times AG[(n*p + i)*R + r],
// stage shifts Z[i*K + k].  Column k of a problem is cols[oCol + k] = (term << 1) | kind:
// kind 0 is amp*time(t) (shift factor e^{as} or cos(ws)), kind 1 the partner amp*cos(wt+phi)
// of a sinusoid (shift factor sin(ws)).
__global__ void b_time_tables_kernel(const BProb* __restrict__ probs, const int64_t* __restrict__ tt_prefix, int P,
                                     int64_t total, const pe_term* __restrict__ terms,
                                     const short* __restrict__ cols, double* __restrict__ AF,
                                     float* __restrict__ AF32, double* __restrict__ AG, float* __restrict__ AG32,
                                     double* __restrict__ Z, float* __restrict__ Z32) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int p = find_prob(tt_prefix, P, idx);
  const BProb& B = probs[p];
  const int R = B.R, K = B.K;
  const int64_t nrow = (int64_t)B.N * K;
  const int64_t ng = (int64_t)B.N * B.p * R;
  int64_t local = idx - tt_prefix[p];
  if (local < nrow) {
    // one thread per (slice n, column k) walks the substeps m: the factor at T_n + m dt from
    // the one at T_n by the exact step e^{a dt} or the rotation by omega dt (angle addition),
    // two transcendental evaluations per thread instead of one per entry; the rounding grows
    // by about one unit in the last place per substep (M <= 128)
    const int k = (int)(local % K), n = (int)(local / K);
    const int c = cols[B.oCol + k];
    const pe_term& T = terms[B.tf + (c >> 1)];
    const double tn = B.t0 + (double)n * B.dT;
    const int KC = (K + 3) & ~3;
    double* af = AF + B.oAF + (int64_t)n * B.M * K + k;
    float* row32 = AF32 ? AF32 + B.oAF32 + (int64_t)n * B.M * KC : nullptr;
    auto put = [&](int m, double v) {
      af[(int64_t)m * K] = v;
      if (row32) {
        float* row = row32 + (int64_t)m * KC;
        row[k] = (float)v;
        if (k == K - 1)
          for (int e = K; e < KC; ++e) row[e] = 0.f;
      }
    };
    if (T.tkind == PE_T_SIN) {
      double sa, ca, sb, cb;
      sincos(T.tp[0] * tn + T.tp[1], &sa, &ca);
      sincos(T.tp[0] * B.dt, &sb, &cb);
      for (int m = 0; m < B.M; ++m) {
        put(m, T.amp * ((c & 1) ? ca : sa));
        const double s2 = fma(sa, cb, ca * sb);
        ca = fma(ca, cb, -(sa * sb));
        sa = s2;
      }
    } else {
      double e = exp(T.tp[0] * tn);
      const double eb = exp(T.tp[0] * B.dt);
      for (int m = 0; m < B.M; ++m) {
        put(m, T.amp * e);
        e *= eb;
      }
    }
  } else if (local < nrow + ng) {
    local -= nrow;
    int64_t rest = local;
    const int r = (int)(rest % R); rest /= R;
    const int i = (int)(rest % B.p); rest /= B.p;
    const int n = (int)rest;
    const double Tn = B.t0 + (double)n * B.dT;
    const double t = Tn + B.cG[i] * B.dT;
    const pe_term& T = terms[B.tf + r];
    const double v = T.amp * eval_time(T, t);
    AG[B.oAG + local] = v;
    if (AG32) AG32[B.oAG + local] = (float)v;
  } else {
    local -= nrow + ng;
    const int k = (int)(local % K), i = (int)(local / K);
    const int c = cols[B.oCol + k];
    const pe_term& T = terms[B.tf + (c >> 1)];
    const double s = B.cF[i] * B.dt;
    double v;
    if (T.tkind == PE_T_SIN) v = (c & 1) ? sin(T.tp[0] * s) : cos(T.tp[0] * s);
    else v = exp(T.tp[0] * s);
    Z[B.oZ + local] = v;
    if (Z32) Z32[B.oZ + local] = (float)v;
  }
}

// Per-mode stage weights W[oW + k*ndof + J] = P_{r(k),J} sum_i (dt b_i)_J Z[oZ + i*K + k],
// in the arithmetic of T: float64 into W for the float64 fine kernel; float32 (from the
// float factors and shifts) into W32 in the mixed form, whose fine kernel reads only W32.
template <typename T>
__global__ void b_stage_weights_kernel(const BProb* __restrict__ probs, const ModeItem* __restrict__ items,
                                       int n_items, const short* __restrict__ cols, const T* __restrict__ axisF,
                                       const double* __restrict__ coefF, const T* __restrict__ Z,
                                       T* __restrict__ W) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const ModeItem mi = items[it];
    const BProb& B = probs[mi.p];
    const int64_t J = mi.J0 + threadIdx.x;
    if (J >= B.g.ndof) continue;
    const int64_t nd = B.g.ndof;
    int j[PE_MAX_D];
    unflatten(B.g, J, j);
    T b[PE_MAX_S];
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i) b[i] = i < B.q ? (T)coefF[B.oCF + (int64_t)(1 + i) * nd + J] : T(0);
    const T* ax = axisF + B.oAx;
    const T* z = Z + B.oZ;
    for (int k = 0; k < B.K; ++k) {
      const int r = cols[B.oCol + k] >> 1;
      T P = ax[(int64_t)B.R * B.g.off[0] + (int64_t)r * B.g.n[0] + j[0]];
#pragma unroll
      for (int a = 1; a < PE_MAX_D; ++a) if (a < B.g.d)
        P *= ax[(int64_t)B.R * B.g.off[a] + (int64_t)r * B.g.n[a] + j[a]];
      T sum = T(0);
#pragma unroll
      for (int i = 0; i < PE_MAX_S; ++i)
        if (i < B.q) sum = fma(b[i], z[(int64_t)i * B.K + k], sum);
      W[B.oW + (int64_t)k * nd + J] = P * sum;
    }
  }
}

// One CTA per (problem, axis, term): the 1D consistent load of the term's factor
// on that axis, its DST-I (sine table in shared memory) and the division by mu^M.
__global__ void b_axis_factor_kernel(const BProb* __restrict__ probs, const FactorJob* __restrict__ jobs,
                                     const pe_term* __restrict__ terms, Gauss G, const double* __restrict__ muM,
                                     double* __restrict__ axisF, float* __restrict__ axisF32,
                                     double* __restrict__ axisU0) {
  extern __shared__ double sh[];
  const FactorJob job = jobs[blockIdx.x];
  const BProb& B = probs[job.p];
  const int a = job.axis;
  const int n = B.g.n[a];
  const int period = 2 * (n + 1);
  double* F = sh;             // [n]
  double* tab = sh + n;       // [period]: sin(pi m/(n+1))
  const pe_term& T = terms[job.u0 ? B.tu + job.r : B.tf + job.r];
  const double lo = B.lo[a], h = B.h[a];
  for (int m = threadIdx.x; m < period; m += blockDim.x) tab[m] = sinpi((double)m / (double)(n + 1));
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double left = 0.0, right = 0.0;
    for (int qi = 0; qi < G.npts; ++qi) {
      const double xl = lo + ((double)k + G.s[qi]) * h;
      const double xr = lo + ((double)(k + 1) + G.s[qi]) * h;
      left += G.w[qi] * eval_space(T.skind[a], T.sp[a], xl) * G.s[qi];
      right += G.w[qi] * eval_space(T.skind[a], T.sp[a], xr) * (1.0 - G.s[qi]);
    }
    F[k] = h * left + h * right;
  }
  __syncthreads();
  const double scale = sqrt(2.0 / (double)(n + 1));
  const int Rj = job.u0 ? B.Ru : B.R;
  const int64_t obase = (job.u0 ? B.oAxU : B.oAx) + (int64_t)Rj * B.g.off[a] + (int64_t)job.r * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double acc = 0.0;
    int idx = 0;
    const int step = j + 1;
    for (int k = 0; k < n; ++k) {
      idx += step;
      if (idx >= period) idx -= period;
      acc = fma(tab[idx], F[k], acc);
    }
    const double v = scale * acc / muM[B.oMu + B.g.off[a] + j];
    if (job.u0) {
      axisU0[obase + j] = v;
    } else {
      axisF[obase + j] = v;
      if (axisF32) axisF32[obase + j] = (float)v;
    }
  }
}

// U^0 = sum_t amp_t prod_a axisU0 (P_h of separable initial data)
__global__ void b_u0_kernel(const BProb* __restrict__ probs, const ModeItem* __restrict__ items, int n_items,
                            const pe_term* __restrict__ terms, const double* __restrict__ axisU0,
                            double* __restrict__ U) {
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const ModeItem m = items[it];
    const BProb& B = probs[m.p];
    const int64_t J = m.J0 + threadIdx.x;
    if (J >= B.g.ndof) continue;
    int j[PE_MAX_D];
    unflatten(B.g, J, j);
    double acc = 0.0;
    for (int t = 0; t < B.Ru; ++t) {
      double v = axisU0[B.oAxU + (int64_t)B.Ru * B.g.off[0] + (int64_t)t * B.g.n[0] + j[0]];
#pragma unroll
      for (int a = 1; a < PE_MAX_D; ++a) if (a < B.g.d)
        v *= axisU0[B.oAxU + (int64_t)B.Ru * B.g.off[a] + (int64_t)t * B.g.n[a] + j[a]];
      acc += terms[B.tu + t].amp * v;
    }
    U[B.oU + J] = acc;
  }
}

// coarse sweep (k = 0) of every problem; P_{r,J} staged per thread in shared memory
// Slices of loads each thread keeps in flight in the sequential correction (its
// inputs do not depend on the recurrence, so they are fetched kPF slices ahead).
constexpr int kPF = 4;

// Coarse sweep of k = 0 for every problem (item-strided grid: an item is 256 modes of one
// problem), U^{n+1} = E_G U^n + gG_n with the coarse forcing gG_n = sum_i b_i sum_r
// A_r(T_n + c_i dT) P_{r,J} made on the fly: the weights P_{r,J} sit in registers (RB =
// roundup(PE_BATCH_MAX_TERMS, 4), zero past R) and the item's time factors are staged in
// shared memory a chunk of slices at a time (rows of RB, read as float4 / double2
// broadcasts).  TF = float in the mixed form (the coarse forcing only sets the first coarse
// iterate; the affine correction never reads it again).
constexpr int kCoarseRB = (PE_BATCH_MAX_TERMS + 3) / 4 * 4;
constexpr int kCoarseSmem = 16 * 1024;  // bytes of staged time factors per CTA

// LEARN: the learned term of G' = G + delta^ is added per slice, sum_r (A_r cos_{r,n} + B_r sin_{r,n})
// with A_r = P_{r,J} amp_r Im K^, B_r = P_{r,J} amp_r Re K^ (K^ interpolated linearly in
// log(lam dT) between the problem's band centres), as the single-problem coarse sweep does.
struct BLearn {
  const double* ratio;    // per-axis mu^K / mu^M (lam = D sum_a ratio)
  const pe_term* terms;
  const double* Kt;       // band tables
  const float2* Ph;       // phase tables
  int NB;
};

template <typename TF, bool LEARN>
__global__ void __launch_bounds__(256) b_coarse_kernel(const BProb* __restrict__ probs,
                                                       const ModeItem* __restrict__ items, int n_items,
                                                       const double* __restrict__ axisF, const TF* __restrict__ AG,
                                                       const double* __restrict__ coefG, double* __restrict__ U,
                                                       BLearn L, const float* __restrict__ axisF32) {
  constexpr int RB = kCoarseRB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TF* sA = reinterpret_cast<TF*>(smem_raw);  // [chunk * p][RB]
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const ModeItem m = items[it];
    const BProb& B = probs[m.p];
    const int64_t J = m.J0 + threadIdx.x;
    const int64_t nd = B.g.ndof;
    const bool on = J < nd;  // no early exit: the staging below needs every thread's barrier
    const int R = B.R, p = B.p, N = B.N;
    TF P[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) P[r] = TF(0);
    TF b[PE_MAX_S];
#pragma unroll
    for (int i = 0; i < PE_MAX_S; ++i) b[i] = TF(0);
    double E = 0.0, c = 0.0;
    const double* cg = coefG + B.oCG;
    float LA[LEARN ? kCoarseRB : 1], LB[LEARN ? kCoarseRB : 1];
#pragma unroll
    for (int r = 0; r < (LEARN ? kCoarseRB : 1); ++r) {
      LA[r] = 0.f;
      LB[r] = 0.f;
    }
    if (on) {
      int j[PE_MAX_D];
      unflatten(B.g, J, j);
      if constexpr (LEARN) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < PE_MAX_D; ++a) if (a < B.g.d) s += L.ratio[B.oMu + B.g.off[a] + j[a]];
        double pos = (log(B.D * s * B.dT) - B.lloglo) / B.lstep;
        pos = fmin(fmax(pos, 0.0), (double)(L.NB - 1) - 1e-9);
        const int b0 = (int)pos;
        const double f = pos - (double)b0;
#pragma unroll
        for (int r = 0; r < kCoarseRB; ++r) {
          if (r < R && L.terms[B.tf + r].tkind == PE_T_SIN) {
            double Pd = axisF[B.oAx + (int64_t)R * B.g.off[0] + (int64_t)r * B.g.n[0] + j[0]];
#pragma unroll
            for (int a = 1; a < PE_MAX_D; ++a)
              if (a < B.g.d) Pd *= axisF[B.oAx + (int64_t)R * B.g.off[a] + (int64_t)r * B.g.n[a] + j[a]];
            const double* k0 = L.Kt + B.oKt + 2 * ((int64_t)r * L.NB + b0);
            const double Kre = (1.0 - f) * k0[0] + f * k0[2];
            const double Kim = (1.0 - f) * k0[1] + f * k0[3];
            const double cc = Pd * L.terms[B.tf + r].amp;
            LA[r] = (float)(cc * Kim);
            LB[r] = (float)(cc * Kre);
          }
        }
      }
      // the source weights P_{r,J}: in the mixed form from the float32 factors in float32 (as
      // the single-problem sweep forms them; no float64 product and conversion per term)
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        if (r < R) {
          if constexpr (sizeof(TF) == 4) {
            float v = axisF32[B.oAx + (int64_t)R * B.g.off[0] + (int64_t)r * B.g.n[0] + j[0]];
#pragma unroll
            for (int a = 1; a < PE_MAX_D; ++a)
              if (a < B.g.d) v *= axisF32[B.oAx + (int64_t)R * B.g.off[a] + (int64_t)r * B.g.n[a] + j[a]];
            P[r] = v;
          } else {
            double v = axisF[B.oAx + (int64_t)R * B.g.off[0] + (int64_t)r * B.g.n[0] + j[0]];
#pragma unroll
            for (int a = 1; a < PE_MAX_D; ++a)
              if (a < B.g.d) v *= axisF[B.oAx + (int64_t)R * B.g.off[a] + (int64_t)r * B.g.n[a] + j[a]];
            P[r] = (TF)v;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < PE_MAX_S; ++i)
        if (i < p) b[i] = (TF)cg[(1 + i) * nd + J];
      E = cg[J];
      c = U[B.oU + J];
    }
    const TF* ag = AG + B.oAG;
    const int CS = max(1, kCoarseSmem / (int)(p * RB * sizeof(TF)));  // slices per chunk
    for (int n0 = 0; n0 < N; n0 += CS) {
      const int nc = min(CS, N - n0);
      __syncthreads();  // the previous chunk's (or item's) reads of sA are done
      for (int e = threadIdx.x; e < nc * p * RB; e += blockDim.x) {
        const int row = e / RB, r = e - row * RB;
        sA[e] = r < R ? ag[((int64_t)n0 * p + row) * R + r] : TF(0);
      }
      __syncthreads();
      if (on) {
        for (int n = 0; n < nc; ++n) {
          TF acc = TF(0);
#pragma unroll
          for (int i = 0; i < PE_MAX_S; ++i) {
            if (i < p) {
              const TF* a = sA + ((int64_t)n * p + i) * RB;
              TF gi = TF(0);
              if constexpr (sizeof(TF) == 4) {
#pragma unroll
                for (int r = 0; r < RB; r += 4) {
                  const float4 v = *reinterpret_cast<const float4*>(a + r);
                  gi = fmaf(v.x, P[r], gi);
                  gi = fmaf(v.y, P[r + 1], gi);
                  gi = fmaf(v.z, P[r + 2], gi);
                  gi = fmaf(v.w, P[r + 3], gi);
                }
              } else {
#pragma unroll
                for (int r = 0; r < RB; r += 2) {
                  const double2 v = *reinterpret_cast<const double2*>(a + r);
                  gi = fma(v.x, P[r], gi);
                  gi = fma(v.y, P[r + 1], gi);
                }
              }
              acc = fma(b[i], gi, acc);
            }
          }
          double gn;
          if constexpr (sizeof(TF) == 4) gn = widen_f32(acc);  // exact, off the float64 pipe
          else gn = acc;
          if constexpr (LEARN) {
            float dl = 0.f;
            const float2* ph = L.Ph + B.oPh + n0 + n;
#pragma unroll
            for (int r = 0; r < kCoarseRB; ++r)
              if (r < R) {
                const float2 e = __ldg(ph + (int64_t)r * N);
                dl = fmaf(LA[r], e.x, fmaf(LB[r], e.y, dl));
              }
            gn += widen_f32(dl);
          }
          c = fma(E, c, gn);
          U[B.oU + (int64_t)(n0 + n + 1) * nd + J] = c;
        }
      }
    }
  }
}

template <typename T>
__device__ inline T block_sum(T v, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T out = T(0);
  if (threadIdx.x < 32) {
    T x = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : T(0);
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    out = x;
  }
  __syncthreads();
  return out;
}

// correction + residual partial sums of every active problem (item-strided grid).  G is
// affine in its argument, so U^{n+1,(k+1)} = G(U^{n,(k+1)}) + Fbar^{n+1} - G(U^{n,(k)}) is
// evaluated as Fbar^{n+1} + E_G (U^{n,(k+1)} - U^{n,(k)}) (no stored coarse values).
__global__ void __launch_bounds__(256) b_correction_kernel(const BProb* __restrict__ probs,
                                                           const ModeItem* __restrict__ items, int n_items,
                                                           const int* __restrict__ active,
                                                           const double* __restrict__ muM,
                                                           const double* __restrict__ coefG,
                                                           const double* __restrict__ Fbar,
                                                           double* __restrict__ U, double* __restrict__ partials) {
  __shared__ double sh[32];
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const ModeItem m = items[it];
    const BProb& B = probs[m.p];
    if (!active[m.p]) continue;  // uniform over the CTA
    const int64_t J = m.J0 + threadIdx.x;
    double sd = 0.0, su = 0.0, w = 0.0;
    if (J < B.g.ndof) {
      const int64_t nd = B.g.ndof;
      const int N = B.N;
      int j[PE_MAX_D];
      unflatten(B.g, J, j);
      w = muM[B.oMu + B.g.off[0] + j[0]];
#pragma unroll
      for (int a = 1; a < PE_MAX_D; ++a) if (a < B.g.d) w *= muM[B.oMu + B.g.off[a] + j[a]];
      const double E = coefG[B.oCG + J];
      double* Up = U + B.oU;
      const double* fp = Fbar + B.oS;
      // U^0 is the same in every iterate (d = U^n_new - U^n_old starts at 0); the loads of the
      // next kPF slices are issued while the current kPF are combined.  Four FP64 operations
      // per slice: the difference d is both the next slice's correction and this slice's
      // residual term.
      double d = 0.0;
      double f0[kPF], o0[kPF], f1[kPF], o1[kPF];
#pragma unroll
      for (int e = 0; e < kPF; ++e) {
        const int64_t o = (int64_t)e * nd + J;
        const bool in = e < N;
        f0[e] = in ? fp[o] : 0.0;
        o0[e] = in ? Up[o + nd] : 0.0;
      }
      for (int n0 = 0; n0 < N; n0 += kPF) {
#pragma unroll
        for (int e = 0; e < kPF; ++e) {
          const int n = n0 + kPF + e;
          const int64_t o = (int64_t)n * nd + J;
          const bool in = n < N;
          f1[e] = in ? fp[o] : 0.0;
          o1[e] = in ? Up[o + nd] : 0.0;
        }
#pragma unroll
        for (int e = 0; e < kPF; ++e) {
          const int n = n0 + e;
          if (n < N) {
            const double nxt = fma(E, d, f0[e]);
            Up[(int64_t)(n + 1) * nd + J] = nxt;
            d = nxt - o0[e];
            sd = fma(d, d, sd);
            su = fma(nxt, nxt, su);
          }
        }
#pragma unroll
        for (int e = 0; e < kPF; ++e) {
          f0[e] = f1[e];
          o0[e] = o1[e];
        }
      }
    }
    // the weight mu^M_J is the same for every slice of the mode: applied once
    sd *= w;
    su *= w;
    sd = block_sum(sd, sh);
    su = block_sum(su, sh);
    if (threadIdx.x == 0) {
      partials[2 * it] = sd;
      partials[2 * it + 1] = su;
    }
  }
}

// one CTA per problem: residual, iteration count, stop flag, active count
__global__ void b_reduce_kernel(const BProb* __restrict__ probs, int P, const double* __restrict__ partials,
                                int* __restrict__ active, int* __restrict__ kcount, double* __restrict__ resid,
                                double tol, int* __restrict__ n_active, int* __restrict__ nonfinite) {
  __shared__ double sh[32];
  const int p = blockIdx.x;
  if (p >= P) return;
  const BProb& B = probs[p];
  if (!active[p]) return;  // uniform
  double sd = 0.0, su = 0.0;
  for (int i = threadIdx.x; i < B.nItems; i += blockDim.x) {
    sd += partials[2 * (B.oItems + i)];
    su += partials[2 * (B.oItems + i) + 1];
  }
  sd = block_sum(sd, sh);
  su = block_sum(su, sh);
  if (threadIdx.x == 0) {
    const double r = su > 0.0 ? sqrt(sd) / sqrt(su) : sqrt(sd);
    resid[p] = r;
    const int k = kcount[p] + 1;
    kcount[p] = k;
    if (!isfinite(r)) {
      atomicExch(nonfinite, 1);
      active[p] = 0;
    } else if (r <= tol || k >= B.N) {
      active[p] = 0;
    } else {
      atomicAdd(n_active, 1);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
pe_status batch_set_attributes(pe_batch* b) {
  const size_t smem = sizeof(double) * (size_t)(b->nmax + 2 * (b->nmax + 1));
  PE_CUDA_TRY(cudaFuncSetAttribute(b_axis_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));

  return PE_OK;  // the fine kernels stage at most 48 KB (pick_mchunk), the default limit
}

pe_status batch_launch_axis_tables(pe_batch* b) {
  const int64_t total = b->mu_total;
  b_axis_tables_kernel<<<(unsigned)((total + 255) / 256), 256, 0, b->stream>>>(b->d_probs, b->d_mu_prefix, b->P,
                                                                              total, b->muM, b->ratio);
  b->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

// phi/b coefficient tables: a function of lam, the step sizes and the nodes only (made at set-up)
pe_status batch_launch_coef_tables(pe_batch* b) {
  b_coef_tables_kernel<<<b->sm_count * 8, 256, 0, b->stream>>>(b->d_probs, b->d_mode_items, b->n_mode_items,
                                                               b->ratio, b->coefF, b->coefG, b->coefF32);
  b->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status batch_launch_prepare(pe_batch* b) {
  const int grid_items = b->sm_count * 8;
  // time factors
  b_time_tables_kernel<<<(unsigned)((b->tt_total + 255) / 256), 256, 0, b->stream>>>(
      b->d_probs, b->d_tt_prefix, b->P, b->tt_total, b->d_terms, b->d_cols, b->AF, b->AF32, b->AG, b->AG32, b->Z,
      b->Z32);
  // per-axis factors of forcing and initial data
  const size_t smem = sizeof(double) * (size_t)(b->nmax + 2 * (b->nmax + 1));
  b_axis_factor_kernel<<<b->n_factor_jobs, 256, smem, b->stream>>>(b->d_probs, b->d_factor_jobs, b->d_terms,
                                                                   b->gauss, b->muM, b->axisF, b->axisF32,
                                                                   b->axisU0);
  // per-mode stage weights of the fine step
  if (b->precision == PE_MIXED)
    b_stage_weights_kernel<float><<<grid_items, 256, 0, b->stream>>>(
        b->d_probs, b->d_mode_items, b->n_mode_items, b->d_cols, b->axisF32, b->coefF, b->Z32, b->W32);
  else
    b_stage_weights_kernel<double><<<grid_items, 256, 0, b->stream>>>(
        b->d_probs, b->d_mode_items, b->n_mode_items, b->d_cols, b->axisF, b->coefF, b->Z, b->W);
  b_u0_kernel<<<grid_items, 256, 0, b->stream>>>(b->d_probs, b->d_mode_items, b->n_mode_items, b->d_terms, b->axisU0,
                                                 b->U);
  // the tensor-core engine's split operand images of every problem
  if (b->fine_engine == PE_FINE_TC) PE_TRY(batch_tc_prepare(b, b->stream));
  // the coarse forcing is iterate-independent and cancels in G(U^{k+1}) - G(U^k): the mixed
  // form evaluates it in float32, the recurrence stays float64
  // learned correction: band and phase tables first, the term summed inside the coarse sweep
  BLearn L{};
  if (b->mlp) {
    PE_TRY(batch_learned_tables(b, b->stream));
    L.ratio = b->ratio;
    L.terms = b->d_terms;
    L.Kt = b->Kt;
    L.Ph = b->Ph;
    L.NB = kBatchLearnedBands;
  }
  if (b->precision == PE_MIXED && b->mlp)
    b_coarse_kernel<float, true><<<grid_items, 256, kCoarseSmem, b->stream>>>(
        b->d_probs, b->d_mode_items, b->n_mode_items, b->axisF, b->AG32, b->coefG, b->U, L, b->axisF32);
  else if (b->precision == PE_MIXED)
    b_coarse_kernel<float, false><<<grid_items, 256, kCoarseSmem, b->stream>>>(
        b->d_probs, b->d_mode_items, b->n_mode_items, b->axisF, b->AG32, b->coefG, b->U, L, b->axisF32);
  else if (b->mlp)
    b_coarse_kernel<double, true><<<grid_items, 256, kCoarseSmem, b->stream>>>(
        b->d_probs, b->d_mode_items, b->n_mode_items, b->axisF, b->AG, b->coefG, b->U, L, (const float*)nullptr);
  else
    b_coarse_kernel<double, false><<<grid_items, 256, kCoarseSmem, b->stream>>>(
        b->d_probs, b->d_mode_items, b->n_mode_items, b->axisF, b->AG, b->coefG, b->U, L, (const float*)nullptr);
  b->launches += 5;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

// One persistent launch per column class present in the batch, each over its own items
// and counter (counter[c]); grids never exceed the class's item count.
static pe_status launch_fine(pe_batch* b, cudaStream_t st, int threads, int ctas_per_sm) {
  if (b->fine_engine == PE_FINE_TC) return batch_tc_fine(b, st);
  const FineItems& fi = threads == 128 ? b->fine128 : b->fine256;
  BatchArrays A{};
  A.W = b->W; A.W32 = b->W32; A.AF = b->AF; A.AF32 = b->AF32;
  A.coefF = b->coefF; A.coefF32 = b->coefF32; A.U = b->U; A.Fbar = b->Fbar;
  for (int c = 0; c < kBatchClasses; ++c) {
    const int n = fi.begin[c + 1] - fi.begin[c];
    if (n == 0) continue;
    const int grid = std::min(b->sm_count * ctas_per_sm, n);
    const FineItem* items = fi.d_items + fi.begin[c];
    if (b->precision == PE_MIXED)
      PE_TRY(batch_launch_fine_mixed(4 * (c + 1), b->d_probs, items, n, b->active, b->counter + c, A, grid, threads,
                                     fi.smem[c], st));
    else
      PE_TRY(batch_launch_fine_f64(4 * (c + 1), b->d_probs, items, n, b->active, b->counter + c, A, grid, threads,
                                   fi.smem[c], st));
  }
  return PE_OK;
}

int batch_fine_launches(const pe_batch* b) {
  int k = 0;
  if (b->fine_engine == PE_FINE_TC) {
    for (int c = 0; c < 3; ++c) k += b->tc.begin[c + 1] > b->tc.begin[c];
    return k;
  }
  for (int c = 0; c < kBatchClasses; ++c) k += b->fine256.begin[c + 1] > b->fine256.begin[c];
  return k;
}

pe_status batch_enqueue_iteration(pe_batch* b, cudaStream_t st, double tol) {
  PE_CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(int) * kBatchClasses, st));
  PE_CUDA_TRY(cudaMemsetAsync(b->n_active, 0, sizeof(int), st));
  PE_TRY(launch_fine(b, st, b->tune_threads, b->tune_ctas));
  b_correction_kernel<<<b->sm_count * 8, 256, 0, st>>>(b->d_probs, b->d_mode_items, b->n_mode_items, b->active,
                                                       b->muM, b->coefG, b->Fbar, b->U, b->partials);
  b_reduce_kernel<<<b->P, 256, 0, st>>>(b->d_probs, b->P, b->partials, b->active, b->kcount, b->resid, tol,
                                        b->n_active, b->nonfinite);
  PE_CUDA_TRY(cudaMemcpyAsync(b->h_flags, b->n_active, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status batch_time_fine(pe_batch* b, int threads, int ctas, float* ms) {
  cudaEvent_t e0, e1;
  PE_CUDA_TRY(cudaEventCreate(&e0));
  PE_CUDA_TRY(cudaEventCreate(&e1));
  PE_CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(int) * kBatchClasses, b->stream));
  PE_CUDA_TRY(cudaEventRecord(e0, b->stream));
  PE_TRY(launch_fine(b, b->stream, threads, ctas));
  PE_CUDA_TRY(cudaEventRecord(e1, b->stream));
  PE_CUDA_TRY(cudaEventSynchronize(e1));
  PE_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->launches += batch_fine_launches(b);
  return PE_OK;
}
