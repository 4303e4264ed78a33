// Dispatch of the fine propagator sweep over the number K of stage-contracted
// columns (kernels in pe_fine_kernels.cuh, instantiated in pe_fine_kXX_YY.cu).
#include <algorithm>
#include <utility>

#include "pe_internal.h"

template <int K>
pe_status fine_launch(pe_ctx* c, int precision, int from_zero, double* out);

namespace {
template <int... Ks>
struct FineTable {
  static pe_status run(int K, pe_ctx* c, int precision, int from_zero, double* out) {
    pe_status st = PE_EINVAL;
    bool hit = ((K == Ks ? (st = fine_launch<Ks>(c, precision, from_zero, out), true) : false) || ...);
    if (!hit) return pe_fail(PE_EINVAL, "stage-contracted columns must be in 1..64");
    return st;
  }
};

template <int... I>
FineTable<(I + 1)...> make_table(std::integer_sequence<int, I...>);
using Table = decltype(make_table(std::make_integer_sequence<int, 2 * PE_MAX_TERMS>{}));
}  // namespace

namespace {
// F^M(U^n) = exp(-lam M dt) U^n + F^M(0) from the cached forced parts
__global__ void affine_fine_kernel(int64_t ndof, int N, const double* __restrict__ EM, const double* __restrict__ U,
                                   const double* __restrict__ Fz, double* __restrict__ Fbar) {
  const int64_t total = (int64_t)N * ndof;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    Fbar[e] = fma(EM[e % ndof], U[e], Fz[e]);
}
}  // namespace

// one sweep of the fine propagator over every slice (the tensor-core engine for the mixed
// form when it was chosen at setup)
static pe_status run_sweep(pe_ctx* c, int precision, int from_zero, double* out) {
  if (precision == PE_MIXED && c->fine_engine == PE_FINE_TC) return launch_fine_tc(c, from_zero, out);
  return Table::run(c->K, c, precision, from_zero, out);
}

pe_status launch_fine_sweep(pe_ctx* c, int precision) {
  if (precision != PE_MIXED) PE_TRY(launch_stage_weights_f64(c));
  if (!c->cache_forced) {
    c->sweeps += 1;
    return run_sweep(c, precision, 0, c->Fbar);
  }
  // affine cache: one sweep from zero per problem and precision, then E^M U + F^M(0)
  if (c->fz_prec != precision) {
    PE_TRY(run_sweep(c, precision, 1, c->Fz));
    c->fz_prec = precision;
    c->sweeps += 1;
  }
  const int threads = 256;
  const int64_t total = (int64_t)c->N * c->g.ndof;
  const int blocks = (int)std::min<int64_t>((total + threads - 1) / threads, 152 * 16);
  affine_fine_kernel<<<blocks, threads, 0, c->stream>>>(c->g.ndof, c->N, c->coefF + (int64_t)(c->q + 1) * c->g.ndof,
                                                        c->U, c->Fz, c->Fbar);
  c->launches += 1;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}
