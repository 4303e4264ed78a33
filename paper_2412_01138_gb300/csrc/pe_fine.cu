// Dispatch of the fine propagator sweep over the number of forcing terms R
// (kernels in pe_fine_kernels.cuh, instantiated in pe_fine_rXX_YY.cu).
#include "pe_internal.h"
#include "pe_sweep_common.cuh"

template <int R>
pe_status fine_launch(pe_ctx* c, int precision);

namespace {
template <int R>
struct FineLaunch {
  static pe_status run(pe_ctx* c, int precision) { return fine_launch<R>(c, precision); }
};
}  // namespace

pe_status launch_fine_sweep(pe_ctx* c, int precision) { return dispatch_R<FineLaunch>(c->R, c, precision); }
