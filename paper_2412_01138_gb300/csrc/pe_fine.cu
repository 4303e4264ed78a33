// Dispatch of the fine propagator sweep over the number K of stage-contracted
// columns (kernels in pe_fine_kernels.cuh, instantiated in pe_fine_kXX_YY.cu).
#include <utility>

#include "pe_internal.h"

template <int K>
pe_status fine_launch(pe_ctx* c, int precision);

namespace {
template <int... Ks>
struct FineTable {
  static pe_status run(int K, pe_ctx* c, int precision) {
    pe_status st = PE_EINVAL;
    bool hit = ((K == Ks ? (st = fine_launch<Ks>(c, precision), true) : false) || ...);
    if (!hit) return pe_fail(PE_EINVAL, "stage-contracted columns must be in 1..64");
    return st;
  }
};

template <int... I>
FineTable<(I + 1)...> make_table(std::integer_sequence<int, I...>);
using Table = decltype(make_table(std::make_integer_sequence<int, 2 * PE_MAX_TERMS>{}));
}  // namespace

pe_status launch_fine_sweep(pe_ctx* c, int precision) { return Table::run(c->K, c, precision); }
