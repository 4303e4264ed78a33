// Instantiations of the fine-sweep kernels for K = 1..8 stage-contracted columns
// (split across translation units to keep compile times short).
#include "pe_fine_kernels.cuh"

template pe_status fine_launch<1>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<2>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<3>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<4>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<5>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<6>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<7>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<8>(pe_ctx* c, int precision, int from_zero, double* out);
