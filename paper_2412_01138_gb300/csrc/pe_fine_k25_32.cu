// Instantiations of the fine-sweep kernels for K = 25..32 stage-contracted columns
// (split across translation units to keep compile times short).
#include "pe_fine_kernels.cuh"

template pe_status fine_launch<25>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<26>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<27>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<28>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<29>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<30>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<31>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<32>(pe_ctx* c, int precision, int from_zero, double* out);
