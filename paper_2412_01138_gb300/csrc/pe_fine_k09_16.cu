// Instantiations of the fine-sweep kernels for K = 9..16 stage-contracted columns
// (split across translation units to keep compile times short).
#include "pe_fine_kernels.cuh"

template pe_status fine_launch<9>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<10>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<11>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<12>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<13>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<14>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<15>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<16>(pe_ctx* c, int precision, int from_zero, double* out);
