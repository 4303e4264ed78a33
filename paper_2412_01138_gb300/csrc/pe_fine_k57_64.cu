// Instantiations of the fine-sweep kernels for K = 57..64 stage-contracted columns
// (split across translation units to keep compile times short).
#include "pe_fine_kernels.cuh"

template pe_status fine_launch<57>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<58>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<59>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<60>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<61>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<62>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<63>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<64>(pe_ctx* c, int precision, int from_zero, double* out);
