// Instantiations of the fine-sweep kernels for K = 17..24 stage-contracted columns
// (split across translation units to keep compile times short).
#include "pe_fine_kernels.cuh"

template pe_status fine_launch<17>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<18>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<19>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<20>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<21>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<22>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<23>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<24>(pe_ctx* c, int precision, int from_zero, double* out);
