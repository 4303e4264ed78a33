// Instantiations of the fine-sweep kernels for K = 33..40 stage-contracted columns
// (split across translation units to keep compile times short).
#include "pe_fine_kernels.cuh"

template pe_status fine_launch<33>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<34>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<35>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<36>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<37>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<38>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<39>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<40>(pe_ctx* c, int precision, int from_zero, double* out);
