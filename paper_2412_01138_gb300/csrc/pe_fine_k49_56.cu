// Instantiations of the fine-sweep kernels for K = 49..56 stage-contracted columns
// (split across translation units to keep compile times short).
#include "pe_fine_kernels.cuh"

template pe_status fine_launch<49>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<50>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<51>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<52>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<53>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<54>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<55>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<56>(pe_ctx* c, int precision, int from_zero, double* out);
