// Instantiations of the fine-sweep kernels for K = 41..48 stage-contracted columns
// (split across translation units to keep compile times short).
#include "pe_fine_kernels.cuh"

template pe_status fine_launch<41>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<42>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<43>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<44>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<45>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<46>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<47>(pe_ctx* c, int precision, int from_zero, double* out);
template pe_status fine_launch<48>(pe_ctx* c, int precision, int from_zero, double* out);
