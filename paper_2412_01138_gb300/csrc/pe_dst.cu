// Tensor DST-I along every axis (the simultaneous diagonalisation of Sec. 2.3).
//
// Each axis pass is a dense contraction with the symmetric orthonormal matrix
// S_a[j][k] = sqrt(2/(n_a+1)) sin(pi (j+1)(k+1)/(n_a+1)):
//   last axis   : out[o][j]    = sum_k X[o][k] S[k][j]     (one GEMM, outer x n times n x n)
//   other axes  : out[o][j][i] = sum_k S[j][k] X[o][k][i]  (batched over o)
// Both are served by one shared-memory tiled, strided, batched GEMM.  In
// float64 the kernel is bound by GB300's float64 FMA rate; the transform is
// applied only to initial data and output on the separable-forcing path.
#include "pe_internal.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;

struct GemmArgs {
  int rows, cols, K;
  int64_t batch;
  int64_t sAb, sAi, sAk;
  int64_t sBb, sBk, sBj;
  int64_t sCb, sCi;
};

template <typename T>
__global__ void __launch_bounds__(256) strided_gemm_kernel(const T* __restrict__ A, const T* __restrict__ B,
                                                           T* __restrict__ C, GemmArgs g) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const int64_t b = blockIdx.z;
  const T* Ab = A + b * g.sAb;
  const T* Bb = B + b * g.sBb;
  T acc[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int s = 0; s < TN; ++s) acc[r][s] = T(0);

  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int li = tid / 16 + 16 * r, lk = tid % 16;
      const int gi = i0 + li, gk = k0 + lk;
      As[lk][li] = (gi < g.rows && gk < g.K) ? Ab[gi * g.sAi + gk * g.sAk] : T(0);
      const int bk = tid / 64 + 4 * r, bj = tid % 64;
      const int gk2 = k0 + bk, gj = j0 + bj;
      Bs[bk][bj] = (gk2 < g.K && gj < g.cols) ? Bb[gk2 * g.sBk + gj * g.sBj] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], bv[TN];
#pragma unroll
      for (int r = 0; r < TM; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int s = 0; s < TN; ++s) bv[s] = Bs[kk][tx + 16 * s];
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int s = 0; s < TN; ++s) acc[r][s] = fma(a[r], bv[s], acc[r][s]);
    }
    __syncthreads();
  }
  T* Cb = C + b * g.sCb;
#pragma unroll
  for (int r = 0; r < TM; ++r) {
    const int gi = i0 + ty + 16 * r;
    if (gi >= g.rows) continue;
#pragma unroll
    for (int s = 0; s < TN; ++s) {
      const int gj = j0 + tx + 16 * s;
      if (gj < g.cols) Cb[gi * g.sCi + gj] = acc[r][s];
    }
  }
}

template <typename T>
pe_status dst_axis(const T* S, const T* in, T* out, int64_t outer, int n, int64_t inner, cudaStream_t st) {
  GemmArgs g{};
  if (inner == 1) {
    g.rows = (int)outer; g.cols = n; g.K = n; g.batch = 1;
    g.sAb = 0; g.sAi = n; g.sAk = 1;
    g.sBb = 0; g.sBk = n; g.sBj = 1;
    g.sCb = 0; g.sCi = n;
    if (outer > (int64_t)1 << 30) return pe_fail(PE_EINVAL, "dst: too many pencils");
    dim3 grid((n + BN - 1) / BN, (unsigned)((outer + BM - 1) / BM), 1);
    strided_gemm_kernel<T><<<grid, 256, 0, st>>>(in, S, out, g);
  } else {
    g.rows = n; g.cols = (int)inner; g.K = n; g.batch = outer;
    g.sAb = 0; g.sAi = n; g.sAk = 1;
    g.sBb = (int64_t)n * inner; g.sBk = inner; g.sBj = 1;
    g.sCb = (int64_t)n * inner; g.sCi = inner;
    if (outer > 65535) return pe_fail(PE_EINVAL, "dst: batch too large");
    dim3 grid((unsigned)((inner + BN - 1) / BN), (n + BM - 1) / BM, (unsigned)outer);
    strided_gemm_kernel<T><<<grid, 256, 0, st>>>(S, in, out, g);
  }
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

// Apply S_a along every axis; tmp (ndof elements) may be null when d == 1 and in != out.
template <typename T>
pe_status dst_nd(int d, const int* n, T* const* S, const T* in, T* out, T* tmp, cudaStream_t st) {
  int64_t ndof = 1;
  for (int a = 0; a < d; ++a) ndof *= n[a];
  const T* src = in;
  if (in == out && (d % 2 == 1)) {
    PE_CUDA_TRY(cudaMemcpyAsync(tmp, in, sizeof(T) * ndof, cudaMemcpyDeviceToDevice, st));
    src = tmp;
  }
  for (int a = 0; a < d; ++a) {
    T* dst = ((d - 1 - a) % 2 == 0) ? out : tmp;
    int64_t outer = 1, inner = 1;
    for (int b = 0; b < a; ++b) outer *= n[b];
    for (int b = a + 1; b < d; ++b) inner *= n[b];
    PE_TRY(dst_axis<T>(S[a], src, dst, outer, n[a], inner, st));
    src = dst;
  }
  return PE_OK;
}

template <typename T>
__global__ void dst_matrix_kernel_t(int n, T* S) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (k >= n || j >= n) return;
  const int64_t period = 2 * (int64_t)(n + 1);
  const int64_t m = ((int64_t)(j + 1) * (k + 1)) % period;
  S[(int64_t)j * n + k] = (T)(sqrt(2.0 / (double)(n + 1)) * sinpi((double)m / (double)(n + 1)));
}

template <typename T>
pe_status standalone_dst(int32_t d, const int32_t* n, const T* in, T* out, void* stream) {
  if (d < 1 || d > PE_MAX_D || !n || !in || !out) return pe_fail(PE_EINVAL, "pe_dst: bad arguments");
  int nn[PE_MAX_D];
  int64_t ndof = 1;
  for (int a = 0; a < d; ++a) {
    if (n[a] < 1 || n[a] > 16384) return pe_fail(PE_EINVAL, "pe_dst: n_a must be in 1..16384");
    nn[a] = n[a];
    ndof *= n[a];
  }
  cudaStream_t st = (cudaStream_t)stream;
  T* S[PE_MAX_D] = {nullptr, nullptr, nullptr};
  T* tmp = nullptr;
  pe_status rc = PE_OK;
  for (int a = 0; a < d && rc == PE_OK; ++a) {
    cudaError_t e = cudaMallocAsync((void**)&S[a], sizeof(T) * (size_t)nn[a] * nn[a], st);
    if (e != cudaSuccess) { rc = pe_cuda_fail(e, "cudaMallocAsync(S)"); break; }
    dim3 grid((nn[a] + 127) / 128, nn[a]);
    dst_matrix_kernel_t<T><<<grid, 128, 0, st>>>(nn[a], S[a]);
  }
  if (rc == PE_OK && (d > 1 || in == out)) {
    cudaError_t e = cudaMallocAsync((void**)&tmp, sizeof(T) * (size_t)ndof, st);
    if (e != cudaSuccess) rc = pe_cuda_fail(e, "cudaMallocAsync(tmp)");
  }
  if (rc == PE_OK) rc = dst_nd<T>(d, nn, S, in, out, tmp, st);
  for (int a = 0; a < d; ++a)
    if (S[a]) cudaFreeAsync(S[a], st);
  if (tmp) cudaFreeAsync(tmp, st);
  cudaError_t e = cudaGetLastError();
  if (rc == PE_OK && e != cudaSuccess) rc = pe_cuda_fail(e, "pe_dst");
  return rc;
}

}  // namespace

pe_status dst_axis_f64(const double* S, const double* in, double* out, int64_t outer, int n, int64_t inner,
                       cudaStream_t st) {
  return dst_axis<double>(S, in, out, outer, n, inner, st);
}

pe_status dst_axis_f32(const float* S, const float* in, float* out, int64_t outer, int n, int64_t inner,
                       cudaStream_t st) {
  return dst_axis<float>(S, in, out, outer, n, inner, st);
}

pe_status dst_nd_f64(pe_ctx* c, const double* in, double* out) {
  c->launches += c->g.d;
  return dst_nd<double>(c->g.d, c->g.n, c->S, in, out, c->work1, c->stream);
}

extern "C" pe_status pe_dst(int32_t d, const int32_t* n, const double* in, double* out, void* stream) {
  return standalone_dst<double>(d, n, in, out, stream);
}

extern "C" pe_status pe_dst_f32(int32_t d, const int32_t* n, const float* in, float* out, void* stream) {
  return standalone_dst<float>(d, n, in, out, stream);
}
