// Measurement and self-check entry points (no counterpart in the paper):
//
//   pe_measure_fma_peak   the FMA throughput of the CUDA cores in float64 or float32, measured
//                         by a kernel of independent FMA chains, so that the ALU-bound fine
//                         kernels can be quoted against a measured peak beside the one derived
//                         from unit counts and the clock;
//   pe_probe_wait_timeout the bounded mbarrier wait of the tensor-core kernels, run in a tiny
//                         kernel on a barrier that nothing ever arrives at (no tensor-core
//                         instruction and no copy in flight), with a caller-given budget: the
//                         wait gives up, the kernel records the expiry in a status word and
//                         returns, and the host reports PE_ETIMEOUT exactly as it does for the
//                         production kernels;
//   pe_probe_widen_f32    the integer float32 -> float64 widening of the mixed form's coarse
//                         sweeps applied to a caller's array, so that a test can compare it bit
//                         for bit with the hardware conversion.
#include <stdio.h>

#include <algorithm>

#include "pe_internal.h"
#include "pe_tc_common.cuh"

namespace {

constexpr int kFmaChains = 8;  // independent accumulators per thread (covers the FMA latency)

template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T a, T b, int iters, T* __restrict__ sink) {
  T x[kFmaChains];
#pragma unroll
  for (int i = 0; i < kFmaChains; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i) x[i] = fma(x[i], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kFmaChains; ++i) s += x[i];
  // never true for the arguments used (|x| stays near b / (1 - a)); keeps the chains live
  if (s == (T)-1.0) sink[blockIdx.x] = s;
}

// status word: 0 = the barrier completed, 1 = the bounded wait expired
__global__ void wait_probe_kernel(long long budget, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // nothing arrives at `bar`: phase 0 never completes
    *status = mbar_wait_for(&bar, 0u, budget) ? 0 : 1;
  }
}

template <typename T>
pe_status fma_peak(double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  PE_CUDA_TRY(cudaGetDevice(&dev));
  PE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 8;  // 2048 threads per SM
  // float64 runs at 1/64 of the float32 rate on this part: fewer iterations for a similar time
  const int iters = sizeof(T) == 8 ? 4096 : 131072;
  T* sink = nullptr;
  PE_CUDA_TRY(cudaMallocAsync((void**)&sink, sizeof(T) * blocks, st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  pe_status rc = PE_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = pe_cuda_fail(cudaGetLastError(), "pe_measure_fma_peak: events");
  float best = 0.f;
  const T a = (T)0.999999, b = (T)1e-6;
  for (int rep = 0; rep < 6 && rc == PE_OK; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, st);
    fma_peak_kernel<T><<<blocks, threads, 0, st>>>(a, b, iters, sink);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = pe_cuda_fail(e, "pe_measure_fma_peak: kernel");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(sink, st);
  if (rc != PE_OK) return rc;
  const double flops = 2.0 * kFmaChains * (double)iters * threads * blocks;
  *tflops = flops / (best * 1e-3) / 1e12;
  return PE_OK;
}

}  // namespace

extern "C" pe_status pe_measure_fma_peak(int32_t precision, double* tflops_out, void* stream) {
  if (!tflops_out) return pe_fail(PE_EINVAL, "pe_measure_fma_peak: tflops_out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == PE_FP64) return fma_peak<double>(tflops_out, st);
  if (precision == PE_MIXED) return fma_peak<float>(tflops_out, st);
  return pe_fail(PE_EINVAL, "pe_measure_fma_peak: precision must be PE_FP64 or PE_MIXED (float32)");
}

namespace {
__global__ void widen_probe_kernel(const float* __restrict__ x, double* __restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = widen_f32(x[i]);
}
}  // namespace

extern "C" pe_status pe_probe_widen_f32(const float* x, double* y, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return pe_fail(PE_EINVAL, "pe_probe_widen_f32: bad arguments");
  if (n == 0) return PE_OK;
  const int64_t blocks = (n + 255) / 256;
  if (blocks > 0x7FFFFFFFLL) return pe_fail(PE_EINVAL, "pe_probe_widen_f32: n too large");
  widen_probe_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(x, y, n);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

extern "C" pe_status pe_probe_wait_timeout(int64_t budget_cycles, void* stream) {
  if (budget_cycles < 1 || budget_cycles > 100000000LL)
    return pe_fail(PE_EINVAL, "pe_probe_wait_timeout: budget must be in 1..1e8 cycles");
  cudaStream_t st = (cudaStream_t)stream;
  int* dstatus = nullptr;
  PE_CUDA_TRY(cudaMallocAsync((void**)&dstatus, sizeof(int), st));
  int hstatus = -1;
  wait_probe_kernel<<<1, 32, 0, st>>>((long long)budget_cycles, dstatus);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hstatus, dstatus, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(dstatus, st);
  if (e != cudaSuccess) return pe_cuda_fail(e, "pe_probe_wait_timeout");
  if (hstatus == 1) return pe_fail(PE_ETIMEOUT, "pe_probe_wait_timeout: the bounded mbarrier wait expired");
  if (hstatus == 0) return PE_OK;
  return pe_fail(PE_ECUDA, "pe_probe_wait_timeout: no status written");
}
