// Tensor DST-I along every axis (the simultaneous diagonalisation of Sec. 2.3).
//
// Each axis pass is a dense contraction with the symmetric orthonormal matrix
// S_a[j][k] = sqrt(2/(n_a+1)) sin(pi (j+1)(k+1)/(n_a+1)):
//   last axis   : out[o][j]    = sum_k X[o][k] S[k][j]     (one GEMM, outer x n times n x n)
//   other axes  : out[o][j][i] = sum_k S[j][k] X[o][k][i]  (batched over o)
// Two kernels serve every axis pass:
//  * n + 1 = 2^k (n <= 1023): a radix-2 FFT in shared memory.  Two real pencils
//    x, y are packed as z = x + i y; the odd extension of z over 2(n+1) points is
//    transformed by an in-place decimation-in-time FFT (bit-reversed load), and
//    DST(x)_k = -Im V_k / 2, DST(y)_k = Re V_k / 2.  About 5 log2(2n+2) flops per
//    element instead of the 2n of the matrix form.
//  * any other n: a shared-memory tiled, strided, batched GEMM with the matrix S_a
//    (tile shape chosen so that the grid covers the GPU).
#include <algorithm>
#include <mutex>

#include "pe_internal.h"

namespace {

constexpr int BK = 16, TM = 4, TN = 4;

struct GemmArgs {
  int rows, cols, K;
  int64_t batch;
  int64_t sAb, sAi, sAk;
  int64_t sBb, sBk, sBj;
  int64_t sCb, sCi;
};

// BM x BN output tile, (BM/TM) x (BN/TN) threads, each owning a TM x TN block
// (rows ty + r*(BM/TM), columns tx + s*(BN/TN)).
template <typename T, int BM, int BN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) strided_gemm_kernel(const T* __restrict__ A,
                                                                          const T* __restrict__ B,
                                                                          T* __restrict__ C, GemmArgs g) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int TX = BN / TN;  // threads along a row of the tile
  constexpr int TY = BM / TM;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
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
    for (int e = tid; e < BM * BK; e += NT) {
      const int li = e / BK, lk = e % BK;
      const int gi = i0 + li, gk = k0 + lk;
      As[lk][li] = (gi < g.rows && gk < g.K) ? Ab[gi * g.sAi + gk * g.sAk] : T(0);
    }
    for (int e = tid; e < BK * BN; e += NT) {
      const int bk = e / BN, bj = e % BN;
      const int gk2 = k0 + bk, gj = j0 + bj;
      Bs[bk][bj] = (gk2 < g.K && gj < g.cols) ? Bb[gk2 * g.sBk + gj * g.sBj] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], bv[TN];
#pragma unroll
      for (int r = 0; r < TM; ++r) a[r] = As[kk][ty + TY * r];
#pragma unroll
      for (int s = 0; s < TN; ++s) bv[s] = Bs[kk][tx + TX * s];
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
    const int gi = i0 + ty + TY * r;
    if (gi >= g.rows) continue;
#pragma unroll
    for (int s = 0; s < TN; ++s) {
      const int gj = j0 + tx + TX * s;
      if (gj < g.cols) Cb[gi * g.sCi + gj] = acc[r][s];
    }
  }
}

template <typename T, int BM, int BN>
pe_status gemm_axis(const T* S, const T* in, T* out, int64_t outer, int n, int64_t inner, cudaStream_t st) {
  GemmArgs g{};
  constexpr int NT = (BM / TM) * (BN / TN);
  if (inner == 1) {
    g.rows = (int)outer; g.cols = n; g.K = n; g.batch = 1;
    g.sAb = 0; g.sAi = n; g.sAk = 1;
    g.sBb = 0; g.sBk = n; g.sBj = 1;
    g.sCb = 0; g.sCi = n;
    if (outer > (int64_t)1 << 30) return pe_fail(PE_EINVAL, "dst: too many pencils");
    dim3 grid((n + BN - 1) / BN, (unsigned)((outer + BM - 1) / BM), 1);
    strided_gemm_kernel<T, BM, BN><<<grid, NT, 0, st>>>(in, S, out, g);
  } else {
    g.rows = n; g.cols = (int)inner; g.K = n;
    g.sAb = 0; g.sAi = n; g.sAk = 1;
    g.sBb = (int64_t)n * inner; g.sBk = inner; g.sBj = 1;
    g.sCb = (int64_t)n * inner; g.sCi = inner;
    // the batch runs in grid.z, at most 65535 per launch
    for (int64_t b0 = 0; b0 < outer; b0 += 65535) {
      const int64_t nb = std::min<int64_t>(65535, outer - b0);
      g.batch = nb;
      dim3 grid((unsigned)((inner + BN - 1) / BN), (n + BM - 1) / BM, (unsigned)nb);
      strided_gemm_kernel<T, BM, BN><<<grid, NT, 0, st>>>(S, in + b0 * g.sBb, out + b0 * g.sCb, g);
    }
  }
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

// ---------------------------------------------------------------------------
// FFT form (n + 1 a power of two)
// ---------------------------------------------------------------------------
template <typename T>
struct Cplx {
  T re, im;
};

template <typename T>
__device__ inline void sincospi_t(T x, T* s, T* c);
template <>
__device__ inline void sincospi_t<double>(double x, double* s, double* c) { sincospi(x, s, c); }
template <>
__device__ inline void sincospi_t<float>(float x, float* s, float* c) { sincospif(x, s, c); }

// One CTA transforms `pairs` pencil pairs (2*pairs consecutive pencils) of length n,
// L = 2(n+1) = 2^logL.  Pencil p lives at o*n*inner + j*inner + i with o = p / inner,
// i = p % inner.  Dynamic shared memory: pairs*L complex values + L/2 twiddles.
template <typename T>
__global__ void __launch_bounds__(256) dst_fft_kernel(const T* __restrict__ in, T* __restrict__ out, int n,
                                                      int logL, int64_t inner, int64_t npencils, int pairs,
                                                      T scale, const Cplx<T>* __restrict__ twg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 1 << logL;
  Cplx<T>* buf = reinterpret_cast<Cplx<T>*>(smem_raw);
  Cplx<T>* tw = buf + (size_t)pairs * L;
  const int tid = threadIdx.x, B = blockDim.x;
  const int64_t p0 = (int64_t)blockIdx.x * (2 * pairs);
  for (int k = tid; k < L / 2; k += B) tw[k] = twg[k];  // e^{-2 pi i k / L}
  // zero the two fixed points of the odd extension (positions 0 and n+1)
  const int np1 = n + 1;
  const int shift = 32 - logL;
  for (int q = tid; q < pairs; q += B) {
    buf[(size_t)q * L + 0] = Cplx<T>{T(0), T(0)};
    buf[(size_t)q * L + (__brev((unsigned)np1) >> shift)] = Cplx<T>{T(0), T(0)};
  }
  // load: consecutive threads take consecutive pencils (coalesced when inner > 1)
  // or consecutive elements (inner == 1)
  const int npen = 2 * pairs;
  for (int e = tid; e < npen * n; e += B) {
    int pl, j;
    if (inner == 1) {
      pl = e / n;
      j = e - pl * n;
    } else {
      j = e / npen;
      pl = e - j * npen;
    }
    const int64_t p = p0 + pl;
    T v = T(0);
    if (p < npencils) {
      const int64_t o = p / inner, i = p - o * inner;
      v = in[o * (int64_t)n * inner + (int64_t)j * inner + i];
    }
    const int q = pl >> 1;
    const int jj = j + 1;  // 1-based position in the extension
    const unsigned a = __brev((unsigned)jj) >> shift;
    const unsigned b = __brev((unsigned)(L - jj)) >> shift;
    Cplx<T>* row = buf + (size_t)q * L;
    if (pl & 1) {
      row[a].im = v;
      row[b].im = -v;
    } else {
      row[a].re = v;
      row[b].re = -v;
    }
  }
  __syncthreads();
  // radix-2 decimation-in-time stages
  for (int s = 1; s <= logL; ++s) {
    const int half = 1 << (s - 1);
    const int tstride = L >> s;  // twiddle index stride
    for (int bfly = tid; bfly < pairs * (L / 2); bfly += B) {
      const int q = bfly / (L / 2);
      const int r = bfly - q * (L / 2);
      const int grp = r / half, pos = r - grp * half;
      const int i0 = grp * 2 * half + pos, i1 = i0 + half;
      Cplx<T>* row = buf + (size_t)q * L;
      const Cplx<T> w = tw[pos * tstride];
      const Cplx<T> u = row[i0], x = row[i1];
      const T tr = w.re * x.re - w.im * x.im;
      const T ti = w.re * x.im + w.im * x.re;
      row[i0] = Cplx<T>{u.re + tr, u.im + ti};
      row[i1] = Cplx<T>{u.re - tr, u.im - ti};
    }
    __syncthreads();
  }
  // store: DST(x)_k = -Im V_k / 2, DST(y)_k = Re V_k / 2, k = 1..n, times sqrt(2/(n+1))
  for (int e = tid; e < npen * n; e += B) {
    int pl, k;
    if (inner == 1) {
      pl = e / n;
      k = e - pl * n;
    } else {
      k = e / npen;
      pl = e - k * npen;
    }
    const int64_t p = p0 + pl;
    if (p >= npencils) continue;
    const Cplx<T> V = buf[(size_t)(pl >> 1) * L + (k + 1)];
    const T val = (pl & 1) ? V.re * scale : -V.im * scale;
    const int64_t o = p / inner, i = p - o * inner;
    out[o * (int64_t)n * inner + (int64_t)k * inner + i] = val;
  }
}

inline bool fft_size_ok(int n, int* logL) {
  const int np1 = n + 1;
  if (np1 < 2 || np1 > 1024 || (np1 & (np1 - 1)) != 0) return false;
  int l = 0;
  while ((1 << l) < 2 * np1) ++l;
  *logL = l;
  return true;
}

template <typename T>
__global__ void twiddle_kernel(int L, Cplx<T>* tw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L / 2) return;
  T s, c;
  sincospi_t<T>((T)(2 * k) / (T)L, &s, &c);
  tw[k].re = c;
  tw[k].im = -s;
}

// Twiddles e^{-2 pi i k/L}, k < L/2, of every FFT length 2(n+1) <= 2048 (L = 2^1..2^11),
// built once per process and device-resident: table for length L starts at L/2 - 1.
template <typename T>
const Cplx<T>* twiddles(int logL, cudaStream_t st) {
  static Cplx<T>* table[64] = {nullptr};
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!table[dev]) {
    Cplx<T>* p = nullptr;
    if (cudaMalloc((void**)&p, sizeof(Cplx<T>) * 2048) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (int l = 1; l <= 11; ++l) {
      const int L = 1 << l;
      twiddle_kernel<T><<<(L / 2 + 255) / 256, 256, 0, st>>>(L, p + (L / 2 - 1));
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(p);
      return nullptr;
    }
    table[dev] = p;
  }
  const int L = 1 << logL;
  return table[dev] + (L / 2 - 1);
}

template <typename T>
pe_status fft_axis(const T* in, T* out, int64_t outer, int n, int64_t inner, int logL, cudaStream_t st) {
  const int L = 1 << logL;
  const int64_t npencils = outer * inner;
  const Cplx<T>* tw = twiddles<T>(logL, st);
  if (!tw) return pe_fail(PE_ECUDA, "dst: twiddle table allocation failed");
  // pencil pairs per CTA: as many as keep >= 2 CTAs per SM, bounded by shared memory
  int max_pairs = (int)((48 * 1024) / ((size_t)L * sizeof(Cplx<T>)));
  max_pairs = max_pairs < 1 ? 1 : (max_pairs > 16 ? 16 : max_pairs);
  int64_t pairs64 = (npencils + 1) / 2 / (2 * 152);
  int pairs = (int)(pairs64 < 1 ? 1 : (pairs64 > max_pairs ? max_pairs : pairs64));
  const int64_t want_ctas = (npencils + 2 * pairs - 1) / (2 * pairs);
  const size_t smem = sizeof(Cplx<T>) * ((size_t)pairs * L + L / 2);
  if (smem > 48 * 1024) {
    PE_CUDA_TRY(cudaFuncSetAttribute(dst_fft_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  const T scale = (T)(0.5 * sqrt(2.0 / (double)(n + 1)));
  const int threads = L / 2 * pairs >= 256 ? 256 : (L / 2 * pairs >= 128 ? 128 : 64);
  dst_fft_kernel<T><<<(unsigned)want_ctas, threads, smem, st>>>(in, out, n, logL, inner, npencils, pairs, scale, tw);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

template <typename T>
pe_status dst_axis(const T* S, const T* in, T* out, int64_t outer, int n, int64_t inner, cudaStream_t st) {
  int logL = 0;
  if (fft_size_ok(n, &logL)) return fft_axis<T>(in, out, outer, n, inner, logL, st);
  // matrix form: large tiles when they still give >= 2 CTAs per SM, else small ones
  const int64_t rows = inner == 1 ? outer : n;
  const int64_t cols = inner == 1 ? n : inner;
  const int64_t batch = inner == 1 ? 1 : outer;
  const int64_t big = ((rows + 63) / 64) * ((cols + 63) / 64) * batch;
  if (big >= 2 * 152) return gemm_axis<T, 64, 64>(S, in, out, outer, n, inner, st);
  return gemm_axis<T, 32, 32>(S, in, out, outer, n, inner, st);
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

// ---------------------------------------------------------------------------
// pe_dst_noalloc: the same transform with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is being
// captured (an allocation would break or be recorded into the capture), callers
// that own a fixed memory pool and forbid the runtime allocator, and hosts whose
// device memory is fully reserved up front.  This entry point keeps every scratch
// buffer of the transform (the ping-pong array, the DST-I matrices of axes without
// an FFT length, the FFT twiddles) in one file-scope device array.  Every GPU that
// loads the library holds that array (about 14.7 MB) until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoallocMaxNdof = (int64_t)1 << 20;     // ping-pong capacity (doubles)
constexpr int kNoallocMaxMatrixN = 512;                   // axes on the matrix path
constexpr int64_t kNoallocSlot = (int64_t)kNoallocMaxMatrixN * kNoallocMaxMatrixN;  // per axis
constexpr int64_t kNoallocDoubles = kNoallocMaxNdof + PE_MAX_D * kNoallocSlot;

static __device__ __align__(256) double g_dst_scratch[kNoallocDoubles];

// Device address of g_dst_scratch on the current device, looked up once per device.
pe_status noalloc_scratch(double** out) {
  static double* addr[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  PE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return pe_fail(PE_EINVAL, "pe_dst_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_dst_scratch);
    if (e != cudaSuccess) return pe_cuda_fail(e, "pe_dst_noalloc: cudaGetSymbolAddress");
    addr[dev] = (double*)p;
  }
  *out = addr[dev];
  return PE_OK;
}

// FFT pass with caller-provided twiddles (tw: L/2 values for L = 2^logL).
pe_status fft_axis_tw(const double* in, double* out, int64_t outer, int n, int64_t inner, int logL,
                      const Cplx<double>* tw, cudaStream_t st) {
  const int L = 1 << logL;
  const int64_t npencils = outer * inner;
  int max_pairs = (int)((48 * 1024) / ((size_t)L * sizeof(Cplx<double>)));
  max_pairs = max_pairs < 1 ? 1 : (max_pairs > 16 ? 16 : max_pairs);
  int64_t pairs64 = (npencils + 1) / 2 / (2 * 152);
  const int pairs = (int)(pairs64 < 1 ? 1 : (pairs64 > max_pairs ? max_pairs : pairs64));
  const int64_t ctas = (npencils + 2 * pairs - 1) / (2 * pairs);
  const size_t smem = sizeof(Cplx<double>) * ((size_t)pairs * L + L / 2);
  if (smem > 48 * 1024)
    PE_CUDA_TRY(cudaFuncSetAttribute(dst_fft_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  const int threads = L / 2 * pairs >= 256 ? 256 : (L / 2 * pairs >= 128 ? 128 : 64);
  dst_fft_kernel<double><<<(unsigned)ctas, threads, smem, st>>>(in, out, n, logL, inner, npencils, pairs,
                                                                0.5 * sqrt(2.0 / (double)(n + 1)), tw);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

}  // namespace

extern "C" pe_status pe_dst_noalloc(int32_t d, const int32_t* n, const double* in, double* out, void* stream) {
  if (d < 1 || d > PE_MAX_D || !n || !in || !out) return pe_fail(PE_EINVAL, "pe_dst_noalloc: bad arguments");
  int64_t ndof = 1;
  int logL[PE_MAX_D] = {0, 0, 0};
  bool fft[PE_MAX_D] = {false, false, false};
  for (int a = 0; a < d; ++a) {
    if (n[a] < 1) return pe_fail(PE_EINVAL, "pe_dst_noalloc: n_a must be >= 1");
    fft[a] = fft_size_ok(n[a], &logL[a]);
    if (!fft[a] && n[a] > kNoallocMaxMatrixN)
      return pe_fail(PE_EINVAL, "pe_dst_noalloc: an axis with n+1 not a power of two must have n <= 512 "
                                "(its DST-I matrix must fit the built-in scratch array)");
    ndof *= n[a];
    if (ndof > kNoallocMaxNdof)
      return pe_fail(PE_EINVAL, "pe_dst_noalloc: at most 1048576 values (the built-in scratch array's capacity)");
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* scratch = nullptr;
  PE_TRY(noalloc_scratch(&scratch));
  double* tmp = scratch;  // ping-pong buffer, kNoallocMaxNdof values
  // per-axis slot: the DST-I matrix (matrix path) or the twiddles (FFT path); every value the
  // passes read is written here first, so nothing in the array has to start at zero
  for (int a = 0; a < d; ++a) {
    double* slot = scratch + kNoallocMaxNdof + (int64_t)a * kNoallocSlot;
    if (fft[a]) {
      const int L = 1 << logL[a];
      twiddle_kernel<double><<<(L / 2 + 255) / 256, 256, 0, st>>>(L, reinterpret_cast<Cplx<double>*>(slot));
    } else {
      dim3 grid((n[a] + 127) / 128, n[a]);
      dst_matrix_kernel_t<double><<<grid, 128, 0, st>>>(n[a], slot);
    }
  }
  PE_CUDA_TRY(cudaGetLastError());
  // passes: a pass never writes the array it reads (in may alias out)
  const double* src = in;
  if (in == out && (d % 2 == 1)) {
    PE_CUDA_TRY(cudaMemcpyAsync(tmp, in, sizeof(double) * ndof, cudaMemcpyDeviceToDevice, st));
    src = tmp;
  }
  for (int a = 0; a < d; ++a) {
    double* dst = ((d - 1 - a) % 2 == 0) ? out : tmp;
    int64_t outer = 1, inner = 1;
    for (int b = 0; b < a; ++b) outer *= n[b];
    for (int b = a + 1; b < d; ++b) inner *= n[b];
    double* slot = scratch + kNoallocMaxNdof + (int64_t)a * kNoallocSlot;
    if (fft[a]) {
      PE_TRY(fft_axis_tw(src, dst, outer, n[a], inner, logL[a], reinterpret_cast<const Cplx<double>*>(slot), st));
    } else {
      const int64_t rows = inner == 1 ? outer : n[a];
      const int64_t cols = inner == 1 ? n[a] : inner;
      const int64_t batch = inner == 1 ? 1 : outer;
      const int64_t big = ((rows + 63) / 64) * ((cols + 63) / 64) * batch;
      if (big >= 2 * 152) PE_TRY((gemm_axis<double, 64, 64>(slot, src, dst, outer, n[a], inner, st)));
      else PE_TRY((gemm_axis<double, 32, 32>(slot, src, dst, outer, n[a], inner, st)));
    }
    src = dst;
  }
  return PE_OK;
}
