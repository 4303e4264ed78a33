// Tensor DST-I along every axis (the simultaneous diagonalisation of Sec. 2.3).
//
// Each axis pass is a dense contraction with the symmetric orthonormal matrix
// S_a[j][k] = sqrt(2/(n_a+1)) sin(pi (j+1)(k+1)/(n_a+1)):
//   last axis   : out[o][j]    = sum_k X[o][k] S[k][j]     (one GEMM, outer x n times n x n)
//   other axes  : out[o][j][i] = sum_k S[j][k] X[o][k][i]  (batched over o)
// Two kernel families serve every axis pass:
//  * n + 1 = 2^k (n <= 1023): an FFT.  Two real pencils x, y are packed as
//    z = x + i y; the odd extension of z over 2(n+1) points is Fourier
//    transformed, and DST(x)_k = -Im V_k / 2, DST(y)_k = Re V_k / 2.  About
//    5 log2(2n+2) flops per element instead of the 2n of the matrix form.  In
//    float64 with n + 1 >= 128 the half-length form folds each pencil so that the
//    pair needs a complex FFT of n + 1 points only (dst_half_warp_kernel); float32
//    and shorter float64 pencils transform the full odd extension with one warp per
//    pencil pair (dst_fft_warp_kernel); both run self-sorting radix-4..32 passes.
//    Pencils with n + 1 < 16 use a block-wide radix-2 kernel (dst_fft_kernel).
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
  pdl_wait();
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
  // or consecutive elements (inner == 1); the (pencil, element) walk advances by
  // carries instead of a division per element
  const int npen = 2 * pairs;
  const int fast = inner == 1 ? n : npen;  // extent of the fast index
  int e_hi = tid / fast, e_lo = tid - (tid / fast) * fast;
  const int step_hi = B / fast, step_lo = B - (B / fast) * fast;
  for (int e = tid; e < npen * n; e += B) {
    const int pl = inner == 1 ? e_hi : e_lo;
    const int j = inner == 1 ? e_lo : e_hi;
    e_lo += step_lo;
    e_hi += step_hi;
    if (e_lo >= fast) {
      e_lo -= fast;
      ++e_hi;
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
  // radix-2 decimation-in-time stages (L and half are powers of two: shifts and masks)
  for (int s = 1; s <= logL; ++s) {
    const int half = 1 << (s - 1);
    const int tstride = L >> s;  // twiddle index stride
    for (int bfly = tid; bfly < pairs * (L / 2); bfly += B) {
      const int q = bfly >> (logL - 1);
      const int r = bfly & (L / 2 - 1);
      const int grp = r >> (s - 1), pos = r & (half - 1);
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
  e_hi = tid / fast;
  e_lo = tid - e_hi * fast;
  for (int e = tid; e < npen * n; e += B) {
    const int pl = inner == 1 ? e_hi : e_lo;
    const int k = inner == 1 ? e_lo : e_hi;
    e_lo += step_lo;
    e_hi += step_hi;
    if (e_lo >= fast) {
      e_lo -= fast;
      ++e_hi;
    }
    const int64_t p = p0 + pl;
    if (p >= npencils) continue;
    const Cplx<T> V = buf[(size_t)(pl >> 1) * L + (k + 1)];
    const T val = (pl & 1) ? V.re * scale : -V.im * scale;
    const int64_t o = p / inner, i = p - o * inner;
    out[o * (int64_t)n * inner + (int64_t)k * inner + i] = val;
  }
}

// Half-length DST-I of one pencil pair per CTA, for float64 passes with few pencils: the
// fold, complex FFT of N = n + 1 points and unfold of the half-length form (see the warp
// kernel below), with the radix-2 butterflies and the prefix sum spread over the CTA so
// that all four SM sub-partitions' float64 units work on the pair (about half the float64
// work of the odd extension).  Shared memory: the pair (N + 1 values), the FFT buffer (N)
// and the warp totals of the scan.
// The CTA's pencil pair (a at in_a, b at in_b, stride `inner`, b absent when !has_b) in
// x[1..n] on return: x[m] = (F^a_m, F^b_m), the unscaled sine sums.  x, z and wsum are
// shared buffers of N + 1, N and 8 complex values.
template <typename T>
__device__ __forceinline__ void half_block_pair(const T* __restrict__ in_a, const T* __restrict__ in_b, bool has_b,
                                                int64_t inner, int n, int logN, const Cplx<T>* __restrict__ tw,
                                                const T* __restrict__ sinN, Cplx<T>* x, Cplx<T>* z, Cplx<T>* wsum) {
  const int N = 1 << logN, H = N / 2;
  const int tid = threadIdx.x, B = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int j = tid; j <= N; j += B) {
    T va = T(0), vb = T(0);
    if (j >= 1 && j <= n) {
      va = in_a[(int64_t)(j - 1) * inner];
      if (has_b) vb = in_b[(int64_t)(j - 1) * inner];
    }
    x[j] = Cplx<T>{va, vb};
  }
  __syncthreads();
  // fold y_j = sin(pi j/N)(x_j + x_{N-j}) + (x_j - x_{N-j})/2 of both pencils, z = y^a + i y^b
  const int shift = 32 - logN;
  for (int j = tid; j < N; j += B) {
    const Cplx<T> xj = x[j];
    const Cplx<T> xm = j == 0 ? Cplx<T>{T(0), T(0)} : x[N - j];
    const T sj = sinN[j];
    z[__brev((unsigned)j) >> shift] = Cplx<T>{sj * (xj.re + xm.re) + T(0.5) * (xj.re - xm.re),
                                              sj * (xj.im + xm.im) + T(0.5) * (xj.im - xm.im)};
  }
  __syncthreads();
  // radix-2 decimation in time, twiddles e^{-2 pi i k/N}
  for (int st = 1; st <= logN; ++st) {
    const int half = 1 << (st - 1), tstride = N >> st;
    for (int b = tid; b < H; b += B) {
      const int grp = b >> (st - 1), pos = b & (half - 1);
      const int i0 = grp * 2 * half + pos, i1 = i0 + half;
      const Cplx<T> w = tw[pos * tstride];
      const Cplx<T> u = z[i0], v = z[i1];
      const T tr = w.re * v.re - w.im * v.im;
      const T ti = w.re * v.im + w.im * v.re;
      z[i0] = Cplx<T>{u.re + tr, u.im + ti};
      z[i1] = Cplx<T>{u.re - tr, u.im - ti};
    }
    __syncthreads();
  }
  // unfold: F_{2k} = I_k, F_{2k+1} = R_0/2 + R_1 + ... + R_k (k < N/2) for both pencils;
  // thread tid owns the contiguous k = tid*C .. tid*C + C - 1
  constexpr int CMAX = 2;  // N <= 1024 and 256 threads
  const int C = (H + B - 1) / B;
  T ia[CMAX], ib[CMAX], sa[CMAX], sb[CMAX];
  T ta = T(0), tb = T(0);
#pragma unroll
  for (int c = 0; c < CMAX; ++c) {
    const int k = tid * C + c;
    ia[c] = ib[c] = T(0);
    if (c < C && k < H) {
      const Cplx<T> Z = z[k];
      const Cplx<T> Wm = z[(N - k) & (N - 1)];
      T ra = T(0.5) * (Z.re + Wm.re), rb = T(0.5) * (Z.im + Wm.im);
      ia[c] = T(0.5) * (Wm.im - Z.im);
      ib[c] = T(0.5) * (Z.re - Wm.re);
      if (k == 0) {
        ra *= T(0.5);
        rb *= T(0.5);
      }
      ta += ra;
      tb += rb;
    }
    sa[c] = ta;
    sb[c] = tb;
  }
  // exclusive scan of the thread totals: within the warp by shuffles, then over the warps
  T ea = ta, eb = tb;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T ua = __shfl_up_sync(0xffffffffu, ea, d), ub = __shfl_up_sync(0xffffffffu, eb, d);
    if (lane >= d) {
      ea += ua;
      eb += ub;
    }
  }
  if (lane == 31) wsum[warp] = Cplx<T>{ea, eb};
  __syncthreads();
  T pre_a = T(0), pre_b = T(0);
  for (int w = 0; w < warp; ++w) {
    pre_a += wsum[w].re;
    pre_b += wsum[w].im;
  }
  ea += pre_a - ta;
  eb += pre_b - tb;
#pragma unroll
  for (int c = 0; c < CMAX; ++c) {
    const int k = tid * C + c;
    if (c < C && k < H) {
      if (k > 0) x[2 * k] = Cplx<T>{ia[c], ib[c]};
      x[2 * k + 1] = Cplx<T>{sa[c] + ea, sb[c] + eb};
    }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) dst_half_block_kernel(const T* __restrict__ in, T* __restrict__ out, int n,
                                                             int logN, int64_t inner, int64_t npencils, T scale,
                                                             const Cplx<T>* __restrict__ tw,
                                                             const T* __restrict__ sinN) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 1 << logN;
  Cplx<T>* x = reinterpret_cast<Cplx<T>*>(smem_raw);
  Cplx<T>* z = x + (N + 1);
  Cplx<T>* wsum = z + N;
  const int64_t pa = 2 * (int64_t)blockIdx.x, pb = pa + 1;
  const bool has_b = pb < npencils;
  const int64_t oa = (pa / inner) * (int64_t)n * inner + (pa % inner);
  const int64_t ob = has_b ? (pb / inner) * (int64_t)n * inner + (pb % inner) : 0;
  half_block_pair<T>(in + oa, in + ob, has_b, inner, n, logN, tw, sinN, x, z, wsum);
  for (int m = threadIdx.x + 1; m <= n; m += blockDim.x) {
    const Cplx<T> F = x[m];
    out[oa + (int64_t)(m - 1) * inner] = F.re * scale;
    if (has_b) out[ob + (int64_t)(m - 1) * inner] = F.im * scale;
  }
}

// The per-axis source factors of every axis in one launch (blockIdx.y = axis, blockIdx.x =
// pair of terms): the consistent loads L[R off_a + r n_a + j] are transformed along their
// axis and divided by mu^M_a(j), into fac (float64) and fac32 (float32, may be null).
struct AxisFactorJob {
  int d, R;
  int n[PE_MAX_D], off[PE_MAX_D], logN[PE_MAX_D];
  const Cplx<double>* tw[PE_MAX_D];
  const double* sinN[PE_MAX_D];
};
__global__ void __launch_bounds__(256) axis_factor_dst_kernel(AxisFactorJob J, const double* __restrict__ loads,
                                                              const double* __restrict__ muM,
                                                              double* __restrict__ fac, float* __restrict__ fac32) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int a = blockIdx.y;
  const int n = J.n[a], logN = J.logN[a], N = 1 << logN;
  const int ra = 2 * blockIdx.x, rb = ra + 1;
  if (ra >= J.R) return;  // uniform over the CTA
  const bool has_b = rb < J.R;
  Cplx<double>* x = reinterpret_cast<Cplx<double>*>(smem_raw);
  Cplx<double>* z = x + (N + 1);
  Cplx<double>* wsum = z + N;
  const int64_t oa = (int64_t)J.R * J.off[a] + (int64_t)ra * n;
  const int64_t ob = has_b ? oa + n : 0;
  half_block_pair<double>(loads + oa, loads + ob, has_b, 1, n, logN, J.tw[a], J.sinN[a], x, z, wsum);
  const double scale = sqrt(2.0 / (double)N);
  for (int m = threadIdx.x + 1; m <= n; m += blockDim.x) {
    const Cplx<double> F = x[m];
    const double mu = muM[J.off[a] + m - 1];
    const double va = F.re * scale / mu;
    fac[oa + m - 1] = va;
    if (fac32) fac32[oa + m - 1] = (float)va;
    if (has_b) {
      const double vb = F.im * scale / mu;
      fac[ob + m - 1] = vb;
      if (fac32) fac32[ob + m - 1] = (float)vb;
    }
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

// ---------------------------------------------------------------------------
// Warp-per-pencil-pair FFT form (n + 1 = 2^k, 16 <= n + 1 <= 1024): the same odd
// extension of z = x + i y over L = 2(n+1) points, transformed by a self-sorting
// (Stockham) FFT in radix-16/32 passes (a radix-2/4/8 pass finishes the rest).
// One warp owns one pencil pair's L values in shared memory, so the passes need
// only __syncwarp; each lane holds L/32 values in registers between a pass's
// loads and stores.  A CTA stages WARPS pencil pairs: the global loads and
// stores are CTA-wide and coalesced (contiguous for the last axis, rows of
// 2*WARPS consecutive pencils for the others).  Pass twiddles are tabulated per
// CTA as [r][k] (k fastest) so that lanes read consecutive entries.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, Cplx<T> b) {
  return Cplx<T>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// read-only (non-coherent cache) load of one complex value
template <typename T>
__device__ __forceinline__ Cplx<T> ldg_cplx(const Cplx<T>* p) {
  if constexpr (sizeof(T) == 4) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return Cplx<T>{v.x, v.y};
  } else {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return Cplx<T>{v.x, v.y};
  }
}

// padded shared-memory index: one gap every 16 values keeps the strided pass
// stores free of bank conflicts
__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }

// Asynchronous global -> shared copies (cp.async, Ampere and later): the strided-pencil
// paths stage the next block of pencils while the current one is transformed.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst_smem, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Offsets of the P pencils of block blk (o * n * inner + i for pencil p = o * inner + i, -1 past the end).
__device__ __forceinline__ void block_offsets(int64_t blk, int P, int n, int64_t inner, int64_t npencils,
                                              int64_t* off) {
  if ((int)threadIdx.x < P) {
    const int64_t p = blk * P + threadIdx.x;
    off[threadIdx.x] = p < npencils ? (p / inner) * (int64_t)n * inner + (p % inner) : -1;
  }
}

// Stage the block's rows, stage[pl * n + j] = pencil pl's value j (consecutive threads take
// consecutive pencils of one row, so each row is one coalesced run); pencils past the end are 0.
template <typename T>
__device__ __forceinline__ void stage_block_async(const T* __restrict__ in, const int64_t* off, int P, int logP,
                                                  int n, int64_t inner, T* stage) {
  for (int e = threadIdx.x; e < P * n; e += blockDim.x) {
    const int pl = e & (P - 1), j = e >> logP;
    const int64_t o = off[pl];
    if (o >= 0) cp_async_elem(stage + pl * n + j, in + o + (int64_t)j * inner);
    else stage[pl * n + j] = T(0);
  }
  cp_async_commit();
}

constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }
__host__ __device__ constexpr int brevc(int i, int bits) {  // bit reversal of i < 32 over `bits` bits
  return (((i & 1) << 4) | ((i & 2) << 2) | (i & 4) | ((i & 8) >> 2) | ((i & 16) >> 4)) >> (5 - bits);
}

// e^{-2 pi i t/32}, t = 0..15 (cos and -sin of multiples of pi/16)
__device__ __forceinline__ constexpr double w32_re(int t) {
  return t == 0 ? 1.0 : t == 1 ? 0.98078528040323044913 : t == 2 ? 0.92387953251128675613 : t == 3 ? 0.83146961230254523708 : t == 4 ? 0.70710678118654752440 : t == 5 ? 0.55557023301960222474 : t == 6 ? 0.38268343236508977173 : t == 7 ? 0.19509032201612826785 : t == 8 ? 0.0 : t == 9 ? -0.19509032201612826785 : t == 10 ? -0.38268343236508977173 : t == 11 ? -0.55557023301960222474 : t == 12 ? -0.70710678118654752440 : t == 13 ? -0.83146961230254523708 : t == 14 ? -0.92387953251128675613 : -0.98078528040323044913;
}
__device__ __forceinline__ constexpr double w32_im(int t) {
  return t == 0 ? 0.0 : t == 1 ? -0.19509032201612826785 : t == 2 ? -0.38268343236508977173 : t == 3 ? -0.55557023301960222474 : t == 4 ? -0.70710678118654752440 : t == 5 ? -0.83146961230254523708 : t == 6 ? -0.92387953251128675613 : t == 7 ? -0.98078528040323044913 : t == 8 ? -1.0 : t == 9 ? -0.98078528040323044913 : t == 10 ? -0.92387953251128675613 : t == 11 ? -0.83146961230254523708 : t == 12 ? -0.70710678118654752440 : t == 13 ? -0.55557023301960222474 : t == 14 ? -0.38268343236508977173 : -0.19509032201612826785;
}

// In-register forward DFT of R = 2, 4, ..., 32 values: radix-2 decimation in frequency,
// natural-order input, output in bit-reversed order (X[r] = v[brevc(r, log2 R)]).
template <typename T, int R>
__device__ __forceinline__ void dft_regs(Cplx<T> (&v)[R]) {
#pragma unroll
  for (int len = R; len >= 2; len >>= 1) {
#pragma unroll
    for (int s = 0; s < R; s += len) {
#pragma unroll
      for (int k = 0; k < len / 2; ++k) {
        const int t = k * (32 / len);
        const Cplx<T> a = v[s + k], b = v[s + k + len / 2];
        v[s + k] = Cplx<T>{a.re + b.re, a.im + b.im};
        const Cplx<T> d{a.re - b.re, a.im - b.im};
        if (t == 0) v[s + k + len / 2] = d;
        else if (t == 8) v[s + k + len / 2] = Cplx<T>{d.im, -d.re};  // times -i
        else v[s + k + len / 2] = cmul(d, Cplx<T>{(T)w32_re(t), (T)w32_im(t)});
      }
    }
  }
}

// Radix (as log2) of the pass that starts with `left` of the LOGL bits still to combine:
// float32 uses 32-point passes from L = 1024 on ([32, 32], [32, 32, 2]); L = 512 takes
// [16, 16, 2] (a 32-point pass there leaves half the lanes idle: 16 groups of 32), and
// float64 keeps 16-point passes (register budget).
template <typename T>
__host__ __device__ constexpr int pass_bits(int left, int logl) {
  return (sizeof(T) == 4 && logl >= 10 && left >= 5) ? 5 : (left >= 4 ? 4 : left);
}

// radix plans of the pass twiddle tables: the one-warp form (pass_bits), the half-length form
// (half_pass_bits) and the team form (team_pass_bits: radix 16 while 4 bits remain)
constexpr int kPlanWarp = 0, kPlanHalf = 1, kPlanTeam = 2, kPlanTwo = 3;
__host__ __device__ constexpr int team_pass_bits(int left) { return left >= 4 ? 4 : left; }
// the two-pass float32 form at L = 512: radix 32, then radix 16
__host__ __device__ constexpr int two_pass_bits(int left, int logl) { return left == logl ? 5 : left; }
constexpr int team_tw_entries(int left, int ns) {
  return left == 0 ? 0
                   : (ns > 1 ? ns * (1 << team_pass_bits(left)) : 0) +
                         team_tw_entries(left - team_pass_bits(left), ns * (1 << team_pass_bits(left)));
}

// One Stockham pass of radix R after NS points have been combined; tw = this pass's
// table [r][k] = e^{-2 pi i k r / (NS R)}, k < NS (unused when NS == 1).
template <typename T, int LOGL, int R, int NS>
__device__ __forceinline__ void stockham_pass(Cplx<T>* a, const Cplx<T>* tw, int lane) {
  constexpr int L = 1 << LOGL, NG = L / R, G = (NG + 31) / 32;
  Cplx<T> v[G][R];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = lane + 32 * g;
    if (NG % 32 == 0 || j < NG) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[g][r] = a[fpad(j + r * NG)];
      if (NS > 1) {
        const int k = j & (NS - 1);
#pragma unroll
        for (int r = 1; r < R; ++r) v[g][r] = cmul(v[g][r], ldg_cplx(tw + r * NS + k));
      }
      dft_regs<T, R>(v[g]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = lane + 32 * g;
    if (NG % 32 == 0 || j < NG) {
      const int k = j & (NS - 1);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) a[fpad(base + r * NS)] = v[g][brevc(r, ilog2c(R))];
    }
  }
  __syncwarp();
}

// All passes: radix 16 while at least 4 bits remain, then one pass of the rest.
template <typename T, int LOGL, int LEFT, int NS>
struct StockhamPasses {
  static __device__ __forceinline__ void run(Cplx<T>* a, const Cplx<T>* tw, int lane) {
    constexpr int RB = pass_bits<T>(LEFT, LOGL);
    constexpr int R = 1 << RB;
    stockham_pass<T, LOGL, R, NS>(a, tw, lane);
    StockhamPasses<T, LOGL, LEFT - RB, NS * R>::run(a, tw + (NS > 1 ? NS * R : 0), lane);
  }
};
template <typename T, int LOGL, int NS>
struct StockhamPasses<T, LOGL, 0, NS> {
  static __device__ __forceinline__ void run(Cplx<T>*, const Cplx<T>*, int) {}
};

// entries of the pass twiddle tables of a length-2^LOGL transform
template <typename T>
constexpr int pass_tw_entries(int left, int ns, int logl) {
  return left == 0 ? 0
                   : (ns > 1 ? ns * (1 << pass_bits<T>(left, logl)) : 0) +
                         pass_tw_entries<T>(left - pass_bits<T>(left, logl), ns * (1 << pass_bits<T>(left, logl)), logl);
}

// blockDim.x = 32 * warps (warps = 1, 2, 4 or 8): P = 2 * warps pencils per block of work.
template <typename T, int LOGL>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && LOGL <= 9) ? 2 : 1) dst_fft_warp_kernel(const T* __restrict__ in, T* __restrict__ out, int n,
                                                           int64_t inner, int64_t npencils, T scale,
                                                           const Cplx<T>* __restrict__ ptw) {
  // PS: pair-buffer stride, one more than the padded length so that the pair buffers of a
  // block start in different banks (the strided load and store walk across pairs)
  constexpr int L = 1 << LOGL, N = L / 2, PADL = L + L / 16, PS = PADL + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int B = blockDim.x, WARPS = B >> 5, P = 2 * WARPS, logP = __ffs(P) - 1;
  Cplx<T>* bufs = reinterpret_cast<Cplx<T>*>(smem_raw);
  int64_t* off = reinterpret_cast<int64_t*>(bufs + (size_t)WARPS * PS);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (inner == 1) {
    // contiguous pencils (last axis): each warp loads, transforms and stores its own pencil
    // pairs (rows of n consecutive values), with no block-wide barrier
    constexpr int JL = (N + 31) / 32;  // values per lane and pencil (n <= N - 1)
    Cplx<T>* a = bufs + (size_t)warp * PS;
    const int64_t npairs = (npencils + 1) / 2;
    for (int64_t pr = (int64_t)blockIdx.x * WARPS + warp; pr < npairs; pr += (int64_t)gridDim.x * WARPS) {
      const int64_t pa = 2 * pr, pb = pa + 1;
      const bool has_b = pb < npencils;
      const T* xa = in + pa * n;
      const T* xb = in + pb * n;
      T ra[JL], rb[JL];
#pragma unroll
      for (int t = 0; t < JL; ++t) {
        const int j = lane + 32 * t;
        ra[t] = j < n ? xa[j] : T(0);
        rb[t] = (j < n && has_b) ? xb[j] : T(0);
      }
      if (lane == 0) {
        a[fpad(0)] = Cplx<T>{T(0), T(0)};
        a[fpad(N)] = Cplx<T>{T(0), T(0)};
      }
#pragma unroll
      for (int t = 0; t < JL; ++t) {
        const int j = lane + 32 * t;
        if (j < n) {
          a[fpad(j + 1)] = Cplx<T>{ra[t], rb[t]};
          a[fpad(L - 1 - j)] = Cplx<T>{-ra[t], -rb[t]};
        }
      }
      __syncwarp();
      StockhamPasses<T, LOGL, LOGL, 1>::run(a, ptw, lane);
      T* ya = out + pa * n;
      T* yb = out + pb * n;
#pragma unroll
      for (int t = 0; t < JL; ++t) {
        const int k = lane + 32 * t;
        if (k < n) {
          const Cplx<T> Z = a[fpad(k + 1)];
          ya[k] = -Z.im * scale;
          if (has_b) yb[k] = Z.re * scale;
        }
      }
      __syncwarp();
    }
    return;
  }
  // strided pencils: blocks of P consecutive pencils, each row j one contiguous run of P
  // values; the next block's rows are staged (cp.async) while this block is transformed
  const int64_t nblk = (npencils + P - 1) / P;
  int64_t* offs[2] = {off, off + P};
  T* stage = reinterpret_cast<T*>(off + 2 * P);
  int cur = 0;
  if ((int64_t)blockIdx.x < nblk) {
    block_offsets(blockIdx.x, P, n, inner, npencils, offs[0]);
    __syncthreads();
    stage_block_async(in, offs[0], P, logP, n, inner, stage);
  }
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x, cur ^= 1) {
    cp_async_wait_all();
    __syncthreads();
    // z_j = x_j + i y_j at j = 1..n, -z_j at L - j, 0 at the fixed points 0 and N
    if (tid < 2 * WARPS) {
      Cplx<T>* a = bufs + (size_t)(tid >> 1) * PS;
      a[fpad((tid & 1) ? N : 0)] = Cplx<T>{T(0), T(0)};
    }
    for (int e = tid; e < P * n; e += B) {
      const int pl = e & (P - 1), j = e >> logP;
      const T v = stage[pl * n + j];
      Cplx<T>* a = bufs + (size_t)(pl >> 1) * PS;
      reinterpret_cast<T*>(a + fpad(j + 1))[pl & 1] = v;
      reinterpret_cast<T*>(a + fpad(L - 1 - j))[pl & 1] = -v;
    }
    __syncthreads();
    const int64_t next = blk + gridDim.x;
    if (next < nblk) {
      block_offsets(next, P, n, inner, npencils, offs[cur ^ 1]);
      __syncthreads();
      stage_block_async(in, offs[cur ^ 1], P, logP, n, inner, stage);
    }
    StockhamPasses<T, LOGL, LOGL, 1>::run(bufs + (size_t)warp * PS, ptw, lane);
    __syncthreads();
    // store: DST(x)_k = -Im Z_k / 2, DST(y)_k = Re Z_k / 2 (times sqrt(2/(n+1)))
    for (int e = tid; e < P * n; e += B) {
      const int pl = e & (P - 1), k = e >> logP;
      const Cplx<T> Z = bufs[(size_t)(pl >> 1) * PS + fpad(k + 1)];
      const T val = (pl & 1) ? Z.re * scale : -Z.im * scale;
      const int64_t o = offs[cur][pl];
      if (o >= 0) out[o + (int64_t)k * inner] = val;
    }
  }
}

// ---------------------------------------------------------------------------
// Half-length form (128 <= n + 1 = N <= 1024).  The odd extension wastes half of
// a length-2N transform; instead each real pencil x (x_0 = x_N = 0) is folded to
//   y_j = sin(pi j/N) (x_j + x_{N-j}) + (x_j - x_{N-j}) / 2,   j = 0..N-1,
// whose length-N real DFT Y_k = R_k + i I_k (kernel e^{+2 pi i jk/N}) gives the
// sine sums F_m = sum_j x_j sin(pi j m/N) as F_{2k} = I_k and
// F_{2k+1} = R_0/2 + R_1 + ... + R_k (a prefix sum).  Two pencils a, b share one
// complex FFT of z = y^a + i y^b (length N, forward kernel e^{-2 pi i jk/N}):
// with W = conj(Z_{N-k}), Y^a = (Z_k + W)/2 and Y^b = (Z_k - W)/(2i), so
// R^a = (Re Z_k + Re Z_{N-k})/2, I^a = (Im Z_{N-k} - Im Z_k)/2,
// R^b = (Im Z_k + Im Z_{N-k})/2, I^b = (Re Z_k - Re Z_{N-k})/2.
// One warp owns a pair; radices keep all 32 lanes busy (N/R >= 32 groups).  The
// prefix sum runs per lane over a contiguous chunk of N/64 indices, then across
// lanes with warp shuffles.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ constexpr int half_pass_bits(int left, int logn) {
  const int cap = sizeof(T) == 4 ? 5 : 4;
  const int lim = logn - 5 < 2 ? 2 : (logn - 5 > cap ? cap : logn - 5);
  return left >= lim ? lim : left;
}

template <typename T, int LOGN, int LEFT, int NS>
struct HalfPasses {
  static __device__ __forceinline__ void run(Cplx<T>* a, const Cplx<T>* tw, int lane) {
    constexpr int RB = half_pass_bits<T>(LEFT, LOGN);
    constexpr int R = 1 << RB;
    stockham_pass<T, LOGN, R, NS>(a, tw, lane);
    HalfPasses<T, LOGN, LEFT - RB, NS * R>::run(a, tw + (NS > 1 ? NS * R : 0), lane);
  }
};
template <typename T, int LOGN, int NS>
struct HalfPasses<T, LOGN, 0, NS> {
  static __device__ __forceinline__ void run(Cplx<T>*, const Cplx<T>*, int) {}
};

template <typename T>
constexpr int half_tw_entries(int left, int ns, int logn) {
  return left == 0 ? 0
                   : (ns > 1 ? ns * (1 << half_pass_bits<T>(left, logn)) : 0) +
                         half_tw_entries<T>(left - half_pass_bits<T>(left, logn),
                                            ns * (1 << half_pass_bits<T>(left, logn)), logn);
}

// Fold (pre-processing), FFT and unfold (post-processing) of one pencil pair held in a:
// on entry a[fpad(p)] = (x^a_p, x^b_p) for p = 1..N-1 and a[fpad(0)] = 0; on exit
// a[fpad(m)] = (4 F^a_m, 4 F^b_m) for m = 1..N-1 (unscaled sine sums times four: the fold is
// taken times two, y_j = (2s_j + 1) x_j + (2s_j - 1) x_{N-j} with s_j = sin(pi j / N), one
// multiplication and one FMA per value from the table fold = (2s + 1, 2s - 1), and the unfold
// without its halvings; the caller's scale carries the 1/4, a power of two).
template <typename T, int LOGN>
__device__ __forceinline__ void half_dst_pair(Cplx<T>* a, const Cplx<T>* __restrict__ ptw,
                                              const Cplx<T>* __restrict__ fold, int lane) {
  constexpr int N = 1 << LOGN, V = N / 32, C = N / 64;
  // fold
  Cplx<T> z[V];
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const int j = lane + 32 * t;
    const Cplx<T> x = a[fpad(j)];
    const Cplx<T> xm = j == 0 ? Cplx<T>{T(0), T(0)} : a[fpad(N - j)];
    const Cplx<T> f = ldg_cplx(fold + j);
    z[t] = Cplx<T>{fma(f.re, x.re, f.im * xm.re), fma(f.re, x.im, f.im * xm.im)};
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < V; ++t) a[fpad(lane + 32 * t)] = z[t];
  __syncwarp();
  HalfPasses<T, LOGN, LOGN, 1>::run(a, ptw, lane);
  // unfold: lane owns k = lane*C .. lane*C + C - 1 of the N/2 output pairs
  T ia[C], ib[C], sa[C], sb[C];
  T ta = T(0), tb = T(0);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int k = lane * C + c;
    const Cplx<T> Z = a[fpad(k)];
    const Cplx<T> Wm = a[fpad((N - k) & (N - 1))];
    T ra = Z.re + Wm.re, rb = Z.im + Wm.im;
    ia[c] = Wm.im - Z.im;
    ib[c] = Z.re - Wm.re;
    if (k == 0) {
      ra *= T(0.5);
      rb *= T(0.5);
    }
    ta += ra;
    tb += rb;
    sa[c] = ta;
    sb[c] = tb;
  }
  // exclusive scan of the lane totals
  T ea = ta, eb = tb;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T ua = __shfl_up_sync(0xffffffffu, ea, d), ub = __shfl_up_sync(0xffffffffu, eb, d);
    if (lane >= d) {
      ea += ua;
      eb += ub;
    }
  }
  ea -= ta;
  eb -= tb;
  __syncwarp();
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int k = lane * C + c;
    if (k > 0) a[fpad(2 * k)] = Cplx<T>{ia[c], ib[c]};
    a[fpad(2 * k + 1)] = Cplx<T>{sa[c] + ea, sb[c] + eb};
  }
  __syncwarp();
}

// Discrete Hartley transform of a pencil pair of N = 2^LOGN points (a periodic axis): with
// Z = FFT(x^a + i x^b), X^a = (Z_k + conj Z_{N-k})/2, X^b = (Z_k - conj Z_{N-k})/(2i) and
// H_k = Re X_k - Im X_k.  On entry a[fpad(j)] = (x^a_j, x^b_j), j = 0..N-1; on exit
// a[fpad(k)] = (H^a_k, H^b_k) (unscaled).
template <typename T, int LOGN>
__device__ __forceinline__ void dht_pair(Cplx<T>* a, const Cplx<T>* __restrict__ ptw, int lane) {
  constexpr int N = 1 << LOGN, C = N / 32;
  HalfPasses<T, LOGN, LOGN, 1>::run(a, ptw, lane);
  Cplx<T> hv[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int k = lane * C + c;
    const Cplx<T> Z = a[fpad(k)];
    const Cplx<T> Wm = a[fpad((N - k) & (N - 1))];
    const T rea = T(0.5) * (Z.re + Wm.re), ima = T(0.5) * (Z.im - Wm.im);
    const T reb = T(0.5) * (Z.im + Wm.im), imb = T(0.5) * (Wm.re - Z.re);
    hv[c] = Cplx<T>{rea - ima, reb - imb};
  }
  __syncwarp();
#pragma unroll
  for (int c = 0; c < C; ++c) a[fpad(lane * C + c)] = hv[c];
  __syncwarp();
}

// blockDim.x = 32 * warps; one warp per pencil pair (P = 2 * warps pencils per block of
// work for strided pencils).
// DHT = true: the same machinery computes the discrete Hartley transform of periodic
// pencils (n = N points, positions 0..N-1, no fold).
template <typename T, int LOGN, bool DHT = false>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && LOGN <= 9) ? 2 : 1)
    dst_half_warp_kernel(const T* __restrict__ in, T* __restrict__ out, int n, int64_t inner, int64_t npencils,
                         T scale, const Cplx<T>* __restrict__ ptw, const Cplx<T>* __restrict__ fold) {
  constexpr int SH = DHT ? 0 : 1;  // buffer position of value j
  constexpr int N = 1 << LOGN, PADN = N + N / 16, PS = PADN + 1, JL = N / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int B = blockDim.x, WARPS = B >> 5, P = 2 * WARPS, logP = __ffs(P) - 1;
  Cplx<T>* bufs = reinterpret_cast<Cplx<T>*>(smem_raw);
  int64_t* off = reinterpret_cast<int64_t*>(bufs + (size_t)WARPS * PS);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Cplx<T>* a = bufs + (size_t)warp * PS;
  if (inner == 1) {
    const int64_t npairs = (npencils + 1) / 2;
    for (int64_t pr = (int64_t)blockIdx.x * WARPS + warp; pr < npairs; pr += (int64_t)gridDim.x * WARPS) {
      const int64_t pa = 2 * pr, pb = pa + 1;
      const bool has_b = pb < npencils;
      const T* xa = in + pa * n;
      const T* xb = in + pb * n;
      T ra[JL], rb[JL];
#pragma unroll
      for (int t = 0; t < JL; ++t) {
        const int j = lane + 32 * t;
        ra[t] = j < n ? xa[j] : T(0);
        rb[t] = (j < n && has_b) ? xb[j] : T(0);
      }
      if (!DHT && lane == 0) a[fpad(0)] = Cplx<T>{T(0), T(0)};
#pragma unroll
      for (int t = 0; t < JL; ++t) {
        const int j = lane + 32 * t;
        if (j < n) a[fpad(j + SH)] = Cplx<T>{ra[t], rb[t]};
      }
      __syncwarp();
      if constexpr (DHT) dht_pair<T, LOGN>(a, ptw, lane);
      else half_dst_pair<T, LOGN>(a, ptw, fold, lane);
      T* ya = out + pa * n;
      T* yb = out + pb * n;
#pragma unroll
      for (int t = 0; t < JL; ++t) {
        const int k = lane + 32 * t;
        if (k < n) {
          const Cplx<T> F = a[fpad(k + SH)];
          ya[k] = F.re * scale;
          if (has_b) yb[k] = F.im * scale;
        }
      }
      __syncwarp();
    }
    return;
  }
  // strided pencils: as in dst_fft_warp_kernel, the next block is staged while this one runs
  const int64_t nblk = (npencils + P - 1) / P;
  int64_t* offs[2] = {off, off + P};
  T* stage = reinterpret_cast<T*>(off + 2 * P);
  int cur = 0;
  if ((int64_t)blockIdx.x < nblk) {
    block_offsets(blockIdx.x, P, n, inner, npencils, offs[0]);
    __syncthreads();
    stage_block_async(in, offs[0], P, logP, n, inner, stage);
  }
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x, cur ^= 1) {
    cp_async_wait_all();
    __syncthreads();
    if (!DHT && tid < WARPS) bufs[(size_t)tid * PS] = Cplx<T>{T(0), T(0)};
    for (int e = tid; e < P * n; e += B) {
      const int pl = e & (P - 1), j = e >> logP;
      reinterpret_cast<T*>(bufs + (size_t)(pl >> 1) * PS + fpad(j + SH))[pl & 1] = stage[pl * n + j];
    }
    __syncthreads();
    const int64_t next = blk + gridDim.x;
    if (next < nblk) {
      block_offsets(next, P, n, inner, npencils, offs[cur ^ 1]);
      __syncthreads();
      stage_block_async(in, offs[cur ^ 1], P, logP, n, inner, stage);
    }
    if constexpr (DHT) dht_pair<T, LOGN>(a, ptw, lane);
    else half_dst_pair<T, LOGN>(a, ptw, fold, lane);
    __syncthreads();
    for (int e = tid; e < P * n; e += B) {
      const int pl = e & (P - 1), k = e >> logP;
      const Cplx<T> F = bufs[(size_t)(pl >> 1) * PS + fpad(k + SH)];
      const int64_t o = offs[cur][pl];
      if (o >= 0) out[o + (int64_t)k * inner] = ((pl & 1) ? F.im : F.re) * scale;
    }
  }
}

// ---------------------------------------------------------------------------
// Two-pass form of the float32 odd-extension FFT at L = 512 points (n = 255), contiguous
// pencils (the last axis).  A warp owns two pencil pairs, lanes 16 h + j (h = 0, 1) the pair
// h.  Pass 1 (radix 32 over the 16 groups j of a pair) takes its inputs straight from the
// rows in global memory -- z_ext[j + 16 r] = z[j + 16 r - 1] for r < 16 -- and the mirrored
// half z_ext[m] = -z_ext[512 - m] (r >= 16) from the lane 16 - j of the same pair by shuffles;
// its outputs cross shared memory once; pass 2 (radix 16 over the 32 groups of a pair, the
// whole warp on one pair at a time) yields X[j + 32 r] in natural order, of which the DST
// needs only m = 1..255 (r < 8), stored straight to the output rows.  Shared memory carries
// one write and one read per point (the one-warp form: the odd extension and three Stockham
// passes).
// ---------------------------------------------------------------------------
// TI, TO: the input and output element types (float64 data is rounded to float32 on load and
// the float32 result widened on store: the mixed form's transforms of float64 fields).
template <typename TI, typename TO>
__global__ void __launch_bounds__(256, 2) dst512_contig_kernel(const TI* __restrict__ in, TO* __restrict__ out,
                                                               int64_t npencils, float scale,
                                                               const Cplx<float>* __restrict__ tw2) {
  constexpr int L = 512, n = 255, PS = L + L / 16 + 1;
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, WARPS = blockDim.x >> 5;
  const int h = lane >> 4, j = lane & 15;
  Cplx<float>* buf = reinterpret_cast<Cplx<float>*>(smem_raw) + (size_t)warp * 2 * PS;
  const int64_t npairs = (npencils + 1) / 2, nquads = (npairs + 1) / 2;
  const int src = ((16 - j) & 15) | (h << 4);
  for (int64_t q = (int64_t)blockIdx.x * WARPS + warp; q < nquads; q += (int64_t)gridDim.x * WARPS) {
    const int64_t pa = 2 * (2 * q + h), pb = pa + 1;
    const bool has_a = pa < npencils, has_b = pb < npencils;
    const TI* xa = in + pa * n;
    const TI* xb = in + pb * n;
    Cplx<float> v[32];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int m = j + 16 * r;
      v[r].re = (m >= 1 && has_a) ? (float)xa[m - 1] : 0.f;
      v[r].im = (m >= 1 && has_b) ? (float)xb[m - 1] : 0.f;
    }
#pragma unroll
    for (int r = 16; r < 32; ++r) {
      // 512 - m = 16 (31 - r) + (16 - j) for j >= 1; 16 (32 - r) for j = 0 (lane 0's own row)
      float re = __shfl_sync(0xffffffffu, v[31 - r].re, src);
      float im = __shfl_sync(0xffffffffu, v[31 - r].im, src);
      if (j == 0) {
        re = r == 16 ? 0.f : v[32 - r].re;
        im = r == 16 ? 0.f : v[32 - r].im;
      }
      v[r] = Cplx<float>{-re, -im};
    }
    dft_regs<float, 32>(v);
    Cplx<float>* a = buf + h * PS;
#pragma unroll
    for (int r = 0; r < 32; ++r) a[fpad(32 * j + r)] = v[brevc(r, 5)];
    __syncwarp();
#pragma unroll 1
    for (int p = 0; p < 2; ++p) {
      const Cplx<float>* b = buf + p * PS;
      Cplx<float> u[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) u[r] = b[fpad(lane + 32 * r)];
#pragma unroll
      for (int r = 1; r < 16; ++r) u[r] = cmul(u[r], ldg_cplx(tw2 + 32 * r + lane));
      dft_regs<float, 16>(u);
      const int64_t qa = 2 * (2 * q + p), qb = qa + 1;
      TO* ya = out + qa * n;
      TO* yb = out + qb * n;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int m = lane + 32 * r;
        if (m >= 1) {
          const Cplx<float> X = u[brevc(r, 4)];
          if (qa < npencils) ya[m - 1] = (TO)(-X.im * scale);
          if (qb < npencils) yb[m - 1] = (TO)(X.re * scale);
        }
      }
    }
    __syncwarp();
  }
}

// The same two passes for strided pencils: a CTA of W warps owns blocks of 4 W consecutive
// pencils (warp w: pencils 4w .. 4w + 3), staged row by row (row j: the 4 W values of one
// position, contiguous when the pencils are) by cp.async into a double buffer, padded to 4 W + 2
// floats so that a lane reads its pencil pair as one float2; pass 1 reads the rows of the stage,
// pass 2 writes the DST values back into the same stage, and the rows leave it coalesced.
// W warps per CTA: blocks of P = 4 W pencils, stage rows of P + 2 floats.
// (TI = double: the rows are converted on the way into the stage by plain loads.)
template <int W, typename TI, typename TO>
__global__ void __launch_bounds__(32 * W) dst512_strided_kernel(const TI* __restrict__ in, TO* __restrict__ out,
                                                                int64_t inner, int64_t npencils, float scale,
                                                                const Cplx<float>* __restrict__ tw2) {
  constexpr int L = 512, n = 255, PS = L + L / 16 + 1, P = 4 * W, SP = P + 2;
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int h = lane >> 4, j = lane & 15;
  float* stage[2] = {reinterpret_cast<float*>(smem_raw), reinterpret_cast<float*>(smem_raw) + n * SP};
  Cplx<float>* buf = reinterpret_cast<Cplx<float>*>(stage[1] + n * SP) + (size_t)warp * 2 * PS;
  __shared__ int64_t offs[2][P];
  const int64_t nblk = (npencils + P - 1) / P;
  const int src = ((16 - j) & 15) | (h << 4);
  // this lane's pass-2 twiddles e^{-2 pi i lane r / 512}, the same for every pair and block
  Cplx<float> tw[16];
#pragma unroll
  for (int r = 1; r < 16; ++r) tw[r] = ldg_cplx(tw2 + 32 * r + lane);
  // thread tid copies column pl = tid % 32 of rows tid / 32, + 8, ... (a warp: one 128-byte row)
  const int pl = tid & (P - 1), row0 = tid / P;
  constexpr int RSTEP = 32 * W / P;
  auto issue = [&](int64_t blk, int b) {
    if (tid < P) {
      const int64_t p = blk * P + tid;
      offs[b][tid] = p < npencils ? (p / inner) * (int64_t)n * inner + (p % inner) : -1;
    }
    __syncthreads();
    const int64_t o = offs[b][pl];
    float* dst = stage[b] + row0 * SP + pl;
    if (o >= 0) {
      const TI* srcp = in + o + (int64_t)row0 * inner;
      const int64_t step = (int64_t)RSTEP * inner;
      if constexpr (sizeof(TI) == 4) {
        for (int jj = row0; jj < n; jj += RSTEP, dst += RSTEP * SP, srcp += step) cp_async_elem(dst, srcp);
      } else {
        // every load of the thread's rows issued before the first store
        constexpr int NR = (n + RSTEP - 1) / RSTEP;
        float vals[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) vals[q] = row0 + q * RSTEP < n ? (float)__ldg(srcp + q * step) : 0.f;
#pragma unroll
        for (int q = 0; q < NR; ++q)
          if (row0 + q * RSTEP < n) dst[q * RSTEP * SP] = vals[q];
      }
    } else {
      for (int jj = row0; jj < n; jj += RSTEP, dst += RSTEP * SP) *dst = 0.f;
    }
    cp_async_commit();
  };
  int cur = 0;
  if ((int64_t)blockIdx.x < nblk) issue(blockIdx.x, 0);
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x, cur ^= 1) {
    cp_async_wait_all();
    __syncthreads();
    const int64_t next = blk + gridDim.x;
    if (next < nblk) issue(next, cur ^ 1);
    const float* st = stage[cur];
    // pass 1 on this warp's pencil pair h: columns 4 warp + 2 h, + 1 of the stage rows
    const int col = 4 * warp + 2 * h;
    Cplx<float> v[32];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int m = j + 16 * r;
      if (m >= 1) {
        const float2 z = *reinterpret_cast<const float2*>(st + (m - 1) * SP + col);
        v[r] = Cplx<float>{z.x, z.y};
      } else {
        v[r] = Cplx<float>{0.f, 0.f};
      }
    }
#pragma unroll
    for (int r = 16; r < 32; ++r) {
      float re = __shfl_sync(0xffffffffu, v[31 - r].re, src);
      float im = __shfl_sync(0xffffffffu, v[31 - r].im, src);
      if (j == 0) {
        re = r == 16 ? 0.f : v[32 - r].re;
        im = r == 16 ? 0.f : v[32 - r].im;
      }
      v[r] = Cplx<float>{-re, -im};
    }
    dft_regs<float, 32>(v);
    Cplx<float>* a = buf + h * PS;
#pragma unroll
    for (int r = 0; r < 32; ++r) a[fpad(32 * j + r)] = v[brevc(r, 5)];
    // a warp reads and writes only its own four columns of the stage, so its DST values go back
    // into them once its own lanes are done (the pair buffers are per warp too)
    __syncwarp();
    float* ost = stage[cur];
#pragma unroll 1
    for (int p = 0; p < 2; ++p) {
      const Cplx<float>* b = buf + p * PS;
      Cplx<float> u[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) u[r] = b[fpad(lane + 32 * r)];
#pragma unroll
      for (int r = 1; r < 16; ++r) u[r] = cmul(u[r], tw[r]);
      dft_regs<float, 16>(u);
      const int oc = 4 * warp + 2 * p;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int m = lane + 32 * r;
        if (m >= 1) {
          const Cplx<float> X = u[brevc(r, 4)];
          *reinterpret_cast<float2*>(ost + (m - 1) * SP + oc) = make_float2(-X.im * scale, X.re * scale);
        }
      }
    }
    __syncthreads();
    {
      const int64_t o = offs[cur][pl];
      if (o >= 0) {
        TO* dstp = out + o + (int64_t)row0 * inner;
        const float* sp = ost + row0 * SP + pl;
        const int64_t step = (int64_t)RSTEP * inner;
        for (int k = row0; k < n; k += RSTEP, sp += RSTEP * SP, dstp += step) *dstp = (TO)*sp;
      }
    }
  }
  cp_async_wait_all();
}

// Two passes at L = 1024 points (n = 511), strided pencils: radix 32 over the 32 groups of a
// pair (a whole warp, the mirrored half of the extension from lane 32 - j), one exchange through
// shared memory, radix 32 again, of whose outputs X[j + 32 r] the DST needs r < 16.  A CTA of W
// warps owns blocks of 4 W consecutive pencils staged as above (511 rows, double buffered); a warp runs its two pencil pairs one after the other through one pair buffer and
// keeps their outputs in registers until every warp is done with the stage.
template <int W>
__global__ void __launch_bounds__(32 * W) dst1024_strided_kernel(const float* __restrict__ in,
                                                                 float* __restrict__ out, int64_t inner,
                                                                 int64_t npencils, float scale,
                                                                 const Cplx<float>* __restrict__ tw2) {
  constexpr int L = 1024, n = 511, PS = L + L / 16 + 1, P = 4 * W, SP = P + 2;
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* stage[2] = {reinterpret_cast<float*>(smem_raw), reinterpret_cast<float*>(smem_raw) + n * SP};
  Cplx<float>* a = reinterpret_cast<Cplx<float>*>(stage[1] + n * SP) + (size_t)warp * PS;
  __shared__ int64_t offs[2][P];
  const int64_t nblk = (npencils + P - 1) / P;
  const int src = (32 - lane) & 31;
  // this lane's pass-2 twiddles e^{-2 pi i lane r / 1024}, the same for every pair and block
  Cplx<float> tw[32];
#pragma unroll
  for (int r = 1; r < 32; ++r) tw[r] = ldg_cplx(tw2 + 32 * r + lane);
  const int pl = tid & (P - 1), row0 = tid / P;
  constexpr int RSTEP = 32 * W / P;
  auto issue = [&](int64_t blk, int b) {
    if (tid < P) {
      const int64_t p = blk * P + tid;
      offs[b][tid] = p < npencils ? (p / inner) * (int64_t)n * inner + (p % inner) : -1;
    }
    __syncthreads();
    const int64_t o = offs[b][pl];
    float* dst = stage[b] + row0 * SP + pl;
    if (o >= 0) {
      const float* srcp = in + o + (int64_t)row0 * inner;
      const int64_t step = (int64_t)RSTEP * inner;
      for (int jj = row0; jj < n; jj += RSTEP, dst += RSTEP * SP, srcp += step) cp_async_elem(dst, srcp);
    } else {
      for (int jj = row0; jj < n; jj += RSTEP, dst += RSTEP * SP) *dst = 0.f;
    }
    cp_async_commit();
  };
  int cur = 0;
  if ((int64_t)blockIdx.x < nblk) issue(blockIdx.x, 0);
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x, cur ^= 1) {
    cp_async_wait_all();
    __syncthreads();
    const int64_t next = blk + gridDim.x;
    if (next < nblk) issue(next, cur ^ 1);
    float* st = stage[cur];
    // a warp reads and writes only its own four columns of the stage: the DST values of a pair
    // go back into the columns its inputs came from as soon as they are ready
#pragma unroll 1
    for (int p = 0; p < 2; ++p) {
      const int col = 4 * warp + 2 * p;
      Cplx<float> v[32];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int m = lane + 32 * r;
        if (m >= 1) {
          const float2 z = *reinterpret_cast<const float2*>(st + (m - 1) * SP + col);
          v[r] = Cplx<float>{z.x, z.y};
        } else {
          v[r] = Cplx<float>{0.f, 0.f};
        }
      }
#pragma unroll
      for (int r = 16; r < 32; ++r) {
        // 1024 - m = 32 (31 - r) + (32 - j) for j >= 1; 32 (32 - r) for j = 0 (lane 0's own row)
        float re = __shfl_sync(0xffffffffu, v[31 - r].re, src);
        float im = __shfl_sync(0xffffffffu, v[31 - r].im, src);
        if (lane == 0) {
          re = r == 16 ? 0.f : v[32 - r].re;
          im = r == 16 ? 0.f : v[32 - r].im;
        }
        v[r] = Cplx<float>{-re, -im};
      }
      dft_regs<float, 32>(v);
      __syncwarp();  // the previous pair's reads of the pair buffer are done
#pragma unroll
      for (int r = 0; r < 32; ++r) a[fpad(32 * lane + r)] = v[brevc(r, 5)];
      __syncwarp();
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = a[fpad(lane + 32 * r)];
#pragma unroll
      for (int r = 1; r < 32; ++r) v[r] = cmul(v[r], tw[r]);
      dft_regs<float, 32>(v);
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int m = lane + 32 * r;
        const Cplx<float> X = v[brevc(r, 5)];
        if (m >= 1) *reinterpret_cast<float2*>(st + (m - 1) * SP + col) = make_float2(-X.im * scale, X.re * scale);
      }
    }
    __syncthreads();
    const float* ost = st;
    {
      const int64_t o = offs[cur][pl];
      if (o >= 0) {
        float* dstp = out + o + (int64_t)row0 * inner;
        const float* sp = ost + row0 * SP + pl;
        const int64_t step = (int64_t)RSTEP * inner;
        for (int k = row0; k < n; k += RSTEP, sp += RSTEP * SP, dstp += step) *dstp = *sp;
      }
    }
  }
  cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// Team form of the odd-extension FFT for long float32 pencils (L = 2(n+1) = 1024, 2048): a team
// of TW warps (TS = 32 TW threads, synchronised by a named barrier) owns one pencil pair, so a
// lane holds L / (16 TS) radix-16 groups -- 16 complex values -- instead of the L/32 of the
// one-warp form (32 or 64 values, which capped that form at one CTA of 8 warps per SM).
// Passes: radix 16 while at least 4 bits remain, then the remainder ([16, 16, 4] at L = 1024,
// [16, 16, 8] at 2048).  Same loads, stores and odd extension as dst_fft_warp_kernel.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void team_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <typename T, int LOGL, int R, int NS, int TS>
__device__ __forceinline__ void stockham_team_pass(Cplx<T>* a, const Cplx<T>* tw, int tl, int bar) {
  constexpr int L = 1 << LOGL, NG = L / R, G = (NG + TS - 1) / TS;
  Cplx<T> v[G][R];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = tl + TS * g;
    if (NG % TS == 0 || j < NG) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[g][r] = a[fpad(j + r * NG)];
      if (NS > 1) {
        const int k = j & (NS - 1);
#pragma unroll
        for (int r = 1; r < R; ++r) v[g][r] = cmul(v[g][r], ldg_cplx(tw + r * NS + k));
      }
      dft_regs<T, R>(v[g]);
    }
  }
  team_sync(bar, TS);
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = tl + TS * g;
    if (NG % TS == 0 || j < NG) {
      const int k = j & (NS - 1);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) a[fpad(base + r * NS)] = v[g][brevc(r, ilog2c(R))];
    }
  }
  team_sync(bar, TS);
}

template <typename T, int LOGL, int LEFT, int NS, int TS>
struct TeamPasses {
  static __device__ __forceinline__ void run(Cplx<T>* a, const Cplx<T>* tw, int tl, int bar) {
    constexpr int RB = team_pass_bits(LEFT);
    constexpr int R = 1 << RB;
    stockham_team_pass<T, LOGL, R, NS, TS>(a, tw, tl, bar);
    TeamPasses<T, LOGL, LEFT - RB, NS * R, TS>::run(a, tw + (NS > 1 ? NS * R : 0), tl, bar);
  }
};
template <typename T, int LOGL, int NS, int TS>
struct TeamPasses<T, LOGL, 0, NS, TS> {
  static __device__ __forceinline__ void run(Cplx<T>*, const Cplx<T>*, int, int) {}
};

constexpr int kTeamThreads = 256;  // CTA size of the team kernel

// blockDim.x = kTeamThreads: kTeamThreads / TS teams, one pencil pair each (P = 2 teams pencils
// per block of strided work).
template <typename T, int LOGL, int TW>
__global__ void __launch_bounds__(kTeamThreads) dst_fft_team_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                                     int n, int64_t inner, int64_t npencils,
                                                                     T scale, const Cplx<T>* __restrict__ ptw) {
  constexpr int L = 1 << LOGL, N = L / 2, PADL = L + L / 16, PS = PADL + 1, TS = 32 * TW;
  constexpr int TEAMS = kTeamThreads / TS, P = 2 * TEAMS, logP = ilog2c(P);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<T>* bufs = reinterpret_cast<Cplx<T>*>(smem_raw);
  int64_t* off = reinterpret_cast<int64_t*>(bufs + (size_t)TEAMS * PS);
  const int tid = threadIdx.x, team = tid / TS, tl = tid & (TS - 1), bar = 1 + team;
  Cplx<T>* a = bufs + (size_t)team * PS;
  if (inner == 1) {
    // contiguous pencils: each team loads, transforms and stores its own pencil pairs
    constexpr int JL = (N + TS - 1) / TS;
    const int64_t npairs = (npencils + 1) / 2;
    for (int64_t pr = (int64_t)blockIdx.x * TEAMS + team; pr < npairs; pr += (int64_t)gridDim.x * TEAMS) {
      const int64_t pa = 2 * pr, pb = pa + 1;
      const bool has_b = pb < npencils;
      const T* xa = in + pa * n;
      const T* xb = in + pb * n;
      T ra[JL], rb[JL];
#pragma unroll
      for (int t = 0; t < JL; ++t) {
        const int j = tl + TS * t;
        ra[t] = j < n ? xa[j] : T(0);
        rb[t] = (j < n && has_b) ? xb[j] : T(0);
      }
      if (tl == 0) {
        a[fpad(0)] = Cplx<T>{T(0), T(0)};
        a[fpad(N)] = Cplx<T>{T(0), T(0)};
      }
#pragma unroll
      for (int t = 0; t < JL; ++t) {
        const int j = tl + TS * t;
        if (j < n) {
          a[fpad(j + 1)] = Cplx<T>{ra[t], rb[t]};
          a[fpad(L - 1 - j)] = Cplx<T>{-ra[t], -rb[t]};
        }
      }
      team_sync(bar, TS);
      TeamPasses<T, LOGL, LOGL, 1, TS>::run(a, ptw, tl, bar);
      T* ya = out + pa * n;
      T* yb = out + pb * n;
#pragma unroll
      for (int t = 0; t < JL; ++t) {
        const int k = tl + TS * t;
        if (k < n) {
          const Cplx<T> Z = a[fpad(k + 1)];
          ya[k] = -Z.im * scale;
          if (has_b) yb[k] = Z.re * scale;
        }
      }
      team_sync(bar, TS);
    }
    return;
  }
  // strided pencils: blocks of P consecutive pencils staged row by row (cp.async), the next block
  // staged while this one is transformed
  const int64_t nblk = (npencils + P - 1) / P;
  int64_t* offs[2] = {off, off + P};
  T* stage = reinterpret_cast<T*>(off + 2 * P);
  int cur = 0;
  if ((int64_t)blockIdx.x < nblk) {
    block_offsets(blockIdx.x, P, n, inner, npencils, offs[0]);
    __syncthreads();
    stage_block_async(in, offs[0], P, logP, n, inner, stage);
  }
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x, cur ^= 1) {
    cp_async_wait_all();
    __syncthreads();
    if (tid < 2 * TEAMS) {
      Cplx<T>* at = bufs + (size_t)(tid >> 1) * PS;
      at[fpad((tid & 1) ? N : 0)] = Cplx<T>{T(0), T(0)};
    }
    for (int e = tid; e < P * n; e += kTeamThreads) {
      const int pl = e & (P - 1), j = e >> logP;
      const T v = stage[pl * n + j];
      Cplx<T>* at = bufs + (size_t)(pl >> 1) * PS;
      reinterpret_cast<T*>(at + fpad(j + 1))[pl & 1] = v;
      reinterpret_cast<T*>(at + fpad(L - 1 - j))[pl & 1] = -v;
    }
    __syncthreads();
    const int64_t next = blk + gridDim.x;
    if (next < nblk) {
      block_offsets(next, P, n, inner, npencils, offs[cur ^ 1]);
      __syncthreads();
      stage_block_async(in, offs[cur ^ 1], P, logP, n, inner, stage);
    }
    TeamPasses<T, LOGL, LOGL, 1, TS>::run(a, ptw, tl, bar);
    __syncthreads();
    for (int e = tid; e < P * n; e += kTeamThreads) {
      const int pl = e & (P - 1), k = e >> logP;
      const Cplx<T> Z = bufs[(size_t)(pl >> 1) * PS + fpad(k + 1)];
      const T val = (pl & 1) ? Z.re * scale : -Z.im * scale;
      const int64_t o = offs[cur][pl];
      if (o >= 0) out[o + (int64_t)k * inner] = val;
    }
  }
}

// Pass twiddle tables of one length 2^logl, in pass order, each laid out [r][k] (k fastest):
// entry = e^{-2 pi i k r / (NS R)}, evaluated in float64 and rounded to T.  HALF selects the
// radix plan of the half-length form.
template <typename T, int PLAN>
__global__ void pass_twiddle_kernel(int logl, int total, Cplx<T>* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int e0 = 0, ns = 1, left = logl;
  while (left > 0) {
    const int rb = PLAN == kPlanHalf   ? half_pass_bits<T>(left, logl)
                   : PLAN == kPlanTeam ? team_pass_bits(left)
                   : PLAN == kPlanTwo  ? two_pass_bits(left, logl)
                                       : pass_bits<T>(left, logl);
    const int R = 1 << rb;
    if (ns > 1) {
      if (e < e0 + ns * R) {
        const int r = (e - e0) / ns, k = (e - e0) - r * ns;
        double sn, cs;
        sincospi(2.0 * (double)(k * r) / (double)(ns * R), &sn, &cs);
        out[e] = Cplx<T>{(T)cs, (T)(-sn)};
        return;
      }
      e0 += ns * R;
    }
    ns *= R;
    left -= rb;
  }
}

// sin(pi j / N), j < N (the fold of the half-length form)
template <typename T>
__global__ void sin_table_kernel(int N, T* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) out[j] = (T)sinpi((double)j / (double)N);
}

// (2 sin(pi j / N) + 1, 2 sin(pi j / N) - 1), j < N: the fold of the half-length form scaled by
// two, y_j = (2s + 1) x_j + (2s - 1) x_{N-j}, one multiplication and one FMA per value
template <typename T>
__global__ void fold_table_kernel(int N, Cplx<T>* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) {
    const double s2 = 2.0 * sinpi((double)j / (double)N);
    out[j] = Cplx<T>{(T)(s2 + 1.0), (T)(s2 - 1.0)};
  }
}

// Device-resident tables (pass twiddles, the fold's sines), built once per device and length.
template <typename T, int PLAN>
const Cplx<T>* pass_twiddles(int logl, int total, cudaStream_t st) {
  static Cplx<T>* table[64][12] = {};
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || logl < 0 || logl > 11) return nullptr;
  if (table[dev][logl]) return table[dev][logl];
  Cplx<T>* p = nullptr;
  if (cudaMalloc((void**)&p, sizeof(Cplx<T>) * (size_t)std::max(total, 1)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (total > 0) pass_twiddle_kernel<T, PLAN><<<(total + 255) / 256, 256, 0, st>>>(logl, total, p);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p);
    return nullptr;
  }
  table[dev][logl] = p;
  return p;
}

template <typename T>
const Cplx<T>* fold_pairs(int logn, cudaStream_t st) {
  static Cplx<T>* table[64][12] = {};
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || logn < 0 || logn > 11) return nullptr;
  if (table[dev][logn]) return table[dev][logn];
  const int N = 1 << logn;
  Cplx<T>* p = nullptr;
  if (cudaMalloc((void**)&p, sizeof(Cplx<T>) * (size_t)N) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  fold_table_kernel<T><<<(N + 255) / 256, 256, 0, st>>>(N, p);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p);
    return nullptr;
  }
  table[dev][logn] = p;
  return p;
}

template <typename T>
const T* half_sines(int logn, cudaStream_t st) {
  static T* table[64][12] = {};
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || logn < 0 || logn > 11) return nullptr;
  if (table[dev][logn]) return table[dev][logn];
  const int N = 1 << logn;
  T* p = nullptr;
  if (cudaMalloc((void**)&p, sizeof(T) * (size_t)N) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  sin_table_kernel<T><<<(N + 255) / 256, 256, 0, st>>>(N, p);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p);
    return nullptr;
  }
  table[dev][logn] = p;
  return p;
}

// warps per CTA: as many (up to 8, float64 up to 4) as still give >= 2 CTAs per SM
template <typename T>
pe_status fft_grid(const void* kern, int64_t npencils, size_t smem_per_warp, size_t stage_per_pencil,
                   int* warps_out, size_t* smem_out, int64_t* grid_out) {
  int dev = 0, sms = 0;
  PE_CUDA_TRY(cudaGetDevice(&dev));
  PE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int warps = sizeof(T) == 4 ? 8 : 4;
  while (warps > 1 && (npencils + 2 * warps - 1) / (2 * warps) < 2 * (int64_t)sms) warps >>= 1;
  const int P = 2 * warps;
  // pair buffers, two offset lists, and (strided launches) the staged rows of one block
  const size_t smem = smem_per_warp * (size_t)warps + 2 * sizeof(int64_t) * P + stage_per_pencil * P;
  if (smem > 48 * 1024) PE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  PE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem));
  const int64_t nblk = (npencils + P - 1) / P;
  *grid_out = std::max<int64_t>(1, std::min<int64_t>(nblk, (int64_t)sms * std::max(per_sm, 1)));
  *warps_out = warps;
  *smem_out = smem;
  return PE_OK;
}

// DHT of periodic pencils with n = N = 2^LOGN points
template <typename T, int LOGN>
pe_status fft_dht_launch(const T* in, T* out, int64_t inner, int64_t npencils, cudaStream_t st) {
  constexpr int N = 1 << LOGN, PADN = N + N / 16;
  constexpr int NTW = half_tw_entries<T>(LOGN, 1, LOGN);
  const Cplx<T>* ptw = pass_twiddles<T, kPlanHalf>(LOGN, NTW, st);
  if (!ptw) return pe_fail(PE_ECUDA, "dst: twiddle table allocation failed");
  auto kern = dst_half_warp_kernel<T, LOGN, true>;
  int warps = 1;
  size_t smem = 0;
  int64_t grid = 1;
  PE_TRY(fft_grid<T>((const void*)kern, npencils, sizeof(Cplx<T>) * (PADN + 1), inner > 1 ? sizeof(T) * N : 0, &warps,
                     &smem, &grid));
  const T scale = (T)(1.0 / sqrt((double)N));
  kern<<<(unsigned)grid, warps * 32, smem, st>>>(in, out, N, inner, npencils, scale, ptw, nullptr);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

template <typename T>
pe_status dht_fft_axis(const T* in, T* out, int64_t outer, int n, int64_t inner, cudaStream_t st, bool* done) {
  const int64_t np = outer * inner;
  *done = true;
  switch (n) {
    case 128: return fft_dht_launch<T, 7>(in, out, inner, np, st);
    case 256: return fft_dht_launch<T, 8>(in, out, inner, np, st);
    case 512: return fft_dht_launch<T, 9>(in, out, inner, np, st);
    case 1024: return fft_dht_launch<T, 10>(in, out, inner, np, st);
    default:
      break;
  }
  *done = false;
  return PE_OK;
}

template <typename T, int LOGN>
pe_status fft_half_launch(const T* in, T* out, int n, int64_t inner, int64_t npencils, cudaStream_t st) {
  constexpr int N = 1 << LOGN, PADN = N + N / 16;
  constexpr int NTW = half_tw_entries<T>(LOGN, 1, LOGN);
  const Cplx<T>* ptw = pass_twiddles<T, kPlanHalf>(LOGN, NTW, st);
  const Cplx<T>* fold = fold_pairs<T>(LOGN, st);
  if (!ptw || !fold) return pe_fail(PE_ECUDA, "dst: twiddle table allocation failed");
  auto kern = dst_half_warp_kernel<T, LOGN>;
  int warps = 1;
  size_t smem = 0;
  int64_t grid = 1;
  PE_TRY(fft_grid<T>((const void*)kern, npencils, sizeof(Cplx<T>) * (PADN + 1), inner > 1 ? sizeof(T) * n : 0, &warps,
                     &smem, &grid));
  const T scale = (T)(0.25 * sqrt(2.0 / (double)N));  // half_dst_pair leaves the sums times four
  kern<<<(unsigned)grid, warps * 32, smem, st>>>(in, out, n, inner, npencils, scale, ptw, fold);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

template <typename T, int LOGL>
pe_status fft_warp_launch(const T* in, T* out, int n, int64_t inner, int64_t npencils, T scale, cudaStream_t st) {
  constexpr int L = 1 << LOGL, PADL = L + L / 16;
  constexpr int NTW = pass_tw_entries<T>(LOGL, 1, LOGL);
  const Cplx<T>* ptw = pass_twiddles<T, kPlanWarp>(LOGL, NTW, st);
  if (!ptw) return pe_fail(PE_ECUDA, "dst: pass twiddle table allocation failed");
  auto kern = dst_fft_warp_kernel<T, LOGL>;
  int warps = 1;
  size_t smem = 0;
  int64_t grid = 1;
  PE_TRY(fft_grid<T>((const void*)kern, npencils, sizeof(Cplx<T>) * (PADL + 1), inner > 1 ? sizeof(T) * n : 0, &warps,
                     &smem, &grid));
  kern<<<(unsigned)grid, warps * 32, smem, st>>>(in, out, n, inner, npencils, scale, ptw);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

template <typename T, int LOGL, int TW>
pe_status fft_team_launch(const T* in, T* out, int n, int64_t inner, int64_t npencils, T scale, cudaStream_t st) {
  constexpr int L = 1 << LOGL, PADL = L + L / 16, TS = 32 * TW, TEAMS = kTeamThreads / TS, P = 2 * TEAMS;
  constexpr int NTW = team_tw_entries(LOGL, 1);
  const Cplx<T>* ptw = pass_twiddles<T, kPlanTeam>(LOGL, NTW, st);
  if (!ptw) return pe_fail(PE_ECUDA, "dst: pass twiddle table allocation failed");
  auto kern = dst_fft_team_kernel<T, LOGL, TW>;
  const size_t smem = sizeof(Cplx<T>) * (size_t)TEAMS * (PADL + 1) + 2 * sizeof(int64_t) * P +
                      (inner > 1 ? sizeof(T) * (size_t)P * n : 0);
  if (smem > 48 * 1024) PE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, per_sm = 0;
  PE_CUDA_TRY(cudaGetDevice(&dev));
  PE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTeamThreads, smem));
  const int64_t work = inner > 1 ? (npencils + P - 1) / P : ((npencils + 1) / 2 + TEAMS - 1) / TEAMS;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(work, (int64_t)sms * std::max(per_sm, 1)));
  kern<<<(unsigned)grid, kTeamThreads, smem, st>>>(in, out, n, inner, npencils, scale, ptw);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

// the two-pass float32 kernels at n = 255 (L = 512); warps per CTA: 8, or 1 when the pencils
// are too few to give every SM a CTA of 8 warps (the mixed form's transforms of small grids)
template <typename TI, typename TO>
pe_status fft512_contig_launch(const TI* in, TO* out, int64_t npencils, float scale, cudaStream_t st) {
  constexpr int PS = 512 + 512 / 16 + 1;
  const size_t smem8 = sizeof(Cplx<float>) * 2 * PS * 8;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [smem8] {
    attr = cudaFuncSetAttribute(dst512_contig_kernel<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem8);
  });
  if (attr != cudaSuccess) return pe_cuda_fail(attr, "dst: shared-memory attribute");
  const Cplx<float>* tw2 = pass_twiddles<float, kPlanTwo>(9, 16 * 32, st);
  if (!tw2) return pe_fail(PE_ECUDA, "dst: twiddle table allocation failed");
  int dev = 0, sms = 0, per_sm = 0;
  PE_CUDA_TRY(cudaGetDevice(&dev));
  PE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t nquads = ((npencils + 1) / 2 + 1) / 2;
  const int warps = nquads < 8 * (int64_t)sms ? 1 : 8;
  const size_t smem = sizeof(Cplx<float>) * 2 * PS * warps;
  PE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dst512_contig_kernel<TI, TO>, 32 * warps, smem));
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((nquads + warps - 1) / warps,
                                                              (int64_t)sms * std::max(per_sm, 1)));
  PE_CUDA_TRY(launch_pdl(dst512_contig_kernel<TI, TO>, dim3((unsigned)grid), dim3(32 * warps), smem, st, in, out,
                         npencils, scale, tw2));
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

constexpr int kStridedWarps = 8;  // warps per CTA of the strided two-pass kernels (32 pencils per block)
template <int W, typename TI, typename TO>
pe_status fft512_strided_launch_w(const TI* in, TO* out, int64_t inner, int64_t npencils, float scale,
                                  cudaStream_t st) {
  constexpr int PS = 512 + 512 / 16 + 1, P = 4 * W;
  const size_t smem = sizeof(float) * 2 * 255 * (P + 2) + sizeof(Cplx<float>) * 2 * PS * W;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [smem] {
    attr = cudaFuncSetAttribute(dst512_strided_kernel<W, TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  });
  if (attr != cudaSuccess) return pe_cuda_fail(attr, "dst: shared-memory attribute");
  const Cplx<float>* tw2 = pass_twiddles<float, kPlanTwo>(9, 16 * 32, st);
  if (!tw2) return pe_fail(PE_ECUDA, "dst: twiddle table allocation failed");
  int dev = 0, sms = 0, per_sm = 0;
  PE_CUDA_TRY(cudaGetDevice(&dev));
  PE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dst512_strided_kernel<W, TI, TO>, 32 * W, smem));
  const int64_t nblk = (npencils + P - 1) / P;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(nblk, (int64_t)sms * std::max(per_sm, 1)));
  PE_CUDA_TRY(launch_pdl(dst512_strided_kernel<W, TI, TO>, dim3((unsigned)grid), dim3(32 * W), smem, st, in, out,
                         inner, npencils, scale, tw2));
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

template <typename TI, typename TO>
pe_status fft512_strided_launch(const TI* in, TO* out, int64_t inner, int64_t npencils, float scale, cudaStream_t st) {
  int dev = 0, sms = 0;
  PE_CUDA_TRY(cudaGetDevice(&dev));
  PE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (npencils < 4 * kStridedWarps * (int64_t)sms)
    return fft512_strided_launch_w<1, TI, TO>(in, out, inner, npencils, scale, st);
  return fft512_strided_launch_w<kStridedWarps, TI, TO>(in, out, inner, npencils, scale, st);
}

// the two-pass float32 kernel: strided pencils of n = 511 (L = 1024)
pe_status fft1024_strided_launch(const float* in, float* out, int64_t inner, int64_t npencils, float scale,
                                 cudaStream_t st) {
  constexpr int PS = 1024 + 1024 / 16 + 1, W = kStridedWarps, P = 4 * W;
  const size_t smem = sizeof(float) * 2 * 511 * (P + 2) + sizeof(Cplx<float>) * PS * W;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [smem] {
    attr = cudaFuncSetAttribute(dst1024_strided_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (attr != cudaSuccess) return pe_cuda_fail(attr, "dst: shared-memory attribute");
  const Cplx<float>* tw2 = pass_twiddles<float, kPlanTwo>(10, 32 * 32, st);
  if (!tw2) return pe_fail(PE_ECUDA, "dst: twiddle table allocation failed");
  int dev = 0, sms = 0, per_sm = 0;
  PE_CUDA_TRY(cudaGetDevice(&dev));
  PE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dst1024_strided_kernel<W>, 32 * W, smem));
  if (per_sm < 1) return pe_fail(PE_ECUDA, "dst: the 1024-point strided kernel does not fit an SM");
  const int64_t nblk = (npencils + P - 1) / P;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(nblk, (int64_t)sms * per_sm));
  PE_CUDA_TRY(launch_pdl(dst1024_strided_kernel<W>, dim3((unsigned)grid), dim3(32 * W), smem, st, in, out, inner,
                         npencils, scale, tw2));
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

template <typename T>
pe_status fft_warp_axis(const T* in, T* out, int64_t outer, int n, int64_t inner, int logL, cudaStream_t st,
                        bool* done) {
  const int64_t np = outer * inner;
  const T scale = (T)(0.5 * sqrt(2.0 / (double)(n + 1)));
  *done = true;
  // float64: the half-length form (half the FP64 work; its prefix sum amplifies the FFT's
  // rounding by about sqrt(n+1)/2, harmless at float64 precision).  float32: the full
  // odd extension, whose error stays at the FFT's own level.
  if constexpr (sizeof(T) == 8) {
    switch (logL) {
      case 5: return fft_warp_launch<T, 5>(in, out, n, inner, np, scale, st);
      case 6: return fft_warp_launch<T, 6>(in, out, n, inner, np, scale, st);
      case 7: return fft_warp_launch<T, 7>(in, out, n, inner, np, scale, st);
      case 8: return fft_half_launch<T, 7>(in, out, n, inner, np, st);
      case 9: return fft_half_launch<T, 8>(in, out, n, inner, np, st);
      case 10: return fft_half_launch<T, 9>(in, out, n, inner, np, st);
      case 11: return fft_half_launch<T, 10>(in, out, n, inner, np, st);
      default:
        break;
    }
  } else {
    switch (logL) {
      case 5: return fft_warp_launch<T, 5>(in, out, n, inner, np, scale, st);
      case 6: return fft_warp_launch<T, 6>(in, out, n, inner, np, scale, st);
      case 7: return fft_warp_launch<T, 7>(in, out, n, inner, np, scale, st);
      case 8: return fft_warp_launch<T, 8>(in, out, n, inner, np, scale, st);
      case 9:
        if (inner == 1) return fft512_contig_launch(in, out, np, scale, st);
        return fft512_strided_launch(in, out, inner, np, scale, st);
      // 1024 and 2048 points: two or four warps per pencil pair (16 complex values per lane)
      case 10:
        if (inner > 1) return fft1024_strided_launch(in, out, inner, np, scale, st);
        return fft_team_launch<T, 10, 2>(in, out, n, inner, np, scale, st);
      case 11: return fft_team_launch<T, 11, 4>(in, out, n, inner, np, scale, st);
      default:
        break;
    }
  }
  *done = false;
  return PE_OK;
}

// Pencil count up to which the block-wide kernel is used (two pencils per SM of 152).
constexpr int64_t kFewPencils = 2 * 152;

template <typename T>
pe_status fft_axis(const T* in, T* out, int64_t outer, int n, int64_t inner, int logL, cudaStream_t st) {
  const int L = 1 << logL;
  const int64_t npencils = outer * inner;
  const Cplx<T>* tw = twiddles<T>(logL, st);
  if (!tw) return pe_fail(PE_ECUDA, "dst: twiddle table allocation failed");
  bool done = false;
  // Few pencils (small problems, the per-axis source factors): a warp per pencil pair
  // would leave most SMs idle behind the FFT's chain of dependent float64 latencies, so
  // those go to the block-wide kernels, which spread every pencil pair over a CTA (float64
  // in the half-length form from N = n + 1 = 16 on).
  if (npencils > kFewPencils) PE_TRY(fft_warp_axis<T>(in, out, outer, n, inner, logL, st, &done));
  if (done) return PE_OK;
  if constexpr (sizeof(T) == 8) {
    const int logN = logL - 1;
    if (npencils <= kFewPencils && logN >= 4) {
      const Cplx<T>* twN = twiddles<T>(logN, st);
      const T* sinN = half_sines<T>(logN, st);
      if (!twN || !sinN) return pe_fail(PE_ECUDA, "dst: twiddle table allocation failed");
      const int N = 1 << logN;
      const size_t smem = sizeof(Cplx<T>) * ((size_t)2 * N + 1 + 8);
      const int threads = N / 2 >= 256 ? 256 : (N / 2 >= 128 ? 128 : (N / 2 >= 64 ? 64 : 32));
      PE_CUDA_TRY(launch_pdl(dst_half_block_kernel<T>, dim3((unsigned)((npencils + 1) / 2)), dim3(threads), smem, st,
                             in, out, n, logN, inner, npencils, (T)sqrt(2.0 / (double)N), twN, sinN));
      PE_CUDA_TRY(cudaGetLastError());
      return PE_OK;
    }
  }
  // few pencils, short transforms (n + 1 < 16) and float64 at n + 1 = 1024: the block-wide radix-2 kernel;
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
  PE_CUDA_TRY(launch_pdl(dst_fft_kernel<T>, dim3((unsigned)want_ctas), dim3(threads), smem, st, in, out, n, logL, inner,
                         npencils, pairs, scale, tw));
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

template <typename T>
pe_status dst_axis(const T* S, const T* in, T* out, int64_t outer, int n, int64_t inner, cudaStream_t st,
                   int periodic = 0) {
  int logL = 0;
  if (!periodic && fft_size_ok(n, &logL)) return fft_axis<T>(in, out, outer, n, inner, logL, st);
  if (periodic) {
    bool done = false;
    PE_TRY(dht_fft_axis<T>(in, out, outer, n, inner, st, &done));
    if (done) return PE_OK;
  }
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
pe_status dst_nd(int d, const int* n, T* const* S, const T* in, T* out, T* tmp, cudaStream_t st,
                 const int* per = nullptr) {
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
    PE_TRY(dst_axis<T>(S[a], src, dst, outer, n[a], inner, st, per ? per[a] : 0));
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

// The library's own stream-ordered memory pool of a device for the scratch of the standalone
// transforms: it keeps freed memory (release threshold unlimited), so that repeated calls of
// one size do not map and unmap it from the driver each time; the process's default pool is
// left as it is.
cudaMemPool_t scratch_pool() {
  static cudaMemPool_t pools[64] = {};
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

template <typename T>
cudaError_t scratch_alloc(T** p, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool = scratch_pool();
  return pool ? cudaMallocFromPoolAsync((void**)p, bytes, pool, st) : cudaMallocAsync((void**)p, bytes, st);
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
  // the DST-I matrix only of axes without an FFT form (n + 1 not a power of two)
  for (int a = 0; a < d && rc == PE_OK; ++a) {
    int logL = 0;
    if (fft_size_ok(nn[a], &logL)) continue;
    cudaError_t e = scratch_alloc(&S[a], sizeof(T) * (size_t)nn[a] * nn[a], st);
    if (e != cudaSuccess) { rc = pe_cuda_fail(e, "cudaMallocAsync(S)"); break; }
    dim3 grid((nn[a] + 127) / 128, nn[a]);
    dst_matrix_kernel_t<T><<<grid, 128, 0, st>>>(nn[a], S[a]);
  }
  if (rc == PE_OK && (d > 1 || in == out)) {
    cudaError_t e = scratch_alloc(&tmp, sizeof(T) * (size_t)ndof, st);
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
                       cudaStream_t st, int periodic) {
  return dst_axis<double>(S, in, out, outer, n, inner, st, periodic);
}

pe_status dst_axis_f32(const float* S, const float* in, float* out, int64_t outer, int n, int64_t inner,
                       cudaStream_t st, int periodic) {
  return dst_axis<float>(S, in, out, outer, n, inner, st, periodic);
}

// Per-axis source factors (a3), all axes in one launch: loads -> DST-I along the axis ->
// division by mu^M.  Returns *done = false (nothing launched) unless every axis is a
// Dirichlet axis with n_a + 1 a power of two between 16 and 1024.
pe_status axis_factors_fused(pe_ctx* c, int R, const double* loads, double* fac, float* fac32, bool* done) {
  *done = false;
  AxisFactorJob J{};
  J.d = c->g.d;
  J.R = R;
  size_t smem = 0;
  for (int a = 0; a < c->g.d; ++a) {
    int logL = 0;
    if (c->g.per[a] || !fft_size_ok(c->g.n[a], &logL) || logL - 1 < 4) return PE_OK;
    J.n[a] = c->g.n[a];
    J.off[a] = c->g.off[a];
    J.logN[a] = logL - 1;
    J.tw[a] = twiddles<double>(logL - 1, c->stream);
    J.sinN[a] = half_sines<double>(logL - 1, c->stream);
    if (!J.tw[a] || !J.sinN[a]) return pe_fail(PE_ECUDA, "dst: twiddle table allocation failed");
    smem = std::max(smem, sizeof(Cplx<double>) * ((size_t)2 * (c->g.n[a] + 1) + 1 + 8));
  }
  int nmax = 1;
  for (int a = 0; a < c->g.d; ++a) nmax = std::max(nmax, c->g.n[a] + 1);
  const int threads = nmax / 2 >= 256 ? 256 : (nmax / 2 >= 128 ? 128 : (nmax / 2 >= 64 ? 64 : 32));
  axis_factor_dst_kernel<<<dim3((unsigned)((R + 1) / 2), (unsigned)c->g.d), threads, smem, c->stream>>>(
      J, loads, c->muM_axis, fac, fac32);
  PE_CUDA_TRY(cudaGetLastError());
  c->launches += 1;
  *done = true;
  return PE_OK;
}

pe_status dst_nd_f64(pe_ctx* c, const double* in, double* out) {
  c->launches += c->gn.d;
  return dst_nd<double>(c->gn.d, c->gn.n, c->S, in, out, c->work1, c->stream, c->gn.per);
}

namespace {
__global__ void f64_to_f32_kernel(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void f32_to_f64_kernel(int64_t n, const float* __restrict__ in, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}
}  // namespace

// Every axis has an FFT form (n + 1 a power of two, or a periodic axis of 128..1024 points),
// so the float32 transform needs no DST-I matrices.
bool dst_nd_f32_ok(const Geom& g) {
  for (int a = 0; a < g.d; ++a) {
    int logL = 0;
    const int n = g.n[a];
    const bool ok = g.per[a] ? (n == 128 || n == 256 || n == 512 || n == 1024) : fft_size_ok(n, &logL);
    if (!ok) return false;
  }
  return true;
}

// The mixed form's transforms between nodal values and modal coefficients (u0 in, the solution
// out): float64 data rounded to float32, the tensor DST-I in float32, widened back to float64.
namespace {
template <typename TI, typename TO>
pe_status fft512_axis(const TI* in, TO* out, int64_t inner, int64_t npencils, float scale, cudaStream_t st) {
  if (inner == 1) return fft512_contig_launch<TI, TO>(in, out, npencils, scale, st);
  return fft512_strided_launch<TI, TO>(in, out, inner, npencils, scale, st);
}
}  // namespace

pe_status dst_nd_mixed(pe_ctx* c, const double* in, double* out) {
  const int64_t nd = c->gn.ndof;
  float* a = c->io32;
  float* b = a + nd;
  float* t = b + nd;
  // every axis n = 255: the two-pass kernels, the first reading the float64 input and the last
  // writing the float64 output (no conversion launches)
  bool two = true;
  for (int ax = 0; ax < c->gn.d; ++ax) two = two && !c->gn.per[ax] && c->gn.n[ax] == 255;
  if (two) {
    const int d = c->gn.d;
    const float scale = (float)(0.5 * sqrt(2.0 / 256.0));
    const int64_t np = nd / 255;
    const float* src = nullptr;
    for (int ax = 0; ax < d; ++ax) {
      int64_t inner = 1;
      for (int q = ax + 1; q < d; ++q) inner *= c->gn.n[q];
      float* dstf = (ax & 1) ? b : a;
      const bool first = ax == 0, last = ax == d - 1;
      pe_status st = PE_OK;
      if (first && last) st = fft512_axis<double, double>(in, out, inner, np, scale, c->stream);
      else if (first) st = fft512_axis<double, float>(in, dstf, inner, np, scale, c->stream);
      else if (last) st = fft512_axis<float, double>(src, out, inner, np, scale, c->stream);
      else st = fft512_axis<float, float>(src, dstf, inner, np, scale, c->stream);
      PE_TRY(st);
      src = dstf;
    }
    c->launches += d;
    return PE_OK;
  }
  const int threads = 256;
  const unsigned blocks = (unsigned)std::min<int64_t>((nd + threads - 1) / threads, 8 * 152);
  f64_to_f32_kernel<<<blocks, threads, 0, c->stream>>>(nd, in, a);
  PE_TRY(dst_nd<float>(c->gn.d, c->gn.n, c->S32, a, b, t, c->stream, c->gn.per));
  f32_to_f64_kernel<<<blocks, threads, 0, c->stream>>>(nd, b, out);
  c->launches += c->gn.d + 2;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
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
// Some callers cannot call cudaMalloc: applications that own a fixed memory pool and
// forbid the runtime allocator, hosts whose device memory is fully reserved up front,
// and latency-critical loops that must not enter the allocator (cudaMalloc and cudaFree
// can synchronise the device).  This entry point keeps every scratch
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
