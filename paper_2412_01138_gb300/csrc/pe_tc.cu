// Tensor-core tensor DST-I (mixed precision) on 5th-generation tensor cores.
//
// Each axis pass of the orthonormal DST-I (the diagonalising transform of Sec. 2.3)
// is a contraction out[p][j] = sum_k X_p[k] S[k][j] over the pencils p of that axis.
// Float32 data are split into nsplit bfloat16 terms x = x0 + x1 (+ x2) and the
// products that carry about 2^-24 of relative weight are concatenated along K,
//   nsplit 2:  [x0 x0 x1] . [s0 s1 s0]                (about 16 bits)
//   nsplit 3:  [x0 x0 x1 x0 x1 x2] . [s0 s1 s0 s2 s1 s0]  (about 24 bits),
// so one bfloat16 GEMM with float32 accumulation gives the pass.
//
// GEMM kernel (one CTA per 128 x 128 output tile, 128 threads):
//   * operands staged in shared memory by TMA (cp.async.bulk.tensor, 2D tiled
//     maps, boxes of 8 elements x rows, i.e. the no-swizzle K-major core-matrix
//     layout: K-chunk c of a stage at c * rows * 16 bytes, 8-row groups 128 bytes
//     apart), two stages, mbarrier transaction counts;
//   * one thread issues tcgen05.mma (kind::f16, bf16 x bf16 -> f32, M = 128,
//     N = 128, K = 16 per instruction) with the accumulators in tensor memory,
//     tcgen05.commit releases each stage.  K tile kt accumulates into TMEM
//     accumulator kt % 4 (4 x 128 columns): the tensor core's float32
//     accumulation error grows with the number of products summed into one
//     accumulator, so four partial sums, added in float32 with round-to-nearest
//     in the epilogue, cut it about fourfold;
//   * epilogue: every warp reads its 32 TMEM lanes (tcgen05.ld 32x32b) of each
//     accumulator and writes its rows straight to the strided destination.
// Every mbarrier wait is bounded (about a second of clock cycles); on expiry the
// CTA records an error code, skips the epilogue, frees its tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "pe_internal.h"

namespace {

constexpr int TBM = 128;  // rows of a CTA tile (TMEM lanes)
constexpr int TBN = 128;  // columns of a CTA tile (TMEM columns)
constexpr int TBK = 64;   // K per stage (4 MMAs of K = 16)
constexpr int TSTAGES = 2;
constexpr int NACC = 4;   // TMEM accumulators (NACC * TBN = 512 columns)
constexpr int A_STAGE_BYTES = TBM * TBK * 2;  // 16 KB
constexpr int B_STAGE_BYTES = TBN * TBK * 2;  // 16 KB
constexpr int STAGE_BYTES = A_STAGE_BYTES + B_STAGE_BYTES;
// shared memory: 1 KB alignment slack + stages + a guard region so that no
// descriptor offset can leave the allocation
constexpr int TC_SMEM = 1024 + TSTAGES * STAGE_BYTES + 64 * 1024;
constexpr long long WAIT_CYCLES = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension byte
// offset (between the two K-adjacent core matrices of one K = 16 MMA), stride byte
// offset (between 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, N, M.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: false once about WAIT_CYCLES have passed
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

struct TcOut {
  float* out;
  int64_t rows_valid;  // pencils
  int n_valid;         // output length of the pass
  int64_t inner;       // pencil p lives at (p / inner) * n * inner + j * inner + (p % inner)
  float scale;
};

__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                         const __grid_constant__ CUtensorMap mapB, int k_tiles,
                                                         TcOut o, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[TSTAGES];
  __shared__ __align__(8) uint64_t empty_bar[TSTAGES];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TBM, n0 = blockIdx.y * TBN;

  if (tid == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(NACC * TBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (tid == 0) {
    const uint32_t idesc = instr_desc_bf16(TBM, TBN);
    auto load_stage = [&](int kt, int s) {
      unsigned char* A = smem + s * STAGE_BYTES;
      unsigned char* Bm = A + A_STAGE_BYTES;
      mbar_expect_tx(&full_bar[s], STAGE_BYTES);
      for (int c = 0; c < TBK / 8; ++c) {
        tma_load_2d(A + c * (TBM * 16), &mapA, kt * TBK + c * 8, m0, &full_bar[s]);
        tma_load_2d(Bm + c * (TBN * 16), &mapB, kt * TBK + c * 8, n0, &full_bar[s]);
      }
    };
    for (int s = 0; s < TSTAGES && s < k_tiles; ++s) load_stage(s, s);
    bool ok = true;
    for (int kt = 0; kt < k_tiles && ok; ++kt) {
      const int s = kt % TSTAGES;
      const uint32_t ph = (uint32_t)((kt / TSTAGES) & 1);
      if (!mbar_wait(&full_bar[s], ph)) {
        ok = false;
        atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES);
      const uint32_t b0 = a0 + A_STAGE_BYTES;
      const uint32_t dacc = tmem + (uint32_t)((kt % NACC) * TBN);
      for (int kk = 0; kk < TBK / 16; ++kk) {
        const uint64_t da = smem_desc(a0 + (2 * kk) * (TBM * 16), TBM * 16, 128);
        const uint64_t db = smem_desc(b0 + (2 * kk) * (TBN * 16), TBN * 16, 128);
        mma_bf16(dacc, da, db, idesc, (kt >= NACC || kk > 0) ? 1u : 0u);
      }
      mma_commit(&empty_bar[s]);
      if (kt + TSTAGES < k_tiles) {
        if (!mbar_wait(&empty_bar[s], ph)) {
          ok = false;
          atomicExch(err, 2);
          break;
        }
        load_stage(kt + TSTAGES, s);
      }
    }
    if (ok) {
      const int last = k_tiles - 1;
      if (!mbar_wait(&empty_bar[last % TSTAGES], (uint32_t)((last / TSTAGES) & 1))) {
        ok = false;
        atomicExch(err, 3);
      }
    }
    if (!ok) s_fail = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (!s_fail) {
    // epilogue: warp w owns TMEM lanes 32w..32w+31 (rows m0 + 32w + lane)
    const int64_t p = (int64_t)m0 + 32 * warp + lane;
    const bool row_ok = p < o.rows_valid;
    const int64_t ob = row_ok ? (p / o.inner) * (int64_t)o.n_valid * o.inner + (p % o.inner) : 0;
    const int nacc = k_tiles < NACC ? k_tiles : NACC;
    for (int c = 0; c < TBN / 16; ++c) {
      float sum[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) sum[e] = 0.f;
      for (int ac = 0; ac < nacc; ++ac) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(ac * TBN + c * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 16; ++e) sum[e] += __uint_as_float(r[e]);
      }
      if (row_ok) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int j = n0 + c * 16 + e;
          if (j < o.n_valid) o.out[ob + (int64_t)j * o.inner] = sum[e] * o.scale;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NACC * TBN) : "memory");
  }
}

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split3(float x, __nv_bfloat16* h) {
  const __nv_bfloat16 a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  const __nv_bfloat16 b = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b);
  h[0] = a;
  h[1] = b;
  h[2] = __float2bfloat16_rn(r2);
}

// segment order of the K-concatenated operands (index of the split term per segment)
__constant__ int c_segA[6] = {0, 0, 1, 0, 1, 2};
__constant__ int c_segB[6] = {0, 1, 0, 2, 1, 0};

// A'[p][seg * kpad + k] for pencils p < rows_pad (zero beyond rows / n); 64 x 64 tiles
// through shared memory so that both the strided read and the row write coalesce.
__global__ void split_pencils_kernel(const float* __restrict__ in, int n, int64_t inner, int64_t rows, int kpad,
                                     int nseg, __nv_bfloat16* __restrict__ Ap) {
  __shared__ float tile[64][65];
  const int64_t p0 = (int64_t)blockIdx.x * 64;
  const int k0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 256 threads: 64 x 4
  for (int r = ty; r < 64; r += 4) {
    float v = 0.f;
    int64_t p;
    int k;
    if (inner == 1) {  // contiguous along k: threads walk k
      p = p0 + r;
      k = k0 + tx;
    } else {           // contiguous along p: threads walk p
      p = p0 + tx;
      k = k0 + r;
    }
    if (p < rows && k < n) v = in[(p / inner) * (int64_t)n * inner + (int64_t)k * inner + (p % inner)];
    if (inner == 1) tile[r][tx] = v;
    else tile[tx][r] = v;
  }
  __syncthreads();
  const int kk = tx;
  for (int r = ty; r < 64; r += 4) {
    const int64_t p = p0 + r;
    const int k = k0 + kk;
    __nv_bfloat16 h[3];
    split3(tile[r][kk], h);
    for (int s = 0; s < nseg; ++s) Ap[p * (int64_t)nseg * kpad + (int64_t)s * kpad + k] = h[c_segA[s]];
  }
}

// B'[j][seg * kpad + k] = split term of S[j][k] = sqrt(2/(n+1)) sin(pi (j+1)(k+1)/(n+1)) (the scale
// is applied in the epilogue), zero padded to npad_rows x kpad
__global__ void split_dst_matrix_kernel(int n, int kpad, int nseg, __nv_bfloat16* __restrict__ Bp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (k >= kpad) return;
  float v = 0.f;
  if (j < n && k < n) {
    const int64_t period = 2 * (int64_t)(n + 1);
    const int64_t m = ((int64_t)(j + 1) * (k + 1)) % period;
    v = (float)sinpi((double)m / (double)(n + 1));
  }
  __nv_bfloat16 h[3];
  split3(v, h);
  for (int s = 0; s < nseg; ++s) Bp[(int64_t)j * nseg * kpad + (int64_t)s * kpad + k] = h[c_segB[s]];
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  }
  return fn;
}

pe_status make_map(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return pe_fail(PE_ECUDA, "tensor-core DST: cuTensorMapEncodeTiled unavailable");
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {8, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return pe_fail(PE_ECUDA, "tensor-core DST: cuTensorMapEncodeTiled failed");
  return PE_OK;
}

inline int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// One axis pass: out = S applied along the axis (pencils of length n, stride inner).
pe_status tc_axis(const float* in, float* out, int64_t outer, int n, int64_t inner, int nsplit, __nv_bfloat16* Ap,
                  __nv_bfloat16* Bp, int* err, cudaStream_t st) {
  const int nseg = nsplit == 2 ? 3 : 6;
  const int kpad = (int)rup(n, TBK);
  const int64_t kprime = (int64_t)nseg * kpad;
  const int64_t rows = outer * inner;
  const int64_t rows_pad = rup(rows, TBM);
  const int npad = (int)rup(n, TBN);
  dim3 g1((unsigned)(rows_pad / 64), kpad / 64);
  split_pencils_kernel<<<g1, 256, 0, st>>>(in, n, inner, rows, kpad, nseg, Ap);
  dim3 g2((kpad + 127) / 128, npad);
  split_dst_matrix_kernel<<<g2, 128, 0, st>>>(n, kpad, nseg, Bp);
  PE_CUDA_TRY(cudaGetLastError());
  CUtensorMap mA, mB;
  PE_TRY(make_map(&mA, Ap, (uint64_t)kprime, (uint64_t)rows_pad, TBM));
  PE_TRY(make_map(&mB, Bp, (uint64_t)kprime, (uint64_t)npad, TBN));
  TcOut o{out, rows, n, inner, (float)sqrt(2.0 / (double)(n + 1))};
  dim3 grid((unsigned)(rows_pad / TBM), (unsigned)(npad / TBN));
  if (grid.x > 2147483647u || grid.y > 65535u) return pe_fail(PE_EINVAL, "tensor-core DST: problem too large");
  tc_gemm_kernel<<<grid, 128, TC_SMEM, st>>>(mA, mB, (int)(kprime / TBK), o, err);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

}  // namespace

extern "C" pe_status pe_dst_tc(int32_t d, const int32_t* n, const float* in, float* out, int32_t nsplit,
                               void* stream) {
  if (d < 1 || d > PE_MAX_D || !n || !in || !out) return pe_fail(PE_EINVAL, "pe_dst_tc: bad arguments");
  if (nsplit != 2 && nsplit != 3) return pe_fail(PE_EINVAL, "pe_dst_tc: nsplit must be 2 or 3");
  int64_t ndof = 1;
  int64_t worstA = 0, worstB = 0;
  for (int a = 0; a < d; ++a) {
    if (n[a] < 1 || n[a] > 1024) return pe_fail(PE_EINVAL, "pe_dst_tc: n_a must be in 1..1024");
    ndof *= n[a];
  }
  const int nseg = nsplit == 2 ? 3 : 6;
  for (int a = 0; a < d; ++a) {
    const int64_t rows = ndof / n[a];
    worstA = std::max<int64_t>(worstA, rup(rows, TBM) * nseg * rup(n[a], TBK));
    worstB = std::max<int64_t>(worstB, rup(n[a], TBN) * nseg * rup(n[a], TBK));
  }
  cudaStream_t st = (cudaStream_t)stream;
  static bool attr_set = false;
  if (!attr_set) {
    PE_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    attr_set = true;
  }
  __nv_bfloat16 *Ap = nullptr, *Bp = nullptr;
  float* tmp = nullptr;
  int* err = nullptr;
  pe_status rc = PE_OK;
  cudaError_t e = cudaMallocAsync((void**)&Ap, sizeof(__nv_bfloat16) * worstA, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&Bp, sizeof(__nv_bfloat16) * worstB, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&tmp, sizeof(float) * ndof, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&err, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e != cudaSuccess) rc = pe_cuda_fail(e, "pe_dst_tc: scratch allocation");
  // ping-pong between tmp and out; a pass never writes the buffer it reads (in may alias out)
  const float* src = in;
  for (int a = 0; a < d && rc == PE_OK; ++a) {
    float* dst = (src == tmp || (src != in && src != out)) ? out : tmp;
    if (src == out) dst = tmp;
    int64_t outer = 1, inner = 1;
    for (int b = 0; b < a; ++b) outer *= n[b];
    for (int b = a + 1; b < d; ++b) inner *= n[b];
    rc = tc_axis(src, dst, outer, n[a], inner, nsplit, Ap, Bp, err, st);
    src = dst;
  }
  if (rc == PE_OK && src != out) {
    e = cudaMemcpyAsync(out, src, sizeof(float) * ndof, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) rc = pe_cuda_fail(e, "pe_dst_tc: copy");
  }
  int herr = 0;
  if (rc == PE_OK) {
    e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = pe_cuda_fail(e, "pe_dst_tc");
  }
  if (Ap) cudaFreeAsync(Ap, st);
  if (Bp) cudaFreeAsync(Bp, st);
  if (tmp) cudaFreeAsync(tmp, st);
  if (err) cudaFreeAsync(err, st);
  if (rc == PE_OK && herr != 0) rc = pe_fail(PE_ETIMEOUT, "pe_dst_tc: a tensor-core pipeline wait expired");
  return rc;
}
