// Tensor-core tensor DST-I (mixed precision) on 5th-generation tensor cores.
//
// Each axis pass of the orthonormal DST-I (the diagonalising transform of Sec. 2.3)
// is a contraction out[p][j] = sum_k X_p[k] S[j][k] over the pencils p of that axis.
// Float32 operands are split into NSPLIT bfloat16 terms x = x0 + x1 (+ x2) and the
// products that carry about 2^-24 of relative weight are summed,
//   NSPLIT 2:  x0 s0 + x0 s1 + x1 s0                         (about 16 bits)
//   NSPLIT 3:  x0 s0 + x0 s1 + x1 s0 + x0 s2 + x1 s1 + x2 s0   (about 24 bits),
// by bfloat16 MMAs with float32 accumulation.
//
// Fused pass kernel (one CTA per 128 pencils x 128 outputs, 160 threads):
//   * warps 0-3 (one pencil row per thread) read the float32 pencils straight from
//     the strided array, split them and store the bfloat16 terms in shared memory
//     in the no-swizzle K-major core-matrix layout (K-chunk c of a term at
//     c * 128 * 16 bytes, row r at r * 16 bytes), so the split operand never goes
//     through HBM; then fence the async proxy and arrive on the stage's barrier;
//   * warp 4, one thread: TMA loads of the split DST matrix (prepared once per pass,
//     2D tiled map, boxes of 8 elements x 128 rows) and the tcgen05.mma issue
//     (kind::f16, M = N = 128, K = 16), accumulators in tensor memory; K tile kt
//     accumulates into TMEM accumulator kt % NACC (partial sums added in float32 in
//     the epilogue: the accumulator's rounding grows with the number of products
//     summed into it); tcgen05.commit releases each stage and finally the tile;
//   * STAGES-deep ring of (A, B) stages with full/empty mbarriers, so the split of
//     the next K tiles and the TMA loads overlap the MMAs;
//   * epilogue (warps 0-3): tcgen05.ld of each lane's row, partial sums added and
//     scaled; strided passes store straight (consecutive lanes are consecutive
//     pencils), the contiguous pass transposes 16-column chunks through shared
//     memory so that each row is written with consecutive addresses.
// Every mbarrier wait is bounded (about half a second of clock cycles); on expiry
// the CTA records an error code, skips the epilogue, frees its tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "pe_internal.h"
#include "pe_tc_common.cuh"

namespace {

constexpr int TBM = 128;  // pencils of a CTA tile (TMEM lanes)
constexpr int TBN = 128;  // outputs of a CTA tile (TMEM columns per accumulator)
constexpr int TBK = 32;   // K per stage (2 MMA K-steps of 16)
constexpr int A_TERM = TBM * TBK * 2;  // one bfloat16 split term of the A stage: 8 KB
constexpr int B_TERM = TBN * TBK * 2;  // one bfloat16 split term of the B stage: 8 KB
constexpr int TC_THREADS = 160;

constexpr int XROW = TBK + 1;             // float32 staging row (one pad word: conflict-free)
constexpr int X_SLOT = TBM * XROW * 4;     // one float32 K tile of the 128 pencils

// per split depth: STAGES split-operand stages, SF float32 staging slots (the pencils'
// K tiles are fetched by cp.async up to SF tiles ahead of the split), NACC accumulators
template <int NSPLIT>
struct TcCfg;
template <>
struct TcCfg<2> {
  static constexpr int STAGES = 4, SF = 4, NACC = 4;
};
template <>
struct TcCfg<3> {
  static constexpr int STAGES = 3, SF = 3, NACC = 4;
};
template <int NSPLIT>
constexpr int tc_smem_bytes() {
  return 1024 + TcCfg<NSPLIT>::STAGES * NSPLIT * (A_TERM + B_TERM) + TcCfg<NSPLIT>::SF * X_SLOT;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// named barrier over the four converter / epilogue warps
__device__ __forceinline__ void conv_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// (A term, B term) of every product kept at each split depth
__device__ __forceinline__ void prod_terms(int nsplit, int q, int* ta, int* tb) {
  const int a2[3] = {0, 0, 1}, b2[3] = {0, 1, 0};
  const int a3[6] = {0, 0, 1, 0, 1, 2}, b3[6] = {0, 1, 0, 2, 1, 0};
  *ta = nsplit == 2 ? a2[q] : a3[q];
  *tb = nsplit == 2 ? b2[q] : b3[q];
}

struct TcPass {
  const float* in;
  float* out;
  int64_t rows;   // pencils of the pass
  int n;          // pencil (and output) length
  int kpad;       // roundup(n, TBK)
  int64_t inner;  // pencil p lives at (p / inner) * n * inner + j * inner + (p % inner)
  float scale;    // sqrt(2 / (n + 1))
};

// Asynchronous 4-byte copy global -> shared; src_bytes = 0 writes a zero.
__device__ __forceinline__ void cp_async4(void* dst_smem, const float* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst_smem)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// Fetch the TBK pencil values of K tile kt of this thread's row into its staging row
// (zeros past n or past the last pencil), one commit group per tile.
__device__ __forceinline__ void fetch_row_tile(const TcPass& P, bool rok, int64_t rb, int kt, float* xrow) {
#pragma unroll
  for (int e = 0; e < TBK; ++e) {
    const int k = kt * TBK + e;
    const bool in = rok && k < P.n;
    cp_async4(xrow + e, in ? P.in + rb + (int64_t)k * P.inner : P.in, in ? 4 : 0);
  }
}

// Split one row's K tile and store the NSPLIT bfloat16 terms in the core-matrix layout
// (pairs of values converted together: cvt.rn.bf16x2.f32).
template <int NSPLIT>
__device__ __forceinline__ void store_row_tile(unsigned char* A, int row, const float (&x)[TBK]) {
#pragma unroll
  for (int c = 0; c < TBK / 8; ++c) {
    uint32_t pk[NSPLIT][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      float r0 = x[8 * c + e], r1 = x[8 * c + e + 1];
#pragma unroll
      for (int t = 0; t < NSPLIT; ++t) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(r0, r1);  // .x = r0 (low half)
        pk[t][e / 2] = *reinterpret_cast<const uint32_t*>(&h);
        if (t + 1 < NSPLIT) {
          r0 -= __low2float(h);
          r1 -= __high2float(h);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < NSPLIT; ++t)
      *reinterpret_cast<uint4*>(A + t * A_TERM + c * (TBM * 16) + row * 16) =
          make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
  }
}

template <int NSPLIT>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_dst_kernel(const __grid_constant__ CUtensorMap mapB, TcPass P,
                                                                int* __restrict__ err) {
  constexpr int STAGES = TcCfg<NSPLIT>::STAGES, NACC = TcCfg<NSPLIT>::NACC;
  constexpr int NPROD = NSPLIT == 2 ? 3 : 6;
  constexpr int STAGE_BYTES = NSPLIT * (A_TERM + B_TERM);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t fullA[STAGES];
  __shared__ __align__(8) uint64_t fullB[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int n0 = blockIdx.x * TBN;
  const int64_t m0 = (int64_t)blockIdx.y * TBM;
  const int KT = P.kpad / TBK;
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&fullA[s], 128);
      mbar_init(&fullB[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(NACC * TBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp < 4) {
    // split-operand producers: thread tid owns pencil row tid of the tile.  Its float32
    // K tiles arrive by cp.async in its own staging row, SF - 1 tiles ahead of the
    // split, so no barrier is needed between the copy and the split.
    constexpr int SF = TcCfg<NSPLIT>::SF;
    const int64_t p = m0 + tid;
    const bool rok = p < P.rows;
    const int64_t rb = rok ? (p / P.inner) * (int64_t)P.n * P.inner + (p % P.inner) : 0;
    float* xs = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES);  // [SF][TBM][XROW]
#pragma unroll
    for (int f = 0; f < SF - 1; ++f) {
      if (f < KT) fetch_row_tile(P, rok, rb, f, xs + (f * TBM + tid) * XROW);
      cp_async_commit();
    }
    for (int kt = 0; kt < KT; ++kt) {
      const int kf = kt + SF - 1;
      if (kf < KT) fetch_row_tile(P, rok, rb, kf, xs + ((kf % SF) * TBM + tid) * XROW);
      cp_async_commit();
      cp_async_wait<SF - 1>();  // tile kt has landed
      float x[TBK];
      const float* xr = xs + ((kt % SF) * TBM + tid) * XROW;
#pragma unroll
      for (int e = 0; e < TBK; ++e) x[e] = xr[e];
      const int s = kt % STAGES;
      if (kt >= STAGES && !mbar_wait(&empty_bar[s], (uint32_t)(((kt / STAGES) - 1) & 1))) {
        atomicExch(err, 4);
        s_fail = 1;
        break;
      }
      store_row_tile<NSPLIT>(smem + s * STAGE_BYTES, tid, x);
      fence_proxy_async();
      mbar_arrive(&fullA[s]);
    }
    cp_async_wait<0>();
  } else if (tid == 128) {
    // TMA producer of the split DST matrix and MMA issuer
    const uint32_t idesc = instr_desc_bf16(TBM, TBN);
    auto load_B = [&](int kt) {
      const int s = kt % STAGES;
      unsigned char* Bst = smem + s * STAGE_BYTES + NSPLIT * A_TERM;
      mbar_expect_tx(&fullB[s], NSPLIT * B_TERM);
      for (int t = 0; t < NSPLIT; ++t)
        for (int c = 0; c < TBK / 8; ++c)
          tma_load_2d(Bst + t * B_TERM + c * (TBN * 16), &mapB, t * P.kpad + kt * TBK + c * 8, n0, &fullB[s]);
    };
    for (int kt = 0; kt < STAGES && kt < KT; ++kt) load_B(kt);
    bool ok = true;
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)((kt / STAGES) & 1);
      if (!mbar_wait(&fullB[s], ph) || !mbar_wait(&fullA[s], ph)) {
        ok = false;
        atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES);
      const uint32_t b0 = a0 + NSPLIT * A_TERM;
      const uint32_t dacc = tmem + (uint32_t)((kt % NACC) * TBN);
      for (int kk = 0; kk < TBK / 16; ++kk) {
        for (int q = 0; q < NPROD; ++q) {
          int ta, tb;
          prod_terms(NSPLIT, q, &ta, &tb);
          const uint64_t da = smem_desc(a0 + ta * A_TERM + (2 * kk) * (TBM * 16), TBM * 16, 128);
          const uint64_t db = smem_desc(b0 + tb * B_TERM + (2 * kk) * (TBN * 16), TBN * 16, 128);
          mma_bf16(dacc, da, db, idesc, (kt >= NACC || kk > 0 || q > 0) ? 1u : 0u);
        }
      }
      mma_commit(&empty_bar[s]);
      // refill the stage of the previous K tile once its MMAs have completed
      const int kr = kt - 1 + STAGES;
      if (kt >= 1 && kr < KT) {
        if (!mbar_wait(&empty_bar[(kt - 1) % STAGES], (uint32_t)(((kt - 1) / STAGES) & 1))) {
          ok = false;
          atomicExch(err, 2);
          break;
        }
        load_B(kr);
      }
    }
    if (ok) mma_commit(&done_bar);
    else s_fail = 1;
  }
  __syncthreads();

  if (warp < 4) {
    if (!s_fail && !mbar_wait(&done_bar, 0)) {
      atomicExch(err, 3);
      s_fail = 1;
    }
    conv_bar();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fail) {
      // warp w reads TMEM lanes 32w..32w+31 = rows of the tile
      const int nacc = KT < NACC ? KT : NACC;
      const int64_t p = m0 + tid;
      const bool rok = p < P.rows;
      float* tile = reinterpret_cast<float*>(smem);  // contiguous pass: 128 x 17 floats
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
        if (P.inner > 1) {
          // strided pass: lanes are consecutive pencils, so every store instruction coalesces
          if (rok) {
            const int64_t ob = (p / P.inner) * (int64_t)P.n * P.inner + (p % P.inner);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int j = n0 + c * 16 + e;
              if (j < P.n) P.out[ob + (int64_t)j * P.inner] = sum[e] * P.scale;
            }
          }
        } else {
          // contiguous pass: transpose the 128 x 16 chunk through shared memory, then
          // half-warps write 16 consecutive outputs of one pencil
#pragma unroll
          for (int e = 0; e < 16; ++e) tile[tid * 17 + e] = sum[e] * P.scale;
          conv_bar();
          const int col = tid & 15;
          const int j = n0 + c * 16 + col;
          for (int rr = tid >> 4; rr < TBM; rr += 8) {
            const int64_t pr = m0 + rr;
            if (pr < P.rows && j < P.n) P.out[pr * (int64_t)P.n + j] = tile[rr * 17 + col];
          }
          conv_bar();
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 4) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TcCfg<NSPLIT>::NACC * TBN)
                 : "memory");
  }
}

// B'[j][t * kpad + k] = split term t of S[j][k] = sin(pi (j+1)(k+1)/(n+1)) (the orthonormal
// scale is applied in the epilogue), zero padded to npad rows x kpad columns per term
__global__ void split_dst_matrix_kernel(int n, int kpad, int nsplit, __nv_bfloat16* __restrict__ Bp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (k >= kpad) return;
  float v = 0.f;
  if (j < n && k < n) {
    const int64_t period = 2 * (int64_t)(n + 1);
    const int64_t m = ((int64_t)(j + 1) * (k + 1)) % period;
    v = (float)sinpi((double)m / (double)(n + 1));
  }
  float r = v;
  for (int t = 0; t < nsplit; ++t) {
    const __nv_bfloat16 h = __float2bfloat16_rn(r);
    Bp[(int64_t)j * nsplit * kpad + (int64_t)t * kpad + k] = h;
    r -= __bfloat162float(h);
  }
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

template <int NSPLIT>
pe_status tc_launch(const CUtensorMap& mB, const TcPass& P, dim3 grid, int* err, cudaStream_t st) {
  static bool attr_set = false;  // the same value for every device and call
  if (!attr_set) {
    PE_CUDA_TRY(cudaFuncSetAttribute(tc_dst_kernel<NSPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     tc_smem_bytes<NSPLIT>()));
    attr_set = true;
  }
  tc_dst_kernel<NSPLIT><<<grid, TC_THREADS, tc_smem_bytes<NSPLIT>(), st>>>(mB, P, err);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

// One axis pass: out = S applied along the axis (pencils of length n, stride inner).
pe_status tc_axis(const float* in, float* out, int64_t outer, int n, int64_t inner, int nsplit, __nv_bfloat16* Bp,
                  int* err, cudaStream_t st) {
  const int kpad = (int)rup(n, TBK);
  const int npad = (int)rup(n, TBN);
  const int64_t rows = outer * inner;
  dim3 g2((kpad + 127) / 128, npad);
  split_dst_matrix_kernel<<<g2, 128, 0, st>>>(n, kpad, nsplit, Bp);
  PE_CUDA_TRY(cudaGetLastError());
  CUtensorMap mB;
  PE_TRY(make_map(&mB, Bp, (uint64_t)nsplit * kpad, (uint64_t)npad, TBN));
  const TcPass P{in, out, rows, n, kpad, inner, (float)sqrt(2.0 / (double)(n + 1))};
  // output tiles of one pencil block are adjacent in launch order, so the block's
  // float32 rows are read from HBM once and from L2 for the other output tiles
  const int64_t mt = rup(rows, TBM) / TBM;
  if (mt > 65535) return pe_fail(PE_EINVAL, "tensor-core DST: problem too large");
  const dim3 grid((unsigned)(npad / TBN), (unsigned)mt);
  return nsplit == 2 ? tc_launch<2>(mB, P, grid, err, st) : tc_launch<3>(mB, P, grid, err, st);
}

}  // namespace

extern "C" pe_status pe_dst_tc(int32_t d, const int32_t* n, const float* in, float* out, int32_t nsplit,
                               void* stream) {
  if (d < 1 || d > PE_MAX_D || !n || !in || !out) return pe_fail(PE_EINVAL, "pe_dst_tc: bad arguments");
  if (nsplit != 2 && nsplit != 3) return pe_fail(PE_EINVAL, "pe_dst_tc: nsplit must be 2 or 3");
  int64_t ndof = 1;
  int64_t worstB = 0;
  for (int a = 0; a < d; ++a) {
    if (n[a] < 1 || n[a] > 1024) return pe_fail(PE_EINVAL, "pe_dst_tc: n_a must be in 1..1024");
    ndof *= n[a];
  }
  for (int a = 0; a < d; ++a) worstB = std::max<int64_t>(worstB, rup(n[a], TBN) * nsplit * rup(n[a], TBK));
  cudaStream_t st = (cudaStream_t)stream;
  __nv_bfloat16* Bp = nullptr;
  float* tmp = nullptr;
  int* err = nullptr;
  pe_status rc = PE_OK;
  cudaError_t e = cudaMallocAsync((void**)&Bp, sizeof(__nv_bfloat16) * worstB, st);
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
    rc = tc_axis(src, dst, outer, n[a], inner, nsplit, Bp, err, st);
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
  if (Bp) cudaFreeAsync(Bp, st);
  if (tmp) cudaFreeAsync(tmp, st);
  if (err) cudaFreeAsync(err, st);
  if (rc == PE_OK && herr != 0) rc = pe_fail(PE_ETIMEOUT, "pe_dst_tc: a tensor-core pipeline wait expired");
  return rc;
}
