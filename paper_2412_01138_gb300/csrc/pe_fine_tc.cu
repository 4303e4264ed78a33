// Tensor-core engine of the mixed-precision fine sweep (pe_options.fine_engine = PE_FINE_TC).
//
// The forced part of the fine propagator over one slice n (the EIFE stage recurrence of
// Sec. 3 with its stage columns contracted) is, per mode J,
//   w_{m+1} = E_F w_m + a_m,   a_m = sum_k W[k][J] Y_n[m][k],   m = 0..M-1,   w_0 = 0,
// and F^M(U^n)_J = exp(-lam_J M dt) U^n_J + w_M.  For a tile of 128 modes and a group of G
// slices the inputs a_m of all G*M substeps form one dense contraction
//   D[J][s*M + m] = sum_k W[k][J] Y_{gG+s}[m][k]        (128 x NR, NR = G*M <= 256, K <= 64),
// which runs on the 5th-generation tensor cores: both operands are split into three
// bfloat16 terms x = x0 + x1 + x2 (about 24 bits together) and the six products whose
// weight is at least 2^-24 (x0y0, x0y1, x1y0, x0y2, x1y1, x2y0) are accumulated in float32
// in tensor memory, the five small ones first.  The recurrence (hi/lo E_F, float32) and
// the float64 homogeneous term then run per mode on the CUDA cores from tcgen05.ld rows.
//
// Kernel roles (one persistent CTA per SM, 288 threads, items = (slice group, mode tile)
// pairs, group-major, a contiguous range per CTA):
//   * warps 0-7 (two warpgroups): the epilogue of each item: wait for its accumulator,
//     read rows with tcgen05.ld, 32 substeps of two slices per read (warp w reads TMEM lanes
//     32 (w % 4) ..; warpgroup h takes the slices h, h + 2, ... of the group), run the
//     recurrence four substeps per step, write F; the next item's epilogue inputs are
//     loaded meanwhile;
//   * warp 8, one thread: bulk copies of the split operands, both prepared once per problem
//     in global memory in the exact shared-memory layout (the time factors of the current
//     slice group; the stage weights of each item's mode tile, a ring of three), and the
//     tcgen05.mma issue into one of two accumulators (2 x NR TMEM columns), released by
//     tcgen05.commit.
// Every mbarrier wait is bounded; on expiry the CTA records an error code, writes a NaN
// into the first output value (so that the Parareal residual reports it), frees its
// tensor memory and exits.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "pe_batch.h"
#include "pe_internal.h"
#include "pe_tc_common.cuh"

namespace {

constexpr int FT_ROWS = 128;                 // modes of a tile (TMEM lanes)
constexpr int FT_WORKERS = 256;              // warps 0-7: two warpgroups
constexpr int FT_THREADS = FT_WORKERS + 32;  // + warp 8 (copies and MMA issue)
constexpr int FT_CHUNK = 16 * 1024;          // bytes per bulk copy instruction
constexpr int FT_MIN_SMEM = 120 * 1024;      // at most one CTA per SM (its TMEM allocation)
constexpr int FT_ABUF = 3;                   // ring of A-operand tiles

// rows of the B operand (G*M) a K padding allows, and the shared-memory budget
__host__ __device__ constexpr int ft_rows_max(int KP) { return KP <= 32 ? 256 : 128; }
__host__ __device__ constexpr int ft_a_bytes(int KP) { return 3 * FT_ROWS * KP * 2; }
__host__ __device__ constexpr int ft_smem_bytes(int KP) {
  return std::max(1024 + 3 * ft_rows_max(KP) * KP * 2 + FT_ABUF * ft_a_bytes(KP), FT_MIN_SMEM);
}

// Operand images use the swizzled K-major layout whose swizzle width equals a row of KP
// bfloat16 (32, 64 or 128 bytes): row r of a term at r * KP * 2 bytes, its 16-byte chunk c
// stored at chunk c ^ ((byte offset >> 7) & (KP / 8 - 1)) (address bits 4.. XOR bits 7..),
// so that the tensor core reads whole rows without bank conflicts.  Terms start on
// 1024-byte boundaries, as the pattern requires.
__host__ __device__ constexpr int ft_kpad(int K) { return K <= 16 ? 16 : (K <= 32 ? 32 : 64); }
__device__ __forceinline__ int64_t ft_swz(int64_t off, int KP) {
  return off ^ (((off >> 7) & (KP / 8 - 1)) << 4);
}
// shared-memory descriptor of a swizzled K-major operand: start address, stride between
// 8-row groups (8 rows of KP * 2 bytes), version 1, layout type 6 / 4 / 2 (32 / 64 / 128-byte
// swizzle); the leading offset is not used by these layouts
__device__ __forceinline__ uint64_t smem_desc_swz(uint32_t saddr, int KP) {
  const uint32_t sbo = 8u * (uint32_t)KP * 2u;
  const uint64_t layout = KP == 16 ? 6 : (KP == 32 ? 4 : 2);
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= layout << 61;
  return d;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
}
// hi + lo pair squared in float32 arithmetic (a double-float product: the low word collects
// the exact rounding error of hi * hi from an FMA and the cross term 2 hi lo; about 2^-44
// relative)
__device__ __forceinline__ void df_square(float h, float l, float& oh, float& ol) {
  const float p = h * h;
  float e = fmaf(h, h, -p);
  e = fmaf(2.f * h, l, e);
  oh = p + e;
  ol = e - (oh - p);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int e = 0; e < 32; ++e) v[e] = __uint_as_float(r[e]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Three bfloat16 terms of eight consecutive values (x = t0 + t1 + t2 up to about 2^-24
// relative), each packed as one 16-byte core-matrix row.
__device__ __forceinline__ void split8(const float (&x)[8], uint4 (&o)[3]) {
  uint32_t pk[3][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float r0 = x[2 * e], r1 = x[2 * e + 1];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(r0, r1);  // .x = r0 (low half)
      pk[t][e] = *reinterpret_cast<const uint32_t*>(&h);
      r0 -= __low2float(h);
      r1 -= __high2float(h);
    }
  }
#pragma unroll
  for (int t = 0; t < 3; ++t) o[t] = make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
}

// Split time factors of every slice group, in the B-operand layout of the kernel below:
// group g occupies 3 * NR * KP * 2 bytes, [term][row r][k] swizzled as above, row r = s * M + m
// holding Y_{gG+s}[m][k] (zero past the last slice and past K).
__global__ void ft_split_time_kernel(const float* __restrict__ Y, int N, int M, int K, int KC, int G, int NR,
                                     int KP, int ngroups, uint4* __restrict__ Bsp) {
  pdl_wait();
  const int chunks = KP / 8;
  const int64_t total = (int64_t)ngroups * NR * chunks;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int c = (int)(e % chunks);
  const int64_t gr = e / chunks;
  const int r = (int)(gr % NR);
  const int g = (int)(gr / NR);
  const int s = r / M, m = r - s * M, n = g * G + s;
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = 8 * c + j;
    x[j] = (n < N && k < K) ? Y[((int64_t)n * M + m) * KC + k] : 0.f;
  }
  uint4 o[3];
  split8(x, o);
  const int64_t term = (int64_t)NR * KP * 2;
#pragma unroll
  for (int t = 0; t < 3; ++t)
    Bsp[(((int64_t)g * 3 + t) * term + ft_swz((int64_t)r * KP * 2 + c * 16, KP)) / 16] = o[t];
}

// Stage weights of every mode tile formed and split in one pass, in the A-operand layout of the
// kernel below: tile q occupies 3 * 128 * KP * 2 bytes, [term][row r][k] swizzled as above, row
// r holding W[k][128 q + r] (zero past the last mode and past K).  A thread per row and group of
// eight columns (consecutive threads: the 16-byte chunks of one row, then the next row): the same
// float32 arithmetic as the SIMT engine's stage-weight table, W[k][J] = P_{r(k),J} sum_i
// (dt b_i)_J Z_k(c_i dt) with P the product of the per-axis modal factors, so that table is never
// written or read by this engine.
template <int Q>
__global__ void __launch_bounds__(256) ft_weights_image_kernel(Geom g, StageCols C, int R,
                                                               const float* __restrict__ axisF,
                                                               const float* __restrict__ coef_b,
                                                               const double* __restrict__ Z, int KP, int64_t tiles,
                                                               uint4* __restrict__ Asp) {
  pdl_wait();
  __shared__ float sZ[PE_MAX_S * 2 * PE_MAX_TERMS];
  __shared__ int sTerm[2 * PE_MAX_TERMS];
  const int K = C.K;
  for (int e = threadIdx.x; e < Q * K; e += blockDim.x) sZ[e] = (float)Z[e];
  for (int e = threadIdx.x; e < K; e += blockDim.x) sTerm[e] = C.term[e];
  __syncthreads();
  const int chunks = KP / 8;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= tiles * FT_ROWS * chunks) return;
  const int c = (int)(e % chunks);
  const int64_t J = e / chunks;
  const int r = (int)(J % FT_ROWS);
  const int64_t tile = J / FT_ROWS, nd = g.ndof;
  const int64_t term = (int64_t)FT_ROWS * KP * 2;
  if (J >= nd || 8 * c >= K) {
    // padding rows past the last mode and columns past K: zero in every split term
#pragma unroll
    for (int t = 0; t < 3; ++t)
      Asp[((tile * 3 + t) * term + ft_swz((int64_t)r * KP * 2 + c * 16, KP)) / 16] = make_uint4(0u, 0u, 0u, 0u);
    return;
  }
  int j[PE_MAX_D];
  unflatten(g, J, j);
  // the row's entries of the per-axis factor tables (term rt of axis a at ax[a][rt * n_a])
  const float* ax[PE_MAX_D];
#pragma unroll
  for (int a = 0; a < PE_MAX_D; ++a) ax[a] = axisF + (int64_t)R * g.off[a] + j[a];
  float b[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) b[i] = coef_b[(int64_t)i * nd + J];
  {
    float x[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int k = 8 * c + jj;
      float v = 0.f;
      if (k < K) {
        const int rt = sTerm[k];
        float P = ax[0][rt * g.n[0]];
#pragma unroll
        for (int a = 1; a < PE_MAX_D; ++a) if (a < g.d) P *= ax[a][rt * g.n[a]];
        float sw = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) sw = fmaf(b[i], sZ[i * K + k], sw);
        v = P * sw;
      }
      x[jj] = v;
    }
    uint4 o[3];
    split8(x, o);
#pragma unroll
    for (int t = 0; t < 3; ++t) Asp[((tile * 3 + t) * term + ft_swz((int64_t)r * KP * 2 + c * 16, KP)) / 16] = o[t];
  }
}

struct FtArgs {
  const float* coefF32;  // E_hi [ndof], E_lo [ndof]
  const double* EM;      // exp(-lam M dt) [ndof]
  const double* U;       // U^n at n * ndof
  double* out;           // F^M(U^n) (or F^M(0)) at n * ndof
  const unsigned char* Asp;  // split stage weights of every mode tile
  const unsigned char* Bsp;  // split time factors of every slice group
  int64_t ndof, tiles, items;
  int N, M, K, G, NR, from_zero;
  int* err;
};

template <int KP>
__global__ void __launch_bounds__(FT_THREADS, 1) fine_tc_kernel(FtArgs a) {
  pdl_wait();
  constexpr int A_TERM = FT_ROWS * KP * 2;          // one split term of the A operand
  constexpr int A_BYTES = 3 * A_TERM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t fullA[FT_ABUF], emptyA[FT_ABUF], fullD[2], emptyD[2], fullB, freeB, drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sB = smem;
  unsigned char* sA = smem + 3 * ft_rows_max(KP) * KP * 2;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int NR = a.NR, M = a.M;
  const int B_BYTES = 3 * NR * KP * 2;
  const int64_t nd = a.ndof;
  const int64_t i0 = (int64_t)blockIdx.x * a.items / gridDim.x;
  const int64_t i1 = (int64_t)(blockIdx.x + 1) * a.items / gridDim.x;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(2 * NR)) ncols <<= 1;
  volatile int* fail = &s_fail;
  auto set_fail = [&](int code) {
    atomicExch(a.err, code);
    *fail = 1;
    a.out[0] = __longlong_as_double(0x7ff8000000000000LL);
  };
  if (tid == 0) {
    for (int b = 0; b < FT_ABUF; ++b) {
      mbar_init(&fullA[b], 1);
      mbar_init(&emptyA[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&fullD[b], 1);
      mbar_init(&emptyD[b], FT_WORKERS / 32);
    }
    mbar_init(&fullB, 1);
    mbar_init(&freeB, 1);
    mbar_init(&drain, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == FT_WORKERS / 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp < FT_WORKERS / 32) {
    // thread (h, r): warpgroup h of two, row r of the tile (TMEM lane r)
    const int r = tid & (FT_ROWS - 1), h = tid >> 7, lane = tid & 31;
    // the epilogue inputs of item i + 1 (E_hi, E_lo, exp(-lam M dt)) are loaded while item i
    // waits for its accumulator and runs, into two alternating register sets
    struct Pre {
      float eh, el;
      double em;
    };
    Pre P0, P1;
    auto load_epi = [&](Pre& P, int64_t i) {
      const int64_t g = i / a.tiles, J = (i % a.tiles) * FT_ROWS + r;
      const bool ok = J < nd;
      P.eh = ok ? a.coefF32[J] : 0.f;
      P.el = ok ? a.coefF32[nd + J] : 0.f;
      P.em = ok ? a.EM[J] : 0.0;
    };
    auto step = [&](int64_t i, const Pre& cur, Pre& nxt) -> bool {
      const int j = (int)(i - i0);
      if (i + 1 < i1) load_epi(nxt, i + 1);
      // U^n of the slices, loaded ahead: the first pair's before the wait for the accumulator,
      // each later pair's (more than four slices per group) while the pair before it runs
      const int64_t g = i / a.tiles;
      const int64_t J = (i % a.tiles) * FT_ROWS + r;
      const bool ok = J < nd;
      auto load_u = [&](int s) -> double {
        const int64_t n = g * a.G + s;
        return (!a.from_zero && ok && s < a.G && n < a.N) ? a.U[n * nd + J] : 0.0;
      };
      double u0 = load_u(h), u1 = load_u(h + 2);
      if (!mbar_wait(&fullD[j & 1], (uint32_t)((j >> 1) & 1))) {
        set_fail(5);
        return false;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float e2h, e2l, e4h, e4l;
      df_square(cur.eh, cur.el, e2h, e2l);
      df_square(e2h, e2l, e4h, e4l);
      const float eh = cur.eh, e2 = e2h, e3 = e2h * eh;
      const uint32_t row = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((j & 1) * NR);
      // this thread's slices s = h + 2t of the group, two at a time (warp-uniform); each
      // TMEM read brings 32 substeps of both, and the chains run four substeps per step:
      // w <- E^4 w + (E^3 a_m + E^2 a_{m+1} + E a_{m+2} + a_{m+3}), the bracket independent of
      // w and E^4 applied as a hi/lo pair
      auto chain4 = [&](float& w, float x0, float x1, float x2, float x3) {
        const float b = fmaf(e3, x0, fmaf(e2, x1, fmaf(eh, x2, x3)));
        w = fmaf(e4h, w, fmaf(e4l, w, b));
      };
      auto finish = [&](double u, int s, float w) {
        const int64_t n = g * a.G + s;
        if (ok && n < a.N) a.out[n * nd + J] = a.from_zero ? (double)w : fma(cur.em, u, (double)w);
      };
#pragma unroll 1
      for (int p = 0; p < 4; ++p) {
        const int s0 = h + 4 * p, s1 = s0 + 2;
        if (s0 >= a.G) break;
        const bool two = s1 < a.G;
        const double n0 = load_u(s0 + 4), n1 = load_u(s1 + 4);
        float w0 = 0.f, w1 = 0.f;
        int m0 = 0;
        for (; m0 + 32 <= M; m0 += 32) {
          float v0[32], v1[32];
          tmem_ld32(row + (uint32_t)(s0 * M + m0), v0);
          if (two) tmem_ld32(row + (uint32_t)(s1 * M + m0), v1);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 32; e += 4) {
            chain4(w0, v0[e], v0[e + 1], v0[e + 2], v0[e + 3]);
            if (two) chain4(w1, v1[e], v1[e + 1], v1[e + 2], v1[e + 3]);
          }
        }
        if (m0 < M) {  // a tail of 16 substeps
          float v0[16], v1[16];
          tmem_ld16(row + (uint32_t)(s0 * M + m0), v0);
          if (two) tmem_ld16(row + (uint32_t)(s1 * M + m0), v1);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 16; e += 4) {
            chain4(w0, v0[e], v0[e + 1], v0[e + 2], v0[e + 3]);
            if (two) chain4(w1, v1[e], v1[e + 1], v1[e + 2], v1[e + 3]);
          }
        }
        finish(u0, s0, w0);
        if (two) finish(u1, s1, w1);
        u0 = n0;
        u1 = n1;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&emptyD[j & 1]);
      return true;
    };
    if (i0 < i1) load_epi(P0, i0);
    for (int64_t i = i0; i < i1; i += 2) {
      if (*fail || !step(i, P0, P1)) break;
      if (i + 1 < i1 && (*fail || !step(i + 1, P1, P0))) break;
    }
  } else if (tid == FT_WORKERS) {
    const uint32_t idesc = instr_desc_bf16(FT_ROWS, NR);
    const int ta[6] = {2, 1, 0, 1, 0, 0}, tb[6] = {0, 1, 2, 0, 1, 0};  // small products first
    const int n = (int)(i1 - i0);
    // item i0 + jj's split weights into A buffer jj % FT_ABUF
    auto load_A = [&](int jj) {
      const int b = jj % FT_ABUF;
      const unsigned char* src = a.Asp + ((i0 + jj) % a.tiles) * (int64_t)A_BYTES;
      mbar_expect_tx(&fullA[b], (uint32_t)A_BYTES);
      for (int off = 0; off < A_BYTES; off += FT_CHUNK)
        bulk_g2s(sA + b * A_BYTES + off, src + off, (uint32_t)(A_BYTES - off < FT_CHUNK ? A_BYTES - off : FT_CHUNK),
                 &fullA[b]);
    };
    int nl = 0;  // items whose A copy has been issued
    for (; nl < FT_ABUF && nl < n; ++nl) load_A(nl);
    int j = 0;
    int64_t gcur = -1;
    int nB = 0;
    bool issued = false;
    for (; j < n; ++j) {
      const int64_t g = (i0 + j) / a.tiles;
      if (g != gcur) {
        // the previous group's MMAs must be done with sB before it is overwritten
        if (gcur >= 0) {
          mma_commit(&freeB);
          if (!mbar_wait(&freeB, (uint32_t)((nB - 1) & 1))) {
            set_fail(6);
            break;
          }
        }
        mbar_expect_tx(&fullB, (uint32_t)B_BYTES);
        const unsigned char* src = a.Bsp + g * (int64_t)B_BYTES;
        for (int off = 0; off < B_BYTES; off += FT_CHUNK)
          bulk_g2s(sB + off, src + off, (uint32_t)(B_BYTES - off < FT_CHUNK ? B_BYTES - off : FT_CHUNK), &fullB);
        if (!mbar_wait(&fullB, (uint32_t)(nB & 1))) {
          set_fail(7);
          break;
        }
        ++nB;
        gcur = g;
      }
      const int b = j % FT_ABUF;
      if (!mbar_wait(&fullA[b], (uint32_t)((j / FT_ABUF) & 1))) {
        set_fail(8);
        break;
      }
      if (j >= 2 && !mbar_wait(&emptyD[j & 1], (uint32_t)(((j >> 1) - 1) & 1))) {
        set_fail(9);
        break;
      }
      if (*fail) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA + b * A_BYTES), b0 = smem_u32(sB);
      const uint32_t d = tmem + (uint32_t)((j & 1) * NR);
      bool first = true;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
#pragma unroll
        for (int ks = 0; ks < KP / 16; ++ks) {
          const uint64_t da = smem_desc_swz(a0 + ta[q] * A_TERM + 32 * ks, KP);
          const uint64_t db = smem_desc_swz(b0 + tb[q] * (NR * KP * 2) + 32 * ks, KP);
          mma_bf16(d, da, db, idesc, first ? 0u : 1u);
          first = false;
        }
      }
      mma_commit(&fullD[j & 1]);
      mma_commit(&emptyA[b]);
      issued = true;
      // refill the buffer of item j - 1 (its MMAs ran ahead of item j's) with item j + 2
      if (j >= 1 && j + FT_ABUF - 1 < n) {
        if (!mbar_wait(&emptyA[(j - 1) % FT_ABUF], (uint32_t)(((j - 1) / FT_ABUF) & 1))) {
          set_fail(11);
          break;
        }
        load_A(j + FT_ABUF - 1);
        ++nl;
      }
    }
    // after a failure: wait (bounded) for the A copies still in flight into shared memory
    if (*fail)
      for (int jj = j; jj < nl; ++jj) mbar_wait(&fullA[jj % FT_ABUF], (uint32_t)((jj / FT_ABUF) & 1));
    // every MMA and copy of this CTA has completed before the tensor memory is freed
    if (issued) {
      mma_commit(&drain);
      if (!mbar_wait(&drain, 0)) set_fail(10);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == FT_WORKERS / 32) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Batched form: the same engine over the work items (problem p, slice group g, mode tile t)
// of many problems at once, one persistent launch per column padding KP.  Each item reads
// its problem's record (sizes, slice-group shape NR = TG * M, arena offsets); the B operand
// (the group's split time factors) is reloaded when (p, g) changes, the A operand (the tile's
// split stage weights) every item through the same ring; the MMA instruction takes the item's
// N = NR.  Items of converged problems run too (the batched correction leaves those problems
// unchanged), which keeps both pipeline sides' item sequences fixed inside the captured graph.
// ---------------------------------------------------------------------------
struct BtcArgs {
  const BProb* probs;
  const BTcItem* items;
  int64_t n_items;
  const float* coefF32;  // arena: E_hi, E_lo at oCF
  const double* coefF;   // arena: exp(-lam M dt) at oCF + (q + 1) ndof
  const double* U;       // arena at oU
  double* Fbar;          // arena at oS
  const unsigned char* A;
  const unsigned char* B;
  int* err;
};

template <int KP>
__global__ void __launch_bounds__(FT_THREADS, 1) b_fine_tc_kernel(BtcArgs a) {
  constexpr int A_TERM = FT_ROWS * KP * 2;
  constexpr int A_BYTES = 3 * A_TERM;
  constexpr int NRMAX = ft_rows_max(KP);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t fullA[FT_ABUF], emptyA[FT_ABUF], fullD[2], emptyD[2], fullB, freeB, drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sB = smem;
  unsigned char* sA = smem + 3 * NRMAX * KP * 2;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * a.n_items / gridDim.x;
  const int64_t i1 = (int64_t)(blockIdx.x + 1) * a.n_items / gridDim.x;
  constexpr uint32_t ncols = 2 * NRMAX;  // 512 or 256: a power of two
  volatile int* fail = &s_fail;
  auto set_fail = [&](int code) {
    atomicExch(a.err, code);
    *fail = 1;
    a.Fbar[0] = __longlong_as_double(0x7ff8000000000000LL);
  };
  if (tid == 0) {
    for (int b = 0; b < FT_ABUF; ++b) {
      mbar_init(&fullA[b], 1);
      mbar_init(&emptyA[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&fullD[b], 1);
      mbar_init(&emptyD[b], FT_WORKERS / 32);
    }
    mbar_init(&fullB, 1);
    mbar_init(&freeB, 1);
    mbar_init(&drain, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == FT_WORKERS / 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp < FT_WORKERS / 32) {
    const int r = tid & (FT_ROWS - 1), h = tid >> 7, lane = tid & 31;
    struct Pre {
      float eh, el;
      double em;
    };
    Pre P0, P1;
    auto load_epi = [&](Pre& P, int64_t i) {
      const BTcItem it = a.items[i];
      const BProb& B = a.probs[it.p];
      const int64_t nd = B.g.ndof, J = it.t * FT_ROWS + r;
      const bool ok = J < nd;
      P.eh = ok ? a.coefF32[B.oCF + J] : 0.f;
      P.el = ok ? a.coefF32[B.oCF + nd + J] : 0.f;
      P.em = ok ? a.coefF[B.oCF + (int64_t)(B.q + 1) * nd + J] : 0.0;
    };
    auto step = [&](int64_t i, const Pre& cur, Pre& nxt) -> bool {
      const int j = (int)(i - i0);
      if (i + 1 < i1) load_epi(nxt, i + 1);
      const BTcItem it = a.items[i];
      const BProb& B = a.probs[it.p];
      const int M = B.M, TG = B.TG, N = B.N;
      const int64_t nd = B.g.ndof;
      const int64_t J = it.t * FT_ROWS + r;
      const bool ok = J < nd;
      // U^n loaded ahead, as in the single-problem kernel: the first pair's before the wait
      auto load_u = [&](int s) -> double {
        const int64_t n = (int64_t)it.g * TG + s;
        return (ok && s < TG && n < N) ? a.U[B.oU + n * nd + J] : 0.0;
      };
      double u0 = load_u(h), u1 = load_u(h + 2);
      if (!mbar_wait(&fullD[j & 1], (uint32_t)((j >> 1) & 1))) {
        set_fail(5);
        return false;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float e2h, e2l, e4h, e4l;
      df_square(cur.eh, cur.el, e2h, e2l);
      df_square(e2h, e2l, e4h, e4l);
      const float eh = cur.eh, e2 = e2h, e3 = e2h * eh;
      const uint32_t row = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((j & 1) * NRMAX);
      auto chain4 = [&](float& w, float x0, float x1, float x2, float x3) {
        const float bsum = fmaf(e3, x0, fmaf(e2, x1, fmaf(eh, x2, x3)));
        w = fmaf(e4h, w, fmaf(e4l, w, bsum));
      };
      auto finish = [&](double u, int s, float w) {
        const int64_t n = (int64_t)it.g * TG + s;
        if (ok && n < N) a.Fbar[B.oS + n * nd + J] = fma(cur.em, u, (double)w);
      };
#pragma unroll 1
      for (int pq = 0; pq < 8; ++pq) {
        const int s0 = h + 4 * pq, s1 = s0 + 2;
        if (s0 >= TG) break;
        const bool two = s1 < TG;
        const double n0 = load_u(s0 + 4), n1 = load_u(s1 + 4);
        float w0 = 0.f, w1 = 0.f;
        int m0 = 0;
        for (; m0 + 32 <= M; m0 += 32) {
          float v0[32], v1[32];
          tmem_ld32(row + (uint32_t)(s0 * M + m0), v0);
          if (two) tmem_ld32(row + (uint32_t)(s1 * M + m0), v1);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 32; e += 4) {
            chain4(w0, v0[e], v0[e + 1], v0[e + 2], v0[e + 3]);
            if (two) chain4(w1, v1[e], v1[e + 1], v1[e + 2], v1[e + 3]);
          }
        }
        if (m0 < M) {
          float v0[16], v1[16];
          tmem_ld16(row + (uint32_t)(s0 * M + m0), v0);
          if (two) tmem_ld16(row + (uint32_t)(s1 * M + m0), v1);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 16; e += 4) {
            chain4(w0, v0[e], v0[e + 1], v0[e + 2], v0[e + 3]);
            if (two) chain4(w1, v1[e], v1[e + 1], v1[e + 2], v1[e + 3]);
          }
        }
        finish(u0, s0, w0);
        if (two) finish(u1, s1, w1);
        u0 = n0;
        u1 = n1;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&emptyD[j & 1]);
      return true;
    };
    if (i0 < i1) load_epi(P0, i0);
    for (int64_t i = i0; i < i1; i += 2) {
      if (*fail || !step(i, P0, P1)) break;
      if (i + 1 < i1 && (*fail || !step(i + 1, P1, P0))) break;
    }
  } else if (tid == FT_WORKERS) {
    const int ta[6] = {2, 1, 0, 1, 0, 0}, tb[6] = {0, 1, 2, 0, 1, 0};
    const int n = (int)(i1 - i0);
    auto load_A = [&](int jj) {
      const int b = jj % FT_ABUF;
      const BTcItem it = a.items[i0 + jj];
      const unsigned char* src = a.A + a.probs[it.p].oTA + it.t * (int64_t)A_BYTES;
      mbar_expect_tx(&fullA[b], (uint32_t)A_BYTES);
      for (int off = 0; off < A_BYTES; off += FT_CHUNK)
        bulk_g2s(sA + b * A_BYTES + off, src + off, (uint32_t)(A_BYTES - off < FT_CHUNK ? A_BYTES - off : FT_CHUNK),
                 &fullA[b]);
    };
    int nl = 0;
    for (; nl < FT_ABUF && nl < n; ++nl) load_A(nl);
    int j = 0;
    int cur_p = -1, cur_g = -1, nB = 0;
    bool issued = false;
    for (; j < n; ++j) {
      const BTcItem it = a.items[i0 + j];
      const BProb& B = a.probs[it.p];
      const int NR = B.NR;
      if (it.p != cur_p || it.g != cur_g) {
        if (cur_p >= 0) {
          mma_commit(&freeB);
          if (!mbar_wait(&freeB, (uint32_t)((nB - 1) & 1))) {
            set_fail(6);
            break;
          }
        }
        const int B_BYTES = 3 * NR * KP * 2;
        mbar_expect_tx(&fullB, (uint32_t)B_BYTES);
        const unsigned char* src = a.B + B.oTB + (int64_t)it.g * B_BYTES;
        for (int off = 0; off < B_BYTES; off += FT_CHUNK)
          bulk_g2s(sB + off, src + off, (uint32_t)(B_BYTES - off < FT_CHUNK ? B_BYTES - off : FT_CHUNK), &fullB);
        if (!mbar_wait(&fullB, (uint32_t)(nB & 1))) {
          set_fail(7);
          break;
        }
        ++nB;
        cur_p = it.p;
        cur_g = it.g;
      }
      const int b = j % FT_ABUF;
      if (!mbar_wait(&fullA[b], (uint32_t)((j / FT_ABUF) & 1))) {
        set_fail(8);
        break;
      }
      if (j >= 2 && !mbar_wait(&emptyD[j & 1], (uint32_t)(((j >> 1) - 1) & 1))) {
        set_fail(9);
        break;
      }
      if (*fail) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t idesc = instr_desc_bf16(FT_ROWS, NR);
      const uint32_t a0 = smem_u32(sA + b * A_BYTES), b0 = smem_u32(sB);
      const uint32_t d = tmem + (uint32_t)((j & 1) * NRMAX);
      bool first = true;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
#pragma unroll
        for (int ks = 0; ks < KP / 16; ++ks) {
          const uint64_t da = smem_desc_swz(a0 + ta[q] * A_TERM + 32 * ks, KP);
          const uint64_t db = smem_desc_swz(b0 + tb[q] * (NR * KP * 2) + 32 * ks, KP);
          mma_bf16(d, da, db, idesc, first ? 0u : 1u);
          first = false;
        }
      }
      mma_commit(&fullD[j & 1]);
      mma_commit(&emptyA[b]);
      issued = true;
      if (j >= 1 && j + FT_ABUF - 1 < n) {
        if (!mbar_wait(&emptyA[(j - 1) % FT_ABUF], (uint32_t)(((j - 1) / FT_ABUF) & 1))) {
          set_fail(11);
          break;
        }
        load_A(j + FT_ABUF - 1);
        ++nl;
      }
    }
    if (*fail)
      for (int jj = j; jj < nl; ++jj) mbar_wait(&fullA[jj % FT_ABUF], (uint32_t)((jj / FT_ABUF) & 1));
    if (issued) {
      mma_commit(&drain);
      if (!mbar_wait(&drain, 0)) set_fail(10);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == FT_WORKERS / 32) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// Split images of every problem of a batch.  Job index e of a prefix table: the problem whose
// first job is the largest prefix <= e (binary search), then that problem's local job.
__device__ inline int prefix_owner(const int64_t* __restrict__ prefix, int P, int64_t e) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void b_split_time_kernel(const BProb* __restrict__ probs, const int64_t* __restrict__ prefix, int P,
                                    int64_t total, const float* __restrict__ AF32, unsigned char* __restrict__ Bimg) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int p = prefix_owner(prefix, P, e);
  const BProb& B = probs[p];
  const int KP = B.KP, chunks = KP / 8, NR = B.NR, M = B.M, K = B.K, KC = (K + 3) / 4 * 4;
  const int64_t le = e - prefix[p];
  const int c = (int)(le % chunks);
  const int64_t gr = le / chunks;
  const int rr = (int)(gr % NR);
  const int g = (int)(gr / NR);
  const int sl = rr / M, m = rr - sl * M, n = g * B.TG + sl;
  float x[8];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int k = 8 * c + jj;
    x[jj] = (n < B.N && k < K) ? AF32[B.oAF32 + ((int64_t)n * M + m) * KC + k] : 0.f;
  }
  uint4 o[3];
  split8(x, o);
  const int64_t term = (int64_t)NR * KP * 2;
  uint4* dst = reinterpret_cast<uint4*>(Bimg + B.oTB);
#pragma unroll
  for (int t = 0; t < 3; ++t) dst[(((int64_t)g * 3 + t) * term + ft_swz((int64_t)rr * KP * 2 + c * 16, KP)) / 16] = o[t];
}

__global__ void b_split_w_kernel(const BProb* __restrict__ probs, const int64_t* __restrict__ prefix, int P,
                                 int64_t total, const float* __restrict__ W32, unsigned char* __restrict__ Aimg) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int p = prefix_owner(prefix, P, e);
  const BProb& B = probs[p];
  const int KP = B.KP, chunks = KP / 8, K = B.K;
  const int64_t nd = B.g.ndof;
  const int64_t le = e - prefix[p];
  const int rr = (int)(le % FT_ROWS);
  const int64_t rest = le / FT_ROWS;
  const int c = (int)(rest % chunks);
  const int64_t tile = rest / chunks;
  const int64_t J = tile * FT_ROWS + rr;
  float x[8];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int k = 8 * c + jj;
    x[jj] = (J < nd && k < K) ? W32[B.oW + (int64_t)k * nd + J] : 0.f;
  }
  uint4 o[3];
  split8(x, o);
  const int64_t term = (int64_t)FT_ROWS * KP * 2;
  uint4* dst = reinterpret_cast<uint4*>(Aimg + B.oTA);
#pragma unroll
  for (int t = 0; t < 3; ++t) dst[((tile * 3 + t) * term + ft_swz((int64_t)rr * KP * 2 + c * 16, KP)) / 16] = o[t];
}

template <int KP>
pe_status btc_launch(const BtcArgs& args, int grid, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(b_fine_tc_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, ft_smem_bytes(KP));
  });
  if (attr != cudaSuccess) return pe_cuda_fail(attr, "batched fine sweep (tensor cores): shared-memory attribute");
  b_fine_tc_kernel<KP><<<grid, FT_THREADS, ft_smem_bytes(KP), st>>>(args);
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

template <int KP>
pe_status ft_launch(const FtArgs& args, int grid, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(fine_tc_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, ft_smem_bytes(KP));
  });
  if (attr != cudaSuccess) return pe_cuda_fail(attr, "fine sweep (tensor cores): shared-memory attribute");
  PE_CUDA_TRY(launch_pdl(fine_tc_kernel<KP>, dim3(grid), dim3(FT_THREADS), ft_smem_bytes(KP), st, args));
  return PE_OK;
}

// slice-group shape of a column padding KP at M substeps: G slices, NR = G * M rows
void ft_shape(int KP, int M, int N, int* G, int* NR, int* ngroups) {
  *G = std::max(1, ft_rows_max(KP) / M);
  *NR = *G * M;
  *ngroups = (N + *G - 1) / *G;
}

}  // namespace

bool fine_tc_supported(int M) { return M >= 16 && M <= 128 && M % 16 == 0; }

size_t fine_tc_buffer_bytes(int M, int N) {
  size_t most = 0;
  for (int KP = 16; KP <= 64; KP *= 2) {
    int G, NR, ng;
    ft_shape(KP, M, N, &G, &NR, &ng);
    most = std::max(most, (size_t)ng * 3 * NR * KP * 2);
  }
  return most;
}

// The split operand images depend only on the problem (stage weights, time factors): made
// once by pe_set_problem (after the stage weights) and reused by every sweep of the problem.
static pe_status ft_check(pe_ctx* c) {
  if (!fine_tc_supported(c->M) || c->K < 1 || c->K > 64 || !c->tcB || !c->tc_err)
    return pe_fail(PE_EINVAL, "fine sweep (tensor cores): unsupported shape");
  return PE_OK;
}

pe_status fine_tc_prepare_time(pe_ctx* c) {
  PE_TRY(ft_check(c));
  const int M = c->M, K = c->K, N = c->N;
  const int KP = ft_kpad(K), KC = (K + 3) / 4 * 4;
  int G, NR, ngroups;
  ft_shape(KP, M, N, &G, &NR, &ngroups);
  const int64_t nsplit = (int64_t)ngroups * NR * (KP / 8);
  PE_CUDA_TRY(launch_pdl(ft_split_time_kernel, dim3((unsigned)((nsplit + 255) / 256)), dim3(256), 0, c->stream,
                         (const float*)c->AF32, N, M, K, KC, G, NR, KP, ngroups, (uint4*)c->tcB));
  c->launches += 1;
  return PE_OK;
}

pe_status fine_tc_prepare_weights(pe_ctx* c) {
  PE_TRY(ft_check(c));
  const int KP = ft_kpad(c->K);
  const int64_t tiles = (c->g.ndof + FT_ROWS - 1) / FT_ROWS;
  const size_t a_need = (size_t)tiles * ft_a_bytes(KP);
  if (a_need > c->tcA_cap) {
    PE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->tcA) PE_CUDA_TRY(cudaFree(c->tcA));
    c->tcA = nullptr;
    c->tcA_cap = 0;
    PE_CUDA_TRY(cudaMalloc((void**)&c->tcA, a_need));
    c->tcA_cap = a_need;
  }
  // a thread per (row, group of eight columns)
  const int64_t nsw = tiles * FT_ROWS * (KP / 8);
  const dim3 grid((unsigned)((nsw + 255) / 256));
  const float* ax = c->axisF32;
  const float* cb = c->coefF32 + 2 * c->g.ndof;
  switch (c->q) {
#define PE_FW_CASE(Q)                                                                                          \
  case Q:                                                                                                      \
    PE_CUDA_TRY(launch_pdl(ft_weights_image_kernel<Q>, grid, dim3(256), 0, c->stream, c->g, c->cols, c->R, ax, cb, \
                           (const double*)c->Zst, KP, tiles, (uint4*)c->tcA));                                  \
    break;
    PE_FW_CASE(1) PE_FW_CASE(2) PE_FW_CASE(3) PE_FW_CASE(4) PE_FW_CASE(5) PE_FW_CASE(6) PE_FW_CASE(7) PE_FW_CASE(8)
#undef PE_FW_CASE
    default:
      return pe_fail(PE_EINVAL, "fine sweep (tensor cores): unsupported number of stages");
  }
  c->launches += 1;
  return PE_OK;
}

pe_status fine_tc_prepare(pe_ctx* c) {
  PE_TRY(fine_tc_prepare_time(c));
  PE_TRY(fine_tc_prepare_weights(c));
  c->tc_split_ok = true;
  return PE_OK;
}

pe_status launch_fine_tc(pe_ctx* c, int from_zero, double* out) {
  const int M = c->M, K = c->K, N = c->N;
  if (!fine_tc_supported(M) || K < 1 || K > 64 || !c->tcB || !c->tc_err)
    return pe_fail(PE_EINVAL, "fine sweep (tensor cores): unsupported shape");
  if (!c->tc_split_ok) PE_TRY(fine_tc_prepare(c));
  const int KP = ft_kpad(K);
  int G, NR, ngroups;
  ft_shape(KP, M, N, &G, &NR, &ngroups);
  const int64_t tiles = (c->g.ndof + FT_ROWS - 1) / FT_ROWS;
  FtArgs args{};
  args.coefF32 = c->coefF32;
  args.EM = c->coefF + (int64_t)(c->q + 1) * c->g.ndof;
  args.U = c->U;
  args.out = out;
  args.Asp = c->tcA;
  args.Bsp = c->tcB;
  args.ndof = c->g.ndof;
  args.tiles = tiles;
  args.items = args.tiles * ngroups;
  args.N = N;
  args.M = M;
  args.K = K;
  args.G = G;
  args.NR = NR;
  args.from_zero = from_zero;
  args.err = c->tc_err;
  int dev = 0, sms = 0;
  PE_CUDA_TRY(cudaGetDevice(&dev));
  PE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::min<int64_t>(args.items, sms);
  pe_status st = PE_OK;
  switch (KP) {
    case 16: st = ft_launch<16>(args, grid, c->stream); break;
    case 32: st = ft_launch<32>(args, grid, c->stream); break;
    default: st = ft_launch<64>(args, grid, c->stream); break;
  }
  c->launches += 1;
  return st;
}

pe_status fine_tc_status(pe_ctx* c) {
  if (!c->tc_err) return PE_OK;
  int herr = 0;
  PE_CUDA_TRY(cudaMemcpyAsync(&herr, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (herr != 0) {
    cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->stream);
    return pe_fail(PE_ETIMEOUT, "fine sweep (tensor cores): a pipeline wait expired (code " + std::to_string(herr) + ")");
  }
  return PE_OK;
}

// ---------------------------------------------------------------------------
// batched form (pe_batch with fine_engine = PE_FINE_TC)
// ---------------------------------------------------------------------------
bool batch_tc_shape(int K, int M, int* KP, int* TG, int* NR) {
  if (!fine_tc_supported(M) || K < 1 || K > 64) return false;
  *KP = ft_kpad(K);
  int ng = 0;
  ft_shape(*KP, M, 1, TG, NR, &ng);
  return true;
}

pe_status batch_tc_prepare(pe_batch* b, cudaStream_t st) {
  const unsigned threads = 256;
  if (b->tc.y_jobs > 0)
    b_split_time_kernel<<<(unsigned)((b->tc.y_jobs + threads - 1) / threads), threads, 0, st>>>(
        b->d_probs, b->tc.d_y_prefix, b->P, b->tc.y_jobs, b->AF32, b->tc.B);
  if (b->tc.w_jobs > 0)
    b_split_w_kernel<<<(unsigned)((b->tc.w_jobs + threads - 1) / threads), threads, 0, st>>>(
        b->d_probs, b->tc.d_w_prefix, b->P, b->tc.w_jobs, b->W32, b->tc.A);
  b->launches += 2;
  PE_CUDA_TRY(cudaGetLastError());
  return PE_OK;
}

pe_status batch_tc_fine(pe_batch* b, cudaStream_t st) {
  for (int cls = 0; cls < 3; ++cls) {
    const int n = b->tc.begin[cls + 1] - b->tc.begin[cls];
    if (n == 0) continue;
    BtcArgs args{};
    args.probs = b->d_probs;
    args.items = b->tc.d_items + b->tc.begin[cls];
    args.n_items = n;
    args.coefF32 = b->coefF32;
    args.coefF = b->coefF;
    args.U = b->U;
    args.Fbar = b->Fbar;
    args.A = b->tc.A;
    args.B = b->tc.B;
    args.err = b->tc.err;
    const int grid = std::min(n, b->sm_count);
    if (cls == 0) PE_TRY(btc_launch<16>(args, grid, st));
    else if (cls == 1) PE_TRY(btc_launch<32>(args, grid, st));
    else PE_TRY(btc_launch<64>(args, grid, st));
  }
  return PE_OK;
}

pe_status batch_tc_status(pe_batch* b) {
  if (!b->tc.err) return PE_OK;
  int herr = 0;
  PE_CUDA_TRY(cudaMemcpy(&herr, b->tc.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr != 0) {
    cudaMemset(b->tc.err, 0, sizeof(int));
    return pe_fail(PE_ETIMEOUT, "batched fine sweep (tensor cores): a pipeline wait expired (code " +
                                    std::to_string(herr) + ")");
  }
  return PE_OK;
}
