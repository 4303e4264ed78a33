// Internal declarations shared by the libpe translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "pe.h"

#define PE_MAX_D 3
#define PE_MAX_S 8
#define PE_NEV 10  // timing events of a context

// ---------------------------------------------------------------------------
// error reporting (thread-local message behind pe_last_error)
// ---------------------------------------------------------------------------
void pe_set_error(const std::string& msg);
pe_status pe_fail(pe_status st, const std::string& msg);
pe_status pe_cuda_fail(cudaError_t err, const char* what);

#define PE_CUDA_TRY(call)                                  \
  do {                                                     \
    cudaError_t err__ = (call);                            \
    if (err__ != cudaSuccess) return pe_cuda_fail(err__, #call); \
  } while (0)

#define PE_TRY(call)                          \
  do {                                        \
    pe_status st__ = (call);                  \
    if (st__ != PE_OK) return st__;           \
  } while (0)

// ---------------------------------------------------------------------------
// geometry shared by the kernels: per-axis sizes and strides of a mode index
// ---------------------------------------------------------------------------
struct Geom {
  int d;
  int n[PE_MAX_D];        // interior nodes per axis (all nodes of a periodic axis)
  int off[PE_MAX_D];      // offset of axis a in concatenated per-axis tables
  int per[PE_MAX_D];      // 1: periodic axis (DHT basis), 0: Dirichlet (DST-I basis)
  int64_t ndof;
};

// Decompose a flat C-ordered mode index into per-axis indices (0-based); j[a] for a >= g.d is
// left unset.  Unrolled over PE_MAX_D axes so that j stays in registers when the caller's axis
// loops are unrolled too; 32-bit divisions while J fits (every grid of up to 2^32 modes).
__host__ __device__ inline void unflatten(const Geom& g, int64_t J, int* j) {
  if (J >= 0 && J <= (int64_t)0xFFFFFFFFu) {
    unsigned u = (unsigned)J;
#pragma unroll
    for (int a = PE_MAX_D - 1; a >= 0; --a)
      if (a < g.d) {
        const unsigned n = (unsigned)g.n[a], q = u / n;
        j[a] = (int)(u - q * n);
        u = q;
      }
    return;
  }
#pragma unroll
  for (int a = PE_MAX_D - 1; a >= 0; --a)
    if (a < g.d) {
      j[a] = (int)(J % g.n[a]);
      J /= g.n[a];
    }
}

// Separable forcing, device layout (R terms, K stage-contracted columns):
//   axisF[R * off[a] + r * n_a + j]         = modal factor (S_a F_{r,a})_j / mu^M_a(j)
//   AF[(n * M + m) * K + k]                 = Y_k(T_n + m dt)   (substep-start time factors)
//   Zst[i * K + k]                          = Z_k(c_i dt)       (stage shifts)
//   Wst[k * ndof + J]                       = P_{r(k),J} sum_i dt b_i(J) Z_k(c_i dt)
//   AG[(n * p + i) * R + r]                 = amp_r * time_r(T_n + c_i dT)
// Column k belongs to term colTerm[k]: an exponential time factor gives one
// column (Y = amp e^{at}, Z = e^{as}); a sinusoid gives two (kind 0:
// Y = amp sin(wt+phi), Z = cos(ws); kind 1: Y = amp cos(wt+phi), Z = sin(ws)).
struct StageCols {
  int K;
  signed char term[2 * PE_MAX_TERMS];
  signed char kind[2 * PE_MAX_TERMS];
};
// Device-resident state of a solve whose Parareal loop runs as a CUDA graph (device_loop):
// the correction kernel's last CTA appends r_k, advances k and sets the graph's loop condition.
struct LoopCtl {
  int k, max_iter, nonfinite, hist_cap;
  double tol, r;
  double* hist;   // [hist_cap] residuals r_1 .. r_k (device)
  LoopCtl* host;  // device address of the mapped pinned mirror that receives k, r, nonfinite
};

struct pe_ctx {
  // problem
  Geom g;    // the modes this context owns (every mode unless it owns a block of axis-0 modes)
  Geom gn;   // the whole grid (nodal arrays, DST-I passes, per-axis loads); equals g unsharded
  bool sharded = false;  // owns the axis-0 modes [base0, base0 + g.n[0]) of gn.n[0]
  int base0 = 0;
  double lo[PE_MAX_D], hi[PE_MAX_D], h[PE_MAX_D];
  double D, t0, T, dT, dt;
  int N, M, q, p;
  double cF[PE_MAX_S], cG[PE_MAX_S];
  double lagF[PE_MAX_S][PE_MAX_S], lagG[PE_MAX_S][PE_MAX_S];  // Lagrange monomial coefficients
  int nsum;       // sum_a n_a of g (per-axis modal tables)
  int nsum_full;  // sum_a n_a of gn (per-axis nodal loads)
  // a sharded context: per-axis tables of the whole axes (compacted into the tables above),
  // and a whole-grid buffer for its nodal transforms
  double* muM_full = nullptr;   // [nsum_full]
  double* ratio_full = nullptr; // [nsum_full]
  double* fac_full = nullptr;   // [PE_MAX_TERMS * nsum_full]
  double* work2 = nullptr;      // [gn.ndof]
  void (*reduce)(double*, void*) = nullptr;  // residual sums across contexts (pe_options.residual_reduce)
  void* reduce_user = nullptr;
  // options
  int precision, dst_backend, quad_pts, max_iter, forcing_path, cache_forced;
  int fine_engine = 0;  // PE_FINE_SIMT | PE_FINE_TC
  cudaStream_t stream;
  // device memory
  double* muM_axis = nullptr;   // [nsum]
  double* ratio_axis = nullptr; // [nsum] mu^K/mu^M
  double* S[PE_MAX_D] = {nullptr, nullptr, nullptr};  // DST-I matrices n_a x n_a
  float* S32[PE_MAX_D] = {nullptr, nullptr, nullptr};  // float copies (general path, mixed)
  // general forcing path: stage-time loads and their transforms for a chunk of slices
  double* gen_L = nullptr;      // [stages][R * nsum] 1D loads
  double* gen_buf = nullptr;    // [stages][ndof] transformed loads (float in the mixed fine sweep)
  double* gen_tmp = nullptr;    // same size, DST ping-pong
  double* lam = nullptr;        // [ndof]
  double* coefF = nullptr;      // [(q+2) * ndof]: E, dt*b_1..q, exp(-lam M dt)
  double* coefG = nullptr;      // [(p+1) * ndof]: E, dT*b_1..p
  float* coefF32 = nullptr;     // [(q+2) * ndof]: E_hi, E_lo, dt*b_i (float)
  double* U = nullptr;          // [(N+1) * ndof]
  double* Fz = nullptr;         // [N * ndof] cached F^M(0) per slice (cache_forced)
  int fz_prec = -1;             // precision Fz was computed in, -1: none for this problem
  int64_t sweeps = 0;           // fine sweeps executed since the last reset
  double* Fbar = nullptr;       // [N * ndof]
  double* gG = nullptr;         // [N * ndof] coarse forcing of each slice
  double* work0 = nullptr;      // [gn.ndof] nodal / DST scratch
  double* work1 = nullptr;      // [gn.ndof]
  float* io32 = nullptr;        // [3 gn.ndof] float32 transform scratch of the mixed form (null: float64 transforms)
  double* muM_inv = nullptr;    // [nsum of the whole grid] 1 / mu^M per axis node
  double* out_nodal = nullptr;  // [gn.ndof] inverse DST of U^N after pe_solve
  double* partials = nullptr;   // [2 * max_blocks]
  double* red = nullptr;        // [2] device
  unsigned int* done_ctr = nullptr;  // correction: CTAs finished (0 between launches)
  unsigned char* tcB = nullptr;  // tensor-core fine engine: split time factors of every slice group
  unsigned char* tcA = nullptr;  // tensor-core fine engine: split stage weights of every mode tile
  size_t tcA_cap = 0;            // bytes allocated in tcA
  bool tc_split_ok = false;      // tcA / tcB hold the current problem's split operands
  int* tc_err = nullptr;         // tensor-core fine engine: error code of an expired wait (0: none)
  cudaStream_t side = nullptr;  // second stream: the nodal u0 transform beside the forcing tables
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_tables = nullptr;
  double* h_red = nullptr;      // [2] pinned host
  int max_blocks = 0;
  int sms = 0;                      // SMs of the context's device
  // forcing (set by pe_set_problem)
  int R = 0;
  pe_term terms[PE_MAX_TERMS];
  signed char lkind[PE_MAX_TERMS][PE_MAX_D] = {};  // load kinds of terms (Dirichlet lifting)
  // non-homogeneous Dirichlet data (pe_set_dirichlet): separable terms on the closed box
  int nbd = 0;
  pe_term bterms[PE_MAX_TERMS];
  double* axisF = nullptr;      // [PE_MAX_TERMS * nsum]
  float* axisF32 = nullptr;     // [PE_MAX_TERMS * nsum]
  double* axisU0 = nullptr;     // [PE_MAX_TERMS * nsum] factors of separable u0
  double* AF = nullptr;         // [N*M*2*PE_MAX_TERMS]
  float* AF32 = nullptr;
  int K = 0;                    // stage-contracted columns of the current forcing
  StageCols cols{};
  double* Zst = nullptr;        // [PE_MAX_S * 2*PE_MAX_TERMS]
  double* Wst = nullptr;        // [K * ndof] (allocated on first use, grown with K)
  float* Wst32 = nullptr;       // [K * ndof] (mixed precision)
  int Wcap = 0;                 // columns allocated in Wst / Wst32
  bool Wst_valid = false;       // Wst holds the current problem's float64 weights
  double* AG = nullptr;         // [N*p*PE_MAX_TERMS]
  float* AG32 = nullptr;
  double* loads = nullptr;      // [PE_MAX_TERMS * nsum_full] 1D loads before the DST
  // learned coarse correction (optional)
  const struct pe_mlp* mlp = nullptr;
  double* Ktab = nullptr;       // [PE_MAX_TERMS][bands][2]
  void* phase_tab = nullptr;    // [PE_MAX_TERMS][N] float2
  // accounting
  int64_t launches = 0;     // kernels launched since the last reset
  double ms_fine = 0.0;     // device time of fine-propagator kernels since the last reset
  double ms_corr = 0.0;     // device time of correction kernels since the last reset
  // state
  int k = 0;
  bool have_problem = false;
  bool have_output = false;
  cudaEvent_t ev[PE_NEV];
  // device-resident Parareal loop (pe_options.device_loop)
  int device_loop = 0;
  cudaGraphExec_t loop_exec = nullptr;
  int loop_K = -1, loop_prec = -1;  // what the graph was built for
  int64_t loop_body_launches = 0;   // kernels of one pass of the graph's body
  LoopCtl* loopctl = nullptr;       // device
  LoopCtl* h_loop = nullptr;        // mapped pinned mirror of the loop state (host address)
  LoopCtl* h_loop_dev = nullptr;    //   its device address
  double* loop_hist = nullptr;      // device [N]
  // device_loop = 2: the set-up and output phases of a repeated problem replayed as CUDA graphs
  cudaStream_t cap_stream = nullptr;  // capture stream (the context's own may be the legacy stream)
  cudaGraphExec_t setup_exec = nullptr, out_exec = nullptr;
  uint64_t graph_key = 0;           // problem the graphs were captured for
  int graph_key_seen = 0;           // solves of graph_key so far (captured at the second)
  // a solve enqueued by pe_solve_async (or the first half of pe_solve), reported by pe_solve_wait
  bool pend = false, pend_on_device = false;
  double pend_tol = 0.0, pend_r = 0.0;
  std::vector<double> pend_hist;    // residuals of the host-driven loop
  int64_t setup_launches = 0, out_launches = 0;
  int u0_dev_hint = -1;             // u0 nodal pointer is device memory (1) / host (0) / unknown (-1)
  int capturing = 0;                // the phase being run is captured (timing events become graph nodes)
};

// Substeps of time factors (per_m values each) staged per shared-memory fill.
inline int pick_mchunk(int M, int per_m, size_t elem) {
  const size_t budget = 48 * 1024;
  int mc = (int)(budget / (elem * (size_t)per_m));
  if (mc < 1) mc = 1;
  return mc < M ? mc : M;
}

// ---------------------------------------------------------------------------
// launchers (each returns a pe_status and reports errors through pe_set_error)
// ---------------------------------------------------------------------------
// pe_api.cu (shared host helpers)
pe_status pe_resolve_nodes(const pe_tableau* tb, const char* name, int* s_out, double* c);
void pe_lagrange_coeffs(int s, const double* c, double a[PE_MAX_S][PE_MAX_S]);
bool pe_is_device_ptr(const void* p);
pe_status pe_validate_terms(int n, const pe_term* t, int d, const char* what, bool allow_moving = false);

// pe_tables.cu
pe_status launch_axis_tables(pe_ctx* c);
pe_status launch_coef_tables(pe_ctx* c);
pe_status build_dst_matrix(int n, double* S, cudaStream_t st, int periodic = 0);  // DST-I, or the DHT
pe_status build_dst_matrix_f32(int n, float* S, cudaStream_t st, int periodic = 0);

// pe_forcing.cu
pe_status launch_time_tables(pe_ctx* c);   // also sets c->K, c->cols and Zst
pe_status launch_stage_weights(pe_ctx* c);  // Wst (float64 form) or Wst32 (mixed form)
pe_status launch_stage_weights_f64(pe_ctx* c);  // Wst, if not yet made for this problem
// rows of whole-axis per-axis tables [R * nsum_full] kept by a sharded context, in its layout
pe_status compact_axis_tables(pe_ctx* c, int R, const double* in, double* out, float* out32);
pe_status launch_separable_factors(pe_ctx* c, const pe_term* terms, int nterms, double* axis_out, int mode,
                                   const signed char (*lk)[PE_MAX_D] = nullptr);
pe_status launch_outer_sum(pe_ctx* c, const double* axis_fac, const pe_term* terms, int nterms, double* out,
                           int accumulate);
pe_status launch_forcing_modal(pe_ctx* c, double t, double* out);

// pe_dst.cu
// periodic: the axis' transform is the DHT held in S (matrix form; no FFT)
pe_status dst_axis_f64(const double* S, const double* in, double* out, int64_t outer, int n, int64_t inner,
                       cudaStream_t st, int periodic = 0);
pe_status dst_axis_f32(const float* S, const float* in, float* out, int64_t outer, int n, int64_t inner,
                       cudaStream_t st, int periodic = 0);
pe_status dst_nd_f64(pe_ctx* c, const double* in, double* out);
// float64 data transformed in float32 arithmetic through c->io32 (FFT-length axes only)
bool dst_nd_f32_ok(const Geom& g);
pe_status dst_nd_mixed(pe_ctx* c, const double* in, double* out);  // whole grid (c->gn); uses c->S, c->work1
// Per-axis source factors of every axis in one launch (loads -> DST-I -> / mu^M); *done = false when
// an axis is periodic or n_a + 1 is not a power of two in 16..1024 (nothing launched then).
pe_status axis_factors_fused(pe_ctx* c, int R, const double* loads, double* fac, float* fac32, bool* done);

// pe_sweep.cu
pe_status launch_coarse_sweep(pe_ctx* c);
pe_status launch_fine_sweep(pe_ctx* c, int precision);
pe_status launch_correction(pe_ctx* c, double* num, double* den, cudaEvent_t after = nullptr);
// the correction kernel alone; with loop != NULL its last CTA also runs the stopping decision of a
// device-resident loop (appends r, advances k, sets the graph condition `handle`)
pe_status launch_correction_kernel(pe_ctx* c, LoopCtl* loop, unsigned long long handle);
// Arms the device-resident loop's state for one solve (k = 0, tol, the history, the mirror).
pe_status launch_loop_init(pe_ctx* c, double tol);
pe_status launch_scale_by_muM(pe_ctx* c, double* x, int inverse);

// pe_learned.cu
pe_status launch_learned_correction(pe_ctx* c);

// pe_general.cu
int general_slices_per_chunk(const pe_ctx* c);
pe_status launch_general_coarse_forcing(pe_ctx* c);
pe_status launch_general_fine_sweep(pe_ctx* c, int precision);

// pe_fine_tc.cu (tensor-core engine of the mixed fine sweep)
bool fine_tc_supported(int M);                 // M a multiple of 16 in 16..128
size_t fine_tc_buffer_bytes(int M, int N);     // split time factors, any K <= 64
// Threads per CTA of a kernel with one thread per mode: when the modes fit one wave of CTAs,
// as many warps as an even share of the SMs needs (every SM then runs one CTA of equal size,
// rather than some SMs two CTAs of 256 threads and others one); 256 otherwise.
inline int per_mode_block(int64_t units, int sms) {
  if (sms <= 0) return 256;
  const int64_t per_sm = (units + sms - 1) / sms;
  if (per_sm > 512) return 256;
  const int64_t t = (per_sm + 31) / 32 * 32;
  return (int)(t < 64 ? 64 : t);
}

// Programmatic dependent launch: a kernel launched by launch_pdl may be scheduled while its
// predecessor on the stream is still running.  Each such kernel calls pdl_wait() first, before
// it touches global memory: it waits there until the predecessor has completed and its writes
// are visible, then lets its own successor be scheduled early in turn.  Without the launch
// attribute (a plain launch) both instructions do nothing.
// Exact float32 -> float64 widening.  GB300 runs the F2F conversion on its float64 pipe (two
// lanes per SM), where the recurrences that add a float32 sum into a float64 state already
// spend their float64 budget; a normal float32 is widened here with integer operations instead
// (IEEE 754 binary32 -> binary64: exponent rebiased by 1023 - 127 = 896, fraction shifted left
// by 29), zero by its sign alone, and the rare subnormal, infinite or NaN values by the
// conversion, behind a call so that it is not issued for the common case.
static __device__ __noinline__ double widen_f32_rare(float x) { return (double)x; }
__device__ __forceinline__ double widen_f32(float x) {
  const unsigned u = __float_as_uint(x), mag = u & 0x7FFFFFFFu;
  if (mag - 0x00800000u < 0x7F000000u)
    return __hiloint2double((int)((u & 0x80000000u) | ((mag >> 3) + 0x38000000u)), (int)(u << 29));
  if (mag == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  return widen_f32_rare(x);
}

__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Drops the cached set-up and output graphs of a repeated problem (pe_api.cu).
void drop_solve_graphs(pe_ctx* c);
pe_status fine_tc_prepare(pe_ctx* c);          // split operand images of the current problem
pe_status fine_tc_prepare_time(pe_ctx* c);     //   the time factors' image (after the time tables)
pe_status fine_tc_prepare_weights(pe_ctx* c);  //   the stage weights' image (after tables and factors)
pe_status launch_fine_tc(pe_ctx* c, int from_zero, double* out);
pe_status fine_tc_status(pe_ctx* c);           // PE_ETIMEOUT if a pipeline wait expired
