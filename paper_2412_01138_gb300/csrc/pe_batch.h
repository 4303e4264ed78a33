// Internal layout of the batched solver (pe_batch): per-problem records,
// work items and arenas.  Not part of the ABI.
#pragma once
#include <vector>

#include "pe_forcing_common.cuh"
#include "pe_internal.h"

// One problem of the batch, as the kernels see it (offsets index the arenas).
struct BProb {
  Geom g;
  int N, M, q, p, R, Ru;   // slices, substeps, fine/coarse stages, forcing / u0 terms
  int K;                   // stage-contracted columns of the fine step (one per exponential, two per sinusoid)
  int mchunk;              // substeps of time factors staged per shared-memory fill
  int dbuf;                // mixed: 1 if two whole [M][KC] slice blocks fit the staging buffer
  int tf, tu;              // first forcing / u0 term in the terms array
  double D, t0, dT, dt;
  double lo[PE_MAX_D], h[PE_MAX_D];
  double cF[PE_MAX_S], cG[PE_MAX_S];
  double lagF[PE_MAX_S][PE_MAX_S], lagG[PE_MAX_S][PE_MAX_S];
  int64_t oU;    // U arena: (N+1)*ndof
  int64_t oS;    // Fbar arena: N*ndof
  int64_t oCF;   // coefF / coefF32 arenas: (q+2)*ndof
  int64_t oCG;   // coefG arena: (p+1)*ndof
  int64_t oAx;   // axisF / axisF32: R*nsum
  int64_t oAxU;  // axisU0: Ru*nsum
  int64_t oAF;   // AF: substep-start time factors Y, N*M*K
  int64_t oAF32; // AF32: the same in float, rows padded to KC = roundup(K, 4) (zeros), N*M*KC
  int64_t oW;    // W / W32: per-mode stage weights, K*ndof
  int64_t oZ;    // Z: stage shifts, q*K
  int64_t oCol;  // column map: K entries, (term << 1) | kind
  int64_t oAG;   // AG: N*p*R
  int64_t oMu;   // muM / ratio: nsum
  int64_t oItems;  // first mode item of this problem
  int nItems;
  // tensor-core fine engine (pe_options.fine_engine = PE_FINE_TC): column padding KP, slice
  // groups of TG slices (NR = TG * M rows of the B operand), the operand images' byte offsets
  int KP, TG, NR, groups;
  int64_t tiles;  // 128-mode tiles
  int64_t oTA;    // split stage weights, tiles * 3 * 128 * KP bf16
  int64_t oTB;    // split time factors, groups * 3 * NR * KP bf16
  // learned coarse correction (pe_batch_set_learned): band table K^[r][band] (re, im) at oKt,
  // bands log-spaced in log(lam dT) from lloglo by lstep; phase table (cos, sin)(w_r T_n + phi_r)
  // [r][n] at oPh
  int64_t oKt, oPh;
  double lloglo, lstep;
};

// A work item of the batched tensor-core fine sweep: slice group g and 128-mode tile t of problem p.
struct BTcItem {
  int p, g;
  int64_t t;
};

// tensor-core images of one batch and its work items (one list per column padding 16 / 32 / 64)
struct BatchTc {
  unsigned char* A = nullptr;  // split stage weights of every problem's tiles
  unsigned char* B = nullptr;  // split time factors of every problem's slice groups
  BTcItem* d_items = nullptr;
  int begin[4] = {};           // items of padding class c (KP = 16 << c): [begin[c], begin[c + 1])
  int64_t* d_w_prefix = nullptr;  // per problem: first split-weight job (tiles * 128 * KP / 8)
  int64_t* d_y_prefix = nullptr;  // per problem: first split-time job (groups * NR * KP / 8)
  int64_t w_jobs = 0, y_jobs = 0;
  int* err = nullptr;          // error code of an expired pipeline wait (0: none)
};

// Modes per thread of the mixed-precision fine tile for a problem with K stage columns
// (the work items and the kernel's tile dispatch both use it).
__host__ __device__ constexpr int batch_mixed_mpt(int KC) { return KC <= 16 ? 4 : (KC <= 24 ? 3 : 2); }

struct ModeItem {
  int p;
  int pad;
  int64_t J0;
};

struct FineItem {
  int p;
  int unused;   // padding (an item covers every slice of its problem)
  int64_t J0;
};

struct FactorJob {
  int p, axis, r, u0;
};

struct BatchArrays {
  const double* W;
  const float* W32;
  const double* AF;
  const float* AF32;
  const double* coefF;
  const float* coefF32;
  const double* U;
  double* Fbar;
};

// Fine work items of one tile width, grouped by column class: the items of class c
// (KC = 4(c+1)) are d_items[begin[c] .. begin[c+1]).
constexpr int kBatchClasses = (2 * PE_BATCH_MAX_TERMS + 3) / 4;
struct FineItems {
  FineItem* d_items = nullptr;
  int n = 0;
  int begin[kBatchClasses + 1] = {};
  size_t smem[kBatchClasses] = {};
};

struct pe_batch {
  int P = 0;
  int precision = PE_MIXED;
  int quad_pts = 3;
  int sm_count = 152;
  cudaStream_t stream = nullptr;   // owned, non-blocking (graph capture needs one)
  cudaStream_t user_stream = nullptr;
  std::vector<BProb> probs;
  BProb* d_probs = nullptr;
  std::vector<pe_term> terms;
  pe_term* d_terms = nullptr;
  Gauss gauss;
  int nmax = 1;
  // items
  ModeItem* d_mode_items = nullptr;
  int n_mode_items = 0;
  FineItems fine128, fine256;
  FactorJob* d_factor_jobs = nullptr;
  int n_factor_jobs = 0;
  int64_t* d_mu_prefix = nullptr;
  int64_t mu_total = 0;
  int64_t* d_tt_prefix = nullptr;
  int64_t tt_total = 0;
  // arenas
  double *muM = nullptr, *ratio = nullptr;
  double *coefF = nullptr, *coefG = nullptr;
  float* coefF32 = nullptr;
  double *U = nullptr, *Fbar = nullptr;
  double *axisF = nullptr, *axisU0 = nullptr;
  float* axisF32 = nullptr;
  double *AF = nullptr, *AG = nullptr;
  float* AF32 = nullptr;
  double *W = nullptr, *Z = nullptr;
  float* AG32 = nullptr;
  float* Z32 = nullptr;  // mixed: float copy of the stage shifts Z
  float* W32 = nullptr;
  short* d_cols = nullptr;
  double* partials = nullptr;
  // per-problem iteration state
  int *active = nullptr, *kcount = nullptr;
  double* resid = nullptr;
  int* counter = nullptr;
  int* dflags = nullptr;   // [0] active problems after the last iteration, [1] non-finite seen
  int* n_active = nullptr;
  int* nonfinite = nullptr;
  int* h_flags = nullptr;  // pinned copy of dflags
  // graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  double graph_tol = -1.0;
  int graph_threads = 0, graph_ctas = 0;
  // learned coarse correction (pe_batch_set_learned)
  const struct pe_mlp* mlp = nullptr;
  double* Kt = nullptr;       // band tables of every problem
  float2* Ph = nullptr;       // phase tables of every problem
  int64_t* d_kt_prefix = nullptr;  // per problem: first band-table job (R * bands)
  int64_t* d_ph_prefix = nullptr;  // per problem: first phase-table job (R * N)
  int64_t kt_jobs = 0, ph_jobs = 0;
  // tensor-core fine engine (PE_FINE_TC)
  int fine_engine = PE_FINE_SIMT;
  BatchTc tc;
  // launch shape of the persistent fine kernel
  int tune_threads = 256, tune_ctas = 2;
  bool tuned = false;
  bool have_problem = false;
  int64_t launches = 0;
  uint64_t signature = 0;
};

// pe_batch.cu
pe_status batch_set_attributes(pe_batch* b);
pe_status batch_launch_axis_tables(pe_batch* b);
pe_status batch_launch_coef_tables(pe_batch* b);
pe_status batch_launch_prepare(pe_batch* b);
pe_status batch_enqueue_iteration(pe_batch* b, cudaStream_t st, double tol);
pe_status batch_time_fine(pe_batch* b, int threads, int ctas, float* ms);
int batch_fine_launches(const pe_batch* b);  // fine kernels per iteration (one per column class)
// pe_learned.cu: band and phase tables of the learned correction for every problem of a batch
constexpr int kBatchLearnedBands = 2048;
pe_status batch_learned_tables(pe_batch* b, cudaStream_t st);
// pe_fine_tc.cu: the batched tensor-core fine sweep
bool batch_tc_shape(int K, int M, int* KP, int* TG, int* NR);  // false: M unsupported
pe_status batch_tc_prepare(pe_batch* b, cudaStream_t st);        // split images of every problem
pe_status batch_tc_fine(pe_batch* b, cudaStream_t st);           // one launch per padding class present
pe_status batch_tc_status(pe_batch* b);                          // PE_ETIMEOUT if a wait expired
// pe_batch_fine_*.cu (KC: the column class of the launch)
pe_status batch_launch_fine_mixed(int KC, const BProb* probs, const FineItem* items, int n_items, const int* active,
                                  int* counter, BatchArrays A, int grid, int threads, size_t smem, cudaStream_t st);
pe_status batch_launch_fine_f64(int KC, const BProb* probs, const FineItem* items, int n_items, const int* active,
                                int* counter, BatchArrays A, int grid, int threads, size_t smem, cudaStream_t st);
