/*
 * pe.h -- C-ABI of libpe, a GB300 (sm_103a) implementation of the data-parallel
 * hot path of the Parareal exponential-integrator Q1 finite element method
 * (PEIFE-linear) of Huang & Xu, arXiv 2412.01138.
 *
 * Problem (Sec. 2, Eq. (1-1) with homogeneous Dirichlet data, Eq. (3-1)):
 *     u_t = D Lap u + f(t, x)  on a rectangle  Omega = prod_a (lo_a, hi_a),
 *     u = 0 on the boundary,  u(t0) = u0,  t in [t0, t0 + T].
 * Space: Q1 elements on a uniform grid with n_a interior nodes per axis
 * (h_a = (hi_a - lo_a)/(n_a + 1)), Sec. 2.1.  The mass and stiffness matrices
 * are diagonalised at once by the orthonormal tensor DST-I V = kron_a S_a
 * (closing paragraph of Sec. 2.3), which turns the semi-discrete system
 * Eq. (1-5) into independent scalar ODEs c_J' = -lam_J c_J + ghat_J(t).
 * Time: the exponential Runge-Kutta step Eq. (1-7) with weights Eq. (3-12);
 * coarse propagator G = one step of dT = T/N with p nodes, fine propagator
 * F^M = M steps of dt = dT/M with q nodes, combined by Algorithm 1.
 *
 * Array layout: nodal and modal arrays are C-ordered, shape (n_0, .., n_{d-1}),
 * axis d-1 contiguous, float64 unless stated.  Slice arrays are [N+1][Ndof].
 *
 * Ownership: the caller owns every buffer it passes; the library copies what
 * it needs during the call and keeps no caller pointer.  A pointer argument
 * may be host or device memory wherever a comment says "host or device"; the
 * library inspects it with cudaPointerGetAttributes.  All device work is
 * issued on the stream given in pe_options (NULL: the legacy default stream);
 * every call that returns data to a host pointer synchronises that stream.
 *
 * Errors: every function returns a pe_status; no exception crosses the ABI.
 * pe_last_error() returns a message for the most recent failure on the
 * calling thread.  A context is not thread-safe: use one per thread.
 */
#ifndef PE_H
#define PE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pe_ctx pe_ctx; /* opaque; owns its device memory */

typedef enum {
  PE_OK = 0,
  PE_EINVAL = -1,      /* invalid argument (sizes, D <= 0, duplicate nodes, ...) */
  PE_ENOMEM = -2,      /* device or host allocation failed */
  PE_ECUDA = -3,       /* a CUDA call failed; message in pe_last_error() */
  PE_ENOCONV = -4,     /* pe_solve: residual above tol after max_iter iterations */
  PE_ENONFINITE = -5,  /* a NaN/Inf reached the Parareal residual */
  PE_ETIMEOUT = -6,    /* a bounded device-side wait expired */
  PE_ESTATE = -7       /* call out of order (e.g. iterate before a problem is set) */
} pe_status;

/* precision of the fine propagator (pe_options.precision) */
enum { PE_FP64 = 0,   /* every step in float64 */
       PE_MIXED = 1   /* fine stages in float32 on the zero-start forced part, the
                         homogeneous part e^{-lam M dt} v, tables, correction and
                         residual in float64 */ };

/* engine of the mixed-precision fine sweep (pe_options.fine_engine), separable forcing only:
 * SIMT = float32 FMAs on the CUDA cores; TC = the stage contraction of every 128 modes x
 * (slice group) on the tensor cores (tcgen05, three-term bfloat16 split of both operands,
 * six products, float32 accumulation; about the accuracy of the float32 form), the
 * recurrence and the float64 homogeneous term on the CUDA cores.  TC needs M (substeps
 * per slice) a multiple of 16 in 16..128: pe_setup returns PE_EINVAL otherwise, and for
 * PE_FP64 or PE_FORCING_GENERAL.  The float64 refinement (pe_refine) is unaffected. */
enum { PE_FINE_SIMT = 0, PE_FINE_TC = 1 };

/* DST-I backend of the general forcing path (pe_options.dst_backend): AUTO = radix-2 FFT
 * when n+1 is a power of two, else the matrix form; TC = tensor cores (mixed precision
 * only, split bfloat16, about 3e-6 relative per pass at n = 255) */
enum { PE_DST_AUTO = 0, PE_DST_MATRIX = 1, PE_DST_TC = 2 };

/* separable factor kinds: spatial  S_ONE 1 | S_SIN sin(p0 x + p1) |
 * S_GAUSS exp(-(x-p0)^2/(2 p1^2)) | S_POLY p0 + p1 x + p2 x^2 + p3 x^3 |
 * S_MOVING_HAT max(1 - |x - c(t)|/p3, 0), c(t) = p0 + p1 sin(2 pi p2 t) (a factor that
 * moves with t, the source of Example 4 of Sec. 5; PE_FORCING_GENERAL only);
 * time  T_EXP exp(p0 t) | T_SIN sin(p0 t + p1) */
enum { PE_S_ONE = 0, PE_S_SIN = 1, PE_S_GAUSS = 2, PE_S_POLY = 3, PE_S_MOVING_HAT = 4 };

/* how P_h f(t) is formed (pe_options.forcing_path) */
enum { PE_FORCING_SEPARABLE = 0, /* modal factors of every term once, products per mode and stage */
       PE_FORCING_GENERAL = 1    /* at every stage time: consistent load assembled in nodal space
                                    (element Gauss quadrature), tensor DST-I, division by Lambda_M */ };
enum { PE_T_EXP = 0, PE_T_SIN = 1 };

/* One separable term  amp * time(t) * prod_{a<d} spatial_a(x_a). */
typedef struct {
  double amp;
  int32_t tkind;
  double tp[2];
  int32_t skind[3];
  double sp[3][4];
} pe_term;

/* Interpolation nodes c_1..c_s in [0,1] of one exponential RK tableau (Eq. (1-7)).
 * c == NULL and random == 0: c_i = (i-1)/s.  random != 0: s nodes drawn from
 * SplitMix64(seed) as doubles (x >> 11) * 2^-53, sorted, the whole set redrawn
 * while two nodes are closer than 1e-3 (Theorem 3.1 holds for any distinct
 * nodes).  Nodes must be distinct (Lagrange basis of Eq. (3-12)): else PE_EINVAL. */
typedef struct {
  int32_t s;          /* 1 <= s <= 8 */
  const double* c;    /* host, s values, or NULL */
  int32_t random;
  uint64_t seed;
} pe_tableau;

typedef struct {
  int32_t precision;    /* PE_FP64 | PE_MIXED */
  int32_t dst_backend;  /* PE_DST_AUTO | PE_DST_MATRIX */
  int32_t quad_pts;     /* Gauss points per axis per element for loads (1..8, 0 = 3) */
  int32_t max_iter;     /* pe_solve iteration cap, 0 = N (Theorem 4.3: k = N is exact) */
  void* cuda_stream;    /* cudaStream_t or NULL */
  int32_t forcing_path; /* PE_FORCING_SEPARABLE (default) | PE_FORCING_GENERAL */
  int32_t cache_forced; /* 1: keep the forced part F^M(0) of every slice after the first fine
                           sweep and reuse it in later iterations (exact, since the fine
                           propagator is affine: F^M(v) = exp(-lam M dt) v + F^M(0)); later
                           iterations then run no fine sweep.  Separable forcing only; the
                           float64 refinement of a mixed run makes its own float64 copy. */
  int32_t periodic_mask;  /* bit a set: axis a is periodic -- n_a nodes x_k = lo + k h, k < n_a,
                             h = (hi - lo)/n_a, node n_a identified with node 0; the circulant Q1
                             matrices are diagonalised by the discrete Hartley transform
                             (DHT) in place of the DST-I, theta_j = 2 pi j / n_a, and the mode
                             j = 0 of an all-periodic problem has lam = 0.  Not with Dirichlet
                             data or the learned correction. */
  int32_t fine_engine;    /* PE_FINE_SIMT (default) | PE_FINE_TC, see above */
  /* Mode sharding (modes are independent after the diagonalisation of Sec. 2.3; only the
   * residual of the stopping rule couples them).  mode_begin <= j_0 < mode_end: this context
   * owns the modes whose index along axis 0 (the slowest axis) lies in that range (0-based),
   * a contiguous block of the C-ordered modal array; both 0: every mode.  A context that owns
   * a block: pe_get_modal, pe_get_lambda, pe_get_coefficients, pe_forcing_modal and
   * pe_save_state hold its (mode_end - mode_begin) * prod_{a>0} n_a modes; nodal u0
   * (PE_FIELD_NODAL) is the whole grid's; pe_get_solution returns the whole grid's nodal
   * values of its modes alone (the other modes taken as zero), so that the sum of these
   * fields over contexts covering every mode once is the nodal solution.  Its residual sums
   * are its own: pe_parareal_iter_sums returns them, and pe_parareal_iter / pe_solve need
   * residual_reduce to combine them across contexts (PE_EINVAL otherwise).  Separable forcing
   * only, no Dirichlet data, u0 nodal or PE_FIELD_TERMS_SEPARABLE. */
  int32_t mode_begin, mode_end;
  /* Called by pe_parareal_iter / pe_solve after the correction of every iteration with the
   * two residual sums of this context (sums[0] = sum mu^M (U_new - U_old)^2, sums[1] =
   * sum mu^M U_new^2 over its modes and slices); it must replace them by their totals over
   * every context of the solve (an all-reduce: MPI, NCCL, a host loop) and return.  NULL:
   * the context's own sums are the totals (the unsharded solve). */
  void (*residual_reduce)(double* sums, void* user);
  void* residual_reduce_user;
  /* 1: pe_solve runs Algorithm 1's loop on the device -- one CUDA graph whose conditional
   * (while) node repeats {fine sweep, correction + residual} and whose correction kernel
   * decides, from the float64 residual, whether to go on (r > tol and k < max_iter) -- so the
   * host waits once per solve instead of once per iteration.  Same kernels and results as the
   * host-driven loop; per-kernel times (pe_result.ms_fine_kernel, ms_correction_kernel) are not
   * measured in this mode (0).  The graph is built at the first such solve of a column count K
   * and reused.  Falls back to the host loop for cache_forced, the general forcing path and
   * contexts with residual_reduce.  0 (default): the host-driven loop of the paper's Algorithm 1.
   * 2: as 1, and a problem solved again -- the same u0 description (or the same device pointer
   * of nodal u0: its values are read anew each solve), forcing terms, Dirichlet data and network
   * pointer -- replays the set-up (transform of u0, forcing factors, stage weights, coarse
   * sweep) and output (inverse transform, lifting) phases as CUDA graphs captured at its second
   * solve, so that a solve costs a few graph launches.  Same kernels, same results.  Nodal u0 in
   * host memory, or any pe_set_problem / pe_set_dirichlet / pe_set_learned call in between, runs
   * the phases directly (and drops the graphs).  Other values: PE_EINVAL. */
  int32_t device_loop;
} pe_options;

/* Initial data: u0 = sum of separable terms (time factors ignored), projected
 * onto V_h by P_h (L2 projection, Eq. (3-11)), or nodal values of a V_h function. */
enum { PE_FIELD_TERMS_SEPARABLE = 0, /* P_h by per-axis 1D loads and 1D DST-I */
       PE_FIELD_TERMS_QUADRATURE = 1, /* P_h by d-D element quadrature + d-D DST-I */
       PE_FIELD_NODAL = 2 };          /* u0 already in V_h: c0 = V^T u0 */
typedef struct {
  int32_t kind;
  int32_t n_terms;
  const pe_term* terms;  /* host */
  const double* nodal;   /* host or device, Ndof values (kind == PE_FIELD_NODAL) */
} pe_field;

/* Source f = sum of separable terms (host array, 0 <= n_terms <= PE_MAX_TERMS). */
#define PE_MAX_TERMS 32
typedef struct {
  int32_t n_terms;
  const pe_term* terms;
} pe_forcing;

typedef struct {
  int32_t k;                 /* Parareal iterations performed */
  double residual;           /* last relative residual r_k (defined at pe_parareal_iter) */
  double* residual_history;  /* host, caller-owned, capacity history_cap (may be NULL) */
  int32_t history_cap;
  int64_t fine_sweeps;       /* fine propagator sweeps executed (= k; 1 with cache_forced) */
  double ms_tables;          /* device time of the forcing tables (time factors, per-axis modal
                                factors, fine-step stage weights); the phi/b coefficient tables
                                depend only on pe_setup's arguments and are made there */
  double ms_prepare;         /* projection of u0, coarse sweep */
  double ms_iterations;      /* all fine sweeps + corrections + residuals */
  double ms_output;          /* inverse DST of the final slice */
  double ms_fine_kernel;     /* device time of the fine-propagator kernels alone (sum over sweeps) */
  int64_t kernel_launches;   /* kernels this call launched */
  double ms_correction_kernel; /* device time of the correction + residual kernel (sum over iterations) */
  double ms_coarse_kernel;   /* device time of the coarse sweep of k = 0 (its kernels alone) */
} pe_result;

/*
 * pe_setup -- validate the problem, allocate the context and its device memory
 * (slice arrays U, F^M(U) and the coarse forcing of N x Ndof float64 each, plus tables).
 * d in 1..3; n: host int32[d], n_a >= 1; box: host double[2d] as lo0,hi0,lo1,hi1,..;
 * D > 0; T > 0; n_slices = N >= 1; n_substeps = M >= 1; fine (q nodes) and
 * coarse (p nodes) tableaux; opt may be NULL (defaults).  On success *out owns
 * everything; release with pe_destroy.
 */
pe_status pe_setup(pe_ctx** out, int32_t d, const int32_t* n, const double* box, double D,
                   double t0, double T, int32_t n_slices, int32_t n_substeps,
                   const pe_tableau* fine, const pe_tableau* coarse, const pe_options* opt);

/*
 * pe_set_problem -- Algorithm 1 up to its loop: compute lam_J (Sec. 2.3) and the
 * phi/b tables (Eq. (3-12)) for the fine and coarse steps, the modal factors of
 * P_h f (outer products of 1D projections of each separable term), U^0 = P_h u0,
 * and the coarse sweep U^{n+1,(0)} = G(U^{n,(0)}).  Sets k = 0.
 */
pe_status pe_set_problem(pe_ctx* ctx, const pe_field* u0, const pe_forcing* f);

/*
 * pe_set_dirichlet -- non-homogeneous Dirichlet data u = g on the boundary, for the
 * following pe_set_problem / pe_solve calls (n_terms = 0 restores u = 0).  The paper
 * treats u = 0 and states (openings of Sec. 3 and Sec. 4) that its results extend to
 * non-homogeneous data, without formulas; this library's reading: g is given as
 * separable terms (time factor exp or sin, spatial factors of the pe_term kinds except
 * the moving hat) on the CLOSED box, its values on the boundary are the data, and the
 * lifting is the Q1 interpolant I_h g on all nodes.  The solver integrates
 * w = u_h - I_h g (zero on the boundary) with the extra load
 * -(M d/dt I_h g + K I_h g) on interior nodes, from w(t0) = P_h(u0 - I_h g(t0))
 * (descriptor u0) or u0 - I_h g(t0) (nodal u0); pe_get_solution returns the interior
 * nodal values of u_h = w + I_h g, pe_get_modal the modal coefficients of w.  Each data
 * term adds 1 + d separable forcing terms (at most 32 in all).  Separable forcing path
 * only, not with the learned correction (PE_EINVAL).  g is copied (host array).
 */
pe_status pe_set_dirichlet(pe_ctx* ctx, int32_t n_terms, const pe_term* g);

/*
 * pe_parareal_iter -- one pass of Algorithm 1's loop: the fine propagator from
 * every slice start in parallel, then the sequential correction
 *   U^{n+1,(k+1)} = G(U^{n,(k+1)}) + F^M(U^{n,(k)}) - G(U^{n,(k)}),
 * and the relative residual
 *   r = sqrt(sum_{n=1}^N ||U^{n,(k+1)} - U^{n,(k)}||_0^2) / sqrt(sum_{n=1}^N ||U^{n,(k+1)}||_0^2)
 * in float64 (the paper leaves the stopping rule open; this relative residual is the rule used).
 * rel_residual_out: host, may be NULL.  Returns PE_ENONFINITE if a sum is not finite.
 */
pe_status pe_parareal_iter(pe_ctx* ctx, double* rel_residual_out);

/*
 * pe_parareal_iter_sums -- the same pass as pe_parareal_iter, returning the two float64
 * residual sums of this context's modes before any combination or division:
 * sums_out[0] = sum_{n=1}^N sum_J mu^M_J (U^{n,(k+1)}_J - U^{n,(k)}_J)^2 and
 * sums_out[1] = sum_{n=1}^N sum_J mu^M_J (U^{n,(k+1)}_J)^2 (host, 2 values).  The relative
 * residual of a mode-sharded solve is sqrt(sum of sums_out[0]) / sqrt(sum of sums_out[1])
 * over the contexts.  Returns PE_ENONFINITE if a sum is not finite.
 */
pe_status pe_parareal_iter_sums(pe_ctx* ctx, double* sums_out);

/*
 * pe_refine -- one Parareal iteration exactly like pe_parareal_iter but with the
 * fine propagator in float64 whatever pe_options.precision says.  Because G and
 * F share the homogeneous propagator e^{-lam dT} (up to rounding), one float64
 * iteration from a mixed-precision iterate reproduces the float64 fine solution
 * (the float64 refinement of the mixed form).  rel_residual_out: host, may be NULL.
 */
pe_status pe_refine(pe_ctx* ctx, double* rel_residual_out);

/*
 * pe_solve -- pe_set_problem, then pe_parareal_iter until r <= tol or k = N
 * (or max_iter), then the inverse DST of U^N into the context's output buffer
 * (read with pe_get_solution).  Returns PE_ENOCONV if max_iter < N stopped it
 * above tol.  out may be NULL.
 */
pe_status pe_solve(pe_ctx* ctx, const pe_field* u0, const pe_forcing* f, double tol, pe_result* out);

/*
 * pe_solve_out -- pe_solve, and the nodal solution u_h(T_N) = V U^N (Ndof values, the
 * whole grid also for a context that owns a block of modes: its modes' share) written
 * into nodal_out (host or device, caller-owned) in the same stream order before the
 * call returns: what pe_get_solution(ctx, N, nodal_out) gives afterwards, without a
 * second synchronisation.  PE_EINVAL if nodal_out is NULL; on PE_ENOCONV the buffer is
 * filled as well.
 */
pe_status pe_solve_out(pe_ctx* ctx, const pe_field* u0, const pe_forcing* f, double tol, double* nodal_out,
                       pe_result* out);

/*
 * pe_solve_async / pe_solve_wait -- pe_solve_out in two calls.  pe_solve_async enqueues the
 * whole solve (set-up, Algorithm 1's loop, the inverse DST of U^N and, if nodal_out is not
 * NULL, its copy into nodal_out) on the context's stream and returns; with the loop on the
 * device (pe_options.device_loop = 1 or 2) it does not wait for the GPU, with the host-driven
 * loop it waits for every residual as pe_solve does.  pe_solve_wait waits for the stream and
 * fills out (may be NULL) and returns what pe_solve would have returned (PE_ENOCONV,
 * PE_ENONFINITE, ...).  One solve may be pending per context: until pe_solve_wait, the
 * context's other calls that read or change its state return PE_ESTATE, and nodal_out
 * (caller-owned) and a device u0 must stay valid.  nodal_out in pageable host memory makes
 * the copy, and so the call, wait for the solve (device or pinned host memory does not).
 * pe_solve_wait without a pending solve: PE_ESTATE.
 */
pe_status pe_solve_async(pe_ctx* ctx, const pe_field* u0, const pe_forcing* f, double tol, double* nodal_out);
pe_status pe_solve_wait(pe_ctx* ctx, pe_result* out);

/* Nodal values u_h(T_slice) = V U^{slice} (slice in 0..N) into nodal_out (host or device, Ndof). */
pe_status pe_get_solution(pe_ctx* ctx, int32_t slice, double* nodal_out);

/* Modal coefficients U^{slice} (slice in 0..N) into modal_out (host or device, Ndof). */
pe_status pe_get_modal(pe_ctx* ctx, int32_t slice, double* modal_out);

/* lam_J into out (host or device, Ndof): lam_J = D sum_a mu^K_a(j_a)/mu^M_a(j_a). */
pe_status pe_get_lambda(pe_ctx* ctx, double* out);

/* Coefficient table of one propagator (which = 0 fine, 1 coarse) into out (host or
 * device, (s+1) x Ndof): row 0 = e^{-lam tau}, row 1+i = tau * b_i(-lam tau). */
pe_status pe_get_coefficients(pe_ctx* ctx, int32_t which, double* out);

/* Modal coefficients of P_h f(t) into out (host or device, Ndof); needs a problem. */
pe_status pe_forcing_modal(pe_ctx* ctx, double t, double* out);

/* Interpolation nodes actually used (which = 0 fine, 1 coarse) into host c_out[s]. */
pe_status pe_get_nodes(pe_ctx* ctx, int32_t which, double* c_out);

/* Parareal state (k, U^0..U^N) to / from a host buffer: resume gives identical results
 * (the correction needs no stored coarse values: G is affine in its argument).
 * pe_save_state with buf == NULL reports the size in *bytes. */
pe_status pe_save_state(pe_ctx* ctx, void* buf, size_t* bytes);
pe_status pe_load_state(pe_ctx* ctx, const void* buf, size_t bytes);

/*
 * pe_dst -- orthonormal tensor DST-I (S_a[k][j] = sqrt(2/(n_a+1)) sin(pi j k/(n_a+1)))
 * applied along every axis of a C-ordered float64 array: out = (kron_a S_a) in.
 * V is symmetric and orthogonal, so the same call is the forward and the inverse
 * transform (Sec. 2.3).  in/out: device, Ndof values, may alias.  d in 1..3.
 * stream: cudaStream_t or NULL.  Scratch (a ping-pong array; the DST-I matrix of axes whose
 * n + 1 is not a power of two) comes stream-ordered from a memory pool the library creates per
 * device, which keeps freed memory for the next call until the process exits.
 */
pe_status pe_dst(int32_t d, const int32_t* n, const double* in, double* out, void* stream);

/* Same transform in float32 (device in/out). */
pe_status pe_dst_f32(int32_t d, const int32_t* n, const float* in, float* out, void* stream);

/*
 * pe_dst_noalloc -- pe_dst for callers that cannot allocate device memory (applications
 * that own a fixed memory pool and forbid the runtime allocator, hosts whose device memory
 * is reserved up front, latency-critical loops that must not enter the allocator, which
 * can synchronise the device).  The
 * paper has no counterpart: this is an interface variant, not a step of the method.
 * It calls no cudaMalloc, cudaFree or other allocating routine; its scratch (ping-pong
 * array, DST-I matrices, FFT twiddles) is one file-scope device array of 1,835,008
 * doubles (about 14.7 MB) that every GPU loading the library holds until the process
 * exits.  Limits: at most 1,048,576 values in total; an axis whose n+1 is not a power
 * of two must have n <= 512.  Larger sizes return PE_EINVAL with a message.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current: make that first call before any stream capture.  The address
 * is kept for the life of the process: do not use this call across a cudaDeviceReset.
 * Every call shares the one array and leaves its contents behind; nothing in it has to
 * start at zero (each call writes what it reads), but calls that overlap on the GPU
 * (different streams, or different host threads on one device) race on it.
 * in/out: device float64, may alias; stream: cudaStream_t or NULL.
 */
pe_status pe_dst_noalloc(int32_t d, const int32_t* n, const double* in, double* out, void* stream);

/* ------------------------------------------------------------------------
 * Batched solver: many independent problems (uneven grids, D, sources and
 * slice counts) advanced together.  Every phase of Algorithm 1 over all
 * problems is one kernel launch whose CTAs pull (problem, slice, mode-tile)
 * work items from a queue; the Parareal iteration (fine sweep, correction,
 * per-problem residuals and stop flags) is captured once as a CUDA graph and
 * replayed; problems whose residual reached tol (or k = N) drop out.  Only
 * separable initial data (PE_FIELD_TERMS_SEPARABLE) is accepted; each
 * problem has at most PE_BATCH_MAX_TERMS forcing terms.
 * ------------------------------------------------------------------------ */
#define PE_BATCH_MAX_TERMS 20
typedef struct pe_batch pe_batch; /* opaque */

typedef struct {
  int32_t d;
  int32_t n[3];
  double box[6];        /* lo0, hi0, lo1, hi1, lo2, hi2 (first 2d used) */
  double D, t0, T;
  int32_t n_slices, n_substeps;
  pe_tableau fine, coarse;
  pe_field u0;
  pe_forcing forcing;
} pe_problem;

typedef struct {
  int32_t graph_replays;      /* Parareal iterations run (graph launches) */
  int32_t max_k;              /* largest per-problem iteration count */
  double max_residual;        /* largest per-problem final relative residual */
  int64_t fine_dof_substeps;  /* sum over problems of Ndof * N * M * (its fine sweeps) */
  double ms_prepare;          /* forcing tables, u0 projection, coarse sweeps (phi/b tables: set-up) */
  double ms_iterations;       /* all graph replays */
  int64_t kernel_launches;    /* kernels launched (graph nodes counted per replay) */
  int32_t threads, ctas_per_sm; /* launch shape of the persistent fine kernel */
} pe_batch_result;

/* Validate and lay out all problems (one arena per array kind), compute their
 * spectra and DST-I-free 1D factor transforms.  opt->precision selects the fine
 * stages (PE_MIXED: float32 stages, float64 tables/correction/residual);
 * opt->fine_engine = PE_FINE_TC (PE_MIXED only) runs the stage contraction of every
 * problem on the tensor cores (work items: problem x slice group x 128-mode tile, one
 * persistent launch per column padding; every problem needs M a multiple of 16 in
 * 16..128, else PE_EINVAL).  problems: host array of n_problems. */
pe_status pe_setup_batch(pe_batch** out, int32_t n_problems, const pe_problem* problems, const pe_options* opt);

/* Pick the persistent fine kernel's launch shape (threads per CTA x CTAs per SM)
 * by timing the candidates on this batch; cache_path (may be NULL) is a text file
 * of previous choices keyed by device and batch signature, read and appended. */
pe_status pe_batch_autotune(pe_batch* b, const char* cache_path);

/* Tables, P_h f, U^0, coarse sweeps, then graph replays of the Parareal iteration
 * until every problem has r <= tol or k = N.  res may be NULL. */
pe_status pe_batch_solve(pe_batch* b, double tol, pe_batch_result* res);

/* Per-problem modal U^{slice} / nodal u_h(T) (host or device out, Ndof of that problem). */
pe_status pe_batch_get_modal(pe_batch* b, int32_t problem, int32_t slice, double* out);
pe_status pe_batch_get_solution(pe_batch* b, int32_t problem, double* nodal_out);

/* Per-problem final relative residuals and iteration counts (host arrays of n_problems; may be NULL). */
pe_status pe_batch_status(pe_batch* b, double* residuals, int32_t* iterations);

void pe_batch_destroy(pe_batch* b);

/* ------------------------------------------------------------------------
 * Learned coarse correction.  F^M(v) - G(v) does not depend on v (G and F share
 * e^{-lam dT}); per mode J and sine source term amp sin(w t + phi) prod_a g_a it is
 * P_{r,J} amp Im(e^{i(w T_n + phi)} K(lam_J, w)) with K the response of F^M - G to
 * the unit source e^{i w t} over one slice.  A 3-layer MLP (2 -> 64 -> 64 -> 2,
 * tanh, float16 weights / float32 accumulation at inference) learns K from
 * features x = (log(lam dT)/6, w dT - 1) and targets K~ = 4 K (1 + lam dT)/(dT (w dT)^2).
 * With a network attached, the coarse step becomes G'(v) = G(v) + delta^ (band
 * table of K^ over log lam, linear interpolation per mode); the correction of
 * Algorithm 1 cancels delta^, so the converged result is unchanged and only the
 * iteration count can change.  Sources of other kinds get no correction.
 * Buffers x, t, y, lam, omega, K are device memory; grad_out, params are host.
 * ------------------------------------------------------------------------ */
typedef struct pe_mlp pe_mlp; /* opaque */

/* New network with Xavier-uniform weights drawn from SplitMix64(seed), zero biases. */
pe_status pe_mlp_create(pe_mlp** out, uint64_t seed);
/* Number of float parameters (W1[64][2], b1, W2[64][64], b2, W3[2][64], b3). */
int32_t pe_mlp_num_params(void);
/* Adam (beta 0.9/0.999, cosine-decayed step lr -> lr/100) on 0.5 |y - t|^2, mean over
 * each batch, `epochs` passes over the n samples in order.  final_loss: mean loss of
 * the trained weights over all samples (host, may be NULL). */
pe_status pe_mlp_train(pe_mlp* m, const float* x, const float* t, int32_t n, int32_t epochs, int32_t batch,
                       float lr, float* final_loss);
/* Gradient of the mean loss over n samples (float32 weights) into host grad_out[num_params]. */
pe_status pe_mlp_gradient(pe_mlp* m, const float* x, const float* t, int32_t n, float* grad_out, float* loss_out);
/* Inference with the float16 weights: y[n][2] = net(x[n][2]). */
pe_status pe_mlp_forward(pe_mlp* m, const float* x, int32_t n, float* y);
pe_status pe_mlp_get_params(pe_mlp* m, float* out);
pe_status pe_mlp_set_params(pe_mlp* m, const float* in);
void pe_mlp_destroy(pe_mlp* m);
/* Training pairs generated by the method: for each (lam_s, w_s), run the fine
 * propagator (M steps, q nodes) and the coarse step of this context on the unit
 * source e^{i w t} and return features x[n][2], normalised targets t[n][2] and the
 * raw K[n][2] (re, im; K may be NULL). */
pe_status pe_learned_samples(pe_ctx* ctx, int32_t n, const double* lam, const double* omega, float* x, float* t,
                             double* K);
/* Attach (m != NULL) or detach the learned correction; takes effect at the next pe_set_problem / pe_solve.
 * The network must outlive its use by the context. */
pe_status pe_set_learned(pe_ctx* ctx, const pe_mlp* m);
/* Attach (m != NULL) or detach the learned coarse correction for every problem of the batch
 * (G'(v) = G(v) + delta^ per problem, as pe_set_learned does for one context; band tables of
 * 2048 log-spaced bands per problem and sine term, the learned term summed inside the batched
 * coarse sweep); takes effect at the next pe_batch_solve.  The network must outlive its use. */
pe_status pe_batch_set_learned(pe_batch* b, const pe_mlp* m);

/*
 * pe_dst_tc -- the same orthonormal tensor DST-I for float32 data on the tensor cores:
 * every axis pass is one bfloat16 GEMM (tcgen05.mma, float32 accumulation in tensor
 * memory, operands staged by TMA) after splitting data and DST matrix into nsplit
 * bfloat16 terms (2: three products, about 1e-5 relative; 3: six products, about
 * 1e-7).  in/out: device float32, Ndof values, may alias; n_a <= 1024.  Allocates its
 * operand buffers with cudaMallocAsync on the stream.  PE_ETIMEOUT if a pipeline wait
 * in the kernel expired (the kernel then skips its output).
 */
pe_status pe_dst_tc(int32_t d, const int32_t* n, const float* in, float* out, int32_t nsplit, void* stream);

/* ------------------------------------------------------------------------
 * Measurement and self-check calls (the paper has no counterpart).
 * ------------------------------------------------------------------------ */

/*
 * pe_measure_fma_peak -- FMA throughput of the CUDA cores in TFLOP/s (2 FLOP per FMA),
 * measured by a kernel of independent FMA chains (8 per thread, 2048 threads per SM), the
 * best of five timed launches after one warm-up: precision PE_FP64 for float64 FMAs,
 * PE_MIXED for float32 FMAs.  The ALU-bound fine kernels are quoted against it beside
 * the peak derived from unit counts and the clock.  tflops_out: host.  Allocates 40 KB
 * with cudaMallocAsync on the stream for the duration of the call.
 */
pe_status pe_measure_fma_peak(int32_t precision, double* tflops_out, void* stream);

/*
 * pe_probe_wait_timeout -- runs the bounded mbarrier wait of the tensor-core kernels
 * on a barrier that nothing arrives at, in a one-warp kernel with no tensor-core
 * instruction and no copy in flight, giving up after budget_cycles SM clock cycles
 * (1..1e8; 2e6 is about a millisecond).  Returns PE_ETIMEOUT (the status the
 * tensor-core kernels report when one of their waits expires) after the kernel has
 * recorded the expiry and returned; the context stays usable.  PE_EINVAL for a budget
 * out of range.  Allocates 4 bytes with cudaMallocAsync for the status word.
 */
pe_status pe_probe_wait_timeout(int64_t budget_cycles, void* stream);

/*
 * pe_probe_widen_f32 -- y[i] = x[i] widened from float32 to float64 by the integer
 * operations the mixed form's coarse sweeps use in place of the conversion instruction
 * (normal values: exponent rebiased, fraction shifted; zero, subnormal, infinite and NaN
 * values as the conversion gives them), for i < n; x (n floats) and y (n doubles) device
 * memory, enqueued on stream.  A self-check of that step: the result equals the hardware
 * conversion bit for bit.  PE_EINVAL for n < 0 or NULL buffers with n > 0.
 */
pe_status pe_probe_widen_f32(const float* x, double* y, int64_t n, void* stream);

/* Most recent error message on this thread ("" if none). */
const char* pe_last_error(void);

void pe_destroy(pe_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PE_H */
