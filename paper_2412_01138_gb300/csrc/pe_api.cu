// Host side of libpe: the C-ABI declared in include/pe.h.
//
// Validates arguments, owns device memory, and sequences the kernels of
// Algorithm 1 (PEIFE-linear): tables -> P_h u0 -> coarse sweep -> loop of
// {fine sweep, correction + residual} -> inverse DST of the last slice.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <new>
#include <string>

#include "pe_internal.h"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

void pe_set_error(const std::string& msg) { g_err = msg; }

pe_status pe_fail(pe_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

pe_status pe_cuda_fail(cudaError_t err, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
  return err == cudaErrorMemoryAllocation ? PE_ENOMEM : PE_ECUDA;
}

extern "C" const char* pe_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// interpolation nodes
// ---------------------------------------------------------------------------
namespace {

// SplitMix64 (Steele, Lea & Flood 2014): counter += golden gamma, two xor-shift-multiply rounds.
uint64_t splitmix64_next(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

const double kMinNodeGap = 1e-3;

}  // namespace

pe_status pe_resolve_nodes(const pe_tableau* tb, const char* name, int* s_out, double* c) {
  if (!tb) return pe_fail(PE_EINVAL, std::string(name) + " tableau is NULL");
  const int s = tb->s;
  if (s < 1 || s > PE_MAX_S) return pe_fail(PE_EINVAL, std::string(name) + " tableau: s must be in 1..8");
  if (tb->random) {
    uint64_t state = tb->seed;
    for (int attempt = 0; attempt < 100000; ++attempt) {
      for (int i = 0; i < s; ++i) c[i] = (double)(splitmix64_next(state) >> 11) * (1.0 / 9007199254740992.0);
      std::sort(c, c + s);
      double gap = 1.0;
      for (int i = 1; i < s; ++i) gap = std::min(gap, c[i] - c[i - 1]);
      if (s == 1 || gap >= kMinNodeGap) {
        *s_out = s;
        return PE_OK;
      }
    }
    return pe_fail(PE_EINVAL, std::string(name) + " tableau: could not draw separated random nodes");
  }
  for (int i = 0; i < s; ++i) c[i] = tb->c ? tb->c[i] : (double)i / (double)s;
  for (int i = 0; i < s; ++i) {
    if (!(c[i] >= 0.0 && c[i] <= 1.0)) return pe_fail(PE_EINVAL, std::string(name) + " tableau: nodes must lie in [0,1]");
    for (int j = 0; j < i; ++j)
      if (c[i] == c[j]) return pe_fail(PE_EINVAL, std::string(name) + " tableau: nodes must be distinct");
  }
  *s_out = s;
  return PE_OK;
}

// a[i][m]: coefficient of theta^m in the Lagrange basis polynomial l_i.
void pe_lagrange_coeffs(int s, const double* c, double a[PE_MAX_S][PE_MAX_S]) {
  for (int i = 0; i < PE_MAX_S; ++i)
    for (int m = 0; m < PE_MAX_S; ++m) a[i][m] = 0.0;
  for (int i = 0; i < s; ++i) {
    double poly[PE_MAX_S + 1] = {1.0};
    int deg = 0;
    for (int m = 0; m < s; ++m) {
      if (m == i) continue;
      const double den = c[i] - c[m];
      double nxt[PE_MAX_S + 1] = {0.0};
      for (int k = 0; k <= deg; ++k) {
        nxt[k + 1] += poly[k] / den;
        nxt[k] -= poly[k] * c[m] / den;
      }
      ++deg;
      for (int k = 0; k <= deg; ++k) poly[k] = nxt[k];
    }
    for (int k = 0; k < s; ++k) a[i][k] = poly[k];
  }
}

bool pe_is_device_ptr(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

namespace {

template <typename T>
pe_status dev_alloc(T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return pe_fail(PE_ENOMEM, "cudaMalloc of " + std::to_string(sizeof(T) * count) + " bytes failed");
  }
  return PE_OK;
}

void free_ctx(pe_ctx* c) {
  if (!c) return;
  void* ptrs[] = {c->muM_axis, c->ratio_axis, c->S[0], c->S[1], c->S[2], c->S32[0], c->S32[1], c->S32[2],
                  c->gen_L, c->gen_buf, c->gen_tmp, c->lam, c->coefF, c->coefG,
                  c->coefF32, c->U, c->Fbar, c->gG, c->work0, c->work1, c->out_nodal, c->partials,
                  c->red, c->axisF, c->axisF32, c->axisU0, c->AF, c->AF32, c->AG, c->AG32, c->loads,
                  c->Ktab, c->phase_tab, c->Zst, c->Wst, c->Wst32, c->Fz, c->done_ctr, c->tcB, c->tc_err, c->tcA,
                  c->muM_full, c->ratio_full, c->fac_full, c->work2, c->loopctl, c->loop_hist, c->io32, c->muM_inv};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_red) cudaFreeHost(c->h_red);
  if (c->h_loop) cudaFreeHost(c->h_loop);
  if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
  if (c->setup_exec) cudaGraphExecDestroy(c->setup_exec);
  if (c->out_exec) cudaGraphExecDestroy(c->out_exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (int i = 0; i < PE_NEV; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_tables) cudaEventDestroy(c->ev_tables);
  if (c->side) cudaStreamDestroy(c->side);
  delete c;
}

pe_status copy_out(pe_ctx* c, const double* src_dev, double* out, size_t count) {
  if (!out) return pe_fail(PE_EINVAL, "output pointer is NULL");
  const bool dev = pe_is_device_ptr(out);
  PE_CUDA_TRY(cudaMemcpyAsync(out, src_dev, sizeof(double) * count,
                              dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  PE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PE_OK;
}

}  // namespace

pe_status pe_validate_terms(int n, const pe_term* t, int d, const char* what, bool allow_moving) {
  if (n < 0 || n > PE_MAX_TERMS) return pe_fail(PE_EINVAL, std::string(what) + ": n_terms must be in 0..32");
  if (n > 0 && !t) return pe_fail(PE_EINVAL, std::string(what) + ": terms is NULL");
  for (int i = 0; i < n; ++i) {
    if (t[i].tkind != PE_T_EXP && t[i].tkind != PE_T_SIN)
      return pe_fail(PE_EINVAL, std::string(what) + ": unknown time factor kind");
    for (int a = 0; a < d; ++a) {
      const int k = t[i].skind[a];
      if (k == PE_S_MOVING_HAT && !allow_moving)
        return pe_fail(PE_EINVAL, std::string(what) + ": moving factors need PE_FORCING_GENERAL");
      if (k == PE_S_MOVING_HAT && !(t[i].sp[a][3] > 0.0))
        return pe_fail(PE_EINVAL, std::string(what) + ": moving hat half-width must be positive");
      if (k < PE_S_ONE || k > PE_S_MOVING_HAT) return pe_fail(PE_EINVAL, std::string(what) + ": unknown spatial kind");
      if (k == PE_S_GAUSS && !(t[i].sp[a][1] != 0.0))
        return pe_fail(PE_EINVAL, std::string(what) + ": Gaussian width must be nonzero");
    }
  }
  return PE_OK;
}

namespace {

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

}  // namespace

// ---------------------------------------------------------------------------
// setup / destroy
// ---------------------------------------------------------------------------
extern "C" pe_status pe_setup(pe_ctx** out, int32_t d, const int32_t* n, const double* box, double D, double t0,
                              double T, int32_t n_slices, int32_t n_substeps, const pe_tableau* fine,
                              const pe_tableau* coarse, const pe_options* opt) {
  if (!out) return pe_fail(PE_EINVAL, "pe_setup: out is NULL");
  *out = nullptr;
  if (d < 1 || d > PE_MAX_D) return pe_fail(PE_EINVAL, "pe_setup: d must be 1, 2 or 3");
  if (!n || !box) return pe_fail(PE_EINVAL, "pe_setup: n or box is NULL");
  if (!(D > 0.0) || !isfinite(D)) return pe_fail(PE_EINVAL, "pe_setup: D must be positive");
  if (!(T > 0.0) || !isfinite(T) || !isfinite(t0)) return pe_fail(PE_EINVAL, "pe_setup: T must be positive");
  if (n_slices < 1 || n_substeps < 1) return pe_fail(PE_EINVAL, "pe_setup: n_slices and n_substeps must be >= 1");
  if (n_slices > 65535) return pe_fail(PE_EINVAL, "pe_setup: n_slices must be <= 65535");
  int64_t ndof = 1;
  int nsum = 0;
  for (int a = 0; a < d; ++a) {
    if (n[a] < 1 || n[a] > 16384) return pe_fail(PE_EINVAL, "pe_setup: n_a must be in 1..16384");
    if (!(box[2 * a + 1] > box[2 * a])) return pe_fail(PE_EINVAL, "pe_setup: box needs lo < hi on every axis");
    ndof *= n[a];
    nsum += n[a];
  }
  if (ndof > ((int64_t)1 << 31)) return pe_fail(PE_EINVAL, "pe_setup: too many degrees of freedom");

  pe_ctx* c = new (std::nothrow) pe_ctx();
  if (!c) return pe_fail(PE_ENOMEM, "pe_setup: host allocation failed");
  for (int i = 0; i < PE_NEV; ++i) c->ev[i] = nullptr;
  c->g.d = d;
  c->g.ndof = ndof;
  c->nsum = nsum;
  int off = 0;
  for (int a = 0; a < PE_MAX_D; ++a) {
    c->g.n[a] = a < d ? n[a] : 1;
    c->g.off[a] = off;
    if (a < d) {
      c->lo[a] = box[2 * a];
      c->hi[a] = box[2 * a + 1];
      c->h[a] = (c->hi[a] - c->lo[a]) / (double)(n[a] + 1);
      off += n[a];
    } else {
      c->lo[a] = 0.0; c->hi[a] = 1.0; c->h[a] = 1.0;
    }
  }
  c->D = D; c->t0 = t0; c->T = T;
  c->N = n_slices; c->M = n_substeps;
  c->dT = T / (double)n_slices;
  c->dt = c->dT / (double)n_substeps;
  pe_status st = pe_resolve_nodes(fine, "fine", &c->q, c->cF);
  if (st == PE_OK) st = pe_resolve_nodes(coarse, "coarse", &c->p, c->cG);
  if (st != PE_OK) { delete c; return st; }
  pe_lagrange_coeffs(c->q, c->cF, c->lagF);
  pe_lagrange_coeffs(c->p, c->cG, c->lagG);
  pe_options o{};
  if (opt) o = *opt;
  if (o.precision != PE_FP64 && o.precision != PE_MIXED) { delete c; return pe_fail(PE_EINVAL, "pe_setup: bad precision"); }
  if (o.quad_pts == 0) o.quad_pts = 3;
  if (o.quad_pts < 1 || o.quad_pts > 8) { delete c; return pe_fail(PE_EINVAL, "pe_setup: quad_pts must be in 1..8"); }
  if (o.max_iter < 0) { delete c; return pe_fail(PE_EINVAL, "pe_setup: max_iter must be >= 0"); }
  if (o.forcing_path != PE_FORCING_SEPARABLE && o.forcing_path != PE_FORCING_GENERAL) {
    delete c;
    return pe_fail(PE_EINVAL, "pe_setup: bad forcing_path");
  }
  if (o.periodic_mask < 0 || o.periodic_mask >= (1 << d)) {
    delete c;
    return pe_fail(PE_EINVAL, "pe_setup: periodic_mask has bits beyond the problem's axes");
  }
  for (int a = 0; a < PE_MAX_D; ++a) {
    c->g.per[a] = a < d ? ((o.periodic_mask >> a) & 1) : 0;
    if (c->g.per[a]) c->h[a] = (c->hi[a] - c->lo[a]) / (double)n[a];  // n nodes, node n is node 0
  }
  if (o.cache_forced && o.forcing_path == PE_FORCING_GENERAL) {
    delete c;
    return pe_fail(PE_EINVAL, "pe_setup: cache_forced needs PE_FORCING_SEPARABLE");
  }
  if (o.fine_engine != PE_FINE_SIMT && o.fine_engine != PE_FINE_TC) {
    delete c;
    return pe_fail(PE_EINVAL, "pe_setup: bad fine_engine");
  }
  if (o.fine_engine == PE_FINE_TC &&
      (o.precision != PE_MIXED || o.forcing_path != PE_FORCING_SEPARABLE || !fine_tc_supported(n_substeps))) {
    delete c;
    return pe_fail(PE_EINVAL,
                   "pe_setup: PE_FINE_TC needs PE_MIXED, PE_FORCING_SEPARABLE and M a multiple of 16 in 16..128");
  }
  // mode sharding: this context owns the axis-0 modes [mode_begin, mode_end)
  c->gn = c->g;
  c->nsum_full = nsum;
  if (!(o.mode_begin == 0 && o.mode_end == 0) && !(o.mode_begin == 0 && o.mode_end == n[0])) {
    if (o.mode_begin < 0 || o.mode_end <= o.mode_begin || o.mode_end > n[0]) {
      delete c;
      return pe_fail(PE_EINVAL, "pe_setup: mode range must satisfy 0 <= mode_begin < mode_end <= n_0");
    }
    if (o.forcing_path != PE_FORCING_SEPARABLE) {
      delete c;
      return pe_fail(PE_EINVAL, "pe_setup: a context that owns a block of modes needs PE_FORCING_SEPARABLE");
    }
    c->sharded = true;
    c->base0 = o.mode_begin;
    c->g.n[0] = o.mode_end - o.mode_begin;
    c->g.ndof = ndof / n[0] * c->g.n[0];
    int offl = 0;
    for (int a = 0; a < d; ++a) {
      c->g.off[a] = offl;
      offl += c->g.n[a];
    }
    c->nsum = offl;
  }
  c->reduce = o.residual_reduce;
  c->reduce_user = o.residual_reduce_user;
  if (o.device_loop < 0 || o.device_loop > 2) {
    delete c;
    return pe_fail(PE_EINVAL, "pe_setup: device_loop must be 0, 1 or 2");
  }
  c->device_loop = o.device_loop;
  c->fine_engine = o.fine_engine;
  c->forcing_path = o.forcing_path;
  c->cache_forced = o.cache_forced ? 1 : 0;
  c->precision = o.precision;
  c->dst_backend = o.dst_backend;
  c->quad_pts = o.quad_pts;
  c->max_iter = o.max_iter == 0 ? n_slices : std::min(o.max_iter, n_slices);
  c->stream = (cudaStream_t)o.cuda_stream;

  const int threads = 256;
  // modal arrays hold this context's modes (nd); nodal arrays and per-axis loads the whole grid
  const size_t N = (size_t)n_slices, nd = (size_t)c->g.ndof, ndn = (size_t)ndof, MT = PE_MAX_TERMS;
  const int nsl = c->nsum;
  // CTAs of the one-thread-per-mode kernels: at most one per 64 modes (per_mode_block)
  c->max_blocks = (int)((nd + 63) / 64) + 1;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      c->sms = 0;
    }
  }
  st = PE_OK;
  if (st == PE_OK) st = dev_alloc(&c->muM_axis, nsl);
  if (st == PE_OK) st = dev_alloc(&c->muM_inv, nsum);
  if (st == PE_OK) st = dev_alloc(&c->ratio_axis, nsl);
  if (st == PE_OK && c->sharded) st = dev_alloc(&c->muM_full, nsum);
  if (st == PE_OK && c->sharded) st = dev_alloc(&c->ratio_full, nsum);
  if (st == PE_OK && c->sharded) st = dev_alloc(&c->fac_full, MT * nsum);
  if (st == PE_OK && c->sharded) st = dev_alloc(&c->work2, ndn);
  for (int a = 0; a < d && st == PE_OK; ++a) st = dev_alloc(&c->S[a], (size_t)n[a] * n[a]);
  if (st == PE_OK) st = dev_alloc(&c->lam, nd);
  if (st == PE_OK) st = dev_alloc(&c->coefF, (size_t)(c->q + 2) * nd);
  if (st == PE_OK) st = dev_alloc(&c->coefG, (size_t)(c->p + 1) * nd);
  if (st == PE_OK && c->precision == PE_MIXED) st = dev_alloc(&c->coefF32, (size_t)(c->q + 2) * nd);
  if (st == PE_OK) st = dev_alloc(&c->U, (N + 1) * nd);
  if (st == PE_OK) st = dev_alloc(&c->Fbar, N * nd);
  if (st == PE_OK && c->cache_forced) st = dev_alloc(&c->Fz, N * nd);
  if (st == PE_OK) st = dev_alloc(&c->gG, N * nd);
  if (st == PE_OK) st = dev_alloc(&c->work0, ndn + 64);
  if (st == PE_OK) st = dev_alloc(&c->work1, ndn + 64);
  // the mixed form transforms u0 and the solution in float32 (grids of at least 4096 nodes whose
  // axes all have FFT forms; below that the float64 transform is cheaper than the two conversions)
  if (st == PE_OK && o.precision == PE_MIXED && ndn >= 4096 && dst_nd_f32_ok(c->gn))
    st = dev_alloc(&c->io32, 3 * ndn + 64);
  if (st == PE_OK) st = dev_alloc(&c->out_nodal, ndn);
  if (st == PE_OK) st = dev_alloc(&c->partials, 2 * (size_t)c->max_blocks + 64);
  if (st == PE_OK) st = dev_alloc(&c->red, 2);
  if (st == PE_OK) st = dev_alloc(&c->done_ctr, 1);
  if (st == PE_OK && c->fine_engine == PE_FINE_TC) {
    st = dev_alloc(&c->tcB, fine_tc_buffer_bytes(n_substeps, n_slices));
    if (st == PE_OK) st = dev_alloc(&c->tc_err, 1);
    if (st == PE_OK && cudaMemset(c->tc_err, 0, sizeof(int)) != cudaSuccess)
      st = pe_fail(PE_ECUDA, "pe_setup: error flag initialisation failed");
  }
  if (st == PE_OK && cudaMemset(c->done_ctr, 0, sizeof(unsigned int)) != cudaSuccess)
    st = pe_fail(PE_ECUDA, "pe_setup: counter initialisation failed");
  if (st == PE_OK) st = dev_alloc(&c->axisF, MT * nsl);
  if (st == PE_OK && c->precision == PE_MIXED) st = dev_alloc(&c->axisF32, MT * nsl);
  if (st == PE_OK) st = dev_alloc(&c->axisU0, MT * nsl);
  if (st == PE_OK) st = dev_alloc(&c->loads, MT * nsum);
  if (st == PE_OK) st = dev_alloc(&c->AF, N * n_substeps * 2 * MT);
  if (st == PE_OK && c->precision == PE_MIXED) st = dev_alloc(&c->AF32, N * n_substeps * 2 * MT);
  if (st == PE_OK) st = dev_alloc(&c->Zst, (size_t)PE_MAX_S * 2 * MT);
  if (st == PE_OK) st = dev_alloc(&c->AG, N * c->p * MT);
  if (st == PE_OK && c->precision == PE_MIXED) st = dev_alloc(&c->AG32, N * c->p * MT);
  if (st == PE_OK && c->forcing_path == PE_FORCING_GENERAL &&
      ((int64_t)n_substeps * c->q > 65535 || (int64_t)n_slices * c->p > 65535))
    st = pe_fail(PE_EINVAL, "pe_setup: general forcing path needs M*q and N*p <= 65535");
  if (st == PE_OK && c->forcing_path == PE_FORCING_GENERAL) {
    // stage-time buffers of one chunk of slices (also holding the N*p coarse stage times)
    const int chunk = general_slices_per_chunk(c);
    const size_t stages = std::max((size_t)chunk * n_substeps * c->q, N * c->p);
    st = dev_alloc(&c->gen_buf, stages * nd);
    if (st == PE_OK) st = dev_alloc(&c->gen_tmp, stages * nd);
    if (st == PE_OK) st = dev_alloc(&c->gen_L, stages * MT * nsum);
    for (int a = 0; a < d && st == PE_OK && c->precision == PE_MIXED; ++a)
      st = dev_alloc(&c->S32[a], (size_t)n[a] * n[a]);
  }
  if (st == PE_OK && cudaMallocHost((void**)&c->h_red, 4 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    st = pe_fail(PE_ENOMEM, "pe_setup: pinned host allocation failed");
  }
  if (st == PE_OK && c->device_loop == 2 &&
      cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    st = pe_cuda_fail(cudaGetLastError(), "pe_setup: capture stream");
  if (st == PE_OK && c->device_loop) {
    st = dev_alloc(&c->loopctl, 1);
    if (st == PE_OK) st = dev_alloc(&c->loop_hist, N);
    if (st == PE_OK && (cudaHostAlloc((void**)&c->h_loop, sizeof(LoopCtl), cudaHostAllocMapped) != cudaSuccess ||
                        cudaHostGetDevicePointer((void**)&c->h_loop_dev, c->h_loop, 0) != cudaSuccess)) {
      cudaGetLastError();
      st = pe_fail(PE_ENOMEM, "pe_setup: mapped pinned host allocation failed");
    }
  }
  for (int i = 0; i < PE_NEV && st == PE_OK; ++i)
    if (cudaEventCreate(&c->ev[i]) != cudaSuccess) st = pe_cuda_fail(cudaGetLastError(), "cudaEventCreate");
  if (st == PE_OK && (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
                      cudaEventCreateWithFlags(&c->ev_tables, cudaEventDisableTiming) != cudaSuccess))
    st = pe_cuda_fail(cudaGetLastError(), "pe_setup: side stream");
  if (st == PE_OK) st = launch_axis_tables(c);
  for (int a = 0; a < d && st == PE_OK; ++a) st = build_dst_matrix(n[a], c->S[a], c->stream, c->g.per[a]);
  for (int a = 0; a < d && st == PE_OK; ++a)
    if (c->S32[a]) st = build_dst_matrix_f32(n[a], c->S32[a], c->stream, c->g.per[a]);
  if (st == PE_OK) st = launch_coef_tables(c);
  if (st == PE_OK) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = pe_cuda_fail(e, "pe_setup");
  }
  if (st != PE_OK) {
    free_ctx(c);
    return st;
  }
  *out = c;
  return PE_OK;
}

extern "C" void pe_destroy(pe_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

// ---------------------------------------------------------------------------
// non-homogeneous Dirichlet data by lifting
//
// Data g(t, x) = sum_s A_s theta_s(t) prod_a gamma_{s,a}(x_a) on the closed box; the lifting
// is the Q1 interpolant I_h g on all nodes and the solver integrates w = u_h - I_h g, which
// vanishes on the boundary.  Testing with the interior hat functions adds the load
//   r_i = -(M_full d/dt I_h g + K_full I_h g)_i,
// a sum of separable terms whose per-axis 1D vectors are interior rows of the full-grid
// 1D mass and stiffness matrices applied to gamma's nodal values (load kinds 1 and 2): per
// data term one mass term with time factor -A theta' and d stiffness terms -A D theta.
// ---------------------------------------------------------------------------
static double time_factor(const pe_term& t, double tt) {
  return t.tkind == PE_T_SIN ? sin(t.tp[0] * tt + t.tp[1]) : exp(t.tp[0] * tt);
}

static pe_status expand_dirichlet_terms(pe_ctx* c) {
  const int d = c->g.d;
  for (int s = 0; s < c->nbd; ++s) {
    const pe_term& b = c->bterms[s];
    if (c->R + 1 + d > PE_MAX_TERMS)
      return pe_fail(PE_EINVAL, "pe_set_problem: forcing plus Dirichlet terms exceed 32 (each data term adds 1 + d)");
    // mass term: time factor d/dt theta (exp(a t) -> a exp(a t); sin(w t + phi) -> w sin(w t + phi + pi/2))
    pe_term m = b;
    if (b.tkind == PE_T_SIN) {
      m.amp = -b.amp * b.tp[0];
      m.tp[1] = b.tp[1] + 0.5 * M_PI;
    } else {
      m.amp = -b.amp * b.tp[0];
    }
    if (m.amp != 0.0) {
      c->terms[c->R] = m;
      for (int a = 0; a < d; ++a) c->lkind[c->R][a] = 1;
      c->R += 1;
    }
    for (int a = 0; a < d; ++a) {
      pe_term k = b;
      k.amp = -b.amp * c->D;
      c->terms[c->R] = k;
      for (int e = 0; e < d; ++e) c->lkind[c->R][e] = e == a ? 2 : 1;
      c->R += 1;
    }
  }
  if (c->R == 0) {  // data only through terms that vanished: keep one zero term
    c->R = 1;
    memset(&c->terms[0], 0, sizeof(pe_term));
  }
  return PE_OK;
}

// out += sign * I_h g(t) in one of three forms: kind 1 the modal P_h of the interpolant,
// kind 2 the modal V^T of its interior values, kind 3 its interior nodal values.
static pe_status add_lift(pe_ctx* c, double t, double sign, int kind, double* out) {
  if (c->nbd == 0) return PE_OK;
  pe_term tt[PE_MAX_TERMS];
  signed char lk[PE_MAX_TERMS][PE_MAX_D] = {};
  for (int s = 0; s < c->nbd; ++s) {
    tt[s] = c->bterms[s];
    tt[s].amp = sign * c->bterms[s].amp * time_factor(c->bterms[s], t);
    for (int a = 0; a < c->g.d; ++a) lk[s][a] = kind == 1 ? 1 : 3;
  }
  const int mode = kind == 1 ? 1 : (kind == 2 ? 2 : 0);
  PE_TRY(launch_separable_factors(c, tt, c->nbd, c->axisU0, mode, lk));
  return launch_outer_sum(c, c->axisU0, tt, c->nbd, out, 1);
}

// The set-up and output graphs of a repeated problem (pe_options.device_loop = 2) hold the host
// state of the solve that captured them; every call that changes that state drops them.
void drop_solve_graphs(pe_ctx* c) {
  if (c->setup_exec) cudaGraphExecDestroy(c->setup_exec);
  if (c->out_exec) cudaGraphExecDestroy(c->out_exec);
  c->setup_exec = c->out_exec = nullptr;
  c->graph_key = 0;
  c->graph_key_seen = 0;
}

extern "C" pe_status pe_set_dirichlet(pe_ctx* c, int32_t n_terms, const pe_term* g) {
  if (c && c->pend) return pe_fail(PE_ESTATE, "pe_set_dirichlet: a solve is pending (pe_solve_wait first)");
  if (!c) return pe_fail(PE_EINVAL, "pe_set_dirichlet: ctx is NULL");
  if (n_terms < 0 || n_terms > PE_MAX_TERMS) return pe_fail(PE_EINVAL, "pe_set_dirichlet: n_terms out of range");
  if (n_terms > 0 && !g) return pe_fail(PE_EINVAL, "pe_set_dirichlet: terms is NULL");
  PE_TRY(pe_validate_terms(n_terms, g, c->g.d, "Dirichlet data"));
  if (n_terms > 0 && c->forcing_path == PE_FORCING_GENERAL)
    return pe_fail(PE_EINVAL, "pe_set_dirichlet: Dirichlet data need PE_FORCING_SEPARABLE");
  drop_solve_graphs(c);
  if (n_terms > 0 && (c->g.per[0] || c->g.per[1] || c->g.per[2]))
    return pe_fail(PE_EINVAL, "pe_set_dirichlet: Dirichlet data with periodic axes");
  if (n_terms > 0 && c->sharded)
    return pe_fail(PE_EINVAL, "pe_set_dirichlet: Dirichlet data in a context that owns a block of modes");
  c->nbd = n_terms;
  for (int i = 0; i < n_terms; ++i) c->bterms[i] = g[i];
  c->have_problem = false;  // the next pe_set_problem / pe_solve takes the data into account
  return PE_OK;
}

// ---------------------------------------------------------------------------
// nodal <-> modal for the modes this context owns.  A sharded context owns the axis-0 modes
// [base0, base0 + g.n[0]): a contiguous block of the whole grid's modal array starting at
// base0 * (the product of the other axes' sizes).
// ---------------------------------------------------------------------------
static int64_t slab_offset(const pe_ctx* c) { return (int64_t)c->base0 * (c->gn.ndof / c->gn.n[0]); }

// modal_out = this context's modes of V^T nodal (nodal: whole grid, device; not work1 / work2)
// the whole grid's transform: float32 arithmetic in the mixed form (where every axis has an FFT
// form), float64 otherwise
static pe_status dst_whole(pe_ctx* c, const double* in, double* out) {
  return c->io32 ? dst_nd_mixed(c, in, out) : dst_nd_f64(c, in, out);
}

static pe_status nodal_to_modal(pe_ctx* c, const double* nodal, double* modal_out) {
  if (!c->sharded) return dst_whole(c, nodal, modal_out);
  PE_TRY(dst_whole(c, nodal, c->work2));
  PE_CUDA_TRY(cudaMemcpyAsync(modal_out, c->work2 + slab_offset(c), sizeof(double) * c->g.ndof,
                              cudaMemcpyDeviceToDevice, c->stream));
  return PE_OK;
}

// nodal_out (whole grid, device; not work1 / work2) = V applied to this context's modes, the
// other modes taken as zero
static pe_status modal_to_nodal(pe_ctx* c, const double* modal, double* nodal_out) {
  if (!c->sharded) return dst_whole(c, modal, nodal_out);
  PE_CUDA_TRY(cudaMemsetAsync(c->work2, 0, sizeof(double) * c->gn.ndof, c->stream));
  PE_CUDA_TRY(cudaMemcpyAsync(c->work2 + slab_offset(c), modal, sizeof(double) * c->g.ndof,
                              cudaMemcpyDeviceToDevice, c->stream));
  return dst_whole(c, c->work2, nodal_out);
}

// ---------------------------------------------------------------------------
// problem, iteration, solve
// ---------------------------------------------------------------------------
// grids below this many nodes run pe_set_problem on one stream (their kernels are launch-bound)
constexpr int64_t kForkMinDof = 4096;

// A timing event on the context's stream; inside a captured phase it becomes an event-record node
// of the graph, so that its replays record it too.
static cudaError_t record_timing(pe_ctx* c, cudaEvent_t e) {
  return cudaEventRecordWithFlags(e, c->stream, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
}

static pe_status set_problem_impl(pe_ctx* c, const pe_field* u0, const pe_forcing* f) {
  if (!u0) return pe_fail(PE_EINVAL, "pe_set_problem: u0 is NULL");
  const int nf = f ? f->n_terms : 0;
  const bool general = c->forcing_path == PE_FORCING_GENERAL;
  PE_TRY(pe_validate_terms(nf, f ? f->terms : nullptr, c->g.d, "forcing", general));
  if (general && c->mlp) return pe_fail(PE_EINVAL, "pe_set_problem: the learned correction needs PE_FORCING_SEPARABLE");
  if (c->nbd > 0 && general) return pe_fail(PE_EINVAL, "pe_set_problem: Dirichlet data need PE_FORCING_SEPARABLE");
  if (c->nbd > 0 && c->mlp) return pe_fail(PE_EINVAL, "pe_set_problem: Dirichlet data and the learned correction");
  const bool any_periodic = c->g.per[0] || c->g.per[1] || c->g.per[2];
  if (any_periodic && c->mlp) return pe_fail(PE_EINVAL, "pe_set_problem: periodic axes and the learned correction");
  if (c->sharded && u0->kind == PE_FIELD_TERMS_QUADRATURE)
    return pe_fail(PE_EINVAL, "pe_set_problem: a context that owns a block of modes takes nodal or separable u0");
  memset(c->lkind, 0, sizeof(c->lkind));
  c->tc_split_ok = false;
  if (nf == 0 && c->nbd == 0) {
    // no source: one zero term keeps every kernel shape valid
    c->R = 1;
    memset(&c->terms[0], 0, sizeof(pe_term));
  } else {
    c->R = nf;
    for (int i = 0; i < nf; ++i) c->terms[i] = f->terms[i];
    PE_TRY(expand_dirichlet_terms(c));
  }
  // Two streams for grids large enough that their set-up kernels run side by side: the side
  // stream makes the time tables, then the forward transform of nodal u0 (after its copy, for
  // host u0), then the tensor-core engine's split time factors; the main stream makes the
  // per-axis forcing factors, waits for the time tables (the stage weights take their shifts
  // Z), makes the stage weights, and waits for the side stream before the coarse sweep.
  // (Small grids, whose kernels are launch-bound, keep everything on the main stream.)
  double* U0 = c->U;
  const bool fork_u0 = u0->kind == PE_FIELD_NODAL && u0->nodal != nullptr;
  const bool fork = fork_u0 && c->gn.ndof >= kForkMinDof;
  const bool inline_u0 = fork_u0 && !fork;  // nodal u0, transformed below on the main stream
  const bool tc = !general && c->precision == PE_MIXED && c->fine_engine == PE_FINE_TC;
  if (fork) {
    PE_CUDA_TRY(cudaEventRecord(c->ev_fork, c->stream));
    PE_CUDA_TRY(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    cudaStream_t main_stream = c->stream;
    c->stream = c->side;
    pe_status st = PE_OK;
    if (!general) {
      st = launch_time_tables(c);
      if (st == PE_OK && cudaEventRecord(c->ev_tables, c->side) != cudaSuccess)
        st = pe_cuda_fail(cudaGetLastError(), "pe_set_problem: event record");
    }
    if (st == PE_OK) {
      // device u0 is read in place by the transform; host u0 is copied in first
      const bool dev = c->u0_dev_hint >= 0 ? c->u0_dev_hint == 1 : pe_is_device_ptr(u0->nodal);
      const double* src = static_cast<const double*>(u0->nodal);
      if (!dev) {
        const cudaError_t e = cudaMemcpyAsync(c->work0, u0->nodal, sizeof(double) * c->gn.ndof,
                                              cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) st = pe_cuda_fail(e, "pe_set_problem: u0 copy");
        src = c->work0;
      }
      if (st == PE_OK) st = nodal_to_modal(c, src, U0);
    }
    if (st == PE_OK && tc) st = fine_tc_prepare_time(c);
    c->stream = main_stream;
    PE_TRY(st);
    PE_CUDA_TRY(cudaEventRecord(c->ev_join, c->side));
  } else if (!general) {
    PE_TRY(launch_time_tables(c));
  }
  // The phi/b coefficient tables depend only on lam, dt, dT and the nodes: pe_setup made them.
  // Forcing: per-axis modal factors, then the stage weights of the fine step.
  if (!general) PE_TRY(launch_separable_factors(c, c->terms, c->R, c->axisF, 1, c->lkind));
  if (fork && !general) PE_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->ev_tables, 0));
  if (!general) PE_TRY(launch_stage_weights(c));
  // the tensor-core engine's split operand images of the stage weights and time factors
  if (tc) PE_TRY(fine_tc_prepare_weights(c));
  if (tc && !fork) PE_TRY(fine_tc_prepare_time(c));
  if (fork) PE_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  if (tc) c->tc_split_ok = true;
  PE_CUDA_TRY(record_timing(c, c->ev[1]));
  // U^0 = P_h u0
  if (fork_u0 && !inline_u0) {
    // made on the side stream above
  } else if (u0->kind == PE_FIELD_TERMS_SEPARABLE || u0->kind == PE_FIELD_TERMS_QUADRATURE) {
    PE_TRY(pe_validate_terms(u0->n_terms, u0->terms, c->g.d, "u0"));
    if (u0->n_terms == 0) {
      PE_CUDA_TRY(cudaMemsetAsync(U0, 0, sizeof(double) * c->g.ndof, c->stream));
    } else if (u0->kind == PE_FIELD_TERMS_SEPARABLE) {
      PE_TRY(launch_separable_factors(c, u0->terms, u0->n_terms, c->axisU0, 1));
      PE_TRY(launch_outer_sum(c, c->axisU0, u0->terms, u0->n_terms, U0, 0));
    } else {
      // nodal consistent load F = sum_t amp_t kron_a F_{t,a}, then c0 = Lambda_M^{-1} V^T F
      PE_TRY(launch_separable_factors(c, u0->terms, u0->n_terms, c->axisU0, 0));
      PE_TRY(launch_outer_sum(c, c->axisU0, u0->terms, u0->n_terms, c->work0, 0));
      PE_TRY(dst_nd_f64(c, c->work0, U0));
      PE_TRY(launch_scale_by_muM(c, U0, 1));
    }
  } else if (u0->kind == PE_FIELD_NODAL) {
    if (!u0->nodal) return pe_fail(PE_EINVAL, "pe_set_problem: nodal u0 is NULL");
    const bool dev = c->u0_dev_hint >= 0 ? c->u0_dev_hint == 1 : pe_is_device_ptr(u0->nodal);
    PE_CUDA_TRY(cudaMemcpyAsync(c->work0, u0->nodal, sizeof(double) * c->gn.ndof,
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    PE_TRY(nodal_to_modal(c, c->work0, U0));
  } else {
    return pe_fail(PE_EINVAL, "pe_set_problem: unknown u0 kind");
  }
  // Dirichlet lifting: w(t0) = P_h(u0 - I_h g(t0)) for descriptor data, u0 - I_h g(t0) for
  // nodal data (taken as already in V_h)
  if (c->nbd > 0) {
    const bool nodal = u0->kind == PE_FIELD_NODAL;
    PE_TRY(add_lift(c, c->t0, -1.0, nodal ? 2 : 1, U0));
  }
  // k = 0: coarse sweep
  PE_CUDA_TRY(record_timing(c, c->ev[8]));
  PE_TRY(launch_coarse_sweep(c));
  PE_CUDA_TRY(record_timing(c, c->ev[9]));
  c->fz_prec = -1;
  c->k = 0;
  c->have_problem = true;
  c->have_output = false;
  return PE_OK;
}

extern "C" pe_status pe_set_problem(pe_ctx* c, const pe_field* u0, const pe_forcing* f) {
  if (c && c->pend) return pe_fail(PE_ESTATE, "pe_set_problem: a solve is pending (pe_solve_wait first)");
  if (!c) return pe_fail(PE_EINVAL, "pe_set_problem: ctx is NULL");
  c->have_problem = false;
  drop_solve_graphs(c);
  PE_CUDA_TRY(cudaEventRecord(c->ev[0], c->stream));
  PE_TRY(set_problem_impl(c, u0, f));
  PE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return PE_OK;
}

// One pass of Algorithm 1's loop.  sums_out (may be NULL): this context's two residual sums;
// r_out (may be NULL): the relative residual of the totals (after residual_reduce, if any).
static pe_status iter_impl(pe_ctx* c, double* r_out, int precision, double* sums_out = nullptr) {
  PE_CUDA_TRY(cudaEventRecord(c->ev[5], c->stream));
  if (c->forcing_path == PE_FORCING_GENERAL) PE_TRY(launch_general_fine_sweep(c, precision));
  else PE_TRY(launch_fine_sweep(c, precision));
  PE_CUDA_TRY(cudaEventRecord(c->ev[6], c->stream));
  double num = 0.0, den = 0.0;
  PE_TRY(launch_correction(c, &num, &den, c->ev[7]));  // synchronises the stream
  c->ms_fine += elapsed(c->ev[5], c->ev[6]);
  c->ms_corr += elapsed(c->ev[6], c->ev[7]);
  c->k += 1;
  if (sums_out) {
    sums_out[0] = num;
    sums_out[1] = den;
  }
  if (!isfinite(num) || !isfinite(den)) {
    c->have_problem = false;
    if (precision == PE_MIXED && c->fine_engine == PE_FINE_TC) PE_TRY(fine_tc_status(c));
    return pe_fail(PE_ENONFINITE, "Parareal residual is not finite (NaN/Inf in the iterate)");
  }
  if (r_out) {
    if (c->reduce) {
      double tot[2] = {num, den};
      c->reduce(tot, c->reduce_user);
      num = tot[0];
      den = tot[1];
      if (!isfinite(num) || !isfinite(den))
        return pe_fail(PE_ENONFINITE, "Parareal residual is not finite after the combination across contexts");
    }
    *r_out = den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
  }
  return PE_OK;
}

static pe_status need_totals(const pe_ctx* c, const char* who) {
  if (c->sharded && !c->reduce)
    return pe_fail(PE_EINVAL, std::string(who) + ": a context that owns a block of modes needs "
                              "pe_options.residual_reduce (or pe_parareal_iter_sums)");
  return PE_OK;
}

extern "C" pe_status pe_parareal_iter(pe_ctx* c, double* rel_residual_out) {
  if (c && c->pend) return pe_fail(PE_ESTATE, "pe_parareal_iter: a solve is pending (pe_solve_wait first)");
  if (!c) return pe_fail(PE_EINVAL, "pe_parareal_iter: ctx is NULL");
  if (!c->have_problem) return pe_fail(PE_ESTATE, "pe_parareal_iter: no problem set (call pe_set_problem)");
  PE_TRY(need_totals(c, "pe_parareal_iter"));
  c->have_output = false;
  double r = 0.0;
  PE_TRY(iter_impl(c, &r, c->precision));
  if (rel_residual_out) *rel_residual_out = r;
  return PE_OK;
}

extern "C" pe_status pe_parareal_iter_sums(pe_ctx* c, double* sums_out) {
  if (c && c->pend) return pe_fail(PE_ESTATE, "pe_parareal_iter_sums: a solve is pending (pe_solve_wait first)");
  if (!c || !sums_out) return pe_fail(PE_EINVAL, "pe_parareal_iter_sums: NULL argument");
  if (!c->have_problem) return pe_fail(PE_ESTATE, "pe_parareal_iter_sums: no problem set (call pe_set_problem)");
  c->have_output = false;
  return iter_impl(c, nullptr, c->precision, sums_out);
}

extern "C" pe_status pe_refine(pe_ctx* c, double* rel_residual_out) {
  if (c && c->pend) return pe_fail(PE_ESTATE, "pe_refine: a solve is pending (pe_solve_wait first)");
  if (!c) return pe_fail(PE_EINVAL, "pe_refine: ctx is NULL");
  if (!c->have_problem) return pe_fail(PE_ESTATE, "pe_refine: no problem set (call pe_set_problem)");
  PE_TRY(need_totals(c, "pe_refine"));
  c->have_output = false;
  double r = 0.0;
  PE_TRY(iter_impl(c, &r, PE_FP64));
  if (rel_residual_out) *rel_residual_out = r;
  return PE_OK;
}

// ---------------------------------------------------------------------------
// device-resident Parareal loop: a CUDA graph with one conditional (while) node whose body is
// one pass of Algorithm 1's loop -- the fine sweep from every slice and the correction, whose
// last CTA appends r_k, advances k and sets the condition (r > tol and k < max_iter)
// ---------------------------------------------------------------------------
static bool loop_on_device(const pe_ctx* c) {
  return c->device_loop && !c->cache_forced && c->forcing_path == PE_FORCING_SEPARABLE && !c->reduce &&
         !c->sharded;
}

static pe_status build_loop_graph(pe_ctx* c) {
  if (c->loop_exec && c->loop_K == c->K && c->loop_prec == c->precision) return PE_OK;
  if (c->loop_exec) {
    PE_CUDA_TRY(cudaGraphExecDestroy(c->loop_exec));
    c->loop_exec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  PE_CUDA_TRY(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle handle;
  pe_status st = PE_OK;
  cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1u, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np{};
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return pe_cuda_fail(e, "device loop: conditional node");
  }
  // the body: the launches of one iteration, captured on the side stream (the context's own
  // stream may be the legacy default stream, which cannot be captured)
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t main_stream = c->stream;
  const int64_t launches0 = c->launches, sweeps0 = c->sweeps;
  e = cudaStreamBeginCaptureToGraph(c->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    c->stream = c->side;
    st = launch_fine_sweep(c, c->precision);
    if (st == PE_OK) st = launch_correction_kernel(c, c->loopctl, (unsigned long long)handle);
    c->stream = main_stream;
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(c->side, &captured);
    if (st == PE_OK && e2 != cudaSuccess) st = pe_cuda_fail(e2, "device loop: capture");
  } else {
    st = pe_cuda_fail(e, "device loop: begin capture");
  }
  c->loop_body_launches = c->launches - launches0;
  c->launches = launches0;
  c->sweeps = sweeps0;
  if (st == PE_OK) {
    e = cudaGraphInstantiate(&c->loop_exec, graph, 0);
    if (e != cudaSuccess) st = pe_cuda_fail(e, "device loop: instantiate");
  }
  cudaGraphDestroy(graph);
  if (st != PE_OK) {
    cudaGetLastError();
    c->loop_exec = nullptr;
    return st;
  }
  c->loop_K = c->K;
  c->loop_prec = c->precision;
  return PE_OK;
}

// Iterations of pe_solve on the device, enqueued: a kernel arms the loop state, the graph runs
// the loop, and the stop decision of every iteration also writes k, r and the non-finite flag
// into the mapped pinned mirror that the host reads after the solve's wait (no copies).
static pe_status enqueue_loop_on_device(pe_ctx* c, double tol) {
  PE_TRY(build_loop_graph(c));
  volatile LoopCtl* h = c->h_loop;
  h->k = 0;
  h->nonfinite = 0;
  h->r = INFINITY;
  PE_TRY(launch_loop_init(c, tol));
  PE_CUDA_TRY(cudaGraphLaunch(c->loop_exec, c->stream));
  return PE_OK;
}

// After the stream has completed: k, the last residual in *r, the history.
static pe_status finish_loop_on_device(pe_ctx* c, pe_result* res, double* r) {
  volatile LoopCtl* h = c->h_loop;
  const int k = h->k;
  c->k += k;
  c->sweeps += k;
  c->launches += (int64_t)k * c->loop_body_launches;
  *r = h->r;
  if (res && res->residual_history && res->history_cap > 0) {
    const int cnt = std::min(k, res->history_cap);
    PE_CUDA_TRY(cudaMemcpy(res->residual_history, c->loop_hist, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
  }
  if (h->nonfinite) {
    c->have_problem = false;
    if (c->precision == PE_MIXED && c->fine_engine == PE_FINE_TC) PE_TRY(fine_tc_status(c));
    return pe_fail(PE_ENONFINITE, "Parareal residual is not finite (NaN/Inf in the iterate)");
  }
  return PE_OK;
}

// ---------------------------------------------------------------------------
// device_loop = 2: a problem solved again (same u0 description or device pointer, same source,
// Dirichlet data and network) replays its set-up and output phases as CUDA graphs captured at its
// second solve (the first solve runs them directly, which makes every lazily built table and
// buffer exist before the capture).  The graphs re-execute every kernel; only the per-launch
// overhead goes.
// ---------------------------------------------------------------------------
static uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 0x100000001B3ull;
  }
  return h;
}

static uint64_t problem_key(const pe_ctx* c, const pe_field* u0, const pe_forcing* f) {
  uint64_t h = 0xcbf29ce484222325ull;
  h = fnv(h, &u0->kind, sizeof(u0->kind));
  h = fnv(h, &u0->n_terms, sizeof(u0->n_terms));
  if (u0->terms && u0->n_terms > 0) h = fnv(h, u0->terms, sizeof(pe_term) * (size_t)u0->n_terms);
  h = fnv(h, &u0->nodal, sizeof(u0->nodal));
  const int nf = f ? f->n_terms : 0;
  h = fnv(h, &nf, sizeof(nf));
  if (nf > 0 && f->terms) h = fnv(h, f->terms, sizeof(pe_term) * (size_t)nf);
  h = fnv(h, &c->nbd, sizeof(c->nbd));
  if (c->nbd > 0) h = fnv(h, c->bterms, sizeof(pe_term) * (size_t)c->nbd);
  h = fnv(h, &c->mlp, sizeof(c->mlp));
  return h;
}

// Captures body() (which enqueues on c->stream) into *exec; *launches = the kernels it enqueued.
// Returns false, with nothing enqueued and *exec null, when the phase cannot be captured.
template <typename F>
static bool capture_phase(pe_ctx* c, cudaGraphExec_t* exec, int64_t* launches, F body) {
  cudaStream_t main_stream = c->stream;
  const int64_t l0 = c->launches;
  *exec = nullptr;
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->stream = c->cap_stream;
  c->capturing = 1;
  const pe_status st = body();
  c->capturing = 0;
  c->stream = main_stream;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  *launches = c->launches - l0;
  c->launches = l0;
  bool ok = st == PE_OK && e == cudaSuccess && g != nullptr;
  if (ok && cudaGraphInstantiate(exec, g, 0) != cudaSuccess) {
    *exec = nullptr;
    ok = false;
  }
  if (g) cudaGraphDestroy(g);
  if (!ok) cudaGetLastError();
  return ok;
}

static pe_status output_phase(pe_ctx* c) {
  PE_TRY(modal_to_nodal(c, c->U + (int64_t)c->N * c->g.ndof, c->out_nodal));
  return add_lift(c, c->t0 + c->T, 1.0, 3, c->out_nodal);
}

// The solve in two halves: solve_begin enqueues the whole solve on the context's stream (with
// the loop on the device nothing in it waits for the GPU; the host-driven loop waits for every
// residual), solve_end waits for the stream and reports.
static pe_status solve_begin(pe_ctx* c, const pe_field* u0, const pe_forcing* f, double tol, double* nodal_out) {
  if (!c) return pe_fail(PE_EINVAL, "pe_solve: ctx is NULL");
  if (c->pend) return pe_fail(PE_ESTATE, "pe_solve: a solve is pending (pe_solve_wait first)");
  if (!(tol >= 0.0)) return pe_fail(PE_EINVAL, "pe_solve: tol must be >= 0");
  PE_TRY(need_totals(c, "pe_solve"));
  c->have_problem = false;
  c->launches = 0;
  c->ms_fine = 0.0;
  c->ms_corr = 0.0;
  c->sweeps = 0;
  // graphs of the set-up and output phases: a device-resident loop, and u0 not in host memory
  // (a copy from pageable host memory cannot be captured)
  bool use_graphs = false;
  c->u0_dev_hint = -1;
  if (c->device_loop == 2 && loop_on_device(c) && u0) {
    const bool host_u0 = u0->kind == PE_FIELD_NODAL && u0->nodal && !pe_is_device_ptr(u0->nodal);
    if (!host_u0) {
      if (u0->kind == PE_FIELD_NODAL) c->u0_dev_hint = 1;
      const uint64_t key = problem_key(c, u0, f);
      if (key != c->graph_key) {
        drop_solve_graphs(c);
        c->graph_key = key;
      }
      use_graphs = ++c->graph_key_seen >= 2;
    }
  }
  PE_CUDA_TRY(cudaEventRecord(c->ev[0], c->stream));
  if (use_graphs && !c->setup_exec &&
      !capture_phase(c, &c->setup_exec, &c->setup_launches, [&] { return set_problem_impl(c, u0, f); })) {
    use_graphs = false;  // not capturable: this problem runs its phases directly from now on
    c->graph_key_seen = INT_MIN / 2;
  }
  if (use_graphs) {
    // the host-side state is that of the previous solve of this problem (any other call that
    // changes it drops the graphs); only the iteration state restarts
    c->fz_prec = -1;
    c->k = 0;
    c->have_problem = true;
    c->have_output = false;
    PE_CUDA_TRY(cudaGraphLaunch(c->setup_exec, c->stream));
    c->launches += c->setup_launches;
  } else {
    PE_TRY(set_problem_impl(c, u0, f));
  }
  c->u0_dev_hint = -1;
  PE_CUDA_TRY(cudaEventRecord(c->ev[2], c->stream));
  double r = INFINITY;
  const bool on_device = loop_on_device(c);
  c->pend_hist.clear();
  if (on_device) {
    PE_TRY(enqueue_loop_on_device(c, tol));
  } else {
    while (c->k < c->max_iter) {
      PE_TRY(iter_impl(c, &r, c->precision));
      c->pend_hist.push_back(r);
      if (r <= tol) break;
    }
  }
  PE_CUDA_TRY(cudaEventRecord(c->ev[3], c->stream));
  if (use_graphs && !c->out_exec && !capture_phase(c, &c->out_exec, &c->out_launches, [&] { return output_phase(c); }))
    use_graphs = false;
  if (use_graphs) {
    PE_CUDA_TRY(cudaGraphLaunch(c->out_exec, c->stream));
    c->launches += c->out_launches;
  } else {
    PE_TRY(output_phase(c));
  }
  PE_CUDA_TRY(cudaEventRecord(c->ev[4], c->stream));
  // the nodal solution into the caller's buffer in the same stream order
  if (nodal_out)
    PE_CUDA_TRY(cudaMemcpyAsync(nodal_out, c->out_nodal, sizeof(double) * c->gn.ndof,
                                pe_is_device_ptr(nodal_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream));
  c->pend = true;
  c->pend_on_device = on_device;
  c->pend_tol = tol;
  c->pend_r = r;
  return PE_OK;
}

static pe_status solve_end(pe_ctx* c, pe_result* res) {
  if (!c) return pe_fail(PE_EINVAL, "pe_solve_wait: ctx is NULL");
  if (!c->pend) return pe_fail(PE_ESTATE, "pe_solve_wait: no solve pending");
  c->pend = false;
  PE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  double r = c->pend_r;
  if (c->pend_on_device) {
    PE_TRY(finish_loop_on_device(c, res, &r));
  } else if (res && res->residual_history) {
    const int cnt = std::min((int)c->pend_hist.size(), res->history_cap);
    for (int i = 0; i < cnt; ++i) res->residual_history[i] = c->pend_hist[i];
  }
  c->have_output = true;
  if (res) {
    res->k = c->k;
    res->residual = r;
    res->fine_sweeps = c->sweeps;
    res->ms_tables = elapsed(c->ev[0], c->ev[1]);
    res->ms_prepare = elapsed(c->ev[1], c->ev[2]);
    res->ms_iterations = elapsed(c->ev[2], c->ev[3]);
    res->ms_output = elapsed(c->ev[3], c->ev[4]);
    res->ms_fine_kernel = c->ms_fine;
    res->kernel_launches = c->launches;
    res->ms_correction_kernel = c->ms_corr;
    res->ms_coarse_kernel = elapsed(c->ev[8], c->ev[9]);
  }
  if (r > c->pend_tol && c->k < c->N)
    return pe_fail(PE_ENOCONV, "pe_solve: residual above tol after max_iter iterations");
  return PE_OK;
}

extern "C" pe_status pe_solve(pe_ctx* c, const pe_field* u0, const pe_forcing* f, double tol, pe_result* res) {
  PE_TRY(solve_begin(c, u0, f, tol, nullptr));
  return solve_end(c, res);
}

extern "C" pe_status pe_solve_out(pe_ctx* c, const pe_field* u0, const pe_forcing* f, double tol, double* nodal_out,
                                  pe_result* res) {
  if (!nodal_out) return pe_fail(PE_EINVAL, "pe_solve_out: nodal_out is NULL");
  PE_TRY(solve_begin(c, u0, f, tol, nodal_out));
  return solve_end(c, res);
}

extern "C" pe_status pe_solve_async(pe_ctx* c, const pe_field* u0, const pe_forcing* f, double tol,
                                    double* nodal_out) {
  return solve_begin(c, u0, f, tol, nodal_out);
}

extern "C" pe_status pe_solve_wait(pe_ctx* c, pe_result* res) { return solve_end(c, res); }

// ---------------------------------------------------------------------------
// getters, state
// ---------------------------------------------------------------------------
extern "C" pe_status pe_get_solution(pe_ctx* c, int32_t slice, double* nodal_out) {
  if (c && c->pend) return pe_fail(PE_ESTATE, "pe_get_solution: a solve is pending (pe_solve_wait first)");
  if (!c) return pe_fail(PE_EINVAL, "pe_get_solution: ctx is NULL");
  if (slice < 0 || slice > c->N) return pe_fail(PE_EINVAL, "pe_get_solution: slice out of range");
  if (!c->have_problem) return pe_fail(PE_ESTATE, "pe_get_solution: no problem set");
  if (slice == c->N && c->have_output) return copy_out(c, c->out_nodal, nodal_out, c->gn.ndof);
  PE_TRY(modal_to_nodal(c, c->U + (int64_t)slice * c->g.ndof, c->work0));
  PE_TRY(add_lift(c, c->t0 + slice * c->dT, 1.0, 3, c->work0));
  return copy_out(c, c->work0, nodal_out, c->gn.ndof);
}

extern "C" pe_status pe_get_modal(pe_ctx* c, int32_t slice, double* modal_out) {
  if (c && c->pend) return pe_fail(PE_ESTATE, "pe_get_modal: a solve is pending (pe_solve_wait first)");
  if (!c) return pe_fail(PE_EINVAL, "pe_get_modal: ctx is NULL");
  if (slice < 0 || slice > c->N) return pe_fail(PE_EINVAL, "pe_get_modal: slice out of range");
  if (!c->have_problem) return pe_fail(PE_ESTATE, "pe_get_modal: no problem set");
  return copy_out(c, c->U + (int64_t)slice * c->g.ndof, modal_out, c->g.ndof);
}

extern "C" pe_status pe_get_lambda(pe_ctx* c, double* out) {
  if (!c) return pe_fail(PE_EINVAL, "pe_get_lambda: ctx is NULL");
  return copy_out(c, c->lam, out, c->g.ndof);
}

extern "C" pe_status pe_get_coefficients(pe_ctx* c, int32_t which, double* out) {
  if (!c) return pe_fail(PE_EINVAL, "pe_get_coefficients: ctx is NULL");
  if (which == 0) return copy_out(c, c->coefF, out, (size_t)(c->q + 1) * c->g.ndof);
  if (which == 1) return copy_out(c, c->coefG, out, (size_t)(c->p + 1) * c->g.ndof);
  return pe_fail(PE_EINVAL, "pe_get_coefficients: which must be 0 (fine) or 1 (coarse)");
}

extern "C" pe_status pe_forcing_modal(pe_ctx* c, double t, double* out) {
  if (!c) return pe_fail(PE_EINVAL, "pe_forcing_modal: ctx is NULL");
  if (!c->have_problem) return pe_fail(PE_ESTATE, "pe_forcing_modal: no problem set");
  if (c->forcing_path != PE_FORCING_SEPARABLE) return pe_fail(PE_EINVAL, "pe_forcing_modal: separable path only");
  PE_TRY(launch_forcing_modal(c, t, c->work0));
  return copy_out(c, c->work0, out, c->g.ndof);
}

extern "C" pe_status pe_get_nodes(pe_ctx* c, int32_t which, double* c_out) {
  if (!c || !c_out) return pe_fail(PE_EINVAL, "pe_get_nodes: NULL argument");
  if (which == 0) memcpy(c_out, c->cF, sizeof(double) * c->q);
  else if (which == 1) memcpy(c_out, c->cG, sizeof(double) * c->p);
  else return pe_fail(PE_EINVAL, "pe_get_nodes: which must be 0 or 1");
  return PE_OK;
}

namespace {
// the problem a state belongs to: grid (every axis), box, D, time interval and partition
struct StateHeader {
  uint64_t magic;
  int32_t d, N, k, M;
  int64_t ndof;
  int32_t n[3], periodic_mask;
  double box[6], D, t0, T;
  int32_t mode_begin, mode_end;  // the axis-0 modes of the state (a sharded context's block)
};
const uint64_t kStateMagic = 0x3330353135504550ull;  // "PEP51503"

void fill_header(const pe_ctx* c, StateHeader* h) {
  memset(h, 0, sizeof(*h));
  h->magic = kStateMagic;
  h->d = c->g.d; h->N = c->N; h->k = c->k; h->M = c->M; h->ndof = c->g.ndof;
  for (int a = 0; a < 3; ++a) {
    h->n[a] = c->gn.n[a];
    h->periodic_mask |= c->g.per[a] << a;
    h->box[2 * a] = c->lo[a];
    h->box[2 * a + 1] = c->hi[a];
  }
  h->D = c->D; h->t0 = c->t0; h->T = c->T;
  h->mode_begin = c->base0;
  h->mode_end = c->base0 + c->g.n[0];
}
}  // namespace

extern "C" pe_status pe_save_state(pe_ctx* c, void* buf, size_t* bytes) {
  if (c && c->pend) return pe_fail(PE_ESTATE, "pe_save_state: a solve is pending (pe_solve_wait first)");
  if (!c || !bytes) return pe_fail(PE_EINVAL, "pe_save_state: NULL argument");
  const size_t nd = (size_t)c->g.ndof, N = (size_t)c->N;
  const size_t need = sizeof(StateHeader) + sizeof(double) * (N + 1) * nd;
  if (!buf) {
    *bytes = need;
    return PE_OK;
  }
  if (*bytes < need) return pe_fail(PE_EINVAL, "pe_save_state: buffer too small");
  if (!c->have_problem) return pe_fail(PE_ESTATE, "pe_save_state: no problem set");
  StateHeader h;
  fill_header(c, &h);
  memcpy(buf, &h, sizeof(h));
  char* p = (char*)buf + sizeof(h);
  PE_CUDA_TRY(cudaMemcpyAsync(p, c->U, sizeof(double) * (N + 1) * nd, cudaMemcpyDeviceToHost, c->stream));
  PE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  *bytes = need;
  return PE_OK;
}

extern "C" pe_status pe_load_state(pe_ctx* c, const void* buf, size_t bytes) {
  if (c && c->pend) return pe_fail(PE_ESTATE, "pe_load_state: a solve is pending (pe_solve_wait first)");
  if (!c || !buf) return pe_fail(PE_EINVAL, "pe_load_state: NULL argument");
  if (!c->have_problem) return pe_fail(PE_ESTATE, "pe_load_state: set the same problem first (pe_set_problem)");
  const size_t nd = (size_t)c->g.ndof, N = (size_t)c->N;
  const size_t need = sizeof(StateHeader) + sizeof(double) * (N + 1) * nd;
  if (bytes < need) return pe_fail(PE_EINVAL, "pe_load_state: buffer too small");
  StateHeader h, mine;
  memcpy(&h, buf, sizeof(h));
  fill_header(c, &mine);
  if (h.magic != kStateMagic) return pe_fail(PE_EINVAL, "pe_load_state: not a libpe state (bad magic)");
  // everything but k must match: a state of another grid (also the same Ndof with the axes
  // swapped), box, D, time interval or partition would put the modes in the wrong places
  mine.k = h.k;
  if (memcmp(&h, &mine, sizeof(h)) != 0)
    return pe_fail(PE_EINVAL, "pe_load_state: state belongs to another problem (grid, box, D, time interval "
                              "or partition differ)");
  const char* p = (const char*)buf + sizeof(h);
  PE_CUDA_TRY(cudaMemcpyAsync(c->U, p, sizeof(double) * (N + 1) * nd, cudaMemcpyHostToDevice, c->stream));
  PE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->k = h.k;
  c->have_output = false;
  return PE_OK;
}
