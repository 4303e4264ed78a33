// Host side of the batched solver (pe_setup_batch / pe_batch_*): validation,
// arena layout, work-item lists, the captured Parareal iteration graph and
// the launch-shape autotuner.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "pe_batch.h"

namespace {

template <typename T>
pe_status balloc(T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return pe_fail(PE_ENOMEM, "batch: cudaMalloc of " + std::to_string(sizeof(T) * count) + " bytes failed");
  }
  return PE_OK;
}

template <typename T>
pe_status upload(T** d, const std::vector<T>& h, cudaStream_t st) {
  PE_TRY(balloc(d, h.size()));
  if (!h.empty()) PE_CUDA_TRY(cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
  return PE_OK;
}

void free_batch(pe_batch* b) {
  if (!b) return;
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  void* ptrs[] = {b->d_probs, b->d_terms, b->d_mode_items, b->fine128.d_items, b->fine256.d_items,
                  b->d_factor_jobs, b->d_mu_prefix, b->d_tt_prefix, b->muM, b->ratio, b->coefF, b->coefG,
                  b->coefF32, b->U, b->Fbar, b->axisF, b->axisU0, b->axisF32, b->AF, b->AG,
                  b->AF32, b->partials, b->active, b->kcount, b->resid, b->counter, b->dflags,
                  b->W, b->W32, b->Z, b->d_cols, b->AG32, b->Z32, b->tc.A, b->tc.B, b->tc.d_items,
                  b->tc.d_w_prefix, b->tc.d_y_prefix, b->tc.err, b->Kt, b->Ph, b->d_kt_prefix,
                  b->d_ph_prefix};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->h_flags) cudaFreeHost(b->h_flags);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

uint64_t fnv1a(uint64_t h, const void* data, size_t n) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 0x100000001B3ull;
  }
  return h;
}

// Fine work items (problem, tile of threads*MPT modes; the item runs every slice of its
// problem), grouped by column class, longest (most slices) first within a class, and the
// dynamic shared memory each class needs (its widest staged chunk of time factors).
pe_status build_fine_items(pe_batch* b, int threads, FineItems* out) {
  std::vector<FineItem> items;
  const size_t elem = b->precision == PE_MIXED ? sizeof(float) : sizeof(double);
  std::vector<int> order((size_t)b->P);
  for (int p = 0; p < b->P; ++p) order[(size_t)p] = p;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return (int64_t)b->probs[x].N * b->probs[x].M > (int64_t)b->probs[y].N * b->probs[y].M; });
  for (int c = 0; c < kBatchClasses; ++c) {
    out->begin[c] = (int)std::min<size_t>(items.size(), INT32_MAX);
    out->smem[c] = 0;
    for (int p : order) {
      const BProb& B = b->probs[p];
      const int KC = (B.K + 3) / 4 * 4;
      if (KC != 4 * (c + 1)) continue;
      const size_t need = B.dbuf ? 2 * sizeof(float) * (size_t)B.M * KC : elem * (size_t)B.mchunk * KC;
      out->smem[c] = std::max(out->smem[c], need);
      const int mpt = b->precision == PE_MIXED ? batch_mixed_mpt(KC) : 1;
      const int64_t tile = (int64_t)threads * mpt;
      for (int64_t J0 = 0; J0 < B.g.ndof; J0 += tile) items.push_back(FineItem{p, 0, J0});
    }
  }
  if (items.size() > (size_t)INT32_MAX) return pe_fail(PE_EINVAL, "batch: too many work items");
  out->begin[kBatchClasses] = (int)items.size();
  out->n = (int)items.size();
  return upload(&out->d_items, items, b->stream);
}

}  // namespace

extern "C" pe_status pe_setup_batch(pe_batch** out, int32_t n_problems, const pe_problem* problems,
                                    const pe_options* opt) {
  if (!out) return pe_fail(PE_EINVAL, "pe_setup_batch: out is NULL");
  *out = nullptr;
  if (n_problems < 1 || !problems) return pe_fail(PE_EINVAL, "pe_setup_batch: need at least one problem");
  pe_options o{};
  if (opt) o = *opt;
  if (o.precision != PE_FP64 && o.precision != PE_MIXED) return pe_fail(PE_EINVAL, "pe_setup_batch: bad precision");
  if (o.quad_pts == 0) o.quad_pts = 3;
  if (o.quad_pts < 1 || o.quad_pts > 8) return pe_fail(PE_EINVAL, "pe_setup_batch: quad_pts must be in 1..8");
  if (o.fine_engine != PE_FINE_SIMT && o.fine_engine != PE_FINE_TC)
    return pe_fail(PE_EINVAL, "pe_setup_batch: bad fine_engine");
  if (o.fine_engine == PE_FINE_TC && o.precision != PE_MIXED)
    return pe_fail(PE_EINVAL, "pe_setup_batch: PE_FINE_TC needs PE_MIXED");

  pe_batch* b = new (std::nothrow) pe_batch();
  if (!b) return pe_fail(PE_ENOMEM, "pe_setup_batch: host allocation failed");
  b->P = n_problems;
  b->precision = o.precision;
  b->fine_engine = o.fine_engine;
  b->quad_pts = o.quad_pts;
  b->user_stream = (cudaStream_t)o.cuda_stream;
  b->gauss = make_gauss(o.quad_pts);
  pe_status st = PE_OK;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      st = pe_cuda_fail(cudaGetLastError(), "pe_setup_batch: device query");
    }
  }
  if (st == PE_OK && cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
    st = pe_cuda_fail(cudaGetLastError(), "pe_setup_batch: stream");
  if (st != PE_OK) {
    free_batch(b);
    return st;
  }

  // ---- validate and lay out every problem --------------------------------
  int64_t oU = 0, oS = 0, oCF = 0, oCG = 0, oAx = 0, oAxU = 0, oAF = 0, oAF32 = 0, oAG = 0, oMu = 0, oItems = 0;
  int64_t oW = 0, oZ = 0, oTA = 0, oTB = 0, wjobs = 0, yjobs = 0;
  std::vector<int64_t> mu_prefix, tt_prefix, w_prefix, y_prefix;
  std::vector<short> cols;
  int64_t tt = 0;
  uint64_t sig = 0xcbf29ce484222325ull;
  b->probs.resize(n_problems);
  for (int p = 0; p < n_problems && st == PE_OK; ++p) {
    const pe_problem& q = problems[p];
    BProb& B = b->probs[p];
    memset(&B, 0, sizeof(B));
    const std::string tag = "problem " + std::to_string(p) + ": ";
    if (q.d < 1 || q.d > PE_MAX_D) { st = pe_fail(PE_EINVAL, tag + "d must be 1..3"); break; }
    if (!(q.D > 0.0) || !(q.T > 0.0) || !isfinite(q.D) || !isfinite(q.T) || !isfinite(q.t0)) {
      st = pe_fail(PE_EINVAL, tag + "D and T must be positive");
      break;
    }
    if (q.n_slices < 1 || q.n_substeps < 1) { st = pe_fail(PE_EINVAL, tag + "slices/substeps must be >= 1"); break; }
    int64_t ndof = 1;
    int nsum = 0;
    for (int a = 0; a < PE_MAX_D; ++a) {
      if (a < q.d) {
        if (q.n[a] < 1 || q.n[a] > 4096) { st = pe_fail(PE_EINVAL, tag + "n_a must be in 1..4096"); break; }
        if (!(q.box[2 * a + 1] > q.box[2 * a])) { st = pe_fail(PE_EINVAL, tag + "box needs lo < hi"); break; }
        B.g.n[a] = q.n[a];
        B.g.off[a] = nsum;
        B.lo[a] = q.box[2 * a];
        B.h[a] = (q.box[2 * a + 1] - q.box[2 * a]) / (double)(q.n[a] + 1);
        ndof *= q.n[a];
        nsum += q.n[a];
        b->nmax = std::max(b->nmax, q.n[a]);
      } else {
        B.g.n[a] = 1;
        B.g.off[a] = nsum;
        B.lo[a] = 0.0;
        B.h[a] = 1.0;
      }
    }
    if (st != PE_OK) break;
    B.g.d = q.d;
    B.g.ndof = ndof;
    B.N = q.n_slices;
    B.M = q.n_substeps;
    B.D = q.D;
    B.t0 = q.t0;
    B.dT = q.T / (double)q.n_slices;
    B.dt = B.dT / (double)q.n_substeps;
    if ((st = pe_resolve_nodes(&q.fine, "fine", &B.q, B.cF)) != PE_OK) break;
    if ((st = pe_resolve_nodes(&q.coarse, "coarse", &B.p, B.cG)) != PE_OK) break;
    pe_lagrange_coeffs(B.q, B.cF, B.lagF);
    pe_lagrange_coeffs(B.p, B.cG, B.lagG);
    if (q.u0.kind != PE_FIELD_TERMS_SEPARABLE) {
      st = pe_fail(PE_EINVAL, tag + "a batch takes separable initial data (PE_FIELD_TERMS_SEPARABLE)");
      break;
    }
    const int nf = q.forcing.n_terms;
    if (nf > PE_BATCH_MAX_TERMS) { st = pe_fail(PE_EINVAL, tag + "at most 20 forcing terms in a batch"); break; }
    if ((st = pe_validate_terms(nf, q.forcing.terms, q.d, "forcing")) != PE_OK) break;
    if ((st = pe_validate_terms(q.u0.n_terms, q.u0.terms, q.d, "u0")) != PE_OK) break;
    B.tf = (int)b->terms.size();
    if (nf == 0) {
      pe_term z;
      memset(&z, 0, sizeof(z));
      b->terms.push_back(z);
      B.R = 1;
    } else {
      for (int i = 0; i < nf; ++i) b->terms.push_back(q.forcing.terms[i]);
      B.R = nf;
    }
    B.tu = (int)b->terms.size();
    if (q.u0.n_terms == 0) {
      pe_term z;
      memset(&z, 0, sizeof(z));
      b->terms.push_back(z);
      B.Ru = 1;
    } else {
      for (int i = 0; i < q.u0.n_terms; ++i) b->terms.push_back(q.u0.terms[i]);
      B.Ru = q.u0.n_terms;
    }
    if (B.Ru > PE_MAX_TERMS) { st = pe_fail(PE_EINVAL, tag + "too many u0 terms"); break; }
    // stage-contracted columns of the fine step: one per exponential term, two per sinusoid
    B.oCol = (int64_t)cols.size();
    for (int r = 0; r < B.R; ++r) {
      cols.push_back((short)(r << 1));
      if (b->terms[B.tf + r].tkind == PE_T_SIN) cols.push_back((short)((r << 1) | 1));
    }
    B.K = (int)((int64_t)cols.size() - B.oCol);
    // tile bodies run with K rounded up to a multiple of 4 (zero-padded staging rows)
    const int KC = (B.K + 3) / 4 * 4;
    const size_t elem = b->precision == PE_MIXED ? sizeof(float) : sizeof(double);
    B.mchunk = pick_mchunk(B.M, KC, elem);
    B.dbuf = b->precision == PE_MIXED && 2 * (size_t)B.M * KC * sizeof(float) <= 48 * 1024 ? 1 : 0;
    B.oU = oU; oU += (int64_t)(B.N + 1) * ndof;
    B.oS = oS; oS += (int64_t)B.N * ndof;
    B.oCF = oCF; oCF += (int64_t)(B.q + 2) * ndof;
    B.oCG = oCG; oCG += (int64_t)(B.p + 1) * ndof;
    B.oAx = oAx; oAx += (int64_t)B.R * nsum;
    B.oAxU = oAxU; oAxU += (int64_t)B.Ru * nsum;
    B.oAF = oAF; oAF += (int64_t)B.N * B.M * B.K;
    B.oAF32 = oAF32; oAF32 += (int64_t)B.N * B.M * KC;
    B.oW = oW; oW += (int64_t)B.K * ndof;
    B.oZ = oZ; oZ += (int64_t)B.q * B.K;
    B.oAG = oAG; oAG += (int64_t)B.N * B.p * B.R;
    B.oMu = oMu;
    mu_prefix.push_back(oMu);
    oMu += nsum;
    tt_prefix.push_back(tt);
    tt += (int64_t)B.N * B.K + (int64_t)B.N * B.p * B.R + (int64_t)B.q * B.K;  // b_time_tables_kernel's threads
    B.oItems = oItems;
    B.nItems = (int)((ndof + 255) / 256);
    oItems += B.nItems;
    if (b->fine_engine == PE_FINE_TC) {
      // tensor-core operand images: split stage weights per 128-mode tile, split time factors
      // per slice group, each in the byte layout the kernel copies into shared memory
      if (!batch_tc_shape(B.K, B.M, &B.KP, &B.TG, &B.NR)) {
        st = pe_fail(PE_EINVAL, tag + "PE_FINE_TC needs M a multiple of 16 in 16..128");
        break;
      }
      B.groups = (B.N + B.TG - 1) / B.TG;
      B.tiles = (ndof + 127) / 128;
      B.oTA = oTA;
      oTA += B.tiles * 3 * 128 * B.KP * 2;
      B.oTB = oTB;
      oTB += (int64_t)B.groups * 3 * B.NR * B.KP * 2;
      w_prefix.push_back(wjobs);
      wjobs += B.tiles * 128 * (B.KP / 8);
      y_prefix.push_back(yjobs);
      yjobs += (int64_t)B.groups * B.NR * (B.KP / 8);
    }
    sig = fnv1a(sig, &B.g, sizeof(B.g));
    sig = fnv1a(sig, &B.N, sizeof(int) * 6);
  }
  if (st != PE_OK) {
    free_batch(b);
    return st;
  }
  b->signature = fnv1a(fnv1a(sig, &b->precision, sizeof(int)), &b->fine_engine, sizeof(int));
  b->mu_total = oMu;
  b->tt_total = tt;

  // ---- arenas --------------------------------------------------------------
  const bool mixed = b->precision == PE_MIXED;
  if (st == PE_OK) st = balloc(&b->muM, oMu);
  if (st == PE_OK) st = balloc(&b->ratio, oMu);
  if (st == PE_OK) st = balloc(&b->coefF, oCF);
  if (st == PE_OK && mixed) st = balloc(&b->coefF32, oCF);
  if (st == PE_OK) st = balloc(&b->coefG, oCG);
  if (st == PE_OK) st = balloc(&b->U, oU);
  if (st == PE_OK) st = balloc(&b->Fbar, oS);
  if (st == PE_OK) st = balloc(&b->axisF, oAx);
  if (st == PE_OK && mixed) st = balloc(&b->axisF32, oAx);
  if (st == PE_OK) st = balloc(&b->axisU0, oAxU);
  if (st == PE_OK) st = balloc(&b->AF, oAF);
  if (st == PE_OK && mixed) st = balloc(&b->AF32, oAF32);
  if (st == PE_OK) st = balloc(&b->AG, oAG);
  if (st == PE_OK && mixed) st = balloc(&b->AG32, oAG);
  // float64 weights for the float64 fine kernel; the mixed form keeps only the float copy
  if (st == PE_OK && !mixed) st = balloc(&b->W, oW);
  if (st == PE_OK && mixed) st = balloc(&b->W32, oW);
  if (st == PE_OK) st = balloc(&b->Z, oZ);
  if (st == PE_OK && mixed) st = balloc(&b->Z32, oZ);
  if (st == PE_OK) st = balloc(&b->partials, 2 * (size_t)oItems);
  if (st == PE_OK) st = balloc(&b->active, (size_t)b->P);
  if (st == PE_OK) st = balloc(&b->kcount, (size_t)b->P);
  if (st == PE_OK) st = balloc(&b->resid, (size_t)b->P);
  if (st == PE_OK) st = balloc(&b->counter, (size_t)kBatchClasses);
  if (st == PE_OK) st = balloc(&b->dflags, 2);
  if (st == PE_OK && b->fine_engine == PE_FINE_TC) {
    st = balloc(&b->tc.A, (size_t)oTA);
    if (st == PE_OK) st = balloc(&b->tc.B, (size_t)oTB);
    if (st == PE_OK) st = balloc(&b->tc.err, 1);
    if (st == PE_OK && cudaMemset(b->tc.err, 0, sizeof(int)) != cudaSuccess)
      st = pe_cuda_fail(cudaGetLastError(), "pe_setup_batch: error flag");
    b->tc.w_jobs = wjobs;
    b->tc.y_jobs = yjobs;
  }
  if (st == PE_OK && cudaMallocHost((void**)&b->h_flags, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    st = pe_fail(PE_ENOMEM, "pe_setup_batch: pinned allocation failed");
  }
  if (st != PE_OK) {
    free_batch(b);
    return st;
  }
  b->n_active = b->dflags;
  b->nonfinite = b->dflags + 1;

  // ---- work items ----------------------------------------------------------
  {
    std::vector<ModeItem> mitems;
    mitems.reserve((size_t)oItems);
    for (int p = 0; p < b->P; ++p)
      for (int64_t J0 = 0; J0 < b->probs[p].g.ndof; J0 += 256) mitems.push_back(ModeItem{p, 0, J0});
    b->n_mode_items = (int)mitems.size();
    std::vector<FactorJob> jobs;
    for (int p = 0; p < b->P; ++p) {
      const BProb& B = b->probs[p];
      for (int a = 0; a < B.g.d; ++a) {
        for (int r = 0; r < B.R; ++r) jobs.push_back(FactorJob{p, a, r, 0});
        for (int r = 0; r < B.Ru; ++r) jobs.push_back(FactorJob{p, a, r, 1});
      }
    }
    b->n_factor_jobs = (int)jobs.size();
    st = upload(&b->d_probs, b->probs, b->stream);
    if (st == PE_OK) st = upload(&b->d_terms, b->terms, b->stream);
    if (st == PE_OK) st = upload(&b->d_mode_items, mitems, b->stream);
    if (st == PE_OK) st = upload(&b->d_factor_jobs, jobs, b->stream);
    if (st == PE_OK) st = upload(&b->d_mu_prefix, mu_prefix, b->stream);
    if (st == PE_OK) st = upload(&b->d_tt_prefix, tt_prefix, b->stream);
    if (st == PE_OK) st = upload(&b->d_cols, cols, b->stream);
    if (st == PE_OK) st = build_fine_items(b, 128, &b->fine128);
    if (st == PE_OK) st = build_fine_items(b, 256, &b->fine256);
    if (st == PE_OK && b->fine_engine == PE_FINE_TC) {
      // items per column padding (16, 32, 64), each problem's (slice group, tile) pairs
      // group-major, so that a CTA's consecutive items share the group's B operand
      std::vector<BTcItem> titems;
      for (int cls = 0; cls < 3; ++cls) {
        b->tc.begin[cls] = (int)titems.size();
        for (int p = 0; p < b->P; ++p) {
          const BProb& B = b->probs[p];
          if (B.KP != (16 << cls)) continue;
          for (int g = 0; g < B.groups; ++g)
            for (int64_t t = 0; t < B.tiles; ++t) titems.push_back(BTcItem{p, g, t});
        }
      }
      if (titems.size() > (size_t)INT32_MAX) st = pe_fail(PE_EINVAL, "batch: too many tensor-core work items");
      b->tc.begin[3] = (int)titems.size();
      if (st == PE_OK) st = upload(&b->tc.d_items, titems, b->stream);
      if (st == PE_OK) st = upload(&b->tc.d_w_prefix, w_prefix, b->stream);
      if (st == PE_OK) st = upload(&b->tc.d_y_prefix, y_prefix, b->stream);
    }
  }
  if (st == PE_OK) st = batch_set_attributes(b);
  if (st == PE_OK) st = batch_launch_axis_tables(b);
  if (st == PE_OK) st = batch_launch_coef_tables(b);
  if (st == PE_OK) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) st = pe_cuda_fail(e, "pe_setup_batch");
  }
  if (st != PE_OK) {
    free_batch(b);
    return st;
  }
  *out = b;
  return PE_OK;
}

extern "C" void pe_batch_destroy(pe_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

namespace {

pe_status reset_iteration_state(pe_batch* b) {
  std::vector<int> ones((size_t)b->P, 1);
  PE_CUDA_TRY(cudaMemcpyAsync(b->active, ones.data(), sizeof(int) * b->P, cudaMemcpyHostToDevice, b->stream));
  PE_CUDA_TRY(cudaMemsetAsync(b->kcount, 0, sizeof(int) * b->P, b->stream));
  PE_CUDA_TRY(cudaMemsetAsync(b->resid, 0, sizeof(double) * b->P, b->stream));
  PE_CUDA_TRY(cudaMemsetAsync(b->dflags, 0, 2 * sizeof(int), b->stream));
  // the host vector must stay alive until the copy has been issued from it
  PE_CUDA_TRY(cudaStreamSynchronize(b->stream));
  return PE_OK;
}

pe_status ensure_graph(pe_batch* b, double tol) {
  if (b->graph_exec && b->graph_tol == tol && b->graph_threads == b->tune_threads && b->graph_ctas == b->tune_ctas)
    return PE_OK;
  if (b->graph_exec) {
    cudaGraphExecDestroy(b->graph_exec);
    b->graph_exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  PE_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  pe_status st = batch_enqueue_iteration(b, b->stream, tol);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (st != PE_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return pe_cuda_fail(e, "batch: graph capture");
  b->graph = g;
  PE_CUDA_TRY(cudaGraphInstantiate(&b->graph_exec, g, 0));
  b->graph_tol = tol;
  b->graph_threads = b->tune_threads;
  b->graph_ctas = b->tune_ctas;
  return PE_OK;
}

float ms_between(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

}  // namespace

extern "C" pe_status pe_batch_autotune(pe_batch* b, const char* cache_path) {
  if (!b) return pe_fail(PE_EINVAL, "pe_batch_autotune: NULL batch");
  if (b->fine_engine == PE_FINE_TC) {  // one CTA of 288 threads per SM: no launch shape to choose
    b->tuned = true;
    return PE_OK;
  }
  cudaDeviceProp prop;
  int dev = 0;
  PE_CUDA_TRY(cudaGetDevice(&dev));
  PE_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  char key[320];
  snprintf(key, sizeof(key), "%s|%016llx", prop.name, (unsigned long long)b->signature);
  for (char* c = key; *c; ++c)
    if (*c == ' ') *c = '_';
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      std::istringstream ss(line);
      std::string k;
      int th = 0, ct = 0;
      if (ss >> k >> th >> ct && k == key && (th == 128 || th == 256) && ct >= 1 && ct <= 8) {
        b->tune_threads = th;
        b->tune_ctas = ct;
        b->tuned = true;
        return PE_OK;
      }
    }
  }
  // time every candidate on a prepared state (writes only the fine-propagator outputs)
  PE_TRY(reset_iteration_state(b));
  PE_TRY(batch_launch_prepare(b));
  const int cand_threads[2] = {128, 256};
  float best = 1e30f;
  int best_t = 256, best_c = 2;
  for (int ti = 0; ti < 2; ++ti) {
    for (int ct = 1; ct <= 4; ++ct) {
      if (cand_threads[ti] == 256 && ct > 2) continue;  // 256 x 128 registers: at most 2 CTAs per SM
      float ms = 0.f, tot = 0.f;
      PE_TRY(batch_time_fine(b, cand_threads[ti], ct, &ms));  // warm
      for (int rep = 0; rep < 2; ++rep) {
        PE_TRY(batch_time_fine(b, cand_threads[ti], ct, &ms));
        tot += ms;
      }
      if (tot < best) {
        best = tot;
        best_t = cand_threads[ti];
        best_c = ct;
      }
    }
  }
  b->tune_threads = best_t;
  b->tune_ctas = best_c;
  b->tuned = true;
  if (cache_path) {
    std::ofstream outf(cache_path, std::ios::app);
    if (outf) outf << key << " " << best_t << " " << best_c << "\n";
  }
  return PE_OK;
}

extern "C" pe_status pe_batch_solve(pe_batch* b, double tol, pe_batch_result* res) {
  if (!b) return pe_fail(PE_EINVAL, "pe_batch_solve: NULL batch");
  if (!(tol >= 0.0)) return pe_fail(PE_EINVAL, "pe_batch_solve: tol must be >= 0");
  cudaEvent_t ev[3];
  for (int i = 0; i < 3; ++i) PE_CUDA_TRY(cudaEventCreate(&ev[i]));
  if (b->user_stream) {
    PE_CUDA_TRY(cudaEventRecord(ev[0], b->user_stream));
    PE_CUDA_TRY(cudaStreamWaitEvent(b->stream, ev[0], 0));
  }
  b->launches = 0;
  PE_TRY(reset_iteration_state(b));
  PE_TRY(ensure_graph(b, tol));
  PE_CUDA_TRY(cudaEventRecord(ev[0], b->stream));
  PE_TRY(batch_launch_prepare(b));
  PE_CUDA_TRY(cudaEventRecord(ev[1], b->stream));
  int replays = 0;
  int maxN = 0;
  for (const BProb& B : b->probs) maxN = std::max(maxN, B.N);
  for (;;) {
    PE_CUDA_TRY(cudaGraphLaunch(b->graph_exec, b->stream));
    PE_CUDA_TRY(cudaStreamSynchronize(b->stream));
    ++replays;
    b->launches += batch_fine_launches(b) + 2;  // graph: fine kernels, correction, reduction
    if (b->h_flags[1]) {
      b->have_problem = false;
      if (b->fine_engine == PE_FINE_TC) PE_TRY(batch_tc_status(b));
      return pe_fail(PE_ENONFINITE, "batch: a problem's Parareal residual is not finite");
    }
    if (b->h_flags[0] == 0 || replays >= maxN) break;
  }
  PE_CUDA_TRY(cudaEventRecord(ev[2], b->stream));
  PE_CUDA_TRY(cudaEventSynchronize(ev[2]));
  b->have_problem = true;
  if (b->user_stream) {
    PE_CUDA_TRY(cudaEventRecord(ev[0], b->stream));
    PE_CUDA_TRY(cudaStreamWaitEvent(b->user_stream, ev[0], 0));
  }
  if (res) {
    std::vector<int> k((size_t)b->P);
    std::vector<double> r((size_t)b->P);
    PE_CUDA_TRY(cudaMemcpy(k.data(), b->kcount, sizeof(int) * b->P, cudaMemcpyDeviceToHost));
    PE_CUDA_TRY(cudaMemcpy(r.data(), b->resid, sizeof(double) * b->P, cudaMemcpyDeviceToHost));
    res->graph_replays = replays;
    res->max_k = 0;
    res->max_residual = 0.0;
    res->fine_dof_substeps = 0;
    for (int p = 0; p < b->P; ++p) {
      const BProb& B = b->probs[p];
      res->max_k = std::max(res->max_k, k[p]);
      res->max_residual = std::max(res->max_residual, r[p]);
      res->fine_dof_substeps += B.g.ndof * (int64_t)B.N * B.M * k[p];
    }
    res->ms_prepare = ms_between(ev[0], ev[1]);
    res->ms_iterations = ms_between(ev[1], ev[2]);
    res->kernel_launches = b->launches;
    res->threads = b->fine_engine == PE_FINE_TC ? 288 : b->tune_threads;
    res->ctas_per_sm = b->fine_engine == PE_FINE_TC ? 1 : b->tune_ctas;
  }
  for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
  return PE_OK;
}

extern "C" pe_status pe_batch_get_modal(pe_batch* b, int32_t problem, int32_t slice, double* out) {
  if (!b || !out) return pe_fail(PE_EINVAL, "pe_batch_get_modal: NULL argument");
  if (problem < 0 || problem >= b->P) return pe_fail(PE_EINVAL, "pe_batch_get_modal: problem out of range");
  const BProb& B = b->probs[problem];
  if (slice < 0 || slice > B.N) return pe_fail(PE_EINVAL, "pe_batch_get_modal: slice out of range");
  if (!b->have_problem) return pe_fail(PE_ESTATE, "pe_batch_get_modal: no solve has completed");
  const bool dev = pe_is_device_ptr(out);
  PE_CUDA_TRY(cudaMemcpyAsync(out, b->U + B.oU + (int64_t)slice * B.g.ndof, sizeof(double) * B.g.ndof,
                              dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
  PE_CUDA_TRY(cudaStreamSynchronize(b->stream));
  return PE_OK;
}

extern "C" pe_status pe_batch_get_solution(pe_batch* b, int32_t problem, double* nodal_out) {
  if (!b || !nodal_out) return pe_fail(PE_EINVAL, "pe_batch_get_solution: NULL argument");
  if (problem < 0 || problem >= b->P) return pe_fail(PE_EINVAL, "pe_batch_get_solution: problem out of range");
  if (!b->have_problem) return pe_fail(PE_ESTATE, "pe_batch_get_solution: no solve has completed");
  const BProb& B = b->probs[problem];
  double* tmp = nullptr;
  PE_CUDA_TRY(cudaMallocAsync((void**)&tmp, sizeof(double) * B.g.ndof, b->stream));
  int n[PE_MAX_D] = {B.g.n[0], B.g.n[1], B.g.n[2]};
  pe_status st = pe_dst(B.g.d, n, b->U + B.oU + (int64_t)B.N * B.g.ndof, tmp, b->stream);
  if (st == PE_OK) {
    const bool dev = pe_is_device_ptr(nodal_out);
    cudaError_t e = cudaMemcpyAsync(nodal_out, tmp, sizeof(double) * B.g.ndof,
                                    dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) st = pe_cuda_fail(e, "pe_batch_get_solution");
  }
  cudaFreeAsync(tmp, b->stream);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (st == PE_OK && e != cudaSuccess) st = pe_cuda_fail(e, "pe_batch_get_solution");
  return st;
}

// Learned correction for every problem: the band range of each problem (its slowest and fastest
// closed-form lam, times dT), table offsets and job prefixes; the tables themselves are made by
// the next pe_batch_solve (batch_learned_tables).
extern "C" pe_status pe_batch_set_learned(pe_batch* b, const pe_mlp* m) {
  if (!b) return pe_fail(PE_EINVAL, "pe_batch_set_learned: NULL batch");
  if (!m) {
    b->mlp = nullptr;
    return PE_OK;
  }
  PE_CUDA_TRY(cudaStreamSynchronize(b->stream));
  const int NB = kBatchLearnedBands;
  std::vector<int64_t> kp, pp;
  int64_t okt = 0, oph = 0;
  for (int p = 0; p < b->P; ++p) {
    BProb& B = b->probs[p];
    double lmin = 0.0, lmax = 0.0;
    for (int a = 0; a < B.g.d; ++a) {
      const int n = B.g.n[a];
      auto ratio = [&](int j) {
        const double th = M_PI * (double)j / (double)(n + 1);
        const double sh = sin(0.5 * th);
        return ((4.0 / B.h[a]) * sh * sh) / ((B.h[a] / 3.0) * (2.0 + cos(th)));
      };
      lmin += ratio(1);
      lmax += ratio(n);
    }
    const double loglo = log(B.D * lmin * B.dT) - 1e-6, loghi = log(B.D * lmax * B.dT) + 1e-6;
    B.lloglo = loglo;
    B.lstep = (loghi - loglo) / (double)(NB - 1);
    B.oKt = okt;
    kp.push_back(okt / 2);
    okt += 2 * (int64_t)B.R * NB;
    B.oPh = oph;
    pp.push_back(oph);
    oph += (int64_t)B.R * B.N;
  }
  if (b->Kt) cudaFree(b->Kt);
  if (b->Ph) cudaFree(b->Ph);
  if (b->d_kt_prefix) cudaFree(b->d_kt_prefix);
  if (b->d_ph_prefix) cudaFree(b->d_ph_prefix);
  b->Kt = nullptr;
  b->Ph = nullptr;
  b->d_kt_prefix = nullptr;
  b->d_ph_prefix = nullptr;
  PE_TRY(balloc(&b->Kt, (size_t)okt));
  PE_TRY(balloc(&b->Ph, (size_t)oph));
  PE_TRY(upload(&b->d_kt_prefix, kp, b->stream));
  PE_TRY(upload(&b->d_ph_prefix, pp, b->stream));
  PE_CUDA_TRY(cudaMemcpyAsync(b->d_probs, b->probs.data(), sizeof(BProb) * b->P, cudaMemcpyHostToDevice, b->stream));
  PE_CUDA_TRY(cudaStreamSynchronize(b->stream));
  b->kt_jobs = okt / 2;
  b->ph_jobs = oph;
  b->mlp = m;
  return PE_OK;
}

extern "C" pe_status pe_batch_status(pe_batch* b, double* residuals, int32_t* iterations) {
  if (!b) return pe_fail(PE_EINVAL, "pe_batch_status: NULL batch");
  if (residuals)
    PE_CUDA_TRY(cudaMemcpy(residuals, b->resid, sizeof(double) * b->P, cudaMemcpyDeviceToHost));
  if (iterations)
    PE_CUDA_TRY(cudaMemcpy(iterations, b->kcount, sizeof(int) * b->P, cudaMemcpyDeviceToHost));
  return PE_OK;
}
