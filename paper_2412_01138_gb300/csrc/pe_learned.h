// Internal declarations of the learned coarse correction (pe_learned.cu).
#pragma once
#include "pe_internal.h"
#include "pe_phi.cuh"

#define PE_MLP_WIDTH 64
#define PE_LEARNED_BANDS 4096

struct pe_mlp {
  float* params = nullptr;    // float32 master weights (training)
  void* params16 = nullptr;   // float16 copy used for inference
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* loss_dev = nullptr;
  float* partial = nullptr;   // per-CTA partial gradients of the training kernel [CTAs][NPARAM + 1]
  int partial_cap = 0;        // CTAs partial has room for
  unsigned* sync = nullptr;   // grid barrier of the training kernel: arrival count, unused, error flag
  int64_t step = 0;
};

struct Nodes8 {
  double c[PE_MAX_S];
};

// per source term: sine kind flag, frequency, phase, amplitude
struct TermsW {
  int R;
  int is_sin[PE_MAX_TERMS];
  double omega[PE_MAX_TERMS];
  double phase[PE_MAX_TERMS];
  double amp[PE_MAX_TERMS];
};

// What the coarse sweep needs to add the learned term itself: the band table K^(lam, w_r)
// (Ktab, NB bands log-spaced from loglo by logstep in log(lam dT)), the phase table
// (cos, sin)(w_r T_n + phi_r) [R][N] (cs), and per term the sine flag and amplitude.
struct LearnedTerms {
  int NB;
  double loglo, logstep, dT;
  const double* Ktab;
  const float2* cs;
  int is_sin[PE_MAX_TERMS];
  double amp[PE_MAX_TERMS];
};

// Band and phase tables of the attached network (two launches); fills *L.
pe_status launch_learned_tables(pe_ctx* c, LearnedTerms* L);
pe_status launch_learned_correction(pe_ctx* c);
