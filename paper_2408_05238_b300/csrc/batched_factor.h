// Persistent batched factorization (batched_factor.cu): the randUTV step
// loop and block SVDs (Fig. 2, steps a1-a7) of many FP64 problems in one
// kernel launch, writing each problem's factors as the solver's step loop
// does.
#pragma once

#include "internal.h"

namespace lls {

// Largest block size of the persistent path (one tile of 64 columns).
constexpr int kPbMaxNb = 64;

// One problem: its input, its factor buffers (as in Factor: T with W_U below
// the diagonal, W_V in WV, per-step nb x nb T_V, T_U, U_SVD, V_SVD, R_11 and
// per-step tau_V, tau_U, sigma) and its workspace (G, W, P, P2: m x nb, ld m;
// Q, Q2: nb x n, ld nb; S: nb x nb).  flags[0] is raised for a non-finite
// entry of A, flags[1] receives LLS_ERR_SVD_NOCONV.
struct PBProblem {
  int m, n, nb, q, steps, nphases;
  uint64_t seed;
  const double* A;
  int64_t lda;
  double* T;
  int64_t ldt;
  double* WV;
  int64_t ldw;
  double *TV, *TU, *US, *VS, *Rblk;
  double *tauV, *tauU, *sigma;
  double *G, *W, *P, *P2, *Q, *Q2, *S;
  int* flags;
};

// Scheduler state (device memory, zero before the launch): per problem a
// 64-bit word (phase << 32 | tasks claimed) and a count of finished tasks of
// the current phase; the number of finished problems; the error word.
struct PBArgs {
  int count;
  const PBProblem* probs;  // device array, largest problems first
  unsigned long long* state;
  unsigned int* done;
  unsigned int* finished;
  int* err;
  long long poll_limit;  // polls of a CTA that finds no task before it gives up
};

// Phases of one problem (copy, 8 + 2q per step, then three for the SVDs).
int pb_num_phases(int m, int n, int nb, int q);
// Doubles of one problem's workspace (G, W, P, P2, Q, Q2, S).
size_t pb_workspace_doubles(int64_t m, int64_t n, int nb);
// Enqueues the persistent kernel on st.
Status batched_factor_launch(const PBArgs& args, cudaStream_t st);
// Whether this build has the persistent kernel (the host test harness, which
// links the host code with plain-loop stand-ins, emulates it).
bool batched_factor_available();

}  // namespace lls
