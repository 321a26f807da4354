// Per-kernel-family and per-phase tracing: CUDA events recorded on the
// launching stream around each launch (and around each phase of the method),
// with the algorithmic flops and bytes of the launch.
// Off unless a handle enables it; the counters mirror the paper's per-task
// time table (average time and count per elementary task).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

namespace lls {

enum TraceKind {
  kTrGemm = 0,     // dgemm_kernel
  kTrSplitK,       // split-K reduction
  kTrPanelQR,      // cooperative Householder panel
  kTrTFactor,      // compact-WY T factor
  kTrSketch,       // Philox + Box-Muller
  kTrSvd,          // batched Jacobi SVD
  kTrSmall,        // copies, rank scan, gathers, TRSM blocks
  kTrBf16Gemm,     // tcgen05 BF16 sampling GEMM
  kTrConvert,      // FP64 -> exact BF16 digit slices and TF32 split planes
  kTrOzGemm,       // FP64-accurate GEMM on tensor cores (exact BF16 slices)
  kTrTf32Gemm,     // split-operand TF32 GEMM on tensor cores (3xTF32 / TF32)
  kTrBatchedFactor,  // persistent batched factorization
  kTrThin,         // small kernels of the <= 16 right-hand-side path (T, S blocks, chunk sums)
  kTrThinN,        // thin_n_kernel: op(A) x, rows of A per thread
  kTrThinT,        // thin_t_kernel: A^T x, lanes along the rows of A
  kTrTrsmDiag,     // trsm_diag_kernel: diagonal blocks of the triangular solves
  kTrConvertBf16,  // max |A| and the BF16 copies of the trailing block for the sample
  kTrReplay,       // replay_kernel: a replay's reflector steps in one cooperative launch
  // phases of the method (each spans the kernels above that it launches)
  kTrPhaseSample,   // a1/a2 sketch and sample Y
  kTrPhaseQrY,      // a3 QR of Y and its T factor
  kTrPhaseRight,    // a4 right update, all m rows
  kTrPhasePanel,    // a5 panel QR of the block column and its T factor
  kTrPhaseLeft,     // a6 left update
  kTrPhaseSvd,      // a7 block SVDs and their updates
  kTrPhaseRank,     // a8 rank decision
  kTrPhaseNullify,  // a9 Nullify
  kTrPhaseSolve,    // a10 solve
  kTrPhaseRefine,   // iterative refinement after the solve
  kTrCount
};
constexpr int kTrFirstPhase = kTrPhaseSample;

const char* trace_kind_name(int k);

struct Tracer {
  struct Rec {
    int kind;
    cudaEvent_t a, b;
    double flops, bytes;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  int64_t launches[kTrCount] = {};
  double seconds[kTrCount] = {};
  double flops[kTrCount] = {};
  double bytes[kTrCount] = {};
  cudaEvent_t get();
  void flush();  // waits for the recorded events and accumulates
  void reset();
  ~Tracer();
};

// The tracer of the handle currently running on this thread (or null).
extern thread_local Tracer* g_tracer;
// Kernels launched by the library since load (all handles, all threads).
extern std::atomic<int64_t> g_launches;
// Device allocations made by DevBuf (lls_alloc_count).
extern std::atomic<int64_t> g_allocs;
// Poll limit of the grid barrier of the cooperative panel kernels
// (kBarrierSpinLimit; lls_debug_barrier_limit lowers it for tests).
extern std::atomic<long long> g_barrier_spin_limit;

// Records a start event in the constructor and a stop event in the
// destructor when a tracer is active.
struct TraceScope {
  Tracer* t;
  int kind;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  double flops, bytes;
  TraceScope(int k, cudaStream_t s, double f = 0.0, double by = 0.0)
      : t(g_tracer), kind(k), st(s), flops(f), bytes(by) {
    if (t) {
      a = t->get();
      cudaEventRecord(a, st);
    }
  }
  ~TraceScope() {
    if (t) {
      cudaEvent_t b = t->get();
      cudaEventRecord(b, st);
      t->recs.push_back(Tracer::Rec{kind, a, b, flops, bytes});
    }
  }
};

}  // namespace lls
