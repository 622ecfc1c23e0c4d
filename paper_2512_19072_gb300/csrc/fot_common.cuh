// Shared device helpers and the context layout of the FOT library (internal header).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "../../include/fot.h"

namespace fot {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// 2^x with the MUFU.EX2 unit (PTX ex2.approx.ftz.f32: relative error ~2^-22, results
// below 2^-126 flush to zero, ex2(-inf) = 0).
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// log2(x) with the MUFU.LG2 unit (PTX lg2.approx.ftz.f32: absolute error about 2^-22 for
// normal x; subnormal x flushes to zero and gives -inf).
__device__ __forceinline__ float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Latch the first device-side error of a context (later errors are dropped).
__device__ __forceinline__ void raise_error(int* err, int code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ bool error_latched(const int* err) {
  return *(volatile const int*)err != 0;
}

// Optional per-kernel-class timing of the Sinkhorn loop (fot_set_kernel_timing): while a
// context with timing on runs its loop, g_ktimer points at its timer and every launch site
// brackets its kernel with a pair of events; fot_kernel_times sums them per class.
enum KernelClass : int {
  kKPlan = FOT_KERNEL_PLAN,       // band_plan_kernel
  kKBand = FOT_KERNEL_BAND,       // band_pass_kernel
  kKTensor = FOT_KERNEL_TENSOR,   // tc_pass_kernel
  kKDense = FOT_KERNEL_DENSE,     // axis_pass_kernel (dense exact pass)
  kKClasses = FOT_KERNEL_CLASSES
};

struct KernelTimer {
  std::vector<cudaEvent_t> ev;   // (start, end) pairs, created on first use and reused
  std::vector<int> cls;          // class of each pair
  size_t used = 0;               // pairs recorded since the last read
  bool failed = false;           // an event could not be created or recorded
};

extern thread_local KernelTimer* g_ktimer;
void ktimer_begin(cudaStream_t s, int cls);   // no-op unless g_ktimer is set
void ktimer_end(cudaStream_t s);

}  // namespace fot

// Context (opaque to callers).  Every device buffer is owned here.
struct fot_ctx {
  int rows = 0, cols = 0, device = 0, precision = 0;
  cudaStream_t stream = nullptr;
  // device images, rows x cols unless noted
  float* la = nullptr;       // log a (natural), -inf on zero mass
  float* lb = nullptr;       // log b
  float* f = nullptr;        // source potential, px^2
  float* psi = nullptr;      // target potential, px^2
  float* R = nullptr;        // axis-pass intermediate, transposed (cols x rows), log2 units
  float* R2 = nullptr;       // second intermediate (moments / stats), cols x rows
  float* S_last = nullptr;   // natural-log kernel sum of the last u-update (Eqs. 9-10)
  float* tmp = nullptr;      // rows x cols scratch (stats, moments)
  float* tmp2 = nullptr;     // rows x cols scratch
  float* phi = nullptr;      // rows x cols phase (host-buffer entry point)
  float* col_phi = nullptr;  // rows: phase along the centre column
  float* plan = nullptr;     // per-(row, 16-output tile) window plan of a banded pass, 3 words each
  double* red = nullptr;     // reduction scratch (partials + results)
  float* lam_hat = nullptr;  // cFOT: the spectra of lambda (allocated by the first cFOT solve)
  int* err = nullptr;        // latched device status
  unsigned long long* terms = nullptr;  // device counters of evaluated (row, output, m) terms on
                                        // the CUDA cores: [0] banded GEMM, [1] exact windows
  int64_t host_terms = 0;    // terms of passes whose count is known on the host (dense)
  int red_blocks = 0;
  // host-side state
  double dx = 0.0;
  double eps_last = 0.0;
  bool have_problem = false;
  bool have_solution = false;
  int64_t launches = 0;
  // CUDA events bracketing the last Sinkhorn loop (only axis passes run inside it)
  cudaEvent_t ev_loop0 = nullptr, ev_loop1 = nullptr;
  int64_t loop_passes = 0;   // axis-pass launches inside the last loop
  std::vector<double> sched; // eps (px^2) of every iteration since the last fot_solve
  // the Sinkhorn loop as a CUDA graph (captured on `cap`, replayed on `stream`) and the
  // per-iteration eps (px^2) it was captured for
  cudaStream_t cap = nullptr;
  cudaGraphExec_t loop_exec = nullptr;
  std::vector<double> loop_key;
  int64_t loop_kernels = 0;
  // mixed-precision (tensor-core) resources, owned by fot_tc.cu
  void* tc = nullptr;
  fot::KernelTimer* ktimer = nullptr;   // per-kernel-class loop timing, when switched on
};

namespace fot {
// Implemented in fot_api.cu
cudaError_t launch_error_check(fot_ctx* c);
}  // namespace fot
