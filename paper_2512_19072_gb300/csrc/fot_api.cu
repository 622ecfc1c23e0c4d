// C ABI of the FOT library (include/fot.h): context lifetime, argument checking, the
// Sinkhorn loop of Algorithm 1 and the phase step, on top of the kernels in fot_simt.cu
// (exact FP32 passes), fot_tc.cu (tensor-core passes) and fot_ctransform.cu.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "fot_common.cuh"

namespace fot {
void half_step_simt(fot_ctx* c, const float* pot_in, const float* lmarg, double eps,
                    float* pot_out, float* logsum, float* tmp);
cudaError_t simt_configure();
void moments_simt(fot_ctx* c, const float* psi, const float* S, double eps, double dx,
                  float* Dx, float* Dy);
void set_problem_simt(fot_ctx* c, const float* g, const float* G, float* psi0, float psi0_val);
void fill(fot_ctx* c, float* p, size_t N, float v);
void source_stats(fot_ctx* c, const float* f, const float* S, double eps, double* out);
bool intensity_supported(int rows, int cols);
bool cfot_supported(int rows, int cols);
void cfot_run(fot_ctx* c, const double* eps_px, int iters);
size_t cfot_spectrum_floats();
void intensity_loss_gpu(fot_ctx* c, const float* phi, double* out);
void marginal_stats(fot_ctx* c, const float* f, const float* S, const float* psi,
                    const float* T, double eps, double* out);
void integrate_phase(fot_ctx* c, const float* Dx, const float* Dy, double dx, float* phi);
void c_transform_envelope(fot_ctx* c, const float* pot_in, float* out);
void half_step_band(fot_ctx* c, const float* pot_in, const float* lmarg, double eps,
                    float* pot_out, float* logsum, float* tmp);
// tensor-core path (fot_tc.cu)
bool tc_supported(int rows, int cols);
int tc_create(fot_ctx* c);
void tc_destroy(fot_ctx* c);
void half_step_tc(fot_ctx* c, const float* pot_in, const float* lmarg, double eps,
                  float* pot_out, float* logsum);
int64_t tc_terms(fot_ctx* c);
void tc_begin(fot_ctx* c);
}  // namespace fot

using namespace fot;

static const int kMaxDim = 4096;

namespace fot {
thread_local KernelTimer* g_ktimer = nullptr;

void ktimer_begin(cudaStream_t s, int cls) {
  KernelTimer* t = g_ktimer;
  if (!t || t->failed) return;
  const size_t need = 2 * (t->used + 1);
  while (t->ev.size() < need) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      t->failed = true;
      return;
    }
    t->ev.push_back(e);
  }
  if (t->cls.size() < t->used + 1) t->cls.resize(t->used + 1);
  t->cls[t->used] = cls;
  if (cudaEventRecord(t->ev[2 * t->used], s) != cudaSuccess) t->failed = true;
}

void ktimer_end(cudaStream_t s) {
  KernelTimer* t = g_ktimer;
  if (!t || t->failed) return;
  if (cudaEventRecord(t->ev[2 * t->used + 1], s) != cudaSuccess) t->failed = true;
  ++t->used;
}
}  // namespace fot

static void ktimer_free(fot_ctx* c) {
  if (!c->ktimer) return;
  for (cudaEvent_t e : c->ktimer->ev) cudaEventDestroy(e);
  delete c->ktimer;
  c->ktimer = nullptr;
}

#define FOT_CUDA(call)                                \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return FOT_ECUDA;          \
  } while (0)

static fot_status check_launch(fot_ctx* c) {
  (void)c;
  return cudaGetLastError() == cudaSuccess ? FOT_OK : FOT_ECUDA;
}

static fot_status read_latched(fot_ctx* c) {
  int e = 0;
  FOT_CUDA(cudaMemcpyAsync(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  FOT_CUDA(cudaStreamSynchronize(c->stream));
  return (fot_status)e;
}

static bool bad_ptr(const void* p) { return p == nullptr; }

static double eps_px(const fot_ctx* c, double e, int units) {
  if (units == FOT_EPS_PAPER) {
    const double n = (double)(c->rows > c->cols ? c->rows : c->cols);
    return e * n * n;
  }
  return e;
}

static fot_status check_eps(const double* eps, int n_eps, int iters) {
  if (iters < 0 || eps == nullptr || n_eps < 1) return FOT_EINVAL;
  if (!(n_eps == 1 || n_eps == iters)) return FOT_EINVAL;
  for (int i = 0; i < n_eps; ++i)
    if (!(eps[i] > 0.0) || !isfinite(eps[i])) return FOT_EINVAL;
  return FOT_OK;
}

extern "C" {

const char* fot_status_string(fot_status s) {
  switch (s) {
    case FOT_OK: return "ok";
    case FOT_EINVAL: return "invalid argument or input (negative / non-finite amplitude)";
    case FOT_ENOMEM: return "out of memory";
    case FOT_ECUDA: return "CUDA runtime error";
    case FOT_ENONFINITE: return "non-finite potential during the iteration";
    case FOT_ETIMEOUT: return "bounded device wait timed out";
    case FOT_EMASS: return "zero total power in g or G";
    case FOT_EUNSUPPORTED: return "unsupported precision or shape";
    case FOT_ESTATE: return "call out of order";
  }
  return "unknown status";
}

fot_status fot_create(fot_ctx** out, int rows, int cols, int precision, int device,
                      void* cuda_stream) {
  if (!out) return FOT_EINVAL;
  *out = nullptr;
  if (rows < 1 || cols < 1 || rows > kMaxDim || cols > kMaxDim) return FOT_EINVAL;
  if (precision != FOT_FP32 && precision != FOT_MIXED && precision != FOT_FP32_DENSE &&
      precision != FOT_BF16)
    return FOT_EINVAL;
  if (getenv("FOT_FAULT_INJECT_ENOMEM")) return FOT_ENOMEM;   // host-side fault injection
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FOT_EINVAL;
  FOT_CUDA(cudaSetDevice(device));
  fot_ctx* c = new (std::nothrow) fot_ctx();
  if (!c) return FOT_ENOMEM;
  c->rows = rows;
  c->cols = cols;
  c->device = device;
  c->precision = precision;
  c->stream = (cudaStream_t)cuda_stream;
  const size_t N = (size_t)rows * cols;
  c->red_blocks = (int)((N + 1023) / 1024 < 1024 ? (N + 1023) / 1024 : 1024);
  if (c->red_blocks < 1) c->red_blocks = 1;
  float** bufs[] = {&c->la, &c->lb, &c->f, &c->psi, &c->R, &c->R2, &c->S_last, &c->tmp, &c->tmp2,
                    &c->phi};
  bool ok = true;
  for (float** b : bufs) ok = ok && cudaMalloc((void**)b, N * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&c->col_phi, (size_t)rows * sizeof(float)) == cudaSuccess;
  // the per-(16-output tile, row) plan of the larger banded pass (3 words each; rows padded to
  // a multiple of 128, the plan's tile-major stride)
  const size_t pr = (size_t)(rows + 127) / 128 * 128, pc = (size_t)(cols + 127) / 128 * 128;
  const size_t plan_words = 3 * std::max(pr * ((cols + 15) / 16), pc * ((rows + 15) / 16));
  ok = ok && cudaMalloc((void**)&c->plan, plan_words * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&c->red, (size_t)(4 * c->red_blocks + 16) * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&c->err, sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&c->terms, 2 * sizeof(unsigned long long)) == cudaSuccess;
  if (ok) ok = cudaMemsetAsync(c->terms, 0, 2 * sizeof(unsigned long long), c->stream) == cudaSuccess;
  if (ok) ok = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream) == cudaSuccess;
  if (ok) ok = cudaEventCreate(&c->ev_loop0) == cudaSuccess && cudaEventCreate(&c->ev_loop1) == cudaSuccess;
  if (ok && simt_configure() != cudaSuccess) {   // per-device kernel attributes
    cudaGetLastError();
    fot_destroy(c);
    return FOT_ECUDA;
  }
  if (ok && (precision == FOT_MIXED || precision == FOT_BF16)) {
    if (!tc_supported(rows, cols)) {
      fot_destroy(c);
      return FOT_EUNSUPPORTED;
    }
    ok = tc_create(c) == 0;
  }
  if (!ok) {
    cudaGetLastError();
    fot_destroy(c);
    return FOT_ENOMEM;
  }
  *out = c;
  return FOT_OK;
}

void fot_destroy(fot_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->tc) tc_destroy(c);
  ktimer_free(c);
  if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
  if (c->cap) cudaStreamDestroy(c->cap);
  float* bufs[] = {c->la, c->lb, c->f, c->psi, c->R, c->R2, c->S_last, c->tmp, c->tmp2, c->phi,
                   c->col_phi, c->plan};
  for (float* b : bufs)
    if (b) cudaFree(b);
  if (c->red) cudaFree(c->red);
  if (c->lam_hat) cudaFree(c->lam_hat);
  if (c->err) cudaFree(c->err);
  if (c->terms) cudaFree(c->terms);
  if (c->ev_loop0) cudaEventDestroy(c->ev_loop0);
  if (c->ev_loop1) cudaEventDestroy(c->ev_loop1);
  delete c;
}

fot_status fot_set_stream(fot_ctx* c, void* s) {
  if (!c) return FOT_EINVAL;
  c->stream = (cudaStream_t)s;
  return FOT_OK;
}

int64_t fot_launch_count(const fot_ctx* c) { return c ? c->launches : -1; }

fot_status fot_work_count(fot_ctx* c, int64_t* terms_out, int64_t* tensor_terms_out) {
  if (!c || !terms_out) return FOT_EINVAL;
  FOT_CUDA(cudaSetDevice(c->device));
  int64_t w[4];
  const fot_status s = fot_work_split(c, w);
  if (s != FOT_OK) return s;
  *terms_out = w[0] + w[1] + w[2] + w[3];
  if (tensor_terms_out) *tensor_terms_out = w[2];
  return FOT_OK;
}

fot_status fot_work_split(fot_ctx* c, int64_t* out4) {
  if (!c || !out4) return FOT_EINVAL;
  FOT_CUDA(cudaSetDevice(c->device));
  unsigned long long t[2] = {0, 0};
  FOT_CUDA(cudaMemcpyAsync(t, c->terms, sizeof(t), cudaMemcpyDeviceToHost, c->stream));
  FOT_CUDA(cudaStreamSynchronize(c->stream));
  out4[0] = (int64_t)t[0];
  out4[1] = (int64_t)t[1];
  out4[2] = c->tc ? tc_terms(c) : 0;
  out4[3] = c->host_terms;
  return FOT_OK;
}

fot_status fot_set_kernel_timing(fot_ctx* c, int on) {
  if (!c) return FOT_EINVAL;
  if (!on) {
    if (c->ktimer) {
      FOT_CUDA(cudaSetDevice(c->device));
      FOT_CUDA(cudaStreamSynchronize(c->stream));
    }
    ktimer_free(c);
    return FOT_OK;
  }
  if (!c->ktimer) {
    c->ktimer = new (std::nothrow) KernelTimer();
    if (!c->ktimer) return FOT_ENOMEM;
  }
  return FOT_OK;
}

fot_status fot_kernel_times(fot_ctx* c, double* ms_out, int64_t* launches_out) {
  if (!c || !ms_out || !launches_out) return FOT_EINVAL;
  for (int k = 0; k < kKClasses; ++k) {
    ms_out[k] = 0.0;
    launches_out[k] = 0;
  }
  KernelTimer* t = c->ktimer;
  if (!t) return FOT_ESTATE;
  FOT_CUDA(cudaSetDevice(c->device));
  if (t->failed) {
    t->used = 0;
    t->failed = false;
    return FOT_ECUDA;
  }
  if (t->used) FOT_CUDA(cudaEventSynchronize(t->ev[2 * t->used - 1]));
  for (size_t i = 0; i < t->used; ++i) {
    float ms = 0.f;
    FOT_CUDA(cudaEventElapsedTime(&ms, t->ev[2 * i], t->ev[2 * i + 1]));
    ms_out[t->cls[i]] += ms;
    launches_out[t->cls[i]] += 1;
  }
  t->used = 0;
  return FOT_OK;
}

fot_status fot_loop_time(fot_ctx* c, double* ms_out, int64_t* passes_out) {
  if (!c || !ms_out) return FOT_EINVAL;
  if (!c->have_solution) return FOT_ESTATE;
  FOT_CUDA(cudaSetDevice(c->device));
  FOT_CUDA(cudaEventSynchronize(c->ev_loop1));
  float ms = 0.f;
  FOT_CUDA(cudaEventElapsedTime(&ms, c->ev_loop0, c->ev_loop1));
  *ms_out = ms;
  if (passes_out) *passes_out = c->loop_passes;
  return FOT_OK;
}

fot_status fot_set_problem(fot_ctx* c, const float* g, const float* G) {
  if (!c || bad_ptr(g) || bad_ptr(G)) return FOT_EINVAL;
  FOT_CUDA(cudaSetDevice(c->device));
  FOT_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
  set_problem_simt(c, g, G, nullptr, 0.f);
  c->have_problem = true;
  c->have_solution = false;
  return check_launch(c);
}

static void half_step(fot_ctx* c, const float* pot_in, const float* lmarg, double eps,
                      float* pot_out, float* logsum) {
  if ((c->precision == FOT_MIXED || c->precision == FOT_BF16) && c->tc)
    half_step_tc(c, pot_in, lmarg, eps, pot_out, logsum);
  else if (c->precision == FOT_FP32_DENSE)
    half_step_simt(c, pot_in, lmarg, eps, pot_out, logsum, c->R);
  else
    half_step_band(c, pot_in, lmarg, eps, pot_out, logsum, c->R);
}

// the loop of Algorithm 1 for per-iteration eps e (px^2), enqueued on c->stream
static void loop_body(fot_ctx* c, const std::vector<double>& e) {
  const int iters = (int)e.size();
  if (c->tc) tc_begin(c);
  for (int t = 0; t < iters; ++t) {
    // Eq. 7: f = eps (log a - log(Lambda V Lambda)); keep S of the last u-update (Eqs. 9-10)
    half_step(c, c->psi, c->la, e[(size_t)t], c->f, t == iters - 1 ? c->S_last : nullptr);
    // Eq. 8: psi = eps (log b - log(Lambda u Lambda))
    half_step(c, c->f, c->lb, e[(size_t)t], c->psi, nullptr);
  }
}

// Capture the loop for schedule e into c->loop_exec (on the context's private stream: the
// legacy default stream cannot be captured).  False when capture is not possible.
static bool capture_loop(fot_ctx* c, const std::vector<double>& e) {
  if (c->loop_exec) {
    cudaGraphExecDestroy(c->loop_exec);
    c->loop_exec = nullptr;
    c->loop_key.clear();
  }
  if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    c->cap = nullptr;
    return false;
  }
  cudaStream_t user = c->stream;
  const int64_t l0 = c->launches;
  if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  c->stream = c->cap;
  loop_body(c, e);
  c->stream = user;
  cudaGraph_t g = nullptr;
  const bool ok = cudaStreamEndCapture(c->cap, &g) == cudaSuccess && g &&
                  cudaGraphInstantiate(&c->loop_exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  c->loop_kernels = c->launches - l0;
  c->launches = l0;
  if (!ok) {
    cudaGetLastError();
    c->loop_exec = nullptr;
    return false;
  }
  c->loop_key = e;
  return true;
}

// The Sinkhorn loop.  It is replayed as a CUDA graph when kernel timing is off: captured on
// first use for a schedule (or when at least 16 iterations make the capture pay for itself in
// the call) and reused while the schedule stays the same.
static fot_status run_iterations(fot_ctx* c, const double* eps, int n_eps, int units, int iters) {
  std::vector<double> e((size_t)iters);
  for (int t = 0; t < iters; ++t) e[(size_t)t] = eps_px(c, eps[n_eps == 1 ? 0 : t], units);
  const int64_t l0 = c->launches;
  bool graph = c->ktimer == nullptr && iters > 0;
  if (graph && !(c->loop_exec && c->loop_key == e)) graph = (iters >= 16 || c->loop_key.empty()) && capture_loop(c, e);
  if (graph) {
    cudaEventRecord(c->ev_loop0, c->stream);
    if (cudaGraphLaunch(c->loop_exec, c->stream) != cudaSuccess) return FOT_ECUDA;
    cudaEventRecord(c->ev_loop1, c->stream);
    c->launches += c->loop_kernels;
    // the host no longer knows which B table the device holds: the next pass rewrites it
    if (c->tc) tc_begin(c);
  } else {
    g_ktimer = c->ktimer;                  // null unless kernel timing is on
    cudaEventRecord(c->ev_loop0, c->stream);
    loop_body(c, e);
    cudaEventRecord(c->ev_loop1, c->stream);
    g_ktimer = nullptr;
  }
  for (int t = 0; t < iters; ++t) c->sched.push_back(e[(size_t)t]);
  if (iters > 0) c->eps_last = e[(size_t)iters - 1];
  c->loop_passes = c->launches - l0;
  if (iters > 0) c->have_solution = true;
  return check_launch(c);
}

// load the problem and the Algorithm 1 start (arguments already checked)
static fot_status start_solve(fot_ctx* c, const float* g, const float* G, double dx,
                              const double* eps, int eps_units) {
  FOT_CUDA(cudaSetDevice(c->device));
  FOT_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
  const double n = (double)(c->rows > c->cols ? c->rows : c->cols);
  c->dx = dx > 0.0 ? dx : 1.0 / sqrt(n);
  // Algorithm 1 initialisation: V = 1/(rows cols)  ->  psi0 = eps_0 log(1/(rows cols))
  const double e0 = eps_px(c, eps[0], eps_units);
  const float psi0 = (float)(e0 * log(1.0 / ((double)c->rows * c->cols)));
  set_problem_simt(c, g, G, c->psi, psi0);
  c->have_problem = true;
  c->have_solution = false;
  c->sched.clear();
  return FOT_OK;
}

fot_status fot_solve(fot_ctx* c, const float* g, const float* G, double dx, const double* eps,
                     int n_eps, int eps_units, int iters) {
  if (!c || bad_ptr(g) || bad_ptr(G)) return FOT_EINVAL;
  fot_status s = check_eps(eps, n_eps, iters);
  if (s != FOT_OK) return s;
  if (eps_units != FOT_EPS_PX2 && eps_units != FOT_EPS_PAPER) return FOT_EINVAL;
  if (!isfinite(dx)) return FOT_EINVAL;
  s = start_solve(c, g, G, dx, eps, eps_units);
  if (s != FOT_OK) return s;
  return run_iterations(c, eps, n_eps, eps_units, iters);
}

fot_status fot_cfot_solve(fot_ctx* c, const float* g, const float* G, double dx, const double* eps,
                          int n_eps, int eps_units, int iters) {
  if (!c || bad_ptr(g) || bad_ptr(G) || iters < 1) return FOT_EINVAL;
  fot_status s = check_eps(eps, n_eps, iters);
  if (s != FOT_OK) return s;
  if (eps_units != FOT_EPS_PX2 && eps_units != FOT_EPS_PAPER) return FOT_EINVAL;
  if (!isfinite(dx)) return FOT_EINVAL;
  if (!cfot_supported(c->rows, c->cols)) return FOT_EUNSUPPORTED;
  FOT_CUDA(cudaSetDevice(c->device));
  if (!c->lam_hat && cudaMalloc((void**)&c->lam_hat, cfot_spectrum_floats() * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    c->lam_hat = nullptr;
    return FOT_ENOMEM;
  }
  s = start_solve(c, g, G, dx, eps, eps_units);
  if (s != FOT_OK) return s;
  std::vector<double> e((size_t)iters);
  for (int t = 0; t < iters; ++t) e[(size_t)t] = eps_px(c, eps[n_eps == 1 ? 0 : t], eps_units);
  const int64_t l0 = c->launches;
  cudaEventRecord(c->ev_loop0, c->stream);
  cfot_run(c, e.data(), iters);
  cudaEventRecord(c->ev_loop1, c->stream);
  c->loop_passes = c->launches - l0;
  c->eps_last = e[(size_t)iters - 1];
  c->have_solution = true;              // no schedule recorded: fot_backward does not apply
  return check_launch(c);
}

fot_status fot_solve_tol(fot_ctx* c, const float* g, const float* G, double dx, const double* eps,
                         int n_eps, int eps_units, int max_iters, double tol, int check_every,
                         int* iters_out, double* tv_out) {
  if (!c || bad_ptr(g) || bad_ptr(G) || !iters_out) return FOT_EINVAL;
  if (max_iters < 1 || check_every < 1 || !(tol >= 0.0) || !isfinite(tol)) return FOT_EINVAL;
  fot_status s = check_eps(eps, n_eps, max_iters);
  if (s != FOT_OK) return s;
  if (eps_units != FOT_EPS_PX2 && eps_units != FOT_EPS_PAPER) return FOT_EINVAL;
  if (!isfinite(dx)) return FOT_EINVAL;
  s = start_solve(c, g, G, dx, eps, eps_units);
  if (s != FOT_OK) return s;
  int done = 0;
  double tv = INFINITY;
  while (done < max_iters) {
    const int k = max_iters - done < check_every ? max_iters - done : check_every;
    s = run_iterations(c, n_eps == 1 ? eps : eps + done, n_eps == 1 ? 1 : k, eps_units, k);
    if (s != FOT_OK) return s;
    done += k;
    // the row sums of Gamma(f, psi) at eps_last: S(psi) from one more u-half (its potentials
    // are thrown away), then sum |exp(f/eps + S) - a| in FP64
    half_step(c, c->psi, c->la, c->eps_last, c->tmp2, c->tmp);
    double* out = c->red + 4 * c->red_blocks;
    source_stats(c, c->f, c->tmp, c->eps_last, out);
    double h[3];
    FOT_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    s = read_latched(c);
    if (s != FOT_OK) return s;
    tv = h[0];
    if (tv <= tol) break;
  }
  *iters_out = done;
  if (tv_out) *tv_out = tv;
  return FOT_OK;
}

// the marginal violation sum |Gamma 1 - a| of the context's iterate (f, psi) at eps_last: the
// measurement of fot_solve_tol (synchronising)
static fot_status source_violation(fot_ctx* c, double* tv) {
  half_step(c, c->psi, c->la, c->eps_last, c->tmp2, c->tmp);
  double* out = c->red + 4 * c->red_blocks;
  source_stats(c, c->f, c->tmp, c->eps_last, out);
  double h[3];
  FOT_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  fot_status s = read_latched(c);
  if (s != FOT_OK) return s;
  *tv = h[0];
  return isfinite(h[0]) ? FOT_OK : FOT_ENONFINITE;
}

fot_status fot_select_eps(fot_ctx* c, const float* g, const float* G, double dx, const double* cand,
                          int n_cand, int eps_units, int probe_iters, int check_every,
                          double min_decrease, int use_cfot, int* index_out, double* tv_out) {
  if (!c || bad_ptr(g) || bad_ptr(G) || !cand || n_cand < 1 || !index_out) return FOT_EINVAL;
  if (check_every < 1 || probe_iters <= check_every || !(min_decrease >= 0.0) || !(min_decrease < 1.0))
    return FOT_EINVAL;
  if (eps_units != FOT_EPS_PX2 && eps_units != FOT_EPS_PAPER) return FOT_EINVAL;
  if (!isfinite(dx)) return FOT_EINVAL;
  for (int i = 0; i < n_cand; ++i)
    if (!(cand[i] > 0.0) || !isfinite(cand[i])) return FOT_EINVAL;
  if (use_cfot && !cfot_supported(c->rows, c->cols)) return FOT_EUNSUPPORTED;
  *index_out = -1;
  std::vector<int> order((size_t)n_cand);
  for (int i = 0; i < n_cand; ++i) order[(size_t)i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return cand[x] < cand[y]; });
  for (int i : order) {
    const double e = cand[i];
    // the first check_every iterations, then the rest of the probe from the same start
    double tv1 = INFINITY, tv2 = INFINITY;
    fot_status s = use_cfot ? fot_cfot_solve(c, g, G, dx, &e, 1, eps_units, check_every)
                            : fot_solve(c, g, G, dx, &e, 1, eps_units, check_every);
    if (s == FOT_OK) s = source_violation(c, &tv1);
    if (s == FOT_OK)
      s = use_cfot ? fot_cfot_solve(c, g, G, dx, &e, 1, eps_units, probe_iters)
                   : fot_resume(c, &e, 1, eps_units, probe_iters - check_every);
    if (s == FOT_OK) s = source_violation(c, &tv2);
    if (s == FOT_ENONFINITE) continue;               // unstable at this eps: try the next larger
    if (s != FOT_OK) return s;
    if (tv2 <= (1.0 - min_decrease) * tv1) {
      *index_out = i;
      if (tv_out) *tv_out = tv2;
      return FOT_OK;
    }
  }
  return FOT_OK;
}

fot_status fot_resume(fot_ctx* c, const double* eps, int n_eps, int eps_units, int iters) {
  if (!c) return FOT_EINVAL;
  if (!c->have_problem) return FOT_ESTATE;
  fot_status s = check_eps(eps, n_eps, iters);
  if (s != FOT_OK) return s;
  FOT_CUDA(cudaSetDevice(c->device));
  return run_iterations(c, eps, n_eps, eps_units, iters);
}

fot_status fot_sync(fot_ctx* c) {
  if (!c) return FOT_EINVAL;
  FOT_CUDA(cudaSetDevice(c->device));
  return read_latched(c);
}

fot_status fot_potentials(fot_ctx* c, float* f_out, float* psi_out) {
  if (!c) return FOT_EINVAL;
  if (!c->have_solution) return FOT_ESTATE;
  FOT_CUDA(cudaSetDevice(c->device));
  const size_t bytes = (size_t)c->rows * c->cols * sizeof(float);
  if (f_out) FOT_CUDA(cudaMemcpyAsync(f_out, c->f, bytes, cudaMemcpyDeviceToDevice, c->stream));
  if (psi_out) FOT_CUDA(cudaMemcpyAsync(psi_out, c->psi, bytes, cudaMemcpyDeviceToDevice, c->stream));
  return read_latched(c);
}

fot_status fot_set_potentials(fot_ctx* c, const float* f, const float* psi) {
  if (!c || bad_ptr(psi)) return FOT_EINVAL;
  if (!c->have_problem) return FOT_ESTATE;
  c->sched.clear();   // the backward recomputes from the standard start: no longer valid
  FOT_CUDA(cudaSetDevice(c->device));
  const size_t bytes = (size_t)c->rows * c->cols * sizeof(float);
  if (f) FOT_CUDA(cudaMemcpyAsync(c->f, f, bytes, cudaMemcpyDeviceToDevice, c->stream));
  FOT_CUDA(cudaMemcpyAsync(c->psi, psi, bytes, cudaMemcpyDeviceToDevice, c->stream));
  return FOT_OK;
}

fot_status fot_phase(fot_ctx* c, float* phi_out, float* dphidx_out, float* dphidy_out) {
  if (!c) return FOT_EINVAL;
  if (!c->have_solution) return FOT_ESTATE;
  FOT_CUDA(cudaSetDevice(c->device));
  float* Dx = dphidx_out ? dphidx_out : c->tmp;
  float* Dy = dphidy_out ? dphidy_out : c->tmp2;
  moments_simt(c, c->psi, c->S_last, c->eps_last, c->dx, Dx, Dy);
  if (phi_out) integrate_phase(c, Dx, Dy, c->dx, phi_out);
  fot_status s = check_launch(c);
  if (s != FOT_OK) return s;
  return read_latched(c);
}

fot_status fot_moments(fot_ctx* c, const float* psi, const float* logsum_u, double eps, double dx,
                       float* phi_out, float* dphidx_out, float* dphidy_out) {
  if (!c || bad_ptr(psi) || bad_ptr(logsum_u) || !(eps > 0.0) || !isfinite(eps) || !isfinite(dx))
    return FOT_EINVAL;
  FOT_CUDA(cudaSetDevice(c->device));
  const double n = (double)(c->rows > c->cols ? c->rows : c->cols);
  const double h = dx > 0.0 ? dx : 1.0 / sqrt(n);
  float* Dx = dphidx_out ? dphidx_out : c->tmp;
  float* Dy = dphidy_out ? dphidy_out : c->tmp2;
  moments_simt(c, psi, logsum_u, eps, h, Dx, Dy);
  if (phi_out) integrate_phase(c, Dx, Dy, h, phi_out);
  fot_status s = check_launch(c);
  if (s != FOT_OK) return s;
  return read_latched(c);
}

fot_status fot_marginal_error(fot_ctx* c, double* l1_out, double* dual_out) {
  if (!c || !l1_out) return FOT_EINVAL;
  if (!c->have_solution) return FOT_ESTATE;
  FOT_CUDA(cudaSetDevice(c->device));
  const double e = c->eps_last;
  // exact FP32 evaluation of log(Lambda V Lambda) and log(Lambda u Lambda) on the stored
  // potentials; tmp2 receives throw-away potentials
  half_step_simt(c, c->psi, c->la, e, c->tmp2, c->tmp, c->R);    // tmp = S(psi)
  half_step_simt(c, c->f, c->lb, e, c->tmp2, c->R2, c->R);       // R2 = T(f)
  double* out = c->red + 4 * c->red_blocks;
  marginal_stats(c, c->f, c->tmp, c->psi, c->R2, e, out);
  double h[6];
  FOT_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  fot_status s = read_latched(c);
  if (s != FOT_OK) return s;
  *l1_out = h[0] + h[3];
  if (dual_out) *dual_out = h[2] + h[5] - e * h[1] + e;
  return FOT_OK;
}

fot_status fot_intensity_loss(fot_ctx* c, const float* phi, double* loss_out, float* intensity_out) {
  if (!c || bad_ptr(phi) || !loss_out) return FOT_EINVAL;
  if (!c->have_problem) return FOT_ESTATE;
  if (!intensity_supported(c->rows, c->cols)) return FOT_EUNSUPPORTED;
  FOT_CUDA(cudaSetDevice(c->device));
  double* out = c->red + 4 * c->red_blocks + 8;      // [0] loss, [1] total power
  intensity_loss_gpu(c, phi, out);
  if (intensity_out)
    FOT_CUDA(cudaMemcpyAsync(intensity_out, c->tmp, (size_t)c->rows * c->cols * sizeof(float),
                             cudaMemcpyDeviceToDevice, c->stream));
  double h[2];
  FOT_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  fot_status s = read_latched(c);
  if (s != FOT_OK) return s;
  *loss_out = h[0];
  return FOT_OK;
}

fot_status fot_u_update(fot_ctx* c, const float* psi_in, double eps, float* f_out,
                        float* logsum_out) {
  if (!c || bad_ptr(psi_in) || bad_ptr(f_out) || !(eps > 0.0) || !isfinite(eps)) return FOT_EINVAL;
  if (!c->have_problem) return FOT_ESTATE;
  FOT_CUDA(cudaSetDevice(c->device));
  if (c->tc) tc_begin(c);
  half_step(c, psi_in, c->la, eps, f_out, logsum_out);
  return check_launch(c);
}

fot_status fot_v_update(fot_ctx* c, const float* f_in, double eps, float* psi_out,
                        float* logsum_out) {
  if (!c || bad_ptr(f_in) || bad_ptr(psi_out) || !(eps > 0.0) || !isfinite(eps)) return FOT_EINVAL;
  if (!c->have_problem) return FOT_ESTATE;
  FOT_CUDA(cudaSetDevice(c->device));
  if (c->tc) tc_begin(c);
  half_step(c, f_in, c->lb, eps, psi_out, logsum_out);
  return check_launch(c);
}

fot_status fot_c_transform(fot_ctx* c, const float* pot_in, float* out) {
  if (!c || bad_ptr(pot_in) || bad_ptr(out)) return FOT_EINVAL;
  FOT_CUDA(cudaSetDevice(c->device));
  c_transform_envelope(c, pot_in, out);
  return check_launch(c);
}

fot_status fot_solve_phase_host(fot_ctx* c, const float* g_host, const float* G_host, double dx,
                                const double* eps, int n_eps, int eps_units, int iters,
                                float* phi_host) {
  if (!c || !g_host || !G_host || !phi_host) return FOT_EINVAL;
  FOT_CUDA(cudaSetDevice(c->device));
  const size_t bytes = (size_t)c->rows * c->cols * sizeof(float);
  // stage the inputs in context scratch that the solve does not touch before prep
  FOT_CUDA(cudaMemcpyAsync(c->tmp, g_host, bytes, cudaMemcpyHostToDevice, c->stream));
  FOT_CUDA(cudaMemcpyAsync(c->tmp2, G_host, bytes, cudaMemcpyHostToDevice, c->stream));
  fot_status s = fot_solve(c, c->tmp, c->tmp2, dx, eps, n_eps, eps_units, iters);
  if (s != FOT_OK) return s;
  moments_simt(c, c->psi, c->S_last, c->eps_last, c->dx, c->tmp, c->tmp2);
  integrate_phase(c, c->tmp, c->tmp2, c->dx, c->phi);
  s = check_launch(c);
  if (s != FOT_OK) return s;
  FOT_CUDA(cudaMemcpyAsync(phi_host, c->phi, bytes, cudaMemcpyDeviceToHost, c->stream));
  return read_latched(c);
}

}  // extern "C"

namespace fot {
// the configured half-step (FP32 banded, dense or tensor-core) for the adjoint
void half_step_dispatch(fot_ctx* c, const float* pot_in, const float* lmarg, double eps, float* pot_out,
                        float* logsum) {
  half_step(c, pot_in, lmarg, eps, pot_out, logsum);
}
}  // namespace fot
