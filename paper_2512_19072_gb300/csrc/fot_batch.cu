// Batched solve: many independent beam-shaping problems of different grid sizes in one
// stream of multi-problem launches.
//
// Every axis pass of every problem goes into the same two launches (the window plan, then the
// banded window sums on the CUDA cores or, for the mixed form, on the tensor cores):
// the kernels take a table of up to 64 problems by value and map each warp / CTA to its
// problem by prefix sums (BandTable).  The whole solve - problem setup and all iterations
// with each iteration's eps baked into its launches - is captured once into a CUDA graph and
// replayed with a single cudaGraphLaunch; the graph is rebuilt only when the inputs, the
// schedule or the iteration count change.
//
// Precision FOT_AUTO times one iteration of the FP32 and of the mixed (tensor-core) passes
// on the batch itself at graph-build time and keeps the faster for every problem.
#include <math.h>
#include <string.h>

#include <chrono>
#include <new>
#include <vector>

#include "fot_band.cuh"

namespace fot {
void set_problem_simt(fot_ctx* c, const float* g, const float* G, float* psi0, float psi0_val);
BandArgs band_args(fot_ctx* c, const float* x, int n_rows, int len, double eps, float x_scale);
int tc_create(fot_ctx* c);
}  // namespace fot

using namespace fot;

struct fot_batch {
  int count = 0, precision = 0, device = 0;
  cudaStream_t stream = nullptr;       // the caller's stream: graph launches
  cudaStream_t cap = nullptr;          // private non-blocking stream the graph is captured on
  std::vector<fot_ctx*> ctx;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // what the captured graph was built for
  std::vector<const float*> key_g, key_G;
  std::vector<double> key_eps;
  int key_iters = -1, key_neps = -1;
  bool use_tc = false;     // precision decided for the graph (FOT_AUTO resolves it)
  int64_t nodes = 0;       // kernels per graph launch
};

static void capture_solve(fot_batch* b, cudaStream_t st, const float* const* g, const float* const* G,
                          const double* eps, int n_eps, int iters, bool use_tc, int64_t* kernels) {
  const int n = b->count;
  for (fot_ctx* c : b->ctx) c->stream = st;
  int64_t k = 0;
  for (int q = 0; q < n; ++q) {
    fot_ctx* c = b->ctx[q];
    const double e0 = eps[(size_t)q * n_eps];
    const float psi0 = (float)(e0 * log(1.0 / ((double)c->rows * c->cols)));
    set_problem_simt(c, g[q], G[q], c->psi, psi0);
    k += 3;
  }
  // one table per pass and tile width: a problem runs the same kernels as its single solve
  static const int kWidths[4] = {64, 32, 16, 0};
  BandTable<kMaxBatch>* tab = new BandTable<kMaxBatch>();
  std::vector<BandArgs> p1(n), p2(n);
  std::vector<int> width(n);
  std::vector<fot_ctx*> tctx(n);
  if (use_tc)
    for (fot_ctx* c : b->ctx) tc_begin(c);
  for (int it = 0; it < iters; ++it) {
    for (int half = 0; half < 2; ++half) {
      for (int q = 0; q < n; ++q) {
        fot_ctx* c = b->ctx[q];
        const double e = eps[(size_t)q * n_eps + (n_eps == 1 ? 0 : it)];
        const float* pin = half == 0 ? c->psi : c->f;
        float* pout = half == 0 ? c->f : c->psi;
        BandArgs a1 = band_args(c, pin, c->rows, c->cols, e, (float)(1.4426950408889634 / e));
        a1.y = c->R;
        BandArgs a2 = band_args(c, c->R, c->cols, c->rows, e, 1.f);
        a2.y = pout;
        a2.lmarg = half == 0 ? c->la : c->lb;
        a2.logsum = (half == 0 && it == iters - 1) ? c->S_last : nullptr;
        p1[q] = a1;
        p2[q] = a2;
        width[q] = use_tc ? tc_width_for(a1.c) : -1;
      }
      for (int pass = 0; pass < 2; ++pass) {
        const std::vector<BandArgs>& pa = pass == 0 ? p1 : p2;
        for (int wi = 0; wi < (use_tc ? 4 : 1); ++wi) {
          tab->n = 0;
          for (int q = 0; q < n; ++q)
            if (width[q] == (use_tc ? kWidths[wi] : -1)) {
              tctx[tab->n] = b->ctx[q];
              tab->p[tab->n++] = pa[q];
            }
          if (tab->n == 0) continue;
          if (use_tc) {
            for (int j = 0; j < tab->n; ++j) tc_bind(tctx[j], tab->p[j]);
            k += pass == 0 ? tc_pass<0>(st, *tab, kWidths[wi], tctx.data())
                           : tc_pass<1>(st, *tab, kWidths[wi], tctx.data());
          } else {
            band_table_finish(*tab);
            band_prepare(st, *tab);
            if (pass == 0)
              band_simt<0>(st, *tab);
            else
              band_simt<1>(st, *tab);
            k += 2;
          }
        }
      }
    }
  }
  delete tab;
  for (int q = 0; q < n; ++q) {
    fot_ctx* c = b->ctx[q];
    c->stream = b->stream;
    c->eps_last = eps[(size_t)q * n_eps + (n_eps == 1 ? 0 : iters - 1)];
    c->sched.clear();
    for (int it = 0; it < iters; ++it) c->sched.push_back(eps[(size_t)q * n_eps + (n_eps == 1 ? 0 : it)]);
  }
  *kernels = k;
}

static fot_status build_graph(fot_batch* b, const float* const* g, const float* const* G, const double* eps,
                              int n_eps, int iters, bool use_tc) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  // capture on the private stream (capture is not allowed on the legacy default stream)
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return FOT_ECUDA;
  int64_t k = 0;
  capture_solve(b, b->cap, g, G, eps, n_eps, iters, use_tc, &k);
  if (cudaStreamEndCapture(b->cap, &b->graph) != cudaSuccess) return FOT_ECUDA;
  if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return FOT_ECUDA;
  b->nodes = k;
  b->use_tc = use_tc;
  return FOT_OK;
}

// one iteration of each form on the batch, timed with events (FOT_AUTO)
static bool tc_faster(fot_batch* b, const float* const* g, const float* const* G, const double* eps, int n_eps) {
  float ms[2] = {0.f, 0.f};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int v = 0; v < 2; ++v) {
    int64_t k = 0;
    capture_solve(b, b->stream, g, G, eps, n_eps, 1, v == 1, &k);   // warm (also loads the problems)
    cudaEventRecord(e0, b->stream);
    capture_solve(b, b->stream, g, G, eps, n_eps, 2, v == 1, &k);
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms[v], e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms[1] < ms[0];
}

extern "C" {

fot_status fot_batch_create(fot_batch** out, int count, const int* rows, const int* cols, int precision,
                            int device, void* cuda_stream) {
  if (!out || !rows || !cols || count < 1 || count > kMaxBatch) return FOT_EINVAL;
  *out = nullptr;
  if (precision != FOT_FP32 && precision != FOT_MIXED && precision != FOT_AUTO) return FOT_EINVAL;
  fot_batch* b = new (std::nothrow) fot_batch();
  if (!b) return FOT_ENOMEM;
  b->count = count;
  b->precision = precision;
  b->device = device;
  b->stream = (cudaStream_t)cuda_stream;
  if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return FOT_ECUDA;
  }
  for (int q = 0; q < count; ++q) {
    fot_ctx* c = nullptr;
    const int p = precision == FOT_FP32 ? FOT_FP32 : FOT_MIXED;   // AUTO keeps both ready
    fot_status s = fot_create(&c, rows[q], cols[q], p, device, cuda_stream);
    if (s != FOT_OK) {
      fot_batch_destroy(b);
      return s;
    }
    b->ctx.push_back(c);
  }
  *out = b;
  return FOT_OK;
}

void fot_batch_destroy(fot_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (fot_ctx* c : b->ctx) fot_destroy(c);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

fot_ctx* fot_batch_context(fot_batch* b, int index) {
  if (!b || index < 0 || index >= b->count) return nullptr;
  return b->ctx[index];
}

fot_status fot_batch_solve(fot_batch* b, const float* const* g, const float* const* G, double dx,
                           const double* eps, int n_eps, int eps_units, int iters) {
  if (!b || !g || !G || !eps || iters < 1 || !(n_eps == 1 || n_eps == iters)) return FOT_EINVAL;
  if (eps_units != FOT_EPS_PX2 && eps_units != FOT_EPS_PAPER) return FOT_EINVAL;
  const int n = b->count;
  std::vector<double> e((size_t)n * n_eps);
  for (int q = 0; q < n; ++q) {
    if (!g[q] || !G[q]) return FOT_EINVAL;
    const fot_ctx* c = b->ctx[q];
    const double nn = (double)(c->rows > c->cols ? c->rows : c->cols);
    for (int t = 0; t < n_eps; ++t) {
      const double v = eps[(size_t)q * n_eps + t];
      if (!(v > 0.0) || !isfinite(v)) return FOT_EINVAL;
      e[(size_t)q * n_eps + t] = eps_units == FOT_EPS_PAPER ? v * nn * nn : v;
    }
  }
  if (cudaSetDevice(b->device) != cudaSuccess) return FOT_ECUDA;
  for (fot_ctx* c : b->ctx) {
    c->stream = b->stream;
    if (cudaMemsetAsync(c->err, 0, sizeof(int), b->stream) != cudaSuccess) return FOT_ECUDA;
    const double nn = (double)(c->rows > c->cols ? c->rows : c->cols);
    c->dx = dx > 0.0 ? dx : 1.0 / sqrt(nn);
  }
  const bool same = b->exec && b->key_iters == iters && b->key_neps == n_eps && b->key_eps == e &&
                    memcmp(b->key_g.data(), g, n * sizeof(float*)) == 0 &&
                    memcmp(b->key_G.data(), G, n * sizeof(float*)) == 0;
  if (!same) {
    bool use_tc = b->precision == FOT_MIXED;
    if (b->precision == FOT_AUTO) use_tc = tc_faster(b, g, G, e.data(), n_eps);
    fot_status s = build_graph(b, g, G, e.data(), n_eps, iters, use_tc);
    if (s != FOT_OK) return s;
    b->key_g.assign(g, g + n);
    b->key_G.assign(G, G + n);
    b->key_eps = e;
    b->key_iters = iters;
    b->key_neps = n_eps;
  }
  if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return FOT_ECUDA;
  for (fot_ctx* c : b->ctx) {
    c->have_problem = true;
    c->have_solution = true;
    c->launches += b->nodes / n;
  }
  return FOT_OK;
}

fot_status fot_batch_info(fot_batch* b, int64_t* kernels_per_solve, int* tensor_path) {
  if (!b) return FOT_EINVAL;
  if (kernels_per_solve) *kernels_per_solve = b->nodes;
  if (tensor_path) *tensor_path = b->use_tc ? 1 : 0;
  return FOT_OK;
}

}  // extern "C"
