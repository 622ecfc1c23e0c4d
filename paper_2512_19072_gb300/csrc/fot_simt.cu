// Exact log-domain axis passes on the CUDA cores (the FP32 form of the FOT iteration),
// plus the elementwise, reduction and scan kernels of the solve and the phase step.
//
// One "axis pass" is one 1-D contraction of the separable kernel Lambda (Sec. 2-3):
//     y[o][r] = log2 sum_m 2^( x[r][m]*scale - (o - m)^2 * c2 ),  c2 = log2(e) / (2 eps),
// over the contiguous axis m of a row-major input, written TRANSPOSED so that the next
// pass again contracts a contiguous axis.  Two passes make one application of
// log(Lambda . exp(pot/eps) . Lambda) (Eqs. 7-8); the second pass carries the potential
// update f = eps (log a - S) as a fused epilogue.
//
// Every output takes its own exact maximum (first sweep) before the exponentials
// (second sweep), so no offset choice can underflow: this is the robust FP32 path, bound
// by the MUFU exponential throughput (one ex2 per term).  Inputs are staged once per
// CTA in shared memory, interleaved [m][RB] so one 16-byte broadcast load feeds RB rows.
#include "fot_common.cuh"

#include <algorithm>

namespace fot {

enum PassMode : int { kLse = 0, kLsePot = 1, kLseMean = 2, kMoment = 3 };

struct PassArgs {
  const float* x;       // [n_rows][len] input
  const float* w;       // kMoment: per-term weights [n_rows][len]
  const float* off;     // kMoment: per-output natural-log divisor, layout of y
  const float* lmarg;   // kLsePot: natural log of the marginal, layout of y
  float* y;             // [len][n_rows] output (transposed)
  float* y2;            // kLseMean: weighted mean; kMoment: second moment output
  float* logsum;        // kLsePot: optional natural-log LSE output, layout of y
  int* err;
  float x_scale;        // x * x_scale -> log2 units
  float c2;             // log2(e) / (2 eps)
  float eps;            // kLsePot
  float coord0, coord_step;  // coordinate of index m: coord0 + m * coord_step
  int n_rows, len;
};

template <int RB, int MODE>
__global__ void __launch_bounds__(256) axis_pass_kernel(PassArgs p) {
  extern __shared__ __align__(16) float smem[];
  float* sx = smem;                              // [len][RB]
  float* sw = smem + (size_t)p.len * RB;         // [len][RB] (kMoment only)
  if (error_latched(p.err)) return;
  const int r0 = blockIdx.y * RB;
  const int len = p.len;
  for (int i = threadIdx.x; i < len * RB; i += blockDim.x) {
    const int r = i / len, m = i - r * len;
    const bool ok = r0 + r < p.n_rows;
    const size_t gi = (size_t)(r0 + r) * len + m;
    sx[m * RB + r] = ok ? p.x[gi] * p.x_scale : -INFINITY;
    if (MODE == kMoment) sw[m * RB + r] = ok ? p.w[gi] : 0.f;
  }
  __syncthreads();
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= len) return;
  const float nc2 = -p.c2;

  // sweep 1: exact maximum of every output
  float mx[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) mx[r] = -INFINITY;
  float df = (float)o;
  for (int m = 0; m < len; ++m, df -= 1.f) {
    const float t = df * df;
    const float4* xv = reinterpret_cast<const float4*>(sx + m * RB);
#pragma unroll
    for (int q = 0; q < RB / 4; ++q) {
      const float4 v = xv[q];
      mx[4 * q + 0] = fmaxf(mx[4 * q + 0], fmaf(t, nc2, v.x));
      mx[4 * q + 1] = fmaxf(mx[4 * q + 1], fmaf(t, nc2, v.y));
      mx[4 * q + 2] = fmaxf(mx[4 * q + 2], fmaf(t, nc2, v.z));
      mx[4 * q + 3] = fmaxf(mx[4 * q + 3], fmaf(t, nc2, v.w));
    }
  }
  bool empty[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    empty[r] = (mx[r] == -INFINITY);
    if (empty[r]) mx[r] = 0.f;   // every term is 2^-inf = 0
  }

  // sweep 2: sum of 2^(e - max) (and weighted sums)
  float acc[RB], accx[RB], accy[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) acc[r] = accx[r] = accy[r] = 0.f;
  df = (float)o;
  for (int m = 0; m < len; ++m, df -= 1.f) {
    const float t = df * df;
    const float cm = p.coord0 + (float)m * p.coord_step;
    const float* xr = sx + m * RB;
    const float* wr = sw + m * RB;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const float e = ex2(fmaf(t, nc2, xr[r]) - mx[r]);
      if (MODE == kLseMean) {
        acc[r] += e;
        accx[r] = fmaf(e, cm, accx[r]);
      } else if (MODE == kMoment) {
        accx[r] = fmaf(e, cm, accx[r]);
        accy[r] = fmaf(e, wr[r], accy[r]);
      } else {
        acc[r] += e;
      }
    }
  }

  // epilogues; output (o, r0 + r) lives at y[o * n_rows + r0 + r]
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    if (r0 + r >= p.n_rows) break;
    const size_t yi = (size_t)o * p.n_rows + r0 + r;
    if (MODE == kLse) {
      p.y[yi] = empty[r] ? -INFINITY : mx[r] + log2f(acc[r]);
    } else if (MODE == kLsePot) {
      const float s = empty[r] ? -INFINITY : (mx[r] + log2f(acc[r])) * kLn2;
      const float lm = p.lmarg[yi];
      float pot;
      if (lm == -INFINITY) {
        pot = -INFINITY;
      } else {
        pot = p.eps * (lm - s);
        if (!isfinite(pot)) raise_error(p.err, FOT_ENONFINITE);
      }
      p.y[yi] = pot;
      if (p.logsum) p.logsum[yi] = s;
    } else if (MODE == kLseMean) {
      p.y[yi] = empty[r] ? -INFINITY : mx[r] + log2f(acc[r]);
      p.y2[yi] = empty[r] ? 0.f : accx[r] / acc[r];
    } else {  // kMoment
      const float sc = empty[r] ? 0.f : ex2(mx[r] - p.off[yi] * kLog2e);
      p.y[yi] = accx[r] * sc;
      p.y2[yi] = accy[r] * sc;
    }
  }
}

template <int RB, int MODE>
static void launch_pass(fot_ctx* c, const PassArgs& p) {
  const int threads = std::min(256, ((p.len + 31) / 32) * 32);
  dim3 grid((p.len + threads - 1) / threads, (p.n_rows + RB - 1) / RB);
  size_t smem = (size_t)p.len * RB * sizeof(float) * (MODE == kMoment ? 2 : 1);
  // (the dynamic shared-memory limit was raised for this device by simt_configure)
  ktimer_begin(c->stream, kKDense);
  axis_pass_kernel<RB, MODE><<<grid, threads, smem, c->stream>>>(p);
  ktimer_end(c->stream);
  c->launches++;
  c->host_terms += (int64_t)p.n_rows * p.len * p.len;
}

// Raise the dynamic shared-memory limit of every axis-pass instance on the current device
// (a per-device function attribute: fot_create calls this with the context's device
// current, before any stream capture).  The staged rows need len * RB floats (twice that
// for the moment pass), i.e. more than the 48 KB default once len > 1536.
cudaError_t simt_configure() {
  const int lim = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(axis_pass_kernel<8, kLse>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(axis_pass_kernel<8, kLsePot>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(axis_pass_kernel<8, kLseMean>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(axis_pass_kernel<4, kMoment>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  return e;
}

static PassArgs base_args(fot_ctx* c, double eps) {
  PassArgs p{};
  p.err = c->err;
  p.c2 = (float)(1.4426950408889634 / (2.0 * eps));
  p.eps = (float)eps;
  return p;
}

// One half-step: pot_out = eps (lmarg - log(Lambda exp(pot_in/eps) Lambda)).
// pot_in, pot_out, lmarg, logsum: rows x cols; tmp: cols x rows.
void half_step_simt(fot_ctx* c, const float* pot_in, const float* lmarg, double eps,
                    float* pot_out, float* logsum, float* tmp) {
  PassArgs p = base_args(c, eps);
  // pass over the contiguous axis: rows of pot_in, outputs along cols, written [k][L]
  p.x = pot_in; p.x_scale = (float)(1.4426950408889634 / eps);
  p.n_rows = c->rows; p.len = c->cols; p.y = tmp;
  launch_pass<8, kLse>(c, p);
  // pass over the row axis with the fused potential update, written [j][k]
  PassArgs q = base_args(c, eps);
  q.x = tmp; q.x_scale = 1.f; q.n_rows = c->cols; q.len = c->rows;
  q.y = pot_out; q.lmarg = lmarg; q.logsum = logsum;
  launch_pass<8, kLsePot>(c, q);
}

// Phase-gradient moments (Eqs. 9-10, ratio form with u/g^2 = exp(-S_last)).
void moments_simt(fot_ctx* c, const float* psi, const float* S, double eps, double dx,
                  float* Dx, float* Dy) {
  const int rows = c->rows, cols = c->cols;
  // row pass with the final psi: log2 row sums Rf[k][L] and the conditional mean of Y_M
  PassArgs p = base_args(c, eps);
  p.x = psi; p.x_scale = (float)(1.4426950408889634 / eps);
  p.n_rows = rows; p.len = cols; p.y = c->R; p.y2 = c->R2;
  p.coord0 = (float)(-(double)(cols / 2) / (cols * dx));
  p.coord_step = (float)(1.0 / (cols * dx));
  launch_pass<8, kLseMean>(c, p);
  // column pass: Dx = sum_L X_L w, Dy = sum_L E[Y|L,k] w, w = 2^(Rf - d^2 c2) / e^S_last
  PassArgs q = base_args(c, eps);
  q.x = c->R; q.w = c->R2; q.off = S; q.x_scale = 1.f;
  q.n_rows = cols; q.len = rows; q.y = Dx; q.y2 = Dy;
  q.coord0 = (float)(-(double)(rows / 2) / (rows * dx));
  q.coord_step = (float)(1.0 / (rows * dx));
  launch_pass<4, kMoment>(c, q);
}

// ------------------------------------------------------------------------------------
// problem setup: a = g^2 / sum g^2, log a (and the same for G), validation
// ------------------------------------------------------------------------------------
__global__ void power_partials_kernel(const float* __restrict__ g, const float* __restrict__ G,
                                      size_t N, double* __restrict__ part, int* err) {
  __shared__ double sa[256], sb[256];
  double s0 = 0.0, s1 = 0.0;
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    const float x = g[i], y = G[i];
    bad |= !(isfinite(x) && isfinite(y) && x >= 0.f && y >= 0.f);
    s0 += (double)x * x;
    s1 += (double)y * y;
  }
  if (bad) raise_error(err, FOT_EINVAL);
  sa[threadIdx.x] = s0;
  sb[threadIdx.x] = s1;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sa[0];
    part[2 * blockIdx.x + 1] = sb[0];
  }
}

// Sum `nparts` pairs of partials in a fixed order (deterministic); out[0..1].
__global__ void sum_pairs_kernel(const double* __restrict__ part, int nparts, double* out,
                                 int* err, int check_mass) {
  __shared__ double sa[256], sb[256];
  double s0 = 0.0, s1 = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    s0 += part[2 * i];
    s1 += part[2 * i + 1];
  }
  sa[threadIdx.x] = s0;
  sb[threadIdx.x] = s1;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sa[0];
    out[1] = sb[0];
    if (check_mass && !(sa[0] > 0.0 && sb[0] > 0.0)) raise_error(err, FOT_EMASS);
  }
}

__global__ void log_marginals_kernel(const float* __restrict__ g, const float* __restrict__ G,
                                     size_t N, const double* __restrict__ tot,
                                     float* __restrict__ la, float* __restrict__ lb,
                                     float* __restrict__ psi0, float psi0_val, int* err) {
  if (error_latched(err)) return;
  const float lga = (float)log(tot[0]);
  const float lgb = (float)log(tot[1]);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    const float x = g[i], y = G[i];
    // log(g^2 / sum g^2) without forming g^2 (no FP32 underflow for faint pixels)
    la[i] = x > 0.f ? 2.f * logf(x) - lga : -INFINITY;
    lb[i] = y > 0.f ? 2.f * logf(y) - lgb : -INFINITY;
    if (psi0) psi0[i] = psi0_val;
  }
}

void set_problem_simt(fot_ctx* c, const float* g, const float* G, float* psi0, float psi0_val) {
  const size_t N = (size_t)c->rows * c->cols;
  power_partials_kernel<<<c->red_blocks, 256, 0, c->stream>>>(g, G, N, c->red, c->err);
  sum_pairs_kernel<<<1, 256, 0, c->stream>>>(c->red, c->red_blocks, c->red + 2 * c->red_blocks,
                                             c->err, 1);
  log_marginals_kernel<<<c->red_blocks, 256, 0, c->stream>>>(
      g, G, N, c->red + 2 * c->red_blocks, c->la, c->lb, psi0, psi0_val, c->err);
  c->launches += 3;
}

__global__ void fill_kernel(float* __restrict__ p, size_t N, float v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x)
    p[i] = v;
}

void fill(fot_ctx* c, float* p, size_t N, float v) {
  fill_kernel<<<c->red_blocks, 256, 0, c->stream>>>(p, N, v);
  c->launches++;
}

// ------------------------------------------------------------------------------------
// marginal violation and dual objective (double accumulation, deterministic order)
// ------------------------------------------------------------------------------------
// part[4*b + {0,1,2,3}] = { sum |row - a|, sum Gamma, sum_a f a, 0 } for the source image,
// and the same for the target with psi, b in a second launch.
__global__ void marginal_partials_kernel(const float* __restrict__ pot,
                                         const float* __restrict__ logsum,
                                         const float* __restrict__ lmarg, size_t N, double inv_eps,
                                         double* __restrict__ part) {
  __shared__ double s[3][256];
  double e1 = 0.0, e2 = 0.0, e3 = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    const float lm = lmarg[i];
    const double m = lm == -INFINITY ? 0.0 : exp((double)lm);
    double r = 0.0;
    if (pot[i] != -INFINITY && logsum[i] != -INFINITY)
      r = exp((double)pot[i] * inv_eps + (double)logsum[i]);
    e1 += fabs(r - m);
    e2 += r;
    if (m > 0.0) e3 += (double)pot[i] * m;
  }
  s[0][threadIdx.x] = e1;
  s[1][threadIdx.x] = e2;
  s[2][threadIdx.x] = e3;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 3; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) part[3 * blockIdx.x + q] = s[q][0];
}

__global__ void sum_triples_kernel(const double* __restrict__ part, int nparts, double* out) {
  __shared__ double s[3][256];
  double e[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < nparts; i += blockDim.x)
    for (int q = 0; q < 3; ++q) e[q] += part[3 * i + q];
  for (int q = 0; q < 3; ++q) s[q][threadIdx.x] = e[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 3; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) out[q] = s[q][0];
}

// out[0..2] = source {L1, mass, <f,a>} alone (the convergence check of fot_solve_tol)
void source_stats(fot_ctx* c, const float* f, const float* S, double eps, double* out) {
  const size_t N = (size_t)c->rows * c->cols;
  marginal_partials_kernel<<<c->red_blocks, 256, 0, c->stream>>>(f, S, c->la, N, 1.0 / eps, c->red);
  sum_triples_kernel<<<1, 256, 0, c->stream>>>(c->red, c->red_blocks, out);
  c->launches += 2;
}

// out[0..2] = source {L1, mass, <f,a>}; out[3..5] = target {L1, mass, <psi,b>}
void marginal_stats(fot_ctx* c, const float* f, const float* S, const float* psi,
                    const float* T, double eps, double* out) {
  const size_t N = (size_t)c->rows * c->cols;
  double* part = c->red;
  marginal_partials_kernel<<<c->red_blocks, 256, 0, c->stream>>>(f, S, c->la, N, 1.0 / eps, part);
  sum_triples_kernel<<<1, 256, 0, c->stream>>>(part, c->red_blocks, out);
  marginal_partials_kernel<<<c->red_blocks, 256, 0, c->stream>>>(psi, T, c->lb, N, 1.0 / eps,
                                                                 part);
  sum_triples_kernel<<<1, 256, 0, c->stream>>>(part, c->red_blocks, out + 3);
  c->launches += 4;
}

// ------------------------------------------------------------------------------------
// trapezoid integration of the phase gradient (the "Integrate" step of Algorithm 1)
// ------------------------------------------------------------------------------------
// Inclusive warp scan of one float per lane.
__device__ __forceinline__ float warp_scan(float v) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float t = __shfl_up_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) >= d) v += t;
  }
  return v;
}

// Outward trapezoid sums along a line of n values v[i * stride] from the centre c:
// out[c] = base, out[i] = base + h/2 sum_{q=c+1..i} (v[q-1] + v[q]) for i > c,
// out[i] = base - h/2 sum_{q=i..c-1} (v[q] + v[q+1]) for i < c.  One warp per line.
__device__ void trapezoid_line(const float* v, int stride, int n, int c, float h, float base,
                               float* out, int ostride) {
  const int lane = threadIdx.x & 31;
  // forward half: increments q = c+1 .. n-1
  float carry = base;
  if (lane == 0) out[(size_t)c * ostride] = base;
  for (int q0 = c + 1; q0 < n; q0 += 32) {
    const int q = q0 + lane;
    const float inc = q < n ? 0.5f * h * (v[(size_t)(q - 1) * stride] + v[(size_t)q * stride]) : 0.f;
    const float s = warp_scan(inc) + carry;
    if (q < n) out[(size_t)q * ostride] = s;
    carry = __shfl_sync(0xffffffffu, s, 31);
  }
  // backward half: q = c-1 .. 0
  carry = base;
  for (int q0 = c - 1; q0 >= 0; q0 -= 32) {
    const int q = q0 - lane;
    const float inc = q >= 0 ? 0.5f * h * (v[(size_t)q * stride] + v[(size_t)(q + 1) * stride]) : 0.f;
    const float s = carry - warp_scan(inc);
    if (q >= 0) out[(size_t)q * ostride] = s;
    carry = __shfl_sync(0xffffffffu, s, 31);
  }
}

__global__ void trapezoid_column_kernel(const float* __restrict__ Dx, int rows, int cols,
                                        float h, float* __restrict__ col) {
  // centre column k = cols/2, along j
  trapezoid_line(Dx + cols / 2, cols, rows, rows / 2, h, 0.f, col, 1);
}

__global__ void trapezoid_rows_kernel(const float* __restrict__ Dy, const float* __restrict__ col,
                                      int rows, int cols, float h, float* __restrict__ phi) {
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (j >= rows) return;
  trapezoid_line(Dy + (size_t)j * cols, 1, cols, cols / 2, h, col[j], phi + (size_t)j * cols, 1);
}

void integrate_phase(fot_ctx* c, const float* Dx, const float* Dy, double dx, float* phi) {
  trapezoid_column_kernel<<<1, 32, 0, c->stream>>>(Dx, c->rows, c->cols, (float)dx, c->col_phi);
  const int wpb = 8;
  trapezoid_rows_kernel<<<(c->rows + wpb - 1) / wpb, 32 * wpb, 0, c->stream>>>(
      Dy, c->col_phi, c->rows, c->cols, (float)dx, phi);
  c->launches += 2;
}

}  // namespace fot

// ------------------------------------------------------------------------------------
// Allocation-free u-update (fot_u_update_noalloc in include/fot.h).
//
// For callers that may not allocate device memory at call time: it runs the same two
// axis passes as fot_u_update, but its intermediate lives in the file-scope device array
// below instead of context-owned cudaMalloc memory.  Every GPU that loads this library
// keeps these FOT_NOALLOC_MAX_PIXELS floats (4 MiB) until the process exits.  All calls
// share the array, so calls whose work overlaps on the GPU race on it.
// ------------------------------------------------------------------------------------
static __device__ __align__(256) float g_noalloc_scratch[FOT_NOALLOC_MAX_PIXELS];
// The pass kernels latch a non-finite potential into an error word and skip their work
// while it is set.  This entry point reads nothing back (it never synchronises), so the word
// is not reported: it is cleared at the start of every call so that a value latched by an
// earlier call never makes a later one skip its passes.  A non-finite result shows up as a
// non-finite value in f_out.
static __device__ int g_noalloc_err;

namespace {
constexpr int kNoallocMaxDevices = 64;
struct NoallocDevice {
  float* scratch = nullptr;   // device address of g_noalloc_scratch on this device
  int* err = nullptr;         // device address of g_noalloc_err on this device
  bool ready = false;
};
NoallocDevice g_noalloc_devices[kNoallocMaxDevices];

template <int RB, int MODE>
cudaError_t launch_pass_noalloc(const fot::PassArgs& p, cudaStream_t s) {
  const int threads = std::min(256, ((p.len + 31) / 32) * 32);
  dim3 grid((p.len + threads - 1) / threads, (p.n_rows + RB - 1) / RB);
  const size_t smem = (size_t)p.len * RB * sizeof(float);
  fot::axis_pass_kernel<RB, MODE><<<grid, threads, smem, s>>>(p);
  return cudaGetLastError();
}
}  // namespace

extern "C" fot_status fot_u_update_noalloc(const float* psi_in, const float* log_a, int rows,
                                           int cols, double eps, float* f_out,
                                           float* logsum_out, void* cuda_stream) {
  if (!psi_in || !log_a || !f_out) return FOT_EINVAL;
  if (rows < 1 || cols < 1 || rows > 4096 || cols > 4096) return FOT_EINVAL;
  if ((size_t)rows * (size_t)cols > (size_t)FOT_NOALLOC_MAX_PIXELS) return FOT_EINVAL;
  if (!(eps > 0.0) || !isfinite(eps)) return FOT_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FOT_ECUDA;
  if (dev < 0 || dev >= kNoallocMaxDevices) return FOT_EUNSUPPORTED;
  NoallocDevice& d = g_noalloc_devices[dev];
  if (!d.ready) {
    // one-time set-up on this device (current): the symbols' device addresses and the
    // shared-memory limit of the two pass kernels (both per-device state)
    if (cudaGetSymbolAddress((void**)&d.scratch, g_noalloc_scratch) != cudaSuccess) return FOT_ECUDA;
    if (cudaGetSymbolAddress((void**)&d.err, g_noalloc_err) != cudaSuccess) return FOT_ECUDA;
    if (fot::simt_configure() != cudaSuccess) return FOT_ECUDA;
    d.ready = true;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (cudaMemsetAsync(d.err, 0, sizeof(int), s) != cudaSuccess) return FOT_ECUDA;
  fot::PassArgs p{};
  p.err = d.err;
  p.c2 = (float)(1.4426950408889634 / (2.0 * eps));
  p.eps = (float)eps;
  fot::PassArgs q = p;
  // pass over the contiguous axis into the static scratch, written [k][L]
  p.x = psi_in; p.x_scale = (float)(1.4426950408889634 / eps);
  p.n_rows = rows; p.len = cols; p.y = d.scratch;
  if (launch_pass_noalloc<8, fot::kLse>(p, s) != cudaSuccess) return FOT_ECUDA;
  // pass over the row axis with the fused update f = eps (log a - S), written [j][k]
  q.x = d.scratch; q.x_scale = 1.f; q.n_rows = cols; q.len = rows;
  q.y = f_out; q.lmarg = log_a; q.logsum = logsum_out;
  if (launch_pass_noalloc<8, fot::kLsePot>(q, s) != cudaSuccess) return FOT_ECUDA;
  return FOT_OK;
}
