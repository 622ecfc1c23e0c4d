// Adjoint (reverse mode) of the FOT solve: gradients of a scalar loss of the phase and/or the
// final potentials with respect to the input and target amplitudes g and G, through every
// unrolled iteration (Eqs. 7-8), the moments (Eqs. 9-10), the trapezoid integration and the
// marginal normalisation a = g^2 / sum g^2, b = G^2 / sum G^2.
//
// Half-step VJPs.  f = eps (log a - S(psi)), S_jk = log sum_LM exp(psi_LM/eps - C_jkLM/eps):
//     dL/dlog a += eps fbar,   psibar_LM -= sum_jk fbar_jk exp(psi_LM/eps - C/eps - S_jk),
// and likewise for psi = eps (log b - T(f)).  The sum is a Gaussian-kernel application to
// the signed weights z_jk = fbar_jk e^{-S_jk}; it is evaluated in the log domain by the same
// separable axis passes as the forward solve, once on the positive and once on the negative
// part:  sum_jk z e^{-C/eps} = e^{L+} - e^{L-},  L+- = log(Lambda e^{log z+-} Lambda).
//
// Moments: with W_jk,LM = exp((f_jk + psi_LM - C)/eps - log a_jk) (the plan over g^2),
// Dx_jk = sum_LM X_L W, Dy_jk = sum_LM Y_M W, so
//     psibar_LM += (1/eps) e^{psi_LM/eps} [X_L K(Dxbar e^{-S}) + Y_M K(Dybar e^{-S})]_LM,
//     fbar_jk += (Dxbar Dx + Dybar Dy)_jk / eps,   dL/dlog a_jk -= (Dxbar Dx + Dybar Dy)_jk.
// Trapezoid: the transpose of the linear integration map (suffix / prefix sums).
// Normalisation: log a = 2 log g - log sum g^2, so dL/dg = 2 (abar - a sum abar) / g (0 where
// g = 0), abar = dL/dlog a.
//
// Memory: the forward is recomputed from potentials checkpointed every k iterations; one
// segment of k iterations (psi_t, S_t, f_t+1, T_t) is held at a time.
#include <math.h>

#include <vector>

#include "fot_common.cuh"

namespace fot {
void tc_begin(fot_ctx* c);
void half_step_dispatch(fot_ctx* c, const float* pot_in, const float* lmarg, double eps, float* pot_out,
                        float* logsum);
void moments_simt(fot_ctx* c, const float* psi, const float* S, double eps, double dx, float* Dx, float* Dy);
void set_problem_simt(fot_ctx* c, const float* g, const float* G, float* psi0, float psi0_val);
void fill(fot_ctx* c, float* p, size_t N, float v);
}  // namespace fot

using namespace fot;

namespace {

__global__ void split_kernel(const float* __restrict__ z, const float* __restrict__ off, float eps, size_t N,
                             float* __restrict__ pos, float* __restrict__ neg) {
  // pos = eps (log z+ - off), neg = eps (log z- - off); -inf where that part is zero
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const float v = z[i];
    const float o = off ? off[i] : 0.f;
    const bool fin = isfinite(o);
    pos[i] = (v > 0.f && fin) ? eps * (logf(v) - o) : -INFINITY;
    neg[i] = (v < 0.f && fin) ? eps * (logf(-v) - o) : -INFINITY;
  }
}

// out -= (e^{base/eps + Lp} - e^{base/eps + Ln}) * scale   (base = -inf contributes 0)
__global__ void combine_kernel(const float* __restrict__ base, float inv_eps, const float* __restrict__ Lp,
                               const float* __restrict__ Ln, float scale, size_t N, float* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const float b = base[i];
    if (b == -INFINITY) continue;
    const float x = b * inv_eps;
    const float p = Lp[i] == -INFINITY ? 0.f : expf(x + Lp[i]);
    const float q = Ln[i] == -INFINITY ? 0.f : expf(x + Ln[i]);
    out[i] -= scale * (p - q);
  }
}

__global__ void axpy_kernel(float* __restrict__ y, const float* __restrict__ x, float s, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    y[i] += s * x[i];
}

// moments VJP, elementwise part: fbar += (Dxbar Dx + Dybar Dy)/eps; abar -= (Dxbar Dx +
// Dybar Dy).  (The kernel applications to Dxbar e^{-S}, Dybar e^{-S} take S as the log
// offset of split_kernel: e^{-S} alone overflows FP32 where S is very negative.)
__global__ void moments_vjp_pre(const float* __restrict__ Dxb, const float* __restrict__ Dyb,
                                const float* __restrict__ Dx, const float* __restrict__ Dy, float inv_eps,
                                size_t N, float* __restrict__ fbar, float* __restrict__ abar) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const float d = Dxb[i] * Dx[i] + Dyb[i] * Dy[i];
    fbar[i] += d * inv_eps;
    abar[i] -= d;
  }
}

// psibar_LM += (1/eps) e^{psi/eps} [X_L (e^{Lx+} - e^{Lx-}) + Y_M (e^{Ly+} - e^{Ly-})]
__global__ void moments_vjp_post(const float* __restrict__ psi, float inv_eps, const float* __restrict__ Lxp,
                                 const float* __restrict__ Lxn, const float* __restrict__ Lyp,
                                 const float* __restrict__ Lyn, int rows, int cols, float dX, float dY,
                                 float* __restrict__ psibar) {
  const size_t N = (size_t)rows * cols;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    if (psi[i] == -INFINITY) continue;
    const int L = (int)(i / cols), M = (int)(i % cols);
    const float X = (float)(L - rows / 2) * dX, Y = (float)(M - cols / 2) * dY;
    const float x = psi[i] * inv_eps;
    const float kx = (Lxp[i] == -INFINITY ? 0.f : expf(x + Lxp[i])) - (Lxn[i] == -INFINITY ? 0.f : expf(x + Lxn[i]));
    const float ky = (Lyp[i] == -INFINITY ? 0.f : expf(x + Lyp[i])) - (Lyn[i] == -INFINITY ? 0.f : expf(x + Lyn[i]));
    psibar[i] += inv_eps * (X * kx + Y * ky);
  }
}

// transpose of the trapezoid integration: one thread per row for the row sweeps (with
// column-bar accumulation), then one thread for the centre column
__global__ void trapezoid_vjp_rows(const float* __restrict__ phib, int rows, int cols, float h,
                                   float* __restrict__ Dyb, float* __restrict__ colb) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= rows) return;
  const float* p = phib + (size_t)j * cols;
  float* d = Dyb + (size_t)j * cols;
  const int cc = cols / 2;
  float tot = 0.f;
  for (int k = 0; k < cols; ++k) {
    tot += p[k];
    d[k] = 0.f;
  }
  colb[j] = tot;
  // k > cc: phi[k] = col + sum_{q=cc+1..k} h/2 (Dy[q-1] + Dy[q])
  float suf = 0.f;                 // sum_{k >= q} phib[k], built from the right
  for (int q = cols - 1; q >= cc; --q) {
    const float suf_next = suf;    // sum_{k >= q+1}
    suf += p[q];
    if (q >= cc + 1) d[q] += 0.5f * h * suf;
    d[q] += 0.5f * h * suf_next;
  }
  // k < cc: phi[k] = col - sum_{q=k..cc-1} h/2 (Dy[q] + Dy[q+1])
  float pre = 0.f;                 // sum_{k <= q} phib[k], k < cc
  for (int q = 0; q <= cc; ++q) {
    const float pre_prev = pre;    // sum_{k <= q-1}
    if (q <= cc - 1) pre += p[q];
    if (q <= cc - 1) d[q] -= 0.5f * h * pre;
    if (q >= 1) d[q] -= 0.5f * h * pre_prev;
  }
}

__global__ void trapezoid_vjp_col(const float* __restrict__ colb, int rows, int cols, float h, float* __restrict__ Dxb) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int cc = cols / 2, cr = rows / 2;
  for (int j = 0; j < rows; ++j) Dxb[(size_t)j * cols + cc] = 0.f;
  float suf = 0.f;
  for (int q = rows - 1; q >= cr; --q) {
    const float suf_next = suf;
    suf += colb[q];
    if (q >= cr + 1) Dxb[(size_t)q * cols + cc] += 0.5f * h * suf;
    Dxb[(size_t)q * cols + cc] += 0.5f * h * suf_next;
  }
  float pre = 0.f;
  for (int q = 0; q <= cr; ++q) {
    const float pre_prev = pre;
    if (q <= cr - 1) pre += colb[q];
    if (q <= cr - 1) Dxb[(size_t)q * cols + cc] -= 0.5f * h * pre;
    if (q >= 1) Dxb[(size_t)q * cols + cc] -= 0.5f * h * pre_prev;
  }
}

// sums of abar and of amp^2 (double, one block), then grad = 2 (abar - a sum abar) / amp
__global__ void grad_from_logmarg(const float* __restrict__ abar, const float* __restrict__ amp, size_t N,
                                  float* __restrict__ grad) {
  __shared__ double s1[256], s2[256];
  double t1 = 0.0, t2 = 0.0;
  for (size_t i = threadIdx.x; i < N; i += blockDim.x) {
    t1 += (double)abar[i];
    t2 += (double)amp[i] * amp[i];
  }
  s1[threadIdx.x] = t1;
  s2[threadIdx.x] = t2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  const double sa = s1[0], sg = s2[0];
  for (size_t i = threadIdx.x; i < N; i += blockDim.x) {
    const float x = amp[i];
    grad[i] = x > 0.f ? (float)(2.0 * ((double)abar[i] - (double)x * x / sg * sa) / x) : 0.f;
  }
}

inline dim3 grid_for(size_t N) {
  size_t b = (N + 255) / 256;
  return dim3((unsigned)(b < 2048 ? (b < 1 ? 1 : b) : 2048));
}

}  // namespace

extern "C" fot_status fot_backward(fot_ctx* c, const float* g, const float* G, const float* dL_dphi,
                                   const float* dL_df, const float* dL_dpsi, int checkpoint_every,
                                   float* dL_dg, float* dL_dG) {
  if (!c || !g || !G || !dL_dg || !dL_dG || checkpoint_every < 1) return FOT_EINVAL;
  if (!c->have_solution || c->sched.empty()) return FOT_ESTATE;
  if (cudaSetDevice(c->device) != cudaSuccess) return FOT_ECUDA;
  const int T = (int)c->sched.size();
  const int K = checkpoint_every;
  const int nseg = (T + K - 1) / K;
  const size_t N = (size_t)c->rows * c->cols;
  const size_t B = N * sizeof(float);
  cudaStream_t s = c->stream;
  // device memory of the backward: checkpoints, one segment, adjoints and temporaries
  std::vector<float*> bufs;
  int failed = 0;
  auto alloc = [&](size_t words) -> float* {
    float* p = nullptr;
    if (cudaMalloc((void**)&p, words * sizeof(float)) != cudaSuccess) {
      ++failed;
      return nullptr;
    }
    bufs.push_back(p);
    return p;
  };
  float* ckpt = alloc(N * nseg);                 // psi at t = 0, K, 2K, ...
  float* seg_psi = alloc(N * K);                 // psi_t (input of the u-half)
  float* seg_S = alloc(N * K);                   // S_t
  float* seg_f = alloc(N * K);                   // f_{t+1}
  float* seg_T = alloc(N * K);                   // T_t
  float* psib = alloc(N);
  float* fb = alloc(N);
  float* ab = alloc(N);
  float* bb = alloc(N);
  float* neg_inf = alloc(N);
  float* tA = alloc(N);
  float* tB = alloc(N);
  float* Lp = alloc(N);
  float* Ln = alloc(N);
  float* scratch = alloc(N);
  float* psi_cur = alloc(N);
  float* f_cur = alloc(N);
  float* lxp = alloc(N);
  float* lxn = alloc(N);
  float* lyp = alloc(N);
  float* lyn = alloc(N);
  float* pp = alloc(N);
  float* pn = alloc(N);
  const bool ok = failed == 0;
  auto cleanup = [&]() {
    cudaStreamSynchronize(s);
    for (float* p : bufs)
      if (p) cudaFree(p);
  };
  if (!ok) {
    cleanup();
    return FOT_ENOMEM;
  }
  const dim3 gN = grid_for(N);
  if (c->tc) tc_begin(c);
  fill(c, neg_inf, N, -INFINITY);
  cudaMemsetAsync(psib, 0, B, s);
  cudaMemsetAsync(fb, 0, B, s);
  cudaMemsetAsync(ab, 0, B, s);
  cudaMemsetAsync(bb, 0, B, s);
  // 1. forward with checkpoints (bitwise the solve: same kernels, same order)
  const double e0 = c->sched[0];
  fill(c, psi_cur, N, (float)(e0 * log(1.0 / (double)N)));
  for (int t = 0; t < T; ++t) {
    if (t % K == 0) cudaMemcpyAsync(ckpt + (size_t)(t / K) * N, psi_cur, B, cudaMemcpyDeviceToDevice, s);
    half_step_dispatch(c, psi_cur, c->la, c->sched[t], f_cur, nullptr);
    half_step_dispatch(c, f_cur, c->lb, c->sched[t], psi_cur, nullptr);
  }
  // 2. seeds at the end of the solve: psi_T = psi_cur, f_T = f_cur, S_{T-1} = c->S_last
  const double eT = c->sched[T - 1];
  if (dL_dpsi) axpy_kernel<<<gN, 256, 0, s>>>(psib, dL_dpsi, 1.f, N);
  if (dL_df) axpy_kernel<<<gN, 256, 0, s>>>(fb, dL_df, 1.f, N);
  if (dL_dphi) {
    float* Dxb = tA;
    float* Dyb = tB;
    float* colb = scratch;
    cudaMemsetAsync(Dxb, 0, B, s);
    trapezoid_vjp_rows<<<(c->rows + 127) / 128, 128, 0, s>>>(dL_dphi, c->rows, c->cols, (float)c->dx, Dyb, colb);
    trapezoid_vjp_col<<<1, 1, 0, s>>>(colb, c->rows, c->cols, (float)c->dx, Dxb);
    float* Dx = Lp;
    float* Dy = Ln;
    moments_simt(c, psi_cur, c->S_last, eT, c->dx, Dx, Dy);
    moments_vjp_pre<<<gN, 256, 0, s>>>(Dxb, Dyb, Dx, Dy, (float)(1.0 / eT), N, fb, ab);
    // K(Dxbar e^{-S}), K(Dybar e^{-S}) on the target grid (4 log-domain applications)
    split_kernel<<<gN, 256, 0, s>>>(Dxb, c->S_last, (float)eT, N, pp, pn);
    half_step_dispatch(c, pp, neg_inf, eT, scratch, lxp);
    half_step_dispatch(c, pn, neg_inf, eT, scratch, lxn);
    split_kernel<<<gN, 256, 0, s>>>(Dyb, c->S_last, (float)eT, N, pp, pn);
    half_step_dispatch(c, pp, neg_inf, eT, scratch, lyp);
    half_step_dispatch(c, pn, neg_inf, eT, scratch, lyn);
    moments_vjp_post<<<gN, 256, 0, s>>>(psi_cur, (float)(1.0 / eT), lxp, lxn, lyp, lyn, c->rows, c->cols,
                                        (float)(1.0 / (c->rows * c->dx)), (float)(1.0 / (c->cols * c->dx)), psib);
  }
  // 3. reverse sweep, one recomputed segment at a time
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int t0 = sg * K, t1 = t0 + K < T ? t0 + K : T;
    cudaMemcpyAsync(psi_cur, ckpt + (size_t)sg * N, B, cudaMemcpyDeviceToDevice, s);
    for (int t = t0; t < t1; ++t) {
      const int q = t - t0;
      cudaMemcpyAsync(seg_psi + (size_t)q * N, psi_cur, B, cudaMemcpyDeviceToDevice, s);
      half_step_dispatch(c, psi_cur, c->la, c->sched[t], seg_f + (size_t)q * N, seg_S + (size_t)q * N);
      half_step_dispatch(c, seg_f + (size_t)q * N, c->lb, c->sched[t], psi_cur, seg_T + (size_t)q * N);
    }
    for (int t = t1 - 1; t >= t0; --t) {
      const int q = t - t0;
      const double e = c->sched[t];
      const float ie = (float)(1.0 / e);
      const float* f1 = seg_f + (size_t)q * N;
      // V-half: psi_{t+1} = eps (log b - T_t(f_{t+1}))
      axpy_kernel<<<gN, 256, 0, s>>>(bb, psib, (float)e, N);
      split_kernel<<<gN, 256, 0, s>>>(psib, seg_T + (size_t)q * N, (float)e, N, tA, tB);   // psibar e^{-T}
      half_step_dispatch(c, tA, neg_inf, e, scratch, Lp);
      half_step_dispatch(c, tB, neg_inf, e, scratch, Ln);
      combine_kernel<<<gN, 256, 0, s>>>(f1, ie, Lp, Ln, 1.f, N, fb);
      cudaMemsetAsync(psib, 0, B, s);
      // U-half: f_{t+1} = eps (log a - S_t(psi_t))
      axpy_kernel<<<gN, 256, 0, s>>>(ab, fb, (float)e, N);
      split_kernel<<<gN, 256, 0, s>>>(fb, seg_S + (size_t)q * N, (float)e, N, tA, tB);     // fbar e^{-S}
      half_step_dispatch(c, tA, neg_inf, e, scratch, Lp);
      half_step_dispatch(c, tB, neg_inf, e, scratch, Ln);
      combine_kernel<<<gN, 256, 0, s>>>(seg_psi + (size_t)q * N, ie, Lp, Ln, 1.f, N, psib);
      cudaMemsetAsync(fb, 0, B, s);
    }
  }
  // 4. through the normalisation to the amplitudes
  grad_from_logmarg<<<1, 256, 0, s>>>(ab, g, N, dL_dg);
  grad_from_logmarg<<<1, 256, 0, s>>>(bb, G, N, dL_dG);
  c->launches += 8;
  const cudaError_t le = cudaGetLastError();
  cleanup();
  if (le != cudaSuccess) return FOT_ECUDA;
  int e = 0;
  if (cudaMemcpy(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FOT_ECUDA;
  return (fot_status)e;
}
