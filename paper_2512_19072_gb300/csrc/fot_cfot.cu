// cFOT (Sec. 3.1): Algorithm 1 in the exponential domain with every product by the Toeplitz
// matrix Lambda replaced by a linear convolution with lambda_j = exp(-j^2 / (2 eps)),
// j = -(n-1) .. n-1, evaluated with FFTs:
//
//   u = a / (lambda * V * lambda),   V = b / (lambda * u * lambda).
//
// On its n outputs, the linear convolution of a line of length n with lambda equals the
// circular convolution of length P >= 2n - 1 (a power of two) of the zero-padded line with
// lambda wrapped around (lambda_j at index j mod P).  One CTA per line: a decimation-in-frequency
// FFT leaves the padded line in bit-reversed order, where it is multiplied by lambda's spectrum
// (real, lambda being even, and stored in that same order), and a decimation-in-time inverse FFT
// returns natural order.  Pass 0 convolves the rows and writes them transposed; pass 1
// convolves the columns and applies the update (u = e^{log a} / y, and log y for S_last).
//
// FP32 throughout, like the exponential-domain iteration the paper's cFOT is: an FFT
// convolution carries an absolute error of a few ulp of the line's largest value, so entries
// far below it lose their relative accuracy, and u, V leave the FP32 range once eps is small
// against the spread of the potentials.  A non-positive or non-finite convolution where the
// marginal has mass latches FOT_ENONFINITE: the cFOT instability Sec. 5 reports at small eps.
#include <math.h>

#include "fot_common.cuh"

namespace fot {
namespace {

constexpr int kConvThreads = 256;
constexpr int kConvMaxP = 4096;

__device__ __forceinline__ int bitrev(int i, int log2p) { return (int)(__brev((unsigned)i) >> (32 - log2p)); }

// hat[bitrev(q)] = sum_{|j| <= n-1} lambda_j e^{-2 pi i j q / P} = 1 + 2 sum_{j >= 1} lambda_j cos(2 pi j q / P)
__global__ void lambda_spectrum_kernel(float* __restrict__ hat, int n, int P, int log2p, double eps) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P) return;
  double acc = 1.0;
  for (int j = 1; j < n; ++j) {
    const double lam = exp(-(double)j * (double)j / (2.0 * eps));
    if (lam == 0.0) break;                                    // decreasing in j
    acc += 2.0 * lam * cospi(2.0 * (double)(((long long)j * q) % P) / (double)P);
  }
  hat[bitrev(q, log2p)] = (float)acc;
}

// PASS 0: y = (line of x) * lambda, written transposed: out[k][line].
// PASS 1: y likewise, then out[k][line] = e^{lmarg} / y and logsum[k][line] = log y.
template <int PASS>
__global__ void __launch_bounds__(kConvThreads) conv_line_kernel(const float* __restrict__ x,
                                                                 const float* __restrict__ hat,
                                                                 float* __restrict__ out,
                                                                 const float* __restrict__ lmarg,
                                                                 float* __restrict__ logsum, int* err,
                                                                 int n_lines, int n, int P, int log2p) {
  __shared__ float s_re[kConvMaxP], s_im[kConvMaxP];
  const int line = blockIdx.x;
  const float* xl = x + (size_t)line * n;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    s_re[i] = i < n ? xl[i] : 0.f;
    s_im[i] = 0.f;
  }
  // forward, decimation in frequency: pairs (i0, i0 + h) of each 2h block, twiddle e^{-i pi pos/h}
  for (int h = P >> 1; h >= 1; h >>= 1) {
    __syncthreads();
    for (int b = threadIdx.x; b < (P >> 1); b += blockDim.x) {
      const int pos = b & (h - 1);
      const int i0 = ((b - pos) << 1) + pos, i1 = i0 + h;
      float ws, wc;
      sincospif(-(float)pos / (float)h, &ws, &wc);
      const float ar = s_re[i0], ai = s_im[i0], br = s_re[i1], bi = s_im[i1];
      s_re[i0] = ar + br;
      s_im[i0] = ai + bi;
      const float dr = ar - br, di = ai - bi;
      s_re[i1] = dr * wc - di * ws;
      s_im[i1] = dr * ws + di * wc;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P; i += blockDim.x) {          // both in bit-reversed order
    const float hq = hat[i];
    s_re[i] *= hq;
    s_im[i] *= hq;
  }
  // inverse, decimation in time from bit-reversed order: twiddle e^{+i pi pos/h}
  for (int h = 1; h < P; h <<= 1) {
    __syncthreads();
    for (int b = threadIdx.x; b < (P >> 1); b += blockDim.x) {
      const int pos = b & (h - 1);
      const int i0 = ((b - pos) << 1) + pos, i1 = i0 + h;
      float ws, wc;
      sincospif((float)pos / (float)h, &ws, &wc);
      const float tr = wc * s_re[i1] - ws * s_im[i1];
      const float ti = wc * s_im[i1] + ws * s_re[i1];
      const float ar = s_re[i0], ai = s_im[i0];
      s_re[i1] = ar - tr;
      s_im[i1] = ai - ti;
      s_re[i0] = ar + tr;
      s_im[i0] = ai + ti;
    }
  }
  __syncthreads();
  const float scale = 1.f / (float)P;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const float y = s_re[k] * scale;
    const size_t o = (size_t)k * n_lines + line;
    if (PASS == 0) {
      out[o] = y;
    } else {
      const float lm = lmarg[o];
      float v = 0.f;
      if (lm != -INFINITY) {
        v = expf(lm) / y;
        if (!(y > 0.f) || !isfinite(v)) raise_error(err, FOT_ENONFINITE);
      }
      out[o] = v;
      if (logsum) logsum[o] = logf(y);
    }
  }
}

__global__ void fill_value_kernel(float* __restrict__ p, size_t N, float v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// exponential-domain scaling -> potential: p <- eps log p (-inf where p = 0)
__global__ void to_potential_kernel(float* __restrict__ p, size_t N, float eps) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const float v = p[i];
    p[i] = v > 0.f ? eps * logf(v) : -INFINITY;
  }
}

int pad_log2(int n) {                 // log2 of the smallest power of two >= 2n - 1
  int l = 0;
  while ((1 << l) < 2 * n - 1) ++l;
  return l;
}

}  // namespace

bool cfot_supported(int rows, int cols) {
  return rows >= 2 && cols >= 2 && (1 << pad_log2(rows)) <= kConvMaxP && (1 << pad_log2(cols)) <= kConvMaxP;
}

// eps_px: the px^2 value of every iteration (host array of iters).  The context's f and psi
// hold u and V during the loop and the potentials afterwards; c->lam_hat holds the two spectra
// (rows at 0, cols at kConvMaxP).
void cfot_run(fot_ctx* c, const double* eps_px, int iters) {
  const int nr = c->rows, nc = c->cols;
  const size_t N = (size_t)nr * nc;
  const int lr = pad_log2(nr), lc = pad_log2(nc), Pr = 1 << lr, Pc = 1 << lc;
  float* hat_r = c->lam_hat;
  float* hat_c = c->lam_hat + kConvMaxP;
  const int fill_blocks = c->red_blocks;
  fill_value_kernel<<<fill_blocks, 256, 0, c->stream>>>(c->psi, N, (float)(1.0 / ((double)nr * nc)));
  int64_t k = 1;
  double e_prev = -1.0;
  for (int t = 0; t < iters; ++t) {
    const double e = eps_px[t];
    if (e != e_prev) {
      lambda_spectrum_kernel<<<(Pr + 255) / 256, 256, 0, c->stream>>>(hat_r, nr, Pr, lr, e);
      lambda_spectrum_kernel<<<(Pc + 255) / 256, 256, 0, c->stream>>>(hat_c, nc, Pc, lc, e);
      k += 2;
      e_prev = e;
    }
    for (int half = 0; half < 2; ++half) {
      const float* in = half == 0 ? c->psi : c->f;       // V, then u
      float* outp = half == 0 ? c->f : c->psi;           // u, then V
      const float* lm = half == 0 ? c->la : c->lb;
      float* ls = (half == 0 && t == iters - 1) ? c->S_last : nullptr;
      conv_line_kernel<0><<<nr, kConvThreads, 0, c->stream>>>(in, hat_c, c->R, nullptr, nullptr, c->err, nr, nc,
                                                              Pc, lc);
      conv_line_kernel<1><<<nc, kConvThreads, 0, c->stream>>>(c->R, hat_r, outp, lm, ls, c->err, nc, nr, Pr,
                                                              lr);
      k += 2;
    }
  }
  const float el = (float)eps_px[iters - 1];
  to_potential_kernel<<<fill_blocks, 256, 0, c->stream>>>(c->f, N, el);
  to_potential_kernel<<<fill_blocks, 256, 0, c->stream>>>(c->psi, N, el);
  c->launches += k + 2;
}

size_t cfot_spectrum_floats() { return 2 * (size_t)kConvMaxP; }

}  // namespace fot
