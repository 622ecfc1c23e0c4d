// Far-field intensity and the L1 intensity loss of a phase solution (Sec. 5).
//
//   I = |F[g e^{2 pi i phi}]|^2,   loss = sum_LM | I_LM / sum I - b_LM |,
//
// F the 2-D DFT between the centred grids of Sec. 2 (x_j = (j - floor(n/2)) dx, X_L =
// (L - floor(n/2)) dX, dx dX = 1/n).  The centring multiplies each output of the plain DFT by a
// unit-modulus factor that depends on the output index alone, so I at (L, M) is the squared
// modulus of the plain DFT at ((L - c_r) mod n_r, (M - c_c) mod n_c): the kernels compute plain
// DFTs and write each intensity at its shifted position.  The amplitude is sqrt(a) = e^{log a / 2}
// (a = g^2 / sum g^2; the overall scale cancels in I / sum I).
//
// One radix-2 kernel, launched twice (power-of-two lengths up to 4096): one CTA per line, the
// line held in shared memory in bit-reversed order, log2(len) butterfly stages with twiddles
// from sincospif.  Pass 0 transforms the rows of the field and writes the spectrum transposed as
// split real / imaginary planes; pass 1 transforms those lines (the columns) and writes
// |.|^2 at the shifted position.  Two FP64 reductions follow: the total power, then
// sum |I / P - b| (which also leaves I / P in place).
#include "fot_common.cuh"

namespace fot {
namespace {

constexpr int kFftThreads = 256;
constexpr int kFftMaxLen = 4096;

template <int PASS>
__global__ void __launch_bounds__(kFftThreads) fft_line_kernel(
    const float* __restrict__ la, const float* __restrict__ phi,       // pass 0: [n_lines][len]
    const float* __restrict__ re_in, const float* __restrict__ im_in,  // pass 1: [n_lines][len]
    float* __restrict__ re_out, float* __restrict__ im_out,            // pass 0: [len][n_lines]
    float* __restrict__ inten,                                          // pass 1: [len][n_lines]
    int n_lines, int len, int log2len, int c_len, int c_line) {
  __shared__ float s_re[kFftMaxLen], s_im[kFftMaxLen];
  const int line = blockIdx.x;
  const size_t base = (size_t)line * len;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    float re, im;
    if (PASS == 0) {
      const float amp = expf(0.5f * la[base + i]);           // log a = -inf -> 0
      float sn, cs;
      sincospif(2.f * phi[base + i], &sn, &cs);                  // e^{2 pi i phi}, phi in cycles
      re = amp * cs;
      im = amp * sn;
    } else {
      re = re_in[base + i];
      im = im_in[base + i];
    }
    const int r = (int)(__brev((unsigned)i) >> (32 - log2len));
    s_re[r] = re;
    s_im[r] = im;
  }
  // butterflies: stage with half-size h pairs i0 = 2h*group + pos and i1 = i0 + h, twiddle
  // e^{-i pi pos / h}
  for (int h = 1; h < len; h <<= 1) {
    __syncthreads();
    for (int b = threadIdx.x; b < len / 2; b += blockDim.x) {
      const int pos = b & (h - 1);
      const int i0 = ((b - pos) << 1) + pos, i1 = i0 + h;
      float ws, wc;
      sincospif(-(float)pos / (float)h, &ws, &wc);
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
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    if (PASS == 0) {
      re_out[(size_t)i * n_lines + line] = s_re[i];
      im_out[(size_t)i * n_lines + line] = s_im[i];
    } else {
      // line = spectral column index, i = spectral row index
      const int L = (i + c_len) & (len - 1), M = (line + c_line) & (n_lines - 1);
      inten[(size_t)L * n_lines + M] = s_re[i] * s_re[i] + s_im[i] * s_im[i];
    }
  }
}

// STEP 0: part[b] = sum of v over the block's share; STEP 1: with P = *total,
// v <- v / P in place and part[b] = sum |v / P - e^{lb}|
template <int STEP>
__global__ void __launch_bounds__(256) intensity_partials_kernel(float* __restrict__ v,
                                                                const float* __restrict__ lb,
                                                                const double* __restrict__ total,
                                                                size_t N, double* __restrict__ part) {
  __shared__ double s[256];
  double acc = 0.0;
  const double inv = STEP == 1 ? 1.0 / *total : 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    if (STEP == 0) {
      acc += (double)v[i];
    } else {
      const double q = (double)v[i] * inv;
      v[i] = (float)q;
      const float l = lb[i];
      acc += fabs(q - (l == -INFINITY ? 0.0 : exp((double)l)));
    }
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(256) sum_parts_kernel(const double* __restrict__ part, int n, double* out) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

int log2_exact(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return (1 << l) == n ? l : -1;
}

}  // namespace

bool intensity_supported(int rows, int cols) {
  return rows >= 2 && cols >= 2 && rows <= kFftMaxLen && cols <= kFftMaxLen && log2_exact(rows) > 0 &&
         log2_exact(cols) > 0;
}

// I / P into c->tmp and the loss into out[0] (device); c->R, c->R2 hold the spectrum between
// the passes.  The caller checked intensity_supported.
void intensity_loss_gpu(fot_ctx* c, const float* phi, double* out) {
  const int nr = c->rows, nc = c->cols;
  const size_t N = (size_t)nr * nc;
  fft_line_kernel<0><<<nr, kFftThreads, 0, c->stream>>>(c->la, phi, nullptr, nullptr, c->R, c->R2, nullptr,
                                                        nr, nc, log2_exact(nc), 0, 0);
  fft_line_kernel<1><<<nc, kFftThreads, 0, c->stream>>>(nullptr, nullptr, c->R, c->R2, nullptr, nullptr,
                                                        c->tmp, nc, nr, log2_exact(nr), nr / 2, nc / 2);
  double* part = c->red;
  intensity_partials_kernel<0><<<c->red_blocks, 256, 0, c->stream>>>(c->tmp, nullptr, nullptr, N, part);
  sum_parts_kernel<<<1, 256, 0, c->stream>>>(part, c->red_blocks, out + 1);
  intensity_partials_kernel<1><<<c->red_blocks, 256, 0, c->stream>>>(c->tmp, c->lb, out + 1, N, part);
  sum_parts_kernel<<<1, 256, 0, c->stream>>>(part, c->red_blocks, out);
  c->launches += 6;
}

}  // namespace fot
