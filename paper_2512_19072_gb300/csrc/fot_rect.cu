// Algorithm 1 between an input grid and an output grid of different sizes (fot_solve_rect).
//
// Sec. 2 notes that square, equal arrays are not essential.  With centre-aligned unit-spaced
// pixel coordinates on both planes the cost still separates and each Lambda product becomes a
// rectangular 1-D contraction.  Every axis pass here is dense and exact:
//     y[o][r] = log2 sum_m 2^( x[r][m]*scale - (o - m + shift)^2 c ),   c = log2(e)/(2 eps),
// o over the output axis (len_out), m over the input axis (len_in), shift = (len_in - len_out)/2
// the offset between the two centre-aligned axes; the result is written transposed.  Two sweeps
// per output: its exact maximum, then the sum of 2^(e - max) (the FP32 dense form of the square
// passes, FOT_FP32_DENSE).  The second pass of a half-step applies the potential update
// f = eps (log a - S) in its epilogue.
#include "fot_common.cuh"

#include <algorithm>
#include <vector>

namespace fot {

namespace {

constexpr int kRectRows = 4;             // input rows per CTA (staged in shared memory)
constexpr int kRectThreads = 256;        // outputs per CTA
constexpr int kRectMaxLen = 3072;        // longest axis: kRectRows * len floats in 48 KB

template <bool POT>
__global__ void __launch_bounds__(kRectThreads) rect_pass_kernel(const float* __restrict__ x, int n_rows, int len_in,
                                                                  int len_out, float shift, float x_scale, float c,
                                                                  const float* __restrict__ lmarg, float eps,
                                                                  float* __restrict__ y, int* err) {
  extern __shared__ float sx[];                           // [len_in][kRectRows]
  const int r0 = blockIdx.y * kRectRows;
  for (int i = threadIdx.x; i < len_in * kRectRows; i += blockDim.x) {
    const int r = i / len_in, m = i - r * len_in;
    sx[m * kRectRows + r] = r0 + r < n_rows ? x[(size_t)(r0 + r) * len_in + m] * x_scale : -INFINITY;
  }
  __syncthreads();
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= len_out) return;
  const float d0 = (float)o + shift;                      // distance to m = 0
  float mx[kRectRows];
#pragma unroll
  for (int r = 0; r < kRectRows; ++r) mx[r] = -INFINITY;
  for (int m = 0; m < len_in; ++m) {
    const float d = d0 - (float)m;
    const float t = -d * d * c;
#pragma unroll
    for (int r = 0; r < kRectRows; ++r) mx[r] = fmaxf(mx[r], t + sx[m * kRectRows + r]);
  }
  float acc[kRectRows];
#pragma unroll
  for (int r = 0; r < kRectRows; ++r) acc[r] = 0.f;
  for (int m = 0; m < len_in; ++m) {
    const float d = d0 - (float)m;
    const float t = -d * d * c;
#pragma unroll
    for (int r = 0; r < kRectRows; ++r)
      if (mx[r] != -INFINITY) acc[r] += ex2(t + sx[m * kRectRows + r] - mx[r]);
  }
#pragma unroll
  for (int r = 0; r < kRectRows; ++r) {
    if (r0 + r >= n_rows) break;
    const size_t yi = (size_t)o * n_rows + r0 + r;
    const float s2 = mx[r] == -INFINITY ? -INFINITY : mx[r] + log2f(acc[r]);
    if (!POT) {
      y[yi] = s2;
    } else {
      const float lm = lmarg[yi];
      float pot;
      if (lm == -INFINITY) {
        pot = -INFINITY;
      } else {
        pot = eps * (lm - s2 * kLn2);
        if (!isfinite(pot)) raise_error(err, FOT_ENONFINITE);
      }
      y[yi] = pot;
    }
  }
}

// sum of amp^2 in FP64 (one CTA)
__global__ void rect_power_kernel(const float* __restrict__ amp, size_t n, double* out) {
  __shared__ double s[1024];
  double acc = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = amp[i];
    acc += v * v;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// log of the marginal g^2 / sum g^2 (log 0 = -inf)
__global__ void rect_logmarg_kernel(const float* __restrict__ amp, size_t n, const double* sum,
                                    float* __restrict__ lm) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = amp[i];
  lm[i] = v == 0.0 ? -INFINITY : (float)log(v * v / *sum);
}

__global__ void rect_fill_kernel(float* p, size_t n, float v) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

template <bool POT>
void rect_pass(cudaStream_t s, const float* x, int n_rows, int len_in, int len_out, double eps, float x_scale,
               const float* lmarg, float* y, int* err) {
  const dim3 grid((len_out + kRectThreads - 1) / kRectThreads, (n_rows + kRectRows - 1) / kRectRows);
  const float c = (float)(1.4426950408889634 / (2.0 * eps));
  const float shift = 0.5f * (float)(len_in - len_out);
  rect_pass_kernel<POT><<<grid, kRectThreads, (size_t)len_in * kRectRows * sizeof(float), s>>>(
      x, n_rows, len_in, len_out, shift, x_scale, c, lmarg, (float)eps, y, err);
}

}  // namespace

}  // namespace fot

using namespace fot;

extern "C" fot_status fot_solve_rect(const float* g, int rows_in, int cols_in, const float* G, int rows_out,
                                     int cols_out, const double* eps, int n_eps, int iters, float* f_out,
                                     float* psi_out, void* cuda_stream) {
  if (!g || !G || !eps || !f_out || !psi_out || iters < 1) return FOT_EINVAL;
  if (n_eps != 1 && n_eps != iters) return FOT_EINVAL;
  for (int d : {rows_in, cols_in, rows_out, cols_out})
    if (d < 1 || d > kRectMaxLen) return FOT_EINVAL;
  for (int t = 0; t < n_eps; ++t)
    if (!(eps[t] > 0.0) || !isfinite(eps[t])) return FOT_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t ni = (size_t)rows_in * cols_in, no = (size_t)rows_out * cols_out;
  const size_t nr = std::max((size_t)cols_in * rows_out, (size_t)cols_out * rows_in);
  float *la = nullptr, *lb = nullptr, *R = nullptr;
  double* sums = nullptr;
  int* err = nullptr;
  bool ok = cudaMalloc((void**)&la, ni * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&lb, no * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&R, nr * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&sums, 2 * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&err, sizeof(int)) == cudaSuccess;
  fot_status st = FOT_OK;
  if (!ok) {
    cudaGetLastError();
    st = FOT_ENOMEM;
  } else {
    double h[2] = {0.0, 0.0};
    cudaMemsetAsync(err, 0, sizeof(int), s);
    rect_power_kernel<<<1, 1024, 0, s>>>(g, ni, sums);
    rect_power_kernel<<<1, 1024, 0, s>>>(G, no, sums + 1);
    cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      st = FOT_ECUDA;
    } else if (!(h[0] > 0.0) || !(h[1] > 0.0) || !isfinite(h[0]) || !isfinite(h[1])) {
      st = FOT_EMASS;
    } else {
      rect_logmarg_kernel<<<(unsigned)((ni + 255) / 256), 256, 0, s>>>(g, ni, sums, la);
      rect_logmarg_kernel<<<(unsigned)((no + 255) / 256), 256, 0, s>>>(G, no, sums + 1, lb);
      // Algorithm 1 start: V = 1 / (rows_out cols_out)  ->  psi0 = eps_0 log(1 / (rows_out cols_out))
      rect_fill_kernel<<<(unsigned)((no + 255) / 256), 256, 0, s>>>(psi_out, no,
                                                                     (float)(eps[0] * log(1.0 / (double)no)));
      for (int t = 0; t < iters; ++t) {
        const double e = eps[n_eps == 1 ? 0 : t];
        const float xs = (float)(1.4426950408889634 / e);
        // Eq. 7: S over the input grid from psi (columns, then rows), f = eps (log a - S)
        rect_pass<false>(s, psi_out, rows_out, cols_out, cols_in, e, xs, nullptr, R, err);   // R[k][L]
        rect_pass<true>(s, R, cols_in, rows_out, rows_in, e, 1.f, la, f_out, err);          // f[j][k]
        // Eq. 8: T over the output grid from f, psi = eps (log b - T)
        rect_pass<false>(s, f_out, rows_in, cols_in, cols_out, e, xs, nullptr, R, err);      // R[M][j]
        rect_pass<true>(s, R, cols_out, rows_in, rows_out, e, 1.f, lb, psi_out, err);       // psi[L][M]
      }
      int herr = 0;
      cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        st = FOT_ECUDA;
      else if (herr != 0)
        st = (fot_status)herr;
    }
  }
  cudaFree(la);
  cudaFree(lb);
  cudaFree(R);
  cudaFree(sums);
  cudaFree(err);
  return st;
}
