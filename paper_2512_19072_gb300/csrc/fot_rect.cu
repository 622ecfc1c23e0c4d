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
// f = eps (log a - S) in its epilogue.  The same kernels in FP64 (exp2 / log2 of the CUDA math
// library in double precision) give fot_solve_rect_fp64, a GPU reference for equal or unequal
// grids.
#include "fot_common.cuh"

#include <algorithm>
#include <vector>

namespace fot {

namespace {

constexpr int kRectRows = 4;             // input rows per CTA (staged in shared memory)
constexpr int kRectThreads = 256;        // outputs per CTA
constexpr int kRectMaxLen = 3072;        // longest axis: kRectRows * len floats in 48 KB

// 2^x and log2 x in the working precision: the MUFU forms in FP32, the math library in FP64
__device__ __forceinline__ float rect_ex2(float x) { return ex2(x); }
__device__ __forceinline__ double rect_ex2(double x) { return exp2(x); }
__device__ __forceinline__ float rect_lg2(float x) { return log2f(x); }
__device__ __forceinline__ double rect_lg2(double x) { return log2(x); }

template <bool POT, typename T>
__global__ void __launch_bounds__(kRectThreads) rect_pass_kernel(const T* __restrict__ x, int n_rows, int len_in,
                                                                  int len_out, T shift, T x_scale, T c,
                                                                  const T* __restrict__ lmarg, T eps,
                                                                  T* __restrict__ y, int* err) {
  extern __shared__ __align__(16) unsigned char rect_smem[];
  T* sx = reinterpret_cast<T*>(rect_smem);                // [len_in][kRectRows]
  const int r0 = blockIdx.y * kRectRows;
  for (int i = threadIdx.x; i < len_in * kRectRows; i += blockDim.x) {
    const int r = i / len_in, m = i - r * len_in;
    sx[m * kRectRows + r] = r0 + r < n_rows ? x[(size_t)(r0 + r) * len_in + m] * x_scale : (T)-INFINITY;
  }
  __syncthreads();
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= len_out) return;
  const T d0 = (T)o + shift;                              // distance to m = 0
  T mx[kRectRows];
#pragma unroll
  for (int r = 0; r < kRectRows; ++r) mx[r] = (T)-INFINITY;
  for (int m = 0; m < len_in; ++m) {
    const T d = d0 - (T)m;
    const T t = -d * d * c;
#pragma unroll
    for (int r = 0; r < kRectRows; ++r) mx[r] = fmax(mx[r], t + sx[m * kRectRows + r]);
  }
  T acc[kRectRows];
#pragma unroll
  for (int r = 0; r < kRectRows; ++r) acc[r] = (T)0;
  for (int m = 0; m < len_in; ++m) {
    const T d = d0 - (T)m;
    const T t = -d * d * c;
#pragma unroll
    for (int r = 0; r < kRectRows; ++r)
      if (mx[r] != (T)-INFINITY) acc[r] += rect_ex2(t + sx[m * kRectRows + r] - mx[r]);
  }
  const T ln2 = (T)0.69314718055994530942;
#pragma unroll
  for (int r = 0; r < kRectRows; ++r) {
    if (r0 + r >= n_rows) break;
    const size_t yi = (size_t)o * n_rows + r0 + r;
    const T s2 = mx[r] == (T)-INFINITY ? (T)-INFINITY : mx[r] + rect_lg2(acc[r]);
    if (!POT) {
      y[yi] = s2;
    } else {
      const T lm = lmarg[yi];
      T pot;
      if (lm == (T)-INFINITY) {
        pot = (T)-INFINITY;
      } else {
        pot = eps * (lm - s2 * ln2);
        if (!isfinite(pot)) raise_error(err, FOT_ENONFINITE);
      }
      y[yi] = pot;
    }
  }
}

// sum of amp^2 in FP64 (one CTA)
template <typename T>
__global__ void rect_power_kernel(const T* __restrict__ amp, size_t n, double* out) {
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
template <typename T>
__global__ void rect_logmarg_kernel(const T* __restrict__ amp, size_t n, const double* sum, T* __restrict__ lm) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = amp[i];
  lm[i] = v == 0.0 ? (T)-INFINITY : (T)log(v * v / *sum);
}

template <typename T>
__global__ void rect_fill_kernel(T* p, size_t n, T v) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

template <bool POT, typename T>
void rect_pass(cudaStream_t s, const T* x, int n_rows, int len_in, int len_out, double eps, T x_scale,
               const T* lmarg, T* y, int* err) {
  const dim3 grid((len_out + kRectThreads - 1) / kRectThreads, (n_rows + kRectRows - 1) / kRectRows);
  const T c = (T)(1.4426950408889634 / (2.0 * eps));
  const T shift = (T)0.5 * (T)(len_in - len_out);
  rect_pass_kernel<POT, T><<<grid, kRectThreads, (size_t)len_in * kRectRows * sizeof(T), s>>>(
      x, n_rows, len_in, len_out, shift, x_scale, c, lmarg, (T)eps, y, err);
}

template <typename T>
fot_status solve_rect(const T* g, int rows_in, int cols_in, const T* G, int rows_out, int cols_out,
                      const double* eps, int n_eps, int iters, T* f_out, T* psi_out, void* cuda_stream) {
  if (!g || !G || !eps || !f_out || !psi_out || iters < 1) return FOT_EINVAL;
  if (n_eps != 1 && n_eps != iters) return FOT_EINVAL;
  const int max_len = sizeof(T) == 4 ? kRectMaxLen : kRectMaxLen / 2;   // staged rows in 48 KB
  for (int d : {rows_in, cols_in, rows_out, cols_out})
    if (d < 1 || d > max_len) return FOT_EINVAL;
  for (int t = 0; t < n_eps; ++t)
    if (!(eps[t] > 0.0) || !isfinite(eps[t])) return FOT_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t ni = (size_t)rows_in * cols_in, no = (size_t)rows_out * cols_out;
  const size_t nr = std::max((size_t)cols_in * rows_out, (size_t)cols_out * rows_in);
  T *la = nullptr, *lb = nullptr, *R = nullptr;
  double* sums = nullptr;
  int* err = nullptr;
  bool ok = cudaMalloc((void**)&la, ni * sizeof(T)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&lb, no * sizeof(T)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&R, nr * sizeof(T)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&sums, 2 * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&err, sizeof(int)) == cudaSuccess;
  fot_status st = FOT_OK;
  if (!ok) {
    cudaGetLastError();
    st = FOT_ENOMEM;
  } else {
    double h[2] = {0.0, 0.0};
    cudaMemsetAsync(err, 0, sizeof(int), s);
    rect_power_kernel<T><<<1, 1024, 0, s>>>(g, ni, sums);
    rect_power_kernel<T><<<1, 1024, 0, s>>>(G, no, sums + 1);
    cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      st = FOT_ECUDA;
    } else if (!(h[0] > 0.0) || !(h[1] > 0.0) || !isfinite(h[0]) || !isfinite(h[1])) {
      st = FOT_EMASS;
    } else {
      rect_logmarg_kernel<T><<<(unsigned)((ni + 255) / 256), 256, 0, s>>>(g, ni, sums, la);
      rect_logmarg_kernel<T><<<(unsigned)((no + 255) / 256), 256, 0, s>>>(G, no, sums + 1, lb);
      // Algorithm 1 start: V = 1 / (rows_out cols_out)  ->  psi0 = eps_0 log(1 / (rows_out cols_out))
      rect_fill_kernel<T><<<(unsigned)((no + 255) / 256), 256, 0, s>>>(psi_out, no, (T)(eps[0] * log(1.0 / (double)no)));
      for (int t = 0; t < iters; ++t) {
        const double e = eps[n_eps == 1 ? 0 : t];
        const T xs = (T)(1.4426950408889634 / e);
        // Eq. 7: S over the input grid from psi (columns, then rows), f = eps (log a - S)
        rect_pass<false, T>(s, psi_out, rows_out, cols_out, cols_in, e, xs, nullptr, R, err);   // R[k][L]
        rect_pass<true, T>(s, R, cols_in, rows_out, rows_in, e, (T)1, la, f_out, err);         // f[j][k]
        // Eq. 8: T over the output grid from f, psi = eps (log b - T)
        rect_pass<false, T>(s, f_out, rows_in, cols_in, cols_out, e, xs, nullptr, R, err);      // R[M][j]
        rect_pass<true, T>(s, R, cols_out, rows_in, rows_out, e, (T)1, lb, psi_out, err);      // psi[L][M]
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

}  // namespace

}  // namespace fot

using namespace fot;

extern "C" fot_status fot_solve_rect(const float* g, int rows_in, int cols_in, const float* G, int rows_out,
                                     int cols_out, const double* eps, int n_eps, int iters, float* f_out,
                                     float* psi_out, void* cuda_stream) {
  return solve_rect<float>(g, rows_in, cols_in, G, rows_out, cols_out, eps, n_eps, iters, f_out, psi_out, cuda_stream);
}

extern "C" fot_status fot_solve_rect_fp64(const double* g, int rows_in, int cols_in, const double* G, int rows_out,
                                          int cols_out, const double* eps, int n_eps, int iters, double* f_out,
                                          double* psi_out, void* cuda_stream) {
  return solve_rect<double>(g, rows_in, cols_in, G, rows_out, cols_out, eps, n_eps, iters, f_out, psi_out,
                            cuda_stream);
}
