// Exact c-transform of a potential image for the quadratic cost, the eps -> 0 limit of a
// half-step (Eqs. 7-8 with the entropic log-sum-exp replaced by its maximum):
//     out_jk = min_LM [ ((j-L)^2 + (k-M)^2)/2 - pot_LM ].
// The cost is separable (Sec. 2), so this is one 1-D transform along each row followed by
// one along each column.  Each 1-D transform
//     Y(o) = max_m [ z_m - (o - m)^2 / 2 ]
// is the lower envelope of the parabolas (o - m)^2/2 - z_m (Felzenszwalb and Huttenlocher,
// "Distance transforms of sampled functions", 2012): O(len) per line.  One thread scans one
// line; the envelope (parabola apex index and left boundary) lives in per-line scratch.
// -inf inputs (zero mass) are not parabolas; a line with none yields -inf.
#include "fot_common.cuh"

namespace fot {

// One line: x[m] (stride 1), writes y[o * ystride] = sign * max_m (x[m] - (o-m)^2/2).
// v: apex index of envelope parabola i, zb: left boundary of parabola i (float).
__device__ void envelope_line(const float* __restrict__ x, int len, float* y, size_t ystride,
                              float sign, int* __restrict__ v, float* __restrict__ zb) {
  int top = -1;
  for (int q = 0; q < len; ++q) {
    const float xq = x[q];
    if (xq == -INFINITY) continue;
    // parabola q: P_q(o) = (o - q)^2 / 2 - xq; intersection with the top parabola p:
    // s = ((q^2/2 - xq) - (p^2/2 - xp)) / (q - p)
    const double hq = 0.5 * (double)q * q - (double)xq;
    double s = -INFINITY;
    while (top >= 0) {
      const int p = v[top];
      const double hp = 0.5 * (double)p * p - (double)x[p];
      s = (hq - hp) / (double)(q - p);
      if (s > (double)zb[top]) break;
      --top;   // parabola p never attains the minimum
    }
    if (top < 0) s = -INFINITY;
    ++top;
    v[top] = q;
    zb[top] = (float)s;
  }
  if (top < 0) {
    for (int o = 0; o < len; ++o) y[(size_t)o * ystride] = sign * -INFINITY;
    return;
  }
  int i = 0;
  for (int o = 0; o < len; ++o) {
    while (i < top && (double)zb[i + 1] <= (double)o) ++i;
    const int p = v[i];
    const double d = (double)(o - p);
    y[(size_t)o * ystride] = sign * (float)((double)x[p] - 0.5 * d * d);
  }
}

// rows of x [n_rows][len] -> y[o][r] (transposed), y = sign * envelope max
__global__ void envelope_pass_kernel(const float* __restrict__ x, int n_rows, int len, float* y,
                                     float sign, int* vscr, float* zscr, const int* err) {
  if (error_latched(err)) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  envelope_line(x + (size_t)r * len, len, y + r, (size_t)n_rows, sign, vscr + (size_t)r * len,
                zscr + (size_t)r * len);
}

void c_transform_envelope(fot_ctx* c, const float* pot_in, float* out) {
  // scratch: envelope indices in tmp (as int), boundaries in tmp2; intermediate in R
  int* vscr = reinterpret_cast<int*>(c->tmp);
  float* zscr = c->tmp2;
  const int t = 64;
  // along rows (contiguous M): R[k][L] = max_M (pot_LM - (k-M)^2/2)
  envelope_pass_kernel<<<(c->rows + t - 1) / t, t, 0, c->stream>>>(pot_in, c->rows, c->cols, c->R,
                                                                   1.f, vscr, zscr, c->err);
  // along columns (contiguous L in R): out[j][k] = -max_L (R[k][L] - (j-L)^2/2)
  envelope_pass_kernel<<<(c->cols + t - 1) / t, t, 0, c->stream>>>(c->R, c->cols, c->rows, out,
                                                                   -1.f, vscr, zscr, c->err);
  c->launches += 2;
}

}  // namespace fot
