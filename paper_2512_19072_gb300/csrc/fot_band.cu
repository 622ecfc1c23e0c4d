// Banded axis passes: the same contraction as the exact pass,
//     y[o][r] = log2 sum_m 2^( x[r][m]*scale - (o - m)^2 c ),   c = log2(e) / (2 eps),
// but each output only visits the terms that can matter, and for large eps the inner loop
// is a plain FP32 multiply-add GEMM instead of one exponential per term.
//
// Work unit: one warp, 16 input rows r x one tile of 16 consecutive outputs o = k0 + i; lane
// (h, i) = (lane / 16, lane % 16) owns rows 8h .. 8h+7 and output i.  Steps 1-2 run in
// band_plan_kernel (one CTA per row) and leave (alpha, lo, window length) per (row, tile);
// steps 3-4 run in band_pass_kernel.
//
// 1. Exact offset at every tile centre kc = k0 + 8:  alpha_r = max_m e_r(m, kc),
//    e_r(m, o) = x_r[m] - (o - m)^2 c, and its argmax, found by scanning only the 32-wide
//    chunks of m whose upper bound (chunk maximum of x, nearest distance) beats the best
//    term found so far.
// 2. A provable window: every o in the tile has max_m e_r(m, o) >= LB_r, with LB_r the
//    value of the centre's argmax term at the worse tile end.  A 32-wide chunk of m whose
//    upper bound (chunk maximum of x, nearest distance) over the whole tile is below
//    LB_r - 40 holds only terms below 2^-40 of every output of the tile; the window is the
//    hull of the remaining chunks (relative truncation error < len * 2^-40).
// 3. Tilt identity (large eps).  With o = kc + kap:
//      e_r(m, o) = [x_r[m] - (kc - m)^2 c - alpha_r] + [2 kap (m - Mref_r) c - kap^2 c]
//                  + alpha_r + 2 kap (Mref_r - kc) c,
//    so  sum_m 2^e = 2^(alpha_r + 2 kap (Mref_r - kc) c) * sum_m' A[r][m'] B[m'][kap]
//    with A[r][m'] = 2^(e_r(lo_r + m', kc) - alpha_r) <= 1 (one exponential per row and
//    window position, shared by the tile's outputs) and B[m'][kap] = 2^(2 kap (m' - W/2) c -
//    kap^2 c), the same for every row once each row's window is indexed from its own start
//    lo_r (Mref_r = lo_r + W/2).  This is a GEMM over the window, done with FFMAs; the
//    per-row offsets are the "online softmax" max-offsets of the paper's Toeplitz
//    contraction (Sec. 3.1).  It is used when |B| stays within 2^+-40 and kap^2 c <= 32.
// 4. Otherwise (small eps: narrow kernel, narrow windows) each output takes its exact
//    maximum and sum over the window only.
#include "fot_band_item.cuh"

#include <algorithm>

namespace fot {

// Per (row, tile) plan (tiles of tile_w = 16 or 64 outputs): exact centre offset alpha, window
// start lo and length wl.  One CTA per row.  The row, scaled to log2 units, is staged in shared memory with one pad
// word per 32-wide chunk (threads scanning different chunks at the same offset hit different
// banks), together with the chunk maxima and the row maximum.  Each thread then plans its
// own tiles:
//   a. alpha: scan the chunk holding the centre kc, then every chunk whose upper bound
//      (chunk maximum less the nearest squared distance times c) beats the running best.
//      The bound never undershoots the rounded terms it stands for (d*d is exact and the
//      fused multiply-add rounds monotonically), so the maximum is exact for any input;
//      chunks farther from kc than sqrt((row max - best) / c) cannot qualify and are not
//      visited.  For the concave rows of converged potentials one or two chunks qualify.
//   b. the window of step 2 above, from the same chunk maxima.
constexpr int kPlanThreads = 128;
constexpr int kMaxChunks = 4096 / kCW;        // longest axis 4096
constexpr int kMaskWords = kMaxChunks / 32;

template <int MAXP>
__global__ void __launch_bounds__(kPlanThreads) band_plan_kernel(const __grid_constant__ BandTable<MAXP> tab) {
  __shared__ float s_x[kMaxChunks * (kCW + 1)];
  __shared__ float s_cm[kMaxChunks];
  __shared__ float s_rowmax;
  const BandArgs& a = tab.p[find_prob<MAXP, 1>(tab, (int)blockIdx.x)];
  if (error_latched(a.err)) return;                       // CTA-uniform
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = (int)blockIdx.x - a.plan_base;
  const int T = a.n_tiles, len = a.len, nch = a.n_chunks;
  const float c = a.c, sc = a.x_scale;
  const float* xr = a.x + (size_t)row * len;
  for (int m = tid; m < nch * kCW; m += kPlanThreads)
    s_x[(m >> 5) * (kCW + 1) + (m & 31)] = m < len ? xr[m] * sc : -INFINITY;
  __syncthreads();
  // max(x) * sc == max(x * sc): sc > 0 and rounding is monotone
  for (int j = warp; j < nch; j += kPlanThreads / 32) {
    const float v = warp_max(s_x[j * (kCW + 1) + lane]);
    if (lane == 0) s_cm[j] = v;
  }
  __syncthreads();
  if (warp == 0) {
    float v = -INFINITY;
    for (int j = lane; j < nch; j += 32) v = fmaxf(v, s_cm[j]);
    v = warp_max(v);
    if (lane == 0) s_rowmax = v;
  }
  __syncthreads();
  const float X = s_rowmax;
  const size_t np = (size_t)a.n_rows * T;
  float* p_alpha = a.plan;
  int* p_lo = reinterpret_cast<int*>(a.plan + np);
  int* p_wl = reinterpret_cast<int*>(a.plan + 2 * np);

  const int tw = a.tile_w;
  for (int t = tid; t < T; t += kPlanThreads) {
    const int k0 = t * tw, kc = k0 + tw / 2, k1 = min(k0 + tw, len) - 1;
    float best = -INFINITY;
    int arg = 0;
    auto scan = [&](int j) {
      const float* xs = &s_x[j * (kCW + 1)];
      const float d0 = (float)(kc - j * kCW);
#pragma unroll 8
      for (int u = 0; u < kCW; ++u) {
        const float d = d0 - (float)u;
        const float v = fmaf(-d * d, c, xs[u]);
        if (v > best) {
          best = v;
          arg = j * kCW + u;
        }
      }
    };
    // a. exact centre maximum
    const int jc = min(kc, len - 1) / kCW;
    scan(jc);
    int jlo = 0, jhi = nch - 1;
    if (best != -INFINITY) {          // a chunk at distance dist needs X - dist^2 c > best
      const float R = sqrtf((X - best) / c) * 1.01f + 2.f * kCW;
      jlo = (int)fmaxf(0.f, floorf(((float)kc - R) / (float)kCW));
      jhi = (int)fminf((float)(nch - 1), floorf(((float)kc + R) / (float)kCW));
    }
    unsigned cand[kMaskWords];
#pragma unroll
    for (int w = 0; w < kMaskWords; ++w) {
      unsigned mk = 0;
      const int ja = max(jlo, 32 * w), jb = min(jhi, 32 * w + 31);
      for (int j = ja; j <= jb; ++j) {
        const float d = (float)chunk_dist(j, kc, kc, len);
        if (j != jc && fmaf(-d * d, c, s_cm[j]) > best) mk |= 1u << (j - 32 * w);
      }
      cand[w] = mk;
    }
#pragma unroll
    for (int w = 0; w < kMaskWords; ++w) {
      unsigned mk = cand[w];
      while (mk) {
        const int j = 32 * w + __ffs(mk) - 1;
        mk &= mk - 1;
        const float d = (float)chunk_dist(j, kc, kc, len);
        if (fmaf(-d * d, c, s_cm[j]) > best) scan(j);   // best may have risen meanwhile
      }
    }
    const size_t pi = (size_t)row * T + t;
    if (best == -INFINITY) {                              // no finite term: empty row
      p_alpha[pi] = -INFINITY;
      p_lo[pi] = 0;
      p_wl[pi] = 0;
      continue;
    }
    // b. window: lower bound over the tile from the argmax term at the worse tile end, then
    // the first and the last chunk whose bound over the tile reaches lb - kCut
    const float dM = (float)(arg - kc);
    const float ka = (float)(k0 - kc), kb = (float)(k1 - kc);
    const float lb = best + fminf(fmaf(2.f * ka, dM * c, -ka * ka * c), fmaf(2.f * kb, dM * c, -kb * kb * c));
    const float R2 = sqrtf((X - (lb - kCut)) / c) * 1.01f + 2.f * kCW;
    const int ja = (int)fmaxf(0.f, floorf(((float)k0 - R2) / (float)kCW));
    const int jb = (int)fminf((float)(nch - 1), floorf(((float)k1 + R2) / (float)kCW));
    int wlo = ja, whi = jb;
    for (; wlo < jb; ++wlo) {
      const float d = (float)chunk_dist(wlo, k0, k1, len);
      if (fmaf(-d * d, c, s_cm[wlo]) >= lb - kCut) break;
    }
    for (; whi > wlo; --whi) {
      const float d = (float)chunk_dist(whi, k0, k1, len);
      if (fmaf(-d * d, c, s_cm[whi]) >= lb - kCut) break;
    }
    p_alpha[pi] = best;
    p_lo[pi] = wlo * kCW;
    p_wl[pi] = min((whi + 1) * kCW, len) - wlo * kCW;
  }
}

#ifndef FOT_BAND_MIN_BLOCKS
#define FOT_BAND_MIN_BLOCKS 2   // resident CTAs per SM the register budget is sized for (at 3
                                // the 80-register budget spills; measured slower)
#endif

template <int MODE, int MAXP>
__global__ void __launch_bounds__(kBW * 32, FOT_BAND_MIN_BLOCKS) band_pass_kernel(const __grid_constant__ BandTable<MAXP> tab) {
  __shared__ __align__(16) float sA[kBW][2 * kSA];
  const int warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * kBW + warp;
  if (gw >= tab.items) return;                            // warp-uniform
  const BandArgs& a = tab.p[find_prob<MAXP, 2>(tab, gw)];
  if (error_latched(a.err)) return;
  const int lw = gw - a.item_base;
  const int tile = lw % a.n_tiles, r0 = (lw / a.n_tiles) * 2 * kBR;
  // each item takes exactly one of the two (warp-uniform choice inside band_item)
  band_item<MODE, 0>(a, r0, tile, tile * kBT, sA[warp]);
  band_item<MODE, 1>(a, r0, tile, tile * kBT, sA[warp]);
}

template <int MAXP>
void band_table_finish(BandTable<MAXP>& t) {
  int rows = 0, plans = 0, items = 0, ctas = 0;
  for (int q = 0; q < t.n; ++q) {
    BandArgs& a = t.p[q];
    a.n_chunks = (a.len + kCW - 1) / kCW;
    a.n_tiles = (a.len + a.tile_w - 1) / a.tile_w;
    a.row_base = rows;
    a.plan_base = plans;
    a.item_base = items;
    a.cta_base = ctas;
    rows += a.n_rows;
    plans += a.n_rows;
    items += ((a.n_rows + 2 * kBR - 1) / (2 * kBR)) * a.n_tiles;
    ctas += ((a.n_rows + 127) / 128) * a.n_tiles;
  }
  t.rows = rows;
  t.plans = plans;
  t.items = items;
  t.ctas = ctas;
}

template <int MAXP>
void band_prepare(cudaStream_t s, const BandTable<MAXP>& t) {
  ktimer_begin(s, kKPlan);
  band_plan_kernel<MAXP><<<t.plans, kPlanThreads, 0, s>>>(t);
  ktimer_end(s);
}

template <int MODE, int MAXP>
void band_simt(cudaStream_t s, const BandTable<MAXP>& t) {
  ktimer_begin(s, kKBand);
  band_pass_kernel<MODE, MAXP><<<(t.items + kBW - 1) / kBW, kBW * 32, 0, s>>>(t);
  ktimer_end(s);
}

template void band_table_finish<1>(BandTable<1>&);
template void band_table_finish<kMaxBatch>(BandTable<kMaxBatch>&);
template void band_prepare<1>(cudaStream_t, const BandTable<1>&);
template void band_prepare<kMaxBatch>(cudaStream_t, const BandTable<kMaxBatch>&);
template void band_simt<kBandLse, 1>(cudaStream_t, const BandTable<1>&);
template void band_simt<kBandPot, 1>(cudaStream_t, const BandTable<1>&);
template void band_simt<kBandLse, kMaxBatch>(cudaStream_t, const BandTable<kMaxBatch>&);
template void band_simt<kBandPot, kMaxBatch>(cudaStream_t, const BandTable<kMaxBatch>&);

// the two passes of one half-step for one context
BandArgs band_args(fot_ctx* c, const float* x, int n_rows, int len, double eps, float x_scale) {
  BandArgs a{};
  a.x = x;
  a.plan = c->plan;
  a.err = c->err;
  a.terms = c->terms;
  a.x_scale = x_scale;
  a.c = (float)(1.4426950408889634 / (2.0 * eps));
  a.eps = (float)eps;
  a.n_rows = n_rows;
  a.len = len;
  a.tile_w = kBT;
  return a;
}

// One half-step with banded passes: pot_out = eps (lmarg - log(Lambda exp(pot_in/eps) Lambda)).
void half_step_band(fot_ctx* c, const float* pot_in, const float* lmarg, double eps,
                    float* pot_out, float* logsum, float* tmp) {
  BandTable<1> t{};
  t.n = 1;
  // pass over the contiguous axis: rows of pot_in, outputs along cols, written [k][L]
  t.p[0] = band_args(c, pot_in, c->rows, c->cols, eps, (float)(1.4426950408889634 / eps));
  t.p[0].y = tmp;
  band_table_finish(t);
  band_prepare(c->stream, t);
  band_simt<kBandLse>(c->stream, t);
  // pass over the row axis (input tmp[k][L], log2 units) with the fused potential update
  t.p[0] = band_args(c, tmp, c->cols, c->rows, eps, 1.f);
  t.p[0].y = pot_out;
  t.p[0].lmarg = lmarg;
  t.p[0].logsum = logsum;
  band_table_finish(t);
  band_prepare(c->stream, t);
  band_simt<kBandPot>(c->stream, t);
  c->launches += 4;
}

}  // namespace fot
