// Banded axis passes: the same contraction as the exact pass,
//     y[o][r] = log2 sum_m 2^( x[r][m]*scale - (o - m)^2 c ),   c = log2(e) / (2 eps),
// but each output only visits the terms that can matter, and for large eps the inner loop
// is a plain FP32 multiply-add GEMM instead of one exponential per term.
//
// Work unit: one warp, 16 input rows r x one tile of 16 consecutive outputs o = k0 + i; lane
// (h, i) = (lane / 16, lane % 16) owns rows 8h .. 8h+7 and output i.  Steps 1-2 run in
// band_plan_kernel (one warp per row) and leave (alpha, lo, window length) per (row, tile);
// steps 3-4 run in band_pass_kernel.
//
// 1. Offset at every tile centre kc = k0 + 8: alpha_r, the largest term
//    e_r(m, kc) = x_r[m] - (kc - m)^2 c over the positions that can hold the maximum, and the
//    position where it is reached; within kPlanSlack below the exact maximum (see
//    band_plan_kernel).
// 2. A provable window: every o in the tile has max_m e_r(m, o) >= LB_r, with LB_r the
//    value of that position's term at the worse tile end.  A 32-wide chunk of m whose
//    upper bound (chunk maximum of x, nearest distance) over the whole tile is below
//    LB_r - 40 holds only terms below 2^-40 of every output of the tile; the window is the
//    hull of the remaining chunks (relative truncation error < len * 2^-40).
// 3. Tilt identity (large eps).  With o = kc + kap:
//      e_r(m, o) = [x_r[m] - (kc - m)^2 c - alpha_r] + [2 kap (m - Mref_r) c - kap^2 c]
//                  + alpha_r + 2 kap (Mref_r - kc) c,
//    so  sum_m 2^e = 2^(alpha_r + 2 kap (Mref_r - kc) c) * sum_m' A[r][m'] B[m'][kap]
//    with A[r][m'] = 2^(e_r(lo_r + m', kc) - alpha_r) <= 2^kPlanSlack (one exponential per row and
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

// Per (row, tile) plan (tiles of tile_w = 16, 32 or 64 outputs): offset alpha, window start
// lo and window length wl.  One warp per row; the row is staged in shared memory as
// z[m] = x[m] * scale in 32-wide chunks (one pad word per chunk), with each chunk's maximum
// cm[j] and the position p[j] where it is reached.  Lane t then takes tiles t, t + 32, ...:
//   a. alpha: the largest term e(m, kc) = z[m] - (kc - m)^2 c at the tile centre kc over the
//      positions of the chunks scanned: first the chunk whose own maximum gives the best
//      term at kc (e(p[j], kc)), then every chunk whose bound cm[j] - d_j^2 c (d_j its
//      nearest distance to kc) exceeds the best term found so far by more than kPlanSlack.
//      Every unscanned chunk is then within kPlanSlack of alpha, so
//          alpha_exact - kPlanSlack <= alpha <= alpha_exact.
//      An offset below the exact maximum only raises the operands 2^(e - alpha) (by at most
//      2^kPlanSlack): the range arguments of the GEMM paths only need alpha <= alpha_exact.
//   b. the window of step 2 above, with the lower bound LB = min over the tile ends o of
//      e(mh, o) for the position mh that gave alpha (valid for every output of the tile, as
//      e(mh, o) is concave in o): the first and the last chunk whose bound over the tile
//      reaches LB - kCut.
constexpr int kPlanWarps = 8;        // rows per CTA (fewer for long rows: see band_prepare)
constexpr float kPlanSlack = 8.f;    // log2 units

// shared memory of one row (floats): z[n_chunks * 33], cm[n_chunks], p[n_chunks] (as float)
__host__ __device__ inline int plan_row_floats(int n_chunks) { return n_chunks * (kCW + 3); }

template <int MAXP>
__global__ void __launch_bounds__(kPlanWarps * 32) band_plan_kernel(const __grid_constant__ BandTable<MAXP> tab) {
  extern __shared__ __align__(16) float s_plan[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  // every warp of a CTA belongs to one problem and one 128-row block: each problem's plan rows
  // start at a multiple of 8 and nwarps divides 8
  const int grow = blockIdx.x * nwarps + warp;
  const BandArgs& a = tab.p[find_prob<MAXP, 1>(tab, (int)blockIdx.x * nwarps)];
  const int row = grow - a.plan_base;                       // may be a padding row (>= n_rows)
  const int T = a.n_tiles, len = a.len, nch = a.n_chunks, tw = a.tile_w;
  const bool live = row < a.n_rows && !error_latched(a.err);
  const bool ext = a.ext_lo != nullptr;
  int* s_ulo = reinterpret_cast<int*>(s_plan + (size_t)nwarps * tab.plan_row_stride);
  int* s_uhi = s_ulo + tab.plan_tiles;
  if (a.ext_lo_next) {
    // reset the next pass's unit extents (the problem's plan rows take strided shares; the
    // next pass's plan kernel reduces into them): the whole array, since the next pass may
    // contract the other axis with another tile width
    for (int i = row * 32 + lane; i < a.ext_units; i += a.plan_rows * 32) {
      a.ext_lo_next[i] = 0x7F7F7F7F;
      a.ext_hi_next[i] = 0;
    }
  }
  if (ext) {
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
      s_ulo[t] = 0x7F7F7F7F;
      s_uhi[t] = 0;
    }
    __syncthreads();                                       // CTA-uniform (ext is per problem)
  }
  if (live) {
    const float c = a.c, sc = a.x_scale;
    const float* xr = a.x + (size_t)row * len;
    float* z = s_plan + (size_t)warp * tab.plan_row_stride;
    float* cm = z + nch * (kCW + 1);
    float* cp = cm + nch;

    // stage the row (coalesced: one 128-byte chunk per warp load)
#pragma unroll 4
    for (int j = 0; j < nch; ++j) {
      const int m = j * kCW + lane;
      z[j * (kCW + 1) + lane] = m < len ? __fmul_rn(xr[m], sc) : -INFINITY;
    }
    __syncwarp();
    // chunk maxima and their leftmost positions: lane j takes chunks j, j + 32, ... (the pad
    // word puts the 32 lanes on 32 different banks)
    for (int j = lane; j < nch; j += 32) {
      const float* zj = z + j * (kCW + 1);
      float best = -INFINITY;
      int arg = 0;
#pragma unroll 8
      for (int u = 0; u < kCW; ++u) {
        const float v = zj[u];
        if (v > best) {
          best = v;
          arg = u;
        }
      }
      cm[j] = best;
      cp[j] = (float)(j * kCW + arg);
    }
    __syncwarp();

    const size_t np = (size_t)a.plan_stride * T;
    float* p_alpha = a.plan;
    int* p_lo = reinterpret_cast<int*>(a.plan + np);
    int* p_wl = reinterpret_cast<int*>(a.plan + 2 * np);
    for (int t = lane; t < T; t += 32) {
      const int k0 = t * tw, kc = k0 + tw / 2, k1 = min(k0 + tw, len) - 1;
      const float fkc = (float)kc;
      // a. the chunk whose maximum gives the best term at kc
      float vb = -INFINITY;
      int jb = -1;
      for (int j = 0; j < nch; ++j) {
        const float d = fkc - cp[j];
        const float v = fmaf(-d * d, c, cm[j]);
        if (v > vb) {
          vb = v;
          jb = j;
        }
      }
      float alpha = -INFINITY;
      int mh = 0;
      auto scan = [&](int j) {                            // exact maximum over chunk j
        const float* zj = z + j * (kCW + 1);
        float d = fkc - (float)(j * kCW);
#pragma unroll 8
        for (int u = 0; u < kCW; ++u, d -= 1.f) {
          const float v = fmaf(-d * d, c, zj[u]);
          if (v > alpha) {
            alpha = v;
            mh = j * kCW + u;
          }
        }
      };
      if (jb >= 0) {
        scan(jb);
        for (int j = 0; j < nch; ++j) {
          if (j == jb) continue;
          const int clo = j * kCW, chi = min(clo + kCW, len) - 1;
          const int dd = clo > kc ? clo - kc : (chi < kc ? kc - chi : 0);
          if (fmaf(-(float)dd * (float)dd, c, cm[j]) > alpha + kPlanSlack) scan(j);
        }
      }
      // b. window
      int wlo = -1, whi = -1;
      if (alpha != -INFINITY) {
        const float zm = z[(mh / kCW) * (kCW + 1) + mh % kCW];
        const float da = (float)(k0 - mh), db = (float)(k1 - mh);
        const float lb = fminf(fmaf(-da * da, c, zm), fmaf(-db * db, c, zm));
        for (int j = 0; j < nch; ++j) {
          const int clo = j * kCW, chi = min(clo + kCW, len) - 1;
          const int d = clo > k1 ? clo - k1 : (chi < k0 ? k0 - chi : 0);
          if (fmaf(-(float)d * (float)d, c, cm[j]) >= lb - kCut) {
            if (wlo < 0) wlo = j;
            whi = j;
          }
        }
      }
      const size_t pi = (size_t)t * a.plan_stride + row;
      if (alpha == -INFINITY) {                           // no finite term: empty row
        p_alpha[pi] = -INFINITY;
        p_lo[pi] = 0;
        p_wl[pi] = 0;
      } else {
        const int lo = wlo * kCW, hi = min((whi + 1) * kCW, len);
        p_alpha[pi] = alpha;
        p_lo[pi] = lo;
        p_wl[pi] = hi - lo;
        if (ext) {
          atomicMin(&s_ulo[t], lo);
          atomicMax(&s_uhi[t], hi);
        }
      }
    }
  }
  if (ext) {
    // the CTA's rows share one row block: one global atomic pair per tile
    __syncthreads();
    const int rb = ((int)blockIdx.x * nwarps - a.plan_base) / 128;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
      if (s_uhi[t] > 0) {
        atomicMin(&a.ext_lo[rb * T + t], s_ulo[t]);
        atomicMax(&a.ext_hi[rb * T + t], s_uhi[t]);
      }
    }
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
  int rows = 0, plans = 0, items = 0, ctas = 0, tiles = 1;
  for (int q = 0; q < t.n; ++q) {
    BandArgs& a = t.p[q];
    a.n_chunks = (a.len + kCW - 1) / kCW;
    a.n_tiles = (a.len + a.tile_w - 1) / a.tile_w;
    a.plan_stride = (a.n_rows + 127) / 128 * 128;
    a.plan_rows = (a.n_rows + kPlanWarps - 1) / kPlanWarps * kPlanWarps;
    a.row_base = rows;
    a.plan_base = plans;
    a.item_base = items;
    a.cta_base = ctas;
    rows += a.n_rows;
    plans += a.plan_rows;
    items += ((a.n_rows + 2 * kBR - 1) / (2 * kBR)) * a.n_tiles;
    ctas += ((a.n_rows + 127) / 128) * a.n_tiles;
    tiles = std::max(tiles, a.n_tiles);
  }
  t.rows = rows;
  t.plans = plans;
  t.items = items;
  t.ctas = ctas;
  t.plan_tiles = tiles;
}

template <int MAXP>
void band_prepare(cudaStream_t s, BandTable<MAXP>& t) {
  int nch = 1;
  for (int q = 0; q < t.n; ++q) nch = std::max(nch, t.p[q].n_chunks);
  t.plan_row_stride = plan_row_floats(nch);
  // rows per CTA: a power of two up to kPlanWarps (so that a CTA never straddles two problems
  // or two 128-row blocks), as many as fit the default 48 KB of shared memory together with the
  // per-tile unit extents
  const size_t tile_bytes = 2 * sizeof(int) * (size_t)t.plan_tiles;
  int wpb = kPlanWarps;
  while (wpb > 1 && wpb * t.plan_row_stride * sizeof(float) + tile_bytes > 48 * 1024) wpb /= 2;
  const size_t smem = (size_t)wpb * t.plan_row_stride * sizeof(float) + tile_bytes;
  ktimer_begin(s, kKPlan);
  band_plan_kernel<MAXP><<<t.plans / wpb, wpb * 32, smem, s>>>(t);
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
template void band_prepare<1>(cudaStream_t, BandTable<1>&);
template void band_prepare<kMaxBatch>(cudaStream_t, BandTable<kMaxBatch>&);
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
