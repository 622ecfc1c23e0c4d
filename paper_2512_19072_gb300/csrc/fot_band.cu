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
// 1. Offset at every tile centre kc = k0 + 8: a term alpha_r = e_r(m_r, kc) within 16 (log2
//    units) of max_m e_r(m, kc), e_r(m, o) = x_r[m] - (o - m)^2 c, found by scanning only the
//    32-wide chunks of m whose upper bound (chunk maximum of x, nearest distance) exceeds the
//    best term found so far by more than that.
// 2. A provable window: every o in the tile has max_m e_r(m, o) >= LB_r, with LB_r the
//    value of the centre's argmax term at the worse tile end.  A 32-wide chunk of m whose
//    upper bound (chunk maximum of x, nearest distance) over the whole tile is below
//    LB_r - 40 holds only terms below 2^-40 of every output of the tile; the window is the
//    hull of the remaining chunks (relative truncation error < len * 2^-40).
// 3. Tilt identity (large eps).  With o = kc + kap:
//      e_r(m, o) = [x_r[m] - (kc - m)^2 c - alpha_r] + [2 kap (m - Mref_r) c - kap^2 c]
//                  + alpha_r + 2 kap (Mref_r - kc) c,
//    so  sum_m 2^e = 2^(alpha_r + 2 kap (Mref_r - kc) c) * sum_m' A[r][m'] B[m'][kap]
//    with A[r][m'] = 2^(e_r(lo_r + m', kc) - alpha_r) <= 2^16 (one exponential per row and
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

// Per (row, tile) plan (tiles of tile_w = 16, 32 or 64 outputs): centre offset alpha, window
// start lo and length wl.  One CTA of four warps per row.  The row is staged in shared memory
// as z[m] = x[m] * scale - u^2 c (u = m mod 32, one pad word per 32-wide chunk), with the
// maxima of x * scale over 32-wide chunks and over 8-wide sub-chunks.  Each warp then plans
// tiles one at a time:
//   a. alpha: with d0 = kc - 32 j, e(32 j + u, kc) = z[32 j + u] + 2 c d0 u - c d0^2.  Lane l
//      takes element l of the chunk holding the centre kc, and every sub-chunk it owns whose
//      upper bound (sub-chunk maximum less the nearest squared distance times c) exceeds that
//      chunk's best term by more than kAlphaSlack; one warp argmax over the lanes' best terms
//      gives alpha and its index.  Every sub-chunk left out is bounded by alpha + kAlphaSlack,
//      so alpha is a term within kAlphaSlack of the maximum: it only scales the window sums'
//      operands (A <= 2^kAlphaSlack instead of <= 1, far from overflow, and the largest term
//      of every output keeps A >= 2^-2 kTiltMax), and the window bound below needs a term.
//   b. the window of step 2 above: the first and the last 32-wide chunk whose bound over the
//      tile reaches LB - kCut (one ballot per 32 chunks).
constexpr int kPlanThreads = 128;
constexpr int kSub = 8;                       // sub-chunk width
constexpr float kAlphaSlack = 16.f;           // alpha may sit this far (log2) below the maximum

template <int MAXP>
__global__ void __launch_bounds__(kPlanThreads) band_plan_kernel(const __grid_constant__ BandTable<MAXP> tab) {
  extern __shared__ float s_plan[];   // [n_chunks * 33] z, [n_chunks] chunk maxima, [4 n_chunks] sub
  const BandArgs& a = tab.p[find_prob<MAXP, 1>(tab, (int)blockIdx.x)];
  if (error_latched(a.err)) return;                       // CTA-uniform
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int row = (int)blockIdx.x - a.plan_base;
  const int T = a.n_tiles, len = a.len, nch = a.n_chunks;
  const int nsub = nch * (kCW / kSub);
  const int nwords = (nch + 31) / 32, nswords = (nsub + 31) / 32;
  const float c = a.c, sc = a.x_scale;
  const float* xr = a.x + (size_t)row * len;
  float* s_z = s_plan;
  float* s_cm = s_plan + nch * (kCW + 1);
  float* s_c8 = s_cm + nch;
  // stage: each warp takes whole chunks, four at a time (lane = position in the chunk; the
  // four loads are issued together); max(x) * sc equals max(x * sc) since sc > 0 and rounding
  // is monotone
  const float uc = -(float)(lane * lane) * c;
  for (int j0 = warp * 4; j0 < nch; j0 += nw * 4) {
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = (j0 + q) * kCW + lane;
      v[q] = (j0 + q < nch && m < len) ? __fmul_rn(xr[m], sc) : -INFINITY;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (j0 + q >= nch) break;                           // warp-uniform
      s_z[(j0 + q) * (kCW + 1) + lane] = __fadd_rn(v[q], uc);   // no contraction: the same
                                                                  // rounding in every instance
      float mx = v[q];
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
      if ((lane & (kSub - 1)) == 0) s_c8[(j0 + q) * (kCW / kSub) + lane / kSub] = mx;
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
      if (lane == 0) s_cm[j0 + q] = mx;
    }
  }
  __syncthreads();
  const size_t np = (size_t)a.n_rows * T;
  float* p_alpha = a.plan;
  int* p_lo = reinterpret_cast<int*>(a.plan + np);
  int* p_wl = reinterpret_cast<int*>(a.plan + 2 * np);
  const int tw = a.tile_w;

  for (int t = warp; t < T; t += nw) {
    const int k0 = t * tw, kc = k0 + tw / 2, k1 = min(k0 + tw, len) - 1;
    // a. element `lane` of the centre's chunk, then this lane's qualifying sub-chunks
    const int jc = min(kc, len - 1) / kCW;
    const float dc = (float)(kc - jc * kCW);
    float best = fmaf((float)lane, 2.f * c * dc, s_z[jc * (kCW + 1) + lane]);
    best = fmaf(-dc * dc, c, best);
    int arg = jc * kCW + lane;
    const float floor_ = warp_max(best) + kAlphaSlack;  // sub-chunks at or below: left out
#pragma unroll 1
    for (int w = 0; w < nswords; ++w) {
      const int sj = 32 * w + lane;
      const int m0 = sj * kSub, m1 = min(m0 + kSub, len) - 1;
      const int d = m0 > kc ? m0 - kc : (m1 < kc ? kc - m1 : 0);
      const float c8 = sj < nsub ? s_c8[sj] : -INFINITY;
      if (sj / (kCW / kSub) != jc && fmaf(-(float)d * (float)d, c, c8) > floor_) {
        const int j = sj / (kCW / kSub), u0 = m0 - j * kCW;
        const float d0 = (float)(kc - j * kCW);
        const float t2 = 2.f * c * d0;
        const float* zs = &s_z[j * (kCW + 1) + u0];
#pragma unroll
        for (int v = 0; v < kSub; ++v) {
          const float e = fmaf(-d0 * d0, c, fmaf((float)(u0 + v), t2, zs[v]));
          if (e > best) {
            best = e;
            arg = m0 + v;
          }
        }
      }
    }
    warp_argmax(best, arg);
    const size_t pi = (size_t)row * T + t;
    if (best == -INFINITY) {                              // no finite term: empty row
      if (lane == 0) {
        p_alpha[pi] = -INFINITY;
        p_lo[pi] = 0;
        p_wl[pi] = 0;
      }
      continue;
    }
    const float al = best;
    // b. window: lower bound over the tile from the argmax term at the worse tile end, then
    // the first and the last chunk whose bound over the tile reaches lb - kCut
    const float dM = (float)(arg - kc);
    const float ka = (float)(k0 - kc), kb = (float)(k1 - kc);
    const float lb = al + fminf(fmaf(2.f * ka, dM * c, -ka * ka * c), fmaf(2.f * kb, dM * c, -kb * kb * c));
    int wlo = -1, whi = -1;
#pragma unroll 1
    for (int w = 0; w < nwords; ++w) {
      const int j = 32 * w + lane;
      const int clo = j * kCW, chi = min(clo + kCW, len) - 1;
      const int d = clo > k1 ? clo - k1 : (chi < k0 ? k0 - chi : 0);
      const float cmj = j < nch ? s_cm[j] : -INFINITY;
      const bool in = fmaf(-(float)d * (float)d, c, cmj) >= lb - kCut;
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      if (bal) {
        if (wlo < 0) wlo = 32 * w + __ffs(bal) - 1;
        whi = 32 * w + 31 - __clz(bal);
      }
    }
    if (lane == 0) {
      p_alpha[pi] = al;
      p_lo[pi] = wlo * kCW;
      p_wl[pi] = min((whi + 1) * kCW, len) - wlo * kCW;
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
  int max_chunks = 1;
  for (int q = 0; q < t.n; ++q) max_chunks = std::max(max_chunks, t.p[q].n_chunks);
  const size_t smem = (size_t)max_chunks * (kCW + 2 + kCW / kSub) * sizeof(float);
  ktimer_begin(s, kKPlan);
  band_plan_kernel<MAXP><<<t.plans, kPlanThreads, smem, s>>>(t);
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
