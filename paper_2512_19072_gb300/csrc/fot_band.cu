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
// 1. Offset at every tile centre kc = k0 + 8: alpha_r = max_m e_r(m, kc) (up to rounding),
//    e_r(m, o) = x_r[m] - (o - m)^2 c, and its argmax, from the upper convex hulls of the
//    32-wide chunks (see band_plan_kernel).
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

// Per (row, tile) plan (tiles of tile_w = 16, 32 or 64 outputs): centre offset alpha, window
// start lo and length wl.  One CTA of four warps per row.  The row is staged in shared memory
// as z[m] = x[m] * scale - u^2 c (u = m mod 32, one pad word per 32-wide chunk), with the
// chunk maxima of x * scale.
//   a. alpha: with d0 = kc - 32 j, e(32 j + u, kc) = z[32 j + u] + t u - c d0^2, t = 2 c d0,
//      so the maximum of chunk j at any centre is the support function of the upper convex
//      hull of the points (u, z[32 j + u]) at slope t.  One thread per chunk builds that hull
//      (monotone chain, at most 32 vertices) and the slopes of its edges, which decrease; a
//      query is a binary search for the first edge slope <= -t.  S threads per tile (S * T
//      about the CTA's 128 threads) share its chunks, each skipping every chunk whose bound
//      (chunk maximum less the nearest squared distance times c) cannot beat its best so far,
//      all starting from the chunk that holds kc; a shuffle reduction gives alpha (the maximum
//      at kc up to rounding) and its index.
//   b. the window of step 2 above: the first and the last 32-wide chunk whose bound over the
//      tile reaches LB - kCut.
constexpr int kPlanThreads = 128;

// shared memory of one row: z[n_chunks * 33], cm[n_chunks], hull vertex count[n_chunks],
// edge slopes[n_chunks * 33], vertex positions[n_chunks * 36] (bytes); the odd word strides
// keep threads that work on different chunks on different banks
constexpr int kHullS = kCW + 1;      // slope row stride (floats)
constexpr int kHullU = kCW + 4;      // vertex row stride (bytes)
__host__ __device__ inline size_t plan_smem_bytes(int n_chunks) {
  return (size_t)n_chunks * (kCW + 1 + 1 + 1 + kHullS) * 4 + (size_t)n_chunks * kHullU;
}

template <int MAXP>
__global__ void __launch_bounds__(kPlanThreads) band_plan_kernel(const __grid_constant__ BandTable<MAXP> tab) {
  extern __shared__ __align__(16) float s_plan[];
  const BandArgs& a = tab.p[find_prob<MAXP, 1>(tab, (int)blockIdx.x)];
  if (error_latched(a.err)) return;                       // CTA-uniform
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = (int)blockIdx.x - a.plan_base;
  const int T = a.n_tiles, len = a.len, nch = a.n_chunks, tw = a.tile_w;
  const float c = a.c, sc = a.x_scale;
  const float* xr = a.x + (size_t)row * len;
  float* s_z = s_plan;
  float* s_cm = s_z + nch * (kCW + 1);
  int* s_hn = reinterpret_cast<int*>(s_cm + nch);
  float* s_hs = reinterpret_cast<float*>(s_hn + nch);                          // [j][k] edge k slope
  unsigned char* s_hu = reinterpret_cast<unsigned char*>(s_hs + nch * kHullS);   // [j][k] vertex u

  // stage: each warp takes whole chunks, four at a time (lane = position in the chunk)
  const float uc = -(float)(lane * lane) * c;
  for (int j0 = warp * 4; j0 < nch; j0 += kPlanThreads / 8) {
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
      const float mx = warp_max(v[q]);
      if (lane == 0) s_cm[j0 + q] = mx;
    }
  }
  __syncthreads();
  // upper hulls, one thread per chunk (the padded rows keep the threads on different banks);
  // the top two vertices of the stack live in registers
  for (int j = tid; j < nch; j += kPlanThreads) {
    const float* zs = &s_z[j * (kCW + 1)];
    unsigned char* hu = &s_hu[j * kHullU];
    float* hs = &s_hs[j * kHullS];
    int n = 0;
    int u0 = 0, u1 = 0;                                   // second and top vertex
    float z0 = 0.f, z1 = 0.f;
    for (int u = 0; u < kCW; ++u) {
      const float zu = zs[u];
      if (zu == -INFINITY) continue;
      // pop while the top lies on or below the segment from the one below it to u
      while (n >= 2 && (z1 - z0) * (float)(u - u0) <= (zu - z0) * (float)(u1 - u0)) {
        --n;
        u1 = u0;
        z1 = z0;
        if (n >= 2) {
          u0 = hu[n - 2];
          z0 = zs[u0];
        }
      }
      hu[n++] = (unsigned char)u;
      u0 = u1;
      z0 = z1;
      u1 = u;
      z1 = zu;
    }
    // edge slopes (they only steer the vertex search: the fast division is enough)
    for (int k = 0; k + 1 < n; ++k)
      hs[k] = __fdividef(zs[hu[k + 1]] - zs[hu[k]], (float)(hu[k + 1] - hu[k]));
    s_hn[j] = n;
  }
  __syncthreads();

  const size_t np = (size_t)a.n_rows * T;
  float* p_alpha = a.plan;
  int* p_lo = reinterpret_cast<int*>(a.plan + np);
  int* p_wl = reinterpret_cast<int*>(a.plan + 2 * np);
  // S threads per tile (S a power of two, S * T about the CTA's 128 threads, within a warp):
  // the S threads of a tile take its chunks in turn (every S-th), each skipping the chunks whose
  // bound (chunk maximum less the nearest squared distance times c) cannot beat its best so
  // far, all starting from the chunk that holds the centre; a shuffle reduction then gives the
  // tile's maximum (leftmost index on ties) and its window
  int S = 1;
  while (S < 32 && 2 * S * T <= kPlanThreads) S *= 2;
  const int per_pass = kPlanThreads / S;
  const int slot = tid / S, sub = tid % S;
  for (int base = 0; base < T; base += per_pass) {       // uniform across the CTA
    const int t = base + slot;
    const bool live = t < T;
    const int k0 = t * tw, kc = k0 + tw / 2, k1 = min(k0 + tw, len) - 1;
    float best = -INFINITY;
    int arg = 0x7fffffff;
    auto query = [&](int j) {
      const int n = s_hn[j];
      if (n == 0) return;
      const int clo = j * kCW;
      const float d0 = (float)(kc - clo);
      const float t2 = 2.f * c * d0;
      const float* hs = &s_hs[j * kHullS];
      int lo = 0, hi = n - 1;                             // first edge with slope <= -t2
      while (lo < hi) {
        const int md = (lo + hi) >> 1;
        if (hs[md] <= -t2)
          hi = md;
        else
          lo = md + 1;
      }
      const int u = s_hu[j * kHullU + lo];
      const float v = fmaf(-d0 * d0, c, fmaf((float)u, t2, s_z[j * (kCW + 1) + u]));
      if (v > best || (v == best && clo + u < arg)) {
        best = v;
        arg = clo + u;
      }
    };
    if (live) {
      const int jc = min(kc, len - 1) / kCW;
      query(jc);
      for (int j = sub; j < nch; j += S) {
        if (j == jc) continue;
        const int clo = j * kCW, chi = min(clo + kCW, len) - 1;
        const int dd = clo > kc ? clo - kc : (chi < kc ? kc - chi : 0);
        if (fmaf(-(float)dd * (float)dd, c, s_cm[j]) > best) query(j);
      }
    }
    for (int off = S / 2; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oa = __shfl_xor_sync(0xffffffffu, arg, off);
      if (ob > best || (ob == best && oa < arg)) {
        best = ob;
        arg = oa;
      }
    }
    // b. window: lower bound over the tile from the argmax term at the worse tile end, then
    // the first and the last chunk whose bound over the tile reaches lb - kCut
    int wlo = 0x7fffffff, whi = -1;
    if (live && best != -INFINITY) {
      const float dM = (float)(arg - kc);
      const float ka = (float)(k0 - kc), kb = (float)(k1 - kc);
      const float lb = best + fminf(fmaf(2.f * ka, dM * c, -ka * ka * c), fmaf(2.f * kb, dM * c, -kb * kb * c));
      for (int j = sub; j < nch; j += S) {
        const int clo = j * kCW, chi = min(clo + kCW, len) - 1;
        const int d = clo > k1 ? clo - k1 : (chi < k0 ? k0 - chi : 0);
        if (fmaf(-(float)d * (float)d, c, s_cm[j]) >= lb - kCut) {
          wlo = min(wlo, j);
          whi = j;
        }
      }
    }
    for (int off = S / 2; off > 0; off >>= 1) {
      wlo = min(wlo, __shfl_xor_sync(0xffffffffu, wlo, off));
      whi = max(whi, __shfl_xor_sync(0xffffffffu, whi, off));
    }
    if (live && sub == 0) {
      const size_t pi = (size_t)row * T + t;
      if (best == -INFINITY) {                            // no finite term: empty row
        p_alpha[pi] = -INFINITY;
        p_lo[pi] = 0;
        p_wl[pi] = 0;
      } else {
        p_alpha[pi] = best;
        p_lo[pi] = wlo * kCW;
        p_wl[pi] = min((whi + 1) * kCW, len) - wlo * kCW;
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
  size_t smem = 0;
  for (int q = 0; q < t.n; ++q) smem = std::max(smem, plan_smem_bytes(t.p[q].n_chunks));
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
