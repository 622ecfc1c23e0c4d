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
// lo and window length wl.  A CTA takes R whole rows; each row is staged once in shared memory
// as z[m] = x[m] * scale in 32-wide chunks (one pad word per chunk), with each chunk's maximum
// cm[j] and the position p[j] where it is reached.  Then four lanes (q = 0..3) work on each
// tile, eight tiles per warp, splitting the chunks (j = q mod 4) and the positions of a
// scanned chunk (8 each) between them:
//   a. alpha: the largest term e(m, kc) = z[m] - (kc - m)^2 c at the tile centre kc over the
//      positions of the chunks scanned: first the chunk whose own maximum gives the best
//      term at kc (e(p[j], kc)), then every chunk whose bound cm[j] - d_j^2 c (d_j its
//      nearest distance to kc) exceeds the best term found so far by more than kPlanSlack,
//      lowest first.  Every unscanned chunk is then within kPlanSlack of alpha, so
//          alpha_exact - kPlanSlack <= alpha <= alpha_exact.
//      An offset below the exact maximum only raises the operands 2^(e - alpha) (by at most
//      2^kPlanSlack): the range arguments of the GEMM paths only need alpha <= alpha_exact.
//   b. the window of step 2 above, with the lower bound LB = min over the tile ends o of
//      e(mh, o) for the position mh that gave alpha (valid for every output of the tile, as
//      e(mh, o) is concave in o): the first and the last chunk whose bound over the tile
//      reaches LB - kCut.
// With unit extents requested (tensor-core passes) the CTA also reduces, per tile, the union
// of its rows' windows into the unit's [ext_lo, ext_hi) (all R rows lie in one 128-row block).
constexpr int kPlanWarps = 8;                 // rows per CTA at most (plan rows are padded to a multiple)
constexpr int kPlanMaxChunks = 4096 / kCW;    // 32-wide chunks of the longest row
constexpr int kPlanQ = 4;                     // lanes per tile
constexpr int kPlanTPW = 32 / kPlanQ;         // tiles per warp
constexpr float kPlanSlack = 14.f;            // log2 units (a looser offset scans fewer chunks; the
                                              // window test stays provable for any slack)

// shared memory of one row (floats): z[n_chunks * 33], cm[n_chunks], p[n_chunks] (as float)
__host__ __device__ inline int plan_row_floats(int n_chunks) { return n_chunks * (kCW + 3); }

// max with the smaller key on ties, over the kPlanQ lanes of a tile
__device__ __forceinline__ void quad_argmax(float& v, int& k) {
#pragma unroll
  for (int d = 1; d < kPlanQ; d <<= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, d);
    const int ok = __shfl_xor_sync(0xffffffffu, k, d);
    if (ov > v || (ov == v && ok < k)) {
      v = ov;
      k = ok;
    }
  }
}

template <int MAXP>
__global__ void __launch_bounds__(1024) band_plan_kernel(const __grid_constant__ BandTable<MAXP> tab) {
  extern __shared__ __align__(16) float s_plan[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wpr = tab.plan_wpr;                           // warps per row
  const int R = (blockDim.x >> 5) / wpr;                  // rows of this CTA
  const int rr = warp / wpr, wr = warp % wpr;             // this warp's row and tile group
  // every row of a CTA belongs to one problem and one 128-row block: each problem's plan rows
  // start at a multiple of 8 and R divides 8
  const int grow0 = (int)blockIdx.x * R;
  const BandArgs& a = tab.p[find_prob<MAXP, 1>(tab, grow0)];
  const int row = grow0 + rr - a.plan_base;               // may be a padding row (>= n_rows)
  const int T = a.n_tiles, len = a.len, nch = a.n_chunks, tw = a.tile_w;
  const bool live = row < a.n_rows && !error_latched(a.err);
  const bool ext = a.ext_lo != nullptr;
  float* z = s_plan + (size_t)rr * tab.plan_row_stride;
  float* cm = z + nch * (kCW + 1);
  float* cp = cm + nch;
  int* s_ulo = reinterpret_cast<int*>(s_plan + (size_t)R * tab.plan_row_stride);
  int* s_uhi = s_ulo + tab.plan_tiles;
  if (a.ext_lo_next) {
    // reset the next pass's unit extents (the problem's plan rows take strided shares; the
    // next pass's plan kernel reduces into them): the whole array, since the next pass may
    // contract the other axis with another tile width
    if (wr == 0)
      for (int i = row * 32 + lane; i < a.ext_units; i += a.plan_rows * 32) {
        a.ext_lo_next[i] = 0x7F7F7F7F;
        a.ext_hi_next[i] = 0;
      }
  }
  if (ext)
    for (int t = tid; t < T; t += blockDim.x) {
      s_ulo[t] = 0x7F7F7F7F;
      s_uhi[t] = 0;
    }
  const float c = a.c, sc = a.x_scale;
  // stage the rows (each warp of a row loads every wpr-th chunk, coalesced, eight in flight)
  if (live) {
    const float* xr = a.x + (size_t)row * len;
    for (int j0 = wr; j0 < nch; j0 += 8 * wpr) {
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = j0 + q * wpr, m = j * kCW + lane;
        v[q] = (j < nch && m < len) ? __fmul_rn(__ldg(xr + m), sc) : -INFINITY;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = j0 + q * wpr;
        if (j < nch) z[j * (kCW + 1) + lane] = v[q];
      }
    }
  }
  __syncthreads();
  // chunk maxima and their leftmost positions (thread per chunk; the pad word puts the lanes
  // of a warp on different banks)
  if (live) {
    for (int j = wr * 32 + lane; j < nch; j += wpr * 32) {
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
  }
  __syncthreads();

  if (live) {
    const size_t np = (size_t)a.plan_stride * T;
    float* p_alpha = a.plan;
    int* p_lo = reinterpret_cast<int*>(a.plan + np);
    int* p_wl = reinterpret_cast<int*>(a.plan + 2 * np);
    const int q = lane & (kPlanQ - 1);
    // warp-uniform loop over this warp's groups of eight tiles (the combines and the candidate
    // rounds below are warp-wide); lanes of a missing tile compute nothing and write nothing
    for (int tg = wr * kPlanTPW; tg < T; tg += wpr * kPlanTPW) {
      const int t = tg + lane / kPlanQ;
      const bool has = t < T;
      const int k0 = min(t, T - 1) * tw, kc = k0 + tw / 2, k1 = min(k0 + tw, len) - 1;
      const float fkc = (float)kc;
      auto bound = [&](int j) {                           // chunk j's bound at kc
        const int clo = j * kCW, chi = min(clo + kCW, len) - 1;
        const int dd = clo > kc ? clo - kc : (chi < kc ? kc - chi : 0);
        return fmaf(-(float)dd * (float)dd, c, cm[j]);
      };
      // a. the chunk whose maximum gives the best term at kc
      float vb = -INFINITY;
      int jb = 0x7fffffff;
      for (int j = q; j < nch && has; j += kPlanQ) {
        const float d = fkc - cp[j];
        const float v = fmaf(-d * d, c, cm[j]);
        if (v > vb) {
          vb = v;
          jb = j;
        }
      }
      quad_argmax(vb, jb);
      float alpha = -INFINITY;
      int mh = 0x7fffffff;
      // exact maximum over chunk j, the four lanes taking eight positions each; every lane of
      // the warp runs it (the combine is warp-wide), a lane whose tile has nothing to scan
      // passes valid = false and keeps its maximum
      auto scan = [&](int j, bool valid) {
        const float* zj = z + j * (kCW + 1) + q * (kCW / kPlanQ);
        float d = fkc - (float)(j * kCW + q * (kCW / kPlanQ));
        float v0 = -INFINITY;
        int m0 = 0x7fffffff;
#pragma unroll
        for (int u = 0; u < kCW / kPlanQ; ++u, d -= 1.f) {
          const float v = fmaf(-d * d, c, zj[u]);
          if (v > v0) {
            v0 = v;
            m0 = j * kCW + q * (kCW / kPlanQ) + u;
          }
        }
        quad_argmax(v0, m0);
        if (valid && (v0 > alpha || (v0 == alpha && m0 < mh))) {
          alpha = v0;
          mh = m0;
        }
      };
      const bool any = has && vb != -INFINITY;
      if (__any_sync(0xffffffffu, any)) {
        scan(any ? jb : 0, any);
        // the candidate chunks (this lane's share), then rounds in which every tile scans its
        // lowest remaining candidate together; each is tested again against the maximum so far
        uint32_t cand[kPlanMaxChunks / 32 / kPlanQ + 1];
#pragma unroll
        for (int w = 0; w < kPlanMaxChunks / 32 / kPlanQ + 1; ++w) cand[w] = 0u;
        if (any)
          for (int j = q, b = 0; j < nch; j += kPlanQ, ++b)
            if (j != jb && bound(j) > alpha + kPlanSlack) cand[b >> 5] |= 1u << (b & 31);
        for (;;) {
          int mine = 0x7fffffff;                          // this lane's lowest candidate chunk
#pragma unroll
          for (int w = 0; w < kPlanMaxChunks / 32 / kPlanQ + 1; ++w)
            if (mine == 0x7fffffff && cand[w] != 0u) mine = (w * 32 + __ffs(cand[w]) - 1) * kPlanQ + q;
          float dummy = 0.f;
          int next = mine;
          quad_argmax(dummy, next);                       // the tile's lowest candidate
          if (!__any_sync(0xffffffffu, next != 0x7fffffff)) break;
          if (next != 0x7fffffff && next == mine) {
            const int b = (mine - q) / kPlanQ;
            cand[b >> 5] &= ~(1u << (b & 31));
          }
          const bool doscan = next != 0x7fffffff && bound(next) > alpha + kPlanSlack;
          scan(doscan ? next : 0, doscan);
        }
      }
      // b. window
      int wlo = 0x7fffffff, whi = -1;
      if (has && alpha != -INFINITY) {
        const float zm = z[(mh / kCW) * (kCW + 1) + mh % kCW];
        const float da = (float)(k0 - mh), db = (float)(k1 - mh);
        const float lb = fminf(fmaf(-da * da, c, zm), fmaf(-db * db, c, zm));
        for (int j = q; j < nch; j += kPlanQ) {
          const int clo = j * kCW, chi = min(clo + kCW, len) - 1;
          const int d = clo > k1 ? clo - k1 : (chi < k0 ? k0 - chi : 0);
          if (fmaf(-(float)d * (float)d, c, cm[j]) >= lb - kCut) {
            wlo = min(wlo, j);
            whi = max(whi, j);
          }
        }
      }
#pragma unroll
      for (int d = 1; d < kPlanQ; d <<= 1) {
        wlo = min(wlo, __shfl_xor_sync(0xffffffffu, wlo, d));
        whi = max(whi, __shfl_xor_sync(0xffffffffu, whi, d));
      }
      if (!has || q != 0) continue;
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
    const int rb = (grow0 - a.plan_base) / 128;
    for (int t = tid; t < T; t += blockDim.x) {
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
  // warps per row: enough tile groups of eight for the widest row of tiles (at most 32); rows
  // per CTA: a power of two up to 8 (a CTA never straddles two problems or two 128-row
  // blocks) within 8 warps per CTA (or the row's own warps) and the default 48 KB of shared
  // memory together with the per-tile unit extents
  int wpr = std::max(1, std::min(32, (t.plan_tiles + kPlanTPW - 1) / kPlanTPW));
  t.plan_wpr = wpr;
  const size_t tile_bytes = 2 * sizeof(int) * (size_t)t.plan_tiles;
  int R = 8;
  while (R > 1 && (R * wpr > std::max(8, wpr) || R * t.plan_row_stride * sizeof(float) + tile_bytes > 48 * 1024)) R /= 2;
  const size_t smem = (size_t)R * t.plan_row_stride * sizeof(float) + tile_bytes;
  ktimer_begin(s, kKPlan);
  band_plan_kernel<MAXP><<<t.plans / R, R * wpr * 32, smem, s>>>(t);
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
