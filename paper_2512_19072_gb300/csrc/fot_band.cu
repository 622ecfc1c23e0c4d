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
// 1. Exact offset at every tile centre kc = k0 + 8:  alpha_r = max_m e_r(m, kc),
//    e_r(m, o) = x_r[m] - (o - m)^2 c, and its argmax.  e_r(m, o) - e_r(m', o) =
//    x_m - x_m' - (m^2 - m'^2) c + 2 o (m - m') c grows with o when m > m', so the leftmost
//    argmax is non-decreasing in o for any input: a divide-and-conquer monotone search finds
//    the maxima of a group of 16 centres with O(len log 16) evaluations.
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
#include "fot_band.cuh"

#include <algorithm>

namespace fot {

constexpr int kBT = 16;          // outputs per tile
constexpr int kBR = 8;           // rows per lane (16 per warp)
constexpr int kBW = 8;           // warps per CTA
constexpr int kCW = 32;          // chunk width of the chunk maxima
constexpr float kCut = 40.f;     // window cut-off, log2 units
constexpr float kTiltMax = 40.f; // largest |log2 B| allowed on the GEMM path.  The largest
                                 // term of an output has A >= 2^(-2 kTiltMax), and an A that
                                 // flushes below 2^-126 is < 2^(2 kTiltMax - 126) = 2^-46 of it.

enum BandMode : int { kBandLse = 0, kBandPot = 1 };

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d));
  return v;
}

// warp-wide argmax (ties -> smallest index); every lane gets the result
__device__ __forceinline__ void warp_argmax(float& v, int& i) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, d);
    const int oi = __shfl_xor_sync(0xffffffffu, i, d);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
}

__device__ __forceinline__ int chunk_dist(int j, int a, int b, int len) {
  // distance from chunk j's index interval to the index interval [a, b]
  const int lo = j * kCW, hi = min(lo + kCW, len) - 1;
  return b < lo ? lo - b : (a > hi ? a - hi : 0);
}

// chunk maxima: cmax[r][j] = scale * max_{m in chunk j} x[r][m]; one warp per row
template <int MAXP>
__global__ void chunk_max_kernel(const __grid_constant__ BandTable<MAXP> t) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= t.rows) return;
  const BandArgs& a = t.p[find_prob<MAXP, 0>(t, gw)];
  if (error_latched(a.err)) return;
  const int row = gw - a.row_base;
  const float* xr = a.x + (size_t)row * a.len;
  for (int j = 0; j < a.n_chunks; ++j) {
    const int m = j * kCW + lane;
    const float v = warp_max(m < a.len ? xr[m] : -INFINITY);
    if (lane == 0) a.cmax[(size_t)row * a.n_chunks + j] = v * a.x_scale;
  }
}

// Per (row, tile) plan: exact centre offset alpha, window start lo and length wl.  One warp
// per (row, group of 16 tiles): the monotone search runs over the group's centres with
// lane-parallel scans of contiguous ranges of m (the group's first scan covers the whole
// row); the windows are then found with one lane per tile.
constexpr int kPlanGroup = 16;

template <int MAXP>
__global__ void __launch_bounds__(256) band_plan_kernel(const __grid_constant__ BandTable<MAXP> tab) {
  __shared__ float s_al[8][kPlanGroup];
  __shared__ int s_arg[8][kPlanGroup];
  __shared__ int4 s_stack[8][16];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * 8 + w;
  if (gw >= tab.plans) return;                            // warp-uniform
  const BandArgs& a = tab.p[find_prob<MAXP, 1>(tab, gw)];
  if (error_latched(a.err)) return;
  const int T = a.n_tiles, len = a.len;
  const int groups = (T + kPlanGroup - 1) / kPlanGroup;
  const int lw = gw - a.plan_base;
  const size_t np = (size_t)a.n_rows * T;
  float* p_alpha = a.plan;
  int* p_lo = reinterpret_cast<int*>(a.plan + np);
  int* p_wl = reinterpret_cast<int*>(a.plan + 2 * np);
  const int row = lw / groups, t0 = (lw % groups) * kPlanGroup;
  const int t1 = min(t0 + kPlanGroup, T) - 1;
  const float c = a.c, sc = a.x_scale;
  const float* xr = a.x + (size_t)row * len;
  // 1. monotone divide and conquer over the group's centres (depth-first, left child first)
  int sp = 1;
  if (lane == 0) s_stack[w][0] = make_int4(t0, t1, 0, len - 1);
  bool row_empty = false;
  __syncwarp();
  while (sp > 0) {
    const int4 e = s_stack[w][sp - 1];
    --sp;
    if (e.x > e.y) continue;
    const int mid = (e.x + e.y) >> 1;
    const int kc = mid * kBT + kBT / 2;
    float best = -INFINITY;
    int arg = 0x7fffffff;
    for (int pass = 0; pass < 2; ++pass) {
      // pass 1 only when the restricted range held no finite term (rounding can break the
      // monotone order by an ulp): then scan the whole row
      const int mlo = pass == 0 ? e.z : 0, mhi = pass == 0 ? e.w : len - 1;
#pragma unroll 4
      for (int m = mlo + lane; m <= mhi; m += 32) {
        const float d = (float)(kc - m);
        const float v = fmaf(-d * d, c, xr[m] * sc);
        if (v > best) {
          best = v;
          arg = m;
        }
      }
      warp_argmax(best, arg);
      if (best != -INFINITY || row_empty || (mlo == 0 && mhi == len - 1)) break;
    }
    if (best == -INFINITY) {                              // no finite term anywhere: empty row
      row_empty = true;
      arg = e.z;
    }
    __syncwarp();
    if (lane == 0) {
      s_al[w][mid - t0] = best;
      s_arg[w][mid - t0] = arg;
      s_stack[w][sp] = make_int4(mid + 1, e.y, arg, e.w);
      s_stack[w][sp + 1] = make_int4(e.x, mid - 1, e.z, arg);
    }
    sp += 2;
    __syncwarp();
  }
  // 2. windows, one lane per tile
  const float* cm = a.cmax + (size_t)row * a.n_chunks;
  const int t = t0 + lane;
  if (lane >= kPlanGroup || t > t1) return;
  const size_t pi = (size_t)row * T + t;
  const float al = s_al[w][lane];
  if (al == -INFINITY) {
    p_alpha[pi] = -INFINITY;
    p_lo[pi] = 0;
    p_wl[pi] = 0;
    return;
  }
  const int k0 = t * kBT, kc = k0 + kBT / 2, k1 = min(k0 + kBT, len) - 1;
  const float dM = (float)(s_arg[w][lane] - kc);
  const float ka = (float)(k0 - kc), kb = (float)(k1 - kc);
  const float lb = al + fminf(fmaf(2.f * ka, dM * c, -ka * ka * c), fmaf(2.f * kb, dM * c, -kb * kb * c));
  int jlo = a.n_chunks, jhi = -1;
  for (int j = 0; j < a.n_chunks; ++j) {
    const float d = (float)chunk_dist(j, k0, k1, len);
    if (fmaf(-d * d, c, cm[j]) >= lb - kCut) {
      jlo = min(jlo, j);
      jhi = j;
    }
  }
  p_alpha[pi] = al;
  p_lo[pi] = jlo * kCW;
  p_wl[pi] = min((jhi + 1) * kCW, len) - jlo * kCW;
}

// PATH 0 handles the items that take the tilted GEMM, PATH 1 the exact-window items; the two
// variants are launched back to back and each skips the other's items (lean registers).
constexpr int kSA = 8 * 36 + 4;   // floats per half-warp A block (8 rows x 36, +4: banks)

template <int MODE, int PATH, int MAXP>
__global__ void __launch_bounds__(kBW * 32, 3) band_pass_kernel(const __grid_constant__ BandTable<MAXP> tab) {
  __shared__ __align__(16) float sA[kBW][2 * kSA];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h = lane >> 4, i = lane & 15;
  const int gw = blockIdx.x * kBW + warp;
  if (gw >= tab.items) return;                            // warp-uniform
  const BandArgs& a = tab.p[find_prob<MAXP, 2>(tab, gw)];
  if (error_latched(a.err)) return;
  const int lw = gw - a.item_base;
  const int tile = lw % a.n_tiles, r0 = (lw / a.n_tiles) * 2 * kBR;
  if (a.skip && a.skip[(size_t)(r0 / 128) * a.n_tiles + tile]) return;   // done on the tensor cores
  const size_t np = (size_t)a.n_rows * a.n_tiles;
  const float* __restrict__ p_alpha = a.plan;
  const int* __restrict__ p_lo = reinterpret_cast<const int*>(a.plan + np);
  const int* __restrict__ p_wl = reinterpret_cast<const int*>(a.plan + 2 * np);
  const int rh = r0 + h * kBR;                             // this half's first row
  const int k0 = tile * kBT, kc = k0 + kBT / 2;
  const int k1 = min(k0 + kBT, a.len) - 1;
  const float c = a.c, sc = a.x_scale;

  float alpha[kBR];
  int lo[kBR], wl[kBR];
  int W = 0;
#pragma unroll
  for (int rr = 0; rr < kBR; ++rr) {
    const int r = rh + rr;
    if (r < a.n_rows) {
      const size_t pi = (size_t)r * a.n_tiles + tile;
      alpha[rr] = p_alpha[pi];
      lo[rr] = p_lo[pi];
      wl[rr] = p_wl[pi];
    } else {
      alpha[rr] = -INFINITY;
      lo[rr] = 0;
      wl[rr] = 0;
    }
    W = max(W, wl[rr]);
  }
  W = max(W, __shfl_xor_sync(0xffffffffu, W, 16));        // common to both halves
  const int k = k0 + i;
  const float kap = (float)(k - kc);
  const float kmax = (float)(kBT / 2);
  float out[kBR];
#pragma unroll
  for (int rr = 0; rr < kBR; ++rr) out[rr] = -INFINITY;

  const bool gemm = W > 0 && kmax * (float)W * c <= kTiltMax && kmax * kmax * c <= 32.f;
  if (gemm != (PATH == 0)) return;                        // the other variant's item
  if (i == 0) {                                           // lanes 0 and 16: per-half count
    unsigned long long t = 0;
    if (gemm) {
      if (h == 0) t = (unsigned long long)W * kBT * 2 * kBR;
    } else {
#pragma unroll
      for (int rr = 0; rr < kBR; ++rr) t += (unsigned long long)wl[rr] * kBT;
    }
    if (t) atomicAdd(a.terms, t);
  }
  float* sAh = &sA[warp][h * kSA];
  if (PATH == 0) {
    // 3. tilted GEMM over the common window length W.  Lane (h, i) produces window
    // positions m0 + 2i, m0 + 2i + 1 of its half's 8 rows; the next chunk's inputs are
    // loaded before the current chunk's multiply-adds.
    float acc[kBR], xn[2 * kBR];
#pragma unroll
    for (int rr = 0; rr < kBR; ++rr) {
      acc[rr] = 0.f;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int mp = 2 * i + u, m = lo[rr] + mp;
        xn[2 * rr + u] = (alpha[rr] != -INFINITY && mp < W && m < a.len)
                             ? a.x[(size_t)(rh + rr) * a.len + m] : -INFINITY;
      }
    }
    const float halfW = 0.5f * (float)W;
    const float t2 = 2.f * kap * c, tk = -kap * kap * c;
    for (int m0 = 0; m0 < W; m0 += 32) {
#pragma unroll
      for (int rr = 0; rr < kBR; ++rr) {
        float2 v;
        const int mp = m0 + 2 * i;
        const float d0 = (float)(kc - (lo[rr] + mp)), d1 = d0 - 1.f;
        v.x = ex2(fmaf(-d0 * d0, c, xn[2 * rr] * sc) - alpha[rr]);      // x = -inf -> 0
        v.y = ex2(fmaf(-d1 * d1, c, xn[2 * rr + 1] * sc) - alpha[rr]);
        *reinterpret_cast<float2*>(&sAh[rr * 36 + 2 * i]) = v;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int mq = m0 + 32 + 2 * i + u, m = lo[rr] + mq;
          xn[2 * rr + u] = (alpha[rr] != -INFINITY && mq < W && m < a.len)
                               ? a.x[(size_t)(rh + rr) * a.len + m] : -INFINITY;
        }
      }
      __syncwarp();
      float mp = (float)m0 - halfW;
#pragma unroll 2
      for (int j = 0; j < 32; j += 4) {
        float b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) b[u] = ex2(fmaf(t2, mp + (float)u, tk));
        mp += 4.f;
#pragma unroll
        for (int rr = 0; rr < kBR; ++rr) {
          const float4 av = *reinterpret_cast<const float4*>(&sAh[rr * 36 + j]);
          acc[rr] = fmaf(av.x, b[0], acc[rr]);
          acc[rr] = fmaf(av.y, b[1], acc[rr]);
          acc[rr] = fmaf(av.z, b[2], acc[rr]);
          acc[rr] = fmaf(av.w, b[3], acc[rr]);
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int rr = 0; rr < kBR; ++rr) {
      if (alpha[rr] == -INFINITY) continue;
      if (!(acc[rr] > 0.f) || !isfinite(acc[rr])) {
        raise_error(a.err, FOT_ENONFINITE);               // outside the tilt bounds: a bug
        continue;
      }
      const float mref = (float)lo[rr] + halfW;
      out[rr] = alpha[rr] + 2.f * kap * (mref - (float)kc) * c + log2f(acc[rr]);
    }
  } else {
    // 4. exact log-sum-exp over each row's own window; the two halves step through their
    // rows together (loop bounds from the larger of the two windows)
#pragma unroll
    for (int rr = 0; rr < kBR; ++rr) {
      const int wr = max(wl[rr], __shfl_xor_sync(0xffffffffu, wl[rr], 16));
      const float* xr = a.x + (size_t)min(rh + rr, a.n_rows - 1) * a.len;
      float mx = -INFINITY, sum = 0.f;
      // both sweeps run for every lane (the two halves own different rows and sync per warp)
      for (int sweep = 0; sweep < 2; ++sweep) {
        const float mref = (sweep == 1 && mx == -INFINITY) ? 0.f : mx;   // empty: all terms 0
        for (int m0 = 0; m0 < wr; m0 += 32) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int mp = m0 + 2 * i + u;
            sAh[2 * i + u] = (alpha[rr] != -INFINITY && mp < wl[rr]) ? xr[lo[rr] + mp] * sc : -INFINITY;
          }
          __syncwarp();
          for (int j = 0; j < 32; ++j) {
            const float d = (float)(k - (lo[rr] + m0 + j));
            const float e = fmaf(-d * d, c, sAh[j]);
            if (sweep == 0)
              mx = fmaxf(mx, e);
            else
              sum += ex2(e - mref);
          }
          __syncwarp();
        }
      }
      if (alpha[rr] != -INFINITY && mx != -INFINITY) out[rr] = mx + log2f(sum);
    }
  }

  if (k > k1) return;
  // epilogue: output (o = k, r) at y[k * n_rows + r]
#pragma unroll
  for (int rr = 0; rr < kBR; ++rr) {
    const int r = rh + rr;
    if (r >= a.n_rows) break;
    const size_t yi = (size_t)k * a.n_rows + r;
    if (MODE == kBandLse) {
      a.y[yi] = out[rr];
    } else {
      const float s = out[rr] * kLn2;
      const float lm = a.lmarg[yi];
      float pot;
      if (lm == -INFINITY) {
        pot = -INFINITY;
      } else {
        pot = a.eps * (lm - s);
        if (!isfinite(pot)) raise_error(a.err, FOT_ENONFINITE);
      }
      a.y[yi] = pot;
      if (a.logsum) a.logsum[yi] = s;
    }
  }
}

template <int MAXP>
void band_table_finish(BandTable<MAXP>& t) {
  int rows = 0, plans = 0, items = 0, ctas = 0;
  for (int q = 0; q < t.n; ++q) {
    BandArgs& a = t.p[q];
    a.n_chunks = (a.len + kCW - 1) / kCW;
    a.n_tiles = (a.len + kBT - 1) / kBT;
    a.row_base = rows;
    a.plan_base = plans;
    a.item_base = items;
    a.cta_base = ctas;
    rows += a.n_rows;
    plans += a.n_rows * ((a.n_tiles + kPlanGroup - 1) / kPlanGroup);
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
  chunk_max_kernel<MAXP><<<(t.rows + 7) / 8, 256, 0, s>>>(t);
  band_plan_kernel<MAXP><<<(t.plans + 7) / 8, 256, 0, s>>>(t);
}

template <int MODE, int MAXP>
void band_simt(cudaStream_t s, const BandTable<MAXP>& t) {
  band_pass_kernel<MODE, 0, MAXP><<<(t.items + kBW - 1) / kBW, kBW * 32, 0, s>>>(t);
  band_pass_kernel<MODE, 1, MAXP><<<(t.items + kBW - 1) / kBW, kBW * 32, 0, s>>>(t);
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
  a.cmax = c->cmax;
  a.plan = c->cmax + (size_t)c->rows * ((c->cols + kCW - 1) / kCW) + (size_t)c->cols * ((c->rows + kCW - 1) / kCW);
  a.err = c->err;
  a.terms = c->terms;
  a.x_scale = x_scale;
  a.c = (float)(1.4426950408889634 / (2.0 * eps));
  a.eps = (float)eps;
  a.n_rows = n_rows;
  a.len = len;
  return a;
}

// One half-step with banded passes: pot_out = eps (lmarg - log(Lambda exp(pot_in/eps) Lambda)).
void half_step_band(fot_ctx* c, const float* pot_in, const float* lmarg, double eps,
                    float* pot_out, float* logsum, float* tmp, float* cmax) {
  (void)cmax;
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
  c->launches += 8;
}

}  // namespace fot
