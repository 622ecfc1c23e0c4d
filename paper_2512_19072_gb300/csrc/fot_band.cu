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
//    all centres' maxima with O(len log n_tiles) evaluations per row.
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
constexpr int kMaxTiles = 4096 / kBT;
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
__global__ void chunk_max_kernel(const float* __restrict__ x, float scale, int n_rows, int len,
                                 int n_chunks, float* __restrict__ cmax, const int* err) {
  if (error_latched(err)) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n_rows) return;
  const float* xr = x + (size_t)warp * len;
  for (int j = 0; j < n_chunks; ++j) {
    const int m = j * kCW + lane;
    const float v = warp_max(m < len ? xr[m] : -INFINITY);
    if (lane == 0) cmax[(size_t)warp * n_chunks + j] = v * scale;
  }
}

// Per (row, tile) plan: exact centre offset alpha, window start lo and length wl.  One warp
// per row: the monotone search evaluates lane-parallel scans of contiguous ranges of m; the
// windows are then found with one lane per tile.
__global__ void __launch_bounds__(256) band_plan_kernel(BandArgs a, float* __restrict__ p_alpha,
                                                        int* __restrict__ p_lo, int* __restrict__ p_wl) {
  __shared__ float s_al[8][kMaxTiles];
  __shared__ int s_arg[8][kMaxTiles];
  __shared__ int4 s_stack[8][40];
  if (error_latched(a.err)) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + w;
  if (row >= a.n_rows) return;                            // warp-uniform
  const float c = a.c, sc = a.x_scale;
  const int T = a.n_tiles, len = a.len;
  const float* xr = a.x + (size_t)row * len;
  // 1. monotone divide and conquer over the tile centres (depth-first, left child first)
  int sp = 1;
  if (lane == 0) s_stack[w][0] = make_int4(0, T - 1, 0, len - 1);
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
      s_al[w][mid] = best;
      s_arg[w][mid] = arg;
      s_stack[w][sp] = make_int4(mid + 1, e.y, arg, e.w);
      s_stack[w][sp + 1] = make_int4(e.x, mid - 1, e.z, arg);
    }
    sp += 2;
    __syncwarp();
  }
  // 2. windows, one lane per tile
  const float* cm = a.cmax + (size_t)row * a.n_chunks;
  for (int t = lane; t < T; t += 32) {
    const size_t pi = (size_t)row * T + t;
    const float al = s_al[w][t];
    if (al == -INFINITY) {
      p_alpha[pi] = -INFINITY;
      p_lo[pi] = 0;
      p_wl[pi] = 0;
      continue;
    }
    const int k0 = t * kBT, kc = k0 + kBT / 2, k1 = min(k0 + kBT, len) - 1;
    const float dM = (float)(s_arg[w][t] - kc);
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
}

// PATH 0 handles the items that take the tilted GEMM, PATH 1 the exact-window items; the two
// variants are launched back to back and each skips the other's items (lean registers).
constexpr int kSA = 8 * 36 + 4;   // floats per half-warp A block (8 rows x 36, +4: banks)

template <int MODE, int PATH>
__global__ void __launch_bounds__(kBW * 32, 3) band_pass_kernel(BandArgs a, const float* __restrict__ p_alpha,
                                                                const int* __restrict__ p_lo,
                                                                const int* __restrict__ p_wl,
                                                                const unsigned char* __restrict__ skip) {
  __shared__ __align__(16) float sA[kBW][2 * kSA];
  if (error_latched(a.err)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h = lane >> 4, i = lane & 15;
  const int gw = blockIdx.x * kBW + warp;
  const int n_rg = (a.n_rows + 2 * kBR - 1) / (2 * kBR);
  if (gw >= n_rg * a.n_tiles) return;                     // warp-uniform
  const int tile = gw % a.n_tiles, r0 = (gw / a.n_tiles) * 2 * kBR;
  if (skip && skip[(size_t)(r0 / 128) * a.n_tiles + tile]) return;   // done on the tensor cores
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
      for (int sweep = 0; sweep < 2; ++sweep) {
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
              sum += ex2(e - mx);
          }
          __syncwarp();
        }
        if (mx == -INFINITY) break;
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

static void chunk_max(fot_ctx* c, const float* x, float scale, int n_rows, int len, float* cmax) {
  const int nch = (len + kCW - 1) / kCW;
  const int warps_per_block = 8;
  chunk_max_kernel<<<(n_rows + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0,
                     c->stream>>>(x, scale, n_rows, len, nch, cmax, c->err);
  c->launches++;
}

void band_prepare(fot_ctx* c, const BandArgs& a, float* plan) {
  chunk_max(c, a.x, a.x_scale, a.n_rows, a.len, const_cast<float*>(a.cmax));
  const size_t np = (size_t)a.n_rows * a.n_tiles;
  band_plan_kernel<<<(a.n_rows + 7) / 8, 256, 0, c->stream>>>(
      a, plan, reinterpret_cast<int*>(plan + np), reinterpret_cast<int*>(plan + 2 * np));
  c->launches++;
}

template <int MODE>
void band_simt(fot_ctx* c, const BandArgs& a, const float* plan, const unsigned char* skip) {
  const size_t np = (size_t)a.n_rows * a.n_tiles;
  const float* p_alpha = plan;
  const int* p_lo = reinterpret_cast<const int*>(plan + np);
  const int* p_wl = reinterpret_cast<const int*>(plan + 2 * np);
  const int n_rg = (a.n_rows + 2 * kBR - 1) / (2 * kBR);
  const int warps = n_rg * a.n_tiles;
  band_pass_kernel<MODE, 0><<<(warps + kBW - 1) / kBW, kBW * 32, 0, c->stream>>>(a, p_alpha, p_lo, p_wl, skip);
  band_pass_kernel<MODE, 1><<<(warps + kBW - 1) / kBW, kBW * 32, 0, c->stream>>>(a, p_alpha, p_lo, p_wl, skip);
  c->launches += 2;
}
template void band_simt<kBandLse>(fot_ctx*, const BandArgs&, const float*, const unsigned char*);
template void band_simt<kBandPot>(fot_ctx*, const BandArgs&, const float*, const unsigned char*);

// One half-step with banded passes: pot_out = eps (lmarg - log(Lambda exp(pot_in/eps) Lambda)).
void half_step_band(fot_ctx* c, const float* pot_in, const float* lmarg, double eps,
                    float* pot_out, float* logsum, float* tmp, float* cmax) {
  float* plan = cmax + (size_t)c->rows * ((c->cols + kCW - 1) / kCW) + (size_t)c->cols * ((c->rows + kCW - 1) / kCW);
  const float cc = (float)(1.4426950408889634 / (2.0 * eps));
  const float scale = (float)(1.4426950408889634 / eps);
  // pass over the contiguous axis: rows = rows of pot_in, outputs along cols
  BandArgs p{};
  p.x = pot_in; p.cmax = cmax; p.y = tmp; p.err = c->err; p.terms = c->terms;
  p.x_scale = scale; p.c = cc; p.eps = (float)eps;
  p.n_rows = c->rows; p.len = c->cols;
  p.n_chunks = (c->cols + kCW - 1) / kCW; p.n_tiles = (c->cols + kBT - 1) / kBT;
  band_prepare(c, p, plan);
  band_simt<kBandLse>(c, p, plan, nullptr);
  // pass over the row axis (input tmp[k][L], log2 units) with the fused potential update
  BandArgs q{};
  q.x = tmp; q.cmax = cmax; q.y = pot_out; q.lmarg = lmarg; q.logsum = logsum; q.err = c->err;
  q.terms = c->terms;
  q.x_scale = 1.f; q.c = cc; q.eps = (float)eps;
  q.n_rows = c->cols; q.len = c->rows;
  q.n_chunks = (c->rows + kCW - 1) / kCW; q.n_tiles = (c->rows + kBT - 1) / kBT;
  band_prepare(c, q, plan);
  band_simt<kBandPot>(c, q, plan, nullptr);
}

}  // namespace fot
