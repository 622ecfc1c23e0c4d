// Banded pass building blocks shared by the CUDA-core kernels (fot_band.cu) and the
// tensor-core kernel (fot_tc.cu), which runs the CUDA-core window sums itself for the tiles
// whose tilt bounds it cannot meet.  The algorithm is described in fot_band.cu.
#pragma once

#include "fot_band.cuh"

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

// PATH 0 handles the items that take the tilted GEMM, PATH 1 the exact-window items; callers
// invoke both and each returns at once on the other's items (the choice is warp-uniform).
constexpr int kSA = 8 * 36 + 4;   // floats per half-warp A block (8 rows x 36, +4: banks)

// The work of one (16-row group from row r0, 16 outputs from k0) item; PATH 0 = tilted GEMM,
// PATH 1 = exact window sums.  Returns at once when the item belongs to the other PATH.
// The plan entry is (row, pt): with a 16-wide plan pt = k0 / 16; a wider plan tile holding
// these outputs gives a window that covers theirs, and then its alpha is not the maximum at
// this item's centre: either only PATH 1 may be used (EXACT_ONLY), or the item first takes
// every row's exact maximum over its window at its own centre (OWN_ALPHA, one sweep of the
// window without exponentials) and then both paths apply.
// sAw: this warp's 2 * kSA floats of shared memory.
template <int MODE, int PATH, bool EXACT_ONLY = false, bool OWN_ALPHA = false>
__device__ __forceinline__ void band_item(const BandArgs& a, int r0, int pt, int k0, float* sAw) {
  const int lane = threadIdx.x & 31;
  const int h = lane >> 4, i = lane & 15;
  const size_t np = (size_t)a.plan_stride * a.n_tiles;
  const float* __restrict__ p_alpha = a.plan;
  const int* __restrict__ p_lo = reinterpret_cast<const int*>(a.plan + np);
  const int* __restrict__ p_wl = reinterpret_cast<const int*>(a.plan + 2 * np);
  const int rh = r0 + h * kBR;                             // this half's first row
  const int kc = k0 + kBT / 2;
  const int k1 = min(k0 + kBT, a.len) - 1;
  const float c = a.c, sc = a.x_scale;

  float alpha[kBR];
  int lo[kBR], wl[kBR];
  int W = 0;
#pragma unroll
  for (int rr = 0; rr < kBR; ++rr) {
    const int r = rh + rr;
    if (r < a.n_rows) {
      const size_t pi = (size_t)pt * a.plan_stride + r;
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
  if (OWN_ALPHA) {
    // alpha_r = max over the row's window of x_r[m] sc - (kc - m)^2 c (the exponent PATH 0
    // forms), lanes of a half-warp striding the window, then a max over the half-warp
#pragma unroll
    for (int rr = 0; rr < kBR; ++rr) {
      float mx = -INFINITY;
      if (alpha[rr] != -INFINITY) {
        const float* xr = a.x + (size_t)(rh + rr) * a.len;
        for (int mp = i; mp < wl[rr]; mp += kBT) {
          const int m = lo[rr] + mp;
          const float d = (float)(kc - m);
          mx = fmaxf(mx, fmaf(-d * d, c, xr[m] * sc));
        }
      }
#pragma unroll
      for (int o = kBT / 2; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (alpha[rr] != -INFINITY) alpha[rr] = mx;
    }
  }
  const int k = k0 + i;
  const float kap = (float)(k - kc);
  const float kmax = (float)(kBT / 2);
  float out[kBR];
#pragma unroll
  for (int rr = 0; rr < kBR; ++rr) out[rr] = -INFINITY;

  const bool gemm = !EXACT_ONLY && W > 0 && kmax * (float)W * c <= kTiltMax && kmax * kmax * c <= 32.f;
  if (gemm != (PATH == 0)) return;                        // the other variant's item
  if (i == 0) {                                           // lanes 0 and 16: per-half count
    unsigned long long t = 0;
    if (gemm) {
      if (h == 0) t = (unsigned long long)W * kBT * 2 * kBR;
    } else {
#pragma unroll
      for (int rr = 0; rr < kBR; ++rr) t += (unsigned long long)wl[rr] * kBT;
    }
    if (t) atomicAdd(a.terms + PATH, t);
  }
  float* sAh = &sAw[h * kSA];
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
    const float rstep = ex2(t2);                          // B[m' + 1] / B[m']
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
        // B at four consecutive positions: one exponential, then the constant ratio 2^t2
        float b[4];
        b[0] = ex2(fmaf(t2, mp, tk));
#pragma unroll
        for (int u = 1; u < 4; ++u) b[u] = __fmul_rn(b[u - 1], rstep);
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
      out[rr] = __fadd_rn(fmaf(2.f * kap * (mref - (float)kc), c, alpha[rr]), log2f(acc[rr]));
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
      if (alpha[rr] != -INFINITY && mx != -INFINITY) out[rr] = __fadd_rn(mx, log2f(sum));
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
      const float s = __fmul_rn(out[rr], kLn2);
      const float lm = a.lmarg[yi];
      float pot;
      if (lm == -INFINITY) {
        pot = -INFINITY;
      } else {
        pot = __fmul_rn(a.eps, __fsub_rn(lm, s));
        if (!isfinite(pot)) raise_error(a.err, FOT_ENONFINITE);
      }
      a.y[yi] = pot;
      if (a.logsum) a.logsum[yi] = s;
    }
  }
}


}  // namespace fot
