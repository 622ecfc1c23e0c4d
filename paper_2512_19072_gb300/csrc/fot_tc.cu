// Tensor-core (tcgen05) form of the banded axis pass.
//
// The window sums of the banded pass (fot_band.cu, steps 3-4) are a GEMM:
//     C[r][kap] = sum_{m' < W} A[r][m'] B[m'][kap],
//     A[r][m'] = 2^(x_r[lo_r + m'] - (kc - lo_r - m')^2 c - alpha_r)   (<= 1, per row)
//     B[m'][kap] = 2^(2 kap (m' - W/2) c - kap^2 c)                     (same for all rows)
// after which y[kc + kap][r] = alpha_r + 2 kap (lo_r + W/2 - kc) c + log2 C[r][kap] (the
// per-row max-offsets of Sec. 3.1's Toeplitz contraction, plus the tilt).  One CTA computes
// a 128-row x TN-output tile (TN = 16, 32 or 64) with tcgen05.mma (M = 128, N = TN, K = 16
// per instruction), the FP32 accumulator in tensor memory.  A wider tile shares one A operand
// (one exponential per row and window position) between more outputs; the host picks the
// widest one whose tilt bound the problem's eps allows.
//
// Warp roles: eight producer warps generate the operands of each 32-position stage in shared
// memory (canonical no-swizzle K-major layout) and arrive on the stage's "full" mbarrier; one
// more warp owns the tensor memory and issues the stage's MMAs once all producers have
// arrived, committing to the stage's "empty" mbarrier, which the producers wait on before
// reusing it (a ring of four stages).  A last commit signals the epilogue, in which the producers read
// the accumulator (the potential-update pass prefetches its marginals during the last MMAs).
//
// Precision: each operand is split into two BF16 parts, v = hi + lo (hi = bf16(v),
// lo = bf16(v - hi)), and the product is accumulated as hi*hi + hi*lo + lo*hi (three MMAs):
// about 2^-16 relative per product instead of 2^-8, FP32 accumulation.  The epilogue takes
// log2 of the accumulator with the MUFU unit (about 2^-22 absolute), far below that.
//
// A CTA uses the tensor cores only when the tilt bound holds for the common window length W
// of its 128 rows: |kap| W c <= 48 with |kap| <= TN / 2.  Then every output's largest term has
// A >= 2^-96, and the A values that flush below 2^-126 add less than W 2^-30 relative: below
// the 2^-16 of the split-BF16 products.  Otherwise its producer warps compute the tile with the
// CUDA-core window sums of the banded pass (16 rows each; for a wider tile the exact window
// sums over the tile's window, which covers the windows of its 16-wide parts).  Every mbarrier
// wait is bounded: on time-out the kernel latches FOT_ETIMEOUT, stops issuing, waits (again
// bounded) for the MMAs in flight, frees its tensor memory and returns.
#include "fot_band_item.cuh"

#include <cuda_bf16.h>

#include <new>

namespace fot {

namespace {

constexpr int kTM = 128;            // rows per CTA (MMA M, TMEM lanes)
constexpr int kKC = 32;             // window positions per pipeline stage
constexpr int kStages = 4;          // operand stages in flight
constexpr int kPH = kKC / 2;        // window positions per producer thread and stage
constexpr int kGroupBytes = (kKC / 8) * 128;   // bytes between 8-row core-matrix groups
constexpr int kRouteKC = 64;        // window rounding of the host's tile-width estimate
constexpr int kProducerWarps = 8;   // operand producers (256 threads)
constexpr int kThreadsTC = kProducerWarps * 32 + 32;   // + the MMA-issuing warp
constexpr float kTiltMaxTC = 48.f;
constexpr int kSpin = 1 << 20;      // bounded mbarrier polls

// shared-memory layout of one stage (bytes): A_hi, A_lo (128 x 32 bf16 each), B_hi, B_lo
// (TN x 32 bf16 each), in 8 x 16-byte core matrices: core (g, kg) at g * 512 + kg * 128.
constexpr int kABytes = kTM * kKC * 2;   // 8192
template <int TN> struct TcShape {
  static constexpr int kBBytes = TN * kKC * 2;
  static constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;
  static constexpr int kSmemBytes = kStages * kStageBytes + 1024;   // the ring + slack
  static constexpr uint32_t kTmemCols = TN < 32 ? 32 : TN;    // power of two >= 32
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle, K-major:
// start address, leading (K-direction core-matrix) byte offset, stride (M/N-direction
// 8-row group) byte offset, fixed version bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :: "r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
  return ok != 0;
}

// bounded wait; false (and FOT_ETIMEOUT latched) if the phase never completes
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int* err) {
  for (int i = 0; i < kSpin; ++i)
    if (mbar_try(mbar, parity)) return true;
  raise_error(err, FOT_ETIMEOUT);
  return false;
}

// split 8 consecutive values into hi / lo BF16 parts (hi = round(v), lo = round(v - hi)) and
// store one 16-byte row of a core matrix for each (plain shared-memory stores; the caller
// fences them for the tensor core's async proxy)
__device__ __forceinline__ void store_split8(const float* v, unsigned char* hi_p, unsigned char* lo_p) {
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 hf = __bfloat1622float2(h2);
    const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
    hw[i] = *reinterpret_cast<const uint32_t*>(&h2);
    lw[i] = *reinterpret_cast<const uint32_t*>(&l2);
  }
  *reinterpret_cast<uint4*>(hi_p) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  *reinterpret_cast<uint4*>(lo_p) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// CUDA-core window sums of a declined tile (kept out of line: rarely run, and large)
template <int MODE, int TN>
__device__ __noinline__ void tc_declined_tile(const BandArgs& a, int rw, int tile, int k0, float* sAw) {
  if (TN == kBT) {
    band_item<MODE, 0>(a, rw, tile, k0, sAw);
    band_item<MODE, 1>(a, rw, tile, k0, sAw);
  } else {
    for (int q = 0; q < TN / kBT && k0 + q * kBT < a.len; ++q)
      band_item<MODE, 1, true>(a, rw, tile, k0 + q * kBT, sAw);
  }
}

template <int MODE, int TN, int MAXP>
__global__ void __launch_bounds__(kThreadsTC, 2) tc_pass_kernel(const __grid_constant__ BandTable<MAXP> tab) {
  constexpr int kTN = TN;
  constexpr int kStageBytes = TcShape<TN>::kStageBytes;
  constexpr int kBBytes = TcShape<TN>::kBBytes;
  constexpr uint32_t kTmemCols = TcShape<TN>::kTmemCols;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t full[kStages], empty[kStages], done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_wm[kTM / 32], s_err;
  const BandArgs& a = tab.p[find_prob<MAXP, 3>(tab, (int)blockIdx.x)];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lb = (int)blockIdx.x - a.cta_base;
  const int blk = lb / a.n_tiles, tile = lb % a.n_tiles;
  const int r0 = blk * kTM;
  const int k0 = tile * kTN, kc = k0 + kTN / 2;
  const int k1 = min(k0 + kTN, a.len) - 1;
  const float c = a.c, sc = a.x_scale;
  const bool producer = warp < kProducerWarps;

  // producer roles: A row r0 + ar (ar = tid % 128, which is also the accumulator row, i.e.
  // the tensor-memory lane 32 (warp % 4) + lane, that this thread reads in the epilogue),
  // half ah = tid / 128 (16 window positions each); B: core rows q = tid, tid + 256, ... of
  // TN outputs x 8 groups of 8 positions.  Both threads of a row read its plan entry straight
  // from global memory and start the loads of its first window chunk before any barrier, so
  // that the CTA waits out one memory latency before its first stage instead of three.
  const int ar = tid & (kTM - 1), ah = (tid >> 7) & 1;
  float a_alpha = -INFINITY;
  int a_lo = 0, a_wl = 0;
  if (producer && r0 + ar < a.n_rows) {
    const size_t np = (size_t)a.n_rows * a.n_tiles;
    const size_t pi = (size_t)(r0 + ar) * a.n_tiles + tile;
    a_alpha = a.plan[pi];
    a_lo = reinterpret_cast<const int*>(a.plan + np)[pi];
    a_wl = reinterpret_cast<const int*>(a.plan + 2 * np)[pi];
  }
  // window positions m' >= the row's own window length hold only terms below 2^-kCut of every
  // output of the tile (the provable window): their A values are written as zeros, with no
  // load and no exponential (rows with short windows cost little in a long tile)
  const float* xr = a.x + (size_t)min(r0 + ar, a.n_rows - 1) * a.len;
  // x of the next chunk, prefetched: 16 consecutive window positions of row ar.  lo and each
  // chunk start are multiples of 32, so the float4 loads are aligned; positions at or
  // beyond len read -inf (the kernel skips rows without mass).
  const bool a_live = producer && a_alpha != -INFINITY;
  // the 16-byte vector load needs the row base aligned too: x + row * len is 16-byte aligned
  // only when row * len is a multiple of 4 (window starts are multiples of 32)
  const bool vec_ok = (reinterpret_cast<uintptr_t>(xr) & 15u) == 0;
  float4 xq[kPH / 4];
  auto load_x = [&](int m0) {
    if (m0 + ah * kPH >= a_wl) return;                  // outside the row's window
    const int mb = a_lo + m0 + ah * kPH;
#pragma unroll
    for (int q = 0; q < kPH / 4; ++q) {
      const int m = mb + 4 * q;
      if (a_live && vec_ok && m + 3 < a.len) {
        xq[q] = __ldg(reinterpret_cast<const float4*>(xr + m));
      } else {
        xq[q].x = (a_live && m < a.len) ? xr[m] : -INFINITY;
        xq[q].y = (a_live && m + 1 < a.len) ? xr[m + 1] : -INFINITY;
        xq[q].z = (a_live && m + 2 < a.len) ? xr[m + 2] : -INFINITY;
        xq[q].w = (a_live && m + 3 < a.len) ? xr[m + 3] : -INFINITY;
      }
    }
  };
  if (producer) load_x(0);                  // in flight while the CTA sets up

  // the common window length of the 128 rows: warps 0-3 hold one thread per row
  int wm = a_wl;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) wm = max(wm, __shfl_xor_sync(0xffffffffu, wm, off));
  if (lane == 0 && warp < kTM / 32) s_wm[warp] = wm;
  if (tid == 0) s_err = error_latched(a.err) ? 1 : 0;   // one read: the exit is CTA-uniform

  // the MMA warp owns the tensor memory (128 x TN FP32 accumulator) and the barriers:
  // full[s] (256 producer arrivals: stage s written), empty[s] (the commit of the MMAs that
  // read stage s), done (the commit after the last chunk)
  if (warp == kProducerWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base_sh)), "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    if (lane == 0) {
      for (int i = 0; i < kStages; ++i) {
        mbar_init(smem_u32(&full[i]), kProducerWarps * 32);
        mbar_init(smem_u32(&empty[i]), 1);
      }
      mbar_init(smem_u32(&done), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int wmax = max(max(s_wm[0], s_wm[1]), max(s_wm[2], s_wm[3]));
  const int W = ((wmax + kKC - 1) / kKC) * kKC;
  const float kmax = (float)(kTN / 2);
  const bool take = wmax > 0 && kmax * (float)W * c <= kTiltMaxTC && kmax * kmax * c <= 32.f;
  if (s_err || !take) {                                 // CTA-uniform
    if (warp == kProducerWarps)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem_base_sh),
                   "r"(kTmemCols) : "memory");
    if (s_err) return;
    const int rw = r0 + warp * 2 * kBR;                 // producer warp w: rows rw .. rw + 15
    if (warp < kProducerWarps && rw < a.n_rows)
      tc_declined_tile<MODE, TN>(a, rw, tile, k0, reinterpret_cast<float*>(smem) + warp * 2 * kSA);
    return;
  }
  if (tid == 0) atomicAdd(a.tc_terms, (unsigned long long)W * kTN * kTM);

  const uint32_t sbase = smem_u32(smem);
  const float halfW = 0.5f * (float)W;
  const int nchunk = W / kKC;
  const uint32_t tmem_d = tmem_base_sh;
  bool ok = true;

  if (!producer) {
    // MMA warp: lane 0 issues each stage's MMAs once its 256 producers have arrived
    if (lane == 0) {
      const uint32_t idesc = instr_desc(kTM, kTN);
      for (int ch = 0; ch < nchunk; ++ch) {
        const int s = ch % kStages;
        if (!mbar_wait(smem_u32(&full[s]), (ch / kStages) & 1, a.err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = sbase + s * kStageBytes;
        const uint32_t sAhi = st, sAlo = st + kABytes, sBhi = st + 2 * kABytes, sBlo = sBhi + kBBytes;
#pragma unroll
        for (int ks = 0; ks < kKC / 16; ++ks) {
          const uint64_t dAh = smem_desc(sAhi + ks * 256, 128, kGroupBytes);
          const uint64_t dAl = smem_desc(sAlo + ks * 256, 128, kGroupBytes);
          const uint64_t dBh = smem_desc(sBhi + ks * 256, 128, kGroupBytes);
          const uint64_t dBl = smem_desc(sBlo + ks * 256, 128, kGroupBytes);
          mma_bf16(tmem_d, dAh, dBh, idesc, (ch > 0 || ks > 0) ? 1u : 0u);
          mma_bf16(tmem_d, dAh, dBl, idesc, 1u);
          mma_bf16(tmem_d, dAl, dBh, idesc, 1u);
        }
        mma_commit(smem_u32(&empty[s]));
      }
      // arrives when every MMA issued above has completed; the producers wait on it before
      // reading the accumulator, and this thread before the tensor memory is released
      mma_commit(smem_u32(&done));
      ok = mbar_wait(smem_u32(&done), 0, a.err) && ok;
    }
    __syncwarp();
  } else {
    for (int ch = 0; ch < nchunk; ++ch) {
      const int s = ch % kStages;
      // stage free again: the MMAs of chunk ch - kStages (its previous use) have completed
      if (ch >= kStages && !mbar_wait(smem_u32(&empty[s]), ((ch - kStages) / kStages) & 1, a.err)) {
        ok = false;
        break;
      }
      unsigned char* const stp = smem + s * kStageBytes;
      const int m0 = ch * kKC;
      float xv[kPH];
#pragma unroll
      for (int q = 0; q < kPH / 4; ++q) {
        xv[4 * q] = xq[q].x;
        xv[4 * q + 1] = xq[q].y;
        xv[4 * q + 2] = xq[q].z;
        xv[4 * q + 3] = xq[q].w;
      }
      if (ch + 1 < nchunk) load_x(m0 + kKC);
      // A: 16 consecutive window positions of row ar -> 2 core-matrix rows of 8 values
      const float dbase = (float)(kc - (a_lo + m0 + ah * kPH));
      if (!a_live || m0 + ah * kPH >= a_wl) {
        // no term of this row here: zeros
#pragma unroll
        for (int g = 0; g < kPH / 8; ++g) {
          const uint32_t off = (uint32_t)((ar >> 3) * kGroupBytes + (ah * (kPH / 8) + g) * 128 + (ar & 7) * 16);
          *reinterpret_cast<uint4*>(stp + off) = make_uint4(0u, 0u, 0u, 0u);
          *reinterpret_cast<uint4*>(stp + kABytes + off) = make_uint4(0u, 0u, 0u, 0u);
        }
      } else {
#pragma unroll
        for (int g = 0; g < kPH / 8; ++g) {
          float v[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float d = dbase - (float)(g * 8 + i);
            v[i] = ex2(fmaf(-d * d, c, xv[g * 8 + i] * sc) - a_alpha);   // x = -inf -> 0
          }
          const int kg = ah * (kPH / 8) + g;              // core-matrix column in the stage
          const uint32_t off = (uint32_t)((ar >> 3) * kGroupBytes + kg * 128 + (ar & 7) * 16);
          store_split8(v, stp + off, stp + kABytes + off);
        }
      }
      // B: 8 window positions of output bn per core row
#pragma unroll
      for (int q = tid; q < kTN * (kKC / 8); q += kProducerWarps * 32) {
        const int bn = q % kTN, bq = q / kTN;
        const float bkap = (float)(bn - kTN / 2);
        const float bt2 = 2.f * bkap * c, btk = -bkap * bkap * c;
        // eight consecutive positions: one exponential, then the constant ratio 2^bt2
        float v[8];
        v[0] = ex2(fmaf(bt2, (float)(m0 + bq * 8) - halfW, btk));
        const float rstep = ex2(bt2);
#pragma unroll
        for (int i = 1; i < 8; ++i) v[i] = __fmul_rn(v[i - 1], rstep);
        const uint32_t off = (uint32_t)((bn >> 3) * kGroupBytes + bq * 128 + (bn & 7) * 16);
        store_split8(v, stp + 2 * kABytes + off, stp + 2 * kABytes + kBBytes + off);
      }
      // make the stores visible to the tensor core's async proxy, then arrive
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&full[s]));
    }
  }
  // epilogue geometry: accumulator row = TMEM lane = 32 * (warp % 4) + lane; warps w and w + 4
  // take the two halves of the TN columns, 8 at a time
  const int lq = warp & 3, half = (warp >> 2) & 1;
  const int rloc = 32 * lq + lane;
  const int r_out = r0 + rloc;
  // potential update: the marginals of this thread's outputs, loaded while the last MMAs run
  float lm_pre[kTN / 2];
#pragma unroll
  for (int u = 0; u < kTN / 2; ++u) {
    const int k = k0 + half * (kTN / 2) + u;
    lm_pre[u] = (MODE == 1 && producer && r_out < a.n_rows && k <= k1)
                    ? a.lmarg[(size_t)k * a.n_rows + r_out] : 0.f;
  }
  if (producer) ok = ok && mbar_wait(smem_u32(&done), 0, a.err);
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (ok && producer) {
    const float al = a_alpha;                       // rloc == ar: this thread's own row
    const float mref = (float)a_lo + halfW;
#pragma unroll
    for (int cg = 0; cg < kTN / 2; cg += 8) {
      const int n0 = half * (kTN / 2) + cg;
      uint32_t acc[8];
      const uint32_t taddr = tmem_d + ((uint32_t)(32 * lq) << 16) + (uint32_t)n0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(acc[0]), "=r"(acc[1]), "=r"(acc[2]), "=r"(acc[3]), "=r"(acc[4]), "=r"(acc[5]),
            "=r"(acc[6]), "=r"(acc[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r_out < a.n_rows) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int n = n0 + u;
          const int k = k0 + n;
          if (k > k1) break;
          const float kap = (float)(n - kTN / 2);
          const float cv = __uint_as_float(acc[u]);
          float out = -INFINITY;
          if (al != -INFINITY) {
            if (cv > 0.f && isfinite(cv))
              out = __fadd_rn(fmaf(2.f * kap * (mref - (float)kc), c, al), lg2(cv));
            else
              raise_error(a.err, FOT_ENONFINITE);
          }
          const size_t yi = (size_t)k * a.n_rows + r_out;
          if (MODE == 0) {
            a.y[yi] = out;
          } else {
            const float sv = __fmul_rn(out, kLn2);
            const float lm = lm_pre[cg + u];
            float pot;
            if (lm == -INFINITY) {
              pot = -INFINITY;
            } else {
              pot = __fmul_rn(a.eps, __fsub_rn(lm, sv));
              if (!isfinite(pot)) raise_error(a.err, FOT_ENONFINITE);
            }
            a.y[yi] = pot;
            if (a.logsum) a.logsum[yi] = sv;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kProducerWarps)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem_d), "r"(kTmemCols)
                 : "memory");
}

struct TcState {
  unsigned long long* tc_terms = nullptr; // window terms computed on the tensor cores
};

}  // namespace

bool tc_supported(int rows, int cols) { return rows >= 1 && cols >= 1; }

int tc_create(fot_ctx* c) {
  TcState* t = new (std::nothrow) TcState();
  if (!t) return 1;
  if (cudaMalloc((void**)&t->tc_terms, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemsetAsync(t->tc_terms, 0, sizeof(unsigned long long), c->stream) != cudaSuccess) {
    if (t->tc_terms) cudaFree(t->tc_terms);
    delete t;
    return 1;
  }
  // dynamic shared memory above 48 KB, for every instance (before any stream capture)
  bool ok = true;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<0, 16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<16>::kSmemBytes) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<1, 16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<16>::kSmemBytes) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<0, 16, kMaxBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<16>::kSmemBytes) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<1, 16, kMaxBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<16>::kSmemBytes) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<0, 32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<32>::kSmemBytes) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<1, 32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<32>::kSmemBytes) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<0, 32, kMaxBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<32>::kSmemBytes) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<1, 32, kMaxBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<32>::kSmemBytes) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<0, 64, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<64>::kSmemBytes) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<1, 64, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<64>::kSmemBytes) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<0, 64, kMaxBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<64>::kSmemBytes) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<1, 64, kMaxBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<64>::kSmemBytes) == cudaSuccess;
  if (!ok) {
    cudaFree(t->tc_terms);
    delete t;
    return 1;
  }
  c->tc = t;
  return 0;
}

void tc_destroy(fot_ctx* c) {
  TcState* t = (TcState*)c->tc;
  if (!t) return;
  cudaFree(t->tc_terms);
  delete t;
  c->tc = nullptr;
}

int64_t tc_terms(fot_ctx* c) {
  TcState* t = (TcState*)c->tc;
  if (!t) return 0;
  unsigned long long v = 0;
  cudaMemcpyAsync(&v, t->tc_terms, sizeof(v), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  return (int64_t)v;
}

// Tile width of a tensor-core pass for a problem with kernel constant c: the widest TN in
// {64, 32} whose tile is expected to meet the tilt bound |kap| W c <= kTiltMaxTC with room to
// spare: W is taken as twice the window of a smooth potential (the tile plus sqrt(kCut / c) on
// each side, where the Gaussian kernel alone has fallen by 2^-kCut), rounded up to a multiple
// of 64 positions, since the hull of a tile's windows grows where the transport map jumps across
// zero-mass gaps; else 16 when a 16-wide tile meets the bound with a window of kRouteKC
// positions; else 0: the CUDA-core kernel.  A declined wide tile costs exact window sums.
int tc_width_for(float c) {
  for (int tn = 64; tn >= 32; tn /= 2) {
    const float w = (float)tn + 2.f * sqrtf(kCut / c);
    const float wr = 2.f * ceilf(w / (float)kRouteKC) * (float)kRouteKC;
    if ((float)(tn / 2) * wr * c <= kTiltMaxTC && (float)(tn / 2) * (float)(tn / 2) * c <= 32.f) return tn;
  }
  if ((float)(kBT / 2) * (float)kRouteKC * c <= kTiltMaxTC) return 16;
  return 0;
}

// tw: the tile width every problem of the table uses (tc_width_for of its c)
template <int MODE, int MAXP>
int tc_pass(cudaStream_t s, BandTable<MAXP>& t, int tw) {
  for (int q = 0; q < t.n; ++q) t.p[q].tile_w = tw == 0 ? kBT : tw;
  band_table_finish(t);
  band_prepare(s, t);
  if (tw == 0) {
    band_simt<MODE>(s, t);
    return 2;
  }
  ktimer_begin(s, kKTensor);
  if (tw == 64)
    tc_pass_kernel<MODE, 64, MAXP><<<t.ctas, kThreadsTC, TcShape<64>::kSmemBytes, s>>>(t);
  else if (tw == 32)
    tc_pass_kernel<MODE, 32, MAXP><<<t.ctas, kThreadsTC, TcShape<32>::kSmemBytes, s>>>(t);
  else
    tc_pass_kernel<MODE, 16, MAXP><<<t.ctas, kThreadsTC, TcShape<16>::kSmemBytes, s>>>(t);
  ktimer_end(s);
  return 2;
}

unsigned long long* tc_terms_ptr(fot_ctx* c) { return c->tc ? ((TcState*)c->tc)->tc_terms : nullptr; }
template int tc_pass<0, 1>(cudaStream_t, BandTable<1>&, int);
template int tc_pass<1, 1>(cudaStream_t, BandTable<1>&, int);
template int tc_pass<0, kMaxBatch>(cudaStream_t, BandTable<kMaxBatch>&, int);
template int tc_pass<1, kMaxBatch>(cudaStream_t, BandTable<kMaxBatch>&, int);

BandArgs band_args(fot_ctx* c, const float* x, int n_rows, int len, double eps, float x_scale);

// One half-step with the tensor-core banded passes.
void half_step_tc(fot_ctx* c, const float* pot_in, const float* lmarg, double eps, float* pot_out,
                  float* logsum) {
  TcState* ts = (TcState*)c->tc;
  BandTable<1> t{};
  t.n = 1;
  t.p[0] = band_args(c, pot_in, c->rows, c->cols, eps, (float)(1.4426950408889634 / eps));
  t.p[0].y = c->R;
  t.p[0].tc_terms = ts->tc_terms;
  const int tw = tc_width_for(t.p[0].c);
  int k = tc_pass<0>(c->stream, t, tw);
  t.p[0] = band_args(c, c->R, c->cols, c->rows, eps, 1.f);
  t.p[0].y = pot_out;
  t.p[0].lmarg = lmarg;
  t.p[0].logsum = logsum;
  t.p[0].tc_terms = ts->tc_terms;
  k += tc_pass<1>(c->stream, t, tw);
  c->launches += k;
}

}  // namespace fot
