// Tensor-core (tcgen05) form of the banded axis pass.
//
// The window sums of the banded pass (fot_band.cu, steps 3-4) are a GEMM.  A unit is a
// 128-row block of the input x and a tile of TN consecutive outputs o = kc + kap around the
// tile centre kc.  The plan kernel gives every row r its offset alpha_r (at most the largest
// term at kc) and its window, and the union of the 128 windows [lo, lo + W) (W a multiple of
// 32).  Indexing the union window from its own start (m = lo + m'),
//     C[r][kap] = sum_{m' < W} A[r][m'] B[m'][kap],
//     A[r][m'] = 2^(x_r[lo + m'] - (kc - lo - m')^2 c - alpha_r)      (per row)
//     B[m'][kap] = 2^(2 kap (m' - W/2) c - kap^2 c)                    (the same for all rows)
// and y[kc + kap][r] = alpha_r + 2 kap (lo + W/2 - kc) c + log2 C[r][kap]: the per-row
// max-offsets of Sec. 3.1's Toeplitz contraction plus the tilt of the tile.  The union window
// holds every row's own window, so each row's sum covers at least its provable window; the
// extra positions only add exact (small) terms.
//
// One persistent CTA per SM.  The stages (32 window positions each) of all units of the pass
// are laid end to end and every CTA takes an equal contiguous share of them (stream-K).  A
// unit is accumulated in chunks of kChunk stages, each in a fresh accumulator, and the chunk
// sums are added in chunk order; a CTA takes the chunks that start in its share.  A unit whose
// chunks fall into several shares is split: each contributor writes its chunk sums to global
// slots and the last one to arrive adds them in chunk order and writes the outputs.  The
// arithmetic of every output is thus the same whatever the split (and whatever else shares the
// launch, e.g. the other problems of a batch): results do not depend on the grid.
//
// Warp roles (576 threads):
//  * warp 8, one lane (TMA): per stage, the 128 x 32 FP32 tile of x by a 2-D tensor copy
//    (128-byte swizzle) and the stage's B operand (a 1-D bulk copy from the pass's B table); at
//    a unit's first stage also the 128 row offsets alpha (1-D bulk copies for the producers and
//    for the epilogue) and, in the potential-update pass, the unit's [TN][128] block of log a
//    (a 2-D tensor copy) into the epilogue's slot.
//  * warps 0-7 (producers): thread (row ar, half ah) turns its 16 window positions into A,
//    split into two BF16 parts (v = hi + lo), stored in the canonical K-major core-matrix
//    layout.
//  * warp 9, one lane (MMA): per 16-position K step two tcgen05.mma (kind::f16, M = 128):
//    A_hi x [B_hi | B_lo] (N = 2 TN) and A_lo x B_hi (N = TN) into an FP32 accumulator in
//    tensor memory, so that hi*hi + hi*lo + lo*hi is accumulated (about 2^-16 relative per
//    product instead of 2^-8); two accumulators alternate between consecutive chunks.
//  * warps 10-17 (epilogue, two per tensor-memory lane quarter, each with half of the tile's
//    columns): read the accumulator (tcgen05.ld), add its two halves, take log2 (MUFU lg2),
//    add the offsets; the potential-update pass also applies f = eps (log a - S).
// Every barrier wait is bounded: on time-out the kernel latches FOT_ETIMEOUT, all roles leave
// their loops, the copies and MMAs in flight are waited for (again bounded) and the tensor
// memory is freed.
//
// A unit takes the tensor cores when its tilt bound holds: |kap| W c <= 48 with |kap| <= TN/2
// (and kap^2 c <= 32).  The largest term of every output then has A >= 2^-96 (alpha is at most
// the largest term at kc), and the A values that flush below 2^-126 add less than W 2^-30
// relative.  Other units (and units whose rows carry no mass) are summed on the CUDA cores by
// the producer warps after the tensor work, as 16-row x 16-output items dealt round-robin over
// all CTAs: each item takes its rows' exact maxima at its own centre, then the banded pass's
// tilted FP32 GEMM (or exact window sums where the item's own tilt bound fails too).
//
// Shared-memory hand-offs between the generic proxy (thread loads and stores) and the async
// proxy (TMA writes, MMA reads) are ordered by fence.proxy.async.shared::cta on the thread
// side, in both directions: after a thread's A stores (before the MMA reads them) and after its
// reads of an x tile or an epilogue slot (before the next tensor copy overwrites it).
#include "fot_band_item.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdlib.h>

#include <algorithm>
#include <new>

namespace fot {

namespace {

constexpr int kTM = 128;                 // rows per unit (MMA M, TMEM lanes)
constexpr int kKC = 32;                  // window positions per stage
constexpr int kXStages = 4;              // x tiles in flight
constexpr int kOpStagesMax = 4;          // operand stages in flight (TcShape::kOpStages)
constexpr int kAccBufs = 2;              // tensor-memory accumulators
constexpr int kEpiBufs = 2;              // epilogue slots in flight (a unit's alpha and log a)
constexpr int kProdWarps = 8;
constexpr int kProd = kProdWarps * 32;   // 256 producer threads
constexpr int kTmaWarp = 8, kMmaWarp = 9, kEpiWarp0 = 10, kEpiWarps = 8;
constexpr int kThreads = (kEpiWarp0 + kEpiWarps) * 32;   // 576
constexpr int kWarps = kThreads / 32;
constexpr int kEpi = kEpiWarps * 32;     // 256 epilogue threads: two per accumulator row (the
                                         // halves of the tile's columns)
constexpr int kXBytes = kTM * kKC * 4;   // 16 KB x tile
constexpr int kAlphaBytes = kTM * 4;     // 512 B of offsets
constexpr int kABytes = kTM * kKC * 2;   // 8 KB per BF16 part of A
constexpr int kGroupBytes = (kKC / 8) * 128;   // 512 B between 8-row core-matrix groups
constexpr float kTiltMaxTC = 48.f;
constexpr int kMaxPieces = 128;          // units one CTA's share may touch
constexpr int kChunk = 4;                // stages per accumulation chunk
constexpr int kMaxDecl = 1024;           // CUDA-core items (16 rows x 16 outputs) per CTA: every
                                         // unit of the largest table declined, dealt over 152 CTAs
constexpr int kUnitsPerThread = 8;       // units each thread holds during the set-up scan
constexpr int kSpinDefault = 1 << 20;    // bounded mbarrier polls
constexpr int kRouteKC = 64;             // window rounding of the host's tile-width estimate

// dynamic shared memory (bytes from a 1024-aligned base): the x ring, the producers' alpha per
// x slot, the epilogue's ring (per slot a unit's alpha, then in the potential-update pass its
// [TN][128] block of log a), the operand ring
template <int TN> struct TcShape {
  // operand stages in flight: four, three for 64-wide tiles (four do not fit in shared memory
  // beside the epilogue's two slots of log a)
  static constexpr int kOpStages = TN == 64 ? 3 : kOpStagesMax;
  static constexpr int kBBytes = 2 * TN * kKC * 2;          // B_hi rows, then B_lo rows
  static constexpr int kOpBytes = 2 * kABytes + kBBytes;
  static constexpr int kXAlphaOff = kXStages * kXBytes;
  static constexpr int kEpiOff = kXAlphaOff + kXStages * kAlphaBytes;
  static constexpr int kLmBytes = TN * kTM * 4;
  static constexpr int kEpiSlot = kAlphaBytes + kLmBytes;
  static constexpr int kOpOff = kEpiOff + kEpiBufs * kEpiSlot;
  static constexpr int kSmemBytes = kOpOff + kOpStages * kOpBytes + 1024;
  static_assert(kSmemBytes <= 227 * 1024 - 12 * 1024, "shared memory per CTA (dynamic + static)");
  // 2 accumulators of 2TN columns, then the TN-column running sum of a unit's chunks
  static constexpr uint32_t kTmemCols = 5 * TN <= 32 ? 32 : 5 * TN <= 64 ? 64 : 5 * TN <= 128 ? 128 : 5 * TN <= 256 ? 256 : 512;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle, K-major: start address, leading
// (K-direction core-matrix) byte offset, stride (M/N-direction 8-row group) byte offset,
// fixed version bits 46-48 = 0b001.
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

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
  return ok != 0;
}

// the same with a suspend-time hint: the thread may sleep up to hint_ns until the phase
// completes instead of spinning (its warp then takes no issue slots from the others)
__device__ __forceinline__ bool mbar_try_sleep(uint32_t mbar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok) : "r"(mbar), "r"(parity), "r"(hint_ns) : "memory");
  return ok != 0;
}

constexpr uint32_t kSleepNs = 2000;      // suspend-time hint of a poll (normal wait limit only)

// Bounded wait.  Returns false when another role has aborted the CTA, or when `limit` polls
// pass (then FOT_ETIMEOUT is latched and the CTA aborted).  With the normal limit each poll
// may sleep up to kSleepNs; a shorter limit (the test setting) polls without sleeping.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit, int* err,
                                          volatile int* abort) {
  const bool sleep = limit >= kSpinDefault;
  for (int i = 0; i < limit; ++i) {
    if (sleep ? mbar_try_sleep(mbar, parity, kSleepNs) : mbar_try(mbar, parity)) return true;
    if ((i & 31) == 31 && *abort) return false;
  }
  raise_error(err, FOT_ETIMEOUT);
  *abort = 1;
  return false;
}

// bounded wait that ignores the abort flag (the drain after an abort)
__device__ __forceinline__ void mbar_drain(uint32_t mbar, uint32_t parity) {
  for (int i = 0; i < kSpinDefault; ++i)
    if (mbar_try(mbar, parity)) return;
}

// AND of pred over the kEpi epilogue threads (named barrier 2): a decision they all take alike
__device__ __forceinline__ bool epi_all(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 2, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r) : "r"((uint32_t)pred), "r"(kEpi) : "memory");
  return r != 0;
}

// 2-D tensor copy of one box (x tile) into shared memory, completing on mbar
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int c0, int c1, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      :: "r"(dst), "l"(tmap), "r"(c0), "r"(c1), "r"(mbar) : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

// split 8 consecutive values into hi / lo BF16 parts (hi = round(v), lo = round(v - hi)) and
// store one 16-byte core-matrix row of each
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

// the hi part only (single BF16 operands)
__device__ __forceinline__ void store_hi8(const float* v, unsigned char* hi_p) {
  uint32_t hw[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    hw[i] = *reinterpret_cast<const uint32_t*>(&h2);
  }
  *reinterpret_cast<uint4*>(hi_p) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
}

// tensor-memory load / store of N consecutive 32-bit columns of this warp's 32 lanes
template <int N> __device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t* v);
template <> __device__ __forceinline__ void tmem_ld<4>(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(taddr));
}
// Wait for this thread's tensor-memory loads and pin their destination registers: the
// registers pass through the wait as read-write operands, so no use of them can be scheduled
// before the wait (a "memory" clobber orders memory accesses only, not register arithmetic).
template <int N> __device__ __forceinline__ void reg_pin(uint32_t* v);
template <> __device__ __forceinline__ void reg_pin<4>(uint32_t* v) {
  asm volatile("" : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]) :: "memory");
}
template <int N> __device__ __forceinline__ void tmem_wait_ld(uint32_t* a) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  reg_pin<N>(a);
}
template <int N> __device__ __forceinline__ void tmem_wait_ld(uint32_t* a, uint32_t* b) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  reg_pin<N>(a);
  reg_pin<N>(b);
}

template <int N> __device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t* v);
template <> __device__ __forceinline__ void tmem_st<4>(uint32_t taddr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};"
               :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]) : "memory");
}

// the CTA holding stage x of the pass when S stages are shared out over C CTAs (CTA k takes
// [k S / C, (k + 1) S / C))
// (32-bit arithmetic: the host keeps S * C below 2^32)
__device__ __forceinline__ int cta_of(uint32_t x, uint32_t S, uint32_t C) {
  return (int)(((x + 1u) * C - 1u) / S);
}
__device__ __forceinline__ uint32_t share_start(uint32_t k, uint32_t S, uint32_t C) { return k * S / C; }

// what a unit needs: its stage count when it takes the tensor cores (0 otherwise), whether it
// takes the CUDA-core sums instead, its union window start.  Every CTA must derive the same
// partition, so nothing here may change while the kernel runs (the error latch, which another
// CTA may set meanwhile, is not consulted).
template <int TN, int MAXP>
__device__ __forceinline__ void unit_info(const BandTable<MAXP>& tab, int u, int& S, int& decl, int& lo) {
  const BandArgs& a = tab.p[find_prob<MAXP, 3>(tab, u)];
  const int lu = u - a.cta_base;
  lo = a.ext_lo[lu];
  const int hi = a.ext_hi[lu];
  const int W = hi > lo ? (hi - lo + kKC - 1) / kKC * kKC : 0;
  const float kmax = (float)(TN / 2);
  const bool take = W > 0 && kmax * (float)W * a.c <= kTiltMaxTC && kmax * kmax * a.c <= 32.f;
  S = take ? W / kKC : 0;
  decl = take ? 0 : 1;
}

// CUDA-core window sums of one 16-row x 16-output item of a unit outside the tensor path
// (item it: rows r0 + 16 (it % 8), outputs k0 + 16 (it / 8)).  For a wider tile the item first
// takes its rows' maxima at its own centre, then the tilted GEMM or, where the item's own tilt
// bound fails too, the exact window sums.
constexpr int kRowItems = kTM / (2 * kBR);               // 8 row groups of 16 per unit
template <int MODE, int TN>
__device__ __noinline__ void tc_cuda_core_item(const BandArgs& a, int r0, int tile, int k0, int it, float* sAw) {
  const int rw = r0 + (it % kRowItems) * 2 * kBR;
  const int kq = k0 + (it / kRowItems) * kBT;
  if (rw >= a.n_rows || kq >= a.len) return;             // warp-uniform
  if (TN == kBT) {
    band_item<MODE, 0>(a, rw, tile, kq, sAw);
    band_item<MODE, 1>(a, rw, tile, kq, sAw);
  } else {
    band_item<MODE, 0, false, true>(a, rw, tile, kq, sAw);
    band_item<MODE, 1, false, true>(a, rw, tile, kq, sAw);
  }
}

template <int MODE, int TN, int MAXP>
__global__ void __launch_bounds__(kThreads, 1) tc_pass_kernel(const __grid_constant__ BandTable<MAXP> tab) {
  using Sh = TcShape<TN>;
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned base (the 128-byte swizzle of the x tiles), formed by pointer arithmetic
  // on the shared array so that every access through it compiles as a shared-memory access
  unsigned char* const smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ uint64_t xfull[kXStages], xempty[kXStages];
  __shared__ uint64_t opfull[Sh::kOpStages], opempty[Sh::kOpStages], bfull[Sh::kOpStages];
  __shared__ uint64_t accfull[kAccBufs], accempty[kAccBufs];
  __shared__ uint64_t eafull[kEpiBufs], eaempty[kEpiBufs];
  __shared__ uint64_t drain;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort, s_np, s_nd, s_first, s_last;
  __shared__ int4 s_piece[kMaxPieces];   // unit, first stage of the unit in the pass, stages, lo
  __shared__ int4 s_pcon[kMaxPieces];    // first and last contributor CTA, contributors
  __shared__ int s_decl[kMaxDecl];
  __shared__ long long s_wsum[kWarps][2];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int C = (int)gridDim.x, cta = (int)blockIdx.x;
  const int spin = tab.spin_limit;
  const bool single = tab.tc_single != 0;               // one BF16 MMA per term (FOT_BF16)
  volatile int* abort_flag = &s_abort;
  int* err0 = tab.p[0].err;

  if (tid == 0) {
    s_abort = 0;
    s_np = 0;
    s_nd = 0;
    s_first = 0x7fffffff;
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&s_tmem)), "r"(Sh::kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (warp == kTmaWarp && lane == 0) {
    for (int i = 0; i < kXStages; ++i) {
      mbar_init(smem_u32(&xfull[i]), 1);
      mbar_init(smem_u32(&xempty[i]), kProd);
    }
    for (int i = 0; i < Sh::kOpStages; ++i) {
      mbar_init(smem_u32(&opfull[i]), kProd);
      mbar_init(smem_u32(&opempty[i]), 1);
      mbar_init(smem_u32(&bfull[i]), 1);
    }
    for (int i = 0; i < kAccBufs; ++i) {
      mbar_init(smem_u32(&accfull[i]), 1);
      mbar_init(smem_u32(&accempty[i]), kEpi);
    }
    for (int i = 0; i < kEpiBufs; ++i) {
      mbar_init(smem_u32(&eafull[i]), 1);
      mbar_init(smem_u32(&eaempty[i]), kEpi);
    }
    mbar_init(smem_u32(&drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  // ---- set-up: the stage counts of all units, their prefix sums, this CTA's share -------------
  const int U = tab.ctas;
  const int per = (U + kThreads - 1) / kThreads;          // <= kUnitsPerThread (host check)
  const int u0 = min(U, tid * per), u1 = min(U, u0 + per);
  int uS[kUnitsPerThread], uD[kUnitsPerThread], uL[kUnitsPerThread];
  long long my_s = 0, my_t = 0;                           // stages; tensor units | CUDA-core units << 32
#pragma unroll
  for (int i = 0; i < kUnitsPerThread; ++i) {
    uS[i] = 0;
    uD[i] = 0;
    uL[i] = 0;
    if (u0 + i < u1) {
      unit_info<TN>(tab, u0 + i, uS[i], uD[i], uL[i]);
      my_s += uS[i];
      my_t += (uS[i] > 0 ? 1ll : 0ll) + ((long long)uD[i] << 32);
    }
  }
  // block-wide exclusive scan of (stages, counts) in unit order
  long long inc_s = my_s, inc_t = my_t;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long vs = __shfl_up_sync(0xffffffffu, inc_s, d);
    const long long vt = __shfl_up_sync(0xffffffffu, inc_t, d);
    if (lane >= d) {
      inc_s += vs;
      inc_t += vt;
    }
  }
  if (lane == 31) {
    s_wsum[warp][0] = inc_s;
    s_wsum[warp][1] = inc_t;
  }
  __syncthreads();
  long long base_s = inc_s - my_s, base_t = inc_t - my_t, tot_s = 0, tot_t = 0;
  for (int w = 0; w < kWarps; ++w) {
    if (w < warp) {
      base_s += s_wsum[w][0];
      base_t += s_wsum[w][1];
    }
    tot_s += s_wsum[w][0];
    tot_t += s_wsum[w][1];
  }
  const uint32_t S_tot = (uint32_t)tot_s;
  const uint32_t sb = S_tot > 0 ? share_start(cta, S_tot, C) : 0u;
  const uint32_t se = S_tot > 0 ? share_start(cta + 1, S_tot, C) : 0u;
  // this CTA takes the chunks of unit u that start in [sb, se): chunks [jlo, jhi)
  auto chunks_here = [&](uint32_t P, int S, int& jlo, int& jhi) {
    const int nc = (S + kChunk - 1) / kChunk;
    jlo = sb > P ? min(nc, (int)((sb - P + kChunk - 1) / kChunk)) : 0;
    jhi = se > P ? min(nc, (int)((se - P + kChunk - 1) / kChunk)) : 0;
  };
  {
    long long P = base_s, R = base_t & 0xffffffffll;
#pragma unroll
    for (int i = 0; i < kUnitsPerThread; ++i) {
      if (uS[i] > 0) {
        int jlo, jhi;
        chunks_here(P, uS[i], jlo, jhi);
        if (jlo < jhi) atomicMin(&s_first, (int)R);
      }
      P += uS[i];
      R += uS[i] > 0 ? 1 : 0;
    }
  }
  __syncthreads();
  {
    long long P = base_s, R = base_t & 0xffffffffll, D = base_t >> 32;
#pragma unroll
    for (int i = 0; i < kUnitsPerThread; ++i) {
      if (uS[i] > 0) {
        int jlo, jhi;
        chunks_here(P, uS[i], jlo, jhi);
        if (jlo < jhi) {
          const int idx = (int)(R - s_first);
          if (idx >= 0 && idx < kMaxPieces) {
            s_piece[idx] = make_int4(u0 + i, (int)P, uS[i], uL[i]);
            // contributors: the distinct CTAs holding a chunk start of the unit (a share
            // shorter than a chunk can hold none)
            const int nc = (uS[i] + kChunk - 1) / kChunk;
            int ncon = 0, prev = -1;
            for (int jj = 0; jj < nc; ++jj) {
              const int k = cta_of((uint32_t)P + (uint32_t)(jj * kChunk), S_tot, C);
              if (k != prev) {
                ++ncon;
                prev = k;
              }
            }
            s_pcon[idx] = make_int4(cta_of((uint32_t)P, S_tot, C), prev, ncon, 0);
            atomicMax(&s_np, idx + 1);
          } else {
            raise_error(err0, FOT_EUNSUPPORTED);
          }
        }
      }
      if (uD[i]) {
        // the declined unit's items q = D * IPU + it are dealt round-robin over the CTAs
        constexpr int IPU = kRowItems * (TN / kBT);
        const long long q0 = D * IPU;
        for (int it = (int)((cta - q0 % C + C) % C); it < IPU; it += C) {
          const int idx = atomicAdd(&s_nd, 1);
          if (idx < kMaxDecl)
            s_decl[idx] = ((u0 + i) << 8) | it;
          else
            raise_error(err0, FOT_EUNSUPPORTED);
        }
      }
      P += uS[i];
      R += uS[i] > 0 ? 1 : 0;
      D += uD[i];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const int np = s_np, nd = s_nd;

  // piece i: unit, its chunks [jlo, jhi) here (stages [b, e)), whether it is split, and the
  // first contributor (whose index names the split unit's slots)
  // (the problem's fields are copied into the piece once: read through a pointer into the
  // kernel's parameters they would be reloaded after every barrier operation)
  struct Piece {
    const BandArgs* a;
    int lu, r0, tile, k0, kc, lo, S, nc, jlo, jhi, b, e, P, ca, ncon;
    bool split;
    int* err;
    int len, n_rows;
    float c, sc, eps;
  };
  auto piece = [&](int i) {
    const int4 q = s_piece[i];
    const int4 con = s_pcon[i];
    Piece p;
    p.a = &tab.p[find_prob<MAXP, 3>(tab, q.x)];
    p.lu = q.x - p.a->cta_base;
    p.r0 = (p.lu / p.a->n_tiles) * kTM;
    p.tile = p.lu % p.a->n_tiles;
    p.k0 = p.tile * TN;
    p.kc = p.k0 + TN / 2;
    p.lo = q.w;
    p.S = q.z;
    p.P = q.y;
    p.nc = (q.z + kChunk - 1) / kChunk;
    chunks_here(q.y, q.z, p.jlo, p.jhi);
    p.b = p.jlo * kChunk;
    p.e = min(p.jhi * kChunk, p.S);
    p.ca = con.x;
    p.ncon = con.z;
    p.split = con.x != con.y;
    p.err = p.a->err;
    p.len = p.a->len;
    p.n_rows = p.a->n_rows;
    p.c = p.a->c;
    p.sc = p.a->x_scale;
    p.eps = p.a->eps;
    return p;
  };

  unsigned char* const xring = smem;
  unsigned char* const xalpha = smem + Sh::kXAlphaOff;
  unsigned char* const epiring = smem + Sh::kEpiOff;
  unsigned char* const opring = smem + Sh::kOpOff;
  int issued_x = 0, issued_o = 0, issued_ea = 0, issued_mma = 0;   // for the drain after an abort

  if (warp == kTmaWarp) {
    // ---------------------------------------------------------------- TMA issue (one lane)
    if (lane == 0) {
      int xi = 0, oi = 0;
      bool ok = true;
      for (int i = 0; i < np && ok; ++i) {
        const Piece p = piece(i);
        const BandArgs& a = *p.a;
        const float* alpha_src = a.plan + (size_t)p.tile * a.plan_stride + p.r0;
        const unsigned char* btab = a.btab + (size_t)(a.s_max - p.S) * Sh::kBBytes;
        const void* xmap = a.xmap;
        const void* lmap = a.lmap;
        for (int ch = p.b; ch < p.e && ok; ++ch) {
          const int s = xi % kXStages;
          if (xi >= kXStages && !(ok = mbar_wait(smem_u32(&xempty[s]), ((xi / kXStages) - 1) & 1, spin, p.err, abort_flag))) break;
          const bool first = ch == p.b;
          mbar_expect_tx(smem_u32(&xfull[s]), kXBytes + (first ? kAlphaBytes : 0));
          tma_load_2d(smem_u32(xring + s * kXBytes), xmap, p.lo + ch * kKC, p.r0, smem_u32(&xfull[s]));
          if (first) bulk_load(smem_u32(xalpha + s * kAlphaBytes), alpha_src, kAlphaBytes, smem_u32(&xfull[s]));
          ++xi;
          issued_x = xi;
          if (first) {
            // the epilogue's slot: alpha, and log a of the unit's outputs (rows r0.., outputs
            // k0..; outside the image read as zeros, which the epilogue does not use)
            const int eb = i % kEpiBufs;
            if (i >= kEpiBufs && !(ok = mbar_wait(smem_u32(&eaempty[eb]), ((i / kEpiBufs) - 1) & 1, spin, p.err, abort_flag))) break;
            unsigned char* const slot = epiring + eb * Sh::kEpiSlot;
            const bool lm = MODE == 1 && a.lm_tma;
            mbar_expect_tx(smem_u32(&eafull[eb]), kAlphaBytes + (lm ? Sh::kLmBytes : 0));
            bulk_load(smem_u32(slot), alpha_src, kAlphaBytes, smem_u32(&eafull[eb]));
            if (lm) tma_load_2d(smem_u32(slot + kAlphaBytes), lmap, p.r0, p.k0, smem_u32(&eafull[eb]));
            issued_ea = i + 1;
          }
          const int so = oi % Sh::kOpStages;
          if (oi >= Sh::kOpStages && !(ok = mbar_wait(smem_u32(&opempty[so]), ((oi / Sh::kOpStages) - 1) & 1, spin, p.err, abort_flag))) break;
          mbar_expect_tx(smem_u32(&bfull[so]), Sh::kBBytes);
          bulk_load(smem_u32(opring + so * Sh::kOpBytes + 2 * kABytes), btab + (size_t)(2 * ch) * Sh::kBBytes,
                    Sh::kBBytes, smem_u32(&bfull[so]));
          ++oi;
          issued_o = oi;
        }
      }
    }
    __syncwarp();                                         // reconverge before the CTA barriers
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------------- MMA issue (one lane)
    if (lane == 0) {
      const uint32_t idesc1 = instr_desc(kTM, single ? TN : 2 * TN), idesc2 = instr_desc(kTM, TN);
      int oi = 0, ai = 0;
      bool ok = true;
      for (int i = 0; i < np && ok; ++i) {
        const Piece p = piece(i);
        for (int j = p.jlo; j < p.jhi && ok; ++j) {
          // chunk j: a fresh accumulator over its stages
          const int ab = ai % kAccBufs;
          if (ai >= kAccBufs && !(ok = mbar_wait(smem_u32(&accempty[ab]), ((ai / kAccBufs) - 1) & 1, spin, p.err, abort_flag))) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dcol = tmem + (uint32_t)(ab * 2 * TN);
          const int s0 = j * kChunk, s1 = min(s0 + kChunk, p.S);
          for (int ch = s0; ch < s1; ++ch) {
            const int so = oi % Sh::kOpStages;
            const uint32_t par = (oi / Sh::kOpStages) & 1;
            if (!(ok = mbar_wait(smem_u32(&opfull[so]), par, spin, p.err, abort_flag))) break;
            if (!(ok = mbar_wait(smem_u32(&bfull[so]), par, spin, p.err, abort_flag))) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = smem_u32(opring + so * Sh::kOpBytes);
            const uint32_t sAhi = st, sAlo = st + kABytes, sB = st + 2 * kABytes;
#pragma unroll
            for (int ks = 0; ks < kKC / 16; ++ks) {
              const uint64_t dAh = smem_desc(sAhi + ks * 256, 128, kGroupBytes);
              const uint64_t dAl = smem_desc(sAlo + ks * 256, 128, kGroupBytes);
              const uint64_t dB = smem_desc(sB + ks * 256, 128, kGroupBytes);
              mma_bf16(dcol, dAh, dB, idesc1, (ch > s0 || ks > 0) ? 1u : 0u);   // hi x [B_hi | B_lo]
              if (!single) mma_bf16(dcol, dAl, dB, idesc2, 1u);                  // lo x B_hi
            }
            mma_commit(smem_u32(&opempty[so]));
            issued_mma = 1;
            ++oi;
          }
          if (!ok) break;
          mma_commit(smem_u32(&accfull[ab]));
          ++ai;
        }
      }
    }
    __syncwarp();
  } else if (warp < kProdWarps) {
    // ---------------------------------------------------------------- producers
    // thread (row ar, half ah) makes window positions 16 ah .. 16 ah + 15 of the stage, as two
    // groups of 8 (one core-matrix row of A each)
    const int ar = tid & (kTM - 1), ah = tid >> 7;
    // 128-byte swizzle of the x tile: 16-byte chunk j of row r sits at chunk j ^ (r % 8)
    const uint32_t xrow = (uint32_t)ar * 128u;
    uint32_t xc[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) xc[t] = xrow + (uint32_t)(((4 * ah + t) ^ (ar & 7)) * 16);
    const uint32_t aoff = (uint32_t)((ar >> 3) * kGroupBytes + 2 * ah * 128 + (ar & 7) * 16);
    int xi = 0, oi = 0;
    bool ok = true;
    for (int i = 0; i < np && ok; ++i) {
      const Piece p = piece(i);
      const float c = p.c, sc = p.sc;
      const int len = p.len;
      const bool rowok = p.r0 + ar < p.n_rows;
      float alpha = -INFINITY;
      for (int ch = p.b; ch < p.e; ++ch) {
        const int s = xi % kXStages;
        if (!(ok = mbar_wait(smem_u32(&xfull[s]), (xi / kXStages) & 1, spin, p.err, abort_flag))) break;
        if (ch == p.b && rowok) alpha = reinterpret_cast<const float*>(xalpha + s * kAlphaBytes)[ar];
        float4 xv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) xv[t] = *reinterpret_cast<const float4*>(xring + s * kXBytes + xc[t]);
        const int so = oi % Sh::kOpStages;
        if (oi >= Sh::kOpStages && !(ok = mbar_wait(smem_u32(&opempty[so]), ((oi / Sh::kOpStages) - 1) & 1, spin, p.err, abort_flag))) break;
        unsigned char* const stp = opring + so * Sh::kOpBytes;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          float v[8];
          const int m0 = p.lo + ch * kKC + ah * 16 + g * 8;   // absolute position of v[0]
          if (alpha == -INFINITY) {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = 0.f;
          } else {
            // exponent e_j = x_j sc - (kc - m0 - j)^2 c - alpha = x_j sc + P + Q j - c j^2
            const float dbase = (float)(p.kc - m0);
            const float P = fmaf(-dbase * dbase, c, -alpha), Q = 2.f * dbase * c;
            const float4 a0 = xv[2 * g], a1 = xv[2 * g + 1];
            const float xs[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float K = fmaf(Q, (float)j, fmaf(-(float)(j * j), c, P));
              v[j] = (m0 + j < len) ? ex2(fmaf(xs[j], sc, K)) : 0.f;   // x = -inf -> 0
            }
          }
          if (single)
            store_hi8(v, stp + aoff + g * 128);
          else
            store_split8(v, stp + aoff + g * 128, stp + kABytes + aoff + g * 128);
        }
        // one proxy fence orders this thread's generic accesses of the stage against the async
        // proxy: its A stores before the MMA reads them, and its reads of the x slot (and of
        // alpha) before the next tensor copy into that slot overwrites them (without the
        // fence the copy was seen to land before the reads)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&xempty[s]));
        ++xi;
        mbar_arrive(smem_u32(&opfull[so]));
        ++oi;
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    // two warps per tensor-memory lane quarter (warp % 4), each taking half of the columns
    constexpr int HN = TN / 2;                            // columns of this thread
    // columns per step: the column loops are not unrolled, so that the epilogue's code stays
    // small (it runs once per unit, between long stretches of producer code, and a large
    // unrolled body was fetched cold every time)
    constexpr int CH = 4;
    const int q4 = warp & 3;
    const int hcol = ((warp - kEpiWarp0) >> 2) * HN;      // first column of this thread's half
    const int rl = 32 * q4 + lane;                        // accumulator row
    const bool lead = rl == 0 && hcol == 0;               // one thread per CTA for the counters
    const uint32_t tlane = tmem + ((uint32_t)(32 * q4) << 16);
    const uint32_t tfold = tlane + (uint32_t)(4 * TN);    // running sum of the unit's chunks
    int ai = 0;
    bool ok = true;
    for (int i = 0; i < np && ok; ++i) {
      const Piece p = piece(i);
      const BandArgs& a = *p.a;
      const int n_rows = p.n_rows;
      const int row = p.r0 + rl;
      const bool rowok = row < n_rows;
      const int k1 = min(p.k0 + TN, p.len) - 1;
      float* const y = a.y;
      float* const logsum = a.logsum;
      int* const err = p.err;
      const float peps = p.eps;
      // this piece's slot: alpha, then (potential update) log a as [TN][128]
      const int eb = i % kEpiBufs;
      const unsigned char* const eslot = epiring + eb * Sh::kEpiSlot;
      const float* const s_lm = reinterpret_cast<const float*>(eslot + kAlphaBytes);
      const bool lm_tma = a.lm_tma;      // else (rows not 16-byte aligned) log a from global
      const float* const lmarg = a.lmarg;
      ok = mbar_wait(smem_u32(&eafull[eb]), (i / kEpiBufs) & 1, spin, err, abort_flag);
      float alpha = -INFINITY;
      if (ok && rowok) alpha = reinterpret_cast<const float*>(eslot)[rl];
      if (!epi_all(ok)) break;                            // the same for all epilogue threads
      if (lead) atomicAdd(a.tc_terms, (unsigned long long)(p.e - p.b) * kKC * TN * kTM);
      const float c = p.c;
      const float mref = (float)p.lo + 0.5f * (float)(p.S * kKC);
      // the tilt of output column n: alpha + 2 (n - TN/2) (mref - kc) c
      const float tilt0 = fmaf(2.f * (float)(-TN / 2) * (mref - (float)p.kc), c, alpha);
      const float tstep = 2.f * (mref - (float)p.kc) * c;
      // outputs (o = k0 + c0 + u, r = row) from CH sums: all log2 first, then (potential
      // update) all loads of log a, then the stores; one error check per call
      const int nvalid = k1 - p.k0 + 1;                   // outputs of this tile inside the image
      auto emit = [&](int c0, const float* cv) {
        if (!rowok) return;
        float out[CH];
        bool bad = false;
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const bool okv = cv[u] > 0.f && cv[u] <= 3.4e38f;
          out[u] = okv ? __fadd_rn(fmaf((float)(c0 + u), tstep, tilt0), lg2(cv[u])) : -INFINITY;
          bad |= alpha != -INFINITY && !okv;
        }
        if (alpha == -INFINITY) {
#pragma unroll
          for (int u = 0; u < CH; ++u) out[u] = -INFINITY;
        }
        float* const yp = y + (size_t)(p.k0 + c0) * n_rows + row;
        if (MODE == 0) {
#pragma unroll
          for (int u = 0; u < CH; ++u)
            if (c0 + u < nvalid) yp[(size_t)u * n_rows] = out[u];
        } else {
          float lm[CH];
          if (lm_tma) {
#pragma unroll
            for (int u = 0; u < CH; ++u) lm[u] = s_lm[(c0 + u) * kTM + rl];
          } else {
#pragma unroll
            for (int u = 0; u < CH; ++u) lm[u] = c0 + u < nvalid ? __ldg(lmarg + (size_t)(p.k0 + c0 + u) * n_rows + row) : 0.f;
          }
          float pot[CH], sv[CH];
#pragma unroll
          for (int u = 0; u < CH; ++u) {
            sv[u] = __fmul_rn(out[u], kLn2);
            pot[u] = lm[u] == -INFINITY ? -INFINITY : __fmul_rn(peps, __fsub_rn(lm[u], sv[u]));
            bad |= lm[u] != -INFINITY && !isfinite(pot[u]) && c0 + u < nvalid;
          }
#pragma unroll
          for (int u = 0; u < CH; ++u)
            if (c0 + u < nvalid) yp[(size_t)u * n_rows] = pot[u];
          if (logsum) {
            float* const lp = logsum + (size_t)(p.k0 + c0) * n_rows + row;
#pragma unroll
            for (int u = 0; u < CH; ++u)
              if (c0 + u < nvalid) lp[(size_t)u * n_rows] = sv[u];
          }
        }
        if (bad) raise_error(err, FOT_ENONFINITE);
      };
      for (int j = p.jlo; j < p.jhi; ++j) {
        const int ab = ai % kAccBufs;
        ok = mbar_wait(smem_u32(&accfull[ab]), (ai / kAccBufs) & 1, spin, err, abort_flag);
        if (!epi_all(ok)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t tacc = tlane + (uint32_t)(ab * 2 * TN);
        const bool last = j == p.nc - 1;
        // chunk sum = D[0:TN) + D[TN:2TN) (the three split products), CH columns at a time; a
        // split unit's chunk sums go to its slots, the others are added to the running sum
        float* slot = tab.slots + (((size_t)p.ca * tab.slot_chunks + j) * kTM + rl) * TN;
#pragma unroll 1
        for (int c0 = hcol; c0 < hcol + HN; c0 += CH) {
          uint32_t d1[CH], d2[CH];
          tmem_ld<CH>(tacc + (uint32_t)c0, d1);
          if (!single) tmem_ld<CH>(tacc + (uint32_t)(TN + c0), d2);
          tmem_wait_ld<CH>(d1, d2);
          float cv[CH];
#pragma unroll
          for (int u = 0; u < CH; ++u) cv[u] = single ? __uint_as_float(d1[u]) : __uint_as_float(d1[u]) + __uint_as_float(d2[u]);
          if (p.split) {
#pragma unroll
            for (int u = 0; u < CH; u += 4)
              *reinterpret_cast<float4*>(slot + c0 + u) = make_float4(cv[u], cv[u + 1], cv[u + 2], cv[u + 3]);
          } else {
            if (j > 0) {                                  // running sum of chunks 0 .. j-1
              uint32_t f[CH];
              tmem_ld<CH>(tfold + (uint32_t)c0, f);
              tmem_wait_ld<CH>(f);
#pragma unroll
              for (int u = 0; u < CH; ++u) cv[u] = __uint_as_float(f[u]) + cv[u];
            }
            if (last) {
              emit(c0, cv);
            } else {
              uint32_t f[CH];
#pragma unroll
              for (int u = 0; u < CH; ++u) f[u] = __float_as_uint(cv[u]);
              tmem_st<CH>(tfold + (uint32_t)c0, f);
            }
          }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(smem_u32(&accempty[ab]));
        ++ai;
      }
      if (!ok) break;
      if (p.split) {
        // the last contributor adds all chunk sums of the unit in chunk order (the same sums,
        // in the same order, as an unsplit unit) and writes the outputs.  (The grid
        // synchronisation pattern: the epilogue's writes are gathered by the barrier, one
        // thread publishes them with a device-scope fence before the count and fences again
        // after reading the final count, before the barrier that releases the readers.)
        asm volatile("bar.sync 1, %0;" :: "r"(kEpi) : "memory");
        if (lead) {
          __threadfence();
          s_last = atomicAdd(&a.ucnt[p.lu], 1) == p.ncon - 1;
          __threadfence();
        }
        asm volatile("bar.sync 1, %0;" :: "r"(kEpi) : "memory");
        if (s_last) {
#pragma unroll 1
          for (int c0 = hcol; c0 < hcol + HN; c0 += CH) {
            float cv[CH];
            const float* sl0 = tab.slots + (((size_t)p.ca * tab.slot_chunks) * kTM + rl) * TN + c0;
            const size_t jstride = (size_t)kTM * TN;
#pragma unroll 1
            for (int j0 = 0; j0 < p.nc; j0 += 2) {
              // two chunks' loads in flight, then added in chunk order
              float4 t4[2][CH / 4];
#pragma unroll
              for (int jj = 0; jj < 2; ++jj)
#pragma unroll
                for (int u = 0; u < CH; u += 4)
                  t4[jj][u / 4] = (j0 + jj < p.nc) ? __ldcg(reinterpret_cast<const float4*>(sl0 + (j0 + jj) * jstride + u))
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
              for (int jj = 0; jj < 2; ++jj) {
                if (j0 + jj >= p.nc) break;
#pragma unroll
                for (int u = 0; u < CH; u += 4) {
                  const float4 q = t4[jj][u / 4];
                  if (j0 + jj == 0) {
                    cv[u] = q.x;
                    cv[u + 1] = q.y;
                    cv[u + 2] = q.z;
                    cv[u + 3] = q.w;
                  } else {
                    cv[u] += q.x;
                    cv[u + 1] += q.y;
                    cv[u + 2] += q.z;
                    cv[u + 3] += q.w;
                  }
                }
              }
            }
            emit(c0, cv);
          }
          if (lead) a.ucnt[p.lu] = 0;
        }
      }
      // the slot is free once every epilogue thread is done with this piece's alpha and log a
      // (reads ordered before the next copies into the slot by a proxy fence)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&eaempty[eb]));
    }
  }

  // ---- units outside the tensor path: CUDA-core window sums by the producer warps ------------
  // The x ring serves as their scratch once every producer warp has read its last x tile (a
  // barrier of the producer warps: a warp that finishes early must not overwrite a tile that
  // another warp still reads).
  if (warp < kProdWarps) asm volatile("bar.sync 3, %0;" :: "r"(kProd) : "memory");
  if (warp < kProdWarps && !*abort_flag) {
    float* sAw = reinterpret_cast<float*>(xring) + warp * 2 * kSA;
    for (int d = warp; d < min(nd, kMaxDecl); d += kProdWarps) {
      const int u = s_decl[d] >> 8, it = s_decl[d] & 255;
      const BandArgs& a = tab.p[find_prob<MAXP, 3>(tab, u)];
      const int lu = u - a.cta_base;
      const int tile = lu % a.n_tiles;
      tc_cuda_core_item<MODE, TN>(a, (lu / a.n_tiles) * kTM, tile, tile * TN, it, sAw);
    }
  }

  // ---- tear-down --------------------------------------------------------------------------
  __syncthreads();
  if (*abort_flag) {
    // wait (bounded, with the full limit) for the copies and MMAs this CTA started
    if (warp == kTmaWarp && lane == 0) {
      for (int s = 0; s < kXStages && s < issued_x; ++s)
        mbar_drain(smem_u32(&xfull[s]), ((issued_x - 1 - s) / kXStages) & 1);
      for (int s = 0; s < Sh::kOpStages && s < issued_o; ++s)
        mbar_drain(smem_u32(&bfull[s]), ((issued_o - 1 - s) / Sh::kOpStages) & 1);
      for (int s = 0; s < kEpiBufs && s < issued_ea; ++s)
        mbar_drain(smem_u32(&eafull[s]), ((issued_ea - 1 - s) / kEpiBufs) & 1);
    }
    if (warp == kMmaWarp && lane == 0 && issued_mma) {
      mma_commit(smem_u32(&drain));
      mbar_drain(smem_u32(&drain), 0);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(Sh::kTmemCols) : "memory");
}

// B operand table of one pass: for every half-shift s = e - s_max (e in [0, 2 s_max)) the
// block of 2 TN rows x 32 positions in the canonical K-major core-matrix layout, rows n < TN
// B_hi and rows TN + n B_lo of B(u, kap) = 2^(2 kap (16 s + u) c - kap^2 c), kap = n - TN/2
// (a stage at window offset 32 ch in a window of nW stages reads block e = 2 ch - nW + s_max:
// m' - W/2 = 16 (2 ch - nW) + u).  Exponents are clamped to [-126, 126]: blocks whose values
// would leave that range only serve units outside the tilt bound, which never read them.
template <int TN>
__global__ void btab_kernel(unsigned char* tab, int s_max, float c) {
  constexpr int kBBytes = 2 * TN * kKC * 2;
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;   // (e, n, kg)
  const int kg = gi & 3, n = (gi >> 2) % TN, e = (gi >> 2) / TN;
  if (e >= 2 * s_max) return;
  const float kap = (float)(n - TN / 2);
  const float sh = 16.f * (float)(e - s_max) + (float)(8 * kg);
  float v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const float ex = fmaf(2.f * kap * (sh + (float)u), c, -kap * kap * c);
    v[u] = ex2(fminf(fmaxf(ex, -126.f), 126.f));
  }
  unsigned char* blk = tab + (size_t)e * kBBytes;
  const int rh = n, rl = TN + n;
  store_split8(v, blk + (rh >> 3) * kGroupBytes + kg * 128 + (rh & 7) * 16,
               blk + (rl >> 3) * kGroupBytes + kg * 128 + (rl & 7) * 16);
}

// ---- host side ---------------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// the x tensor map of a pass: [n_rows][len] FP32, boxes of 32 positions x 128 rows, 128-byte
// swizzle; positions and rows outside the image read as zeros (the kernel masks them)
bool encode_xmap(BandArgs& a) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  if ((a.len & 3) != 0 || (reinterpret_cast<uintptr_t>(a.x) & 15u) != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)a.len, (cuuint64_t)a.n_rows};
  cuuint64_t strides[1] = {(cuuint64_t)a.len * 4};
  cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)kTM};
  cuuint32_t estr[2] = {1, 1};
  static_assert(sizeof(CUtensorMap) == sizeof(a.xmap), "tensor map size");
  return fn(reinterpret_cast<CUtensorMap*>(a.xmap), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(a.x), dims,
            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the log-marginal tensor map of a potential-update pass: lmarg as [len][n_rows] FP32 (the
// layout of y), boxes of 128 rows x tn outputs, no swizzle; outside the image reads as zeros
bool encode_lmap(BandArgs& a, int tn) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  if ((a.n_rows & 3) != 0 || (reinterpret_cast<uintptr_t>(a.lmarg) & 15u) != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)a.n_rows, (cuuint64_t)a.len};
  cuuint64_t strides[1] = {(cuuint64_t)a.n_rows * 4};
  cuuint32_t box[2] = {(cuuint32_t)kTM, (cuuint32_t)tn};
  cuuint32_t estr[2] = {1, 1};
  static_assert(sizeof(CUtensorMap) == sizeof(a.lmap), "tensor map size");
  return fn(reinterpret_cast<CUtensorMap*>(a.lmap), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(a.lmarg),
            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcState {
  unsigned long long* tc_terms = nullptr;   // window terms computed on the tensor cores
  int* ext = nullptr;          // [2 parities][lo, hi][max units]
  int* ucnt = nullptr;         // [max units]
  unsigned char* btab = nullptr;
  float* slots = nullptr;      // chunk sums of split units: [sms][slot_chunks][128][64]
  int max_units = 0, s_max = 0, slot_chunks = 0, sms = 0, parity = 0, spin = kSpinDefault;
  float btab_c = 0.f;          // parameters of the B table as last written on the stream
  int btab_tn = 0;
};

size_t btab_bytes(int s_max) { return (size_t)2 * s_max * TcShape<64>::kBBytes; }

template <int TN, int MAXP>
void set_smem_attr(bool& ok) {
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<0, TN, MAXP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  TcShape<TN>::kSmemBytes) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(tc_pass_kernel<1, TN, MAXP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  TcShape<TN>::kSmemBytes) == cudaSuccess;
}

}  // namespace

bool tc_supported(int rows, int cols) { return rows >= 1 && cols >= 1; }

int tc_create(fot_ctx* c) {
  TcState* t = new (std::nothrow) TcState();
  if (!t) return 1;
  const int rows = c->rows, cols = c->cols;
  t->max_units = std::max(((rows + 127) / 128) * ((cols + 15) / 16), ((cols + 127) / 128) * ((rows + 15) / 16));
  t->s_max = (std::max(rows, cols) + kKC - 1) / kKC;
  t->slot_chunks = (t->s_max + kChunk - 1) / kChunk;
  if (cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || t->sms < 1) t->sms = 1;
  if (const char* e = getenv("FOT_TEST_WAIT_LIMIT")) {   // test-only: a short wait limit
    const int v = atoi(e);
    if (v > 0) t->spin = v;
  }
  bool ok = cudaMalloc((void**)&t->tc_terms, sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&t->ext, (size_t)4 * t->max_units * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&t->ucnt, (size_t)t->max_units * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&t->btab, btab_bytes(t->s_max)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&t->slots, (size_t)t->sms * t->slot_chunks * kTM * 64 * sizeof(float)) == cudaSuccess;
  if (ok) {
    // reset state of the unit extents (lo = 0x7F7F7F7F, hi = 0) and the split counters
    for (int p = 0; p < 2; ++p) {
      ok = ok && cudaMemsetAsync(t->ext + (size_t)(2 * p) * t->max_units, 0x7F, (size_t)t->max_units * sizeof(int), c->stream) == cudaSuccess;
      ok = ok && cudaMemsetAsync(t->ext + (size_t)(2 * p + 1) * t->max_units, 0, (size_t)t->max_units * sizeof(int), c->stream) == cudaSuccess;
    }
    ok = ok && cudaMemsetAsync(t->ucnt, 0, (size_t)t->max_units * sizeof(int), c->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(t->tc_terms, 0, sizeof(unsigned long long), c->stream) == cudaSuccess;
  }
  // dynamic shared memory above 48 KB, for every instance (per device; before any capture)
  set_smem_attr<16, 1>(ok);
  set_smem_attr<32, 1>(ok);
  set_smem_attr<64, 1>(ok);
  set_smem_attr<16, kMaxBatch>(ok);
  set_smem_attr<32, kMaxBatch>(ok);
  set_smem_attr<64, kMaxBatch>(ok);
  c->tc = t;
  if (!ok) return 1;   // fot_create destroys the context (tc_destroy frees what was made)
  return 0;
}

void tc_destroy(fot_ctx* c) {
  TcState* t = (TcState*)c->tc;
  if (!t) return;
  if (t->tc_terms) cudaFree(t->tc_terms);
  if (t->ext) cudaFree(t->ext);
  if (t->ucnt) cudaFree(t->ucnt);
  if (t->btab) cudaFree(t->btab);
  if (t->slots) cudaFree(t->slots);
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

unsigned long long* tc_terms_ptr(fot_ctx* c) { return c->tc ? ((TcState*)c->tc)->tc_terms : nullptr; }

// Start of a sequence of passes of one API call (a solve, a graph capture, a standalone
// half-step): the B table is rewritten at its first tensor pass, and the split counters start
// from zero (a pass that timed out can leave them set).
void tc_begin(fot_ctx* c) {
  TcState* t = (TcState*)c->tc;
  if (!t) return;
  t->btab_tn = 0;
  cudaMemsetAsync(t->ucnt, 0, (size_t)t->max_units * sizeof(int), c->stream);
}

// The tensor-core fields of one pass's arguments: unit extents of the current parity (and the
// other parity, which this pass's plan kernel resets), split counters, B table.  Toggles the
// parity: call once per pass.
void tc_bind(fot_ctx* c, BandArgs& a) {
  TcState* t = (TcState*)c->tc;
  const int p = t->parity;
  t->parity ^= 1;
  a.ext_lo = t->ext + (size_t)(2 * p) * t->max_units;
  a.ext_hi = t->ext + (size_t)(2 * p + 1) * t->max_units;
  a.ext_lo_next = t->ext + (size_t)(2 * (p ^ 1)) * t->max_units;
  a.ext_hi_next = t->ext + (size_t)(2 * (p ^ 1) + 1) * t->max_units;
  a.ext_units = t->max_units;
  a.ucnt = t->ucnt;
  a.btab = t->btab;
  a.s_max = t->s_max;
  a.tc_terms = t->tc_terms;
}

// whether the B table of ctx c needs writing for (kernel constant cc, tile width tw); records
// the new parameters
bool tc_btab_stale(fot_ctx* c, float cc, int tw) {
  TcState* t = (TcState*)c->tc;
  if (t->btab_tn == tw && t->btab_c == cc) return false;
  t->btab_tn = tw;
  t->btab_c = cc;
  return true;
}

float* tc_slots(fot_ctx* c) { return ((TcState*)c->tc)->slots; }
int tc_sms(fot_ctx* c) { return ((TcState*)c->tc)->sms; }
int tc_spin(fot_ctx* c) { return ((TcState*)c->tc)->spin; }

// Tile width of a tensor-core pass for a problem with kernel constant c: the widest TN in
// {64, 32} whose tile is expected to meet the tilt bound |kap| W c <= kTiltMaxTC with room to
// spare: W is taken as twice the window of a smooth potential (the tile plus sqrt(kCut / c) on
// each side, where the Gaussian kernel alone has fallen by 2^-kCut), rounded up to a multiple
// of 64 positions, since the hull of a tile's windows grows where the transport map jumps across
// zero-mass gaps; else 16 when a 16-wide tile meets the bound with a window of kRouteKC
// positions; else 0: the CUDA-core kernel.  A unit outside the bound costs CUDA-core window sums.
int tc_width_for(float c) {
  for (int tn = 64; tn >= 32; tn /= 2) {
    const float w = (float)tn + 2.f * sqrtf(kCut / c);
    const float wr = 2.f * ceilf(w / (float)kRouteKC) * (float)kRouteKC;
    if ((float)(tn / 2) * wr * c <= kTiltMaxTC && (float)(tn / 2) * (float)(tn / 2) * c <= 32.f) return tn;
  }
  if ((float)(kBT / 2) * (float)kRouteKC * c <= kTiltMaxTC) return 16;
  return 0;
}

template <int TN, int MAXP>
static void launch_btab(cudaStream_t s, const BandArgs& a) {
  const int threads = 2 * a.s_max * TN * 4;
  ktimer_begin(s, kKPlan);                 // timed with the window plans (set-up of a pass)
  btab_kernel<TN><<<(threads + 255) / 256, 256, 0, s>>>(const_cast<unsigned char*>(a.btab), a.s_max, a.c);
  ktimer_end(s);
}

// tw: the tile width every problem of the table uses (tc_width_for of its c); ctx[q]: the
// context of problem q (its B table is rewritten first when stale); ctx[0] also lends the
// split slots, the SM count and the wait limit.  Returns the number of kernels launched.
template <int MODE, int MAXP>
int tc_pass(cudaStream_t s, BandTable<MAXP>& t, int tw, fot_ctx* const* ctx) {
  // the problems the tensor kernel can take (rows 16-byte aligned for the tensor copies) and
  // the others, each in a table of its own
  BandTable<MAXP>* tt = new BandTable<MAXP>();
  BandTable<MAXP>* tf = new BandTable<MAXP>();
  fot_ctx* tctx[MAXP];
  for (int q = 0; q < t.n; ++q) {
    BandArgs a = t.p[q];
    a.tile_w = tw == 0 ? kBT : tw;
    if (tw != 0 && encode_xmap(a)) {
      a.lm_tma = MODE == 1 && encode_lmap(a, tw);
      tctx[tt->n] = ctx[q];
      tt->p[tt->n++] = a;
    } else {
      a.ext_lo = a.ext_hi = nullptr;   // the plan kernel still resets the next pass's extents
      a.tile_w = kBT;
      tf->p[tf->n++] = a;
    }
  }
  int k = 0;
  if (tt->n > 0) {
    band_table_finish(*tt);
    // the context with the most slot chunks lends its slots (every problem's chunks fit)
    TcState* ts = (TcState*)tctx[0]->tc;
    for (int q = 1; q < tt->n; ++q) {
      TcState* o = (TcState*)tctx[q]->tc;
      if (o->slot_chunks > ts->slot_chunks) ts = o;
    }
    const int sms = ts->sms;
    int smax_all = 1;
    for (int q = 0; q < tt->n; ++q) smax_all = std::max(smax_all, tt->p[q].s_max);
    const long long items_max = (long long)tt->ctas * (kTM / (2 * kBR)) * (tw / kBT);
    if (tt->ctas > kThreads * kUnitsPerThread || tt->ctas > (kMaxPieces / 2) * sms ||
        items_max > (long long)kMaxDecl * std::min(sms, tt->ctas) ||
        (uint64_t)tt->ctas * (uint64_t)smax_all * (uint64_t)sms >= (1ull << 32)) {
      // more units than the kernel's set-up holds (or stage positions beyond its 32-bit
      // partition arithmetic): the CUDA-core sums for all of them
      for (int q = 0; q < tt->n; ++q) {
        BandArgs a = tt->p[q];
        a.ext_lo = a.ext_hi = nullptr;
        a.tile_w = kBT;
        tf->p[tf->n++] = a;
      }
      tt->n = 0;
    } else {
      for (int q = 0; q < tt->n; ++q) {
        if (!tc_btab_stale(tctx[q], tt->p[q].c, tw)) continue;
        if (tw == 64) launch_btab<64, MAXP>(s, tt->p[q]);
        else if (tw == 32) launch_btab<32, MAXP>(s, tt->p[q]);
        else launch_btab<16, MAXP>(s, tt->p[q]);
        ++k;
      }
      band_prepare(s, *tt);
      tt->slots = ts->slots;
      tt->slot_chunks = ts->slot_chunks;
      tt->spin_limit = ts->spin;
      tt->tc_single = tctx[0]->precision == FOT_BF16 ? 1 : 0;
      const int grid = std::max(1, std::min(sms, tt->ctas));
      ktimer_begin(s, kKTensor);
      if (tw == 64)
        tc_pass_kernel<MODE, 64, MAXP><<<grid, kThreads, TcShape<64>::kSmemBytes, s>>>(*tt);
      else if (tw == 32)
        tc_pass_kernel<MODE, 32, MAXP><<<grid, kThreads, TcShape<32>::kSmemBytes, s>>>(*tt);
      else
        tc_pass_kernel<MODE, 16, MAXP><<<grid, kThreads, TcShape<16>::kSmemBytes, s>>>(*tt);
      ktimer_end(s);
      k += 2;
    }
  }
  if (tf->n > 0) {
    band_table_finish(*tf);
    band_prepare(s, *tf);
    band_simt<MODE>(s, *tf);
    k += 2;
  }
  delete tt;
  delete tf;
  return k;
}

template int tc_pass<0, 1>(cudaStream_t, BandTable<1>&, int, fot_ctx* const*);
template int tc_pass<1, 1>(cudaStream_t, BandTable<1>&, int, fot_ctx* const*);
template int tc_pass<0, kMaxBatch>(cudaStream_t, BandTable<kMaxBatch>&, int, fot_ctx* const*);
template int tc_pass<1, kMaxBatch>(cudaStream_t, BandTable<kMaxBatch>&, int, fot_ctx* const*);

BandArgs band_args(fot_ctx* c, const float* x, int n_rows, int len, double eps, float x_scale);

// One half-step with the tensor-core banded passes.
void half_step_tc(fot_ctx* c, const float* pot_in, const float* lmarg, double eps, float* pot_out,
                  float* logsum) {
  BandTable<1> t{};
  t.n = 1;
  t.p[0] = band_args(c, pot_in, c->rows, c->cols, eps, (float)(1.4426950408889634 / eps));
  t.p[0].y = c->R;
  tc_bind(c, t.p[0]);
  const int tw = tc_width_for(t.p[0].c);
  int k = tc_pass<0>(c->stream, t, tw, &c);
  t.p[0] = band_args(c, c->R, c->cols, c->rows, eps, 1.f);
  t.p[0].y = pot_out;
  t.p[0].lmarg = lmarg;
  t.p[0].logsum = logsum;
  tc_bind(c, t.p[0]);
  k += tc_pass<1>(c->stream, t, tw, &c);
  c->launches += k;
}

}  // namespace fot
