// Banded axis pass: arguments and entry points shared by the CUDA-core kernels
// (fot_band.cu), the tensor-core kernel (fot_tc.cu) and the batched solver (fot_batch.cu).
#pragma once

#include "fot_common.cuh"

namespace fot {

// One problem's pass.  plan holds alpha (float), window start and window length (int) per
// (tile of tile_w outputs, row), tile-major: entry (t, r) at t * plan_stride + r, with
// plan_stride = n_rows rounded up to 128 (a 128-row block's alphas are contiguous), the three
// arrays n_tiles * plan_stride words each, consecutive.
struct BandArgs {
  const float* x;      // [n_rows][len] input
  float* plan;
  const float* lmarg;  // potential-update mode: natural log marginal, layout of y
  float* y;            // [len][n_rows] output (transposed)
  float* logsum;       // potential-update mode: optional natural-log LSE, layout of y
  int* err;
  unsigned long long* terms;     // [2]: += (row, output, m) triples evaluated on the CUDA cores,
                                 // [0] tilted-GEMM items, [1] exact-window items
  unsigned long long* tc_terms;  // += triples evaluated on the tensor cores
  // tensor-core pass only (null / 0 otherwise): per 128-row unit (row block, tile) the union
  // of its rows' windows [ext_lo, ext_hi), reduced by the plan kernel with atomics into the
  // current buffers; the plan kernel also resets the other pair (the next pass's).  Reset
  // state: ext_lo = 0x7F7F7F7F, ext_hi = 0.
  int* ext_lo;
  int* ext_hi;
  int* ext_lo_next;
  int* ext_hi_next;
  int ext_units;       // entries of each extent array
  int* ucnt;           // per unit: contributions of a unit split between CTAs (reset to 0)
  const unsigned char* btab;   // B operand table of this pass (tc_btab_fill)
  float x_scale, c, eps;
  int tile_w;          // outputs per plan tile: 16 (CUDA-core and 16-wide tensor passes) or 64
  int n_rows, len, n_chunks, n_tiles;
  int plan_stride;     // n_rows rounded up to 128
  int s_max;           // B table: window stages of the longest possible window (len / 32 up)
  int row_base, plan_base, item_base, cta_base;   // first global work index of each kernel
  int plan_rows;       // rows of the plan kernel's grid for this problem (n_rows rounded up to 8)
  int lm_tma;          // potential-update tensor pass: lmap holds lmarg (else read directly)
  alignas(64) unsigned char xmap[128];   // CUtensorMap of x for the tensor-core pass
  alignas(64) unsigned char lmap[128];   // CUtensorMap of lmarg (potential-update tensor pass)
};

constexpr int kMaxBatch = 64;

// A launch covers every problem of the table; each kernel maps its global warp (or CTA)
// index to a problem by the *_base prefix sums.  Passed by value (__grid_constant__).
template <int MAXP>
struct BandTable {
  int n;                                 // problems
  int rows, plans, items, ctas;          // totals of the four work kinds (ctas: 128-row units)
  int plan_row_stride;                   // floats of plan-kernel shared memory per row
  int plan_tiles;                        // largest n_tiles of the table
  int plan_wpr;                          // plan kernel: warps per row
  // tensor-core pass: chunk sums of units split between CTAs ([grid][slot_chunks][128][tile_w]
  // floats, indexed by the unit's first contributor) and the wait limit of the pipeline barriers
  float* slots;
  int slot_chunks;
  int spin_limit;
  int tc_single;                         // tensor pass: single BF16 operands (one MMA per term)
  BandArgs p[MAXP];
};
static_assert(sizeof(BandTable<kMaxBatch>) <= 32764, "kernel parameter limit");

// problem owning global work index gi of kind WHICH (0 rows, 1 plan rows, 2 band items,
// 3 tensor-core units): binary search over the prefix sums (a single problem needs none)
template <int MAXP, int WHICH>
__device__ __forceinline__ int find_prob(const BandTable<MAXP>& t, int gi) {
  if (MAXP == 1) return 0;
  int lo = 0, hi = t.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const BandArgs& q = t.p[mid];
    const int b = WHICH == 0 ? q.row_base : WHICH == 1 ? q.plan_base : WHICH == 2 ? q.item_base : q.cta_base;
    if (b <= gi)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// fill n_chunks, n_tiles, the *_base prefix sums and the totals
template <int MAXP>
void band_table_finish(BandTable<MAXP>& t);

// per-(row, tile) plan of every problem
template <int MAXP>
void band_prepare(cudaStream_t s, BandTable<MAXP>& t);

// the CUDA-core window sums (MODE 0: log-sum output; MODE 1: potential update)
template <int MODE, int MAXP>
void band_simt(cudaStream_t s, const BandTable<MAXP>& t);

// tile width of the tensor-core pass for kernel constant c: 64, 32, 16, or 0 (CUDA cores)
int tc_width_for(float c);

// a whole pass on the tensor cores (fot_tc.cu) at tile width tw (every problem of the table
// must have tc_width_for(c) == tw and its tensor-core fields set by tc_bind; ctx[q] is problem
// q's context): finishes the table, writes stale B tables, plans and launches; units outside
// the tilt bound take CUDA-core sums inside the same kernel, and tw = 0 (or a table the
// tensor kernel cannot take: rows not 16-byte aligned, too many units) runs band_simt.
// Returns the number of kernels launched.
template <int MODE, int MAXP>
int tc_pass(cudaStream_t s, BandTable<MAXP>& t, int tw, fot_ctx* const* ctx);

// tensor-core fields of one pass of context c (toggles its unit-extent parity: once per pass)
void tc_bind(fot_ctx* c, BandArgs& a);
// start of an API call's sequence of passes on context c (B table rewritten at the first pass)
void tc_begin(fot_ctx* c);

}  // namespace fot
