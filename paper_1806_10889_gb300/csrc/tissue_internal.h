// Internal declarations shared by the CUDA translation units of libtissue.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "tissue.h"

#include <cstddef>
#include <cstdint>

namespace tsg {

constexpr uint32_t kTagChi = 1u, kTagSx = 2u, kTagSy = 3u, kTagInit = 4u;
constexpr uint32_t kTagSx2 = 5u, kTagSy2 = 6u;  // second half-steps of Strang splitting
constexpr uint32_t kTagPlace = 7u;  // placement of a well-mixed cell's D (7), N (8), R (9)
constexpr uint32_t kHillTab = 4096;  // tabulated Hill production for R < kHillTab
constexpr int kErrOverflow = 1;
constexpr int kErrEventIndex = 2;
constexpr int kErrInternal = 4;  // a selection invariant failed (never expected)
constexpr int kErrState = 8;     // promoter model: more bound sites than sites in a voxel
constexpr int kErrBounds = 16;   // checked build: an array index was out of range
// 16-bit counts: a count passed 65535 and the cell is redone with 32-bit
// counts (never reported; the launcher handles it).
constexpr int kErrNarrow = 32;
constexpr uint32_t kModelND = 0u;        // Hill-repressed Notch-Delta lattice model
constexpr uint32_t kModelPromoter = 1u;  // the paper's promoter model (Sec. III-A1)
constexpr int kCountMax = (1 << 30) - 1;      // largest count a voxel may hold
constexpr uint64_t kPropLimit = 1ull << 52;  // a voxel or face channel must stay below

// Quantised model: every rate as an integer in units of 2^-32 per unit time.
// The promoter model maps onto the same fields: gD = gN = d, hopD = hopN =
// hop, k_in = k_a (slot 17, X = N F), k_bind = k_N (face conversion), and
// gR = hopR = k_off = kN = 0; tD and kd are its own.
struct QRates {
  uint64_t kN, gD, gN, gR, hopD, hopN, hopR, k_in, k_off, k_bind;
  uint64_t cD[5], cN[5], cR[5];  // g + nn * hop for nn existing neighbours
  uint64_t cRo[5];               // cR[nn] + k_off
  double kD, K;
  const uint64_t* hill;  // device table, kHillTab entries
  uint32_t small;        // counts all below this keep every voxel total below 2^52
  uint32_t kind;         // kModelND or kModelPromoter
  uint64_t tD, kd;       // promoter: transcription by a free site, unbinding of a bound one
  double k_in_raw, ka_raw;  // unquantised k_in / k_a: well-mixed cells use q(k / V)
};

// One recorded event (tissue_event of the C ABI; the oracle's trace record).
struct TraceRec {
  uint32_t step, kind, unit, e;
  double t;
  uint32_t site, channel;
};

// One tissue as the kernels see it.
struct TissueView {
  int32_t* counts;      // [cell][3][V]
  uint32_t width, height, n, V;
  uint32_t magic;       // ceil(2^16 / n)
  uint32_t tissue_id;
  uint64_t seed;
  QRates q;
  uint64_t* ev_last;    // [3][cells] events of the last step
  double* t_last;       // [3][cells] time of the last event of the last step
  uint64_t* ev_total;   // [3][cells] events since creation
  const uint32_t* step; // device step counter
  int* err;             // device error flag (bit mask)
  const uint8_t* wm;    // per cell: 1 = well-mixed chi; nullptr when no cell is
  uint32_t wm_cells;    // number of well-mixed cells
  uint32_t trace_cap;   // capacity of trace (records)
  TraceRec* trace;      // event trace (tests); nullptr when off
  uint32_t* trace_len;  // events recorded (may exceed trace_cap)
};

// Record one event in the tissue's trace, if it has one (any order).
__device__ __forceinline__ void trace_event(const TissueView& t, uint32_t step, uint32_t kind,
                                            uint32_t unit, uint32_t e, double time, uint32_t site,
                                            uint32_t channel) {
  if (t.trace == nullptr) return;
  const uint32_t i = atomicAdd(t.trace_len, 1u);
  if (i < t.trace_cap) t.trace[i] = TraceRec{step, kind, unit, e, time, site, channel};
}

// NVTX range over a host-side library call (seen by profilers; no cost
// without one attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device allocation by the library: cudaMalloc, unless a test armed the
// host-side fault injector (tissue_debug_fail_allocs), in which case it
// fails as an out-of-memory cudaMalloc would, touching no GPU state.
cudaError_t lib_malloc(void** p, size_t bytes);

// Launchers (enqueue on `stream`; return the launch error).
cudaError_t launch_hill_table(const QRates& q, uint64_t* table, cudaStream_t stream);
cudaError_t launch_init(const TissueView& t, const double p0[3], const double lam[3],
                        cudaStream_t stream);
cudaError_t launch_chi(const TissueView& t, uint32_t step_off, double dt, int warps_per_block,
                       cudaStream_t stream);
// Persistent segmented chi over a work list: d_items = nullptr means the cells
// of d_views[0] in order.  H = 16 or 32 lanes per cell; vmax_cells is the
// largest V among the listed tissues (sizes shared memory).  blocks <= 0
// picks a grid that fills every SM.
// pre: keep the per-voxel prefix array (layout 0) or recompute the selected
// block (layout 1, at most 4 warps per block).
// gen: the models of the listed tissues: 0 Notch-Delta only (the fast
// path), 1 either or a trace is on (each cell tests its tissue's model), 2
// promoter only.
// redo: scratch for the 16-bit-count pass, used when the listed cells have
// more than 256 voxels, gen = 0 and pre (shared memory then bounds how many
// cells an SM holds): items holds n_items entries, counters three words
// {work counter of the first pass, redo count, work counter of the 32-bit
// pass}, all three cleared by the caller before the call (counters[0] is
// then d_counter).  nullptr: 32-bit counts only.
struct ChiRedo {
  uint2* items;
  uint32_t* counters;
};
cudaError_t launch_chi_seg(const TissueView* d_views, const uint2* d_items, uint32_t n_items,
                           uint32_t* d_counter, uint32_t vmax_cells, int H, int warps_per_block,
                           int blocks, uint32_t step_off, double dt, bool pre, int gen,
                           const ChiRedo* redo, cudaStream_t stream, int priority = 0);
using ChiSegKernel = void (*)(const TissueView*, const uint2*, uint32_t, uint32_t*, uint32_t,
                              uint32_t, double, uint2*, uint32_t*, const uint32_t*);
ChiSegKernel chi_seg_kernel_nd(int H, bool pre, bool qb);   // k_chi_seg.cu
ChiSegKernel chi_seg_kernel_gen(int H, bool pre, bool qb);  // k_chi_seg_gen.cu
ChiSegKernel chi_seg_kernel_pm(int H, bool pre, bool qb);   // k_chi_seg_pm.cu
// 16-bit counts, Notch-Delta only (prefix layout at 8, 16 or 32 lanes; the
// counts-only layout at 32 lanes, or at 16 with sub-blocks); nullptr where
// not built.
ChiSegKernel chi_seg_kernel_narrow(int H, bool pre, bool qb);  // k_chi_seg_narrow.cu
uint32_t seg_bytes_for(uint32_t V, int H, bool pre, bool narrow = false);
// Whether the counts-only (recompute) layout takes cells of V voxels with H
// lanes for launches of model code gen (k_chi_seg.cu): V <= H^2, or for the
// Notch-Delta model (gen 0) blocks of up to four sub-blocks of H voxels
// (V <= 4 H^2 at 8 or 16 lanes).
bool recompute_covers(uint32_t V, int H, int gen);
// Well-mixed cells (k_chi_wm.cu): one warp per (tissue, cell) item;
// vmax_cells is the largest V among the listed cells.
cudaError_t launch_chi_wm(const TissueView* d_views, const uint2* d_items, uint32_t n_items,
                          uint32_t vmax_cells, uint32_t step_off, double dt, cudaStream_t stream);
cudaError_t launch_sig_list(const TissueView* d_views, const uint2* d_items, uint32_t n_items,
                            int axis, uint32_t tag, double dt, cudaStream_t stream);
cudaError_t launch_advance_list(const TissueView* d_views, uint32_t n, cudaStream_t stream);
// Batch checkpoint I/O (k_sig.cu): set step counters (d_steps may be null) and
// clear error flags; flag a count outside [0, kCountMax]; gather error flags.
cudaError_t launch_set_steps_list(const TissueView* d_views, const uint32_t* d_steps, uint32_t n,
                                  cudaStream_t stream);
cudaError_t launch_check_counts_list(const TissueView* d_views, uint32_t n, int* d_bad,
                                     cudaStream_t stream);
cudaError_t launch_gather_err_list(const TissueView* d_views, uint32_t n, int* d_out,
                                   cudaStream_t stream);

// Library-internal access to a tissue handle (tissue_lib.cu).
struct TissueInfo {
  tissue_desc desc;
  TissueView view;
  cudaStream_t stream;
  bool has_model;
  const uint8_t* wm_host;  // per cell: 1 = well-mixed (host copy); nullptr if none
};
bool tissue_info(const tissue* t, TissueInfo* out);
// The default chi launch for `cells` cells of V voxels (one launch).
constexpr uint64_t kFewCells = 1024;
// Above these cell counts the default launch takes the counts-only layout:
// past one wave of the prefix launch it would otherwise use, on a 152-SM
// GB300.  Cells of 257..1,024 voxels: one per warp in the prefix layout fit
// 14 per SM (2,128 cells); cells of 65..256 voxels: two per warp, 40 per SM
// (6,080 cells).
constexpr uint64_t kRecCellsLarge = 2128;
constexpr uint64_t kRecCellsMid = 6080;
tissue_launch default_launch(uint32_t V, uint64_t cells);
// The default among prefix-layout launches (the fallback of a counts-only
// launch that cannot take a tissue's model).
tissue_launch prefix_launch(uint32_t V, uint64_t cells);
void tissue_advance_host_step(tissue* t, uint32_t n);
void tissue_set_host_step(tissue* t, uint32_t step_index);
// A latched device error flag as the C ABI's status code.
int error_code_of(int flag);
int seg_lanes_for(uint32_t V, int want);

// tag: the Philox stream tag of this face phase (kTagSx, kTagSy, kTagSx2, kTagSy2).
cudaError_t launch_sig(const TissueView& t, int axis, uint32_t tag, uint32_t step_off, double dt,
                       cudaStream_t stream);
cudaError_t launch_step_advance(uint32_t* step, uint32_t n, cudaStream_t stream);
cudaError_t launch_selftest_time(uint64_t n, uint64_t seed, unsigned long long* mismatches,
                                 cudaStream_t stream);

// Validate and quantise the twelve rates (kD, K, kN, gD, gN, gR, hopD, hopN,
// hopR, k_in, k_off, k_bind) into q; q->hill is set to `hill`.  false when a
// rate is out of range.
bool make_qrates(const double rates[12], const uint64_t* hill, QRates* q);
// The promoter model (tD, ka, kd, kN, d, hop) into q; false when a rate is out
// of range.
bool make_qrates_promoter(const double rates[6], const uint64_t* hill, QRates* q);

// Largest power of two T <= 2^30 such that counts below T keep a voxel's total
// propensity below 2^52 (so the fast path needs no overflow checks).
uint32_t small_count_bound(const QRates& q, uint64_t hill_max);

}  // namespace tsg
