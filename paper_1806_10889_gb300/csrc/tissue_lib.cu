// libtissue: the C ABI of include/tissue.h.
//
// The orchestration role of the paper's Dask DAG (Sec. II-C, Fig. 4) is taken
// by stream order: each splitting step enqueues K_chi over all cells, then
// K_sig over the x-faces, then over the y-faces, on the tissue's stream.  The
// state never leaves device memory between steps (the paper's per-module
// input/output files become in-place reads and writes of one array).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "tissue.h"
#include "tissue_internal.h"

using namespace tsg;

struct tissue {
  tissue_desc d{};
  int32_t* counts = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  bool has_model = false;
  QRates q{};
  unsigned char* scratch = nullptr;
  uint64_t* hill = nullptr;
  uint64_t* ev_last = nullptr;
  double* t_last = nullptr;
  uint64_t* ev_total = nullptr;
  uint32_t* d_step = nullptr;
  int* d_err = nullptr;
  uint32_t step_index = 0;
  tissue_launch cfg{TISSUE_KERNEL_WARP, 32, 4, 0, TISSUE_LAYOUT_PREFIX};
  uint32_t scheme = TISSUE_SPLIT_LIE;
  TissueView* d_view = nullptr;   // device copy of the view, for the persistent kernel
  uint32_t* d_work = nullptr;     // work-list counters of the persistent kernel (3 words)
  uint2* d_redo = nullptr;        // cells the 16-bit-count pass gives up on
  uint8_t* d_wm = nullptr;        // per cell: 1 = well-mixed chi
  uint32_t wm_cells = 0;
  std::vector<uint8_t> wm_host;   // host copy of d_wm (empty: no well-mixed cell)
  uint2* d_lat_items = nullptr;   // (0, cell) of the lattice cells, when some are well-mixed
  uint2* d_wm_items = nullptr;    // (0, cell) of the well-mixed cells
  TraceRec* d_trace = nullptr;    // event trace (tissue_trace_begin); nullptr when off
  uint32_t* d_trace_len = nullptr;
  uint32_t trace_cap = 0;
};

namespace {

bool desc_ok(const tissue_desc* d) {
  if (!d) return false;
  if (d->width < 1 || d->height < 1 || d->n < 2 || d->n > 32) return false;
  if (d->tissue_id >= (1u << 24)) return false;
  if (static_cast<uint64_t>(d->width) * d->height > 0xFFFFFFFFull) return false;
  for (int s = 0; s < 3; ++s)
    if (!(d->init_lambda[s] >= 0.0 && d->init_lambda[s] <= 700.0)) return false;
  return true;
}

uint64_t cells_of(const tissue_desc* d) { return static_cast<uint64_t>(d->width) * d->height; }

struct ScratchLayout {
  size_t hill, ev_last, t_last, ev_total, step, err, view, work, wm, lat_items, wm_items, redo,
      total;
};

ScratchLayout layout(const tissue_desc* d) {
  const size_t cells = cells_of(d);
  auto up = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
  ScratchLayout L{};
  size_t o = 0;
  L.hill = o;
  o = up(o + sizeof(uint64_t) * kHillTab);
  L.ev_last = o;
  o = up(o + sizeof(uint64_t) * 3 * cells);
  L.t_last = o;
  o = up(o + sizeof(double) * 3 * cells);
  L.ev_total = o;
  o = up(o + sizeof(uint64_t) * 3 * cells);
  L.step = o;
  o = up(o + sizeof(uint32_t));
  L.err = o;
  o = up(o + sizeof(int));
  L.view = o;
  o = up(o + sizeof(TissueView));
  L.work = o;  // work counter, redo count, work counter of the 32-bit redo pass
  o = up(o + 3 * sizeof(uint32_t));
  L.wm = o;
  o = up(o + cells);
  L.lat_items = o;
  o = up(o + sizeof(uint2) * cells);
  L.wm_items = o;
  o = up(o + sizeof(uint2) * cells);
  L.redo = o;  // cells the 16-bit-count pass hands to the 32-bit one
  o = up(o + sizeof(uint2) * cells);
  L.total = o;
  return L;
}

TissueView view_of(const tissue* t) {
  TissueView v{};
  v.counts = t->counts;
  v.width = t->d.width;
  v.height = t->d.height;
  v.n = t->d.n;
  v.V = t->d.n * t->d.n;
  v.magic = (65536u + t->d.n - 1) / t->d.n;
  v.tissue_id = t->d.tissue_id;
  v.seed = t->d.seed;
  v.q = t->q;
  v.ev_last = t->ev_last;
  v.t_last = t->t_last;
  v.ev_total = t->ev_total;
  v.step = t->d_step;
  v.err = t->d_err;
  v.wm = t->wm_cells ? t->d_wm : nullptr;
  v.wm_cells = t->wm_cells;
  v.trace = t->d_trace;
  v.trace_len = t->d_trace_len;
  v.trace_cap = t->trace_cap;
  return v;
}

}  // namespace

namespace {
std::atomic<uint32_t> g_fail_allocs{0};
}  // namespace

cudaError_t tsg::lib_malloc(void** p, size_t bytes) {
  uint32_t n = g_fail_allocs.load();
  while (n > 0) {
    if (g_fail_allocs.compare_exchange_weak(n, n - 1)) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  return cudaMalloc(p, bytes);
}

tissue_launch tsg::prefix_launch(uint32_t V, uint64_t cells) {
  // Up to ~1,000 cells the machine is not full and each cell's event chain
  // sets the time: one cell per warp has the shortest chain (measured:
  // 2,790 against 2,930 and 3,220 SM cycles per event with 16 and 8 lanes on
  // four 8x8 cells).  Beyond that, cells sharing a warp share its
  // instruction issue.
  if (cells <= kFewCells) return tissue_launch{TISSUE_KERNEL_PERSISTENT, 32, 2, 0,
                                               TISSUE_LAYOUT_PREFIX};
  if (V <= 64) return tissue_launch{TISSUE_KERNEL_PERSISTENT, 8, 4, 0, TISSUE_LAYOUT_PREFIX};
  if (V <= 256) return tissue_launch{TISSUE_KERNEL_PERSISTENT, 16, 4, 0, TISSUE_LAYOUT_PREFIX};
  return tissue_launch{TISSUE_KERNEL_PERSISTENT, 32, 2, 0, TISSUE_LAYOUT_PREFIX};
}

tissue_launch tsg::default_launch(uint32_t V, uint64_t cells) {
  // Past one wave of the prefix launch, the counts-only layout, each event
  // recomputing one sub-block of the selected block (one voxel per lane):
  // - cells of 257..1,024 voxels two per warp (16-bit counts, 6.4 KB per
  //   cell: 32 per SM against 14 in the prefix layout);
  // - cells of 65..256 voxels four per warp (64 per SM against 40).
  // Same-box A/B, chi ms per step (prefix launch -> this one): 32x32-voxel
  // cells 25.8 -> 32.4 at 1,024 cells (one prefix wave: kept), 50.8 -> 36.5
  // at 2,304, 68.5 -> 51.4 at 4,096, 876 -> 542 at 65,536; 16x16-voxel cells
  // 9.4 -> 10.1 at 4,096 (kept), 18.8 -> 14.1 at 9,216, 32.0 -> 25.3 at
  // 16,384.  Smaller launches keep the prefix layout, whose event chains are
  // shorter.  Launches the counts-only layout cannot take (the promoter
  // model, a trace) run prefix_launch.
  if (V > 256 && V <= 1024 && cells > kRecCellsLarge)
    return tissue_launch{TISSUE_KERNEL_PERSISTENT, 16, 2, 0, TISSUE_LAYOUT_RECOMPUTE};
  if (V > 64 && V <= 256 && cells > kRecCellsMid)
    return tissue_launch{TISSUE_KERNEL_PERSISTENT, 8, 2, 0, TISSUE_LAYOUT_RECOMPUTE};
  return prefix_launch(V, cells);
}

namespace {

// chi for step offset i, in the tissue's launch configuration.
cudaError_t launch_chi_cfg(tissue* t, const TissueView& v, uint32_t i, double dt) {
  tissue_launch c = t->cfg;
  if (c.kernel == TISSUE_KERNEL_PERSISTENT) {
    const uint32_t cells = t->d.width * t->d.height;
    const int gen = t->q.kind == kModelPromoter ? 2 : t->d_trace != nullptr ? 1 : 0;
    // A counts-only launch with several voxels per lane runs Notch-Delta
    // launches without a trace only; others take the prefix launch of the
    // cell size (the same trajectory, bit for bit).
    if (c.smem_layout == TISSUE_LAYOUT_RECOMPUTE &&
        !recompute_covers(v.V, static_cast<int>(c.lanes_per_cell), gen))
      c = prefix_launch(v.V, cells - t->wm_cells);
    cudaError_t e = cudaSuccess;
    if (t->wm_cells) {  // well-mixed cells first, then the lattice cells by list
      e = launch_chi_wm(t->d_view, t->d_wm_items, t->wm_cells, v.V, i, dt, t->stream);
      if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(t->d_work, 0, 3 * sizeof(uint32_t), t->stream);
    if (e != cudaSuccess) return e;
    const ChiRedo redo{t->d_redo, t->d_work};
    const bool pre = c.smem_layout == TISSUE_LAYOUT_PREFIX;
    return launch_chi_seg(t->d_view, t->wm_cells ? t->d_lat_items : nullptr, cells - t->wm_cells,
                          t->d_work, v.V, static_cast<int>(c.lanes_per_cell),
                          static_cast<int>(c.warps_per_block), static_cast<int>(c.blocks), i, dt,
                          pre, gen, &redo, t->stream);
  }
  return launch_chi(v, i, dt, static_cast<int>(c.warps_per_block), t->stream);
}

// One splitting step at step offset i.  `mark`, if given, is recorded right
// before and right after the chi launch (for the timed variant).
int enqueue_split_step(tissue* t, const TissueView& v, uint32_t i, double dt, cudaEvent_t before,
                       cudaEvent_t after) {
  auto chi = [&]() -> bool {
    if (before && cudaEventRecord(before, t->stream) != cudaSuccess) return false;
    if (launch_chi_cfg(t, v, i, dt) != cudaSuccess) return false;
    return !after || cudaEventRecord(after, t->stream) == cudaSuccess;
  };
  if (t->scheme == TISSUE_SPLIT_LIE) {
    if (!chi() || launch_sig(v, 0, kTagSx, i, dt, t->stream) != cudaSuccess ||
        launch_sig(v, 1, kTagSy, i, dt, t->stream) != cudaSuccess)
      return TISSUE_E_CUDA;
  } else {
    const double h = dt * 0.5;
    if (launch_sig(v, 0, kTagSx, i, h, t->stream) != cudaSuccess ||
        launch_sig(v, 1, kTagSy, i, h, t->stream) != cudaSuccess || !chi() ||
        launch_sig(v, 1, kTagSy2, i, h, t->stream) != cudaSuccess ||
        launch_sig(v, 0, kTagSx2, i, h, t->stream) != cudaSuccess)
      return TISSUE_E_CUDA;
  }
  return TISSUE_OK;
}

int device_error(tissue* t) {
  int h = 0;
  if (cudaMemcpyAsync(&h, t->d_err, sizeof(int), cudaMemcpyDeviceToHost, t->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  if (cudaStreamSynchronize(t->stream) != cudaSuccess) return TISSUE_E_CUDA;
  return tsg::error_code_of(h);
}

// The one-warp-per-cell kernel computes lattice cells of the Notch-Delta
// model only.
bool launch_fits_model(const tissue* t) {
  return (t->q.kind == kModelND && t->wm_cells == 0 && t->d_trace == nullptr) ||
         t->cfg.kernel == TISSUE_KERNEL_PERSISTENT;
}

int upload_view(tissue* t) {
  const TissueView v = view_of(t);
  return cudaMemcpyAsync(t->d_view, &v, sizeof(v), cudaMemcpyHostToDevice, t->stream) == cudaSuccess
             ? TISSUE_OK
             : TISSUE_E_CUDA;
}

bool rate_ok(double x) { return std::isfinite(x) && x >= 0.0 && x < 1048576.0; }

// Rate x as an integer number of 2^-32 units: round-half-even(x * 2^32).
uint64_t quantise(double x) { return static_cast<uint64_t>(std::nearbyint(x * 4294967296.0)); }

}  // namespace

bool tsg::make_qrates(const double r[12], const uint64_t* hill, QRates* q) {
  for (int i = 0; i < 12; ++i)
    if (!rate_ok(r[i])) return false;
  if (!(r[1] > 0.0)) return false;
  *q = QRates{};
  q->kD = r[0];
  q->K = r[1];
  q->kN = quantise(r[2]);
  q->gD = quantise(r[3]);
  q->gN = quantise(r[4]);
  q->gR = quantise(r[5]);
  q->hopD = quantise(r[6]);
  q->hopN = quantise(r[7]);
  q->hopR = quantise(r[8]);
  q->k_in = quantise(r[9]);
  q->k_off = quantise(r[10]);
  q->k_bind = quantise(r[11]);
  q->k_in_raw = r[9];
  for (int nn = 0; nn <= 4; ++nn) {
    q->cD[nn] = q->gD + static_cast<uint64_t>(nn) * q->hopD;
    q->cN[nn] = q->gN + static_cast<uint64_t>(nn) * q->hopN;
    q->cR[nn] = q->gR + static_cast<uint64_t>(nn) * q->hopR;
    q->cRo[nn] = q->cR[nn] + q->k_off;
  }
  q->hill = hill;
  // the Hill term is largest at R = 0, where it is quantise(kD) (kD / 1)
  q->small = small_count_bound(*q, quantise(r[0]));
  return true;
}

bool tsg::make_qrates_promoter(const double r[6], const uint64_t* hill, QRates* q) {
  for (int i = 0; i < 6; ++i)
    if (!rate_ok(r[i])) return false;
  *q = QRates{};
  q->kind = kModelPromoter;
  q->tD = quantise(r[0]);
  q->k_in = quantise(r[1]);    // k_a: slot 17, N + F -> R
  q->ka_raw = r[1];
  q->kd = quantise(r[2]);
  q->k_bind = quantise(r[3]);  // k_N: Delta -> NICD across a face
  q->gD = q->gN = quantise(r[4]);
  q->hopD = q->hopN = quantise(r[5]);
  q->K = 1.0;
  for (int nn = 0; nn <= 4; ++nn) {
    q->cD[nn] = q->gD + static_cast<uint64_t>(nn) * q->hopD;
    q->cN[nn] = q->gN + static_cast<uint64_t>(nn) * q->hopN;
  }
  q->hill = hill;
  // c0 + c1 = tD F + kd R <= max(tD, kd) since F + R <= 1
  q->small = small_count_bound(*q, q->tD > q->kd ? q->tD : q->kd);
  return true;
}

bool tsg::tissue_info(const tissue* t, TissueInfo* out) {
  if (!t || !out) return false;
  out->desc = t->d;
  out->view = view_of(t);
  out->stream = t->stream;
  out->has_model = t->has_model;
  out->wm_host = t->wm_cells ? t->wm_host.data() : nullptr;
  return true;
}

void tsg::tissue_advance_host_step(tissue* t, uint32_t n) { t->step_index += n; }

void tsg::tissue_set_host_step(tissue* t, uint32_t step_index) { t->step_index = step_index; }

int tsg::error_code_of(int h) {
  if (h & kErrBounds) return TISSUE_E_BOUNDS;
  if (h & kErrInternal) return TISSUE_E_CUDA;
  if (h & kErrState) return TISSUE_E_STATE;
  return h ? TISSUE_E_OVERFLOW : TISSUE_OK;
}

extern "C" {

size_t tissue_state_bytes(const tissue_desc* d) {
  if (!desc_ok(d)) return 0;
  return static_cast<size_t>(cells_of(d)) * 3 * d->n * d->n * sizeof(int32_t);
}

size_t tissue_scratch_bytes(const tissue_desc* d) {
  if (!desc_ok(d)) return 0;
  return layout(d).total;
}

int tissue_create(const tissue_desc* d, void* dev_counts, size_t bytes, void* cuda_stream,
                  tissue** out) {
  NvtxRange range("tissue_create");
  if (!out) return TISSUE_E_ARG;
  *out = nullptr;
  if (!desc_ok(d) || !dev_counts) return TISSUE_E_ARG;
  if (bytes < tissue_state_bytes(d)) return TISSUE_E_ARG;
  if (reinterpret_cast<uintptr_t>(dev_counts) % 16 != 0) return TISSUE_E_ARG;
  tissue* t = new (std::nothrow) tissue();
  if (!t) return TISSUE_E_NOMEM;
  t->d = *d;
  t->counts = static_cast<int32_t*>(dev_counts);
  t->bytes = bytes;
  t->stream = static_cast<cudaStream_t>(cuda_stream);
  // Default chi launch (measured on GB300): the persistent kernel with four
  // cells per warp for V <= 64, two for V <= 256, one (2 warps per block)
  // above.
  t->cfg = default_launch(d->n * d->n, cells_of(d));
  const ScratchLayout L = layout(d);
  if (lib_malloc(reinterpret_cast<void**>(&t->scratch), L.total) != cudaSuccess) {
    cudaGetLastError();
    delete t;
    return TISSUE_E_NOMEM;
  }
  t->hill = reinterpret_cast<uint64_t*>(t->scratch + L.hill);
  t->ev_last = reinterpret_cast<uint64_t*>(t->scratch + L.ev_last);
  t->t_last = reinterpret_cast<double*>(t->scratch + L.t_last);
  t->ev_total = reinterpret_cast<uint64_t*>(t->scratch + L.ev_total);
  t->d_step = reinterpret_cast<uint32_t*>(t->scratch + L.step);
  t->d_err = reinterpret_cast<int*>(t->scratch + L.err);
  t->d_view = reinterpret_cast<TissueView*>(t->scratch + L.view);
  t->d_work = reinterpret_cast<uint32_t*>(t->scratch + L.work);
  t->d_redo = reinterpret_cast<uint2*>(t->scratch + L.redo);
  t->d_wm = reinterpret_cast<uint8_t*>(t->scratch + L.wm);
  t->d_lat_items = reinterpret_cast<uint2*>(t->scratch + L.lat_items);
  t->d_wm_items = reinterpret_cast<uint2*>(t->scratch + L.wm_items);
  if (cudaMemsetAsync(t->scratch, 0, L.total, t->stream) != cudaSuccess) {
    cudaFree(t->scratch);
    delete t;
    return TISSUE_E_CUDA;
  }
  double p0[3], lam[3];
  for (int s = 0; s < 3; ++s) {
    lam[s] = d->init_lambda[s];
    p0[s] = std::exp(-lam[s]);
  }
  if (launch_init(view_of(t), p0, lam, t->stream) != cudaSuccess) {
    cudaFree(t->scratch);
    delete t;
    return TISSUE_E_CUDA;
  }
  *out = t;
  return TISSUE_OK;
}

int tissue_set_model(tissue* t, const tissue_model* m) {
  if (!t || !m) return TISSUE_E_ARG;
  const double r[12] = {m->kD, m->K, m->kN, m->gD, m->gN, m->gR,
                        m->hopD, m->hopN, m->hopR, m->k_in, m->k_off, m->k_bind};
  QRates q{};
  if (!make_qrates(r, t->hill, &q)) return TISSUE_E_ARG;
  if (launch_hill_table(q, t->hill, t->stream) != cudaSuccess) return TISSUE_E_CUDA;
  t->q = q;
  const TissueView v = view_of(t);
  if (cudaMemcpyAsync(t->d_view, &v, sizeof(v), cudaMemcpyHostToDevice, t->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  t->has_model = true;
  return TISSUE_OK;
}

int tissue_set_promoter_model(tissue* t, const tissue_promoter_model* m) {
  if (!t || !m) return TISSUE_E_ARG;
  const double r[6] = {m->tD, m->ka, m->kd, m->kN, m->d, m->hop};
  QRates q{};
  if (!make_qrates_promoter(r, t->hill, &q)) return TISSUE_E_ARG;
  t->q = q;
  const TissueView v = view_of(t);
  if (cudaMemcpyAsync(t->d_view, &v, sizeof(v), cudaMemcpyHostToDevice, t->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  t->has_model = true;
  return TISSUE_OK;
}

int tissue_set_cell_fidelity(tissue* t, const uint8_t* host, size_t n) {
  if (!t || !host || n != cells_of(&t->d)) return TISSUE_E_ARG;
  uint32_t count = 0;
  for (size_t i = 0; i < n; ++i) {
    if (host[i] > 1) return TISSUE_E_ARG;
    count += host[i];
  }
  std::vector<uint2> lat, wm;
  for (uint32_t c = 0; c < n; ++c) (host[c] ? wm : lat).push_back(make_uint2(0u, c));
  if (cudaMemcpyAsync(t->d_wm, host, n, cudaMemcpyHostToDevice, t->stream) != cudaSuccess ||
      (!lat.empty() && cudaMemcpyAsync(t->d_lat_items, lat.data(), sizeof(uint2) * lat.size(),
                                       cudaMemcpyHostToDevice, t->stream) != cudaSuccess) ||
      (!wm.empty() && cudaMemcpyAsync(t->d_wm_items, wm.data(), sizeof(uint2) * wm.size(),
                                      cudaMemcpyHostToDevice, t->stream) != cudaSuccess))
    return TISSUE_E_CUDA;
  t->wm_cells = count;
  if (count) t->wm_host.assign(host, host + n);
  else t->wm_host.clear();
  const TissueView v = view_of(t);
  if (cudaMemcpyAsync(t->d_view, &v, sizeof(v), cudaMemcpyHostToDevice, t->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  // the host arrays (the caller's and the item lists) are released on return
  return cudaStreamSynchronize(t->stream) == cudaSuccess ? TISSUE_OK : TISSUE_E_CUDA;
}

int tissue_write_counts(tissue* t, const int32_t* host, size_t n, uint32_t step_index) {
  NvtxRange range("tissue_write_counts");
  if (!t || !host) return TISSUE_E_ARG;
  const size_t want = tissue_state_bytes(&t->d) / sizeof(int32_t);
  if (n != want) return TISSUE_E_ARG;
  // 0 <= count <= TISSUE_COUNT_MAX, as one unsigned compare (a negative count
  // is a large unsigned value); a branch-free reduction the compiler vectorises
  uint32_t worst = 0;
  for (size_t i = 0; i < n; ++i) {
    const uint32_t x = static_cast<uint32_t>(host[i]);
    worst = x > worst ? x : worst;
  }
  if (worst > static_cast<uint32_t>(TISSUE_COUNT_MAX)) return TISSUE_E_ARG;
  if (cudaMemcpyAsync(t->counts, host, n * sizeof(int32_t), cudaMemcpyHostToDevice, t->stream) !=
      cudaSuccess)
    return TISSUE_E_CUDA;
  if (cudaMemcpyAsync(t->d_step, &step_index, sizeof(uint32_t), cudaMemcpyHostToDevice,
                      t->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  if (cudaMemsetAsync(t->d_err, 0, sizeof(int), t->stream) != cudaSuccess) return TISSUE_E_CUDA;
  if (cudaStreamSynchronize(t->stream) != cudaSuccess) return TISSUE_E_CUDA;
  t->step_index = step_index;
  return TISSUE_OK;
}

int tissue_step(tissue* t, double dt, uint32_t n_steps) {
  NvtxRange range("tissue_step");
  if (!t) return TISSUE_E_ARG;
  if (!t->has_model) return TISSUE_E_NOMODEL;
  if (!(dt > 0.0) || !std::isfinite(dt) || !launch_fits_model(t)) return TISSUE_E_ARG;
  if (n_steps == 0) return TISSUE_OK;
  const TissueView v = view_of(t);
  for (uint32_t i = 0; i < n_steps; ++i) {
    const int rc = enqueue_split_step(t, v, i, dt, nullptr, nullptr);
    if (rc != TISSUE_OK) return rc;
  }
  if (launch_step_advance(t->d_step, n_steps, t->stream) != cudaSuccess) return TISSUE_E_CUDA;
  t->step_index += n_steps;
  return TISSUE_OK;
}

int tissue_step_timed(tissue* t, double dt, uint32_t n_steps, double* ms_chi, double* ms_sig) {
  NvtxRange range("tissue_step_timed");
  if (!t) return TISSUE_E_ARG;
  if (!t->has_model) return TISSUE_E_NOMODEL;
  if (!(dt > 0.0) || !std::isfinite(dt) || !launch_fits_model(t)) return TISSUE_E_ARG;
  // per step: start, chi start, chi end, end
  std::vector<cudaEvent_t> ev(4 * static_cast<size_t>(n_steps), nullptr);
  int rc = TISSUE_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) rc = TISSUE_E_CUDA;
  const TissueView v = view_of(t);
  for (uint32_t i = 0; i < n_steps && rc == TISSUE_OK; ++i) {
    if (cudaEventRecord(ev[4 * i], t->stream) != cudaSuccess) rc = TISSUE_E_CUDA;
    if (rc == TISSUE_OK) rc = enqueue_split_step(t, v, i, dt, ev[4 * i + 1], ev[4 * i + 2]);
    if (rc == TISSUE_OK && cudaEventRecord(ev[4 * i + 3], t->stream) != cudaSuccess)
      rc = TISSUE_E_CUDA;
  }
  if (rc == TISSUE_OK && launch_step_advance(t->d_step, n_steps, t->stream) != cudaSuccess)
    rc = TISSUE_E_CUDA;
  if (rc == TISSUE_OK && cudaStreamSynchronize(t->stream) != cudaSuccess) rc = TISSUE_E_CUDA;
  double chi = 0.0, all = 0.0;
  for (uint32_t i = 0; i < n_steps && rc == TISSUE_OK; ++i) {
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, ev[4 * i + 1], ev[4 * i + 2]) != cudaSuccess ||
        cudaEventElapsedTime(&b, ev[4 * i], ev[4 * i + 3]) != cudaSuccess)
      rc = TISSUE_E_CUDA;
    chi += a;
    all += b;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (rc != TISSUE_OK) return rc;
  t->step_index += n_steps;
  if (ms_chi) *ms_chi = chi;
  if (ms_sig) *ms_sig = all - chi;
  return device_error(t);
}

int tissue_set_splitting(tissue* t, uint32_t scheme) {
  if (!t || (scheme != TISSUE_SPLIT_LIE && scheme != TISSUE_SPLIT_STRANG)) return TISSUE_E_ARG;
  t->scheme = scheme;
  return TISSUE_OK;
}

int tissue_read_counts(tissue* t, int32_t* host, size_t n) {
  NvtxRange range("tissue_read_counts");
  if (!t || !host) return TISSUE_E_ARG;
  if (n != tissue_state_bytes(&t->d) / sizeof(int32_t)) return TISSUE_E_ARG;
  if (cudaMemcpyAsync(host, t->counts, n * sizeof(int32_t), cudaMemcpyDeviceToHost, t->stream) !=
      cudaSuccess)
    return TISSUE_E_CUDA;
  return device_error(t);
}

int tissue_read_stats(tissue* t, uint64_t* n_events, double* t_last, size_t n) {
  if (!t) return TISSUE_E_ARG;
  const size_t want = 3 * static_cast<size_t>(cells_of(&t->d));
  if (n != want) return TISSUE_E_ARG;
  if (n_events && cudaMemcpyAsync(n_events, t->ev_last, n * sizeof(uint64_t),
                                  cudaMemcpyDeviceToHost, t->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  if (t_last && cudaMemcpyAsync(t_last, t->t_last, n * sizeof(double), cudaMemcpyDeviceToHost,
                                t->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  return device_error(t);
}

int tissue_total_events(tissue* t, uint64_t out[3]) {
  if (!t || !out) return TISSUE_E_ARG;
  const size_t cells = cells_of(&t->d);
  std::vector<uint64_t> h(3 * cells);
  if (cudaMemcpyAsync(h.data(), t->ev_total, h.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                      t->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  const int rc = device_error(t);
  for (int k = 0; k < 3; ++k) {
    uint64_t s = 0;
    for (size_t c = 0; c < cells; ++c) s += h[k * cells + c];
    out[k] = s;
  }
  return rc;
}

int tissue_get_step(const tissue* t, uint32_t* step_index) {
  if (!t || !step_index) return TISSUE_E_ARG;
  *step_index = t->step_index;
  return TISSUE_OK;
}

int tissue_sync(tissue* t) {
  if (!t) return TISSUE_E_ARG;
  return device_error(t);
}

int tissue_set_launch(tissue* t, uint32_t chi_warps_per_block) {
  if (!t || chi_warps_per_block < 1 || chi_warps_per_block > 16) return TISSUE_E_ARG;
  t->cfg = tissue_launch{TISSUE_KERNEL_WARP, 32, chi_warps_per_block, 0, TISSUE_LAYOUT_PREFIX};
  return TISSUE_OK;
}

int tissue_set_launch_config(tissue* t, const tissue_launch* c) {
  if (!t || !c) return TISSUE_E_ARG;
  const uint32_t V = t->d.n * t->d.n;
  if (c->kernel == TISSUE_KERNEL_WARP) {
    if (c->warps_per_block < 1 || c->warps_per_block > 16) return TISSUE_E_ARG;
  } else if (c->kernel == TISSUE_KERNEL_PERSISTENT) {
    if (c->lanes_per_cell != 32 && c->lanes_per_cell != 16 && c->lanes_per_cell != 8)
      return TISSUE_E_ARG;
    // the recompute layout needs a block to fit the segment's lanes
    // (V <= lanes^2), or 16 lanes and V <= 1024 for the Notch-Delta model
    if (c->smem_layout == TISSUE_LAYOUT_RECOMPUTE &&
        !recompute_covers(V, static_cast<int>(c->lanes_per_cell), 0))
      return TISSUE_E_ARG;
    if (c->smem_layout != TISSUE_LAYOUT_PREFIX && c->smem_layout != TISSUE_LAYOUT_RECOMPUTE)
      return TISSUE_E_ARG;
    const bool pre = c->smem_layout == TISSUE_LAYOUT_PREFIX;
    if (c->warps_per_block < 1 || c->warps_per_block > (pre ? 8u : 4u)) return TISSUE_E_ARG;
    if (static_cast<size_t>(c->warps_per_block) * (32 / c->lanes_per_cell) *
            seg_bytes_for(V, static_cast<int>(c->lanes_per_cell), pre) > 227 * 1024)
      return TISSUE_E_ARG;
  } else {
    return TISSUE_E_ARG;
  }
  t->cfg = *c;
  return TISSUE_OK;
}

int tissue_get_launch_config(const tissue* t, tissue_launch* c) {
  if (!t || !c) return TISSUE_E_ARG;
  *c = t->cfg;
  return TISSUE_OK;
}

int tissue_trace_begin(tissue* t, size_t capacity) {
  if (!t || capacity == 0 || capacity > 0xFFFFFFFFull) return TISSUE_E_ARG;
  tissue_trace_end(t);
  if (cudaStreamSynchronize(t->stream) != cudaSuccess) return TISSUE_E_CUDA;
  void* p = nullptr;
  if (lib_malloc(&p, sizeof(TraceRec) * capacity + 256) != cudaSuccess) {
    cudaGetLastError();
    return TISSUE_E_NOMEM;
  }
  t->d_trace_len = static_cast<uint32_t*>(p);
  t->d_trace = reinterpret_cast<TraceRec*>(static_cast<unsigned char*>(p) + 256);
  t->trace_cap = static_cast<uint32_t>(capacity);
  if (cudaMemsetAsync(t->d_trace_len, 0, sizeof(uint32_t), t->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  return upload_view(t);
}

int tissue_trace_read(tissue* t, tissue_event* host, size_t capacity, size_t* n_recorded) {
  static_assert(sizeof(tissue_event) == sizeof(TraceRec), "trace record layout");
  if (!t || !n_recorded || (capacity && !host)) return TISSUE_E_ARG;
  if (!t->d_trace) return TISSUE_E_ARG;
  uint32_t n = 0;
  if (cudaMemcpyAsync(&n, t->d_trace_len, sizeof(n), cudaMemcpyDeviceToHost, t->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(t->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  *n_recorded = n;
  const size_t k = std::min<size_t>(std::min<size_t>(n, t->trace_cap), capacity);
  if (k && cudaMemcpy(host, t->d_trace, sizeof(TraceRec) * k, cudaMemcpyDeviceToHost) != cudaSuccess)
    return TISSUE_E_CUDA;
  return device_error(t);
}

int tissue_trace_end(tissue* t) {
  if (!t) return TISSUE_E_ARG;
  if (!t->d_trace_len) return TISSUE_OK;
  if (cudaStreamSynchronize(t->stream) != cudaSuccess) return TISSUE_E_CUDA;
  cudaFree(t->d_trace_len);
  t->d_trace = nullptr;
  t->d_trace_len = nullptr;
  t->trace_cap = 0;
  return upload_view(t);
}

void tissue_destroy(tissue* t) {
  if (!t) return;
  cudaStreamSynchronize(t->stream);
  if (t->d_trace_len) cudaFree(t->d_trace_len);
  cudaFree(t->scratch);
  delete t;
}

int tissue_selftest_time(uint64_t n_samples, uint64_t seed, uint64_t* mismatches) {
  if (!mismatches) return TISSUE_E_ARG;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, sizeof(*d)) != cudaSuccess) {
    cudaGetLastError();
    return TISSUE_E_NOMEM;
  }
  unsigned long long h = 0;
  int rc = TISSUE_OK;
  if (cudaMemset(d, 0, sizeof(*d)) != cudaSuccess ||
      launch_selftest_time(n_samples, seed, d, nullptr) != cudaSuccess ||
      cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = TISSUE_E_CUDA;
  cudaFree(d);
  *mismatches = h;
  return rc;
}

int tissue_debug_fail_allocs(uint32_t n) {
  g_fail_allocs.store(n);
  return TISSUE_OK;
}

const char* tissue_strerror(int code) {
  switch (code) {
    case TISSUE_OK: return "ok";
    case TISSUE_E_ARG: return "invalid argument";
    case TISSUE_E_NOMEM: return "out of device memory";
    case TISSUE_E_NOMODEL: return "no model set";
    case TISSUE_E_OVERFLOW: return "count or propensity overflow";
    case TISSUE_E_CUDA: return "CUDA runtime error";
    case TISSUE_E_TIMEOUT: return "device wait timed out";
    case TISSUE_E_BUDGET: return "memory budget exceeded";
    case TISSUE_E_STATE: return "more bound promoter sites than sites";
    case TISSUE_E_BOUNDS: return "an index out of range (checked build)";
    default: return "unknown error";
  }
}

}  // extern "C"
