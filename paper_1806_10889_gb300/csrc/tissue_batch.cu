// tissue_batch: many tissues advanced by one persistent launch per step.
//
// Each member keeps its own state buffer, statistics and step counter; the
// batch holds a device table of the members' views, the chi work list of
// every cell-size class (V) and the face lists of both phases.  One
// splitting step is: for every class, the persistent chi kernel over the
// class's (tissue, cell) items; then one face kernel over all x-faces of all
// members, one over all y-faces; then every member's step counter advances.
// The step is captured once in a CUDA graph per dt and replayed, so a batch
// step costs a handful of graph launches regardless of how many tissues it
// holds.  Work items never enter the random streams (which are keyed by a
// tissue's seed, id, cell and step), so a tissue's trajectory is the same
// alone and in any batch.
#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <vector>

#include "tissue.h"
#include "tissue_internal.h"

using namespace tsg;

namespace {

struct ClassPlan {
  uint32_t V;
  uint32_t lanes, warps_per_block, layout;
  size_t items_off;  // offset (in uint2) into the item buffer
  uint32_t n_items;
  int gen;           // 0: Notch-Delta only; 2: promoter only; 1: both, or a trace is on
};

}  // namespace

struct tissue_batch {
  std::vector<tissue*> members;
  cudaStream_t stream = nullptr;
  std::vector<ClassPlan> classes;
  unsigned char* dmem = nullptr;
  TissueView* d_views = nullptr;
  uint2* d_items = nullptr;   // chi items of every class, then x-faces, then y-faces
  uint32_t* d_counters = nullptr;  // per class: work counter, redo count, redo-pass work counter
  uint2* d_redo = nullptr;         // cells a class's 16-bit-count pass gives up on
  uint32_t* d_io_steps = nullptr;  // checkpoint writes: the members' new step indices
  int* d_io_err = nullptr;         // checkpoint reads: the members' error flags
  int* d_io_bad = nullptr;         // checkpoint writes: a count out of range
  // pinned host staging of the state I/O's small copies (step indices in,
  // error flags out), so none of them goes through pageable memory
  uint32_t* h_io_steps = nullptr;  // count entries
  int* h_io_flags = nullptr;       // count error flags, then the range flag
  size_t xface_off = 0, yface_off = 0, wm_off = 0;
  uint32_t n_xfaces = 0, n_yfaces = 0;
  uint32_t n_wm = 0, wm_vmax = 0;  // well-mixed cells of all members (one launch)
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0.0;
  uint32_t steps_per_graph = 1;
  uint32_t scheme = TISSUE_SPLIT_LIE;
  // timing (tissue_batch_set_timing): events at the step's start and end,
  // before the well-mixed launch and after it, and after each class
  bool timing = false, timed_once = false, timed_overlap = false;
  // [0] step start, [1] step end, [2] chi start, [3] after the well-mixed
  // launch (the classes' start), [4 + i] end of class i, [4 + classes] chi end
  std::vector<cudaEvent_t> tev;
  // Overlapped classes: the largest-cell class runs on the batch stream at
  // the highest launch priority; every other class on a stream of its own at
  // the lowest, forked after the well-mixed launch and joined before the
  // faces, so its blocks take the SMs the large class's last wave frees.
  bool overlap = true;
  std::vector<cudaStream_t> side;  // one per class after the first
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  int prio_hi = 0, prio_lo = 0;
};

namespace {

// Record timing event i on the batch stream (an event-record node when the
// stream is being captured).
int mark(tissue_batch* b, size_t i, cudaStream_t stream) {
  if (!b->timing) return TISSUE_OK;
  return cudaEventRecordWithFlags(b->tev[i], stream, cudaEventRecordExternal) == cudaSuccess
             ? TISSUE_OK
             : TISSUE_E_CUDA;
}

int mark(tissue_batch* b, size_t i) { return mark(b, i, b->stream); }

bool overlapped(const tissue_batch* b) {
  return b->overlap && b->stream != nullptr && b->classes.size() > 1 &&
         b->side.size() + 1 == b->classes.size();
}

int chi_all(tissue_batch* b, double dt) {
  if (mark(b, 2) != TISSUE_OK) return TISSUE_E_CUDA;
  if (b->n_wm && launch_chi_wm(b->d_views, b->d_items + b->wm_off, b->n_wm, b->wm_vmax, 0u, dt,
                               b->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  if (mark(b, 3) != TISSUE_OK) return TISSUE_E_CUDA;
  const size_t nc = b->classes.size();
  const bool ov = overlapped(b);
  if (ov && cudaEventRecord(b->ev_fork, b->stream) != cudaSuccess) return TISSUE_E_CUDA;
  for (size_t c = 0; c < nc; ++c) {
    const ClassPlan& p = b->classes[c];
    const cudaStream_t st = (ov && c > 0) ? b->side[c - 1] : b->stream;
    if (ov && c > 0 && cudaStreamWaitEvent(st, b->ev_fork, 0) != cudaSuccess) return TISSUE_E_CUDA;
    uint32_t* counters = b->d_counters + 3 * c;
    if (cudaMemsetAsync(counters, 0, 3 * sizeof(uint32_t), st) != cudaSuccess)
      return TISSUE_E_CUDA;
    // each class has its own part of the redo list (classes may run at once)
    const ChiRedo redo{b->d_redo + p.items_off, counters};
    // as for single tissues: a counts-only launch with several voxels per
    // lane takes Notch-Delta classes without a trace; others run the prefix
    // launch of the class (the same trajectories)
    tissue_launch lc{TISSUE_KERNEL_PERSISTENT, p.lanes, p.warps_per_block, 0, p.layout};
    if (lc.smem_layout == TISSUE_LAYOUT_RECOMPUTE &&
        !recompute_covers(p.V, static_cast<int>(p.lanes), p.gen))
      lc = prefix_launch(p.V, p.n_items);
    const int prio = ov ? (c == 0 ? b->prio_hi : b->prio_lo) : 0;
    if (launch_chi_seg(b->d_views, b->d_items + p.items_off, p.n_items, counters, p.V,
                       static_cast<int>(lc.lanes_per_cell), static_cast<int>(lc.warps_per_block),
                       0, 0u, dt, lc.smem_layout == TISSUE_LAYOUT_PREFIX, p.gen, &redo, st,
                       prio) != cudaSuccess)
      return TISSUE_E_CUDA;
    if (mark(b, 4 + c, st) != TISSUE_OK) return TISSUE_E_CUDA;
    if (ov && c > 0 && cudaEventRecord(b->ev_join[c - 1], st) != cudaSuccess)
      return TISSUE_E_CUDA;
  }
  if (ov)
    for (size_t c = 1; c < nc; ++c)
      if (cudaStreamWaitEvent(b->stream, b->ev_join[c - 1], 0) != cudaSuccess)
        return TISSUE_E_CUDA;
  if (mark(b, 4 + nc) != TISSUE_OK) return TISSUE_E_CUDA;
  if (b->timing) b->timed_overlap = ov;
  return TISSUE_OK;
}

int faces(tissue_batch* b, int axis, uint32_t tag, double dt) {
  const uint2* items = b->d_items + (axis == 0 ? b->xface_off : b->yface_off);
  const uint32_t n = axis == 0 ? b->n_xfaces : b->n_yfaces;
  return launch_sig_list(b->d_views, items, n, axis, tag, dt, b->stream) == cudaSuccess
             ? TISSUE_OK
             : TISSUE_E_CUDA;
}

int enqueue_step(tissue_batch* b, double dt) {
  int rc;
  if ((rc = mark(b, 0))) return rc;
  if (b->scheme == TISSUE_SPLIT_LIE) {
    if ((rc = chi_all(b, dt)) || (rc = faces(b, 0, kTagSx, dt)) || (rc = faces(b, 1, kTagSy, dt)))
      return rc;
  } else {
    const double h = dt * 0.5;
    if ((rc = faces(b, 0, kTagSx, h)) || (rc = faces(b, 1, kTagSy, h)) || (rc = chi_all(b, dt)) ||
        (rc = faces(b, 1, kTagSy2, h)) || (rc = faces(b, 0, kTagSx2, h)))
      return rc;
  }
  if (launch_advance_list(b->d_views, static_cast<uint32_t>(b->members.size()), b->stream) !=
      cudaSuccess)
    return TISSUE_E_CUDA;
  if ((rc = mark(b, 1))) return rc;
  if (b->timing) b->timed_once = true;
  return TISSUE_OK;
}

void drop_events(tissue_batch* b) {
  for (cudaEvent_t e : b->tev) cudaEventDestroy(e);
  b->tev.clear();
}

// The side streams and fork/join events of overlapped classes.
void drop_side(tissue_batch* b) {
  for (cudaStream_t st : b->side) cudaStreamDestroy(st);
  b->side.clear();
  for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
  b->ev_join.clear();
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  b->ev_fork = nullptr;
}

bool make_side(tissue_batch* b) {
  if (b->classes.size() < 2) return true;
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return false;
  b->prio_lo = least;
  b->prio_hi = greatest;
  if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) return false;
  for (size_t c = 1; c < b->classes.size(); ++c) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, least) != cudaSuccess)
      return false;
    b->side.push_back(st);
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return false;
    b->ev_join.push_back(ev);
  }
  return true;
}

void drop_graph(tissue_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

}  // namespace

extern "C" {

int tissue_batch_create(tissue* const* members, uint32_t count, void* cuda_stream,
                        tissue_batch** out) {
  if (!out) return TISSUE_E_ARG;
  *out = nullptr;
  if (!members || count == 0) return TISSUE_E_ARG;
  std::vector<TissueInfo> info(count);
  for (uint32_t i = 0; i < count; ++i) {
    if (!tissue_info(members[i], &info[i])) return TISSUE_E_ARG;
    if (!info[i].has_model) return TISSUE_E_NOMODEL;
    for (uint32_t j = 0; j < i; ++j)
      if (members[j] == members[i]) return TISSUE_E_ARG;  // a tissue may appear once
  }
  tissue_batch* b = new (std::nothrow) tissue_batch();
  if (!b) return TISSUE_E_NOMEM;
  b->members.assign(members, members + count);
  b->stream = static_cast<cudaStream_t>(cuda_stream);

  // chi items by class, largest cells first; faces of both phases
  std::map<uint32_t, std::vector<uint2>, std::greater<uint32_t>> by_v;
  std::map<uint32_t, int> nd_v, pm_v, tr_v;  // per class: members of each model, traced
  std::vector<uint2> xf, yf, wm_items;
  for (uint32_t i = 0; i < count; ++i) {
    const tissue_desc& d = info[i].desc;
    const uint32_t V = d.n * d.n, cells = d.width * d.height;
    std::vector<uint2>& list = by_v[V];
    (info[i].view.q.kind == kModelPromoter ? pm_v : nd_v)[V] += 1;
    if (info[i].view.trace != nullptr) tr_v[V] += 1;
    const uint8_t* wm = info[i].wm_host;
    for (uint32_t c = 0; c < cells; ++c) {
      if (wm && wm[c]) {
        wm_items.push_back(make_uint2(i, c));
        b->wm_vmax = std::max(b->wm_vmax, V);
      } else {
        list.push_back(make_uint2(i, c));
      }
    }
    for (uint32_t c = 0; c < cells; ++c) {
      const uint32_t cx = c % d.width, cy = c / d.width;
      if (cx + 1 < d.width) xf.push_back(make_uint2(i, c));
      if (cy + 1 < d.height) yf.push_back(make_uint2(i, c));
    }
  }
  std::vector<uint2> items;
  for (auto& kv : by_v) {
    if (kv.second.empty()) continue;  // every cell of this size is well-mixed
    ClassPlan p{};
    p.V = kv.first;
    const tissue_launch dl = default_launch(kv.first, kv.second.size());
    p.lanes = dl.lanes_per_cell;
    p.warps_per_block = dl.warps_per_block;
    p.layout = dl.smem_layout;
    p.items_off = items.size();
    p.n_items = static_cast<uint32_t>(kv.second.size());
    const uint32_t V = kv.first;
    p.gen = (nd_v[V] == 0 && pm_v[V] > 0) ? 2 : (pm_v[V] > 0 || tr_v[V] > 0) ? 1 : 0;
    items.insert(items.end(), kv.second.begin(), kv.second.end());
    b->classes.push_back(p);
  }
  b->wm_off = items.size();
  b->n_wm = static_cast<uint32_t>(wm_items.size());
  items.insert(items.end(), wm_items.begin(), wm_items.end());
  b->xface_off = items.size();
  b->n_xfaces = static_cast<uint32_t>(xf.size());
  items.insert(items.end(), xf.begin(), xf.end());
  b->yface_off = items.size();
  b->n_yfaces = static_cast<uint32_t>(yf.size());
  items.insert(items.end(), yf.begin(), yf.end());

  const size_t views_bytes = (sizeof(TissueView) * count + 255) & ~static_cast<size_t>(255);
  const size_t items_bytes = (sizeof(uint2) * items.size() + 255) & ~static_cast<size_t>(255);
  size_t redo_items = 0;  // every class has its part (at its items' offset)
  for (const ClassPlan& p : b->classes) redo_items = std::max<size_t>(redo_items, p.items_off + p.n_items);
  const size_t redo_bytes = (sizeof(uint2) * redo_items + 255) & ~static_cast<size_t>(255);
  const size_t io_bytes = (2 * sizeof(uint32_t) * count + 255) & ~static_cast<size_t>(255);
  const size_t counters_bytes =
      (3 * sizeof(uint32_t) * b->classes.size() + 255) & ~static_cast<size_t>(255);
  const size_t total = views_bytes + items_bytes + redo_bytes + counters_bytes + io_bytes + 256;
  if (lib_malloc(reinterpret_cast<void**>(&b->dmem), total) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return TISSUE_E_NOMEM;
  }
  b->d_views = reinterpret_cast<TissueView*>(b->dmem);
  b->d_items = reinterpret_cast<uint2*>(b->dmem + views_bytes);
  b->d_redo = reinterpret_cast<uint2*>(b->dmem + views_bytes + items_bytes);
  b->d_counters = reinterpret_cast<uint32_t*>(b->dmem + views_bytes + items_bytes + redo_bytes);
  unsigned char* io = b->dmem + views_bytes + items_bytes + redo_bytes + counters_bytes;
  b->d_io_steps = reinterpret_cast<uint32_t*>(io);
  b->d_io_err = reinterpret_cast<int*>(io + sizeof(uint32_t) * count);
  b->d_io_bad = reinterpret_cast<int*>(io + io_bytes);
  if (cudaMallocHost(reinterpret_cast<void**>(&b->h_io_steps), sizeof(uint32_t) * count) !=
          cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&b->h_io_flags), sizeof(int) * (count + 1)) !=
          cudaSuccess) {
    cudaGetLastError();
    if (b->h_io_steps) cudaFreeHost(b->h_io_steps);
    cudaFree(b->dmem);
    delete b;
    return TISSUE_E_NOMEM;
  }
  std::vector<TissueView> views(count);
  for (uint32_t i = 0; i < count; ++i) views[i] = info[i].view;
  // Members' pending work (creation, earlier steps) must finish before the
  // batch stream uses their buffers.
  auto fail = [b]() {
    drop_side(b);
    cudaFreeHost(b->h_io_steps);
    cudaFreeHost(b->h_io_flags);
    cudaFree(b->dmem);
    delete b;
    return TISSUE_E_CUDA;
  };
  if (!make_side(b)) return fail();
  for (uint32_t i = 0; i < count; ++i)
    if (cudaStreamSynchronize(info[i].stream) != cudaSuccess) return fail();
  if (cudaMemcpy(b->d_views, views.data(), sizeof(TissueView) * count, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(b->d_items, items.data(), sizeof(uint2) * items.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return fail();
  *out = b;
  return TISSUE_OK;
}

int tissue_batch_set_class_launch(tissue_batch* b, uint32_t V, uint32_t lanes_per_cell,
                                  uint32_t warps_per_block, uint32_t smem_layout) {
  if (!b) return TISSUE_E_ARG;
  if (lanes_per_cell != 8 && lanes_per_cell != 16 && lanes_per_cell != 32) return TISSUE_E_ARG;
  if (smem_layout != TISSUE_LAYOUT_PREFIX && smem_layout != TISSUE_LAYOUT_RECOMPUTE)
    return TISSUE_E_ARG;
  if (smem_layout == TISSUE_LAYOUT_RECOMPUTE &&
      !recompute_covers(V, static_cast<int>(lanes_per_cell), 0))
    return TISSUE_E_ARG;
  const bool pre = smem_layout == TISSUE_LAYOUT_PREFIX;
  if (warps_per_block < 1 || warps_per_block > (pre ? 8u : 4u)) return TISSUE_E_ARG;
  if (static_cast<size_t>(warps_per_block) * (32 / lanes_per_cell) *
          seg_bytes_for(V, static_cast<int>(lanes_per_cell), pre) > 227 * 1024)
    return TISSUE_E_ARG;
  for (ClassPlan& p : b->classes)
    if (p.V == V) {
      p.lanes = lanes_per_cell;
      p.warps_per_block = warps_per_block;
      p.layout = smem_layout;
      drop_graph(b);
      return TISSUE_OK;
    }
  return TISSUE_E_ARG;
}

int tissue_batch_step(tissue_batch* b, double dt, uint32_t n_steps) {
  NvtxRange range("tissue_batch_step");
  if (!b) return TISSUE_E_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return TISSUE_E_ARG;
  if (n_steps == 0) return TISSUE_OK;
  if (!b->graph || b->graph_dt != dt) {
    drop_graph(b);
    // A legacy default stream cannot be captured: fall back to direct launches.
    if (b->stream == nullptr) {
      for (uint32_t s = 0; s < n_steps; ++s) {
        const int rc = enqueue_step(b, dt);
        if (rc != TISSUE_OK) return rc;
      }
      for (tissue* m : b->members) tissue_advance_host_step(m, n_steps);
      return TISSUE_OK;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return TISSUE_E_CUDA;
    int rc = TISSUE_OK;
    for (uint32_t s = 0; s < b->steps_per_graph && rc == TISSUE_OK; ++s) rc = enqueue_step(b, dt);
    const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
    if (rc != TISSUE_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return TISSUE_E_CUDA;
    }
    // node priorities: the overlapped large-cell class goes first
    const cudaError_t ie =
        cudaGraphInstantiateWithFlags(&b->graph, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      b->graph = nullptr;
      return TISSUE_E_CUDA;
    }
    b->graph_dt = dt;
  }
  // whole graphs, then single steps for the remainder
  const uint32_t k = b->steps_per_graph;
  for (uint32_t s = 0; s + k <= n_steps; s += k)
    if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return TISSUE_E_CUDA;
  for (uint32_t s = n_steps - n_steps % k; s < n_steps; ++s) {
    const int rc = enqueue_step(b, dt);
    if (rc != TISSUE_OK) return rc;
  }
  for (tissue* m : b->members) tissue_advance_host_step(m, n_steps);
  return TISSUE_OK;
}

int tissue_batch_set_schedule(tissue_batch* b, uint32_t steps_per_graph) {
  if (!b || steps_per_graph < 1 || steps_per_graph > 64) return TISSUE_E_ARG;
  if (steps_per_graph != b->steps_per_graph) drop_graph(b);
  b->steps_per_graph = steps_per_graph;
  return TISSUE_OK;
}

int tissue_batch_set_splitting(tissue_batch* b, uint32_t scheme) {
  if (!b || (scheme != TISSUE_SPLIT_LIE && scheme != TISSUE_SPLIT_STRANG)) return TISSUE_E_ARG;
  if (scheme != b->scheme) drop_graph(b);
  b->scheme = scheme;
  return TISSUE_OK;
}

int tissue_batch_sync(tissue_batch* b) {
  if (!b) return TISSUE_E_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TISSUE_E_CUDA;
  int worst = TISSUE_OK;
  for (tissue* m : b->members) {
    const int rc = tissue_sync(m);
    if (rc != TISSUE_OK) worst = rc;
  }
  return worst;
}

int tissue_batch_write_counts(tissue_batch* b, const int32_t* const* host,
                              const uint32_t* step_index) {
  NvtxRange range("tissue_batch_write_counts");
  if (!b || !host) return TISSUE_E_ARG;
  const uint32_t n = static_cast<uint32_t>(b->members.size());
  for (uint32_t i = 0; i < n; ++i)
    if (!host[i]) return TISSUE_E_ARG;
  for (uint32_t i = 0; i < n; ++i) {
    TissueInfo info;
    if (!tissue_info(b->members[i], &info)) return TISSUE_E_ARG;
    if (cudaMemcpyAsync(info.view.counts, host[i], tissue_state_bytes(&info.desc),
                        cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
      return TISSUE_E_CUDA;
  }
  if (step_index) {
    // the previous call's copies out of the staging area are complete: every
    // call ends with a wait on the batch stream
    std::copy(step_index, step_index + n, b->h_io_steps);
    if (cudaMemcpyAsync(b->d_io_steps, b->h_io_steps, sizeof(uint32_t) * n,
                        cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
      return TISSUE_E_CUDA;
  }
  if (cudaMemsetAsync(b->d_io_bad, 0, sizeof(int), b->stream) != cudaSuccess ||
      launch_set_steps_list(b->d_views, step_index ? b->d_io_steps : nullptr, n, b->stream) !=
          cudaSuccess ||
      launch_check_counts_list(b->d_views, n, b->d_io_bad, b->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  if (cudaMemcpyAsync(b->h_io_flags + n, b->d_io_bad, sizeof(int), cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  const int bad = b->h_io_flags[n];
  if (step_index)
    for (uint32_t i = 0; i < n; ++i) tissue_set_host_step(b->members[i], step_index[i]);
  return bad ? TISSUE_E_ARG : TISSUE_OK;
}

int tissue_batch_read_counts(tissue_batch* b, int32_t* const* host) {
  NvtxRange range("tissue_batch_read_counts");
  if (!b || !host) return TISSUE_E_ARG;
  const uint32_t n = static_cast<uint32_t>(b->members.size());
  for (uint32_t i = 0; i < n; ++i)
    if (!host[i]) return TISSUE_E_ARG;
  for (uint32_t i = 0; i < n; ++i) {
    TissueInfo info;
    if (!tissue_info(b->members[i], &info)) return TISSUE_E_ARG;
    if (cudaMemcpyAsync(host[i], info.view.counts, tissue_state_bytes(&info.desc),
                        cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
      return TISSUE_E_CUDA;
  }
  if (launch_gather_err_list(b->d_views, n, b->d_io_err, b->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  if (cudaMemcpyAsync(b->h_io_flags, b->d_io_err, sizeof(int) * n, cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  for (uint32_t i = 0; i < n; ++i)
    if (b->h_io_flags[i]) return error_code_of(b->h_io_flags[i]);
  return TISSUE_OK;
}

int tissue_batch_class_info(const tissue_batch* b, uint32_t i, uint32_t* V,
                            uint32_t* lanes_per_cell, uint32_t* warps_per_block,
                            uint32_t* smem_layout, uint32_t* cells) {
  if (!b || i >= b->classes.size()) return TISSUE_E_ARG;
  const ClassPlan& p = b->classes[i];
  if (V) *V = p.V;
  if (lanes_per_cell) *lanes_per_cell = p.lanes;
  if (warps_per_block) *warps_per_block = p.warps_per_block;
  if (smem_layout) *smem_layout = p.layout;
  if (cells) *cells = p.n_items;
  return TISSUE_OK;
}

int tissue_batch_set_timing(tissue_batch* b, uint32_t on) {
  if (!b || on > 1) return TISSUE_E_ARG;
  if ((on != 0) == b->timing) return TISSUE_OK;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TISSUE_E_CUDA;
  drop_graph(b);
  drop_events(b);
  b->timing = false;
  b->timed_once = false;
  if (!on) return TISSUE_OK;
  const size_t n = 5 + b->classes.size();
  for (size_t i = 0; i < n; ++i) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      drop_events(b);
      return TISSUE_E_CUDA;
    }
    b->tev.push_back(e);
  }
  b->timing = true;
  return TISSUE_OK;
}

int tissue_batch_read_timing(tissue_batch* b, double* step_ms, double* chi_ms, double* wm_ms,
                             double* class_ms, uint32_t n) {
  if (!b || !b->timing || !b->timed_once || n > b->classes.size()) return TISSUE_E_ARG;
  if (n > 0 && !class_ms) return TISSUE_E_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TISSUE_E_CUDA;
  float ms = 0.0f;
  auto span = [&](size_t a, size_t z, double* out) -> bool {
    if (!out) return true;
    if (cudaEventElapsedTime(&ms, b->tev[a], b->tev[z]) != cudaSuccess) return false;
    *out = ms;
    return true;
  };
  const size_t nc = b->classes.size();
  if (!span(0, 1, step_ms) || !span(2, 4 + nc, chi_ms) || !span(2, 3, wm_ms)) return TISSUE_E_CUDA;
  for (uint32_t i = 0; i < n; ++i) {
    // a class starts when its launches become ready: after the previous
    // class, or, overlapped, when the classes fork
    const size_t from = (b->timed_overlap || i == 0) ? 3 : 3 + i;
    if (!span(from, 4 + i, class_ms + i)) return TISSUE_E_CUDA;
  }
  return TISSUE_OK;
}

int tissue_batch_set_overlap(tissue_batch* b, uint32_t on) {
  if (!b || on > 1) return TISSUE_E_ARG;
  if ((on != 0) != b->overlap) drop_graph(b);
  b->overlap = on != 0;
  return TISSUE_OK;
}

int tissue_batch_info(const tissue_batch* b, uint32_t* n_members, uint32_t* n_classes,
                      uint64_t* n_cells) {
  if (!b) return TISSUE_E_ARG;
  if (n_members) *n_members = static_cast<uint32_t>(b->members.size());
  if (n_classes) *n_classes = static_cast<uint32_t>(b->classes.size());
  if (n_cells) {
    uint64_t s = b->n_wm;
    for (const ClassPlan& p : b->classes) s += p.n_items;
    *n_cells = s;
  }
  return TISSUE_OK;
}

void tissue_batch_destroy(tissue_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  drop_events(b);
  drop_side(b);
  cudaFreeHost(b->h_io_steps);
  cudaFreeHost(b->h_io_flags);
  cudaFree(b->dmem);
  delete b;
}

}  // extern "C"
