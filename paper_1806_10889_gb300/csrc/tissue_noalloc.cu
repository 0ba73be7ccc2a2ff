// tissue_step_noalloc: splitting steps without any device allocation.
//
// The regular entry points allocate a small scratch area per tissue with
// cudaMalloc (Hill table, step counter, error flag, cumulative event
// counters).  Some callers cannot do that: an application that hands this
// library a fixed device-memory budget it manages itself, code running where a
// cudaMalloc would stall every stream on the device (cudaMalloc may
// synchronise), or a host framework whose allocator owns all device memory.
// This entry point serves them.  The caller passes the state and the output
// statistics; the scratch lives in one file-scope __device__ array below,
// sized for tissues of up to TISSUE_NOALLOC_MAX_CELLS cells.
//
// The array is a single object per device for the whole process: every call
// on a device uses the same bytes and leaves its contents behind.  Each call
// therefore re-initialises what must start from a known value (error flag,
// step counter, cumulative counters, Hill table) before its kernels run.
// Two calls whose work overlaps on the same device (different streams, or
// different host threads without ordering) race on that memory.
#include <cmath>
#include <mutex>

#include "tissue.h"
#include "tissue_internal.h"

using namespace tsg;

namespace {

struct StaticScratch {
  uint64_t hill[kHillTab];
  uint64_t ev_total[3 * TISSUE_NOALLOC_MAX_CELLS];
  uint32_t step;
  int err;
};

// The scratch itself: ~416 KB of device memory on every device that loads
// this library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(StaticScratch)];

// Device address of g_noalloc_scratch per device.  In host code the symbol
// name is only a host-side stand-in; the device address comes from
// cudaGetSymbolAddress, taken once per device with that device current.
constexpr int kMaxDevices = 128;
std::mutex g_setup_mu;
StaticScratch* g_scratch_addr[kMaxDevices] = {};

int scratch_on_current_device(StaticScratch** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TISSUE_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return TISSUE_E_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
      return TISSUE_E_CUDA;
    g_scratch_addr[dev] = static_cast<StaticScratch*>(p);
  }
  *out = g_scratch_addr[dev];
  return TISSUE_OK;
}

bool finite_rate(double x) { return std::isfinite(x) && x >= 0.0 && x < 1048576.0; }

}  // namespace

extern "C" int tissue_step_noalloc(const tissue_desc* d, const tissue_model* m,
                                   int32_t* dev_counts, uint32_t step_index, double dt,
                                   uint32_t n_steps, uint64_t* dev_n_events, double* dev_t_last,
                                   void* cuda_stream) {
  if (!d || !m || !dev_counts || !dev_n_events || !dev_t_last) return TISSUE_E_ARG;
  if (d->width < 1 || d->height < 1 || d->n < 2 || d->n > 32) return TISSUE_E_ARG;
  if (d->tissue_id >= (1u << 24)) return TISSUE_E_ARG;
  const uint64_t cells = static_cast<uint64_t>(d->width) * d->height;
  if (cells > TISSUE_NOALLOC_MAX_CELLS) return TISSUE_E_ARG;  // beyond the static scratch
  if (reinterpret_cast<uintptr_t>(dev_counts) % 16 != 0) return TISSUE_E_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return TISSUE_E_ARG;
  const double r[12] = {m->kD, m->K, m->kN, m->gD, m->gN, m->gR,
                        m->hopD, m->hopN, m->hopR, m->k_in, m->k_off, m->k_bind};
  for (double x : r)
    if (!finite_rate(x)) return TISSUE_E_ARG;
  if (!(m->K > 0.0)) return TISSUE_E_ARG;

  StaticScratch* s = nullptr;
  int rc = scratch_on_current_device(&s);
  if (rc != TISSUE_OK) return rc;
  // Like tissue_step, zero steps do nothing: the outputs keep their contents.
  // The address lookup above has been made, so such a call also serves as the
  // device's set-up call.
  if (n_steps == 0) return TISSUE_OK;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

  QRates q{};
  if (!make_qrates(r, s->hill, &q)) return TISSUE_E_ARG;

  TissueView v{};
  v.counts = dev_counts;
  v.width = d->width;
  v.height = d->height;
  v.n = d->n;
  v.V = d->n * d->n;
  v.magic = (65536u + d->n - 1) / d->n;
  v.tissue_id = d->tissue_id;
  v.seed = d->seed;
  v.q = q;
  v.ev_last = dev_n_events;
  v.t_last = dev_t_last;
  v.ev_total = s->ev_total;
  v.step = &s->step;
  v.err = &s->err;

  // Reset everything the kernels read before they write: the previous call's
  // values are still in the array.  The outputs are cleared too, because the
  // face rows of cells that own no face are never written by the kernels.
  const size_t stat_bytes = 3 * static_cast<size_t>(cells) * sizeof(uint64_t);
  if (cudaMemsetAsync(s->ev_total, 0, stat_bytes, stream) != cudaSuccess ||
      cudaMemsetAsync(&s->step, 0, sizeof(uint32_t), stream) != cudaSuccess ||
      cudaMemsetAsync(&s->err, 0, sizeof(int), stream) != cudaSuccess ||
      cudaMemsetAsync(dev_n_events, 0, stat_bytes, stream) != cudaSuccess ||
      cudaMemsetAsync(dev_t_last, 0, 3 * static_cast<size_t>(cells) * sizeof(double), stream) !=
          cudaSuccess)
    return TISSUE_E_CUDA;
  if (launch_step_advance(&s->step, step_index, stream) != cudaSuccess) return TISSUE_E_CUDA;
  if (launch_hill_table(q, s->hill, stream) != cudaSuccess) return TISSUE_E_CUDA;
  for (uint32_t i = 0; i < n_steps; ++i) {
    if (launch_chi(v, i, dt, 4, stream) != cudaSuccess) return TISSUE_E_CUDA;
    if (launch_sig(v, 0, kTagSx, i, dt, stream) != cudaSuccess) return TISSUE_E_CUDA;
    if (launch_sig(v, 1, kTagSy, i, dt, stream) != cudaSuccess) return TISSUE_E_CUDA;
  }
  int flag = 0;
  if (cudaMemcpyAsync(&flag, &s->err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
    return TISSUE_E_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return TISSUE_E_CUDA;
  if (flag & kErrBounds) return TISSUE_E_BOUNDS;
  if (flag & kErrInternal) return TISSUE_E_CUDA;
  return flag ? TISSUE_E_OVERFLOW : TISSUE_OK;
}
