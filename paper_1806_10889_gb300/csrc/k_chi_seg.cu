// K_chi, persistent segmented form: the Notch-Delta-only instantiations and
// the launcher (the kernel template is in chi_seg.cuh; the model-generic and
// promoter-only instantiations are in k_chi_seg_gen.cu and k_chi_seg_pm.cu).
#include "chi_seg.cuh"

namespace tsg {

namespace {

template <int GEN>
ChiSegKernel pick(int H, bool pre, bool qb) {
  if (H == 8) {
    if (!pre) return qb ? k_chi_seg<8, false, true, GEN, false> : k_chi_seg<8, false, false, GEN, false>;
    return qb ? k_chi_seg<8, true, true, GEN, false> : k_chi_seg<8, true, false, GEN, false>;
  }
  if (H == 16) {
    // the counts-only layout with several voxels per lane: Notch-Delta only
    if (!pre) return qb ? k_chi_seg<16, false, true, GEN, false> : k_chi_seg<16, false, false, GEN, false>;
    return qb ? k_chi_seg<16, true, true, GEN, false> : k_chi_seg<16, true, false, GEN, false>;
  }
  if (!pre) return k_chi_seg<32, false, false, GEN, false>;
  return qb ? k_chi_seg<32, true, true, GEN, false> : k_chi_seg<32, true, false, GEN, false>;
}

}  // namespace

ChiSegKernel chi_seg_kernel_nd(int H, bool pre, bool qb) { return pick<0>(H, pre, qb); }

bool recompute_covers(uint32_t V, int H, int gen) {
  return V <= static_cast<uint32_t>(H * H) ||
         (gen == 0 && ((H == 16 && V <= 1024) || (H == 8 && V <= 256)));
}

int seg_lanes_for(uint32_t V, int want) {
  if (want == 16 && V <= 256) return 16;
  return 32;
}

uint32_t seg_bytes_for(uint32_t V, int H, bool pre, bool narrow) {
  int B = 1;
  while (static_cast<uint32_t>(H * B) < V) B <<= 1;
  const int per_voxel = (pre ? 8 : 0) + (narrow ? 6 : 12);
  return static_cast<uint32_t>(kViewBytes + per_voxel * H * B);
}

namespace {

// One launch of kernel k over items[0 .. n) (n = *n_dev when given; n_items
// bounds it and sizes the grid).
cudaError_t launch_one(ChiSegKernel k, const TissueView* d_views, const uint2* d_items,
                       uint32_t n_items, const uint32_t* n_dev, uint32_t* d_counter,
                       uint32_t seg_bytes, int H, int warps_per_block, int blocks,
                       uint32_t step_off, double dt, uint2* redo, uint32_t* redo_n,
                       cudaStream_t stream, int priority) {
  const size_t smem = static_cast<size_t>(warps_per_block) * (32 / H) * seg_bytes;
  const int threads = 32 * warps_per_block;
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024)
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  if (blocks <= 0) {
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem)) != cudaSuccess)
      return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    blocks = sms * per_sm;
    const uint32_t segs_per_block = static_cast<uint32_t>(warps_per_block * (32 / H));
    const uint32_t need = (n_items + segs_per_block - 1) / segs_per_block;
    if (need < static_cast<uint32_t>(blocks)) blocks = static_cast<int>(need);
  }
  if (priority == 0) {
    k<<<blocks, threads, smem, stream>>>(d_views, d_items, n_items, d_counter, seg_bytes,
                                         step_off, dt, redo, redo_n, n_dev);
    return cudaGetLastError();
  }
  // a launch priority (kept by a captured kernel node as its attribute)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(blocks));
  cfg.blockDim = dim3(static_cast<unsigned>(threads));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = priority;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, d_views, d_items, n_items, d_counter, seg_bytes, step_off, dt,
                            redo, redo_n, n_dev);
}

}  // namespace

cudaError_t launch_chi_seg(const TissueView* d_views, const uint2* d_items, uint32_t n_items,
                           uint32_t* d_counter, uint32_t vmax_cells, int H, int warps_per_block,
                           int blocks, uint32_t step_off, double dt, bool pre, int gen,
                           const ChiRedo* redo, cudaStream_t stream, int priority) {
  if (n_items == 0) return cudaSuccess;
  if (H != 8 && H != 16 && H != 32) return cudaErrorInvalidValue;
  if (!pre && warps_per_block > 4) return cudaErrorInvalidValue;
  // B > H (a lane covers several voxels of a block) only when V > H^2; the
  // recompute layout allows that only for the Notch-Delta model, up to four
  // voxels per lane (16 lanes and V <= 1024, or 8 lanes and V <= 256).
  const bool qb = vmax_cells > static_cast<uint32_t>(H * H);
  if (gen < 0 || gen > 2) return cudaErrorInvalidValue;
  if (!pre && qb && !recompute_covers(vmax_cells, H, gen)) return cudaErrorInvalidValue;
  const ChiSegKernel k = gen == 2   ? chi_seg_kernel_pm(H, pre, qb)
                         : gen == 1 ? chi_seg_kernel_gen(H, pre, qb)
                                    : chi_seg_kernel_nd(H, pre, qb);
  const uint32_t seg_bytes = seg_bytes_for(vmax_cells, H, pre);
  // Large cells: 16-bit counts first (more cells per SM), then the cells that
  // held or reached a count above 65535 with 32-bit counts, from the state
  // they started the step with.
  const ChiSegKernel kn =
      (redo && gen == 0 && vmax_cells > 256) ? chi_seg_kernel_narrow(H, pre, qb) : nullptr;
  if (!kn)
    return launch_one(k, d_views, d_items, n_items, nullptr, d_counter, seg_bytes, H,
                      warps_per_block, blocks, step_off, dt, nullptr, nullptr, stream, priority);
  cudaError_t e = launch_one(kn, d_views, d_items, n_items, nullptr, d_counter,
                             seg_bytes_for(vmax_cells, H, pre, true), H, warps_per_block, blocks,
                             step_off, dt, redo->items, redo->counters + 1, stream, priority);
  if (e != cudaSuccess) return e;
  return launch_one(k, d_views, redo->items, n_items, redo->counters + 1, redo->counters + 2,
                    seg_bytes, H, warps_per_block, blocks, step_off, dt, nullptr, nullptr, stream,
                    priority);
}

}  // namespace tsg
