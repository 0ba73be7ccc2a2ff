// K_chi, persistent segmented form: the Notch-Delta-only instantiations and
// the launcher (the kernel template is in chi_seg.cuh; the model-generic and
// promoter-only instantiations are in k_chi_seg_gen.cu and k_chi_seg_pm.cu).
#include "chi_seg.cuh"

namespace tsg {

namespace {

template <int GEN>
ChiSegKernel pick(int H, bool pre, bool qb) {
  if (H == 8) {
    if (!pre) return k_chi_seg<8, false, false, GEN, false>;
    return qb ? k_chi_seg<8, true, true, GEN, false> : k_chi_seg<8, true, false, GEN, false>;
  }
  if (H == 16) {
    if (!pre) return k_chi_seg<16, false, false, GEN, false>;
    return qb ? k_chi_seg<16, true, true, GEN, false> : k_chi_seg<16, true, false, GEN, false>;
  }
  if (!pre) return k_chi_seg<32, false, false, GEN, false>;
  return qb ? k_chi_seg<32, true, true, GEN, false> : k_chi_seg<32, true, false, GEN, false>;
}

}  // namespace

ChiSegKernel chi_seg_kernel_nd(int H, bool pre, bool qb) { return pick<0>(H, pre, qb); }

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
                       cudaStream_t stream) {
  const size_t smem = static_cast<size_t>(warps_per_block) * (32 / H) * seg_bytes;
  const int threads = 32 * warps_per_block;
  // all of an SM's unified memory as shared memory, for every instantiation:
  // two chi launches then share SMs without waiting for a carveout change
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
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
  k<<<blocks, threads, smem, stream>>>(d_views, d_items, n_items, d_counter, seg_bytes, step_off,
                                       dt, redo, redo_n, n_dev);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_chi_seg(const TissueView* d_views, const uint2* d_items, uint32_t n_items,
                           uint32_t* d_counter, uint32_t vmax_cells, int H, int warps_per_block,
                           int blocks, uint32_t step_off, double dt, bool pre, int gen,
                           const ChiRedo* redo, cudaStream_t stream) {
  if (n_items == 0) return cudaSuccess;
  if (H != 8 && H != 16 && H != 32) return cudaErrorInvalidValue;
  if (!pre && warps_per_block > 4) return cudaErrorInvalidValue;
  // B > H (a lane covers several voxels of a block) only when V > H^2; the
  // recompute layout requires V <= H^2.
  const bool qb = vmax_cells > static_cast<uint32_t>(H * H);
  if (!pre && qb) return cudaErrorInvalidValue;
  if (gen < 0 || gen > 2) return cudaErrorInvalidValue;
  const ChiSegKernel k = gen == 2   ? chi_seg_kernel_pm(H, pre, qb)
                         : gen == 1 ? chi_seg_kernel_gen(H, pre, qb)
                                    : chi_seg_kernel_nd(H, pre, qb);
  const uint32_t seg_bytes = seg_bytes_for(vmax_cells, H, pre);
  // Large cells: 16-bit counts first (more cells per SM), then the cells that
  // held or reached a count above 65535 with 32-bit counts, from the state
  // they started the step with.
  const ChiSegKernel kn =
      (redo && pre && gen == 0 && vmax_cells > 256) ? chi_seg_kernel_narrow(H, qb) : nullptr;
  if (!kn)
    return launch_one(k, d_views, d_items, n_items, nullptr, d_counter, seg_bytes, H,
                      warps_per_block, blocks, step_off, dt, nullptr, nullptr, stream);
  cudaError_t e = launch_one(kn, d_views, d_items, n_items, nullptr, d_counter,
                             seg_bytes_for(vmax_cells, H, pre, true), H, warps_per_block, blocks,
                             step_off, dt, redo->items, redo->counters + 1, stream);
  if (e != cudaSuccess) return e;
  return launch_one(k, d_views, redo->items, n_items, redo->counters + 1, redo->counters + 2,
                    seg_bytes, H, warps_per_block, blocks, step_off, dt, nullptr, nullptr, stream);
}

namespace {

// Heavy/light partition of one tissue's cells by their last chi event counts
// (a cell is heavy when its count exceeds 33/32 of the mean; at most `cap`
// cells, the heavy launch's segments, are heavy: the rest stay light so that
// no heavy cell waits for a segment), one block.  It also clears the two
// launches' work counters: counts = {heavy cells, light cells, heavy work
// counter, light work counter}.
__global__ void __launch_bounds__(1024) k_split_cells(const uint64_t* __restrict__ ev_last,
                                                      uint32_t cells, uint32_t cap, uint2* heavy,
                                                      uint2* light, uint32_t* counts) {
  __shared__ unsigned long long part[32];
  __shared__ uint32_t nh, nl;
  if (threadIdx.x == 0) nh = nl = 0u;
  unsigned long long sum = 0;
  for (uint32_t c = threadIdx.x; c < cells; c += blockDim.x) sum += ev_last[c];
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(kFull, sum, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long w = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(kFull, w, o);
    if (threadIdx.x == 0) part[0] = w;
  }
  __syncthreads();
  sum = part[0];
  // exact in 64 bits: cells <= 2^16 and a cell's events per step < 2^32
  for (uint32_t c = threadIdx.x; c < cells; c += blockDim.x) {
    const uint32_t h = 32ull * cells * ev_last[c] > 33ull * sum ? atomicAdd(&nh, 1u) : cap;
    if (h < cap)
      heavy[h] = make_uint2(0u, c);
    else
      light[atomicAdd(&nl, 1u)] = make_uint2(0u, c);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    counts[0] = nh < cap ? nh : cap;
    counts[1] = nl;
    counts[2] = 0u;
    counts[3] = 0u;
  }
}

}  // namespace

bool chi_split_fits(uint32_t V, int H, int warps_per_block, uint32_t cells, int gen) {
  if (H != 16 || V > 256 || cells > 65536u || gen == 1) return false;
  const ChiSegKernel k = gen == 2 ? chi_seg_kernel_pm(16, true, false) : chi_seg_kernel_nd(16, true, false);
  const size_t smem =
      static_cast<size_t>(warps_per_block) * 2 * seg_bytes_for(V, 16, true);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * warps_per_block, smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  // one wave: every cell has a segment from the start
  return static_cast<uint64_t>(cells) <= static_cast<uint64_t>(sms) * per_sm * warps_per_block * 2;
}

cudaError_t launch_chi_seg_split(const TissueView* d_view, const uint64_t* ev_last, uint32_t cells,
                                 uint2* heavy_items, uint2* light_items, uint32_t* counters,
                                 uint32_t V, int warps_per_block, uint32_t step_off, double dt,
                                 int gen, cudaStream_t stream, cudaStream_t side, cudaEvent_t fork,
                                 cudaEvent_t join) {
  if (cells == 0) return cudaSuccess;
  // heavy cells, one per warp, on a grid of cells/8 segments (2 per block)
  const uint32_t heavy_cap = cells / 8 > 0 ? cells / 8 : 1;
  k_split_cells<<<1, 1024, 0, stream>>>(ev_last, cells, heavy_cap, heavy_items, light_items,
                                        counters);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const ChiSegKernel k32 = gen == 2 ? chi_seg_kernel_pm(32, true, false) : chi_seg_kernel_nd(32, true, false);
  const ChiSegKernel k16 = gen == 2 ? chi_seg_kernel_pm(16, true, false) : chi_seg_kernel_nd(16, true, false);
  if ((e = cudaEventRecord(fork, stream)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess)
    return e;
  e = launch_one(k32, d_view, heavy_items, heavy_cap, counters, counters + 2,
                 seg_bytes_for(V, 32, true), 32, 2, 0, step_off, dt, nullptr, nullptr, side);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventRecord(join, side)) != cudaSuccess) return e;
  e = launch_one(k16, d_view, light_items, cells, counters + 1, counters + 3,
                 seg_bytes_for(V, 16, true), 16, warps_per_block, 0, step_off, dt, nullptr,
                 nullptr, stream);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(stream, join, 0);
}

}  // namespace tsg
