// K_chi for well-mixed cells: the coarse single-cell module of a
// mixed-fidelity tissue (arXiv 1806.10889, Sec. IV: detailed modules where
// cells signal, coarser ones where they do not).  The cells are taken from
// a list of (tissue, cell) items, one warp per item; the lattice cells of the
// same tissues run in the persistent lattice kernel, launched after this one
// on the same stream.
//
// A well-mixed cell keeps the voxel layout between module calls: this chi
// sums the voxels (the translation S -> chi), simulates the totals, and
// places the molecules again (chi -> S), so the face kernels and every
// reader see one format.
#include "tissue_dev.cuh"

namespace tsg {

namespace {

// chi of one well-mixed cell by one warp: totals of the cell's voxels
// (coalesced loads, a warp reduction), the direct-method SSA on the totals
// with compartment rates, then every molecule placed in a uniformly random
// voxel (Philox tags 7..9; the bound promoter stays on its voxel) by shared-
// memory atomics, written back coalesced.  A well-mixed cell has about a
// hundred times fewer events than a lattice cell (no hops), so every lane
// runs the same scalar event loop.  On an error the cell is left unchanged.
__device__ __forceinline__ void wm_cell(const TissueView& t, const uint32_t cell, const int sl,
                                        int32_t* cnt, const int vmax, const uint32_t step_off,
                                        const double dt) {
  constexpr int H = 32;
  const int V = static_cast<int>(t.V), n = static_cast<int>(t.n);
  const int centre = (n >> 1) * n + (n >> 1);
  const bool pm = t.q.kind == kModelPromoter;
  const QRates& q = t.q;
  if (kChecked && (V > vmax || cell >= t.width * t.height)) {
    // checked build: the cell does not fit the launch or is not in its tissue
    if (sl == 0) atomicOr(t.err, kErrBounds);
    __syncwarp(kFull);
    return;
  }
  bool oob = false;  // checked build (see TSG_IDX)
  int32_t* g = t.counts + static_cast<size_t>(cell) * 3 * V;
  const uint32_t step = *t.step + step_off;
  const uint32_t key0 = static_cast<uint32_t>(t.seed), key1 = static_cast<uint32_t>(t.seed >> 32);
  uint64_t D = 0, N = 0, R = 0;
  bool bad = false;
  for (int v = sl; v < V; v += H) {
    const int32_t r = g[2 * V + v];
    D += static_cast<uint32_t>(g[v]);
    N += static_cast<uint32_t>(g[V + v]);
    R += static_cast<uint32_t>(r);
    if (pm && r > static_cast<int32_t>(v == centre)) bad = true;
  }
#pragma unroll
  for (int o = H / 2; o > 0; o >>= 1) {
    D += __shfl_xor_sync(kFull, D, o, H);
    N += __shfl_xor_sync(kFull, N, o, H);
    R += __shfl_xor_sync(kFull, R, o, H);
  }
  int err = __any_sync(kFull, bad) ? kErrState : 0;
  const uint64_t cmax = static_cast<uint64_t>(kCountMax);
  if (!err && (D > cmax || N > cmax || R > cmax)) err = kErrOverflow;
  const double Vd = static_cast<double>(V);
  const uint64_t k17 =
      __double2ull_rn(__dmul_rn(__ddiv_rn(pm ? q.ka_raw : q.k_in_raw, Vd), 4294967296.0));
  const uint32_t word3 = t.tissue_id | (kTagChi << 24);
  double tnow = 0.0;
  uint32_t e = 0;
  while (!err) {
    uint64_t a[7];
    bool ovf = false;
    if (pm) {  // transcription, unbinding, decay D, decay N, binding
      const uint64_t F = 1ull - R;
      a[0] = q.tD * F;
      a[1] = q.kd * R;
      a[2] = mul_lim(q.gD, D, ovf);
      a[3] = mul_lim(q.gN, N, ovf);
      a[4] = mul_lim(k17, N * F, ovf);
      a[5] = a[6] = 0ull;
    } else {   // Hill production, N production, decays, D + N -> R, R -> D + N
      const double x = __ddiv_rn(static_cast<double>(R), __dmul_rn(Vd, q.K));
      const double val = __ddiv_rn(__dmul_rn(Vd, q.kD), __dadd_rn(1.0, __dmul_rn(x, x)));
      a[0] = __double2ull_rn(__dmul_rn(val, 4294967296.0));
      a[1] = q.kN * static_cast<uint64_t>(V);
      a[2] = mul_lim(q.gD, D, ovf);
      a[3] = mul_lim(q.gN, N, ovf);
      a[4] = mul_lim(q.gR, R, ovf);
      a[5] = mul_lim(k17, D * N, ovf);
      a[6] = mul_lim(q.k_off, R, ovf);
    }
    uint64_t A = 0;
#pragma unroll
    for (int j = 0; j < 7; ++j) A += a[j];
    if (ovf || (A >> 52) != 0ull) {
      err = kErrOverflow;
      break;
    }
    if (A == 0ull) break;
    uint64_t Em, Rb;
    int Ek;
    draw_event(e, step, cell, word3, key0, key1, Em, Ek, Rb);
    const double tn = __dadd_rn(tnow, tau_from(F53{Em, Ek}, Ek < 0, A));
    if (!before(tn, dt)) break;
    tnow = tn;
    uint64_t r = __umul64hi(Rb, A);
    int j = 0;
    while (j < 6 && r >= a[j]) {
      r -= a[j];
      ++j;
    }
    if (sl == 0) trace_event(t, step, kTagChi, cell, e, tnow, 0u, static_cast<uint32_t>(j));
    // effects on (D, N, R) of each channel
    int dD, dN, dR;
    if (pm) {
      dD = j == 0 ? 1 : j == 2 ? -1 : 0;
      dN = j == 1 ? 1 : (j == 3 || j == 4) ? -1 : 0;
      dR = j == 1 ? -1 : j == 4 ? 1 : 0;
    } else {
      dD = (j == 0 || j == 6) ? 1 : (j == 2 || j == 5) ? -1 : 0;
      dN = (j == 1 || j == 6) ? 1 : (j == 3 || j == 5) ? -1 : 0;
      dR = j == 5 ? 1 : (j == 4 || j == 6) ? -1 : 0;
    }
    D += static_cast<uint64_t>(static_cast<int64_t>(dD));
    N += static_cast<uint64_t>(static_cast<int64_t>(dN));
    R += static_cast<uint64_t>(static_cast<int64_t>(dR));
    if (D > cmax || N > cmax || R > cmax) err = kErrOverflow;
    ++e;
    if (e == 0xFFFFFFFFu) err |= kErrEventIndex;
  }
  if (!err) {
    for (int sp = 0; sp < 3; ++sp)
      for (int v = sl; v < V; v += H) cnt[sp * vmax + v] = 0;
    __syncwarp(kFull);
    for (int sp = 0; sp < 3; ++sp) {
      const uint64_t T = sp == 0 ? D : sp == 1 ? N : R;
      if (pm && sp == 2) {
        if (sl == 0) cnt[2 * vmax + TSG_IDX(centre, vmax, oob)] = static_cast<int32_t>(T);
        continue;
      }
      const uint32_t w3 = t.tissue_id | ((kTagPlace + static_cast<uint32_t>(sp)) << 24);
      for (uint64_t blk = static_cast<uint64_t>(sl); 4 * blk < T; blk += H) {
        const U4 w = philox10(static_cast<uint32_t>(blk), step, cell, w3, key0, key1);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (4 * blk + k < T)
            atomicAdd(&cnt[sp * vmax + TSG_IDX(static_cast<int>(__umulhi(
                                                        ws[k], static_cast<uint32_t>(V))),
                                                    vmax, oob)],
                      1);
      }
    }
    __syncwarp(kFull);
    for (int sp = 0; sp < 3; ++sp)
      for (int v = sl; v < V; v += H) g[sp * V + v] = cnt[sp * vmax + v];
  }
  if (kChecked && __any_sync(kFull, oob)) err |= kErrBounds;
  if (sl == 0) {
    t.ev_last[cell] = e;
    t.t_last[cell] = tnow;
    t.ev_total[cell] += e;
    if (err) atomicOr(t.err, err);
  }
  __syncwarp(kFull);
}

constexpr int kWmWarps = 4;

__global__ void __launch_bounds__(32 * kWmWarps) k_chi_wm(const TissueView* __restrict__ views,
                                                          const uint2* __restrict__ items,
                                                          const uint32_t n_items,
                                                          const uint32_t vmax,
                                                          const uint32_t step_off,
                                                          const double dt) {
  extern __shared__ __align__(16) int32_t wm_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* cnt = wm_smem + static_cast<size_t>(wib) * 3 * vmax;
  for (uint32_t it = blockIdx.x * kWmWarps + wib; it < n_items; it += gridDim.x * kWmWarps) {
    const uint2 w = items[it];  // whole warp: same item
    wm_cell(views[w.x], w.y, lane, cnt, static_cast<int>(vmax), step_off, dt);
  }
}

}  // namespace

cudaError_t launch_chi_wm(const TissueView* d_views, const uint2* d_items, uint32_t n_items,
                          uint32_t vmax_cells, uint32_t step_off, double dt, cudaStream_t stream) {
  if (n_items == 0) return cudaSuccess;
  const size_t smem = static_cast<size_t>(kWmWarps) * 3 * vmax_cells * sizeof(int32_t);
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024)
    e = cudaFuncSetAttribute(k_chi_wm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const uint32_t want = (n_items + kWmWarps - 1) / kWmWarps;
  const uint32_t blocks = want < 152u * 16u ? want : 152u * 16u;
  k_chi_wm<<<blocks, 32 * kWmWarps, smem, stream>>>(d_views, d_items, n_items, vmax_cells,
                                                     step_off, dt);
  return cudaGetLastError();
}

}  // namespace tsg
