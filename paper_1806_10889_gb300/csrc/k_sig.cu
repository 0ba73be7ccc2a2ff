// K_sig: the signalling module S (arXiv 1806.10889, Sec. II-A2) for one
// phase of faces, with the translations T_{chi->S} / T_{S->chi} (Sec. II-B)
// fused in: the warp of a face gathers the boundary voxels of both cells
// straight from the state array and writes the result back in place.
//
// A face joins cell c (the owner, the lower id) and its +x (axis 0) or +y
// (axis 1) neighbour.  Lane p holds voxel pair p -- voxel a_p of c on the
// face and voxel b_p of the neighbour facing it -- in registers, with the
// two binding channels D(a)+N(b) -> R(b) and D(b)+N(a) -> R(a) (promoter
// model: the conversions Delta(a) -> NICD(b) and Delta(b) -> NICD(a)).  Within a
// phase no voxel belongs to two faces (the single-face coupling rule,
// Sec. III-A1), so all faces of the phase run concurrently and
// deterministically.  The direct-method SSA runs over [0, dt) exactly as in
// chi, with the face's own Philox stream.
//
// This file also holds the initial-state kernel (Poisson counts by CDF
// inversion), the Hill-production table and the step-counter update.
#include "tissue_dev.cuh"

namespace tsg {

namespace {

// The face owned by cell c on `axis`, advanced over [0, dt) by one warp.
__device__ __forceinline__ void sig_face(const TissueView& t, const uint32_t c, const int axis,
                                         const uint32_t tag, const uint32_t step_off,
                                         const double dt) {
  const int lane = threadIdx.x & 31;
  const uint32_t W = t.width, H = t.height;
  bool oob = false;  // checked build: a cell outside the tissue (see TSG_IDX)
  const uint32_t nb = static_cast<uint32_t>(TSG_IDX(axis == 0 ? c + 1 : c + W, W * H, oob));
  const uint32_t ca = static_cast<uint32_t>(TSG_IDX(c, W * H, oob));
  const int n = static_cast<int>(t.n), V = static_cast<int>(t.V);
  int32_t* ga = t.counts + static_cast<size_t>(ca) * 3 * V;
  int32_t* gb = t.counts + static_cast<size_t>(nb) * 3 * V;
  const bool act = lane < n;
  const int va = axis == 0 ? lane * n + (n - 1) : (n - 1) * n + lane;
  const int vb = axis == 0 ? lane * n : lane;

  uint32_t Da = 0, Na = 0, Ra = 0, Db = 0, Nb = 0, Rb = 0;
  if (act) {
    Da = ga[va];
    Na = ga[V + va];
    Ra = ga[2 * V + va];
    Db = gb[vb];
    Nb = gb[V + vb];
    Rb = gb[2 * V + vb];
  }
  // Notch-Delta: D(a) + N(b) -> R(b) at k_bind D(a) N(b), and the mirror.
  // Promoter model: Delta(a) -> NICD(b) at k_N D(a), and the mirror.
  const bool pm = t.q.kind == kModelPromoter;
  const uint64_t kb = t.q.k_bind;
  bool ovf = false;
  uint64_t c0 = mul_lim(kb, static_cast<uint64_t>(Da) * (pm ? 1u : Nb), ovf);
  uint64_t c1 = mul_lim(kb, static_cast<uint64_t>(Db) * (pm ? 1u : Na), ovf);
  uint64_t s = c0 + c1;
  uint64_t P = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(kFull, P, o);
    if (lane >= o) P += y;
  }
  uint64_t A = __shfl_sync(kFull, P, 31);

  const uint32_t step = *t.step + step_off;
  const uint32_t key0 = static_cast<uint32_t>(t.seed), key1 = static_cast<uint32_t>(t.seed >> 32);
  const uint32_t word3 = t.tissue_id | (tag << 24);
  int err = __any_sync(kFull, ovf) ? kErrOverflow : 0;
  if (kChecked && oob) err = kErrBounds;  // then no event runs and nothing is written
  double tnow = 0.0;
  uint32_t e = 0, e0 = 0;
  uint64_t Em = 0, Rnd = 0;
  int Ek = -1;
  bool have = false;

  while (A != 0ull && !err) {
    int j = static_cast<int>(e - e0);
    if (!have || j == 32) {
      if (have) e0 += 32;
      have = true;
      j = 0;
      draw_event(e0 + lane, step, c, word3, key0, key1, Em, Ek, Rnd);
    }
    const uint64_t mE = __shfl_sync(kFull, Em, j);
    const int kE = __shfl_sync(kFull, Ek, j);
    const uint64_t R64 = __shfl_sync(kFull, Rnd, j);
    const double tn = __dadd_rn(tnow, tau_from(F53{mE, kE}, kE < 0, A));
    const uint64_t r = __umul64hi(R64, A);
    const unsigned m1 = __ballot_sync(kFull, r < P);
    const int L = m1 ? __ffs(m1) - 1 : 0;
    if (m1 == 0u || L >= n) {  // impossible while the prefix sums are consistent
      err |= kErrInternal;
      break;
    }
    const uint64_t Pl = __shfl_sync(kFull, P, L > 0 ? L - 1 : 0);
    const uint64_t r1 = r - (L > 0 ? Pl : 0ull);
    const uint64_t c0L = __shfl_sync(kFull, c0, L);
    if (!before(tn, dt)) break;
    tnow = tn;
    uint64_t delta = 0;
    if (lane == L) {
      trace_event(t, step, tag, c, e, tn, static_cast<uint32_t>(L), r1 < c0L ? 0u : 1u);
      if (r1 < c0L) {  // D(a) + N(b) -> R(b), or Delta(a) -> NICD(b)
        Da -= 1;
        Nb = pm ? Nb + 1 : Nb - 1;
        Rb += pm ? 0 : 1;
        ovf |= Rb > static_cast<uint32_t>(kCountMax) || Nb > static_cast<uint32_t>(kCountMax);
      } else {         // D(b) + N(a) -> R(a), or Delta(b) -> NICD(a)
        Db -= 1;
        Na = pm ? Na + 1 : Na - 1;
        Ra += pm ? 0 : 1;
        ovf |= Ra > static_cast<uint32_t>(kCountMax) || Na > static_cast<uint32_t>(kCountMax);
      }
      c0 = mul_lim(kb, static_cast<uint64_t>(Da) * (pm ? 1u : Nb), ovf);
      c1 = mul_lim(kb, static_cast<uint64_t>(Db) * (pm ? 1u : Na), ovf);
      const uint64_t s2 = c0 + c1;
      delta = s2 - s;
      s = s2;
    }
    delta = __shfl_sync(kFull, delta, L);
    P += lane >= L ? delta : 0ull;
    A += delta;
    ++e;
    if (__any_sync(kFull, ovf)) err = kErrOverflow;
    if (e == 0xFFFFFFFFu) err |= kErrEventIndex;
  }

  if (act && !(kChecked && oob)) {
    ga[va] = Da;
    ga[V + va] = Na;
    ga[2 * V + va] = Ra;
    gb[vb] = Db;
    gb[V + vb] = Nb;
    gb[2 * V + vb] = Rb;
  }
  if (lane == 0) {
    const uint32_t cells = W * H;
    const size_t row = static_cast<size_t>(1 + axis) * cells;
    t.ev_last[row + ca] = e;
    t.t_last[row + ca] = tnow;
    t.ev_total[row + ca] += e;
    if (err) atomicOr(t.err, err);
  }
}

__global__ void __launch_bounds__(256) k_sig(const TissueView t, const int axis,
                                             const uint32_t tag, const uint32_t step_off,
                                             const double dt) {
  const uint32_t W = t.width, H = t.height;
  const uint32_t nfaces = axis == 0 ? (W - 1) * H : W * (H - 1);
  const uint32_t f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (f >= nfaces) return;  // whole warp
  sig_face(t, axis == 0 ? (f / (W - 1)) * W + f % (W - 1) : f, axis, tag, step_off, dt);
}

// Faces of many tissues: item = (tissue index, owner cell).
__global__ void __launch_bounds__(256) k_sig_list(const TissueView* __restrict__ views,
                                                  const uint2* __restrict__ items,
                                                  const uint32_t n_items, const int axis,
                                                  const uint32_t tag, const double dt) {
  const uint32_t f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (f >= n_items) return;  // whole warp
  const uint2 w = items[f];
  sig_face(views[w.x], w.y, axis, tag, 0u, dt);
}

// Advance the step counter of every tissue of a batch by one.
__global__ void k_advance_list(const TissueView* __restrict__ views, const uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) *const_cast<uint32_t*>(views[i].step) += 1u;
}

// Batch checkpoint writes: every member's step counter from steps[] (if
// given) and its error flag cleared.
__global__ void k_set_steps_list(const TissueView* __restrict__ views, const uint32_t* steps,
                                 const uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (steps) *const_cast<uint32_t*>(views[i].step) = steps[i];
  *views[i].err = 0;
}

// Set *bad if any count of any member lies outside [0, TISSUE_COUNT_MAX]
// (one unsigned compare: a negative int32 is a large unsigned value).  Blocks
// stride over the members (y) and over each member's state (x), 16 bytes per
// load where the state allows it.
__global__ void k_check_counts_list(const TissueView* __restrict__ views, const uint32_t n,
                                    int* bad) {
  for (uint32_t m = blockIdx.y; m < n; m += gridDim.y) {
    const TissueView& t = views[m];
    const uint64_t total = static_cast<uint64_t>(t.width) * t.height * 3 * t.V;
    const uint32_t* c = reinterpret_cast<const uint32_t*>(t.counts);
    uint32_t worst = 0;
    const uint64_t n4 = total >> 2;  // the buffer is 16-byte aligned
    const uint4* c4 = reinterpret_cast<const uint4*>(c);
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n4;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
      const uint4 x = c4[i];
      worst = max(worst, max(max(x.x, x.y), max(x.z, x.w)));
    }
    for (uint64_t i = (n4 << 2) + blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
         i < total; i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
      worst = max(worst, c[i]);
    if (__any_sync(kFull, worst > static_cast<uint32_t>(kCountMax)) && (threadIdx.x & 31) == 0)
      atomicOr(bad, 1);
  }
}

// Every member's error flag into out[] (one copy back for the whole batch).
__global__ void k_gather_err_list(const TissueView* __restrict__ views, const uint32_t n,
                                  int* out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = *views[i].err;
}

// Initial counts: Poisson(lambda_s) per voxel and species by inversion,
// accumulating p_k = p_{k-1} * lambda / k; p0 = exp(-lambda) from the host.
__global__ void k_init(const TissueView t, const double p0_0, const double p0_1, const double p0_2,
                       const double l0, const double l1, const double l2) {
  const uint32_t V = t.V;
  const uint64_t total = static_cast<uint64_t>(t.width) * t.height * 3 * V;
  const uint32_t key0 = static_cast<uint32_t>(t.seed), key1 = static_cast<uint32_t>(t.seed >> 32);
  const uint32_t word3 = t.tissue_id | (kTagInit << 24);
  for (uint64_t idx = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t cs = static_cast<uint32_t>(idx / V);
    const uint32_t v = static_cast<uint32_t>(idx - static_cast<uint64_t>(cs) * V);
    const uint32_t c = cs / 3, s = cs - 3 * c;
    const double lam = s == 0 ? l0 : s == 1 ? l1 : l2;
    const double p0 = s == 0 ? p0_0 : s == 1 ? p0_1 : p0_2;
    const U4 w = philox10(v, s, c, word3, key0, key1);
    const uint64_t bits = ((static_cast<uint64_t>(w.y) << 32) | w.x) >> 11;
    const double u = __dmul_rn(__ull2double_rn(bits), 0x1p-53);
    int k = 0;
    double p = p0, F = p0;
    while (u >= F && k < 4096) {
      k += 1;
      p = __ddiv_rn(__dmul_rn(p, lam), static_cast<double>(k));
      F = __dadd_rn(F, p);
    }
    t.counts[idx] = k;
  }
}

__global__ void k_hill(const QRates q, uint64_t* table) {
  const uint32_t R = blockIdx.x * blockDim.x + threadIdx.x;
  if (R < kHillTab) table[R] = hill_direct(q, R);
}

__global__ void k_step_advance(uint32_t* step, uint32_t n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += n;
}

}  // namespace

cudaError_t launch_sig(const TissueView& t, int axis, uint32_t tag, uint32_t step_off, double dt,
                       cudaStream_t stream) {
  const uint32_t nfaces = axis == 0 ? (t.width - 1) * t.height : t.width * (t.height - 1);
  if (nfaces == 0) return cudaSuccess;
  constexpr int kWarps = 8;
  k_sig<<<(nfaces + kWarps - 1) / kWarps, 32 * kWarps, 0, stream>>>(t, axis, tag, step_off, dt);
  return cudaGetLastError();
}

cudaError_t launch_sig_list(const TissueView* d_views, const uint2* d_items, uint32_t n_items,
                            int axis, uint32_t tag, double dt, cudaStream_t stream) {
  if (n_items == 0) return cudaSuccess;
  constexpr int kWarps = 8;
  k_sig_list<<<(n_items + kWarps - 1) / kWarps, 32 * kWarps, 0, stream>>>(d_views, d_items, n_items,
                                                                         axis, tag, dt);
  return cudaGetLastError();
}

cudaError_t launch_advance_list(const TissueView* d_views, uint32_t n, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  k_advance_list<<<(n + 255) / 256, 256, 0, stream>>>(d_views, n);
  return cudaGetLastError();
}

cudaError_t launch_set_steps_list(const TissueView* d_views, const uint32_t* d_steps, uint32_t n,
                                  cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  k_set_steps_list<<<(n + 255) / 256, 256, 0, stream>>>(d_views, d_steps, n);
  return cudaGetLastError();
}

cudaError_t launch_check_counts_list(const TissueView* d_views, uint32_t n, int* d_bad,
                                     cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const dim3 grid(16, n < 65535u ? n : 65535u);
  k_check_counts_list<<<grid, 256, 0, stream>>>(d_views, n, d_bad);
  return cudaGetLastError();
}

cudaError_t launch_gather_err_list(const TissueView* d_views, uint32_t n, int* d_out,
                                   cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  k_gather_err_list<<<(n + 255) / 256, 256, 0, stream>>>(d_views, n, d_out);
  return cudaGetLastError();
}

cudaError_t launch_init(const TissueView& t, const double p0[3], const double lam[3],
                        cudaStream_t stream) {
  const uint64_t total = static_cast<uint64_t>(t.width) * t.height * 3 * t.V;
  const uint64_t want = (total + 255) / 256;
  const uint32_t blocks = static_cast<uint32_t>(want < 152ull * 64 ? want : 152ull * 64);
  k_init<<<blocks, 256, 0, stream>>>(t, p0[0], p0[1], p0[2], lam[0], lam[1], lam[2]);
  return cudaGetLastError();
}

cudaError_t launch_hill_table(const QRates& q, uint64_t* table, cudaStream_t stream) {
  k_hill<<<(kHillTab + 255) / 256, 256, 0, stream>>>(q, table);
  return cudaGetLastError();
}

cudaError_t launch_step_advance(uint32_t* step, uint32_t n, cudaStream_t stream) {
  k_step_advance<<<1, 32, 0, stream>>>(step, n);
  return cudaGetLastError();
}

}  // namespace tsg
