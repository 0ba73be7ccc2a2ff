// K_chi: the intracellular module chi (arXiv 1806.10889, Sec. II-A1) as a
// lattice RDME advanced by the direct-method SSA over one splitting step
// [0, dt), one warp per cell.
//
// Data layout per warp in shared memory:
//   pre[v]    uint64  inclusive prefix of the voxel propensities a_v inside the
//                     lane block of v (lane l owns voxels l*B .. l*B+B-1)
//   cnt[s][v] int32   D, N, R counts
// and per lane in registers:
//   P         uint64  inclusive prefix of the block totals over lanes 0..l
// Propensities are exact integers (units of 2^-32 per unit time), so the
// prefix sums are exact and are updated by adding the change of the touched
// voxels instead of being rebuilt: after an event only 1 or 2 voxels change.
//
// Event selection for r in [0, A): one ballot over P finds the lane block,
// one ballot over pre[] finds the voxel, and a 19-lane shuffle scan over the
// channels of that voxel finds the channel -- the same first-index-whose-
// running-sum-exceeds-r rule as a linear scan in voxel-major, channel-minor
// order.  Random numbers for 32 consecutive events are drawn at once, one
// Philox block and one exponential variate per lane.  The waiting time uses
// the integer binary64 quotient of tissue_dev.cuh, so the only FP64-pipe
// instruction per event is the clock addition t + tau.
#include "tissue_dev.cuh"

namespace tsg {

namespace {

// Total propensity of voxel v.  Counts below q.small cannot reach the 2^52
// limit, so the common case needs no overflow checks; otherwise every term is
// checked exactly.
template <int VMAX>
__device__ __forceinline__ uint64_t voxel_total(const int32_t* cnt, int v, const TissueView& t,
                                                bool& ovf) {
  const uint32_t D = static_cast<uint32_t>(cnt[v]);
  const uint32_t N = static_cast<uint32_t>(cnt[VMAX + v]);
  const uint32_t R = static_cast<uint32_t>(cnt[2 * VMAX + v]);
  const int n = static_cast<int>(t.n);
  const int vy = div_n(v, t.magic), vx = v - vy * n;
  const int nn = (vx > 0) + (vx < n - 1) + (vy > 0) + (vy < n - 1);
  const uint64_t base = hill_q(t.q, R) + t.q.kN;
  if ((D | N | R) < t.q.small) {
    return base + t.q.cD[nn] * D + t.q.cN[nn] * N + t.q.cRo[nn] * R +
           t.q.k_in * (static_cast<uint64_t>(D) * N);
  }
  uint64_t a = base;
  a += mul_lim(t.q.cD[nn], D, ovf);
  a += mul_lim(t.q.cN[nn], N, ovf);
  a += mul_lim(t.q.cR[nn], R, ovf);
  a += mul_lim(t.q.k_in, static_cast<uint64_t>(D) * N, ovf);
  a += mul_lim(t.q.k_off, R, ovf);
  ovf |= (a >> 52) != 0ull;
  return a;
}

// Channel lanes: lane j < 19 evaluates channel j of the selected voxel.
//   0 Hill production of D, 1 production of N, 2..4 decay of D, N, R,
//   5..8 / 9..12 / 13..16 hop of D / N / R toward -x, +x, -y, +y,
//   17 D + N -> R, 18 R -> D + N.
enum : int { kOne = 0, kD = 1, kN = 2, kR = 3, kDN = 4, kHill = 5 };

__device__ __forceinline__ void channel_of_lane(int lane, const QRates& q, uint64_t& rate,
                                                int& factor, int& dir) {
  rate = 0;
  factor = kOne;
  dir = -1;
  if (lane == 0) {
    factor = kHill;
  } else if (lane == 1) {
    rate = q.kN;
  } else if (lane <= 4) {
    rate = lane == 2 ? q.gD : lane == 3 ? q.gN : q.gR;
    factor = lane == 2 ? kD : lane == 3 ? kN : kR;
  } else if (lane <= 16) {
    const int s = (lane - 5) >> 2;
    rate = s == 0 ? q.hopD : s == 1 ? q.hopN : q.hopR;
    factor = s == 0 ? kD : s == 1 ? kN : kR;
    dir = (lane - 5) & 3;
  } else if (lane == 17) {
    rate = q.k_in;
    factor = kDN;
  } else if (lane == 18) {
    rate = q.k_off;
    factor = kR;
  }
}

template <int B>
__global__ void __launch_bounds__(512) k_chi(const TissueView t, const uint32_t step_off,
                                             const double dt) {
  constexpr int VMAX = 32 * B;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const uint32_t ncells = t.width * t.height;
  const uint32_t cell = blockIdx.x * (blockDim.x >> 5) + wib;
  if (cell >= ncells) return;  // the whole warp leaves together

  uint64_t* pre = reinterpret_cast<uint64_t*>(smem + static_cast<size_t>(wib) * (VMAX * 20));
  int32_t* cnt = reinterpret_cast<int32_t*>(pre + VMAX);
  const int V = static_cast<int>(t.V);
  const int n = static_cast<int>(t.n);
  int32_t* g = t.counts + static_cast<size_t>(cell) * 3 * V;

  // T_{S->chi}: the cell's state, as left by the previous step, into shared memory.
  if ((V & 3) == 0) {
    const int V4 = V >> 2;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int4* src = reinterpret_cast<const int4*>(g + s * V);
      int4* dst = reinterpret_cast<int4*>(cnt + s * VMAX);
      for (int i = lane; i < V4; i += 32) dst[i] = src[i];
    }
  } else {
    for (int s = 0; s < 3; ++s)
      for (int i = lane; i < V; i += 32) cnt[s * VMAX + i] = g[s * V + i];
  }
  __syncwarp();

  const uint32_t step = *t.step + step_off;
  const uint32_t key0 = static_cast<uint32_t>(t.seed), key1 = static_cast<uint32_t>(t.seed >> 32);
  const uint32_t word3 = t.tissue_id | (kTagChi << 24);
  bool ovf = false;

  // Block prefixes and lane prefixes of the voxel propensities.
  uint64_t S = 0;
  for (int i = 0; i < B; ++i) {
    const int v = lane * B + i;
    if (v < V) {
      S += voxel_total<VMAX>(cnt, v, t, ovf);
      pre[v] = S;
    }
  }
  uint64_t P = S;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(kFull, P, o);
    if (lane >= o) P += y;
  }
  uint64_t A = __shfl_sync(kFull, P, 31);
  __syncwarp();

  uint64_t ch_rate;
  int ch_factor, ch_dir;
  channel_of_lane(lane, t.q, ch_rate, ch_factor, ch_dir);

  double tnow = 0.0;
  uint32_t e = 0, e0 = 0;
  uint64_t Em, Rb;
  int Ek;
  draw_event(e0 + lane, step, cell, word3, key0, key1, Em, Ek, Rb);
  int err = __any_sync(kFull, ovf) ? kErrOverflow : 0;

  while (A != 0ull && !err) {
    int j = static_cast<int>(e - e0);
    if (j == 32) {
      e0 += 32;
      j = 0;
      draw_event(e0 + lane, step, cell, word3, key0, key1, Em, Ek, Rb);
    }
    const uint64_t mE = __shfl_sync(kFull, Em, j);
    const int kE = __shfl_sync(kFull, Ek, j);
    const uint64_t R64 = __shfl_sync(kFull, Rb, j);
    // waiting time: tau = E / (A 2^-32); the event fires iff t + tau < dt
    const double tn = __dadd_rn(tnow, tau_from(F53{mE, kE}, kE < 0, A));

    // selection (independent of the time test, so it overlaps its latency)
    const uint64_t r = __umul64hi(R64, A);
    const unsigned m1 = __ballot_sync(kFull, r < P);
    const int L = m1 ? __ffs(m1) - 1 : 0;
    const uint64_t Pl = __shfl_sync(kFull, P, L > 0 ? L - 1 : 0);
    const uint64_t r1 = r - (L > 0 ? Pl : 0ull);
    const int vb = L * B;
    uint64_t pv = ~0ull;
    if (lane < B && vb + lane < V) pv = pre[vb + lane];
    const unsigned m2 = __ballot_sync(kFull, r1 < pv);
    const int i2 = m2 ? __ffs(m2) - 1 : 0;
    const uint64_t pp = __shfl_sync(kFull, pv, i2 > 0 ? i2 - 1 : 0);
    const uint64_t r2 = r1 - (i2 > 0 ? pp : 0ull);
    const int v = vb + i2;
    // The prefix invariants make these impossible; if they ever broke, stop
    // this cell with an error instead of touching memory outside it.
    if (m1 == 0u || m2 == 0u || i2 >= B || v >= V) {
      err |= kErrInternal;
      break;
    }
    const uint32_t D = static_cast<uint32_t>(cnt[v]);
    const uint32_t N = static_cast<uint32_t>(cnt[VMAX + v]);
    const uint32_t R = static_cast<uint32_t>(cnt[2 * VMAX + v]);
    const int vy = div_n(v, t.magic), vx = v - vy * n;
    uint64_t x = ch_factor == kD ? D : ch_factor == kN ? N : ch_factor == kR ? R : 1u;
    if (ch_factor == kDN) x = static_cast<uint64_t>(D) * N;
    uint64_t cum = ch_rate * x;
    if (ch_dir >= 0) {
      const bool has = ch_dir == 0 ? vx > 0 : ch_dir == 1 ? vx < n - 1 : ch_dir == 2 ? vy > 0 : vy < n - 1;
      if (!has) cum = 0;
    }
    if (ch_factor == kHill) cum = hill_q(t.q, R);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(kFull, cum, o);
      if (lane >= o) cum += y;
    }
    const unsigned m3 = __ballot_sync(kFull, lane < 19 && r2 < cum);
    const int ch = m3 ? __ffs(m3) - 1 : 0;
    const uint64_t a_old_v = __shfl_sync(kFull, cum, 18);
    if (m3 == 0u) {
      err |= kErrInternal;
      break;
    }

    if (!before(tn, dt)) break;
    tnow = tn;

    // the channel's effect: up to three (species, voxel, +-1) changes
    int sp0, sp1 = 0, sp2 = 0, d0, d1 = 0, d2 = 0, u = -1;
    if (ch <= 1) {
      sp0 = ch;
      d0 = 1;
    } else if (ch <= 4) {
      sp0 = ch - 2;
      d0 = -1;
    } else if (ch <= 16) {
      const int s = (ch - 5) >> 2, dir = (ch - 5) & 3;
      u = v + (dir == 0 ? -1 : dir == 1 ? 1 : dir == 2 ? -n : n);
      if (u < 0 || u >= V) {
        err |= kErrInternal;
        break;
      }
      sp0 = s;
      d0 = -1;
      sp1 = s;
      d1 = 1;
    } else if (ch == 17) {
      sp0 = 0; d0 = -1; sp1 = 1; d1 = -1; sp2 = 2; d2 = 1;
    } else {
      sp0 = 2; d0 = -1; sp1 = 0; d1 = 1; sp2 = 1; d2 = 1;
    }
    uint64_t a_old_u = 0;
    if (u >= 0) a_old_u = pre[u] - ((u & (B - 1)) ? pre[u - 1] : 0ull);
    __syncwarp();
    if (lane < 3) {
      const int sp = lane == 0 ? sp0 : lane == 1 ? sp1 : sp2;
      const int dd = lane == 0 ? d0 : lane == 1 ? d1 : d2;
      const int xv = (lane == 1 && u >= 0) ? u : v;
      if (dd != 0) {
        int32_t* c = &cnt[sp * VMAX + xv];
        const int nv = *c + dd;
        *c = nv;
        ovf |= nv > kCountMax;
      }
    }
    __syncwarp();
    // New totals: lane 1 evaluates u (when a hop moved a molecule there), the
    // others v; one call site, so the warp does not split.
    const uint64_t a_new = voxel_total<VMAX>(cnt, (lane == 1 && u >= 0) ? u : v, t, ovf);
    const uint64_t dv = __shfl_sync(kFull, a_new, 0) - a_old_v;
    const uint64_t du = __shfl_sync(kFull, a_new, 1) - a_old_u;
    const int bv = v / B;
    P += lane >= bv ? dv : 0ull;
    A += dv;
    if (u >= 0) {
      const int bu = u / B;
      P += lane >= bu ? du : 0ull;
      A += du;
    }
    if (lane < B) {
      const int iv = bv * B + lane;
      if (lane >= (v & (B - 1)) && iv < V) pre[iv] += dv;
      if (u >= 0) {
        const int iu = (u / B) * B + lane;
        if (lane >= (u & (B - 1)) && iu < V) pre[iu] += du;
      }
    }
    __syncwarp();
    ++e;
    if (__any_sync(kFull, ovf)) err = kErrOverflow;
    if (e == 0xFFFFFFFFu) err |= kErrEventIndex;
  }

  // T_{chi->S}: write the cell back for the signalling phases.
  __syncwarp();
  if ((V & 3) == 0) {
    const int V4 = V >> 2;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      int4* dst = reinterpret_cast<int4*>(g + s * V);
      const int4* src = reinterpret_cast<const int4*>(cnt + s * VMAX);
      for (int i = lane; i < V4; i += 32) dst[i] = src[i];
    }
  } else {
    for (int s = 0; s < 3; ++s)
      for (int i = lane; i < V; i += 32) g[s * V + i] = cnt[s * VMAX + i];
  }
  if (lane == 0) {
    t.ev_last[cell] = e;
    t.t_last[cell] = tnow;
    t.ev_total[cell] += e;
    if (err) atomicOr(t.err, err);
  }
}

template <int B>
cudaError_t launch_chi_b(const TissueView& t, uint32_t step_off, double dt, int wpb,
                         cudaStream_t stream) {
  const size_t smem = static_cast<size_t>(wpb) * 32 * B * 20;
  // The attribute belongs to the current device's copy of the kernel, so it is
  // set on every launch that needs more than the default 48 KB (a host-side
  // call, cheap next to the launch): a cache of it would have to be kept per
  // device and guarded against concurrent callers.
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_chi<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  const uint32_t cells = t.width * t.height;
  const uint32_t blocks = (cells + wpb - 1) / wpb;
  k_chi<B><<<blocks, 32 * wpb, smem, stream>>>(t, step_off, dt);
  return cudaGetLastError();
}

// Self-check of the integer binary64 time arithmetic against the FP64 unit:
// random and structured (E, A) pairs, the quotient and the clock test.
__global__ void k_selftest_time(uint64_t n, uint64_t seed, unsigned long long* mismatches) {
  unsigned long long bad = 0;
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const U4 w = philox10(static_cast<uint32_t>(i), static_cast<uint32_t>(i >> 32), 7u, 7u,
                          static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    const uint64_t w01 = (static_cast<uint64_t>(w.y) << 32) | w.x;
    const uint64_t w23 = (static_cast<uint64_t>(w.w) << 32) | w.z;
    uint64_t eq;
    switch (i & 3) {
      case 0: eq = neg_ln_q58((w01 >> 11) + 1); break;           // as drawn
      case 1: eq = w01 >> (w.z & 63); break;                     // any magnitude
      case 2: eq = (1ull << (w.z % 63)) + (w.w & 7) - 3; break;  // near powers of two
      default: eq = w01 & 0xFFFFFull; break;                     // small
    }
    uint64_t A;
    switch ((i >> 2) & 3) {
      case 0: A = w23 >> (2 + (w.x % 62)); break;                // 1 .. 2^62
      case 1: A = 1ull << (w.x % 62); break;                     // powers of two
      case 2: A = (1ull << (w.x % 62)) + (w.y & 15) - 7; break;  // around them
      default: A = (w23 >> 9) | (1ull << 54); break;             // needs rounding to 53 bits
    }
    if (A == 0ull || (A >> 62) != 0ull) A = 1ull + (A & 0x3FFFFFFFFFFFFFFEull);
    const F53 f = round53(eq | static_cast<uint64_t>(eq == 0ull));
    const double mine = tau_from(f, eq == 0ull, A);
    const double ref = __ddiv_rn(__dmul_rn(__ull2double_rn(eq), 0x1p-58),
                                 __dmul_rn(__ull2double_rn(A), 0x1p-32));
    bad += __double_as_longlong(mine) != __double_as_longlong(ref);
    const double t0 = __dmul_rn(__ull2double_rn(w23 >> 11), 0x1p-53);
    const double sum = __dadd_rn(t0, ref);
    bad += before(sum, 0.5) != (sum < 0.5);
  }
  if (bad) atomicAdd(mismatches, bad);
}

}  // namespace

cudaError_t launch_chi(const TissueView& t, uint32_t step_off, double dt, int wpb,
                       cudaStream_t stream) {
  const uint32_t V = t.V;
  if (V <= 32) return launch_chi_b<1>(t, step_off, dt, wpb, stream);
  if (V <= 64) return launch_chi_b<2>(t, step_off, dt, wpb, stream);
  if (V <= 128) return launch_chi_b<4>(t, step_off, dt, wpb, stream);
  if (V <= 256) return launch_chi_b<8>(t, step_off, dt, wpb, stream);
  if (V <= 512) return launch_chi_b<16>(t, step_off, dt, wpb, stream);
  if (V <= 1024) return launch_chi_b<32>(t, step_off, dt, wpb, stream);
  return cudaErrorInvalidValue;
}

cudaError_t launch_selftest_time(uint64_t n, uint64_t seed, unsigned long long* mismatches,
                                 cudaStream_t stream) {
  k_selftest_time<<<152 * 8, 256, 0, stream>>>(n, seed, mismatches);
  return cudaGetLastError();
}

uint32_t small_count_bound(const QRates& q, uint64_t hill_max) {
  using u128 = unsigned __int128;
  uint64_t cmax = 0;
  for (int nn = 0; nn <= 4; ++nn) {
    const uint64_t c = q.cD[nn] + q.cN[nn] + q.cRo[nn];
    cmax = c > cmax ? c : cmax;
  }
  uint32_t best = 0;
  for (int j = 1; j <= 30; ++j) {
    const u128 T = (static_cast<u128>(1) << j) - 1;  // largest count below 2^j
    const u128 a = static_cast<u128>(hill_max) + q.kN + static_cast<u128>(cmax) * T +
                   static_cast<u128>(q.k_in) * T * T;
    if (a < (static_cast<u128>(1) << 52)) best = 1u << j;
  }
  return best;
}

}  // namespace tsg
