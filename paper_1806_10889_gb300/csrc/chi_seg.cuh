// K_chi, persistent segmented form: the intracellular module chi (arXiv
// 1806.10889, Sec. II-A1) over a work list of cells, H lanes per cell.
//
// A warp is split into 32/H segments (H = 32, 16 or 8); each segment runs one
// cell's direct-method SSA exactly as the one-warp-per-cell kernel does
// (same Philox stream, same integer propensities, same binary64 clock), so
// both kernels give identical results.  With H < 32 every uniform
// instruction of the event loop -- waiting time, selection arithmetic,
// decoding -- serves several cells at once.  When a segment's cell reaches
// the end of the step it writes the cell back and takes the next item from
// the work list (one atomic add), so cells of different cost and tissues of
// different size share one launch without idle warps.
//
// Per segment, shared memory holds a copy of its tissue's view (model,
// pointers) and the counts cnt[][], and in the prefix layout the
// within-block prefix pre[] as in the one-warp kernel.  Lane l of a segment
// owns voxels l*B .. l*B+B-1 (B a power of two, H*B >= V) and keeps the
// inclusive prefix P of the block totals in a register; selection takes a
// block by one ballot over P, then a voxel inside it: from pre[] (prefix
// layout), or by recomputing the block's voxel totals, one voxel per lane,
// and scanning them (counts-only layout).  When a block is wider than the
// segment (B > H) the counts-only layout first picks one of the block's
// sub-blocks of H voxels from the running sums its owning lane keeps in
// registers, and recomputes only that sub-block.  The channel of the
// selected voxel is found without a scan: lane j evaluates the running sum
// C_j of channels 0..j in closed form (hop channels enter through the count
// of existing neighbour directions); with H = 16, C_16..C_18 follow from
// C_15 by three additions.
//
// Both single-cell models share the 19 channel slots.  Per voxel a model
// contributes three terms -- c0 (slot 0), c1 (slot 1) and the bimolecular
// product X of slot 17 -- and affine terms in D, N and R:
//   Notch-Delta:  c0 = Hill(R), c1 = kN,        X = D N
//   promoter:     c0 = t_D F,   c1 = k_d R,     X = N F
// where F = [v is the promoter voxel] - R counts the free promoter sites
// (the paper's Notch model, Sec. III-A1: R counts bound sites).
//
// Template parameters: H lanes per cell; PRE the shared-memory layout; QB
// whether a lane may cover several voxels of a block (B > H, i.e. V > H^2);
// GEN the models the launch holds: 0 Notch-Delta only, 1 either (each cell
// tests its tissue's model), 2 promoter only (the test folded away); NARROW
// 16-bit counts in shared memory (14 instead of 20 bytes per voxel, so more
// large cells fit on an SM).  A NARROW segment whose cell holds or reaches a
// count above 65535 leaves that cell untouched and appends it to a redo list,
// which the launcher then runs through the 32-bit instantiation from the same
// state and random streams: the results are those of a 32-bit run.  The
// launcher picks QB and GEN from the largest cell and the listed tissues.
#pragma once
#include <type_traits>

#include "tissue_dev.cuh"

namespace tsg {

namespace {

constexpr int kViewBytes = (static_cast<int>(sizeof(TissueView)) + 15) & ~15;
static_assert(sizeof(TissueView) % 8 == 0, "view copy uses 8-byte words");

struct Seg {
  int V, n, B, lb;  // voxels, side, voxels per lane block, log2 B
  uint32_t magic;
  int qb;           // log2 of the voxels each lane covers inside one block (B > H)
  int centre;       // the promoter voxel (n/2, n/2)
  int ls;           // log2 of a sub-block's voxels, lb - qb (counts-only layout, B > H)
};

// The model terms c0, c1 and X of a voxel (see the file comment); hR is the
// Hill production Hill(R) of the Notch-Delta model (unused by the promoter).
template <bool GEN>
__device__ __forceinline__ void voxel_terms(bool pm, const QRates& q, int v, const Seg& s,
                                            uint32_t D, uint32_t N, uint32_t R, uint64_t hR,
                                            uint64_t& c0, uint64_t& c1, uint64_t& X) {
  if (GEN && pm) {
    const uint32_t F = static_cast<uint32_t>(v == s.centre) - R;
    c0 = q.tD * F;
    c1 = q.kd * R;
    X = static_cast<uint64_t>(N) * F;
  } else {
    c0 = hR;
    c1 = q.kN;
    X = static_cast<uint64_t>(D) * N;
  }
}

// Hill values held in registers: lane j of a segment keeps Hill(j) (SETS = 1)
// and Hill(j + H) (SETS = 2), read from its tissue's table when the segment
// takes a cell.  Repressor counts per voxel are small (a few tens in a
// running tissue), so most lookups of the event loop become register
// shuffles instead of table loads on the event's dependency chain; larger
// counts fall back to the table.  The kernel uses one set with one cell per
// warp (H = 32) and in the counts-only layout, which looks up every voxel of
// the selected block, one set at 16 lanes and two at 8 (R < 16); with the
// prefix layout at 16 or 8 lanes the extra registers cost more than they
// save (a resident block per SM at 16 lanes; same-box A/B), so those read
// the table (SETS = 0).
template <int H, int SETS>
struct HillRegs {
  static constexpr int kSets = SETS;
  static constexpr uint32_t kCover = static_cast<uint32_t>(kSets * H);
  uint64_t h0 = 0, h1 = 0;

  __device__ __forceinline__ void load(const QRates& q, int sl) {
    if (kSets >= 1) h0 = __ldg(q.hill + sl);
    if (kSets >= 2) h1 = __ldg(q.hill + sl + H);
  }

  // Hill(R) for this lane's R; every lane of the warp must call it (the
  // shuffles are warp-wide).  `act` gates the table fallback so an idle
  // segment reads nothing.
  __device__ __forceinline__ uint64_t get(const QRates& q, uint32_t R, bool act) const {
    uint64_t x = 0ull;
    if (kSets >= 1) {
      const int src = static_cast<int>(R & static_cast<uint32_t>(H - 1));
      x = __shfl_sync(kFull, h0, src, H);
      if (kSets >= 2) {
        const uint64_t y = __shfl_sync(kFull, h1, src, H);
        x = (R & static_cast<uint32_t>(H)) ? y : x;
      }
    }
    return R < kCover ? x : (act ? hill_q(q, R) : 0ull);
  }
};

// Existence mask of the four neighbour directions (-x, +x, -y, +y) of v.
__device__ __forceinline__ uint32_t dir_mask(int v, const Seg& s) {
  const int vy = div_n(v, s.magic), vx = v - vy * s.n;
  return static_cast<uint32_t>(vx > 0) | (static_cast<uint32_t>(vx < s.n - 1) << 1) |
         (static_cast<uint32_t>(vy > 0) << 2) | (static_cast<uint32_t>(vy < s.n - 1) << 3);
}

// Total propensity of voxel v (see voxel_total in k_chi.cu; same value),
// given the voxel's counts and its Hill value hR.
template <bool GEN>
__device__ __forceinline__ uint64_t voxel_total_of(int v, uint32_t D, uint32_t N, uint32_t R,
                                                   uint64_t hR, const Seg& s, const QRates& q,
                                                   bool pm, bool& ovf) {
  const int nn = __popc(dir_mask(v, s));
  uint64_t c0, c1, X;
  voxel_terms<GEN>(pm, q, v, s, D, N, R, hR, c0, c1, X);
  const uint64_t base = c0 + c1;
  if ((D | N | R) < q.small) {
    return base + q.cD[nn] * D + q.cN[nn] * N + q.cRo[nn] * R + q.k_in * X;
  }
  uint64_t a = base;
  a += mul_lim(q.cD[nn], D, ovf);
  a += mul_lim(q.cN[nn], N, ovf);
  a += mul_lim(q.cR[nn], R, ovf);
  a += mul_lim(q.k_in, X, ovf);
  a += mul_lim(q.k_off, R, ovf);
  ovf |= (a >> 52) != 0ull;
  return a;
}

// Total propensity of voxel v from the counts in shared memory, its Hill
// value read from the table.
template <bool GEN, typename CT>
__device__ __forceinline__ uint64_t seg_voxel_total(const CT* cnt, int vmax, int v,
                                                    const Seg& s, const QRates& q, bool pm,
                                                    bool& ovf, bool& oob) {
  const int vi = static_cast<int>(TSG_IDX(v, vmax, oob));
  const uint32_t D = static_cast<uint32_t>(cnt[vi]);
  const uint32_t N = static_cast<uint32_t>(cnt[vmax + vi]);
  const uint32_t R = static_cast<uint32_t>(cnt[2 * vmax + vi]);
  const uint64_t hR = (GEN && pm) ? 0ull : hill_q(q, R);
  return voxel_total_of<GEN>(v, D, N, R, hR, s, q, pm, ovf);
}

// Lane constants for the closed-form running sum C_j of channel j: which of
// the first five channels are included, which hop directions of D, N and R.
struct ChanLane {
  uint32_t mD, mN, mR;   // direction masks counted in C_j
  bool f1, f2, f3, f4, f17, f18, valid;
};

__device__ __forceinline__ ChanLane chan_lane(int j) {
  ChanLane c;
  c.valid = j < 19;
  c.f1 = j >= 1;
  c.f2 = j >= 2;
  c.f3 = j >= 3;
  c.f4 = j >= 4;
  c.f17 = j >= 17;
  c.f18 = j >= 18;
  c.mD = j < 5 ? 0u : j <= 8 ? (2u << (j - 5)) - 1u : 0xFu;
  c.mN = j < 9 ? 0u : j <= 12 ? (2u << (j - 9)) - 1u : 0xFu;
  c.mR = j < 13 ? 0u : j <= 16 ? (2u << (j - 13)) - 1u : 0xFu;
  return c;
}

// PRE selects the shared-memory layout: true keeps the within-block prefix
// pre[] of the voxel propensities (20 B per voxel); false keeps only the
// counts (12 B per voxel, 6 with 16-bit counts) and recomputes, per event,
// the propensities of the selected block -- or, when a block is wider than
// the segment, of one sub-block of H voxels found from the owning lane's
// sub-block sums -- one voxel per lane, so that more cells fit on an SM.
// A lane's channel-sum coefficients for one tissue, in registers (set when the
// segment takes a cell): the per-count terms of the channels up to the lane's.
// The hop terms depend on the voxel's neighbours and are added per voxel.
struct LaneK {
  uint64_t aD, aN, aR, k17;  // gD, gN, gR + k_off and k_in where counted in C_j
};

__device__ __forceinline__ LaneK lane_k(const ChanLane& c, const QRates& q) {
  LaneK k;
  k.aD = c.f2 ? q.gD : 0ull;
  k.aN = c.f3 ? q.gN : 0ull;
  k.aR = (c.f4 ? q.gR : 0ull) + (c.f18 ? q.k_off : 0ull);
  k.k17 = c.f17 ? q.k_in : 0ull;
  return k;
}

// Running sum C_j of the channels 0..j of a voxel (~0 for j >= 19). The hop
// rates, the same for every lane, come from the view in shared memory: holding
// them in registers too costs a resident block per SM.
__device__ __forceinline__ uint64_t chan_cum(const ChanLane& c, const LaneK& k, const QRates& q,
                                             uint64_t c0, uint64_t c1, uint32_t D, uint32_t N,
                                             uint32_t R, uint64_t X, uint32_t hm) {
  if (!c.valid) return ~0ull;
  return c0 + (c.f1 ? c1 : 0ull) + D * (k.aD + q.hopD * __popc(hm & c.mD)) +
         N * (k.aN + q.hopN * __popc(hm & c.mN)) + R * (k.aR + q.hopR * __popc(hm & c.mR)) +
         k.k17 * X;
}

// items[0 .. n) are the work (n = *n_items_dev when that is given, else
// n_items); NARROW appends the cells it gives up on to redo[*redo_n ...].
template <int H, bool PRE, bool QB, int GEN, bool NARROW>
__global__ void __launch_bounds__(PRE ? 256 : 128, PRE ? 1 : (QB ? 4 : (NARROW ? 5 : 8))) k_chi_seg(
                                                 const TissueView* __restrict__ views,
                                                 const uint2* __restrict__ items,
                                                 const uint32_t n_items, uint32_t* counter,
                                                 const uint32_t seg_bytes,
                                                 const uint32_t step_off, const double dt,
                                                 uint2* __restrict__ redo, uint32_t* redo_n,
                                                 const uint32_t* n_items_dev) {
  static_assert(!NARROW || GEN == 0, "16-bit counts: Notch-Delta only");
  using CT = typename std::conditional<NARROW, uint16_t, int32_t>::type;
  constexpr int G = 32 / H;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int seg = lane / H, sl = lane % H;
  constexpr unsigned kSegBits = H == 32 ? kFull : ((1u << H) - 1u);
  const unsigned segmask = H == 32 ? kFull : (kSegBits << (H * seg));
  unsigned char* base = smem + static_cast<size_t>(wib * G + seg) * seg_bytes;
  TissueView* sv = reinterpret_cast<TissueView*>(base);
  constexpr int kBytesPerVoxel = (PRE ? 8 : 0) + 3 * static_cast<int>(sizeof(CT));
  const int vmax = static_cast<int>((seg_bytes - kViewBytes) / kBytesPerVoxel);
  uint64_t* pre = reinterpret_cast<uint64_t*>(base + kViewBytes);  // used only if PRE
  CT* cnt = reinterpret_cast<CT*>(base + kViewBytes + (PRE ? 8 * vmax : 0));
  const ChanLane cl = chan_lane(sl);
  const ChanLane cl2 = chan_lane(sl + H);  // second channel of each lane when H = 8
  LaneK lk{}, lk2{};                         // their coefficients for the current cell
  HillRegs<H, (!PRE && H == 8) ? 2 : (H == 32 || (!PRE && H == 16)) ? 1 : 0> hreg;

  // The counts-only layout with blocks wider than the segment (B > H, up to
  // four sub-blocks of H voxels: 16 lanes for V <= 1024, 8 for V <= 256):
  // lane l keeps the running sums sb[k] of its own block's sub-blocks 0..k,
  // so that an event finds the sub-block from lane L's sums and recomputes
  // only its H voxels, one per lane, instead of the whole block.
  static_assert(PRE || !QB || H == 16 || H == 8, "recompute layout with B > H: 8 or 16 lanes");
  constexpr bool SUB = !PRE && QB;
  uint64_t sb[4] = {0ull, 0ull, 0ull, 0ull};
  bool have = false, done = false, pm = false;
  bool oob = false;  // checked build: an index out of range (see TSG_IDX)
  Seg s{0, 2, 1, 0, 1, 0, 0, 0};
  uint32_t cell = 0, vidx = 0, step = 0, word3 = 0, key0 = 0, key1 = 0, e = 0, e0 = 0;
  uint64_t A = 0, P = 0, Em = 0, Rb = 0, Em2 = 0, Rb2 = 0;
  int Ek = -1, Ek2 = -1, err = 0;
  bool next_ok = false;  // the draws of events e0+H+sl are in Em2/Ek2/Rb2
  double tnow = 0.0;
  int32_t* g = nullptr;

  for (;;) {
    // ---- a segment without a cell takes the next work item ----------------
    if (!have && !done) {
      uint32_t it = 0;
      if (sl == 0) it = atomicAdd(counter, 1u);
      it = __shfl_sync(segmask, it, 0, H);
      if (it >= (n_items_dev ? *n_items_dev : n_items)) {
        done = true;
      } else {
        const uint2 w = items ? items[it] : make_uint2(0u, it);
        cell = w.y;
        vidx = w.x;
        const uint64_t* src = reinterpret_cast<const uint64_t*>(views + w.x);
        uint64_t* dst = reinterpret_cast<uint64_t*>(sv);
        for (int i = sl; i < static_cast<int>(sizeof(TissueView) / 8); i += H) dst[i] = src[i];
        __syncwarp(segmask);
        s.V = static_cast<int>(sv->V);
        s.n = static_cast<int>(sv->n);
        s.magic = sv->magic;
        s.lb = 0;
        while ((H << s.lb) < s.V) ++s.lb;
        s.B = 1 << s.lb;
        s.qb = 0;
        while ((H << s.qb) < s.B) ++s.qb;
        s.centre = (s.n >> 1) * s.n + (s.n >> 1);
        s.ls = s.lb - s.qb;
        pm = GEN == 2 || (GEN == 1 && sv->q.kind == kModelPromoter);
        lk = lane_k(cl, sv->q);
        if (H == 8) lk2 = lane_k(cl2, sv->q);
        if (GEN != 2) hreg.load(sv->q, sl);
        const bool skip = kChecked && (s.V > vmax || cell >= sv->width * sv->height);
        if (skip) {
          // the cell does not fit this launch's shared memory, or is not in
          // its tissue: report it; the segment stays idle this pass and takes
          // the next item on the next one
          if (sl == 0) atomicOr(sv->err, kErrBounds);
          __syncwarp(segmask);
        } else {
          g = sv->counts + static_cast<size_t>(cell) * 3 * s.V;
          bool big = false;  // NARROW: a count above 65535 (the cell goes to the redo list)
          if ((s.V & 3) == 0) {
            const int V4 = s.V >> 2;
            for (int sp = 0; sp < 3; ++sp) {
              const int4* a = reinterpret_cast<const int4*>(g + sp * s.V);
              if (NARROW) {
                uint2* b = reinterpret_cast<uint2*>(cnt + sp * vmax);
                for (int i = sl; i < V4; i += H) {
                  const int4 x = a[i];
                  const uint32_t x0 = static_cast<uint32_t>(x.x), x1 = static_cast<uint32_t>(x.y);
                  const uint32_t x2 = static_cast<uint32_t>(x.z), x3 = static_cast<uint32_t>(x.w);
                  big |= (x0 | x1 | x2 | x3) > 0xFFFFu;
                  b[i] = make_uint2((x0 & 0xFFFFu) | (x1 << 16), (x2 & 0xFFFFu) | (x3 << 16));
                }
              } else {
                int4* b = reinterpret_cast<int4*>(cnt + sp * vmax);
                for (int i = sl; i < V4; i += H) b[i] = a[i];
              }
            }
          } else {
            for (int sp = 0; sp < 3; ++sp)
              for (int i = sl; i < s.V; i += H) {
                const int32_t x = g[sp * s.V + i];
                if (NARROW) big |= static_cast<uint32_t>(x) > 0xFFFFu;
                cnt[sp * vmax + i] = static_cast<CT>(x);
              }
          }
          __syncwarp(segmask);
          step = *sv->step + step_off;
          key0 = static_cast<uint32_t>(sv->seed);
          key1 = static_cast<uint32_t>(sv->seed >> 32);
          word3 = sv->tissue_id | (kTagChi << 24);
          bool ovf = false, bad_state = false;
          const bool bad_qb = !QB && s.qb > 0;  // the launcher never lets this happen
          uint64_t S = 0;
          for (int i = 0; i < s.B; ++i) {
            const int v = (sl << s.lb) + i;
            if (v < s.V) {
              // promoter model: bound sites never exceed the voxel's sites
              if (pm && cnt[2 * vmax + v] > static_cast<int32_t>(v == s.centre)) bad_state = true;
              S += seg_voxel_total<(GEN != 0)>(cnt, vmax, v, s, sv->q, pm, ovf, oob);
              if (PRE) pre[TSG_IDX(v, vmax, oob)] = S;
            }
            if (SUB && ((i + 1) & ((1 << s.ls) - 1)) == 0) {
              // the end of sub-block i >> ls (voxels past V add nothing); the
              // entries past the block's last sub-block end as its total
              const int kk = i >> s.ls;
#pragma unroll
              for (int k = 0; k < 4; ++k)
                if (k >= kk) sb[k] = S;
            }
          }
          P = S;
  #pragma unroll
          for (int o = 1; o < H; o <<= 1) {
            const uint64_t y = __shfl_up_sync(segmask, P, o, H);
            if (sl >= o) P += y;
          }
          A = __shfl_sync(segmask, P, H - 1, H);
          tnow = 0.0;
          e = 0;
          e0 = 0;
          draw_event(e0 + sl, step, cell, word3, key0, key1, Em, Ek, Rb);
          next_ok = false;
          err = (NARROW && __any_sync(segmask, big)) ? kErrNarrow
                : bad_qb                            ? kErrInternal
                : __any_sync(segmask, bad_state)    ? kErrState
                : __any_sync(segmask, ovf)          ? kErrOverflow
                                                    : 0;
          have = true;
          __syncwarp(segmask);
        }
      }
    }
    if (__all_sync(kFull, done)) break;

    // ---- one event of every active segment (the whole warp in step) -------
    const bool act = have;
    const bool PM = GEN == 2 ? true : pm;  // this segment's cell runs the promoter model
    const int qb = QB ? s.qb : 0;  // log2 of the voxels a lane covers in the selected block
    int j = static_cast<int>(e - e0);
    // Draws come in batches of H events per segment.  A segment that has used
    // its batch takes the prepared next one if it has it; when some segment
    // has none, every segment without a prepared batch draws in the same
    // pass, so the segments of a warp share the Philox / -ln work.
    bool must = false;
    if (act && j == H) {
      if (next_ok) {
        Em = Em2;
        Ek = Ek2;
        Rb = Rb2;
        next_ok = false;
        e0 += H;
        j = 0;
      } else {
        must = true;
      }
    }
    if (__any_sync(kFull, must)) {
      if (must || (act && !next_ok)) {
        const uint32_t base = e0 + H;  // the batch after the one in use
        uint64_t m_, r_;
        int k_;
        draw_event(base + sl, step, cell, word3, key0, key1, m_, k_, r_);
        if (must) {
          Em = m_;
          Ek = k_;
          Rb = r_;
          e0 += H;
          j = 0;
        } else {
          Em2 = m_;
          Ek2 = k_;
          Rb2 = r_;
          next_ok = true;
        }
      }
    }
    const uint64_t mE = __shfl_sync(kFull, Em, j, H);
    const int kE = __shfl_sync(kFull, Ek, j, H);
    const uint64_t R64 = __shfl_sync(kFull, Rb, j, H);
    const uint64_t Aa = act ? A : 0ull;
    const double tn = __dadd_rn(tnow, tau_from(F53{mE, kE}, kE < 0 || Aa == 0ull, Aa | (Aa == 0ull)));

    const uint64_t r = __umul64hi(R64, Aa);
    const unsigned m1 = (__ballot_sync(kFull, r < P && act) >> (seg * H)) & kSegBits;
    const int L = m1 ? __ffs(m1) - 1 : 0;
    const uint64_t Pl = __shfl_sync(kFull, P, L > 0 ? L - 1 : 0, H);
    uint64_t r1 = r - (L > 0 ? Pl : 0ull);
    // The second level searches the nsec voxels from vb, lane sl covering
    // voxels vb + sl*2^lq .. + 2^lq - 1 (lq = qb in the prefix layout, else 0)
    int vb = L << s.lb;
    int nsec = s.B;
    const int lq = PRE ? qb : 0;
    const QRates& q = sv->q;
    uint64_t pv = ~0ull;
    bool bad_s = false;
    if (PRE) {
      const int q0 = vb + (sl << qb);
      if ((sl << qb) < s.B && q0 < s.V)
        pv = pre[TSG_IDX(min(q0 + (1 << qb) - 1, s.V - 1), vmax, oob)];
    } else {
      if (SUB) {
        // the sub-block of lane L's block that holds r1: every lane finds
        // the first of its own running sums above r1, and lane L's answer is
        // taken (an empty sub-block is never chosen: its sum equals the one
        // before it)
        int kq = -1;
        uint64_t below = 0ull;
#pragma unroll
        for (int k = 3; k >= 0; --k)
          if (k < (1 << qb) && r1 < sb[k]) {
            kq = k;
            below = k > 0 ? sb[k > 0 ? k - 1 : 0] : 0ull;
          }
        const int ks = __shfl_sync(kFull, kq, L, H);
        const uint64_t bs = __shfl_sync(kFull, below, L, H);
        bad_s = ks < 0;
        if (ks > 0) {
          vb += ks << s.ls;
          r1 -= bs;
        }
        nsec = 1 << s.ls;
      }
      // the propensities of those voxels, recomputed (one per lane) and
      // scanned across the segment
      bool unused = false;
      const bool mine = act && sl < nsec && vb + sl < s.V;
      const int bx = mine ? vb + sl : 0;
      const int bi = static_cast<int>(TSG_IDX(bx, vmax, oob));
      const uint32_t bD = static_cast<uint32_t>(cnt[bi]);
      const uint32_t bN = static_cast<uint32_t>(cnt[vmax + bi]);
      const uint32_t bR = static_cast<uint32_t>(cnt[2 * vmax + bi]);
      const uint64_t bh = GEN == 2 ? 0ull : hreg.get(q, bR, mine && !PM);
      uint64_t cx = mine ? voxel_total_of<(GEN != 0)>(bx, bD, bN, bR, bh, s, q, PM, unused) : 0ull;
#pragma unroll
      for (int o = 1; o < H; o <<= 1) {
        const uint64_t y = __shfl_up_sync(kFull, cx, o, H);
        if (sl >= o) cx += y;
      }
      if (sl < nsec && vb + sl < s.V) pv = cx;
    }
    const unsigned m2 = (__ballot_sync(kFull, r1 < pv) >> (seg * H)) & kSegBits;
    const int i2 = m2 ? __ffs(m2) - 1 : 0;
    const uint64_t pp = __shfl_sync(kFull, pv, i2 > 0 ? i2 - 1 : 0, H);
    uint64_t r2 = r1 - (i2 > 0 ? pp : 0ull);
    int v = vb + (i2 << lq);
    bool bad_q = false;
    if (PRE && QB) {
      // the voxel inside lane i2's run of Q = 2^qb voxels: the segment's
      // lanes read H of the run's prefix entries at a time and one ballot
      // finds the first that exceeds r1 (Q = 1 re-finds lane i2's voxel).
      // Every lane of the warp runs the same trip count (the warp's largest
      // Q), so the collectives inside stay converged.
      const int qmax = static_cast<int>(__reduce_max_sync(kFull, 1u << qb));
      uint64_t before_v = i2 > 0 ? pp : 0ull;
      int pick = -1;
      for (int k0 = 0; k0 < qmax; k0 += H) {
        const int idx = v + k0 + sl;
        const bool in = k0 + sl < (1 << qb) && idx < s.V;
        const uint64_t x = in ? pre[TSG_IDX(idx, vmax, oob)] : ~0ull;
        const unsigned mq = (__ballot_sync(kFull, in && r1 < x) >> (seg * H)) & kSegBits;
        const int kq = mq ? __ffs(mq) - 1 : 0;
        const uint64_t xprev = __shfl_sync(kFull, x, kq > 0 ? kq - 1 : 0, H);
        const uint64_t xlast = __shfl_sync(kFull, x, H - 1, H);
        if (pick < 0 && mq) {
          pick = v + k0 + kq;
          r2 = r1 - (kq > 0 ? xprev : before_v);
        }
        before_v = xlast;
      }
      bad_q = pick < 0;
      v = pick < 0 ? v : pick;
    }
    const bool bad1 = act && Aa != 0ull &&
                      (m1 == 0u || m2 == 0u || (i2 << lq) >= nsec || v >= s.V || bad_q || bad_s);
    if (bad1 || v >= s.V) v = 0;

    // channel: closed-form running sums
    const int vi = static_cast<int>(TSG_IDX(v, vmax, oob));
    const uint32_t D = static_cast<uint32_t>(cnt[vi]);
    const uint32_t N = static_cast<uint32_t>(cnt[vmax + vi]);
    const uint32_t R = static_cast<uint32_t>(cnt[2 * vmax + vi]);
    const uint32_t hm = dir_mask(v, s);
    const uint64_t hR = GEN == 2 ? 0ull : hreg.get(q, R, act && !PM);
    uint64_t c0, c1, X;
    voxel_terms<(GEN != 0)>(PM, q, v, s, D, N, R, hR, c0, c1, X);
    const uint64_t C = chan_cum(cl, lk, q, c0, c1, D, N, R, X, hm);
    const uint64_t Cb = H == 8 ? chan_cum(cl2, lk2, q, c0, c1, D, N, R, X, hm) : ~0ull;
    uint64_t C16 = 0, C17 = 0, C18;
    if (H <= 16) {
      // C_16..C_18 from C_15: +x hop of R (if that neighbour exists), slots 17, 18
      const uint64_t C15 = __shfl_sync(kFull, H == 16 ? C : Cb, H == 16 ? 15 : 7, H);
      C16 = C15 + (((hm >> 3) & 1u) ? q.hopR * R : 0ull);
      C17 = C16 + q.k_in * X;
      C18 = C17 + q.k_off * R;
    } else {
      C18 = __shfl_sync(kFull, C, 18, H);
    }
    const unsigned m3 = (__ballot_sync(kFull, r2 < C) >> (seg * H)) & kSegBits;
    const unsigned m3b = H == 8 ? (__ballot_sync(kFull, r2 < Cb) >> (seg * H)) & kSegBits : 0u;
    int ch = m3 ? __ffs(m3) - 1
                : m3b ? H + __ffs(m3b) - 1
                      : 16 + static_cast<int>(r2 >= C16) + static_cast<int>(r2 >= C17);
    const bool bad = bad1 || (act && Aa != 0ull && !(r2 < C18));
    const uint64_t a_old_v = C18;
    if (ch > 18) ch = 18;

    const bool fire = act && err == 0 && !bad && Aa != 0ull && before(tn, dt);
    // the channel's effect, decoded without branches
    const bool hop = ch >= 5 && ch <= 16;
    const int hs = (ch - 5) >> 2, hd = (ch - 5) & 3;
    int u = hop ? v + (hd == 0 ? -1 : hd == 1 ? 1 : hd == 2 ? -s.n : s.n) : -1;
    const bool bad_u = fire && hop && (u < 0 || u >= s.V);
    if (u >= s.V) u = -1;
    const bool fire_ok = fire && !bad_u;
    uint64_t a_old_u = 0;
    if (PRE && u >= 0)
      a_old_u = pre[TSG_IDX(u, vmax, oob)] -
                ((u & (s.B - 1)) ? pre[TSG_IDX(u - 1, vmax, oob)] : 0ull);
    __syncwarp();
    if (fire_ok && sl < 3) {
      // Notch-Delta: slot 17 is D + N -> R, 18 is R -> D + N.  Promoter:
      // slot 1 (unbinding) also frees the site (R - 1), slot 17 (binding) is
      // N + F -> R, and slots 4, 13..16 and 18 have no propensity.
      const bool pm1 = GEN != 0 && PM && ch == 1, pm17 = GEN != 0 && PM && ch == 17;
      // the three lanes' (species, change, voxel), chosen without branches
      const int sp0 = ch <= 1 ? ch : ch <= 4 ? ch - 2 : hop ? hs : ch == 17 ? (pm17 ? 1 : 0) : 2;
      const int dd0 = ch <= 1 ? 1 : -1;
      const int sp1 = hop ? hs : ch == 17 ? 1 : 0;
      const int dd1 = hop ? 1 : ch == 17 ? (pm17 ? 0 : -1) : ch == 18 ? 1 : 0;
      const int sp2 = (ch == 17 || pm1) ? 2 : 1;
      const int dd2 = ch >= 17 ? 1 : pm1 ? -1 : 0;
      const int sp = sl == 0 ? sp0 : sl == 1 ? sp1 : sp2;
      const int dd = sl == 0 ? dd0 : sl == 1 ? dd1 : dd2;
      const int xv = (sl == 1 && hop) ? u : v;
      if (dd != 0) {
        CT* c = &cnt[TSG_IDX(sp * vmax + xv, 3 * vmax, oob)];
        const int nv = static_cast<int>(*c) + dd;
        *c = static_cast<CT>(nv);
        if (nv > (NARROW ? 0xFFFF : kCountMax)) err |= NARROW ? kErrNarrow : kErrOverflow;
      }
    }
    __syncwarp();
    bool ovf = false;
    uint64_t dv, du;
    if (PRE) {
      // lane 0 the new total of v, lane 1 that of u (the hop's target)
      const int xv = (sl == 1 && u >= 0) ? u : v;
      uint64_t a_new;
      if (decltype(hreg)::kSets == 0) {  // table lookups, inside the active branch
        a_new = act ? seg_voxel_total<(GEN != 0)>(cnt, vmax, xv, s, q, PM, ovf, oob) : 0ull;
      } else {  // register lookups: every lane takes part in the shuffles
        const int xi = static_cast<int>(TSG_IDX(xv, vmax, oob));
        const uint32_t xD = static_cast<uint32_t>(cnt[xi]);
        const uint32_t xN = static_cast<uint32_t>(cnt[vmax + xi]);
        const uint32_t xR = static_cast<uint32_t>(cnt[2 * vmax + xi]);
        const uint64_t xh = GEN == 2 ? 0ull : hreg.get(q, xR, act && !PM);
        a_new = act ? voxel_total_of<(GEN != 0)>(xv, xD, xN, xR, xh, s, q, PM, ovf) : 0ull;
      }
      dv = __shfl_sync(kFull, a_new, 0, H) - a_old_v;
      du = __shfl_sync(kFull, a_new, 1, H) - a_old_u;
    } else {
      const int vi2 = static_cast<int>(TSG_IDX(v, vmax, oob));
      const uint32_t vD = static_cast<uint32_t>(cnt[vi2]);
      const uint32_t vN = static_cast<uint32_t>(cnt[vmax + vi2]);
      const uint32_t vR = static_cast<uint32_t>(cnt[2 * vmax + vi2]);
      const uint64_t vh = GEN == 2 ? 0ull : hreg.get(q, vR, act && !PM);
      dv = (act ? voxel_total_of<(GEN != 0)>(v, vD, vN, vR, vh, s, q, PM, ovf) : 0ull) - a_old_v;
      // one molecule of species hs arrived at u: the change of u's total in
      // closed form (the total is affine in D and N apart from k_in X)
      du = 0;
      if (act && u >= 0) {
        const int ui = static_cast<int>(TSG_IDX(u, vmax, oob));
        const uint32_t Du = static_cast<uint32_t>(cnt[ui]);
        const uint32_t Nu = static_cast<uint32_t>(cnt[vmax + ui]);
        const uint32_t Ru = static_cast<uint32_t>(cnt[2 * vmax + ui]);
        const int nnu = __popc(dir_mask(u, s));
        if (GEN != 0 && PM) {  // X = N F: a Delta adds cD, a NICD adds cN + k_a F (R never hops)
          const uint32_t Fu = static_cast<uint32_t>(u == s.centre) - Ru;
          du = hs == 0 ? q.cD[nnu] : q.cN[nnu] + q.k_in * Fu;
        } else if (hs == 0) {
          du = q.cD[nnu] + q.k_in * Nu;
        } else if (hs == 1) {
          du = q.cN[nnu] + q.k_in * Du;
        } else {
          du = q.cRo[nnu] + (hill_q(q, Ru) - hill_q(q, Ru - 1u));
        }
        if (((Du | Nu | Ru) >= q.small) && fire_ok) {
          bool o2 = false;  // large counts: check the new total exactly
          seg_voxel_total<(GEN != 0)>(cnt, vmax, u, s, q, PM, o2, oob);
          ovf |= o2;
        }
      }
    }
    if (fire_ok) {
      const int bv = v >> s.lb;
      P += sl >= bv ? dv : 0ull;
      A += dv;
      if (SUB) {  // the owning lane's sub-block sums from v's sub-block on
        const int kv = (v & (s.B - 1)) >> s.ls;
#pragma unroll
        for (int k = 0; k < 4; ++k) sb[k] += (sl == bv && k >= kv) ? dv : 0ull;
      }
      if (u >= 0) {
        const int bu = u >> s.lb;
        P += sl >= bu ? du : 0ull;
        A += du;
        if (SUB) {
          const int ku = (u & (s.B - 1)) >> s.ls;
#pragma unroll
          for (int k = 0; k < 4; ++k) sb[k] += (sl == bu && k >= ku) ? du : 0ull;
        }
      }
      if (PRE && (sl << qb) < s.B) {
        // prefix entries from the changed voxel to the end of its block
        for (int kq = 0; kq < (1 << qb); ++kq) {
          const int off = (sl << qb) + kq;  // position inside the block
          const int iv = (bv << s.lb) + off;
          if (off >= (v & (s.B - 1)) && iv < s.V) pre[TSG_IDX(iv, vmax, oob)] += dv;
          if (u >= 0) {
            const int iu = ((u >> s.lb) << s.lb) + off;
            if (off >= (u & (s.B - 1)) && iu < s.V) pre[TSG_IDX(iu, vmax, oob)] += du;
          }
        }
      }
      if (GEN != 0 && sl == 0) trace_event(*sv, step, kTagChi, cell, e, tn, static_cast<uint32_t>(v),
                                      static_cast<uint32_t>(ch));
      tnow = tn;
      ++e;
      if (e == 0xFFFFFFFFu) err |= kErrEventIndex;
      if (ovf) err |= kErrOverflow;
    }
    if (bad || bad_u) err |= kErrInternal;
    if (kChecked && oob && act) err |= kErrBounds;
    __syncwarp();

    // ---- a segment whose cell is finished writes it back ------------------
    const unsigned seg_err = (__ballot_sync(kFull, err != 0) >> (seg * H)) & kSegBits;
    const bool finish = act && (!fire_ok || seg_err != 0u);
    if (finish) {
      if (NARROW && __any_sync(segmask, (err & kErrNarrow) != 0)) {
        // a count passed 65535: the cell stays as it was, for the 32-bit pass
        if (sl == 0) redo[atomicAdd(redo_n, 1u)] = make_uint2(vidx, cell);
      } else {
        if ((s.V & 3) == 0) {
          const int V4 = s.V >> 2;
          for (int sp = 0; sp < 3; ++sp) {
            int4* a = reinterpret_cast<int4*>(g + sp * s.V);
            if (NARROW) {
              const uint2* b = reinterpret_cast<const uint2*>(cnt + sp * vmax);
              for (int i = sl; i < V4; i += H) {
                const uint2 x = b[i];
                a[i] = make_int4(static_cast<int>(x.x & 0xFFFFu), static_cast<int>(x.x >> 16),
                                 static_cast<int>(x.y & 0xFFFFu), static_cast<int>(x.y >> 16));
              }
            } else {
              const int4* b = reinterpret_cast<const int4*>(cnt + sp * vmax);
              for (int i = sl; i < V4; i += H) a[i] = b[i];
            }
          }
        } else {
          for (int sp = 0; sp < 3; ++sp)
            for (int i = sl; i < s.V; i += H)
              g[sp * s.V + i] = static_cast<int32_t>(cnt[sp * vmax + i]);
        }
        const int e_or = static_cast<int>(__reduce_or_sync(segmask, static_cast<unsigned>(err)));
        if (sl == 0) {
          sv->ev_last[cell] = e;
          sv->t_last[cell] = tnow;
          sv->ev_total[cell] += e;
          if (e_or) atomicOr(sv->err, e_or);
        }
      }
      err = 0;
      have = false;
      __syncwarp(segmask);
    }
  }
}

}  // namespace

}  // namespace tsg
