/*
 * tissue.h -- C ABI of the GB300 operator-split tissue SSA (libtissue.so).
 *
 * The method (arXiv 1806.10889, "Orchestral"):
 *   A tissue is a layer of identical cells, each with at most four neighbours
 *   (Sec. III-A1).  Time advances by Lie operator splitting (Sec. II; Fig. 1):
 *   in every step of length dt the intracellular module chi advances every
 *   cell independently (Sec. II-A1), then the signalling module S advances
 *   every pair of neighbouring cells independently (Sec. II-A2).  The
 *   translations T_{chi->S} and T_{S->chi} (Sec. II-B) gather a face's
 *   boundary voxels from the two cells and write the result back.  Every
 *   module call runs on its own clock over [0, dt) (the per-cell "end_time"
 *   of the network file, Fig. 2) and draws from its own seeded stream
 *   (the "-seed" of the module command lines, Fig. 3).
 *
 *   chi here is a lattice RDME on an n x n voxel grid solved by the exact
 *   direct-method SSA, with one of two single-cell models (tissue_model, or
 *   the paper's promoter model, tissue_promoter_model); S is the Delta-Notch
 *   reaction across a shared face, with
 *   every boundary voxel coupled to a single face (Sec. III-A1), realised as
 *   an x-face phase followed by a y-face phase.
 *
 * State layout (device memory, owned by the caller):
 *   int32 counts[cell][species][voxel], species D = 0, N = 1, R = 2,
 *   cell c = cy * width + cx, voxel v = vy * n + vx.
 *   tissue_state_bytes() gives its size.  The base must be 16-byte aligned.
 *
 * Arithmetic contract (exactly reproducible; the CPU oracle defines it):
 *   - Philox4x32-10, key = seed, counter = (event, step, unit,
 *     tissue_id | tag << 24) with tag 1 = chi, 2 = x-face, 3 = y-face,
 *     4 = initial counts, 5 and 6 = the second face half-steps of Strang
 *     splitting, 7..9 = placement of a well-mixed cell's D, N, R.
 *   - Propensities are integers in units of 2^-32 per unit time; a rate x is
 *     quantised once as round-half-even(x * 2^32).
 *   - Event times are IEEE binary64: tau = E / (A * 2^-32) with E the
 *     fixed-point -ln(u1); an event fires iff t + tau < dt.
 *
 * Threading: a tissue handle is not thread-safe; use one handle per host
 * thread.  All device work is ordered on the stream given at creation.
 *
 * Errors: every int-returning call returns TISSUE_OK (0) or a negative
 * TISSUE_E_* code; nothing is thrown across the ABI.  Device-side errors
 * (count or propensity overflow) are latched in a device flag and reported
 * by the next synchronising call (tissue_read_counts, tissue_read_stats,
 * tissue_total_events, tissue_sync).
 */
#ifndef TISSUE_H
#define TISSUE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TISSUE_OK 0
#define TISSUE_E_ARG (-1)      /* invalid argument (sizes, ranges, null pointers) */
#define TISSUE_E_NOMEM (-2)    /* library scratch allocation failed */
#define TISSUE_E_NOMODEL (-3)  /* tissue_step before tissue_set_model */
#define TISSUE_E_OVERFLOW (-4) /* a count passed 2^30-1 or a propensity reached 2^52 */
#define TISSUE_E_CUDA (-5)     /* a CUDA runtime call failed */
#define TISSUE_E_TIMEOUT (-6)  /* a bounded device wait gave up */
#define TISSUE_E_BUDGET (-7)   /* admission refused: memory budget exceeded */
#define TISSUE_E_STATE (-9)    /* promoter model: a voxel holds more bound sites than sites */
#define TISSUE_E_BOUNDS (-10)  /* checked build only: a kernel caught an index out of range */

#define TISSUE_COUNT_MAX ((1 << 30) - 1)

typedef struct tissue tissue; /* opaque, library-owned */

typedef struct {
  uint32_t width, height; /* cells; the tissue is width x height, not periodic; >= 1 each */
  uint32_t n;             /* voxels per cell side, 2..32 (V = n*n voxels per cell) */
  uint32_t tissue_id;     /* < 2^24; part of every Philox counter */
  uint64_t seed;          /* Philox key */
  double init_lambda[3];  /* Poisson mean of the initial D, N, R count per voxel, 0..700 */
} tissue_desc;

/* Rates (all finite, >= 0 and < 2^20; K > 0).  Per voxel:
 *   D production kD / (1 + (R/K)^2)      N production kN
 *   decay gD*D, gN*N, gR*R
 *   hop of each molecule to each existing neighbour voxel at hopD, hopN, hopR
 *   D + N -> R at k_in*D*N and R -> D + N at k_off*R (in-voxel; 0 in the tissue model)
 * Across a face, for every voxel pair (i in one cell, j in the other):
 *   D(i) + N(j) -> R(j) at k_bind*D(i)*N(j), in both directions. */
typedef struct {
  double kD, K, kN, gD, gN, gR, hopD, hopN, hopR, k_in, k_off, k_bind;
} tissue_model;

/* The paper's own Notch model (arXiv 1806.10889, Sec. III-A1, Table I) on the
 * voxel lattice.  Each cell holds one DNA promoter site at voxel (n/2, n/2).
 * The species slots are read as D = Delta, N = NICD, and R = bound promoter
 * sites (0 or 1 at the promoter voxel, 0 elsewhere).  A voxel's free sites
 * are F = [v is the promoter voxel] - R.  Per voxel:
 *   transcription F -> F + D at tD*F; NICD binding N + F -> R at ka*N*F;
 *   unbinding R -> N + F at kd*R; decay of D and N at d each (DNA does not
 *   decay); hop of each Delta and NICD to each existing neighbour voxel at hop.
 * Across a face, for every voxel pair (i in one cell, j facing it in the other):
 *   Delta(i) -> NICD(j) at kN*D(i), in both directions.
 * Rates are per unit time in lattice units (all finite, >= 0 and < 2^20).
 * A state may not hold more bound sites than sites; if it does, the next
 * step's chi leaves that cell unchanged and latches TISSUE_E_STATE.  Initial
 * counts with init_lambda[2] = 0 start with every promoter free. */
typedef struct {
  double tD, ka, kd, kN, d, hop;
} tissue_promoter_model;

/* Bytes of the caller-owned state buffer: width*height*3*n*n*4.
 * Returns 0 for an invalid descriptor. */
size_t tissue_state_bytes(const tissue_desc* desc);

/* Bytes the library itself allocates for one tissue (statistics, flags,
 * tables), for memory-budget admission.  0 for an invalid descriptor. */
size_t tissue_scratch_bytes(const tissue_desc* desc);

/* Bind a tissue to a caller-owned device buffer (>= tissue_state_bytes,
 * 16-byte aligned) and a CUDA stream (NULL = legacy default stream), and
 * enqueue the Poisson initial counts (Sec. III-A1 tissue; per-cell seeds of
 * Fig. 2).  The buffer must outlive the handle.  On success *out receives the
 * handle and the global step index is 0. */
int tissue_create(const tissue_desc* desc, void* dev_counts, size_t bytes, void* cuda_stream,
                  tissue** out);

/* Set (or replace, between steps) the model; the rates are copied. */
int tissue_set_model(tissue* t, const tissue_model* model);

/* Set (or replace, between steps) the promoter model instead; the rates are
 * copied.  A promoter-model tissue steps with the persistent chi kernel only:
 * tissue_step returns TISSUE_E_ARG while the launch configuration selects
 * TISSUE_KERNEL_WARP, and tissue_step_noalloc does not take it. */
int tissue_set_promoter_model(tissue* t, const tissue_promoter_model* model);

/* Mixed-fidelity tissues (arXiv 1806.10889, Sec. IV: detailed modules where
 * cells signal, coarser ones elsewhere).  host[c] (n = width*height bytes)
 * selects the chi of cell c: 0 = the lattice RDME (default), 1 = well mixed.
 * A well-mixed cell keeps its molecules in the same voxel layout between
 * steps, so S and every reader see one format.  Its chi:
 *   1. sums the cell's voxels into totals D, N, R;
 *   2. runs the direct-method SSA on the totals over [0, dt), the cell one
 *      compartment of V voxel volumes:
 *      - Notch-Delta: D production V*kD / (1 + (R/(V*K))^2), N production
 *        V*kN, decays gD*D, gN*N, gR*R, D + N -> R at (k_in/V)*D*N,
 *        R -> D + N at k_off*R;
 *      - promoter: transcription tD*F with F = 1 - R, unbinding kd*R,
 *        decays d*D, d*N, binding (ka/V)*N*F;
 *   3. places every molecule in a uniformly random voxel
 *      v = floor(w * V / 2^32), where w is word (i mod 4) of the Philox block
 *      (i / 4, step, cell, tissue_id | (7 + species) << 24) for the i-th
 *      molecule of the species.  The promoter model's bound site stays on the
 *      promoter voxel.
 * The Hill term is binary64, left to right, rounded to nearest at each
 * operation, then quantised.  k/V is one binary64 division, then quantised.
 * On an error the cell is left unchanged.  Copies the array and waits for
 * the copy.  Only the persistent chi kernel runs well-mixed cells
 * (tissue_step returns TISSUE_E_ARG with TISSUE_KERNEL_WARP). */
int tissue_set_cell_fidelity(tissue* t, const uint8_t* host, size_t n);

/* Overwrite the state from host memory (n int32 values, exactly
 * width*height*3*V) and set the global step index (checkpoint resume).
 * Synchronises the stream.  Clears the device error flag. */
int tissue_write_counts(tissue* t, const int32_t* host, size_t n, uint32_t step_index);

/* Enqueue n_steps splitting steps of length dt (> 0, finite): for each step
 * k, chi on every cell, S on every x-face, then S on every y-face.
 * Asynchronous on the tissue's stream; advances the global step index. */
int tissue_step(tissue* t, double dt, uint32_t n_steps);

/* Splitting scheme of tissue_step (arXiv 1806.10889, Sec. II: modules run one
 * after the other over dt; the scheme fixes the order).
 *   TISSUE_SPLIT_LIE (default): chi(dt), S_x(dt), S_y(dt).
 *   TISSUE_SPLIT_STRANG: S_x(dt/2), S_y(dt/2), chi(dt), S_y(dt/2), S_x(dt/2);
 *     second order in dt; the second half-steps draw from Philox tags 5 and
 *     6.  The face rows of tissue_read_stats then hold the last half-step. */
#define TISSUE_SPLIT_LIE 0u
#define TISSUE_SPLIT_STRANG 1u
int tissue_set_splitting(tissue* t, uint32_t scheme);

/* As tissue_step, but also measures the device time of each phase with CUDA
 * events recorded on the tissue's stream around every launch, and waits for
 * the work to finish.  ms_chi receives the summed duration of the chi
 * launches, ms_sig that of the face phases (either may be NULL). */
int tissue_step_timed(tissue* t, double dt, uint32_t n_steps, double* ms_chi, double* ms_sig);

/* Copy the state to host memory (n int32 values) after the queued work;
 * synchronises the stream and reports a latched device error. */
int tissue_read_counts(tissue* t, int32_t* host, size_t n);

/* Statistics of the LAST step, each laid out [3][cells]: row 0 chi of the
 * cell, row 1 the x-face the cell owns (its +x face), row 2 its y-face
 * (0 where the cell owns no such face).  n_events: fired events; t_last:
 * local time of the last fired event (0.0 if none).  n = 3*cells.
 * Either pointer may be NULL.  Synchronises. */
int tissue_read_stats(tissue* t, uint64_t* n_events, double* t_last, size_t n);

/* Events fired since creation: out[0] chi, out[1] x-faces, out[2] y-faces.
 * Synchronises. */
int tissue_total_events(tissue* t, uint64_t out[3]);

/* Global step index (the next step to run). */
int tissue_get_step(const tissue* t, uint32_t* step_index);

/* Wait for the queued work; report a latched device error. */
int tissue_sync(tissue* t);

/* Launch shape of the chi kernel: warps (cells) per block, 1..16, of the
 * one-warp-per-cell kernel.  Results never depend on it. */
int tissue_set_launch(tissue* t, uint32_t chi_warps_per_block);

/* Kernel choice for chi.  Results never depend on it: every configuration
 * computes the same trajectory bit for bit. */
#define TISSUE_KERNEL_WARP 0u       /* one warp per cell, one launch over all cells */
#define TISSUE_KERNEL_PERSISTENT 1u /* persistent kernel, cells taken from a work list */
#define TISSUE_LAYOUT_PREFIX 0u    /* persistent kernel keeps per-voxel prefix sums (20 B/voxel; 14 B with 16-bit counts, cells of V > 256) */
#define TISSUE_LAYOUT_RECOMPUTE 1u /* counts only (12 B/voxel; 6 with 16-bit counts, cells of V > 256); <= 4 warps per block, V <= lanes^2 or, for the Notch-Delta model, 16 lanes and V <= 1024 or 8 lanes and V <= 256 */
typedef struct {
  uint32_t kernel;          /* TISSUE_KERNEL_WARP or TISSUE_KERNEL_PERSISTENT */
  uint32_t lanes_per_cell;  /* persistent kernel: 32, 16 or 8 (1, 2 or 4 cells per warp) */
  uint32_t warps_per_block; /* 1..16 (warp kernel) or 1..8 (persistent kernel) */
  uint32_t blocks;          /* persistent kernel grid; 0 = enough to fill every SM */
  uint32_t smem_layout;     /* persistent kernel: TISSUE_LAYOUT_PREFIX or _RECOMPUTE */
} tissue_launch;
/* The default after tissue_create: persistent kernel; for a tissue of at
 * most 1024 cells 32 lanes and 2 warps per block, prefix layout (one cell per
 * warp: the shortest event chain, which sets the time when the machine is
 * not full); otherwise by cell size: V <= 64, 8 lanes and 4 warps per block,
 * prefix layout; 64 < V <= 256, 8 lanes, 2 warps per block and the recompute
 * layout above 6080 cells, else 16 lanes and 4 warps, prefix layout;
 * 256 < V <= 1024, 16 lanes, 2 warps per block and the recompute layout
 * above 2128 cells, else 32 lanes and 2 warps, prefix layout (the recompute
 * layout holds more cells per SM; the thresholds are one wave of the prefix
 * launch on a 152-SM GB300).  A recompute launch with more voxels per block
 * than lanes that the tissue's model cannot take (the promoter model, a
 * trace) runs the prefix launch of its cell size instead; results never
 * depend on it. */
int tissue_set_launch_config(tissue* t, const tissue_launch* config);
int tissue_get_launch_config(const tissue* t, tissue_launch* config);

/* ---- Batching: many tissues in one persistent launch per step ----------
 * The members keep their own buffers, models, statistics and step indices;
 * one batch step runs chi for the cells of every member with the persistent
 * kernel (one launch per cell-size class, cells taken from a work list),
 * then all members' x-faces, then all y-faces, then advances every member's
 * step index.  The step is captured in a CUDA graph on first use (per dt) and
 * replayed.  Each tissue's trajectory is bit-identical to stepping it alone.
 * While a batch exists, step its members only through it; a member's model
 * must not change (recreate the batch instead).  The members must outlive
 * the batch.  Members of both models may share a batch and a chi launch. */
typedef struct tissue_batch tissue_batch;

/* count >= 1 distinct tissues with models set, on the current device.
 * cuda_stream: the stream batch steps run on (NULL = legacy default stream,
 * which is not graph-captured).  Waits for the members' pending work. */
int tissue_batch_create(tissue* const* members, uint32_t count, void* cuda_stream,
                        tissue_batch** out);

/* Launch shape of the chi launch of the class of cells with V voxels:
 * 8, 16 or 32 lanes per cell, 1..8 warps per block (1..4 with the recompute
 * layout, which also needs V <= lanes^2, or for a Notch-Delta class 16 lanes
 * and V <= 1024 or 8 lanes and V <= 256), shared-memory layout
 * TISSUE_LAYOUT_*.  The default is
 * the single-tissue default for that V.  Results never depend on it. */
int tissue_batch_set_class_launch(tissue_batch* b, uint32_t V, uint32_t lanes_per_cell,
                                  uint32_t warps_per_block, uint32_t smem_layout);

/* Split-step schedule: how many splitting steps one captured graph holds
 * (1..64, default 1); n_steps not divisible by it end with direct launches. */
int tissue_batch_set_schedule(tissue_batch* b, uint32_t steps_per_graph);

/* Splitting scheme of the batch's steps (TISSUE_SPLIT_LIE or _STRANG). */
int tissue_batch_set_splitting(tissue_batch* b, uint32_t scheme);

/* Enqueue n_steps batch steps of length dt on the batch stream. */
int tissue_batch_step(tissue_batch* b, double dt, uint32_t n_steps);

/* Wait for the batch stream; report the first member's latched device error. */
int tissue_batch_sync(tissue_batch* b);

/* Members, cell-size classes and total cells of the batch (any may be NULL). */
int tissue_batch_info(const tissue_batch* b, uint32_t* n_members, uint32_t* n_classes,
                      uint64_t* n_cells);

/* State I/O of a whole batch: the batch form of tissue_write_counts and
 * tissue_read_counts (in the paper the modules hand each cell's state on
 * through files every step, Sec. II-B; these calls move the states of all
 * members between host and device memory instead), with every member's copy
 * queued on the batch stream and one wait for all of them.
 * host[i] (count entries, i in member order): member i's state, exactly
 * width*height*3*V int32 in the layout of tissue_read_counts; pinned host
 * memory makes the copies asynchronous DMA.  The caller owns the arrays. */

/* Write every member's state; step_index[i] (or NULL: unchanged) becomes
 * member i's global step index.  After the copies one device pass checks
 * every count lies in [0, TISSUE_COUNT_MAX], and the members' device error
 * flags are cleared; the call waits for all of it.  TISSUE_E_ARG if a count
 * is out of range (the members' states are then unspecified). */
int tissue_batch_write_counts(tissue_batch* b, const int32_t* const* host,
                              const uint32_t* step_index);

/* Copy every member's state to host[i] and wait; reports the first member's
 * latched device error in member order, as tissue_read_counts does. */
int tissue_batch_read_counts(tissue_batch* b, int32_t* const* host);

/* Cell-size class i (0 <= i < n_classes of tissue_batch_info; largest cells
 * first): its cell size V, the launch shape of its chi launch and its number
 * of lattice cells (any pointer may be NULL). */
int tissue_batch_class_info(const tissue_batch* b, uint32_t i, uint32_t* V,
                            uint32_t* lanes_per_cell, uint32_t* warps_per_block,
                            uint32_t* smem_layout, uint32_t* cells);

/* Diagnostic timing of batch steps (a measurement aid; the paper has no
 * counterpart).  With on = 1 every following step records CUDA events on the
 * batch stream around each class's chi launches and around the whole step;
 * a captured step holds them as event-record nodes of its graph.  Results
 * never depend on it.  Toggling it drops the captured graph. */
int tissue_batch_set_timing(tissue_batch* b, uint32_t on);

/* Device milliseconds of the last step enqueued with timing on (any pointer
 * may be NULL): the whole step; the chi phase (well-mixed and lattice
 * classes); the well-mixed chi launch (0 when the batch has no well-mixed
 * cell); and for each class i < n its chi launches (the 16-bit-count launch
 * and its 32-bit redo pass together), from when they became ready to run to
 * their end.  Classes run one after another, or overlapped (see
 * tissue_batch_set_overlap): then every class is ready from the start of the
 * chi phase, and a class that waits for SMs held by another counts that wait.
 * Waits for the batch stream.  TISSUE_E_ARG if timing is off or no timed
 * step has run. */
int tissue_batch_read_timing(tissue_batch* b, double* step_ms, double* chi_ms, double* wm_ms,
                             double* class_ms, uint32_t n);

/* Overlapped classes (on = 1, the default) or one after another (0).  The
 * chi launches of a step's classes run on separate streams: the first class
 * (the largest cells, which take longest) at the device's highest launch
 * priority, the others at the lowest, so their blocks fill the SMs the first
 * class's last wave frees instead of waiting for its slowest cells.  Results
 * never depend on it.  Changing it drops the captured graph. */
int tissue_batch_set_overlap(tissue_batch* b, uint32_t on);

void tissue_batch_destroy(tissue_batch* b);

/* Largest tissue (width*height cells) tissue_step_noalloc accepts. */
#define TISSUE_NOALLOC_MAX_CELLS 16384

/* Allocation-free steps (Lie splitting).  The paper has no counterpart; this exists for
 * callers that cannot allocate device memory when they advance a tissue (an
 * application that owns a fixed device-memory budget itself, or code where a
 * cudaMalloc would synchronise the device).  No cudaMalloc, cudaFree or
 * allocating library call is made: the scratch (Hill table, step counter,
 * error flag, cumulative counters; about 416 KB) is one static device array
 * that every device loading this library keeps until the process exits.
 *
 * dev_counts (in/out, device, 16-byte aligned): the state as in tissue_create.
 * step_index: global index of the first step (the Philox step word).
 * dev_n_events / dev_t_last (out, device, 3*width*height each): statistics of
 * the last step laid out as in tissue_read_stats.
 * Runs n_steps steps exactly as tissue_step would, on cuda_stream, and waits
 * for them; returns TISSUE_E_ARG if width*height > TISSUE_NOALLOC_MAX_CELLS
 * or an argument is invalid, TISSUE_E_OVERFLOW as tissue_read_counts would.
 * n_steps == 0 leaves the state and both outputs untouched, as tissue_step
 * does.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), also when n_steps == 0; make that first call before
 * any stream capture.
 * All calls share the one array: calls whose work overlaps on a device race. */
int tissue_step_noalloc(const tissue_desc* desc, const tissue_model* model, int32_t* dev_counts,
                        uint32_t step_index, double dt, uint32_t n_steps,
                        uint64_t* dev_n_events, double* dev_t_last, void* cuda_stream);

/* Diagnostic: check the event loop's integer implementation of the binary64
 * waiting time (tau = E / (A 2^-32), IEEE round-to-nearest) and clock test
 * against the GPU's FP64 unit on n_samples random and structured inputs
 * (seeded); *mismatches receives the number of differing results (0 expected).
 * Synchronises the device. */
int tissue_selftest_time(uint64_t n_samples, uint64_t seed, uint64_t* mismatches);

/* Event trace (tests and diagnostics; the paper has no counterpart).  While
 * a trace is on, every fired event of chi (lattice and well-mixed cells) and
 * of both face phases is recorded, in no particular order (sort by step,
 * kind, unit, e):
 *   step  global step index       kind  Philox tag of the module call
 *                                       (1 chi, 2/3 x/y faces, 5/6 their
 *                                       Strang second halves)
 *   unit  cell, or owner of the face  e  event index within the call
 *   t     local time of the event in [0, dt)
 *   site  voxel (chi lattice cells), 0 (well-mixed cells) or voxel pair (faces)
 *   channel  channel slot 0..18 (lattice), 0..6 (well mixed) or 0/1 (faces:
 *            0 = from the owner's side)
 * The layout equals the CPU oracle's trace record.  tissue_trace_begin
 * allocates room for `capacity` records (device memory) and clears the
 * count; recording starts with the next step and uses the persistent chi
 * kernel (tissue_step returns TISSUE_E_ARG with TISSUE_KERNEL_WARP).
 * tissue_trace_read waits for the stream, copies min(count, capacity,
 * host capacity) records and stores the count (which may exceed the
 * capacity: the excess was dropped).  tissue_trace_end frees the buffer. */
typedef struct {
  uint32_t step, kind, unit, e;
  double t;
  uint32_t site, channel;
} tissue_event;
int tissue_trace_begin(tissue* t, size_t capacity);
int tissue_trace_read(tissue* t, tissue_event* host, size_t capacity, size_t* n_recorded);
int tissue_trace_end(tissue* t);

/* Host-side fault injection for tests: the next n device allocations the
 * library makes (tissue_create, tissue_batch_create, tissue_trace_begin)
 * fail as an out-of-memory cudaMalloc would (TISSUE_E_NOMEM), without
 * touching the GPU.  n = 0 disarms it. */
int tissue_debug_fail_allocs(uint32_t n);

/* Release library scratch (not the caller's buffer or stream). */
void tissue_destroy(tissue* t);

const char* tissue_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
