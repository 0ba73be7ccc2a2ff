/*
 * tissue_oracle.h -- plain, slow CPU oracle of the operator-split tissue SSA.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Method (arXiv 1806.10889, "Orchestral"):
 *   - Lie operator splitting: each step of length dt runs the intracellular
 *     module chi on every cell independently, then the pairwise signalling
 *     module S on every pair of neighbouring cells (Sec. II; Fig. 1 text).
 *   - chi: per-cell internal kinetics, embarrassingly parallel over dt
 *     (Sec. II-A1).  Here a lattice RDME on an n x n voxel grid solved by the
 *     exact direct-method SSA.
 *   - S: interactions involving exactly two cells, all pairs independent
 *     (Sec. II-A2).  Here Delta-Notch binding across the shared face; each
 *     molecule near a boundary belongs to a single face (Sec. III-A1 coupling
 *     rule), realised as two phases: x-faces, then y-faces.
 *   - The translations T_{chi->S}, T_{S->chi} (Sec. II-B) are the gather of a
 *     face's boundary voxels from both cells and the write-back of the result.
 *   - Each module call runs on its own local clock over [0, dt) (the per-cell
 *     "end_time" of the network file, Fig. 2) with its own seed (Fig. 3).
 *
 * Every arithmetic step is defined exactly (integer fixed-point propensities,
 * IEEE-754 binary64 time arithmetic with no contraction), so a faithful
 * implementation reproduces this oracle bit for bit.
 */
#ifndef TISSUE_ORACLE_H
#define TISSUE_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_E_ARG (-1)
#define ORC_E_OVERFLOW (-4)
#define ORC_E_STATE (-9)   /* a promoter-model state with more bound sites than sites */

/* Philox counter word 3 carries the tissue id in its low 24 bits and a tag
 * naming the stream in its high 8 bits. */
#define ORC_TAG_CHI 1u
#define ORC_TAG_SX 2u
#define ORC_TAG_SY 3u
#define ORC_TAG_INIT 4u
#define ORC_TAG_SX2 5u   /* second half-step of x-faces (Strang splitting) */
#define ORC_TAG_SY2 6u   /* second half-step of y-faces (Strang splitting) */
#define ORC_TAG_PLACE 7u /* placement of a well-mixed cell's D (7), N (8), R (9) */

/* Species index in the state layout counts[cell][species][voxel]. */
#define ORC_D 0
#define ORC_N 1
#define ORC_R 2

#define ORC_NCH 19          /* channels per voxel in chi */
#define ORC_COUNT_MAX ((1 << 30) - 1)
#define ORC_PROP_LIMIT (1ull << 52)   /* a voxel (chi) or a channel (S) must stay below */

typedef struct {
  uint32_t width, height;   /* cells; cell id c = cy*width + cx; no wrap-around */
  uint32_t n;               /* voxels per cell side; voxel id v = vy*n + vx */
  uint32_t tissue_id;       /* < 2^24 */
  uint64_t seed;            /* Philox key */
  double init_lambda[3];    /* Poisson mean of the initial count of D, N, R per voxel */
  const uint8_t* wm;        /* per cell: 0 lattice RDME, 1 well-mixed; NULL = all lattice */
} orc_desc;

/* The paper's own Notch model (Sec. III-A1, Table I) on the voxel lattice.
 * One DNA promoter site per cell, at the centre voxel (n/2, n/2).  Species
 * slots: D = Delta, N = NICD, R = bound promoter sites (0 or 1 at the centre
 * voxel, 0 elsewhere); the free sites of voxel v are F_v = [v is the centre]
 * - R_v.  Within a cell:
 *   free promoter transcribes Delta        F -> F + D      t_D * F
 *   NICD binds the free promoter           N + F -> R      k_a * N * F
 *   NICD unbinds                           R -> N + F      k_d * R
 *   Delta and NICD degrade (DNA does not)  D -> 0, N -> 0  d * D, d * N
 *   Delta and NICD hop to each existing neighbour voxel at `hop` each.
 * Across a face (the signalling module): each Delta in a face voxel turns
 * into NICD in the facing voxel of the other cell at k_N per molecule.
 * Rates are per unit time, already in lattice units (hop = diffusion
 * constant / h^2, k_a = bimolecular constant / voxel volume). */
typedef struct {
  double tD, ka, kd, kN, d, hop;
} orc_promoter;

#define ORC_MODEL_ND 0        /* Hill-repressed Delta-Notch lattice model (the rates below) */
#define ORC_MODEL_PROMOTER 1  /* the paper's promoter model (pm below) */

typedef struct {
  double kD, K, kN, gD, gN, gR, hopD, hopN, hopR, k_in, k_off, k_bind;
  int32_t kind;             /* ORC_MODEL_ND or ORC_MODEL_PROMOTER */
  int32_t reserved;
  orc_promoter pm;          /* used when kind == ORC_MODEL_PROMOTER */
} orc_model;

/* Well-mixed cells (the coarse single-cell module of the paper's mixed-
 * fidelity tissues, Sec. IV).  A well-mixed cell keeps its molecules in the
 * same voxel layout between module calls, but its chi ignores position:
 *   1. T_{S->chi}: the totals of D, N, R over the cell's voxels;
 *   2. the direct-method SSA on the totals over [0, dt), with the cell as one
 *      compartment of V voxel volumes:
 *        Notch-Delta   0 D production V kD / (1 + (R / (V K))^2)
 *                      1 N production V kN
 *                      2..4 decay gD D, gN N, gR R
 *                      5 D + N -> R at (k_in / V) D N
 *                      6 R -> D + N at k_off R
 *        promoter      0 transcription t_D F (F = 1 - R, one site per cell)
 *                      1 unbinding k_d R
 *                      2, 3 decay d D, d N
 *                      4 binding (k_a / V) N F
 *   3. T_{chi->S}: every molecule is placed in a voxel drawn uniformly at
 *      random (the well-mixed assumption), v = floor(w V / 2^32) with w the
 *      (i mod 4)-th word of Philox block (i / 4, step, cell, tissue_id |
 *      (7 + species) << 24) for the i-th molecule of the species; the
 *      promoter model's bound site stays on the promoter voxel.
 * The Hill term is evaluated in binary64 as written, left to right, each
 * operation rounded to nearest, then quantised; k_in / V and k_a / V are one
 * binary64 division each, then quantised.  On an error the cell's counts are
 * left unchanged. */

/* One fired event, for full-trace comparisons on small cases. */
typedef struct {
  uint32_t step;     /* global step index k */
  uint32_t kind;     /* ORC_TAG_CHI / ORC_TAG_SX / ORC_TAG_SY */
  uint32_t unit;     /* cell id (chi) or owner cell id of the face (S) */
  uint32_t e;        /* event index within this module call */
  double t;          /* local time of the event in [0, dt) */
  uint32_t site;     /* voxel (chi) or voxel pair p (S) */
  uint32_t channel;  /* channel slot 0..18 (chi) or 0/1 within the pair (S) */
} orc_event;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint64_t orc_neg_ln_q58(uint64_t k);
double orc_exp_variate(uint32_t w0, uint32_t w1);
int orc_quantize(double x, uint64_t* q);
int orc_hill_q(const orc_model* m, int64_t R, uint64_t* q);
int orc_validate(const orc_desc* d, const orc_model* m);

int orc_init_counts(const orc_desc* d, int32_t* counts);
int orc_init_cell(const orc_desc* d, int32_t* counts, uint32_t c);
int orc_chi_cell(const orc_desc* d, const orc_model* m, int32_t* counts, uint32_t c,
                 uint32_t step, double dt, uint64_t* n_events, double* t_last,
                 orc_event* trace, size_t trace_cap, size_t* trace_len);
int orc_sig_face(const orc_desc* d, const orc_model* m, int32_t* counts, uint32_t c,
                 int axis, uint32_t step, double dt, uint64_t* n_events, double* t_last,
                 orc_event* trace, size_t trace_cap, size_t* trace_len);
int orc_step(const orc_desc* d, const orc_model* m, int32_t* counts, uint32_t step0,
             uint32_t n_steps, double dt, uint64_t* n_events, double* t_last, int n_threads);
/* scheme 0: Lie (chi, S_x, S_y); 1: Strang (S_x/2, S_y/2, chi, S_y/2, S_x/2). */
int orc_step_scheme(const orc_desc* d, const orc_model* m, int32_t* counts, uint32_t step0,
                    uint32_t n_steps, double dt, int scheme, uint64_t* n_events, double* t_last,
                    int n_threads);
int orc_step_traced(const orc_desc* d, const orc_model* m, int32_t* counts, uint32_t step0,
                    uint32_t n_steps, double dt, orc_event* trace, size_t trace_cap,
                    size_t* trace_len);
/* As orc_step_traced, with the splitting scheme of orc_step_scheme. */
int orc_step_traced_scheme(const orc_desc* d, const orc_model* m, int32_t* counts,
                           uint32_t step0, uint32_t n_steps, double dt, int scheme,
                           orc_event* trace, size_t trace_cap, size_t* trace_len);

/* Test hooks: 0 = faithful.  A nonzero value plants one known mistake so the
 * pin tests can show that they catch it. */
void orc_set_mutation(int which);
/* 1 = recompute every voxel's propensity after each event (slow cross-check). */
void orc_set_paranoid(int on);
int orc_get_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
