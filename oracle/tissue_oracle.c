/*
 * tissue_oracle.c -- plain, slow, obviously-correct CPU oracle of the
 * operator-split tissue SSA.  TEST INFRASTRUCTURE ONLY (see tissue_oracle.h).
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
 * (no FMA contraction: every binary64 operation is one IEEE round-to-nearest).
 *
 * Definitions restated here, in the order the method applies them:
 *   1. Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 *      key = seed, counter = (event, step, unit, tissue_id | tag << 24).
 *   2. Waiting time: E = -ln(u1) as a Q.58 fixed-point value, converted once
 *      to binary64; tau = E / (A * 2^-32); the event fires iff t + tau < dt.
 *   3. Propensities: integers in units of 2^-32 per unit time.  Each rate is
 *      quantised once, q(x) = round-half-even(x * 2^32); mass action then
 *      multiplies integers, so every sum is exact and order-free.
 *   4. Selection: r = floor(R64 * A / 2^64); the event is the first
 *      (voxel, channel) in canonical order whose running sum exceeds r.
 * Two single-cell models: the Notch-Delta lattice model of the tissue
 * workloads (Hill-repressed Delta production), and the paper's own Notch
 * model with one DNA promoter per cell (Sec. III-A1, Table I).
 */
#include "tissue_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

static int g_mutation = 0;
static int g_paranoid = 0;
void orc_set_mutation(int which) { g_mutation = which; }
void orc_set_paranoid(int on) { g_paranoid = on; }

int orc_get_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* 1. Philox4x32-10 (SC'11, "Parallel random numbers: as easy as 1, 2, 3").  */
/*    One round: two 32x32->64 products of counter words 0 and 2 with the    */
/*    round multipliers; the high halves are xored with the other counter    */
/*    words and the key.  The key is bumped by the Weyl constants between    */
/*    rounds.                                                                 */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = (g_mutation == 5) ? 0xD2511F55u : 0xD2511F53u;
  const uint32_t M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * x0;
    uint64_t p1 = (uint64_t)M1 * x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw(const orc_desc* d, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                 uint32_t out[4]) {
  uint32_t ctr[4] = {w0, w1, w2, w3};
  uint32_t key[2] = {(uint32_t)d->seed, (uint32_t)(d->seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* 2. -ln(u) in fixed point, u = k * 2^-53, k in [1, 2^53].                  */
/*    k = 2^j * m with m in [1, 2).  For m <= sqrt 2:  ln m = ln(1 + x);     */
/*    otherwise ln(m / 2) = ln(1 - w) and j grows by one.  Both use           */
/*    ln(1 +- 2h) = +-2 atanh(h / (1 +- h)) (Abramowitz & Stegun 4.1.27 with */
/*    h = x/2 or w/2), the atanh series summed to z^11 with z = s^2, and a   */
/*    Newton-Raphson reciprocal for 1 / (1 +- h).                              */
/* ------------------------------------------------------------------------ */
#define LN2_Q64 0xB17217F7D1CF79ACull    /* round(ln 2 * 2^64) */
#define SQRT2_Q63 0xB504F333F9DE6484ull  /* floor(sqrt 2 * 2^63) */

static uint64_t mulshr(uint64_t a, uint64_t b, int sh) {
  return (uint64_t)(((u128)a * b) >> sh);
}

static uint64_t atanh_coef_q63(int j) { /* round(2^63 / (2j + 1)) */
  uint64_t den = 2u * (uint64_t)j + 1u;
  return ((1ull << 63) + den / 2) / den;
}

uint64_t orc_neg_ln_q58(uint64_t k) {
  int j = 63 - __builtin_clzll(k);       /* k >= 1 */
  uint64_t m = k << (63 - j);            /* Q1.63, in [1, 2) */
  uint64_t h, d;
  uint64_t n;                            /* multiple of ln 2 */
  int case_b = m > SQRT2_Q63;
  if (!case_b) {
    h = m - (1ull << 63);                /* x/2 in Q0.64 */
    d = (1ull << 62) + (h >> 2);         /* 1 + x/2 in Q2.62 */
    n = (uint64_t)(53 - j);
  } else {
    h = (0 - m) >> 1;                    /* w/2 = (2 - m)/4 in Q0.64 */
    d = (1ull << 62) - (h >> 2);         /* 1 - w/2 in Q2.62 */
    n = (uint64_t)(52 - j);
  }
  uint64_t y = (1ull << 63) - d;         /* 2 - d: first guess of 1/d, Q2.62 */
  for (int it = 0; it < 4; ++it) {
    uint64_t dy = mulshr(d, y, 62);      /* d*y, Q2.62 */
    y = mulshr(y, (1ull << 63) - dy, 62);/* y*(2 - d*y) */
  }
  uint64_t s = mulshr(h, y, 62);         /* h/d, Q0.64 */
  uint64_t z = mulshr(s, s, 64);         /* s^2, Q0.64 */
  uint64_t p = atanh_coef_q63(11);       /* sum_j z^j/(2j+1), Q1.63 */
  for (int i = 10; i >= 0; --i) p = mulshr(p, z, 64) + atanh_coef_q63(i);
  uint64_t two_atanh = mulshr(s, p, 62); /* 2*s*p, Q0.64 */
  int sign_plus = case_b;
  if (g_mutation == 7) sign_plus = !sign_plus;
  u128 acc = (u128)n * LN2_Q64;
  if (sign_plus) acc += two_atanh; else acc -= two_atanh;
  return (uint64_t)(acc >> 6);           /* Q.58 */
}

/* Unit-mean exponential variate from Philox words 0 and 1. */
double orc_exp_variate(uint32_t w0, uint32_t w1) {
  uint64_t bits = (((uint64_t)w1 << 32) | w0) >> 11;
  uint64_t e_q58 = orc_neg_ln_q58(bits + 1);   /* u1 = (bits + 1) * 2^-53 in (0, 1] */
  return (double)e_q58 * 0x1p-58;
}

/* ------------------------------------------------------------------------ */
/* 3. Rates and propensities.                                                */
/* ------------------------------------------------------------------------ */
static int rate_ok(double x) { return isfinite(x) && x >= 0.0 && x < 1048576.0; }

int orc_quantize(double x, uint64_t* q) {
  if (!rate_ok(x)) return ORC_E_ARG;
  *q = (uint64_t)nearbyint(x * 4294967296.0);  /* exact scaling, then round half even */
  return ORC_OK;
}

typedef struct {
  int kind;
  uint64_t kN, gD, gN, gR, hopD, hopN, hopR, k_in, k_off, k_bind;
  double kD, K;
  uint64_t tD, ka, kd, kNc, d, hop;  /* promoter model (kNc: the face's k_N) */
  double k_in_raw, ka_raw;           /* for the well-mixed compartment rates */
} qmodel;

int orc_validate(const orc_desc* d, const orc_model* m) {
  if (d) {
    if (d->width < 1 || d->height < 1 || d->n < 2 || d->n > 32) return ORC_E_ARG;
    if (d->tissue_id >= (1u << 24)) return ORC_E_ARG;
    if ((uint64_t)d->width * d->height > 0xFFFFFFFFull) return ORC_E_ARG;
    for (int s = 0; s < 3; ++s)
      if (!(d->init_lambda[s] >= 0.0 && d->init_lambda[s] <= 700.0)) return ORC_E_ARG;
  }
  if (m) {
    if (m->kind == ORC_MODEL_ND) {
      const double r[12] = {m->kD, m->K, m->kN, m->gD, m->gN, m->gR,
                            m->hopD, m->hopN, m->hopR, m->k_in, m->k_off, m->k_bind};
      for (int i = 0; i < 12; ++i)
        if (!rate_ok(r[i])) return ORC_E_ARG;
      if (!(m->K > 0.0)) return ORC_E_ARG;
    } else if (m->kind == ORC_MODEL_PROMOTER) {
      const double r[6] = {m->pm.tD, m->pm.ka, m->pm.kd, m->pm.kN, m->pm.d, m->pm.hop};
      for (int i = 0; i < 6; ++i)
        if (!rate_ok(r[i])) return ORC_E_ARG;
    } else {
      return ORC_E_ARG;
    }
  }
  return ORC_OK;
}

static int make_qmodel(const orc_model* m, qmodel* q) {
  int rc = orc_validate(NULL, m);
  if (rc) return rc;
  memset(q, 0, sizeof(*q));
  q->kind = m->kind;
  if (m->kind == ORC_MODEL_PROMOTER) {
    orc_quantize(m->pm.tD, &q->tD);
    orc_quantize(m->pm.ka, &q->ka);
    orc_quantize(m->pm.kd, &q->kd);
    orc_quantize(m->pm.kN, &q->kNc);
    orc_quantize(m->pm.d, &q->d);
    orc_quantize(m->pm.hop, &q->hop);
    q->ka_raw = m->pm.ka;
    return ORC_OK;
  }
  orc_quantize(m->kN, &q->kN);
  orc_quantize(m->gD, &q->gD);
  orc_quantize(m->gN, &q->gN);
  orc_quantize(m->gR, &q->gR);
  orc_quantize(m->hopD, &q->hopD);
  orc_quantize(m->hopN, &q->hopN);
  orc_quantize(m->hopR, &q->hopR);
  orc_quantize(m->k_in, &q->k_in);
  orc_quantize(m->k_off, &q->k_off);
  orc_quantize(m->k_bind, &q->k_bind);
  if (g_mutation == 3) q->gR = q->gD;
  q->kD = m->kD;
  q->K = m->K;
  q->k_in_raw = m->k_in;
  return ORC_OK;
}

/* Hill-repressed Delta production kD / (1 + (R/K)^2), binary64, quantised. */
static uint64_t hill_q(const qmodel* q, int64_t R) {
  double x = (double)R / q->K;
  double den = (g_mutation == 1) ? 1.0 + x : 1.0 + x * x;
  double val = q->kD / den;
  return (uint64_t)nearbyint(val * 4294967296.0);
}

int orc_hill_q(const orc_model* m, int64_t R, uint64_t* out) {
  qmodel q;
  int rc = make_qmodel(m, &q);
  if (rc) return rc;
  *out = hill_q(&q, R);
  return ORC_OK;
}

/* Neighbour of voxel v in direction dir (0:-x 1:+x 2:-y 3:+y), or -1 at a
 * cell wall (walls reflect: there is no channel across them). */
static int neighbour(int n, int v, int dir) {
  int vx = v % n, vy = v / n;
  switch (dir) {
    case 0: return vx > 0 ? v - 1 : -1;
    case 1: return vx < n - 1 ? v + 1 : -1;
    case 2: return vy > 0 ? v - n : -1;
    default: return vy < n - 1 ? v + n : -1;
  }
}

/* The voxel of a cell that holds its promoter: (n/2, n/2). */
static int centre_voxel(int n) {
  if (g_mutation == 9) return (n / 2 - 1) * n + n / 2;
  return (n / 2) * n + n / 2;
}

/* The 19 channel slots of voxel v, in canonical order.
 * Notch-Delta model:
 *   0 Delta production (Hill)      1 Notch production
 *   2..4 decay of D, N, R
 *   5..8 hop of D toward -x,+x,-y,+y   9..12 hop of N   13..16 hop of R
 *   17 D + N -> R (in-voxel)       18 R -> D + N
 * Promoter model (R = bound sites, F = free sites):
 *   0 transcription F -> F + D     1 unbinding R -> N + F
 *   2, 3 decay of D, N             4 (none: DNA does not decay)
 *   5..8 hop of D   9..12 hop of N   13..16 (none: DNA does not move)
 *   17 binding N + F -> R          18 (none)
 * Values are exact (128-bit) so the overflow rule can be applied exactly. */
static void voxel_channels(const qmodel* q, const int32_t* cell, int n, int v, u128 c[ORC_NCH]) {
  const int V = n * n;
  const uint64_t D = (uint64_t)cell[ORC_D * V + v];
  const uint64_t N = (uint64_t)cell[ORC_N * V + v];
  const uint64_t R = (uint64_t)cell[ORC_R * V + v];
  if (q->kind == ORC_MODEL_PROMOTER) {
    const uint64_t F = (uint64_t)(v == centre_voxel(n)) - R;  /* R <= sites, checked */
    for (int j = 0; j < ORC_NCH; ++j) c[j] = 0;
    c[0] = (u128)q->tD * F;
    c[1] = (u128)q->kd * R;
    c[2] = (u128)q->d * D;
    c[3] = (u128)q->d * N;
    for (int dir = 0; dir < 4; ++dir) {
      int has = neighbour(n, v, dir) >= 0;
      c[5 + dir] = has ? (u128)q->hop * D : 0;
      c[9 + dir] = has ? (u128)q->hop * N : 0;
    }
    c[17] = (u128)q->ka * (N * F);
    return;
  }
  c[0] = hill_q(q, (int64_t)R);
  c[1] = q->kN;
  c[2] = (u128)q->gD * D;
  c[3] = (u128)q->gN * N;
  c[4] = (u128)q->gR * R;
  for (int dir = 0; dir < 4; ++dir) {
    int has = neighbour(n, v, dir) >= 0;
    c[5 + dir] = has ? (u128)q->hopD * D : 0;
    c[9 + dir] = has ? (u128)q->hopN * N : 0;
    c[13 + dir] = has ? (u128)q->hopR * R : 0;
  }
  c[17] = (u128)q->k_in * (D * N);
  c[18] = (u128)q->k_off * R;
}

/* Total propensity of voxel v; returns 0 and sets *ovf if it reaches 2^52. */
static uint64_t voxel_total(const qmodel* q, const int32_t* cell, int n, int v, int* ovf) {
  u128 c[ORC_NCH], s = 0;
  voxel_channels(q, cell, n, v, c);
  for (int j = 0; j < ORC_NCH; ++j) s += c[j];
  if (s >= (u128)ORC_PROP_LIMIT) {
    *ovf = 1;
    return 0;
  }
  return (uint64_t)s;
}

static int bump(int32_t* x, int delta) {
  int64_t y = (int64_t)*x + delta;
  if (y < 0 || y > ORC_COUNT_MAX) return ORC_E_OVERFLOW;
  *x = (int32_t)y;
  return ORC_OK;
}

static void record(orc_event* trace, size_t cap, size_t* len, uint32_t step, uint32_t kind,
                   uint32_t unit, uint32_t e, double t, uint32_t site, uint32_t ch) {
  if (!trace || !len) return;
  if (*len < cap) {
    orc_event* ev = &trace[*len];
    ev->step = step; ev->kind = kind; ev->unit = unit; ev->e = e;
    ev->t = t; ev->site = site; ev->channel = ch;
  }
  *len += 1;
}

/* ------------------------------------------------------------------------ */
/* Initial state: Poisson(lambda_s) per voxel and species, by inversion of    */
/* the CDF accumulated term by term, p_k = p_{k-1} * lambda / k.              */
/* ------------------------------------------------------------------------ */
static int32_t poisson_voxel(const orc_desc* d, double lam, double p0, uint32_t c, int s, int v) {
  uint32_t w[4];
  draw(d, (uint32_t)v, (uint32_t)s, c, d->tissue_id | (ORC_TAG_INIT << 24), w);
  double u = (double)((((uint64_t)w[1] << 32) | w[0]) >> 11) * 0x1p-53;
  int k = 0;
  double p = p0, F = p0;
  while (u >= F && k < 4096) {
    k += 1;
    p = (p * lam) / (double)k;
    F = F + p;
  }
  return k;
}

/* Initial counts of one cell c only (the other cells are left untouched). */
int orc_init_cell(const orc_desc* d, int32_t* counts, uint32_t c) {
  int rc = orc_validate(d, NULL);
  if (rc) return rc;
  if ((uint64_t)c >= (uint64_t)d->width * d->height) return ORC_E_ARG;
  const int V = (int)(d->n * d->n);
  for (int s = 0; s < 3; ++s) {
    const double lam = d->init_lambda[s] + (g_mutation == 4 ? 0.5 : 0.0);
    const double p0 = exp(-lam);
    for (int v = 0; v < V; ++v)
      counts[((int64_t)c * 3 + s) * V + v] = poisson_voxel(d, lam, p0, c, s, v);
  }
  return ORC_OK;
}

int orc_init_counts(const orc_desc* d, int32_t* counts) {
  int rc = orc_validate(d, NULL);
  if (rc) return rc;
  const int64_t cells = (int64_t)d->width * d->height;
  const int V = (int)(d->n * d->n);
  for (int s = 0; s < 3; ++s) {
    const double lam = d->init_lambda[s] + (g_mutation == 4 ? 0.5 : 0.0);
    const double p0 = exp(-lam);
    for (int64_t c = 0; c < cells; ++c) {
      for (int v = 0; v < V; ++v)
        counts[(c * 3 + s) * V + v] = poisson_voxel(d, lam, p0, (uint32_t)c, s, v);
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* chi: one cell over [0, dt) by the direct method (Gillespie 1977).          */
/* ------------------------------------------------------------------------ */
static int chi_cell_q(const orc_desc* d, const qmodel* q, int32_t* counts, uint32_t c,
                      uint32_t step, double dt, uint64_t* n_events, double* t_last,
                      orc_event* trace, size_t cap, size_t* len) {
  const int n = (int)d->n, V = n * n;
  int32_t* cell = counts + (size_t)c * 3 * V;
  uint64_t* a = (uint64_t*)malloc(sizeof(uint64_t) * V);
  if (!a) return ORC_E_ARG;
  int ovf = 0, bad_state = 0;
  if (q->kind == ORC_MODEL_PROMOTER) /* bound sites never exceed the voxel's sites */
    for (int v = 0; v < V; ++v)
      if (cell[ORC_R * V + v] > (v == centre_voxel(n))) bad_state = 1;
  for (int v = 0; v < V && !bad_state; ++v) a[v] = voxel_total(q, cell, n, v, &ovf);
  double t = 0.0;
  uint32_t e = 0;
  int rc = bad_state ? ORC_E_STATE : ovf ? ORC_E_OVERFLOW : ORC_OK;
  while (rc == ORC_OK) {
    uint64_t A = 0;
    for (int v = 0; v < V; ++v) A += a[v];
    if (A == 0) break;
    uint32_t w[4];
    draw(d, e, step, c, d->tissue_id | (ORC_TAG_CHI << 24), w);
    const double E = orc_exp_variate(w[0], w[1]);
    const double tau = E / ((double)A * 0x1p-32);
    const double tn = t + tau;
    if (!(tn < dt)) break;
    t = tn;
    /* select (voxel, channel) */
    const uint64_t R64 = ((uint64_t)w[3] << 32) | w[2];
    uint64_t r = (uint64_t)(((u128)R64 * A) >> 64);
    int v = 0;
    while (r >= a[v]) { r -= a[v]; ++v; }
    u128 ch[ORC_NCH];
    voxel_channels(q, cell, n, v, ch);
    int j = 0;
    while ((u128)r >= ch[j]) { r -= (uint64_t)ch[j]; ++j; }
    record(trace, cap, len, step, ORC_TAG_CHI, c, e, t, (uint32_t)v, (uint32_t)j);
    /* apply */
    int32_t* Dv = &cell[ORC_D * V + v];
    int32_t* Nv = &cell[ORC_N * V + v];
    int32_t* Rv = &cell[ORC_R * V + v];
    int u = -1;
    if (q->kind == ORC_MODEL_PROMOTER && (j == 1 || j == 17)) {
      if (j == 1) /* unbinding releases the NICD into the promoter's voxel */
        rc = (g_mutation == 8 ? 0 : bump(Nv, +1)) | bump(Rv, -1);
      else        /* binding takes one NICD and occupies the site */
        rc = bump(Nv, -1) | bump(Rv, +1);
    } else switch (j) {
      case 0: rc = bump(Dv, +1); break;
      case 1: rc = bump(Nv, +1); break;
      case 2: rc = bump(Dv, -1); break;
      case 3: rc = bump(Nv, -1); break;
      case 4: rc = bump(Rv, -1); break;
      case 17: rc = bump(Dv, -1) | bump(Nv, -1) | bump(Rv, +1); break;
      case 18: rc = bump(Rv, -1) | bump(Dv, +1) | bump(Nv, +1); break;
      default: {
        const int sp = (j - 5) / 4, dir = (j - 5) % 4;
        u = neighbour(n, v, dir);
        rc = bump(&cell[sp * V + v], -1) | bump(&cell[sp * V + u], +1);
      }
    }
    if (rc) { rc = ORC_E_OVERFLOW; break; }
    a[v] = voxel_total(q, cell, n, v, &ovf);
    if (u >= 0) a[u] = voxel_total(q, cell, n, u, &ovf);
    if (ovf) { rc = ORC_E_OVERFLOW; break; }
    if (g_paranoid) /* recompute every voxel: must not change anything */
      for (int x = 0; x < V; ++x) a[x] = voxel_total(q, cell, n, x, &ovf);
    e += 1;
    if (e == 0xFFFFFFFFu) { rc = ORC_E_OVERFLOW; break; }
  }
  free(a);
  if (n_events) *n_events = e;
  if (t_last) *t_last = t;
  return rc;
}

/* ------------------------------------------------------------------------ */
/* chi of a well-mixed cell (see the header): totals, direct-method SSA on    */
/* the totals, uniform placement.                                             */
/* ------------------------------------------------------------------------ */
#define WM_NCH 7

static int wm_channels(const qmodel* q, int V, const int64_t T[3], u128 a[WM_NCH]) {
  for (int j = 0; j < WM_NCH; ++j) a[j] = 0;
  const uint64_t D = (uint64_t)T[0], N = (uint64_t)T[1], R = (uint64_t)T[2];
  uint64_t k17;
  if (q->kind == ORC_MODEL_PROMOTER) {
    const uint64_t F = 1 - R;
    if (orc_quantize(q->ka_raw / (double)V, &k17)) return ORC_E_ARG;
    a[0] = (u128)q->tD * F;
    a[1] = (u128)q->kd * R;
    a[2] = (u128)q->d * D;
    a[3] = (u128)q->d * N;
    a[4] = (u128)k17 * (N * F);
    return ORC_OK;
  }
  const double Kc = (g_mutation == 12) ? q->K : (double)V * q->K;
  const double x = (double)R / Kc;
  const double val = ((double)V * q->kD) / (1.0 + x * x);
  if (orc_quantize(q->k_in_raw / (double)V, &k17)) return ORC_E_ARG;
  a[0] = (uint64_t)nearbyint(val * 4294967296.0);
  a[1] = (u128)q->kN * (uint64_t)V;
  a[2] = (u128)q->gD * D;
  a[3] = (u128)q->gN * N;
  a[4] = (u128)q->gR * R;
  a[5] = (u128)k17 * ((u128)D * N);
  a[6] = (u128)q->k_off * R;
  return ORC_OK;
}

/* The voxel of the i-th placed molecule of species s. */
static int wm_voxel(const orc_desc* d, uint32_t c, uint32_t step, int s, uint64_t i, int V) {
  uint32_t w[4];
  draw(d, (uint32_t)(i >> 2), step, c, d->tissue_id | ((ORC_TAG_PLACE + (uint32_t)s) << 24), w);
  const uint64_t v = ((uint64_t)w[i & 3] * (uint64_t)V) >> 32;
  if (g_mutation == 11 && v == (uint64_t)(V - 1)) return 0;
  return (int)v;
}

static int wm_cell_q(const orc_desc* d, const qmodel* q, int32_t* counts, uint32_t c,
                     uint32_t step, double dt, uint64_t* n_events, double* t_last,
                     orc_event* trace, size_t cap, size_t* len) {
  const int n = (int)d->n, V = n * n;
  int32_t* cell = counts + (size_t)c * 3 * V;
  const int pm = q->kind == ORC_MODEL_PROMOTER;
  int64_t T[3] = {0, 0, 0};
  int rc = ORC_OK;
  for (int sp = 0; sp < 3; ++sp)
    for (int v = 0; v < V; ++v) T[sp] += cell[sp * V + v];
  if (pm)
    for (int v = 0; v < V; ++v)
      if (cell[ORC_R * V + v] > (v == centre_voxel(n))) rc = ORC_E_STATE;
  for (int sp = 0; sp < 3; ++sp)
    if (T[sp] > ORC_COUNT_MAX) rc = rc ? rc : ORC_E_OVERFLOW;
  double t = 0.0;
  uint32_t e = 0;
  while (rc == ORC_OK) {
    u128 a[WM_NCH], A128 = 0;
    if ((rc = wm_channels(q, V, T, a))) break;
    for (int j = 0; j < WM_NCH; ++j) A128 += a[j];
    if (A128 >= (u128)ORC_PROP_LIMIT) { rc = ORC_E_OVERFLOW; break; }
    const uint64_t A = (uint64_t)A128;
    if (A == 0) break;
    uint32_t w[4];
    draw(d, e, step, c, d->tissue_id | (ORC_TAG_CHI << 24), w);
    const double E = orc_exp_variate(w[0], w[1]);
    const double tn = t + E / ((double)A * 0x1p-32);
    if (!(tn < dt)) break;
    t = tn;
    const uint64_t R64 = ((uint64_t)w[3] << 32) | w[2];
    uint64_t r = (uint64_t)(((u128)R64 * A) >> 64);
    int j = 0;
    while ((u128)r >= a[j]) { r -= (uint64_t)a[j]; ++j; }
    record(trace, cap, len, step, ORC_TAG_CHI, c, e, t, 0u, (uint32_t)j);
    static const int dnd[WM_NCH][3] = {{1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                                       {0, 0, -1}, {-1, -1, 1}, {1, 1, -1}};
    static const int dpm[WM_NCH][3] = {{1, 0, 0}, {0, 1, -1}, {-1, 0, 0}, {0, -1, 0},
                                       {0, -1, 1}, {0, 0, 0}, {0, 0, 0}};
    for (int sp = 0; sp < 3; ++sp) {
      T[sp] += pm ? dpm[j][sp] : dnd[j][sp];
      if (T[sp] < 0 || T[sp] > ORC_COUNT_MAX) rc = ORC_E_OVERFLOW;
    }
    e += 1;
    if (e == 0xFFFFFFFFu) rc = ORC_E_OVERFLOW;
  }
  if (rc == ORC_OK) { /* placement */
    memset(cell, 0, sizeof(int32_t) * 3 * V);
    for (int sp = 0; sp < 3; ++sp) {
      if (pm && sp == ORC_R) {
        cell[ORC_R * V + centre_voxel(n)] = (int32_t)T[ORC_R];
        continue;
      }
      for (int64_t i = 0; i < T[sp]; ++i) cell[sp * V + wm_voxel(d, c, step, sp, (uint64_t)i, V)] += 1;
    }
  }
  if (n_events) *n_events = e;
  if (t_last) *t_last = t;
  return rc;
}

static int chi_any_q(const orc_desc* d, const qmodel* q, int32_t* counts, uint32_t c,
                     uint32_t step, double dt, uint64_t* n_events, double* t_last,
                     orc_event* trace, size_t cap, size_t* len) {
  if (d->wm && d->wm[c])
    return wm_cell_q(d, q, counts, c, step, dt, n_events, t_last, trace, cap, len);
  return chi_cell_q(d, q, counts, c, step, dt, n_events, t_last, trace, cap, len);
}

int orc_chi_cell(const orc_desc* d, const orc_model* m, int32_t* counts, uint32_t c,
                 uint32_t step, double dt, uint64_t* n_events, double* t_last,
                 orc_event* trace, size_t trace_cap, size_t* trace_len) {
  qmodel q;
  int rc = orc_validate(d, m);
  if (rc) return rc;
  if (!(dt > 0.0) || !isfinite(dt)) return ORC_E_ARG;
  make_qmodel(m, &q);
  if (c >= d->width * d->height) return ORC_E_ARG;
  return chi_any_q(d, &q, counts, c, step, dt, n_events, t_last, trace, trace_cap, trace_len);
}

/* ------------------------------------------------------------------------ */
/* S: one face between cell c (owner, lower id) and its +x (axis 0) or +y     */
/* (axis 1) neighbour.  Pair p couples voxel a_p of c with voxel b_p of the   */
/* neighbour across the face.  Channel 2p: D(a)+N(b) -> R(b); channel 2p+1:   */
/* D(b)+N(a) -> R(a); both at k_bind * D * N.                                  */
/* ------------------------------------------------------------------------ */
static void face_voxels(int n, int axis, int p, int* va, int* vb) {
  if (axis == 0) {            /* right column of c, left column of c+1 */
    *va = p * n + (n - 1);
    *vb = p * n + 0;
    if (g_mutation == 6) *va = (n - 1) * n + p;
  } else {                    /* top row of c, bottom row of c+W */
    *va = (n - 1) * n + p;
    *vb = 0 * n + p;
  }
}

static int sig_face_q(const orc_desc* d, const qmodel* q, int32_t* counts, uint32_t c, int axis,
                      uint32_t tag, uint32_t step, double dt, uint64_t* n_events, double* t_last,
                      orc_event* trace, size_t cap, size_t* len) {
  const int n = (int)d->n, V = n * n;
  const uint32_t nb = axis == 0 ? c + 1 : c + d->width;
  int32_t* ca = counts + (size_t)c * 3 * V;
  int32_t* cb = counts + (size_t)nb * 3 * V;
  const int nch = 2 * n;
  uint64_t* a = (uint64_t*)malloc(sizeof(uint64_t) * nch);
  if (!a) return ORC_E_ARG;
  double t = 0.0;
  uint32_t e = 0;
  int rc = ORC_OK;
  for (;;) {
    /* channel propensities, recomputed from the counts at every event */
    uint64_t A = 0;
    for (int p = 0; p < n && rc == ORC_OK; ++p) {
      int va, vb;
      face_voxels(n, axis, p, &va, &vb);
      u128 x0, x1;
      if (q->kind == ORC_MODEL_PROMOTER) { /* Delta(a) -> NICD(b), Delta(b) -> NICD(a) */
        x0 = (u128)q->kNc * (uint64_t)ca[ORC_D * V + va];
        x1 = (u128)q->kNc * (uint64_t)cb[ORC_D * V + vb];
      } else {                             /* D(a) + N(b) -> R(b), D(b) + N(a) -> R(a) */
        x0 = (u128)q->k_bind * ((uint64_t)ca[ORC_D * V + va] * (uint64_t)cb[ORC_N * V + vb]);
        x1 = (u128)q->k_bind * ((uint64_t)cb[ORC_D * V + vb] * (uint64_t)ca[ORC_N * V + va]);
      }
      if (x0 >= (u128)ORC_PROP_LIMIT || x1 >= (u128)ORC_PROP_LIMIT) rc = ORC_E_OVERFLOW;
      a[2 * p] = (uint64_t)x0;
      a[2 * p + 1] = (uint64_t)x1;
      A += a[2 * p] + a[2 * p + 1];
    }
    if (rc || A == 0) break;
    uint32_t w[4];
    draw(d, e, step, c, d->tissue_id | (tag << 24), w);
    const double E = orc_exp_variate(w[0], w[1]);
    const double tau = E / ((double)A * 0x1p-32);
    const double tn = t + tau;
    if (!(tn < dt)) break;
    t = tn;
    const uint64_t R64 = ((uint64_t)w[3] << 32) | w[2];
    uint64_t r = (uint64_t)(((u128)R64 * A) >> 64);
    int j = 0;
    while (r >= a[j]) { r -= a[j]; ++j; }
    const int p = j / 2, dirn = j % 2;
    record(trace, cap, len, step, tag, c, e, t, (uint32_t)p, (uint32_t)dirn);
    int va, vb;
    face_voxels(n, axis, p, &va, &vb);
    int32_t* donor = dirn == 0 ? ca : cb;       /* cell giving Delta */
    int32_t* recv = dirn == 0 ? cb : ca;        /* cell giving Notch, receiving R */
    const int vd = dirn == 0 ? va : vb, vr = dirn == 0 ? vb : va;
    if (q->kind == ORC_MODEL_PROMOTER) {
      /* the Delta leaves the donor; NICD appears in the facing voxel */
      int32_t* ncell = (g_mutation == 10) ? donor : recv;
      const int vN = (g_mutation == 10) ? vd : vr;
      rc = bump(&donor[ORC_D * V + vd], -1) | bump(&ncell[ORC_N * V + vN], +1);
    } else {
      int32_t* rcell = (g_mutation == 2) ? donor : recv;
      const int vR = (g_mutation == 2) ? vd : vr;
      rc = bump(&donor[ORC_D * V + vd], -1) | bump(&recv[ORC_N * V + vr], -1) |
           bump(&rcell[ORC_R * V + vR], +1);
    }
    if (rc) { rc = ORC_E_OVERFLOW; break; }
    e += 1;
    if (e == 0xFFFFFFFFu) { rc = ORC_E_OVERFLOW; break; }
  }
  free(a);
  if (n_events) *n_events = e;
  if (t_last) *t_last = t;
  return rc;
}

int orc_sig_face(const orc_desc* d, const orc_model* m, int32_t* counts, uint32_t c, int axis,
                 uint32_t step, double dt, uint64_t* n_events, double* t_last,
                 orc_event* trace, size_t trace_cap, size_t* trace_len) {
  qmodel q;
  int rc = orc_validate(d, m);
  if (rc) return rc;
  if (!(dt > 0.0) || !isfinite(dt)) return ORC_E_ARG;
  make_qmodel(m, &q);
  const uint32_t cx = c % d->width, cy = c / d->width;
  if (c >= d->width * d->height) return ORC_E_ARG;
  if (axis == 0 && cx + 1 >= d->width) return ORC_E_ARG;
  if (axis == 1 && cy + 1 >= d->height) return ORC_E_ARG;
  return sig_face_q(d, &q, counts, c, axis, axis == 0 ? ORC_TAG_SX : ORC_TAG_SY, step, dt,
                    n_events, t_last, trace, trace_cap, trace_len);
}

/* ------------------------------------------------------------------------ */
/* One splitting step per k.
 *   Lie (scheme 0): chi over dt on every cell, then S over dt on every
 *     x-face, then on every y-face.
 *   Strang (scheme 1): S on x-faces over dt/2, S on y-faces over dt/2, chi
 *     over dt, S on y-faces over dt/2, S on x-faces over dt/2 (the symmetric
 *     composition; the second halves draw from their own tagged streams).
 * Within a phase the units touch disjoint voxels, so running them in
 * parallel (OpenMP) cannot change the result.  n_events / t_last (optional)
 * receive the LAST step's statistics laid out [3][cells]: row 0 chi per cell,
 * row 1 the x-face owned by the cell, row 2 its y-face (the last phase of
 * that axis in the step; 0 where the cell owns no such face). */
static int face_phase(const orc_desc* d, const qmodel* q, int32_t* counts, int axis, uint32_t tag,
                      uint32_t k, double dt, int last, uint64_t* n_events, double* t_last,
                      int n_threads, orc_event* trace, size_t cap, size_t* len) {
  const int64_t cells = (int64_t)d->width * d->height;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(| : err)
  for (int64_t c = 0; c < cells; ++c) {
    const uint32_t cx = (uint32_t)(c % d->width), cy = (uint32_t)(c / d->width);
    if (axis == 0 && cx + 1 >= d->width) continue;
    if (axis == 1 && cy + 1 >= d->height) continue;
    uint64_t ne; double tl;
    err |= -sig_face_q(d, q, counts, (uint32_t)c, axis, tag, k, dt, &ne, &tl, trace, cap, len);
    if (last && n_events) n_events[(1 + axis) * cells + c] = ne;
    if (last && t_last) t_last[(1 + axis) * cells + c] = tl;
  }
  return err;
}

static int chi_phase(const orc_desc* d, const qmodel* q, int32_t* counts, uint32_t k, double dt,
                     int last, uint64_t* n_events, double* t_last, int n_threads,
                     orc_event* trace, size_t cap, size_t* len) {
  const int64_t cells = (int64_t)d->width * d->height;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(| : err)
  for (int64_t c = 0; c < cells; ++c) {
    uint64_t ne; double tl;
    err |= -chi_any_q(d, q, counts, (uint32_t)c, k, dt, &ne, &tl, trace, cap, len);
    if (last && n_events) n_events[c] = ne;
    if (last && t_last) t_last[c] = tl;
  }
  return err;
}

static int step_impl(const orc_desc* d, const orc_model* m, int32_t* counts, uint32_t step0,
                     uint32_t n_steps, double dt, int scheme, uint64_t* n_events, double* t_last,
                     int n_threads, orc_event* trace, size_t cap, size_t* len) {
  qmodel q;
  int rc = orc_validate(d, m);
  if (rc) return rc;
  if (!(dt > 0.0) || !isfinite(dt) || (scheme != 0 && scheme != 1)) return ORC_E_ARG;
  make_qmodel(m, &q);
  const int64_t cells = (int64_t)d->width * d->height;
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#else
  (void)n_threads;
#endif
  if (trace) n_threads = 1; /* trace order: unit by unit */
  const double half = dt * 0.5;
  for (uint32_t s = 0; s < n_steps && rc == ORC_OK; ++s) {
    const uint32_t k = step0 + s;
    const int last = (s + 1 == n_steps);
    if (last && n_events) memset(n_events, 0, sizeof(uint64_t) * 3 * cells);
    if (last && t_last) memset(t_last, 0, sizeof(double) * 3 * cells);
    int err = 0;
    if (scheme == 0) {
      err |= chi_phase(d, &q, counts, k, dt, last, n_events, t_last, n_threads, trace, cap, len);
      if (!err) err |= face_phase(d, &q, counts, 0, ORC_TAG_SX, k, dt, last, n_events, t_last,
                                  n_threads, trace, cap, len);
      if (!err) err |= face_phase(d, &q, counts, 1, ORC_TAG_SY, k, dt, last, n_events, t_last,
                                  n_threads, trace, cap, len);
    } else {
      err |= face_phase(d, &q, counts, 0, ORC_TAG_SX, k, half, last, n_events, t_last,
                        n_threads, trace, cap, len);
      if (!err) err |= face_phase(d, &q, counts, 1, ORC_TAG_SY, k, half, last, n_events, t_last,
                                  n_threads, trace, cap, len);
      if (!err) err |= chi_phase(d, &q, counts, k, dt, last, n_events, t_last, n_threads, trace,
                                 cap, len);
      if (!err) err |= face_phase(d, &q, counts, 1, ORC_TAG_SY2, k, half, last, n_events, t_last,
                                  n_threads, trace, cap, len);
      if (!err) err |= face_phase(d, &q, counts, 0, ORC_TAG_SX2, k, half, last, n_events, t_last,
                                  n_threads, trace, cap, len);
    }
    if (err) rc = (err & -ORC_E_STATE) == -ORC_E_STATE ? ORC_E_STATE : ORC_E_OVERFLOW;
  }
  return rc;
}

int orc_step(const orc_desc* d, const orc_model* m, int32_t* counts, uint32_t step0,
             uint32_t n_steps, double dt, uint64_t* n_events, double* t_last, int n_threads) {
  return step_impl(d, m, counts, step0, n_steps, dt, 0, n_events, t_last, n_threads, NULL, 0,
                   NULL);
}

int orc_step_scheme(const orc_desc* d, const orc_model* m, int32_t* counts, uint32_t step0,
                    uint32_t n_steps, double dt, int scheme, uint64_t* n_events, double* t_last,
                    int n_threads) {
  return step_impl(d, m, counts, step0, n_steps, dt, scheme, n_events, t_last, n_threads, NULL,
                   0, NULL);
}

int orc_step_traced(const orc_desc* d, const orc_model* m, int32_t* counts, uint32_t step0,
                    uint32_t n_steps, double dt, orc_event* trace, size_t trace_cap,
                    size_t* trace_len) {
  return orc_step_traced_scheme(d, m, counts, step0, n_steps, dt, 0, trace, trace_cap,
                                trace_len);
}

int orc_step_traced_scheme(const orc_desc* d, const orc_model* m, int32_t* counts,
                           uint32_t step0, uint32_t n_steps, double dt, int scheme,
                           orc_event* trace, size_t trace_cap, size_t* trace_len) {
  *trace_len = 0;
  return step_impl(d, m, counts, step0, n_steps, dt, scheme, NULL, NULL, 1, trace, trace_cap,
                   trace_len);
}
