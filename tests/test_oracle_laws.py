"""Pins of the oracle against closed-form laws of the stochastic kinetics.

Each test runs the oracle's full Lie splitting step (chi, then both S phases)
on a synthetic tissue whose model reduces to a process with a known law:
  - immigration-death-migration from a product-Poisson start stays product
    Poisson with mean m(t) = lam e^{-gt} + (b/g)(1 - e^{-gt}) (exact);
  - pure decay thins a Poisson start to Poisson(lam e^{-gt});
  - in-voxel D + N <-> R has the detailed-balance law
    pi(c+1)/pi(c) = k_in (a0-c)(b0-c) / (k_off (c+1));
  - a single lattice walker with reflecting walls has the exact per-axis law
    exp(Q t) of the tridiagonal generator, hence an exact mean-square
    displacement;
  - hops conserve per-cell totals; binding conserves D+R and N+R.
Rates enter through the integer propensities, i.e. as q(x)/2^32.
"""
import math

import numpy as np
import pytest
from scipy import linalg, stats

import oracle as O
from tests._util import discrete_gof, poisson_gof, q_exact, q_rate

ZERO = dict(kD=0.0, K=20.0, kN=0.0, gD=0.0, gN=0.0, gR=0.0, hopD=0.0, hopN=0.0, hopR=0.0,
            k_in=0.0, k_off=0.0, k_bind=0.0)


def _model(**kw):
    m = dict(ZERO)
    m.update(kw)
    return O.Model(**m)


def _species(d, counts, s):
    return counts.reshape(d.cells, 3, d.V)[:, s, :]


def test_poisson_initial_law():
    d = O.Desc(64, 32, 4, seed=31, init_lambda=(5.0, 0.5, 40.0))
    counts = O.init_counts(d)
    for s, lam in enumerate(d.init_lambda):
        p, z = poisson_gof(_species(d, counts, s), lam)
        assert p > 0.01 and abs(z) < 3, (s, p, z)


def test_poisson_initial_planted_mistake_is_caught():
    d = O.Desc(64, 32, 4, seed=31, init_lambda=(5.0, 5.0, 5.0))
    O.set_mutation(4)  # mean shifted by 0.5
    counts = O.init_counts(d)
    O.set_mutation(0)
    p, z = poisson_gof(_species(d, counts, 0), 5.0)
    assert p < 1e-6 or abs(z) > 5


def _immigration_death(lam, b, g, t):
    return lam * math.exp(-g * t) + (b / g) * (1.0 - math.exp(-g * t))


def test_immigration_death_transient_law():
    d = O.Desc(32, 32, 2, seed=41, init_lambda=(0.0, 7.0, 0.0))
    m = _model(kN=5.0, gN=0.1, hopN=1.0, k_bind=0.01)  # no Delta: binding never fires
    counts = O.init_counts(d)
    O.step(d, m, counts, 0, 30, 0.5)
    mean = _immigration_death(7.0, q_rate(5.0), q_rate(0.1), 15.0)
    p, z = poisson_gof(_species(d, counts, 1), mean)
    assert p > 0.01 and abs(z) < 3, (p, z, mean)


def _hill_setup(mutation=0):
    d = O.Desc(64, 64, 2, seed=44, init_lambda=(3.0, 0.0, 0.0))
    m = _model(kD=10.0, K=20.0, gD=0.5, hopD=1.0)
    counts = O.init_counts(d)
    counts.reshape(d.cells, 3, d.V)[:, 2, :] = 40  # repressor held at R = 40
    O.set_mutation(mutation)
    try:
        O.step(d, m, counts, 0, 20, 0.5)
    finally:
        O.set_mutation(0)
    b = O.hill_q(m, 40) / 2 ** 32
    assert b == 2.0  # 10 / (1 + (40/20)^2) is exact in binary64
    mean = _immigration_death(3.0, b, q_rate(0.5), 10.0)
    return poisson_gof(_species(d, counts, 0), mean)


def test_hill_production_law():
    p, z = _hill_setup()
    assert p > 0.01 and abs(z) < 3, (p, z)


def test_hill_planted_mistake_is_caught():
    p, z = _hill_setup(mutation=1)  # Hill exponent 1 instead of 2
    assert p < 1e-6 or abs(z) > 5


def _decay_setup(mutation=0):
    d = O.Desc(32, 32, 2, seed=47, init_lambda=(0.0, 0.0, 20.0))
    m = _model(gR=0.2, gD=0.1, hopR=1.0)
    counts = O.init_counts(d)
    O.set_mutation(mutation)
    try:
        O.step(d, m, counts, 0, 10, 0.5)
    finally:
        O.set_mutation(0)
    return poisson_gof(_species(d, counts, 2), 20.0 * math.exp(-q_rate(0.2) * 5.0))


def test_pure_decay_thinning_law():
    p, z = _decay_setup()
    assert p > 0.01 and abs(z) < 3, (p, z)


def test_decay_planted_mistake_is_caught():
    p, z = _decay_setup(mutation=3)  # R decays at the Delta rate
    assert p < 1e-6 or abs(z) > 5


def test_reversible_binding_equilibrium():
    a0, b0 = 6, 4
    d = O.Desc(32, 32, 2, seed=53, init_lambda=(0.0, 0.0, 0.0))
    m = _model(k_in=0.3, k_off=1.0)
    counts = np.zeros(d.cells * 3 * d.V, dtype=np.int32)
    v = counts.reshape(d.cells, 3, d.V)
    v[:, 0, :] = a0
    v[:, 1, :] = b0
    O.step(d, m, counts, 0, 20, 1.0)
    R = v[:, 2, :].ravel()
    assert np.all(v[:, 0, :].ravel() + R == a0) and np.all(v[:, 1, :].ravel() + R == b0)
    ratio = q_exact(0.3) / q_exact(1.0)
    w = np.array([ratio ** c / (math.factorial(c) * math.factorial(a0 - c) * math.factorial(b0 - c))
                  for c in range(b0 + 1)])
    pi = w / w.sum()
    obs = np.bincount(R, minlength=b0 + 1).astype(float)
    assert discrete_gof(obs, pi) > 0.01
    mean = (pi * np.arange(b0 + 1)).sum()
    sd = math.sqrt((pi * (np.arange(b0 + 1) - mean) ** 2).sum() / R.size)
    assert abs(R.mean() - mean) < 3 * sd


def _walk_law(n, x0, rate, t):
    Q = np.zeros((n, n))
    for x in range(n):
        for y in (x - 1, x + 1):
            if 0 <= y < n:
                Q[y, x] += rate
                Q[x, x] -= rate
    p0 = np.zeros(n)
    p0[x0] = 1.0
    return linalg.expm(Q * t) @ p0


def test_diffusion_mean_square_displacement():
    n, M, t = 32, 4000, 4.0
    x0, y0 = 5, 9
    d = O.Desc(1, 1, n, seed=59, init_lambda=(0.0, 0.0, 0.0))
    m = _model(hopD=1.0)
    counts = np.zeros(3 * n * n, dtype=np.int32)
    counts[y0 * n + x0] = M
    O.step(d, m, counts, 0, 8, 0.5)
    D = counts[: n * n].reshape(n, n)  # [vy][vx]
    assert D.sum() == M
    px = _walk_law(n, x0, q_rate(1.0), t)
    py = _walk_law(n, y0, q_rate(1.0), t)
    xs = np.arange(n)
    dx2, dy2 = (xs - x0) ** 2, (xs - y0) ** 2
    msd_exact = (px * dx2).sum() + (py * dy2).sum()
    var = (px * dx2 ** 2).sum() - (px * dx2).sum() ** 2 + (py * dy2 ** 2).sum() - (py * dy2).sum() ** 2
    msd = (D * (dy2[:, None] + dx2[None, :])).sum() / M
    assert abs(msd - msd_exact) < 3 * math.sqrt(var / M), (msd, msd_exact)
    assert discrete_gof(D.sum(axis=0).astype(float), px) > 0.01
    assert discrete_gof(D.sum(axis=1).astype(float), py) > 0.01
    # short-time limit of a 2-D lattice walk: MSD ~ 4 d t away from walls
    assert abs(msd_exact - 4 * t) < 0.35 * 4 * t


def test_hops_conserve_cell_totals():
    d = O.Desc(5, 3, 6, seed=61)
    m = _model(hopD=1.0, hopN=2.0, hopR=0.5)
    counts = O.init_counts(d)
    before = counts.reshape(d.cells, 3, d.V).sum(axis=2)
    for k in range(4):
        O.step(d, m, counts, k, 1, 0.3)
        assert np.array_equal(counts.reshape(d.cells, 3, d.V).sum(axis=2), before)


def test_binding_conserves_d_plus_r_and_n_plus_r():
    d = O.Desc(4, 3, 4, seed=67, init_lambda=(8.0, 8.0, 0.0))
    m = _model(hopD=1.0, hopN=1.0, hopR=1.0, k_bind=0.2)
    counts = O.init_counts(d)
    v = counts.reshape(d.cells, 3, d.V)
    dr, nr = v[:, 0].sum() + v[:, 2].sum(), v[:, 1].sum() + v[:, 2].sum()
    total_s = 0
    for k in range(5):
        ne, _ = O.step(d, m, counts, k, 1, 0.5)
        total_s += int(ne[1:].sum())
        assert v[:, 0].sum() + v[:, 2].sum() == dr
        assert v[:, 1].sum() + v[:, 2].sum() == nr
    assert total_s > 0 and v[:, 2].sum() == total_s


def test_incremental_propensities_equal_full_recompute():
    d = O.Desc(2, 2, 8, seed=1)
    m = O.Model()
    a = O.init_counts(d)
    b = a.copy()
    na, ta = O.step(d, m, a, 0, 5, 0.1)
    O.set_paranoid(True)
    nb, tb = O.step(d, m, b, 0, 5, 0.1)
    O.set_paranoid(False)
    assert np.array_equal(a, b) and np.array_equal(na, nb) and np.array_equal(ta, tb)


def test_thread_count_does_not_change_results():
    d = O.Desc(6, 5, 8, seed=71)
    m = O.Model(k_bind=0.05)
    a = O.init_counts(d)
    b = a.copy()
    na, ta = O.step(d, m, a, 0, 3, 0.1, n_threads=1)
    nb, tb = O.step(d, m, b, 0, 3, 0.1, n_threads=4)
    assert np.array_equal(a, b) and np.array_equal(na, nb) and np.array_equal(ta, tb)
