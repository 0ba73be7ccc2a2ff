"""Pins of the oracle's promoter model (the paper's Notch model: one DNA
promoter per cell transcribing Delta while free, NICD binding and unbinding
it, Delta turning into NICD across a face; Sec. III-A1, Table I) against
laws fixed by the mathematics:

  - transcription from a promoter that never binds is an immigration-death
    process: the cell's Delta total is exactly Poisson(t_D/d (1 - e^{-d t}));
  - a promoter facing m NICD molecules that neither move nor decay is a
    two-state chain: P(bound at t) = a/(a+b) (1 - e^{-(a+b) t}), a = k_a m,
    b = k_d, and NICD + bound sites stays m;
  - each Delta on a face turns into NICD across it independently, so the
    converted count is Binomial(D0, 1 - e^{-k_N dt});
  - the exact law of the split process on tiny spaces (brute-force CME).
Each pin also shows that it catches a planted mistake."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from tests._util import discrete_gof, poisson_gof, q_rate
from tests.cme import split_law


def _cells(d, counts):
    return counts.reshape(d.cells, 3, d.V)


def _run(d, m, counts, n_steps, dt, mutation=0, scheme=O.LIE):
    O.set_mutation(mutation)
    try:
        O.step(d, m, counts, 0, n_steps, dt, scheme=scheme)
    finally:
        O.set_mutation(0)


def _transcription(mutation=0):
    d = O.Desc(64, 64, 4, seed=201, init_lambda=(0.0, 0.0, 0.0))
    m = O.Promoter(tD=10.0, ka=0.0, kd=0.0, kN=0.0, d=1.0, hop=2.0)
    counts = O.init_counts(d)
    _run(d, m, counts, 4, 0.5, mutation)
    x = _cells(d, counts)
    assert x[:, 1:].sum() == 0  # no NICD, no binding
    mean = q_rate(10.0) / q_rate(1.0) * (1.0 - math.exp(-q_rate(1.0) * 2.0))
    return poisson_gof(x[:, 0].sum(axis=1), mean)


def test_promoter_transcription_law():
    p, z = _transcription()
    assert p > 0.01 and abs(z) < 3, (p, z)


def _two_state(mutation=0, m_nicd=3, ka=0.4, kd=1.5, T=1.0):
    d = O.Desc(64, 64, 4, seed=203, init_lambda=(0.0, 0.0, 0.0))
    m = O.Promoter(tD=0.0, ka=ka, kd=kd, kN=0.0, d=0.0, hop=0.0)
    counts = O.init_counts(d)
    centre = (d.n // 2) * d.n + d.n // 2
    _cells(d, counts)[:, 1, centre] = m_nicd
    _run(d, m, counts, 4, T / 4, mutation)
    x = _cells(d, counts)
    bound = x[:, 2, centre]
    a, b = q_rate(ka) * m_nicd, q_rate(kd)
    p_bound = a / (a + b) * (1.0 - math.exp(-(a + b) * T))
    z = (bound.mean() - p_bound) / math.sqrt(p_bound * (1 - p_bound) / d.cells)
    conserved = bool(np.all(x[:, 1].sum(axis=1) + x[:, 2].sum(axis=1) == m_nicd))
    return z, conserved, x


def test_promoter_two_state_law():
    z, conserved, x = _two_state()
    assert conserved
    assert abs(z) < 3, z
    # the site is the only place a bound state can be, and never above one
    centre = 2 * 4 + 2
    assert x[:, 2].max() == 1 and x[:, 2].sum() == x[:, 2, centre].sum()


def test_promoter_unbinding_mistake_is_caught():
    z, conserved, _ = _two_state(mutation=8)  # unbinding loses the NICD
    assert not conserved


def test_promoter_centre_mistake_is_caught():
    z, conserved, _ = _two_state(mutation=9)  # the site one row lower
    assert abs(z) > 5


def _face(mutation=0, D0=30, kN=1.0, dt=0.5):
    n = 4
    d = O.Desc(2, 512, n, seed=205, init_lambda=(0.0, 0.0, 0.0))
    m = O.Promoter(tD=0.0, ka=0.0, kd=0.0, kN=kN, d=0.0, hop=0.0)
    counts = O.init_counts(d)
    x = _cells(d, counts)
    left, right = np.arange(0, d.cells, 2), np.arange(1, d.cells, 2)
    x[left, 0, 1 * n + 3] = D0    # cell 0, (vx=3, vy=1): on the x-face
    x[right, 0, 2 * n + 0] = D0   # cell 1, (vx=0, vy=2): on the x-face
    x[left, 0, 1 * n + 1] = D0    # cell 0, (1, 1): inside, never converts
    _run(d, m, counts, 1, dt, mutation)
    x = _cells(d, counts)
    return n, D0, x, left, right, 1.0 - math.exp(-q_rate(kN) * dt)


def test_promoter_face_conversion_binomial():
    n, D0, x, left, right, p = _face()
    conv_lr = D0 - x[left, 0, 1 * n + 3]
    conv_rl = D0 - x[right, 0, 2 * n + 0]
    # the NICD appears exactly in the facing voxel of the other cell
    assert np.array_equal(x[right, 1, 1 * n + 0], conv_lr)
    assert np.array_equal(x[left, 1, 2 * n + 3], conv_rl)
    assert x[:, 1].sum() == conv_lr.sum() + conv_rl.sum()
    assert np.all(x[left, 0, 1 * n + 1] == D0)
    ks = np.arange(D0 + 1)
    pmf = stats.binom.pmf(ks, D0, p)
    for conv in (conv_lr, conv_rl):
        assert discrete_gof(np.bincount(conv, minlength=D0 + 1).astype(float), pmf) > 0.01


def test_promoter_face_mistake_is_caught():
    n, D0, x, left, right, p = _face(mutation=10)  # NICD left in the donor cell
    assert x[right, 1, 1 * n + 0].sum() == 0


def test_promoter_invalid_state_is_rejected():
    d = O.Desc(2, 2, 4, seed=1, init_lambda=(0.0, 0.0, 0.0))
    counts = O.init_counts(d)
    _cells(d, counts)[1, 2, 0] = 1  # a bound site away from the promoter voxel
    with pytest.raises(O.OracleError) as e:
        O.step(d, O.Promoter(), counts, 0, 1, 0.1)
    assert e.value.code == O.E_STATE


# ---- exact law of the split process (brute-force CME) ---------------------

PM_RATES = dict(tD=0.0, ka=1.3, kd=0.9, kN=0.8, d=0.3, hop=0.7)


def _qr(r):
    return {k: q_rate(v) for k, v in r.items()}


def _pm_ensemble(W, H, n, x0, rates, replicas, dt, k_steps, seed, scheme=O.LIE, mutation=0):
    m = O.Promoter(**rates)
    finals = []
    O.set_mutation(mutation)
    try:
        for r in range(replicas):
            d = O.Desc(W, H, n, seed=seed, tissue_id=r, init_lambda=(0.0, 0.0, 0.0))
            x = x0.copy()
            O.step(d, m, x, 0, k_steps, dt, n_threads=1, scheme=scheme)
            finals.append(tuple(int(v) for v in x))
    finally:
        O.set_mutation(0)
    return finals


def _pm_initial_two_cells():
    n, V = 2, 4
    x = np.zeros(2 * 3 * V, dtype=np.int32)
    x[(0 * 3 + 0) * V + 1] = 1  # Delta in cell 0 at (1, 0): on the x-face
    x[(1 * 3 + 0) * V + 2] = 1  # Delta in cell 1 at (0, 1): on the x-face
    x[(0 * 3 + 1) * V + 3] = 1  # NICD in cell 0 at its promoter voxel (1, 1)
    return n, x


def _pm_pvalue(scheme=O.LIE, mutation=0, replicas=12000, dt=0.5, k_steps=3, seed=211):
    n, x0 = _pm_initial_two_cells()
    finals = _pm_ensemble(2, 1, n, x0, PM_RATES, replicas, dt, k_steps, seed, scheme, mutation)
    states, idx, p, _ = split_law(2, 1, n, _qr(PM_RATES), x0, dt, k_steps,
                                  "lie" if scheme == O.LIE else "strang", model="promoter")
    obs = np.zeros(len(states))
    unreachable = 0
    for f in finals:
        if f in idx:
            obs[idx[f]] += 1
        else:
            unreachable += 1
    return (discrete_gof(obs, p) if not unreachable else 0.0), len(states), unreachable


@pytest.mark.parametrize("scheme", [O.LIE, O.STRANG])
def test_promoter_split_process_matches_exact_law(scheme):
    p, S, unreachable = _pm_pvalue(scheme)
    assert unreachable == 0 and S > 50
    assert p > 0.01, p


@pytest.mark.parametrize("mutation", [8, 9, 10])
def test_promoter_planted_mistakes_fail_exact_law(mutation):
    p, _, unreachable = _pm_pvalue(mutation=mutation, replicas=3000)
    assert unreachable > 0 or p < 1e-4


def test_promoter_transcription_matches_exact_law():
    """One cell of 2x2 voxels with transcription on: the space is truncated
    at 7 Delta molecules, which the law crosses with probability < 1e-4."""
    rates = dict(tD=1.0, ka=1.1, kd=0.8, kN=0.0, d=0.7, hop=0.9)
    n, V = 2, 4
    x0 = np.zeros(3 * V, dtype=np.int32)
    x0[1 * V + 0] = 1  # one NICD at (0, 0)
    dt, k_steps = 0.5, 3
    finals = _pm_ensemble(1, 1, n, x0, rates, 12000, dt, k_steps, 213)
    states, idx, p, _ = split_law(1, 1, n, _qr(rates), x0, dt, k_steps, model="promoter",
                                  max_delta=7)
    lost = 1.0 - p.sum()
    assert 0.0 <= lost < 1e-4
    obs = np.zeros(len(states))
    outside = 0
    for f in finals:
        if f in idx:
            obs[idx[f]] += 1
        else:
            outside += 1
    assert outside <= 3
    assert discrete_gof(obs, p / p.sum()) > 0.01
