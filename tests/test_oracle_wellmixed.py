"""Pins of the oracle's well-mixed cells (the coarse single-cell module of a
mixed-fidelity tissue, Sec. IV) against laws fixed by the mathematics:

  - transcription from a promoter that never binds, in a well-mixed cell, is
    an immigration-death process (Poisson law of the Delta total), and every
    molecule lands in a uniformly random voxel;
  - a well-mixed promoter facing m fixed NICD is the two-state chain with the
    compartment binding rate k_a / V;
  - Notch-Delta production in a well-mixed cell at a fixed repressor total R
    runs at V kD / (1 + (R / (V K))^2);
  - the exact law (brute-force CME) of a tissue with one well-mixed and one
    lattice cell coupled by face conversion.
Each pin also shows that it catches a planted mistake."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from tests._util import discrete_gof, poisson_gof, q_rate
from tests.cme import wm_split_law


def _cells(d, counts):
    return counts.reshape(d.cells, 3, d.V)


def _run(d, m, counts, n_steps, dt, mutation=0):
    O.set_mutation(mutation)
    try:
        O.step(d, m, counts, 0, n_steps, dt)
    finally:
        O.set_mutation(0)


def _all_wm(w, h, n, seed, lam=(0.0, 0.0, 0.0)):
    return O.Desc(w, h, n, seed=seed, init_lambda=lam, wm=np.ones(w * h, dtype=np.uint8))


def _transcription(mutation=0):
    d = _all_wm(64, 64, 4, 301)
    m = O.Promoter(tD=10.0, ka=0.0, kd=0.0, kN=0.0, d=1.0, hop=2.0)
    counts = O.init_counts(d)
    _run(d, m, counts, 4, 0.5, mutation)
    x = _cells(d, counts)
    mean = q_rate(10.0) / q_rate(1.0) * (1.0 - math.exp(-q_rate(1.0) * 2.0))
    p_tot, z = poisson_gof(x[:, 0].sum(axis=1), mean)
    per_voxel = x[:, 0].sum(axis=0).astype(float)  # pooled over cells: uniform over voxels
    p_uni = stats.chisquare(per_voxel).pvalue
    return p_tot, z, p_uni


def test_wm_transcription_and_uniform_placement():
    p_tot, z, p_uni = _transcription()
    assert p_tot > 0.01 and abs(z) < 3, (p_tot, z)
    assert p_uni > 0.01, p_uni


def test_wm_placement_mistake_is_caught():
    _, _, p_uni = _transcription(mutation=11)  # the last voxel never receives a molecule
    assert p_uni < 1e-6


def test_wm_two_state_law():
    n, m_nicd, ka, kd, T = 4, 3, 6.4, 1.5, 1.0
    d = _all_wm(64, 64, n, 303)
    model = O.Promoter(tD=0.0, ka=ka, kd=kd, kN=0.0, d=0.0, hop=0.0)
    counts = O.init_counts(d)
    _cells(d, counts)[:, 1, 5] = m_nicd  # anywhere: the cell is well mixed
    _run(d, model, counts, 4, T / 4)
    x = _cells(d, counts)
    centre = (n // 2) * n + n // 2
    bound = x[:, 2, centre]
    assert x[:, 2].sum() == bound.sum()  # the bound site stays on the promoter voxel
    assert np.all(x[:, 1].sum(axis=1) + bound == m_nicd)
    a, b = q_rate(ka / (n * n)) * m_nicd, q_rate(kd)
    p_bound = a / (a + b) * (1.0 - math.exp(-(a + b) * T))
    z = (bound.mean() - p_bound) / math.sqrt(p_bound * (1 - p_bound) / d.cells)
    assert abs(z) < 3, z


def _hill(mutation=0):
    n, R_each = 2, 40  # R total 160 = V * 40: x = 160 / (4 * 20) = 2
    d = _all_wm(64, 64, n, 305)
    m = O.Model(kD=10.0, K=20.0, kN=0.0, gD=0.5, gN=0.0, gR=0.0, hopD=1.0, hopN=0.0, hopR=0.0,
                k_in=0.0, k_off=0.0, k_bind=0.0)
    counts = O.init_counts(d)
    _cells(d, counts)[:, 2, :] = R_each
    _run(d, m, counts, 20, 0.5, mutation)
    x = _cells(d, counts)
    assert np.all(x[:, 2].sum(axis=1) == n * n * R_each)
    b = n * n * 10.0 / (1.0 + 2.0 ** 2)  # = 8, exact in binary64
    g = q_rate(0.5)
    return poisson_gof(x[:, 0].sum(axis=1), b / g * (1.0 - math.exp(-g * 10.0)))


def test_wm_hill_production_law():
    p, z = _hill()
    assert p > 0.01 and abs(z) < 3, (p, z)


def test_wm_hill_mistake_is_caught():
    p, z = _hill(mutation=12)  # R / K instead of R / (V K)
    assert p < 1e-6 or abs(z) > 5


RATES = dict(tD=0.0, ka=1.3, kd=0.9, kN=0.8, d=0.3, hop=0.7)


def _mixed_pvalue(wm, mutation=0, replicas=12000, dt=0.5, k_steps=2, seed=311):
    n, V = 2, 4
    x0 = np.zeros(2 * 3 * V, dtype=np.int32)
    x0[(0 * 3 + 0) * V + 1] = 1  # Delta in cell 0 at (1, 0): on the x-face
    x0[(0 * 3 + 0) * V + 0] = 1  # Delta in cell 0 at (0, 0)
    x0[(1 * 3 + 0) * V + 2] = 1  # Delta in cell 1 at (0, 1): on the x-face
    x0[(1 * 3 + 1) * V + 0] = 1  # NICD in cell 1
    model = O.Promoter(**RATES)
    finals = []
    O.set_mutation(mutation)
    try:
        for r in range(replicas):
            d = O.Desc(2, 1, n, seed=seed, tissue_id=r, init_lambda=(0.0, 0.0, 0.0),
                       wm=np.array(wm, dtype=np.uint8))
            x = x0.copy()
            O.step(d, model, x, 0, k_steps, dt, n_threads=1)
            finals.append(tuple(int(v) for v in x))
    finally:
        O.set_mutation(0)
    rates = {k: q_rate(v) for k, v in RATES.items()}
    rates["ka_cell"] = q_rate(RATES["ka"] / V)
    states, idx, p = wm_split_law(2, 1, n, rates, x0, dt, k_steps, wm)
    assert abs(p.sum() - 1.0) < 1e-9
    obs = np.zeros(len(states))
    unreachable = 0
    for f in finals:
        if f in idx:
            obs[idx[f]] += 1
        else:
            unreachable += 1
    return (discrete_gof(obs, p) if not unreachable else 0.0), len(states), unreachable


@pytest.mark.parametrize("wm", [(1, 0), (0, 1), (1, 1)])
def test_mixed_fidelity_tissue_matches_exact_law(wm):
    p, S, unreachable = _mixed_pvalue(list(wm))
    assert unreachable == 0 and S > 20, (S, unreachable)
    assert p > 0.01, p


def test_mixed_fidelity_exact_law_reduces_to_lattice():
    """With no well-mixed cell the helper's law is the lattice split law."""
    from tests.cme import split_law
    n, V = 2, 4
    x0 = np.zeros(2 * 3 * V, dtype=np.int32)
    x0[1] = 1
    x0[(1 * 3 + 1) * V + 3] = 1
    rates = {k: q_rate(v) for k, v in RATES.items()}
    rates["ka_cell"] = q_rate(RATES["ka"] / V)
    s1, i1, p1 = wm_split_law(2, 1, n, rates, x0, 0.5, 2, [0, 0])
    s2, i2, p2, _ = split_law(2, 1, n, rates, x0, 0.5, 2, model="promoter")
    q2 = np.array([p2[i2[s]] if s in i2 else 0.0 for s in s1])
    assert np.allclose(p1, q2, atol=1e-12)


@pytest.mark.parametrize("mutation", [11])
def test_mixed_fidelity_planted_mistake_fails_exact_law(mutation):
    p, _, unreachable = _mixed_pvalue([1, 0], mutation=mutation, replicas=4000)
    assert unreachable > 0 or p < 1e-4
