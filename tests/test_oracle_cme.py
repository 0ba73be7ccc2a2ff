"""Pin of the whole oracle step against the exact law of the Lie-split
process (operator splitting, Sec. II), computed by brute force on tiny state
spaces: two cells of 2x2 voxels holding a few molecules, with decay, hops and
face binding in both directions.  A mistake in the time sampling, the
selection, a channel's effect, the face geometry or the splitting order moves
the law and fails the chi-square test."""
import numpy as np
import pytest
from scipy import linalg

import oracle as O
from tests._util import discrete_gof, q_rate
from tests.cme import split_law

RATES = dict(kD=0.0, K=20.0, kN=0.0, gD=0.3, gN=0.2, gR=0.5, hopD=0.7, hopN=1.1,
             hopR=0.4, k_in=0.0, k_off=0.0, k_bind=1.5)


def _qrates():
    return {k: q_rate(v) for k, v in RATES.items()}


def _initial(W, H, n, axis):
    V = n * n
    x = np.zeros(W * H * 3 * V, dtype=np.int32)
    if axis == 0:   # cells 0 | 1 side by side
        x[(0 * 3 + 0) * V + 1] = 1  # D in cell 0 at (vx=1, vy=0): on the face
        x[(1 * 3 + 1) * V + 2] = 1  # N in cell 1 at (vx=0, vy=1)
        x[(1 * 3 + 0) * V + 0] = 1  # D in cell 1 at (0, 0): on the face
        x[(0 * 3 + 1) * V + 0] = 1  # N in cell 0 at (0, 0): off the face
    else:           # cell 0 below cell 1
        x[(0 * 3 + 0) * V + 2] = 1  # D in cell 0 at (0, 1): on the face
        x[(1 * 3 + 1) * V + 1] = 1  # N in cell 1 at (1, 0): on the face
        x[(1 * 3 + 0) * V + 3] = 1  # D in cell 1 at (1, 1): off the face
        x[(0 * 3 + 1) * V + 3] = 1  # N in cell 0 at (1, 1): on the face
    return x


def _ensemble(W, H, n, axis, replicas, dt, k_steps, seed, scheme=O.LIE):
    x0 = _initial(W, H, n, axis)
    m = O.Model(**RATES)
    finals = []
    for r in range(replicas):
        d = O.Desc(W, H, n, seed=seed, tissue_id=r, init_lambda=(0.0, 0.0, 0.0))
        x = x0.copy()
        O.step(d, m, x, 0, k_steps, dt, n_threads=1, scheme=scheme)
        finals.append(tuple(int(v) for v in x))
    return x0, finals


def _law_pvalue(W, H, n, axis, replicas=12000, dt=0.5, k_steps=3, seed=77, scheme=O.LIE):
    x0, finals = _ensemble(W, H, n, axis, replicas, dt, k_steps, seed, scheme)
    states, idx, p, _ = split_law(W, H, n, _qrates(), x0, dt, k_steps,
                                  "lie" if scheme == O.LIE else "strang")
    obs = np.zeros(len(states))
    for f in finals:
        assert f in idx, "oracle reached a state the CME says is unreachable"
        obs[idx[f]] += 1
    return discrete_gof(obs, p), len(states)


@pytest.mark.parametrize("W,H,axis", [(2, 1, 0), (1, 2, 1)])
def test_split_process_matches_exact_law(W, H, axis):
    p, S = _law_pvalue(W, H, 2, axis)
    assert S > 100
    assert p > 0.01, p


@pytest.mark.parametrize("W,H,axis", [(2, 1, 0), (1, 2, 1)])
def test_strang_split_process_matches_exact_law(W, H, axis):
    p, S = _law_pvalue(W, H, 2, axis, seed=79, scheme=O.STRANG)
    assert p > 0.01, p


def test_strang_differs_from_lie_in_law():
    """The two schemes are different processes at finite dt: the Lie
    ensemble fails the Strang law."""
    x0, finals = _ensemble(2, 1, 2, 0, 12000, 1.0, 2, 81, O.LIE)
    states, idx, p, _ = split_law(2, 1, 2, _qrates(), x0, 1.0, 2, "strang")
    obs = np.zeros(len(states))
    for f in finals:
        obs[idx[f]] += 1
    assert discrete_gof(obs, p) < 1e-3


@pytest.mark.parametrize("mutation", [2, 6])
def test_face_planted_mistakes_are_caught(mutation):
    # 2: the repressor appears in the Delta donor; 6: x-face uses the top row
    O.set_mutation(mutation)
    try:
        x0, finals = _ensemble(2, 1, 2, 0, 3000, 0.5, 3, 78)
    finally:
        O.set_mutation(0)
    states, idx, p, _ = split_law(2, 1, 2, _qrates(), x0, 0.5, 3)
    obs = np.zeros(len(states))
    unreachable = 0
    for f in finals:
        if f in idx:
            obs[idx[f]] += 1
        else:
            unreachable += 1
    assert unreachable > 0 or discrete_gof(obs, p) < 1e-4


def test_strang_splitting_converges_at_second_order():
    """Strang's symmetric composition is second order: halving dt quarters
    the distance of the split law from the unsplit law."""
    x0 = _initial(2, 1, 2, 0)
    T = 1.0
    errs = {"lie": [], "strang": []}
    for scheme in errs:
        for k in (2, 4, 8, 16):
            states, idx, p, Q = split_law(2, 1, 2, _qrates(), x0, T / k, k, scheme)
            p0 = np.zeros(len(states))
            p0[0] = 1.0
            exact = linalg.expm((Q["chi"] + Q["sx"] + Q["sy"]) * T) @ p0
            errs[scheme].append(np.abs(p - exact).sum())
    r = errs["strang"]
    ratios = [r[i] / r[i + 1] for i in range(len(r) - 1)]
    assert ratios == sorted(ratios) and 3.6 < ratios[-1] < 4.4, (r, ratios)  # -> 4
    assert r[-1] < errs["lie"][-1] / 4


def test_lie_splitting_converges_as_dt_shrinks():
    """The split law approaches the unsplit law exp((Q_chi+Q_S) T) p0 at first
    order in dt (the convergence the framework relies on, Sec. II)."""
    x0 = _initial(2, 1, 2, 0)
    T = 1.0
    errs = []
    for k in (1, 2, 4, 8):
        states, idx, p, Q = split_law(2, 1, 2, _qrates(), x0, T / k, k)
        p0 = np.zeros(len(states))
        p0[0] = 1.0
        exact = linalg.expm((Q["chi"] + Q["sx"] + Q["sy"]) * T) @ p0
        errs.append(np.abs(p - exact).sum())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(1.7 < r < 2.7 for r in ratios), (errs, ratios)  # first order: -> 2
