"""Shared test helpers: conversions from workload specs and small statistics."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
from scipy import stats

import oracle as O
from paper_1806_10889_gb300.workloads import TissueSpec

SCALE = 2 ** 32


def orc_desc(spec: TissueSpec) -> O.Desc:
    from paper_1806_10889_gb300.workloads import fidelity_mask
    return O.Desc(spec.width, spec.height, spec.n, seed=spec.seed, tissue_id=spec.tissue_id,
                  init_lambda=tuple(spec.init_lambda), wm=fidelity_mask(spec))


def orc_model(spec: TissueSpec):
    if spec.model.get("kind") == "promoter":
        return O.Promoter(**{k: v for k, v in spec.model.items() if k != "kind"})
    return O.Model(**spec.model)


def q_exact(x: float) -> int:
    """round-half-even(x * 2^32) in exact rational arithmetic."""
    f = Fraction(x) * SCALE
    fl = f.numerator // f.denominator
    rem = f - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return fl


def q_rate(x: float) -> float:
    """The rate the integer SSA actually simulates: q(x) / 2^32."""
    return q_exact(x) / SCALE


def poisson_gof(samples: np.ndarray, mean: float, min_expected: float = 5.0):
    """Chi-square goodness of fit of integer samples to Poisson(mean).

    Returns (p_value, z_of_sample_mean)."""
    samples = np.asarray(samples).ravel()
    n = samples.size
    hi = int(max(samples.max(), mean + 10 * np.sqrt(mean + 1) + 10))
    ks = np.arange(hi + 1)
    pmf = stats.poisson.pmf(ks, mean)
    pmf[-1] += stats.poisson.sf(hi, mean)
    obs = np.bincount(samples, minlength=hi + 1)[: hi + 1].astype(float)
    exp = pmf * n
    # merge bins from both tails until every bin expects >= min_expected
    bins_o, bins_e, acc_o, acc_e = [], [], 0.0, 0.0
    for o, e in zip(obs, exp):
        acc_o += o
        acc_e += e
        if acc_e >= min_expected:
            bins_o.append(acc_o)
            bins_e.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0 or acc_o > 0:
        bins_o[-1] += acc_o
        bins_e[-1] += acc_e
    bins_e = np.array(bins_e)
    bins_o = np.array(bins_o)
    bins_e *= bins_o.sum() / bins_e.sum()
    p = stats.chisquare(bins_o, bins_e).pvalue if len(bins_o) > 1 else 1.0
    z = (samples.mean() - mean) / np.sqrt(mean / n) if mean > 0 else 0.0
    return float(p), float(z)


def discrete_gof(obs_counts: np.ndarray, probs: np.ndarray, min_expected: float = 5.0):
    """Chi-square of observed category counts against exact probabilities
    (categories with small expectation are pooled)."""
    n = obs_counts.sum()
    exp = probs * n
    order = np.argsort(exp)
    bins_o, bins_e, acc_o, acc_e = [], [], 0.0, 0.0
    for i in order:
        acc_o += obs_counts[i]
        acc_e += exp[i]
        if acc_e >= min_expected:
            bins_o.append(acc_o)
            bins_e.append(acc_e)
            acc_o = acc_e = 0.0
    if bins_o:
        bins_o[-1] += acc_o
        bins_e[-1] += acc_e
    bins_o, bins_e = np.array(bins_o), np.array(bins_e)
    if len(bins_o) < 2:
        return 1.0
    bins_e *= bins_o.sum() / bins_e.sum()
    return float(stats.chisquare(bins_o, bins_e).pvalue)
