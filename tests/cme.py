"""Exact chemical master equation of the split process on tiny state spaces.

The test side's own restatement of the reaction network as three generator
matrices -- Q_chi (per-cell kinetics), Q_Sx and Q_Sy (face binding) -- over
the states reachable from one initial count vector.  The law after k Lie
splitting steps of length dt is
    p_k = (exp(Q_Sy dt) exp(Q_Sx dt) exp(Q_chi dt))^k p_0.
Only models without production (kD = kN = 0) are used so the space is finite,
except for the promoter model, whose transcription is handled by truncating
the space at a Delta count the law almost never reaches.
"""
from __future__ import annotations

from collections import deque

import numpy as np
from scipy import linalg, sparse


def _nbr(n, v, d):
    vx, vy = v % n, v // n
    if d == 0:
        return v - 1 if vx > 0 else -1
    if d == 1:
        return v + 1 if vx < n - 1 else -1
    if d == 2:
        return v - n if vy > 0 else -1
    return v + n if vy < n - 1 else -1


def _idx(n, c, s, v):
    return (c * 3 + s) * n * n + v


def chi_moves(W, H, n, r, x):
    """(rate, new_state) of every chi reaction from state x (a tuple)."""
    V = n * n
    out = []
    for c in range(W * H):
        for v in range(V):
            D, N, R = x[_idx(n, c, 0, v)], x[_idx(n, c, 1, v)], x[_idx(n, c, 2, v)]
            for s, cnt, g in ((0, D, r["gD"]), (1, N, r["gN"]), (2, R, r["gR"])):
                if cnt and g:
                    y = list(x)
                    y[_idx(n, c, s, v)] -= 1
                    out.append((g * cnt, tuple(y)))
            for s, cnt, h in ((0, D, r["hopD"]), (1, N, r["hopN"]), (2, R, r["hopR"])):
                if not (cnt and h):
                    continue
                for d in range(4):
                    u = _nbr(n, v, d)
                    if u < 0:
                        continue
                    y = list(x)
                    y[_idx(n, c, s, v)] -= 1
                    y[_idx(n, c, s, u)] += 1
                    out.append((h * cnt, tuple(y)))
            if D and N and r["k_in"]:
                y = list(x)
                y[_idx(n, c, 0, v)] -= 1
                y[_idx(n, c, 1, v)] -= 1
                y[_idx(n, c, 2, v)] += 1
                out.append((r["k_in"] * D * N, tuple(y)))
            if R and r["k_off"]:
                y = list(x)
                y[_idx(n, c, 2, v)] -= 1
                y[_idx(n, c, 0, v)] += 1
                y[_idx(n, c, 1, v)] += 1
                out.append((r["k_off"] * R, tuple(y)))
    return out


def face_pairs(W, H, n, axis):
    """(cell a, voxel a, cell b, voxel b) of every voxel pair across the faces."""
    pairs = []
    for c in range(W * H):
        cx, cy = c % W, c // W
        if axis == 0 and cx + 1 < W:
            pairs += [(c, p * n + n - 1, c + 1, p * n) for p in range(n)]
        if axis == 1 and cy + 1 < H:
            pairs += [(c, (n - 1) * n + p, c + W, p) for p in range(n)]
    return pairs


def sig_moves(W, H, n, r, x, axis):
    out = []
    for ca, va, cb, vb in face_pairs(W, H, n, axis):
        for (cd, vd, cr, vr) in ((ca, va, cb, vb), (cb, vb, ca, va)):
            Dd, Nr = x[_idx(n, cd, 0, vd)], x[_idx(n, cr, 1, vr)]
            if Dd and Nr and r["k_bind"]:
                y = list(x)
                y[_idx(n, cd, 0, vd)] -= 1
                y[_idx(n, cr, 1, vr)] -= 1
                y[_idx(n, cr, 2, vr)] += 1
                out.append((r["k_bind"] * Dd * Nr, tuple(y)))
    return out


def promoter_chi_moves(W, H, n, r, x):
    """chi reactions of the promoter model (Sec. III-A1): slot 0 Delta, slot 1
    NICD, slot 2 bound promoter sites; one site per cell at voxel (n/2, n/2)."""
    V = n * n
    centre = (n // 2) * n + n // 2
    out = []

    def moved(changes):
        y = list(x)
        for (c, s, v), dv in changes:
            y[_idx(n, c, s, v)] += dv
        return tuple(y)

    for c in range(W * H):
        for v in range(V):
            D, N, B = x[_idx(n, c, 0, v)], x[_idx(n, c, 1, v)], x[_idx(n, c, 2, v)]
            free = (1 if v == centre else 0) - B
            assert free >= 0
            if free and r["tD"]:
                out.append((r["tD"] * free, moved([((c, 0, v), +1)])))
            if free and N and r["ka"]:
                out.append((r["ka"] * N * free, moved([((c, 1, v), -1), ((c, 2, v), +1)])))
            if B and r["kd"]:
                out.append((r["kd"] * B, moved([((c, 2, v), -1), ((c, 1, v), +1)])))
            for s, cnt in ((0, D), (1, N)):
                if cnt and r["d"]:
                    out.append((r["d"] * cnt, moved([((c, s, v), -1)])))
                if cnt and r["hop"]:
                    for d in range(4):
                        u = _nbr(n, v, d)
                        if u >= 0:
                            out.append((r["hop"] * cnt, moved([((c, s, v), -1), ((c, s, u), +1)])))
    return out


def promoter_sig_moves(W, H, n, r, x, axis):
    """Face reactions of the promoter model: a Delta in a face voxel becomes
    NICD in the facing voxel of the other cell."""
    out = []
    for ca, va, cb, vb in face_pairs(W, H, n, axis):
        for (cd, vd, cr, vr) in ((ca, va, cb, vb), (cb, vb, ca, va)):
            Dd = x[_idx(n, cd, 0, vd)]
            if Dd and r["kN"]:
                y = list(x)
                y[_idx(n, cd, 0, vd)] -= 1
                y[_idx(n, cr, 1, vr)] += 1
                out.append((r["kN"] * Dd, tuple(y)))
    return out


def split_law(W, H, n, rates, x0, dt, k_steps, scheme="lie", model="nd", max_delta=None):
    """Return (states list, index dict, law after k_steps, generators).

    Lie:    p <- E_Sy(dt) E_Sx(dt) E_chi(dt) p
    Strang: p <- E_Sx(dt/2) E_Sy(dt/2) E_chi(dt) E_Sy(dt/2) E_Sx(dt/2) p
    (the rightmost factor acts first).
    model "promoter" uses the promoter model's reactions.  max_delta, if
    given, truncates the space at that many Delta molecules in the tissue:
    moves above it are dropped but keep their rate on the diagonal, so the
    law then sums to 1 minus the probability of having crossed the bound."""
    chi_f, sig_f = (promoter_chi_moves, promoter_sig_moves) if model == "promoter" else \
        (chi_moves, sig_moves)
    V = n * n

    def delta_total(y):
        return sum(y[_idx(n, c, 0, v)] for c in range(W * H) for v in range(V))

    x0 = tuple(int(v) for v in x0)
    idx = {x0: 0}
    states = [x0]
    edges = {"chi": [], "sx": [], "sy": []}
    leak = {"chi": [], "sx": [], "sy": []}
    q = deque([x0])
    while q:
        x = q.popleft()
        i = idx[x]
        for name, moves in (("chi", chi_f(W, H, n, rates, x)),
                            ("sx", sig_f(W, H, n, rates, x, 0)),
                            ("sy", sig_f(W, H, n, rates, x, 1))):
            for rate, y in moves:
                if max_delta is not None and delta_total(y) > max_delta:
                    leak[name].append((i, rate))
                    continue
                if y not in idx:
                    idx[y] = len(states)
                    states.append(y)
                    q.append(y)
                edges[name].append((i, idx[y], rate))
    S = len(states)
    Q = {}
    for name, es in edges.items():
        M = np.zeros((S, S))
        for i, j, rate in es:
            M[j, i] += rate
            M[i, i] -= rate
        for i, rate in leak[name]:
            M[i, i] -= rate
        Q[name] = M
    p = np.zeros(S)
    p[0] = 1.0
    if scheme == "lie":
        P = {name: linalg.expm(M * dt) for name, M in Q.items()}
        for _ in range(k_steps):
            p = P["sy"] @ (P["sx"] @ (P["chi"] @ p))
    else:
        chi = linalg.expm(Q["chi"] * dt)
        hx, hy = linalg.expm(Q["sx"] * dt / 2), linalg.expm(Q["sy"] * dt / 2)
        for _ in range(k_steps):
            p = hx @ (hy @ (chi @ (hy @ (hx @ p))))
    return states, idx, p, Q


# ---- tissues with well-mixed cells (promoter model) -----------------------
#
# A well-mixed cell's chi ignores position: it runs the SSA on the cell's
# totals, then places every molecule in a uniformly random voxel (the bound
# promoter site stays on the promoter voxel).  As a Markov kernel on full
# voxel states that is  K_chi = Place . exp(Q_hyb dt) . Aggregate,  where the
# hybrid state keeps the lattice cells' voxels and the well-mixed cells'
# totals, and Q_hyb is the sum of the lattice RDME generator and the
# well-mixed generators (cells are independent within chi).

def _wm_total_moves(r, V, T):
    """(rate, new totals) of a well-mixed promoter cell with totals T = (D, N, R)."""
    D, N, R = T
    F = 1 - R
    out = []
    ka_c = r["ka_cell"]
    if F and r["tD"]:
        out.append((r["tD"] * F, (D + 1, N, R)))
    if R and r["kd"]:
        out.append((r["kd"] * R, (D, N + 1, R - 1)))
    if D and r["d"]:
        out.append((r["d"] * D, (D - 1, N, R)))
    if N and r["d"]:
        out.append((r["d"] * N, (D, N - 1, R)))
    if N and F and ka_c:
        out.append((ka_c * N * F, (D, N - 1, R + 1)))
    return out


def _placements(n, total, centre=None):
    """Every voxel vector of `total` molecules over n*n voxels with its
    multinomial probability (all at `centre` if given)."""
    V = n * n
    if centre is not None:
        vec = [0] * V
        vec[centre] = total
        return [(tuple(vec), 1.0)]
    out = []

    def rec(i, left, vec):
        if i == V - 1:
            vec = vec + [left]
            # multinomial: total! / prod(k!) * V^-total
            from math import factorial
            p = factorial(total)
            for k in vec:
                p //= factorial(k)
            out.append((tuple(vec), p / V ** total))
            return
        for k in range(left + 1):
            rec(i + 1, left - k, vec + [k])

    rec(0, total, [])
    return out


def wm_split_law(W, H, n, rates, x0, dt, k_steps, wm):
    """Exact law of the Lie-split promoter model on a tissue whose cells with
    wm[c] = 1 are well-mixed.  rates: the quantised lattice rates plus
    "ka_cell", the quantised compartment binding rate k_a / V."""
    V = n * n
    C = W * H
    centre = (n // 2) * n + n // 2
    lattice = [c for c in range(C) if not wm[c]]
    mixed = [c for c in range(C) if wm[c]]

    def hyb(x):
        part = tuple(x[_idx(n, c, s, v)] for c in lattice for s in range(3) for v in range(V))
        tot = tuple(sum(x[_idx(n, c, s, v)] for v in range(V)) for c in mixed for s in range(3))
        return part + tot

    def full_from(h, placements_of):
        """All full states (with probabilities) of hybrid state h."""
        base = [0] * (C * 3 * V)
        k = 0
        for c in lattice:
            for s in range(3):
                for v in range(V):
                    base[_idx(n, c, s, v)] = h[k]
                    k += 1
        outs = [(base, 1.0)]
        for j, c in enumerate(mixed):
            T = h[k + 3 * j:k + 3 * j + 3]
            new = []
            for vec, p in outs:
                for pd, qd in placements_of(T[0], None):
                    for pn, qn in placements_of(T[1], None):
                        for pr, qr in placements_of(T[2], centre):
                            y = list(vec)
                            for v in range(V):
                                y[_idx(n, c, 0, v)] = pd[v]
                                y[_idx(n, c, 1, v)] = pn[v]
                                y[_idx(n, c, 2, v)] = pr[v]
                            new.append((y, p * qd * qn * qr))
            outs = new
        return [(tuple(y), p) for y, p in outs]

    cache = {}

    def placements_of(total, ctr):
        key = (total, ctr)
        if key not in cache:
            cache[key] = _placements(n, total, ctr)
        return cache[key]

    def hyb_moves(h):
        x = full_from(h, lambda t, ctr: [(tuple([t] + [0] * (V - 1)), 1.0)] if ctr is None
                      else [(tuple(t if v == ctr else 0 for v in range(V)), 1.0)])[0][0]
        out = []
        # lattice cells: RDME moves on their voxels
        for rate, y in promoter_chi_moves(W, H, n, rates, x):
            changed = {i // (3 * V) for i in range(len(x)) if x[i] != y[i]}
            if changed <= set(lattice):
                out.append((rate, hyb(y)[:len(h) - 3 * len(mixed)] + h[len(h) - 3 * len(mixed):]))
        k0 = len(h) - 3 * len(mixed)
        for j in range(len(mixed)):
            T = h[k0 + 3 * j:k0 + 3 * j + 3]
            for rate, T2 in _wm_total_moves(rates, V, T):
                out.append((rate, h[:k0 + 3 * j] + tuple(T2) + h[k0 + 3 * j + 3:]))
        return out

    # closure of full states and hybrid states
    x0 = tuple(int(v) for v in x0)
    full_idx, fulls = {x0: 0}, [x0]
    hyb_idx, hybs = {}, []
    qf = deque([x0])

    def add_full(y):
        if y not in full_idx:
            full_idx[y] = len(fulls)
            fulls.append(y)
            qf.append(y)

    def add_hyb(h):
        if h in hyb_idx:
            return False
        hyb_idx[h] = len(hybs)
        hybs.append(h)
        return True

    while qf:
        x = qf.popleft()
        for axis in (0, 1):
            for _, y in promoter_sig_moves(W, H, n, rates, x, axis):
                add_full(y)
        h0 = hyb(x)
        if add_hyb(h0):
            qh = deque([h0])
            while qh:
                h = qh.popleft()
                for y, _ in full_from(h, placements_of):
                    add_full(y)
                for _, h2 in hyb_moves(h):
                    if add_hyb(h2):
                        qh.append(h2)
    S, Hn = len(fulls), len(hybs)
    A = np.zeros((Hn, S))
    for i, x in enumerate(fulls):
        A[hyb_idx[hyb(x)], i] = 1.0
    Qh = np.zeros((Hn, Hn))
    for i, h in enumerate(hybs):
        for rate, h2 in hyb_moves(h):
            j = hyb_idx[h2]
            Qh[j, i] += rate
            Qh[i, i] -= rate
    Pm = np.zeros((S, Hn))
    for i, h in enumerate(hybs):
        for y, p in full_from(h, placements_of):
            Pm[full_idx[y], i] += p
    Qs = {}
    for axis, name in ((0, "sx"), (1, "sy")):
        M = np.zeros((S, S))
        for i, x in enumerate(fulls):
            for rate, y in promoter_sig_moves(W, H, n, rates, x, axis):
                j = full_idx[y]
                M[j, i] += rate
                M[i, i] -= rate
        Qs[name] = M
    K_chi = Pm @ linalg.expm(Qh * dt) @ A
    Ex, Ey = linalg.expm(Qs["sx"] * dt), linalg.expm(Qs["sy"] * dt)
    p = np.zeros(S)
    p[0] = 1.0
    for _ in range(k_steps):
        p = Ey @ (Ex @ (K_chi @ p))
    return fulls, full_idx, p
