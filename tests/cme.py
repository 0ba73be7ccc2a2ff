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
