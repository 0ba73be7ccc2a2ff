"""Golden fixtures: the paper's example network (Fig. 2) and a regression
record of the oracle on the tiny tissue (written by tests/golden/make_golden.py
from oracle/ only)."""
import json
import os

import numpy as np

import oracle as O

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_face_topology_matches_paper_network_file():
    """Fig. 2 lists a 2x2 layer: each cell's neighbours are the cells one
    position step away.  Our tissue puts cell c = cy*W + cx at (cx, cy) and
    defines one S unit per shared face; the two must describe the same pairs."""
    with open(os.path.join(HERE, "fig2_network.json")) as f:
        net = json.load(f)["cells"]
    step = 1e-6
    pos = {int(k): (round(v["position"][0] / step), round(v["position"][1] / step))
           for k, v in net.items()}
    paper_pairs = set()
    for k, v in net.items():
        for nb in v["neighbors"]:
            paper_pairs.add(frozenset((pos[int(k)], pos[nb])))
    W = H = 2
    d = O.Desc(W, H, 4, seed=1)
    m = O.Model()
    counts = O.init_counts(d)
    ours = set()
    for c in range(W * H):
        for axis in (0, 1):
            try:
                O.sig_face(d, m, counts.copy(), c, axis, 0, 0.1)
            except O.OracleError:
                continue
            nb = c + 1 if axis == 0 else c + W
            ours.add(frozenset(((c % W, c // W), (nb % W, nb // W))))
    assert ours == paper_pairs
    # every module call in Fig. 2 advances its cell by end_time = 0.1, the dt used here
    assert {v["end_time"] for v in net.values()} == {0.1}


def test_oracle_matches_its_recorded_tiny_run():
    with open(os.path.join(HERE, "tiny_oracle.json")) as f:
        g = json.load(f)
    dd = g["desc"]
    d = O.Desc(dd["width"], dd["height"], dd["n"], seed=dd["seed"], tissue_id=dd["tissue_id"],
               init_lambda=tuple(dd["init_lambda"]))
    counts = O.init_counts(d)
    assert counts.reshape(4, 3, 64).sum(axis=2).tolist() == g["totals"]["0"]
    done = 0
    for upto in (1, 10, 100):
        ne, tl = O.step(d, O.Model(), counts, done, upto - done, g["dt"])
        done = upto
        assert counts.reshape(4, 3, 64).sum(axis=2).tolist() == g["totals"][str(upto)]
    assert ne.tolist() == g["last_step_events"]
    assert [[x.hex() for x in row] for row in tl] == g["last_step_t_last_hex"]
