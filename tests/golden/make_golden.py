"""Write tests/golden/tiny_oracle.json from the CPU oracle alone.

The tiny tissue (2x2 cells of 8x8 voxels, seed 1, Notch-Delta model, dt 0.1)
is advanced 100 steps (T = 10); the file stores per-cell species totals after
steps 0, 1, 10 and 100 and the event counts of the last step.  Run:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402


def main():
    d = O.Desc(2, 2, 8, seed=1, tissue_id=0, init_lambda=(5.0, 5.0, 5.0))
    m = O.Model()
    counts = O.init_counts(d)
    out = {"_source": "written by tests/golden/make_golden.py from oracle/ only",
           "desc": {"width": 2, "height": 2, "n": 8, "seed": 1, "tissue_id": 0,
                    "init_lambda": [5.0, 5.0, 5.0]},
           "dt": 0.1, "totals": {}}
    out["totals"]["0"] = counts.reshape(4, 3, 64).sum(axis=2).tolist()
    done = 0
    for upto in (1, 10, 100):
        ne, tl = O.step(d, m, counts, done, upto - done, 0.1)
        done = upto
        out["totals"][str(upto)] = counts.reshape(4, 3, 64).sum(axis=2).tolist()
    out["last_step_events"] = ne.tolist()
    out["last_step_t_last_hex"] = [[float(x).hex() for x in row] for row in tl]
    with open(os.path.join(HERE, "tiny_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
