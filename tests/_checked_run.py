"""Run representative workloads on the range-checked library build
(TISSUE_CHECKED=1) and compare every step with the oracle.  Executed in its
own process by test_gpu_checked_build.py; exits non-zero on any mismatch
or reported out-of-range index."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1806_10889_gb300 import tissue as T  # noqa: E402
from paper_1806_10889_gb300 import workloads as W  # noqa: E402
from paper_1806_10889_gb300.batching import Batch  # noqa: E402
from paper_1806_10889_gb300.workloads import TissueSpec  # noqa: E402
from dataclasses import replace  # noqa: E402
from tests._util import orc_desc, orc_model  # noqa: E402

P, PRE, REC = T.KERNEL_PERSISTENT, T.LAYOUT_PREFIX, T.LAYOUT_RECOMPUTE


def same(spec, dt, n_steps, config=None, scheme=O.LIE, x0=None):
    d, m = orc_desc(spec), orc_model(spec)
    ref = O.init_counts(d) if x0 is None else x0.copy()
    g = T.Tissue(spec)
    if x0 is not None:
        g.write_counts(x0, 0)
    if config:
        g.set_launch_config(*config)
    if scheme == O.STRANG:
        g.set_splitting(T.SPLIT_STRANG)
    for k in range(n_steps):
        ne, tl = O.step(d, m, ref, k, 1, dt, scheme=scheme)
        g.step(dt, 1)
        got = g.read_counts()  # raises TissueError(E_BOUNDS) on a caught index
        gne, gtl = g.read_stats()
        assert np.array_equal(got, ref), (spec, config, k)
        assert np.array_equal(gne, ne) and np.array_equal(gtl.view(np.uint64), tl.view(np.uint64))
    g.close()


def main():
    assert T.checked() and T.library_path().endswith("libtissue_checked.so")
    same(W.tiny().tissue, 0.1, 10)
    strong = dict(k_bind=0.05)
    for w, h, n, dt in ((5, 3, 16, 0.1), (3, 2, 10, 0.1), (2, 2, 32, 0.05), (4, 1, 2, 0.5),
                        (1, 3, 7, 0.2), (1, 1, 8, 0.1)):
        spec = TissueSpec(w, h, n, seed=3000 + n, tissue_id=w * h).with_model(**strong)
        for cfg in (None, (T.KERNEL_WARP, 32, 4, 0, PRE), (P, 8, 4, 0, PRE), (P, 16, 2, 0, PRE),
                    (P, 32, 2, 0, PRE), (P, 16, 4, 0, REC), (P, 8, 2, 0, REC), (P, 16, 1, 2, PRE)):
            # the counts-only layout: V <= lanes^2, or up to four voxels a lane
            if cfg and cfg[4] == REC and n * n > cfg[1] ** 2 and \
                    not (cfg[1] == 16 and n * n <= 1024) and not (cfg[1] == 8 and n * n <= 256):
                continue
            try:
                same(spec, dt, 2, cfg)
            except T.TissueError as e:
                if e.code != T.E_ARG:  # E_ARG: shape does not fit shared memory
                    raise
    # 32x32-voxel cells with 16-bit counts: one cell starts above 65535 and one
    # passes it mid-step, so both go through the 32-bit redo pass
    big = TissueSpec(3, 2, 32, seed=71, tissue_id=3).with_model(hopD=0.0, k_off=1.0, k_in=0.0)
    x = O.init_counts(orc_desc(big)).reshape(big.cells, 3, big.V)
    x[1, 0, 0] = 70000
    x[4, 0, 5] = 65000
    x[4, 2, 5] = 0xFFFF
    for cfg in (None, (P, 16, 2, 0, PRE), (P, 8, 2, 0, PRE), (P, 32, 2, 0, REC),
                (P, 16, 2, 0, REC)):
        same(big, 0.05, 2, cfg, x0=x.ravel())
    model = W.promoter_model(8)
    model["kd"] = 3.0
    pm = TissueSpec(4, 3, 8, seed=7, init_lambda=(0.6, 0.4, 0.0), model=model)
    same(pm, 0.1, 3)
    same(pm, 0.1, 2, scheme=O.STRANG)
    same(replace(pm, fidelity="edge:1"), 0.1, 3)
    same(replace(TissueSpec(4, 4, 16, seed=8), fidelity="well_mixed"), 0.1, 2)
    # a batch mixing cell sizes, models and fidelities
    specs = [TissueSpec(3, 2, 8, seed=9, tissue_id=0), replace(pm, tissue_id=1),
             TissueSpec(2, 2, 32, seed=9, tissue_id=2),
             replace(TissueSpec(3, 3, 16, seed=9, tissue_id=3), fidelity="edge:1")]
    members = [T.Tissue(s) for s in specs]
    b = Batch(members)
    refs = [O.init_counts(orc_desc(s)) for s in specs]
    for k in range(2):
        b.step(0.1, 1)
        b.sync()
        for i, s in enumerate(specs):
            O.step(orc_desc(s), orc_model(s), refs[i], k, 1, 0.1)
            assert np.array_equal(members[i].read_counts(), refs[i]), (k, i)
    b.close()
    for m in members:
        m.close()
    print("checked build ok")


if __name__ == "__main__":
    main()
