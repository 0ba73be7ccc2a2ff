"""Host-side logic of bench.py on the CPU: the wavefront bound against brute
force, the chi kernel keys, the instruction-count table's freshness, and the
samples the benchmark draws from its workloads."""
import numpy as np

import bench
from paper_1806_10889_gb300 import workloads as W


def test_wavefront_bound_matches_brute_force():
    rng = np.random.default_rng(7)
    K, H, Wd = 6, 4, 5
    e = rng.integers(1, 1000, size=(K, H, Wd)).astype(float)
    F = {}
    for k in range(K):
        for y in range(H):
            for x in range(Wd):
                prev = max(F.get((k - 1, yy, xx), 0.0)
                           for yy in range(y - 1, y + 2) for xx in range(x - 1, x + 2)
                           if 0 <= yy < H and 0 <= xx < Wd)
                F[(k, y, x)] = prev + e[k, y, x]
    got = bench.wavefront_bound(e.reshape(K, -1), Wd, H)
    assert got["wavefront_events"] == max(F[(K - 1, y, x)] for y in range(H) for x in range(Wd))
    assert got["barrier_events"] == e.max(axis=(1, 2)).sum()
    assert got["slowest_cell_events"] == e.sum(axis=0).max()
    # the wavefront never beats the slowest cell's own chain, nor loses to the barrier
    assert got["slowest_cell_events"] <= got["wavefront_events"] <= got["barrier_events"]


def test_wavefront_bound_is_zero_when_one_cell_is_slowest_every_step():
    e = np.ones((4, 3, 3))
    e[:, 1, 1] = 10.0
    got = bench.wavefront_bound(e.reshape(4, -1), 3, 3)
    assert got["gain_bound"] == 0.0


def test_chi_kernel_keys():
    assert bench.chi_kernel_key(1024, 32, 0) == "V1024/H32/pre/qb0/nd/u16"
    assert bench.chi_kernel_key(1024, 16, 0) == "V1024/H16/pre/qb1/nd/u16"
    assert bench.chi_kernel_key(1024, 32, 1) == "V1024/H32/rec/qb0/nd/u16"
    assert bench.chi_kernel_key(256, 16, 0) == "V256/H16/pre/qb0/nd/u32"
    assert bench.chi_kernel_key(64, 8, 1) == "V64/H8/rec/qb0/nd/u32"


def test_instruction_counts_were_measured_on_the_current_kernel():
    """The issue roofline multiplies live event rates by ncu's instructions per
    event; a kernel change without a new measurement must fail here."""
    assert bench.CHI_IPE["sources"] == bench.chi_sources_sha(), (
        "the persistent chi kernel changed since its instructions per event were measured: "
        "re-run the ncu commands in profiles/k_chi_inst_per_event_by_cell_size.md")
    # the default launches of the benchmark's workloads (the batch's 16x16-voxel
    # class: 8 lanes, counts only, above 6,080 cells) and the former default
    for key in ("batch:V1024/H16/rec/qb1/nd/u16", "batch:V256/H8/rec/qb1/nd/u32",
                "batch:V256/H16/pre/qb0/nd/u32", "batch:V64/H8/pre/qb0/nd/u32",
                "medium:V256/H16/pre/qb0/nd/u32", "large:V1024/H16/rec/qb1/nd/u16"):
        ipe, bpe = bench.CHI_IPE["kernels"][key]
        assert 100 < ipe < 1000 and 0 < bpe < 10


def test_oracle_sample_has_every_cell_size():
    runs = W.batch()
    idx = bench.oracle_sample(runs)
    assert sorted(runs[i].tissue.n for i in idx) == [8, 16, 32]
    sub = bench.profile_subset(runs)
    assert {runs[i].tissue.n for i in sub} == {8, 16, 32} and len(sub) == 48


def test_serving_requests_cap_replicas_only():
    full = W.serving()[:20]
    capped = bench.serving_requests(20, 2)
    for a, b in zip(full, capped):
        assert b.replicas == min(a.replicas, 2)
        assert (a.index, a.arrival_s, a.side, a.n, a.n_steps) == (b.index, b.arrival_s, b.side,
                                                                  b.n, b.n_steps)


def test_kernel_hash_ignores_comments_but_not_code():
    import os
    base = {f: open(os.path.join(bench.CSRC, f)).read() for f in bench.CHI_SOURCES}
    sha = bench.chi_sources_sha(base.get)
    commented = dict(base, **{"chi_seg.cuh": "// a note\n" + base["chi_seg.cuh"] + "\n/* more */\n"})
    assert bench.chi_sources_sha(commented.get) == sha
    hosty = dict(base, **{"tissue_internal.h": base["tissue_internal.h"] + "\nint host_only(int);\n"})
    assert bench.chi_sources_sha(hosty.get) == sha
    changed = dict(base, **{"tissue_dev.cuh": base["tissue_dev.cuh"].replace(
        "0xD2511F53u", "0xD2511F55u", 1)})
    assert bench.chi_sources_sha(changed.get) != sha
