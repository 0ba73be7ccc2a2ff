"""GB300-native operator-split tissue SSA (arXiv 1806.10889, "Orchestral").

The hot path -- per-cell lattice RDME by the direct-method SSA (the module chi)
and the Delta-Notch binding across cell faces (the module S), run in a Lie
splitting step -- is hand-written CUDA for sm_103a behind the C ABI declared
in ``include/tissue.h``.  ``paper_1806_10889_gb300.tissue`` is the thin Python
binding; ``workloads`` generates the seeded synthetic inputs.

Submodules are imported explicitly; importing the package loads nothing.
"""
__all__ = ["tissue", "workloads", "batching", "serving", "autotune"]
