"""Plain CPU oracle of the operator-split tissue SSA -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_1806_10889_gb300``) and never imports it.

The C source (``tissue_oracle.c``) is compiled on first use into
``oracle/_build/liboracle.so`` with ``-O2 -ffp-contract=off -fno-fast-math``.
"""
from .oracle import (  # noqa: F401
    Desc,
    Model,
    Promoter,
    ND,
    PROMOTER,
    E_STATE,
    EVENT_DTYPE,
    build,
    lib,
    philox,
    neg_ln_q58,
    exp_variate,
    quantize,
    hill_q,
    init_counts,
    init_cell,
    chi_cell,
    sig_face,
    step,
    step_traced,
    set_mutation,
    set_paranoid,
    max_threads,
    OracleError,
    LIE,
    STRANG,
)
