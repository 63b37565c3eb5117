"""qcw: GB300-native density-matrix evolution (the QCWAVE hot path) behind a C ABI.

The compute path is libqcw.so (hand-written CUDA for sm_103a, built in-tree by
``build.build()``); this package only binds it.
"""

from ._binding import (  # noqa: F401
    QCW_EINVAL,
    QCW_ENOMEM,
    QCW_ENOTSUP,
    QCW_ETIMEOUT,
    QCW_EZEROPROB,
    QCW_MODE_FUSED,
    QCW_MODE_PLAIN,
    QCW_OK,
    SIGNATURES,
    Batch,
    Density,
    Ensemble,
    Server,
    QcwResult,
    PackedOps,
    QcwOp,
    QcwError,
    lib,
    run_circuit,
)
