"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only *draws* inputs: gate kinds, qubit choices, the 2x2 / 4x4 gate matrices,
Kraus operator sets and initial density matrices.  It applies none of them; both the
oracle and the CUDA library receive the same arrays and do the arithmetic themselves.

Conventions (paper Sec. 2.3, Eq. staten): qubit index ``i`` in these lists is the paper's
qubit i_s = i + 1, so qubit 0 is the most significant bit of a basis label.  A two-qubit
matrix is indexed 2*q(first) + q(second), the paper's amplitude-quartet order (Eq. resmat2).
"""

from .circuits import (  # noqa: F401
    Op,
    Circuit,
    GATE_KINDS_MIXED,
    haar_su2,
    haar_state,
    gate_matrix,
    kraus_ad,
    kraus_pd,
    kraus_depolarising,
    kraus_pauli_multiverse,
    config1_circuit,
    config2_circuit,
    config3_circuit,
    config4_batch,
    config5_requests,
    random_circuit,
    random_density_matrix,
    zero_state,
    mixed_plus_haar_state,
    seed_for,
    MVExperiment,
    MV_ALGORITHMS,
    NOISE_SWITCHES,
    PAULI_NAMES,
    mv_experiment,
    mv_trajectories,
)
