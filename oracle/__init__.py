"""FP64 CPU oracle for the clover solve of stochastic noise sources.

TEST INFRASTRUCTURE, not product code. Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline / reference leg of ``bench.py`` may
import it. It shares no code with the CUDA path (``paper_1405_4524_gb300``)
and imports nothing from it; both sides take their inputs from the seeded
generators in ``paper_1405_4524_gb300.inputs``.

Every function here is pinned by a check in ``tests/test_oracle_pins.py``
(``tests/test_oracle_diagrams.py`` for the diagram contractions of
``oracle.diagrams``) against something other than itself (closed forms,
invariants, dense LU).
"""

from . import diagrams  # noqa: F401
from .dirac import (  # noqa: F401
    GAMMA,
    GAMMA5,
    PLANES,
    apply_M,
    bicgstab,
    clover_apply,
    clover_matrices,
    dagger,
    dilute,
    field_strength,
    hopping,
    hopping_eo,
    inner,
    parity_field,
    pion_correlator,
    propagator_trace,
    stochastic_operator,
    stochastic_operator_correlator,
    stochastic_propagator,
    stochastic_propagator_trace,
    plaquette_leaves,
    restrict,
    schur_apply,
    schur_reconstruct,
    schur_source,
    shift,
    sigma,
    site_apply,
    solve,
)
