"""FP64 CPU oracle (test infrastructure only; see ``oracle.lindblad``)."""

from .lindblad import (  # noqa: F401
    THETA,
    vec,
    unvec,
    lindbladian,
    drive_generator,
    slice_generator,
    pade13_coefficients,
    onenorm,
    squaring_count,
    lu_gepp,
    lu_solve,
    expm_pade13,
    slice_propagators,
    frechet_expm,
    propagate_step,
    propagate,
    propagate_chain,
    trace_of,
    grape_fidelity_grad,
)
