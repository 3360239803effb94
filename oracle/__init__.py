"""FP64 CPU oracle of the phase-field lattice Boltzmann step.

Test infrastructure only: the tests, the package smoke check and the CPU
baseline leg of the benchmark may import this package; the product path must
not.  It shares no code with the CUDA library.
"""
from .oracle import (  # noqa: F401
    OracleLattice,
    OrcParams,
    build_oracle,
    cell_collide,
    chem_pot,
    delta_theta,
    filtered_collide,
    force_and_eq,
    gamma_vec,
    ghost_values,
    h_eq,
    lattice_tables,
    macros_cell,
    tanh_phi,
    tau_mix,
    cd_stencil,
)
