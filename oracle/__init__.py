"""FP64 CPU oracle of the sheared model-H step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and ``--impl reference``) may import anything here.  The
product (the CUDA library and its Python binding) never imports this package,
and this package never imports the product.

Pinned against the paper and mathematics in ``tests/test_oracle_*.py``; every
function of ``scheme`` is pinned (none is marked "parity unpinned").
"""
from .scheme import (  # noqa: F401
    Params, REMAP_SHIFT, REMAP_NONE, strain, shifted, d_x, d_y_sheared,
    lap_sheared, bracket, chemical_potential, body_force_curl, wavenumbers,
    sheared_k2, remap_rows, advect, cahn_hilliard_spectral, vorticity_poisson_solve,
    stokes_solve, flow_substep, step, run,
    mean_phi, structure_factor_moments, structure_factor_binned, gradient_tensor, principal_lengths,
)
