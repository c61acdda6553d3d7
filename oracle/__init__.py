"""CPU oracle for the 1D PIC polar-cap tube (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and ``--impl reference`` arm) may import this package.
The CUDA library and its Python binding never import it, and it imports
nothing from them.
"""

from .sclf_oracle import (  # noqa: F401
    C_LIGHT, E_CHARGE, M_ELECTRON, G_NEWTON, M_SUN, FIXED_SCALE,
    RHO_FLAT, RHO_GR, code_units, rho_gj_profile, poisson_potential, initial_fields,
    base_weight_fixed, injection_count, macro_charge_for, default_dt,
    gather, push, fractions, quantized_fraction, fixed_fractions, accumulate, deposit_fractions, current_from,
    field_update, rho_nodes, fix32_bits, gather_fix32, push_fix32, fix32_fractions,
    deposit_fix32, base_weight_fix32, Tube,
)
