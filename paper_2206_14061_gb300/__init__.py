"""GB300 (sm_103a) Lagrangian-particle granular-flow step with mu(I) rheology.

The hot path (neighbour search, GFD least-squares fits, mu(I) closure,
stress-divergence update, adjoint) runs in the CUDA library built from
``csrc/`` behind the C ABI of ``include/lp.h``; ``capi`` is its thin binding.
"""
from .capi import (LP_FP64, LP_MIXED, LP_MIXED_FF, LP_MIRROR_FREESLIP, LP_MIRROR_NONE, LP_MIRROR_NOSLIP,  # noqa: F401
                   Context, LpError, Neighbors, lp_build_neighbors, lp_fit_derivatives,
                   lp_mui_stress, lp_step, lp_step_adjoint)
