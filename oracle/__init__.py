"""Oracle for CFNEB: plain FP64 CPU reference implementation.

TEST INFRASTRUCTURE ONLY.  ``tests/``, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference legs of ``bench.py`` are the only callers.  The CUDA
product path never imports, links or executes anything here, and nothing here
imports the product.

Parity status: every function is pinned by ``tests/test_oracle_*.py``
(finite differences, closed-form lattice sums, published equilibrium values,
the Mueller-Brown saddle, symmetry and invariance checks).  The converged
barriers of the synthetic workloads have no published value.  The LJ and
Tersoff vacancy-hop barriers are pinned by a constrained minimisation of the
symmetric midpoint image (an independent route to the same saddle); the
graphite -> hexagonal-diamond barriers are pinned only through their
ingredients: for them parity is "parity unpinned".
"""
from . import _native  # noqa: F401
from .cfneb import (LJ, Tersoff, TERSOFF_C1988, ROTFREE_B, DEFGRAD_D, NotSPD,  # noqa: F401
                    energy_forces_virial, sym_sqrt, to_generalized, from_generalized,
                    generalized_force, AtomicImage, upwind_tangent, climbing_index,
                    neb_forces, Fire, row_fmax, Band, interpolate, unwrap_final, make_band,
                    relax_single)
from .nep import NEP  # noqa: F401


def build():
    """Compile the C part of the oracle (gcc)."""
    return _native.build()
