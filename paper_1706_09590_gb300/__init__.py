"""GB300 (sm_103a) library for the multi-state quantum hierarchical Fokker-Planck equation
(Ikeda & Tanimura 2017): C ABI in include/qhfpe.h, thin binding in .qhfpe."""
from .qhfpe import (Batch, COMMUTATOR, FP64, LEFT, MIXED, MIXED_BF16X3, RIGHT, TERMINATOR, TRUNCATE,  # noqa: F401
                    TERM_ALL, TERM_DAMPING, TERM_KINETIC, TERM_POTENTIAL, TERM_TIER_DOWN, TERM_TIER_UP,
                    Propagator, QhfpeError, lib)
