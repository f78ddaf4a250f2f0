"""GB300 implementation of the planar photoacoustic operator H, its adjoint H*
and FISTA (Küçükkömürcü et al., depth-dependent transverse shift-invariant
operator). Compute runs in libpat.so (hand-written CUDA for sm_103a); this
package only marshals arguments to its C ABI."""
from .pat import (FLAG_FORCE_COMPLEX, FLAG_FP64, Medium, PatError, Plan, apply,  # noqa: F401
                  lib)
