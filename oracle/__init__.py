"""CPU oracle (TEST INFRASTRUCTURE ONLY).

Plain single-threaded FP64 restatement of the randomized small-block Lanczos
null-space method (Kressner & Shao, Alg. 2 with locking and FP64 refinement).
Only tests/, the smoke check and the bench's CPU-baseline / reference leg may
import this package; the CUDA library never does, and the two share no code.
"""

from .philox import philox4x32_10, uniform01, gaussian, perturbation_diagonal, start_block  # noqa: F401
from .lanczos import lanczos_nullspace, refine_null, Operator, norm2_A, qr_pos, U_FP64  # noqa: F401
from .checks import principal_sine, indicator_basis, copy_pair_basis, components  # noqa: F401
