"""h2bem on GB300: the boundary double-layer operator of the Fredkin-Koehler
FEM/BEM method as an H2 matrix (arXiv:1811.05731), assembled and applied by
hand-written CUDA kernels for sm_103a.

The compute path is the C-ABI library ``libh2bem`` (``include/h2bem.h``); this
package only marshals arguments to it.  The functions carry the C names:

* :func:`h2_build_geometry` - closed surface mesh -> geometry handle
  (mesh checks, solid angle Psi at every node; Eq. mainInt)
* :func:`h2_assemble`       - geometry + parameters -> H2 operator
  (Section "H2-Matrix Compression")
* :func:`h2_matvec`         - u2 = M u1 for r right-hand sides (Eq. denseMat)
* :func:`h2_free`           - release a handle
* :func:`h2_fem_create`, :func:`h2_fem_solve` - the finite-element half of the
  field evaluation on a tetrahedral mesh (u1 Neumann solve, u2 boundary values
  through the operator and Dirichlet solve, energy; Section "Basic Equations")

:class:`Geometry`, :class:`Operator` and :class:`Fem` wrap the handles.  There is no CPU
fallback: if the library is missing or cannot be loaded, every call raises.
"""
from ._lib import (  # noqa: F401
    H2Error, Params, Stats, FP64, FP32, TF32X3, BF16X3, matvec_batched, h2_matvec_batched, h2_autotune, SCHEDULE_FLOW, SCHEDULE_LEVELS,
    COUPLING_STORED, COUPLING_ON_THE_FLY, NEAR_FP64, NEAR_F32PAIR, lib, load,
    h2_default_params, h2_build_geometry, h2_assemble, h2_matvec, h2_matvec_noalloc, h2_free,
    h2_stats, h2_plan_check, PlanReport,
    h2_get_tree, h2_get_blocks, h2_get_psi, h2_device_status, h2_error_string,
    Geometry, Operator, Fem, FemReport, h2_fem_create, h2_fem_solve,
)
from .build import build, lib_path  # noqa: F401
