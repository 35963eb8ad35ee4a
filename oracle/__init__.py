"""FP64 CPU oracle for the collocation BEM operators (test infrastructure only).

Only the tests, the smoke check and the bench's CPU-baseline leg import this
package.  It shares no code with the CUDA library.
"""
from .oracle import (  # noqa: F401
    FLAG_NO_HALF,
    FLAG_NO_REFINE,
    FLAG_RULE1,
    adjoint,
    apply,
    assemble,
    entries,
    eval_points,
    eval_points_grad,
    geometry,
    grad,
    lu_solve,
    num_threads,
)
from .isosurface import isosurface  # noqa: F401,E402
from .topological import point_source_field, topological_derivative  # noqa: F401,E402
from . import levelset  # noqa: F401,E402
from . import burton_miller  # noqa: F401,E402
from . import fem  # noqa: F401,E402
