"""GB300 (sm_103a) implementation of the PCG Hessian solve of the modified
interior-point method (Zhang & Lavaei, arXiv 1703.10973), behind the libsdpgb
C ABI declared in include/sdpgb.h."""
from ._build import LIB, build  # noqa: F401
from ._lib import SDPError, load  # noqa: F401
from .api import SDPBatch, SDPProblem, default_params, hessian_matvec_static  # noqa: F401

__all__ = ["SDPBatch", "SDPProblem", "default_params", "hessian_matvec_static", "SDPError", "build", "load", "LIB"]
