"""FP64 CPU oracle (test infrastructure only; see sfs_oracle's header)."""
from .sfs_oracle import *  # noqa: F401,F403
from .sfs_oracle import Geometry, LateralFFTOperator  # noqa: F401
from . import crb_oracle, lista_oracle, mixing_oracle  # noqa: F401
