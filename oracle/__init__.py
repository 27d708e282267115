"""FP64 CPU oracle (test infrastructure only; see ``oracle.sdp_oracle``)."""
from .sdp_oracle import *  # noqa: F401,F403
