"""FP64 CPU oracle (test infrastructure only; see ``pd_oracle``)."""

from .pd_oracle import *  # noqa: F401,F403
