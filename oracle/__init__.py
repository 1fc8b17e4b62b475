"""FP64 CPU oracle (test infrastructure only; see ``lsgg_oracle``)."""
from . import lsgg_oracle  # noqa: F401
