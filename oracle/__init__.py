"""FP64 CPU oracle (test infrastructure only; see oracle/elph.py)."""
from . import elph  # noqa: F401
