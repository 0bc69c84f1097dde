"""CPU FP64 oracle (test infrastructure only; see fe_oracle's module docstring)."""
from . import fe_oracle  # noqa: F401
