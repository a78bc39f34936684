"""CPU FP64 oracle (test infrastructure only; see rimg_oracle's header)."""
from . import rimg_oracle  # noqa: F401
