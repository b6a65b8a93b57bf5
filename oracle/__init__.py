"""FP64 CPU oracle of the thermal pseudopotential MRT-LBM step (test infrastructure only)."""
from .oracle import Oracle, feq19, tables, PERIODIC, WALL, OPEN  # noqa: F401
