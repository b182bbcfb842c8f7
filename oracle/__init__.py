"""CPU oracle of the InIm cartogram iteration (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
import this package; the product path never does.
"""
from . import inim_oracle  # noqa: F401
