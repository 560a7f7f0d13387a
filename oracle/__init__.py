"""FP64 CPU oracle for the MOFF imaging step.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg, never by the CUDA library or its Python binding.  It shares no code
with them.  `moff` is the direct route (grid -> zero-pad -> DFT -> |.|^2 -> average),
`fx` the independent visibility (FX / software-holography) route.
"""
from . import moff, fx  # noqa: F401
