"""FP64 CPU oracle of the LETKF analysis (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and reference
legs import this package. It shares no code with the CUDA library.
"""
from .letkf_oracle import *  # noqa: F401,F403
from . import letkf_domains  # noqa: F401,E402
from . import letkf_dm  # noqa: F401,E402
