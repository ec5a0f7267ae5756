"""FP64 CPU oracle for the SHARP RAAR hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA library never does.
"""
from .sharp_oracle import *  # noqa: F401,F403
from .sharp_oracle import (D_REL_THRESHOLD, PROBE_REL_THRESHOLD,  # noqa: F401
                           frame_indices, global_phase, norm)
