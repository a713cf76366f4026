"""X-drop oracle: TEST INFRASTRUCTURE ONLY.

A plain C restatement of the X-drop seed-and-extend alignment (the reading
"Definition C" documented at the top of ``xdrop_oracle.c``), loaded with
ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this package; the CUDA library never does, and the
two share no code.
"""
from .oracle import (  # noqa: F401
    NO_BEST,
    ORC_PAIR,
    ORC_RESULT,
    accept,
    align_pairs,
    best_seeds,
    build,
    extend,
    load,
    unpack,
)
