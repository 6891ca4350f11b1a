"""CPU FP64 oracle for the discrete-ordinates radiative-transfer operator.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import or run anything here.  The
product path (the C-ABI library and its Python binding) never calls it and
shares no code with it; the two meet only in the seeded input generators of
``paper_2602_21958_gb300.workloads``.

Every function cites the passage of the paper it restates.  Functions whose
results are not pinned by a check independent of this module say
"parity unpinned" in their docstring.
"""
from .rt_oracle import *  # noqa: F401,F403
