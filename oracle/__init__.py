"""FP64 CPU oracle for the QG beta-plane LES step.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_2508_06678_gb300``)
never imports it and has no CPU fallback.  The oracle shares no code with the
CUDA path; both receive their inputs from ``synth``.

Every function cites the part of the paper (section / equation) it follows.
Where the paper is silent or garbled the reading taken is documented beside
the function.  Parity status per function is stated in ``qg.__doc__`` and
``apost.__doc__``.
"""
from .qg import *  # noqa: F401,F403
from .apost import *  # noqa: F401,F403
from .adjoint import *  # noqa: F401,F403
