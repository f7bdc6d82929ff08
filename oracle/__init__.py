"""CPU oracle (numpy complex128) for the batched RGF path.  TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA library and
imports nothing from it; both sides read their inputs from ``workloads``.
"""
from .negf_oracle import *  # noqa: F401,F403
from . import negf_oracle  # noqa: F401
