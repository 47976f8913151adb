"""CPU oracle for the server-side homomorphic matrix product (Algorithm 1).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA library (see he_oracle.c's header).
"""
from .core import build_oracle, lib  # noqa: F401
from .bfv import *  # noqa: F401,F403
