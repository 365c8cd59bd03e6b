"""Plain FP64 CPU oracle of the hybrid LB/FD step of arXiv:1102.3094 (Sec. 2).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.
"""
from . import oracle, diag  # noqa: F401
