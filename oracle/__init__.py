"""FP64 CPU oracle for the adjoint rules of arXiv 2202.10297 (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_2202_10297_gb300``.
"""
