"""paper_2508_06628_b300 -- batched pair-potential MD / FIRE / adjoint engine for B300.

The compute path is the C-ABI library ``libts.so`` (hand-written CUDA for
sm_103a, declared in ``include/ts.h``); ``paper_2508_06628_b300.ts`` is the thin
Python binding over it.  Importing this package does not load CUDA; the
binding loads ``libts.so`` on first use and raises if it is missing.
"""
__all__ = ["ts", "workloads"]
