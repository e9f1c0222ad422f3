"""Band-limited PDE-constrained LDDMM with Gauss-Newton-Krylov optimisation on
GB300 (sm_103a).

The compute path is the C-ABI library ``libblr.so`` (CUDA kernels in ``csrc/``);
``blr`` is its thin ctypes binding.  Importing this package does not load the
library; ``paper_1807_05117_gb300.blr`` does, and fails loudly if it is missing.
"""

__all__ = ["blr", "synth", "build"]
