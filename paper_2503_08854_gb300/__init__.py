"""GB300-native non-linear digital tracking (after arXiv 2503.08854).

The compute path is the CUDA library ``csrc/`` behind the C ABI declared in
``include/ndt.h``; ``paper_2503_08854_gb300.ndt`` is its thin ctypes binding.
``paper_2503_08854_gb300.synth`` draws seeded synthetic survey inputs.  Neither
is imported here, so importing the package loads no native code.
"""
__all__ = ["ndt", "synth"]
