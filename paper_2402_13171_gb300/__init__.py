"""GB300-native D3Q27 cumulant LBM + actuator line (arxiv 2402.13171).

The compute path lives in the CUDA library ``csrc/`` behind the C ABI declared
in ``include/lbm_gb300.h``; ``lbm`` is the thin ctypes binding.  Importing the
package does not load the library; ``lbm.load()`` does, and raises if it was
not built.
"""
__all__ = ["lbm", "inputs"]
