"""GB300-native DD/TD/QD matrix multiplication (arXiv 2101.06584).

The compute path is the C-ABI library ``libmpgemm.so`` (CUDA, sm_103a) built
from ``csrc/``; ``mpgemm`` is its thin Python binding.  Importing this package
does not load the library; the first call through ``mpgemm`` does, and fails
loudly if it is missing.
"""
__all__ = ["mpgemm", "inputs"]
