"""GB300-native linear-complexity Silhouette (arXiv 2303.14102).

The compute path is the CUDA library ``libsil.so`` (sources in ``csrc/``,
C ABI declared in ``include/sil.h``); ``paper_2303_14102_gb300.sil`` is its
thin ctypes binding and ``paper_2303_14102_gb300.autograd`` the
``torch.autograd.Function`` around it.  Importing this package loads
nothing; the library is loaded on first use and fails loudly when missing.
"""
__all__ = ["sil", "autograd", "synth"]
