"""GB300-native OSLQ / OSA-IOP log-determinant estimation (arXiv 2606.07004).

The compute path is the CUDA library ``liblogdet.so`` (sources in ``csrc/``,
C-ABI in ``include/logdet.h``); ``binding`` is its ctypes front end.  Import
``paper_2606_07004_gb300.binding`` to load the library: it raises if the
library has not been built.
"""
__all__ = ["binding", "build"]
