"""GB300-native hot path of the MOR-based adaptive parareal method (arXiv 2601.10981).

The compute lives in the CUDA library built from ``csrc/`` (``build.py``) behind the C
ABI of ``include/parareal.h``; ``binding`` is its ctypes binding.  Importing the package
does not load the library; ``from paper_2601_10981_gb300 import binding`` does, and fails
if it has not been built.
"""
__all__ = ["binding", "build", "report"]
