"""GB300-native Scheduled Relaxation Jacobi (SRJ) solver.

The compute path lives in the CUDA library ``libsrj.so`` built from
``csrc/``; ``srj.py`` is its thin ctypes binding.  Importing this package does
not load the library: ``from paper_2011_06636_gb300 import srj`` does.
"""
__all__ = ["srj", "inputs"]
