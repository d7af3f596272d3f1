"""GB300-native explicit phase-field PVD time step (arXiv 2312.05410, Materials and Methods).

The package holds the CUDA kernels and C-ABI library (``csrc/``), the ctypes
binding (``pf``), the in-tree build step (``build``) and the seeded synthetic
input generators (``inputs``).  Importing the package loads nothing native;
``paper_2312_05410_gb300.pf`` loads ``libpf.so`` and fails loudly if it is
missing.
"""

__all__ = ["inputs", "pf", "build"]
__version__ = "0.1.0"
