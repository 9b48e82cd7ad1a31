"""B300-native lattice gap map-seeking IK (arXiv 1906.10678).

The compute path is the CUDA library ``libik_b300.so`` behind the C ABI in
``include/ik.h``; ``paper_1906_10678_b300.ik`` is its Python binding.  Import
the binding explicitly (``from paper_1906_10678_b300 import ik``); it raises
ImportError when the library has not been built.
"""
__all__ = ["ik", "build"]
