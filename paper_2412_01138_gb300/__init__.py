"""GB300-native Parareal exponential-integrator Q1 FEM (Huang & Xu, arXiv 2412.01138).

The compute path lives in the CUDA shared library ``libpe`` (sources under
``csrc/``, C-ABI declared in ``include/pe.h``); ``pe`` is its thin ctypes
binding.  ``inputs`` generates seeded problem descriptors.  Importing this
package loads nothing; ``from paper_2412_01138_gb300 import pe`` loads the
library and fails loudly when it has not been built.
"""
__all__ = ["inputs", "pe"]
