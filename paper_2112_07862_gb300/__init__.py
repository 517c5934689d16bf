"""GB300 (sm_103a) implementation of generalized-eigenvector manifold graph embedding.

The hot path -- two-hop CSR assembly, Q, eps, mu, A and B (Sec. 4), and the LOBPCG
iteration for the first K generalized eigenpairs of (A, B) -- runs in the CUDA kernels of
libmge.so behind the C ABI in include/mge.h.  ``mge`` is its Python binding.
"""
from . import mge  # noqa: F401
