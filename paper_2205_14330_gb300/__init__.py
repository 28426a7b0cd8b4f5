"""GB300-native differentiable point-splat renderer (Zhang et al. 2022, Sec. 3).

Importing the package loads nothing: ``scenes`` holds the seeded synthetic
input generators, ``pbr`` the ctypes binding of the CUDA library ``libpbr.so``
(which fails loudly when the library is missing).
"""
__all__ = ["scenes", "pbr"]
