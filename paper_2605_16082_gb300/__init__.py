"""GB300-native (sm_103a) implementation of the prismatic DG ocean-model hot path
of arXiv 2605.16082 (SLIM): 3D residual, 3D/2D mode coupling and column-wise
implicit vertical solves, behind the C ABI of include/slim.h.

``slim`` is the ctypes binding of libslim.so; ``build`` compiles it."""
__all__ = ["slim", "build"]
