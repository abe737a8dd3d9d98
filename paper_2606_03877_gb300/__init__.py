"""GB300 (sm_103a) hot path of MLP-Splatting: sparse volumetric compositing over ray-primitive
interactions, each primitive an ellipsoid-supported MLP (arxiv 2606.03877).

Layout: ``csrc/`` holds the CUDA kernels and the C ABI (``include/mlps.h``), ``_lib`` the ctypes
binding, ``render`` the torch wrapper, ``synth`` the seeded synthetic inputs and ``build`` the
in-tree nvcc build of ``_build/libmlps.so``.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "build", "render", "_lib"]
