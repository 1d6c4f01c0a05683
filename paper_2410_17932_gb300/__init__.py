"""GB300-native tile-based Gaussian-splatting rasterizer for VR-Splatting's periphery.

The compute path is the C-ABI library ``libvrs.so`` (hand-written CUDA for
sm_103a); ``_lib`` marshals its arguments and ``render`` wraps it for PyTorch
tensors.  Importing this package does not load the library; the first call
into it does, and fails loudly if it has not been built.
"""
__all__ = ["inputs"]
