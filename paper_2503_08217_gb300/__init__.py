"""GB300-native S3R-GS render-and-backprop hot path.

The package is a thin layer over the CUDA library ``libs3r.so`` (built from
``csrc/`` for sm_103a). ``scenegen`` draws the synthetic street corridors;
``binding`` is the ctypes binding of the C ABI; ``render`` holds the
autograd function and the batched multi-camera runner. Submodules are loaded
lazily so that importing the scene generator does not load the CUDA library.
"""

__all__ = ["scenegen", "binding", "render"]
