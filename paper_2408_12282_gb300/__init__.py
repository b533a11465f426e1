"""GB300-native differentiable OLAT render of relightable 3D Gaussians with a
learned subsurface-scattering residual (arXiv 2408.12282).

The compute path is libsssgs.so (CUDA, sm_103a) behind the C ABI in
include/sssgs.h; `binding` marshals torch tensors into it and `pipeline`
sequences the calls. Importing the package does not load the library;
`load_library()` does, and raises if it has not been built.
"""
from .binding import SSSGSError, load_library, library_path  # noqa: F401

__all__ = ["SSSGSError", "load_library", "library_path"]
