"""GB300-native irregular wavefront propagation (IWPP): morphological
reconstruction by dilation and the Euclidean distance transform by
nearest-feature propagation (Teodoro et al., arXiv:1209.3314).

The computation lives in the CUDA library ``libiwpp`` (C ABI in
``include/iwpp.h``); ``binding`` is a ctypes layer over it and ``synth``
produces seeded synthetic inputs.  Importing the package loads nothing;
``Context`` loads the library and fails loudly if it is not built.
"""
from .binding import Context, IWPPError, load_library  # noqa: F401

__all__ = ["Context", "IWPPError", "load_library"]
