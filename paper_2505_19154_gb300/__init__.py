"""GB300-native hot path of FHGS feature splatting (arXiv 2505.19154).

The compute runs in hand-written CUDA kernels for sm_103a behind the C ABI
declared in ``include/fhgs.h`` (``libfhgs.so``).  ``paper_2505_19154_gb300.api``
is the Python binding (ctypes argument marshalling plus a
``torch.autograd.Function``); importing this package does not load the
library.
"""
__all__ = ["api", "synth"]
