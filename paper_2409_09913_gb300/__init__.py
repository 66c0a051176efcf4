"""GB300-native extended-RaBitQ search (arXiv 2409.09913) behind a C ABI.

``erq`` is the ctypes binding of liberq.so (include/erq.h); ``autograd`` wraps
the estimated scores and their query gradient in a torch.autograd.Function.
"""
from . import erq  # noqa: F401
from .erq import Index, build_index, encode, rotate, version  # noqa: F401
