"""GB300 compressed-column transfer and decode (ZipFlow, arXiv 2602.08190).

A thin ctypes binding of ``libzf.so``: every function keeps the name of the
C entry point it calls (see ``include/zf.h``) and only marshals arguments.
Device buffers and streams may come from PyTorch (``tensor.data_ptr()``,
``torch.cuda.Stream.cuda_stream``); the library does everything else.
Importing fails loudly if the library has not been built.
"""
from .binding import *  # noqa: F401,F403
from .binding import __all__  # noqa: F401
