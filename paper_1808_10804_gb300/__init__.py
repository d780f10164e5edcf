"""Block-sparse U(1)-symmetric tensor contraction and CTMRG moves on GB300.

The computation lives in the CUDA library libbst.so (C ABI: include/bst.h);
``bst`` is its thin ctypes binding.
"""
from . import bst  # noqa: F401
from .bst import Context, Env, Layout, Leg, BstError  # noqa: F401
