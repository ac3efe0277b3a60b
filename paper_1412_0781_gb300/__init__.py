"""GB300-native fast Fourier-Bessel steerable PCA (Zhao, Shkolnisky & Singer).

The computation lives in the C-ABI library ``libffb.so`` (``include/ffb.h``),
built from ``csrc/`` for sm_103a; ``ffb`` is its ctypes binding and
``autograd`` wraps the expansion and its adjoint as torch autograd functions.
"""
from .ffb import Plan, Group, FFBError, load, PRECISION, DENOISE  # noqa: F401

__all__ = ["Plan", "Group", "FFBError", "load", "PRECISION", "DENOISE"]
