"""GB300 (sm_103a) kernels for products of Householder reflectors.

Rusu, "Approximate Eigenvalue Decompositions of Linear Transformations with a
Few Householder Reflectors" (arXiv 1811.07624): the data-parallel hot path,
applying W = H_1 ... H_h, W^T and S = D W diag(d) W^T D to batches of vectors,
behind the C ABI of ``include/hh.h``.
"""

from ._lib import HHError, header_symbols, lib  # noqa: F401
from .api import Batch, Plan, batch_shapes, tune, tune_clear, tune_get, tune_load, tune_save, tune_set  # noqa: F401
from . import autograd  # noqa: F401
from .autograd import ReflectorTransform  # noqa: F401

__all__ = ["Plan", "Batch", "batch_shapes", "tune", "tune_get", "tune_set", "tune_save",
           "tune_load", "tune_clear", "HHError", "lib", "header_symbols", "autograd", "ReflectorTransform"]
