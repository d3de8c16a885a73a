"""GB300-native Tensor Train Multiplication (arXiv:2410.19747).

The product Omega = A o B of two tensor trains by the paper's swap-and-contract
sweep, run in hand-written sm_103a CUDA kernels behind the C ABI of
``include/ttm.h`` (libttm.so). This package holds the CUDA sources (``csrc/``),
the in-tree build (``_build.py``) and the ctypes binding (``binding.py``).
"""

from .binding import (  # noqa: F401
    EXPORTED, Handle, TTMError, load_library, library_path, output_capacity,
    ttm_backward, ttm_gemm, ttm_inner, ttm_inner3, ttm_multiply, ttm_multiply_batched,
)
from ._build import build  # noqa: F401
from .autograd import TTMProductLoss, product_loss  # noqa: F401
