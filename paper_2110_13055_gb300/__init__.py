"""GB300-native pore-scale capacitive-deionization solver (arXiv 2110.13055).

The product is the CUDA library ``libcdi.so`` behind the C ABI of
``include/cdi.h``; ``cdi`` is its Python binding and ``inputs`` holds the
seeded geometry generators.
"""
from . import cdi, inputs  # noqa: F401

__all__ = ["inputs", "cdi"]
