"""GB300-native triangle-triangle intersection energy (TTIE).

The hot path (LBVH broad phase, Möller narrow phase, energy / gradient / PSD
Hessian, block-CSR assembly, PCG inexact Newton with line search) runs in the
CUDA kernels of ``libttie.so`` behind the C ABI of ``include/ttie.h``;
``ttie`` is its Python binding.
"""
from .build import build  # noqa: F401
