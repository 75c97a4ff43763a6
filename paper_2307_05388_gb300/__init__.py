"""GB300-native cached direct solves for FDFD adjoint inverse design (arXiv 2307.05388).

The compute path is libfdfd.so (CUDA, sm_103a) behind the C ABI in include/fdfd.h;
`fdfd` is its Python binding, `autograd` the torch.autograd.Function built on it and
`autotune` the measured choice of the factorisation's launch parameters and `optimize`
the L-BFGS-B host loop over the design density.
Importing `fdfd` raises when the library has not been built.
"""
__all__ = ["fdfd", "autograd", "autotune", "optimize", "build"]
