"""csx: clustered parametric CMB component separation on NVIDIA B300 (sm_103a).

The hot path of arxiv 2604.08463 (mixing matrix, clustered spectral likelihood, its adjoint
gradient, the batched on-device fit and the W.d reconstruction with residual diagnostics) runs in
hand-written CUDA kernels behind the C ABI of include/csx.h; `csx` is its Python binding.
"""
from . import csx  # noqa: F401
from .csx import (CsxError, Model, Sky, SpectralLikelihood, build_cells, fit_batch,  # noqa: F401
                  mixing, reconstruct, select, spectral_grad, spectral_like)
