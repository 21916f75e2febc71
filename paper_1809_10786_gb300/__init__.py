"""GB300-native non-lattice fast SGL Fourier transforms (Wuelker, arXiv:1809.10786).

The transform, its adjoint and its point gradient run in hand-written sm_103a
CUDA kernels behind the C-ABI library ``libsgl.so`` (declared in
``include/sgl.h``).  This package is the thin Python binding: it marshals
arguments and nothing else.  Importing the package loads nothing; the first
transform call loads the library and fails loudly when it is missing.
"""
_BINDING_NAMES = (
    "Plan", "BatchPlan", "SGLError", "num_coeffs", "library_path", "load_library",
    "PREC_FP64", "PREC_FP32_MIXED", "WIN_KB", "WIN_GAUSS", "nfft_error_bound", "choose_cutoff", "choose_params",
)


def __getattr__(name):
    if name in _BINDING_NAMES:
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)
