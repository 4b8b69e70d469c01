"""GB300-native Pinv-Recon: explicit Tikhonov pseudoinverse MRI reconstruction.

The compute path lives in libpinv.so (CUDA, sm_103a) behind the C ABI of
include/pinv.h; `Plan` is its torch front end. Importing the package does not
load the library; creating a Plan does, and fails loudly if it is missing.
"""
from ._lib import (C64, C128, EXPORT_CHOL, EXPORT_GINV, EXPORT_GRAM, EXPORT_RECON, FP64,  # noqa: F401
                   LAMBDA_ABS, LAMBDA_REL_MEAN_DIAG, MIXED_BF16X3, MIXED_BF16X6, RECON_AUTO,
                   RECON_NONE, RECON_STORE, PinvError)


def __getattr__(name):
    if name == "Plan":
        from .plan import Plan
        return Plan
    raise AttributeError(name)
