"""libcholdiff for GB300: blocked Cholesky factorisation and its forward- and
reverse-mode derivatives (Murray, arXiv:1602.07527, Sec. 4.2) as hand-written
sm_103a CUDA kernels behind a C ABI (include/libcholdiff.h).

The Python layer only marshals arguments; see ``native`` for the binding,
``autograd`` for the torch.autograd.Function and ``serving`` for the
continuous-batching request loop.
"""
from .native import (CholDiffError, chol_fwd, chol_fwd_and_sens, chol_fwd_and_sens_batched,  # noqa: F401
                     chol_fwd_batched, chol_fwd_sens, chol_fwd_sens_batched, chol_jacobian, chol_rev, chol_rev_batched, device_error,
                     launch_count, profile_enable, profile_read, profile_timeline, reserve, version,
                     workspace_size)

__all__ = ["CholDiffError", "chol_fwd", "chol_fwd_and_sens", "chol_fwd_and_sens_batched", "chol_fwd_batched",
           "chol_jacobian", "chol_fwd_sens", "chol_fwd_sens_batched",
           "chol_rev", "chol_rev_batched", "device_error", "launch_count", "profile_enable", "profile_read", "profile_timeline",
           "reserve", "version",
           "workspace_size"]
