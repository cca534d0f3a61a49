"""Spin summations on GB300 (sm_103a): B = alpha * sum_sigma a_sigma pi_sigma(A) + beta * B
for d = 2, 3 and 4 (Springer, Matthews & Bientinesi, arXiv 1705.06661), and the
packing and unpacking of antisymmetric tensors over the permuted indices.

The compute path is the CUDA library behind include/spinsum.h; this package
is its thin Python binding (``_binding``: same names as the C-ABI) plus a
torch-tensor convenience layer (``api``). Importing fails if the library has
not been built; there is no CPU fallback.
"""
from ._binding import (SPINSUM_ADJOINT, SPINSUM_EXPANDED, SPINSUM_F32, SPINSUM_F64, SPINSUM_FACTORIZED,
                       SPINSUM_STATIC_MAX_PROBLEMS, SPINSUM_STRICT, SPINSUM_TMA, LIBRARY_PATH, SpinsumError, spinsum_2d, spinsum_3d, spinsum_4d, spinsum_pack, spinsum_unpack, spinsum_contract, spinsum_2d_host, spinsum_3d_host, spinsum_4d_host, spinsum_batch_static, spinsum_check_status,
                       spinsum_last_error, spinsum_launch_count, spinsum_plan_create, spinsum_plan_describe,
                       spinsum_plan_destroy, spinsum_plan_execute, spinsum_problem, spinsum_version)
from .api import Plan, contract, pack, unpack, spinsum_host, SpinSumFunction, colmajor_empty, colmajor_like, spinsum, spinsum_autograd, to_colmajor

__all__ = [
    "SPINSUM_ADJOINT", "SPINSUM_EXPANDED", "SPINSUM_F32", "SPINSUM_F64", "SPINSUM_FACTORIZED", "SPINSUM_STRICT",
    "SPINSUM_TMA", "SPINSUM_STATIC_MAX_PROBLEMS", "spinsum_batch_static", "LIBRARY_PATH", "SpinsumError", "spinsum_2d", "spinsum_3d", "spinsum_4d", "spinsum_pack", "spinsum_unpack", "spinsum_contract", "contract", "spinsum_2d_host", "spinsum_3d_host", "spinsum_4d_host", "spinsum_check_status", "spinsum_last_error",
    "spinsum_launch_count", "spinsum_plan_create", "spinsum_plan_describe", "spinsum_plan_destroy",
    "spinsum_plan_execute", "spinsum_problem", "spinsum_version", "Plan", "pack", "unpack", "spinsum_host", "SpinSumFunction", "colmajor_empty",
    "colmajor_like", "spinsum", "spinsum_autograd", "to_colmajor",
]
