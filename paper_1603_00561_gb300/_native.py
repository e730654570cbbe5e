"""ctypes declarations of the C ABI in ``include/dsrg.h`` (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdsrg.so")

# dsrg_status_t
OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_NONFINITE, ERR_UNSUPPORTED = range(7)
STATUS_NAMES = {0: "DSRG_OK", 1: "DSRG_ERR_INVALID_ARG", 2: "DSRG_ERR_CUDA", 3: "DSRG_ERR_OOM",
                4: "DSRG_ERR_TIMEOUT", 5: "DSRG_ERR_NONFINITE", 6: "DSRG_ERR_UNSUPPORTED"}
# dsrg_precision_t
PREC = {"fp64": 0, "tf32x3": 1, "bf16x3": 2}
PLAN_HOST_IO = 1
PLAN_GRAD = 2

# every exported symbol of include/dsrg.h
EXPORTS = [
    "dsrg_df_plan", "dsrg_plan_destroy", "dsrg_plan_set_stream", "dsrg_mrpt2_energy",
    "dsrg_ccvv_pair_energies", "dsrg_mrpt2_energy_grad", "dsrg_mrpt2_energy_host",
    "dsrg_plan_sync", "dsrg_plan_last_launch_count", "dsrg_plan_workspace_bytes",
    "dsrg_status_string", "dsrg_plan_last_error",
    "dsrg_batch_plan", "dsrg_batch_destroy", "dsrg_mrpt2_energy_batched", "dsrg_batch_sync",
    "dsrg_batch_launch_count", "dsrg_batch_last_error", "dsrg_ccvv_energy_noalloc",
    "dsrg_plan_autotune", "dsrg_batch_autotune", "dsrg_plan_item_order", "dsrg_batch_item_order",
    "dsrg_plan_time_ccvv", "dsrg_plan_set_item_order", "dsrg_batch_set_item_order",
    "dsrg_plan_selftest_wait_timeout", "dsrg_plan_branch_counts", "dsrg_mrpt2_energy_ext",
    "dsrg_mrpt2_energy_grad_ext", "dsrg_sc_plan_create", "dsrg_sc_plan_destroy", "dsrg_generalized_fock",
    "dsrg_semicanonicalize", "dsrg_sc_last_sweeps", "dsrg_sc_last_error",
    "dsrg_df_mo_transform_work_bytes", "dsrg_df_mo_transform", "dsrg_cd_factors_work_bytes",
    "dsrg_cd_factors", "dsrg_plan_set_shard", "dsrg_shard_pairs", "dsrg_batch_branches",
    "dsrg_batch_set_branches", "dsrg_batch_autotune_branches", "dsrg_tune_cache_get",
    "dsrg_tune_cache_put",
]
# indices of dsrg_plan_branch_counts
NCOUNTERS = 8
COUNTERS = {"ccvv_far": 0, "ccvv_factored": 1, "ccvv_direct": 2, "ccvv_unfactorable": 3,
            "cavv_near": 4, "cavv_unfactorable": 5}


class Sizes(C.Structure):
    _fields_ = [("ncore", C.c_int32), ("nactive", C.c_int32), ("nvirt", C.c_int32),
                ("naux", C.c_int32)]


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load ``libdsrg.so`` and declare the signatures. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1603_00561_gb300.build()")
    lib = C.CDLL(path)
    vp, dp, st = C.c_void_p, C.POINTER(C.c_double), C.c_int
    lib.dsrg_df_plan.argtypes = [C.POINTER(vp), C.POINTER(Sizes), C.c_int, vp, C.c_uint32]
    lib.dsrg_df_plan.restype = st
    lib.dsrg_plan_destroy.argtypes = [vp]
    lib.dsrg_plan_destroy.restype = st
    lib.dsrg_plan_set_stream.argtypes = [vp, vp]
    lib.dsrg_plan_set_stream.restype = st
    lib.dsrg_mrpt2_energy.argtypes = [vp, vp, vp, vp, vp, C.c_double, vp]
    lib.dsrg_mrpt2_energy.restype = st
    lib.dsrg_ccvv_pair_energies.argtypes = [vp, vp, vp, C.c_double, vp]
    lib.dsrg_ccvv_pair_energies.restype = st
    lib.dsrg_mrpt2_energy_grad.argtypes = [vp, vp, vp, vp, vp, C.c_double, vp, vp, vp, vp]
    lib.dsrg_mrpt2_energy_grad.restype = st
    lib.dsrg_mrpt2_energy_ext.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.c_double, vp]
    lib.dsrg_mrpt2_energy_ext.restype = st
    lib.dsrg_mrpt2_energy_grad_ext.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.c_double, vp, vp, vp,
                                               vp]
    lib.dsrg_mrpt2_energy_grad_ext.restype = st
    lib.dsrg_mrpt2_energy_host.argtypes = [vp, vp, vp, vp, vp, C.c_double, vp]
    lib.dsrg_mrpt2_energy_host.restype = st
    lib.dsrg_plan_sync.argtypes = [vp]
    lib.dsrg_plan_sync.restype = st
    lib.dsrg_plan_selftest_wait_timeout.argtypes = [vp]
    lib.dsrg_plan_selftest_wait_timeout.restype = st
    lib.dsrg_sc_plan_create.argtypes = [C.POINTER(vp), C.POINTER(Sizes), vp]
    lib.dsrg_sc_plan_create.restype = st
    lib.dsrg_sc_plan_destroy.argtypes = [vp]
    lib.dsrg_sc_plan_destroy.restype = st
    lib.dsrg_generalized_fock.argtypes = [vp, vp, vp, vp, vp]
    lib.dsrg_generalized_fock.restype = st
    lib.dsrg_semicanonicalize.argtypes = [vp] + [vp] * 12
    lib.dsrg_semicanonicalize.restype = st
    lib.dsrg_sc_last_sweeps.argtypes = [vp]
    lib.dsrg_sc_last_sweeps.restype = C.c_int32
    i32 = C.c_int32
    lib.dsrg_df_mo_transform_work_bytes.argtypes = [i32, i32, i32, i32]
    lib.dsrg_df_mo_transform_work_bytes.restype = C.c_size_t
    lib.dsrg_df_mo_transform.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, i32, i32, vp, vp,
                                         C.c_size_t, vp]
    lib.dsrg_df_mo_transform.restype = st
    lib.dsrg_cd_factors_work_bytes.argtypes = [i32]
    lib.dsrg_cd_factors_work_bytes.restype = C.c_size_t
    lib.dsrg_cd_factors.argtypes = [vp, i32, i32, C.c_double, i32, vp, C.POINTER(i32), vp,
                                    C.c_size_t, vp]
    lib.dsrg_cd_factors.restype = st
    lib.dsrg_plan_set_shard.argtypes = [vp, i32, i32]
    lib.dsrg_plan_set_shard.restype = st
    lib.dsrg_shard_pairs.argtypes = [i32, i32, i32, C.POINTER(i32)]
    lib.dsrg_shard_pairs.restype = i32
    lib.dsrg_sc_last_error.argtypes = [vp]
    lib.dsrg_sc_last_error.restype = C.c_char_p
    lib.dsrg_plan_branch_counts.argtypes = [vp, C.POINTER(C.c_uint64), C.c_int32]
    lib.dsrg_plan_branch_counts.restype = st
    lib.dsrg_plan_last_launch_count.argtypes = [vp]
    lib.dsrg_plan_last_launch_count.restype = C.c_int32
    lib.dsrg_plan_workspace_bytes.argtypes = [vp]
    lib.dsrg_plan_workspace_bytes.restype = C.c_size_t
    lib.dsrg_status_string.argtypes = [C.c_int]
    lib.dsrg_status_string.restype = C.c_char_p
    lib.dsrg_plan_last_error.argtypes = [vp]
    lib.dsrg_plan_last_error.restype = C.c_char_p
    lib.dsrg_batch_plan.argtypes = [C.POINTER(vp), C.c_int32, C.POINTER(Sizes), C.c_int, vp, C.c_uint32]
    lib.dsrg_batch_plan.restype = st
    lib.dsrg_batch_destroy.argtypes = [vp]
    lib.dsrg_batch_destroy.restype = st
    lib.dsrg_mrpt2_energy_batched.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                              C.POINTER(vp), C.POINTER(C.c_double), vp]
    lib.dsrg_mrpt2_energy_batched.restype = st
    lib.dsrg_batch_sync.argtypes = [vp]
    lib.dsrg_batch_sync.restype = st
    lib.dsrg_batch_launch_count.argtypes = [vp]
    lib.dsrg_batch_launch_count.restype = C.c_int32
    lib.dsrg_batch_last_error.argtypes = [vp]
    lib.dsrg_batch_last_error.restype = C.c_char_p
    lib.dsrg_ccvv_energy_noalloc.argtypes = [C.POINTER(Sizes), vp, vp, C.c_double, vp, vp]
    lib.dsrg_ccvv_energy_noalloc.restype = st
    lib.dsrg_plan_autotune.argtypes = [vp, vp, vp, C.c_double, C.c_int32, C.POINTER(C.c_int32)]
    lib.dsrg_plan_autotune.restype = st
    lib.dsrg_batch_autotune.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_double),
                                        C.c_int32, C.POINTER(C.c_int32)]
    lib.dsrg_batch_autotune.restype = st
    lib.dsrg_plan_item_order.argtypes = [vp]
    lib.dsrg_plan_item_order.restype = C.c_int32
    lib.dsrg_batch_item_order.argtypes = [vp]
    lib.dsrg_batch_item_order.restype = C.c_int32
    lib.dsrg_plan_time_ccvv.argtypes = [vp, vp, vp, C.c_double, C.c_int32, C.POINTER(C.c_float)]
    lib.dsrg_plan_time_ccvv.restype = st
    lib.dsrg_plan_set_item_order.argtypes = [vp, C.c_int32]
    lib.dsrg_plan_set_item_order.restype = st
    lib.dsrg_batch_set_item_order.argtypes = [vp, C.c_int32]
    lib.dsrg_batch_set_item_order.restype = st
    lib.dsrg_batch_branches.argtypes = [vp]
    lib.dsrg_batch_branches.restype = C.c_int32
    lib.dsrg_batch_set_branches.argtypes = [vp, C.c_int32]
    lib.dsrg_batch_set_branches.restype = st
    lib.dsrg_batch_autotune_branches.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                                 C.POINTER(vp), C.POINTER(C.c_double), vp,
                                                 C.c_int32, C.POINTER(C.c_int32)]
    lib.dsrg_batch_autotune_branches.restype = st
    lib.dsrg_tune_cache_get.argtypes = [C.c_char_p, C.c_char_p, C.POINTER(C.c_int64)]
    lib.dsrg_tune_cache_get.restype = C.c_int32
    lib.dsrg_tune_cache_put.argtypes = [C.c_char_p, C.c_char_p, C.c_int64]
    lib.dsrg_tune_cache_put.restype = st
    _ = dp
    _lib = lib
    return lib


class DSRGError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {detail}")
