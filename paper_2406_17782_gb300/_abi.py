"""ctypes declarations of the C ABI in include/fabric.h.

Loading fails loudly when the compiled library is missing: there is no CPU
fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
HEADER = os.path.join(ROOT, "include", "fabric.h")
LIB_PATH = os.path.join(PKG, "_build", "libfabric.so")

FABRIC_OK = 0
STATUS_NAMES = {0: "FABRIC_OK", 1: "FABRIC_ERR_INVALID_ARG", 2: "FABRIC_ERR_CUDA", 3: "FABRIC_ERR_OOM",
                4: "FABRIC_ERR_TIMEOUT", 5: "FABRIC_ERR_IO", 6: "FABRIC_ERR_UNSUPPORTED", 7: "FABRIC_ERR_DEVICE"}
PREC = {"fp32": 0, "bf16": 1, "fp8": 2, "fp16": 3}
LOSS = {"eq11": 0, "rendered": 1}
PAPER_STRUCTURES = {"full": 0, "no_oneblob": 1, "no_fusion": 2}   # the paper decoder and its two ablations


class FabricMaterial(ctypes.Structure):
    _fields_ = [("pattern_id", ctypes.c_int32), ("twist_deg", ctypes.c_float), ("incl_deg", ctypes.c_float),
                ("alpha", ctypes.c_float * 2), ("beta", ctypes.c_float * 2),
                ("kd", (ctypes.c_float * 3) * 2), ("ks", (ctypes.c_float * 3) * 2),
                ("gap", ctypes.c_float), ("w_blend", ctypes.c_float)]


class FabricGBuffer(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("radius", ctypes.c_void_p),
                ("wi", ctypes.c_void_p), ("wo", ctypes.c_void_p), ("material", ctypes.c_void_p),
                ("n", ctypes.c_int64)]


class FabricTrainBatch(ctypes.Structure):
    _fields_ = [("queries", FabricGBuffer), ("target", ctypes.c_void_p)]


class FabricDatasetOut(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("u", "v", "radius", "wi", "wo", "material", "target")]


class FabricSegment(ctypes.Structure):
    _fields_ = [("g", FabricGBuffer), ("rgb_dev", ctypes.c_void_p), ("comps_dev", ctypes.c_void_p)]


class FabricError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def header_functions() -> list[str]:
    """Names of every function the public header declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fabric_\w+)\s*\(", text)))


def load(path: str | None = None):
    """Load libfabric.so (built in-tree by ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libfabric.so not found at {path}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    P, vp, i32, i64, u64 = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
    st = ctypes.c_int
    sig = {
        "fabric_create": (st, [P(vp), i32]),
        "fabric_destroy": (None, [vp]),
        "fabric_last_error": (ctypes.c_char_p, [vp]),
        "fabric_status_string": (ctypes.c_char_p, [st]),
        "fabric_sync_status": (st, [vp, vp]),
        "fabric_sm_count": (i32, [vp]),
        "fabric_set_launch_config": (st, [vp, i32, i32, i32]),
        "fabric_set_decoder_tile_warpgroups": (st, [vp, i32]),
        "fabric_set_train_loss": (st, [vp, i32]),
        "fabric_set_train_precision": (st, [vp, i32]),
        "fabric_shade_neural_host": (st, [vp, vp, i32, vp, vp, i64, vp]),
        "fabric_set_materials": (st, [vp, vp, i32]),
        "fabric_set_train_materials": (st, [vp, vp, i32]),
        "fabric_decoder_param_count": (i64, []),
        "fabric_encoder_param_count": (i64, []),
        "fabric_set_params": (st, [vp, vp, vp]),
        "fabric_get_params": (st, [vp, vp, vp]),
        "fabric_param_pointers": (st, [vp, P(vp), P(vp)]),
        "fabric_checkpoint_save": (st, [vp, ctypes.c_char_p]),
        "fabric_checkpoint_load": (st, [vp, ctypes.c_char_p]),
        "fabric_encode_params": (st, [vp, vp, i32, vp, vp]),
        "fabric_shade_reference": (st, [vp, P(FabricGBuffer), i32, i32, u64, vp, vp, vp]),
        "fabric_shade_neural": (st, [vp, P(FabricGBuffer), vp, st, vp, vp, vp]),
        "fabric_prepare_neural": (st, [vp, vp, st, vp]),
        "fabric_shade_neural_prepared": (st, [vp, P(FabricGBuffer), st, vp, vp, vp]),
        "fabric_train_step": (st, [vp, P(FabricTrainBatch), ctypes.c_float, vp, vp]),
        "fabric_shuffle_dataset": (st, [vp, P(FabricTrainBatch), P(FabricDatasetOut), u64, vp]),
        "fabric_train_steps": (st, [vp, P(FabricTrainBatch), i64, i32, i64, i64, ctypes.c_double, ctypes.c_double,
                                    vp, vp]),
        "fabric_decoder_forward": (st, [vp, P(FabricGBuffer), vp, i32, vp, vp, vp]),
        "fabric_decoder_backward": (st, [vp, P(FabricGBuffer), vp, i32, vp, vp, vp, vp, vp]),
        "fabric_encoder_forward": (st, [vp, vp, i32, vp, vp, vp]),
        "fabric_encoder_backward": (st, [vp, vp, i32, vp, vp, vp, vp]),
        "fabric_error_stats": (st, [vp, vp, vp, i64, vp, i32, i32, vp, vp]),
        "fabric_selftest_mma": (st, [vp, vp, vp, i32, i32, i32, vp, vp]),
        "fabric_selftest_mma_e4m3": (st, [vp, vp, vp, i32, i32, vp, vp]),
        "fabric_selftest_mma_mn": (st, [vp, vp, vp, i32, i32, vp, vp]),
        "fabric_selftest_wait_timeout": (st, [vp, i32, vp]),
        "fabric_shade_neural_noalloc": (st, [vp, P(FabricGBuffer), vp, st, vp, vp, vp]),
        "fabric_plan_create": (st, [vp, vp, i32, P(vp)]),
        "fabric_plan_shade": (st, [vp, vp, st, vp]),
        "fabric_plan_points": (i64, [vp]),
        "fabric_plan_destroy": (None, [vp]),
        "fabric_paper_param_count": (i64, [i32, i32]),
        "fabric_paper_set_params": (st, [vp, i32, vp, vp]),
        "fabric_paper_get_params": (st, [vp, vp, vp]),
        "fabric_paper_prepare": (st, [vp, vp, st, vp]),
        "fabric_paper_shade_prepared": (st, [vp, P(FabricGBuffer), st, vp, vp, vp]),
        "fabric_paper_shade_neural": (st, [vp, P(FabricGBuffer), vp, st, vp, vp, vp]),
        "fabric_paper_encode_params": (st, [vp, vp, i32, vp, vp]),
        "fabric_paper_train_step": (st, [vp, P(FabricTrainBatch), ctypes.c_float, vp, vp]),
        "fabric_paper_get_gradient": (st, [vp, vp]),
        "fabric_set_visibility": (st, [vp, i32]),
        "fabric_paper_structure_param_count": (i64, [i32, i32]),
        "fabric_paper_set_structure": (st, [vp, i32, i32, vp, vp]),
        "fabric_paper_shade_fp32": (st, [vp, P(FabricGBuffer), vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        if not hasattr(L, name):
            continue
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status: int, handle=None):
    if status != FABRIC_OK:
        msg = ""
        if handle is not None and _lib is not None:
            raw = _lib.fabric_last_error(handle)
            msg = raw.decode() if raw else ""
        raise FabricError(status, msg)
