"""FP64 CPU oracle for the footprint-filtered woven-fabric reflectance and its
neural decoder (Chen, Wang and Wang, "Real-time Neural Woven Fabric Rendering",
SIGGRAPH 2024).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and imports nothing from it.

* :mod:`oracle.fabric_oracle` (C, FP64): the shading model of Eq. 1-2, the
  aggregation of Eq. 3-5 split into the components of Eq. 7 and recombined by
  Eq. 8, the stratified footprint estimator and a whole-period quadrature.
* :mod:`oracle.mlp` (numpy, FP64): the query encoding, the decoder and encoder
  forward/backward passes, the loss of Eq. 9-11, Adam and BF16 / E4M3 rounding.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fabric_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAT_STRIDE = 21


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, no contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            d, u32, u64, i64 = ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64
            L.ora_mix64.restype = u64
            L.ora_mix64.argtypes = [u64]
            L.ora_pattern_info.restype = ctypes.c_int
            L.ora_pattern_info.argtypes = [ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int),
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.ora_frame.restype = ctypes.c_int
            L.ora_frame.argtypes = [ctypes.c_void_p, u32, u32, ctypes.c_void_p, ctypes.c_void_p]
            L.ora_sggx_D.restype = d
            L.ora_sggx_D.argtypes = [d, ctypes.c_void_p, ctypes.c_void_p]
            L.ora_sggx_sigma.restype = d
            L.ora_sggx_sigma.argtypes = [d, ctypes.c_void_p, ctypes.c_void_p]
            L.ora_point_eval.restype = None
            L.ora_point_eval.argtypes = [ctypes.c_void_p, u32, u32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]
            L.ora_point_contrib.restype = None
            L.ora_point_contrib.argtypes = [ctypes.c_void_p, u32, u32, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]
            L.ora_sample_position.restype = None
            L.ora_sample_position.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                              i64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              u64, P(u32), P(u32)]
            L.ora_shade_reference.restype = None
            L.ora_shade_reference.argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 6 + [
                i64, ctypes.c_int, ctypes.c_int, u64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                ctypes.c_void_p]
            L.ora_period_quadrature.restype = None
            L.ora_period_quadrature.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
            L.ora_shade_reference_vis.restype = None
            L.ora_shade_reference_vis.argtypes = L.ora_shade_reference.argtypes + [ctypes.c_int, d,
                                                                                  ctypes.c_void_p]
            L.ora_height.restype = d
            L.ora_height.argtypes = [ctypes.c_void_p, u32, u32]
            L.ora_height_max.restype = d
            L.ora_height_max.argtypes = [ctypes.c_void_p]
            L.ora_visible.restype = ctypes.c_int
            L.ora_visible.argtypes = [ctypes.c_void_p, u32, u32, ctypes.c_void_p, d, P(ctypes.c_int)]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# material records
# --------------------------------------------------------------------------
def material_rows(materials: np.ndarray) -> np.ndarray:
    """Flatten a structured material array (float32 fields, see
    ``workloads.MATERIAL_DTYPE``) into the oracle's 21-double rows.  The
    float32 -> float64 conversion is exact, so both paths see the same values."""
    m = np.atleast_1d(materials)
    rows = np.zeros((len(m), MAT_STRIDE), np.float64)
    rows[:, 0] = m["pattern"].astype(np.float64)
    rows[:, 1] = m["twist_deg"].astype(np.float64)
    rows[:, 2] = m["incl_deg"].astype(np.float64)
    rows[:, 3:5] = m["alpha"].astype(np.float64)
    rows[:, 5:7] = m["beta"].astype(np.float64)
    rows[:, 7:10] = m["kd"][:, 0].astype(np.float64)
    rows[:, 10:13] = m["kd"][:, 1].astype(np.float64)
    rows[:, 13:16] = m["ks"][:, 0].astype(np.float64)
    rows[:, 16:19] = m["ks"][:, 1].astype(np.float64)
    rows[:, 19] = m["gap"].astype(np.float64)
    rows[:, 20] = m["w_blend"].astype(np.float64)
    return np.ascontiguousarray(rows)


# --------------------------------------------------------------------------
# thin wrappers
# --------------------------------------------------------------------------
def mix64(z: int) -> int:
    return int(lib().ora_mix64(ctypes.c_uint64(z & 0xFFFFFFFFFFFFFFFF)))


def pattern_info(pid: int):
    R, C = ctypes.c_int(), ctypes.c_int()
    bits = np.zeros(256, np.uint8)
    rl = np.zeros(256, np.uint8)
    ro = np.zeros(256, np.uint8)
    if lib().ora_pattern_info(pid, ctypes.byref(R), ctypes.byref(C), _ptr(bits), _ptr(rl), _ptr(ro)) != 0:
        raise ValueError(f"unknown pattern {pid}")
    r, c = R.value, C.value
    return (bits.reshape(16, 16)[:r, :c].copy(), rl.reshape(16, 16)[:r, :c].copy(),
            ro.reshape(16, 16)[:r, :c].copy())


def frame(mat_row: np.ndarray, pu: int, pv: int):
    n = np.zeros(3)
    t = np.zeros(3)
    m = np.ascontiguousarray(mat_row, np.float64)
    yarn = lib().ora_frame(_ptr(m), pu & 0xFFFFFFFF, pv & 0xFFFFFFFF, _ptr(n), _ptr(t))
    return yarn, n, t


def sggx_D(alpha: float, t, h) -> float:
    t = np.ascontiguousarray(t, np.float64)
    h = np.ascontiguousarray(h, np.float64)
    return float(lib().ora_sggx_D(alpha, _ptr(t), _ptr(h)))


def sggx_sigma(alpha: float, t, w) -> float:
    t = np.ascontiguousarray(t, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    return float(lib().ora_sggx_sigma(alpha, _ptr(t), _ptr(w)))


def point_eval(mat_row, pu: int, pv: int, wi, wo) -> np.ndarray:
    m = np.ascontiguousarray(mat_row, np.float64)
    wi = np.ascontiguousarray(wi, np.float64)
    wo = np.ascontiguousarray(wo, np.float64)
    out = np.zeros(4)
    lib().ora_point_eval(_ptr(m), pu & 0xFFFFFFFF, pv & 0xFFFFFFFF, _ptr(wi), _ptr(wo), _ptr(out))
    return out


def point_contrib(mat_row, pu: int, pv: int, wi, wo) -> np.ndarray:
    m = np.ascontiguousarray(mat_row, np.float64)
    wi = np.ascontiguousarray(wi, np.float64)
    wo = np.ascontiguousarray(wo, np.float64)
    out = np.zeros(5)
    lib().ora_point_contrib(_ptr(m), pu & 0xFFFFFFFF, pv & 0xFFFFFFFF, _ptr(wi), _ptr(wo), _ptr(out))
    return out


def sample_position(u, v, r, pixel, k, nx, ny, seed):
    pu, pv = ctypes.c_uint32(), ctypes.c_uint32()
    lib().ora_sample_position(float(np.float32(u)), float(np.float32(v)), float(np.float32(r)),
                              int(pixel), int(k), int(nx), int(ny),
                              ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF),
                              ctypes.byref(pu), ctypes.byref(pv))
    return pu.value, pv.value


def shade_reference(materials, gbuf: dict, spp_x: int, spp_y: int, seed: int, nthreads: int = 0,
                    pixel_index=None, visibility: bool = False, eps: float = 1e-6):
    """Stratified footprint estimator over a G-buffer (dict of numpy arrays
    u, v, radius float32 [n]; wi, wo float32 [n,3]; material uint16 [n]).
    `pixel_index` (int64 [n]) gives each point's index in the full buffer when
    the arrays are a subset of it.  Returns (comps [n,4], rgb [n,3]) in FP64;
    with `visibility` (the proposed inter-yarn visibility model) also
    ambiguous [n] bool: points where some march came within `eps` of the
    surface without a clear occluder."""
    rows = material_rows(materials)
    u = np.ascontiguousarray(gbuf["u"], np.float32)
    v = np.ascontiguousarray(gbuf["v"], np.float32)
    r = np.ascontiguousarray(gbuf["radius"], np.float32)
    wi = np.ascontiguousarray(gbuf["wi"], np.float32)
    wo = np.ascontiguousarray(gbuf["wo"], np.float32)
    mat = np.ascontiguousarray(gbuf["material"], np.uint16)
    n = len(u)
    comps = np.zeros((n, 4))
    rgb = np.zeros((n, 3))
    idx = None if pixel_index is None else np.ascontiguousarray(pixel_index, np.int64)
    if not visibility:
        lib().ora_shade_reference(_ptr(rows), len(rows), _ptr(u), _ptr(v), _ptr(r), _ptr(wi), _ptr(wo),
                                  _ptr(mat), n, spp_x, spp_y, ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF),
                                  _ptr(comps), _ptr(rgb), int(nthreads), None if idx is None else _ptr(idx))
        return comps, rgb
    amb = np.zeros(n, np.uint8)
    lib().ora_shade_reference_vis(_ptr(rows), len(rows), _ptr(u), _ptr(v), _ptr(r), _ptr(wi), _ptr(wo),
                                  _ptr(mat), n, spp_x, spp_y, ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF),
                                  _ptr(comps), _ptr(rgb), int(nthreads), None if idx is None else _ptr(idx),
                                  1, float(eps), _ptr(amb))
    return comps, rgb, amb.astype(bool)


def height(mat_row, pu: int, pv: int) -> float:
    """Height of the proposed visibility model's surface at a fixed-point
    position (repeat units)."""
    m = np.ascontiguousarray(mat_row, np.float64)
    return float(lib().ora_height(_ptr(m), pu & 0xFFFFFFFF, pv & 0xFFFFFFFF))


def height_max(mat_row) -> float:
    m = np.ascontiguousarray(mat_row, np.float64)
    return float(lib().ora_height_max(_ptr(m)))


def visible(mat_row, pu: int, pv: int, w, eps: float = 1e-6):
    """(V, ambiguous) of the proposed visibility model from the surface point
    at (pu, pv) along w."""
    m = np.ascontiguousarray(mat_row, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    a = ctypes.c_int()
    v = lib().ora_visible(_ptr(m), pu & 0xFFFFFFFF, pv & 0xFFFFFFFF, _ptr(w), float(eps), ctypes.byref(a))
    return int(v), bool(a.value)


def period_quadrature(mat_row, wi, wo, grid: int, nthreads: int = 0) -> np.ndarray:
    """Whole-period average of the Eq. 3 numerators and of A (Eq. 5) by
    midpoint quadrature; returns [Cw, Cf, Sw, Sf, A] averages."""
    m = np.ascontiguousarray(mat_row, np.float64)
    wi = np.ascontiguousarray(wi, np.float64)
    wo = np.ascontiguousarray(wo, np.float64)
    out = np.zeros(5)
    lib().ora_period_quadrature(_ptr(m), _ptr(wi), _ptr(wo), int(grid), _ptr(out), int(nthreads))
    return out


from . import mlp  # noqa: E402,F401
