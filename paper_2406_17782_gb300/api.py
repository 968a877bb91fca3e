"""Python binding of the fabric library: argument marshalling only.

PyTorch supplies device memory and streams; every step of the shading path
runs in the library's CUDA kernels behind the C ABI of include/fabric.h.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _abi
from ._abi import PAPER_STRUCTURES, FabricDatasetOut, FabricGBuffer, FabricMaterial, FabricTrainBatch, check

LATENT = 32


def _stream_handle(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def material_array(materials) -> ctypes.Array:
    """Host array of fabric_material from a structured numpy array with the
    fields of ``workloads.MATERIAL_DTYPE`` (same 84-byte layout)."""
    m = np.ascontiguousarray(np.atleast_1d(materials))
    if m.dtype.itemsize != ctypes.sizeof(FabricMaterial):
        raise ValueError("material records must be 84-byte structured records")
    arr = (FabricMaterial * len(m))()
    ctypes.memmove(arr, m.ctypes.data, m.nbytes)
    return arr


@dataclass
class GBuffer:
    """Device G-buffer (structure of arrays): u, v, radius float32 [n];
    wi, wo float32 [n, 3]; material uint16 bits stored in an int16 [n]."""
    u: torch.Tensor
    v: torch.Tensor
    radius: torch.Tensor
    wi: torch.Tensor
    wo: torch.Tensor
    material: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.u.shape[0])

    @classmethod
    def from_numpy(cls, g: dict, device="cuda", pin: bool = False) -> "GBuffer":
        def conv(a, dt):
            t = torch.from_numpy(np.ascontiguousarray(a).view(dt) if dt == np.int16 else np.ascontiguousarray(a, dt))
            if device == "cpu":
                return t.pin_memory() if pin else t
            return t.to(device)
        return cls(u=conv(g["u"], np.float32), v=conv(g["v"], np.float32), radius=conv(g["radius"], np.float32),
                   wi=conv(g["wi"], np.float32), wo=conv(g["wo"], np.float32),
                   material=conv(np.asarray(g["material"], np.uint16), np.int16))

    def to(self, device, non_blocking=False) -> "GBuffer":
        return GBuffer(*(getattr(self, k).to(device, non_blocking=non_blocking)
                         for k in ("u", "v", "radius", "wi", "wo", "material")))

    def copy_(self, src: "GBuffer", non_blocking=True) -> "GBuffer":
        for k in ("u", "v", "radius", "wi", "wo", "material"):
            getattr(self, k).copy_(getattr(src, k), non_blocking=non_blocking)
        return self

    def nbytes(self) -> int:
        return sum(getattr(self, k).numel() * getattr(self, k).element_size()
                   for k in ("u", "v", "radius", "wi", "wo", "material"))

    def struct(self, host: bool = False) -> FabricGBuffer:
        for k in ("u", "v", "radius", "wi", "wo", "material"):
            t = getattr(self, k)
            if t.is_cuda == host or not t.is_contiguous():
                where = "host" if host else "CUDA"
                raise ValueError(f"G-buffer field {k} must be a contiguous {where} tensor")
        return FabricGBuffer(self.u.data_ptr(), self.v.data_ptr(), self.radius.data_ptr(), self.wi.data_ptr(),
                             self.wo.data_ptr(), self.material.data_ptr(), self.n)


class Fabric:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = _abi.load()
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        h = ctypes.c_void_p()
        check(self.lib.fabric_create(ctypes.byref(h), device))
        self.h = h
        self.n_dec = int(self.lib.fabric_decoder_param_count())
        self.n_enc = int(self.lib.fabric_encoder_param_count())
        self.n_mat = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.fabric_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status):
        check(status, self.h)

    @property
    def sm_count(self) -> int:
        return int(self.lib.fabric_sm_count(self.h))

    def sync_status(self, stream=None):
        self._check(self.lib.fabric_sync_status(self.h, _stream_handle(stream)))

    def set_launch_config(self, decoder_ctas_per_sm: int = 0, decoder_warpgroups: int = 0, reference_lanes: int = 0,
                          decoder_tile_warpgroups: int = 0):
        self._check(self.lib.fabric_set_launch_config(self.h, int(decoder_ctas_per_sm), int(decoder_warpgroups),
                                                      int(reference_lanes)))
        self._check(self.lib.fabric_set_decoder_tile_warpgroups(self.h, int(decoder_tile_warpgroups)))
        self.launch_config = (int(decoder_ctas_per_sm), int(decoder_warpgroups), int(reference_lanes))
        self.tile_warpgroups = int(decoder_tile_warpgroups)

    # ---------------------------------------------------------------- setup
    def set_materials(self, materials):
        arr = material_array(materials)
        self._check(self.lib.fabric_set_materials(self.h, arr, len(arr)))
        self.n_mat = len(arr)

    def set_train_materials(self, materials):
        arr = material_array(materials)
        self._check(self.lib.fabric_set_train_materials(self.h, arr, len(arr)))

    def set_params(self, decoder=None, encoder=None):
        d = None if decoder is None else np.ascontiguousarray(decoder, np.float32)
        e = None if encoder is None else np.ascontiguousarray(encoder, np.float32)
        if d is not None and d.size != self.n_dec:
            raise ValueError(f"decoder needs {self.n_dec} parameters")
        if e is not None and e.size != self.n_enc:
            raise ValueError(f"encoder needs {self.n_enc} parameters")
        self._check(self.lib.fabric_set_params(self.h, None if d is None else d.ctypes.data_as(ctypes.c_void_p),
                                               None if e is None else e.ctypes.data_as(ctypes.c_void_p)))

    def get_params(self):
        d = np.empty(self.n_dec, np.float32)
        e = np.empty(self.n_enc, np.float32)
        self._check(self.lib.fabric_get_params(self.h, d.ctypes.data_as(ctypes.c_void_p),
                                               e.ctypes.data_as(ctypes.c_void_p)))
        return d, e

    def param_tensors(self):
        """Views of the context's FP32 master parameters as CUDA tensors."""
        pd, pe = ctypes.c_void_p(), ctypes.c_void_p()
        self._check(self.lib.fabric_param_pointers(self.h, ctypes.byref(pd), ctypes.byref(pe)))
        return pd.value, pe.value

    def checkpoint_save(self, path: str):
        self._check(self.lib.fabric_checkpoint_save(self.h, path.encode()))

    def checkpoint_load(self, path: str):
        self._check(self.lib.fabric_checkpoint_load(self.h, path.encode()))

    # ----------------------------------------------------------- the path
    def encode_params(self, materials, stream=None) -> torch.Tensor:
        arr = material_array(materials)
        z = torch.empty((len(arr), LATENT), dtype=torch.float32, device=self.device)
        self._check(self.lib.fabric_encode_params(self.h, arr, len(arr), _ptr(z), _stream_handle(stream)))
        return z

    def shade_reference(self, g: GBuffer, spp_x: int, spp_y: int, seed: int, comps: bool = False,
                        out_rgb=None, out_comps=None, stream=None):
        rgb = out_rgb if out_rgb is not None else torch.empty((g.n, 3), dtype=torch.float32, device=self.device)
        cp = out_comps if out_comps is not None else (
            torch.empty((g.n, 4), dtype=torch.float32, device=self.device) if comps else None)
        gs = g.struct()
        self._check(self.lib.fabric_shade_reference(self.h, ctypes.byref(gs), spp_x, spp_y,
                                                    ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), _ptr(rgb), _ptr(cp),
                                                    _stream_handle(stream)))
        return rgb, cp

    def shade_neural(self, g: GBuffer, latents: torch.Tensor, precision: str = "fp16", comps: bool = False,
                     out_rgb=None, out_comps=None, stream=None):
        rgb = out_rgb if out_rgb is not None else torch.empty((g.n, 3), dtype=torch.float32, device=self.device)
        cp = out_comps if out_comps is not None else (
            torch.empty((g.n, 4), dtype=torch.float32, device=self.device) if comps else None)
        lat = latents.contiguous()
        gs = g.struct()
        self._check(self.lib.fabric_shade_neural(self.h, ctypes.byref(gs), _ptr(lat), _abi.PREC[precision],
                                                 _ptr(rgb), _ptr(cp), _stream_handle(stream)))
        return rgb, cp

    def prepare_neural(self, latents: torch.Tensor, precision: str = "fp16", stream=None):
        """Fold the latents and pack the decoder operands (once per edit)."""
        self._prepared_latents = latents.contiguous()
        self._check(self.lib.fabric_prepare_neural(self.h, _ptr(self._prepared_latents), _abi.PREC[precision],
                                                   _stream_handle(stream)))

    def shade_neural_prepared(self, g: GBuffer, precision: str = "fp16", comps: bool = False, out_rgb=None,
                              out_comps=None, stream=None):
        """Draw one G-buffer with the last prepared state (one kernel)."""
        rgb = out_rgb if out_rgb is not None else torch.empty((g.n, 3), dtype=torch.float32, device=self.device)
        cp = out_comps if out_comps is not None else (
            torch.empty((g.n, 4), dtype=torch.float32, device=self.device) if comps else None)
        gs = g.struct()
        self._check(self.lib.fabric_shade_neural_prepared(self.h, ctypes.byref(gs), _abi.PREC[precision],
                                                          _ptr(rgb), _ptr(cp), _stream_handle(stream)))
        return rgb, cp

    def shade_neural_host(self, g: GBuffer, precision: str = "fp16", out_rgb=None, out_comps=None,
                          chunk_points: int = 0, stream=None):
        """Draw a G-buffer held in host memory (CPU tensors, ideally pinned)
        into host outputs, with chunked, overlapped copies and decoder
        launches (fabric_shade_neural_host).  Asynchronous on `stream`."""
        rgb = out_rgb if out_rgb is not None else torch.empty((g.n, 3), dtype=torch.float32).pin_memory()
        for t in (rgb, out_comps):
            if t is not None and (t.is_cuda or not t.is_contiguous()):
                raise ValueError("shade_neural_host writes contiguous host tensors")
        gs = g.struct(host=True)
        self._check(self.lib.fabric_shade_neural_host(self.h, ctypes.byref(gs), _abi.PREC[precision], _ptr(rgb),
                                                      _ptr(out_comps), int(chunk_points), _stream_handle(stream)))
        return rgb, out_comps

    def plan(self, segments) -> "Plan":
        """Batched draw over (GBuffer, rgb_out, comps_out or None) triples."""
        return Plan(self, segments)

    def set_train_loss(self, loss: str = "eq11"):
        """'eq11' (the paper's Eq. 11) or 'rendered' (squared error of the
        components weighted by max(wi.z, 0))."""
        self._check(self.lib.fabric_set_train_loss(self.h, _abi.LOSS[loss]))

    def set_visibility(self, on: bool):
        """The reference's proposed inter-yarn visibility model (V of Eq. 3-5)
        on or off (default off: V = 1)."""
        self._check(self.lib.fabric_set_visibility(self.h, 1 if on else 0))

    def set_train_precision(self, precision: str = "fp32"):
        """'fp32' (SIMT kernels) or 'bf16' (tensor cores) for the decoder's
        training forward and backward."""
        self._check(self.lib.fabric_set_train_precision(self.h, _abi.PREC[precision]))

    def train_step(self, batch: GBuffer, target: torch.Tensor, lr: float, loss_out=None, stream=None):
        loss = loss_out if loss_out is not None else torch.empty((), dtype=torch.float64, device=self.device)
        tb = FabricTrainBatch(batch.struct(), target.contiguous().data_ptr())
        self._check(self.lib.fabric_train_step(self.h, ctypes.byref(tb), ctypes.c_float(lr), _ptr(loss),
                                               _stream_handle(stream)))
        return loss

    def train_steps(self, data: GBuffer, target: torch.Tensor, batch: int, n_steps: int, first_step: int,
                    total_steps: int, lr0: float, lr1: float, loss_out=None, stream=None):
        """n_steps steps of train_step over consecutive batch-sized slices of
        data (wrapping after n // batch steps), with the cosine learning
        rate lr1 + (lr0 - lr1) (1 + cos(pi t / total_steps)) / 2 at step
        t = first_step + k, in one call (fabric_train_steps).  loss_out:
        optional float64 device tensor of at least n_steps entries."""
        if loss_out is not None:
            assert loss_out.dtype == torch.float64 and loss_out.is_contiguous() and loss_out.numel() >= n_steps
        tb = FabricTrainBatch(data.struct(), target.contiguous().data_ptr())
        self._check(self.lib.fabric_train_steps(self.h, ctypes.byref(tb), int(batch), int(n_steps), int(first_step),
                                                int(total_steps), float(lr0), float(lr1),
                                                _ptr(loss_out) if loss_out is not None else None,
                                                _stream_handle(stream)))

    def shuffle_dataset(self, data: GBuffer, target: torch.Tensor, seed: int, out: tuple = None, stream=None):
        """A shuffled copy (GBuffer, target) of a training dataset in one pass
        on the device (fabric_shuffle_dataset): every field of point p is
        point pi(p) of the input, pi the permutation of [0, n) that `seed`
        selects.  out: optional (GBuffer, target) to write into (not
        overlapping the input)."""
        target = target.contiguous()
        if out is None:
            out = (GBuffer(*(torch.empty_like(getattr(data, k)) for k in ("u", "v", "radius", "wi", "wo", "material"))),
                   torch.empty_like(target))
        og, ot = out
        tb = FabricTrainBatch(data.struct(), target.data_ptr())
        do = FabricDatasetOut(*(getattr(og, k).data_ptr() for k in ("u", "v", "radius", "wi", "wo", "material")),
                              ot.data_ptr())
        self._check(self.lib.fabric_shuffle_dataset(self.h, ctypes.byref(tb), ctypes.byref(do),
                                                    ctypes.c_uint64(seed & (2 ** 64 - 1)), _stream_handle(stream)))
        return og, ot

    def error_stats(self, a: torch.Tensor, b: torch.Tensor, weights: torch.Tensor = None, group: int = 1,
                    weight_stride: int = 1, out=None, stream=None) -> torch.Tensor:
        """[sum (w(a-b))^2, sum (w b)^2, max |w(a-b)|] in FP64 on the device;
        w = weights[i // group * weight_stride] (e.g. wi.z per RGB pixel)."""
        out = out if out is not None else torch.empty(3, dtype=torch.float64, device=self.device)
        a = a.contiguous()
        b = b.contiguous()
        self._check(self.lib.fabric_error_stats(self.h, _ptr(a), _ptr(b), a.numel(),
                                                _ptr(weights) if weights is not None else None, int(group),
                                                int(weight_stride), _ptr(out), _stream_handle(stream)))
        return out

    def selftest_mma(self, a: torch.Tensor, b: torch.Tensor, a_in_tmem: bool = False) -> torch.Tensor:
        n, k = b.shape
        d = torch.empty((128, n), dtype=torch.float32, device=self.device)
        self._check(self.lib.fabric_selftest_mma(self.h, _ptr(a.contiguous()), _ptr(b.contiguous()), n, k,
                                                 int(a_in_tmem), _ptr(d), _stream_handle(None)))
        return d

    def selftest_mma_e4m3(self, a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
        """128 x n x k product with E4M3 operands (A in tensor memory)."""
        n, k = b.shape
        d = torch.empty((128, n), dtype=torch.float32, device=self.device)
        self._check(self.lib.fabric_selftest_mma_e4m3(self.h, _ptr(a.contiguous()), _ptr(b.contiguous()), n, k,
                                                      _ptr(d), _stream_handle(None)))
        return d

    def selftest_wait_timeout(self, sleep: bool = False):
        """Launch the bounded-wait self-test (a wait that can never complete
        gives up after about 1 ms); the next sync_status raises TIMEOUT."""
        self._check(self.lib.fabric_selftest_wait_timeout(self.h, int(sleep), _stream_handle(None)))

    def selftest_mma_mn(self, a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
        """128 x n x k BF16 product with both operands MN-major in shared memory."""
        n, k = b.shape
        d = torch.empty((128, n), dtype=torch.float32, device=self.device)
        self._check(self.lib.fabric_selftest_mma_mn(self.h, _ptr(a.contiguous()), _ptr(b.contiguous()), n, k,
                                                    _ptr(d), _stream_handle(None)))
        return d

    # ------------------------------- the paper's decoder structure (Sec. 4.2)
    def paper_set_params(self, width: int, decoder=None, encoder=None, ablation: str = "full"):
        """Parameters of the paper's decoder (width 64 or 128; the full
        structure or one of its ablations, PAPER_STRUCTURES) and its 64-wide
        latent encoder; a new width or structure needs both."""
        a = PAPER_STRUCTURES[ablation]
        nd = int(self.lib.fabric_paper_structure_param_count(int(width), a))
        ne = int(self.lib.fabric_paper_param_count(int(width), 1))
        d = None if decoder is None else np.ascontiguousarray(decoder, np.float32)
        e = None if encoder is None else np.ascontiguousarray(encoder, np.float32)
        if d is not None and d.size != nd:
            raise ValueError(f"paper decoder ({ablation}) of width {width} needs {nd} parameters")
        if e is not None and e.size != ne:
            raise ValueError(f"paper encoder needs {ne} parameters")
        self._check(self.lib.fabric_paper_set_structure(self.h, int(width), a,
                                                        None if d is None else d.ctypes.data_as(ctypes.c_void_p),
                                                        None if e is None else e.ctypes.data_as(ctypes.c_void_p)))
        self.paper_width = int(width)
        self.paper_ablation = ablation

    def _paper_n_dec(self) -> int:
        return int(self.lib.fabric_paper_structure_param_count(self.paper_width,
                                                               PAPER_STRUCTURES[self.paper_ablation]))

    def paper_get_params(self):
        nd = self._paper_n_dec()
        ne = int(self.lib.fabric_paper_param_count(self.paper_width, 1))
        d = np.empty(nd, np.float32)
        e = np.empty(ne, np.float32)
        self._check(self.lib.fabric_paper_get_params(self.h, d.ctypes.data_as(ctypes.c_void_p),
                                                     e.ctypes.data_as(ctypes.c_void_p)))
        return d, e

    def paper_encode_params(self, materials, stream=None) -> torch.Tensor:
        arr = material_array(materials)
        z = torch.empty((len(arr), 64), dtype=torch.float32, device=self.device)
        self._check(self.lib.fabric_paper_encode_params(self.h, arr, len(arr), _ptr(z), _stream_handle(stream)))
        return z

    def paper_prepare(self, latents: torch.Tensor, precision: str = "fp16", stream=None):
        self._paper_latents = latents.contiguous()
        self._check(self.lib.fabric_paper_prepare(self.h, _ptr(self._paper_latents), _abi.PREC[precision],
                                                  _stream_handle(stream)))

    def paper_shade_prepared(self, g: GBuffer, precision: str = "fp16", comps: bool = False, out_rgb=None,
                             out_comps=None, stream=None):
        rgb = out_rgb if out_rgb is not None else torch.empty((g.n, 3), dtype=torch.float32, device=self.device)
        cp = out_comps if out_comps is not None else (
            torch.empty((g.n, 4), dtype=torch.float32, device=self.device) if comps else None)
        gs = g.struct()
        self._check(self.lib.fabric_paper_shade_prepared(self.h, ctypes.byref(gs), _abi.PREC[precision], _ptr(rgb),
                                                         _ptr(cp), _stream_handle(stream)))
        return rgb, cp

    def paper_shade_neural(self, g: GBuffer, latents: torch.Tensor, precision: str = "fp16", comps: bool = False,
                           out_rgb=None, out_comps=None, stream=None):
        rgb = out_rgb if out_rgb is not None else torch.empty((g.n, 3), dtype=torch.float32, device=self.device)
        cp = out_comps if out_comps is not None else (
            torch.empty((g.n, 4), dtype=torch.float32, device=self.device) if comps else None)
        lat = latents.contiguous()
        gs = g.struct()
        self._check(self.lib.fabric_paper_shade_neural(self.h, ctypes.byref(gs), _ptr(lat), _abi.PREC[precision],
                                                       _ptr(rgb), _ptr(cp), _stream_handle(stream)))
        return rgb, cp

    def paper_train_step(self, batch: GBuffer, target: torch.Tensor, lr: float, loss_out=None, stream=None):
        loss = loss_out if loss_out is not None else torch.empty((), dtype=torch.float64, device=self.device)
        tb = FabricTrainBatch(batch.struct(), target.contiguous().data_ptr())
        self._check(self.lib.fabric_paper_train_step(self.h, ctypes.byref(tb), ctypes.c_float(lr), _ptr(loss),
                                                     _stream_handle(stream)))
        return loss

    def paper_gradient(self) -> np.ndarray:
        """The last paper-network training step's gradient [decoder | encoder]."""
        n = self._paper_n_dec() + int(self.lib.fabric_paper_param_count(self.paper_width, 1))
        out = np.empty(n, np.float32)
        self._check(self.lib.fabric_paper_get_gradient(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def paper_shade_fp32(self, g: GBuffer, latents: torch.Tensor, comps: bool = False, stream=None):
        """The paper network (any structure) in FP32 on CUDA cores."""
        rgb = torch.empty((g.n, 3), dtype=torch.float32, device=self.device)
        cp = torch.empty((g.n, 4), dtype=torch.float32, device=self.device) if comps else None
        lat = latents.contiguous()
        gs = g.struct()
        self._check(self.lib.fabric_paper_shade_fp32(self.h, ctypes.byref(gs), _ptr(lat), _ptr(rgb), _ptr(cp),
                                                     _stream_handle(stream)))
        return rgb, cp

    # ---------------------------------------------- autograd building blocks
    def decoder_forward(self, g: GBuffer, latents, dec, stream=None):
        y = torch.empty((g.n, 4), dtype=torch.float32, device=self.device)
        gs = g.struct()
        self._check(self.lib.fabric_decoder_forward(self.h, ctypes.byref(gs), _ptr(latents.contiguous()),
                                                    latents.shape[0], _ptr(dec.contiguous()), _ptr(y),
                                                    _stream_handle(stream)))
        return y

    def decoder_backward(self, g: GBuffer, latents, dec, dy, stream=None):
        ddec = torch.empty(self.n_dec, dtype=torch.float32, device=self.device)
        dlat = torch.empty_like(latents)
        gs = g.struct()
        self._check(self.lib.fabric_decoder_backward(self.h, ctypes.byref(gs), _ptr(latents.contiguous()),
                                                     latents.shape[0], _ptr(dec.contiguous()),
                                                     _ptr(dy.contiguous()), _ptr(ddec), _ptr(dlat),
                                                     _stream_handle(stream)))
        return ddec, dlat

    def encoder_forward(self, feats, enc, stream=None):
        z = torch.empty((feats.shape[0], LATENT), dtype=torch.float32, device=self.device)
        self._check(self.lib.fabric_encoder_forward(self.h, _ptr(feats.contiguous()), feats.shape[0],
                                                    _ptr(enc.contiguous()), _ptr(z), _stream_handle(stream)))
        return z

    def encoder_backward(self, feats, enc, dz, stream=None):
        denc = torch.empty(self.n_enc, dtype=torch.float32, device=self.device)
        self._check(self.lib.fabric_encoder_backward(self.h, _ptr(feats.contiguous()), feats.shape[0],
                                                     _ptr(enc.contiguous()), _ptr(dz.contiguous()), _ptr(denc),
                                                     _stream_handle(stream)))
        return denc


class Plan:
    """Segments (views, ragged tiles) shaded by one persistent launch; the
    tensors stay referenced for the plan's lifetime."""

    def __init__(self, fab: Fabric, segments):
        self.fab = fab
        self.segments = list(segments)
        arr = (_abi.FabricSegment * len(self.segments))()
        for k, (g, rgb, comps) in enumerate(self.segments):
            arr[k] = _abi.FabricSegment(g.struct(), rgb.data_ptr(), comps.data_ptr() if comps is not None else None)
        h = ctypes.c_void_p()
        fab._check(fab.lib.fabric_plan_create(fab.h, arr, len(arr), ctypes.byref(h)))
        self.h = h
        self.points = int(fab.lib.fabric_plan_points(h))
        self.n_segs = len(self.segments)

    def shade(self, precision: str = "fp16", stream=None):
        self.fab._check(self.fab.lib.fabric_plan_shade(self.fab.h, self.h, _abi.PREC[precision],
                                                       _stream_handle(stream)))

    def close(self):
        if getattr(self, "h", None):
            self.fab.lib.fabric_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DecoderFunction(torch.autograd.Function):
    """y = decoder(latents[material], query; dec) with the library's FP32
    forward and deterministic backward kernels."""

    @staticmethod
    def forward(ctx, dec: torch.Tensor, latents: torch.Tensor, fab: Fabric, g: GBuffer):
        ctx.fab, ctx.g = fab, g
        ctx.save_for_backward(dec, latents)
        return fab.decoder_forward(g, latents, dec)

    @staticmethod
    def backward(ctx, dy):
        dec, latents = ctx.saved_tensors
        ddec, dlat = ctx.fab.decoder_backward(ctx.g, latents, dec, dy)
        return ddec, dlat, None, None


class EncoderFunction(torch.autograd.Function):
    """z = encoder(features; enc) with the library's kernels."""

    @staticmethod
    def forward(ctx, enc: torch.Tensor, feats: torch.Tensor, fab: Fabric):
        ctx.fab = fab
        ctx.save_for_backward(enc, feats)
        return fab.encoder_forward(feats, enc)

    @staticmethod
    def backward(ctx, dz):
        enc, feats = ctx.saved_tensors
        return ctx.fab.encoder_backward(feats, enc, dz), None, None
