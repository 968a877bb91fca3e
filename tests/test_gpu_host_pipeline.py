"""fabric_shade_neural_host: a G-buffer in host memory, read directly by the
decoder (mapped page-locked memory) or chunked through three device staging
slots on their own streams, must give exactly the outputs of the
device-resident call (the same kernels on the same points), for ragged
sizes, any chunk size, pinned or pageable memory and every precision; and
it must refuse what it cannot do."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_2406_17782_gb300 import FabricError
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def frame(fab):
    mats = W.frame_materials()
    fab.set_materials(mats)
    fab.set_params(W.decoder_init(), W.encoder_init())
    lat = torch.from_numpy(W.random_latents(len(mats))).cuda()
    host = W.subset(W.frame_gbuffer(), np.arange(5000, 5000 + 300_001))
    return lat, host


# chunk 0 with page-locked buffers takes the direct path (the decoder reads
# and writes host memory itself); a chunk size, or pageable memory, the
# staged three-stream path
@pytest.mark.parametrize("prec,chunk,pin", [("fp16", 0, True), ("fp16", 1000, True), ("fp16", 65536, False),
                                            ("fp16", 0, False), ("bf16", 0, True), ("fp8", 100_000, True),
                                            ("fp8", 0, True), ("fp32", 50_000, True), ("fp32", 0, True)])
def test_host_call_equals_device_call(fab, frame, prec, chunk, pin):
    lat, host = frame
    fab.prepare_neural(lat, prec)
    gd = GBuffer.from_numpy(host)
    want_rgb, want_c = fab.shade_neural_prepared(gd, prec, comps=True)
    gh = GBuffer.from_numpy(host, device="cpu", pin=pin)
    rgb = torch.full((gh.n, 3), float("nan"))
    comps = torch.full((gh.n, 4), float("nan"))
    if pin:
        rgb, comps = rgb.pin_memory(), comps.pin_memory()
    fab.shade_neural_host(gh, prec, out_rgb=rgb, out_comps=comps, chunk_points=chunk)
    fab.sync_status()
    assert torch.equal(rgb, want_rgb.cpu()) and torch.equal(comps, want_c.cpu())


def test_host_call_repeats_and_refuses(fab, frame):
    lat, host = frame
    fab.prepare_neural(lat, "fp16")
    gh = GBuffer.from_numpy(host, device="cpu", pin=True)
    a = torch.empty((gh.n, 3)).pin_memory()
    b = torch.empty((gh.n, 3)).pin_memory()
    fab.shade_neural_host(gh, "fp16", out_rgb=a)
    fab.shade_neural_host(gh, "fp16", out_rgb=b, chunk_points=4096)
    fab.sync_status()
    assert torch.equal(a, b)
    empty = GBuffer.from_numpy(W.subset(host, np.arange(0)), device="cpu")
    fab.shade_neural_host(empty, "fp16", out_rgb=torch.empty((0, 3)))
    with pytest.raises(FabricError):                     # prepared for FP16 only
        fab.shade_neural_host(gh, "bf16", out_rgb=a)
    with pytest.raises(ValueError):                      # a device G-buffer
        fab.shade_neural_host(GBuffer.from_numpy(host), "fp16")
