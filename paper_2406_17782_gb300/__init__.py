"""GB300 (sm_103a) footprint-filtered woven-fabric reflectance: supersampled
reference integrator, tensor-core neural decoder and its training kernels,
behind the C ABI of include/fabric.h (Chen, Wang and Wang, "Real-time Neural
Woven Fabric Rendering", SIGGRAPH 2024).
"""
from ._abi import FabricError, header_functions, load  # noqa: F401


def __getattr__(name):
    # the torch-facing binding is imported lazily so that the ABI module can be
    # inspected on machines without a GPU
    if name in ("Fabric", "GBuffer", "DecoderFunction", "EncoderFunction", "material_array"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
