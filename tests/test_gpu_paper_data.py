"""The paper's data generation (Sec. 5.1, Table 2) on the GPU: the query set
of one material (8x8 footprint centres x 20 footprint sizes x every valid
pair of 8x8-stratified directions, about 3.2 million queries) integrated by
the reference kernel at the paper's 2048 samples (64 x 32 strata), with
sampled queries recomputed by the FP64 oracle on the same sample sequence
(|gpu - oracle| <= 1e-4 |oracle| + 1e-7 per component, as for every
reference-kernel test)."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-4, 1e-7


@pytest.mark.parametrize("material", [0, 81, 464])     # plain, twill 3x3, satin 5x10
def test_paper_query_set_at_2048_spp(fab, material):
    mats = W.paper_materials()
    fab.set_materials(mats)
    q = W.paper_queries(material)
    n = len(q["u"])
    assert abs(n - 3.2e6) / 3.2e6 < 0.05
    rgb, comps = fab.shade_reference(GBuffer.from_numpy(q), 64, 32, 0xDA7A + material, comps=True)
    fab.sync_status()
    c = comps.cpu().numpy()
    assert np.isfinite(c).all() and (c >= 0).all()
    idx = W.sample_indices(n, 48, stream=f"paper-data-{material}")
    want_c, want_rgb = oracle.shade_reference(mats, W.subset(q, idx), 64, 32, 0xDA7A + material, pixel_index=idx)
    err = np.abs(c[idx].astype(np.float64) - want_c) - (RTOL * np.abs(want_c) + ATOL)
    print(f"material {material} (weave {int(mats[material]['pattern'])}): {n} queries; "
          f"worst excess {err.max():.2e}")
    assert (err <= 0).all()
    err = np.abs(rgb.cpu().numpy()[idx].astype(np.float64) - want_rgb) - (RTOL * np.abs(want_rgb) + ATOL)
    assert (err <= 0).all()
