"""A small disorder-averaging campaign through the GPU path (needs a GB300): the gap ratio averaged
per realization, then over realizations, sits near the GOE value at weak disorder and near the
Poisson value at strong disorder (characterization section: r_GOE = 0.5307, r_Poisson = 2 ln 2 - 1),
and the binned statistics of the campaign equal those recomputed from its bins."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_gap_ratio_limits_through_the_gpu_path():
    import paper_1411_0660_gb300 as g
    from paper_1411_0660_gb300 import campaign as cp

    ctx = g.Context(0)
    data = cp.run_campaign(ctx, [14], [0.5, 6.0], range(24), eps=0.5, nev=30, observable="r", slots=6)
    ctx.close()
    assert data["converged"] == data["requested"]
    weak, dw = cp.mean_stderr(data["bins"][(14, 0.5)])
    strong, ds = cp.mean_stderr(data["bins"][(14, 6.0)])
    r_goe, r_poi = 0.5307, 2 * math.log(2) - 1
    assert abs(weak - r_goe) < max(4 * dw, 0.02)
    assert abs(strong - r_poi) < max(4 * ds, 0.03)
    assert weak - strong > 0.08
    b = np.asarray(data["bins"][(14, 0.5)])
    assert abs(weak - b.mean()) < 1e-15
