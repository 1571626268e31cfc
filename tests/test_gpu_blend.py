"""The blend-localisation scenes (n spheres combined by sharp, compact smooth
or classical smooth unions): traced frames against the oracle, and the A-buffer
sizes that make the difference (a classical blend's volumes of interest cover
the scene, so every tile lists every sphere)."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg
from gpu_util import gpu_lists, parity, render

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [8, 16])
@pytest.mark.parametrize("blend,k", [("sharp", 0.0), ("compact", 0.06), ("compact", 0.12), ("classical", 0.06)])
def test_blend_scenes_parity(stlib, orc, cuda, n, blend, k):
    s = sg.blend_spheres(n, blend, k)
    cam = sg.default_camera(240, 160)
    g = render(stlib, s, cam)
    info = parity(orc, s, cam, g, orc.trace(s, cam))
    assert info["n_hit"] > 1000
    lists = gpu_lists(stlib, s, cam, 16)
    counts = np.diff(lists["off"].astype(np.int64))
    if blend == "classical":
        assert np.all(counts == n)
    else:
        assert counts.mean() < 0.5 * n
