"""Host logic of the workload generators: seeded determinism and the view
sizes table that the SSIM-only bench uses without building a scene."""
import numpy as np
import pytest

from paper_2606_11390_gb300 import scenes


@pytest.mark.parametrize("name", sorted(scenes.NAMED))
def test_view_sizes_table_matches_the_generators(name):
    s = scenes.make(name, N=1000)
    np.testing.assert_array_equal(s["sizes"], scenes.make_sizes(name))


def test_generators_are_seeded():
    a, b = scenes.make("tiny", N=500), scenes.make("tiny", N=500)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "target"):
        np.testing.assert_array_equal(a[k], b[k])
