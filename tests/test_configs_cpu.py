"""The configuration table without a GPU: the ensemble spec of the batched runs."""
import math

from paper_0710_5912_gb300 import configs


def test_ensemble_spec_matches_the_batched_configuration():
    sizes, params = configs.ensemble_spec()
    assert len(sizes) == 96
    assert sizes.count(128) == sizes.count(256) == sizes.count(512) == 32
    gd = [p[6] for p in params]
    assert math.isclose(gd[0], 1e-4) and math.isclose(gd[-1], 3e-2)
    assert all(b > a for a, b in zip(gd, gd[1:]))                  # log-spaced, increasing
    assert [p[5] for p in params[:4]] == [0.0, 1.0, 0.0, 1.0]
    assert set(configs.CONFIGS) == {"c1_stokes_64_fp64", "c2_inertial_256_fp32", "c3_side_by_side_1024_fp32",
                                    "c4_ensemble_fp32", "c5_inertial_4096_fp32"}
