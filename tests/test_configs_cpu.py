"""The configuration table without a GPU: the ensemble spec of the batched runs."""
import math
import os

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


def _golden_lengths():
    path = os.path.join(os.path.dirname(__file__), "golden", "table_I_lengths.txt")
    out = {}
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, ldv, lvi = line.split()
                out[name] = (float(ldv), float(lvi))
    return out


def test_table_I_sets_reproduce_the_printed_crossover_lengths():
    """Every Table I set's (eta, rho, l) gives the L_DV and L_VI columns the
    paper prints for it (Section VI's definitions), to their 3 digits (0.2%).
    One printed value disagrees with its own row: R022bs's L_VI = 0.00349,
    where eta = 0.339, rho = 22590, l = 0.00156 give 0.003459 (0.9% lower);
    the row's parameters are kept and that entry is held to 1%."""
    gold = _golden_lengths()
    assert set(gold) == set(configs.TABLE_I)
    for name, t in configs.TABLE_I.items():
        ldv = t["l"] * math.sqrt(t["eta"])
        sigma = 2.0 * math.sqrt(2.0) * t["l"] / 3.0
        lvi = math.inf if t["rho"] == 0 else t["eta"] ** 2 / (t["rho"] * sigma)
        g_dv, g_vi = gold[name]
        assert math.isclose(ldv, g_dv, rel_tol=2e-3), (name, ldv, g_dv)
        if math.isinf(g_vi):
            assert math.isinf(lvi), name
        else:
            tol = 1e-2 if name == "R022bs" else 2e-3
            assert math.isclose(lvi, g_vi, rel_tol=tol), (name, lvi, g_vi)


def test_paper_units_fix_tau0_and_the_mesh():
    """In the paper's units (Section IV) G = 1 and tau_0 = (sqrt(2) l)^3 /
    (3 M sigma) = 1 with sigma = 2 sqrt(2) l G / 3; Lambda_y = Ny dx = 1 and
    Lambda_x = Nx dx."""
    for name, t in configs.TABLE_I.items():
        nx, ny, dx, p = configs.paper_units(name)
        sigma = 2.0 * math.sqrt(2.0) * t["l"] * p["a"] / 3.0
        tau0 = (math.sqrt(2.0) * t["l"]) ** 3 / (3.0 * p["M"] * sigma)
        assert math.isclose(tau0, 1.0, rel_tol=1e-12), name
        assert p["a"] == p["b"] == 1.0 and math.isclose(p["kappa"], t["l"] ** 2)
        assert math.isclose(ny * dx, 1.0) and math.isclose(nx * dx, t["Lx"])
        assert (p["eta"], p["rho"], p["gdot"], p["dt"]) == (t["eta"], t["rho"], t["gdot"], t["dt"])
