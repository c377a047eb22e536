"""The five benchmark configurations of the sheared model-H step, as data.

Each entry gives the grid, precision, model parameters (a, b, kappa, M, eta,
rho, gdot, dt), the quench (seeded +-amp uniform noise on phi = 0, Section VII)
and the step count; ``make`` builds the Grid (or the Ensemble for the batched
configuration) ready to step.  Lengths and times are in grid units (dx = 1).
"""
from __future__ import annotations

from . import SHF_FP32, SHF_FP64, Ensemble, Grid

UNIT = dict(a=1.0, b=1.0, kappa=1.0, M=1.0)

CONFIGS = {
    "c1_stokes_64_fp64": dict(nx=64, ny=64, precision=SHF_FP64, params=dict(UNIT, eta=1.0, rho=0.0, gdot=0.01,
                                                                            dt=0.005),
                              seed=0, amp=0.01, steps=2000),
    "c2_inertial_256_fp32": dict(nx=256, ny=256, precision=SHF_FP32,
                                 params=dict(UNIT, eta=1.0, rho=1.0, gdot=0.003, dt=0.005),
                                 seed=0, amp=0.01, steps=20000, gdot_values=(0.001, 0.003, 0.01)),
    "c3_side_by_side_1024_fp32": dict(nx=1024, ny=1024, precision=SHF_FP32,
                                      params=dict(UNIT, eta=1.0, rho=1.0, gdot=0.003, dt=0.005),
                                      seed=0, amp=0.01, steps=100000, rho_values=(0.0, 0.1, 1.0)),
    "c4_ensemble_fp32": dict(runs=96, precision=SHF_FP32, seed=0, amp=0.01, steps=100),
    "c5_inertial_4096_fp32": dict(nx=4096, ny=4096, precision=SHF_FP32,
                                  params=dict(UNIT, eta=1.0, rho=1.0, gdot=0.001, dt=0.005),
                                  seed=0, amp=0.01, steps=200000),
}


# The paper's run parameters (Table I): eta, rho, interface width l, gdot,
# Lambda_x, Nx, Ny, dt, in the paper's units (Section IV: lengths in units of
# Lambda_y, stresses of G, times of tau_0).  Sets of Table Ia/Ib are unsheared
# (512^2); Ic/Id are sheared with Lambda_x = 2 (1024 x 512).
TABLE_I = {
    # (a) zero shear, viscous to inertial
    "R028u": dict(eta=0.111, rho=136.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.008),
    "R022u": dict(eta=0.196, rho=2510.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.008),
    "R029u": dict(eta=0.0467, rho=893.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.008),
    "R020u": dict(eta=0.0785, rho=16180.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.008),
    "R030u": dict(eta=0.0122, rho=6250.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.008),
    "R019u": dict(eta=0.00876, rho=32814.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.008),
    "R032u": dict(eta=0.00391, rho=20067.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.008),
    # (b) zero shear, diffusive to viscous (no inertia)
    "DV1u": dict(eta=1000.0, rho=0.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.016),
    "DV2u": dict(eta=100.0, rho=0.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.016),
    "DV3u": dict(eta=10.0, rho=0.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.016),
    "DV4u": dict(eta=1.0, rho=0.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.016),
    "DV5u": dict(eta=0.3, rho=0.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.016),
    "DV6u": dict(eta=0.1, rho=0.0, l=0.00156, gdot=0.0, Lx=1.0, nx=512, ny=512, dt=0.016),
    # (c) applied shear, with inertia
    "R028s": dict(eta=0.111, rho=136.0, l=0.00156, gdot=0.0765, Lx=2.0, nx=1024, ny=512, dt=0.008),
    "R028bs": dict(eta=0.444, rho=8704.0, l=0.00156, gdot=0.0765, Lx=2.0, nx=1024, ny=512, dt=0.008),
    "R022s": dict(eta=0.196, rho=2510.0, l=0.00156, gdot=0.0205, Lx=2.0, nx=1024, ny=512, dt=0.008),
    "R022bs": dict(eta=0.339, rho=22590.0, l=0.00156, gdot=0.0355, Lx=2.0, nx=1024, ny=512, dt=0.008),
    "R029s": dict(eta=0.0467, rho=893.0, l=0.00156, gdot=0.0341, Lx=2.0, nx=1024, ny=512, dt=0.008),
    "R029bs": dict(eta=0.0809, rho=8037.0, l=0.00156, gdot=0.0591, Lx=2.0, nx=1024, ny=512, dt=0.008),
    "R020s": dict(eta=0.0785, rho=16180.0, l=0.00156, gdot=0.0256, Lx=2.0, nx=1024, ny=512, dt=0.008),
    "R030s": dict(eta=0.0122, rho=6250.0, l=0.00156, gdot=0.0410, Lx=2.0, nx=1024, ny=512, dt=0.004),
    "R019s": dict(eta=0.00876, rho=32814.0, l=0.00156, gdot=0.0251, Lx=2.0, nx=1024, ny=512, dt=0.004),
    "R032s": dict(eta=0.00391, rho=20067.0, l=0.00156, gdot=0.051, Lx=2.0, nx=1024, ny=512, dt=0.004),
    # (d) applied shear, without inertia
    "DV1s": dict(eta=1000.0, rho=0.0, l=0.00156, gdot=0.01, Lx=2.0, nx=1024, ny=512, dt=0.016),
    "DV2s": dict(eta=100.0, rho=0.0, l=0.00156, gdot=0.01, Lx=2.0, nx=1024, ny=512, dt=0.016),
    "DV3s": dict(eta=10.0, rho=0.0, l=0.00156, gdot=0.01, Lx=2.0, nx=1024, ny=512, dt=0.016),
    "DV4s": dict(eta=1.0, rho=0.0, l=0.00156, gdot=0.01, Lx=2.0, nx=1024, ny=512, dt=0.016),
    "DV5s": dict(eta=0.3, rho=0.0, l=0.00156, gdot=0.01, Lx=2.0, nx=1024, ny=512, dt=0.016),
    "DV6s": dict(eta=0.1, rho=0.0, l=0.00156, gdot=0.03, Lx=2.0, nx=1024, ny=512, dt=0.016),
}


def paper_units(name):
    """Grid arguments of Table I set ``name`` in the paper's units (Section IV):
    Lambda_y = G = tau_0 = 1, so mu = phi(phi^2 - 1) - l^2 lap phi (a = b = 1,
    kappa = l^2) and d_t phi + v.grad phi = l^2 lap mu (M = l^2), on a mesh of
    spacing dx = Lambda_y / Ny.  Returns (nx, ny, dx, params) with params the
    keyword arguments of Grid.set_params."""
    t = TABLE_I[name]
    l2 = t["l"] * t["l"]
    params = dict(a=1.0, b=1.0, kappa=l2, M=l2, eta=t["eta"], rho=t["rho"], gdot=t["gdot"], dt=t["dt"])
    return t["nx"], t["ny"], 1.0 / t["ny"], params


def ensemble_spec(runs=96, dt=0.005):
    """The batched runs: run r has N = 128 * 2^(r // 32), rho = r mod 2,
    gdot = 1e-4 * 300^(r / 95), eta = 1, seed r."""
    sizes = [128 * 2 ** (r // 32) for r in range(runs)]
    params = [[1.0, 1.0, 1.0, 1.0, 1.0, float(r % 2), 1e-4 * 300.0 ** (r / max(runs - 1, 1)), dt]
              for r in range(runs)]
    return sizes, params


def make(name, **overrides):
    """A Grid (or Ensemble) for configuration ``name`` with its quench applied;
    keyword overrides replace model parameters (e.g. gdot=0.01, rho=0.1)."""
    cfg = CONFIGS[name]
    if name.startswith("c4"):
        sizes, params = ensemble_spec(cfg["runs"])
        return Ensemble(sizes, sizes, params, seeds=list(range(cfg["runs"])), amp=cfg["amp"],
                        precision=cfg["precision"])
    params = dict(cfg["params"], **overrides)
    g = Grid(cfg["nx"], cfg["ny"], 1.0, cfg["precision"])
    g.set_params(**params)
    g.init_noise(cfg["seed"], cfg["amp"])
    return g
