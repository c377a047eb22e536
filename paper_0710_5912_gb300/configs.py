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
