"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Tolerances (relative L2 per field): FP64 <= 1e-10 and FP32 <= 2e-5 after 200
steps from the same seeded state; single steps from rough random states
FP64 <= 1e-11, FP32 <= 1e-5.  Every field is held to these, FP32 psi
included: inertial runs carry omega in spectral form and take the force's
lowest modes from compensated sums; Stokes runs (rho = 0, psi_hat =
g_hat / (eta k^4)) form the force beyond FP32 for its lowest modes.  The
one exception is the 3-step 1024^2 quench, whose psi is held to the FP32
error model (fp32_model.psi32_model_ratio; see that test).  Index work (the
wrap remap, checkpoint resume, graph replay, ensemble batching, the
phi -> -phi symmetry) is bit-exact.
"""
import math
import os

import numpy as np
import pytest

import oracle
import paper_0710_5912_gb300 as shf
from paper_0710_5912_gb300 import configs, inputs
from fp32_model import PSI32_MODEL_MAX, psi32_model_ratio

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32, FP64 = shf.SHF_FP32, shf.SHF_FP64
TOL_200 = {FP64: 1e-10, FP32: 2e-5}
TOL_1 = {FP64: 1e-11, FP32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    shf.lib()


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def gpu_run(nx, ny, prec, p, fields, n0, nsteps, remap=shf.SHF_REMAP_SHIFT, chunks=None):
    with shf.Grid(nx, ny, p.dx, prec, remap) as g:
        g.set_params(p.a, p.b, p.kappa, p.M, p.eta, p.rho, p.gdot, p.dt)
        g.set_fields(*fields)
        g.set_step(n0)
        for c in (chunks or [nsteps]):
            g.step(c)
        g.sync()
        out = g.get_fields()
        assert g.get_time()[0] == n0 + nsteps
    return out


def oracle_run(p, fields, n0, nsteps, remap=oracle.REMAP_SHIFT):
    return oracle.run(*fields, nsteps, p, n0=n0, remap=remap)


def rough_state(nx, ny, seed, inertial=True):
    phi = inputs.quench_noise(nx, ny, seed, 0.5)
    psi = inputs.quench_noise(nx, ny, seed + 1, 0.05)
    om = inputs.quench_noise(nx, ny, seed + 2, 0.05) if inertial else np.zeros((ny, nx))
    return phi, psi, om


def assert_close(got, want, tol, rho, what="", prec=FP64, s=0.0, dx=1.0, psi_model=False):
    """Relative L2 per field; with psi_model, FP32 psi is held instead to the
    FP32 error model of fp32_model.psi32_model_ratio."""
    names = ("phi", "psi", "omega")
    for name, a, b in zip(names, got, want):
        if rho == 0 and name == "omega":
            assert np.abs(a).max() == 0.0
            continue
        if name == "psi" and prec == FP32 and psi_model:
            q = psi32_model_ratio(a, b, s, dx, rho)
            assert q <= PSI32_MODEL_MAX, f"{what} psi: error/model {q:.2f} > {PSI32_MODEL_MAX} " \
                                         f"(rel L2 {rel_l2(a, b):.2e})"
            continue
        err = rel_l2(a, b)
        assert err <= tol, f"{what} {name}: rel L2 {err:.3e} > {tol:g}"


# ------------------------------------------------------------- single steps

SHAPES = [(16, 16), (32, 16), (64, 64), (128, 32), (256, 256), (512, 64)]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("rho", [0.0, 0.7])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("strain", ["zero", "pos", "neg"])
def test_one_step_from_rough_state(prec, rho, shape, strain):
    nx, ny = shape
    gdot = {"zero": 0.0, "pos": 0.3, "neg": -0.3}[strain]
    p = oracle.Params(a=0.9, b=1.1, kappa=0.8, M=1.2, eta=0.6, rho=rho, gdot=gdot, dt=0.01, dx=0.9)
    fields = rough_state(nx, ny, 17, rho > 0)
    n0 = 37
    got = gpu_run(nx, ny, prec, p, fields, n0, 2)
    want = oracle_run(p, fields, n0, 2)
    s_end = oracle.strain(n0 + 2, p.gdot, p.dt, nx, ny)[0]
    assert_close(got, want, TOL_1[prec], rho, f"{shape} {strain}", prec, s_end, p.dx)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("rho", [0.0, 1.0])
@pytest.mark.parametrize("shape", [(32, 32), (64, 32), (64, 16)])
@pytest.mark.parametrize("remap", [shf.SHF_REMAP_SHIFT, shf.SHF_REMAP_NONE])
def test_steps_across_strain_wraps(prec, rho, shape, remap):
    nx, ny = shape
    r = nx // ny
    gd = 2.0 ** -5           # gdot*dt: the strain wraps every 16 r steps
    p = oracle.Params(a=1.0, b=1.0, kappa=1.0, M=1.0, eta=1.0, rho=rho, gdot=gd / 0.01, dt=0.01)
    fields = rough_state(nx, ny, 5, rho > 0)
    nsteps = 50 * r
    s_end, K_end = oracle.strain(3 + nsteps, p.gdot, p.dt, nx, ny)
    assert K_end >= 2
    got = gpu_run(nx, ny, prec, p, fields, 3, nsteps, remap)
    want = oracle_run(p, fields, 3, nsteps, remap)
    assert_close(got, want, TOL_200[prec], rho, f"wrap {shape} remap={remap}", prec, s_end, 1.0)


# ------------------------------------------------------------ 200-step runs

def test_config_small_stokes_fp64_full_run():
    """64x64 Stokes, FP64, gdot = 0.01, dt = 0.005, seed 0: 200 steps and the full
    2000-step run against the oracle."""
    nx = ny = 64
    p = oracle.Params(a=1, b=1, kappa=1, M=1, eta=1, rho=0.0, gdot=0.01, dt=0.005)
    fields = inputs.quench_state(nx, ny, 0)
    with shf.Grid(nx, ny, 1.0, FP64) as g:
        g.set_params(p.a, p.b, p.kappa, p.M, p.eta, p.rho, p.gdot, p.dt)
        g.init_noise(0, 0.01)
        assert np.array_equal(g.get_fields()[0], fields[0])
        g.step(200)
        g.sync()
        got200 = g.get_fields()
        g.step(1800)
        g.sync()
        got2000 = g.get_fields()
    want200 = oracle_run(p, fields, 0, 200)
    assert_close(got200, want200, 1e-10, 0.0, "200 steps")
    want2000 = oracle_run(p, want200, 200, 1800)
    assert_close(got2000, want2000, 1e-10, 0.0, "2000 steps")


@pytest.mark.parametrize("gdot", [0.001, 0.003, 0.01])
def test_inertial_256_fp32_200_steps(gdot):
    nx = ny = 256
    p = oracle.Params(a=1, b=1, kappa=1, M=1, eta=1, rho=1.0, gdot=gdot, dt=0.005)
    fields = inputs.quench_state(nx, ny, 1)
    got = gpu_run(nx, ny, FP32, p, fields, 0, 200)
    want = oracle_run(p, fields, 0, 200)
    assert_close(got, want, 2e-5, 1.0, f"256^2 gdot={gdot}", FP32, oracle.strain(200, gdot, p.dt, nx, ny)[0])


@pytest.mark.parametrize("rho", [0.0, 1.0])
def test_fp64_200_steps_rect(rho):
    nx, ny = 128, 64
    p = oracle.Params(a=1, b=1, kappa=1, M=1, eta=1, rho=rho, gdot=0.05, dt=0.01)
    fields = inputs.quench_state(nx, ny, 2, 0.3)
    got = gpu_run(nx, ny, FP64, p, fields, 0, 200)
    want = oracle_run(p, fields, 0, 200)
    assert_close(got, want, 1e-10, rho, "128x64 fp64")


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("rho", [0.0, 0.05])
def test_paper_geometry_1024x512_across_a_wrap(prec, rho):
    """The paper's sheared geometry Lx = 2 Ly (Table I, 1024 x 512): the remap
    shifts row j by 2j cells.  gdot dt = 2^-5 puts the wrap at step 32; steps
    28..36 cross it."""
    nx, ny = 1024, 512
    p = oracle.Params(a=1, b=1, kappa=1, M=1, eta=1, rho=rho, gdot=2.0 ** -5 / 0.004, dt=0.004)
    fields = rough_state(nx, ny, 21, rho > 0)
    fields = tuple(0.1 * f for f in fields)
    K0 = oracle.strain(28, p.gdot, p.dt, nx, ny)[1]
    s_end, K1 = oracle.strain(36, p.gdot, p.dt, nx, ny)
    assert K1 == K0 + 1
    got = gpu_run(nx, ny, prec, p, fields, 28, 8)
    want = oracle_run(p, fields, 28, 8)
    assert_close(got, want, TOL_200[prec], rho, f"1024x512 rho={rho}", prec, s_end, 1.0)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("name", ["R028s", "R030s", "DV4s", "DV6s"])
def test_table_I_parameters_across_the_first_wrap(prec, name):
    """Table I sets (c: sheared with inertia; d: sheared without) in the
    paper's units (Section IV: dx = Lambda_y / 512, kappa = M = l^2,
    Lambda_x = 2) on 1024 x 512: 8 steps across the first strain wrap, where
    |s| reaches 1 and the remap shifts row j by 2j cells, from a rough phi
    (+-0.05) at rest, against the oracle."""
    nx, ny, dx, pp = configs.paper_units(name)
    p = oracle.Params(dx=dx, **pp)
    n_wrap = int(math.ceil(1.0 / (p.gdot * p.dt)))
    while oracle.strain(n_wrap, p.gdot, p.dt, nx, ny)[1] == 0:
        n_wrap += 1
    while oracle.strain(n_wrap - 1, p.gdot, p.dt, nx, ny)[1] == 1:
        n_wrap -= 1
    n0 = n_wrap - 4
    s_before = oracle.strain(n0 + 3, p.gdot, p.dt, nx, ny)[0]
    assert s_before > 0.95                              # |s| near 1 just before the wrap
    phi = 0.1 * inputs.quench_noise(nx, ny, 31, 0.5)
    zero = np.zeros((ny, nx))
    fields = (phi, zero, zero)
    got = gpu_run(nx, ny, prec, p, fields, n0, 8)
    want = oracle_run(p, fields, n0, 8)
    s_end = oracle.strain(n0 + 8, p.gdot, p.dt, nx, ny)[0]
    for nm, a, b in zip(("phi", "psi", "omega"), got, want):
        print(f"{name} {'fp32' if prec == FP32 else 'fp64'} {nm}: rel L2 {rel_l2(a, b):.3e}")
    assert_close(got, want, TOL_200[prec], p.rho, f"{name}", prec, s_end, dx)


@pytest.mark.parametrize("rho", [0.0, 0.1, 1.0])
def test_config_1024_side_by_side(rho):
    """1024x1024 FP32, eta = 1, gdot = 0.003, dt = 0.005: three steps from the
    quench against the oracle.  psi is held to the FP32 error model here: three
    steps in, its lowest modes have grown to only a small fraction of what they
    reach after 200 steps, where the 2e-5 gate applies (test_config_1024_200_steps)."""
    nx = ny = 1024
    p = oracle.Params(a=1, b=1, kappa=1, M=1, eta=1, rho=rho, gdot=0.003, dt=0.005)
    fields = inputs.quench_state(nx, ny, 3)
    got = gpu_run(nx, ny, FP32, p, fields, 0, 3)
    want = oracle_run(p, fields, 0, 3)
    print(f"1024^2 rho={rho} 3 steps psi: rel L2 {rel_l2(got[1], want[1]):.3e}")
    assert_close(got, want, 1e-5, rho, f"1024^2 rho={rho}", FP32, oracle.strain(3, p.gdot, p.dt, nx, ny)[0],
                 psi_model=True)


@pytest.mark.parametrize("rho", [0.0, 0.1, 1.0])
def test_config_1024_200_steps(rho):
    """1024x1024 FP32, eta = 1, gdot = 0.003, dt = 0.005, from the seeded +-0.01
    quench: 200 steps against the oracle at 2e-5 relative L2 for every field
    (the values are printed)."""
    nx = ny = 1024
    p = oracle.Params(a=1, b=1, kappa=1, M=1, eta=1, rho=rho, gdot=0.003, dt=0.005)
    fields = inputs.quench_state(nx, ny, 3)
    got = gpu_run(nx, ny, FP32, p, fields, 0, 200)
    want = oracle_run(p, fields, 0, 200)
    for name, a, b in zip(("phi", "psi", "omega"), got, want):
        print(f"1024^2 rho={rho} 200 steps {name}: rel L2 {rel_l2(a, b):.3e}")
    assert_close(got, want, TOL_200[FP32], rho, f"1024^2 rho={rho} 200 steps", FP32,
                 oracle.strain(200, p.gdot, p.dt, nx, ny)[0])


def test_config_4096_inertial_full_size_step():
    """4096x4096 FP32 inertial (rho = eta = 1, gdot = 0.001): one step in the bench's
    launch configuration against the oracle, every point compared."""
    nx = ny = 4096
    p = oracle.Params(a=1, b=1, kappa=1, M=1, eta=1, rho=1.0, gdot=0.001, dt=0.005)
    phi = inputs.quench_noise(nx, ny, 0)
    psi = 1e-3 * inputs.quench_noise(nx, ny, 1, 1.0)
    om = 1e-3 * inputs.quench_noise(nx, ny, 2, 1.0)
    fields = (phi, psi, om)
    got = gpu_run(nx, ny, FP32, p, fields, 1234, 1)
    want = oracle_run(p, fields, 1234, 1)
    assert_close(got, want, 1e-5, 1.0, "4096^2", FP32, oracle.strain(1235, p.gdot, p.dt, nx, ny)[0])


# --------------------------------------------------------------- invariants

@pytest.mark.parametrize("prec,tol", [(FP64, 1e-15), (FP32, 1e-9)])
def test_mass_is_conserved(prec, tol):
    nx = ny = 128
    with shf.Grid(nx, ny, 1.0, prec) as g:
        g.set_params(rho=1.0, gdot=0.01, dt=0.005)
        g.init_noise(9, 0.01)
        m0 = g.mass()
        want0 = oracle.mean_phi(inputs.quench_noise(nx, ny, 9))
        if prec == FP64:
            assert abs(m0 - want0) <= 1e-18
        g.step(1000)
        g.sync()
        m1 = g.mass()
        phi = g.get_fields()[0]
    assert abs(m1 - m0) <= tol
    assert abs(m1 - oracle.mean_phi(phi)) <= 1e-18


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("rho", [0.0, 1.0])
def test_phi_sign_symmetry_bit_exact(prec, rho):
    nx, ny = 64, 32
    p = oracle.Params(rho=rho, gdot=0.4, dt=0.01)
    phi, psi, om = rough_state(nx, ny, 23, rho > 0)
    a = gpu_run(nx, ny, prec, p, (phi, psi, om), 5, 30)
    b = gpu_run(nx, ny, prec, p, (-phi, psi, om), 5, 30)
    assert np.array_equal(a[0], -b[0])
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_remap_is_an_exact_permutation(prec):
    """With M -> tiny and no flow the step is (numerically) the identity except for
    the remap at the wrap, which must permute the stored values exactly."""
    nx = ny = 32
    gd = 2.0 ** -5
    p = oracle.Params(a=0.0, b=0.0, kappa=1.0, M=1e-300, eta=1.0, rho=0.0, gdot=gd / 0.01, dt=0.01)
    phi = inputs.quench_noise(nx, ny, 4, 1.0)
    if prec == FP32:
        phi = phi.astype(np.float32).astype(np.float64)
    zero = np.zeros_like(phi)
    before = gpu_run(nx, ny, prec, p, (phi, zero, zero), 15, 0)[0]
    after = gpu_run(nx, ny, prec, p, (phi, zero, zero), 15, 1)[0]     # step 15 -> 16 wraps
    assert oracle.strain(16, p.gdot, p.dt, nx, ny)[1] == 1
    # the stage-1 FFT round trip is not bit-exact, so compare after the same round trip:
    # apply the permutation to a run that does not wrap
    nowrap = gpu_run(nx, ny, prec, p, (phi, zero, zero), 14, 1)[0]
    assert np.array_equal(np.sort(after.ravel()), np.sort(nowrap.ravel()))
    assert np.array_equal(after, oracle.remap_rows(nowrap, 1))
    assert before.shape == after.shape


# ------------------------------------------------- graphs, checkpoints, ensembles

@pytest.mark.parametrize("prec", [FP64, FP32])
def test_graph_replay_equals_direct_launches(prec):
    nx = ny = 64
    p = oracle.Params(rho=1.0, gdot=0.02, dt=0.01)
    fields = rough_state(nx, ny, 31)
    a = gpu_run(nx, ny, prec, p, fields, 0, 250)                           # 2 graph replays + 50
    b = gpu_run(nx, ny, prec, p, fields, 0, 250, chunks=[1] * 250)          # all direct
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("rho", [0.0, 1.0])
def test_checkpoint_resume_is_bit_identical(prec, rho, tmp_path):
    nx, ny = 64, 32
    p = oracle.Params(rho=rho, gdot=0.05, dt=0.01)
    straight = gpu_run(nx, ny, prec, p, rough_state(nx, ny, 41, rho > 0), 0, 200)
    path = tmp_path / "ck.shf"
    with shf.Grid(nx, ny, 1.0, prec) as g:
        g.set_params(p.a, p.b, p.kappa, p.M, p.eta, p.rho, p.gdot, p.dt)
        g.set_fields(*rough_state(nx, ny, 41, rho > 0))
        g.step(100)
        g.save(path)
    with shf.Grid(nx, ny, 1.0, prec) as g2:
        g2.load(path)
        assert g2.get_time()[0] == 100
        g2.step(100)
        resumed = g2.get_fields()
    for x, y in zip(straight, resumed):
        assert np.array_equal(x, y)


def test_checkpoint_load_across_regimes_after_graph(tmp_path):
    """Loading an inertial checkpoint into a grid that captured a Stokes graph
    must drop that graph: the flow column pass is chosen per regime."""
    nx, ny = 64, 32
    pi = oracle.Params(rho=1.0, gdot=0.05, dt=0.01)
    ps = oracle.Params(rho=0.0, gdot=0.05, dt=0.01)
    path = tmp_path / "inertial.shf"
    with shf.Grid(nx, ny, 1.0, FP32) as g:
        g.set_params(pi.a, pi.b, pi.kappa, pi.M, pi.eta, pi.rho, pi.gdot, pi.dt)
        g.set_fields(*rough_state(nx, ny, 43))
        g.step(100)
        g.save(path)
    with shf.Grid(nx, ny, 1.0, FP32) as ref:
        ref.load(path)
        ref.step(100)
        want = ref.get_fields()
    with shf.Grid(nx, ny, 1.0, FP32) as g2:
        g2.set_params(ps.a, ps.b, ps.kappa, ps.M, ps.eta, ps.rho, ps.gdot, ps.dt)
        g2.set_fields(*rough_state(nx, ny, 44, False))
        g2.step(100)                                    # captures a Stokes graph
        g2.load(path)
        g2.step(100)
        got = g2.get_fields()
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


def test_checkpoint_errors(tmp_path):
    with shf.Grid(32, 32, 1.0, FP32) as g:
        g.set_params()
        g.init_noise(1)
        path = tmp_path / "a.shf"
        g.save(path)
        data = bytearray(path.read_bytes())
        data[-5] ^= 0xFF
        bad = tmp_path / "bad.shf"
        bad.write_bytes(bytes(data))
        with pytest.raises(shf.ShfError) as e:
            g.load(bad)
        assert e.value.code == shf.SHF_EIO
        short = tmp_path / "short.shf"
        short.write_bytes(path.read_bytes()[:100])
        with pytest.raises(shf.ShfError) as e:
            g.load(short)
        assert e.value.code == shf.SHF_EIO
        with pytest.raises(shf.ShfError) as e:
            g.load(tmp_path / "missing.shf")
        assert e.value.code == shf.SHF_EIO
    with shf.Grid(64, 32, 1.0, FP32) as g:
        with pytest.raises(shf.ShfError) as e:
            g.load(path)
        assert e.value.code == shf.SHF_EINVAL
    with shf.Grid(32, 32, 0.5, FP32) as g:          # same size and precision, another dx
        g.set_params()
        g.init_noise(2)
        before = g.get_fields()
        with pytest.raises(shf.ShfError) as e:
            g.load(path)
        assert e.value.code == shf.SHF_EINVAL
        after = g.get_fields()
        assert all(np.array_equal(a, b) for a, b in zip(before, after))


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_ensemble_members_match_single_runs(prec):
    nxs = [32, 64, 32, 128, 64]
    nys = [32, 32, 32, 64, 64]
    params = []
    for r in range(5):
        params.append([1.0, 1.0, 1.0, 1.0, 1.0, float(r % 2), 10 ** (-3 + r * 0.5), 0.01])
    ens = shf.Ensemble(nxs, nys, params, seeds=list(range(5)), amp=0.2, precision=prec)
    ens.step(120)
    ens.sync()
    for r in range(5):
        a, b, kap, M, eta, rho, gdot, dt = params[r]
        p = oracle.Params(a=a, b=b, kappa=kap, M=M, eta=eta, rho=rho, gdot=gdot, dt=dt)
        fields = inputs.quench_state(nxs[r], nys[r], r, 0.2)
        single = gpu_run(nxs[r], nys[r], prec, p, fields, 0, 120)
        got = ens.members[r].get_fields()
        for x, y in zip(got, single):
            assert np.array_equal(x, y), f"member {r}"
        want = oracle_run(p, fields, 0, 120)
        assert_close(got, want, TOL_200[prec], rho, f"member {r}", prec,
                     oracle.strain(120, gdot, dt, nxs[r], nys[r])[0])
        assert ens.members[r].get_time()[0] == 120
    ens.close()


def test_ensemble_with_tma_rows_and_class_streams_matches_single_runs():
    """An FP32 ensemble whose two 1024 x 512 members take the TMA-loaded inverse
    row passes (one tensor map per member) and the chunk column kernel, beside a
    256^2 member in its own size class (its own stream): every member bit-equal
    to its single run after 120 steps (one graph replay plus direct launches),
    across a strain wrap for the sheared 1024 x 512 members."""
    nxs, nys = [1024, 256, 1024], [512, 256, 512]
    params = [[1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 2.0, 0.005],
              [1.0, 1.0, 1.0, 1.0, 1.0, 0.0, 0.01, 0.005],
              [1.0, 1.0, 1.0, 1.0, 1.0, 0.0, 2.0, 0.005]]
    ens = shf.Ensemble(nxs, nys, params, seeds=[7, 8, 9], amp=0.2, precision=FP32)
    ens.step(120)
    ens.sync()
    for r in range(3):
        a, b, kap, M, eta, rho, gdot, dt = params[r]
        p = oracle.Params(a=a, b=b, kappa=kap, M=M, eta=eta, rho=rho, gdot=gdot, dt=dt)
        fields = inputs.quench_state(nxs[r], nys[r], 7 + r, 0.2)
        single = gpu_run(nxs[r], nys[r], FP32, p, fields, 0, 120)
        got = ens.members[r].get_fields()
        for name, x, y in zip(("phi", "psi", "omega"), got, single):
            assert np.array_equal(x, y), f"member {r} {name}"
        if nxs[r] == 1024:
            assert ens.members[r].get_time()[3] >= 1        # the strain wrapped
    ens.close()


def c4_ensemble_spec():
    """The batched-ensemble configuration: 96 runs, 32 each of 128^2, 256^2 and
    512^2, rho = r mod 2, gdot log-spaced over 1e-4 .. 3e-2, seed r."""
    nxs = [128 * 2 ** (r // 32) for r in range(96)]
    params = [[1.0, 1.0, 1.0, 1.0, 1.0, float(r % 2), 1e-4 * 300.0 ** (r / 95.0), 0.005] for r in range(96)]
    return nxs, params


def test_c4_ensemble_members_match_single_runs_and_oracle():
    nxs, params = c4_ensemble_spec()
    ens = shf.Ensemble(nxs, nxs, params, seeds=list(range(96)), amp=0.01, precision=FP32)
    ens.step(20)
    ens.sync()
    for r in (0, 33, 95):
        a, b, kap, M, eta, rho, gdot, dt = params[r]
        p = oracle.Params(a=a, b=b, kappa=kap, M=M, eta=eta, rho=rho, gdot=gdot, dt=dt)
        fields = inputs.quench_state(nxs[r], nxs[r], r, 0.01)
        single = gpu_run(nxs[r], nxs[r], FP32, p, fields, 0, 20)
        got = ens.members[r].get_fields()
        for x, y in zip(got, single):
            assert np.array_equal(x, y), f"member {r}"
        if nxs[r] <= 256:
            want = oracle_run(p, fields, 0, 20)
            assert_close(got, want, 1e-5, rho, f"C4 member {r}", FP32, oracle.strain(20, gdot, dt, nxs[r], nxs[r])[0])
    ens.close()


def test_autotune_keeps_the_state_and_parity(tmp_path):
    nx = ny = 256
    p = oracle.Params(a=1, b=1, kappa=1, M=1, eta=1, rho=1.0, gdot=0.01, dt=0.005)
    fields = inputs.quench_state(nx, ny, 6, 0.2)
    cache = tmp_path / "tune.json"
    with shf.Grid(nx, ny, 1.0, FP32) as g:
        g.set_params(p.a, p.b, p.kappa, p.M, p.eta, p.rho, p.gdot, p.dt)
        g.set_fields(*fields)
        g.step(100)                                       # the graph path is captured before tuning
        before = g.get_fields()
        choices = g.autotune(cache)
        assert len(choices) == 1 and choices[0][0] in (8, 16) and choices[0][1] == 16
        after = g.get_fields()
        for x, y in zip(before, after):
            assert np.array_equal(x, y)                   # tuning runs only scratch-writing kernels
        assert g.get_time()[0] == 100
        g.step(100)                                       # graph re-captured with the tuned shapes
        got = g.get_fields()
    want = oracle_run(p, fields, 0, 200)
    assert_close(got, want, 2e-5, 1.0, "autotuned 256^2", FP32, oracle.strain(200, p.gdot, p.dt, nx, ny)[0])
    text = cache.read_text()
    assert '"256x256:fp32:inertial"' in text
    with shf.Grid(nx, ny, 1.0, FP32) as g2:                # the cached choice is applied as is
        g2.set_params(p.a, p.b, p.kappa, p.M, p.eta, p.rho, p.gdot, p.dt)
        assert g2.autotune(cache) == choices
    assert cache.read_text() == text


def test_autotune_ensemble_per_size_class():
    nxs = [64, 128, 64, 128]
    params = [[1.0, 1.0, 1.0, 1.0, 1.0, float(r % 2), 0.01, 0.005] for r in range(4)]
    ens = shf.Ensemble(nxs, nxs, params, seeds=list(range(4)), amp=0.1, precision=FP32)
    choices = ens.autotune()
    assert len(choices) == 2
    ens.step(20)
    ens.sync()
    for r in range(4):
        a, b, kap, M, eta, rho, gdot, dt = params[r]
        pr = oracle.Params(a=a, b=b, kappa=kap, M=M, eta=eta, rho=rho, gdot=gdot, dt=dt)
        fields = inputs.quench_state(nxs[r], nxs[r], r, 0.1)
        want = oracle_run(pr, fields, 0, 20)
        assert_close(ens.members[r].get_fields(), want, 1e-5, rho, f"tuned member {r}", FP32,
                     oracle.strain(20, gdot, dt, nxs[r], nxs[r])[0])
    ens.close()


def test_float_host_fields_round_trip_and_match_double_path():
    nx, ny = 128, 64
    p = oracle.Params(rho=1.0, gdot=0.02, dt=0.005)
    fields = inputs.quench_state(nx, ny, 12, 0.2)
    f32 = tuple(np.asarray(f, dtype=np.float32) for f in fields)
    with shf.Grid(nx, ny, 1.0, FP32) as a, shf.Grid(nx, ny, 1.0, FP32) as b:
        for g in (a, b):
            g.set_params(p.a, p.b, p.kappa, p.M, p.eta, p.rho, p.gdot, p.dt)
        a.set_fields_f32(*f32)
        b.set_fields(*fields)                           # doubles, rounded to float on the device
        got_a = a.get_fields_f32()
        for x, y in zip(got_a, f32):
            assert np.array_equal(x, y)
        a.step(10)
        b.step(10)
        for x, y in zip(a.get_fields_f32(), b.get_fields()):
            assert np.array_equal(x.astype(np.float64), y)
    with shf.Grid(32, 32, 1.0, FP64) as g:
        with pytest.raises(shf.ShfError) as e:
            g.set_fields_f32(np.zeros((32, 32), np.float32))
        assert e.value.code == shf.SHF_EINVAL


@pytest.mark.parametrize("rho", [1.0, 0.0])
@pytest.mark.parametrize("nsteps", [0, 1, 3, 101])
def test_step_host_matches_set_step_get(rho, nsteps):
    """shf_step_host_f32 (upload, steps, download with phi copied while the
    flow passes run) gives the same bits as set_fields_f32 + step +
    get_fields_f32, also across a graph replay (101 steps)."""
    nx, ny = 128, 64
    p = oracle.Params(rho=rho, gdot=0.02, dt=0.005)
    fields = [np.asarray(f, dtype=np.float32) for f in inputs.quench_state(nx, ny, 5, 0.2)]
    if rho == 0.0:
        fields[2][:] = 0.0
    with shf.Grid(nx, ny, 1.0, FP32) as a, shf.Grid(nx, ny, 1.0, FP32) as b:
        for g in (a, b):
            g.set_params(p.a, p.b, p.kappa, p.M, p.eta, p.rho, p.gdot, p.dt)
        out = a.step_host_f32(nsteps, *fields)
        b.set_fields_f32(*fields)
        b.step(nsteps)
        want = b.get_fields_f32()
        for x, y in zip(out, want):
            assert np.array_equal(x, y)
        assert a.get_time()[0] == nsteps
        # no inputs: continue from the device state; outputs may be skipped
        phi_only = np.empty((ny, nx), np.float32)
        a.step_host_f32(2, out=(phi_only, None, None))
        b.step(2)
        assert np.array_equal(phi_only, b.get_fields_f32()[0])
        assert np.array_equal(a.get_fields_f32()[1], b.get_fields_f32()[1])


def test_regime_switch_after_graph_capture():
    """The flow column pass is compiled per regime and chosen on the host, so
    a CUDA graph captured for an inertial run must not survive set_params to
    the Stokes regime: 100 graph steps inertial, then 100 Stokes, against the
    oracle over the same sequence."""
    nx = ny = 64
    pi = oracle.Params(rho=1.0, gdot=0.01, dt=0.005)
    ps = oracle.Params(rho=0.0, gdot=0.01, dt=0.005)
    fields = rough_state(nx, ny, 21)
    mid = oracle_run(pi, fields, 0, 100)
    want = oracle_run(ps, mid, 100, 100)
    with shf.Grid(nx, ny, 1.0, FP32) as g:
        g.set_params(pi.a, pi.b, pi.kappa, pi.M, pi.eta, pi.rho, pi.gdot, pi.dt)
        g.set_fields(*fields)
        g.step(100)
        g.set_params(ps.a, ps.b, ps.kappa, ps.M, ps.eta, ps.rho, ps.gdot, ps.dt)
        g.step(100)
        got = g.get_fields()
    assert_close(got, want, 1e-5, 0.0, "inertial then Stokes", FP32,
                 oracle.strain(200, ps.gdot, ps.dt, nx, ny)[0])


def test_step_host_rejects_bad_calls():
    with shf.Grid(32, 32, 1.0, FP64) as g:
        g.set_params(1, 1, 1, 1, 1, 1, 0.01, 0.005)
        with pytest.raises(shf.ShfError) as e:
            g.step_host_f32(1, np.zeros((32, 32), np.float32))
        assert e.value.code == shf.SHF_EINVAL
    with shf.Grid(32, 32, 1.0, FP32) as g:
        with pytest.raises(shf.ShfError) as e:
            g.step_host_f32(1)
        assert e.value.code == shf.SHF_ESTATE
        g.set_params(1, 1, 1, 1, 1, 1, 0.01, 0.005)
        z = np.zeros((32, 32), np.float32)
        rc = shf.lib().shf_step_host_f32(g.handle, 1, None, z.ctypes.data_as(shf._native.P_float), None,
                                         None, None, None)
        assert rc == shf.SHF_EINVAL
    ens = shf.Ensemble([32, 32], [32, 32], [[1, 1, 1, 1, 1, 1, 0.01, 0.005]] * 2, seeds=[0, 1], amp=0.1,
                       precision=FP32)
    rc = shf.lib().shf_step_host_f32(ens.handle, 1, None, None, None, None, None, None)
    assert rc == shf.SHF_EINVAL
    ens.close()


# --------------------------------------------------------------- diagnostics

@pytest.mark.parametrize("prec,tol", [(FP64, 1e-11), (FP32, 1e-5)])
def test_structure_factor_matches_oracle(prec, tol):
    nx, ny = 128, 64
    p = oracle.Params(rho=1.0, gdot=0.07, dt=0.01)
    fields = inputs.quench_state(nx, ny, 8, 0.3)
    with shf.Grid(nx, ny, 1.0, prec) as g:
        g.set_params(p.a, p.b, p.kappa, p.M, p.eta, p.rho, p.gdot, p.dt)
        g.set_fields(*fields)
        g.step(50)
        moments, bins = g.structure_factor(nbins=48)
        phi = g.get_fields()[0]
        n, t, s, K = g.get_time()
    assert (s, K) == oracle.strain(50, p.gdot, p.dt, nx, ny)
    want = oracle.structure_factor_moments(phi, s, 1.0)
    wbins = oracle.structure_factor_binned(phi, s, 48, 1.0)
    for a, b in zip(moments, want):
        assert math.isclose(a, b, rel_tol=tol), (moments, want)
    assert np.allclose(bins, wbins, rtol=tol, atol=tol * wbins.max())


def test_structure_factor_single_mode_closed_form():
    nx = ny = 64
    A, m, n = 0.4, 3, -2
    with shf.Grid(nx, ny, 1.0, FP64) as g:
        g.set_params(gdot=0.0)
        g.set_fields(inputs.cosine_mode(nx, ny, m, n, amp=A))
        moments, _ = g.structure_factor()
    k = 2 * math.pi * math.hypot(m, n) / nx
    assert math.isclose(moments[0], A * A / 2, rel_tol=1e-13)
    assert math.isclose(moments[3], 2 * math.pi / k, rel_tol=1e-13)
    assert math.isclose(moments[4], 1 / k, rel_tol=1e-13)


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (FP32, 2e-6)])
@pytest.mark.parametrize("shape,gdot", [((128, 64), 0.07), ((64, 64), -0.2), ((256, 128), 0.0)])
def test_gradient_tensor_matches_oracle(prec, tol, shape, gdot):
    """Eq. L_matrix on a stepped state (strain nonzero, and past a wrap for the
    first shape) against the oracle on the same phi."""
    nx, ny = shape
    p = oracle.Params(rho=1.0, gdot=gdot, dt=0.01)
    fields = inputs.quench_state(nx, ny, 4, 0.3)
    with shf.Grid(nx, ny, 1.0, prec) as g:
        g.set_params(p.a, p.b, p.kappa, p.M, p.eta, p.rho, p.gdot, p.dt)
        g.set_fields(*fields)
        g.step(60)
        G, L = g.gradient_tensor()
        phi = g.get_fields()[0]
        _, _, s, _ = g.get_time()
    want = oracle.gradient_tensor(phi, s, 1.0)
    scale = max(abs(want[0]), abs(want[2]))
    for a, b in zip(G, want):
        assert abs(a - b) <= tol * scale, (G, want)
    wl = oracle.principal_lengths(want, math.sqrt(p.kappa / p.a))
    for a, b in zip(L, wl):
        assert math.isclose(a, b, rel_tol=10 * tol), (L, wl)


def test_gradient_tensor_two_modes_closed_form():
    nx, ny, s_gdot = 64, 32, 0.3
    A, B, c = 0.5, 0.2, 0.1
    phi = (c + inputs.cosine_mode(nx, ny, 2, 1, amp=A) + inputs.cosine_mode(nx, ny, -1, 3, amp=B, phase=0.4))
    with shf.Grid(nx, ny, 1.0, FP64) as g:
        g.set_params(kappa=2.0, gdot=s_gdot, dt=0.01)
        g.set_fields(phi)
        g.set_step(37)
        _, _, s, _ = g.get_time()
        G, L = g.gradient_tensor()
    num = np.zeros((2, 2))
    for m, n, a in ((2, 1, A), (-1, 3, B)):
        qx, qy = 2 * math.pi * m / nx, 2 * math.pi * n / ny
        q = np.array([qx, qy - s * qx])
        num += a * a / 2 * np.outer(q, q)
    want = num / (c * c + (A * A + B * B) / 2)
    assert np.allclose(G, [want[0, 0], want[0, 1], want[1, 1]], rtol=1e-13, atol=1e-15)
    ev = np.linalg.eigvalsh(want)
    assert np.allclose(L, [1 / (math.sqrt(2.0) * ev[0]), 1 / (math.sqrt(2.0) * ev[1])], rtol=1e-12)


# --------------------------------------------------------------- error paths

def test_error_paths():
    with shf.Grid(32, 32, 1.0, FP32) as g:
        with pytest.raises(shf.ShfError) as e:
            g.step(1)
        assert e.value.code == shf.SHF_ESTATE
        for bad in (dict(kappa=0.0), dict(M=-1.0), dict(eta=0.0), dict(dt=0.0), dict(rho=-1.0),
                    dict(gdot=float("nan")), dict(a=float("inf"))):
            with pytest.raises(shf.ShfError) as e:
                g.set_params(**bad)
            assert e.value.code == shf.SHF_EINVAL
        g.set_params()
        phi = inputs.quench_noise(32, 32, 0)
        phi[5, 7] = np.nan
        g.set_fields(phi)
        g.step(3)
        with pytest.raises(shf.ShfError) as e:
            g.sync()
        assert e.value.code == shf.SHF_ENONFINITE
        with pytest.raises(shf.ShfError) as e:
            g.mass()
        assert e.value.code == shf.SHF_ENONFINITE
        # the grid stays usable after the error
        g.set_fields(inputs.quench_noise(32, 32, 0))
        g.step(3)
        g.sync()


def test_bound_torch_buffers_give_identical_results():
    nx = ny = 64
    p = oracle.Params(rho=1.0, gdot=0.03, dt=0.01)
    fields = rough_state(nx, ny, 51)
    ref = gpu_run(nx, ny, FP32, p, fields, 0, 20)
    bufs = [torch.zeros((ny, nx), dtype=torch.float32, device="cuda") for _ in range(3)]
    stream = torch.cuda.Stream()
    with shf.Grid(nx, ny, 1.0, FP32, stream=stream) as g:
        g.set_params(p.a, p.b, p.kappa, p.M, p.eta, p.rho, p.gdot, p.dt)
        g.set_fields(*fields)
        g.bind_device_fields(*bufs)
        g.step(20)
        g.sync()
        got = g.get_fields()
        stream.synchronize()
        assert np.array_equal(bufs[0].cpu().numpy().astype(np.float64), got[0])
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)


# ---------------------------------------------------------- arithmetic peaks

def test_fma_peak_is_plausible_and_checks_arguments():
    """The measured FMA rates lie between a tenth of and just above what the
    SM count and clock allow (128 FP32 FMA lanes per SM per clock), and FP64
    runs below FP32."""
    props = torch.cuda.get_device_properties(0)
    clock_hz = 2.1e9
    nominal32 = props.multi_processor_count * 128 * 2 * clock_hz
    f32 = shf.shf_fma_peak(FP32, 0)
    f64 = shf.shf_fma_peak(FP64, 0)
    assert 0.1 * nominal32 < f32 < 1.05 * nominal32, f"{f32:.3e} vs {nominal32:.3e}"
    assert 0 < f64 < f32
    for prec, dev in ((7, 0), (FP32, -1), (FP32, torch.cuda.device_count())):
        with pytest.raises(shf.ShfError) as e:
            shf.shf_fma_peak(prec, dev)
        assert e.value.code == shf.SHF_EINVAL
