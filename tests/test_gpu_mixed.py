"""Mixed precision (DG_MIXED): FP32 Schur vmults inside FP64 iterative
refinement.  Checked against the FP64 oracle: the FP32 vmult to FP32
accuracy, the refined solve and whole steps to FP64-solver accuracy, and
the perturbation fields after 10 steps to <= 1e-6 relative L2."""
import numpy as np
import pytest

from oracle import dg_oracle as O
from paper_2605_29598_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    from paper_2605_29598_gb300 import build, dgimex
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return dgimex


@pytest.fixture(scope="module")
def ctx(D):
    return D.Context(0)


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t, shape):
    return t.cpu().numpy().reshape(shape)


def case(name):
    if name == "2d_nc":
        return I.box_mesh((9, 4), (9e3, 4e3), refine_level=lambda c: 1 if 2e3 < c[0] < 5e3 else 0), 2
    return I.box_mesh((5, 4, 3), (5e3, 4e3, 3e3), hill=dict(h0=300.0, a_c=1e3, xc=2.5e3, yc=2e3),
                      refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3 else 0), 3


def setup(D, ctx, name, seed):
    mesh, r = case(name)
    disc = O.Discretisation(mesh, r)
    gm = D.Mesh(ctx, mesh, r)
    q = I.perturb(I.stratified_state(disc.node_points(), wind=(8.0, -3.0, 1.0)),
                  np.random.default_rng(seed), rel=2e-2)
    return disc, gm, q


def coeffs(D, q, adt):
    u, p = O.nodal_primitives(q, 1.4)
    cf = O.StageCoeffs(rho=q[0], p_lag=p, u_lag=u, adt=adt)
    keep = (dev(q[0].reshape(-1)), dev(p.reshape(-1)), dev(u.reshape(3, -1)))
    return cf, keep, D.Mesh.coeffs(*keep, adt)


@pytest.mark.parametrize("name", ["2d_nc", "3d_hill_nc"])
def test_fp32_vmult_accuracy(D, ctx, name):
    disc, gm, q = setup(D, ctx, name, 1)
    cf, keep, dcf = coeffs(D, q, 3.0)
    ph = O.Phys(f=1.3e-4)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(cf.p_lag.shape) * 100.0          # a correction-sized vector
    ref = O.schur_apply(disc, cf, ph, x)
    y = host(gm.apply_implicit(D.make_phys(f=1.3e-4, precision="mixed"), dcf, dev(x.reshape(-1))),
             ref.shape)
    err = np.abs(y - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err
    assert err > 1e-12          # really computed in FP32


@pytest.mark.parametrize("name", ["2d_nc", "3d_hill_nc"])
def test_refined_solve_reaches_fp64_accuracy(D, ctx, name):
    disc, gm, q = setup(D, ctx, name, 2)
    cf, keep, dcf = coeffs(D, q, 2.0)
    ph = O.Phys(f=1.1e-4)
    rng = np.random.default_rng(4)
    b = O.schur_apply(disc, cf, ph, cf.p_lag * (1 + 1e-3 * rng.standard_normal(cf.p_lag.shape)))
    xr, its, rr, ok = O.gmres(lambda v: O.schur_apply(disc, cf, ph, v), b, cf.p_lag, rtol=1e-12,
                              restart=30, maxit=600)
    assert ok
    x = dev(cf.p_lag.reshape(-1))
    info = gm.gmres_solve(D.make_phys(f=1.1e-4, precision="mixed"), dcf, dev(b.reshape(-1)), x,
                          rtol=1e-12, restart=30, maxit=600, inner_rtol=1e-4)
    assert info.relres <= 1e-12 and info.refinements >= 1
    x = host(x, xr.shape)
    assert np.abs(x - xr).max() / np.abs(xr).max() < 1e-10


@pytest.mark.parametrize("name,steps,dt", [("2d_nc", 10, 6.0), ("3d_hill_nc", 3, 1.0)])
def test_mixed_steps_match_fp64_oracle(D, ctx, name, steps, dt):
    """Perturbation fields rho', theta', u', v, w (about the initial state)
    after the steps: relative L2 error vs the FP64 oracle <= 1e-6."""
    disc, gm, q = setup(D, ctx, name, 5)
    ph = O.Phys(f=1e-4)
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=400)
    qd = dev(q.reshape(5, -1))
    dph = D.make_phys(f=1e-4, precision="mixed")
    qo = q
    for _ in range(steps):
        qo = O.imex_ark2_step(disc, ph, qo, dt, opts)
        info = gm.step(dph, qd, dt, picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50,
                       gmres_maxit=2000, gmres_inner_rtol=1e-4)
        assert info.refinements_total > 0
    qg = host(qd, qo.shape)

    def fields(s):
        u, p = O.nodal_primitives(s, 1.4)
        theta = p / (287.0 * s[0]) * (1e5 / p) ** (0.4 / 1.4)
        return [s[0], theta, u[0], u[1], u[2]]

    f0, fg, fo = fields(q), fields(qg), fields(qo)
    for k in range(5):
        pert_o = fo[k] - f0[k]
        err = np.linalg.norm(fg[k] - fo[k]) / np.linalg.norm(pert_o)
        assert err < 1e-6, (k, err)
