"""Floor of the non-stiff Rusanov coefficient (dg_phys.lambda_min, not in
the paper) through the C ABI: explicit rates and whole steps against the
oracle with the same floor, the FP32 perturbation form, graph mode."""
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


def relerr(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def case(name):
    if name == "2d_nc":
        return I.box_mesh((9, 4), (9e3, 4e3), refine_level=lambda c: 1 if 2e3 < c[0] < 5e3 else 0), 2
    return I.box_mesh((5, 4, 3), (5e3, 4e3, 3e3), hill=dict(h0=300.0, a_c=1e3, xc=2.5e3, yc=2e3),
                      refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3 else 0), 3


def slow_state(disc, seed):
    """Nearly at rest (winds of ~0.5 m/s): the floor is active on most faces."""
    return I.perturb(I.stratified_state(disc.node_points(), wind=(0.4, -0.2, 0.1)), np.random.default_rng(seed),
                     rel=1e-3)


@pytest.mark.parametrize("name", ["2d_nc", "3d_hill_nc"])
def test_floor_rates_parity(D, ctx, name):
    mesh, r = case(name)
    disc = O.Discretisation(mesh, r)
    gm = D.Mesh(ctx, mesh, r)
    q = slow_state(disc, 3)
    Fns, Fs = O.explicit_rates(disc, q, O.Phys(f=1.2e-4, lambda_min=1.0))
    F0, _ = O.explicit_rates(disc, q, O.Phys(f=1.2e-4))
    assert np.abs(Fns - F0).max() > 1e-8 * np.abs(Fns).max()          # the floor acts
    fns, fs = gm.apply_explicit(D.make_phys(f=1.2e-4, lambda_min=1.0), dev(q.reshape(5, -1)))
    torch.cuda.synchronize()
    fns, fs = host(fns, Fns.shape), host(fs, (4,) + Fns.shape[1:])
    for k in range(5):
        assert relerr(fns[k], Fns[k]) < 1e-11, ("ns", k, relerr(fns[k], Fns[k]))
    for k in range(4):
        assert relerr(fs[k], Fs[k + 1]) < 1e-11, ("s", k)


def test_floor_step_parity(D, ctx):
    """10 steps of the 2D case with the floor: 1e-9 against the oracle."""
    mesh, r = case("2d_nc")
    disc = O.Discretisation(mesh, r)
    gm = D.Mesh(ctx, mesh, r)
    q = slow_state(disc, 5)
    ph = O.Phys(f=1e-4, lambda_min=1.0)
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=400)
    qd = dev(q.reshape(5, -1))
    dph = D.make_phys(f=1e-4, lambda_min=1.0)
    qo = q
    for _ in range(10):
        qo = O.imex_ark2_step(disc, ph, qo, 6.0, opts)
        gm.step(dph, qd, 6.0, picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=400)
    qg = host(qd, qo.shape)
    for k in range(5):
        assert relerr(qg[k], qo[k]) < 1e-9, (k, relerr(qg[k], qo[k]))


def test_floor_fp32_perturbation_rates(D, ctx):
    """DG_MIXED_EXPLICIT about a background at rest (the floor acts on both
    the full and the background coefficients): F' to FP32 accuracy."""
    mesh, r = case("3d_hill_nc")
    disc = O.Discretisation(mesh, r)
    gm = D.Mesh(ctx, mesh, r)
    qb = I.stratified_state(disc.node_points())
    q = I.perturb(I.stratified_state(disc.node_points(), wind=(0.4, -0.2, 0.1)), np.random.default_rng(11),
                  rel=1e-2)
    ph = O.Phys(f=1.2e-4, lambda_min=1.0)
    Fns, Fs = O.explicit_rates(disc, q, ph)
    Bns, Bs = O.explicit_rates(disc, qb, ph)
    gm.set_background(D.make_phys(f=1.2e-4, lambda_min=1.0), dev(qb.reshape(5, -1)))
    fns, fs = gm.apply_explicit(D.make_phys(f=1.2e-4, lambda_min=1.0, precision="mixed_explicit"),
                                dev(q.reshape(5, -1)))
    torch.cuda.synchronize()
    fns, fs = host(fns, Fns.shape), host(fs, (4,) + Fns.shape[1:])
    for k in range(5):
        dref = Fns[k] - Bns[k]
        assert np.abs((fns[k] - Bns[k]) - dref).max() < 2e-5 * np.abs(dref).max(), ("ns", k)
    for k in range(4):
        dref = Fs[k + 1] - Bs[k + 1]
        assert np.abs((fs[k] - Bs[k + 1]) - dref).max() < 2e-5 * np.abs(dref).max(), ("s", k)


def test_floor_graph_matches_host_and_rejects_negative(D, ctx):
    mesh, r = case("2d_nc")
    disc = O.Discretisation(mesh, r)
    q = slow_state(disc, 6)
    ga, gb = D.Mesh(ctx, mesh, r), D.Mesh(ctx, mesh, r)
    qa, qh = dev(q.reshape(5, -1)), dev(q.reshape(5, -1))
    ph = D.make_phys(f=1e-4, lambda_min=1.0)
    opts = dict(picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=400)
    for _ in range(3):
        ga.step(ph, qa, 6.0, graph=True, **opts)
        gb.step(ph, qh, 6.0, **opts)
    assert relerr(host(qa, q.shape), host(qh, q.shape)) < 1e-10
    with pytest.raises(D.DGError):
        gb.step(D.make_phys(lambda_min=-1.0), qh, 6.0, **opts)
