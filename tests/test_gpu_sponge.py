"""Rayleigh damping layers (Section 4, eq. damping) through the C ABI:
explicit rates and whole steps against the oracle, graph mode against the
host-driven step, and switching the layers off."""
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


CASES = {
    # mesh, degree, layers (lam_bar, z_b, z_t, x_layers, y_layers)
    "2d_nc": (lambda: I.box_mesh((9, 4), (9e3, 4e3), refine_level=lambda c: 1 if 2e3 < c[0] < 5e3 else 0), 2,
              (0.04, 2e3, 4e3, (0.0, 9e3, 2e3), None)),
    "3d_hill_nc": (lambda: I.box_mesh((5, 4, 3), (5e3, 4e3, 3e3), hill=dict(h0=300.0, a_c=1e3, xc=2.5e3, yc=2e3),
                                      refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3 else 0), 3,
                   (0.05, 1.5e3, 3e3, (0.0, 5e3, 1e3), (0.0, 4e3, 1e3))),
}


def setup(D, ctx, name, seed=7):
    build, r, lay = CASES[name]
    mesh = build()
    disc = O.Discretisation(mesh, r)
    gm = D.Mesh(ctx, mesh, r)
    pts = disc.node_points()
    qb = I.stratified_state(pts, wind=(8.0, -3.0, 0.0))
    q = I.perturb(I.stratified_state(pts, wind=(8.0, -3.0, 1.0)), np.random.default_rng(seed), rel=2e-2)
    lam_bar, z_b, z_t, xl, yl = lay
    sp = O.Sponge(lam_bar=lam_bar, z_b=z_b, z_t=z_t, x_layers=xl, y_layers=yl, q_bar=qb)
    gm.set_sponge(dev(qb.reshape(5, -1)), lambda_bar=lam_bar, z_b=z_b, z_t=z_t, x_layers=xl, y_layers=yl)
    return mesh, r, disc, gm, q, qb, sp


@pytest.mark.parametrize("name", list(CASES))
def test_sponge_rates_parity(D, ctx, name):
    mesh, r, disc, gm, q, qb, sp = setup(D, ctx, name)
    Fns, Fs = O.explicit_rates(disc, q, O.Phys(f=1.2e-4, sponge=sp))
    F0, _ = O.explicit_rates(disc, q, O.Phys(f=1.2e-4))
    assert np.abs(Fns - F0).max() > 1e-6 * np.abs(Fns).max()       # the layers do act here
    fns, fs = gm.apply_explicit(D.make_phys(f=1.2e-4), dev(q.reshape(5, -1)))
    torch.cuda.synchronize()
    fns, fs = host(fns, Fns.shape), host(fs, (4,) + Fns.shape[1:])
    for k in range(5):
        assert relerr(fns[k], Fns[k]) < 1e-11, ("ns", k, relerr(fns[k], Fns[k]))
    for k in range(4):
        assert relerr(fs[k], Fs[k + 1]) < 1e-11, ("s", k)
    # switched off: the rates without layers
    gm.set_sponge(None)
    g0, _ = gm.apply_explicit(D.make_phys(f=1.2e-4), dev(q.reshape(5, -1)))
    assert relerr(host(g0, F0.shape), F0) < 1e-11


@pytest.mark.parametrize("variant", ["R2", "R1"])
def test_sponge_step_parity(D, ctx, variant):
    """10 steps of the 2D case with strong layers (lambda_bar dt = 1.2 as in
    the paper) against the oracle: 1e-9 relative max-norm."""
    mesh, r, disc, gm, q, qb, sp = setup(D, ctx, "2d_nc")
    dt = 6.0
    sp.lam_bar = 1.2 / dt
    lay = CASES["2d_nc"][2]
    gm.set_sponge(dev(qb.reshape(5, -1)), lambda_bar=sp.lam_bar, z_b=lay[1], z_t=lay[2], x_layers=lay[3])
    ph = O.Phys(f=1e-4, variant=variant, sponge=sp)
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=400)
    qd = dev(q.reshape(5, -1))
    dph = D.make_phys(f=1e-4, variant=variant)
    qo = q
    for _ in range(10):
        qo = O.imex_ark2_step(disc, ph, qo, dt, opts)
        gm.step(dph, qd, dt, picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=400)
    qg = host(qd, qo.shape)
    for k in range(5):
        assert relerr(qg[k], qo[k]) < 1e-9, (k, relerr(qg[k], qo[k]))
        assert relerr(qg[k] - q[k], qo[k] - q[k]) < 1e-6


def test_sponge_graph_mode_matches_host(D, ctx):
    """The device-driven step carries the damping pass, and switching the
    layers off re-captures the step."""
    mesh, r, disc, gm, q, qb, sp = setup(D, ctx, "3d_hill_nc")
    _, _, _, gh, _, _, _ = setup(D, ctx, "3d_hill_nc")
    ph = D.make_phys(f=1e-4)
    opts = dict(picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=400)
    qg, qh = dev(q.reshape(5, -1)), dev(q.reshape(5, -1))
    for _ in range(2):
        gm.step(ph, qg, 2.0, graph=True, **opts)
        gh.step(ph, qh, 2.0, **opts)
    assert relerr(host(qg, q.shape), host(qh, q.shape)) < 1e-10
    gm.set_sponge(None)
    gh.set_sponge(None)
    for _ in range(2):
        gm.step(ph, qg, 2.0, graph=True, **opts)
        gh.step(ph, qh, 2.0, **opts)
    assert relerr(host(qg, q.shape), host(qh, q.shape)) < 1e-10


def test_sponge_rejects_bad_layers(D, ctx):
    mesh, r, disc, gm, q, qb, sp = setup(D, ctx, "2d_nc")
    qbd = dev(qb.reshape(5, -1))
    with pytest.raises(D.DGError):
        gm.set_sponge(qbd, lambda_bar=0.1, z_b=3e3, z_t=2e3)
    with pytest.raises(D.DGError):
        gm.set_sponge(qbd, lambda_bar=0.1, z_b=1e3, z_t=2e3, x_layers=(0.0, 9e3, 0.0))


def test_sponge_with_fp32_increments(D, ctx):
    """DG_MIXED_EXPLICIT without a background evaluates the later stages'
    rates as FP32 increments; the damping pass follows those too: 3 steps
    stay within the FP32 error level (1e-4 relative to the change) of the
    FP64 oracle with the layers."""
    mesh, r, disc, gm, q, qb, sp = setup(D, ctx, "2d_nc")
    ph = O.Phys(f=1e-4, sponge=sp)
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=400)
    qd = dev(q.reshape(5, -1))
    dph = D.make_phys(f=1e-4, precision="mixed_explicit")
    qo = q
    for _ in range(3):
        qo = O.imex_ark2_step(disc, ph, qo, 6.0, opts)
        gm.step(dph, qd, 6.0, picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=2000,
                gmres_inner_rtol=1e-4)
    qg = host(qd, qo.shape)
    for k in range(5):
        assert relerr(qg[k] - q[k], qo[k] - q[k]) < 1e-4, (k, relerr(qg[k] - q[k], qo[k] - q[k]))
