"""Far-field faces (the non-reflecting top of Section 4.3, read as a face
whose outer state is a given background state) on the GPU against the
oracle (`set_far_state`, `far_affine`): explicit rates, the Schur operator,
its right-hand side and the velocity recovery with the outer data moved to
the right-hand sides, and whole steps.  Bars: 1e-11 per apply, 1e-9 after
the steps."""
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


def relerr(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


def to_dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def from_dev(t, shape):
    return t.detach().cpu().numpy().reshape(shape)


def top_far(mesh):
    return I.with_boundary(mesh, (2 * mesh.dim - 1,), I.BC_FARFIELD)


def top_bottom_far(mesh):
    d = mesh.dim
    return I.with_boundary(mesh, (2 * (d - 1), 2 * (d - 1) + 1), I.BC_FARFIELD)


CASES = {
    "2d_r2_top": (lambda: top_far(I.box_mesh((7, 3), (7e3, 3e3))), 2),
    "2d_r3_nc_topbottom": (lambda: top_bottom_far(I.box_mesh((6, 4), (6e3, 4e3),
                                                             refine_level=lambda c: 1 if c[0] < 2e3 else 0)), 3),
    "3d_r2_hill_nc_topbottom": (lambda: top_bottom_far(I.box_mesh(
        (4, 3, 3), (4e3, 3e3, 3e3), hill=dict(h0=250.0, a_c=1e3, xc=2e3, yc=1.5e3),
        refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3 else 0)), 2),
    "3d_r3_top": (lambda: top_far(I.box_mesh((3, 3, 2), (3e3, 3e3, 2e3))), 3),
}


def make_case(D, ctx, name, seed=0):
    build_mesh, r = CASES[name]
    mesh = build_mesh()
    disc = O.Discretisation(mesh, r)
    gm = D.Mesh(ctx, mesh, r)
    X = disc.node_points()
    rng = np.random.default_rng(seed)
    q = I.perturb(I.stratified_state(X, wind=(8.0, -3.0, 1.5)), rng, rel=2e-2)
    qfar = I.perturb(I.stratified_state(X, wind=(10.0, 2.0, -1.0)), rng, rel=1e-2)
    disc.set_far_state(qfar)
    gm.set_far_state(to_dev(qfar.reshape(5, -1)))
    return mesh, disc, gm, q, qfar


def dev_coeffs(D, cf):
    t = (to_dev(cf.rho.reshape(-1)), to_dev(cf.p_lag.reshape(-1)), to_dev(cf.u_lag.reshape(3, -1)))
    return t, D.Mesh.coeffs(*t, cf.adt)


@pytest.mark.parametrize("name", list(CASES))
def test_far_explicit_parity(D, ctx, name):
    mesh, disc, gm, q, _ = make_case(D, ctx, name)
    Fns, Fs = O.explicit_rates(disc, q, O.Phys(f=1.2e-4))
    fns, fs = gm.apply_explicit(D.make_phys(f=1.2e-4), to_dev(q.reshape(5, -1)))
    fns = from_dev(fns, Fns.shape)
    fs = from_dev(fs, (4,) + Fns.shape[1:])
    for k in range(5):
        assert relerr(fns[k], Fns[k]) < 1e-11, (k, relerr(fns[k], Fns[k]))
    for k in range(4):
        assert relerr(fs[k], Fs[k + 1]) < 1e-11, (k, relerr(fs[k], Fs[k + 1]))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("variant,penalty", [("R2", True), ("R1", True), ("R2", False)])
def test_far_schur_operators(D, ctx, name, variant, penalty):
    """Linear Schur operator (inner halves only), then the right-hand side and
    the recovery with the outer data b_far, g_far moved to them."""
    mesh, disc, gm, q, _ = make_case(D, ctx, name, seed=1)
    rng = np.random.default_rng(3)
    u, p = O.nodal_primitives(q, 1.4)
    cf = O.StageCoeffs(rho=q[0], p_lag=p, u_lag=u * (1 + 1e-2 * rng.standard_normal(u.shape)), adt=2.5)
    ph = O.Phys(f=1.1e-4, variant=variant, penalty=penalty)
    dph = D.make_phys(f=1.1e-4, variant=variant, penalty=penalty)
    keep, dcf = dev_coeffs(D, cf)
    x = p * (1 + 1e-2 * rng.standard_normal(p.shape))
    ref = O.schur_apply(disc, cf, ph, x)
    for stage in ((0, 1), (1, 0)):
        gm.set_fused_stage(*stage)
        y = from_dev(gm.apply_implicit(dph, dcf, to_dev(x.reshape(-1))), ref.shape)
        assert relerr(y, ref) < 1e-11, (stage, relerr(y, ref))
        assert relerr(y - x, ref - x) < 1e-9
    mhat = q[1:4] * (1 + 1e-3 * rng.standard_normal(q[1:4].shape))
    ehat = q[4] * (1 + 1e-4 * rng.standard_normal(q[4].shape))
    f_w = disc.vol_weak(disc.at_quad(mhat))
    g_w = disc.vol_weak(disc.at_quad(ehat))
    fb, gb = O.far_affine(disc, cf, ph)
    assert np.abs(fb).max() > 0 and np.abs(gb).max() > 0
    rref = O.schur_rhs(disc, cf, ph, f_w - fb, g_w - gb)
    rhs = from_dev(gm.schur_rhs(dph, dcf, to_dev(mhat.reshape(3, -1)), to_dev(ehat.reshape(-1))), rref.shape)
    assert relerr(rhs, rref) < 1e-11, relerr(rhs, rref)
    uref = O.recover_velocity(disc, cf, ph, f_w - fb, x)
    ug = from_dev(gm.recover_velocity(dph, dcf, to_dev(mhat.reshape(3, -1)), to_dev(x.reshape(-1))), uref.shape)
    for c in range(3):
        if np.abs(uref[c]).max() > 0:
            assert relerr(ug[c], uref[c]) < 1e-10, (c, relerr(ug[c], uref[c]))


@pytest.mark.parametrize("name", ["2d_r2_top", "3d_r2_hill_nc_topbottom"])
@pytest.mark.parametrize("variant", ["R1", "R2"])
def test_far_steps_match_oracle(D, ctx, name, variant):
    mesh, disc, gm, q, _ = make_case(D, ctx, name, seed=2)
    ph = O.Phys(f=1e-4, variant=variant)
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-13, gmres_restart=40, gmres_maxit=2000)
    qd = to_dev(q.reshape(5, -1)).contiguous()
    dph = D.make_phys(f=1e-4, variant=variant)
    qo = q
    for _ in range(4):
        qo = O.imex_ark2_step(disc, ph, qo, 2.0, opts)
        gm.step(dph, qd, 2.0, picard_fixed=2, gmres_rtol=1e-13, gmres_restart=40, gmres_maxit=2000)
    qg = from_dev(qd, qo.shape)
    for k in range(5):
        assert relerr(qg[k], qo[k]) < 1e-9, (k, relerr(qg[k], qo[k]))
    # the same steps as one graph launch each, and in mixed precision
    qd2 = to_dev(q.reshape(5, -1)).contiguous()
    qd3 = to_dev(q.reshape(5, -1)).contiguous()
    for _ in range(4):
        gm.step(dph, qd2, 2.0, picard_fixed=2, gmres_rtol=1e-13, gmres_restart=40, gmres_maxit=2000, graph=True)
        gm.step(D.make_phys(f=1e-4, variant=variant, precision="mixed"), qd3, 2.0, picard_fixed=2,
                gmres_rtol=1e-12, gmres_restart=40, gmres_maxit=2000, gmres_inner_rtol=1e-4)
    for k in range(5):
        assert relerr(from_dev(qd2, qo.shape)[k], qo[k]) < 1e-9
        assert relerr(from_dev(qd3, qo.shape)[k], qo[k]) < 1e-7
    # and with the vmults in pairs of FP32 numbers (FP64 GMRES); momentum
    # against the momentum vector's scale, as in the pair tests
    qd4 = to_dev(q.reshape(5, -1)).contiguous()
    for _ in range(4):
        gm.step(D.make_phys(f=1e-4, variant=variant, precision="pairs"), qd4, 2.0, picard_fixed=2,
                gmres_rtol=1e-13, gmres_restart=40, gmres_maxit=2000)
    q4 = from_dev(qd4, qo.shape)
    mscale = np.abs(qo[1:4]).max()
    for k in range(5):
        scale = mscale if 1 <= k <= 3 else np.abs(qo[k]).max()
        assert np.abs(q4[k] - qo[k]).max() / scale < 1e-9, k


@pytest.mark.parametrize("name", list(CASES))
def test_far_pairs_vmult(D, ctx, name):
    """The pair vmult on meshes with far-field faces (every schedule it
    takes), at the FP64 bar."""
    mesh, disc, gm, q, _ = make_case(D, ctx, name, seed=3)
    rng = np.random.default_rng(5)
    u, p = O.nodal_primitives(q, 1.4)
    cf = O.StageCoeffs(rho=q[0], p_lag=p, u_lag=u * (1 + 1e-2 * rng.standard_normal(u.shape)), adt=2.5)
    keep, dcf = dev_coeffs(D, cf)
    x = p * (1 + 1e-2 * rng.standard_normal(p.shape))
    for penalty in (True, False):
        ref = O.schur_apply(disc, cf, O.Phys(f=1.1e-4, penalty=penalty), x)
        dph = D.make_phys(f=1.1e-4, penalty=penalty, precision="pairs")
        for stage in (0, 1, 2):
            gm.set_fused_stage(1, 1, stage)
            y = from_dev(gm.apply_implicit(dph, dcf, to_dev(x.reshape(-1))), ref.shape)
            assert relerr(y, ref) < 1e-11, (penalty, stage, relerr(y, ref))
            assert relerr(y - x, ref - x) < 1e-9


def test_uniform_flow_through_far_boundaries_is_steady(D, ctx):
    """GPU form of the oracle pin: a uniform flow crossing far-field top and
    bottom with the outer state equal to it stays steady through whole
    steps (g = f = 0)."""
    mesh = top_bottom_far(I.box_mesh((3, 3, 3), (3e3, 3e3, 2e3), hill=dict(h0=300.0, a_c=0.8e3, xc=1.5e3,
                                                                            yc=1.5e3),
                                     refine_level=lambda c: 1 if c[0] < 1e3 and c[2] < 700 else 0))
    gm = D.Mesh(ctx, mesh, 2)
    n = gm.N
    u = np.array([8.0, -3.0, 2.5])
    rho, p = 1.1, 9.0e4
    q = np.zeros((5, n))
    q[0] = rho
    q[1:4] = rho * u[:, None]
    q[4] = p / 0.4 + 0.5 * rho * (u @ u)
    qd = to_dev(q)
    gm.set_far_state(qd)
    fns, fs = gm.apply_explicit(D.make_phys(f=0.0, g=0.0), qd)
    assert fns.abs().max().item() < 1e-9 and fs.abs().max().item() < 1e-9
    for variant in ("R1", "R2"):
        qs = qd.clone()
        for _ in range(2):
            gm.step(D.make_phys(f=0.0, g=0.0, variant=variant), qs, 5.0, picard_fixed=2, gmres_rtol=1e-13)
        qs = qs.cpu().numpy()
        for k in range(5):
            assert np.abs(qs[k] - q[k]).max() <= 1e-9 * max(np.abs(q[k]).max(), 1.0), (variant, k)


def test_far_faces_need_an_outer_state(D, ctx):
    mesh = top_far(I.box_mesh((3, 2), (3e3, 2e3)))
    gm = D.Mesh(ctx, mesh, 1)
    q = to_dev(np.ones((5, gm.N)))
    with pytest.raises(D.DGError) as ei:
        gm.apply_explicit(D.make_phys(), q)
    assert ei.value.status == -1 and "far_state" in str(ei.value)
