"""Gauss-Lobatto nodes on the GPU against the oracle's Gauss-Lobatto path.

The library evaluates every operator in the Gauss-Legendre nodal basis of
the same polynomials with the same quadrature and changes basis per cell on
the way in and out (the GLL inverse mass S^{-1} W^{-1} S^{-T} of Section 3.1
becomes the GL inverse mass followed by G^{-1}); the oracle assembles dense
GLL mass matrices, interpolation and inverses instead.  Bars as for the
Gauss-Legendre path: 1e-11 per apply, 1e-9 after 10 steps."""
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


CASES = {
    "2d_r2": (lambda: I.box_mesh((7, 3), (21e3, 6e3)), 2),
    "2d_r3_nc": (lambda: I.box_mesh((6, 4), (6e3, 4e3), refine_level=lambda c: 1 if 2e3 < c[0] < 4e3 else 0), 3),
    "3d_r2_hill_nc": (lambda: I.box_mesh((4, 3, 3), (4e3, 3e3, 3e3), hill=dict(h0=250.0, a_c=1e3, xc=2e3, yc=1.5e3),
                                         refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3 else 0), 2),
    "3d_r1": (lambda: I.box_mesh((3, 4, 2), (3e3, 4e3, 2e3)), 1),
}


def make_case(D, ctx, name, seed=0):
    build_mesh, r = CASES[name]
    mesh = build_mesh()
    disc = O.Discretisation(mesh, r, node_set="gll")
    gm = D.Mesh(ctx, mesh, r, node_set=D.DG_NODES_GLL)
    q = I.perturb(I.stratified_state(disc.node_points(), wind=(8.0, -3.0, 1.0)), np.random.default_rng(seed),
                  rel=2e-2)
    return mesh, disc, gm, q


def dev_coeffs(D, cf):
    t = (to_dev(cf.rho.reshape(-1)), to_dev(cf.p_lag.reshape(-1)), to_dev(cf.u_lag.reshape(3, -1)))
    return t, D.Mesh.coeffs(*t, cf.adt)


@pytest.mark.parametrize("name", list(CASES))
def test_gll_node_coords_and_explicit(D, ctx, name):
    mesh, disc, gm, q = make_case(D, ctx, name)
    xyz = from_dev(gm.node_coords(), (disc.d, disc.E, disc.Np))
    assert relerr(xyz, np.moveaxis(disc.node_points(), -1, 0)) < 1e-14
    Fns, Fs = O.explicit_rates(disc, q, O.Phys(f=1.2e-4))
    fns, fs = gm.apply_explicit(D.make_phys(f=1.2e-4), to_dev(q.reshape(5, -1)))
    fns = from_dev(fns, Fns.shape)
    fs = from_dev(fs, (4,) + Fns.shape[1:])
    for k in range(5):
        assert relerr(fns[k], Fns[k]) < 1e-11, (k, relerr(fns[k], Fns[k]))
    for k in range(4):
        assert relerr(fs[k], Fs[k + 1]) < 1e-11, (k, relerr(fs[k], Fs[k + 1]))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("variant", ["R1", "R2"])
def test_gll_schur_operators(D, ctx, name, variant):
    """Schur vmult (FP64, and FP32 within its rounding), right-hand side and
    velocity recovery in the GLL basis."""
    mesh, disc, gm, q = make_case(D, ctx, name, seed=3)
    rng = np.random.default_rng(9)
    u, p = O.nodal_primitives(q, 1.4)
    cf = O.StageCoeffs(rho=q[0], p_lag=p, u_lag=u * (1 + 1e-2 * rng.standard_normal(u.shape)), adt=2.5)
    ph = O.Phys(f=1.1e-4, variant=variant)
    dph = D.make_phys(f=1.1e-4, variant=variant)
    keep, dcf = dev_coeffs(D, cf)
    x = p * (1 + 1e-2 * rng.standard_normal(p.shape))
    ref = O.schur_apply(disc, cf, ph, x)
    y = from_dev(gm.apply_implicit(dph, dcf, to_dev(x.reshape(-1))), ref.shape)
    assert relerr(y, ref) < 1e-11, relerr(y, ref)
    assert relerr(y - x, ref - x) < 1e-9
    y32 = from_dev(gm.apply_implicit(D.make_phys(f=1.1e-4, variant=variant, precision="mixed"), dcf,
                                     to_dev(x.reshape(-1))), ref.shape)
    assert relerr(y32 - x, ref - x) < 1e-4
    # in pairs of FP32 numbers: the FP64 bar
    ydf = from_dev(gm.apply_implicit(D.make_phys(f=1.1e-4, variant=variant, precision="pairs"), dcf,
                                     to_dev(x.reshape(-1))), ref.shape)
    assert relerr(ydf, ref) < 1e-11, relerr(ydf, ref)
    assert relerr(ydf - x, ref - x) < 1e-9
    mhat = q[1:4] * (1 + 1e-3 * rng.standard_normal(q[1:4].shape))
    ehat = q[4] * (1 + 1e-4 * rng.standard_normal(q[4].shape))
    f_w = disc.vol_weak(disc.at_quad(mhat))
    g_w = disc.vol_weak(disc.at_quad(ehat))
    rref = O.schur_rhs(disc, cf, ph, f_w, g_w)
    rhs = from_dev(gm.schur_rhs(dph, dcf, to_dev(mhat.reshape(3, -1)), to_dev(ehat.reshape(-1))), rref.shape)
    assert relerr(rhs, rref) < 1e-11, relerr(rhs, rref)
    uref = O.recover_velocity(disc, cf, ph, f_w, x)
    ug = from_dev(gm.recover_velocity(dph, dcf, to_dev(mhat.reshape(3, -1)), to_dev(x.reshape(-1))), uref.shape)
    for c in range(3):
        if np.abs(uref[c]).max() > 0:
            assert relerr(ug[c], uref[c]) < 1e-10, (c, relerr(ug[c], uref[c]))


@pytest.mark.parametrize("precision", ["fp64", "mixed", "pairs"])
@pytest.mark.parametrize("nx", [20, 100])
def test_gll_steps_match_oracle(D, ctx, precision, nx):
    """Ten ARK2 steps of the 2D inertia-gravity wave (periodic 300 km x 10
    km channel, walls top and bottom, degree 2 on 3 x 3 Gauss-Lobatto nodes,
    dt = 12 s), on its full 100 x 5 mesh and a reduced 20 x 5 one: the fixed
    Picard count and tight GMRES make the two paths take the same
    iterations."""
    case = I.igw2d_case(nx=nx, nz=5)
    mesh, r = case["mesh"], case["degree"]
    disc = O.Discretisation(mesh, r, node_set="gll")
    gm = D.Mesh(ctx, mesh, r, node_set=D.DG_NODES_GLL)
    q = I.stratified_state(disc.node_points(), **case["state_params"])
    q = I.perturb(q, np.random.default_rng(5), rel=1e-4)
    ph = O.Phys(f=case["f"])
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-13, gmres_restart=40, gmres_maxit=2000)
    qd = to_dev(q.reshape(5, -1)).contiguous()
    dph = D.make_phys(f=case["f"], precision=precision)
    # mixed: FP64 refinement to 1e-12 around FP32 inner solves
    extra = {"mixed": dict(gmres_inner_rtol=1e-4, gmres_rtol=1e-12),
             "pairs": dict(gmres_rtol=1e-12)}.get(precision, dict(gmres_rtol=1e-13))
    qo = q
    for _ in range(10):
        qo = O.imex_ark2_step(disc, ph, qo, case["dt"], opts)
        gm.step(dph, qd, case["dt"], picard_fixed=2, gmres_restart=40, gmres_maxit=2000, **extra)
    qg = from_dev(qd, qo.shape)
    # FP64: the step parity bar; mixed: FP32 inner solves under FP64
    # refinement to 1e-12 leave relative errors of a few 1e-9 in the small
    # vertical momentum (itself a perturbation field, so far below 1e-6);
    # pairs: the FP64 bar with the momentum components against the momentum
    # vector's scale, as in the other pair tests
    bar = 1e-7 if precision == "mixed" else 1e-9
    mscale = np.abs(qo[1:4]).max()
    for k in range(5):
        if np.abs(qo[k]).max() > 0:
            scale = mscale if precision == "pairs" and 1 <= k <= 3 else np.abs(qo[k]).max()
            err = np.abs(qg[k] - qo[k]).max() / scale
            assert err < bar, (k, err)


def test_gll_unsupported_paths_say_so(D, ctx):
    mesh, disc, gm, q = make_case(D, ctx, "2d_r2")
    qd = to_dev(q.reshape(5, -1)).contiguous()
    with pytest.raises(D.DGError) as ei:
        gm.step(D.make_phys(), qd, 1.0, graph=True)
    assert ei.value.status == -2
    with pytest.raises(D.DGError) as ei:
        gm.step(D.make_phys(), qd, 1.0, gmres_precond=True)
    assert ei.value.status == -2
    with pytest.raises(D.DGError) as ei:
        gm.set_sponge(qd, lambda_bar=0.1, z_b=1e3, z_t=6e3)
    assert ei.value.status == -2
