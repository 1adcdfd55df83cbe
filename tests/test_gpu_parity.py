"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (stated for the FP64 path): 1e-11 relative max-norm per operator
apply, 1e-9 after 10 ARK2 steps.  Inputs are seeded synthetic states on
meshes that span several blocks of cells with ragged tails, 2:1 hanging
faces, walls, periodic pairs and terrain-following (curved) cells."""
import math

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
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def to_dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def from_dev(t, shape):
    return t.detach().cpu().numpy().reshape(shape)


def sheared(mesh, sx, sy=0.0):
    """The mesh with x += sx z (and y += sy z): cells are no longer
    terrain-following (x depends on the vertical reference coordinate), so
    the cell kernels take their general-metric path.  Periodic and wall
    faces stay matched."""
    v = mesh.vertices.copy()
    v[..., 0] += sx * v[..., -1]
    if mesh.dim == 3:
        v[..., 1] += sy * v[..., -1]
    return I.Mesh(dim=mesh.dim, vertices=v, int_faces=mesh.int_faces, hang_faces=mesh.hang_faces,
                  bdry_faces=mesh.bdry_faces, level=mesh.level, name=mesh.name + "_sheared")


CASES = {
    # name: (mesh builder, degree)
    "2d_r1": (lambda: I.box_mesh((7, 3), (7e3, 3e3)), 1),
    "2d_r2_nc": (lambda: I.box_mesh((9, 4), (9e3, 4e3),
                                    refine_level=lambda c: 1 if 2e3 < c[0] < 5e3 else 0), 2),
    "2d_r4_nc": (lambda: I.box_mesh((6, 3), (6e3, 3e3),
                                    refine_level=lambda c: 2 if c[0] < 1e3 and c[1] < 1e3 else 0), 4),
    "3d_r3_hill_nc": (lambda: I.box_mesh((5, 4, 3), (5e3, 4e3, 3e3),
                                         hill=dict(h0=300.0, a_c=1e3, xc=2.5e3, yc=2e3),
                                         refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3 else 0), 3),
    "3d_r2": (lambda: I.box_mesh((3, 5, 2), (3e3, 5e3, 2e3)), 2),
    "2d_r2_nc_sheared": (lambda: sheared(I.box_mesh((9, 4), (9e3, 4e3),
                                                    refine_level=lambda c: 1 if 2e3 < c[0] < 5e3 else 0), 0.3), 2),
    "3d_r3_hill_nc_sheared": (lambda: sheared(I.box_mesh((5, 4, 3), (5e3, 4e3, 3e3),
                                                         hill=dict(h0=300.0, a_c=1e3, xc=2.5e3, yc=2e3),
                                                         refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3
                                                         else 0), 0.2, -0.15), 3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_terrain_following_detection(D, ctx, name):
    """Box and Gal-Chen meshes take the terrain-following kernels (metric
    terms that vanish exactly are skipped); sheared meshes the general ones."""
    mesh, disc, gm, _ = make_case(D, ctx, name)
    assert gm.stats().terrain_following == (0 if name.endswith("sheared") else 1)


def make_case(D, ctx, name, seed=0):
    build_mesh, r = CASES[name]
    mesh = build_mesh()
    disc = O.Discretisation(mesh, r)
    gm = D.Mesh(ctx, mesh, r)
    rng = np.random.default_rng(seed)
    q = I.perturb(I.stratified_state(disc.node_points(), wind=(8.0, -3.0, 1.0)), rng, rel=2e-2)
    return mesh, disc, gm, q


@pytest.mark.parametrize("name", list(CASES))
def test_node_coords(D, ctx, name):
    mesh, disc, gm, _ = make_case(D, ctx, name)
    xyz = from_dev(gm.node_coords(), (disc.d, disc.E, disc.Np))
    ref = np.moveaxis(disc.node_points(), -1, 0)
    assert relerr(xyz, ref) < 1e-14


@pytest.mark.parametrize("name", list(CASES))
def test_explicit_parity(D, ctx, name):
    mesh, disc, gm, q = make_case(D, ctx, name)
    for f, g in ((1.2e-4, 9.81), (0.0, 0.0)):
        ph = O.Phys(f=f, g=g)
        Fns, Fs = O.explicit_rates(disc, q, ph)
        fns, fs = gm.apply_explicit(D.make_phys(f=f, g=g), to_dev(q.reshape(5, -1)))
        torch.cuda.synchronize()
        fns = from_dev(fns, Fns.shape)
        fs = from_dev(fs, (4,) + Fns.shape[1:])
        for k in range(5):
            assert relerr(fns[k], Fns[k]) < 1e-11, (name, "ns", k, relerr(fns[k], Fns[k]))
        for k in range(4):
            assert relerr(fs[k], Fs[k + 1]) < 1e-11, (name, "s", k, relerr(fs[k], Fs[k + 1]))
        assert np.abs(Fs[0]).max() == 0.0


def stage(disc, q, adt):
    u, p = O.nodal_primitives(q, 1.4)
    return O.StageCoeffs(rho=q[0], p_lag=p, u_lag=u, adt=adt)


def dev_coeffs(D, cf):
    t = (to_dev(cf.rho.reshape(-1)), to_dev(cf.p_lag.reshape(-1)), to_dev(cf.u_lag.reshape(3, -1)))
    return t, D.Mesh.coeffs(*t, cf.adt)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("variant,penalty", [("R2", True), ("R1", True), ("R2", False)])
def test_schur_vmult_parity(D, ctx, name, variant, penalty):
    mesh, disc, gm, q = make_case(D, ctx, name, seed=1)
    cf = stage(disc, q, adt=3.0)
    ph = O.Phys(f=1.3e-4, variant=variant, penalty=penalty)
    x = cf.p_lag * (1 + 1e-2 * np.random.default_rng(4).standard_normal(cf.p_lag.shape))
    ref = O.schur_apply(disc, cf, ph, x)
    keep, dcf = dev_coeffs(D, cf)
    y = gm.apply_implicit(D.make_phys(f=1.3e-4, variant=variant, penalty=penalty), dcf,
                          to_dev(x.reshape(-1)))
    torch.cuda.synchronize()
    y = from_dev(y, ref.shape)
    assert relerr(y, ref) < 1e-11, relerr(y, ref)
    # the operator minus identity carries the physics: check it on its own
    assert relerr(y - x, ref - x) < 1e-9, relerr(y - x, ref - x)


@pytest.mark.parametrize("name", ["2d_r2_nc", "3d_r3_hill_nc"])
@pytest.mark.parametrize("variant", ["R1", "R2"])
def test_schur_rhs_and_recovery_parity(D, ctx, name, variant):
    mesh, disc, gm, q = make_case(D, ctx, name, seed=2)
    rng = np.random.default_rng(6)
    cf = stage(disc, q, adt=2.0)
    cf.u_lag = cf.u_lag * (1 + 1e-2 * rng.standard_normal(cf.u_lag.shape))
    ph = O.Phys(f=1.1e-4, variant=variant)
    mhat = q[1:4] * (1 + 1e-3 * rng.standard_normal(q[1:4].shape))
    ehat = q[4] * (1 + 1e-4 * rng.standard_normal(q[4].shape))
    f_w = disc.vol_weak(disc.at_quad(mhat))
    g_w = disc.vol_weak(disc.at_quad(ehat))
    ref = O.schur_rhs(disc, cf, ph, f_w, g_w)
    keep, dcf = dev_coeffs(D, cf)
    dph = D.make_phys(f=1.1e-4, variant=variant)
    rhs = gm.schur_rhs(dph, dcf, to_dev(mhat.reshape(3, -1)), to_dev(ehat.reshape(-1)))
    torch.cuda.synchronize()
    rhs = from_dev(rhs, ref.shape)
    assert relerr(rhs, ref) < 1e-11, relerr(rhs, ref)
    p = cf.p_lag * (1 + 1e-3 * rng.standard_normal(cf.p_lag.shape))
    uref = O.recover_velocity(disc, cf, ph, f_w, p)
    u = gm.recover_velocity(dph, dcf, to_dev(mhat.reshape(3, -1)), to_dev(p.reshape(-1)))
    torch.cuda.synchronize()
    u = from_dev(u, uref.shape)
    for c in range(3):
        assert relerr(u[c], uref[c]) < 1e-10, (c, relerr(u[c], uref[c]))


@pytest.mark.parametrize("name", ["2d_r2_nc", "3d_r3_hill_nc"])
def test_gmres_parity(D, ctx, name):
    mesh, disc, gm, q = make_case(D, ctx, name, seed=3)
    cf = stage(disc, q, adt=2.0)
    ph = O.Phys(f=1.1e-4)
    rng = np.random.default_rng(9)
    b = O.schur_apply(disc, cf, ph, cf.p_lag * (1 + 1e-3 * rng.standard_normal(cf.p_lag.shape)))
    xr, its, rr, ok = O.gmres(lambda v: O.schur_apply(disc, cf, ph, v), b, cf.p_lag, rtol=1e-12,
                              restart=20, maxit=400)
    assert ok
    keep, dcf = dev_coeffs(D, cf)
    x = to_dev(cf.p_lag.reshape(-1))
    info = gm.gmres_solve(D.make_phys(f=1.1e-4), dcf, to_dev(b.reshape(-1)), x, rtol=1e-12,
                          restart=20, maxit=400)
    torch.cuda.synchronize()
    assert info.relres <= 1e-12
    x = from_dev(x, xr.shape)
    # both stop at relative residual 1e-12 along different rounding paths
    assert relerr(x, xr) < 1e-10, relerr(x, xr)
    assert abs(info.iters - its) <= max(2, its // 5)


def test_gmres_not_converged_returns_best_iterate(D, ctx):
    mesh, disc, gm, q = make_case(D, ctx, "2d_r2_nc", seed=3)
    cf = stage(disc, q, adt=50.0)
    keep, dcf = dev_coeffs(D, cf)
    rng = np.random.default_rng(1)
    b = to_dev(rng.standard_normal(disc.E * disc.Np))
    x = torch.zeros_like(b)
    info = gm.gmres_solve(D.make_phys(), dcf, b, x, rtol=1e-14, restart=5, maxit=3,
                          allow_not_converged=True)
    assert info.iters == 3 and 0 < info.relres < 1.0
    with pytest.raises(D.DGError) as ei:
        gm.gmres_solve(D.make_phys(), dcf, b, torch.zeros_like(b), rtol=1e-14, restart=5, maxit=3)
    assert ei.value.status == -4


@pytest.mark.parametrize("name,steps,variant,dt", [("2d_r2_nc", 10, "R2", 6.0),
                                                   ("2d_r1", 10, "R1", 6.0),
                                                   ("3d_r3_hill_nc", 3, "R2", 1.0)])
def test_step_parity(D, ctx, name, steps, variant, dt):
    mesh, disc, gm, q = make_case(D, ctx, name, seed=5)
    ph = O.Phys(f=1e-4, variant=variant)
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=400)
    qd = to_dev(q.reshape(5, -1))
    dph = D.make_phys(f=1e-4, variant=variant)
    qo = q
    for _ in range(steps):
        qo = O.imex_ark2_step(disc, ph, qo, dt, opts)
        gm.step(dph, qd, dt, picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=400)
    torch.cuda.synchronize()
    qg = from_dev(qd, qo.shape)
    for k in range(5):
        assert relerr(qg[k], qo[k]) < 1e-9, (k, relerr(qg[k], qo[k]))
    # the perturbation about the start carries the dynamics: compare it too
    for k in range(5):
        assert relerr(qg[k] - q[k], qo[k] - q[k]) < 1e-6, (k, relerr(qg[k] - q[k], qo[k] - q[k]))


def test_mesh_validation_errors(D, ctx):
    mesh = I.box_mesh((3, 2), (3.0, 2.0))
    bad = I.Mesh(dim=2, vertices=mesh.vertices, int_faces=mesh.int_faces[1:],
                 hang_faces=mesh.hang_faces, bdry_faces=mesh.bdry_faces)
    with pytest.raises(D.DGError) as ei:
        D.Mesh(ctx, bad, 2)
    assert ei.value.status == -1
    with pytest.raises(D.DGError) as ei:
        D.Mesh(ctx, mesh, 2, node_set=7)
    assert ei.value.status == -1
    flipped = mesh.vertices.copy()
    flipped[0] = flipped[0][[1, 0, 3, 2]]
    with pytest.raises(D.DGError) as ei:
        D.Mesh(ctx, I.Mesh(dim=2, vertices=flipped, int_faces=mesh.int_faces,
                           hang_faces=mesh.hang_faces, bdry_faces=mesh.bdry_faces), 2)
    assert ei.value.status == -1


@pytest.mark.parametrize("name", ["2d_r2_nc", "3d_r3_hill_nc"])
def test_autotuned_tiles_keep_parity(D, ctx, name):
    """Every tile multiplier and fused-vmult schedule the autotuner can pick
    gives the same results."""
    mesh, disc, gm, q = make_case(D, ctx, name, seed=7)
    gm.autotune("pairs")
    t64, t32, sched = gm.autotune("mixed")
    assert all(t in (1, 2, 4) for t in t64 + t32) and all(s in (0, 1, 2) for s in sched)
    Fns, Fs = O.explicit_rates(disc, q, O.Phys(f=1e-4))
    fns, fs = gm.apply_explicit(D.make_phys(f=1e-4), to_dev(q.reshape(5, -1)))
    assert relerr(from_dev(fns, Fns.shape), Fns) < 1e-11
    cf = stage(disc, q, adt=3.0)
    ref = O.schur_apply(disc, cf, O.Phys(f=1e-4), cf.p_lag)
    keep, dcf = dev_coeffs(D, cf)
    y = from_dev(gm.apply_implicit(D.make_phys(f=1e-4), dcf, to_dev(cf.p_lag.reshape(-1))),
                 ref.shape)
    assert relerr(y, ref) < 1e-11


@pytest.mark.parametrize("r", [1, 4])
def test_degree_extremes_3d(D, ctx, r):
    """Lowest and highest supported degree on a 3D 2:1 terrain mesh."""
    mesh = I.box_mesh((3, 2, 2), (3e3, 2e3, 2e3), hill=dict(h0=150.0, a_c=1e3, xc=1.5e3, yc=1e3),
                      refine_level=lambda c: 1 if c[0] < 1e3 else 0)
    disc = O.Discretisation(mesh, r)
    gm = D.Mesh(ctx, mesh, r)
    q = I.perturb(I.stratified_state(disc.node_points(), wind=(5.0, 1.0, 0.0)),
                  np.random.default_rng(r), rel=1e-2)
    Fns, Fs = O.explicit_rates(disc, q, O.Phys(f=1e-4))
    fns, fs = gm.apply_explicit(D.make_phys(f=1e-4), to_dev(q.reshape(5, -1)))
    assert relerr(from_dev(fns, Fns.shape), Fns) < 1e-11
    cf = stage(disc, q, adt=2.0)
    ref = O.schur_apply(disc, cf, O.Phys(f=1e-4), cf.p_lag)
    keep, dcf = dev_coeffs(D, cf)
    y = from_dev(gm.apply_implicit(D.make_phys(f=1e-4), dcf, to_dev(cf.p_lag.reshape(-1))), ref.shape)
    assert relerr(y, ref) < 1e-11


def test_fluid_at_rest_degenerate_lambda(D, ctx):
    """u = 0 everywhere: every Rusanov coefficient lambda is zero."""
    mesh, disc, gm, q = make_case(D, ctx, "2d_r2_nc", seed=8)
    q = q.copy()
    q[4] -= 0.5 * np.sum(q[1:4] ** 2, axis=0) / q[0]
    q[1:4] = 0.0
    Fns, Fs = O.explicit_rates(disc, q, O.Phys(f=1e-4))
    fns, fs = gm.apply_explicit(D.make_phys(f=1e-4), to_dev(q.reshape(5, -1)))
    assert relerr(from_dev(fs, (4,) + Fns.shape[1:]), Fs[1:]) < 1e-11
    assert np.abs(from_dev(fns, Fns.shape)).max() < 1e-12 * np.abs(Fs).max()
    cf = stage(disc, q, adt=3.0)
    ref = O.schur_apply(disc, cf, O.Phys(f=1e-4), cf.p_lag * 1.001)
    keep, dcf = dev_coeffs(D, cf)
    y = from_dev(gm.apply_implicit(D.make_phys(f=1e-4), dcf, to_dev(cf.p_lag.reshape(-1) * 1.001)),
                 ref.shape)
    assert relerr(y, ref) < 1e-11


def test_mesh_edge_cases_rejected(D, ctx):
    """Empty mesh, a missing subface of a 2:1 face, out-of-range indices."""
    import ctypes as C
    lib = D.load()
    v = np.zeros((0, 4, 2))
    d = D.MeshDesc(dim=2, degree=2, node_set=0, n_elem=0,
                   vertices=v.ctypes.data_as(C.POINTER(C.c_double)))
    h = C.c_void_p()
    assert lib.dg_mesh_create(ctx.h, C.byref(d), C.byref(h)) == -1
    mesh = I.box_mesh((4, 3), (4.0, 3.0), refine_level=lambda c: 1 if c[0] < 1 else 0)
    assert len(mesh.hang_faces) >= 2
    for bad in (
        I.Mesh(dim=2, vertices=mesh.vertices, int_faces=mesh.int_faces,
               hang_faces=mesh.hang_faces[1:], bdry_faces=mesh.bdry_faces),
        I.Mesh(dim=2, vertices=mesh.vertices,
               int_faces=np.vstack([mesh.int_faces[:-1], [[0, 1, mesh.n_elem, 0]]]),
               hang_faces=mesh.hang_faces, bdry_faces=mesh.bdry_faces)):
        with pytest.raises(D.DGError) as ei:
            D.Mesh(ctx, bad, 2)
        assert ei.value.status == -1


def test_binding_rejects_mis_sized_buffers(D, ctx):
    """Wrong lengths are refused by the binding before any launch: the state,
    the Schur vector, and coefficients built for another mesh."""
    import torch
    gm = D.Mesh(ctx, I.box_mesh((3, 2), (3e3, 2e3)), 2)
    N = gm.N
    opt = dict(dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        gm.apply_explicit(D.make_phys(), torch.ones((5, N - 1), **opt))
    cf = D.Mesh.coeffs(torch.ones(N, **opt), torch.full((N,), 1e5, **opt), torch.zeros((3, N), **opt), 1.0)
    with pytest.raises(ValueError):
        gm.apply_implicit(D.make_phys(), cf, torch.ones(N + 1, **opt))
    with pytest.raises(ValueError):
        D.Mesh.coeffs(torch.ones(N, **opt), torch.ones(N, **opt), torch.zeros((2, N), **opt), 1.0)
    small = D.Mesh.coeffs(torch.ones(N - 9, **opt), torch.ones(N - 9, **opt), torch.zeros((3, N - 9), **opt), 1.0)
    with pytest.raises(ValueError):
        gm.apply_implicit(D.make_phys(), small, torch.ones(N, **opt))
    y = gm.apply_implicit(D.make_phys(), cf, torch.full((N,), 1e5, **opt))
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()

