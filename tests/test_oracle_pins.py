"""Pins of the FP64 oracle against facts fixed by the paper and by
mathematics (closed forms, invariants, library routines, brute force).

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a transposed operand, a wrong node ordering) fails it."""
import math

import numpy as np
import pytest

from oracle import dg_oracle as O
from paper_2605_29598_gb300 import inputs as I


# ----------------------------------------------------------------------------
# time integrator (Section 3, Butcher tableau)
# ----------------------------------------------------------------------------

def test_tableau_order_conditions():
    a, at, b, c = O.ark2_tableau()
    assert abs(O.CHI - (2 - math.sqrt(2))) < 1e-16
    for A in (a, at):
        assert np.allclose(A.sum(axis=1), c, atol=1e-15)       # row sums = c
    assert abs(b.sum() - 1.0) < 1e-15                          # first order
    assert abs(b @ c - 0.5) < 1e-15                            # second order (fixes chi)
    assert np.allclose(at[2], b, atol=0)                       # stiffly accurate
    assert abs(at[1, 1] - at[2, 2]) == 0                       # singly diagonal
    # IMEX coupling conditions of order 2 with b = bt, c = ct
    assert abs(b @ (a @ np.ones(3)) - 0.5) < 1e-15
    assert abs(b @ (at @ np.ones(3)) - 0.5) < 1e-15


def ark2_amplification(z):
    """Stability function of the implicit tableau for y' = lambda y, z = lambda dt."""
    _, at, b, _ = O.ark2_tableau()
    y1 = 1.0
    y2 = (1 + at[1, 0] * z * y1) / (1 - at[1, 1] * z)
    y3 = (1 + at[2, 0] * z * y1 + at[2, 1] * z * y2) / (1 - at[2, 2] * z)
    return 1 + z * (b[0] * y1 + b[1] * y2 + b[2] * y3)


def test_tableau_l_stability_and_order():
    # L-stable: R(z) -> 0 like 1/z as z -> -infinity
    assert abs(ark2_amplification(-1e6)) < 1e-4
    assert abs(ark2_amplification(-1e6)) < 0.2 * abs(ark2_amplification(-1e5))
    for z in (1e-2, 1e-2j, -1e-2 + 5e-3j):
        # error of the stability function vs exp(z) is O(z^3)
        assert abs(ark2_amplification(z) - np.exp(z)) < 0.2 * abs(z) ** 3


# ----------------------------------------------------------------------------
# bases and quadrature
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_basis_and_quadrature(n):
    x, w = O.gauss_legendre01(n)
    for k in range(2 * n):                                     # exact to degree 2n-1
        assert abs(w @ x ** k - 1.0 / (k + 1)) < 1e-14
    for nodes in (x, O.gauss_lobatto01(n)):
        assert np.allclose(O.lagrange(nodes, nodes), np.eye(n), atol=1e-14)
        t = np.linspace(-0.2, 1.3, 7)
        for k in range(n):                                     # reproduces P_{n-1}
            assert np.allclose(O.lagrange(nodes, t) @ nodes ** k, t ** k, atol=1e-12)
            dk = k * t ** (k - 1) if k else 0 * t
            assert np.allclose(O.dlagrange(nodes, t) @ nodes ** k, dk, atol=1e-11)
    gll = O.gauss_lobatto01(n)
    assert gll[0] == 0.0 and gll[-1] == 1.0


# ----------------------------------------------------------------------------
# explicit operator
# ----------------------------------------------------------------------------

def _refine_corner(d):
    return lambda c: 1 if all(ci < 1.6 for ci in c) else 0


def _poly_state(disc, rng, u):
    d = disc.d
    X = disc.node_points()
    coef = rng.uniform(-1, 1, (disc.r + 1,) * d) * 0.05

    def val(X):
        v = np.ones(X.shape[:-1])
        for idx in np.ndindex(*coef.shape):
            t = coef[idx] * np.ones(X.shape[:-1])
            for a in range(d):
                t = t * X[..., a] ** idx[a]
            v = v + t
        return v

    def grad(X):
        g = np.zeros(X.shape)
        for idx in np.ndindex(*coef.shape):
            for b in range(d):
                if idx[b] == 0:
                    continue
                t = coef[idx] * idx[b] * np.ones(X.shape[:-1])
                for a in range(d):
                    t = t * X[..., a] ** (idx[a] - 1 if a == b else idx[a])
                g[..., b] += t
        return g

    rho = val(X)
    q = np.zeros((5,) + rho.shape)
    q[0] = rho
    for c in range(3):
        q[1 + c] = rho * u[c]
    q[4] = 2.0 / 0.4 + 0.5 * rho * (u @ u)
    ugr = sum(u[c] * grad(X)[..., b] for b, c in enumerate(disc.comp))
    return q, ugr


@pytest.mark.parametrize("d,r,refine,nodes", [
    (2, 1, False, "gl"), (2, 3, False, "gl"), (2, 2, True, "gl"), (2, 3, True, "gll"),
    (3, 1, True, "gl"), (3, 2, False, "gll"), (3, 3, True, "gl")])
def test_polynomial_exactness(d, r, refine, nodes):
    """Affine cells, rho in Q_r continuous, constant u and p: the non-stiff
    rates equal -(u.grad rho)(1, u, kappa) at the nodes and the stiff rates
    vanish (g = f = 0), on every cell with no wall face.  Pins cell terms,
    conforming and hanging face traces, normals and the lift."""
    cells = (4,) * d
    mesh = I.box_mesh(cells, (4.0,) * d, periodic=[False] * d,
                      refine_level=_refine_corner(d) if refine else None)
    if refine:
        assert len(mesh.hang_faces) > 0
    disc = O.Discretisation(mesh, r, nodes)
    u = np.array([0.3, -0.2, 0.5])
    q, ugr = _poly_state(disc, np.random.default_rng(3), u)
    Fns, Fs = O.explicit_rates(disc, q, O.Phys(f=0.0, g=0.0))
    inner = np.setdiff1d(np.arange(disc.E), mesh.bdry_faces[:, 0])
    exp = np.stack([-ugr] + [-ugr * u[c] for c in range(3)] + [-ugr * 0.5 * (u @ u)])
    assert np.abs(Fns[:, inner] - exp[:, inner]).max() < 1e-11
    assert np.abs(Fs[:, inner]).max() < 1e-10


def _random_state(disc, rng, wind=(5.0, 2.0, 1.0)):
    X = disc.node_points()
    q = I.stratified_state(X, wind=wind)
    return I.perturb(q, rng, rel=1e-2)


@pytest.mark.parametrize("d,refine,hill", [(2, False, False), (2, True, False),
                                           (3, True, True)])
def test_conservation(d, refine, hill):
    """Periodic horizontally, walls in z: total mass is conserved by the
    explicit operator, total energy too when g = 0 (Coriolis does no work)."""
    cells = (6, 3) if d == 2 else (4, 4, 3)
    ext = (6e3, 3e3) if d == 2 else (4e3, 4e3, 3e3)
    hl = dict(h0=200.0, a_c=1e3, xc=2e3, yc=2e3) if hill else None
    rl = (lambda c: 1 if c[0] < 2e3 else 0) if refine else None
    mesh = I.box_mesh(cells, ext, hill=hl, refine_level=rl)
    disc = O.Discretisation(mesh, 2)
    q = _random_state(disc, np.random.default_rng(7))
    r_ns, r_s = O.explicit_residuals(disc, q, O.Phys(f=1e-4, g=0.0))
    scale = np.abs(r_ns[0]).sum()
    assert abs(r_ns[0].sum()) < 1e-13 * scale
    assert abs(r_s[0]).max() == 0.0
    e_tot = (r_ns[4] + r_s[4]).sum()
    assert abs(e_tot) < 1e-12 * (np.abs(r_ns[4]).sum() + np.abs(r_s[4]).sum())


def test_free_stream_and_closed_cells():
    """Uniform state with wind tangent to the walls gives zero rates on a
    terrain-following mesh; the area-weighted normals of every cell sum to
    zero (closed surfaces), including 2:1 faces."""
    mesh = I.box_mesh((4, 4, 3), (4e3, 4e3, 3e3),
                      hill=dict(h0=300.0, a_c=1e3, xc=2e3, yc=2e3),
                      refine_level=lambda c: 1 if c[0] < 2e3 else 0)
    disc = O.Discretisation(mesh, 2)
    tot = np.zeros((disc.E, 3))
    np.add.at(tot, disc.f_em, disc.f_nS.sum(axis=1))
    inner = ~disc.f_wall
    np.add.at(tot, disc.f_ep[inner], -disc.f_nS[inner].sum(axis=1))
    assert np.abs(tot).max() < 1e-8 * np.abs(disc.f_nS).max()
    q = np.zeros((5, disc.E, disc.Np))
    q[0] = 1.2
    q[1] = 1.2 * 10.0
    q[2] = 1.2 * 4.0
    q[4] = 1e5 / 0.4 + 0.5 * 1.2 * 116.0
    # walls only at z; the hill makes the bottom wall tilt, so use a flat mesh
    flat = I.box_mesh((4, 4, 3), (4e3, 4e3, 3e3),
                      refine_level=lambda c: 1 if c[0] < 2e3 else 0)
    dflat = O.Discretisation(flat, 2)
    qf = q[:, :dflat.E]
    Fns, Fs = O.explicit_rates(dflat, qf, O.Phys(f=0.0, g=0.0))
    assert np.abs(Fns).max() < 1e-9 and np.abs(Fs).max() < 1e-9


# ----------------------------------------------------------------------------
# implicit operators (Section 3, Schur systems and the (A+R)^{-1} factorisation)
# ----------------------------------------------------------------------------

def _stage(disc, rng, adt=2.0):
    q = _random_state(disc, rng)
    u, p = O.nodal_primitives(q, 1.4)
    return O.StageCoeffs(rho=q[0], p_lag=p, u_lag=u, adt=adt), q


@pytest.mark.parametrize("nodes", ["gl", "gll"])
def test_rotation_closed_form(nodes):
    """R is energy-neutral, R = beta A J, and (A+R)^{-1} equals the
    closed-form (I + beta J)^{-1} A^{-1} (the oracle itself uses a dense LU
    of the full cell block)."""
    mesh = I.box_mesh((3, 2, 2), (3e3, 2e3, 2e3))
    disc = O.Discretisation(mesh, 2, nodes)
    rng = np.random.default_rng(11)
    cf, _ = _stage(disc, rng)
    f = 1.3e-4
    u = rng.standard_normal((3, disc.E, disc.Np))
    Ru = O.op_R(disc, cf, u, f)
    assert abs(np.sum(u * Ru)) < 1e-14 * np.sum(np.abs(u * O.op_A(disc, cf, u)))
    beta = cf.adt * f
    Jmat = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 0]], float)
    # R = beta A J
    Ju = np.einsum("ab,bei->aei", Jmat, u)
    assert np.allclose(Ru, beta * O.op_A(disc, cf, Ju), atol=1e-12 * np.abs(Ru).max())
    rhs = rng.standard_normal((3, disc.E, disc.Np))
    x = O.solve_AR(disc, cf, f, rhs, with_R=True)
    Ainv = O.solve_AR(disc, cf, f, rhs, with_R=False)
    inv = np.array([[1, beta, 0], [-beta, 1, 0], [0, 0, 1 + beta ** 2]]) / (1 + beta ** 2)
    cf_form = np.einsum("ab,bei->aei", inv, Ainv)
    assert np.allclose(x, cf_form, rtol=1e-12, atol=1e-14 * np.abs(x).max())


def _dense(op, n_in, shape_in):
    cols = []
    for k in range(n_in):
        e = np.zeros(n_in)
        e[k] = 1.0
        cols.append(op(e.reshape(shape_in)).reshape(-1))
    return np.array(cols).T


@pytest.mark.parametrize("d,refine", [(2, False), (2, True), (3, True)])
def test_adjointness_and_spd(d, refine):
    """With h rho = 1 on affine cells C = -B^T exactly (the quadrature is
    exact for phi . grad psi), so the R1 Schur operator without the
    penalty, D + B^T A^{-1} B, is symmetric positive definite."""
    cells = (3, 2) if d == 2 else (2, 2, 2)
    rl = (lambda c: 1 if c[0] < 1.0 else 0) if refine else None
    mesh = I.box_mesh(cells, tuple(float(c) for c in cells), refine_level=rl)
    disc = O.Discretisation(mesh, 1 if d == 3 else 2)
    rng = np.random.default_rng(5)
    gm = 1.4
    cf = O.StageCoeffs(rho=1.0 + 0.1 * rng.uniform(size=(disc.E, disc.Np)),
                       p_lag=np.full((disc.E, disc.Np), (gm - 1) / gm),
                       u_lag=rng.standard_normal((3, disc.E, disc.Np)), adt=0.7)
    n_p = disc.E * disc.Np
    B = _dense(lambda x: O.op_B(disc, cf, x), n_p, (disc.E, disc.Np))
    C = _dense(lambda u: O.op_C(disc, cf, u, gm), 3 * n_p, (3, disc.E, disc.Np))
    assert np.abs(C + B.T).max() < 1e-13 * np.abs(B).max()
    ph = O.Phys(variant="R1", penalty=False)
    S = _dense(lambda x: O.schur_apply(disc, cf, ph, x), n_p, (disc.E, disc.Np))
    Dm = _dense(lambda x: O.op_D(disc, x, gm), n_p, (disc.E, disc.Np))
    Sw = Dm @ S                                  # unscaled S = D (D^{-1} S)
    assert np.abs(Sw - Sw.T).max() < 1e-12 * np.abs(Sw).max()
    assert np.linalg.eigvalsh(0.5 * (Sw + Sw.T)).min() > 0


@pytest.mark.parametrize("variant", ["R1", "R2"])
def test_schur_solution_solves_coupled_system(variant):
    """The pressure from the Schur system and the recovered velocity satisfy
    the undecomposed coupled system (eq. matrix_form) with the terms that
    the variant lags held at the lagged iterate.  Pins the signs of every
    term of the Schur operator, its right-hand side and the recovery."""
    mesh = I.box_mesh((4, 3), (4e3, 3e3), refine_level=lambda c: 1 if c[0] < 1e3 else 0)
    disc = O.Discretisation(mesh, 2)
    rng = np.random.default_rng(21)
    cf, q = _stage(disc, rng, adt=3.0)
    ph = O.Phys(variant=variant, f=1.2e-4)
    gm = ph.gamma
    f_w = O.op_A(disc, cf, q[1:4] / q[0]) * (1 + 1e-3 * rng.standard_normal(q[1:4].shape))
    g_w = disc.vol_weak(disc.at_quad(q[4])) * (1 + 1e-4 * rng.standard_normal(q[4].shape))
    rhs = O.schur_rhs(disc, cf, ph, f_w, g_w)
    p, its, rr, ok = O.gmres(lambda x: O.schur_apply(disc, cf, ph, x), rhs, cf.p_lag,
                             rtol=1e-13, restart=40, maxit=400)
    assert ok
    u = O.recover_velocity(disc, cf, ph, f_w, p)
    fg = O.vec_fg(disc, cf, ph.g)
    kv = O.vec_k(disc, cf, cf.u_lag)
    if variant == "R2":
        mom = O.op_A(disc, cf, u) + O.op_R(disc, cf, u, ph.f) + O.op_B(disc, cf, p) + fg
        ene = (O.op_C(disc, cf, u, gm) + O.op_Mg(disc, cf, u, ph.g) + O.op_D(disc, p, gm)
               + O.op_P(disc, cf, p, gm) + kv)
    else:
        mom = (O.op_A(disc, cf, u) + O.op_R(disc, cf, cf.u_lag, ph.f)
               + O.op_B(disc, cf, p) + fg)
        ene = (O.op_C(disc, cf, u, gm) + O.op_Mg(disc, cf, cf.u_lag, ph.g)
               + O.op_D(disc, p, gm) + O.op_P(disc, cf, p, gm) + kv)
    assert np.abs(mom - f_w).max() < 1e-9 * np.abs(f_w).max()
    assert np.abs(ene - g_w).max() < 1e-9 * np.abs(g_w).max()


def test_gmres_matches_dense_solve():
    rng = np.random.default_rng(2)
    n = 60
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / math.sqrt(n)
    b = rng.standard_normal(n)
    x, its, rr, ok = O.gmres(lambda v: A @ v, b, np.zeros(n), rtol=1e-13, restart=10,
                             maxit=500)
    assert ok and rr <= 1e-13
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-11, atol=1e-12)


# ----------------------------------------------------------------------------
# whole step
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["R1", "R2"])
def test_inertial_oscillation_closed_form(variant):
    """Uniform state, g = 0, f != 0: every spatial term vanishes and
    u + i v is multiplied by the ARK2 stability function at z = -i f dt per
    step.  R2 holds the Coriolis term implicitly (one Picard iteration is
    exact); R1 lags it and reaches the same value once Picard converges."""
    # 100 km cells keep the acoustic Courant number (and so the conditioning
    # of the Schur system) moderate at dt = 600 s
    mesh = I.box_mesh((3, 2), (300e3, 200e3), periodic=[True, True])
    disc = O.Discretisation(mesh, 2)
    f, dt, U = 1e-4, 600.0, 10.0
    q = np.zeros((5, disc.E, disc.Np))
    q[0] = 1.1
    q[1] = 1.1 * U
    q[4] = 1e5 / 0.4 + 0.5 * 1.1 * U * U
    ph = O.Phys(f=f, g=0.0, variant=variant)
    opts = O.StepOpts(picard_rtol=1e-13, picard_maxit=30, gmres_rtol=1e-13,
                      gmres_maxit=100)
    steps = 4
    for _ in range(steps):
        q = O.imex_ark2_step(disc, ph, q, dt, opts)
    amp = ark2_amplification(-1j * f * dt) ** steps
    exact = U * amp
    got = (q[1] + 1j * q[2]) / q[0]
    # tolerance: GMRES stops at 1e-13 relative residual on p ~ 1e5 Pa
    assert np.abs(got - exact).max() < 1e-10 * U


def test_balanced_rest_state():
    """Discretely balanced background (READING c11): rho = -(G_z p)/g from
    the discrete weak vertical gradient of p.  With u = 0 and f != 0 the
    scheme keeps u = 0 up to the GMRES tolerance (rtol 1e-12 on p ~ 1e5 Pa
    bounds |u| near 1e-10 m/s; the continuous, non-balanced profile leaves
    |u| ~ 1e-4 m/s), so the Schur right-hand side is consistent with p_bar."""
    mesh = I.box_mesh((6, 4), (60e3, 8e3))
    disc = O.Discretisation(mesh, 2)
    X = disc.node_points()
    _, pbar, _, _ = I.exner_background(X[..., -1], 300.0, 0.01)
    gm, g = 1.4, 9.81
    cf = O.StageCoeffs(rho=np.ones_like(pbar), p_lag=pbar, u_lag=np.zeros((3,) + pbar.shape),
                       adt=1.0)
    Gp = disc.mass_solve(O.op_B(disc, cf, pbar))                # = grad p (weak)
    rho = -Gp[2] / g
    assert np.abs(Gp[0]).max() < 1e-9 * np.abs(Gp[2]).max()
    q = np.zeros((5,) + pbar.shape)
    q[0] = rho
    q[4] = pbar / (gm - 1)
    ph = O.Phys(f=1e-4, g=g)
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-12)
    for _ in range(3):
        q = O.imex_ark2_step(disc, ph, q, 10.0, opts)
    u = q[1:4] / q[0]
    assert np.abs(u).max() < 2e-9
    assert np.abs(q[0] - rho).max() < 1e-11 * rho.max()


# ----------------------------------------------------------------------------
# convergence orders on a linear rotating acoustic-inertia plane wave
# ----------------------------------------------------------------------------

def _plane_wave(X, t, k, m, f, rho0=1.2, p0=1e5, eps=1e-4, gm=1.4):
    """Exact plane wave of the vertical-slice equations linearised about a
    uniform rest state with g = 0 (eq. vertical_slice):
    Omega^4 - Omega^2 (f^2 + c^2 (k^2 + m^2)) + c^2 m^2 f^2 = 0,
    u = k Omega p' / (rho0 (Omega^2 - f^2)), v = -i f u / Omega,
    w = m p' / (rho0 Omega), rho' = p' / c^2."""
    c2 = gm * p0 / rho0
    a = f * f + c2 * (k * k + m * m)
    om = math.sqrt((a + math.sqrt(a * a - 4 * c2 * m * m * f * f)) / 2)
    P = eps * p0 * np.exp(1j * (k * X[..., 0] + m * X[..., 1] - om * t))
    uA = k * om / (rho0 * (om * om - f * f))
    u = np.real(uA * P)
    v = np.real(-1j * f * uA / om * P)
    w = np.real(m / (rho0 * om) * P)
    rho = rho0 + np.real(P) / c2
    p = p0 + np.real(P)
    return np.stack([rho, rho * u, rho * v, rho * w,
                     p / (gm - 1) + 0.5 * rho * (u * u + v * v + w * w)])


def _wave_error(n, r, dt, T, L=10e3, f=0.05):
    mesh = I.box_mesh((n, n), (L, L), periodic=[True, True])
    disc = O.Discretisation(mesh, r)
    X = disc.node_points()
    k = m = 2 * math.pi / L
    q = _plane_wave(X, 0.0, k, m, f)
    ph = O.Phys(f=f, g=0.0)
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-12, gmres_maxit=200)
    steps = int(round(T / dt))
    for _ in range(steps):
        q = O.imex_ark2_step(disc, ph, q, dt, opts)
    _, pe = O.nodal_primitives(_plane_wave(X, steps * dt, k, m, f), 1.4)
    _, pn = O.nodal_primitives(q, 1.4)
    return np.sqrt(np.mean((pn - pe) ** 2))


def test_convergence_orders():
    """Spatial order r + 1 (r = 2, tiny dt) and temporal order 2 (r = 4 on a
    fixed mesh, dt halved) of the whole IMEX-DG step."""
    es = [_wave_error(n, 2, 0.01, 0.5) for n in (3, 6, 12)]
    eoc_x = [math.log2(es[i] / es[i + 1]) for i in range(2)]
    assert all(2.8 < e < 3.3 for e in eoc_x), eoc_x
    et = [_wave_error(6, 4, dt, 8.0) for dt in (2.0, 1.0, 0.5)]
    eoc_t = [math.log2(et[i] / et[i + 1]) for i in range(2)]
    assert all(1.9 < e < 2.1 for e in eoc_t), eoc_t


# ----------------------------------------------------------------------------
# geostrophic imbalance E_geo (Section 4, planetary-scale wave)
# ----------------------------------------------------------------------------

def _linear_pressure_state(disc, a, rho0, v0, gamma=1.4):
    pts = disc.node_points()
    p = 9e4 + a * pts[..., 0]
    q = np.zeros((5,) + pts.shape[:-1])
    q[0] = rho0
    q[2] = rho0 * v0
    q[4] = p / (gamma - 1) + 0.5 * rho0 * v0 ** 2
    return q


@pytest.mark.parametrize("d", [2, 3])
def test_geostrophic_error_closed_form(d):
    """Linear pressure p = p0 + a x with uniform rho and v on a flat box with
    walls on every side (2D case with a 2:1 strip): the DG gradient of a
    linear field is exact, so E_geo = |a / rho - f v| everywhere; with
    f v = a / rho (geostrophic balance) it vanishes, which fixes the sign
    of the Coriolis term and of the pressure gradient."""
    if d == 2:
        mesh = I.box_mesh((5, 3), (5e3, 3e3), periodic=(False, False),
                          refine_level=lambda c: 1 if c[0] < 2e3 else 0)
    else:
        mesh = I.box_mesh((3, 2, 2), (3e3, 2e3, 2e3), periodic=(False, False, False))
    disc = O.Discretisation(mesh, 2)
    a, rho0, v0, f = 2e-3, 1.1, 7.0, 1.3e-4
    # rounding scale: p0 = 9e4 Pa differentiated on 500 m cells
    tol = 1e-14 * 9e4 / (rho0 * 500.0)
    e = O.geostrophic_error(disc, _linear_pressure_state(disc, a, rho0, v0), O.Phys(f=f))
    assert abs(e - abs(a / rho0 - f * v0)) <= tol
    vb = a / (rho0 * f)
    e_bal = O.geostrophic_error(disc, _linear_pressure_state(disc, a, rho0, vb), O.Phys(f=f))
    assert e_bal <= tol


def test_geostrophic_error_vanishes_for_layered_rest_state():
    """p = p(z), v = 0 on a flat periodic box: no horizontal pressure
    gradient and no Coriolis force, E_geo = 0 to round-off (relative to the
    vertical gradient scale g)."""
    mesh = I.box_mesh((6, 3), (6e3, 3e3))
    disc = O.Discretisation(mesh, 3)
    q = I.stratified_state(disc.node_points())
    assert O.geostrophic_error(disc, q, O.Phys(f=1e-4)) <= 1e-12 * 9.81


# ----------------------------------------------------------------------------
# Rayleigh damping layers (Section 4, eq. damping)
# ----------------------------------------------------------------------------

def test_sponge_coefficient_closed_form():
    """lambda = 0 below z_b, lam_bar/2 half way up (sin^2(pi/4)), lam_bar at
    z_t; lateral layers ramp the same way towards both ends; overlaps take
    the larger value."""
    s = O.Sponge(lam_bar=0.3, z_b=10e3, z_t=16e3, x_layers=(0.0, 60e3, 20e3), y_layers=(0.0, 40e3, 10e3))
    pts = np.array([[30e3, 20e3, 5e3],      # interior: 0
                    [30e3, 20e3, 13e3],     # top layer, half way: 0.15
                    [30e3, 20e3, 16e3],     # top: 0.3
                    [10e3, 20e3, 5e3],      # x layer, half way from x = 20 km to 0: 0.15
                    [60e3, 20e3, 5e3],      # x boundary: 0.3
                    [30e3, 32.5e3, 5e3],    # y layer, 1/4 of the way from 30 km: sin^2(pi/8) 0.3
                    [55e3, 20e3, 13e3]])    # x layer 3/4 (sin^2(3pi/8) 0.3) over top layer 0.15
    lam = O.sponge_coefficient(pts, s)
    want = [0.0, 0.15, 0.3, 0.15, 0.3, 0.3 * math.sin(math.pi / 8) ** 2, 0.3 * math.sin(3 * math.pi / 8) ** 2]
    assert np.allclose(lam, want, rtol=0, atol=1e-15)
    # 2D: the second coordinate is z, no y layers
    lam2 = O.sponge_coefficient(np.array([[10e3, 13e3]]), s)
    assert np.allclose(lam2, [0.15], rtol=0, atol=1e-15)


def explicit_stability_polynomial(z):
    """R(z) = 1 + z b.1 + z^2 b.A.1 + z^3 b.A^2.1 of the explicit tableau (A
    strictly lower triangular): the factor one explicit step applies to
    y' = lambda y, z = lambda dt."""
    a, _, b, _ = O.ark2_tableau()
    one = np.ones(3)
    return 1.0 + z * b @ one + z ** 2 * b @ a @ one + z ** 3 * b @ a @ a @ one


@pytest.mark.parametrize("variant", ["R2", "R1"])
@pytest.mark.parametrize("lam_dt", [0.6, 1.2, 2.4])
def test_sponge_uniform_state_relaxes_by_explicit_polynomial(variant, lam_dt):
    """A uniform state in one degree-0 cell with walls, g = 0 and f = 0 has
    no dynamics (no gradient, the wall pressures cancel), so one ARK2 step
    only relaxes each conserved field towards q_bar: q+ - q_bar =
    R(-lambda dt) (q - q_bar), R the explicit stability polynomial, since the
    damping is part of the explicit rates.  The node sits half way up the
    layer (lambda = lam_bar / 2); R(-0.6) = 0.5615 by hand."""
    mesh = I.box_mesh((1, 1), (1e3, 1e3), periodic=(False, False))
    disc = O.Discretisation(mesh, 0)

    def state(rho, v, p):
        q = np.zeros((5, 1, 1))
        q[0], q[2], q[4] = rho, rho * v, p / 0.4 + 0.5 * rho * v * v
        return q

    q, qb = state(1.1, 5.0, 9e4), state(1.0, 0.0, 1e5)
    dt = 2.0
    ph = O.Phys(g=0.0, f=0.0, variant=variant,
                sponge=O.Sponge(lam_bar=2.0 * lam_dt / dt, z_b=0.0, z_t=1e3, q_bar=qb))
    q1 = O.imex_ark2_step(disc, ph, q, dt, O.StepOpts(picard_rtol=1e-14, picard_maxit=50, gmres_rtol=1e-14))
    R = explicit_stability_polynomial(-lam_dt)
    if lam_dt == 0.6:
        assert abs(R - 0.5614701) < 1e-7
    for k in (0, 2, 4):
        assert abs((q1[k] - qb[k]) / (q[k] - qb[k]) - R).max() < 1e-11, (k, R)
    assert np.abs(q1[[1, 3]]).max() == 0.0


def test_sponge_inactive_below_layers():
    """Where lambda = 0 (every node below z_b, no lateral layers) the rates
    are those without the sponge, whatever q_bar is."""
    mesh = I.box_mesh((6, 3), (6e3, 3e3), refine_level=lambda c: 1 if c[0] < 2e3 else 0)
    disc = O.Discretisation(mesh, 2)
    q = I.perturb(I.stratified_state(disc.node_points(), wind=(5.0, 1.0, 0.0)), np.random.default_rng(0), 1e-2)
    qb = I.stratified_state(disc.node_points())
    a_ns, a_s = O.explicit_rates(disc, q, O.Phys())
    b_ns, b_s = O.explicit_rates(disc, q, O.Phys(sponge=O.Sponge(lam_bar=0.5, z_b=5e3, z_t=8e3, q_bar=qb)))
    assert np.array_equal(a_s, b_s)
    assert np.abs(a_ns - b_ns).max() <= 1e-14 * np.abs(a_ns).max()


# ----------------------------------------------------------------------------
# Non-stiff Rusanov floor (option, not in the paper)
# ----------------------------------------------------------------------------

def column_step_jacobian(lambda_min, dt=10.0):
    """Spectral radius of the linearised ARK2 step about the isothermal rest
    state (T0 = 250 K) on a 10-cell column (walls at 0 and 10 km, degree 2),
    for horizontally uniform perturbations of rho, rho w and rho E; built
    column by column from finite differences of whole oracle steps."""
    mesh = I.box_mesh((2, 10), (1000e3, 10e3))
    disc = O.Discretisation(mesh, 2)
    pts = disc.node_points()
    q0 = I.isothermal_state(pts.reshape(-1, 2)).reshape((5,) + pts.shape[:-1])
    ph = O.Phys(f=0.0, lambda_min=lambda_min)
    opts = O.StepOpts(picard_rtol=1e-13, picard_maxit=30, gmres_rtol=1e-13, gmres_restart=60, gmres_maxit=5000)
    z, x = pts[..., -1], pts[..., 0]
    cols = [np.where(x.mean(axis=1) < 500e3)[0], np.where(x.mean(axis=1) >= 500e3)[0]]
    cols = [c[np.argsort(z[c].mean(axis=1))] for c in cols]
    n = 3
    idx = [(f, ci, k) for f in (0, 3, 4) for ci in range(10) for k in range(n)]
    scale = {0: 1e-6, 3: 1e-6, 4: 1e-1}
    base = O.imex_ark2_step(disc, ph, q0, dt, opts)
    J = np.zeros((len(idx), len(idx)))
    for j, (f, ci, k) in enumerate(idx):
        dq = np.zeros_like(q0)
        for col in cols:
            dq[f, col[ci], np.arange(n) + n * k] = scale[f]
        d = O.imex_ark2_step(disc, ph, q0 + dq, dt, opts) - base
        J[:, j] = [d[g, cols[0][cj], n * kk] / scale[g] for (g, cj, kk) in idx]
    return np.abs(np.linalg.eigvals(J)).max()


def test_rest_state_checkerboard_needs_rusanov_floor():
    """The paper's lambda = |u.n| leaves the column's linearised step with a
    growing mode (spectral radius about 1.04 at dt = 10 s: a checkerboard of
    vertical momentum at the buoyancy frequency); lambda floored at 1 m/s in
    the non-stiff fluxes brings the radius to 1 (neutral modes of the
    frozen-in quantities only)."""
    assert column_step_jacobian(0.0) > 1.02
    assert column_step_jacobian(1.0) < 1.001


def test_rusanov_floor_inactive_when_flow_faster():
    """Where |u.n| exceeds the floor everywhere the rates do not change."""
    mesh = I.box_mesh((5, 3), (5e3, 3e3), periodic=(True, False))
    disc = O.Discretisation(mesh, 2)
    q = I.stratified_state(disc.node_points(), wind=(20.0, 0.0, 15.0))
    a_ns, a_s = O.explicit_rates(disc, q, O.Phys())
    b_ns, b_s = O.explicit_rates(disc, q, O.Phys(lambda_min=1.0))
    assert np.array_equal(a_s, b_s)
    assert np.abs(a_ns - b_ns).max() <= 1e-13 * np.abs(a_ns).max()


# ----------------------------------------------------------------------------
# far-field faces (outer state = a given background; READING R-farfield)
# ----------------------------------------------------------------------------

def _top_bottom_farfield(mesh):
    d = mesh.dim
    return I.with_boundary(mesh, (2 * (d - 1), 2 * (d - 1) + 1), I.BC_FARFIELD)


@pytest.mark.parametrize("d,r,refine", [(2, 2, False), (2, 3, True), (3, 2, True)])
def test_polynomial_exactness_through_farfield_faces(d, r, refine):
    """rho in Q_r, constant u (with a vertical component) and p, and the
    outer state equal to the same fields: the far-field faces then carry the
    exact flux, so the non-stiff rates equal -(u.grad rho)(1, u, kappa) on
    every cell without a wall face, those touching the far-field top and
    bottom included.  With slip walls in their place those cells are not
    exact."""
    cells = (4,) * d
    base = I.box_mesh(cells, (4.0,) * d, periodic=[False] * d,
                      refine_level=_refine_corner(d) if refine else None)
    mesh = _top_bottom_farfield(base)
    disc = O.Discretisation(mesh, r)
    u = np.array([0.3, -0.2, 0.5])
    q, ugr = _poly_state(disc, np.random.default_rng(3), u)
    disc.set_far_state(q)
    Fns, Fs = O.explicit_rates(disc, q, O.Phys(f=0.0, g=0.0))
    exp = np.stack([-ugr] + [-ugr * u[c] for c in range(3)] + [-ugr * 0.5 * (u @ u)])
    b = mesh.bdry_faces
    keep = np.setdiff1d(np.arange(disc.E), b[b[:, 2] == I.BC_WALL, 0])
    at_far = np.intersect1d(keep, b[b[:, 2] == I.BC_FARFIELD, 0])
    assert len(at_far) > 0
    assert np.abs(Fns[:, keep] - exp[:, keep]).max() < 1e-11
    assert np.abs(Fs[:, keep]).max() < 1e-10
    walls = O.Discretisation(base, r)
    Fw, _ = O.explicit_rates(walls, q, O.Phys(f=0.0, g=0.0))
    assert np.abs(Fw[:, at_far] - exp[:, at_far]).max() > 1e-3


FAR_FLOW_MESHES = {
    "2d": lambda: I.box_mesh((5, 4), (5e3, 2e3)),
    "3d": lambda: I.box_mesh((3, 3, 3), (3e3, 3e3, 2e3)),
    # far-field bottom on the terrain surface: curved faces, and 2:1 faces
    "3d_hill_nc": lambda: I.box_mesh((3, 3, 3), (3e3, 3e3, 2e3),
                                     hill=dict(h0=300.0, a_c=0.8e3, xc=1.5e3, yc=1.5e3),
                                     refine_level=lambda c: 1 if c[0] < 1e3 and c[2] < 700 else 0),
}


@pytest.mark.parametrize("variant", ["R1", "R2"])
@pytest.mark.parametrize("name", list(FAR_FLOW_MESHES))
def test_uniform_flow_through_farfield_boundaries_is_steady(variant, name):
    """A uniform flow crossing the far-field top and bottom (g = f = 0) with
    the outer state equal to it is an exact steady solution of the scheme:
    the explicit rates vanish and whole steps keep it, which pins the outer
    data moved to the right-hand sides of the implicit stage system.  The
    state holds to about 1e-11 relative (GMRES at 1e-13 on p ~ 1e5 Pa);
    dropping or flipping any of the three outer-data terms moves it by 1e-2
    or more."""
    mesh = _top_bottom_farfield(FAR_FLOW_MESHES[name]())
    d = mesh.dim
    disc = O.Discretisation(mesh, 2)
    pts = disc.node_points()
    u = np.array([8.0, -3.0, 2.5]) if d == 3 else np.array([8.0, 0.0, 2.5])
    rho, p = 1.1, 9.0e4
    q = np.zeros((5,) + pts.shape[:-1])
    q[0] = rho
    q[1:4] = rho * u[:, None, None]
    q[4] = p / 0.4 + 0.5 * rho * (u @ u)
    disc.set_far_state(q)
    ph = O.Phys(f=0.0, g=0.0, variant=variant)
    Fns, Fs = O.explicit_rates(disc, q, ph)
    assert np.abs(Fns).max() < 1e-9 and np.abs(Fs).max() < 1e-9
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-13)
    qn = q
    for _ in range(2):
        qn = O.imex_ark2_step(disc, ph, qn, 5.0, opts)
    for k in range(5):
        assert np.abs(qn[k] - q[k]).max() <= 1e-9 * max(np.abs(q[k]).max(), 1.0), k


def test_balanced_rest_state_under_a_farfield_top():
    """The discretely balanced rest state of the wall pin, with the top
    turned into a far-field face whose outer state is that same state: the
    pressure traces match there, so it stays at rest as under a wall."""
    mesh = I.box_mesh((6, 4), (60e3, 8e3))
    disc = O.Discretisation(mesh, 2)
    X = disc.node_points()
    _, pbar, _, _ = I.exner_background(X[..., -1], 300.0, 0.01)
    gm, g = 1.4, 9.81
    cf = O.StageCoeffs(rho=np.ones_like(pbar), p_lag=pbar, u_lag=np.zeros((3,) + pbar.shape),
                       adt=1.0)
    rho = -disc.mass_solve(O.op_B(disc, cf, pbar))[2] / g
    q = np.zeros((5,) + pbar.shape)
    q[0] = rho
    q[4] = pbar / (gm - 1)
    far = O.Discretisation(I.with_boundary(mesh, (3,), I.BC_FARFIELD), 2)
    assert far.f_far.sum() == 6
    far.set_far_state(q)
    ph = O.Phys(f=1e-4, g=g)
    Fw = O.explicit_rates(disc, q, ph)
    Ff = O.explicit_rates(far, q, ph)
    for a, b in zip(Fw, Ff):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-12)
    for _ in range(3):
        q = O.imex_ark2_step(far, ph, q, 10.0, opts)
    u = q[1:4] / q[0]
    assert np.abs(u).max() < 2e-9
    assert np.abs(q[0] - rho).max() < 1e-11 * rho.max()


def test_farfield_faces_need_an_outer_state():
    mesh = _top_bottom_farfield(I.box_mesh((3, 2), (3e3, 2e3)))
    disc = O.Discretisation(mesh, 1)
    q = I.stratified_state(disc.node_points())
    with pytest.raises(ValueError):
        O.explicit_rates(disc, q, O.Phys())
    bad = I.with_boundary(I.box_mesh((3, 2), (3e3, 2e3)), (3,), 7)
    with pytest.raises(ValueError):
        O.Discretisation(bad, 1)


# ----------------------------------------------------------------------------
# the stiff rho e Rusanov term (explicit, g vector) and its implicit
# counterpart P (READING c5), pinned in absolute terms
# ----------------------------------------------------------------------------

def _piecewise_constant_state(disc, rng, u, gm=1.4):
    """rho and p constant in each cell (random per cell), uniform velocity u."""
    rho_c = 1.0 + 0.2 * rng.uniform(size=disc.E)
    p_c = 1e5 * (1.0 + 0.1 * rng.uniform(size=disc.E))
    u = np.asarray(u, dtype=np.float64)
    q = np.zeros((5, disc.E, disc.Np))
    q[0] = rho_c[:, None]
    for c in range(3):
        q[1 + c] = rho_c[:, None] * u[c]
    q[4] = (p_c / (gm - 1.0) + 0.5 * rho_c * (u @ u))[:, None]
    return q, p_c


@pytest.mark.parametrize("d,u", [(2, (12.0, 0.0, 0.0)), (2, (-7.0, 3.0, 0.0)), (3, (9.0, -5.0, 0.0))])
def test_flux_balance_of_piecewise_constant_state_is_upwind(d, u):
    """Cell-wise constant rho and p, uniform horizontal u, g = f = 0, axis-
    aligned box (periodic sides, walls top and bottom).  Summing the test
    functions of a cell removes the volume terms, so each cell mean of the
    rates is a finite-volume balance of the face fluxes.  With u uniform the
    Rusanov flux with lambda = |u.n| is the upwind flux, and the split of the
    energy flux into kappa rho u (non-stiff, Rusanov on rho kappa) and
    h rho u (stiff, Rusanov on rho e) adds up to the upwind flux of the total
    energy plus the centred pressure work {p} u.n.  Expected means:
      mass      -1/|K| sum_F rho_up (u.n) |F|
      momentum  -1/|K| sum_F (m_up (u.n) + {p} n) |F|   (walls: p n)
      energy    -1/|K| sum_F ((rho E)_up + {p}) (u.n) |F|
    A sign slip or a lost factor 1/2 in any Rusanov term (the stiff rho e
    term included), or in a centred pressure / enthalpy flux, moves a mean
    by O(jump)."""
    rng = np.random.default_rng(3 + d)
    cells, ext = ((5, 3), (5e3, 3e3)) if d == 2 else ((3, 3, 2), (3e3, 3e3, 2e3))
    mesh = I.box_mesh(cells, ext)
    disc = O.Discretisation(mesh, 2)
    q, p_c = _piecewise_constant_state(disc, rng, u)
    u = np.asarray(u, dtype=np.float64)
    Fns, Fs = O.explicit_rates(disc, q, O.Phys(f=0.0, g=0.0))
    vol = disc.wJ.sum(axis=1)
    mean = (disc.at_quad(Fns + Fs) * disc.wJ[None]).sum(axis=-1) / vol[None]
    h = np.array(ext) / np.array(cells)                   # cell sizes

    def area(a):
        return np.prod([h[t] for t in range(d) if t != a])

    exp = np.zeros((5, disc.E))
    for eL, fL, eR, _ in mesh.int_faces:
        a = fL // 2
        n = np.zeros(d)
        n[a] = 1.0                                        # outward of eL
        un = sum(u[c] * n[b] for b, c in enumerate(disc.comp))
        up = eL if un >= 0 else eR
        pav = 0.5 * (p_c[eL] + p_c[eR])
        flux = np.array([q[k, up, 0] * un for k in range(5)])
        for b, c in enumerate(disc.comp):
            flux[1 + c] += pav * n[b]
        flux[4] += pav * un
        exp[:, eL] -= flux * area(a)
        exp[:, eR] += flux * area(a)
    for e, f, _ in mesh.bdry_faces:                       # walls: u.n = 0
        a, s = f // 2, f % 2
        for b, c in enumerate(disc.comp):
            if b == a:
                exp[1 + c, e] -= p_c[e] * (1.0 if s else -1.0) * area(a)
    exp /= vol[None]
    for k in range(5):
        scale = np.abs(exp[k]).max()
        if scale == 0.0:
            assert np.abs(mean[k]).max() < 1e-9
            continue
        assert np.abs(mean[k] - exp[k]).max() < 1e-12 * scale, k


def _two_cell_and_nc_meshes():
    return {
        "2cells_2d": I.box_mesh((2, 1), (2e3, 1e3), periodic=[False, False]),
        "2cells_3d": I.box_mesh((2, 1, 1), (2e3, 1e3, 1e3), periodic=[False, False, False]),
        "nc_2d": I.box_mesh((3, 2), (3e3, 2e3), periodic=[False, False],
                            refine_level=lambda c: 1 if c[0] < 1e3 else 0),
        "nc_3d_far": _top_bottom_farfield(
            I.box_mesh((2, 2, 2), (2e3, 2e3, 2e3), refine_level=lambda c: 1 if c[0] < 1e3 else 0)),
    }


@pytest.mark.parametrize("name", ["2cells_2d", "2cells_3d", "nc_2d", "nc_3d_far"])
def test_implicit_rusanov_term_is_the_linearised_explicit_one(name):
    """P (op_P) by brute force on two-cell and 2:1 meshes (one with
    far-field top and bottom):
      * P is symmetric positive semidefinite and nonzero, and P p = 0 for a
        pressure polynomial continuous across every face (no jumps);
      * P is the implicit form of the explicit stiff rho e Rusanov term:
        with rho and m held fixed, u and so lambda are fixed, p is affine in
        rho E, and the stiff energy residual of the explicit operator
        changes by -(C(u; h rho from dp) + P dp) / a_dt when rho E changes
        by dp / (gamma - 1).  This ties P's sign, its factor 1/2, its
        1/(gamma - 1) and its lambda to the explicit term, whose own sign
        and factor the upwind flux balance above fixes."""
    mesh = _two_cell_and_nc_meshes()[name]
    d = mesh.dim
    disc = O.Discretisation(mesh, 2 if d == 2 else 1)
    rng = np.random.default_rng(17)
    gm, adt = 1.4, 2.5
    X = disc.node_points()
    # uniform velocity, so that the explicit operator's u = m / rho at the
    # face points (from traces of m and rho) and P's lambda (from traces of
    # nodal u) see the same velocity; rho and p vary from node to node
    uw = np.array([15.0, -6.0, 4.0])
    q = I.stratified_state(X, wind=tuple(uw))
    rho = q[0] * (1.0 + 2e-2 * rng.standard_normal(q[0].shape))
    pn = 0.4 * (q[4] - 0.5 * q[0] * (uw @ uw)) * (1.0 + 2e-2 * rng.standard_normal(q[0].shape))
    q = np.concatenate([rho[None], rho[None] * uw[:, None, None],
                        (pn / 0.4 + 0.5 * rho * (uw @ uw))[None]])
    if disc.f_far.any():
        disc.set_far_state(I.stratified_state(X, wind=(12.0, 3.0, -2.0)))
    u, p = O.nodal_primitives(q, gm)
    cf = O.StageCoeffs(rho=q[0], p_lag=p, u_lag=u, adt=adt)
    n_p = disc.E * disc.Np
    P = _dense(lambda x: O.op_P(disc, cf, x, gm), n_p, (disc.E, disc.Np))
    scale = np.abs(P).max()
    assert scale > 0
    assert np.abs(P - P.T).max() < 1e-13 * scale
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > -1e-12 * scale
    # continuous pressure: a global polynomial of degree <= r at the nodes
    pc = 1.0 + sum(rng.uniform(-1, 1) * (X[..., a] / 1e3) ** k for a in range(d)
                   for k in range(1, disc.r + 1))
    pc = pc + 0.3 * (X[..., 0] / 1e3) * (X[..., -1] / 1e3)
    if not disc.f_far.any():
        assert np.abs(P @ pc.reshape(-1)).max() < 1e-12 * scale * np.abs(pc).max()
    # the linearisation of the explicit stiff energy residual
    ph = O.Phys(f=0.0, g=0.0)
    dp = rng.standard_normal((disc.E, disc.Np)) * 1e3
    q2 = q.copy()
    q2[4] += dp / (gm - 1.0)
    dr = O.explicit_residuals(disc, q2, ph)[1][4] - O.explicit_residuals(disc, q, ph)[1][4]
    cfd = O.StageCoeffs(rho=q[0], p_lag=dp, u_lag=u, adt=adt)
    got = -adt * dr - O.op_C(disc, cfd, u, gm)
    want = O.op_P(disc, cf, dp, gm)
    assert np.abs(want).max() > 1e-3 * np.abs(got).max()
    assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()


def test_linearised_step_about_uniform_flow_is_stable():
    """Linearised ARK2 step about a uniform moving state on a doubly
    periodic mesh (g = f = 0): every spatial term of the base state
    vanishes, the perturbations are advected and carried by sound waves,
    and the Rusanov terms (explicit and implicit) are their only damping.
    Spectral radius <= 1 (to the finite-difference accuracy): with the sign
    of the stiff rho e Rusanov term flipped the radius is 1.17 per step,
    and an inconsistent factor between the explicit term and P leaves a
    slowly growing mode (1 + 6e-10 to 1 + 2e-9)."""
    mesh = I.box_mesh((3, 3), (3e3, 3e3), periodic=[True, True])
    disc = O.Discretisation(mesh, 1)
    gm, rho0, p0 = 1.4, 1.1, 1e5
    u = np.array([20.0, 0.0, 8.0])
    q0 = np.zeros((5, disc.E, disc.Np))
    q0[0] = rho0
    for c in range(3):
        q0[1 + c] = rho0 * u[c]
    q0[4] = p0 / (gm - 1.0) + 0.5 * rho0 * (u @ u)
    ph = O.Phys(f=0.0, g=0.0)
    opts = O.StepOpts(picard_fixed=3, gmres_rtol=1e-14, gmres_restart=80, gmres_maxit=2000)
    field_scale = np.array([rho0, 10 * rho0, 10 * rho0, 10 * rho0, p0 / (gm - 1.0)]) * 1e-6
    sc = np.repeat(field_scale, disc.E * disc.Np)
    flat = q0.reshape(-1)
    J = np.zeros((flat.size, flat.size))
    for j in range(flat.size):
        dq = np.zeros(flat.size)
        dq[j] = sc[j]
        a = O.imex_ark2_step(disc, ph, (flat + dq).reshape(q0.shape), 1.0, opts).reshape(-1)
        b = O.imex_ark2_step(disc, ph, (flat - dq).reshape(q0.shape), 1.0, opts).reshape(-1)
        J[:, j] = (a - b) / (2.0 * sc) # scaled Jacobian diag(sc)^-1 J diag(sc)
    radius = np.abs(np.linalg.eigvals(J)).max()
    assert radius < 1.0 + 1e-11, radius
    assert radius > 1.0 - 1e-11                     # conserved quantities: neutral
