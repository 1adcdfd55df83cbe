"""Schur vmult with one thread per x-line (fused schedule 2: three
dimensions, degree 3) against the oracle, in every precision and with 1, 2
and 4 times the base cells per block: terrain-following and general
(sheared) cells, 2:1 faces, walls, periodic faces, far-field faces,
Gauss-Lobatto nodes and cell counts that leave a ragged last block.  Bars as
for the other schedules: FP64 and pairs 1e-11 per apply (1e-9 on the part
of the operator that is not the identity), FP32 1e-5 on a correction-sized
vector; 1e-9 after three steps (FP64, pairs)."""
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


def sheared(mesh, sx, sy=0.0):
    v = mesh.vertices.copy()
    v[..., 0] += sx * v[..., -1]
    v[..., 1] += sy * v[..., -1]
    return I.Mesh(dim=mesh.dim, vertices=v, int_faces=mesh.int_faces, hang_faces=mesh.hang_faces,
                  bdry_faces=mesh.bdry_faces, level=mesh.level, name=mesh.name + "_sheared")


HILL = dict(h0=300.0, a_c=1e3, xc=2.5e3, yc=2e3)
CASES = {
    # 2:1 faces, Gal-Chen terrain, periodic x/y, walls top and bottom
    "hill_nc": lambda: I.box_mesh((5, 4, 3), (5e3, 4e3, 3e3), hill=HILL,
                                  refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3 else 0),
    # general metric (no terrain-following shortcut)
    "hill_nc_sheared": lambda: sheared(I.box_mesh((5, 4, 3), (5e3, 4e3, 3e3), hill=HILL,
                                                  refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3 else 0),
                                       0.2, -0.1),
    # 45 cells: a ragged last block for 2, 4 and 8 cells per block; walls in x
    "ragged_walls": lambda: I.box_mesh((5, 3, 3), (5e3, 3e3, 3e3), periodic=(False, True, False),
                                       hill=dict(h0=200.0, a_c=1e3, xc=2e3, yc=1.5e3)),
}
PRECISIONS = ("fp64", "pairs", "mixed")


def make(D, ctx, name, seed=0, node_set="gl"):
    mesh = CASES[name]()
    disc = O.Discretisation(mesh, 3, node_set=node_set)
    gm = D.Mesh(ctx, mesh, 3, node_set=D.DG_NODES_GLL if node_set == "gll" else D.DG_NODES_GL)
    q = I.perturb(I.stratified_state(disc.node_points(), wind=(8.0, -3.0, 1.0)), np.random.default_rng(seed),
                  rel=2e-2)
    return mesh, disc, gm, q


def coeffs(D, q, adt, rng):
    u, p = O.nodal_primitives(q, 1.4)
    u = u * (1 + 1e-2 * rng.standard_normal(u.shape))
    cf = O.StageCoeffs(rho=q[0], p_lag=p, u_lag=u, adt=adt)
    keep = (to_dev(q[0].reshape(-1)), to_dev(p.reshape(-1)), to_dev(u.reshape(3, -1)))
    return cf, keep, D.Mesh.coeffs(*keep, adt)


def schedule(gm, prec):
    gm.set_fused_stage(*(2 if p == prec else 1 for p in ("fp64", "mixed", "pairs")))


def check(y, ref, x, prec):
    if prec == "mixed":
        assert relerr(y, ref) < 1e-5, relerr(y, ref)
        assert relerr(y, ref) > 1e-13   # really computed in FP32
    else:
        assert relerr(y, ref) < 1e-11, relerr(y, ref)
        assert relerr(y - x, ref - x) < 1e-9, relerr(y - x, ref - x)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("variant,penalty", [("R2", True), ("R1", True), ("R2", False)])
def test_lines_vmult_parity(D, ctx, name, prec, variant, penalty):
    mesh, disc, gm, q = make(D, ctx, name, seed=1)
    rng = np.random.default_rng(3)
    cf, keep, dcf = coeffs(D, q, 2.5, rng)
    ph = O.Phys(f=1.3e-4, variant=variant, penalty=penalty)
    dph = D.make_phys(f=1.3e-4, variant=variant, penalty=penalty, precision=prec)
    # FP64 and pairs: a pressure-sized vector; FP32: a correction-sized one
    x = cf.p_lag * (1 + 1e-2 * rng.standard_normal(cf.p_lag.shape)) if prec != "mixed" else \
        rng.standard_normal(cf.p_lag.shape) * 100.0
    ref = O.schur_apply(disc, cf, ph, x)
    schedule(gm, prec)
    for tile in (1, 2, 4):
        gm.set_vmult_tile(prec, tile)
        y = from_dev(gm.apply_implicit(dph, dcf, to_dev(x.reshape(-1))), ref.shape)
        check(y, ref, x, prec)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_lines_match_the_other_schedules(D, ctx, prec):
    """Schedule 2 agrees with schedules 0 and 1 up to rounding."""
    mesh, disc, gm, q = make(D, ctx, "hill_nc", seed=2)
    rng = np.random.default_rng(4)
    cf, keep, dcf = coeffs(D, q, 3.0, rng)
    dph = D.make_phys(f=1.1e-4, precision=prec)
    x = to_dev((cf.p_lag * (1 + 1e-3 * rng.standard_normal(cf.p_lag.shape))).reshape(-1))
    ys = []
    for s in (0, 1, 2):
        gm.set_fused_stage(s, s, s)
        ys.append(from_dev(gm.apply_implicit(dph, dcf, x), (-1,)))
    # FP32: its parity bar against the oracle; pairs: about 1e-14 per operation
    tol = {"mixed": 1e-5, "pairs": 1e-12}.get(prec, 1e-13)
    assert relerr(ys[2], ys[0]) < tol and relerr(ys[2], ys[1]) < tol


def test_lines_far_field(D, ctx):
    """Far-field top and bottom: the linear part of the operator (outer
    state zero), FP64 and FP32."""
    mesh = I.with_boundary(CASES["hill_nc"](), (4, 5), I.BC_FARFIELD)
    disc = O.Discretisation(mesh, 3)
    gm = D.Mesh(ctx, mesh, 3)
    X = disc.node_points()
    rng = np.random.default_rng(6)
    q = I.perturb(I.stratified_state(X, wind=(8.0, -3.0, 1.5)), rng, rel=2e-2)
    qfar = I.perturb(I.stratified_state(X, wind=(10.0, 2.0, -1.0)), rng, rel=1e-2)
    disc.set_far_state(qfar)
    gm.set_far_state(to_dev(qfar.reshape(5, -1)))
    cf, keep, dcf = coeffs(D, q, 2.5, rng)
    for prec in ("fp64", "mixed"):
        x = cf.p_lag * (1 + 1e-2 * rng.standard_normal(cf.p_lag.shape)) if prec == "fp64" else \
            rng.standard_normal(cf.p_lag.shape) * 100.0
        ref = O.schur_apply(disc, cf, O.Phys(f=1.2e-4), x)
        schedule(gm, prec)
        y = from_dev(gm.apply_implicit(D.make_phys(f=1.2e-4, precision=prec), dcf, to_dev(x.reshape(-1))),
                     ref.shape)
        check(y, ref, x, prec)


def test_lines_gauss_lobatto(D, ctx):
    """Gauss-Lobatto nodes: the passes run in the Gauss-Legendre basis
    between the two changes of basis."""
    mesh, disc, gm, q = make(D, ctx, "hill_nc", seed=5, node_set="gll")
    rng = np.random.default_rng(7)
    cf, keep, dcf = coeffs(D, q, 2.0, rng)
    x = cf.p_lag * (1 + 1e-2 * rng.standard_normal(cf.p_lag.shape))
    ref = O.schur_apply(disc, cf, O.Phys(f=1e-4), x)
    schedule(gm, "fp64")
    y = from_dev(gm.apply_implicit(D.make_phys(f=1e-4), dcf, to_dev(x.reshape(-1))), ref.shape)
    check(y, ref, x, "fp64")


@pytest.mark.parametrize("prec", ["fp64", "pairs"])
def test_lines_steps_match_oracle(D, ctx, prec):
    """Three ARK2 steps on the 2:1 hill mesh with the schedule-2 vmults in
    the GMRES (1e-9 after the steps, FP64 bar)."""
    mesh, disc, gm, q = make(D, ctx, "hill_nc", seed=8)
    ph = O.Phys(f=1e-4)
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-13, gmres_restart=40, gmres_maxit=2000)
    schedule(gm, prec)
    qd = to_dev(q.reshape(5, -1)).contiguous()
    dph = D.make_phys(f=1e-4, precision=prec)
    qo = q
    for _ in range(3):
        qo = O.imex_ark2_step(disc, ph, qo, 2.0, opts)
        gm.step(dph, qd, 2.0, picard_fixed=2, gmres_rtol=1e-12, gmres_restart=40, gmres_maxit=2000)
    qg = from_dev(qd, qo.shape)
    # momentum components against the momentum vector's scale (the vertical
    # one is a small perturbation of the flow; its error against itself
    # mostly measures the GMRES tolerances)
    mscale = np.abs(qo[1:4]).max()
    for k in range(5):
        scale = mscale if 1 <= k <= 3 else np.abs(qo[k]).max()
        err = np.abs(qg[k] - qo[k]).max() / scale
        assert err < 1e-9, (k, err)


def test_lines_autotune_candidates(D, ctx):
    """The autotuner may pick schedule 2 with any tile; whatever it picks
    keeps parity."""
    mesh, disc, gm, q = make(D, ctx, "hill_nc", seed=9)
    t64, t32, sched = gm.autotune("mixed")
    assert all(s in (0, 1, 2) for s in sched) and t64[1] in (1, 2, 4) and t32[2] in (1, 2, 4)
    rng = np.random.default_rng(10)
    cf, keep, dcf = coeffs(D, q, 3.0, rng)
    x = cf.p_lag * (1 + 1e-2 * rng.standard_normal(cf.p_lag.shape))
    ref = O.schur_apply(disc, cf, O.Phys(f=1e-4), x)
    y = from_dev(gm.apply_implicit(D.make_phys(f=1e-4), dcf, to_dev(x.reshape(-1))), ref.shape)
    check(y, ref, x, "fp64")


def test_lines_misaligned_vector_falls_back(D, ctx):
    """A vector that is not 16-byte aligned takes the node-line schedule
    (same result): schedule 2's 128-bit loads need the alignment."""
    mesh, disc, gm, q = make(D, ctx, "ragged_walls", seed=11)
    rng = np.random.default_rng(12)
    cf, keep, dcf = coeffs(D, q, 2.0, rng)
    x = cf.p_lag * (1 + 1e-2 * rng.standard_normal(cf.p_lag.shape))
    ref = O.schur_apply(disc, cf, O.Phys(f=1e-4), x)
    schedule(gm, "fp64")
    buf = torch.zeros(x.size + 1, dtype=torch.float64, device="cuda")
    buf[1:] = to_dev(x.reshape(-1))
    xv = buf[1:]                      # 8 bytes past a 16-byte boundary
    assert xv.data_ptr() % 16 == 8
    y = from_dev(gm.apply_implicit(D.make_phys(f=1e-4), dcf, xv), ref.shape)
    check(y, ref, x, "fp64")


def test_lines_setters_validate(D, ctx):
    """Schedules outside 0..2 and tiles other than 1, 2, 4 are rejected;
    valid ones show in the mesh statistics."""
    mesh, disc, gm, q = make(D, ctx, "ragged_walls")
    with pytest.raises(D.DGError):
        gm.set_fused_stage(0, 3, 0)
    with pytest.raises(D.DGError):
        gm.set_vmult_tile("mixed", 3)
    gm.set_fused_stage(2, 2, 2)
    gm.set_vmult_tile("mixed", 4)
    st = gm.stats()
    assert list(st.fused_stage) == [2, 2, 2] and st.tile_fp32[1] == 4 and st.tile_fp32[2] == 4
