"""DG_PAIRS: the Schur vmult on the FP32 pipe in pairs of FP32 numbers
(hi + lo, an emulation of FP64-class accuracy, not IEEE FP64) against the
FP64 oracle: the per-apply parity bar of the FP64 path (1e-11), the
preconditioned and plain GMRES to the same tolerance, and whole steps at
the step bar (1e-9)."""
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


def sheared(mesh, sx):
    """x += sx z: cells that are not terrain-following (general metric)."""
    v = mesh.vertices.copy()
    v[..., 0] += sx * v[..., -1]
    return I.Mesh(dim=mesh.dim, vertices=v, int_faces=mesh.int_faces, hang_faces=mesh.hang_faces,
                  bdry_faces=mesh.bdry_faces)


CASES = {
    "2d_r2_nc": (lambda: I.box_mesh((9, 4), (9e3, 4e3), refine_level=lambda c: 1 if 2e3 < c[0] < 5e3 else 0), 2),
    "3d_r3_hill_nc": (lambda: I.box_mesh((5, 4, 3), (5e3, 4e3, 3e3), hill=dict(h0=300.0, a_c=1e3, xc=2.5e3, yc=2e3),
                                         refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3 else 0), 3),
    "3d_r4": (lambda: I.box_mesh((3, 2, 2), (3e3, 2e3, 2e3)), 4),
    "2d_r1_sheared": (lambda: sheared(I.box_mesh((7, 3), (7e3, 3e3)), 0.3), 1),
}


def make_case(D, ctx, name, seed=0):
    build_mesh, r = CASES[name]
    mesh = build_mesh()
    disc = O.Discretisation(mesh, r)
    gm = D.Mesh(ctx, mesh, r)
    q = I.perturb(I.stratified_state(disc.node_points(), wind=(8.0, -3.0, 1.0)), np.random.default_rng(seed),
                  rel=2e-2)
    return mesh, disc, gm, q


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("variant,penalty", [("R2", True), ("R1", True), ("R2", False)])
def test_pairs_vmult_parity(D, ctx, name, variant, penalty):
    mesh, disc, gm, q = make_case(D, ctx, name, seed=1)
    u, p = O.nodal_primitives(q, 1.4)
    cf = O.StageCoeffs(rho=q[0], p_lag=p, u_lag=u, adt=3.0)
    ph = O.Phys(f=1.3e-4, variant=variant, penalty=penalty)
    x = p * (1 + 1e-2 * np.random.default_rng(4).standard_normal(p.shape))
    ref = O.schur_apply(disc, cf, ph, x)
    t = (to_dev(q[0].reshape(-1)), to_dev(p.reshape(-1)), to_dev(u.reshape(3, -1)))
    dcf = D.Mesh.coeffs(*t, cf.adt)
    for stage in ((0, 1, 0), (0, 1, 1)):   # both schedules of the pair kernels
        gm.set_fused_stage(*stage)
        y = from_dev(gm.apply_implicit(D.make_phys(f=1.3e-4, variant=variant, penalty=penalty, precision="pairs"),
                                       dcf, to_dev(x.reshape(-1))), ref.shape)
        assert relerr(y, ref) < 1e-11, (stage, relerr(y, ref))
        assert relerr(y - x, ref - x) < 1e-9, (stage, relerr(y - x, ref - x))


@pytest.mark.parametrize("precond", [False, True])
def test_pairs_steps_match_oracle(D, ctx, precond):
    """Ten steps of the 2D inertia-gravity wave (reduced to 20 x 5 cells)
    with the vmults in pairs: the FP64 GMRES converges to the same
    solution; with the vertical-line preconditioner too."""
    case = I.igw2d_case(nx=20, nz=5)
    mesh, r = case["mesh"], case["degree"]
    disc = O.Discretisation(mesh, r)
    gm = D.Mesh(ctx, mesh, r)
    q = I.perturb(I.stratified_state(disc.node_points(), **case["state_params"]), np.random.default_rng(5),
                  rel=1e-4)
    ph = O.Phys(f=case["f"])
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-13, gmres_restart=40, gmres_maxit=2000)
    qd = to_dev(q.reshape(5, -1)).contiguous()
    dph = D.make_phys(f=case["f"], precision="pairs")
    qo = q
    for _ in range(10):
        qo = O.imex_ark2_step(disc, ph, qo, case["dt"], opts)
        gm.step(dph, qd, case["dt"], picard_fixed=2, gmres_rtol=1e-12, gmres_restart=40, gmres_maxit=2000,
                gmres_precond=precond)
    qg = from_dev(qd, qo.shape)
    # momentum components against the momentum vector's scale: the vertical
    # one is a small perturbation of the 20 m/s flow, whose relative error
    # against itself mostly measures the GMRES tolerances (1e-12 here, 1e-13
    # in the oracle run)
    mscale = np.abs(qo[1:4]).max()
    for k in range(5):
        scale = mscale if 1 <= k <= 3 else np.abs(qo[k]).max()
        err = np.abs(qg[k] - qo[k]).max() / scale
        assert err < 1e-9, (k, err)
