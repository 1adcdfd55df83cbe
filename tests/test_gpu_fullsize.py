"""Parity at the full sizes the benchmark runs (60x60x20 hexes of degree 3,
4.6 M nodes; the 129 456-cell refined hill), in the same launch
configuration, on sampled cells: the oracle evaluates each operator on a
sub-mesh made of the sampled cells and the rings of neighbours the operator
reaches, so its values at the sampled cells are exact.  Properties that hold
at any size (conservation) are checked on the whole mesh."""
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


_CASES = {}


def full_case(D, ctx, name):
    """Mesh, device mesh and a seeded perturbed state of a benchmark workload."""
    if name not in _CASES:
        case = I.hill3d_case(refine=(name == "hill3d_nc"))
        mesh = case["mesh"]
        gm = D.Mesh(ctx, mesh, case["degree"])
        gm.autotune("mixed")
        xyz = gm.node_coords().cpu().numpy().T
        q = I.stratified_state(xyz, **case["state_params"])
        q = I.perturb(q, np.random.default_rng(42), rel=5e-3)
        _CASES[name] = (case, mesh, gm, q)
    return _CASES[name]


def samples(mesh, rng, k=12):
    """Seeded random cells plus cells at the hill, the walls, the periodic
    seams and (when present) both sides of hanging faces."""
    E = mesh.n_elem
    pick = set(rng.choice(E, size=k, replace=False).tolist())
    pick.add(int(mesh.bdry_faces[0, 0]))
    pick.add(int(mesh.bdry_faces[-1, 0]))
    c = mesh.vertices.mean(axis=1)
    pick.add(int(np.argmin(np.linalg.norm(c[:, :2] - [100e3, 100e3], axis=1) + c[:, 2])))
    pick.add(int(np.argmin(c[:, 0])))
    pick.add(int(np.argmax(c[:, 1])))
    if len(mesh.hang_faces):
        h = mesh.hang_faces[rng.integers(len(mesh.hang_faces))]
        pick.update([int(h[0]), int(h[2])])
    return np.array(sorted(pick), dtype=np.int64)


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name", ["hill3d", "hill3d_nc"])
def test_explicit_sampled_full_size(D, ctx, name):
    case, mesh, gm, q = full_case(D, ctx, name)
    Np = gm.Np
    fns, fs = gm.apply_explicit(D.make_phys(f=case["f"]), torch.tensor(q, device="cuda"))
    fns = fns.cpu().numpy().reshape(5, -1, Np)
    fs = fs.cpu().numpy().reshape(4, -1, Np)
    cells = samples(mesh, np.random.default_rng(1))
    sub, old, pos = O.submesh(mesh, cells, layers=1)
    disc = O.Discretisation(sub, case["degree"])
    qs = q.reshape(5, -1, Np)[:, old]
    Fns, Fs = O.explicit_rates(disc, qs, O.Phys(f=case["f"]))
    for k in range(5):
        assert relerr(fns[k, cells], Fns[k, pos]) < 1e-11, (k, relerr(fns[k, cells], Fns[k, pos]))
    for k in range(4):
        assert relerr(fs[k, cells], Fs[k + 1, pos]) < 1e-11, (k, relerr(fs[k, cells], Fs[k + 1, pos]))


@pytest.mark.parametrize("name", ["hill3d", "hill3d_nc"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_schur_vmult_sampled_full_size(D, ctx, name, precision):
    case, mesh, gm, q = full_case(D, ctx, name)
    Np = gm.Np
    u, p = O.nodal_primitives(q.reshape(5, -1, Np), 1.4)
    adt = (1 - 0.5 * 2 ** 0.5) * case["dt"]
    rho = q[0].reshape(-1, Np)
    x = p * (1 + 1e-3 * np.random.default_rng(3).standard_normal(p.shape))
    keep = [torch.tensor(np.ascontiguousarray(a).reshape(*s), device="cuda")
            for a, s in ((rho, (-1,)), (p, (-1,)), (u, (3, -1)))]
    dcf = D.Mesh.coeffs(*keep, adt)
    y = gm.apply_implicit(D.make_phys(f=case["f"], precision=precision), dcf,
                          torch.tensor(x.reshape(-1), device="cuda"))
    y = y.cpu().numpy().reshape(-1, Np)
    cells = samples(mesh, np.random.default_rng(2), k=6)
    sub, old, pos = O.submesh(mesh, cells, layers=2)
    disc = O.Discretisation(sub, case["degree"])
    cf = O.StageCoeffs(rho=rho[old], p_lag=p[old], u_lag=u[:, old], adt=adt)
    ref = O.schur_apply(disc, cf, O.Phys(f=case["f"]), x[old])
    # FP32: unit roundoff 6e-8 of inputs ~1e5 Pa, amplified by the operator's
    # non-identity part (acoustic Courant numbers up to ~20 in refined cells)
    tol = 1e-11 if precision == "fp64" else 5e-5
    assert relerr(y[cells], ref[pos]) < tol, relerr(y[cells], ref[pos])
    # the part of the operator that is not the identity, on its own
    d_ref = ref[pos] - x[cells]
    assert relerr(y[cells] - x[cells], d_ref) < (1e-9 if precision == "fp64" else 1e-3)


def _mass_weights(mesh, r):
    """w det J at every node, from the oracle's own cell map and GL rule."""
    x1, w1 = O.gauss_legendre01(r + 1)
    pts = O._tensor_points(x1, mesh.dim)
    w = np.prod(O._tensor_points(w1, mesh.dim), axis=1)
    out = np.empty((mesh.n_elem, len(w)))
    for s in range(0, mesh.n_elem, 8192):
        J = O.map_jacobian(mesh.vertices[s:s + 8192], pts)
        out[s:s + 8192] = w[None] * np.linalg.det(J)
    return out


@pytest.mark.parametrize("name", ["hill3d", "hill3d_nc"])
def test_conservation_full_size(D, ctx, name):
    """Mass rate integrates to zero and one full step conserves total mass
    (periodic sides, walls, 2:1 faces) on the whole mesh."""
    case, mesh, gm, q = full_case(D, ctx, name)
    wJ = _mass_weights(mesh, case["degree"]).reshape(-1)
    qd = torch.tensor(q, device="cuda")
    fns, _ = gm.apply_explicit(D.make_phys(f=case["f"]), qd)
    fr = fns[0].cpu().numpy()
    assert abs(np.sum(wJ * fr)) < 1e-12 * np.sum(np.abs(wJ * fr))
    m0 = np.sum(wJ * q[0])
    gm.step(D.make_phys(f=case["f"], precision="mixed"), qd, case["dt"], gmres_rtol=1e-10,
            gmres_inner_rtol=1e-4)
    m1 = np.sum(wJ * qd[0].cpu().numpy())
    assert abs(m1 - m0) < 1e-13 * abs(m0)
