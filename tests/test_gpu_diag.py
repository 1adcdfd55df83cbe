"""Geostrophic imbalance E_geo through the C ABI: parity with the oracle on
perturbed states (2:1 meshes, terrain), the closed form of a linear pressure
field, and the planetary-scale wave's initial state (balanced: E_geo = 0)."""
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


@pytest.mark.parametrize("name", ["2d_nc", "3d_hill_nc"])
def test_geostrophic_error_parity(D, ctx, name):
    if name == "2d_nc":
        mesh, r = I.box_mesh((9, 4), (9e3, 4e3), refine_level=lambda c: 1 if 2e3 < c[0] < 5e3 else 0), 2
    else:
        mesh, r = I.box_mesh((5, 4, 3), (5e3, 4e3, 3e3), hill=dict(h0=300.0, a_c=1e3, xc=2.5e3, yc=2e3),
                             refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3 else 0), 3
    disc = O.Discretisation(mesh, r)
    gm = D.Mesh(ctx, mesh, r)
    q = I.perturb(I.stratified_state(disc.node_points(), wind=(8.0, -3.0, 1.0)), np.random.default_rng(4),
                  rel=1e-2)
    ref = O.geostrophic_error(disc, q, O.Phys(f=1.1e-4))
    got = gm.geostrophic_error(D.make_phys(f=1.1e-4), dev(q.reshape(5, -1)))
    assert abs(got - ref) <= 1e-11 * ref, (got, ref)


def test_geostrophic_error_closed_form(D, ctx):
    mesh = I.box_mesh((5, 3), (5e3, 3e3), periodic=(False, False), refine_level=lambda c: 1 if c[0] < 2e3 else 0)
    disc = O.Discretisation(mesh, 2)
    gm = D.Mesh(ctx, mesh, 2)
    a, rho0, v0, f = 2e-3, 1.1, 7.0, 1.3e-4
    pts = disc.node_points()
    q = np.zeros((5,) + pts.shape[:-1])
    q[0] = rho0
    q[2] = rho0 * v0
    q[4] = (9e4 + a * pts[..., 0]) / 0.4 + 0.5 * rho0 * v0 ** 2
    got = gm.geostrophic_error(D.make_phys(f=f), dev(q.reshape(5, -1)))
    assert abs(got - abs(a / rho0 - f * v0)) <= 1e-14 * 9e4 / (rho0 * 500.0)


def test_planetary_wave_starts_balanced(D, ctx):
    """p' = 0 and u = 0 at t = 0: no horizontal pressure gradient, no
    Coriolis force."""
    case = I.planetary_igw_case()
    gm = D.Mesh(ctx, case["mesh"], case["degree"])
    xyz = gm.node_coords().cpu().numpy().T
    q = dev(I.isothermal_state(xyz, **case["state_params"]))
    e = gm.geostrophic_error(D.make_phys(f=case["f"]), q)
    assert 0.0 <= e <= 1e-12 * 9.81, e
