"""Ensembles: independent instances of uneven sizes, dims, degrees and
Coriolis parameters advanced together (instances sharing (dim, degree)
merged into one mesh, per-cell f).  Each instance is checked against the
FP64 oracle stepping it alone."""
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


def instances():
    return [
        (I.box_mesh((6, 3), (18e3, 3e3)), 2, 1.2e-4, 6.0),
        (I.box_mesh((5, 3), (15e3, 3e3), refine_level=lambda c: 1 if c[0] < 6e3 else 0), 2, 0.3e-4, 6.0),
        (I.box_mesh((4, 3), (12e3, 3e3)), 3, 0.9e-4, 6.0),
        (I.box_mesh((3, 3, 2), (9e3, 9e3, 2e3)), 2, 1.4e-4, 2.0),
        (I.box_mesh((3, 2, 2), (6e3, 4e3, 2e3), hill=dict(h0=200.0, a_c=2e3, xc=3e3, yc=2e3),
                    refine_level=lambda c: 1 if c[0] < 2e3 else 0), 2, 0.0, 2.0),
    ]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ensemble_matches_oracle_per_instance(D, precision):
    ctx = D.Context(0)
    inst = instances()
    ens = D.Ensemble(ctx, [m for m, _, _, _ in inst], [r for _, r, _, _ in inst],
                     [f for _, _, f, _ in inst])
    assert ens.n_groups == 3
    discs, qs = [], []
    for i, (m, r, f, dt) in enumerate(inst):
        disc = O.Discretisation(m, r)
        q = I.perturb(I.stratified_state(disc.node_points(), wind=(8.0, -2.0, 0.5)),
                      np.random.default_rng(10 + i), rel=1e-2)
        assert ens.nodes[i] == disc.E * disc.Np
        ens.set_state(i, torch.tensor(q.reshape(5, -1), dtype=torch.float64, device="cuda"))
        discs.append(disc)
        qs.append(q)
    phys = D.make_phys(precision=precision)
    dts = [dt for _, _, _, dt in inst]
    steps = 2
    for _ in range(steps):
        info = ens.step(phys, dts, picard_fixed=2, gmres_rtol=1e-12, gmres_restart=40,
                        gmres_maxit=3000, gmres_inner_rtol=1e-4)
        if precision == "mixed":
            assert info.refinements_total > 0
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-12, gmres_restart=40, gmres_maxit=400)
    for i, (m, r, f, dt) in enumerate(inst):
        qo = qs[i]
        for _ in range(steps):
            qo = O.imex_ark2_step(discs[i], O.Phys(f=f), qo, dt, opts)
        qg = ens.get_state(i, torch.empty((5, ens.nodes[i]), dtype=torch.float64,
                                          device="cuda")).cpu().numpy().reshape(qo.shape)
        for k in range(5):
            err = np.abs(qg[k] - qo[k]).max() / np.abs(qo[k]).max()
            assert err < 1e-9, (i, k, err)
            pert = np.linalg.norm(qo[k] - qs[i][k])
            assert np.linalg.norm(qg[k] - qo[k]) < 1e-6 * pert, (i, k)


def test_ensemble_rejects_mixed_dt_in_a_group(D):
    ctx = D.Context(0)
    m = I.box_mesh((4, 2), (4e3, 2e3))
    ens = D.Ensemble(ctx, [m, m], [2, 2], [1e-4, 0.0])
    q = torch.ones((5, ens.nodes[0]), dtype=torch.float64, device="cuda")
    ens.set_state(0, q)
    ens.set_state(1, q)
    with pytest.raises(D.DGError) as ei:
        ens.step(D.make_phys(), [4.0, 6.0])
    assert ei.value.status == -1


def test_ensemble_state_roundtrip(D):
    ctx = D.Context(0)
    inst = instances()
    ens = D.Ensemble(ctx, [m for m, _, _, _ in inst], [r for _, r, _, _ in inst],
                     [f for _, _, f, _ in inst])
    qs = [torch.randn((5, ens.nodes[i]), dtype=torch.float64, device="cuda") for i in range(ens.n)]
    for i in range(ens.n):
        ens.set_state(i, qs[i])
    for i in reversed(range(ens.n)):
        back = ens.get_state(i, torch.empty_like(qs[i]))
        assert torch.equal(back, qs[i])
