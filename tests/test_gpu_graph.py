"""Device-driven step (opts.graph = 1): the whole ARK2 step as one CUDA graph
with while nodes for the Picard, refinement, restart and Arnoldi loops.

It computes what the host-driven step computes (same kernels, same
reductions; only the Givens updates run on the GPU instead of the CPU), so
the two agree to rounding, and the graph step keeps the oracle parity of the
step (1e-9 after 10 steps)."""
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
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t, shape):
    return t.cpu().numpy().reshape(shape)


def case(name):
    if name == "2d_nc":
        return I.box_mesh((9, 4), (9e3, 4e3), refine_level=lambda c: 1 if 2e3 < c[0] < 5e3 else 0), 2
    return I.box_mesh((5, 4, 3), (5e3, 4e3, 3e3), hill=dict(h0=300.0, a_c=1e3, xc=2.5e3, yc=2e3),
                      refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3 else 0), 3


def setup(D, ctx, name, seed=5):
    mesh, r = case(name)
    disc = O.Discretisation(mesh, r)
    q = I.perturb(I.stratified_state(disc.node_points(), wind=(8.0, -3.0, 1.0)),
                  np.random.default_rng(seed), rel=2e-2)
    return mesh, r, disc, q


OPTS = dict(picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=400)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "pairs"])
@pytest.mark.parametrize("name", ["2d_nc", "3d_hill_nc"])
def test_graph_step_matches_host_step(D, ctx, name, precision):
    mesh, r, disc, q = setup(D, ctx, name)
    ph = D.make_phys(f=1e-4, precision=precision)
    opts = dict(OPTS, gmres_inner_rtol=1e-4)
    gh, gg = D.Mesh(ctx, mesh, r), D.Mesh(ctx, mesh, r)
    qh, qg = dev(q.reshape(5, -1)), dev(q.reshape(5, -1))
    for _ in range(3):
        ih = gh.step(ph, qh, 3.0, **opts)
        ig = gg.step(ph, qg, 3.0, graph=True, **opts)
        assert list(ig.picard_iters) == list(ih.picard_iters)
        assert abs(ig.gmres_iters_total - ih.gmres_iters_total) <= 2, (ig.gmres_iters_total,
                                                                       ih.gmres_iters_total)
        assert ig.refinements_total == ih.refinements_total or precision == "mixed"
        assert ig.max_relres <= 1e-12
    # both solve every system to rtol 1e-12; the Givens updates round
    # differently, so the iterates differ at that level
    a, b = host(qg, q.shape), host(qh, q.shape)
    for k in range(5):
        assert relerr(a[k] - q[k], b[k] - q[k]) < 1e-8, (k, relerr(a[k] - q[k], b[k] - q[k]))
        assert relerr(a[k], b[k]) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed", "pairs"])
def test_graph_step_with_line_schedule(D, ctx, precision):
    """The one-thread-per-x-line vmult passes (schedule 2, with their
    asynchronous copies) inside the captured step give the host-driven
    step's result."""
    mesh, r, disc, q = setup(D, ctx, "3d_hill_nc", seed=6)
    ph = D.make_phys(f=1e-4, precision=precision)
    opts = dict(OPTS, gmres_inner_rtol=1e-4)
    gh, gg = D.Mesh(ctx, mesh, r), D.Mesh(ctx, mesh, r)
    for gm in (gh, gg):
        gm.set_fused_stage(2, 2, 2)
        gm.set_vmult_tile(precision, 2)
    qh, qg = dev(q.reshape(5, -1)), dev(q.reshape(5, -1))
    for _ in range(3):
        ih = gh.step(ph, qh, 3.0, **opts)
        ig = gg.step(ph, qg, 3.0, graph=True, **opts)
        assert list(ig.picard_iters) == list(ih.picard_iters)
        assert ig.max_relres <= 1e-12
    a, b = host(qg, q.shape), host(qh, q.shape)
    for k in range(5):
        assert relerr(a[k] - q[k], b[k] - q[k]) < 1e-8, (k, relerr(a[k] - q[k], b[k] - q[k]))


@pytest.mark.parametrize("variant", ["R2", "R1"])
def test_graph_step_parity_with_oracle(D, ctx, variant):
    """10 steps of the 2D non-conforming case: 1e-9 relative max-norm."""
    mesh, r, disc, q = setup(D, ctx, "2d_nc")
    gm = D.Mesh(ctx, mesh, r)
    ph = O.Phys(f=1e-4, variant=variant)
    opts = O.StepOpts(picard_fixed=2, gmres_rtol=1e-12, gmres_restart=50, gmres_maxit=400)
    qd = dev(q.reshape(5, -1))
    dph = D.make_phys(f=1e-4, variant=variant)
    qo = q
    for _ in range(10):
        qo = O.imex_ark2_step(disc, ph, qo, 6.0, opts)
        gm.step(dph, qd, 6.0, graph=True, **OPTS)
    qg = host(qd, qo.shape)
    for k in range(5):
        assert relerr(qg[k], qo[k]) < 1e-9, (k, relerr(qg[k], qo[k]))
        assert relerr(qg[k] - q[k], qo[k] - q[k]) < 1e-6


def test_graph_recaptures_on_new_inputs(D, ctx):
    """A new state pointer or dt re-captures; alternating between two states
    gives what the host-driven step gives for each."""
    mesh, r, disc, q = setup(D, ctx, "2d_nc")
    ph = D.make_phys(f=1e-4)
    gg, gh = D.Mesh(ctx, mesh, r), D.Mesh(ctx, mesh, r)
    q2 = I.perturb(q, np.random.default_rng(9), rel=1e-3)
    ga, gb = dev(q.reshape(5, -1)), dev(q2.reshape(5, -1))
    ha, hb = dev(q.reshape(5, -1)), dev(q2.reshape(5, -1))
    for dt in (3.0, 3.0, 5.0):
        gg.step(ph, ga, dt, graph=True, **OPTS)
        gg.step(ph, gb, dt, graph=True, **OPTS)
        gh.step(ph, ha, dt, **OPTS)
        gh.step(ph, hb, dt, **OPTS)
    assert relerr(host(ga, q.shape), host(ha, q.shape)) < 1e-10
    assert relerr(host(gb, q.shape), host(hb, q.shape)) < 1e-10


def test_graph_not_converged_counts(D, ctx):
    """With a GMRES iteration limit the solves stop early in both modes; the
    step still completes, with the same iteration counts."""
    mesh, r, disc, q = setup(D, ctx, "2d_nc")
    ph = D.make_phys(f=1e-4)
    opts = dict(picard_rtol=1e-10, picard_maxit=3, gmres_rtol=1e-14, gmres_restart=5, gmres_maxit=7)
    gg, gh = D.Mesh(ctx, mesh, r), D.Mesh(ctx, mesh, r)
    qg, qh = dev(q.reshape(5, -1)), dev(q.reshape(5, -1))
    ig = gg.step(ph, qg, 3.0, graph=True, **opts)
    ih = gh.step(ph, qh, 3.0, **opts)
    assert list(ig.picard_iters) == list(ih.picard_iters) == [0, 3, 3]
    assert ig.gmres_iters_total == ih.gmres_iters_total == 2 * 3 * 7
    assert relerr(host(qg, q.shape), host(qh, q.shape)) < 1e-10


def test_graph_mode_rejects_profiling(D, ctx):
    mesh, r, disc, q = setup(D, ctx, "2d_nc")
    gm = D.Mesh(ctx, mesh, r)
    qd = dev(q.reshape(5, -1))
    D.profile_begin(gm)
    with pytest.raises(D.DGError) as ei:
        gm.step(D.make_phys(), qd, 3.0, graph=True, **OPTS)
    D.profile_end(gm)
    assert ei.value.status == -2
    assert relerr(host(qd, q.shape), q) == 0.0


def test_graph_ensemble_matches_host(D, ctx):
    """Ensemble groups (merged meshes, own streams) stepped with graphs."""
    inst = [
        (I.box_mesh((6, 3), (18e3, 3e3)), 2, 1.2e-4, 6.0),
        (I.box_mesh((5, 3), (15e3, 3e3), refine_level=lambda c: 1 if c[0] < 6e3 else 0), 2, 0.3e-4, 6.0),
        (I.box_mesh((4, 3), (12e3, 3e3)), 3, 0.9e-4, 6.0),
        (I.box_mesh((3, 3, 2), (9e3, 9e3, 2e3)), 2, 1.4e-4, 2.0),
    ]
    args = ([m for m, _, _, _ in inst], [r for _, r, _, _ in inst], [f for _, _, f, _ in inst])
    eg, eh = D.Ensemble(ctx, *args), D.Ensemble(ctx, *args)
    for i, (m, r, f, dt) in enumerate(inst):
        disc = O.Discretisation(m, r)
        q = I.perturb(I.stratified_state(disc.node_points(), wind=(8.0, -2.0, 0.5)),
                      np.random.default_rng(20 + i), rel=1e-2)
        eg.set_state(i, dev(q.reshape(5, -1)))
        eh.set_state(i, dev(q.reshape(5, -1)))
    ph = D.make_phys(precision="mixed")
    dts = [dt for _, _, _, dt in inst]
    for _ in range(2):
        ig = eg.step(ph, dts, graph=True, gmres_inner_rtol=1e-4, **OPTS)
        ih = eh.step(ph, dts, gmres_inner_rtol=1e-4, **OPTS)
        assert abs(ig.gmres_iters_total - ih.gmres_iters_total) <= 2 * len(inst)
    for i in range(len(inst)):
        a = torch.empty((5, eg.nodes[i]), dtype=torch.float64, device="cuda")
        b = torch.empty((5, eh.nodes[i]), dtype=torch.float64, device="cuda")
        eg.get_state(i, a)
        eh.get_state(i, b)
        torch.cuda.synchronize()
        assert relerr(a.cpu().numpy(), b.cpu().numpy()) < 1e-11
