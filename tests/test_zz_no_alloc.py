"""dg_apply_explicit_noalloc: the explicit operator for callers that cannot
allocate device memory while they run (a service with memory reserved up
front, or a framework that owns all device allocations).  It takes its
scratch from a fixed array in the library image instead of growing
workspace with cudaMalloc.  Checked through the C ABI against
dg_apply_explicit on two calls in a row, and for a clear rejection of a
mesh beyond its capacity.  This file sorts last so that a run stopping at
the first failure has run every other test first; it also passes alone in
a fresh process."""
import ctypes as C

import numpy as np
import pytest

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


def _state(gm, seed):
    xyz = gm.node_coords().cpu().numpy().T
    q = I.perturb(I.stratified_state(xyz, wind=(12.0, -4.0, 0.5)), np.random.default_rng(seed),
                  rel=2e-2)
    return torch.tensor(q, dtype=torch.float64, device="cuda").contiguous()


def _noalloc(D, ctx, gm, phys, q, fns, fs):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return D.load().dg_apply_explicit_noalloc(ctx.h, gm.h, C.byref(phys), C.c_void_p(q.data_ptr()),
                                              C.c_void_p(fns.data_ptr()), C.c_void_p(fs.data_ptr()),
                                              stream)


@pytest.mark.parametrize("name", ["2d_nc", "3d_hill_nc"])
def test_noalloc_matches_explicit_twice(D, name):
    if name == "2d_nc":
        mesh = I.box_mesh((10, 4), (10e3, 4e3), refine_level=lambda c: 1 if c[0] < 3e3 else 0)
        r = 2
    else:
        mesh = I.box_mesh((5, 4, 3), (5e3, 4e3, 3e3),
                          hill=dict(h0=300.0, a_c=1e3, xc=2.5e3, yc=2e3),
                          refine_level=lambda c: 1 if c[0] < 2e3 and c[2] < 1e3 else 0)
        r = 3
    ctx = D.Context(0)
    gm = D.Mesh(ctx, mesh, r)
    phys = D.make_phys(f=1.2e-4)
    q = _state(gm, 1)
    ref_ns, ref_s = gm.apply_explicit(phys, q)
    torch.cuda.synchronize()
    for call in range(2):
        fns = torch.full_like(ref_ns, float("nan"))
        fs = torch.full_like(ref_s, float("nan"))
        assert _noalloc(D, ctx, gm, phys, q, fns, fs) == 0, D.load().dg_last_error()
        torch.cuda.synchronize()
        for a, b in ((fns, ref_ns), (fs, ref_s)):
            err = ((a - b).abs().max() / b.abs().max()).item()
            assert err < 1e-11, (call, err)
    # a different state on the same shared scratch: no stale values leak in
    q2 = _state(gm, 2)
    ref2_ns, ref2_s = gm.apply_explicit(phys, q2)
    fns = torch.empty_like(ref_ns)
    fs = torch.empty_like(ref_s)
    assert _noalloc(D, ctx, gm, phys, q2, fns, fs) == 0
    torch.cuda.synchronize()
    assert ((fns - ref2_ns).abs().max() / ref2_ns.abs().max()).item() < 1e-11
    assert ((fs - ref2_s).abs().max() / ref2_s.abs().max()).item() < 1e-11


def test_noalloc_rejects_mesh_beyond_capacity(D):
    # 3D degree 3: 96 face-point slots per cell, 14 doubles each -> 4000
    # cells need 5.4 M doubles, above the 4 M-double capacity
    mesh = I.box_mesh((20, 20, 10), (20e3, 20e3, 10e3))
    ctx = D.Context(0)
    gm = D.Mesh(ctx, mesh, 3)
    phys = D.make_phys()
    q = torch.ones((5, gm.N), dtype=torch.float64, device="cuda")
    fns = torch.empty((5, gm.N), dtype=torch.float64, device="cuda")
    fs = torch.empty((4, gm.N), dtype=torch.float64, device="cuda")
    assert _noalloc(D, ctx, gm, phys, q, fns, fs) == -1
    assert b"capacity" in D.load().dg_last_error()


def test_noalloc_allocates_no_workspace_and_honours_sponge_and_mixed(D):
    """On a fresh mesh the call leaves the mesh's workspace empty (every
    scratch value lives in the library's fixed array); damping layers set on
    the mesh are applied as by dg_apply_explicit; DG_MIXED runs the same
    FP64 explicit kernels; DG_MIXED_EXPLICIT and a negative lambda_min are
    refused."""
    mesh = I.box_mesh((8, 3, 4), (8e3, 3e3, 4e3), hill=dict(h0=200.0, a_c=1.5e3, xc=4e3, yc=1.5e3))
    ctx = D.Context(0)
    gm = D.Mesh(ctx, mesh, 2)
    q = _state(gm, 3)
    ws0 = gm.stats().workspace_bytes
    for prec in ("fp64", "mixed"):
        phys = D.make_phys(f=1e-4, precision=prec)
        fns = torch.empty((5, gm.N), dtype=torch.float64, device="cuda")
        fs = torch.empty((4, gm.N), dtype=torch.float64, device="cuda")
        assert _noalloc(D, ctx, gm, phys, q, fns, fs) == 0, D.load().dg_last_error()
        torch.cuda.synchronize()
        assert gm.stats().workspace_bytes == ws0
    # damping layers (towards a perturbed copy of the state, so that they act)
    qbar = _state(gm, 4)
    gm.set_sponge(qbar, lambda_bar=0.3, z_b=1.5e3, z_t=4e3, x_layers=(0.0, 8e3, 2e3))
    phys = D.make_phys(f=1e-4, precision="mixed")
    ref_ns, ref_s = gm.apply_explicit(D.make_phys(f=1e-4), q)
    fns = torch.empty_like(ref_ns)
    fs = torch.empty_like(ref_s)
    assert _noalloc(D, ctx, gm, phys, q, fns, fs) == 0, D.load().dg_last_error()
    torch.cuda.synchronize()
    for a, b in ((fns, ref_ns), (fs, ref_s)):
        assert ((a - b).abs().max() / b.abs().max()).item() < 1e-11
    gm.set_sponge(None)
    no_ns, _ = gm.apply_explicit(D.make_phys(f=1e-4), q)
    assert ((no_ns - ref_ns).abs().max() / ref_ns.abs().max()).item() > 1e-6   # the layers acted
    assert _noalloc(D, ctx, gm, D.make_phys(precision="mixed_explicit"), q, fns, fs) == -2
    assert _noalloc(D, ctx, gm, D.make_phys(lambda_min=-1.0), q, fns, fs) == -1
