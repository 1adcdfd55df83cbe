"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/dgimex.h declares (no compute call needs a GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dgimex.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "return")))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_29598_gb300 import build, dgimex
    build.build()
    return dgimex.load()


def test_header_parses():
    names = declared_functions()
    for must in ("dg_mesh_create", "dg_apply_explicit", "dg_apply_implicit", "dg_gmres_solve",
                 "imex_ark2_step"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    from paper_2605_29598_gb300 import dgimex
    assert set(dgimex.EXPORTS) >= set(declared_functions())


def test_status_strings(lib):
    assert lib.dg_status_string(0) == b"DG_OK"
    assert lib.dg_status_string(-4) == b"DG_ERR_NOT_CONVERGED"


def test_null_arguments_rejected_without_gpu(lib):
    # argument checks run before any CUDA call
    assert lib.dg_ctx_create(0, None) == -1
    assert lib.dg_mesh_create(None, None, None) == -1
    assert lib.dg_apply_explicit(None, None, None, None, None, None, None) == -1
    assert lib.dg_gmres_solve(None, None, None, None, None, None, None, None, None) == -1
    assert lib.imex_ark2_step(None, None, None, None, 1.0, None, None, None) == -1
    assert lib.dg_precond_apply(None, None, None, None, 1, None, None, None) == -1
    assert lib.dg_mesh_set_sponge(None, None, None, None, None) == -1
    assert lib.dg_mesh_set_fused_stage(None, 0, 2, 0) == -1
    assert lib.dg_mesh_set_vmult_tile(None, 1, 2) == -1


def test_context_fails_cleanly_without_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.dg_ctx_create(0, ctypes.byref(h)) in (-1, -3)


def test_binding_checks_buffer_sizes_and_devices():
    """The C ABI receives raw pointers, so the binding checks each buffer's
    length and device before the call (no GPU needed for the checks)."""
    torch = pytest.importorskip("torch")
    from paper_2605_29598_gb300 import dgimex as D
    D._validate(15, 0, 15, 0)
    D._validate(15, 1)                     # nothing to check against
    with pytest.raises(ValueError):
        D._validate(14, 0, 15, 0)          # short buffer
    with pytest.raises(ValueError):
        D._validate(16, 0, 15, 0)          # long buffer: a shape mistake all the same
    with pytest.raises(ValueError):
        D._validate(15, 1, 15, 0)          # another GPU than the context's
    with pytest.raises(TypeError):
        D._ptr(torch.zeros(4, dtype=torch.float64))          # host tensor
    with pytest.raises(TypeError):
        D._ptr(torch.zeros(4, dtype=torch.float32))


def test_mesh_validation_on_the_host():
    """dg_mesh_validate runs every host-side rule of dg_mesh_create with no
    GPU: the generator's meshes pass, and each kind of broken list or
    unsupported option gets dg_mesh_create's status and message."""
    import numpy as np
    from paper_2605_29598_gb300 import dgimex as D, inputs as I
    good = [I.box_mesh((3, 2), (3.0, 2.0)),
            I.box_mesh((4, 3), (4.0, 3.0), refine_level=lambda c: 1 if c[0] < 1 else 0),
            I.box_mesh((3, 3, 2), (3e3, 3e3, 2e3), hill=dict(h0=200.0, a_c=1e3, xc=1.5e3, yc=1.5e3),
                       refine_level=lambda c: 1 if c[0] < 1e3 and c[2] < 1e3 else 0)]
    for m in good:
        for r in (1, 4):
            assert D.validate_mesh(m, r) == 0

    def status(m, r=2, node_set=D.DG_NODES_GL):
        with pytest.raises(D.DGError) as ei:
            D.validate_mesh(m, r, node_set)
        return ei.value.status, str(ei.value)

    m = good[1]
    assert len(m.hang_faces) >= 2
    mk = lambda **kw: I.Mesh(dim=kw.get("dim", m.dim), vertices=kw.get("v", m.vertices),
                             int_faces=kw.get("i", m.int_faces), hang_faces=kw.get("h", m.hang_faces),
                             bdry_faces=kw.get("b", m.bdry_faces))
    assert status(m, r=5)[0] == -2                                   # degree > 4: unsupported
    assert status(m, r=0)[0] == -1
    assert D.validate_mesh(m, 2, D.DG_NODES_GLL) == 0                # Gauss-Lobatto nodes accepted
    assert status(m, node_set=7)[0] == -1                            # unknown node set
    assert status(mk(i=m.int_faces[1:]))[0] == -1                     # an uncovered face
    assert "covered 0 times" in status(mk(i=m.int_faces[1:]))[1]
    assert "covered 2 times" in status(mk(i=np.vstack([m.int_faces, m.int_faces[:1]])))[1]
    assert "misses a subface" in status(mk(h=m.hang_faces[1:]))[1]
    bad_cell = m.int_faces.copy()
    bad_cell[0, 2] = m.n_elem
    assert "out of range" in status(mk(i=bad_cell))[1]
    b = m.bdry_faces.copy()
    b[0, 2] = I.BC_FARFIELD                                            # far-field faces accepted
    assert D.validate_mesh(mk(b=b), 2) == 0
    b[0, 2] = 7
    assert "unknown boundary condition" in status(mk(b=b))[1]
    v = m.vertices.copy()
    v[2, 1, 0] = np.nan
    assert "non-finite" in status(mk(v=v))[1]
    empty = I.Mesh(dim=2, vertices=np.zeros((0, 4, 2)), int_faces=np.zeros((0, 4), np.int64),
                   hang_faces=np.zeros((0, 5), np.int64), bdry_faces=np.zeros((0, 3), np.int64))
    assert status(empty)[0] == -1
    assert D.load().dg_mesh_validate(None) == -1
