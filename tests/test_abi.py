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
