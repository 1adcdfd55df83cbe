"""Pins against the values the paper prints (fixtures under tests/golden/,
each citing its passage): the ARK2 tableaux, the sizes of the paper's meshes,
and the convergence tables of the inertia-gravity wave, whose R1/R2 columns
also bound how far the two rotation strategies may differ."""
import math
import os

import numpy as np
import pytest

from oracle import dg_oracle as O
from paper_2605_29598_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


# ----------------------------------------------------------------------------
# Section 3: Butcher tableaux
# ----------------------------------------------------------------------------

def _printed_tableau():
    rows = list(_lines("ark2_tableau.txt"))
    env = {"sqrt": math.sqrt}
    for row in rows:
        if row[0] == "param":
            env[row[1]] = float(eval(row[2], {"__builtins__": {}}, env))
    mats = {k: np.zeros((3, 3)) for k in ("a", "at")}
    vecs = {k: np.zeros(3) for k in ("b", "bt", "c", "ct")}
    for row in rows:
        if row[0] in mats:
            mats[row[0]][int(row[1]) - 1, int(row[2]) - 1] = eval(row[3], {"__builtins__": {}}, env)
        elif row[0] in vecs:
            vecs[row[0]][int(row[1]) - 1] = eval(row[2], {"__builtins__": {}}, env)
    return env, mats, vecs


def test_oracle_tableau_is_the_printed_one():
    env, mats, vecs = _printed_tableau()
    assert O.CHI == env["chi"]
    a, at, b, c = O.ark2_tableau()
    np.testing.assert_array_max_ulp(a, mats["a"], 1)
    np.testing.assert_array_max_ulp(at, mats["at"], 1)
    # one set of weights and nodes serves both tableaux (b = bt, c = ct)
    for key in ("b", "bt"):
        np.testing.assert_array_max_ulp(b, vecs[key], 1)
    for key in ("c", "ct"):
        np.testing.assert_array_max_ulp(c, vecs[key], 1)


# ----------------------------------------------------------------------------
# Section 4: mesh sizes
# ----------------------------------------------------------------------------

def _meshes():
    out = {}
    for row in _lines("paper_meshes.txt"):
        rec = {}
        for kv in row[1:]:
            k, v = kv.split("=")
            rec[k] = [float(x) for x in v.split("x")] if "x" in v or k in ("cells", "extent_km", "eff_m",
                                                                             "cell_m") else float(v)
        out[row[0]] = rec
    return out


@pytest.mark.parametrize("name", list(_meshes()))
def test_paper_mesh_sizes(name):
    rec = _meshes()[name]
    r = int(rec["degree"])
    cells = [int(c) for c in rec["cells"]] if "cells" in rec else None
    d = len(cells) if cells else int(rec["dim"])
    n_elem = int(np.prod(cells)) if cells else int(rec["n_elem"])
    if "n_elem" in rec:
        assert n_elem == int(rec["n_elem"])
    # nodes per cell of the oracle's discretisation, on a one-cell mesh
    one = O.Discretisation(I.box_mesh([1] * d, [1e3] * d, periodic=[False] * d), r)
    assert one.Np == (r + 1) ** d
    if "dof" in rec:
        assert n_elem * one.Np == int(rec["dof"])
    if cells and "extent_km" in rec:
        ext = np.array(rec["extent_km"]) * 1e3
        mesh = I.box_mesh(cells, ext)
        assert mesh.n_elem == n_elem
        v = np.asarray(mesh.vertices).reshape(n_elem, 2 ** d, d)
        span = v.max(axis=1) - v.min(axis=1)
        size = ext / np.array(cells)
        assert np.allclose(span, size[None, :], rtol=1e-12)
        if "eff_m" in rec:
            assert np.allclose(size / r, rec["eff_m"], rtol=1e-12)
        if "cell_m" in rec:
            assert np.allclose(size, rec["cell_m"], rtol=1e-12)


# ----------------------------------------------------------------------------
# Section 4.1: convergence tables, R1 against R2
# ----------------------------------------------------------------------------

def _conv_table():
    rows = []
    for row in _lines("igw_convergence.txt"):
        vals = [None if x == "-" else float(x) for x in row[1:]]
        rows.append((row[0], vals))
    return rows


def eoc(err_coarse, err_fine, h_coarse, h_fine):
    """Experimental order of convergence between two resolutions, as the
    paper defines it in Section 4.1."""
    return math.log(err_fine / err_coarse) / math.log(h_fine / h_coarse)


# The one entry whose printed EOCs disagree with it: the R2 l2 error of w at
# dx = 20 km is printed as 1.16e-4, while the EOCs on both sides of it (5.10
# and 2.23) each imply 1.12e-4.  The fixture keeps the printed value.
INCONSISTENT = ("w", 1, 7)


def test_printed_eocs_follow_the_printed_errors():
    """The EOC columns are the paper's formula applied to the error columns
    (each error is printed to 3 digits, so the EOC agrees to 0.02), except at
    one misprinted error, which both of its neighbouring EOCs place at the
    same other value."""
    rows = _conv_table()
    for var in ("w", "p"):
        tab = [v for k, v in rows if k == var]
        assert len(tab) == 4
        for i in range(1, 4):
            h0, h1 = tab[i - 1][0], tab[i][0]
            assert tab[i][2] == tab[i - 1][2] / 2 and h1 == h0 / 2     # dt halved with dx
            for col in (3, 5, 7, 9):                                    # l2, linf of R1, R2
                bad = (var, i, col) == INCONSISTENT or (var, i - 1, col) == INCONSISTENT
                ok = abs(eoc(tab[i - 1][col], tab[i][col], h0, h1) - tab[i][col + 1]) < 0.02
                assert ok != bad, (var, i, col)
    var, i, col = INCONSISTENT
    tab = [v for k, v in rows if k == var]
    from_coarse = tab[i - 1][col] / 2 ** tab[i][col + 1]
    from_fine = tab[i + 1][col] * 2 ** tab[i + 1][col + 1]
    assert abs(from_coarse - 1.12e-4) < 5e-7 and abs(from_fine - 1.12e-4) < 5e-7
    assert abs(tab[i][col] - 1.12e-4) > 3e-6


def _r1_r2_spread():
    spread = 0.0
    for _, v in _conv_table():
        for c1, c2 in ((3, 7), (5, 9)):
            spread = max(spread, abs(v[c1] - v[c2]) / min(v[c1], v[c2]))
    return spread


def test_r1_and_r2_reach_the_same_state():
    """The paper finds R1 and R2 equivalent: their errors in the tables
    differ by at most 13 %.  On a small slice of the same test (isothermal
    background, Bretherton perturbation, f at 45 degrees, gravity), the
    oracle's two strategies solve the same coupled system, so with Picard
    iterated to convergence their states agree to the solver tolerance, and
    with the two fixed iterations of the timed runs they agree far inside
    the paper's spread.  A slip in the lagged rotation or gravity terms of
    R1, or in their implicit form in R2, breaks the first bound."""
    spread = _r1_r2_spread()
    assert 0.1 < spread < 0.15
    mesh = I.box_mesh((8, 4), (400e3, 10e3))
    disc = O.Discretisation(mesh, 3)
    q0 = I.isothermal_state(disc.node_points(), bubble=dict(dT=0.01, xc=200e3, a=50e3, H=10e3))
    for fixed, bound in ((0, 1e-8), (2, 1e-2 * spread)):
        opts = O.StepOpts(picard_rtol=1e-13, picard_maxit=40, picard_fixed=fixed, gmres_rtol=1e-13,
                          gmres_maxit=400)
        out = {}
        for variant in ("R1", "R2"):
            q = q0
            for _ in range(3):
                q = O.imex_ark2_step(disc, O.Phys(f=1.03126e-4, variant=variant), q, 20.0, opts)
            out[variant] = q - q0
        for k in range(5):
            d = np.abs(out["R1"][k] - out["R2"][k]).max() / np.abs(out["R2"][k]).max()
            assert d < bound, (fixed, k, d)
