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


# ----------------------------------------------------------------------------
# Section 4: the experiments' configurations
# ----------------------------------------------------------------------------

def _workloads():
    out = {}
    for row in _lines("paper_workloads.txt"):
        rec = {}
        for kv in row[1:]:
            k, v = kv.split("=")
            rec[k] = [float(x) for x in v.split("x")] if k in ("extent", "cells", "hill") else float(v)
        out[row[0]] = rec
    return out


GENERATORS = {
    "igw_reference": lambda: I.paper_igw_case(),
    "planetary_igw": lambda: I.planetary_igw_case(),
    "hill_benchmark": lambda: I.paper_hill_benchmark_case(),
    "hill_large": lambda: I.paper_hill_large_case(),
}


@pytest.mark.parametrize("name", list(GENERATORS))
def test_workload_generators_follow_the_printed_configurations(name):
    rec = _workloads()[name]
    case = GENERATORS[name]()
    mesh = case["mesh"]
    cells = [int(c) for c in rec["cells"]]
    ext = np.array(rec["extent"]) * 1e3
    d = len(cells)
    assert mesh.dim == d and mesh.n_elem == int(np.prod(cells))
    assert case["degree"] == int(rec["degree"])
    assert case["dt"] == rec["dt"] and case.get("hours", rec["hours"]) == rec["hours"]
    if "f" in rec:
        assert case["f"] == rec["f"]
    v = np.asarray(mesh.vertices).reshape(-1, d)
    for a in range(d - 1):
        assert v[:, a].min() == 0.0 and abs(v[:, a].max() - ext[a]) < 1e-6 * ext[a]
    assert abs(v[:, -1].max() - ext[-1]) < 1e-6 * ext[-1]
    sp = case["state_params"]
    if "xc" in rec:
        assert sp["bubble"]["xc"] == rec["xc"] * 1e3
    if "a" in rec:
        assert sp["bubble"]["a"] == rec["a"] * 1e3
    if "hill" in rec:
        # bottom vertices follow the bell: h0 at the centre, h0 / (1 + r^2 / a_c^2) around it
        xc, yc = np.array(rec["hill"]) * 1e3
        bottom = v[v[:, 2] < 0.5 * ext[2] / cells[2]]
        r2 = (bottom[:, 0] - xc) ** 2 + (bottom[:, 1] - yc) ** 2
        h = rec["h0_m"] / (1.0 + r2 / (rec["ac"] * 1e3) ** 2)
        assert np.abs(bottom[:, 2] - h).max() < 1e-9 * rec["h0_m"]
        assert abs(bottom[:, 2].max() - rec["h0_m"]) < 1e-9 * rec["h0_m"]
        s = case["sponge"]
        assert abs(s["lambda_bar"] * case["dt"] - rec["lam_dt"]) < 1e-12
        assert s["z_t"] == ext[2] and abs(s["z_t"] - s["z_b"] - rec["damp_top"] * 1e3) < 1e-6
        assert s["x_layers"] == (0.0, ext[0], rec["damp_x"] * 1e3)
        assert s["y_layers"] == (0.0, ext[1], rec["damp_y"] * 1e3)
        assert sp["theta_ref"] == rec["theta_ref"] and sp["wind"][0] == rec["U0"]
        # N as printed (the isothermal case's g / sqrt(c_p T) = 0.0196 is printed as 0.02)
        assert abs(sp["n_bv"] - rec["N"]) < 0.025 * rec["N"]
