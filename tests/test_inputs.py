"""The synthetic mesh generator (CPU): refined terrain-following meshes stay
exactly terrain-following, and their 2:1 faces stay watertight."""
import numpy as np

from paper_2605_29598_gb300 import inputs as I


def _refined_hill():
    # non-dyadic cell sizes (as the 200 km / 60 hill workload), two levels
    # of refinement around a Gal-Chen hill
    return I.box_mesh((6, 5, 4), (6 * 200e3 / 60, 5 * 200e3 / 60, 4e3),
                      hill=dict(h0=400.0, a_c=5e3, xc=10e3, yc=8e3),
                      refine_level=lambda c: 2 if abs(c[0] - 10e3) < 4e3 and c[2] < 2e3 else 0)


def test_refined_gal_chen_cells_are_exactly_terrain_following():
    """Horizontal coordinate c of every corner equals that of the corner with
    only bit c kept, bit for bit (the test the library applies at mesh
    creation to take the five-term metric)."""
    m = _refined_hill()
    assert len(m.hang_faces) > 0 and m.level.max() == 2
    V = m.vertices
    for c in range(m.dim - 1):
        bit = 1 << c
        for k in range(1 << m.dim):
            assert np.array_equal(V[:, k, c], V[:, k & bit, c]), (c, k)


def test_hanging_faces_stay_watertight():
    """The corners of every fine face lie on its coarse face: the coarse
    face's bilinear map at the subface corner equals the fine corner."""
    m = _refined_hill()
    d = m.dim
    bits = np.array([[(v >> t) & 1 for t in range(d)] for v in range(1 << d)])
    worst = 0.0
    for ec, fc, ef, ff, sub in m.hang_faces:
        ac, sc = fc // 2, fc % 2
        af, sf = ff // 2, ff % 2
        tang = [t for t in range(d) if t != ac]
        # corners of the fine face, and their reference position on the coarse face
        fine_corners = [v for v in range(1 << d) if bits[v][af] == sf]
        for v in fine_corners:
            x_f = m.vertices[ef, v]
            xi = np.zeros(d)
            xi[ac] = sc
            for j, t in enumerate(tang):
                half = (sub >> j) & 1
                xi[t] = 0.5 * (half + bits[v][t])
            w = np.prod(np.where(bits > 0, xi, 1.0 - xi), axis=1)
            x_c = w @ m.vertices[ec]
            worst = max(worst, np.abs(x_f - x_c).max())
    assert worst < 1e-9, worst
