"""Pins of oracle.lattice against Appendix A and the algebra of the D3Q27 lattice."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import lattice as L

GOLD = os.path.join(os.path.dirname(__file__), "golden", "velocity_set.txt")


def _golden():
    rows = []
    with open(GOLD) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(v) for v in line.split()])
    return rows


def test_velocity_set_and_weights_match_appendix_listing():
    rows = _golden()
    assert len(rows) == 27
    for i, cx, cy, cz, wn, wd in rows:
        assert tuple(L.C[i]) == (cx, cy, cz)
        assert L.W_EXACT[i] == Fraction(wn, wd)
    assert len({tuple(c) for c in L.C}) == 27, "27 distinct velocities"


def test_opposites_and_weight_shells():
    for i in range(27):
        assert np.all(L.C[L.OPP[i]] == -L.C[i])
        assert L.W[L.OPP[i]] == L.W[i]
        # weight depends only on |c|^2 (rest, face, edge, corner shells)
        n2 = int(np.sum(L.C[i] ** 2))
        assert L.W_EXACT[i] == [Fraction(8, 27), Fraction(2, 27), Fraction(1, 54), Fraction(1, 216)][n2]


def test_lattice_isotropy_up_to_sixth_order():
    """sum w = 1, sum w c_a c_b = cs2 delta_ab, fourth and sixth moments of the
    Maxwellian: sum w c_a c_b c_c c_d = cs4 (d_ab d_cd + d_ac d_bd + d_ad d_bc),
    sum w c_x^2 c_y^2 c_z^2 = cs6, and the odd moments vanish."""
    w = np.array([float(x) for x in L.W_EXACT])
    c = L.C.astype(float)
    cs2 = 1.0 / 3.0
    assert abs(w.sum() - 1) < 1e-15
    d = np.eye(3)
    for a in range(3):
        assert abs(np.sum(w * c[:, a])) < 1e-15
        for b in range(3):
            assert abs(np.sum(w * c[:, a] * c[:, b]) - cs2 * d[a, b]) < 1e-15
            for g in range(3):
                assert abs(np.sum(w * c[:, a] * c[:, b] * c[:, g])) < 1e-15
                for h in range(3):
                    lhs = np.sum(w * c[:, a] * c[:, b] * c[:, g] * c[:, h])
                    rhs = cs2 ** 2 * (d[a, b] * d[g, h] + d[a, g] * d[b, h] + d[a, h] * d[b, g])
                    assert abs(lhs - rhs) < 1e-15
    assert abs(np.sum(w * c[:, 0] ** 2 * c[:, 1] ** 2 * c[:, 2] ** 2) - cs2 ** 3) < 1e-16


def test_moment_matrix_determinant_and_condition():
    """det(M^T) = 3 * 2^32 exactly and cond_2(M^T) = 38.96..., properties of the 27
    polynomial rows of Eq. (Mmatrix) taken together (a wrong row changes them)."""
    assert L.MT_DET == Fraction(12884901888)
    assert L.MT_DET == 3 * 2 ** 32
    assert abs(np.linalg.cond(L.MT) - 38.9634) < 1e-3


def test_exact_inverse_is_an_inverse():
    n = 27
    A = [[Fraction(v) for v in row] for row in L.MT_INT]
    B = L.MT_INV_EXACT
    for i in range(n):
        for j in range(n):
            s = sum(A[i][k] * B[k][j] for k in range(n))
            assert s == (1 if i == j else 0)


def test_moment_rows_are_the_printed_polynomials_at_spot_velocities():
    """Row k evaluated at hand-picked velocities (worked out by hand from Eq. (Mmatrix))."""
    i = 19      # (1, 1, 1)
    expect = [1, 1, 1, 1, 1, 1, 1, 0, 0, 3, 2, 2, 2, 0, 0, 0, 1, 3, 1, 0, 1, 1, 1, 1, 1, 1, 1]
    assert [L.MT_INT[k][i] for k in range(27)] == expect
    i = 12      # (-1, 0, 1)
    expect = [1, -1, 0, 1, 0, -1, 0, 1, 0, 2, -1, 0, 1, 1, 0, 1, 0, 1, 1, -1, 0, 0, 0, 0, 0, 0, 0]
    assert [L.MT_INT[k][i] for k in range(27)] == expect


@pytest.mark.parametrize("k,support,value", [
    (4, {7: 1, 10: 1, 8: -1, 9: -1}, Fraction(1, 4)),
    (5, {11: 1, 14: 1, 12: -1, 13: -1}, Fraction(1, 4)),
    (6, {15: 1, 18: 1, 16: -1, 17: -1}, Fraction(1, 4)),
])
def test_shear_columns_of_the_inverse(k, support, value):
    """Columns 4..6 of (M^T)^{-1}: the populations whose velocity product c_a c_b is +-1
    in the single plane of the moment, with weight 1/4 (solves M^T C = e_k by hand)."""
    col = [L.MT_INV_EXACT[i][k] for i in range(27)]
    for i in range(27):
        assert col[i] == support.get(i, 0) * value
