"""D3Q27 lattice constants and the MRT moment matrix, as printed in Appendix A.

Test infrastructure (see the package docstring): only tests, smoke() and the
bench CPU baseline use it.

* Velocity set: the three columns |c_ix>, |c_iy>, |c_iz> listed at the start of
  Appendix A (the entry printed as "0,0 0" in |c_ix> is read as three zeros, which
  gives 27 distinct vectors).
* Weights: Eq. (omegas), w_0 = 8/27, w_1..6 = w_0/4, w_7..18 = w_0/16,
  w_19..26 = w_0/64.
* Moment matrix: Eq. (Mmatrix), |M_k> for k = 0..26; m = M^T f.
* c_s^2 = 1/3 (stated after Eq. (BoltzmannEquilibriumDistribution)).
"""
from fractions import Fraction

import numpy as np

# Appendix A, the three velocity columns, entry by entry.
CX = (0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1)
CY = (0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1)
CZ = (0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1)

Q = 27
C = np.array([CX, CY, CZ], dtype=np.int64).T          # (27, 3)
CS2 = 1.0 / 3.0

W0 = Fraction(8, 27)
W_EXACT = [W0] + [W0 / 4] * 6 + [W0 / 16] * 12 + [W0 / 64] * 8   # Eq. (omegas)
W = np.array([float(w) for w in W_EXACT])


def opposite():
    """Index of -c_i for every i (the bar-i of the bounce-back rule, Sec. II.A)."""
    opp = np.empty(Q, dtype=np.int64)
    for i in range(Q):
        matches = [j for j in range(Q) if all(C[j, a] == -C[i, a] for a in range(3))]
        assert len(matches) == 1
        opp[i] = matches[0]
    return opp


OPP = opposite()


def _moment_rows(cx, cy, cz):
    """The 27 polynomials |M_k> of Eq. (Mmatrix) evaluated at one velocity."""
    x2, y2, z2 = cx * cx, cy * cy, cz * cz
    return [
        1,                                  # M0
        cx,                                 # M1
        cy,                                 # M2
        cz,                                 # M3
        cx * cy,                            # M4
        cx * cz,                            # M5
        cy * cz,                            # M6
        x2 - y2,                            # M7
        x2 - z2,                            # M8
        x2 + y2 + z2,                       # M9
        cx * y2 + cx * z2,                  # M10
        x2 * cy + cy * z2,                  # M11
        x2 * cz + y2 * cz,                  # M12
        cx * y2 - cx * z2,                  # M13
        x2 * cy - cy * z2,                  # M14
        x2 * cz - y2 * cz,                  # M15
        cx * cy * cz,                       # M16
        x2 * y2 + x2 * z2 + y2 * z2,        # M17
        x2 * y2 + x2 * z2 - y2 * z2,        # M18
        x2 * y2 - x2 * z2,                  # M19
        x2 * cy * cz,                       # M20
        cx * y2 * cz,                       # M21
        cx * cy * z2,                       # M22
        cx * y2 * z2,                       # M23
        x2 * cy * z2,                       # M24
        x2 * y2 * cz,                       # M25
        x2 * y2 * z2,                       # M26
    ]


def moment_matrix_T_int():
    """M^T as integers: row k holds |M_k> over the 27 velocities, so m = M^T f."""
    cols = [_moment_rows(int(C[i, 0]), int(C[i, 1]), int(C[i, 2])) for i in range(Q)]
    return [[cols[i][k] for i in range(Q)] for k in range(Q)]


def exact_inverse(a):
    """Gauss-Jordan inverse of an integer matrix in rational arithmetic.

    Returns (inverse as a list of Fraction rows, determinant as a Fraction)."""
    n = len(a)
    m = [[Fraction(v) for v in row] + [Fraction(int(i == j)) for j in range(n)]
         for i, row in enumerate(a)]
    det = Fraction(1)
    for col in range(n):
        piv = next(r for r in range(col, n) if m[r][col] != 0)
        if piv != col:
            m[col], m[piv] = m[piv], m[col]
            det = -det
        p = m[col][col]
        det *= p
        m[col] = [v / p for v in m[col]]
        for r in range(n):
            if r != col and m[r][col] != 0:
                fac = m[r][col]
                m[r] = [vr - fac * vc for vr, vc in zip(m[r], m[col])]
    return [row[n:] for row in m], det


MT_INT = moment_matrix_T_int()
MT = np.array(MT_INT, dtype=np.float64)               # (27, 27): m = MT @ f
_MT_INV_EXACT, MT_DET = exact_inverse(MT_INT)
MT_INV = np.array([[float(v) for v in row] for row in _MT_INV_EXACT])   # f = MT_INV @ m
MT_INV_EXACT = _MT_INV_EXACT
