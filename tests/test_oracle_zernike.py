"""Pins for the oracle's Zernike basis (CPU only).

Each check is tied to something outside the oracle: the published Noll
table, the paper's ANSI identities (Sec. II), textbook closed forms of the
low-order polynomials, R_n^m(1) = 1, and orthogonality on the unit disk
computed by an independent polar Gauss quadrature.
"""
import math
import os

import numpy as np
import pytest

from oracle import zernike

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "noll_table.txt")


def _noll_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            j, n, m = (int(v) for v in line.split())
            rows.append((j, n, m))
    return rows


@pytest.mark.parametrize("j,n,m", _noll_rows())
def test_noll_table(j, n, m):
    assert zernike.noll_to_nm(j) == (n, m)


def test_noll_is_bijection_in_radial_order():
    seen = set()
    for j in range(1, 300):
        n, m = zernike.noll_to_nm(j)
        assert abs(m) <= n and (n - abs(m)) % 2 == 0
        assert (n, m) not in seen
        seen.add((n, m))
        if j > 1:
            assert n >= zernike.noll_to_nm(j - 1)[0]
    # every valid (n, m) with n <= 20 appears
    for n in range(21):
        for m in range(-n, n + 1, 2):
            assert (n, m) in seen


def test_paper_ansi_identities():
    # Sec. II: x ~ Z_2 = Z_1^1, y ~ Z_1 = Z_1^-1, defocus Z_4 = Z_2^0, spherical Z_12 = Z_4^0
    assert zernike.ansi_index(1, 1) == 2
    assert zernike.ansi_index(1, -1) == 1
    assert zernike.ansi_index(2, 0) == 4
    assert zernike.ansi_index(4, 0) == 12
    for j in range(0, 120):
        assert zernike.ansi_index(*zernike.ansi_to_nm(j)) == j


def _closed_forms(x, y):
    r2 = x * x + y * y
    return {
        1: np.ones_like(x),
        2: x,
        3: y,
        4: 2 * r2 - 1,
        5: 2 * x * y,
        6: x * x - y * y,
        7: (3 * r2 - 2) * y,
        8: (3 * r2 - 2) * x,
        9: 3 * x * x * y - y ** 3,
        10: x ** 3 - 3 * x * y * y,
        11: 6 * r2 * r2 - 6 * r2 + 1,
        12: (4 * r2 - 3) * (x * x - y * y),
        13: (4 * r2 - 3) * 2 * x * y,
    }


def test_closed_forms_on_grid():
    nx, ny = 37, 23
    noll = list(range(1, 14))
    Z = zernike.basis(nx, ny, noll)
    R = min(nx, ny) / 2.0
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    x = (i - (nx - 1) / 2.0) / R
    y = (j - (ny - 1) / 2.0) / R
    ref = _closed_forms(x.ravel(), y.ravel())
    for d, jn in enumerate(noll):
        np.testing.assert_allclose(Z[d], ref[jn], rtol=0, atol=1e-12, err_msg=f"Noll {jn}")


def test_coordinate_reading_small_grid():
    # nx = 4, ny = 2: R = 1, x = i - 1.5, y = j - 0.5, flat index m = j*nx + i
    Z = zernike.basis(4, 2, [2, 3])
    np.testing.assert_allclose(Z[0], [-1.5, -0.5, 0.5, 1.5, -1.5, -0.5, 0.5, 1.5], rtol=0, atol=1e-15)
    np.testing.assert_allclose(Z[1], [-0.5, -0.5, -0.5, -0.5, 0.5, 0.5, 0.5, 0.5], rtol=0, atol=1e-15)


def test_radial_is_one_at_edge():
    one = np.array([1.0])
    for n in range(0, 13):
        for am in range(n % 2, n + 1, 2):
            assert abs(zernike.radial(n, am, one)[0] - 1.0) < 1e-9


def test_orthogonality_on_unit_disk():
    # independent polar quadrature: Gauss-Legendre in rho (exact for the
    # polynomial degrees involved), uniform trapezoid in theta (exact for
    # trigonometric polynomials of degree < 64).
    xg, wg = np.polynomial.legendre.leggauss(24)
    rho = 0.5 * (xg + 1.0)
    wr = 0.5 * wg * rho
    th = np.arange(64) * (2 * math.pi / 64)
    wt = np.full(64, 2 * math.pi / 64)
    RHO, TH = np.meshgrid(rho, th, indexing="ij")
    W = wr[:, None] * wt[None, :]
    modes = [zernike.noll_to_nm(j) for j in range(1, 29)]
    vals = [zernike.zernike_polar(n, m, RHO, TH) for (n, m) in modes]
    for a, (na, ma) in enumerate(modes):
        for b, (nb, mb) in enumerate(modes):
            ip = float(np.sum(W * vals[a] * vals[b]))
            if a == b:
                expect = math.pi / (na + 1) * (1.0 if ma == 0 else 0.5)
                assert abs(ip - expect) < 1e-12, (a, ip, expect)
            else:
                assert abs(ip) < 1e-12, (a, b, ip)
