"""Pins for the oracle's forward / adjoint spot transform (CPU only).

Pinned against: the closed form of an unaberrated spot under a flat-phase
hologram (E = sum A), the phase-conjugate hologram, numpy's FFT for
integer-bin tilts (the DFT special case of the compressed transform,
Sec. II), brute-force pure-Python sums on tiny grids, the adjoint identity
<Kx, y> = <x, K^H y>, and unitarity (Parseval) when all M bins are targeted.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import transform, zernike
from workloads import gaussian_amplitude, random_problem


def _rand_complex(rng, n):
    return rng.normal(size=n) + 1j * rng.normal(size=n)


def test_flat_phase_unaberrated_spot_is_sum_of_amplitude():
    nx, ny = 33, 20
    A = gaussian_amplitude(nx, ny).astype(np.float64)
    Z = zernike.basis(nx, ny, list(range(2, 12)))
    C = np.zeros((3, 10))
    E = transform.forward(transform.field(A, np.zeros((ny, nx))), C, Z)
    np.testing.assert_allclose(E, np.full(3, A.sum()), rtol=1e-14, atol=0)


def test_phase_conjugate_hologram_focuses_each_spot():
    p = random_problem(3, 24, 18, 5, range(2, 12), defocus_max=5.0)
    Z = zernike.basis(p.nx, p.ny, p.noll)
    C = p.coeff.astype(np.float64)
    A = p.amp.astype(np.float64).ravel()
    for n in range(p.N):
        phase = C[n] @ Z
        E = transform.forward(transform.field(A, phase), C, Z)
        assert abs(E[n] - A.sum()) < 1e-12 * A.sum()
        assert abs(E[n].imag) < 1e-12


@pytest.mark.parametrize("nx,ny", [(16, 12), (15, 9), (32, 32)])
def test_integer_bin_tilts_equal_fft_bins(nx, ny):
    rng = np.random.default_rng(7)
    R = min(nx, ny) / 2.0
    f = _rand_complex(rng, nx * ny)
    bins = [(0, 0), (1, 0), (0, 1), (-3, 2), (nx // 2 - 1, -(ny // 2) + 1), (2, -1)]
    C = np.array([[2 * math.pi * kx * R / nx, 2 * math.pi * ky * R / ny] for kx, ky in bins])
    Z = zernike.basis(nx, ny, [2, 3])
    E = transform.forward(f, C, Z)
    F = np.fft.fft2(f.reshape(ny, nx))
    for n, (kx, ky) in enumerate(bins):
        centring = np.exp(1j * math.pi * (kx * (nx - 1) / nx + ky * (ny - 1) / ny))
        expect = F[ky % ny, kx % nx] * centring
        assert abs(E[n] - expect) < 1e-11 * np.abs(f).sum()


def _brute_forward(f, C, Z):
    N, D = C.shape
    M = Z.shape[1]
    out = []
    for n in range(N):
        acc = 0j
        for m in range(M):
            ph = 0.0
            for d in range(D):
                ph += C[n][d] * Z[d][m]
            acc += f[m] * cmath.exp(-1j * ph)
        out.append(acc)
    return np.array(out)


def _brute_adjoint(y, C, Z):
    N, D = C.shape
    M = Z.shape[1]
    out = []
    for m in range(M):
        acc = 0j
        for n in range(N):
            ph = 0.0
            for d in range(D):
                ph += C[n][d] * Z[d][m]
            acc += y[n] * cmath.exp(1j * ph)
        out.append(acc)
    return np.array(out)


@pytest.mark.parametrize("nx,ny,N,noll", [(7, 5, 3, range(2, 12)), (8, 8, 4, range(2, 13)), (3, 11, 2, [4, 2])])
def test_brute_force_tiny(nx, ny, N, noll):
    p = random_problem(11, nx, ny, N, noll, defocus_max=10.0)
    rng = np.random.default_rng(5)
    Z = zernike.basis(nx, ny, p.noll)
    C = p.coeff.astype(np.float64)
    f = _rand_complex(rng, nx * ny)
    y = _rand_complex(rng, N)
    ref_E = _brute_forward(f, C, Z)
    ref_g = _brute_adjoint(y, C, Z)
    np.testing.assert_allclose(transform.forward(f, C, Z, chunk=5), ref_E, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(transform.adjoint(y, C, Z, chunk=5), ref_g, rtol=1e-12, atol=1e-12)
    K = transform.kernel_matrix(C, Z)
    np.testing.assert_allclose(K @ f, ref_E, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(K.conj().T @ y, ref_g, rtol=1e-12, atol=1e-12)


def test_adjoint_identity():
    p = random_problem(21, 40, 31, 17, range(2, 13), defocus_max=20.0)
    rng = np.random.default_rng(9)
    Z = zernike.basis(p.nx, p.ny, p.noll)
    C = p.coeff.astype(np.float64)
    x = _rand_complex(rng, p.M)
    y = _rand_complex(rng, p.N)
    lhs = np.vdot(y, transform.forward(x, C, Z))     # <Kx, y> = y^H K x
    rhs = np.vdot(transform.adjoint(y, C, Z), x)     # <x, K^H y> = (K^H y)^H x
    assert abs(lhs - rhs) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(y) * math.sqrt(p.M * p.N)


def test_all_bins_unitary():
    # With all M integer-bin tilts as spots, K / sqrt(M) is unitary.
    nx, ny = 6, 5
    R = min(nx, ny) / 2.0
    C = np.array([[2 * math.pi * kx * R / nx, 2 * math.pi * ky * R / ny]
                  for ky in range(ny) for kx in range(nx)])
    Z = zernike.basis(nx, ny, [2, 3])
    rng = np.random.default_rng(2)
    f = _rand_complex(rng, nx * ny)
    y = _rand_complex(rng, nx * ny)
    M = nx * ny
    np.testing.assert_allclose(transform.adjoint(transform.forward(f, C, Z), C, Z), M * f, atol=1e-10)
    np.testing.assert_allclose(transform.forward(transform.adjoint(y, C, Z), C, Z), M * y, atol=1e-10)
    E = transform.forward(f, C, Z)
    assert abs(np.sum(np.abs(E) ** 2) - M * np.sum(np.abs(f) ** 2)) < 1e-9 * M * np.sum(np.abs(f) ** 2)


def test_chunking_and_workers_do_not_change_result():
    p = random_problem(4, 50, 41, 9, range(2, 12))
    rng = np.random.default_rng(1)
    Z = zernike.basis(p.nx, p.ny, p.noll)
    C = p.coeff.astype(np.float64)
    f = _rand_complex(rng, p.M)
    y = _rand_complex(rng, p.N)
    E1 = transform.forward(f, C, Z)
    E2 = transform.forward(f, C, Z, chunk=97, workers=3)
    np.testing.assert_allclose(E1, E2, rtol=1e-13, atol=1e-13)
    g1 = transform.adjoint(y, C, Z)
    g2 = transform.adjoint(y, C, Z, chunk=97, workers=3)
    np.testing.assert_allclose(g1, g2, rtol=1e-13, atol=1e-13)


def test_phase_of_zero_is_zero():
    g = np.array([0j, 1j, -1 + 0j, 1 + 1j])
    np.testing.assert_allclose(transform.phase_of(g), [0.0, math.pi / 2, math.pi, math.pi / 4])
