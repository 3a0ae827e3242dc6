"""Principal isoplanatic modes through the C ABI (host FP64 SVD, no GPU)
against the oracle (oracle/svd.py, pinned in test_oracle_wgs_grad_svd)."""
import numpy as np
import pytest

from oracle import svd
from workloads import config_c2, random_problem


def _pm(C, cols, K):
    from paper_2505_08777_gb300 import principal_modes
    return principal_modes(C, cols, K)


def _oracle_mix(C, cols, K):
    """The oracle's rotation as a mixing matrix over the D input modes."""
    D = C.shape[1]
    keep = [d for d in range(D) if d not in cols]
    _, s, Vt = svd.principal_modes(C[:, cols].astype(np.float64), K)
    mix = np.zeros((len(keep) + K, D))
    for r, d in enumerate(keep):
        mix[r, d] = 1.0
    mix[len(keep):, cols] = Vt
    C2, _ = svd.rotate(C.astype(np.float64), np.eye(D), cols, K)
    return mix, C2, svd.principal_modes(C[:, cols].astype(np.float64))[1]


@pytest.mark.parametrize("K", [8, 5, 1])
def test_principal_modes_match_oracle(K):
    p = config_c2(1)                      # 50 isoplanatic patches x Noll 4-11, tilts per spot
    C = p.coeff
    cols = list(range(2, 10))             # every mode but the two tilts
    mix, Cout, sigma = _pm(C, cols, K)
    mix_o, C2_o, sigma_o = _oracle_mix(C, cols, K)
    np.testing.assert_allclose(sigma, sigma_o, rtol=1e-9, atol=1e-12 * sigma_o[0])
    # the rotated problem's coefficient-basis product is sign-free: compare it
    np.testing.assert_allclose(Cout.astype(np.float64) @ mix, C2_o @ mix_o, rtol=0, atol=1e-5 * np.abs(C).max())
    # each principal row equals the oracle's up to sign, rows orthonormal
    for k in range(2, 2 + K):
        assert abs(abs(mix[k] @ mix_o[k]) - 1.0) < 1e-9
    P = mix[2:]
    np.testing.assert_allclose(P @ P.T, np.eye(K), atol=1e-12)
    # the tilts pass through untouched
    np.testing.assert_array_equal(mix[:2, :2], np.eye(2))
    np.testing.assert_array_equal(Cout[:, :2], C[:, :2])
    assert np.all(np.diff(sigma) <= 0)


def test_full_rank_rotation_reproduces_coefficients():
    p = random_problem(4, 32, 32, 300, list(range(2, 14)), defocus_max=4.0)
    cols = [2, 3, 5, 7, 9, 11]
    mix, Cout, sigma = _pm(p.coeff, cols, len(cols))
    np.testing.assert_allclose(Cout.astype(np.float64) @ mix, p.coeff, atol=2e-6 * np.abs(p.coeff).max())


def test_principal_modes_rejects_bad_arguments():
    from paper_2505_08777_gb300._lib import AshError
    C = np.ones((4, 3), np.float32)
    with pytest.raises(AshError):
        _pm(C, [0, 0], 1)                 # repeated column
    with pytest.raises(AshError):
        _pm(C, [0, 5], 1)                 # out of range
    with pytest.raises(AshError):
        _pm(C, [0, 1], 3)                 # K > ncols
