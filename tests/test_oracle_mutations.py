"""The oracle's pins must catch plausible mistakes (CPU).

Each case plants one mistake in an oracle function -- a flipped sign, a
dropped term, a swapped or transposed operand -- and runs a pin that must
then fail. The mistakes are planted with monkeypatch in the oracle on the
CPU and undone after each case; the pins themselves are the unmodified
tests of test_oracle_*.py.
"""
import math

import numpy as np
import pytest

import test_oracle_cg as PC
import test_oracle_transform as PT
import test_oracle_wgs_grad_svd as PW
import test_oracle_zernike as PZ
import test_oracle_zsub as PS
from oracle import cg, grad, svd, transform, wgs, zernike, zsub


def _forward_sign(mp):
    orig = transform.forward
    mp.setattr(transform, "forward", lambda f, C, Z, chunk=transform.CHUNK, workers=1: orig(f, -np.asarray(C), Z,
                                                                                          chunk, workers))


def _adjoint_unconjugated(mp):
    orig = transform.adjoint
    mp.setattr(transform, "adjoint", lambda y, C, Z, chunk=transform.CHUNK, workers=1: orig(y, -np.asarray(C), Z,
                                                                                          chunk, workers))


def _forward_drops_last_chunk(mp):
    orig = transform.forward

    def bad(f, C, Z, chunk=transform.CHUNK, workers=1):
        f = np.asarray(f, np.complex128).ravel().copy()
        M = f.size
        last = ((M - 1) // chunk) * chunk
        if last > 0:
            f[last:] = 0.0
        return orig(f, C, Z, chunk, workers)
    mp.setattr(transform, "forward", bad)


def _radial_no_alternating_sign(mp):
    def bad(n, am, rho):
        out = np.zeros_like(rho, dtype=np.float64)
        for k in range((n - am) // 2 + 1):
            c = math.factorial(n - k) / (math.factorial(k) * math.factorial((n + am) // 2 - k)
                                         * math.factorial((n - am) // 2 - k))
            out = out + c * rho ** (n - 2 * k)
        return out
    mp.setattr(zernike, "radial", bad)


def _noll_m_sign(mp):
    orig = zernike.noll_to_nm
    mp.setattr(zernike, "noll_to_nm", lambda j: (orig(j)[0], -orig(j)[1]))


def _xy_swapped(mp):
    orig = zernike.pixel_coords

    def bad(nx, ny):
        x, y = orig(nx, ny)
        return y, x
    mp.setattr(zernike, "pixel_coords", bad)


def _wgs_ratio_inverted(mp):
    def bad(E, w, target, feedback=1.0, psi=None):
        t = np.asarray(target, np.float64)
        t_hat = t / np.linalg.norm(t)
        a = np.abs(E)
        e_hat = a / np.linalg.norm(a)
        w = w * (e_hat / np.maximum(t_hat, 1e-30)) ** feedback
        w = w / np.linalg.norm(w)
        if psi is None:
            psi = transform.phase_of(E)
        return w, w * np.exp(1j * psi)
    mp.setattr(wgs, "weight_update", bad)


def _uniformity_half_denominator(mp):
    def bad(E, target):
        I = np.abs(E) ** 2 / np.asarray(target, np.float64) ** 2
        return 1.0 - (I.max() - I.min()) / I.max()
    mp.setattr(wgs, "uniformity", bad)


def _grad_drops_mean_coupling(mp):
    def bad(E, t):
        I = np.abs(E) ** 2
        mu = I.mean()
        r = I / mu - np.asarray(t, np.float64)
        return 2.0 * (2.0 / mu) * r * E
    mp.setattr(grad, "grad_E", bad)


def _phase_gradient_sign(mp):
    orig = grad.backward

    def bad(amp, phase, C, Z, ghat):
        dphi, dC = orig(amp, phase, C, Z, ghat)
        return -dphi, dC
    mp.setattr(grad, "backward", bad)


def _svd_transposed(mp):
    orig = svd.principal_modes

    def bad(W, K=None):
        U, s, Vt = orig(W, K)
        return U, s, Vt.T
    mp.setattr(svd, "principal_modes", bad)


def _cg_step_sign(mp):
    def bad(fun, fun_grad, x0, iters, theta):
        x = np.array(x0, np.float64, copy=True)
        L, g = fun_grad(x)
        d = -g
        losses = [L]
        for _ in range(iters):
            s = float(g @ d)
            mx = float(np.max(np.abs(d)))
            if mx == 0.0:
                losses.append(L)
                continue
            a0 = theta / mx
            c = (fun(x + a0 * d) - L - s * a0) / (a0 * a0)
            a = s / (2.0 * c) if c > 0 else 2.0 * a0          # sign lost
            x = x + a * d
            g_old = g
            L, g = fun_grad(x)
            d = -g + max(0.0, float(g @ (g - g_old)) / float(g_old @ g_old)) * d
            losses.append(L)
        return x, losses
    mp.setattr(cg, "minimize", bad)


def _zsub_vertex_sign(mp):
    orig = zsub.estimate
    mp.setattr(zsub, "estimate", lambda I, deltas: -orig(I, deltas))


def _zsub_sweep_sign(mp):
    orig = zsub.sweep
    mp.setattr(zsub, "sweep", lambda amp, phase, C, Z, mode, deltas, workers=1:
               orig(amp, phase, C, Z, mode, -np.asarray(deltas, np.float64), workers))


CASES = [
    ("forward kernel sign", _forward_sign, lambda: PT.test_integer_bin_tilts_equal_fft_bins(16, 12)),
    ("adjoint without conjugation", _adjoint_unconjugated, PT.test_adjoint_identity),
    ("forward drops its last pixel chunk", _forward_drops_last_chunk, PT.test_chunking_and_workers_do_not_change_result),
    ("radial polynomial without (-1)^k", _radial_no_alternating_sign, PZ.test_closed_forms_on_grid),
    ("Noll index with m negated", _noll_m_sign, lambda: PZ.test_noll_table(2, 1, 1)),
    ("pixel x and y swapped", _xy_swapped, PZ.test_coordinate_reading_small_grid),
    ("WGS weight ratio inverted", _wgs_ratio_inverted, PW.test_wgs_matches_fft_implementation_on_integer_bins),
    ("uniformity with max I as denominator", _uniformity_half_denominator, PW.test_uniformity_definition),
    ("loss gradient without the mean coupling", _grad_drops_mean_coupling, PW.test_gradient_matches_finite_differences),
    ("phase gradient sign", _phase_gradient_sign, PW.test_gradient_matches_finite_differences),
    ("SVD right factor transposed", _svd_transposed, PW.test_svd_reconstruction_and_full_rotation),
    ("CG line-search step sign", _cg_step_sign, PC.test_quadratic_is_minimised_in_n_steps),
    ("calibration vertex sign", _zsub_vertex_sign, PS.test_single_spot_vertex_is_the_model_error),
    ("calibration sweep sign", _zsub_sweep_sign, PS.test_sweep_equals_shifted_coefficients),
]


@pytest.mark.parametrize("name,plant,pin", CASES, ids=[c[0] for c in CASES])
def test_pin_catches_planted_mistake(name, plant, pin, monkeypatch):
    pin()            # the pin passes on the oracle as it is
    plant(monkeypatch)
    with pytest.raises(AssertionError):
        pin()
