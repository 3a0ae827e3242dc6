"""Pins for the oracle's conjugate-gradient phase refinement (CPU).

The line search fits a quadratic through the loss, its slope and one trial
point, so on a quadratic objective it is exact and PR+ reduces to linear
CG: an n-dimensional strictly convex quadratic is minimised in n
iterations (textbook property, checked against numpy's solve). On the
hologram loss the descent must lower the loss from a WGS start and raise
the uniformity of a flat-target array (the top-hat refinement the paper
mentions); a zero gradient leaves the phase where it is.
"""
import numpy as np

from oracle import cg, grad, transform, wgs, zernike
from workloads import random_problem


def test_quadratic_is_minimised_in_n_steps():
    rng = np.random.default_rng(7)
    n = 6
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + n * np.eye(n)
    b = rng.normal(size=n)

    def fun(x):
        return 0.5 * x @ A @ x - b @ x

    def fun_grad(x):
        return fun(x), A @ x - b

    x, losses = cg.minimize(fun, fun_grad, np.zeros(n), n, theta=0.3)
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-9)
    assert all(l1 <= l0 + 1e-12 for l0, l1 in zip(losses, losses[1:]))


def test_one_step_solves_a_one_dimensional_quadratic():
    # the trial step is a quarter of the way; the quadratic fit lands on 0
    def fun(x):
        return 0.5 * float(x @ x)

    def fun_grad(x):
        return fun(x), x.copy()

    x, losses = cg.minimize(fun, fun_grad, np.array([1.0]), 1, theta=0.25)
    assert abs(x[0]) < 1e-12 and losses[-1] < 1e-20


def test_zero_gradient_stops_the_descent():
    def fun(x):
        return 3.0

    def fun_grad(x):
        return 3.0, np.zeros_like(x)

    x, losses = cg.minimize(fun, fun_grad, np.array([0.5, -0.25]), 3, theta=0.1)
    assert np.array_equal(x, [0.5, -0.25]) and losses == [3.0] * 4


def _problem():
    p = random_problem(21, 40, 36, 12, [2, 3, 4, 5, 6, 7], aberr_sigma=0.4, target_range=(1.0, 1.0))
    Z = zernike.basis(p.nx, p.ny, p.noll)
    return p, Z, p.coeff.astype(np.float64), p.amp.astype(np.float64).ravel()


def test_refinement_lowers_the_loss_and_raises_uniformity():
    p, Z, C, A = _problem()
    res = wgs.run(A, p.phase0.astype(np.float64).ravel(), C, Z, p.target, 10)
    t = p.target.astype(np.float64) ** 2 / np.mean(p.target.astype(np.float64) ** 2)
    phi, losses = cg.refine(A, res.phase, C, Z, t, 15, theta=0.05)
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
    E = transform.forward(transform.field(A, phi), C, Z)
    assert wgs.uniformity(E, p.target) > res.uniformity
    assert abs(losses[-1] - grad.loss(A, phi, C, Z, t)) <= 1e-12 * max(1.0, losses[-1])


def test_phase_gradient_matches_the_full_gradient():
    p, Z, C, A = _problem()
    t = np.ones(p.N)
    ph = p.phase0.astype(np.float64).ravel()
    L, g = cg.loss_and_phase_grad(A, ph, C, Z, t)
    L2, g2, _ = grad.grad(A, ph, C, Z, t)
    assert L == L2 and np.allclose(g, g2, rtol=0, atol=1e-14 * np.max(np.abs(g2)))
