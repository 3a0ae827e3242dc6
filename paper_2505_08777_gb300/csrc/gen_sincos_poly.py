"""Coefficients of the FP32-pipe sine / cosine (sincos2_poly in common.cuh).

With t = x / (2 pi), r = t - rint(t) in [-1/2, 1/2] and h = pi r (the half
angle), the device evaluates
    S(u) ~ sqrt(2) sin(pi r) / r,   C(u) ~ sqrt(2) cos(pi r),   u = r^2,
as polynomials of degree 4 in u, and then
    sin x = 2 sin h cos h = (r S) C,    cos x = 2 cos^2 h - 1 = C^2 - 1.
The coefficients are a weighted least-squares fit on Chebyshev nodes of r
(near-minimax for these smooth functions), computed in float64 and rounded
to float32. Running this file prints them and the worst absolute error of
sin x and cos x over r in [-1/2, 1/2], evaluated with float32 rounding after
every operation (an upper bound for the fused multiply-adds of the device).
"""
import numpy as np

DEG_S, DEG_C = 4, 4


def fit():
    k = np.arange(4000)
    r = 0.5 * np.cos(np.pi * (k + 0.5) / len(k))      # Chebyshev nodes on [-1/2, 1/2]
    r = r[np.abs(r) > 1e-6]
    u = r * r
    s_target = np.sqrt(2.0) * np.sin(np.pi * r) / r
    c_target = np.sqrt(2.0) * np.cos(np.pi * r)
    # weight the sine fit by |r| (its error enters sin x multiplied by r)
    Vs = np.vander(u, DEG_S + 1, increasing=True)
    Vc = np.vander(u, DEG_C + 1, increasing=True)
    s = np.linalg.lstsq(Vs * np.abs(r)[:, None], s_target * np.abs(r), rcond=None)[0]
    c = np.linalg.lstsq(Vc, c_target, rcond=None)[0]
    return s.astype(np.float32), c.astype(np.float32)


def evaluate(s, c, n=200001):
    f = np.float32
    r = np.linspace(-0.5, 0.5, n).astype(np.float32)
    u = (r * r).astype(f)
    S = np.full_like(u, s[-1])
    for a in s[-2::-1]:
        S = (S * u + a).astype(f)
    C = np.full_like(u, c[-1])
    for a in c[-2::-1]:
        C = (C * u + a).astype(f)
    sinx = ((r * S).astype(f) * C).astype(f)
    cosx = (C * C - f(1.0)).astype(f)
    x = 2.0 * np.pi * r.astype(np.float64)
    return float(np.max(np.abs(sinx - np.sin(x)))), float(np.max(np.abs(cosx - np.cos(x))))


if __name__ == "__main__":
    s, c = fit()
    es, ec = evaluate(s, c)
    print("S:", ", ".join(f"{v:.9e}f" for v in s))
    print("C:", ", ".join(f"{v:.9e}f" for v in c))
    print(f"max |sin error| {es:.3e}, max |cos error| {ec:.3e}")
