"""Property tests of the oracle transforms (Sec. II: F_n = sum_m K_n(m) f_m,
K_n(m) = exp(-i C_n . Z_m), and its adjoint) on random small problems:
linearity, a global phase, spot permutation, conjugate symmetry, and
chunking and thread-pool invariance (the closed-form and brute-force pins
are in test_oracle_transform.py). Each property fails under a plausible
slip: a dropped or doubled term, a sign that does not flip with C, spots
mixed up, a chunk added twice."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import transform  # noqa: E402

shapes = st.tuples(st.integers(1, 9), st.integers(1, 5), st.integers(1, 300), st.integers(0, 2**31 - 1))


def _problem(N, D, M, seed):
    rng = np.random.default_rng(seed)
    C = rng.normal(0.0, 2.0, (N, D))
    Z = rng.normal(0.0, 1.0, (D, M))
    f = rng.normal(size=M) + 1j * rng.normal(size=M)
    g = rng.normal(size=M) + 1j * rng.normal(size=M)
    y = rng.normal(size=N) + 1j * rng.normal(size=N)
    return rng, C, Z, f, g, y


def _close(a, b, tol=1e-12):
    return np.linalg.norm(a - b) <= tol * max(1.0, np.linalg.norm(b))


@settings(max_examples=40, deadline=None)
@given(shapes, st.floats(-3.0, 3.0), st.floats(-3.0, 3.0))
def test_linearity_and_global_phase(s, a, c):
    _, C, Z, f, g, _ = _problem(*s)
    lhs = transform.forward(a * f + 1j * g, C, Z)
    rhs = a * transform.forward(f, C, Z) + 1j * transform.forward(g, C, Z)
    assert _close(lhs, rhs)
    assert _close(transform.forward(np.exp(1j * c) * f, C, Z), np.exp(1j * c) * transform.forward(f, C, Z))


@settings(max_examples=40, deadline=None)
@given(shapes)
def test_spot_permutation_and_conjugate_symmetry(s):
    rng, C, Z, f, _, y = _problem(*s)
    perm = rng.permutation(C.shape[0])
    E = transform.forward(f, C, Z)
    assert _close(transform.forward(f, C[perm], Z), E[perm])
    # conj(F) of conj(f) through -C: the kernel sign flips with C
    assert _close(transform.forward(f.conj(), -C, Z), E.conj())
    assert _close(transform.adjoint(y[perm], C[perm], Z), transform.adjoint(y, C, Z))


@settings(max_examples=25, deadline=None)
@given(shapes, st.integers(1, 64), st.integers(1, 4))
def test_chunking_and_workers_do_not_change_the_sums(s, chunk, workers):
    _, C, Z, f, _, y = _problem(*s)
    assert _close(transform.forward(f, C, Z, chunk=chunk, workers=workers), transform.forward(f, C, Z), 1e-13)
    assert _close(transform.adjoint(y, C, Z, chunk=chunk, workers=workers), transform.adjoint(y, C, Z), 1e-13)
