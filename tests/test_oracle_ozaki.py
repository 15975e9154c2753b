"""Pins of the oracle's Ozaki-scheme product (slice digits, exact slice
products, truncated recombination) against exact arithmetic."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki as OZ


def exact_product(A, B):
    """A B in exact rational arithmetic, rounded once to FP64."""
    M, K = A.shape
    N = B.shape[1]
    C = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            s = Fraction(0)
            for k in range(K):
                s += Fraction(float(A[i, k])) * Fraction(float(B[k, j]))
            C[i, j] = float(s)
    return C


def test_integer_inputs_are_exact():
    rng = np.random.default_rng(1)
    A = rng.integers(-100, 101, size=(7, 33)).astype(np.float64)
    B = rng.integers(-100, 101, size=(33, 5)).astype(np.float64)
    assert np.array_equal(OZ.gemm(A, B), A @ B)


def test_digits_reconstruct_the_factor():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((6, 20)) * np.exp(rng.uniform(-20, 20, (6, 20)))
    e = OZ.exponents(A, axis=1)
    d = OZ.split(A, 8, e, axis=1)
    assert all(np.abs(x).max() <= 127 for x in d)
    rec = sum(np.ldexp(x.astype(np.float64), -7 * (p + 1)) for p, x in enumerate(d))
    err = np.abs(np.ldexp(rec, e[:, None]) - A)
    assert np.all(err < np.ldexp(np.ones_like(A), e[:, None] - 56))
    # entries with exponents within 3 of their row maximum are reproduced exactly
    big = np.abs(A) >= np.ldexp(np.ones_like(A), e[:, None] - 3)
    assert np.all(err[big] == 0.0)


@pytest.mark.parametrize("S", [8, 6, 4])
def test_error_within_bound_against_exact_product(S):
    rng = np.random.default_rng(3 + S)
    A = rng.standard_normal((5, 24))
    B = rng.standard_normal((24, 4))
    C = OZ.gemm(A, B, S)
    X = exact_product(A, B)
    bound = OZ.error_bound(A, B, S)
    assert np.all(np.abs(C - X) <= bound)
    if S == 8:
        # full FP64 accuracy: within a few units of the exact result's magnitude
        assert np.abs(C - X).max() <= 1e-15 * np.abs(A).max(axis=1).max() * np.abs(B).max() * 24
    else:
        # the bound is not vacuous: fewer slices lose accuracy visibly
        assert np.abs(C - X).max() > 1e-15 * np.abs(X).max()


def test_matches_library_product_on_graded_inputs():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((40, 300)) * np.exp(rng.uniform(-5, 5, (40, 1)))
    B = rng.standard_normal((300, 30)) * np.exp(rng.uniform(-5, 5, (1, 30)))
    C = OZ.gemm(A, B)
    assert np.all(np.abs(C - A @ B) <= OZ.error_bound(A, B) + 300 * 2.0 ** -52 * (np.abs(A) @ np.abs(B)))
    rel = np.abs(C - A @ B).max() / (np.abs(A) @ np.abs(B)).max()
    assert rel < 1e-15
