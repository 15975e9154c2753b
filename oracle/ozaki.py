"""FP64 matrix product emulated by exact low-precision slice products (the
Ozaki scheme: Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
multiplication by using fast routines of matrix multiplication and its
applications", Numer. Algorithms 59 (2012); integer-slice form as in Uchino,
Ozaki, Imamura 2024).  Not part of the paper: an FP64 path on tensor cores for
the contractions of the solver.

Test infrastructure only (see ``oracle/__init__.py``).

Definition followed here (integer slices of B_SLICE = 7 bits plus sign, so that
every slice is exact in bf16 and every slice product exact in FP32):
* row i of A is scaled by 2^-e_i, e_i the smallest integer with
  max_j |a_ij| < 2^e_i; column j of B by 2^-f_j likewise;
* the scaled value r in (-1, 1) is cut into S digits d_1..d_S in [-127, 127]:
  d_p = trunc(r 2^7) (toward zero), r <- r 2^7 - d_p, so that
  a_ij = 2^e_i (sum_p d_p 2^{-7p} + rest), |rest| < 2^{-7S};
* C = sum over pairs (p, q) with p + q <= S + 1 of 2^{e_i + f_j - 7(p + q)}
  (A_p B_q)_ij, where the integer products A_p B_q are exact.
Only the final FP64 accumulation over the pairs rounds.
"""

import numpy as np

B_SLICE = 7


def exponents(M, axis):
    """Smallest integer e with max |m| < 2^e along the given axis (0 where all zero)."""
    mx = np.max(np.abs(M), axis=axis)
    e = np.zeros(mx.shape, dtype=np.int64)
    nz = mx > 0
    # frexp: mx = m 2^k with 0.5 <= m < 1, so mx < 2^k
    _, k = np.frexp(mx[nz])
    e[nz] = k
    return e


def split(M, S, scale_exp, axis):
    """Integer digits (S arrays of int64 in [-127, 127]) of M scaled by
    2^-scale_exp along `axis` (rows: axis=1 means per-row exponents)."""
    if axis == 1:
        r = np.ldexp(M, -scale_exp[:, None])
    else:
        r = np.ldexp(M, -scale_exp[None, :])
    digits = []
    for _ in range(S):
        r = r * 2.0 ** B_SLICE          # exact: a power-of-two scaling
        d = np.trunc(r)
        digits.append(d.astype(np.int64))
        r = r - d                       # exact: d holds the leading bits of r
    return digits


def gemm(A, B, S=8):
    """C = A B by the slice products above (FP64 result)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    e = exponents(A, axis=1)
    f = exponents(B, axis=0)
    Ad = split(A, S, e, axis=1)
    Bd = split(B, S, f, axis=0)
    C = np.zeros((A.shape[0], B.shape[1]))
    for d in range(2, S + 2):
        acc = np.zeros((A.shape[0], B.shape[1]), dtype=np.int64)
        for p in range(1, S + 1):
            q = d - p
            if 1 <= q <= S:
                acc += Ad[p - 1] @ Bd[q - 1]          # exact integer product
        C += np.ldexp(acc.astype(np.float64), -B_SLICE * d)
    return np.ldexp(np.ldexp(C, e[:, None]), f[None, :])


def error_bound(A, B, S=8):
    """Bound on |C_emulated - A B| elementwise, in units of 2^{e_i + f_j} K:
    each factor's digits below 2^{-7S} (at most 2^{-7S} per factor, so
    2^{1-7S} for a product of two numbers below 1), the pairs with
    p + q = d > S + 1 (2S - d + 1 pairs, each below 2^{14 - 7d}), and the FP64
    rounding of the S-term recombination (S 2^{-52})."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    K = A.shape[1]
    e = exponents(A, axis=1)
    f = exponents(B, axis=0)
    scale = np.ldexp(np.ldexp(np.ones((A.shape[0], B.shape[1])), e[:, None]), f[None, :])
    dropped = sum((2 * S - d + 1) * 2.0 ** (2 * B_SLICE - B_SLICE * d) for d in range(S + 2, 2 * S + 1))
    return scale * K * (2.0 ** (1 - B_SLICE * S) + dropped + S * 2.0 ** -52)
