"""The tensor-core Ozaki product on the GPU vs the oracle's Ozaki product and
the exact FP64 product, through the C ABI (device pointers from torch).

The GPU and the oracle run the same integer slice products; they differ only in
the order of the FP64 recombination, so both lie within the scheme's error bound
of the exact product."""
import numpy as np
import pytest

from oracle import ozaki as OZ

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2604_16118_gb300 import build, native
    build.build()
    return native


@pytest.fixture(scope="module")
def ctx(nat):
    return nat.Context(0)


def run(nat, ctx, A, B, S=8):
    import torch
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.full((A.shape[0], B.shape[1]), np.nan, dtype=torch.float64, device="cuda")
    nat.gemm_ozaki(ctx, dA, dB, dC, S)
    ctx.sync()
    return dC.cpu().numpy()


@pytest.mark.parametrize("M,N,K,S", [(70, 45, 300, 8), (129, 64, 1000, 8), (17, 200, 33, 6), (64, 64, 16, 4),
                                     (1, 1, 1, 8)])
def test_matches_oracle_and_exact_product(nat, ctx, M, N, K, S):
    rng = np.random.default_rng(M * 1000 + N + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-4, 4, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-4, 4, (1, N)))
    C = run(nat, ctx, A, B, S)
    bound = OZ.error_bound(A, B, S)
    oc = OZ.gemm(A, B, S)
    assert np.all(np.abs(C - oc) <= 2 * bound)
    exact = A @ B
    assert np.all(np.abs(C - exact) <= bound + K * 2.0 ** -52 * (np.abs(A) @ np.abs(B)))


def test_worst_case_digits_stay_exact(nat, ctx):
    """Every digit 127 and K = 1024: the largest FP32 accumulations the kernel
    makes; the result equals the oracle's (exact integer sums) to FP64 rounding."""
    v = np.nextafter(1.0, 0.0)     # 53 one bits below 1: the first seven digits are 127
    K = 1024
    A = np.full((64, K), v)
    B = np.full((K, 64), v)
    A[1::2] *= -1.0
    C = run(nat, ctx, A, B)
    oc = OZ.gemm(A, B)
    assert np.abs(C - oc).max() <= 8 * 2.0 ** -52 * K
    assert np.abs(C - A @ B).max() <= OZ.error_bound(A, B).max()


def test_integer_inputs_exact_and_strided_views(nat, ctx):
    import torch
    rng = np.random.default_rng(5)
    A = rng.integers(-100, 101, size=(50, 77)).astype(np.float64)
    B = rng.integers(-100, 101, size=(77, 30)).astype(np.float64)
    assert np.array_equal(run(nat, ctx, A, B), A @ B)
    # a sub-matrix view (leading dimension larger than the row)
    wide = torch.from_numpy(np.hstack([A, np.full((50, 11), 1e300)])).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.zeros((50, 30), dtype=torch.float64, device="cuda")
    nat.gemm_ozaki(ctx, wide[:, :77], dB, dC)
    ctx.sync()
    assert np.array_equal(dC.cpu().numpy(), A @ B)


def test_empty_sizes(nat, ctx):
    import torch
    A = torch.zeros((5, 0), dtype=torch.float64, device="cuda")
    B = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    C = torch.full((5, 3), 7.0, dtype=torch.float64, device="cuda")
    nat.gemm_ozaki(ctx, A, B, C)
    ctx.sync()
    assert np.array_equal(C.cpu().numpy(), np.zeros((5, 3)))
    E = torch.zeros((0, 4), dtype=torch.float64, device="cuda")
    F = torch.zeros((4, 6), dtype=torch.float64, device="cuda")
    G = torch.zeros((0, 6), dtype=torch.float64, device="cuda")
    nat.gemm_ozaki(ctx, E, F, G)
    ctx.sync()
