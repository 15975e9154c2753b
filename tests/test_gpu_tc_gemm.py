"""The split-precision tensor-core GEMM (bsmps_gemm_tf32x3: tcgen05.mma kind::tf32,
operands split into two TF32 parts, three products accumulated in FP32 in tensor
memory) against the exact FP64 product on the host.

Bound: |C_ij - (AB)_ij| <= 2^-21 (4 + sqrt(K)) sum_k |a_ik| |b_kj|: a few units
of 2^-21 from the split (each operand to 2^-22) and the dropped lo x lo term,
plus the FP32 accumulation over K (random-walk size sqrt(K) 2^-24, with room).
The measured error is printed.  Sizes span several 128 x 64 tiles, ragged tails
and K below, at and above the 32-value chunk, plus the empty cases."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2604_16118_gb300 import build, native
    build.build()
    return native


@pytest.fixture(scope="module")
def ctx(nat):
    return nat.Context(0)


def run(nat, ctx, A, B):
    import torch
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.full((A.shape[0], B.shape[1]), np.nan, dtype=torch.float64, device="cuda")
    nat.gemm_tf32x3(ctx, dA, dB, dC)
    ctx.sync()
    return dC.cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (128, 64, 32), (7, 5, 3), (200, 70, 45), (300, 130, 257),
                                   (1000, 17, 33), (129, 65, 64), (64, 200, 1000)])
def test_split_precision_product_within_bound(nat, ctx, M, N, K):
    rng = np.random.default_rng(M * 7919 + N * 31 + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-3, 3, (1, N)))
    C = run(nat, ctx, A, B)
    ref = A @ B
    scale = np.abs(A) @ np.abs(B)
    err = np.abs(C - ref) / scale
    print(f"M={M} N={N} K={K}: max error / sum|a||b| = {err.max():.2e}")
    assert np.all(np.isfinite(C))
    assert err.max() <= 2.0 ** -21 * (4.0 + np.sqrt(K))


def test_split_precision_is_far_more_accurate_than_one_tf32_product(nat, ctx):
    # the lo parts matter: one TF32 product has errors near 2^-12 of sum |a||b|
    rng = np.random.default_rng(5)
    A, B = rng.standard_normal((256, 96)), rng.standard_normal((96, 128))
    err = np.abs(run(nat, ctx, A, B) - A @ B) / (np.abs(A) @ np.abs(B))
    print(f"256 x 128 x 96: max {err.max():.2e}, mean {err.mean():.2e}")
    assert err.max() <= 2.0 ** -17 and err.mean() <= 2.0 ** -20


def test_empty_and_zero_inner_dimension(nat, ctx):
    import torch
    A = torch.zeros((5, 0), dtype=torch.float64, device="cuda")
    B = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    C = torch.full((5, 3), np.nan, dtype=torch.float64, device="cuda")
    nat.gemm_tf32x3(ctx, A, B, C)
    ctx.sync()
    assert torch.all(C == 0.0)
    E = torch.zeros((0, 4), dtype=torch.float64, device="cuda")
    nat.gemm_tf32x3(ctx, E, torch.zeros((4, 2), dtype=torch.float64, device="cuda"),
                    torch.zeros((0, 2), dtype=torch.float64, device="cuda"))
    ctx.sync()
