"""Truncation of exactly applied MPO x MPS products with sectors of several
hundred rows (the general-size factorisation path, including the grid-wide
one-sided Jacobi) on the GPU vs the oracle, through the C ABI.

Kept dimensions are compared bit-exactly; the truncated tensors through their
Gram matrices (1e-12 relative) and the discarded norms."""
import numpy as np
import pytest

from oracle import bsmps as OB
from synth import random_block_values, spinless_random_chain
from tests._common import n_random, oracle_mpo, oracle_random, to_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2604_16118_gb300 import build, native
    build.build()
    return native


@pytest.fixture(scope="module")
def ctx(nat):
    return nat.Context(0)


@pytest.mark.parametrize("eps_rel", [1e-3, 1e-7, 1e-11])
def test_truncate_large_sectors_matches_oracle(nat, ctx, eps_rel):
    wl = spinless_random_chain(K=10, N=5, seed=1)
    r = 16
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, 0.0)
    vals = random_block_values(n_random(wl, r), 3)
    x = nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r, vals)
    y, _ = nat.apply_H(ctx, W, x)
    oy = OB.apply_exact(oracle_mpo(wl, 0.0), oracle_random(wl, r, vals))
    assert y.bonds() == oy.bonds
    assert max(max(b.values()) for b in oy.bonds if b) > 200      # sectors beyond shared memory
    nrm = float(np.sqrt(OB.dot(oy, oy)))
    z, dt, _ = nat.truncate(ctx, y, eps_rel * nrm)
    oz, odt, _ = OB.truncate(oy, eps_rel * nrm)
    assert z.bonds() == oz.bonds
    gz = OB.dot(to_oracle(wl, z), to_oracle(wl, z))
    assert abs(gz - OB.dot(oz, oz)) <= 1e-12 * OB.dot(oz, oz)
    assert abs(dt - odt) <= 1e-9 * max(odt, eps_rel * nrm * 1e-3)
    # the truncation error bound of Sec. 2.2 on the GPU result
    d = OB.add(to_oracle(wl, z), oy, 1.0, -1.0)
    assert np.sqrt(max(OB.dot(d, d), 0.0)) <= eps_rel * nrm * (1 + 1e-6) + 1e-12 * nrm


@pytest.mark.parametrize("precond", [0, 32, 96])
@pytest.mark.parametrize("eps_rel", [0.3, 1e-6])
def test_truncate_with_wide_sector_svds(nat, ctx, eps_rel, precond):
    """A random spinless K = 20, N = 10 iterate at exact ranks (middle sectors of
    252): the right sweep's SVDs reach k > 110 and run on clusters, with the
    FP64 Jacobi started plainly (precond = 0) or from the FP32 Jacobi for
    k >= precond."""
    from oracle import fermion as OF
    ctx.set_jacobi_precond(precond)
    try:
        _wide_sector_case(nat, ctx, eps_rel, OF)
    finally:
        ctx.set_jacobi_precond(48)


def _wide_sector_case(nat, ctx, eps_rel, OF):
    K, N, r = 20, 10, 1024
    species = OF.site_species(K, 0)
    dims = OB.default_dims(species, (N, 0), r)
    n = OB.BSMPS(species, (N, 0), dims, [dict() for _ in range(K)]).layout()[1]
    vals = random_block_values(n, 7)
    x = nat.mps_create(ctx, K, 0, N, 0, r, vals)
    ox = OB.random_mps(species, (N, 0), r, vals)
    assert x.bonds() == ox.bonds
    nrm = float(np.sqrt(OB.dot(ox, ox)))
    z, dt, _ = nat.truncate(ctx, x, eps_rel * nrm)
    oz, odt, _ = OB.truncate(ox, eps_rel * nrm)
    assert z.bonds() == oz.bonds
    assert max(oz.ranks()) > 110 or eps_rel > 0.1
    gz = OB.dot(to_oracle_k(z, species, N), to_oracle_k(z, species, N))
    assert abs(gz - OB.dot(oz, oz)) <= 1e-12 * OB.dot(oz, oz)
    assert abs(dt - odt) <= 1e-9 * odt
    # the truncated vector itself: the sweep's cuts amplify rounding by the
    # inverse singular-value gaps at the cut (dense random spectra; 2.5e-8 seen
    # at eps = 0.3 with the plain FP64 Jacobi), so this is a check for gross
    # errors, not a rounding bound
    d = OB.add(to_oracle_k(z, species, N), oz, 1.0, -1.0)
    assert np.sqrt(max(OB.dot(d, d), 0.0)) <= 1e-6 * np.sqrt(OB.dot(oz, oz))


def to_oracle_k(z, species, N):
    return OB.BSMPS.from_flat(species, (N, 0), z.bonds(), z.export())


@pytest.mark.parametrize("min_log2", [16, 0])
def test_truncate_with_emulated_block_products(nat, ctx, min_log2):
    """Sectors of up to 560 rows (K = 12, N = 6, r = 24, exact apply), with the
    emulation threshold lowered to 2^16 flops so that the sweeps' block products
    run on the tensor cores (0: all on the FP64 units); both match the oracle."""
    wl = spinless_random_chain(K=12, N=6, seed=1)
    r = 24
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, 0.0)
    vals = random_block_values(n_random(wl, r), 3)
    x = nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r, vals)
    ctx.set_gemm_emulation(min_log2)
    try:
        y, _ = nat.apply_H(ctx, W, x)
        oy = OB.apply_exact(oracle_mpo(wl, 0.0), oracle_random(wl, r, vals))
        assert max(max(b.values()) for b in oy.bonds if b) > 500
        nrm = float(np.sqrt(OB.dot(oy, oy)))
        for eps_rel in (1e-4, 1e-10):
            z, dt, _ = nat.truncate(ctx, y, eps_rel * nrm)
            oz, odt, _ = OB.truncate(oy, eps_rel * nrm)
            assert z.bonds() == oz.bonds
            gz = OB.dot(to_oracle(wl, z), to_oracle(wl, z))
            assert abs(gz - OB.dot(oz, oz)) <= 1e-12 * OB.dot(oz, oz)
            d = OB.add(to_oracle(wl, z), oy, 1.0, -1.0)
            assert np.sqrt(max(OB.dot(d, d), 0.0)) <= eps_rel * nrm * (1 + 1e-6) + 1e-12 * nrm
    finally:
        ctx.set_gemm_emulation(0)


@pytest.mark.parametrize("eps_rel", [1e-7, 1e-9])
@pytest.mark.parametrize("precond", [0, 48])
def test_truncate_graded_spectrum(nat, ctx, precond, eps_rel):
    """x = sum_i 10^(-2i) y_i, i = 0..5, with y_i random iterates of rank 48
    (spinless K = 20, N = 10): each term lives in its own subspace of the wide
    middle sectors (spaces up to 252), so the bond spectra of the sum fall in six
    groups from 1 to 1e-10 -- the regime in which the FP32 Jacobi start has to
    rotate the small columns too (sectors up to 119 wide).  The cuts fall
    between groups (1e-7) and inside the range of singular values near 1e-8 of
    the largest, below what FP32 resolves (1e-9).  With and without that start
    the truncation keeps the oracle's dims and norm, and its discarded norm
    (singular values fixed to about 1e-16 of the largest) agrees to 1e-4.  (A
    distance ||z - x|| from the contracted <d, d> would sit below its own
    rounding floor, sqrt(eps) ||x||, here.)"""
    from oracle import fermion as OF
    K, N, r = 20, 10, 48
    species = OF.site_species(K, 0)
    dims = OB.default_dims(species, (N, 0), r)
    n = OB.BSMPS(species, (N, 0), dims, [dict() for _ in range(K)]).layout()[1]
    ctx.set_jacobi_precond(precond)
    try:
        x = ox = None
        for i in range(6):
            w = 10.0 ** (-2 * i)
            vals = random_block_values(n, 90 + i)
            y = nat.mps_create(ctx, K, 0, N, 0, r, vals)
            oy = OB.random_mps(species, (N, 0), r, vals)
            if x is None:
                x, ox = nat.add(ctx, y, y, w, 0.0), OB.add(oy, oy, w, 0.0)
            else:
                x, ox = nat.add(ctx, x, y, 1.0, w), OB.add(ox, oy, 1.0, w)
        assert x.bonds() == ox.bonds
        assert max(max(b.values()) for b in ox.bonds if b) >= 96   # sectors wide enough for the FP32 start
        nrm = float(np.sqrt(OB.dot(ox, ox)))
        z, dt, _ = nat.truncate(ctx, x, eps_rel * nrm)
        oz, odt, _ = OB.truncate(ox, eps_rel * nrm)
        assert z.bonds() == oz.bonds
        gz = OB.dot(to_oracle_k(z, species, N), to_oracle_k(z, species, N))
        assert abs(gz - OB.dot(oz, oz)) <= 1e-12 * OB.dot(oz, oz)
        assert odt > 0.1 * eps_rel * nrm and abs(dt - odt) <= 1e-4 * odt
    finally:
        ctx.set_jacobi_precond(48)
