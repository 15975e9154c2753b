"""The allocation-free inner product agrees with bsmps_dot and with the oracle.

bsmps_dot_noalloc keeps every temporary in a fixed 32 MiB device array so that
callers which cannot allocate device memory can still take inner products.
This file is collected last on purpose: it runs after every other GPU test
and also passes on its own in a fresh process.
"""
import math

import numpy as np
import pytest

from synth import hubbard_chain, random_block_values, spinless_random_chain
from tests._common import n_random

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2604_16118_gb300 import build, native
    build.build()
    return native


@pytest.fixture(scope="module")
def ctx(nat):
    return nat.Context(0)


def rand(nat, ctx, wl, r, seed):
    vals = random_block_values(n_random(wl, r), seed)
    return nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r, vals)


@pytest.mark.parametrize("wl,r,gamma", [(spinless_random_chain(K=12, N=6, seed=0), 32, 3.0),
                                         (hubbard_chain(L=8, U=4.0), 40, 1.0)])
def test_noalloc_dot_matches_dot_twice(nat, ctx, wl, r, gamma):
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    a, b = rand(nat, ctx, wl, r, 1), rand(nat, ctx, wl, max(2, r // 2), 2)
    na, nb = math.sqrt(nat.dot(ctx, a, a)), math.sqrt(nat.dot(ctx, b, b))
    hb, _ = nat.apply_H(ctx, W, b, shift=0.3)
    nhb = math.sqrt(nat.dot(ctx, hb, hb))
    # two calls in a row on different inputs: the shared scratch keeps the last call's contents
    for (x, y, op, sh, scale) in [(a, b, W, 0.3, na * nhb), (b, a, None, 0.0, na * nb),
                                  (a, b, W, 0.3, na * nhb)]:
        ref = nat.dot(ctx, x, y, op, sh)
        n_alloc = ctx.alloc_count()
        got = nat.dot_noalloc(ctx, x, y, op, sh)
        assert ctx.alloc_count() == n_alloc          # no request reached the allocator
        assert abs(got - ref) <= 1e-12 * scale


def test_noalloc_dot_matches_oracle(nat, ctx):
    # the same inner products against the FP64 oracle (Sec. 2.4 environment recursion)
    from oracle import bsmps as OB
    from tests._common import oracle_mpo, oracle_random
    wl, r, gamma = spinless_random_chain(K=10, N=5, seed=4), 16, 2.0
    va, vb = random_block_values(n_random(wl, r), 7), random_block_values(n_random(wl, 8), 8)
    a = nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r, va)
    b = nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, 8, vb)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    oa, ob = oracle_random(wl, r, va), oracle_random(wl, 8, vb)
    oW = oracle_mpo(wl, gamma)
    na, nb = math.sqrt(OB.dot(oa, oa)), math.sqrt(OB.dot(ob, ob))
    nhb = math.sqrt(OB.dot(OB.apply_exact(oW, ob, 0.3), OB.apply_exact(oW, ob, 0.3)))
    for _ in range(2):
        assert abs(nat.dot_noalloc(ctx, a, b, W, 0.3) - OB.dot(oa, ob, oW, 0.3)) <= 1e-12 * na * nhb
        assert abs(nat.dot_noalloc(ctx, a, b) - OB.dot(oa, ob)) <= 1e-12 * na * nb


def test_noalloc_rejects_contractions_beyond_the_scratch(nat, ctx):
    wl = spinless_random_chain(K=14, N=7, seed=3)
    x = rand(nat, ctx, wl, 32, 3)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, 0, 7, 1.0)
    y, _ = nat.apply_H(ctx, W, x)          # ranks in the thousands: environments of GBs
    with pytest.raises(nat.BsmpsError) as ei:
        nat.dot_noalloc(ctx, y, y, W)
    assert ei.value.code == 4 and "scratch" in str(ei.value)
    # the failed call leaves the entry point usable
    a = rand(nat, ctx, spinless_random_chain(K=8, N=4, seed=1), 8, 4)
    assert abs(nat.dot_noalloc(ctx, a, a) - nat.dot(ctx, a, a)) <= 1e-12 * nat.dot(ctx, a, a)
