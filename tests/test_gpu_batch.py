"""The batched zip-up application (bsmps_apply_zipup_batch): independent problems
of different operators, sites, particle numbers and ranks advanced together,
against the oracle's zip-up per problem and against separate calls."""
import math

import numpy as np
import pytest

from oracle import bsmps as OB
from synth import hubbard_chain, molecule_like, random_block_values, spinless_random_chain
from tests._common import n_random, oracle_mpo, oracle_random, rel_distance, to_oracle

pytestmark = pytest.mark.gpu

BATCH = [
    (spinless_random_chain(K=6, N=3, seed=11), 6, 0.4),
    (spinless_random_chain(K=9, N=4, seed=12), 12, 0.7),
    (hubbard_chain(L=3, n_up=2, n_dn=1, U=2.0), 6, 1.0),
    (hubbard_chain(L=5, U=4.0), 16, 1.5),
    (molecule_like(L=3, n_up=2, n_dn=1, seed=13), 8, 2.0),
    (molecule_like(L=4, n_up=2, n_dn=2, seed=14), 12, 2.5),
    (spinless_random_chain(K=12, N=6, seed=15), 32, 3.0),
    (hubbard_chain(L=6, U=4.0), 24, 0.8),
]


@pytest.fixture(scope="module")
def nat():
    from paper_2604_16118_gb300 import build, native
    build.build()
    return native


@pytest.fixture(scope="module")
def ctx(nat):
    return nat.Context(0)


def test_batched_zipup_matches_oracle_and_separate_calls(nat, ctx):
    Ws, xs, shifts, oys = [], [], [], []
    for i, (wl, r, gamma) in enumerate(BATCH):
        vals = random_block_values(n_random(wl, r), 40 + i)
        xs.append(nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r, vals))
        Ws.append(nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma))
        shifts.append(-0.3 * (i + 1))
        oys.append(OB.apply_zipup(oracle_mpo(wl, gamma), oracle_random(wl, r, vals), shift=shifts[-1]))
    ys, fl = nat.apply_zipup_batch(ctx, Ws, xs, shifts)
    assert len(ys) == len(BATCH) and fl > 0
    for i, (wl, r, gamma) in enumerate(BATCH):
        y1, _ = nat.apply_zipup(ctx, Ws[i], xs[i], shift=shifts[i])
        assert ys[i].bonds() == oys[i].bonds == y1.bonds()
        got = to_oracle(wl, ys[i])
        assert rel_distance(got, oys[i]) <= 1e-12
        a, b = ys[i].export(), y1.export()
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-300)


def test_batch_of_one_and_empty_batch(nat, ctx):
    wl, r, gamma = BATCH[3]
    vals = random_block_values(n_random(wl, r), 3)
    x = nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r, vals)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    ys, _ = nat.apply_zipup_batch(ctx, [W], [x], [0.25])
    y1, _ = nat.apply_zipup(ctx, W, x, shift=0.25)
    assert ys[0].bonds() == y1.bonds()
    assert nat.apply_zipup_batch(ctx, [], [], [])[0] == []


def test_recorded_plan_replays_the_batch(nat):
    """bsmps_plan_apply_zipup_batch: the batch recorded as one CUDA graph; every
    launch reproduces the oracle's zip-up of the values the inputs hold at that
    point (rewritten in place between launches), and counts its kernels."""
    import torch
    stream = torch.cuda.Stream(device=torch.device("cuda", 0))
    ctx = nat.Context(0, stream.cuda_stream)
    Ws, xs, shifts = [], [], []
    for i, (wl, r, gamma) in enumerate(BATCH):
        vals = random_block_values(n_random(wl, r), 60 + i)
        xs.append(nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r, vals))
        Ws.append(nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma))
        shifts.append(0.2 * (i + 1))
    plan = nat.ZipupPlan(ctx, Ws, xs, shifts)
    assert plan.flops > 0 and plan.launch_count() > 0
    for rep, seed0 in enumerate((60, 80, 100)):
        if rep:
            for i, (wl, r, _) in enumerate(BATCH):
                xs[i].write(random_block_values(n_random(wl, r), seed0 + i))
        l0 = ctx.launch_count()
        plan.launch()
        ctx.sync()
        assert ctx.launch_count() - l0 == plan.launch_count()
        for i, (wl, r, gamma) in enumerate(BATCH):
            vals = random_block_values(n_random(wl, r), seed0 + i)
            oy = OB.apply_zipup(oracle_mpo(wl, gamma), oracle_random(wl, r, vals), shift=shifts[i])
            assert plan.outputs[i].bonds() == oy.bonds
            assert rel_distance(to_oracle(wl, plan.outputs[i]), oy) <= 1e-12
    del plan


def test_plan_needs_a_stream(nat, ctx):
    wl, r, gamma = BATCH[0]
    x = nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r, random_block_values(n_random(wl, r), 1))
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    with pytest.raises(nat.BsmpsError):
        nat.ZipupPlan(ctx, [W], [x], [0.0])
