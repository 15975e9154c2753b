"""The zip-up MPO application of the CUDA path (bsmps_apply_zipup, Sec. 2.4 fused
with the QR sweep of Sec. 2.3) against the oracle's apply_zipup.

* bond dims bit-exact (min(stacked rows, exact columns) per sector);
* the result is left-orthonormal and represents (H_gamma + s) x: its distance
  to the oracle's result is below 1e-12 of the norm;
* the gauge of the bond bases is fixed by trunc_eps: truncating both gives the
  same kept dims and block norms to 1e-12 relative to each block;
* bsmps_apply_H with a tolerance (zip-up + right sweep) equals the oracle's
  trunc(apply_exact);
* at the bench's size (Hubbard L = 32, r = 256) the dims, left orthonormality,
  the norm and amplitudes of sampled occupation strings against the oracle's
  exact application.
"""
import math

import numpy as np
import pytest

from oracle import bsmps as OB
from oracle import mpo as OM
from synth import hubbard_chain, molecule_like, random_block_values, spinless_random_chain
from tests._common import (amplitude, block_norms, n_random, oracle_mpo, oracle_random, random_occupations,
                           rel_distance, species_of, target_of, to_oracle)

pytestmark = pytest.mark.gpu

CASES = [
    ("spinless_K7", spinless_random_chain(K=7, N=3, seed=1), 6, 0.4),
    ("hubbard_L4", hubbard_chain(L=4, n_up=2, n_dn=2, U=4.0), 8, 1.0),
    ("molecule_L4", molecule_like(L=4, n_up=2, n_dn=1, seed=2), 10, 2.0),
    ("spinless_K12", spinless_random_chain(K=12, N=6, seed=0), 32, 3.0),
    ("hubbard_L8", hubbard_chain(L=8, U=4.0), 40, 1.0),
]


@pytest.fixture(scope="module")
def nat():
    from paper_2604_16118_gb300 import build, native
    build.build()
    return native


@pytest.fixture(scope="module")
def ctx(nat):
    return nat.Context(0)


def left_orthonormal_error(x):
    worst = 0.0
    for t in range(x.K - 1):
        sp = x.species[t]
        for m2, k in x.bonds[t + 1].items():
            S = np.vstack([x.cores[t][(m, s)] for (m, s) in x.block_keys(t)
                           if OB.add_charge(m, OB.delta(sp, s)) == m2])
            worst = max(worst, np.abs(S.T @ S - np.eye(k)).max())
    return worst


def gpu_random(nat, ctx, wl, r, seed):
    vals = random_block_values(n_random(wl, r), seed)
    return nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r, vals), vals


@pytest.mark.parametrize("name,wl,r,gamma", CASES)
def test_zipup_matches_oracle(nat, ctx, name, wl, r, gamma):
    x, vals = gpu_random(nat, ctx, wl, r, 21)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    oW, ox = oracle_mpo(wl, gamma), oracle_random(wl, r, vals)
    y, fl = nat.apply_zipup(ctx, W, x, shift=-0.8)
    oy = OB.apply_zipup(oW, ox, shift=-0.8)
    assert y.bonds() == oy.bonds
    assert fl > 0
    got = to_oracle(wl, y)
    assert left_orthonormal_error(got) <= 1e-13 * max(r, 8)
    nrm = math.sqrt(sum(np.sum(B * B) for B in oy.cores[-1].values()))
    gnrm = math.sqrt(sum(np.sum(B * B) for B in got.cores[-1].values()))
    assert abs(gnrm - nrm) <= 1e-13 * nrm
    assert rel_distance(got, oy) <= 1e-12
    # trunc_eps fixes the gauge: same kept dims and tensors; where every kept
    # singular value stands well above rounding (rel = 1e-3) also the same blocks
    # (at 1e-13 the kept singular vectors of values near the noise floor are not
    # determined by the data, in any FP64 implementation)
    for rel in (1e-13, 1e-3):
        t, dt, _ = nat.truncate(ctx, y, rel * nrm)
        ot, odt, _ = OB.truncate(oy, rel * nrm)
        assert t.bonds() == ot.bonds
        assert abs(dt - odt) <= 1e-12 * nrm
        assert rel_distance(to_oracle(wl, t), ot) <= 1e-12
        if rel < 1e-6:
            continue
        gn, on = block_norms(to_oracle(wl, t)), block_norms(ot)
        core_max = {}
        for (tt, _), v in on.items():
            core_max[tt] = max(core_max.get(tt, 0.0), v)
        for k in on:
            assert abs(gn[k] - on[k]) <= 1e-12 * max(on[k], 1e-3 * core_max[k[0]]), (rel, k)


@pytest.mark.parametrize("name,wl,r,gamma", CASES[1:4])
def test_apply_with_tolerance_matches_truncated_exact_application(nat, ctx, name, wl, r, gamma):
    x, vals = gpu_random(nat, ctx, wl, r, 22)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    oy = OB.apply_exact(oracle_mpo(wl, gamma), oracle_random(wl, r, vals), shift=0.5)
    nrm = math.sqrt(OB.dot(oy, oy))
    for rel, cap in ((1e-10, 0), (1e-2, 0), (1e-4, 7)):
        y, _ = nat.apply_H(ctx, W, x, shift=0.5, tol=rel * nrm, r_max=cap)
        ot, _, _ = OB.truncate(oy, rel * nrm, cap)
        assert y.bonds() == ot.bonds
        assert rel_distance(to_oracle(wl, y), ot) <= 1e-12 * max(1.0, nrm / math.sqrt(OB.dot(ot, ot)))


def test_zipup_full_size_hubbard(nat, ctx):
    """Hubbard L = 32 (K = 64 spin-orbitals), r = 256: the size of the bench."""
    wl = hubbard_chain(L=32, r_max=256)
    x, vals = gpu_random(nat, ctx, wl, 256, 3)
    ox = oracle_random(wl, 256, vals)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, 1, 32, 4.0)
    oW = OM.build_mpo(wl.h, wl.eri, 1, 32, 4.0)
    y, fl = nat.apply_zipup(ctx, W, x, shift=-1.0)
    got = to_oracle(wl, y)
    # dims: the QR sweep's rank rule on the exact bases, computed on the host
    segs = OB._exact_segments(oW, ox)
    dims = [{m: v[1] for m, v in segs[0].items()}]
    for t in range(wl.n_sites - 1):
        sp = ox.species[t]
        rows = {}
        for m, d in dims[t].items():
            for s in (0, 1):
                m2 = OB.add_charge(m, OB.delta(sp, s))
                if m2 in segs[t + 1]:
                    rows[m2] = rows.get(m2, 0) + d
        dims.append({m2: min(rw, segs[t + 1][m2][1]) for m2, rw in sorted(rows.items())})
    dims.append({m: v[1] for m, v in segs[-1].items()})
    assert got.bonds == dims
    assert left_orthonormal_error(got) <= 1e-12
    # amplitudes of sampled occupation strings against the oracle's exact application
    oy = OB.apply_exact(oW, ox, shift=-1.0)
    gnrm = math.sqrt(sum(np.sum(B * B) for B in got.cores[-1].values()))
    # (amplitudes span many orders of magnitude and some are exactly 0 in the exact
    # cores, rounding noise in the orthogonalised ones: the sampled vector is
    # compared relative to its norm)
    occs = random_occupations(species_of(wl), target_of(wl), 24, 7)
    a_ref = np.array([amplitude(oy, occ) for occ in occs])
    a_got = np.array([amplitude(got, occ) for occ in occs])
    assert np.count_nonzero(a_ref) >= 12
    assert np.linalg.norm(a_got - a_ref) <= 1e-10 * np.linalg.norm(a_ref)
    # the norm against the library's (oracle-checked) inner product of the exact application
    ye, _ = nat.apply_H(ctx, W, x, shift=-1.0)
    assert abs(gnrm ** 2 - nat.dot(ctx, ye, ye)) <= 1e-12 * gnrm ** 2
