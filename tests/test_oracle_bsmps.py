"""Pins of the oracle's block-sparse MPS operations (Sec. 2.2-2.4)."""
import json
import os

import numpy as np
import pytest

from oracle import bsmps as B
from oracle import fermion as F
from oracle import mpo as M
from synth import hubbard_chain, molecule_like, spinless_random_chain

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_mps(species, target, r_max, seed):
    dims = B.default_dims(species, target, r_max)
    tmp = B.BSMPS(species, target, dims, [dict() for _ in species])
    _, tot = tmp.layout()
    return B.BSMPS.from_flat(species, target, dims, np.random.default_rng(seed).standard_normal(tot))


def test_paper_example_block_pattern():
    g = json.load(open(os.path.join(GOLDEN, "paper_example_K5_N2.json")))
    species = (0,) * g["K"]
    target = (g["N"], 0)
    ranges = B.valid_ranges(species, target)
    assert [[q[0] for q in r] for r in ranges] == g["bond_sectors"]
    x = rand_mps(species, target, 100, 0)
    for t in range(g["K"]):
        got = [[n[0], sg] for (n, sg) in x.block_keys(t)]
        assert got == g["site_blocks"][t]


def test_dims_rule_properties():
    species = F.site_species(6, 1)
    x = rand_mps(species, (3, 3), 20, 1)
    r = x.ranks()
    assert r[0] == r[-1] == 1
    assert max(r) <= 20
    for b in range(len(species) + 1):
        for q, d in x.bonds[b].items():
            left, right = B.config_counts(species, (3, 3), b, q)
            assert 0 < d <= min(left, right)


def test_dense_contraction_lives_in_sector():
    species = F.site_species(3, 1)
    x = rand_mps(species, (2, 1), 8, 2)
    v = B.to_dense(x)
    K = len(species)
    for idx in np.nonzero(np.abs(v) > 0)[0]:
        occ = [(idx >> (K - 1 - s)) & 1 for s in range(K)]
        assert sum(occ[0::2]) == 2 and sum(occ[1::2]) == 1


@pytest.mark.parametrize("wl", [spinless_random_chain(K=7, N=3, seed=21),
                                hubbard_chain(L=3, n_up=2, n_dn=1, U=2.0),
                                molecule_like(L=3, n_up=1, n_dn=1, seed=22)])
def test_apply_add_dot_against_dense(wl):
    species = F.site_species(wl.n_orb, wl.spin)
    tgt = (wl.n_up, wl.n_dn)
    Hf = F.full_hamiltonian(wl.h, wl.eri, wl.spin, wl.n_particles, 0.9)
    mpo = M.build_mpo(wl.h, wl.eri, wl.spin, wl.n_particles, 0.9)
    x = rand_mps(species, tgt, 6, 3)
    z = rand_mps(species, tgt, 5, 4)
    xd, zd = B.to_dense(x), B.to_dense(z)
    y = B.apply_exact(mpo, x, shift=-0.25)
    assert np.abs(B.to_dense(y) - (Hf @ xd - 0.25 * xd)).max() < 1e-12
    s = B.add(x, z, 0.5, -1.5)
    assert np.abs(B.to_dense(s) - (0.5 * xd - 1.5 * zd)).max() < 1e-13
    assert abs(B.dot(x, z) - xd @ zd) < 1e-12
    assert abs(B.dot(z, x, mpo) - zd @ Hf @ xd) < 1e-11
    assert abs(B.dot(z, x, mpo, shift=0.3) - zd @ (Hf + 0.3 * np.eye(len(Hf))) @ xd) < 1e-11


def _check_left_orth(y):
    for t in range(y.K - 1):
        sp = y.species[t]
        for m in y.bonds[t + 1]:
            blocks = [y.cores[t][k] for k in y.block_keys(t)
                      if B.add_charge(k[0], B.delta(sp, k[1])) == m]
            G = sum(Bk.T @ Bk for Bk in blocks)
            assert np.abs(G - np.eye(len(G))).max() < 1e-13


def _check_right_orth(y):
    for t in range(1, y.K):
        for n in y.bonds[t]:
            blocks = [y.cores[t][(n, sg)] for sg in (0, 1) if (n, sg) in y.cores[t]]
            G = sum(Bk @ Bk.T for Bk in blocks)
            assert np.abs(G - np.eye(len(G))).max() < 1e-13


def test_orthogonalisation_and_truncation_bounds():
    wl = spinless_random_chain(K=7, N=3, seed=31)
    species = F.site_species(7, 0)
    mpo = M.build_mpo(wl.h, wl.eri, 0, 3, 0.0)
    y = B.apply_exact(mpo, rand_mps(species, (3, 0), 6, 5))
    yd = B.to_dense(y)
    lo = B.left_orthogonalize(y)
    assert np.abs(B.to_dense(lo) - yd).max() < 1e-12
    _check_left_orth(lo)
    nrm = np.linalg.norm(yd)
    for eps in [0.0, 1e-6 * nrm, 0.05 * nrm, 0.3 * nrm]:
        tr, dtol, dcap = B.truncate(y, eps)
        err = np.linalg.norm(B.to_dense(tr) - yd)
        assert err <= eps + 1e-12 * nrm                  # ||x - trunc_eps(x)|| <= eps
        assert abs(err - dtol) <= 1e-10 * nrm              # equals the discarded Schmidt weight
        assert dcap == 0.0
        _check_right_orth(tr)
    # rank cap: ranks never exceed r_max and the cap's share is reported
    tr, dtol, dcap = B.truncate(y, 0.0, r_max=3)
    assert max(tr.ranks()) <= 3 and dcap > 0
    err = np.linalg.norm(B.to_dense(tr) - yd)
    assert err <= np.sqrt(dtol ** 2 + dcap ** 2) + 1e-12


def test_truncation_exact_low_rank_is_lossless():
    # a sum of two copies of x has the ranks of x: truncation recovers them exactly
    species = F.site_species(4, 1)
    x = rand_mps(species, (2, 2), 6, 7)
    s = B.add(x, x, 1.0, 2.0)
    tr, dtol, _ = B.truncate(s, 1e-10)
    assert tr.ranks() == B.truncate(x, 1e-10)[0].ranks()
    assert np.abs(B.to_dense(tr) - 3 * B.to_dense(x)).max() < 1e-12


def test_e1_state_and_edge_cases():
    species = F.site_species(5, 0)
    e1 = B.e1_mps(species, (2, 0))
    v = B.to_dense(e1)
    assert v[int("11000", 2)] == 1.0 and abs(np.linalg.norm(v) - 1) < 1e-15
    # N = 0 and N = K: single configuration
    for N in (0, 5):
        x = rand_mps(species, (N, 0), 4, 8)
        assert max(x.ranks()) == 1 and np.count_nonzero(B.to_dense(x)) == 1
    # everything truncated away gives the zero vector
    tr, dtol, _ = B.truncate(e1, 2.0)
    assert np.abs(B.to_dense(tr)).max() == 0.0 and abs(dtol - 1.0) < 1e-15


def test_choose_cut_clusters_and_ties():
    sv = [(1.0, 0, 0), (0.5, 1, 0), (0.5 * (1 - 1e-12), 0, 1), (1e-3, 1, 1)]
    kept, dt, dc = B.choose_cut(sv, tol2=0.3, r_max=0)
    # the tolerance would cut inside the 0.5-cluster; the cut moves up to keep it whole
    assert kept == {(0, 0), (1, 0), (0, 1)}
    kept, dt, dc = B.choose_cut(sv, tol2=0.0, r_max=2)
    # a cap inside the cluster moves down to its edge
    assert kept == {(0, 0)}
