"""CUDA path vs the FP64 oracle, through the C ABI.

Tolerances (required: energies 1e-10 relative, block Frobenius norms 1e-12
relative, block structure bit-exact):
* index / structure: bit-exact;
* exact application and block copies: 1e-14 relative per element (a single
  multiply per element on both sides);
* inner products: 1e-12 relative to ||a|| ||O b||;
* truncation: identical kept dims, block norms 1e-12 relative to each block
  (floor: 1e-3 of the largest block of its core, where rounding at the core's
  scale takes over), represented tensors within 1e-12 ||x||;
* eigensolver steps: lambda 1e-10 relative.
"""
import math

import numpy as np
import pytest

from oracle import bsmps as OB
from oracle import mpo as OM
from oracle import pinvit as OPI
from synth import hubbard_chain, molecule_like, random_block_values, spinless_random_chain
from tests._common import (block_norms, n_random, oracle_mpo, oracle_random, precond_for, rel_distance,
                           species_of, target_of, to_oracle)

pytestmark = pytest.mark.gpu

CASES = [
    ("spinless_K7", spinless_random_chain(K=7, N=3, seed=1), 6, 0.4),
    ("hubbard_L4", hubbard_chain(L=4, n_up=2, n_dn=2, U=4.0), 8, 1.0),
    ("molecule_L4", molecule_like(L=4, n_up=2, n_dn=1, seed=2), 10, 2.0),
    ("spinless_K12", spinless_random_chain(K=12, N=6, seed=0), 32, 3.0),
]


@pytest.fixture(scope="module")
def nat():
    from paper_2604_16118_gb300 import build, native
    build.build()
    return native


@pytest.fixture(scope="module")
def ctx(nat):
    return nat.Context(0)


def gpu_random(nat, ctx, wl, r, seed):
    vals = random_block_values(n_random(wl, r), seed)
    return nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r, vals), vals


@pytest.mark.parametrize("name,wl,r,gamma", CASES)
def test_block_index_and_values_roundtrip(nat, ctx, name, wl, r, gamma):
    x, vals = gpu_random(nat, ctx, wl, r, 5)
    ox = oracle_random(wl, r, vals)
    assert x.bonds() == ox.bonds
    assert np.array_equal(x.export(), vals)


@pytest.mark.parametrize("name,wl,r,gamma", CASES)
def test_mpo_bit_exact(nat, ctx, name, wl, r, gamma):
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    oW = oracle_mpo(wl, gamma)
    K = wl.n_sites
    assert W.bond_dims(K) == oW.bond_dims
    for b in range(K + 1):
        assert W.channel_charges(b, oW.bond_dims[b]) == [tuple(c) for c in oW.charges[b]]
    for t in range(K):
        ge = W.entries(t)
        oe = oW.entries(t)
        assert [e[:4] for e in ge] == [e[:4] for e in oe]
        assert np.array_equal(np.array([e[4] for e in ge]), np.array([e[4] for e in oe]))


@pytest.mark.parametrize("name,wl,r,gamma", CASES)
def test_apply_exact_elementwise(nat, ctx, name, wl, r, gamma):
    x, vals = gpu_random(nat, ctx, wl, r, 6)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    y, fl = nat.apply_H(ctx, W, x, shift=-0.37)
    oy = OB.apply_exact(oracle_mpo(wl, gamma), oracle_random(wl, r, vals), shift=-0.37)
    assert y.bonds() == oy.bonds
    gv, ov = y.export(), oy.to_flat()
    assert np.abs(gv - ov).max() <= 1e-14 * np.abs(ov).max()
    assert fl > 0


@pytest.mark.parametrize("name,wl,r,gamma", CASES)
def test_dot_with_and_without_operator(nat, ctx, name, wl, r, gamma):
    a, va = gpu_random(nat, ctx, wl, r, 7)
    b, vb = gpu_random(nat, ctx, wl, max(2, r // 2), 8)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    oa, ob = oracle_random(wl, r, va), oracle_random(wl, max(2, r // 2), vb)
    oW = oracle_mpo(wl, gamma)
    na, nb = math.sqrt(OB.dot(oa, oa)), math.sqrt(OB.dot(ob, ob))
    g = nat.dot(ctx, a, b)
    assert abs(g - OB.dot(oa, ob)) <= 1e-12 * na * nb
    nHb = math.sqrt(OB.dot(OB.apply_exact(oW, ob), OB.apply_exact(oW, ob)))
    g = nat.dot(ctx, a, b, W, shift=0.25)
    assert abs(g - OB.dot(oa, ob, oW, shift=0.25)) <= 1e-12 * na * (nHb + 0.25 * nb)


@pytest.mark.parametrize("name,wl,r,gamma", CASES)
def test_add_and_scale(nat, ctx, name, wl, r, gamma):
    a, va = gpu_random(nat, ctx, wl, r, 9)
    b, vb = gpu_random(nat, ctx, wl, max(2, r - 3), 10)
    s = nat.add(ctx, a, b, 0.5, -1.25)
    os_ = OB.add(oracle_random(wl, r, va), oracle_random(wl, max(2, r - 3), vb), 0.5, -1.25)
    assert s.bonds() == os_.bonds
    assert np.abs(s.export() - os_.to_flat()).max() <= 1e-15 * np.abs(os_.to_flat()).max()
    K = wl.n_sites
    f0, f1 = np.linspace(0.5, 1.5, K), np.linspace(2.0, 0.1, K)
    g = nat.scale_sites(ctx, a, f0, f1)
    o = OB.scale_sites(oracle_random(wl, r, va), f0, f1)
    assert np.array_equal(g.export(), o.to_flat())


@pytest.mark.parametrize("name,wl,r,gamma", CASES)
@pytest.mark.parametrize("eps_rel,cap", [(0.0, 0), (1e-8, 0), (0.05, 0), (0.3, 0), (0.0, 3)])
def test_truncate(nat, ctx, name, wl, r, gamma, eps_rel, cap):
    x, vals = gpu_random(nat, ctx, wl, r, 11)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    y, _ = nat.apply_H(ctx, W, x)                      # rank-deficient input (exact apply)
    oy = OB.apply_exact(oracle_mpo(wl, gamma), oracle_random(wl, r, vals))
    nrm = math.sqrt(OB.dot(oy, oy))
    eps = eps_rel * nrm
    t, dt, dc = nat.truncate(ctx, y, eps, cap)
    ot, odt, odc = OB.truncate(oy, eps, cap)
    assert t.bonds() == ot.bonds                       # kept dims per sector, bit-exact
    got = to_oracle(wl, t)
    assert rel_distance(got, ot) <= 1e-12 * max(1.0, nrm / max(math.sqrt(OB.dot(ot, ot)), 1e-300))
    gn, on = block_norms(got), block_norms(ot)
    assert gn.keys() == on.keys()
    # each block's Frobenius norm to 1e-12 relative to itself; blocks below 1e-3 of
    # the largest block of their core to 1e-15 of that block (their rounding error
    # is set by the core's scale, a few units of 1e-16 of it)
    core_max = {}
    for (t, _), v in on.items():
        core_max[t] = max(core_max.get(t, 0.0), v)
    for k in on:
        assert abs(gn[k] - on[k]) <= 1e-12 * max(on[k], 1e-3 * core_max[k[0]]), (k, gn[k], on[k])
    assert abs(dt - odt) <= 1e-12 * nrm and abs(dc - odc) <= 1e-12 * nrm
    err = rel_distance(got, oy) * nrm
    assert err <= eps + math.sqrt(dc ** 2) + 1e-11 * nrm


@pytest.mark.parametrize("name,wl,r,gamma", CASES[:3])
def test_precondition(nat, ctx, name, wl, r, gamma):
    x, vals = gpu_random(nat, ctx, wl, r, 12)
    th, tmin, tmax, prec = precond_for(wl, gamma + 20.0)
    p = nat.make_precond(th, tmin, tmax, 0.1, 0.7)
    ox = oracle_random(wl, r, vals)
    for term in range(prec.n_terms):
        y, nt = nat.precondition(ctx, p, x, term)
        assert nt == prec.n_terms
        f0, f1 = prec.factors(term)
        o = OB.scale_sites(ox, f0, f1)
        assert np.abs(y.export() - o.to_flat()).max() <= 1e-14 * np.abs(o.to_flat()).max()
    y, _ = nat.precondition(ctx, p, x, -1)
    acc = None
    for term in range(prec.n_terms):
        f0, f1 = prec.factors(term)
        acc = OB.scale_sites(ox, f0, f1) if acc is None else OB.add(acc, OB.scale_sites(ox, f0, f1))
    assert y.bonds() == acc.bonds
    assert np.abs(y.export() - acc.to_flat()).max() <= 1e-14 * np.abs(acc.to_flat()).max()


def _small_problem(wl, gamma_lam1=0.5):
    from oracle import fermion as OF
    H0, _ = OF.sector_hamiltonian(wl.h, wl.eri, wl.spin, wl.n_up, wl.n_dn)
    ev = np.linalg.eigvalsh(H0)
    gamma = gamma_lam1 - ev[0]
    lam = ev[:2] + gamma
    return gamma, lam


@pytest.mark.parametrize("wl,r", [(spinless_random_chain(K=6, N=3, seed=4), 6),
                                  (hubbard_chain(L=3, n_up=2, n_dn=1, U=2.0), 6)])
def test_eigensolve_steps_match_oracle(nat, ctx, wl, r):
    gamma, lam = _small_problem(wl)
    th, tmin, tmax, prec = precond_for(wl, gamma, alpha0=0.6)
    c, delta = 0.6, lam[1] / (lam[1] - lam[0])
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    oW = oracle_mpo(wl, gamma)
    p = nat.make_precond(th, tmin, tmax, 0.1, 0.6)
    prm = nat.solver_params(c, delta, tau=1e-9)
    st = nat.solver_state()
    ost = OPI.SolverState()
    oprm = OPI.SolverParams(c, delta, tau=1e-9)
    x, vals = gpu_random(nat, ctx, wl, r, 13)
    ox = oracle_random(wl, r, vals)
    for it in range(4):
        x, info = nat.eigensolve_step(ctx, W, p, prm, st, x)
        ox, oinfo = OPI.step(ox, oW, prec, oprm, ost)
        assert abs(info["lambda"] - oinfo["lambda"]) <= 1e-10 * abs(oinfo["lambda"])
        assert info["eta_tries"] == oinfo["eta_tries"]
        assert abs(info["rho"] - oinfo["rho"]) <= 1e-8 * oinfo["rho"]
        assert info["converged"] == int(oinfo["converged"])
        assert x.bonds() == ox.bonds
        assert info["lambda"] >= lam[0] - 1e-10
        if info["converged"]:
            break


def test_edge_cases(nat, ctx):
    # e_1, N = 0 and N = K, single site; zero after truncation
    wl = spinless_random_chain(K=5, N=2, seed=3)
    e1 = nat.mps_create(ctx, 5, 0, 2, 0)
    assert e1.ranks() == [1] * 6
    oe1 = OB.e1_mps(species_of(wl), target_of(wl))
    assert e1.bonds() == oe1.bonds and np.array_equal(e1.export(), oe1.to_flat())
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, 0, 2, 0.0)
    y, _ = nat.apply_H(ctx, W, e1)
    oy = OB.apply_exact(oracle_mpo(wl, 0.0), oe1)
    assert y.bonds() == oy.bonds and np.abs(y.export() - oy.to_flat()).max() < 1e-14
    z, dt, _ = nat.truncate(ctx, e1, 2.0)
    assert abs(dt - 1.0) < 1e-15 and abs(nat.dot(ctx, z, z)) == 0.0
    for N in (0, 5):
        x, vals = gpu_random(nat, ctx, spinless_random_chain(K=5, N=N, seed=1), 4, 2)
        ox = oracle_random(spinless_random_chain(K=5, N=N, seed=1), 4, vals)
        assert x.bonds() == ox.bonds
        assert abs(nat.dot(ctx, x, x) - OB.dot(ox, ox)) < 1e-12 * OB.dot(ox, ox)
        t, _, _ = nat.truncate(ctx, x, 0.0)
        assert t.bonds() == OB.truncate(ox, 0.0)[0].bonds
    one = spinless_random_chain(K=1, N=1, seed=0)
    x = nat.mps_create(ctx, 1, 0, 1, 0)
    W1 = nat.mpo_from_integrals(ctx, one.h, one.eri, 0, 1, 0.5)
    y, _ = nat.apply_H(ctx, W1, x)
    assert abs(y.export()[0] - (one.h[0, 0] + 0.5)) < 1e-15
    s = nat.add(ctx, x, x, 2.0, 3.0)
    assert abs(s.export()[0] - 5.0) < 1e-15
    with pytest.raises(nat.BsmpsError):
        nat.add(ctx, x, e1)


@pytest.mark.parametrize("seed", [0])
def test_full_size_hubbard_sampled(nat, ctx, seed):
    """Hubbard L=32 (K=64 spin-orbitals), r=256 -- the size the bench times."""
    wl = hubbard_chain(L=32, r_max=256)
    x, vals = gpu_random(nat, ctx, wl, 256, seed)
    ox = oracle_random(wl, 256, vals)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, 1, 32, 4.0)
    oW = OM.build_mpo(wl.h, wl.eri, 1, 32, 4.0)
    assert W.bond_dims(64) == oW.bond_dims
    y, _ = nat.apply_H(ctx, W, x, shift=-1.0)
    oy = OB.apply_exact(oW, ox, shift=-1.0)
    assert y.bonds() == oy.bonds
    gv, ov = y.export(), oy.to_flat()
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, len(ov), 20000)
    assert np.abs(gv[idx] - ov[idx]).max() <= 1e-14 * np.abs(ov).max()
    nx = OB.dot(ox, ox)
    assert abs(nat.dot(ctx, x, x) - nx) <= 1e-12 * nx
    e = OB.dot(ox, ox, oW)
    assert abs(nat.dot(ctx, x, x, W) - e) <= 1e-12 * nx * (abs(e) / nx + 40.0)
