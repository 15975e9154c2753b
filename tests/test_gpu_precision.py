"""Split-precision (3xTF32, tcgen05) contractions in the zip-up MPO application
and in the Alg. 2 step, against the FP64 oracle.

* bsmps_apply_zipup with BSMPS_PREC_TF32X3: identical bond dims, left-orthonormal
  cores (the QR stays FP64), and a distance to the oracle's FP64 result below
  1e-5 of the norm (the split products' relative error is a few 2^-21 of the
  summed magnitudes; the measured distance is printed);
* Alg. 2 on a small problem with exact diagonalisation: the early steps use
  the split precision, the policy switches to FP64 once the split error
  estimate reaches a tenth of eta_res and stays there, every Rayleigh quotient
  stays above lambda_1, and the run converges to the FP64 run's eigenvalue to
  1e-10 relative.
"""
import math

import numpy as np
import pytest

from oracle import bsmps as OB
from oracle import fermion as OF
from oracle import precond as OP
from synth import hubbard_chain, random_block_values, spinless_random_chain
from tests._common import n_random, oracle_mpo, oracle_random, rel_distance, to_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2604_16118_gb300 import build, native
    build.build()
    return native


@pytest.fixture(scope="module")
def ctx(nat):
    c = nat.Context(0)
    yield c
    c.set_precision(nat.PREC_FP64)


@pytest.mark.parametrize("wl,r,gamma", [(spinless_random_chain(K=12, N=6, seed=0), 32, 3.0),
                                        (hubbard_chain(L=8, U=4.0), 40, 1.0)])
def test_split_precision_zipup_against_fp64_oracle(nat, ctx, wl, r, gamma):
    vals = random_block_values(n_random(wl, r), 31)
    x = nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r, vals)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    oy = OB.apply_zipup(oracle_mpo(wl, gamma), oracle_random(wl, r, vals), shift=-0.6)
    ctx.set_precision(nat.PREC_TF32X3)
    ctx.profile(True)
    try:
        y, _ = nat.apply_zipup(ctx, W, x, shift=-0.6)
        stats = ctx.kernel_stats(reset=True)
    finally:
        ctx.profile(False)
        ctx.set_precision(nat.PREC_FP64)
    assert stats["apply"][0] > 0 and stats["apply"][2] > 0      # the contraction ran as its own kind
    assert y.bonds() == oy.bonds
    got = to_oracle(wl, y)
    d = rel_distance(got, oy)
    print(f"{wl.name}: TF32x3 zip-up vs FP64 oracle, relative distance {d:.2e}")
    assert d <= 1e-5
    for t in range(got.K - 1):
        sp = got.species[t]
        for m2, k in got.bonds[t + 1].items():
            S = np.vstack([got.cores[t][(m, s)] for (m, s) in got.block_keys(t)
                           if OB.add_charge(m, OB.delta(sp, s)) == m2])
            assert np.abs(S.T @ S - np.eye(k)).max() <= 1e-12


def _ed_problem():
    K, N = 8, 4
    wl = spinless_random_chain(K=K, N=N, seed=3)
    rng = np.random.default_rng(3)
    g = 0.05 * rng.standard_normal((K, K))
    wl.h = np.diag(0.8 * np.arange(K)) + g + g.T
    wl.eri = 0.3 * wl.eri
    H0, states = OF.sector_hamiltonian(wl.h, wl.eri, 0, N, 0)
    ev = np.linalg.eigvalsh(H0)
    gamma = 0.5 - ev[0]
    t_so, v_so = OP.spin_orbital_accessors(wl.h, wl.eri, 0)
    th = OP.theta_diag(t_so, v_so, N, gamma, K)
    tmin, tmax = OP.spectrum_bounds(th, OF.site_species(K, 0), (N, 0))
    occ = np.array([[(int(m) >> s) & 1 for s in range(K)] for m in states])
    Dv = occ @ th
    Hg = H0 + gamma * np.eye(len(H0))
    mu = np.linalg.eigvalsh(Hg / np.sqrt(np.outer(Dv, Dv)))
    alpha0, c = OP.alpha0_and_c(0.1, tmin, mu[0], mu[-1])
    lam = ev[:2] + gamma
    return wl, gamma, th, tmin, tmax, alpha0, c, lam[1] / (lam[1] - lam[0]), lam[0]


def _run(nat, ctx, prec, wl, gamma, th, tmin, tmax, alpha0, c, delta, vals, r, steps=60):
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, 0, wl.n_up, gamma)
    p = nat.make_precond(th, tmin, tmax, 0.1, alpha0)
    prm = nat.solver_params(c, delta, tau=1e-9, r_max=0)      # no cap: converges in about 30 steps
    st = nat.solver_state()
    x = nat.mps_create(ctx, wl.n_orb, 0, wl.n_up, 0, r, vals)
    ctx.set_precision(prec)
    infos = []
    try:
        for _ in range(steps):
            x, info = nat.eigensolve_step(ctx, W, p, prm, st, x)
            infos.append(info)
            if info["converged"]:
                break
    finally:
        ctx.set_precision(nat.PREC_FP64)
    return infos


def test_mixed_precision_iteration_switches_to_fp64_and_converges(nat, ctx):
    wl, gamma, th, tmin, tmax, alpha0, c, delta, lam1 = _ed_problem()
    r = 8
    vals = random_block_values(n_random(wl, r), 5)
    ref = _run(nat, ctx, nat.PREC_FP64, wl, gamma, th, tmin, tmax, alpha0, c, delta, vals, r)
    mix = _run(nat, ctx, nat.PREC_TF32X3, wl, gamma, th, tmin, tmax, alpha0, c, delta, vals, r)
    assert ref[-1]["converged"] and mix[-1]["converged"]
    precs = [i["precision"] for i in mix]
    assert precs[0] == nat.PREC_TF32X3 and precs[-1] == nat.PREC_FP64
    first64 = precs.index(nat.PREC_FP64)
    assert all(p == nat.PREC_FP64 for p in precs[first64:])        # the switch is final
    assert all(p == nat.PREC_FP64 for p in (i["precision"] for i in ref))
    for i in mix:
        assert i["lambda"] >= lam1 - 1e-10
    assert abs(mix[-1]["lambda"] - ref[-1]["lambda"]) <= 1e-10 * ref[-1]["lambda"]
    assert abs(mix[-1]["lambda"] - lam1) <= 1e-10 * lam1
    print(f"mixed: {len(mix)} steps ({first64} split-precision), FP64: {len(ref)} steps; "
          f"lambda {mix[-1]['lambda']:.14f} vs {ref[-1]['lambda']:.14f}, exact {lam1:.14f}")
