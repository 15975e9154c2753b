"""Joint block MPS operations and the subspace iteration (Alg. 4) on the GPU vs
the oracle, through the C ABI.

Block structure is compared bit-exactly; values, Gram matrices and Ritz values
to the tolerances of the Alg. 2 parity tests (1e-12 relative for single
operations, lambda 1e-10 relative along a trajectory, ranks and eta_res tries
exact)."""
import numpy as np
import pytest

from oracle import bsmps as OB
from oracle import joint as OJ
from oracle import pinvit as OPI
from paper_2604_16118_gb300 import problem
from synth import hubbard_chain, random_block_values, spinless_random_chain
from tests._common import oracle_mpo, precond_for, species_of, target_of, to_oracle
from tests.test_gpu_parity import _small_problem

pytestmark = pytest.mark.gpu

CASES = [("spinless K=6 N=3 D=3", spinless_random_chain(K=6, N=3, seed=4), 6, 3),
         ("hubbard L=3 (2,1) D=2", hubbard_chain(L=3, n_up=2, n_dn=1, U=2.0), 6, 2),
         ("spinless K=12 N=6 D=4", spinless_random_chain(K=12, N=6, seed=0), 32, 4)]


@pytest.fixture(scope="module")
def nat():
    from paper_2604_16118_gb300 import build, native
    build.build()
    return native


@pytest.fixture(scope="module")
def ctx(nat):
    return nat.Context(0)


def joint_pair(nat, ctx, wl, r, D, seed):
    n = nat.mps_joint_random_size(wl.n_orb, wl.spin, wl.n_up, wl.n_dn, r, D)
    vals = random_block_values(n, seed)
    x = nat.mps_create_joint(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, D, r_max=r, values=vals)
    dims = OB.default_dims(species_of(wl), target_of(wl), r, D)
    return x, OB.BSMPS.from_flat(species_of(wl), target_of(wl), dims, vals)


def t_diagonal(wl):
    """t_ii of the sites (spin-orbitals inherit the spatial h_pp)."""
    d = np.diag(wl.h)
    return np.repeat(d, 2) if wl.spin else d.copy()


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("name,wl,r,D", CASES)
def test_joint_layout_and_columns(nat, ctx, name, wl, r, D):
    x, ox = joint_pair(nat, ctx, wl, r, D, 1)
    assert x.bonds() == ox.bonds
    assert nat.num_columns(x) == D == OB.columns(ox)


@pytest.mark.parametrize("name,wl,r,D", CASES)
def test_determinant_start_bit_exact(nat, ctx, name, wl, r, D):
    t_diag = t_diagonal(wl)
    occ = problem.lowest_determinants(t_diag, wl.spin, wl.n_up, wl.n_dn, D)
    oocc = OJ.lowest_determinants(species_of(wl), target_of(wl), t_diag, D)
    assert [tuple(int(v) for v in row) for row in occ] == [tuple(o) for o in oocc]
    x = nat.mps_create_joint(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, D, occ=occ)
    ox = OJ.from_determinants(species_of(wl), target_of(wl), oocc)
    assert x.bonds() == ox.bonds
    assert np.array_equal(x.export(), ox.to_flat())


@pytest.mark.parametrize("name,wl,r,D", CASES)
def test_gram_matches_oracle(nat, ctx, name, wl, r, D):
    gamma, _ = _small_problem(wl)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    oW = oracle_mpo(wl, gamma)
    a, oa = joint_pair(nat, ctx, wl, r, D, 2)
    b, ob = joint_pair(nat, ctx, wl, max(r // 2, 2), max(D - 1, 1), 3)
    for mpo, om in ((W, oW), (None, None)):
        G = nat.gram(ctx, a, b, mpo)
        oG = OB.gram(oa, ob, om)
        assert G.shape == oG.shape
        assert rel(G, oG) <= 1e-12
    # with a shift: <a, (H + s) b> = <a, H b> + s <a, b>
    Gs = nat.gram(ctx, a, b, W, 0.75)
    assert rel(Gs, OB.gram(oa, ob, oW, 0.75)) <= 1e-12


@pytest.mark.parametrize("name,wl,r,D", CASES)
def test_column_shifted_apply_matches_oracle(nat, ctx, name, wl, r, D):
    gamma, _ = _small_problem(wl)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    oW = oracle_mpo(wl, gamma)
    x, ox = joint_pair(nat, ctx, wl, r, D, 4)
    cs = np.linspace(-1.3, 0.4, D)
    y = nat.apply_columns(ctx, W, x, cs)
    oy = OB.apply_exact(oW, ox, 0.0, col_shift=cs)
    assert y.bonds() == oy.bonds
    assert rel(y.export(), oy.to_flat()) <= 1e-13


@pytest.mark.parametrize("name,wl,r,D", CASES)
def test_mix_add_truncate_match_oracle(nat, ctx, name, wl, r, D):
    a, oa = joint_pair(nat, ctx, wl, r, D, 5)
    b, ob = joint_pair(nat, ctx, wl, max(r // 2, 2), D, 6)
    rng = np.random.default_rng(8)
    Wa, Wb = rng.standard_normal((D, D)), rng.standard_normal((D, D))
    s = nat.add(ctx, nat.mix_columns(ctx, a, Wa), nat.mix_columns(ctx, b, Wb))
    os_ = OB.add(OB.mix_columns(oa, Wa), OB.mix_columns(ob, Wb))
    assert s.bonds() == os_.bonds
    assert rel(s.export(), os_.to_flat()) <= 1e-13
    fro = np.sqrt(np.trace(OB.gram(os_, os_)))
    for eps_rel in (1e-2, 1e-6):
        y, dt, _ = nat.truncate(ctx, s, eps_rel * fro)
        oy, odt, _ = OB.truncate(os_, eps_rel * fro)
        assert y.bonds() == oy.bonds
        G = OB.gram(to_oracle(wl, y), to_oracle(wl, y))
        oG = OB.gram(oy, oy)
        assert rel(G, oG) <= 1e-12
        assert abs(dt - odt) <= 1e-10 * fro


def _solver_setup(nat, ctx, wl):
    gamma, lam = _small_problem(wl)
    th, tmin, tmax, prec = precond_for(wl, gamma, alpha0=0.6)
    c, delta = 0.6, lam[1] / (lam[1] - lam[0])
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    p = nat.make_precond(th, tmin, tmax, 0.1, 0.6)
    return gamma, th, prec, c, delta, W, p


@pytest.mark.parametrize("name,wl,r,D", CASES[:2])
def test_joint_steps_match_oracle(nat, ctx, name, wl, r, D):
    gamma, th, prec, c, delta, W, p = _solver_setup(nat, ctx, wl)
    oW = oracle_mpo(wl, gamma)
    x, ox = joint_pair(nat, ctx, wl, r, D, 13)
    prm = nat.solver_params(c, delta, tau=1e-9)
    oprm = OPI.SolverParams(c, delta, tau=1e-9)
    st, ost = nat.solver_state(), OPI.SolverState()
    for n in range(6):
        x, info = nat.eigensolve_joint_step(ctx, W, p, prm, st, x)
        ox, oinfo = OJ.step(ox, oW, prec, oprm, ost)
        assert info["D"] == D
        assert rel(info["lambda"], oinfo["lambda"]) <= 1e-10
        assert rel(info["rho"], oinfo["rho"]) <= 1e-7
        assert info["eta_tries"] == oinfo["eta_tries"]
        assert bool(info["converged"]) == oinfo["converged"]
        if oinfo["converged"]:
            break
        assert rel(info["lambda_star"], oinfo["lambda_star"]) <= 1e-10
        assert info["max_rank"] == max(oinfo["ranks"])
        assert x.bonds() == ox.bonds


def test_joint_d1_matches_alg2_on_gpu(nat, ctx):
    wl = spinless_random_chain(K=6, N=3, seed=4)
    gamma, th, prec, c, delta, W, p = _solver_setup(nat, ctx, wl)
    x1, _ = joint_pair(nat, ctx, wl, 6, 1, 21)
    x2, _ = joint_pair(nat, ctx, wl, 6, 1, 21)
    prm = nat.solver_params(c, delta, tau=1e-9)
    s1, s2 = nat.solver_state(), nat.solver_state()
    for _ in range(4):
        x1, i1 = nat.eigensolve_step(ctx, W, p, prm, s1, x1)
        x2, i2 = nat.eigensolve_joint_step(ctx, W, p, prm, s2, x2)
        assert abs(i2["lambda"][0] - i1["lambda"]) <= 1e-12 * i1["lambda"]
        assert i2["eta_tries"] == i1["eta_tries"]
        if i1["converged"]:
            break
        assert i2["max_rank"] == i1["max_rank"]


def test_joint_iteration_reaches_exact_eigenvalues(nat, ctx):
    """From the D lowest determinants to tau: the D Ritz values against exact
    diagonalisation (column 1 certified by Eq. (releigerr))."""
    from oracle import fermion as OF
    wl = spinless_random_chain(K=6, N=3, seed=4)
    gamma, th, prec, c, delta, W, p = _solver_setup(nat, ctx, wl)
    H0, _ = OF.sector_hamiltonian(wl.h, wl.eri, wl.spin, wl.n_up, wl.n_dn)
    lam_all = np.linalg.eigvalsh(H0) + gamma
    D = 3
    occ = problem.lowest_determinants(t_diagonal(wl), wl.spin, wl.n_up, wl.n_dn, D)
    x = nat.mps_create_joint(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, D, occ=occ)
    prm = nat.solver_params(c, delta, tau=1e-8)
    st = nat.solver_state()
    for _ in range(80):
        x, info = nat.eigensolve_joint_step(ctx, W, p, prm, st, x)
        assert np.all(info["lambda"] >= lam_all[:D] * (1 - 1e-12))
        if info["converged"]:
            break
    assert info["converged"]
    assert (info["lambda"][0] - lam_all[0]) / lam_all[0] <= info["releig_bound"] * (1 + 1e-6) + 1e-13
    assert abs(info["lambda"][1] - lam_all[1]) <= 1e-4 * lam_all[1]
    # A-orthonormal columns: sum_{k,k'} (S_k X)^T H (S_k' X) = I
    ox = to_oracle(wl, x)
    GA = OJ.gram_sums(ox, ox, prec, oracle_mpo(wl, gamma))
    assert np.abs(GA - np.eye(D)).max() < 1e-9


def test_joint_error_paths(nat, ctx):
    """Calls that need one column reject joint MPS; the joint step rejects more
    than BSMPS_MAX_COLUMNS columns; occupations outside the sector are rejected."""
    wl = spinless_random_chain(K=6, N=3, seed=4)
    gamma, th, prec, c, delta, W, p = _solver_setup(nat, ctx, wl)
    x, _ = joint_pair(nat, ctx, wl, 6, 3, 31)
    with pytest.raises(nat.BsmpsError) as e:
        nat.dot(ctx, x, x)
    assert "INVALID_ARG" in str(e.value)
    with pytest.raises(nat.BsmpsError):
        nat.eigensolve_step(ctx, W, p, nat.solver_params(c, delta), nat.solver_state(), x)
    # the rejected step left the handle alive
    assert nat.num_columns(x) == 3
    big, _ = joint_pair(nat, ctx, wl, 20, nat.MAX_COLUMNS + 1, 32)
    with pytest.raises(nat.BsmpsError):
        nat.eigensolve_joint_step(ctx, W, p, nat.solver_params(c, delta), nat.solver_state(), big)
    bad = np.zeros((1, 6), dtype=np.uint8)
    bad[0, :2] = 1                     # two particles where three are required
    with pytest.raises(nat.BsmpsError) as e:
        nat.mps_create_joint(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn, 1, occ=bad)
    assert "CHARGE" in str(e.value)
    # a Gram matrix of a joint MPS with itself is symmetric positive definite
    G = nat.gram(ctx, x, x)
    assert np.allclose(G, G.T, rtol=0, atol=1e-12 * np.abs(G).max())
    assert np.linalg.eigvalsh(G).min() > 0
