"""The library's problem set-up calls (host only, no GPU) against the oracle:
theta of Sec. 7.1.1, the interval [t_min, t_max] of Sec. 4.3, the lower bound
of the ground energy behind the shift gamma (Sec. 3.1), alpha_0 and c of
Cor. lrprecond."""
import numpy as np
import pytest

from oracle import fermion as OF
from oracle import precond as OP
from paper_2604_16118_gb300 import problem
from synth import coulomb_1d, hubbard_chain, molecule_like, spinless_random_chain

WORKLOADS = [
    ("spinless_K12", spinless_random_chain(K=12, N=6, seed=0), True),
    ("hubbard_L8", hubbard_chain(L=8, U=4.0), False),
    ("hubbard_L32", hubbard_chain(L=32, U=4.0), False),
    ("molecule_L6", molecule_like(L=6, n_up=3, n_dn=2, seed=1), True),
    ("coulomb_K14", coulomb_1d(K=14, N=4, n_grid=2048), True),
]


@pytest.mark.parametrize("name,wl,chol", WORKLOADS)
def test_shift_bound_theta_and_interval_match_oracle(name, wl, chol):
    lib_bound = (problem.cholesky_shift(wl.h, wl.eri, wl.n_up, wl.n_dn, wl.spin, margin=0.0) if chol
                 else problem.hubbard_shift(wl.h, wl.n_up, wl.n_dn, margin=0.0))
    e_lb = OP.energy_lower_bound(wl.h, wl.eri, wl.spin, wl.n_up, wl.n_dn, cholesky=chol)
    assert abs(-lib_bound - e_lb) <= 1e-12 * max(1.0, abs(e_lb))
    gamma = 1.0 - e_lb
    th = problem.theta_diagonal(wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    t_so, v_so = OP.spin_orbital_accessors(wl.h, wl.eri, wl.spin)
    ref = OP.theta_diag(t_so, v_so, wl.n_particles, gamma, wl.n_sites)
    assert np.abs(th - ref).max() <= 1e-13 * np.abs(ref).max()
    species = OF.site_species(wl.n_orb, wl.spin)
    for h in (None, wl.h):
        lo, hi = problem.spectrum_bounds(th, wl.spin, wl.n_up, wl.n_dn, h=h)
        t_diag = None if h is None else (np.repeat(np.diag(h), 2) if wl.spin else np.diag(h))
        rlo, rhi = OP.spectrum_bounds(ref, species, (wl.n_up, wl.n_dn), t_diag=t_diag)
        assert abs(lo - rlo) <= 1e-12 * abs(rlo) and abs(hi - rhi) <= 1e-12 * abs(rhi)


@pytest.mark.parametrize("c0,tmin,cl,cu", [(0.1, 1.38, 0.3, 1.5), (0.05, 73.0, 0.23, 1.4), (0.4, 7.35, 1.0, 1.0)])
def test_alpha0_and_c_match_oracle(c0, tmin, cl, cu):
    a, c = problem.alpha0_and_c(c0, tmin, cl, cu)
    ra, rc = OP.alpha0_and_c(c0, tmin, cl, cu)
    assert abs(a - ra) <= 1e-15 * ra and abs(c - rc) <= 1e-15


def test_setup_rejects_invalid_input():
    from paper_2604_16118_gb300.native import BsmpsError
    with pytest.raises(BsmpsError):
        problem.alpha0_and_c(1.5, 1.0, 0.3, 1.5)
    with pytest.raises(BsmpsError):
        problem.spectrum_bounds(np.ones(4), 0, 5, 0)
