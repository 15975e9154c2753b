"""Problem set-up for the solver: the shift gamma, the diagonal D of the
preconditioner, the interval of its spectrum, alpha_0 and the lowest
determinants.  Argument marshalling only: the arithmetic runs in libbsmps.so
(bsmps_energy_lower_bound, bsmps_precond_theta, bsmps_precond_interval,
bsmps_precond_alpha0, bsmps_lowest_determinants in include/bsmps.h).
"""

from . import native as nat


def hubbard_shift(h, n_up, n_dn, margin=1.0):
    """gamma = margin - E_lb for on-site interactions U >= 0 (Sec. 3.1)."""
    return margin - nat.energy_lower_bound(h, None, 1, n_up, n_dn, cholesky=False)


def cholesky_shift(h, eri, n_up, n_dn, spin, margin=1.0):
    """gamma = margin - E_lb for positive semidefinite (pq|rs) (Sec. 3.1)."""
    return margin - nat.energy_lower_bound(h, eri, spin, n_up, n_dn, cholesky=True)


def theta_diagonal(h, eri, spin, n_particles, gamma):
    """theta_i of Sec. 7.1.1."""
    return nat.precond_theta(h, eri, spin, n_particles, gamma)


def spectrum_bounds(theta, spin, n_up, n_dn, h=None):
    """[t_min, t_max] of the exponential-sum interval (Sec. 4.3)."""
    return nat.precond_interval(theta, spin, n_up, n_dn, h=h)


def alpha0_and_c(c0, t_min, c_lower, c_upper):
    """alpha_0 of Eq. (Sdef) and c of Eq. (precondcdef)."""
    return nat.precond_alpha0(c0, t_min, c_lower, c_upper)


def lowest_determinants(t_diag, spin, n_up, n_dn, D, max_configs=2_000_000):
    """Occupation strings (D x K, uint8) of the D lowest determinants (Sec. 7.1.4)."""
    return nat.lowest_determinants(t_diag, spin, n_up, n_dn, D, max_configs)
