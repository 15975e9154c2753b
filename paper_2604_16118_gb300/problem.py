"""Problem set-up for the solver: shift gamma, the diagonal D of the
preconditioner and the bounds of its spectrum (host-side scalars).

* gamma: H_gamma = H + gamma I must be positive definite (Sec. 3.1).  For
  two-electron integrals of the form (pq|rs) = sum_g L^g_pq L^g_rs (positive
  semidefinite) or an on-site U >= 0, H >= the one-body part minus the
  normal-ordering term, so E_0 >= E_lb with E_lb the sum of the lowest
  single-particle levels of h - 1/2 sum_g (L^g)^2 per species.  For the
  Hubbard model (U >= 0) the interaction is nonnegative and E_lb is the
  free-fermion ground energy.  gamma = margin - E_lb makes lambda_1 >= margin.
* d_i = theta_i = gamma/N + t_ii + sum_{j=k_i+1}^{k_i+N} (v_ijji - v_ijij),
  k_i = max(0, i-N) (1-based, Sec. 7.1.1), with v_ijkl = 1/2 (il|jk).
* t_min / t_max: sums of the N_s smallest / largest d_i of each species
  (the spectrum of D on the N-particle space).
"""

import numpy as np


def spin_orbital_pairs(n_orb, spin):
    if spin:
        return [(i // 2, i % 2) for i in range(2 * n_orb)]
    return [(i, 0) for i in range(n_orb)]


def free_fermion_bound(h, n_up, n_dn, spin):
    ev = np.sort(np.linalg.eigvalsh(h))
    if spin:
        return float(ev[:n_up].sum() + ev[:n_dn].sum())
    return float(ev[:n_up].sum())


def hubbard_shift(h, n_up, n_dn, margin=1.0):
    """gamma for U >= 0 on-site interactions."""
    return margin - free_fermion_bound(h, n_up, n_dn, 1)


def cholesky_shift(h, eri, n_up, n_dn, spin, margin=1.0):
    """gamma for PSD (pq|rs): H >= sum_pq (h_pq - 1/2 sum_r (pr|rq)) a_p^* a_q."""
    hk = h - 0.5 * np.einsum("prrq->pq", eri)
    return margin - free_fermion_bound(hk, n_up, n_dn, spin)


def theta_diagonal(h, eri, spin, n_particles, gamma):
    so = spin_orbital_pairs(h.shape[0], spin)
    K = len(so)
    N = n_particles

    def v(i, j, k, l):
        (pi, si), (pj, sj), (pk, sk), (pl, sl) = so[i], so[j], so[k], so[l]
        if si != sl or sj != sk:
            return 0.0
        return 0.5 * eri[pi, pl, pj, pk]

    th = np.zeros(K)
    for i1 in range(1, K + 1):
        i = i1 - 1
        pi, si = so[i]
        acc = gamma / N + h[pi, pi]
        ki = max(0, i1 - N)
        for j1 in range(ki + 1, ki + N + 1):
            j = j1 - 1
            acc += v(i, j, j, i) - v(i, j, i, j)
        th[i] = acc
    return th


def spectrum_bounds(theta, spin, n_up, n_dn, h=None):
    """t_min / t_max of the exponential-sum interval.  With the one-body matrix
    h given and its diagonal strictly increasing along a species' sites (the
    paper's orbital basis), the sums of theta over that species' first / last
    n sites (t_min = D at e_1, as the printed t_min, t_max and T of Sec. 7.2
    require); otherwise the sums of the n smallest / largest theta (the range
    of the spectrum of D)."""
    lo = hi = 0.0
    K = len(theta)
    diag = None
    if h is not None:
        d = np.diag(np.asarray(h, dtype=np.float64))
        diag = np.repeat(d, 2) if spin else d
    groups = [(np.arange(0, K, 2), n_up), (np.arange(1, K, 2), n_dn)] if spin else [(np.arange(K), n_up)]
    for idx, n in groups:
        if not n:
            continue
        vals = np.asarray(theta)[idx]
        if diag is None or not np.all(np.diff(diag[idx]) > 0):
            vals = np.sort(vals)
        lo += float(np.sum(vals[:n]))
        hi += float(np.sum(vals[-n:]))
    return lo, hi
