"""Dense Jordan--Wigner reference for the second-quantized Hamiltonian.

Test infrastructure only (see ``oracle/__init__.py``).

Sites are numbered 0..K-1 (the paper numbers them 1..K).  Occupation
alpha_s = 1 means site s is occupied.  Basis vectors of the Fock space are
ordered lexicographically in (alpha_0, ..., alpha_{K-1}), i.e. the Kronecker
order of (R^2)^{(x)K} with site 0 the slowest index (Sec. 1.1).

Spin: with ``spin=1`` spatial orbital p carries two sites, 2p (species 0,
"up") and 2p+1 (species 1, "down").  The paper treats equal spins only
(Sec. 1.1); the interleaved spin-orbital reading is the one used by the
whole project.
"""

from itertools import combinations

import numpy as np

# Eq. (elementarycomponents)
S_MAT = np.array([[1.0, 0.0], [0.0, -1.0]])
A_MAT = np.array([[0.0, 1.0], [0.0, 0.0]])
I_MAT = np.eye(2)


def site_species(n_orb, spin):
    """Species (0/1) of every site: all 0 when spinless, alternating when spin=1."""
    if spin:
        return tuple(s % 2 for s in range(2 * n_orb))
    return tuple(0 for _ in range(n_orb))


def annihilator_full(K, i):
    """a_i = S^{(x) i} (x) A (x) I^{(x)(K-i-1)} on the full Fock space (Def. anniloperator)."""
    out = np.ones((1, 1))
    for s in range(K):
        f = S_MAT if s < i else (A_MAT if s == i else I_MAT)
        out = np.kron(out, f)
    return out


def spin_orbital_terms(h, eri, spin, n_particles, gamma=0.0):
    """The one- and two-body terms of H_gamma in a fixed enumeration order.

    Returns (one, two): lists of (coef, i, j) for t_ij a_i^* a_j and
    (coef, i, j, k, l) for v_ijkl a_i^* a_j^* a_k a_l, with
    v_ijkl = 1/2 (il|jk) (Eq. (tvdef) in chemist notation) and the shift
    folded into the diagonal as t_ii + gamma/N (Sec. 7.1.1).
    Spatial integrals are expanded to spin-orbitals when spin=1:
    t_{p s, q s} = h_pq, v_{p s, r u, s u, q s} = 1/2 (pq|rs).
    Zero integrals are skipped.  Order: one-body (p, q, spin), two-body
    (p, q, r, s, spin of pq, spin of rs), all ascending.
    """
    n = h.shape[0]
    spins = (0, 1) if spin else (0,)

    def so(p, s):
        return 2 * p + s if spin else p

    shift = gamma / n_particles if n_particles > 0 else 0.0
    one = []
    for p in range(n):
        for q in range(n):
            coef = h[p, q] + (shift if p == q else 0.0)
            if coef != 0.0:
                for s in spins:
                    one.append((coef, so(p, s), so(q, s)))
    two = []
    nz = np.argwhere(eri != 0.0)
    for p, q, r, s_ in nz:
        val = 0.5 * eri[p, q, r, s_]
        for sa in spins:
            for sb in spins:
                two.append((val, so(p, sa), so(r, sb), so(s_, sb), so(q, sa)))
    return one, two


def sector_states(species, n_tuple):
    """All occupation bitmasks (bit s = site s) with the given particle numbers,
    sorted lexicographically in (alpha_0, ..., alpha_{K-1})."""
    K = len(species)
    sites0 = [s for s in range(K) if species[s] == 0]
    sites1 = [s for s in range(K) if species[s] == 1]
    states = []
    for occ0 in combinations(sites0, n_tuple[0]):
        for occ1 in combinations(sites1, n_tuple[1]):
            m = 0
            for s in occ0 + occ1:
                m |= 1 << s
            states.append(m)

    def lexkey(m):
        return tuple((m >> s) & 1 for s in range(K))

    states.sort(key=lexkey)
    return np.array(states, dtype=np.int64)


def _parity_below_table(K):
    """par[m, s] = parity of the number of occupied sites < s in mask m."""
    masks = np.arange(1 << K, dtype=np.int64)
    par = np.zeros((1 << K, K), dtype=np.int8)
    acc = np.zeros(1 << K, dtype=np.int8)
    for s in range(K):
        par[:, s] = acc
        acc ^= ((masks >> s) & 1).astype(np.int8)
    return par


def sector_hamiltonian(h, eri, spin, n_up, n_dn, gamma=0.0):
    """Dense H_gamma on F_N^K by applying every term's Jordan--Wigner action to
    every occupation basis state (Eq. (hamil), Def. (anniloperator)):
    a_s |alpha> = (-1)^{#occupied sites < s} |alpha - e_s> if alpha_s = 1, else 0.
    """
    species = site_species(h.shape[0], spin)
    K = len(species)
    states = sector_states(species, (n_up, n_dn))
    dim = len(states)
    index = -np.ones(1 << K, dtype=np.int64)
    index[states] = np.arange(dim)
    par = _parity_below_table(K)
    H = np.zeros((dim, dim))
    one, two = spin_orbital_terms(h, eri, spin, n_up + n_dn, gamma)

    def apply(ops_right_to_left, coef):
        m = states.copy()
        sign = np.ones(dim)
        ok = np.ones(dim, dtype=bool)
        for site, creation in ops_right_to_left:
            bit = (m >> site) & 1
            ok &= (bit == 0) if creation else (bit == 1)
            sign *= 1.0 - 2.0 * par[m, site]
            m = m ^ (1 << site)
        cols = np.nonzero(ok)[0]
        rows = index[m[cols]]
        good = rows >= 0
        np.add.at(H, (rows[good], cols[good]), coef * sign[cols[good]])

    for coef, i, j in one:
        apply([(j, False), (i, True)], coef)
    for coef, i, j, k, l in two:
        apply([(l, False), (k, False), (j, True), (i, True)], coef)
    return H, states


def full_hamiltonian(h, eri, spin, n_particles, gamma=0.0):
    """H_gamma on the whole Fock space from Kronecker-product annihilators (tiny K)."""
    species = site_species(h.shape[0], spin)
    K = len(species)
    a = [annihilator_full(K, i) for i in range(K)]
    ad = [m.T for m in a]
    H = np.zeros((1 << K, 1 << K))
    one, two = spin_orbital_terms(h, eri, spin, n_particles, gamma)
    for coef, i, j in one:
        H += coef * ad[i] @ a[j]
    for coef, i, j, k, l in two:
        H += coef * ad[i] @ ad[j] @ a[k] @ a[l]
    return H


def number_operator_full(K):
    """P = sum_i a_i^* a_i on the full Fock space (Sec. 1.1)."""
    P = np.zeros((1 << K, 1 << K))
    for i in range(K):
        a = annihilator_full(K, i)
        P += a.T @ a
    return P


def lowest_eigenpairs(H, k=2):
    """Exact diagonalisation of a dense symmetric matrix (library eigh)."""
    w, v = np.linalg.eigh(H)
    return w[:k], v[:, :k]
