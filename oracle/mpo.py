"""Exact MPO for the second-quantized Hamiltonian (Sec. 2.4, Thm. opranks).

Test infrastructure only (see ``oracle/__init__.py``).

Construction (a finite-state reading of the operator sum, written for this
project; the paper relies on cited constructions it does not print):

1. Every term (Eq. (hamil)) is a product of Jordan--Wigner operators
   a_s = Z^{(x)s} (x) A (x) I...  The product of tensor products is taken site
   by site, so a term equals coef * (x)_t L_t with 2x2 local factors L_t.
   At a site t touched by the term, L_t is the ordered product of the factors
   the term's operators put on t (A or A^T at their own site, Z at sites left
   of it, I right of it).  Untouched sites carry Z^{q}, q = number of the
   term's operators to their right.
2. The touched ("active") sites s_1 < ... < s_m and their factors, each
   normalised so its first nonzero entry is +1 (sign moved into coef), form
   the term's canonical key.  Terms with equal keys are merged by adding
   coefficients (enumeration order of ``fermion.spin_orbital_terms``); terms
   whose merged coefficient is exactly 0 are dropped.
3. The MPO channel of a term at bond b (separating sites < b from sites >= b)
   with p of its m active sites left of b is: I (p = 0), F (p = m), the placed
   prefix ("L", key[:p]) if p < m - p, the remaining suffix ("R", key[p:]) if
   p > m - p, and for p = m - p the prefix when b < K//2 else the suffix.
   The coefficient rides on the single transition from {I, L} to {R, F};
   every other transition has weight 1 and is shared by all terms through it.
4. Channels at a bond are ordered I, L-keys (by length, then key), R-keys
   (by length, then key), F.  I exists on bonds 0..K-1, F on bonds 1..K;
   I->I and F->F carry the identity.  Idle sites carry Z^{parity} with the
   parity of the channel's odd (off-diagonal) factors.
5. W_t[a, b] is a 2x2 operator; its structural support is the union of the
   supports of the factors written into it.  Site 0 always has the entry
   (I -> F) with full diagonal support so that a scalar shift s*Id can be
   added to it (used for H_gamma - lambda I).
"""

import numpy as np

from .fermion import site_species, spin_orbital_terms

_A = np.array([[0, 1], [0, 0]], dtype=np.int64)
_AT = _A.T.copy()
_Z = np.array([[1, 0], [0, -1]], dtype=np.int64)
_I = np.eye(2, dtype=np.int64)


def op_code(M):
    """Integer code of a 2x2 matrix with entries in {-1, 0, 1}."""
    return int(sum((int(M[i, j]) + 1) * 3 ** (2 * i + j) for i in range(2) for j in range(2)))


def op_from_code(code):
    M = np.zeros((2, 2), dtype=np.int64)
    for i in range(2):
        for j in range(2):
            M[i, j] = (code // 3 ** (2 * i + j)) % 3 - 1
    return M


def op_is_odd(code):
    """Off-diagonal factor: changes the occupation of its site."""
    M = op_from_code(code)
    return M[0, 1] != 0 or M[1, 0] != 0


def op_charge(code):
    """Occupation change of the factor: +1 for a creation pattern, -1 annihilation."""
    M = op_from_code(code)
    if M[1, 0] != 0:
        return 1
    if M[0, 1] != 0:
        return -1
    return 0


def canonical_term(coef, ops):
    """Canonical key and coefficient of coef * prod(ops) (ops: (site, creation) in
    operator order).  Returns None when the product vanishes."""
    sites = sorted(set(s for s, _ in ops))
    key = []
    sign = 1
    for t in sites:
        M = _I.copy()
        for s, cr in ops:
            if s == t:
                f = _AT if cr else _A
            elif s > t:
                f = _Z
            else:
                f = _I
            M = M @ f
        flat = M.reshape(-1)
        nzi = np.nonzero(flat)[0]
        if len(nzi) == 0:
            return None
        if flat[nzi[0]] < 0:
            M = -M
            sign = -sign
        key.append((t, op_code(M)))
    return tuple(key), sign * coef


def canonical_terms(h, eri, spin, n_particles, gamma=0.0):
    """Merged canonical terms {key: coef} of H_gamma in enumeration order."""
    one, two = spin_orbital_terms(h, eri, spin, n_particles, gamma)
    acc = {}
    for coef, i, j in one:
        ct = canonical_term(coef, [(i, True), (j, False)])
        if ct is not None:
            acc[ct[0]] = acc.get(ct[0], 0.0) + ct[1]
    for coef, i, j, k, l in two:
        ct = canonical_term(coef, [(i, True), (j, True), (k, False), (l, False)])
        if ct is not None:
            acc[ct[0]] = acc.get(ct[0], 0.0) + ct[1]
    return {k: v for k, v in acc.items() if v != 0.0}


def _state(key, b, bmid):
    m = len(key)
    p = sum(1 for s, _ in key if s < b)
    if p == 0:
        return ("I",)
    if p == m:
        return ("F",)
    if p < m - p or (p == m - p and b < bmid):
        return ("L", key[:p])
    return ("R", key[p:])


def _state_sort_key(st):
    kind = st[0]
    if kind == "I":
        return (0, 0, ())
    if kind == "L":
        return (1, len(st[1]), st[1])
    if kind == "R":
        return (2, len(st[1]), st[1])
    return (3, 0, ())


def _parity(st):
    if st[0] in ("I", "F"):
        return 0
    return sum(1 for _, c in st[1] if op_is_odd(c)) % 2


class MPO:
    """Operator-valued cores: per site t a dict (a, b) -> (2x2 float values, 2x2 bool support);
    per bond b the ordered channel keys and their charge shifts (2 species)."""

    def __init__(self, K, species, channels, charges, W):
        self.K = K
        self.species = species
        self.channels = channels      # list over bonds of list of state keys
        self.charges = charges        # list over bonds of list of (d0, d1)
        self.W = W                    # list over sites of dict (a, b) -> (vals, mask)

    @property
    def bond_dims(self):
        return [len(c) for c in self.channels]

    def entries(self, t, shift=0.0):
        """Sparse entries (a, b, s_out, s_in, w) of site t sorted by (a, b, s_out, s_in)."""
        out = []
        F = len(self.channels[t + 1]) - 1
        for (a, b) in sorted(self.W[t].keys()):
            vals, mask = self.W[t][(a, b)]
            for so in range(2):
                for si in range(2):
                    if mask[so, si]:
                        w = vals[so, si]
                        if t == 0 and a == 0 and b == F and so == si:
                            w = w + shift
                        out.append((a, b, so, si, w))
        return out


def build_mpo(h, eri, spin, n_particles, gamma=0.0):
    """MPO of H_gamma = H + gamma I (shift folded in as t_ii + gamma/N)."""
    species = site_species(h.shape[0], spin)
    K = len(species)
    bmid = K // 2
    terms = canonical_terms(h, eri, spin, n_particles, gamma)
    keys = sorted(terms.keys())

    states = [set() for _ in range(K + 1)]
    for b in range(K):
        states[b].add(("I",))
    for b in range(1, K + 1):
        states[b].add(("F",))
    for key in keys:
        s1, sm = key[0][0], key[-1][0]
        for b in range(s1 + 1, sm + 1):
            states[b].add(_state(key, b, bmid))
    channels = [sorted(st, key=_state_sort_key) for st in states]
    index = [{st: i for i, st in enumerate(ch)} for ch in channels]

    def charge(st):
        d = [0, 0]
        if st[0] == "L":
            for s, c in st[1]:
                d[species[s]] += op_charge(c)
        elif st[0] == "R":
            for s, c in st[1]:
                d[species[s]] -= op_charge(c)
        return tuple(d)

    charges = [[charge(st) for st in ch] for ch in channels]
    W = [dict() for _ in range(K)]

    def put(t, a, b, M, weight, accumulate):
        Mf = M.astype(np.float64)
        if (a, b) in W[t]:
            vals, mask = W[t][(a, b)]
            if accumulate:
                vals = vals + weight * Mf
            mask = mask | (M != 0)
            W[t][(a, b)] = (vals, mask)
        else:
            W[t][(a, b)] = (weight * Mf, M != 0)

    # identity rails
    for t in range(K - 1):
        put(t, index[t][("I",)], index[t + 1][("I",)], _I, 1.0, False)
    for t in range(1, K):
        put(t, index[t][("F",)], index[t + 1][("F",)], _I, 1.0, False)
    # shift slot: (I -> F) at site 0 with diagonal support
    W[0][(0, index[1][("F",)])] = (np.zeros((2, 2)), np.eye(2, dtype=bool))

    for key in keys:
        coef = terms[key]
        active = dict(key)
        s1, sm = key[0][0], key[-1][0]
        for t in range(s1, sm + 1):
            prev = _state(key, t, bmid)
            nxt = _state(key, t + 1, bmid)
            a = index[t][prev]
            b = index[t + 1][nxt]
            if t in active:
                M = op_from_code(active[t])
            else:
                M = _Z if _parity(prev) else _I
            is_coef = prev[0] in ("I", "L") and nxt[0] in ("R", "F")
            if is_coef:
                put(t, a, b, M, coef, True)
            else:
                put(t, a, b, M, 1.0, False)
    return MPO(K, species, channels, charges, W)


def mpo_to_dense(mpo, shift=0.0):
    """Contract the MPO to a dense 2^K x 2^K matrix (site 0 slowest), tiny K only."""
    K = mpo.K
    cur = {0: np.ones((1, 1))}
    for t in range(K):
        nxt = {}
        for (a, b, so, si, w) in mpo.entries(t, shift):
            if a not in cur:
                continue
            E = np.zeros((2, 2))
            E[so, si] = w
            term = np.kron(cur[a], E)
            nxt[b] = nxt[b] + term if b in nxt else term
        cur = nxt
    return cur[0]
