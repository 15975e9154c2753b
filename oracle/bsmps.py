"""Block-sparse U(1) x U(1) matrix product states (Sec. 2.1-2.3).

Test infrastructure only (see ``oracle/__init__.py``).

Conventions shared with the product's documentation (the code is not shared):

* Sites t = 0..K-1, bonds b = 0..K; bond b separates sites < b from >= b.
  Site t lies between bond t and bond t+1.
* Every site has a species (0 or 1); occupying it adds 1 to that species'
  particle count.  A sector (charge) at bond b is the pair (n0, n1) of
  particles left of b.  Valid sectors at bond b (Sec. 2.3, the sets K_k):
  n_s in [max(0, N_s - R_s(b)), min(N_s, L_s(b))], with L_s(b)/R_s(b) the number
  of species-s sites left/right of b.  Sectors at a bond are sorted ascending.
* Core t holds one dense block per (left sector n, sigma) whose right sector
  n + delta_t(sigma) exists: sigma=0 is the unoccupied block, sigma=1 the
  occupied one (Eq. (blockstructure)).  A block is rho_{t,n} x rho_{t+1,n'}.
* Flat layout: sites ascending; within a site left sectors ascending, then
  sigma = 0, 1; each block row-major.
"""

import numpy as np


def delta(species_t, sigma):
    d = [0, 0]
    d[species_t] += sigma
    return tuple(d)


def add_charge(a, b):
    return (a[0] + b[0], a[1] + b[1])


def sub_charge(a, b):
    return (a[0] - b[0], a[1] - b[1])


def valid_ranges(species, target):
    """Per bond: list of valid (n0, n1) sectors, ascending (Sec. 2.3, K_k)."""
    K = len(species)
    out = []
    for b in range(K + 1):
        L = [0, 0]
        R = [0, 0]
        for t in range(K):
            (L if t < b else R)[species[t]] += 1
        rng = []
        for s in range(2):
            lo = max(0, target[s] - R[s])
            hi = min(target[s], L[s])
            rng.append(range(lo, hi + 1))
        out.append([(a, c) for a in rng[0] for c in rng[1]])
    return out


def _binom(n, k):
    if k < 0 or k > n:
        return 0
    r = 1
    for i in range(k):
        r = r * (n - i) // (i + 1)
    return r


def config_counts(species, target, b, q):
    """(#left configurations with charge q, #right configurations completing to target)."""
    K = len(species)
    L = [0, 0]
    R = [0, 0]
    for t in range(K):
        (L if t < b else R)[species[t]] += 1
    left = _binom(L[0], q[0]) * _binom(L[1], q[1])
    right = _binom(R[0], target[0] - q[0]) * _binom(R[1], target[1] - q[1])
    return left, right


def default_dims(species, target, r_max, D=1):
    """Block dims rho_{b,q} of a fresh iterate of maximal rank r_max:
    rho = min(left count, right count) when these fit r_max in total, otherwise
    rho = min(left, right, floor(r_max * left*right / sum_q left*right)) (exact
    integer arithmetic); sectors of dim 0 are dropped.  For a joint block MPS of
    D columns (Sec. 6.2, column index after the last site) the right counts are
    multiplied by D, so the last bond has dimension D."""
    K = len(species)
    ranges = valid_ranges(species, target)
    dims = []
    for b in range(K + 1):
        cnt = [(l, r * D) for l, r in (config_counts(species, target, b, q) for q in ranges[b])]
        exact = [min(l, r) for l, r in cnt]
        if sum(exact) <= r_max:
            d = exact
        else:
            wsum = sum(l * r for l, r in cnt)
            d = [min(l, r, (r_max * l * r) // wsum) for l, r in cnt]
        dims.append({q: x for q, x in zip(ranges[b], d) if x > 0})
    return dims


class BSMPS:
    """Block-sparse MPS: bonds[b] = {charge: dim} (ascending), cores[t] = {(n, sigma): block}."""

    def __init__(self, species, target, bonds, cores):
        self.species = tuple(species)
        self.target = tuple(target)
        self.bonds = bonds
        self.cores = cores

    @property
    def K(self):
        return len(self.species)

    def copy(self):
        return BSMPS(self.species, self.target, [dict(b) for b in self.bonds],
                     [{k: v.copy() for k, v in c.items()} for c in self.cores])

    def ranks(self):
        return [sum(b.values()) for b in self.bonds]

    def block_keys(self, t):
        """Ordered block keys of core t (layout order)."""
        keys = []
        for n in sorted(self.bonds[t]):
            for sg in (0, 1):
                m = add_charge(n, delta(self.species[t], sg))
                if m in self.bonds[t + 1]:
                    keys.append((n, sg))
        return keys

    def layout(self):
        """[(t, n, sigma, rows, cols, offset)] in flat order, and the total size."""
        out = []
        off = 0
        for t in range(self.K):
            for (n, sg) in self.block_keys(t):
                m = add_charge(n, delta(self.species[t], sg))
                r, c = self.bonds[t][n], self.bonds[t + 1][m]
                out.append((t, n, sg, r, c, off))
                off += r * c
        return out, off

    def to_flat(self):
        lay, total = self.layout()
        v = np.zeros(total)
        for (t, n, sg, r, c, off) in lay:
            v[off:off + r * c] = self.cores[t][(n, sg)].reshape(-1)
        return v

    @staticmethod
    def from_flat(species, target, bonds, values):
        x = BSMPS(species, target, bonds, [dict() for _ in range(len(species))])
        lay, total = x.layout()
        assert len(values) == total, (len(values), total)
        for (t, n, sg, r, c, off) in lay:
            x.cores[t][(n, sg)] = np.array(values[off:off + r * c], dtype=np.float64).reshape(r, c)
        return x


def random_mps(species, target, r_max, values):
    dims = default_dims(species, target, r_max)
    return BSMPS.from_flat(species, target, dims, values)


def e1_mps(species, target):
    """Rank-one e_1 (Sec. 7.1.4): lowest determinant, the first N_s sites of each
    species occupied."""
    K = len(species)
    occ = []
    seen = [0, 0]
    for t in range(K):
        s = species[t]
        o = 1 if seen[s] < target[s] else 0
        seen[s] += o
        occ.append(o)
    bonds = [{(0, 0): 1}]
    q = (0, 0)
    for t in range(K):
        q = add_charge(q, delta(species[t], occ[t]))
        bonds.append({q: 1})
    cores = []
    q = (0, 0)
    for t in range(K):
        cores.append({(q, occ[t]): np.ones((1, 1))})
        q = add_charge(q, delta(species[t], occ[t]))
    return BSMPS(species, target, bonds, cores)


def to_dense(x):
    """Contract to the full 2^K vector (site 0 slowest), tiny K only (Eq. (mps))."""
    K = x.K
    cur = {(0, 0): np.ones((1, 1))}        # bond charge -> (configs, rho)
    for t in range(K):
        nxt = {}
        for (n, sg), B in x.cores[t].items():
            if n not in cur:
                continue
            m = add_charge(n, delta(x.species[t], sg))
            left = cur[n]
            rows = left.shape[0]
            blk = np.zeros((rows * 2, B.shape[1]))
            blk[sg::2] = left @ B
            nxt[m] = nxt[m] + blk if m in nxt else blk
        cur = nxt
    if x.target not in cur:
        return np.zeros(1 << K)
    return cur[x.target][:, 0]


def columns(x):
    """Number of represented vectors: the dimension of the last bond (1 for a
    plain MPS, D for a joint block MPS with the eigenvector index there, Sec. 6.2)."""
    return sum(x.bonds[x.K].values())


def to_dense_cols(x):
    """Dense 2^K x D matrix of a joint block MPS (column i = vector i), tiny K only."""
    K = x.K
    cur = {(0, 0): np.ones((1, 1))}
    for t in range(K):
        nxt = {}
        for (n, sg), B in x.cores[t].items():
            if n not in cur:
                continue
            m = add_charge(n, delta(x.species[t], sg))
            left = cur[n]
            blk = np.zeros((left.shape[0] * 2, B.shape[1]))
            blk[sg::2] = left @ B
            nxt[m] = nxt[m] + blk if m in nxt else blk
        cur = nxt
    if x.target not in cur:
        return np.zeros((1 << K, columns(x)))
    return cur[x.target]


def scale_sites(x, f0, f1):
    """Multiply every sigma=0 block of site t by f0[t] and every sigma=1 block by f1[t]
    (action of one rank-one diagonal Kronecker factor, Sec. 4.3)."""
    y = x.copy()
    for t in range(x.K):
        for (n, sg) in y.cores[t]:
            y.cores[t][(n, sg)] = y.cores[t][(n, sg)] * (f1[t] if sg else f0[t])
    return y


def scale(x, alpha):
    """alpha * x: multiply every block of the first core (Sec. 2.3)."""
    y = x.copy()
    for k in y.cores[0]:
        y.cores[0][k] = alpha * y.cores[0][k]
    return y


def add(x, y, alpha=1.0, beta=1.0):
    """alpha x + beta y by block concatenation (Sec. 2.3): bond sectors of the
    sum are the union; inner bonds stack x's basis before y's; the scalars
    scale the first core's blocks."""
    K = x.K
    bonds = []
    for b in range(K + 1):
        if b == 0:
            qs = sorted(set(x.bonds[b]) | set(y.bonds[b]))
            bonds.append({q: 1 for q in qs})
        elif b == K:
            # the last bond carries the column index of a joint block MPS (Sec. 6.2):
            # both summands have the same columns, which are added, not stacked
            qs = sorted(set(x.bonds[b]) | set(y.bonds[b]))
            for q in qs:
                if q in x.bonds[b] and q in y.bonds[b]:
                    assert x.bonds[b][q] == y.bonds[b][q], "different column counts"
            bonds.append({q: x.bonds[b].get(q, y.bonds[b].get(q)) for q in qs})
        else:
            qs = sorted(set(x.bonds[b]) | set(y.bonds[b]))
            bonds.append({q: x.bonds[b].get(q, 0) + y.bonds[b].get(q, 0) for q in qs})
    cores = [dict() for _ in range(K)]
    for t in range(K):
        sp = x.species[t]
        for n in bonds[t]:
            for sg in (0, 1):
                m = add_charge(n, delta(sp, sg))
                if m not in bonds[t + 1]:
                    continue
                B = np.zeros((bonds[t][n], bonds[t + 1][m]))
                if (n, sg) in x.cores[t]:
                    X = x.cores[t][(n, sg)] * (alpha if t == 0 else 1.0)
                    B[:X.shape[0], :X.shape[1]] += X
                if (n, sg) in y.cores[t]:
                    Y = y.cores[t][(n, sg)] * (beta if t == 0 else 1.0)
                    r0 = 0 if t == 0 else x.bonds[t].get(n, 0)
                    c0 = 0 if t == K - 1 else x.bonds[t + 1].get(m, 0)
                    B[r0:r0 + Y.shape[0], c0:c0 + Y.shape[1]] += Y
                cores[t][(n, sg)] = B
    return BSMPS(x.species, x.target, bonds, cores)


def apply_exact(mpo, x, shift=0.0, col_shift=None):
    """y = (H + shift I) x without truncation (Sec. 2.4): y's bond-b basis is the
    product of MPO channels a and x's basis; sector m holds segments (a, n) with
    n = m - Delta_a, ordered by channel; sectors outside the valid sets are
    dropped (no complete path runs through them).  Each sub-block (a, b) of
    y's block (m, sigma') equals sum w(a,b,sigma',sigma) X(n_a, sigma).

    col_shift (joint block MPS, Sec. 6.1): column i of y gets col_shift[i] x_i
    added, i.e. y = H X + X diag(col_shift).  The identity reaches the last site
    on the MPO's identity rail (channel I on every bond before the last site),
    so the term is X's last core times diag(col_shift) added to the (I, F)
    sub-block of each last-site block."""
    K = x.K
    ranges = valid_ranges(x.species, x.target)
    segs = []
    bonds = []
    for b in range(K + 1):
        seg = {}
        for m in ranges[b]:
            lst = []
            off = 0
            for a, d in enumerate(mpo.charges[b]):
                n = sub_charge(m, d)
                if n in x.bonds[b]:
                    lst.append((a, n, off, x.bonds[b][n]))
                    off += x.bonds[b][n]
            if off > 0:
                seg[m] = (lst, off)
        segs.append(seg)
        bonds.append({m: v[1] for m, v in seg.items()})
    cores = [dict() for _ in range(K)]
    for t in range(K):
        sp = x.species[t]
        ents = mpo.entries(t, shift)
        for m in bonds[t]:
            for so in (0, 1):
                m2 = add_charge(m, delta(sp, so))
                if m2 not in bonds[t + 1]:
                    continue
                Y = np.zeros((bonds[t][m], bonds[t + 1][m2]))
                rowseg = {a: (n, off, d) for (a, n, off, d) in segs[t][m][0]}
                colseg = {a: (n, off, d) for (a, n, off, d) in segs[t + 1][m2][0]}
                for (a, b, eo, ei, w) in ents:
                    if eo != so or a not in rowseg or b not in colseg:
                        continue
                    n_a, r0, rd = rowseg[a]
                    n_b, c0, cd = colseg[b]
                    if (n_a, ei) not in x.cores[t]:
                        continue
                    assert add_charge(n_a, delta(sp, ei)) == n_b
                    Y[r0:r0 + rd, c0:c0 + cd] += w * x.cores[t][(n_a, ei)]
                if col_shift is not None and t == K - 1:
                    a = mpo.channels[t].index(("I",))
                    if a in rowseg and 0 in colseg and (rowseg[a][0], so) in x.cores[t]:
                        n_a, r0, rd = rowseg[a]
                        _, c0, cd = colseg[0]
                        Y[r0:r0 + rd, c0:c0 + cd] += x.cores[t][(n_a, so)] * np.asarray(col_shift)[None, :]
                cores[t][(m, so)] = Y
    return BSMPS(x.species, x.target, bonds, cores)


def mix_columns(x, W):
    """X W for a joint block MPS (Sec. 6.1): the last core's blocks times the
    D_in x D_out matrix W; the last bond becomes D_out wide."""
    W = np.asarray(W, dtype=np.float64)
    assert W.shape[0] == columns(x)
    y = x.copy()
    K = y.K
    for k in list(y.cores[K - 1].keys()):
        y.cores[K - 1][k] = y.cores[K - 1][k] @ W
    y.bonds[K] = {q: W.shape[1] for q in y.bonds[K]}
    return y


def _environments(a, b, mpo=None, shift=0.0):
    """Environments at bond K of <a, O b> by the left-to-right recursion (Sec. 2.4):
    E_{t+1}[d](n_a', n_b') = sum w(c,d,s',s) A(n_a,s')^T E_t[c](n_a,n_b) B(n_b,s).
    With mpo=None, O is the identity (one channel)."""
    K = a.K
    if mpo is None:
        charges = [[(0, 0)] for _ in range(K + 1)]

        def ents(t):
            return [(0, 0, 0, 0, 1.0), (0, 0, 1, 1, 1.0)]
    else:
        charges = mpo.charges

        def ents(t):
            return mpo.entries(t, shift)
    E = {0: {((0, 0), (0, 0)): np.ones((1, 1))}}
    for t in range(K):
        sp = a.species[t]
        nE = {}
        for (c, d, so, si, w) in ents(t):
            for (na, nb), M in E.get(c, {}).items():
                if (na, so) not in a.cores[t] or (nb, si) not in b.cores[t]:
                    continue
                A = a.cores[t][(na, so)]
                B = b.cores[t][(nb, si)]
                key = (add_charge(na, delta(sp, so)), add_charge(nb, delta(sp, si)))
                val = w * (A.T @ M @ B)
                Ed = nE.setdefault(d, {})
                Ed[key] = Ed[key] + val if key in Ed else val
        E = nE
    return E


def dot(a, b, mpo=None, shift=0.0):
    """<a, O b> (Sec. 2.4) for MPS with one column."""
    tot = 0.0
    for Ec in _environments(a, b, mpo, shift).values():
        for M in Ec.values():
            tot += M[0, 0]
    return tot


def gram(a, b, mpo=None, shift=0.0):
    """The D_a x D_b matrix <a_i, O b_j> of two joint block MPS (Sec. 6.1): the
    same recursion, whose last environment keeps both column indices."""
    G = np.zeros((columns(a), columns(b)))
    for Ec in _environments(a, b, mpo, shift).values():
        for M in Ec.values():
            G += M
    return G


def norm(x):
    return float(np.sqrt(max(dot(x, x), 0.0)))


def _sign_fix_qr(Q, R):
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :], R * d[:, None]


def left_orthogonalize(x):
    """Left-to-right QR sweep (Sec. 2.3): for every bond b = 1..K-1 and sector m,
    QR of the stacked blocks (n, sigma) -> m of core b-1 (rows in layout
    order), R multiplied into core b.  diag(R) >= 0.  New dim = min(rows, cols)."""
    y = x.copy()
    K = y.K
    for t in range(K - 1):
        sp = y.species[t]
        newdims = {}
        for m in sorted(y.bonds[t + 1]):
            keys = [(n, sg) for (n, sg) in y.block_keys(t)
                    if add_charge(n, delta(sp, sg)) == m]
            if not keys:
                newdims[m] = 0
                continue
            M = np.vstack([y.cores[t][k] for k in keys])
            Q, R = np.linalg.qr(M, mode="reduced")
            Q, R = _sign_fix_qr(Q, R)
            k_new = Q.shape[1]
            r0 = 0
            for k in keys:
                rr = y.cores[t][k].shape[0]
                y.cores[t][k] = Q[r0:r0 + rr, :]
                r0 += rr
            for sg in (0, 1):
                if (m, sg) in y.cores[t + 1]:
                    y.cores[t + 1][(m, sg)] = R @ y.cores[t + 1][(m, sg)]
            newdims[m] = k_new
        _set_bond(y, t + 1, newdims)
    return y


def _set_bond(y, b, newdims):
    """Replace bond b's dims; drop sectors of dim 0 and the blocks touching them."""
    y.bonds[b] = {q: d for q, d in sorted(newdims.items()) if d > 0}
    t_left, t_right = b - 1, b
    if t_left >= 0:
        sp = y.species[t_left]
        y.cores[t_left] = {(n, sg): B for (n, sg), B in y.cores[t_left].items()
                           if add_charge(n, delta(sp, sg)) in y.bonds[b]}
    if t_right < y.K:
        y.cores[t_right] = {(n, sg): B for (n, sg), B in y.cores[t_right].items()
                            if n in y.bonds[b]}


CLUSTER_RTOL = 1e-10


def choose_cut(svals, tol2, r_max):
    """Which pooled singular values survive at one bond (Sec. 2.2, trunc_eps).

    svals: list of (sigma, sector_index, j).  Sorted descending with ties by
    (sector_index, j).  The smallest are discarded while their squared sum
    stays <= tol2; a cut inside a cluster (relative gap < CLUSTER_RTOL) moves
    up to keep the whole cluster.  Then at most r_max are kept (r_max <= 0:
    no cap); a cap cut inside a cluster moves down to the cluster edge unless
    that would keep nothing.  Returns (kept set of (sector_index, j),
    discarded squared norm from the tolerance, discarded squared norm from
    the cap)."""
    order = sorted(svals, key=lambda e: (-e[0], e[1], e[2]))
    n = len(order)
    keep = n
    acc = 0.0
    while keep > 0:
        s = order[keep - 1][0]
        if acc + s * s <= tol2:
            acc += s * s
            keep -= 1
        else:
            break
    while 0 < keep < n and order[keep][0] >= order[keep - 1][0] * (1.0 - CLUSTER_RTOL):
        keep += 1
    tol_disc = sum(e[0] ** 2 for e in order[keep:])
    cap_disc = 0.0
    if r_max > 0 and keep > r_max:
        k2 = r_max
        while 0 < k2 and order[k2][0] >= order[k2 - 1][0] * (1.0 - CLUSTER_RTOL):
            k2 -= 1
        if k2 == 0:
            k2 = r_max
        cap_disc = sum(e[0] ** 2 for e in order[k2:keep])
        keep = k2
    return set((e[1], e[2]) for e in order[:keep]), tol_disc, cap_disc


def _sign_fix_svd(U, S, Vt):
    for i in range(Vt.shape[0]):
        j = int(np.argmax(np.abs(Vt[i])))
        if Vt[i, j] < 0:
            Vt[i] = -Vt[i]
            U[:, i] = -U[:, i]
    return U, S, Vt


def truncate(x, eps, r_max=0):
    """trunc_eps (Sec. 2.2): left-orthogonalise, then sweep right to left; at bond
    b = K-1..1 take the SVD of [X_b(n,0) | X_b(n,1)] per left sector n, pool the
    singular values of the bond and drop the tail with squared sum <=
    eps^2/(K-1) (so ||x - trunc|| <= eps by Eq. (ttsvdquasiopt)), cap at r_max,
    keep V^T in core b and multiply U S into core b-1.  Sign: the largest |entry|
    of each row of V^T is positive.  Returns (y, discarded_tol, discarded_cap)
    with the discarded norms (square roots of the summed squares)."""
    y = left_orthogonalize(x)
    K = y.K
    tol2 = (eps * eps) / (K - 1) if K > 1 else 0.0
    tot_tol = 0.0
    tot_cap = 0.0
    for t in range(K - 1, 0, -1):
        sp = y.species[t]
        sectors = sorted(y.bonds[t])
        dec = {}
        svals = []
        for si, n in enumerate(sectors):
            parts = [(sg, y.cores[t][(n, sg)]) for sg in (0, 1) if (n, sg) in y.cores[t]]
            if not parts:
                continue
            M = np.hstack([B for _, B in parts])
            U, S, Vt = np.linalg.svd(M, full_matrices=False)
            U, S, Vt = _sign_fix_svd(U, S, Vt)
            dec[n] = (parts, U, S, Vt)
            for j, s in enumerate(S):
                svals.append((float(s), si, j))
        kept, dt, dc = choose_cut(svals, tol2, r_max)
        tot_tol += dt
        tot_cap += dc
        newdims = {}
        for si, n in enumerate(sectors):
            if n not in dec:
                newdims[n] = 0
                continue
            parts, U, S, Vt = dec[n]
            idx = [j for j in range(len(S)) if (si, j) in kept]
            k = len(idx)
            newdims[n] = k
            c0 = 0
            for sg, B in parts:
                cw = B.shape[1]
                y.cores[t][(n, sg)] = Vt[idx, c0:c0 + cw]
                c0 += cw
            US = U[:, idx] * S[idx][None, :]
            psp = y.species[t - 1]
            for (pn, psg) in list(y.cores[t - 1].keys()):
                if add_charge(pn, delta(psp, psg)) == n:
                    y.cores[t - 1][(pn, psg)] = y.cores[t - 1][(pn, psg)] @ US
        _set_bond(y, t, newdims)
    return y, float(np.sqrt(tot_tol)), float(np.sqrt(tot_cap))


def _exact_segments(mpo, x):
    """Per bond b and valid sector m of y = (H + s) x: the channel segments
    [(a, n, offset, rho_x(n))] of y's exact basis (channel-major, n = m - Delta_a)
    and its total dimension (Sec. 2.4; the bond basis of apply_exact)."""
    K = x.K
    ranges = valid_ranges(x.species, x.target)
    segs = []
    for b in range(K + 1):
        seg = {}
        for m in ranges[b]:
            lst = []
            off = 0
            for a, d in enumerate(mpo.charges[b]):
                n = sub_charge(m, d)
                if n in x.bonds[b]:
                    lst.append((a, n, off, x.bonds[b][n]))
                    off += x.bonds[b][n]
            if off > 0:
                seg[m] = (lst, off)
        segs.append(seg)
    return segs


def apply_zipup(mpo, x, shift=0.0):
    """y = (H + shift I) x in left-orthogonal form, contracted site by site
    (Sec. 2.4 with the left-to-right QR sweep of Sec. 2.3) without forming the
    exact cores of apply_exact.

    The carry C_t[m] (rho_y(m) x rho_exact(m)) maps y's orthogonalised bond-t
    basis to the exact basis (channel a, x's sector n = m - Delta_a).  At site t
        T[(m, s')][:, seg_b] = sum_{(a, s): W_t(a, b, s', s) != 0}
                               w C_t[m][:, seg_a] X_t(n_a, s),
    and for every sector m' of bond t+1 the blocks (m, s') with m + delta(s') = m'
    are stacked in layout order (m ascending, then s') and factorised S = Q R:
    Q gives y's core-t blocks, R = C_{t+1}[m'].  A stack with no more rows than
    columns takes Q = I, R = S (an exact orthogonalisation; its rank is the row
    count); otherwise Householder QR with diag(R) >= 0.  At the last site the
    blocks T are y's last core.  Equal to left_orthogonalize(apply_exact(...))
    in exact arithmetic up to the gauge of the bond bases."""
    K = x.K
    segs = _exact_segments(mpo, x)
    C = {m: np.eye(v[1]) for m, v in segs[0].items()}
    bonds = [{m: v[1] for m, v in segs[0].items()}]
    cores = []
    for t in range(K):
        sp = x.species[t]
        ents = mpo.entries(t, shift)
        T = {}
        for m in sorted(C):
            Cm = C[m]
            rowseg = {a: (n, off, d) for (a, n, off, d) in segs[t][m][0]}
            for so in (0, 1):
                m2 = add_charge(m, delta(sp, so))
                if m2 not in segs[t + 1]:
                    continue
                colseg = {b: (n, off, d) for (b, n, off, d) in segs[t + 1][m2][0]}
                Tb = np.zeros((Cm.shape[0], segs[t + 1][m2][1]))
                for (a, b, eo, ei, w) in ents:
                    if eo != so or a not in rowseg or b not in colseg:
                        continue
                    n_a, r0, rd = rowseg[a]
                    _, c0, cd = colseg[b]
                    if (n_a, ei) not in x.cores[t]:
                        continue
                    Tb[:, c0:c0 + cd] += w * (Cm[:, r0:r0 + rd] @ x.cores[t][(n_a, ei)])
                T[(m, so)] = Tb
        if t == K - 1:
            cores.append(T)
            bonds.append({m: v[1] for m, v in segs[K].items()})
            break
        core = {}
        newC = {}
        for m2 in sorted(segs[t + 1]):
            keys = [(m, so) for (m, so) in sorted(T) if add_charge(m, delta(sp, so)) == m2]
            if not keys:
                continue
            S = np.vstack([T[k] for k in keys])
            rows, cols = S.shape
            if rows <= cols:
                Q, R = np.eye(rows), S
            else:
                Q, R = _sign_fix_qr(*np.linalg.qr(S, mode="reduced"))
            r0 = 0
            for k in keys:
                rr = T[k].shape[0]
                core[k] = Q[r0:r0 + rr, :]
                r0 += rr
            newC[m2] = R
        cores.append(core)
        bonds.append({m2: R.shape[0] for m2, R in sorted(newC.items())})
        C = newC
    return BSMPS(x.species, x.target, bonds, cores)
