"""Shared helpers for the parity tests (the oracle side and the library side)."""

import numpy as np

from oracle import bsmps as OB
from oracle import fermion as OF
from oracle import mpo as OM
from oracle import precond as OP


def species_of(wl):
    return OF.site_species(wl.n_orb, wl.spin)


def target_of(wl):
    return (wl.n_up, wl.n_dn)


def oracle_random(wl, r_max, values):
    return OB.random_mps(species_of(wl), target_of(wl), r_max, values)


def n_random(wl, r_max):
    dims = OB.default_dims(species_of(wl), target_of(wl), r_max)
    tmp = OB.BSMPS(species_of(wl), target_of(wl), dims, [dict() for _ in species_of(wl)])
    return tmp.layout()[1]


def to_oracle(wl, gpu_mps):
    """The library's result in the oracle's representation (same flat layout)."""
    return OB.BSMPS.from_flat(species_of(wl), target_of(wl), gpu_mps.bonds(), gpu_mps.export())


def stable_norm(x):
    """||x|| without cancellation: after a QR sweep the last core carries the norm."""
    lo = OB.left_orthogonalize(x)
    return float(np.sqrt(sum(np.sum(B * B) for B in lo.cores[-1].values())))


def rel_distance(a, b):
    """||a - b|| / max(||a||, ||b||) of the represented tensors (oracle arithmetic)."""
    d = stable_norm(OB.add(a, b, 1.0, -1.0))
    return d / max(stable_norm(a), stable_norm(b), 1e-300)


def block_norms(x):
    out = {}
    for t in range(x.K):
        for k, B in x.cores[t].items():
            out[(t, k)] = float(np.linalg.norm(B))
    return out


def precond_for(wl, gamma, c0=0.1, alpha0=0.7):
    """Diagonal theta of Sec. 7.1.1, [t_min, t_max] and the term factors (oracle)."""
    t_so, v_so = OP.spin_orbital_accessors(wl.h, wl.eri, wl.spin)
    K = wl.n_sites
    th = OP.theta_diag(t_so, v_so, wl.n_particles, gamma, K)
    tmin, tmax = OP.spectrum_bounds(th, species_of(wl), target_of(wl))
    return th, tmin, tmax, OP.Preconditioner(th, tmin, tmax, c0, alpha0)


def oracle_mpo(wl, gamma):
    return OM.build_mpo(wl.h, wl.eri, wl.spin, wl.n_particles, gamma)


def amplitude(x, occ):
    """<occ|x>: the product of the blocks along the occupation string's sector path
    (Eq. (mps)); 0 when the path leaves the stored sectors."""
    v = np.ones((1, 1))
    q = (0, 0)
    for t, s in enumerate(occ):
        key = (q, int(s))
        if key not in x.cores[t]:
            return 0.0
        v = v @ x.cores[t][key]
        q = OB.add_charge(q, OB.delta(x.species[t], int(s)))
    return float(v[0, 0])


def random_occupations(species, target, n, seed):
    """n random occupation strings of the particle sector (target per species)."""
    rng = np.random.default_rng(seed)
    species = np.asarray(species)
    out = []
    for _ in range(n):
        occ = np.zeros(len(species), dtype=np.int64)
        for s in (0, 1):
            sites = np.flatnonzero(species == s)
            if target[s]:
                occ[rng.choice(sites, size=target[s], replace=False)] = 1
        out.append(occ)
    return out
