"""Seeded generators for the synthetic Hamiltonians and initial iterates.

Integrals use the chemist convention (pq|rs) with 8-fold permutational
symmetry; one-body matrices are symmetric.  All arrays are float64, C-ordered.

Recipes (sizes as used by the tests and the bench):

* spinless random chain: K sites, h_pq ~ N(0,1) exp(-|p-q|/3) (symmetric),
  h_pp += 0.5 p (p = 0..K-1); (pq|rs) = sum_g L^g_pq L^g_rs with L^g = 0.1 G^g,
  G^g symmetric with N(0,1) entries, 8 vectors.  PSD and 8-fold symmetric by
  construction.
* Hubbard chain: L spatial sites, h_{p,p+1} = h_{p+1,p} = -t (open ends),
  (pp|pp) = U, everything else zero.
* molecule-like: h_pp = linspace(-2, 2, L); off-diagonal N(0, 0.05) exp(-|p-q|/6)
  (symmetric); (pq|rs) from n_chol Cholesky-like vectors, L^g = 0.1 G^g.
* one-dimensional Coulomb-like model (the paper's Sec. 7.2 Hamiltonian, with
  finite-difference orbitals standing in for the paper's multiwavelet ones):
  N particles of equal spin on [-b, b] with V(x) = -N delta_0(x) and
  V_2(x, y) = c_V exp(-|x - y|).  The orbitals are the K lowest eigenvectors of
  -1/2 d^2/dx^2 + V on a uniform grid (n_grid intervals, Dirichlet ends, the
  delta as -N/h at the node x = 0), so h = diag(omega); (pq|rs) are grid sums
  h sum_s phi_p phi_q (s) [V_2 (phi_r phi_s)](s), the discrete convolution
  with exp(-|x - y|) taken by a forward and a backward recursion.
"""

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    n_orb: int              # spatial orbitals (= sites when spinless)
    spin: int               # 0: spinless sites; 1: spin-orbitals interleaved (p up, p down)
    n_up: int               # particles of species 0 (all particles when spinless)
    n_dn: int               # particles of species 1 (0 when spinless)
    h: np.ndarray           # (n_orb, n_orb)
    eri: np.ndarray         # (n_orb, n_orb, n_orb, n_orb), chemist (pq|rs)
    r_max: int
    seed: int
    extra: dict = field(default_factory=dict)

    @property
    def n_sites(self) -> int:
        return self.n_orb * (2 if self.spin else 1)

    @property
    def n_particles(self) -> int:
        return self.n_up + self.n_dn


def _sym_gauss(rng, n, scale=1.0):
    g = rng.standard_normal((n, n))
    return scale * (np.triu(g) + np.triu(g, 1).T)


def _cholesky_eri(rng, n, n_chol, scale):
    eri = np.zeros((n, n, n, n))
    for _ in range(n_chol):
        lg = _sym_gauss(rng, n, scale)
        eri += np.einsum("pq,rs->pqrs", lg, lg)
    return eri


def spinless_random_chain(K=12, N=6, r_max=32, seed=0, n_chol=8):
    rng = np.random.default_rng(seed)
    p = np.arange(K)
    decay = np.exp(-np.abs(p[:, None] - p[None, :]) / 3.0)
    h = _sym_gauss(rng, K) * decay
    h[p, p] += 0.5 * p
    eri = _cholesky_eri(rng, K, n_chol, 0.1)
    return Workload("spinless_random_chain", K, 0, N, 0, h, eri, r_max, seed)


def hubbard_chain(L=32, n_up=None, n_dn=None, t=1.0, U=4.0, r_max=256, seed=0):
    n_up = L // 2 if n_up is None else n_up
    n_dn = L // 2 if n_dn is None else n_dn
    h = np.zeros((L, L))
    for p in range(L - 1):
        h[p, p + 1] = h[p + 1, p] = -t
    eri = np.zeros((L, L, L, L))
    for p in range(L):
        eri[p, p, p, p] = U
    return Workload("hubbard_chain", L, 1, n_up, n_dn, h, eri, r_max, seed,
                    extra={"t": t, "U": U})


def molecule_like(L=24, n_up=None, n_dn=None, r_max=1024, seed=0, n_chol=None):
    n_up = L // 2 if n_up is None else n_up
    n_dn = L // 2 if n_dn is None else n_dn
    n_chol = 2 * L if n_chol is None else n_chol
    rng = np.random.default_rng(seed)
    p = np.arange(L)
    decay = np.exp(-np.abs(p[:, None] - p[None, :]) / 6.0)
    off = _sym_gauss(rng, L, 0.05) * decay
    np.fill_diagonal(off, 0.0)
    h = off + np.diag(np.linspace(-2.0, 2.0, L))
    eri = _cholesky_eri(rng, L, n_chol, 0.1)
    return Workload("molecule_like", L, 1, n_up, n_dn, h, eri, r_max, seed)


def coulomb_1d(K=14, N=4, b=4.0, c_v=4.0, n_grid=16384, r_max=64):
    import scipy.linalg

    hx = 2.0 * b / n_grid
    m = n_grid - 1                                    # interior nodes
    diag = np.full(m, 1.0 / hx ** 2)
    diag[m // 2] += -N / hx                           # delta potential at x = 0
    off = np.full(m - 1, -0.5 / hx ** 2)
    omega, vec = scipy.linalg.eigh_tridiagonal(diag, off, select="i", select_range=(0, K - 1))
    phi = vec / np.sqrt(hx)                           # L2-normalised on the grid
    prod = np.einsum("sp,sq->pqs", phi, phi).reshape(K * K, m)
    a = np.exp(-hx)
    fwd = np.empty_like(prod)
    bwd = np.empty_like(prod)
    fwd[:, 0] = prod[:, 0]
    for s in range(1, m):
        fwd[:, s] = prod[:, s] + a * fwd[:, s - 1]
    bwd[:, m - 1] = prod[:, m - 1]
    for s in range(m - 2, -1, -1):
        bwd[:, s] = prod[:, s] + a * bwd[:, s + 1]
    conv = c_v * hx * (fwd + bwd - prod)              # [V_2 (phi_r phi_s)] on the grid
    eri = (hx * prod @ conv.T).reshape(K, K, K, K)
    eri = 0.5 * (eri + eri.transpose(2, 3, 0, 1))     # exact pair symmetry against rounding
    return Workload("coulomb_1d", K, 0, N, 0, np.diag(omega), eri, r_max, 0,
                    extra={"b": b, "c_v": c_v, "n_grid": n_grid})


def random_block_values(n, seed=0):
    """n standard-normal float64 entries for the blocks of a random iterate."""
    return np.random.default_rng(seed).standard_normal(n)
