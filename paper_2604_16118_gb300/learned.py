"""Learned preconditioner controller.

A small network (``native.MLP``: 128 -> 256 -> 256 -> 256 -> 2, BF16 weights,
FP32 accumulation, trained by the library's own forward/backward/Adam
kernels) predicts two parameters of the paper's exponential-sum
preconditioner for a problem: the quadrature accuracy c_0 of Eq.
(expsumparams) -- which sets the number of terms M^+ - M^- + 1 and hence the
J = (#S)^2 residual terms of every step -- and the margin of the shift gamma
above the rigorous lower bound of the ground energy.  Inputs are the one-body
diagonal theta of Sec. 7.1.1 (sorted, normalised) and the residual history of
the run.

Training data come from the plain solver: for every problem of a set, each
(c_0, margin) of a small grid runs a few Alg. 2 steps from e_1 and is scored by
the decrease of the energy per GFLOP; the label is the best grid point.  At
run time the prediction is snapped to the grid, so every parameter set the
controller uses is a valid plain-preconditioner parameter set.  The plain
parameters (c_0 = 0.1, the paper's value, margin 1) are the fallback: they are
used when the prediction is not finite, and the controller switches back to
them when a learned step fails to lower the Rayleigh quotient.
"""

import math

import numpy as np

from . import native as nat
from . import problem

WIDTHS = [128, 256, 256, 256, 2]
C0_GRID = (0.05, 0.1, 0.2, 0.4)
MARGIN_GRID = (0.5, 1.0, 2.0)
PLAIN = (0.1, 1.0)
# solver constants used for the controller's problems (no exact diagonalisation)
SOLVER = {"c": 0.7, "delta": 20.0, "t_eig": 0.5, "C_lower": 0.3, "C_upper": 1.5}


def is_hubbard(wl):
    return getattr(wl, "name", "") == "hubbard_chain"


def shift(wl, margin):
    if is_hubbard(wl):
        return problem.hubbard_shift(wl.h, wl.n_up, wl.n_dn, margin=margin)
    return problem.cholesky_shift(wl.h, wl.eri, wl.n_up, wl.n_dn, wl.spin, margin=margin)


def setup(ctx, wl, c0, margin, r_max=64):
    """MPO, preconditioner and solver parameters of one (c_0, margin) choice."""
    gamma = shift(wl, margin)
    th = problem.theta_diagonal(wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    tmin, tmax = problem.spectrum_bounds(th, wl.spin, wl.n_up, wl.n_dn)
    if not (tmin > 0.0):
        raise ValueError("t_min <= 0: the shift margin is too small for this problem")
    alpha0, _ = problem.alpha0_and_c(c0, tmin, SOLVER["C_lower"], SOLVER["C_upper"])   # Eq. (Sdef)
    W = nat.mpo_from_integrals(ctx, wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    p = nat.make_precond(th, tmin, tmax, c0, alpha0)
    sp = nat.solver_params(SOLVER["c"], SOLVER["delta"], t_eig=SOLVER["t_eig"], tau=1e-14, r_max=r_max)
    return dict(W=W, p=p, sp=sp, gamma=gamma, theta=th, tmin=tmin, tmax=tmax)


def features(wl, rho_hist=()):
    """128 inputs: sorted theta / max|theta| (64 slots), spectral summary (8),
    log10 of up to 16 recent rho values (16), zero padding."""
    gamma = shift(wl, 1.0)
    th = problem.theta_diagonal(wl.h, wl.eri, wl.spin, wl.n_particles, gamma)
    tmin, tmax = problem.spectrum_bounds(th, wl.spin, wl.n_up, wl.n_dn)
    f = np.zeros(128, dtype=np.float32)
    s = np.sort(th)[:64]
    scale = max(np.abs(th).max(), 1e-12)
    f[:len(s)] = s / scale
    K = len(th)
    f[64:72] = [K / 64.0, wl.n_particles / max(K, 1), float(wl.spin), math.log(max(tmax / tmin, 1.0)),
                th.std() / scale, (th.max() - th.min()) / scale, tmin / scale / max(wl.n_particles, 1),
                float(is_hubbard(wl))]
    for i, r in enumerate(list(rho_hist)[-16:]):
        f[80 + i] = math.log10(max(r, 1e-300))
    return f


def run(ctx, wl, c0, margin, n_steps, r_max=64):
    """Plain solver from e_1 with the given parameters: energies lambda - gamma at
    the start of every step, flops per step, rho per step."""
    S = setup(ctx, wl, c0, margin, r_max)
    st = nat.solver_state()
    x = nat.mps_create(ctx, wl.n_orb, wl.spin, wl.n_up, wl.n_dn)
    E, F, R = [], [], []
    for _ in range(n_steps):
        x, info = nat.eigensolve_step(ctx, S["W"], S["p"], S["sp"], st, x)
        E.append(info["lambda"] - S["gamma"])
        F.append(info["flops"])
        R.append(info["rho"])
        if info["converged"]:
            break
    return E, F, R


def score(E, F):
    """Energy decrease per GFLOP between the first and the last step start."""
    if len(E) < 2:
        return 0.0
    fl = sum(F[:len(E) - 1]) * 1e-9
    return (E[0] - E[-1]) / max(fl, 1e-12)


def grid_scores(ctx, wl, n_steps=4):
    """{(c0, margin): score} of the plain solver on one problem."""
    out = {}
    for c0 in C0_GRID:
        for m in MARGIN_GRID:
            try:
                E, F, _ = run(ctx, wl, c0, m, n_steps)
                out[(c0, m)] = score(E, F)
            except (ValueError, nat.BsmpsError):
                out[(c0, m)] = -math.inf
    return out


def label(scores):
    best = max(scores, key=lambda k: scores[k])
    return np.array([math.log(best[0]), math.log(best[1])], dtype=np.float32)


def make_dataset(ctx, problems, n_steps=4):
    X, Y, S = [], [], []
    for wl in problems:
        sc = grid_scores(ctx, wl, n_steps)
        X.append(features(wl))
        Y.append(label(sc))
        S.append(sc)
    return np.stack(X), np.stack(Y), S


def init_params(seed=0):
    """He-scaled normal weights, zero biases (float32, flat layout of bsmps_mlp)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(WIDTHS) - 1):
        i, o = WIDTHS[l], WIDTHS[l + 1]
        parts.append(rng.standard_normal(i * o) * np.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def train(ctx, X, Y, steps=400, lr=1e-3, seed=0):
    net = nat.MLP(ctx, WIDTHS, init_params(seed))
    losses = [net.train_step(X, Y, lr) for _ in range(steps)]
    return net, losses


def snap(pred):
    """Nearest grid point to a predicted (log c0, log margin); None if not finite."""
    if not np.all(np.isfinite(pred)):
        return None
    c0 = min(C0_GRID, key=lambda v: abs(math.log(v) - pred[0]))
    m = min(MARGIN_GRID, key=lambda v: abs(math.log(v) - pred[1]))
    return c0, m


def choose(net, wl):
    """Parameters the controller uses for a problem (plain ones when the prediction is unusable)."""
    sel = snap(net.forward(features(wl)[None, :])[0])
    return sel if sel is not None else PLAIN


def solve(ctx, net, wl, n_steps, r_max=64):
    """Alg. 2 steps with the learned parameters; the plain parameters take over
    (from the current iterate's energy scale, restarting from e_1) when a
    learned step raises the Rayleigh quotient or the prediction is unusable.
    Returns (energies, flops, used parameters)."""
    params = choose(net, wl)
    try:
        E, F, _ = run(ctx, wl, params[0], params[1], n_steps, r_max)
    except (ValueError, nat.BsmpsError):
        E, F = [], []
    if len(E) < 2 or any(b > a + 1e-12 * abs(a) for a, b in zip(E, E[1:])) or not all(map(math.isfinite, E)):
        params = PLAIN
        E, F, _ = run(ctx, wl, PLAIN[0], PLAIN[1], n_steps, r_max)
    return E, F, params
