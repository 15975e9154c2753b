#include <limits>
// Exponential-sum preconditioner (Sec. 4) and one step of the perturbed
// preconditioned inverse iteration (Alg. 2), orchestrated on the host over
// device MPS operations.
#include "solver.h"

#include <algorithm>
#include <cmath>

namespace bsm {

// h, M^-, M^+ of Eq. (expsumparams); alpha_m, beta_m of Sec. 4.3 with
// beta_m = e^{mh}/t_min (obtained by substituting Eq. (expsum) into Eq. (Sdef)).
PrecondTerms make_precond(const bsmps_precond* p) {
    BSM_REQUIRE(p && p->d && p->K > 0, BSMPS_ERR_INVALID_ARG, "precond: K > 0 and d required");
    BSM_REQUIRE(p->t_min > 0.0 && p->t_max >= p->t_min, BSMPS_ERR_NOT_SPD,
                "precond: need 0 < t_min <= t_max");
    BSM_REQUIRE(p->c0 > 0.0 && p->c0 < 1.0 && p->alpha0 > 0.0, BSMPS_ERR_INVALID_ARG,
                "precond: need c0 in (0,1) and alpha0 > 0");
    PrecondTerms P;
    const double pi = 3.14159265358979323846;
    P.h = pi * pi / std::log(8.0 * std::sqrt(2.0) / p->c0 + 1.0);
    const double lg = std::fabs(std::log(std::sqrt(pi) * p->c0 / 4.0));
    P.m_plus = (int)std::ceil(std::log(lg) / P.h);
    P.m_minus = -(int)std::ceil((2.0 * lg + std::log(p->t_max / p->t_min)) / P.h);
    const int K = p->K;
    for (int m = P.m_minus; m <= P.m_plus; ++m) {
        const double alpha = P.h * p->alpha0 / std::sqrt(pi) * std::exp(m * P.h / 2.0);
        const double beta = std::exp(m * P.h) / p->t_min;
        const double a = std::pow(alpha, 1.0 / K);
        std::vector<double> f0(K, a), f1(K);
        for (int i = 0; i < K; ++i) f1[i] = a * std::exp(-beta * p->d[i]);
        P.f0.push_back(f0);
        P.f1.push_back(f1);
    }
    return P;
}

// sum_{k,k'} <O S_k a, S_k' b> for several (a, b, O) at once (Eq. (exactrq)).
// sum_{k,k'} <S_k a, O S_k' b> per job (Eq. (exactrq)).  O is symmetric, so
// for a == b the (k, k') and (k', k) terms are equal: only k <= k' is
// computed and the off-diagonal terms count twice.
std::vector<double> pair_sums(Context* ctx, const PrecondTerms& P,
                              const std::vector<std::tuple<const Mps*, const Mps*, const Mpo*>>& jobs) {
    const int nt = P.n_terms();
    std::vector<EnvProblem> probs;
    std::vector<std::pair<int, double>> weight;   // (job, multiplicity) per problem
    for (size_t j = 0; j < jobs.size(); ++j) {
        const bool same = std::get<0>(jobs[j]) == std::get<1>(jobs[j]);
        for (int k = 0; k < nt; ++k)
            for (int kp = same ? k : 0; kp < nt; ++kp) {
                EnvProblem pr{std::get<0>(jobs[j]), std::get<1>(jobs[j]), std::get<2>(jobs[j]), 0.0};
                pr.fa0 = &P.f0[k];
                pr.fa1 = &P.f1[k];
                pr.fb0 = &P.f0[kp];
                pr.fb1 = &P.f1[kp];
                probs.push_back(pr);
                weight.push_back({(int)j, same && kp != k ? 2.0 : 1.0});
            }
    }
    const std::vector<double> v = op_dot_batch(ctx, probs);
    std::vector<double> out(jobs.size(), 0.0);
    for (size_t q = 0; q < v.size(); ++q) out[weight[q].first] += weight[q].second * v[q];
    return out;
}

static double bdelta(double rho, double delta, bool* ok) {
    const double disc = 1.0 - 4.0 * (delta - 1.0) * delta * rho * rho;
    if (disc < 0.0) {
        *ok = false;
        return 0.0;
    }
    *ok = true;
    return 2.0 * delta / (1.0 + 2.0 * delta * rho * rho + std::sqrt(disc));
}

// Thm. aposterbound: 2 sin(1/2 arcsin(sqrt(delta b_delta) rho)); +inf if invalid.
double eigvec_bound(double rho, double delta) {
    bool ok;
    const double b = bdelta(rho, delta, &ok);
    if (!ok) return INFINITY;
    const double arg = std::sqrt(delta * b) * rho;
    if (arg > 1.0) return INFINITY;
    return 2.0 * std::sin(0.5 * std::asin(arg));
}

// Eq. (releigerr); +inf if invalid.
double releig_bound(double rho, double delta) {
    bool ok;
    const double b = bdelta(rho, delta, &ok);
    if (!ok || b * rho * rho >= 1.0) return INFINITY;
    return b / (1.0 - b * rho * rho) * rho * rho;
}

// Lower eigenpair of the symmetric 2x2 pencil (H, E), E positive definite:
// roots of det(H - mu E) = 0 by the cancellation-free quadratic formula, the
// eigenvector from the better-conditioned row of (H - mu E), scaled to
// v^T E v = 1 with v_1 > 0.
void rr2(const double H[2][2], const double E[2][2], double* mu, double v[2]) {
    const double a = E[0][0] * E[1][1] - E[0][1] * E[0][1];
    const double b = -(H[0][0] * E[1][1] + H[1][1] * E[0][0] - 2.0 * H[0][1] * E[0][1]);
    const double c = H[0][0] * H[1][1] - H[0][1] * H[0][1];
    const double disc = std::max(b * b - 4.0 * a * c, 0.0);
    const double q = -0.5 * (b + (b >= 0.0 ? 1.0 : -1.0) * std::sqrt(disc));
    double r1 = q / a, r2 = q != 0.0 ? c / q : r1;
    const double lo = std::min(r1, r2);
    *mu = lo;
    const double m00 = H[0][0] - lo * E[0][0], m01 = H[0][1] - lo * E[0][1], m11 = H[1][1] - lo * E[1][1];
    double x0, x1;
    if (std::fabs(m00) + std::fabs(m01) >= std::fabs(m01) + std::fabs(m11)) {
        x0 = -m01;
        x1 = m00;
    } else {
        x0 = m11;
        x1 = -m01;
    }
    if (x0 == 0.0 && x1 == 0.0) {   // H = mu E: any vector; take e_1
        x0 = 1.0;
        x1 = 0.0;
    }
    const double nrm = std::sqrt(x0 * x0 * E[0][0] + 2.0 * x0 * x1 * E[0][1] + x1 * x1 * E[1][1]);
    x0 /= nrm;
    x1 /= nrm;
    if (x0 < 0.0) {
        x0 = -x0;
        x1 = -x1;
    }
    v[0] = x0;
    v[1] = x1;
}

double delta_A(double rho, double q) {
    const double disc = std::max(1.0 + rho * rho - q * q, 0.0);
    return std::max((-q * rho + std::sqrt(disc)) / (1.0 + rho * rho), 0.0);
}

static void check_finite(double v, const char* what) {
    BSM_REQUIRE(std::isfinite(v), BSMPS_ERR_NUMERIC, std::string("non-finite ") + what);
}

int first_batch_width(int last_tries) { return std::max(1, std::min(kCandidateBatch, last_tries + 1)); }

std::vector<MpsPtr> residual_candidates(Context* ctx, const PrecondTerms& P, const std::vector<MpsPtr>& u,
                                        const std::vector<ResTerm>& terms, const std::vector<double>& etas) {
    const int C = (int)etas.size();
    std::vector<size_t> j0(C, 0);
    std::vector<double> tail(C, 0.0);
    size_t jmin = terms.size();
    for (int c = 0; c < C; ++c) {
        // drop the smallest terms while their norms sum to at most eta/3
        double acc = 0.0;
        while (j0[c] < terms.size() && acc + terms[j0[c]].norm <= etas[c] / 3.0) {
            acc += terms[j0[c]].norm;
            j0[c]++;
        }
        for (size_t j = j0[c]; j < terms.size(); ++j) tail[c] += terms[j].norm;
        jmin = std::min(jmin, j0[c]);
    }
    std::vector<MpsPtr> y(C);
    for (size_t j = jmin; j < terms.size(); ++j) {
        const ResTerm& tm = terms[j];
        std::vector<MpsPtr> z;
        std::vector<const Mps*> zs;
        std::vector<double> eps;
        std::vector<int> who;
        for (int c = 0; c < C; ++c) {
            if (j < j0[c]) continue;
            // y_j = trunc_{eps_j}(y_{j-1} + s_j), eps_j = eta ||s_j|| / (3 sum_{i > J_0} ||s_i||)
            if (!y[c])
                z.push_back(op_scale_sites(ctx, u[tm.kp].get(), P.f0[tm.k], P.f1[tm.k]));
            else
                z.push_back(op_concat(ctx, {{y[c].get(), {}, {}}, {u[tm.kp].get(), P.f0[tm.k], P.f1[tm.k]}}));
            zs.push_back(z.back().get());
            eps.push_back(tail[c] > 0.0 ? etas[c] * tm.norm / (3.0 * tail[c]) : 0.0);
            who.push_back(c);
        }
        std::vector<MpsPtr> t = op_truncate_batch(ctx, zs, eps, 0);
        for (size_t i = 0; i < who.size(); ++i) y[who[i]] = std::move(t[i]);
    }
    // final trunc_{eta/3}
    std::vector<const Mps*> ys;
    std::vector<double> eps;
    std::vector<int> who;
    for (int c = 0; c < C; ++c)
        if (y[c]) {
            ys.push_back(y[c].get());
            eps.push_back(etas[c] / 3.0);
            who.push_back(c);
        }
    std::vector<MpsPtr> out(C);
    std::vector<MpsPtr> t = op_truncate_batch(ctx, ys, eps, 0);
    for (size_t i = 0; i < who.size(); ++i) out[who[i]] = std::move(t[i]);
    return out;
}

MpsPtr eigensolve_step(Context* ctx, const Mpo& W, const PrecondTerms& P, const bsmps_solver_params& prm,
                       bsmps_solver_state& st, const Mps* x_in, bsmps_step_info& info) {
    const double flops0 = ctx->flops;
    const int nt = P.n_terms();
    info = bsmps_step_info{};
    info.precision = BSMPS_PREC_FP64;
    // lambda^n and ||x||_A^2 (Eq. (exactrq))
    const auto ps = pair_sums(ctx, P, {{x_in, x_in, &W}, {x_in, x_in, nullptr}});
    const double num = ps[0], den = ps[1];
    check_finite(num, "Rayleigh numerator");
    BSM_REQUIRE(num > 0.0 && den > 0.0, BSMPS_ERR_NUMERIC, "iterate has zero A-norm");
    const double lam = num / den;
    // x^n / ||x^n||_A
    std::vector<double> s0(x_in->lay.K, 1.0), s1(x_in->lay.K, 1.0);
    s0[0] = s1[0] = 1.0 / std::sqrt(num);
    MpsPtr x = op_scale_sites(ctx, x_in, s0, s1);
    // residual terms: u_k' = (H_gamma - lambda) S_k' x, s_{k,k'} = S_k u_k'.
    // Split-precision contractions while their error estimate, kSplitRel sum_j ||s_j||
    // of the previous step, stays below a tenth of the previous eta_res (the
    // residual error budget of Lemma truncr); FP64 from then on.
    const int prec_saved = ctx->apply_precision;
    bool split = prec_saved != BSMPS_PREC_FP64 && !st.fp64_locked;
    if (split && std::isfinite(st.eta_res) && kSplitRel * st.last_sum_norms > 0.1 * st.eta_res) {
        split = false;
        st.fp64_locked = 1;
    }
    info.precision = split ? prec_saved : BSMPS_PREC_FP64;
    ctx->apply_precision = info.precision;
    std::vector<MpsPtr> u;
    if (prm.u_rel > 0.0) {
        // zip-up application (left-orthogonal u_k', norm in the last core), then one
        // near-lossless compression per term: the right sweep of trunc at u_rel ||u||
        u = op_apply_zipup_scaled(ctx, W, x.get(), -lam, P.f0, P.f1);
        std::vector<const Mps*> ux;
        for (int kp = 0; kp < nt; ++kp) ux.push_back(u[kp].get());
        const std::vector<double> un = op_last_core_norms(ctx, ux);
        std::vector<double> ueps;
        for (int kp = 0; kp < nt; ++kp) ueps.push_back(prm.u_rel * un[kp]);
        std::vector<MpsPtr> uc = op_truncate_batch_left_orthogonal(ctx, ux, ueps, 0);
        for (int kp = 0; kp < nt; ++kp) u[kp] = std::move(uc[kp]);
    } else {
        u = op_apply_exact_scaled(ctx, W, x.get(), -lam, P.f0, P.f1);   // exactly applied terms
    }
    ctx->apply_precision = prec_saved;
    std::vector<EnvProblem> nprobs;
    for (int kp = 0; kp < nt; ++kp)
        for (int k = 0; k < nt; ++k) {
            EnvProblem pr{u[kp].get(), u[kp].get(), nullptr, 0.0};
            pr.fa0 = pr.fb0 = &P.f0[k];
            pr.fa1 = pr.fb1 = &P.f1[k];
            nprobs.push_back(pr);
        }
    const std::vector<double> n2 = op_dot_batch(ctx, nprobs);
    std::vector<ResTerm> terms;
    double sum_norms = 0.0;
    for (int kp = 0; kp < nt; ++kp)
        for (int k = 0; k < nt; ++k) {
            const double nv = std::sqrt(std::max(n2[kp * nt + k], 0.0));
            terms.push_back({nv, k, kp});
            sum_norms += nv;
        }
    std::sort(terms.begin(), terms.end(), [](const ResTerm& a, const ResTerm& b) {
        if (a.norm != b.norm) return a.norm < b.norm;
        if (a.k != b.k) return a.k < b.k;
        return a.kp < b.kp;
    });
    const double zeta = prm.eps_num / (1.0 + prm.c);
    double eta = std::min(2.0 * st.eta_res, 0.8 * zeta * sum_norms);
    // the eta_res loop: pass t uses eta * 0.8^t and is accepted when
    // ||res_eta|| >= (1 + 1/zeta) eta or t reaches the cap; passes are
    // evaluated in batches of candidates
    int tries = 0;
    MpsPtr r;
    double rnorm = 0.0;
    int width = first_batch_width(st.last_tries);
    for (bool done = false; !done;) {
        std::vector<double> etas;
        double e = eta;
        for (int c = 0; c < width && tries + c <= kMaxEtaRetries; ++c) {
            etas.push_back(e);
            e *= 0.8;
        }
        std::vector<MpsPtr> Rs = residual_candidates(ctx, P, u, terms, etas);
        for (size_t c = 0; c < etas.size(); ++c) {
            const double rn = Rs[c] ? op_core0_norm(ctx, Rs[c].get()) : 0.0;
            if (rn >= (1.0 + 1.0 / zeta) * etas[c] || tries >= kMaxEtaRetries) {
                eta = etas[c];
                r = std::move(Rs[c]);
                rnorm = rn;
                done = true;
                break;
            }
            tries++;
        }
        if (!done) eta = e;
        width = kCandidateBatch;
    }
    st.last_tries = tries;
    st.eta_res = eta;
    st.last_sum_norms = sum_norms;
    const double rho = (rnorm + eta) / std::sqrt(1.0 - prm.c);
    check_finite(rho, "rho");
    info.lambda = lam;
    info.rho = rho;
    info.eta_res = eta;
    info.res_norm = rnorm;
    info.eta_tries = tries;
    info.bound = eigvec_bound(rho, prm.delta);
    info.releig_bound = releig_bound(rho, prm.delta);
    if (info.bound <= prm.tau || !r) {
        info.converged = 1;
        int mr = 0;
        for (auto& b : x->lay.bonds) mr = std::max(mr, b.total());
        info.max_rank = mr;
        info.flops = ctx->flops - flops0;
        return x;
    }
    // 2x2 Rayleigh-Ritz in the normalised basis (Remark omegamin)
    // the Gram matrices are symmetric (H_gamma and the S_k are): <x, r> entries once
    const auto g = pair_sums(ctx, P, {{x.get(), x.get(), &W}, {x.get(), r.get(), &W}, {r.get(), r.get(), &W},
                                      {x.get(), x.get(), nullptr}, {x.get(), r.get(), nullptr},
                                      {r.get(), r.get(), nullptr}});
    const double GH[2][2] = {{g[0], g[1]}, {g[1], g[2]}};
    const double GE[2][2] = {{g[3], g[4]}, {g[4], g[5]}};
    const double nrm[2] = {std::sqrt(GE[0][0]), std::sqrt(GE[1][1])};
    double Hn[2][2], En[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            Hn[i][j] = GH[i][j] / (nrm[i] * nrm[j]);
            En[i][j] = GE[i][j] / (nrm[i] * nrm[j]);
        }
    // symmetrise the (numerically) symmetric Gram entries
    Hn[0][1] = Hn[1][0] = 0.5 * (Hn[0][1] + Hn[1][0]);
    En[0][1] = En[1][0] = 0.5 * (En[0][1] + En[1][0]);
    double lam_star, v[2];
    rr2(Hn, En, &lam_star, v);
    check_finite(lam_star, "Ritz value");
    const double c1 = v[0] / nrm[0], c2 = v[1] / nrm[1];
    // x* = c1 x + c2 r: the scalars scale the first core of each part (Sec. 2.3)
    std::vector<double> a0(x->lay.K, 1.0), b0(x->lay.K, 1.0);
    a0[0] = c1;
    b0[0] = c2;
    MpsPtr xstar = op_concat(ctx, {{x.get(), a0, a0}, {r.get(), b0, b0}});
    const double xstar_A = std::sqrt(std::max(lam_star, 0.0));
    const double q = std::sqrt(lam_star / (lam_star + prm.t_eig * (lam - lam_star)));
    const double dA = delta_A(rho, q);
    const double eta_in = dA * xstar_A / std::sqrt(1.0 + prm.c);
    double cap_disc = 0.0;
    MpsPtr xn = op_truncate(ctx, xstar.get(), eta_in, prm.r_max, nullptr, &cap_disc);
    info.cap_discarded = cap_disc;
    info.lambda_star = lam_star;
    info.omega = -c2 / c1;
    info.eta_in = eta_in;
    info.delta_A = dA;
    int mr = 0;
    for (auto& b : xn->lay.bonds) mr = std::max(mr, b.total());
    info.max_rank = mr;
    info.flops = ctx->flops - flops0;
    st.n += 1;
    return xn;
}

static int max_bond(const Mps* x) {
    int mr = 0;
    for (const Bond& b : x->lay.bonds) mr = std::max(mr, b.total());
    return mr;
}

// Outer perturbed inverse iteration (Alg. 3, D = 1): inner Alg. 2 runs to the
// eigenvector tolerance tau_m, the termination test of Eq. (releigerr), and the
// rank-controlling truncation trunc_{theta eta_m} with eta halved per step
// (kappa of Eq. (kappadef), theta and tau_m of Thm. quasioptr).
MpsPtr eigensolve_outer(Context* ctx, const Mpo& W, const PrecondTerms& P, const bsmps_solver_params& prm,
                        double alpha, double tau, int max_outer, int max_inner, const Mps* y0,
                        std::vector<bsmps_outer_record>& records, bool* converged) {
    const int K = y0->lay.K;
    const double kappa = std::sqrt((1.0 + prm.c) / (1.0 - prm.c)) * std::sqrt((double)std::max(K - 1, 1));
    const double theta = (1.0 + alpha) * kappa / (2.0 * (1.0 + (1.0 + alpha) * kappa));
    double eta = 1.0 / (2.0 * theta);
    *converged = false;
    records.clear();
    MpsPtr y;
    const Mps* cur = y0;
    for (int m = 0; m < max_outer; ++m) {
        const double tau_m = eta / (2.0 * (1.0 + (1.0 + alpha) * kappa));
        bsmps_solver_params inner = prm;
        inner.tau = tau_m;
        bsmps_solver_state st{std::numeric_limits<double>::infinity(), 0, 0, 0.0, 0};
        bsmps_outer_record rec{};
        const double fl0 = ctx->flops;
        bsmps_step_info info{};
        for (int n = 0; n < max_inner; ++n) {
            MpsPtr nx = eigensolve_step(ctx, W, P, inner, st, cur, info);
            y = std::move(nx);
            cur = y.get();
            rec.inner_steps = n + 1;
            if (info.converged) break;
        }
        BSM_REQUIRE(rec.inner_steps > 0, BSMPS_ERR_INVALID_ARG, "max_inner must be positive");
        rec.inner_converged = info.converged;
        rec.lambda = info.lambda;
        rec.rho = info.rho;
        rec.releig_bound = info.releig_bound;
        rec.eta_out = eta;
        rec.tau_m = tau_m;
        rec.max_rank_before = max_bond(cur);
        if (info.releig_bound < tau) {
            rec.max_rank_after = rec.max_rank_before;
            rec.flops = ctx->flops - fl0;
            records.push_back(rec);
            *converged = true;
            return y;
        }
        y = op_truncate(ctx, cur, theta * eta, 0, nullptr, nullptr);
        cur = y.get();
        rec.max_rank_after = max_bond(cur);
        rec.flops = ctx->flops - fl0;
        records.push_back(rec);
        eta *= 0.5;
    }
    return y;
}

}  // namespace bsm
