// Perturbed inverse subspace iteration on joint block MPS (Alg. 4, Sec. 6),
// orchestrated on the host over device MPS operations.
//
// X = (x_1, ..., x_D) is one block MPS whose last bond (the target sector) is
// D wide: the eigenvector-specific core of Sec. 6.2 sits after the last site.
// Gram matrices X^T O Y are then the last left environment of one inner-product
// sweep, and column mixing X V multiplies the last core.
#include <algorithm>
#include <cmath>
#include <limits>

#include "solver.h"

namespace bsm {

// sum_{k,k'} (S_k a)^T O (S_k' b) per job, each a columns(a) x columns(b)
// matrix (Sec. 6.1, summation formulas).  O is symmetric, so for a == b the
// (k', k) term is the transpose of the (k, k') term: only k <= k' is computed.
std::vector<std::vector<double>> gram_pair_sums(
    Context* ctx, const PrecondTerms& P, const std::vector<std::tuple<const Mps*, const Mps*, const Mpo*>>& jobs) {
    const int nt = P.n_terms();
    std::vector<EnvProblem> probs;
    std::vector<std::pair<int, int>> tag;   // (job, 1 if the transpose is added too)
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
                tag.push_back({(int)j, same && kp != k ? 1 : 0});
            }
    }
    const std::vector<std::vector<double>> g = op_gram_batch(ctx, probs);
    std::vector<std::vector<double>> out(jobs.size());
    for (size_t j = 0; j < jobs.size(); ++j)
        out[j].assign((size_t)std::get<0>(jobs[j])->lay.columns() * std::get<1>(jobs[j])->lay.columns(), 0.0);
    for (size_t q = 0; q < g.size(); ++q) {
        const int j = tag[q].first;
        const int na = std::get<0>(jobs[j])->lay.columns(), nb = std::get<1>(jobs[j])->lay.columns();
        for (int r = 0; r < na; ++r)
            for (int c = 0; c < nb; ++c) {
                out[j][(size_t)r * nb + c] += g[q][(size_t)r * nb + c];
                if (tag[q].second) out[j][(size_t)r * nb + c] += g[q][(size_t)c * nb + r];
            }
    }
    return out;
}

namespace {

using Mat = std::vector<double>;   // row-major n x n

// Eigenpairs of the symmetric n x n matrix C by cyclic Jacobi rotations
// (Golub & Van Loan, Alg. 8.5.3); eigenvectors are the columns of V.
void sym_eig(int n, Mat C, std::vector<double>& w, Mat& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                const double v = C[(size_t)p * n + q] * C[(size_t)p * n + q];
                tot += v;
                if (p != q) off += v;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = C[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = C[(size_t)p * n + p], aqq = C[(size_t)q * n + q];
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {   // C <- C J
                    const double ckp = C[(size_t)k * n + p], ckq = C[(size_t)k * n + q];
                    C[(size_t)k * n + p] = c * ckp - s * ckq;
                    C[(size_t)k * n + q] = s * ckp + c * ckq;
                }
                for (int k = 0; k < n; ++k) {   // C <- J^T C
                    const double cpk = C[(size_t)p * n + k], cqk = C[(size_t)q * n + k];
                    C[(size_t)p * n + k] = c * cpk - s * cqk;
                    C[(size_t)q * n + k] = s * cpk + c * cqk;
                }
                for (int k = 0; k < n; ++k) {   // V <- V J
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = C[(size_t)i * n + i];
}

// Lowest m eigenpairs of the symmetric-definite pencil (A, B) (n x n): B = L L^T
// (Cholesky), eigenpairs of L^{-1} A L^{-T}, V = L^{-T} Y, so V^T B V = I and
// V^T A V = diag(w); then the columns are scaled by w^{-1/2} (V^T A V = I) and
// the largest-|.| entry of each is made positive.  Returns V as n x m row-major.
void ritz(int n, const Mat& A, const Mat& B, int m, std::vector<double>& w_out, Mat& V_out) {
    Mat L((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = B[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        BSM_REQUIRE(d > 0.0 && std::isfinite(d), BSMPS_ERR_NUMERIC,
                    "Rayleigh-Ritz: the Gram matrix of the subspace basis is not positive definite");
        L[(size_t)j * n + j] = std::sqrt(d);
        for (int i = j + 1; i < n; ++i) {
            double v = B[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = v / L[(size_t)j * n + j];
        }
    }
    // C = L^{-1} A L^{-T}: solve L Z = A, then C^T = L^{-1} Z^T (C symmetric)
    Mat Z = A;
    for (int c = 0; c < n; ++c)
        for (int i = 0; i < n; ++i) {
            double v = Z[(size_t)i * n + c];
            for (int k = 0; k < i; ++k) v -= L[(size_t)i * n + k] * Z[(size_t)k * n + c];
            Z[(size_t)i * n + c] = v / L[(size_t)i * n + i];
        }
    Mat C((size_t)n * n);
    for (int r = 0; r < n; ++r)   // row r of C = (L^{-1} (row r of Z)^T)^T
        for (int i = 0; i < n; ++i) {
            double v = Z[(size_t)r * n + i];
            for (int k = 0; k < i; ++k) v -= L[(size_t)i * n + k] * C[(size_t)r * n + k];
            C[(size_t)r * n + i] = v / L[(size_t)i * n + i];
        }
    for (int r = 0; r < n; ++r)
        for (int c = r + 1; c < n; ++c) {
            const double v = 0.5 * (C[(size_t)r * n + c] + C[(size_t)c * n + r]);
            C[(size_t)r * n + c] = C[(size_t)c * n + r] = v;
        }
    std::vector<double> w;
    Mat Y;
    sym_eig(n, C, w, Y);
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return w[a] != w[b] ? w[a] < w[b] : a < b; });
    w_out.resize(m);
    V_out.assign((size_t)n * m, 0.0);
    for (int c = 0; c < m; ++c) {
        const int e = ord[c];
        w_out[c] = w[e];
        BSM_REQUIRE(w[e] > 0.0 && std::isfinite(w[e]), BSMPS_ERR_NUMERIC, "Ritz value is not positive");
        // v = L^{-T} y (back substitution with L^T)
        std::vector<double> v(n);
        for (int i = n - 1; i >= 0; --i) {
            double s = Y[(size_t)i * n + e];
            for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * v[k];
            v[i] = s / L[(size_t)i * n + i];
        }
        int jmax = 0;
        for (int i = 1; i < n; ++i)
            if (std::fabs(v[i]) > std::fabs(v[jmax])) jmax = i;
        const double sg = v[jmax] < 0.0 ? -1.0 : 1.0;
        const double sc = sg / std::sqrt(w[e]);
        for (int i = 0; i < n; ++i) V_out[(size_t)i * m + c] = v[i] * sc;
    }
}

void check_finite(double v, const char* what) {
    BSM_REQUIRE(std::isfinite(v), BSMPS_ERR_NUMERIC, std::string("non-finite ") + what);
}

double frob_from_gram(const std::vector<double>& g, int n) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += g[(size_t)i * n + i];
    return std::sqrt(std::max(t, 0.0));
}

}  // namespace

MpsPtr eigensolve_joint_step(Context* ctx, const Mpo& W, const PrecondTerms& P, const bsmps_solver_params& prm,
                             bsmps_solver_state& st, const Mps* X_in, bsmps_joint_step_info& info) {
    const double flops0 = ctx->flops;
    const int nt = P.n_terms();
    const int D = X_in->lay.columns();
    BSM_REQUIRE(D >= 1 && D <= BSMPS_MAX_COLUMNS, BSMPS_ERR_INVALID_ARG, "1 <= columns <= BSMPS_MAX_COLUMNS");
    info = bsmps_joint_step_info{};
    info.D = D;
    // Rayleigh--Ritz on span X^n: A-orthonormal columns, Lambda^n
    const auto g0 = gram_pair_sums(ctx, P, {{X_in, X_in, &W}, {X_in, X_in, nullptr}});
    std::vector<double> lam;
    Mat V;
    ritz(D, g0[0], g0[1], D, lam, V);
    MpsPtr X = op_concat(ctx, {ConcatTerm{X_in, {}, {}, V, D}});
    // residual terms u_k' = H_gamma S_k' X - S_k' X Lambda (Eq. (respara)), one exact apply each
    std::vector<double> neg(D);
    for (int i = 0; i < D; ++i) neg[i] = -lam[i];
    std::vector<MpsPtr> u = op_apply_exact_scaled(ctx, W, X.get(), 0.0, P.f0, P.f1, &neg);
    if (prm.u_rel > 0.0) {
        std::vector<EnvProblem> up;
        for (int kp = 0; kp < nt; ++kp) up.push_back({u[kp].get(), u[kp].get(), nullptr, 0.0});
        const auto ug = op_gram_batch(ctx, up);
        std::vector<const Mps*> ux;
        std::vector<double> ueps;
        for (int kp = 0; kp < nt; ++kp) {
            ux.push_back(u[kp].get());
            ueps.push_back(prm.u_rel * frob_from_gram(ug[kp], D));
        }
        std::vector<MpsPtr> uc = op_truncate_batch(ctx, ux, ueps, 0);
        for (int kp = 0; kp < nt; ++kp) u[kp] = std::move(uc[kp]);
    }
    // term norms ||S_k u_k'||_F
    std::vector<EnvProblem> nprobs;
    for (int kp = 0; kp < nt; ++kp)
        for (int k = 0; k < nt; ++k) {
            EnvProblem pr{u[kp].get(), u[kp].get(), nullptr, 0.0};
            pr.fa0 = pr.fb0 = &P.f0[k];
            pr.fa1 = pr.fb1 = &P.f1[k];
            nprobs.push_back(pr);
        }
    const auto n2 = op_gram_batch(ctx, nprobs);
    std::vector<ResTerm> terms;
    double sum_norms = 0.0;
    for (int kp = 0; kp < nt; ++kp)
        for (int k = 0; k < nt; ++k) {
            const double nv = frob_from_gram(n2[kp * nt + k], D);
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
    // the eta_res loop of Alg. 4 (pass t: eta * 0.8^t, accepted when
    // min_i ||r_i|| >= (1 + 1/zeta) eta or t reaches the cap), in batches of
    // candidate passes
    int tries = 0;
    MpsPtr R;
    std::vector<double> rn(D, 0.0);
    int width = first_batch_width(st.last_tries);
    for (bool done = false; !done;) {
        std::vector<double> etas;
        double e = eta;
        for (int c = 0; c < width && tries + c <= kMaxEtaRetries; ++c) {
            etas.push_back(e);
            e *= 0.8;
        }
        std::vector<MpsPtr> Rs = residual_candidates(ctx, P, u, terms, etas);
        std::vector<EnvProblem> gp;
        for (auto& Rc : Rs)
            if (Rc) gp.push_back({Rc.get(), Rc.get(), nullptr, 0.0});
        const auto rg = op_gram_batch(ctx, gp);
        size_t gi = 0;
        for (size_t c = 0; c < etas.size(); ++c) {
            std::vector<double> cn(D, 0.0);
            double rmin = 0.0;
            if (Rs[c]) {
                rmin = std::numeric_limits<double>::infinity();
                for (int i = 0; i < D; ++i) {
                    cn[i] = std::sqrt(std::max(rg[gi][(size_t)i * D + i], 0.0));
                    rmin = std::min(rmin, cn[i]);
                }
                gi++;
            }
            if (rmin >= (1.0 + 1.0 / zeta) * etas[c] || tries >= kMaxEtaRetries) {
                eta = etas[c];
                R = std::move(Rs[c]);
                rn = cn;
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
    std::vector<double> rho(D);
    for (int i = 0; i < D; ++i) {
        rho[i] = (rn[i] + eta) / std::sqrt(1.0 - prm.c);   // ||x_i||_A = 1
        check_finite(rho[i], "rho");
        info.lambda[i] = lam[i];
        info.rho[i] = rho[i];
        info.res_norm[i] = rn[i];
    }
    info.eta_res = eta;
    info.eta_tries = tries;
    info.bound = eigvec_bound(rho[0], prm.delta);
    info.releig_bound = releig_bound(rho[0], prm.delta);
    auto max_rank = [](const Mps* m) {
        int mr = 0;
        for (const Bond& b : m->lay.bonds) mr = std::max(mr, b.total());
        return mr;
    };
    if (info.bound <= prm.tau || !R) {
        info.converged = 1;
        info.max_rank = max_rank(X.get());
        info.flops = ctx->flops - flops0;
        return X;
    }
    // Rayleigh--Ritz on span (X^n R^n) in the normalised basis (Sec. 6.1)
    const auto g = gram_pair_sums(ctx, P, {{X.get(), X.get(), &W}, {X.get(), R.get(), &W}, {R.get(), R.get(), &W},
                                           {X.get(), X.get(), nullptr}, {X.get(), R.get(), nullptr},
                                           {R.get(), R.get(), nullptr}});
    const int n2d = 2 * D;
    Mat GA((size_t)n2d * n2d), GE((size_t)n2d * n2d);
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            GA[(size_t)i * n2d + j] = g[0][(size_t)i * D + j];
            GA[(size_t)i * n2d + D + j] = g[1][(size_t)i * D + j];
            GA[(size_t)(D + j) * n2d + i] = g[1][(size_t)i * D + j];
            GA[(size_t)(D + i) * n2d + D + j] = g[2][(size_t)i * D + j];
            GE[(size_t)i * n2d + j] = g[3][(size_t)i * D + j];
            GE[(size_t)i * n2d + D + j] = g[4][(size_t)i * D + j];
            GE[(size_t)(D + j) * n2d + i] = g[4][(size_t)i * D + j];
            GE[(size_t)(D + i) * n2d + D + j] = g[5][(size_t)i * D + j];
        }
    std::vector<double> xi(n2d);
    for (int i = 0; i < n2d; ++i) {
        xi[i] = std::sqrt(GE[(size_t)i * n2d + i]);
        check_finite(xi[i], "column norm");
    }
    Mat Bm((size_t)n2d * n2d), Mm((size_t)n2d * n2d);
    for (int i = 0; i < n2d; ++i)
        for (int j = 0; j < n2d; ++j) {
            Bm[(size_t)i * n2d + j] = GA[(size_t)i * n2d + j] / (xi[i] * xi[j]);
            Mm[(size_t)i * n2d + j] = GE[(size_t)i * n2d + j] / (xi[i] * xi[j]);
        }
    for (int i = 0; i < n2d; ++i)
        for (int j = i + 1; j < n2d; ++j) {
            const double b = 0.5 * (Bm[(size_t)i * n2d + j] + Bm[(size_t)j * n2d + i]);
            const double m = 0.5 * (Mm[(size_t)i * n2d + j] + Mm[(size_t)j * n2d + i]);
            Bm[(size_t)i * n2d + j] = Bm[(size_t)j * n2d + i] = b;
            Mm[(size_t)i * n2d + j] = Mm[(size_t)j * n2d + i] = m;
        }
    std::vector<double> lam_star;
    Mat Wm;
    ritz(n2d, Bm, Mm, D, lam_star, Wm);
    // X* = X Xi_x^{-1} W_1 + R Xi_r^{-1} W_2 (A-orthonormal columns)
    std::vector<double> W1((size_t)D * D), W2((size_t)D * D);
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            W1[(size_t)i * D + j] = Wm[(size_t)i * D + j] / xi[i];
            W2[(size_t)i * D + j] = Wm[(size_t)(D + i) * D + j] / xi[D + i];
        }
    MpsPtr Xstar = op_concat(ctx, {ConcatTerm{X.get(), {}, {}, W1, D}, ConcatTerm{R.get(), {}, {}, W2, D}});
    double dmin = std::numeric_limits<double>::infinity();
    for (int i = 0; i < D; ++i) {
        const double q = std::sqrt(lam_star[i] / (lam_star[i] + prm.t_eig * (lam[i] - lam_star[i])));
        info.lambda_star[i] = lam_star[i];
        info.delta_A[i] = delta_A(rho[i], q);
        dmin = std::min(dmin, info.delta_A[i]);
    }
    const double eta_in = dmin / std::sqrt(1.0 + prm.c);   // ||X*_i||_A = 1
    check_finite(eta_in, "eta_in");
    double cap_disc = 0.0;
    MpsPtr Xn = op_truncate(ctx, Xstar.get(), eta_in, prm.r_max, nullptr, &cap_disc);
    info.eta_in = eta_in;
    info.cap_discarded = cap_disc;
    info.max_rank = max_rank(Xn.get());
    info.flops = ctx->flops - flops0;
    st.n += 1;
    return Xn;
}

}  // namespace bsm
