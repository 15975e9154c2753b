// Preconditioner terms and the Alg. 2 step.
#pragma once

#include <tuple>
#include <vector>

#include "ops.h"

namespace bsm {

constexpr int kMaxEtaRetries = 60;
// Relative error estimate of the residual terms computed with split-precision
// (3xTF32) contractions, against sum_j ||s_j||: the per-entry bound of a few
// units of 2^-21 of the summed magnitudes, with room for cancellation.
constexpr double kSplitRel = 1.0 / 262144.0;   // 2^-18

struct PrecondTerms {
    double h = 0.0;
    int m_minus = 0, m_plus = 0;
    std::vector<std::vector<double>> f0, f1;   // per term, per site
    int n_terms() const { return (int)f0.size(); }
};

PrecondTerms make_precond(const bsmps_precond* p);

// One residual term s_{k,k'} = S_k u_k' with its norm (Sec. 5.3.1).
struct ResTerm {
    double norm;
    int k, kp;
};
// res_eta for the candidate tolerances etas (consecutive passes of the eta_res
// loop), computed together: the sequential truncated sums of all candidates
// advance term by term, the truncations of one term sharing one batch.  Each
// candidate runs exactly the operations of its own pass.  terms: ascending by
// (norm, k, k').  Entry c is null when candidate c keeps no term.
std::vector<MpsPtr> residual_candidates(Context* ctx, const PrecondTerms& P, const std::vector<MpsPtr>& u,
                                        const std::vector<ResTerm>& terms, const std::vector<double>& etas);
// Width of the first batch of candidates after a step that needed last_tries
// extra passes, and of later batches.
int first_batch_width(int last_tries);
constexpr int kCandidateBatch = 8;
std::vector<double> pair_sums(Context* ctx, const PrecondTerms& P,
                              const std::vector<std::tuple<const Mps*, const Mps*, const Mpo*>>& jobs);
double eigvec_bound(double rho, double delta);
double releig_bound(double rho, double delta);
void rr2(const double H[2][2], const double E[2][2], double* mu, double v[2]);
double delta_A(double rho, double q);
MpsPtr eigensolve_step(Context* ctx, const Mpo& W, const PrecondTerms& P, const bsmps_solver_params& prm,
                       bsmps_solver_state& st, const Mps* x, bsmps_step_info& info);
// Gram-matrix pair sums of joint block MPS (row-major columns(a) x columns(b)).
std::vector<std::vector<double>> gram_pair_sums(
    Context* ctx, const PrecondTerms& P, const std::vector<std::tuple<const Mps*, const Mps*, const Mpo*>>& jobs);
// Alg. 4, one step on a joint iterate.
MpsPtr eigensolve_joint_step(Context* ctx, const Mpo& W, const PrecondTerms& P, const bsmps_solver_params& prm,
                             bsmps_solver_state& st, const Mps* X, bsmps_joint_step_info& info);
// Alg. 3; records: one per outer step taken.
MpsPtr eigensolve_outer(Context* ctx, const Mpo& W, const PrecondTerms& P, const bsmps_solver_params& prm,
                        double alpha, double tau, int max_outer, int max_inner, const Mps* y0,
                        std::vector<bsmps_outer_record>& records, bool* converged);

}  // namespace bsm
