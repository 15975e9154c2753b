// MPS operations on the device (host orchestration of the kernels).
#pragma once

#include <memory>
#include <vector>

#include "common.h"

namespace bsm {

using MpsPtr = std::unique_ptr<Mps>;

void mps_upload(Mps* x, const double* host_flat);
void mps_download(const Mps* x, double* host_flat);

// One term of a block concatenation: x with its sigma=0 / sigma=1 blocks of
// site t scaled by f0[t] / f1[t] (empty vectors: 1).
struct ConcatTerm {
    const Mps* x;
    std::vector<double> f0, f1;
    // optional column mixing x W of a joint block MPS (Sec. 6.1): W is
    // columns(x) x mix_out, row-major; empty: no mixing
    std::vector<double> mix = {};
    int mix_out = 0;
};

// sum_i term_i by block concatenation (Sec. 2.3): union of sectors, inner
// bonds stacked in term order, first core side by side, last core stacked.
// The last bond keeps the common column count of the (mixed) terms.
MpsPtr op_concat(Context* ctx, const std::vector<ConcatTerm>& terms);
MpsPtr op_scale_sites(Context* ctx, const Mps* x, const std::vector<double>& f0,
                      const std::vector<double>& f1);

// y = (H_gamma + shift I) x exactly (Sec. 2.4).
MpsPtr op_apply_exact(Context* ctx, const Mpo& W, const Mps* x, double shift);

// y_i = (H_gamma + shift I) S_i x for site scalings S_i = (f0[i], f1[i]) as in
// ConcatTerm: one layout, one zeroing launch and one copy launch for all i.
// col_shift (joint block MPS, length columns(x)): y_i also gets
// S_i X diag(col_shift), entered on the MPO's identity rail at the last site.
std::vector<MpsPtr> op_apply_exact_scaled(Context* ctx, const Mpo& W, const Mps* x, double shift,
                                          const std::vector<std::vector<double>>& f0,
                                          const std::vector<std::vector<double>>& f1,
                                          const std::vector<double>* col_shift = nullptr);

// u_i = (H_gamma + shift I) S_i x in left-orthogonal form by the zip-up
// application (Sec. 2.4 fused with the QR sweep of Sec. 2.3, csrc/zipup.cpp):
// per site one grouped GEMM for all i (the contraction, profiled as KK_APPLY),
// then per sector Q = I (no more rows than columns) or Householder QR.
std::vector<MpsPtr> op_apply_zipup_scaled(Context* ctx, const Mpo& W, const Mps* x, double shift,
                                          const std::vector<std::vector<double>>& f0,
                                          const std::vector<std::vector<double>>& f1);
// Several independent zip-up applications (different operators, iterates and
// sizes) advanced together: site t of every problem shares the launches of that
// site.  Result j holds the branches of problem j.
struct ZipProblem {
    const Mpo* W;
    const Mps* x;
    double shift;
    std::vector<std::vector<double>> f0, f1;   // per branch (empty inner vector: no scaling)
};
std::vector<std::vector<MpsPtr>> op_apply_zipup_batch(Context* ctx, const std::vector<ZipProblem>& probs);

// trunc_eps of left-orthogonal MPS: the right SVD sweep alone (the left QR
// sweep of a truncation leaves such an MPS as it is, up to the bond gauge).
std::vector<MpsPtr> op_truncate_batch_left_orthogonal(Context* ctx, const std::vector<const Mps*>& xs,
                                                      const std::vector<double>& eps, int r_max);
// Frobenius norms of the last cores (the norms of left-orthogonal MPS), one sync.
std::vector<double> op_last_core_norms(Context* ctx, const std::vector<const Mps*>& xs);

// trunc_eps with rank cap (Sec. 2.2); discarded norms are returned.
MpsPtr op_truncate(Context* ctx, const Mps* x, double eps, int r_max, double* disc_tol,
                   double* disc_cap);

// trunc_eps of several MPS on the same sites, eps[i] for xs[i]; the sweeps of
// all of them share launches.
std::vector<MpsPtr> op_truncate_batch(Context* ctx, const std::vector<const Mps*>& xs,
                                      const std::vector<double>& eps, int r_max);

// Which pooled singular values of one bond survive (Sec. 2.2); entries
// (sigma, sector, j).  Returns kept counts per sector.
struct SvEntry {
    double s;
    int sector, j;
};
std::vector<int> choose_cut(std::vector<SvEntry> sv, int n_sectors, double tol2, int r_max,
                            double* tol_disc2, double* cap_disc2);

// <S_a a, O S_b b> for a batch of problems, O = (H_gamma + shift) or identity.
struct EnvProblem {
    const Mps* a;
    const Mps* b;
    const Mpo* W;               // nullptr: identity
    double shift;
    const std::vector<double>* fa0 = nullptr;   // per-site scalings of a (nullptr: 1)
    const std::vector<double>* fa1 = nullptr;
    const std::vector<double>* fb0 = nullptr;
    const std::vector<double>* fb1 = nullptr;
};
std::vector<double> op_dot_batch(Context* ctx, const std::vector<EnvProblem>& probs);
// The Gram matrices <S_a a_i, O S_b b_j> (columns(a) x columns(b), row-major)
// of joint block MPS, one per problem (Sec. 6.1).
std::vector<std::vector<double>> op_gram_batch(Context* ctx, const std::vector<EnvProblem>& probs);

// <a, O b> with every temporary in a fixed file-scope device array (no allocation).
double op_dot_noalloc(Context* ctx, const Mps* a, const Mps* b, const Mpo* W, double shift);

// Frobenius norm of core 0 (the norm of a right-orthogonalised MPS).
double op_core0_norm(Context* ctx, const Mps* x);

bool same_space(const Layout& a, const Layout& b);

}  // namespace bsm
