// Zip-up application of the Hamiltonian MPO (Sec. 2.4) fused with the
// left-to-right QR sweep of Sec. 2.3: u_i = (H_gamma + shift I) S_i x for a set
// of site scalings S_i, each returned in left-orthogonal form, without forming
// the exact cores (whose bonds are MPO width x rank).
//
// For y = (H + s) S x, the exact bond-t basis of a sector m is the list of
// channel segments (a, n = m - Delta_a) of x's sector dims.  The carry
// C_t[m] (rho_y(m) x rho_exact(m)) maps y's orthogonalised bond basis into it.
// Site t computes, for every block (m, s') of y's core t,
//     T[(m, s')][:, seg_b] = sum_{(a, s): W_t(a, b, s', s) != 0}  w f_s C_t[m][:, seg_a] X_t(n_a, s)
// as one grouped GEMM over all blocks, segments and scalings (the contraction
// stage, whose 2mnk flops are the apply's algorithmic work), then factorises,
// per sector m' of bond t+1, the stack of the blocks (m, s') -> m' (rows in
// layout order): no more rows than columns gives Q = I and C_{t+1}[m'] = the
// stack; otherwise Householder QR (diag R >= 0), Q into y's core t and
// R = C_{t+1}[m'].  The last site's blocks are y's last core.
//
// Several independent problems (different operators, iterates and sizes) run
// together: site t of every problem that has one shares the grouped-GEMM
// launch and the zeroing, gather, QR and scatter launches of that site.
#include <algorithm>
#include <cmath>

#include "kernels.h"
#include "ops.h"

namespace bsm {
namespace {

// One problem of a zip-up batch: its bases, layout, carries and buffers.
struct ZipJob {
    Context* ctx = nullptr;
    const Mpo* W = nullptr;
    const Mps* x = nullptr;
    double shift = 0.0;
    const std::vector<std::vector<double>>* f0 = nullptr;
    const std::vector<std::vector<double>>* f1 = nullptr;
    const double* one = nullptr;
    int K = 0, nb = 0;
    std::vector<Bond> ex;                  // exact bond bases
    std::vector<std::vector<int>> eoff;    // (x sector li, channel a) -> segment offset in its exact sector
    Layout Y;
    std::vector<MpsPtr> ys;
    std::vector<std::vector<const double*>> carry;   // per branch, per sector of Y's bond t
    std::vector<int> carry_ld;
    std::vector<void*> held;               // buffers the carry reads (freed after the next contraction)
    // site state between the contraction and the factorisation
    struct TB {
        int mi, so, em, r0;
    };
    std::vector<TB> tbs;
    std::vector<int> rows;
    std::vector<int64_t> stack_off;
    std::vector<double*> T;

    void init() {
        const Layout& X = x->lay;
        BSM_REQUIRE(W->K == X.K && W->species == X.species, BSMPS_ERR_INVALID_ARG,
                    "MPO and MPS act on different sites");
        BSM_REQUIRE(f0->size() == f1->size() && !f0->empty(), BSMPS_ERR_INVALID_ARG, "scalings mismatch");
        BSM_REQUIRE(X.columns() == 1, BSMPS_ERR_INVALID_ARG, "zip-up application of a single-column MPS");
        K = X.K;
        nb = (int)f0->size();
        const auto valid = valid_sectors(X.species, X.target);
        ex.assign(K + 1, Bond{});
        eoff.assign(K + 1, {});
        for (int b = 0; b <= K; ++b) {
            const int w = W->bond_dim(b), nx = (int)X.bonds[b].q.size();
            eoff[b].assign((size_t)nx * w, -1);
            for (const Charge& m : valid[b]) {
                int tot = 0;
                for (int a = 0; a < w; ++a) {
                    const int li = X.bonds[b].find(m - W->charges[b][a]);
                    if (li < 0) continue;
                    eoff[b][(size_t)li * w + a] = tot;
                    tot += X.bonds[b].dim[li];
                }
                if (tot > 0) {
                    ex[b].q.push_back(m);
                    ex[b].dim.push_back(tot);
                }
            }
        }
        Y.K = K;
        Y.species = X.species;
        Y.target = X.target;
        Y.bonds.assign(K + 1, Bond{});
        Y.bonds[0] = ex[0];
        BSM_REQUIRE(Y.bonds[0].q.size() == 1 && Y.bonds[0].dim[0] == 1, BSMPS_ERR_INVALID_ARG,
                    "bond 0 must have a single sector of dimension 1");
        ys.resize(nb);
        for (int i = 0; i < nb; ++i) {
            ys[i].reset(new Mps);
            ys[i]->ctx = ctx;
            ys[i]->core.assign(K, nullptr);
        }
        carry.assign(nb, std::vector<const double*>(1, one));   // C_0 = [1]
        carry_ld.assign(1, 1);
    }

    // The contraction of site t: allocates the T buffers and appends the outputs.
    void contraction(int t, std::vector<GemmOut>& outs, std::vector<GemmIn>& ins) {
        const Layout& X = x->lay;
        const int sp = X.species[t];
        const int wl = W->bond_dim(t), wr = W->bond_dim(t + 1);
        const Bond& yb = Y.bonds[t];
        const int ny = (int)yb.q.size(), ne = (int)ex[t + 1].q.size();
        std::vector<int> xlook(X.bonds[t].q.size() * 2, -1);   // (li * 2 + sigma) -> block of x's core t
        for (int bi = 0; bi < (int)X.blocks[t].size(); ++bi)
            xlook[X.blocks[t][bi].li * 2 + X.blocks[t][bi].sigma] = bi;
        tbs.clear();
        rows.assign(ne, 0);
        for (int mi = 0; mi < ny; ++mi)
            for (int so = 0; so < 2; ++so) {
                const int em = ex[t + 1].find(yb.q[mi] + site_delta(sp, so));
                if (em < 0) continue;
                tbs.push_back({mi, so, em, rows[em]});
                rows[em] += yb.dim[mi];
            }
        stack_off.assign(ne, 0);
        int64_t tsize = 0;
        for (int em = 0; em < ne; ++em) {
            stack_off[em] = tsize;
            tsize += (int64_t)rows[em] * ex[t + 1].dim[em];
        }
        T.assign(nb, nullptr);
        for (int i = 0; i < nb; ++i) T[i] = tsize > 0 ? (double*)ctx->alloc((size_t)tsize * sizeof(double)) : nullptr;
        // the site's MPO entries by (s', b), in entry order
        std::vector<std::vector<int>> by_sob((size_t)2 * wr);
        for (int ei = 0; ei < (int)W->entries[t].size(); ++ei) {
            const MpoEntry& e = W->entries[t][ei];
            if (e.so >= 0 && e.so < 2 && e.b >= 0 && e.b < wr) by_sob[(size_t)e.so * wr + e.b].push_back(ei);
        }
        for (const TB& tb : tbs) {
            const Charge m = yb.q[tb.mi], m2 = ex[t + 1].q[tb.em];
            const int ldc = ex[t + 1].dim[tb.em];
            // segments b of the exact sector m2: channel b with x sector n_b = m2 - Delta_b
            for (int b = 0; b < wr; ++b) {
                const int rb = X.bonds[t + 1].find(m2 - W->charges[t + 1][b]);
                if (rb < 0) continue;
                const int coff = eoff[t + 1][(size_t)rb * wr + b];
                const int ncols = X.bonds[t + 1].dim[rb];
                for (int i = 0; i < nb; ++i) {
                    GemmOut o{T[i] + stack_off[tb.em] + (int64_t)tb.r0 * ldc + coff, yb.dim[tb.mi], ncols, ldc,
                              (int)ins.size(), (int)ins.size(), 0.0};
                    for (const int ei : by_sob[(size_t)tb.so * wr + b]) {
                        const MpoEntry& e = W->entries[t][ei];
                        const int la = X.bonds[t].find(m - W->charges[t][e.a]);
                        if (la < 0) continue;
                        const int xb = xlook[la * 2 + e.si];
                        if (xb < 0) continue;
                        const Block& bk = X.blocks[t][xb];
                        if (bk.ri != rb) continue;
                        double w = e.w;
                        if (t == 0 && (ei == W->shift_entry[0] || ei == W->shift_entry[1])) w += shift;
                        const std::vector<double>& f = e.si ? (*f1)[i] : (*f0)[i];
                        const double fs = f.empty() ? 1.0 : f[t];
                        const int aoff = eoff[t][(size_t)la * wl + e.a];
                        BSM_REQUIRE(aoff >= 0, BSMPS_ERR_INVALID_ARG, "zip-up: inconsistent bases");
                        ins.push_back({carry[i][tb.mi] + aoff, x->core[t] + bk.off, bk.rows, carry_ld[tb.mi],
                                       bk.cols, 0, w * fs});
                    }
                    o.end = (int)ins.size();
                    outs.push_back(o);
                }
            }
        }
    }

    // After the contraction launch: the previous carry's buffers are free.
    void release_held() {
        for (void* p : held) ctx->free(p);
        held.clear();
    }

    // The factorisation of site t (appended to the site's shared launches), or
    // at the last site the T buffers become the last core.
    void factor(int t, std::vector<double*>& zp, std::vector<int64_t>& zn, std::vector<CopyTask>& gather,
                std::vector<QrTask>& qr, std::vector<CopyTask>& scatter) {
        if (t == K - 1) {
            Y.bonds[K] = ex[K];
            for (int i = 0; i < nb; ++i) ys[i]->core[t] = T[i];
            return;
        }
        const Bond& yb = Y.bonds[t];
        const int ne = (int)ex[t + 1].q.size();
        // new bond t+1: k = min(stacked rows, exact columns) per exact sector
        Bond nbnd;
        std::vector<int> newidx(ne, -1);
        for (int em = 0; em < ne; ++em) {
            if (rows[em] == 0) continue;
            newidx[em] = (int)nbnd.q.size();
            nbnd.q.push_back(ex[t + 1].q[em]);
            nbnd.dim.push_back(std::min(rows[em], ex[t + 1].dim[em]));
        }
        // the blocks of core t, (mi, s') -> (yb.dim[mi] x k(m')), in layout order (= tbs order)
        int64_t csize = 0;
        std::vector<int64_t> boff(tbs.size(), 0);
        for (size_t q = 0; q < tbs.size(); ++q) {
            boff[q] = csize;
            csize += (int64_t)yb.dim[tbs[q].mi] * nbnd.dim[newidx[tbs[q].em]];
        }
        std::vector<double*> core(nb, nullptr);
        for (int i = 0; i < nb; ++i) {
            core[i] = csize > 0 ? (double*)ctx->alloc((size_t)csize * sizeof(double)) : nullptr;
            if (core[i]) {
                zp.push_back(core[i]);
                zn.push_back(csize);
            }
        }
        std::vector<std::vector<const double*>> ncarry(nb, std::vector<const double*>(nbnd.q.size(), nullptr));
        std::vector<int> ncarry_ld(nbnd.q.size(), 1);
        for (int em = 0; em < ne; ++em) {
            const int ni = newidx[em];
            if (ni < 0) continue;
            const int M = rows[em], N = ex[t + 1].dim[em], k = nbnd.dim[ni];
            ncarry_ld[ni] = N;
            for (int i = 0; i < nb; ++i) {
                if (M <= N) {
                    // Q = I: the identity rows of each block, the stack itself is the carry
                    ncarry[i][ni] = T[i] + stack_off[em];
                    for (size_t q = 0; q < tbs.size(); ++q)
                        if (tbs[q].em == em)
                            scatter.push_back({one, core[i] + boff[q] + tbs[q].r0, yb.dim[tbs[q].mi], 1, 0, k + 1, 0,
                                               0, 0, 1.0});
                } else {
                    double* A = (double*)ctx->alloc((size_t)M * N * sizeof(double));
                    double* Q = (double*)ctx->alloc((size_t)M * k * sizeof(double));
                    double* R = (double*)ctx->alloc((size_t)k * N * sizeof(double));
                    double* tau = (double*)ctx->alloc((size_t)k * sizeof(double));
                    gather.push_back({T[i] + stack_off[em], A, M, N, N, M, 0, 1, 0, 1.0});
                    qr.push_back({A, Q, R, tau, M, N});
                    for (size_t q = 0; q < tbs.size(); ++q)
                        if (tbs[q].em == em)
                            scatter.push_back({Q + tbs[q].r0, core[i] + boff[q], yb.dim[tbs[q].mi], k, M, k, 1, 0, 0,
                                               1.0});
                    ncarry[i][ni] = R;
                    // A, Q, tau and R are released one site later (stream order keeps
                    // them alive for the launches of this site)
                    held.push_back(A);
                    held.push_back(Q);
                    held.push_back(tau);
                    held.push_back(R);
                }
            }
        }
        for (int i = 0; i < nb; ++i) {
            ys[i]->core[t] = core[i];
            if (T[i]) held.push_back(T[i]);
        }
        Y.bonds[t + 1] = nbnd;
        carry.swap(ncarry);
        carry_ld.swap(ncarry_ld);
    }

    std::vector<MpsPtr> finish() {
        release_held();
        Y.rebuild_blocks();
        for (int i = 0; i < nb; ++i) ys[i]->lay = Y;
        return std::move(ys);
    }
};

}  // namespace

std::vector<std::vector<MpsPtr>> op_apply_zipup_batch(Context* ctx, const std::vector<ZipProblem>& probs) {
    std::vector<std::vector<MpsPtr>> out(probs.size());
    if (probs.empty()) return out;
    double* one = (double*)ctx->upload(std::vector<double>{1.0});
    std::vector<ZipJob> jobs(probs.size());
    int kmax = 0;
    try {
        for (size_t j = 0; j < probs.size(); ++j) {
            ZipJob& J = jobs[j];
            J.ctx = ctx;
            J.W = probs[j].W;
            J.x = probs[j].x;
            J.shift = probs[j].shift;
            J.f0 = &probs[j].f0;
            J.f1 = &probs[j].f1;
            J.one = one;
            J.init();
            kmax = std::max(kmax, J.K);
        }
        for (int t = 0; t < kmax; ++t) {
            std::vector<GemmOut> outs;
            std::vector<GemmIn> ins;
            for (ZipJob& J : jobs)
                if (t < J.K) J.contraction(t, outs, ins);
            launch_gemm(ctx, outs, ins, KK_APPLY);
            for (ZipJob& J : jobs)
                if (t < J.K) J.release_held();
            std::vector<double*> zp;
            std::vector<int64_t> zn;
            std::vector<CopyTask> gather, scatter;
            std::vector<QrTask> qr;
            for (ZipJob& J : jobs)
                if (t < J.K) J.factor(t, zp, zn, gather, qr, scatter);
            launch_zero(ctx, zp, zn, KK_APPLY_QR);
            launch_copy(ctx, gather, KK_APPLY_QR);
            launch_qr(ctx, qr, KK_APPLY_QR);
            launch_copy(ctx, scatter, KK_APPLY_QR);
        }
    } catch (...) {
        for (ZipJob& J : jobs) J.release_held();
        ctx->free(one);
        throw;
    }
    for (size_t j = 0; j < jobs.size(); ++j) out[j] = jobs[j].finish();
    ctx->free(one);
    return out;
}

std::vector<MpsPtr> op_apply_zipup_scaled(Context* ctx, const Mpo& W, const Mps* x, double shift,
                                          const std::vector<std::vector<double>>& f0,
                                          const std::vector<std::vector<double>>& f1) {
    std::vector<ZipProblem> p{{&W, x, shift, f0, f1}};
    return std::move(op_apply_zipup_batch(ctx, p)[0]);
}

}  // namespace bsm
