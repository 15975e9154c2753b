// Host orchestration of the block-sparse MPS operations (Sec. 2.2-2.4).
#include "ops.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <tuple>

#include "kernels.h"

namespace bsm {

Mps::~Mps() {
    if (ctx && owns_cores)
        for (double* p : core)
            if (p) ctx->free(p);
}

Mps* new_mps(Context* ctx, const Layout& L, bool zero) {
    MpsPtr x(new Mps);
    x->ctx = ctx;
    x->lay = L;
    x->core.assign(L.K, nullptr);
    std::vector<double*> zp;
    std::vector<int64_t> zn;
    for (int t = 0; t < L.K; ++t) {
        const int64_t n = L.core_size[t];
        if (n > 0) {
            x->core[t] = (double*)ctx->alloc((size_t)n * sizeof(double));
            zp.push_back(x->core[t]);
            zn.push_back(n);
        }
    }
    if (zero) launch_zero(ctx, zp, zn);   // every core in one launch
    return x.release();
}

static MpsPtr make_mps(Context* ctx, const Layout& L, bool zero) { return MpsPtr(new_mps(ctx, L, zero)); }

void mps_upload(Mps* x, const double* host) {
    int64_t off = 0;
    for (int t = 0; t < x->lay.K; ++t) {
        const int64_t n = x->lay.core_size[t];
        if (n > 0)
            BSM_CUDA(cudaMemcpyAsync(x->core[t], host + off, (size_t)n * sizeof(double),
                                     cudaMemcpyHostToDevice, x->ctx->stream));
        off += n;
    }
    x->ctx->sync();
}

void mps_download(const Mps* x, double* host) {
    int64_t off = 0;
    for (int t = 0; t < x->lay.K; ++t) {
        const int64_t n = x->lay.core_size[t];
        if (n > 0)
            BSM_CUDA(cudaMemcpyAsync(host + off, x->core[t], (size_t)n * sizeof(double),
                                     cudaMemcpyDeviceToHost, x->ctx->stream));
        off += n;
    }
    x->ctx->sync();
}

bool same_space(const Layout& a, const Layout& b) {
    return a.K == b.K && a.species == b.species && a.target == b.target;
}

// per-site lookup (left sector index, sigma) -> block index
static std::vector<int> block_lookup(const Layout& L, int t) {
    std::vector<int> idx(L.bonds[t].q.size() * 2, -1);
    for (int i = 0; i < (int)L.blocks[t].size(); ++i)
        idx[L.blocks[t][i].li * 2 + L.blocks[t][i].sigma] = i;
    return idx;
}

static void rebuild_site(Layout& L, int t) {
    L.blocks[t].clear();
    int64_t off = 0;
    const Bond& bl = L.bonds[t];
    const Bond& br = L.bonds[t + 1];
    for (int li = 0; li < (int)bl.q.size(); ++li)
        for (int sg = 0; sg < 2; ++sg) {
            const int ri = br.find(bl.q[li] + site_delta(L.species[t], sg));
            if (ri < 0) continue;
            Block bk{li, ri, sg, bl.dim[li], br.dim[ri], off};
            off += (int64_t)bk.rows * bk.cols;
            L.blocks[t].push_back(bk);
        }
    L.core_size[t] = off;
}

MpsPtr op_concat(Context* ctx, const std::vector<ConcatTerm>& terms) {
    BSM_REQUIRE(!terms.empty(), BSMPS_ERR_INVALID_ARG, "concat of nothing");
    const Layout& L0 = terms[0].x->lay;
    for (auto& tm : terms)
        BSM_REQUIRE(same_space(tm.x->lay, L0), BSMPS_ERR_INVALID_ARG,
                    "MPS of different sites or particle numbers");
    const int K = L0.K;
    int D = -1;   // columns of the result
    for (auto& tm : terms) {
        const int din = tm.x->lay.columns();
        int dout = din;
        if (!tm.mix.empty()) {
            BSM_REQUIRE(tm.mix_out > 0 && (int64_t)tm.mix.size() == (int64_t)din * tm.mix_out && K > 1,
                        BSMPS_ERR_INVALID_ARG, "mixing matrix must be columns x mix_out (K > 1)");
            dout = tm.mix_out;
        }
        BSM_REQUIRE(D < 0 || D == dout, BSMPS_ERR_INVALID_ARG, "terms with different column counts");
        D = dout;
    }
    Layout R;
    R.K = K;
    R.species = L0.species;
    R.target = L0.target;
    R.bonds.resize(K + 1);
    // offsets[i][b][sector of R]
    std::vector<std::vector<std::vector<int>>> offs(terms.size(), std::vector<std::vector<int>>(K + 1));
    for (int b = 0; b <= K; ++b) {
        std::vector<Charge> qs;
        for (auto& tm : terms)
            for (auto& q : tm.x->lay.bonds[b].q) qs.push_back(q);
        std::sort(qs.begin(), qs.end());
        qs.erase(std::unique(qs.begin(), qs.end()), qs.end());
        R.bonds[b].q = qs;
        R.bonds[b].dim.assign(qs.size(), 0);
        for (size_t i = 0; i < terms.size(); ++i) offs[i][b].assign(qs.size(), 0);
        for (size_t s = 0; s < qs.size(); ++s) {
            int acc = 0;
            for (size_t i = 0; i < terms.size(); ++i) {
                offs[i][b][s] = (b == 0 || b == K) ? 0 : acc;
                const int j = terms[i].x->lay.bonds[b].find(qs[s]);
                if (j >= 0) acc += terms[i].x->lay.bonds[b].dim[j];
            }
            R.bonds[b].dim[s] = b == 0 ? 1 : (b == K ? D : acc);
        }
    }
    R.rebuild_blocks();
    MpsPtr y = make_mps(ctx, R, true);
    std::vector<std::vector<CopyTask>> per_term(terms.size());
    std::vector<std::vector<int>> looks(K);
    for (int t = 0; t < K; ++t) looks[t] = block_lookup(R, t);
    // mixed terms: their last-site blocks are products X_block W (one GEMM output each)
    Scratch sm(ctx);
    std::vector<GemmOut> gouts;
    std::vector<GemmIn> gins;
    for (size_t i = 0; i < terms.size(); ++i) {
        const Mps* x = terms[i].x;
        const double* dmix = terms[i].mix.empty() ? nullptr : sm.up(terms[i].mix);
        for (int t = 0; t < K; ++t) {
            const std::vector<int>& look = looks[t];
            for (const Block& bk : x->lay.blocks[t]) {
                const int li = R.bonds[t].find(x->lay.bonds[t].q[bk.li]);
                const int ri = R.bonds[t + 1].find(x->lay.bonds[t + 1].q[bk.ri]);
                const Block& rb = R.blocks[t][look[li * 2 + bk.sigma]];
                const int r0 = offs[i][t][li], c0 = offs[i][t + 1][ri];
                double f = 1.0;
                const std::vector<double>& fv = bk.sigma ? terms[i].f1 : terms[i].f0;
                if (!fv.empty()) f = fv[t];
                double* dst = y->core[t] + rb.off + (int64_t)r0 * rb.cols + c0;
                if (dmix && t == K - 1) {
                    gouts.push_back({dst, bk.rows, rb.cols, rb.cols, (int)gins.size(), (int)gins.size() + 1, 0.0});
                    gins.push_back({x->core[t] + bk.off, dmix, bk.cols, bk.cols, rb.cols, 0, f});
                    continue;
                }
                CopyTask ct{x->core[t] + bk.off, dst, bk.rows, bk.cols, bk.cols, rb.cols, 0, 0, K == 1 ? 1 : 0, f};
                per_term[i].push_back(ct);
            }
        }
    }
    launch_gemm(ctx, gouts, gins);
    if (K == 1) {
        for (auto& v : per_term) launch_copy(ctx, v);   // same destination: one launch per term
    } else {
        std::vector<CopyTask> all;
        for (auto& v : per_term) all.insert(all.end(), v.begin(), v.end());
        launch_copy(ctx, all);
    }
    return y;
}

MpsPtr op_scale_sites(Context* ctx, const Mps* x, const std::vector<double>& f0,
                      const std::vector<double>& f1) {
    MpsPtr y = make_mps(ctx, x->lay, false);
    std::vector<CopyTask> tasks;
    for (int t = 0; t < x->lay.K; ++t)
        for (const Block& bk : x->lay.blocks[t]) {
            const double f = bk.sigma ? (f1.empty() ? 1.0 : f1[t]) : (f0.empty() ? 1.0 : f0[t]);
            tasks.push_back({x->core[t] + bk.off, y->core[t] + bk.off, bk.rows, bk.cols, bk.cols,
                             bk.cols, 0, 0, 0, f});
        }
    launch_copy(ctx, tasks);
    return y;
}

std::vector<MpsPtr> op_apply_exact_scaled(Context* ctx, const Mpo& W, const Mps* x, double shift,
                                          const std::vector<std::vector<double>>& f0,
                                          const std::vector<std::vector<double>>& f1,
                                          const std::vector<double>* col_shift) {
    const Layout& X = x->lay;
    BSM_REQUIRE(W.K == X.K && W.species == X.species, BSMPS_ERR_INVALID_ARG,
                "MPO and MPS act on different sites");
    BSM_REQUIRE(f0.size() == f1.size() && !f0.empty(), BSMPS_ERR_INVALID_ARG, "scalings mismatch");
    const int K = X.K;
    const int n = (int)f0.size();
    const auto valid = valid_sectors(X.species, X.target);
    Layout Y;
    Y.K = K;
    Y.species = X.species;
    Y.target = X.target;
    Y.bonds.resize(K + 1);
    // For bond b, X sector li and channel a: the output sector holding the
    // product (-1: none) and the row offset of channel a's segment in it.
    std::vector<std::vector<int>> ysec(K + 1), yoff(K + 1);
    for (int b = 0; b <= K; ++b) {
        const int w = W.bond_dim(b);
        const int nx = (int)X.bonds[b].q.size();
        ysec[b].assign((size_t)nx * w, -1);
        yoff[b].assign((size_t)nx * w, -1);
        for (const Charge& m : valid[b]) {
            const int ml = (int)Y.bonds[b].q.size();
            int tot = 0;
            for (int a = 0; a < w; ++a) {
                const int li = X.bonds[b].find(m - W.charges[b][a]);
                if (li < 0) continue;
                ysec[b][(size_t)li * w + a] = ml;
                yoff[b][(size_t)li * w + a] = tot;
                tot += X.bonds[b].dim[li];
            }
            if (tot > 0) {
                Y.bonds[b].q.push_back(m);
                Y.bonds[b].dim.push_back(tot);
            }
        }
    }
    Y.rebuild_blocks();
    // every output zeroed in one launch, then every piece of every output in one copy launch
    std::vector<MpsPtr> ys;
    std::vector<double*> zp;
    std::vector<int64_t> zn;
    for (int i = 0; i < n; ++i) {
        ys.push_back(make_mps(ctx, Y, false));
        for (int t = 0; t < K; ++t)
            if (Y.core_size[t] > 0) {
                zp.push_back(ys[i]->core[t]);
                zn.push_back(Y.core_size[t]);
            }
    }
    launch_zero(ctx, zp, zn);
    std::vector<CopyTask> tasks;
    double fl = 0.0;
    const int ncol = X.columns();
    if (col_shift) {
        BSM_REQUIRE((int)col_shift->size() == ncol && W.ident_last >= 0 && W.bond_dim(K) == 1,
                    BSMPS_ERR_INVALID_ARG, "one column shift per column and an MPO with an identity rail");
    }
    for (int t = 0; t < K; ++t) {
        const std::vector<int> look = block_lookup(Y, t);
        const int wl = W.bond_dim(t), wr = W.bond_dim(t + 1);
        const auto& ents = W.entries[t];
        const bool rail = col_shift && t == K - 1;   // the (I -> F, s, s) sub-blocks get the column shifts
        for (const Block& bk : X.blocks[t]) {
            bool rail_done = false;
            auto emit = [&](int so, int a, int b, double w, bool on_rail) {
                const size_t il = (size_t)bk.li * wl + a, ir = (size_t)bk.ri * wr + b;
                const int ml = ysec[t][il], mr = ysec[t + 1][ir];
                if (ml < 0 || mr < 0) return;
                const int yb = look[ml * 2 + so];
                if (yb < 0) return;
                const Block& yk = Y.blocks[t][yb];
                const int64_t dst = yk.off + (int64_t)yoff[t][il] * yk.cols + yoff[t + 1][ir];
                for (int i = 0; i < n; ++i) {
                    const std::vector<double>& f = bk.sigma ? f1[i] : f0[i];
                    const double fs = f.empty() ? 1.0 : f[t];
                    if (!on_rail) {
                        tasks.push_back({x->core[t] + bk.off, ys[i]->core[t] + dst, bk.rows, bk.cols, bk.cols,
                                         yk.cols, 0, 0, 0, w * fs});
                    } else {
                        // one task per column j: weight (w + col_shift[j])
                        for (int j = 0; j < bk.cols; ++j)
                            tasks.push_back({x->core[t] + bk.off + j, ys[i]->core[t] + dst + j, bk.rows, 1,
                                             bk.cols, yk.cols, 0, 0, 0, (w + (*col_shift)[j]) * fs});
                    }
                }
                fl += 2.0 * n * bk.rows * bk.cols;
            };
            for (int ei = 0; ei < (int)ents.size(); ++ei) {
                const MpoEntry& e = ents[ei];
                if (bk.sigma != e.si) continue;
                double w = e.w;
                if (t == 0 && (ei == W.shift_entry[0] || ei == W.shift_entry[1])) w += shift;
                const bool on_rail = rail && e.a == W.ident_last && e.b == 0 && e.so == e.si;
                rail_done = rail_done || on_rail;
                emit(e.so, e.a, e.b, w, on_rail);
            }
            if (rail && !rail_done) emit(bk.sigma, W.ident_last, 0, 0.0, true);
        }
    }
    ctx->flops += fl;
    launch_copy(ctx, tasks);
    return ys;
}

MpsPtr op_apply_exact(Context* ctx, const Mpo& W, const Mps* x, double shift) {
    const std::vector<std::vector<double>> none(1);   // one output, unscaled
    std::vector<MpsPtr> ys = op_apply_exact_scaled(ctx, W, x, shift, none, none);
    return std::move(ys[0]);
}

std::vector<int> choose_cut(std::vector<SvEntry> sv, int n_sectors, double tol2, int r_max,
                            double* tol_disc2, double* cap_disc2) {
    std::sort(sv.begin(), sv.end(), [](const SvEntry& a, const SvEntry& b) {
        if (a.s != b.s) return a.s > b.s;
        if (a.sector != b.sector) return a.sector < b.sector;
        return a.j < b.j;
    });
    const double rtol = 1e-10;
    const int n = (int)sv.size();
    int keep = n;
    double acc = 0.0;
    while (keep > 0) {
        const double s = sv[keep - 1].s;
        if (acc + s * s <= tol2) {
            acc += s * s;
            keep -= 1;
        } else {
            break;
        }
    }
    while (keep > 0 && keep < n && sv[keep].s >= sv[keep - 1].s * (1.0 - rtol)) keep += 1;
    double td = 0.0;   // discarded squares, summed from the smallest
    for (int i = n - 1; i >= keep; --i) td += sv[i].s * sv[i].s;
    double cd = 0.0;
    if (r_max > 0 && keep > r_max) {
        int k2 = r_max;
        while (k2 > 0 && sv[k2].s >= sv[k2 - 1].s * (1.0 - rtol)) k2 -= 1;
        if (k2 == 0) k2 = r_max;
        for (int i = k2; i < keep; ++i) cd += sv[i].s * sv[i].s;
        keep = k2;
    }
    *tol_disc2 += td;
    *cap_disc2 += cd;
    std::vector<int> cnt(n_sectors, 0);
    for (int i = 0; i < keep; ++i) cnt[sv[i].sector]++;
    return cnt;
}

namespace {

// One truncation in flight: the sweeps update its layout and cores in place.
// Cores it owns (allocated by a sweep) are freed on destruction unless they
// were handed to the result.
struct TruncJob {
    Context* ctx;
    Layout L;
    std::vector<double*> cores;
    std::vector<char> owned;
    double eps;
    int r_max;
    double td2 = 0.0, cd2 = 0.0;
    TruncJob(Context* c, const Mps* x, double e, int r)
        : ctx(c), L(x->lay), cores(x->core), owned(x->lay.K, 0), eps(e), r_max(r) {}
    TruncJob(const TruncJob&) = delete;
    TruncJob& operator=(const TruncJob&) = delete;
    ~TruncJob() {
        for (size_t t = 0; t < cores.size(); ++t)
            if (owned[t] && cores[t]) ctx->free(cores[t]);
    }
    void release(int t) {
        if (owned[t] && cores[t]) ctx->free(cores[t]);
        cores[t] = nullptr;
        owned[t] = 0;
    }
    double* alloc_core(int64_t n) { return n > 0 ? (double*)ctx->alloc((size_t)n * sizeof(double)) : nullptr; }
    MpsPtr finish() {
        const int K = L.K;
        MpsPtr y(new Mps);
        y->ctx = ctx;
        y->lay = L;
        y->core.assign(K, nullptr);
        for (int t = 0; t < K; ++t) {
            if (owned[t]) {
                y->core[t] = cores[t];
            } else if (L.core_size[t] > 0) {   // untouched core (K == 1): copy
                y->core[t] = alloc_core(L.core_size[t]);
                BSM_CUDA(cudaMemcpyAsync(y->core[t], cores[t], (size_t)L.core_size[t] * sizeof(double),
                                         cudaMemcpyDeviceToDevice, ctx->stream));
            }
            owned[t] = 0;
        }
        return y;
    }
};

// ---- left-to-right QR sweep, one launch per site ----
void left_sweep_sitewise(Context* ctx, TruncJob& J) {
    const int K = J.L.K;
    Layout& L = J.L;
    std::vector<double*>& cores = J.cores;
    std::vector<char>& owned = J.owned;
    auto release = [&](int t) { J.release(t); };
    auto alloc_core = [&](int64_t n) { return J.alloc_core(n); };
    for (int t = 0; t + 1 < K; ++t) {
        Scratch s(ctx);
        const Bond bm = L.bonds[t + 1];   // the old bond (L is updated in place below)
        const int nm = (int)bm.q.size();
        std::vector<int> Mrows(nm, 0), krank(nm, 0);
        std::vector<std::vector<std::pair<int, int>>> stack(nm);   // (block index, row offset)
        for (int bi = 0; bi < (int)L.blocks[t].size(); ++bi) {
            const Block& bk = L.blocks[t][bi];
            stack[bk.ri].push_back({bi, Mrows[bk.ri]});
            Mrows[bk.ri] += bk.rows;
        }
        const std::vector<int> oldlook = block_lookup(L, t + 1);
        const std::vector<Block> oldB_t = L.blocks[t], oldB_t1 = L.blocks[t + 1];
        {
            Bond nb;
            for (int mi = 0; mi < nm; ++mi) {
                if (Mrows[mi] > 0) krank[mi] = std::min(Mrows[mi], bm.dim[mi]);
                if (krank[mi] > 0) {
                    nb.q.push_back(bm.q[mi]);
                    nb.dim.push_back(krank[mi]);
                }
            }
            L.bonds[t + 1] = nb;
            rebuild_site(L, t);
            rebuild_site(L, t + 1);
        }
        double* nt = alloc_core(L.core_size[t]);
        double* nt1 = alloc_core(L.core_size[t + 1]);
        const std::vector<int> newlook_t = block_lookup(L, t);
        // fused path: one CTA per sector does gather, QR, Q scatter and R X
        bool fused = true;
        for (int mi = 0; mi < nm && fused; ++mi) {
            if (Mrows[mi] == 0) continue;
            int64_t rx = 0;
            for (int sg = 0; sg < 2; ++sg) {
                const int ob = oldlook[mi * 2 + sg];
                if (ob >= 0) rx += (int64_t)krank[mi] * bm.dim[mi] * oldB_t1[ob].cols;
            }
            fused = left_site_fits(Mrows[mi], bm.dim[mi], rx);
        }
        if (fused) {
            std::vector<LeftTask> lt;
            std::vector<LeftSrc> ls;
            std::vector<LeftX> lx;
            for (int mi = 0; mi < nm; ++mi) {
                if (Mrows[mi] == 0) continue;
                const int nmi = L.bonds[t + 1].find(bm.q[mi]);
                LeftTask task{Mrows[mi], bm.dim[mi], krank[mi], (int)ls.size(), 0, (int)lx.size(), 0};
                for (auto& pr : stack[mi]) {
                    const Block& ob = oldB_t[pr.first];
                    const Block& nbk = L.blocks[t][newlook_t[ob.li * 2 + ob.sigma]];
                    ls.push_back({cores[t] + ob.off, nt + nbk.off, ob.rows, pr.second});
                }
                task.s_end = (int)ls.size();
                for (const Block& nbk : L.blocks[t + 1]) {
                    if (nbk.li != nmi) continue;
                    const Block& ob = oldB_t1[oldlook[mi * 2 + nbk.sigma]];
                    lx.push_back({cores[t + 1] + ob.off, nt1 + nbk.off, ob.cols});
                }
                task.x_end = (int)lx.size();
                lt.push_back(task);
            }
            launch_left_site(ctx, lt, ls, lx);
        } else {
            std::vector<double*> Am(nm, nullptr), Qm(nm, nullptr), Rm(nm, nullptr);
            std::vector<CopyTask> gather;
            std::vector<QrTask> qr;
            for (int mi = 0; mi < nm; ++mi) {
                const int M = Mrows[mi], N = bm.dim[mi];
                if (M == 0) continue;
                const int k = krank[mi];
                Am[mi] = s.dbl((size_t)M * N);
                Qm[mi] = s.dbl((size_t)M * k);
                Rm[mi] = s.dbl((size_t)k * N);
                double* tau = s.dbl((size_t)k);
                for (auto& pr : stack[mi]) {
                    const Block& bk = oldB_t[pr.first];
                    gather.push_back({cores[t] + bk.off, Am[mi] + pr.second, bk.rows, bk.cols, bk.cols, M,
                                      0, 1, 0, 1.0});
                }
                qr.push_back({Am[mi], Qm[mi], Rm[mi], tau, M, N});
            }
            launch_copy(ctx, gather);
            launch_qr(ctx, qr);
            std::vector<CopyTask> qcopy;
            for (const Block& nbk : L.blocks[t]) {
                const int mi = bm.find(L.bonds[t + 1].q[nbk.ri]);
                int r0 = -1;
                for (auto& pr : stack[mi]) {
                    const Block& ob = oldB_t[pr.first];
                    if (ob.li == nbk.li && ob.sigma == nbk.sigma) r0 = pr.second;
                }
                qcopy.push_back({Qm[mi] + r0, nt + nbk.off, nbk.rows, nbk.cols, Mrows[mi], nbk.cols, 1, 0, 0,
                                 1.0});
            }
            launch_copy(ctx, qcopy);
            std::vector<GemmOut> outs;
            std::vector<GemmIn> ins;
            for (const Block& nbk : L.blocks[t + 1]) {
                const int mi = bm.find(L.bonds[t + 1].q[nbk.li]);
                const Block& ob = oldB_t1[oldlook[mi * 2 + nbk.sigma]];
                outs.push_back({nt1 + nbk.off, nbk.rows, nbk.cols, nbk.cols, (int)ins.size(),
                                (int)ins.size() + 1, 0.0});
                ins.push_back({Rm[mi], cores[t + 1] + ob.off, ob.rows, bm.dim[mi], ob.cols, 0, 1.0});
            }
            launch_gemm(ctx, outs, ins);
        }
        release(t);
        release(t + 1);
        cores[t] = nt;
        owned[t] = 1;
        cores[t + 1] = nt1;
        owned[t + 1] = 1;
    }

}

// ---- right-to-left SVD sweep, one launch per site and a host cut ----
void right_sweep_sitewise(Context* ctx, TruncJob& J) {
    const int K = J.L.K;
    Layout& L = J.L;
    std::vector<double*>& cores = J.cores;
    std::vector<char>& owned = J.owned;
    const int r_max = J.r_max;
    double& td2 = J.td2;
    double& cd2 = J.cd2;
    auto release = [&](int t) { J.release(t); };
    auto alloc_core = [&](int64_t n) { return J.alloc_core(n); };
    const double tol2 = K > 1 ? J.eps * J.eps / (K - 1) : 0.0;
    for (int t = K - 1; t >= 1; --t) {
        Scratch s(ctx);
        const Bond bn = L.bonds[t];   // the old bond (L is updated in place below)
        const int nn = (int)bn.q.size();
        std::vector<int> c0(nn, 0), c1(nn, 0), b0(nn, -1), b1(nn, -1), kk(nn, 0);
        for (int bi = 0; bi < (int)L.blocks[t].size(); ++bi) {
            const Block& bk = L.blocks[t][bi];
            if (bk.sigma == 0) {
                c0[bk.li] = bk.cols;
                b0[bk.li] = bi;
            } else {
                c1[bk.li] = bk.cols;
                b1[bk.li] = bi;
            }
        }
        std::vector<double*> US(nn, nullptr), Vt(nn, nullptr);
        std::vector<int64_t> soff(nn, 0);
        int64_t stot = 0;
        for (int ni = 0; ni < nn; ++ni) {
            const int M = bn.dim[ni], N = c0[ni] + c1[ni];
            kk[ni] = N > 0 ? std::min(M, N) : 0;
            soff[ni] = stot;
            stot += kk[ni];
        }
        double* S_all = s.dbl((size_t)std::max<int64_t>(stot, 1));
        // sectors of this bond: small ones in the fused one-CTA kernel, the others
        // (k >= kClusterJacobiMin, or too large for it) by QR + Jacobi on clusters
        std::vector<int> site_sec, gen_sec;
        for (int ni = 0; ni < nn; ++ni) {
            if (kk[ni] == 0) continue;
            if (kk[ni] < kClusterJacobiMin && svd_site_fits(bn.dim[ni], c0[ni] + c1[ni]))
                site_sec.push_back(ni);
            else
                gen_sec.push_back(ni);
        }
        // the one-CTA sector SVDs overlap the cluster chain of the wide sectors
        // on the context's second stream (joined before the singular values
        // are read; their buffers live in s until the end of the bond)
        const bool overlap = !site_sec.empty() && !gen_sec.empty() && !ctx->profiling && !ctx->rec;
        SideJoin guard(overlap ? ctx : nullptr);   // after s: an error between fork and join still joins first
        if (!site_sec.empty()) {
            std::vector<SvdSiteTask> st;
            std::vector<SvdPart> parts;
            for (int ni : site_sec) {
                const int M = bn.dim[ni], N = c0[ni] + c1[ni], k = kk[ni];
                US[ni] = s.dbl((size_t)M * k);
                Vt[ni] = s.dbl((size_t)k * N);
                SvdSiteTask task{M, N, k, std::max(M, N), M < N ? 1 : 0, (int)parts.size(), 0, S_all + soff[ni],
                                 US[ni], Vt[ni]};
                for (int part = 0; part < 2; ++part) {
                    const int bi = part == 0 ? b0[ni] : b1[ni];
                    if (bi < 0) continue;
                    const Block& bk = L.blocks[t][bi];
                    parts.push_back({cores[t] + bk.off, bk.cols, part == 0 ? 0 : c0[ni]});
                }
                task.p_end = (int)parts.size();
                st.push_back(task);
            }
            launch_svd_site(ctx, st, parts, s, overlap);
        }
        if (!gen_sec.empty()) {
            std::vector<CopyTask> gather;
            std::vector<SvdTask> svd;
            for (int ni : gen_sec) {
                const int M = bn.dim[ni], N = c0[ni] + c1[ni], k = kk[ni];
                const int wide = M < N ? 1 : 0;
                double* G = s.dbl((size_t)M * N);
                double* V = s.dbl((size_t)k * k);
                US[ni] = s.dbl((size_t)M * k);
                Vt[ni] = s.dbl((size_t)k * N);
                for (int part = 0; part < 2; ++part) {
                    const int bi = part == 0 ? b0[ni] : b1[ni];
                    if (bi < 0) continue;
                    const Block& bk = L.blocks[t][bi];
                    const int coff = part == 0 ? 0 : c0[ni];
                    if (wide)
                        gather.push_back({cores[t] + bk.off, G + coff, bk.rows, bk.cols, bk.cols, N, 0, 0, 0, 1.0});
                    else
                        gather.push_back({cores[t] + bk.off, G + (int64_t)coff * M, bk.rows, bk.cols, bk.cols, M,
                                          0, 1, 0, 1.0});
                }
                svd.push_back({G, V, S_all + soff[ni], US[ni], Vt[ni], M, N, wide});
            }
            launch_copy(ctx, gather);
            launch_svd(ctx, svd);
        }
        if (overlap) ctx->join_side();
        std::vector<double> S_h((size_t)stot);
        if (stot > 0) {
            BSM_CUDA(cudaMemcpyAsync(S_h.data(), S_all, (size_t)stot * sizeof(double),
                                     cudaMemcpyDeviceToHost, ctx->stream));
            ctx->sync();
        }
        std::vector<SvEntry> sv;
        for (int ni = 0; ni < nn; ++ni)
            for (int j = 0; j < kk[ni]; ++j) sv.push_back({S_h[soff[ni] + j], ni, j});
        const std::vector<int> keep = choose_cut(sv, nn, tol2, r_max, &td2, &cd2);
        const std::vector<int> oldlook = block_lookup(L, t - 1);
        const std::vector<Block> oldB_tm = L.blocks[t - 1];
        {
            Bond nb;
            for (int ni = 0; ni < nn; ++ni)
                if (keep[ni] > 0) {
                    nb.q.push_back(bn.q[ni]);
                    nb.dim.push_back(keep[ni]);
                }
            L.bonds[t] = nb;
            rebuild_site(L, t - 1);
            rebuild_site(L, t);
        }
        double* nt = alloc_core(L.core_size[t]);
        double* ntm = alloc_core(L.core_size[t - 1]);
        bool fused_apply = true;
        {
            std::vector<int64_t> fma(nn, 0);
            for (const Block& nbk : L.blocks[t - 1]) {
                const int ni = bn.find(L.bonds[t].q[nbk.ri]);
                fma[ni] += (int64_t)nbk.rows * bn.dim[ni] * nbk.cols;
            }
            for (int ni = 0; ni < nn; ++ni)
                if (fma[ni] > kFusedGemmMaxFma) fused_apply = false;
        }
        if (fused_apply) {
            std::vector<RTask> rt(nn);
            std::vector<RCopy> rc;
            std::vector<RGemm> rg;
            std::vector<std::vector<RCopy>> cpn(nn);
            std::vector<std::vector<RGemm>> gmn(nn);
            for (const Block& nbk : L.blocks[t]) {
                const int ni = bn.find(L.bonds[t].q[nbk.li]);
                const int coff = nbk.sigma == 0 ? 0 : c0[ni];
                cpn[ni].push_back({Vt[ni] + coff, nt + nbk.off, nbk.rows, nbk.cols, c0[ni] + c1[ni]});
            }
            for (const Block& nbk : L.blocks[t - 1]) {
                const int ni = bn.find(L.bonds[t].q[nbk.ri]);
                const Block& ob = oldB_tm[oldlook[nbk.li * 2 + nbk.sigma]];
                gmn[ni].push_back({cores[t - 1] + ob.off, US[ni], ntm + nbk.off, nbk.rows, bn.dim[ni], nbk.cols,
                                   kk[ni]});
            }
            std::vector<RTask> tasks;
            for (int ni = 0; ni < nn; ++ni) {
                if (cpn[ni].empty() && gmn[ni].empty()) continue;
                RTask task{(int)rc.size(), 0, (int)rg.size(), 0};
                rc.insert(rc.end(), cpn[ni].begin(), cpn[ni].end());
                rg.insert(rg.end(), gmn[ni].begin(), gmn[ni].end());
                task.c_end = (int)rc.size();
                task.g_end = (int)rg.size();
                tasks.push_back(task);
            }
            launch_right_apply(ctx, tasks, rc, rg);
        } else {
            std::vector<CopyTask> vcopy;
            for (const Block& nbk : L.blocks[t]) {
                const int ni = bn.find(L.bonds[t].q[nbk.li]);
                const int coff = nbk.sigma == 0 ? 0 : c0[ni];
                const int N = c0[ni] + c1[ni];
                vcopy.push_back({Vt[ni] + coff, nt + nbk.off, nbk.rows, nbk.cols, N, nbk.cols, 0, 0, 0, 1.0});
            }
            launch_copy(ctx, vcopy);
            std::vector<GemmOut> outs;
            std::vector<GemmIn> ins;
            for (const Block& nbk : L.blocks[t - 1]) {
                const int ni = bn.find(L.bonds[t].q[nbk.ri]);
                const Block& ob = oldB_tm[oldlook[nbk.li * 2 + nbk.sigma]];
                outs.push_back({ntm + nbk.off, nbk.rows, nbk.cols, nbk.cols, (int)ins.size(),
                                (int)ins.size() + 1, 0.0});
                ins.push_back({cores[t - 1] + ob.off, US[ni], bn.dim[ni], ob.cols, kk[ni], 0, 1.0});
            }
            launch_gemm(ctx, outs, ins);
        }
        release(t);
        release(t - 1);
        cores[t] = nt;
        owned[t] = 1;
        cores[t - 1] = ntm;
        owned[t - 1] = 1;
    }
}

// Planned left sweep of one job: the new layout of every site follows on the
// host from the sector row counts alone (rank = min(rows, cols)).
struct LeftPlan {
    Layout P;
    std::vector<double*> pc;
    std::vector<char> po;
    std::vector<double*> fresh, deferred;
    std::vector<std::vector<LeftTask>> tasks;   // per site
    std::vector<LeftSrc> srcs;
    std::vector<LeftX> xs;
};

// False (nothing allocated) when a site does not fit the fused kernel.
bool plan_left(Context* ctx, const TruncJob& J, LeftPlan& pl) {
    const int K = J.L.K;
    pl.P = J.L;
    pl.pc = J.cores;
    pl.po = J.owned;
    pl.tasks.assign(K - 1, {});
    auto abandon = [&]() {
        for (double* q : pl.fresh) ctx->free(q);
        pl.fresh.clear();
        return false;
    };
    Layout& P = pl.P;
    for (int t = 0; t + 1 < K; ++t) {
        const Bond bm = P.bonds[t + 1];
        const int nm = (int)bm.q.size();
        std::vector<int> Mrows(nm, 0), krank(nm, 0);
        std::vector<std::vector<std::pair<int, int>>> stack(nm);
        for (int bi = 0; bi < (int)P.blocks[t].size(); ++bi) {
            const Block& bk = P.blocks[t][bi];
            stack[bk.ri].push_back({bi, Mrows[bk.ri]});
            Mrows[bk.ri] += bk.rows;
        }
        const std::vector<int> oldlook = block_lookup(P, t + 1);
        const std::vector<Block> oldB_t = P.blocks[t], oldB_t1 = P.blocks[t + 1];
        Bond nb;
        for (int mi = 0; mi < nm; ++mi) {
            if (Mrows[mi] > 0) krank[mi] = std::min(Mrows[mi], bm.dim[mi]);
            if (krank[mi] > 0) {
                nb.q.push_back(bm.q[mi]);
                nb.dim.push_back(krank[mi]);
            }
        }
        for (int mi = 0; mi < nm; ++mi) {
            if (Mrows[mi] == 0) continue;
            int64_t rx = 0;
            for (int sg = 0; sg < 2; ++sg) {
                const int ob = oldlook[mi * 2 + sg];
                if (ob >= 0) rx += (int64_t)krank[mi] * bm.dim[mi] * oldB_t1[ob].cols;
            }
            if (!left_site_fits(Mrows[mi], bm.dim[mi], rx)) return abandon();
        }
        P.bonds[t + 1] = nb;
        rebuild_site(P, t);
        rebuild_site(P, t + 1);
        double* nt = P.core_size[t] > 0 ? (double*)ctx->alloc(sizeof(double) * (size_t)P.core_size[t]) : nullptr;
        double* nt1 =
            P.core_size[t + 1] > 0 ? (double*)ctx->alloc(sizeof(double) * (size_t)P.core_size[t + 1]) : nullptr;
        if (nt) pl.fresh.push_back(nt);
        if (nt1) pl.fresh.push_back(nt1);
        const std::vector<int> newlook_t = block_lookup(P, t);
        for (int mi = 0; mi < nm; ++mi) {
            if (Mrows[mi] == 0) continue;
            const int nmi = P.bonds[t + 1].find(bm.q[mi]);
            LeftTask task{Mrows[mi], bm.dim[mi], krank[mi], (int)pl.srcs.size(), 0, (int)pl.xs.size(), 0};
            for (auto& pr : stack[mi]) {
                const Block& ob = oldB_t[pr.first];
                const Block& nbk = P.blocks[t][newlook_t[ob.li * 2 + ob.sigma]];
                pl.srcs.push_back({pl.pc[t] + ob.off, nt + nbk.off, ob.rows, pr.second});
            }
            task.s_end = (int)pl.srcs.size();
            for (const Block& nbk : P.blocks[t + 1]) {
                if (nbk.li != nmi) continue;
                const Block& ob = oldB_t1[oldlook[mi * 2 + nbk.sigma]];
                pl.xs.push_back({pl.pc[t + 1] + ob.off, nt1 + nbk.off, ob.cols});
            }
            task.x_end = (int)pl.xs.size();
            pl.tasks[t].push_back(task);
        }
        for (int u : {t, t + 1})
            if (pl.po[u] && pl.pc[u]) pl.deferred.push_back(pl.pc[u]);
        pl.pc[t] = nt;
        pl.po[t] = 1;
        pl.pc[t + 1] = nt1;
        pl.po[t + 1] = 1;
    }
    return true;
}

// Left sweeps of several truncations as one persistent launch (site t of
// every job is phase t).  Jobs whose sites do not fit are returned in `rest`.
bool left_sweep_batch(Context* ctx, const std::vector<TruncJob*>& jobs, GridSync* gs,
                      std::vector<TruncJob*>* rest) {
    std::vector<TruncJob*> in;
    std::vector<LeftPlan> plans;
    plans.reserve(jobs.size());
    for (TruncJob* J : jobs) {
        if (J->L.K < 2) {
            rest->push_back(J);
            continue;
        }
        plans.emplace_back();
        if (plan_left(ctx, *J, plans.back())) {
            in.push_back(J);
        } else {
            plans.pop_back();
            rest->push_back(J);
        }
    }
    if (in.empty()) return false;
    const int K = in[0]->L.K;
    std::vector<LeftTask> lt;
    std::vector<LeftSrc> ls;
    std::vector<LeftX> lx;
    std::vector<int> phase_beg{0};
    std::vector<int> soff(plans.size()), xoff(plans.size());
    for (size_t j = 0; j < plans.size(); ++j) {
        soff[j] = (int)ls.size();
        xoff[j] = (int)lx.size();
        ls.insert(ls.end(), plans[j].srcs.begin(), plans[j].srcs.end());
        lx.insert(lx.end(), plans[j].xs.begin(), plans[j].xs.end());
    }
    for (int t = 0; t + 1 < K; ++t) {
        for (size_t j = 0; j < plans.size(); ++j)
            for (LeftTask task : plans[j].tasks[t]) {
                task.s_beg += soff[j];
                task.s_end += soff[j];
                task.x_beg += xoff[j];
                task.x_end += xoff[j];
                lt.push_back(task);
            }
        phase_beg.push_back((int)lt.size());
    }
    if (!launch_left_sweep(ctx, lt, ls, lx, phase_beg, gs)) {
        for (LeftPlan& pl : plans)
            for (double* q : pl.fresh) ctx->free(q);
        rest->insert(rest->end(), in.begin(), in.end());
        return false;
    }
    // the intermediate R X cores and the replaced cores are released behind the launch
    for (size_t j = 0; j < plans.size(); ++j) {
        for (double* q : plans[j].deferred) ctx->free(q);
        in[j]->L = plans[j].P;
        in[j]->cores = plans[j].pc;
        in[j]->owned = plans[j].po;
    }
    return true;
}

// Sizes of one job's device-driven right sweep: padded ranks per bond
// (kpad[K] = 1 for the single sector of bond K) and padded column counts.
struct RightPlan {
    TruncJob* J;
    std::vector<std::vector<int>> kpad, cpad;
    std::vector<int> secoff;   // first sector of bond b in the job's keep / kact arrays
    int nsec = 0;
    std::vector<std::vector<double*>> S, US, Vt;
    int* kact = nullptr;
    int* keep = nullptr;
    double* disc = nullptr;
};

// Jobs with a sector of this many kept columns or more leave the persistent
// right sweep (one CTA per sector) for the per-site sweep, whose larger SVDs run
// on thread-block clusters: one SM's FP64 rate bounds a one-CTA Jacobi.
constexpr int kPersistentSvdMax = 40;

bool plan_right_sizes(const TruncJob& J, RightPlan& rp) {
    const Layout& L = J.L;
    const int K = L.K;
    if (K < 2) return false;
    rp.kpad.assign(K + 1, {});
    rp.cpad.assign(K + 1, {});
    rp.kpad[K].assign(L.bonds[K].q.size(), 1);
    for (int b = K - 1; b >= 1; --b) {
        const Bond& bn = L.bonds[b];
        rp.kpad[b].assign(bn.q.size(), 0);
        rp.cpad[b].assign(bn.q.size(), 0);
        int total = 0;
        for (const Block& bk : L.blocks[b]) rp.cpad[b][bk.li] += (b + 1 == K) ? bk.cols : rp.kpad[b + 1][bk.ri];
        for (size_t n = 0; n < bn.q.size(); ++n) {
            // the SVD keeps min(rows, cols) columns before the cut, so the
            // padding is not reduced by the rank cap
            const int kp = std::min(bn.dim[n], rp.cpad[b][n]);
            rp.kpad[b][n] = kp;
            total += kp;
            if (kp >= kPersistentSvdMax || dyn_svd_smem(bn.dim[n], rp.cpad[b][n]) > 220 * 1024) return false;
            int64_t fma = 0;
            for (const Block& bk : L.blocks[b])
                if (bk.li == (int)n && b + 1 < K) fma += (int64_t)bk.rows * bk.cols * rp.kpad[b + 1][bk.ri];
            if (fma > (int64_t)1 << 20) return false;
        }
        if (total > 2048) return false;
    }
    rp.secoff.assign(K + 1, 0);
    rp.nsec = 0;
    for (int b = 1; b < K; ++b) {
        rp.secoff[b] = rp.nsec;
        rp.nsec += (int)L.bonds[b].q.size();
    }
    return true;
}

// Right sweeps with the cut decided on the device, several truncations in one
// persistent launch (bond K-1-p of every job is phase p).  Every bond's SVDs
// read the kept counts of the previous bond from device memory; the last task
// of a job in a phase runs that job's pooled cut.  The kept counts of all
// bonds are read once at the end.  Jobs that do not fit are returned in `rest`.
bool right_sweep_batch(Context* ctx, const std::vector<TruncJob*>& jobs, GridSync* gs, bool* gs_checked,
                       std::vector<TruncJob*>* rest) {
    std::vector<RightPlan> plans;
    for (TruncJob* J : jobs) {
        RightPlan rp;
        rp.J = J;
        if (plan_right_sizes(*J, rp))
            plans.push_back(std::move(rp));
        else
            rest->push_back(J);
    }
    if (plans.empty()) return false;
    const int K = plans[0].J->L.K;
    const int nj = (int)plans.size();
    // buffers
    Scratch s(ctx);
    int nsec_tot = 0;
    for (RightPlan& rp : plans) nsec_tot += rp.nsec;
    const int n_phase = K - 1;
    const size_t n_ints = 2 * (size_t)std::max(nsec_tot, 1) + (size_t)n_phase * nj;
    int* ints = (int*)ctx->alloc(sizeof(int) * n_ints);
    s.ptrs.push_back(ints);
    double* disc = s.dbl(2 * (size_t)nj);
    BSM_CUDA(cudaMemsetAsync(ints, 0, sizeof(int) * n_ints, ctx->stream));
    BSM_CUDA(cudaMemsetAsync(disc, 0, sizeof(double) * 2 * nj, ctx->stream));
    int* done = ints + 2 * (size_t)std::max(nsec_tot, 1);
    {
        // S, US and Vt of every sector of every bond and job, carved from one allocation
        size_t total = 0;
        for (RightPlan& rp : plans) {
            const Layout& L = rp.J->L;
            for (int b = 1; b < K; ++b)
                for (size_t n = 0; n < L.bonds[b].q.size(); ++n) {
                    const size_t kp = std::max(rp.kpad[b][n], 1), cp = std::max(rp.cpad[b][n], 1);
                    total += kp + (size_t)L.bonds[b].dim[n] * kp + kp * cp;
                }
        }
        double* arena = s.dbl(total);
        size_t at = 0;
        auto carve = [&](size_t n) {
            double* q = arena + at;
            at += n;
            return q;
        };
        int o = 0;
        for (int j = 0; j < nj; ++j) {
            RightPlan& rp = plans[j];
            rp.kact = ints + o;
            rp.keep = ints + std::max(nsec_tot, 1) + o;
            rp.disc = disc + 2 * j;
            o += rp.nsec;
            const Layout& L = rp.J->L;
            rp.S.assign(K, {});
            rp.US.assign(K, {});
            rp.Vt.assign(K, {});
            for (int b = 1; b < K; ++b) {
                const Bond& bn = L.bonds[b];
                for (size_t n = 0; n < bn.q.size(); ++n) {
                    const size_t kp = std::max(rp.kpad[b][n], 1), cp = std::max(rp.cpad[b][n], 1);
                    rp.S[b].push_back(carve(kp));
                    rp.US[b].push_back(carve((size_t)bn.dim[n] * kp));
                    rp.Vt[b].push_back(carve(kp * cp));
                }
            }
        }
    }
    // tasks in sweep order
    std::vector<DynTask> tasks;
    std::vector<DynPart> parts;
    std::vector<CutTask> cuts;
    std::vector<CutSector> secs;
    std::vector<int> phase_beg{0};
    for (int b = K - 1; b >= 1; --b) {
        for (int j = 0; j < nj; ++j) {
            RightPlan& rp = plans[j];
            const Layout& L = rp.J->L;
            const std::vector<double*>& cores = rp.J->cores;
            const Bond& bn = L.bonds[b];
            const int cut_idx = (int)cuts.size();
            std::vector<std::vector<DynPart>> per(bn.q.size());
            for (const Block& bk : L.blocks[b]) {   // layout order: sigma 0 before 1 within a sector
                const int m = bk.ri;
                if (b + 1 == K)
                    per[bk.li].push_back({cores[b] + bk.off, bk.cols, nullptr, 0, nullptr});
                else
                    per[bk.li].push_back({cores[b] + bk.off, bk.cols, rp.US[b + 1][m],
                                          std::max(rp.kpad[b + 1][m], 1), rp.keep + rp.secoff[b + 1] + m});
            }
            for (size_t n = 0; n < bn.q.size(); ++n) {
                DynTask t{bn.dim[n],       std::max(rp.kpad[b][n], 1), std::max(rp.cpad[b][n], 1),
                          (int)parts.size(), 0, rp.S[b][n], rp.US[b][n], rp.Vt[b][n],
                          rp.kact + rp.secoff[b] + (int)n, cut_idx};
                parts.insert(parts.end(), per[n].begin(), per[n].end());
                t.p_end = (int)parts.size();
                tasks.push_back(t);
            }
            const int s_beg = (int)secs.size();
            int cap = 0;
            for (size_t n = 0; n < bn.q.size(); ++n) {
                secs.push_back({rp.S[b][n], rp.kact + rp.secoff[b] + (int)n});
                cap += rp.kpad[b][n];
            }
            const double tol2 = rp.J->eps * rp.J->eps / (K - 1);
            cuts.push_back({(int)bn.q.size(), s_beg, std::max(cap, 1), rp.J->r_max, tol2, rp.keep + rp.secoff[b],
                            rp.disc, (int)bn.q.size(), done + cut_idx});
        }
        phase_beg.push_back((int)tasks.size());
    }
    std::vector<int> prof_idx(1, -1);
    if (!launch_right_sweep(ctx, tasks, parts, phase_beg, cuts, secs, gs + 1, &prof_idx[0])) {
        // grid not co-resident: one SVD launch per bond and one cut launch per job
        prof_idx.clear();
        for (int p = 0; p < n_phase; ++p) {
            std::vector<DynTask> tp(tasks.begin() + phase_beg[p], tasks.begin() + phase_beg[p + 1]);
            prof_idx.push_back(launch_right_dyn(ctx, tp, parts));
            for (int j = 0; j < nj; ++j) launch_cut(ctx, cuts[(size_t)p * nj + j], secs);
        }
    }
    std::vector<int> ints_h(2 * (size_t)std::max(nsec_tot, 1));
    std::vector<double> disc_h(2 * (size_t)nj);
    GridSync gs_h[2];
    BSM_CUDA(cudaMemcpyAsync(ints_h.data(), ints, sizeof(int) * ints_h.size(), cudaMemcpyDeviceToHost,
                             ctx->stream));
    BSM_CUDA(cudaMemcpyAsync(disc_h.data(), disc, sizeof(double) * disc_h.size(), cudaMemcpyDeviceToHost,
                             ctx->stream));
    BSM_CUDA(cudaMemcpyAsync(gs_h, gs, sizeof(gs_h), cudaMemcpyDeviceToHost, ctx->stream));
    ctx->sync();
    BSM_REQUIRE(gs_h[0].err == 0 && gs_h[1].err == 0, BSMPS_ERR_TIMEOUT,
                "truncation sweep: a grid-wide wait gave up");
    *gs_checked = true;
    // compaction of every job: kept rows of Vt into cores 1..K-1, X_0 U S into core 0
    double fl = 0.0;
    std::vector<CopyTask> cp;
    std::vector<GemmOut> go;
    std::vector<GemmIn> gi;
    std::vector<std::vector<double*>> new_cores(nj);
    std::vector<Layout> new_lay(nj);
    for (int j = 0; j < nj; ++j) {
        RightPlan& rp = plans[j];
        TruncJob& J = *rp.J;
        const Layout& L = J.L;
        J.td2 += disc_h[2 * j];
        J.cd2 += disc_h[2 * j + 1];
        const int* keep_h = ints_h.data() + std::max(nsec_tot, 1) + (rp.keep - (ints + std::max(nsec_tot, 1)));
        auto kept = [&](int b, int m) { return b == K ? 1 : keep_h[rp.secoff[b] + m]; };
        std::vector<std::vector<int>> coff1(K);
        for (int b = K - 1; b >= 1; --b) {
            const Bond& bn = L.bonds[b];
            std::vector<int> cols_act(bn.q.size(), 0);
            coff1[b].assign(bn.q.size(), 0);
            for (const Block& bk : L.blocks[b]) {
                const int c = (b + 1 == K) ? bk.cols : kept(b + 1, bk.ri);
                if (bk.sigma == 0) coff1[b][bk.li] = c;
                cols_act[bk.li] += c;
                if (b + 1 < K) fl += 2.0 * bk.rows * (double)bk.cols * c;
            }
            for (size_t n = 0; n < bn.q.size(); ++n) {
                const double M = bn.dim[n], N = cols_act[n], k = std::min(M, N), len = std::max(M, N);
                if (k > 0)
                    fl += 2.0 * len * k * k - (len + k) * k * k + 2.0 / 3.0 * k * k * k + 2.0 * len * k * k -
                          2.0 / 3.0 * k * k * k + 54.0 * k * k * k + 2.0 * len * k * k;
            }
        }
        Layout F = L;
        for (int b = 1; b < K; ++b) {
            Bond nb;
            for (size_t n = 0; n < L.bonds[b].q.size(); ++n)
                if (keep_h[rp.secoff[b] + n] > 0) {
                    nb.q.push_back(L.bonds[b].q[n]);
                    nb.dim.push_back(keep_h[rp.secoff[b] + n]);
                }
            F.bonds[b] = nb;
        }
        F.rebuild_blocks();
        std::vector<double*>& nc = new_cores[j];
        nc.assign(K, nullptr);
        for (int t = 0; t < K; ++t)
            if (F.core_size[t] > 0) nc[t] = (double*)ctx->alloc(sizeof(double) * (size_t)F.core_size[t]);
        for (int t = 0; t < K; ++t) {
            for (const Block& fb : F.blocks[t]) {
                const Charge qn = F.bonds[t].q[fb.li];
                if (t == 0) {
                    const int m = L.bonds[1].find(F.bonds[1].q[fb.ri]);
                    const Block* ob = nullptr;
                    for (const Block& b0 : L.blocks[0])
                        if (b0.sigma == fb.sigma) ob = &b0;
                    go.push_back({nc[0] + fb.off, fb.rows, fb.cols, fb.cols, (int)gi.size(), (int)gi.size() + 1, 0.0});
                    gi.push_back({J.cores[0] + ob->off, rp.US[1][m], ob->cols, ob->cols,
                                  std::max(rp.kpad[1][m], 1), 0, 1.0});
                } else {
                    const int n = L.bonds[t].find(qn);
                    const int coff = fb.sigma == 0 ? 0 : coff1[t][n];
                    cp.push_back({rp.Vt[t][n] + coff, nc[t] + fb.off, fb.rows, fb.cols,
                                  std::max(rp.cpad[t][n], 1), fb.cols, 0, 0, 0, 1.0});
                }
            }
        }
        new_lay[j] = F;
    }
    ctx->flops += fl;
    if (!prof_idx.empty() && prof_idx[0] >= 0) {
        for (int idx : prof_idx) ctx->prof[idx].flops = 0.0;
        ctx->prof[prof_idx[0]].flops = fl;   // attributed to the sweep's first SVD launch record
    }
    launch_copy(ctx, cp);
    launch_gemm(ctx, go, gi);
    for (int j = 0; j < nj; ++j) {
        TruncJob& J = *plans[j].J;
        for (int t = 0; t < K; ++t) {
            if (J.owned[t] && J.cores[t]) ctx->free(J.cores[t]);
            J.cores[t] = new_cores[j][t];
            J.owned[t] = 1;
        }
        J.L = new_lay[j];
    }
    return true;
}

// trunc_eps of several MPS of the same sites (Sec. 2.2): the fused sweeps of
// all of them share launches.
std::vector<MpsPtr> truncate_jobs(Context* ctx, std::vector<std::unique_ptr<TruncJob>>& jobs,
                                  bool left_orthogonal = false) {
    std::vector<TruncJob*> all;
    for (auto& j : jobs) all.push_back(j.get());
    // phase bookkeeping of the two persistent sweeps; err is read back with
    // the right sweep's cut results (or at the end when that path is not taken)
    Scratch gs_scratch(ctx);
    GridSync* gs = (GridSync*)ctx->alloc(2 * sizeof(GridSync));
    gs_scratch.ptrs.push_back(gs);
    BSM_CUDA(cudaMemsetAsync(gs, 0, 2 * sizeof(GridSync), ctx->stream));
    bool gs_checked = false;
    std::vector<TruncJob*> left_rest;
    const bool left_done = !left_orthogonal && left_sweep_batch(ctx, all, gs, &left_rest);
    if (!left_orthogonal)
        for (TruncJob* J : left_rest) left_sweep_sitewise(ctx, *J);
    std::vector<TruncJob*> right_rest;
    right_sweep_batch(ctx, all, gs, &gs_checked, &right_rest);
    for (TruncJob* J : right_rest) right_sweep_sitewise(ctx, *J);
    if (left_done && !gs_checked) {
        GridSync h;
        BSM_CUDA(cudaMemcpyAsync(&h, gs, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
        ctx->sync();
        BSM_REQUIRE(h.err == 0, BSMPS_ERR_TIMEOUT, "left truncation sweep: a grid-wide wait gave up");
    }
    std::vector<MpsPtr> out;
    for (TruncJob* J : all) out.push_back(J->finish());
    return out;
}

}  // namespace

std::vector<MpsPtr> op_truncate_batch_left_orthogonal(Context* ctx, const std::vector<const Mps*>& xs,
                                                      const std::vector<double>& eps, int r_max) {
    BSM_REQUIRE(xs.size() == eps.size(), BSMPS_ERR_INVALID_ARG, "one tolerance per MPS");
    if (xs.empty()) return {};
    std::vector<std::unique_ptr<TruncJob>> jobs;
    for (size_t i = 0; i < xs.size(); ++i) {
        BSM_REQUIRE(same_space(xs[i]->lay, xs[0]->lay), BSMPS_ERR_INVALID_ARG,
                    "batched truncation of MPS on different sites");
        jobs.emplace_back(new TruncJob(ctx, xs[i], eps[i], r_max));
    }
    return truncate_jobs(ctx, jobs, true);
}

std::vector<double> op_last_core_norms(Context* ctx, const std::vector<const Mps*>& xs) {
    std::vector<double> out(xs.size(), 0.0);
    std::vector<const double*> ptr;
    std::vector<int64_t> n;
    std::vector<int> who;
    for (size_t i = 0; i < xs.size(); ++i) {
        const int K = xs[i]->lay.K;
        if (K == 0 || xs[i]->lay.core_size[K - 1] == 0) continue;
        ptr.push_back(xs[i]->core[K - 1]);
        n.push_back(xs[i]->lay.core_size[K - 1]);
        who.push_back((int)i);
    }
    if (ptr.empty()) return out;
    Scratch s(ctx);
    double* d = s.dbl(ptr.size());
    launch_sumsq(ctx, ptr, n, d);
    std::vector<double> h(ptr.size());
    BSM_CUDA(cudaMemcpyAsync(h.data(), d, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    ctx->sync();
    for (size_t q = 0; q < who.size(); ++q) out[who[q]] = std::sqrt(h[q]);
    return out;
}

MpsPtr op_truncate(Context* ctx, const Mps* x, double eps, int r_max, double* disc_tol, double* disc_cap) {
    std::vector<std::unique_ptr<TruncJob>> jobs;
    jobs.emplace_back(new TruncJob(ctx, x, eps, r_max));
    std::vector<MpsPtr> out = truncate_jobs(ctx, jobs);
    if (disc_tol) *disc_tol = std::sqrt(jobs[0]->td2);
    if (disc_cap) *disc_cap = std::sqrt(jobs[0]->cd2);
    return std::move(out[0]);
}

std::vector<MpsPtr> op_truncate_batch(Context* ctx, const std::vector<const Mps*>& xs, const std::vector<double>& eps,
                                      int r_max) {
    BSM_REQUIRE(xs.size() == eps.size(), BSMPS_ERR_INVALID_ARG, "one tolerance per MPS");
    if (xs.empty()) return {};
    std::vector<std::unique_ptr<TruncJob>> jobs;
    for (size_t i = 0; i < xs.size(); ++i) {
        BSM_REQUIRE(same_space(xs[i]->lay, xs[0]->lay), BSMPS_ERR_INVALID_ARG,
                    "batched truncation of MPS on different sites");
        jobs.emplace_back(new TruncJob(ctx, xs[i], eps[i], r_max));
    }
    return truncate_jobs(ctx, jobs);
}

namespace {
struct EnvBlk {
    int c, ia, ib;
    int rows, cols;
    double* ptr;
};

Mpo identity_mpo(const Layout& L) {
    Mpo I;
    I.K = L.K;
    I.species = L.species;
    I.charges.assign(L.K + 1, std::vector<Charge>(1, Charge{0, 0}));
    I.entries.assign(L.K, {{0, 0, 0, 0, 1.0}, {0, 0, 1, 1, 1.0}});
    return I;
}
}  // namespace

// Per-site launches (used when the persistent sweep cannot be resident).
static std::vector<double> dot_batch_sitewise(Context* ctx, const std::vector<EnvProblem>& probs) {
    const int P = (int)probs.size();
    std::vector<double> result(P, 0.0);
    if (P == 0) return result;
    const int K = probs[0].a->lay.K;
    std::vector<Mpo> ids;
    ids.reserve(P);
    std::vector<const Mpo*> ops(P);
    for (int p = 0; p < P; ++p) {
        const EnvProblem& pr = probs[p];
        BSM_REQUIRE(same_space(pr.a->lay, pr.b->lay) && pr.a->lay.K == K, BSMPS_ERR_INVALID_ARG,
                    "dot of MPS of different spaces");
        if (pr.W) {
            BSM_REQUIRE(pr.W->K == K && pr.W->species == pr.a->lay.species, BSMPS_ERR_INVALID_ARG,
                        "MPO and MPS act on different sites");
            ops[p] = pr.W;
        } else {
            ids.push_back(identity_mpo(pr.a->lay));
            ops[p] = &ids.back();
        }
    }
    // bond 0 environments: [[1]] on (channel 0, sector 0, sector 0)
    std::vector<std::vector<EnvBlk>> E(P);
    Scratch keep0(ctx);
    double* one = nullptr;
    {
        std::vector<double> v(1, 1.0);
        one = keep0.up(v);
    }
    for (int p = 0; p < P; ++p) {
        const Layout& A = probs[p].a->lay;
        const Layout& B = probs[p].b->lay;
        if (!A.bonds[0].q.empty() && !B.bonds[0].q.empty()) E[p].push_back({0, 0, 0, 1, 1, one});
    }
    double* prevbuf = nullptr;
    for (int t = 0; t < K; ++t) {
        // ---- structure of this site ----
        struct TBlk {
            int env, sigma, rows, cols;
            int64_t off;
        };
        std::vector<std::vector<TBlk>> T(P);
        // contributions: key (d, ra, rb) -> list of (T index, alpha) and the a-block
        std::vector<std::map<std::tuple<int, int, int>, std::vector<std::tuple<int, int, double>>>> contrib(P);
        int64_t tot_T = 0;
        for (int p = 0; p < P; ++p) {
            const Layout& A = probs[p].a->lay;
            const Layout& B = probs[p].b->lay;
            const std::vector<int> blook = block_lookup(B, t);
            const std::vector<int> alook = block_lookup(A, t);
            // T blocks: env e x b-block (ib, si)
            std::vector<std::array<int, 2>> tidx(E[p].size(), {-1, -1});
            for (int e = 0; e < (int)E[p].size(); ++e)
                for (int si = 0; si < 2; ++si) {
                    const int bb = blook[E[p][e].ib * 2 + si];
                    if (bb < 0) continue;
                    tidx[e][si] = (int)T[p].size();
                    T[p].push_back({e, si, E[p][e].rows, B.blocks[t][bb].cols, tot_T});
                    tot_T += (int64_t)E[p][e].rows * B.blocks[t][bb].cols;
                }
            // env blocks by channel
            std::map<int, std::vector<int>> by_chan;
            for (int e = 0; e < (int)E[p].size(); ++e) by_chan[E[p][e].c].push_back(e);
            const Mpo& W = *ops[p];
            for (int ei = 0; ei < (int)W.entries[t].size(); ++ei) {
                const MpoEntry& me = W.entries[t][ei];
                auto it = by_chan.find(me.a);
                if (it == by_chan.end()) continue;
                double w = me.w;
                if (probs[p].W && t == 0 && (ei == W.shift_entry[0] || ei == W.shift_entry[1]))
                    w += probs[p].shift;
                double fa = 1.0, fb = 1.0;
                if (me.so == 0 ? probs[p].fa0 : probs[p].fa1) fa = (*(me.so == 0 ? probs[p].fa0 : probs[p].fa1))[t];
                if (me.si == 0 ? probs[p].fb0 : probs[p].fb1) fb = (*(me.si == 0 ? probs[p].fb0 : probs[p].fb1))[t];
                const double alpha = w * fa * fb;
                for (int e : it->second) {
                    const int ab = alook[E[p][e].ia * 2 + me.so];
                    const int ti = tidx[e][me.si];
                    if (ab < 0 || ti < 0) continue;
                    const int bb = blook[E[p][e].ib * 2 + me.si];
                    const int ra = A.blocks[t][ab].ri, rb = B.blocks[t][bb].ri;
                    contrib[p][std::make_tuple(me.b, ra, rb)].push_back(std::make_tuple(ti, ab, alpha));
                }
            }
        }
        // ---- buffers ----
        int64_t tot_E = 0;
        std::vector<std::vector<EnvBlk>> En(P);
        for (int p = 0; p < P; ++p) {
            const Layout& A = probs[p].a->lay;
            const Layout& B = probs[p].b->lay;
            for (auto& kv : contrib[p]) {
                const int d = std::get<0>(kv.first), ra = std::get<1>(kv.first), rb = std::get<2>(kv.first);
                En[p].push_back({d, ra, rb, A.bonds[t + 1].dim[ra], B.bonds[t + 1].dim[rb],
                                 (double*)(intptr_t)tot_E});
                tot_E += (int64_t)A.bonds[t + 1].dim[ra] * B.bonds[t + 1].dim[rb];
            }
        }
        Scratch s(ctx);
        double* Tbuf = s.dbl((size_t)std::max<int64_t>(tot_T, 1));
        double* Ebuf = (double*)ctx->alloc(sizeof(double) * (size_t)std::max<int64_t>(tot_E, 1));
        // stage 1: T = E * X_b(ib, si)
        std::vector<GemmOut> o1;
        std::vector<GemmIn> i1;
        for (int p = 0; p < P; ++p) {
            const Layout& B = probs[p].b->lay;
            const std::vector<int> blook = block_lookup(B, t);
            for (const TBlk& tb : T[p]) {
                const EnvBlk& eb = E[p][tb.env];
                const Block& bk = B.blocks[t][blook[eb.ib * 2 + tb.sigma]];
                o1.push_back({Tbuf + tb.off, tb.rows, tb.cols, tb.cols, (int)i1.size(), (int)i1.size() + 1, 0.0});
                i1.push_back({eb.ptr, probs[p].b->core[t] + bk.off, eb.cols, eb.cols, bk.cols, 0, 1.0});
            }
        }
        launch_gemm(ctx, o1, i1);
        // stage 2: E'(d, ra, rb) = sum alpha X_a(ia, so)^T T
        std::vector<GemmOut> o2;
        std::vector<GemmIn> i2;
        for (int p = 0; p < P; ++p) {
            const Layout& A = probs[p].a->lay;
            int q = 0;
            for (auto& kv : contrib[p]) {
                EnvBlk& nb = En[p][q++];
                nb.ptr = Ebuf + (int64_t)(intptr_t)nb.ptr;
                const int beg = (int)i2.size();
                for (auto& c : kv.second) {
                    const TBlk& tb = T[p][std::get<0>(c)];
                    const Block& ab = A.blocks[t][std::get<1>(c)];
                    i2.push_back({probs[p].a->core[t] + ab.off, Tbuf + tb.off, ab.rows, ab.cols, tb.cols, 1,
                                  std::get<2>(c)});
                }
                o2.push_back({nb.ptr, nb.rows, nb.cols, nb.cols, beg, (int)i2.size(), 0.0});
            }
        }
        launch_gemm(ctx, o2, i2);
        if (prevbuf) ctx->free(prevbuf);
        prevbuf = Ebuf;
        E.swap(En);
    }
    // bond K: sum of the remaining 1x1 blocks
    std::vector<CopyTask> g;
    Scratch s(ctx);
    double* res = s.dbl((size_t)P);
    BSM_CUDA(cudaMemsetAsync(res, 0, sizeof(double) * P, ctx->stream));
    std::vector<std::vector<CopyTask>> rounds;
    for (int p = 0; p < P; ++p)
        for (size_t e = 0; e < E[p].size(); ++e) {
            if (rounds.size() <= e) rounds.resize(e + 1);
            rounds[e].push_back({E[p][e].ptr, res + p, 1, 1, 1, 1, 0, 0, 1, 1.0});
        }
    for (auto& r : rounds) launch_copy(ctx, r);
    BSM_CUDA(cudaMemcpyAsync(result.data(), res, sizeof(double) * P, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->sync();
    if (prevbuf) ctx->free(prevbuf);
    return result;
}

// <S_a a, O S_b b> for a batch, all sites in one persistent launch.  The left
// environment E_t of a problem is a list of blocks (MPO channel c, sector ia of
// a, sector ib of b) at bond t; site t takes two phases: T = E X_b(ib, s_in)
// and E'(c', ra, rb) = sum over MPO entries (c -> c', s_out, s_in) of
// alpha X_a(ia, s_out)^T T, with alpha = w f_a f_b.  E lives in two ping-pong
// buffers, T in one buffer; the structure of every site follows on the host
// from the layouts.
// grams != nullptr: also return each problem's last environment, the Gram
// matrix of the columns of a and b.
static std::vector<double> dot_batch_impl(Context* ctx, const std::vector<EnvProblem>& probs,
                                          std::vector<std::vector<double>>* grams) {
    const int P = (int)probs.size();
    std::vector<double> result(P, 0.0);
    if (grams) grams->assign(P, {});
    if (P == 0) return result;
    const int K = probs[0].a->lay.K;
    for (int p = 0; p < P; ++p) {
        const EnvProblem& pr = probs[p];
        BSM_REQUIRE(same_space(pr.a->lay, pr.b->lay) && pr.a->lay.K == K, BSMPS_ERR_INVALID_ARG,
                    "dot of MPS of different spaces");
        if (pr.W)
            BSM_REQUIRE(pr.W->K == K && pr.W->species == pr.a->lay.species, BSMPS_ERR_INVALID_ARG,
                        "MPO and MPS act on different sites");
    }
    // Problems with the same a, b, operator and shift share every block structure
    // and differ only in the per-site scale factors: the structure is planned once
    // per group and replicated for each member with its own factors and buffers.
    std::vector<int> group_of(P, -1), rep;
    std::vector<std::vector<int>> members;
    for (int p = 0; p < P; ++p) {
        for (int g = 0; g < (int)rep.size() && group_of[p] < 0; ++g) {
            const EnvProblem& q = probs[rep[g]];
            if (q.a == probs[p].a && q.b == probs[p].b && q.W == probs[p].W &&
                (q.W == nullptr || q.shift == probs[p].shift))
                group_of[p] = g;
        }
        if (group_of[p] < 0) {
            group_of[p] = (int)rep.size();
            rep.push_back(p);
            members.emplace_back();
        }
        members[group_of[p]].push_back(p);
    }
    const int G = (int)rep.size();
    std::vector<Mpo> ids;
    ids.reserve(G);
    std::vector<const Mpo*> ops(G);
    for (int g = 0; g < G; ++g) {
        if (probs[rep[g]].W) {
            ops[g] = probs[rep[g]].W;
        } else {
            ids.push_back(identity_mpo(probs[rep[g]].a->lay));
            ops[g] = &ids.back();
        }
    }
    // factor table: the distinct per-site scale vectors of all problems
    std::vector<const std::vector<double>*> fvec;
    std::vector<double> ftab;
    auto frow = [&](const std::vector<double>* v) -> int {
        if (!v) return -1;
        for (size_t r = 0; r < fvec.size(); ++r)
            if (fvec[r] == v) return (int)r;
        BSM_REQUIRE((int)v->size() >= K, BSMPS_ERR_INVALID_ARG, "scale factors shorter than the chain");
        fvec.push_back(v);
        ftab.insert(ftab.end(), v->begin(), v->begin() + K);
        return (int)fvec.size() - 1;
    };
    std::vector<EnvMemberFac> mfac;
    std::vector<int> mem_beg(G);
    for (int g = 0; g < G; ++g) {
        mem_beg[g] = (int)mfac.size();
        for (int p : members[g])
            mfac.push_back({{frow(probs[p].fa0), frow(probs[p].fa1), frow(probs[p].fb0), frow(probs[p].fb1)}});
    }
    struct EBlk {
        int c, ia, ib, rows, cols;
        int64_t off;   // within a member's share of the E buffer
    };
    std::vector<EnvOutT> outs;
    std::vector<EnvInT> ins;
    std::vector<EnvTileT> tiles;
    std::vector<EnvGroupPhase> gph;
    std::vector<int> phase_beg{0};
    int64_t maxT = 1, maxE = 1;
    std::vector<std::vector<EBlk>> E(G);              // per group: blocks of E at the current bond
    std::vector<int64_t> E_size(G, 0), E_base(G, 0);  // per group: entries per member, start of its region
    for (int g = 0; g < G; ++g) {
        const Layout& A = probs[rep[g]].a->lay;
        const Layout& B = probs[rep[g]].b->lay;
        if (!A.bonds[0].q.empty() && !B.bonds[0].q.empty()) E[g].push_back({0, 0, 0, 1, 1, 0});
    }
    auto add_tiles = [&](int o, int n_mem) {
        for (int m = 0; m < n_mem; ++m)
            for (int m0 = 0; m0 < outs[o].M; m0 += 32)
                for (int n0 = 0; n0 < outs[o].N; n0 += 32) tiles.push_back({o, m0, n0, m});
    };
    auto group_phase = [&](int g) {
        EnvGroupPhase e{};
        e.mem_beg = mem_beg[g];
        e.n_mem = (int)members[g].size();
        e.shift = probs[rep[g]].W ? probs[rep[g]].shift : 0.0;
        gph.push_back(e);
        return (int)gph.size() - 1;
    };
    struct Contrib {
        uint64_t key;
        int seq, ti, ab, ei;
        int so, si;
    };
    struct TBlk {
        int env, sigma, rows, cols, bb;
        int64_t off;   // within a member's share of the T buffer
    };
    for (int t = 0; t < K; ++t) {
        const int eid = t == 0 ? 3 : 1 + (t % 2);   // buffer of E at bond t
        const int nid = 1 + ((t + 1) % 2);          // buffer of E at bond t + 1
        std::vector<std::vector<TBlk>> T(G);
        std::vector<int64_t> T_size(G, 0);
        std::vector<std::vector<Contrib>> contrib(G);
        // ---- structure of the site, once per group ----
        for (int g = 0; g < G; ++g) {
            const Layout& A = probs[rep[g]].a->lay;
            const Layout& B = probs[rep[g]].b->lay;
            const std::vector<int> blook = block_lookup(B, t);
            const std::vector<int> alook = block_lookup(A, t);
            std::vector<std::array<int, 2>> tidx(E[g].size(), {-1, -1});
            for (int e = 0; e < (int)E[g].size(); ++e)
                for (int si = 0; si < 2; ++si) {
                    const int bb = blook[E[g][e].ib * 2 + si];
                    if (bb < 0) continue;
                    tidx[e][si] = (int)T[g].size();
                    const Block& bk = B.blocks[t][bb];
                    T[g].push_back({e, si, E[g][e].rows, bk.cols, bb, T_size[g]});
                    T_size[g] += (int64_t)E[g][e].rows * bk.cols;
                }
            const Mpo& W = *ops[g];
            const int nch = W.bond_dim(t);
            std::vector<std::vector<int>> by_chan(nch);
            for (int e = 0; e < (int)E[g].size(); ++e) by_chan[E[g][e].c].push_back(e);
            int seq = 0;
            for (int ei = 0; ei < (int)W.entries[t].size(); ++ei) {
                const MpoEntry& me = W.entries[t][ei];
                if (me.a >= nch || by_chan[me.a].empty()) continue;
                for (int e : by_chan[me.a]) {
                    const int ab = alook[E[g][e].ia * 2 + me.so];
                    const int ti = tidx[e][me.si];
                    if (ab < 0 || ti < 0) continue;
                    const int bb = blook[E[g][e].ib * 2 + me.si];
                    const uint64_t ra = (uint64_t)A.blocks[t][ab].ri, rb = (uint64_t)B.blocks[t][bb].ri;
                    const uint64_t key = ((uint64_t)me.b << 42) | (ra << 21) | rb;
                    contrib[g].push_back({key, seq++, ti, ab, ei, me.so, me.si});
                }
            }
            std::sort(contrib[g].begin(), contrib[g].end(), [](const Contrib& x, const Contrib& y) {
                return x.key != y.key ? x.key < y.key : x.seq < y.seq;
            });
        }
        // ---- stage 1: T = E X_b (templates once per group) ----
        int64_t tot_T = 0;
        std::vector<int64_t> T_base(G, 0);
        for (int g = 0; g < G; ++g) {
            T_base[g] = tot_T;
            tot_T += (int64_t)members[g].size() * T_size[g];
            const int gp = group_phase(g);
            gph[gp].base[0] = T_base[g];
            gph[gp].stride[0] = T_size[g];
            if (eid != 3) {
                gph[gp].base[eid] = E_base[g];
                gph[gp].stride[eid] = E_size[g];
            }
            const Mps* b = probs[rep[g]].b;
            for (const TBlk& tb : T[g]) {
                const EBlk& eb = E[g][tb.env];
                const Block& bk = b->lay.blocks[t][tb.bb];
                const int o = (int)outs.size();
                outs.push_back({tb.rows, tb.cols, tb.cols, (int)ins.size(), (int)ins.size() + 1, gp, 0, tb.off});
                ins.push_back({nullptr, b->core[t] + bk.off, eb.off, 0, eid, -1, eb.cols, eb.cols, bk.cols, 0, 1.0,
                               0, -1, -1, t});
                add_tiles(o, (int)members[g].size());
            }
        }
        maxT = std::max(maxT, tot_T);
        phase_beg.push_back((int)tiles.size());
        // ---- stage 2: E'(d, ra, rb) = sum alpha X_a^T T ----
        std::vector<std::vector<EBlk>> En(G);
        std::vector<int64_t> En_size(G, 0), En_base(G, 0);
        int64_t tot_E = 0;
        for (int g = 0; g < G; ++g) {
            const Mps* a_ = probs[rep[g]].a;
            const Layout& A = a_->lay;
            const Layout& B = probs[rep[g]].b->lay;
            const Mpo& W = *ops[g];
            const bool real_op = probs[rep[g]].W != nullptr;
            const std::vector<Contrib>& cs = contrib[g];
            // blocks of E' first (their sizes fix the member stride)
            for (size_t i = 0; i < cs.size();) {
                size_t j = i;
                while (j < cs.size() && cs[j].key == cs[i].key) ++j;
                const int d = (int)(cs[i].key >> 42), ra = (int)((cs[i].key >> 21) & 0x1fffff),
                          rb = (int)(cs[i].key & 0x1fffff);
                const int rows = A.bonds[t + 1].dim[ra], cols = B.bonds[t + 1].dim[rb];
                En[g].push_back({d, ra, rb, rows, cols, En_size[g]});
                En_size[g] += (int64_t)rows * cols;
                i = j;
            }
            En_base[g] = tot_E;
            tot_E += (int64_t)members[g].size() * En_size[g];
            const int gp = group_phase(g);
            gph[gp].base[0] = T_base[g];
            gph[gp].stride[0] = T_size[g];
            gph[gp].base[nid] = En_base[g];
            gph[gp].stride[nid] = En_size[g];
            size_t q = 0;
            for (size_t i = 0; i < cs.size(); ++q) {
                size_t j = i;
                while (j < cs.size() && cs[j].key == cs[i].key) ++j;
                const EBlk& nb = En[g][q];
                const int o = (int)outs.size();
                outs.push_back({nb.rows, nb.cols, nb.cols, (int)ins.size(), 0, gp, nid, nb.off});
                for (size_t u = i; u < j; ++u) {
                    const Contrib& c = cs[u];
                    const MpoEntry& me = W.entries[t][c.ei];
                    const int sf = real_op && t == 0 && (c.ei == W.shift_entry[0] || c.ei == W.shift_entry[1]);
                    const TBlk& tb = T[g][c.ti];
                    const Block& abk = A.blocks[t][c.ab];
                    ins.push_back({a_->core[t] + abk.off, nullptr, 0, tb.off, -1, 0, abk.rows, abk.cols, tb.cols, 1,
                                   me.w, sf, c.so, c.si, t});
                }
                outs[o].end = (int)ins.size();
                add_tiles(o, (int)members[g].size());
                i = j;
            }
        }
        maxE = std::max(maxE, tot_E);
        phase_beg.push_back((int)tiles.size());
        E.swap(En);
        E_size.swap(En_size);
        E_base.swap(En_base);
    }
    // buffers
    Scratch s(ctx);
    double* base[4];
    base[0] = s.dbl((size_t)maxT);
    base[1] = s.dbl((size_t)maxE);
    base[2] = s.dbl((size_t)maxE);
    {
        std::vector<double> one(1, 1.0);
        base[3] = s.up(one);
    }
    double* res = s.dbl((size_t)P);
    GridSync* gs = (GridSync*)ctx->alloc(sizeof(GridSync));
    s.ptrs.push_back(gs);
    BSM_CUDA(cudaMemsetAsync(gs, 0, sizeof(GridSync), ctx->stream));
    // bond K: the remaining 1x1 blocks of every problem
    const int fid = 1 + (K % 2);
    std::vector<const double*> finals;
    std::vector<int> final_beg{0};
    std::vector<int> member_index(P, 0);
    for (int g = 0; g < G; ++g)
        for (size_t m = 0; m < members[g].size(); ++m) member_index[members[g][m]] = (int)m;
    for (int p = 0; p < P; ++p) {
        const int g = group_of[p];
        for (const EBlk& eb : E[g])
            finals.push_back(base[fid] + E_base[g] + (int64_t)member_index[p] * E_size[g] + eb.off);
        final_beg.push_back((int)finals.size());
    }
    if (!launch_env_sweep_t(ctx, outs, ins, tiles, phase_beg, gph, mfac, ftab, K, base, finals, final_beg, res,
                            gs)) {
        BSM_REQUIRE(!grams, BSMPS_ERR_RANK_CAP, "Gram matrices need the persistent environment sweep");
        return dot_batch_sitewise(ctx, probs);
    }
    // Gram matrices: gather every problem's last environment block (one per
    // problem: bond K has one sector and one channel) into one buffer
    std::vector<double> gh;
    double* gd = nullptr;
    std::vector<int64_t> goff(P + 1, 0);
    if (grams) {
        std::vector<CopyTask> gt;
        for (int p = 0; p < P; ++p) {
            const int g = group_of[p];
            const int da = probs[p].a->lay.columns(), db = probs[p].b->lay.columns();
            goff[p + 1] = goff[p] + (int64_t)da * db;
            BSM_REQUIRE(E[g].size() <= 1, BSMPS_ERR_INVALID_ARG, "more than one environment block at bond K");
            for (const EBlk& eb : E[g]) {
                BSM_REQUIRE(eb.rows == da && eb.cols == db, BSMPS_ERR_INVALID_ARG, "Gram block shape");
                gt.push_back({base[fid] + E_base[g] + (int64_t)member_index[p] * E_size[g] + eb.off, nullptr, da, db,
                              db, db, 0, 0, 0, 1.0});
            }
        }
        gd = s.dbl((size_t)std::max<int64_t>(goff[P], 1));
        BSM_CUDA(cudaMemsetAsync(gd, 0, sizeof(double) * std::max<int64_t>(goff[P], 1), ctx->stream));
        size_t k = 0;
        for (int p = 0; p < P; ++p)
            if (!E[group_of[p]].empty()) gt[k++].dst = gd + goff[p];
        launch_copy(ctx, gt);
        gh.assign((size_t)std::max<int64_t>(goff[P], 1), 0.0);
        BSM_CUDA(cudaMemcpyAsync(gh.data(), gd, sizeof(double) * gh.size(), cudaMemcpyDeviceToHost, ctx->stream));
    }
    GridSync h;
    BSM_CUDA(cudaMemcpyAsync(result.data(), res, sizeof(double) * P, cudaMemcpyDeviceToHost, ctx->stream));
    BSM_CUDA(cudaMemcpyAsync(&h, gs, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    ctx->sync();
    BSM_REQUIRE(h.err == 0, BSMPS_ERR_TIMEOUT, "inner-product sweep: a grid-wide wait gave up");
    if (grams)
        for (int p = 0; p < P; ++p) (*grams)[p].assign(gh.begin() + goff[p], gh.begin() + goff[p + 1]);
    return result;
}

std::vector<double> op_dot_batch(Context* ctx, const std::vector<EnvProblem>& probs) {
    return dot_batch_impl(ctx, probs, nullptr);
}

std::vector<std::vector<double>> op_gram_batch(Context* ctx, const std::vector<EnvProblem>& probs) {
    std::vector<std::vector<double>> g;
    dot_batch_impl(ctx, probs, &g);
    return g;
}

double op_core0_norm(Context* ctx, const Mps* x) {
    if (x->lay.K == 0 || x->lay.core_size[0] == 0) return 0.0;
    Scratch s(ctx);
    double* d = s.dbl(1);
    launch_sumsq(ctx, {x->core[0]}, {x->lay.core_size[0]}, d);
    double h = 0.0;
    BSM_CUDA(cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    ctx->sync();
    return std::sqrt(h);
}

}  // namespace bsm
