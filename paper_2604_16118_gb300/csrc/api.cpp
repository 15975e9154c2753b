// extern "C" entry points of the block-sparse MPS library (see include/bsmps.h).
#include <cmath>
#include <cstdint>
#include <cstring>

#include "kernels.h"
#include "problem.h"
#include "solver.h"

struct bsmps_ctx_s {
    bsm::Context c;
};
struct bsmps_mps_s {
    std::unique_ptr<bsm::Mps> m;
};
struct bsmps_mpo_s {
    bsm::Context* ctx;
    bsm::Mpo W;
};
// A recorded batch of zip-up applications: the graph, its memory and the
// outputs its launches write.
struct bsmps_plan_s {
    bsm::Context* ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bsm::PlanArena arena;
    int64_t launches = 0;
    double flops = 0.0;
    ~bsmps_plan_s() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (arena.dev) cudaFree(arena.dev);
        if (arena.host) cudaFreeHost(arena.host);
    }
};

namespace bsm {

Context* context_of(bsmps_ctx c) {
    BSM_REQUIRE(c != nullptr, BSMPS_ERR_INVALID_ARG, "null context");
    BSM_CUDA(cudaSetDevice(c->c.device));
    (void)cudaGetLastError();   // see C(): a stale error is not this call's
    return &c->c;
}

void* Context::alloc(size_t bytes) {
    if (bytes == 0) return nullptr;
    ++alloc_calls;
    const size_t granule = (bytes + 255) & ~size_t(255);
    alloc_bytes += granule;
    if (rec) {
        BSM_REQUIRE(rec->dev_used + granule <= rec->dev_cap, BSMPS_ERR_OOM,
                    "recorded graph: device arena exhausted (the recording took another path than the sizing run)");
        void* p = rec->dev + rec->dev_used;
        rec->dev_used += granule;
        return p;
    }
#ifdef BSM_NO_ALLOC_CACHE   // host-side checking builds: every block goes back to the pool
    {
        void* q = nullptr;
        BSM_CUDA(cudaMallocAsync(&q, bytes, stream));
        return q;
    }
#endif
    int c = 8;   // 256-byte minimum
    while (c <= kMaxClass && (size_t(1) << c) < bytes) ++c;
    void* p = nullptr;
    if (c > kMaxClass) {
        BSM_CUDA(cudaMallocAsync(&p, bytes, stream));
        block_class[p] = -1;
        return p;
    }
    std::vector<void*>& fl = free_blocks[c];
    if (!fl.empty()) {
        p = fl.back();
        fl.pop_back();
        cached_bytes -= size_t(1) << c;
        return p;
    }
    BSM_CUDA(cudaMallocAsync(&p, size_t(1) << c, stream));
    block_class[p] = c;
    return p;
}

void Context::free(void* p) {
    if (!p) return;
    if (rec && rec->owns(p)) return;   // arena blocks live as long as the graph
#ifdef BSM_NO_ALLOC_CACHE
    cudaFreeAsync(p, stream);
    return;
#endif
    auto it = block_class.find(p);
    if (it == block_class.end()) {
        cudaFreeAsync(p, stream);
        return;
    }
    const int c = it->second;
    if (c < 0 || cached_bytes + (size_t(1) << c) > kCacheCap) {
        block_class.erase(it);
        cudaFreeAsync(p, stream);
        return;
    }
    free_blocks[c].push_back(p);
    cached_bytes += size_t(1) << c;
}

void Context::release_cache() {
    for (auto& fl : free_blocks) {
        for (void* p : fl) {
            block_class.erase(p);
            cudaFreeAsync(p, stream);
        }
        fl.clear();
    }
    cached_bytes = 0;
}

void* Context::upload_raw(const void* src, size_t bytes) {
    void* d = alloc(bytes);
    const size_t granule = (bytes + 255) & ~size_t(255);
    upload_bytes += granule;
    if (rec) {
        // recording: the staged copy must outlive the capture (the graph's copy
        // node reads it at every launch)
        BSM_REQUIRE(rec->host_used + granule <= rec->host_cap, BSMPS_ERR_OOM,
                    "recorded graph: host staging arena exhausted");
        unsigned char* h = rec->host + rec->host_used;
        rec->host_used += granule;
        std::memcpy(h, src, bytes);
        BSM_CUDA(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, stream));
        return d;
    }
    const size_t half = kRingBytes / 2;
    if (bytes > half) {
        BSM_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, stream));
        return d;
    }
    if (!ring_host) {
        BSM_CUDA(cudaMallocHost((void**)&ring_host, kRingBytes));
        for (auto& e : half_ev) BSM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ring_head = 0;
        ring_half = 0;
    }
    if (ring_head + bytes > (size_t)(ring_half + 1) * half) {
        // leave this half: its copies complete before the event; wait for the other half's
        BSM_CUDA(cudaEventRecord(half_ev[ring_half], stream));
        half_pending[ring_half] = true;
        ring_half ^= 1;
        ring_head = (size_t)ring_half * half;
        if (half_pending[ring_half]) {
            BSM_CUDA(cudaEventSynchronize(half_ev[ring_half]));
            half_pending[ring_half] = false;
        }
    }
    unsigned char* h = ring_host + ring_head;
    std::memcpy(h, src, bytes);
    BSM_CUDA(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, stream));
    ring_head += (bytes + 255) & ~size_t(255);
    return d;
}

void Context::release_ring() {
    for (auto& e : half_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    if (ring_host) cudaFreeHost(ring_host);
    ring_host = nullptr;
}

}  // namespace bsm

namespace {

thread_local std::string g_err;

template <class F>
bsmps_status guarded(bsmps_ctx ctx, F&& f) {
    try {
        f();
        return BSMPS_OK;
    } catch (const bsm::Error& e) {
        if (ctx) ctx->c.last_error = e.what();
        g_err = e.what();
        return e.code;
    } catch (const std::bad_alloc& e) {
        if (ctx) ctx->c.last_error = "host allocation failed";
        g_err = "host allocation failed";
        return BSMPS_ERR_OOM;
    } catch (const std::exception& e) {
        if (ctx) ctx->c.last_error = e.what();
        g_err = e.what();
        return BSMPS_ERR_INVALID_ARG;
    }
}

bsm::Context* C(bsmps_ctx ctx) {
    BSM_REQUIRE(ctx != nullptr, BSMPS_ERR_INVALID_ARG, "null context");
    BSM_CUDA(cudaSetDevice(ctx->c.device));
    // an error another caller left in the runtime's last-error slot (not a
    // sticky device error, which every later call reports anyway) must not be
    // taken for the result of this call's launches
    (void)cudaGetLastError();
    return &ctx->c;
}

const bsm::Mps* M(bsmps_mps x) {
    BSM_REQUIRE(x != nullptr && x->m, BSMPS_ERR_INVALID_ARG, "null MPS handle");
    return x->m.get();
}

bsmps_mps wrap(bsm::MpsPtr p) {
    bsmps_mps h = new bsmps_mps_s;
    h->m = std::move(p);
    return h;
}

bsm::Charge target_of(int n_up, int n_dn, int spin) {
    BSM_REQUIRE(n_up >= 0 && (spin ? n_dn >= 0 : true), BSMPS_ERR_CHARGE, "negative particle number");
    return spin ? bsm::Charge{n_up, n_dn} : bsm::Charge{n_up, 0};
}

void check_params(const bsmps_solver_params* params) {
    BSM_REQUIRE(params->c > 0.0 && params->c < 1.0 && params->delta > 1.0 && params->eps_num > 0.0 &&
                    params->eps_num < 1.0 - params->c && params->t_eig > 0.0 && params->t_eig < 1.0 &&
                    params->r_max >= 0 && params->u_rel >= 0.0 && params->u_rel < 1e-3,
                BSMPS_ERR_INVALID_ARG, "solver parameters out of range");
}

}  // namespace

extern "C" {

const char* bsmps_status_string(bsmps_status s) {
    switch (s) {
        case BSMPS_OK: return "ok";
        case BSMPS_ERR_INVALID_ARG: return "invalid argument";
        case BSMPS_ERR_CHARGE: return "particle numbers or sectors not realisable";
        case BSMPS_ERR_OOM: return "device out of memory";
        case BSMPS_ERR_RANK_CAP: return "rank capacity exceeded";
        case BSMPS_ERR_NOT_SPD: return "preconditioner data not positive";
        case BSMPS_ERR_NUMERIC: return "non-finite scalar";
        case BSMPS_ERR_TIMEOUT: return "bounded device wait gave up";
        case BSMPS_ERR_CUDA: return "CUDA error";
    }
    return "unknown status";
}

bsmps_status bsmps_ctx_create(int device, void* stream, bsmps_ctx* out) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(out != nullptr, BSMPS_ERR_INVALID_ARG, "null out pointer");
        BSM_CUDA(cudaSetDevice(device));
        cudaMemPool_t pool;
        BSM_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
        uint64_t thr = UINT64_MAX;
        BSM_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        bsmps_ctx c = new bsmps_ctx_s;
        c->c.device = device;
        c->c.stream = (cudaStream_t)stream;
        *out = c;
    });
}

bsmps_status bsmps_ctx_destroy(bsmps_ctx ctx) {
    if (!ctx) return BSMPS_ERR_INVALID_ARG;
    bsmps_status s = guarded(nullptr, [&] {
        ctx->c.sync();
        for (auto& r : ctx->c.prof) {
            cudaEventDestroy(r.e0);
            cudaEventDestroy(r.e1);
        }
        for (auto e : ctx->c.event_pool) cudaEventDestroy(e);
        if (ctx->c.side) {
            cudaStreamSynchronize(ctx->c.side);
            cudaStreamDestroy(ctx->c.side);
            cudaEventDestroy(ctx->c.fork_ev);
            cudaEventDestroy(ctx->c.join_ev);
            ctx->c.side = nullptr;
        }
        ctx->c.release_ring();
        ctx->c.release_cache();
        ctx->c.sync();
        if (ctx->c.dev_err) cudaFree(ctx->c.dev_err);
        ctx->c.dev_err = nullptr;
    });
    delete ctx;
    return s;
}

bsmps_status bsmps_check_grid_wait(bsmps_ctx ctx, int skip_cta, int* timed_out) {
    return guarded(ctx, [&] {
        BSM_REQUIRE(timed_out != nullptr && skip_cta <= 1, BSMPS_ERR_INVALID_ARG, "skip_cta must be < 2");
        *timed_out = bsm::check_grid_wait(C(ctx), skip_cta < 0 ? -1 : skip_cta) != 0 ? 1 : 0;
    });
}

bsmps_status bsmps_ctx_sync(bsmps_ctx ctx) {
    return guarded(ctx, [&] { C(ctx)->sync(); });
}

const char* bsmps_last_error(bsmps_ctx ctx) { return ctx ? ctx->c.last_error.c_str() : g_err.c_str(); }

int64_t bsmps_ctx_launch_count(bsmps_ctx ctx) { return ctx ? ctx->c.launches : 0; }

int64_t bsmps_ctx_alloc_count(bsmps_ctx ctx) { return ctx ? ctx->c.alloc_calls : 0; }

bsmps_status bsmps_ctx_profile(bsmps_ctx ctx, int enable) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        c->profiling = enable != 0;
    });
}

bsmps_status bsmps_ctx_kernel_stats(bsmps_ctx ctx, int kind, int reset, int64_t* launches, double* ms,
                                    double* flops, double* bytes) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(kind >= 0 && kind < bsm::KK_COUNT, BSMPS_ERR_INVALID_ARG, "kernel kind out of range");
        c->sync();
        int64_t n = 0;
        double t = 0.0, f = 0.0, b = 0.0;
        for (auto& r : c->prof) {
            if (r.kind != kind) continue;
            float e = 0.0f;
            BSM_CUDA(cudaEventElapsedTime(&e, r.e0, r.e1));
            n++;
            t += e;
            f += r.flops;
            b += r.bytes;
        }
        if (launches) *launches = n;
        if (ms) *ms = t;
        if (flops) *flops = f;
        if (bytes) *bytes = b;
        if (reset) {
            for (auto& r : c->prof) {
                c->event_pool.push_back(r.e0);
                c->event_pool.push_back(r.e1);
            }
            c->prof.clear();
        }
    });
}

bsmps_status bsmps_ctx_set_jacobi_precond(bsmps_ctx ctx, int min_k) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(min_k >= 0, BSMPS_ERR_INVALID_ARG, "min_k must be >= 0");
        c->jacobi_precond_min = min_k;
    });
}

bsmps_status bsmps_ctx_set_gemm_emulation(bsmps_ctx ctx, int min_log2_flops) {
    return guarded(ctx, [&] {
        BSM_REQUIRE(ctx && min_log2_flops >= 0 && min_log2_flops <= 60, BSMPS_ERR_INVALID_ARG,
                    "need a context and 0 <= min_log2_flops <= 60");
        ctx->c.gemm_emulation_log2 = min_log2_flops;
    });
}

bsmps_status bsmps_gemm_ozaki(bsmps_ctx ctx, int M, int N, int K, const double* A, int lda, const double* B,
                              int ldb, double* Cm, int ldc, int slices) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(M >= 0 && N >= 0 && K >= 0 && lda >= K && ldb >= N && ldc >= N, BSMPS_ERR_INVALID_ARG,
                    "emulated GEMM: need sizes >= 0 and leading dimensions >= row lengths");
        BSM_REQUIRE(M == 0 || N == 0 || (Cm && (K == 0 || (A && B))), BSMPS_ERR_INVALID_ARG, "null matrix");
        bsm::launch_gemm_ozaki(c, M, N, K, A, lda, B, ldb, Cm, ldc, slices, 1.0);
    });
}

bsmps_status bsmps_gemm_tf32x3(bsmps_ctx ctx, int M, int N, int K, const double* A, int lda, const double* B,
                              int ldb, double* Cm, int ldc) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(M >= 0 && N >= 0 && K >= 0 && lda >= K && ldb >= N && ldc >= N, BSMPS_ERR_INVALID_ARG,
                    "split-precision GEMM: need sizes >= 0 and leading dimensions >= row lengths");
        BSM_REQUIRE(M == 0 || N == 0 || (Cm && (K == 0 || (A && B))), BSMPS_ERR_INVALID_ARG, "null matrix");
        if (M == 0 || N == 0) return;
        std::vector<bsm::GemmOut> outs{{Cm, M, N, ldc, 0, K > 0 ? 1 : 0, 0.0}};
        std::vector<bsm::GemmIn> ins;
        if (K > 0) ins.push_back({A, B, K, lda, ldb, 0, 1.0});
        bsm::launch_gemm_tf32x3(c, outs, ins, bsm::KK_GEMM);
    });
}

bsmps_status bsmps_ctx_set_precision(bsmps_ctx ctx, int precision) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(precision == BSMPS_PREC_FP64 || precision == BSMPS_PREC_TF32X3, BSMPS_ERR_INVALID_ARG,
                    "precision must be BSMPS_PREC_FP64 or BSMPS_PREC_TF32X3");
        c->apply_precision = precision;
    });
}

bsmps_status bsmps_mps_joint_random_size(int n_orb, int spin, int n_up, int n_dn, int r_max, int D,
                                         int64_t* n_values) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(n_orb > 0 && r_max > 0 && D >= 1 && n_values, BSMPS_ERR_INVALID_ARG,
                    "n_orb, r_max, D > 0 required");
        bsm::Layout L = bsm::default_layout(bsm::species_of(n_orb, spin), target_of(n_up, n_dn, spin), r_max, D);
        *n_values = L.total();
    });
}

bsmps_status bsmps_mps_create_joint(bsmps_ctx ctx, int n_orb, int spin, int n_up, int n_dn, int D, int init,
                                    const unsigned char* occ, int r_max, const double* values, int64_t n_values,
                                    bsmps_mps* out) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(n_orb > 0 && D >= 1 && out && (init == 0 || init == 1), BSMPS_ERR_INVALID_ARG,
                    "n_orb > 0, D >= 1, init in {0, 1} and out required");
        const auto species = bsm::species_of(n_orb, spin);
        const bsm::Charge tgt = target_of(n_up, n_dn, spin);
        bsm::Layout L;
        std::vector<double> vals;
        const double* src = values;
        if (init == 0) {
            L = bsm::determinant_layout(species, tgt, occ, D, &vals);
            src = vals.data();
        } else {
            BSM_REQUIRE(r_max > 0, BSMPS_ERR_INVALID_ARG, "r_max > 0 required");
            L = bsm::default_layout(species, tgt, r_max, D);
            BSM_REQUIRE(values && n_values == L.total(), BSMPS_ERR_INVALID_ARG,
                        "values must hold exactly bsmps_mps_joint_random_size entries");
        }
        bsm::check_layout(L);
        bsm::MpsPtr x(bsm::new_mps(c, L, false));
        bsm::mps_upload(x.get(), src);
        *out = wrap(std::move(x));
    });
}

bsmps_status bsmps_mps_num_columns(bsmps_mps x, int* D) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(x && D, BSMPS_ERR_INVALID_ARG, "null argument");
        *D = M(x)->lay.columns();
    });
}

bsmps_status bsmps_gram(bsmps_ctx ctx, bsmps_mps a, bsmps_mps b, bsmps_mpo W, double shift, double* out) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(a && b && out, BSMPS_ERR_INVALID_ARG, "null argument");
        bsm::EnvProblem pr{M(a), M(b), W ? &W->W : nullptr, shift};
        const auto g = bsm::op_gram_batch(c, {pr});
        std::copy(g[0].begin(), g[0].end(), out);
    });
}

bsmps_status bsmps_apply_columns(bsmps_ctx ctx, bsmps_mpo W, bsmps_mps x, double shift, const double* col_shift,
                                 bsmps_mps* y) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(W && x && col_shift && y, BSMPS_ERR_INVALID_ARG, "null argument");
        const std::vector<double> cs(col_shift, col_shift + M(x)->lay.columns());
        const std::vector<std::vector<double>> none(1);
        std::vector<bsm::MpsPtr> r = bsm::op_apply_exact_scaled(c, W->W, M(x), shift, none, none, &cs);
        c->sync();
        *y = wrap(std::move(r[0]));
    });
}

bsmps_status bsmps_mix_columns(bsmps_ctx ctx, bsmps_mps x, const double* Wm, int D_out, bsmps_mps* y) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(x && Wm && D_out >= 1 && y, BSMPS_ERR_INVALID_ARG, "null argument or D_out < 1");
        const int din = M(x)->lay.columns();
        bsm::ConcatTerm t{M(x), {}, {}, std::vector<double>(Wm, Wm + (size_t)din * D_out), D_out};
        bsm::MpsPtr r = bsm::op_concat(c, {t});
        c->sync();
        *y = wrap(std::move(r));
    });
}

bsmps_status bsmps_precond_theta(int n_orb, const double* h, const double* eri, int spin, int n_particles,
                                 double gamma, double* theta) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(n_orb > 0 && h && eri && theta && n_particles > 0, BSMPS_ERR_INVALID_ARG,
                    "n_orb, n_particles > 0 and h, eri, theta required");
        const std::vector<double> th = bsm::precond_theta(n_orb, h, eri, spin ? 1 : 0, n_particles, gamma);
        std::memcpy(theta, th.data(), th.size() * sizeof(double));
    });
}

bsmps_status bsmps_precond_interval(int n_orb, int spin, const double* theta, const double* h, int n_up, int n_dn,
                                    double* t_min, double* t_max) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(n_orb > 0 && theta && t_min && t_max && n_up >= 0 && n_dn >= 0, BSMPS_ERR_INVALID_ARG,
                    "n_orb > 0, theta, t_min, t_max required");
        bsm::precond_interval(n_orb, spin ? 1 : 0, theta, h, n_up, spin ? n_dn : 0, t_min, t_max);
    });
}

bsmps_status bsmps_energy_lower_bound(int n_orb, const double* h, const double* eri, int spin, int n_up, int n_dn,
                                      int cholesky, double* e_lb) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(n_orb > 0 && h && e_lb && (eri || !cholesky), BSMPS_ERR_INVALID_ARG,
                    "n_orb > 0, h, e_lb (and eri when cholesky) required");
        BSM_REQUIRE(n_up >= 0 && n_up <= n_orb && n_dn >= 0 && n_dn <= n_orb, BSMPS_ERR_INVALID_ARG,
                    "particle numbers out of range");
        *e_lb = bsm::energy_lower_bound(n_orb, h, eri, spin ? 1 : 0, n_up, n_dn, cholesky);
    });
}

bsmps_status bsmps_precond_alpha0(double c0, double t_min, double c_lower, double c_upper, double* alpha0,
                                  double* c) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(c0 > 0.0 && c0 < 1.0 && t_min > 0.0 && c_lower > 0.0 && c_upper > 0.0 && alpha0 && c,
                    BSMPS_ERR_INVALID_ARG, "need c0 in (0, 1), t_min > 0, C_lower, C_upper > 0");
        bsm::precond_alpha0(c0, t_min, c_lower, c_upper, alpha0, c);
    });
}

bsmps_status bsmps_lowest_determinants(int K, const double* t_diag, int spin, int n_up, int n_dn, int D,
                                       int64_t max_configs, unsigned char* occ) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(K > 0 && t_diag && occ && D > 0, BSMPS_ERR_INVALID_ARG, "K, D > 0, t_diag, occ required");
        bsm::lowest_determinants(K, t_diag, spin ? 1 : 0, n_up, spin ? n_dn : 0, D, max_configs, occ);
    });
}

bsmps_status bsmps_mps_random_size(int n_orb, int spin, int n_up, int n_dn, int r_max, int64_t* n_values) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(n_orb > 0 && r_max > 0 && n_values, BSMPS_ERR_INVALID_ARG, "n_orb, r_max > 0 required");
        bsm::Layout L = bsm::default_layout(bsm::species_of(n_orb, spin), target_of(n_up, n_dn, spin), r_max);
        *n_values = L.total();
    });
}

bsmps_status bsmps_mps_create(bsmps_ctx ctx, int n_orb, int spin, int n_up, int n_dn, int r_max, int init,
                              const double* values, int64_t n_values, bsmps_mps* out) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(n_orb > 0 && out, BSMPS_ERR_INVALID_ARG, "n_orb > 0 and out required");
        const auto species = bsm::species_of(n_orb, spin);
        const bsm::Charge tgt = target_of(n_up, n_dn, spin);
        bsm::Layout L;
        std::vector<double> ones;
        const double* src = values;
        if (init == 0) {
            L = bsm::e1_layout(species, tgt);
            ones.assign((size_t)L.total(), 1.0);
            src = ones.data();
        } else {
            BSM_REQUIRE(r_max > 0, BSMPS_ERR_INVALID_ARG, "r_max > 0 required");
            L = bsm::default_layout(species, tgt, r_max);
            BSM_REQUIRE(values && n_values == L.total(), BSMPS_ERR_INVALID_ARG,
                        "values must hold exactly bsmps_mps_random_size entries");
        }
        bsm::MpsPtr x(bsm::new_mps(c, L, false));
        bsm::mps_upload(x.get(), src);
        *out = wrap(std::move(x));
    });
}

bsmps_status bsmps_mps_import(bsmps_ctx ctx, int n_orb, int spin, int n_up, int n_dn, const int* n_sectors,
                              const int* sectors, const double* values, int64_t n_values, bsmps_mps* out) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(n_orb > 0 && n_sectors && sectors && out, BSMPS_ERR_INVALID_ARG, "null argument");
        bsm::Layout L;
        L.species = bsm::species_of(n_orb, spin);
        L.K = (int)L.species.size();
        L.target = target_of(n_up, n_dn, spin);
        L.bonds.resize(L.K + 1);
        int64_t pos = 0;
        for (int b = 0; b <= L.K; ++b) {
            BSM_REQUIRE(n_sectors[b] >= 0, BSMPS_ERR_INVALID_ARG, "negative sector count");
            for (int i = 0; i < n_sectors[b]; ++i, ++pos) {
                L.bonds[b].q.push_back({sectors[3 * pos], sectors[3 * pos + 1]});
                L.bonds[b].dim.push_back(sectors[3 * pos + 2]);
            }
        }
        bsm::check_layout(L);
        L.rebuild_blocks();
        BSM_REQUIRE(n_values == L.total() && (values || n_values == 0), BSMPS_ERR_INVALID_ARG,
                    "values must match the sector dims");
        bsm::MpsPtr x(bsm::new_mps(c, L, false));
        if (n_values > 0) bsm::mps_upload(x.get(), values);
        *out = wrap(std::move(x));
    });
}

bsmps_status bsmps_mps_num_sites(bsmps_mps x, int* K) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(K, BSMPS_ERR_INVALID_ARG, "null out");
        *K = M(x)->lay.K;
    });
}

bsmps_status bsmps_mps_num_sectors(bsmps_mps x, int* per_bond, int* total) {
    return guarded(nullptr, [&] {
        const bsm::Layout& L = M(x)->lay;
        int tot = 0;
        for (int b = 0; b <= L.K; ++b) {
            if (per_bond) per_bond[b] = (int)L.bonds[b].q.size();
            tot += (int)L.bonds[b].q.size();
        }
        if (total) *total = tot;
    });
}

bsmps_status bsmps_mps_sectors(bsmps_mps x, int* triples) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(triples, BSMPS_ERR_INVALID_ARG, "null out");
        const bsm::Layout& L = M(x)->lay;
        int64_t pos = 0;
        for (int b = 0; b <= L.K; ++b)
            for (size_t i = 0; i < L.bonds[b].q.size(); ++i, ++pos) {
                triples[3 * pos] = L.bonds[b].q[i].q0;
                triples[3 * pos + 1] = L.bonds[b].q[i].q1;
                triples[3 * pos + 2] = L.bonds[b].dim[i];
            }
    });
}

bsmps_status bsmps_mps_size(bsmps_mps x, int64_t* n) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(n, BSMPS_ERR_INVALID_ARG, "null out");
        *n = M(x)->lay.total();
    });
}

bsmps_status bsmps_mps_export(bsmps_mps x, double* values) {
    return guarded(nullptr, [&] {
        const bsm::Mps* m = M(x);
        BSM_REQUIRE(values || m->lay.total() == 0, BSMPS_ERR_INVALID_ARG, "null out");
        BSM_CUDA(cudaSetDevice(m->ctx->device));
        bsm::mps_download(m, values);
    });
}

bsmps_status bsmps_mps_destroy(bsmps_mps x) {
    if (!x) return BSMPS_ERR_INVALID_ARG;
    return guarded(nullptr, [&] {
        if (x->m) BSM_CUDA(cudaSetDevice(x->m->ctx->device));
        delete x;
    });
}

bsmps_status bsmps_mpo_from_integrals(bsmps_ctx ctx, int n_orb, const double* h, const double* eri, int spin,
                                      int n_particles, double gamma, double compress_tol, bsmps_mpo* out) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(out, BSMPS_ERR_INVALID_ARG, "null out");
        BSM_REQUIRE(n_particles > 0, BSMPS_ERR_CHARGE, "n_particles must be positive");
        bsmps_mpo W = new bsmps_mpo_s;
        W->ctx = c;
        try {
            W->W = bsm::build_mpo(n_orb, h, eri, spin, n_particles, gamma, compress_tol);
        } catch (...) {
            delete W;
            throw;
        }
        *out = W;
    });
}

bsmps_status bsmps_mpo_bond_dims(bsmps_mpo W, int* dims) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(W && dims, BSMPS_ERR_INVALID_ARG, "null argument");
        for (int b = 0; b <= W->W.K; ++b) dims[b] = W->W.bond_dim(b);
    });
}

bsmps_status bsmps_mpo_num_entries(bsmps_mpo W, int site, int* n) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(W && n && site >= 0 && site < W->W.K, BSMPS_ERR_INVALID_ARG, "bad argument");
        *n = (int)W->W.entries[site].size();
    });
}

bsmps_status bsmps_mpo_entries(bsmps_mpo W, int site, int* quads, double* w) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(W && quads && w && site >= 0 && site < W->W.K, BSMPS_ERR_INVALID_ARG, "bad argument");
        const auto& E = W->W.entries[site];
        for (size_t i = 0; i < E.size(); ++i) {
            quads[4 * i] = E[i].a;
            quads[4 * i + 1] = E[i].b;
            quads[4 * i + 2] = E[i].so;
            quads[4 * i + 3] = E[i].si;
            w[i] = E[i].w;
        }
    });
}

bsmps_status bsmps_mpo_channel_charges(bsmps_mpo W, int bond, int* pairs) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(W && pairs && bond >= 0 && bond <= W->W.K, BSMPS_ERR_INVALID_ARG, "bad argument");
        const auto& ch = W->W.charges[bond];
        for (size_t i = 0; i < ch.size(); ++i) {
            pairs[2 * i] = ch[i].q0;
            pairs[2 * i + 1] = ch[i].q1;
        }
    });
}

bsmps_status bsmps_mpo_destroy(bsmps_mpo W) {
    if (!W) return BSMPS_ERR_INVALID_ARG;
    delete W;
    return BSMPS_OK;
}

bsmps_status bsmps_apply_H(bsmps_ctx ctx, bsmps_mpo W, bsmps_mps x, double shift, double tol, int r_max,
                           bsmps_mps* y, double* flops) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(W && y, BSMPS_ERR_INVALID_ARG, "null argument");
        BSM_REQUIRE(tol >= 0.0 && r_max >= 0, BSMPS_ERR_INVALID_ARG, "tol >= 0 and r_max >= 0 required");
        const double f0 = c->flops;
        bsm::MpsPtr r;
        if (tol == 0.0 && r_max == 0) {
            r = bsm::op_apply_exact(c, W->W, M(x), shift);
        } else {
            // zip-up application (left-orthogonal result), then the right SVD sweep of trunc_tol
            std::vector<bsm::MpsPtr> u = bsm::op_apply_zipup_scaled(c, W->W, M(x), shift, {{}}, {{}});
            std::vector<bsm::MpsPtr> t = bsm::op_truncate_batch_left_orthogonal(c, {u[0].get()}, {tol}, r_max);
            r = std::move(t[0]);
        }
        c->sync();
        if (flops) *flops = c->flops - f0;
        *y = wrap(std::move(r));
    });
}

bsmps_status bsmps_apply_zipup(bsmps_ctx ctx, bsmps_mpo W, bsmps_mps x, double shift, bsmps_mps* y, double* flops) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(W && y, BSMPS_ERR_INVALID_ARG, "null argument");
        const double f0 = c->flops;
        std::vector<bsm::MpsPtr> u = bsm::op_apply_zipup_scaled(c, W->W, M(x), shift, {{}}, {{}});
        c->sync();
        if (flops) *flops = c->flops - f0;
        *y = wrap(std::move(u[0]));
    });
}

bsmps_status bsmps_apply_zipup_batch(bsmps_ctx ctx, int n, const bsmps_mpo* W, const bsmps_mps* x,
                                     const double* shift, bsmps_mps* y, double* flops) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(n >= 0 && (n == 0 || (W && x && shift && y)), BSMPS_ERR_INVALID_ARG, "null argument");
        std::vector<bsm::ZipProblem> probs;
        for (int i = 0; i < n; ++i) {
            BSM_REQUIRE(W[i] && x[i], BSMPS_ERR_INVALID_ARG, "null handle in the batch");
            probs.push_back({&W[i]->W, M(x[i]), shift[i], {{}}, {{}}});
        }
        const double f0 = c->flops;
        std::vector<std::vector<bsm::MpsPtr>> r = bsm::op_apply_zipup_batch(c, probs);
        c->sync();
        if (flops) *flops = c->flops - f0;
        for (int i = 0; i < n; ++i) y[i] = wrap(std::move(r[i][0]));
    });
}

bsmps_status bsmps_mps_write(bsmps_mps x, const double* values, int64_t n_values) {
    return guarded(nullptr, [&] {
        BSM_REQUIRE(x && x->m, BSMPS_ERR_INVALID_ARG, "null MPS handle");
        bsm::Mps* m = x->m.get();
        BSM_REQUIRE(n_values == m->lay.total() && (values || n_values == 0), BSMPS_ERR_INVALID_ARG,
                    "values must match the sector dims");
        BSM_CUDA(cudaSetDevice(m->ctx->device));
        bsm::mps_upload(m, values);
    });
}

bsmps_status bsmps_plan_apply_zipup_batch(bsmps_ctx ctx, int n, const bsmps_mpo* W, const bsmps_mps* x,
                                          const double* shift, bsmps_plan* plan, bsmps_mps* y, double* flops) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(n > 0 && W && x && shift && y && plan, BSMPS_ERR_INVALID_ARG, "null argument");
        BSM_REQUIRE(c->stream != nullptr, BSMPS_ERR_INVALID_ARG,
                    "recording a plan needs a context on a non-default stream");
        BSM_REQUIRE(c->rec == nullptr, BSMPS_ERR_INVALID_ARG, "the context is already recording");
        std::vector<bsm::ZipProblem> probs;
        for (int i = 0; i < n; ++i) {
            BSM_REQUIRE(W[i] && x[i], BSMPS_ERR_INVALID_ARG, "null handle in the batch");
            probs.push_back({&W[i]->W, M(x[i]), shift[i], {{}}, {{}}});
        }
        // sizing run: the same batch, uncaptured; it also tunes every contraction
        // size class, so the recording makes no timing runs
        const size_t a0 = c->alloc_bytes, u0 = c->upload_bytes;
        {
            std::vector<std::vector<bsm::MpsPtr>> r = bsm::op_apply_zipup_batch(c, probs);
        }
        c->sync();
        c->err_word();   // created outside the capture
        std::unique_ptr<bsmps_plan_s> P(new bsmps_plan_s);
        P->ctx = c;
        P->arena.dev_cap = c->alloc_bytes - a0 + (size_t(1) << 20);
        P->arena.host_cap = c->upload_bytes - u0 + (size_t(1) << 16);
        BSM_CUDA(cudaMalloc((void**)&P->arena.dev, P->arena.dev_cap));
        BSM_CUDA(cudaMallocHost((void**)&P->arena.host, P->arena.host_cap));
        const bool prof = c->profiling;
        const int64_t l0 = c->launches;
        const double f0 = c->flops;
        std::vector<std::vector<bsm::MpsPtr>> r;
        c->profiling = false;
        c->rec = &P->arena;
        BSM_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
        try {
            r = bsm::op_apply_zipup_batch(c, probs);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(c->stream, &g);
            if (g) cudaGraphDestroy(g);
            c->rec = nullptr;
            c->profiling = prof;
            throw;
        }
        const cudaError_t ec = cudaStreamEndCapture(c->stream, &P->graph);
        c->rec = nullptr;
        c->profiling = prof;
        BSM_CUDA(ec);
        BSM_CUDA(cudaGraphInstantiate(&P->exec, P->graph, 0));
        P->launches = c->launches - l0;
        P->flops = c->flops - f0;
        c->launches = l0;   // nothing ran yet: launches count at bsmps_plan_launch
        c->flops = f0;
        if (flops) *flops = P->flops;
        for (int i = 0; i < n; ++i) {
            r[i][0]->owns_cores = false;
            y[i] = wrap(std::move(r[i][0]));
        }
        *plan = P.release();
    });
}

bsmps_status bsmps_plan_launch(bsmps_plan plan) {
    if (!plan) return BSMPS_ERR_INVALID_ARG;
    return guarded(nullptr, [&] {
        bsm::Context* c = plan->ctx;
        BSM_CUDA(cudaSetDevice(c->device));
        BSM_CUDA(cudaGraphLaunch(plan->exec, c->stream));
        c->launches += plan->launches;
        c->flops += plan->flops;
    });
}

int64_t bsmps_plan_launch_count(bsmps_plan plan) { return plan ? plan->launches : -1; }

bsmps_status bsmps_plan_destroy(bsmps_plan plan) {
    if (!plan) return BSMPS_ERR_INVALID_ARG;
    return guarded(nullptr, [&] {
        BSM_CUDA(cudaSetDevice(plan->ctx->device));
        BSM_CUDA(cudaStreamSynchronize(plan->ctx->stream));
        delete plan;
    });
}

bsmps_status bsmps_truncate(bsmps_ctx ctx, bsmps_mps x, double eps, int r_max, bsmps_mps* y, double* disc_tol,
                            double* disc_cap) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(y && eps >= 0.0 && r_max >= 0, BSMPS_ERR_INVALID_ARG, "bad argument");
        bsm::MpsPtr r = bsm::op_truncate(c, M(x), eps, r_max, disc_tol, disc_cap);
        c->sync();
        *y = wrap(std::move(r));
    });
}

bsmps_status bsmps_add(bsmps_ctx ctx, bsmps_mps x, bsmps_mps y, double alpha, double beta, bsmps_mps* out) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(out, BSMPS_ERR_INVALID_ARG, "null out");
        const int K = M(x)->lay.K;
        std::vector<double> a(K, 1.0), b(K, 1.0);
        a[0] = alpha;
        b[0] = beta;
        bsm::MpsPtr r = bsm::op_concat(c, {{M(x), a, a}, {M(y), b, b}});
        c->sync();
        *out = wrap(std::move(r));
    });
}

bsmps_status bsmps_scale_sites(bsmps_ctx ctx, bsmps_mps x, const double* f0, const double* f1, bsmps_mps* out) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(out && f0 && f1, BSMPS_ERR_INVALID_ARG, "null argument");
        const int K = M(x)->lay.K;
        bsm::MpsPtr r = bsm::op_scale_sites(c, M(x), std::vector<double>(f0, f0 + K),
                                            std::vector<double>(f1, f1 + K));
        c->sync();
        *out = wrap(std::move(r));
    });
}

bsmps_status bsmps_precondition(bsmps_ctx ctx, const bsmps_precond* p, int term, bsmps_mps x, bsmps_mps* y,
                                int* n_terms) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(y, BSMPS_ERR_INVALID_ARG, "null out");
        const bsm::PrecondTerms P = bsm::make_precond(p);
        BSM_REQUIRE(p->K == M(x)->lay.K, BSMPS_ERR_INVALID_ARG, "precond K differs from the MPS");
        if (n_terms) *n_terms = P.n_terms();
        BSM_REQUIRE(term >= -1 && term < P.n_terms(), BSMPS_ERR_INVALID_ARG, "term out of range");
        bsm::MpsPtr r;
        if (term >= 0) {
            r = bsm::op_scale_sites(c, M(x), P.f0[term], P.f1[term]);
        } else {
            std::vector<bsm::ConcatTerm> terms;
            for (int k = 0; k < P.n_terms(); ++k) terms.push_back({M(x), P.f0[k], P.f1[k]});
            r = bsm::op_concat(c, terms);
        }
        c->sync();
        *y = wrap(std::move(r));
    });
}

bsmps_status bsmps_dot(bsmps_ctx ctx, bsmps_mps a, bsmps_mps b, bsmps_mpo W, double shift, double* out) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(out, BSMPS_ERR_INVALID_ARG, "null out");
        BSM_REQUIRE(M(a)->lay.columns() == 1 && M(b)->lay.columns() == 1, BSMPS_ERR_INVALID_ARG,
                    "joint block MPS: use bsmps_gram");
        bsm::EnvProblem pr{M(a), M(b), W ? &W->W : nullptr, shift};
        *out = bsm::op_dot_batch(c, {pr})[0];
    });
}

bsmps_status bsmps_dot_noalloc(bsmps_ctx ctx, bsmps_mps a, bsmps_mps b, bsmps_mpo W, double shift,
                               double* out) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(out, BSMPS_ERR_INVALID_ARG, "null out");
        BSM_REQUIRE(M(a)->lay.columns() == 1 && M(b)->lay.columns() == 1, BSMPS_ERR_INVALID_ARG,
                    "joint block MPS: use bsmps_gram");
        *out = bsm::op_dot_noalloc(c, M(a), M(b), W ? &W->W : nullptr, shift);
    });
}

bsmps_status bsmps_eigensolve_outer(bsmps_ctx ctx, bsmps_mpo W, const bsmps_precond* p,
                                    const bsmps_solver_params* params, double alpha, double tau, int max_outer,
                                    int max_inner, bsmps_mps* x, bsmps_outer_record* records, int* n_outer,
                                    int* converged) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(W && params && x && *x && n_outer && converged, BSMPS_ERR_INVALID_ARG, "null argument");
        BSM_REQUIRE(params->c > 0.0 && params->c < 1.0 && params->delta > 1.0 && params->eps_num > 0.0 &&
                        params->eps_num < 1.0 - params->c && params->t_eig > 0.0 && params->t_eig < 1.0 &&
                        params->r_max >= 0 && params->u_rel >= 0.0 && params->u_rel < 1e-3,
                    BSMPS_ERR_INVALID_ARG, "solver parameters out of range");
        BSM_REQUIRE(alpha > 0.0 && tau > 0.0 && max_outer > 0 && max_inner > 0, BSMPS_ERR_INVALID_ARG,
                    "alpha, tau, max_outer and max_inner must be positive");
        const bsm::PrecondTerms P = bsm::make_precond(p);
        BSM_REQUIRE(p->K == M(*x)->lay.K, BSMPS_ERR_INVALID_ARG, "precond K differs from the MPS");
        std::vector<bsmps_outer_record> recs;
        bool ok = false;
        bsm::MpsPtr r = bsm::eigensolve_outer(c, W->W, P, *params, alpha, tau, max_outer, max_inner, M(*x), recs, &ok);
        c->sync();
        if (records)
            for (size_t i = 0; i < recs.size(); ++i) records[i] = recs[i];
        *n_outer = (int)recs.size();
        *converged = ok ? 1 : 0;
        bsmps_mps old = *x;
        *x = wrap(std::move(r));
        delete old;
    });
}

bsmps_status bsmps_eigensolve_joint_step(bsmps_ctx ctx, bsmps_mpo W, const bsmps_precond* p,
                                         const bsmps_solver_params* params, bsmps_solver_state* state, bsmps_mps* x,
                                         bsmps_joint_step_info* info) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(W && params && state && x && *x && info, BSMPS_ERR_INVALID_ARG, "null argument");
        check_params(params);
        const bsm::PrecondTerms P = bsm::make_precond(p);
        BSM_REQUIRE(p->K == M(*x)->lay.K, BSMPS_ERR_INVALID_ARG, "precond K differs from the MPS");
        bsmps_joint_step_info inf;
        bsmps_solver_state st = *state;
        bsm::MpsPtr r = bsm::eigensolve_joint_step(c, W->W, P, *params, st, M(*x), inf);
        c->sync();
        *state = st;
        *info = inf;
        bsmps_mps old = *x;
        *x = wrap(std::move(r));
        delete old;
    });
}

bsmps_status bsmps_eigensolve_step(bsmps_ctx ctx, bsmps_mpo W, const bsmps_precond* p,
                                   const bsmps_solver_params* params, bsmps_solver_state* state, bsmps_mps* x,
                                   bsmps_step_info* info) {
    return guarded(ctx, [&] {
        bsm::Context* c = C(ctx);
        BSM_REQUIRE(W && params && state && x && *x && info, BSMPS_ERR_INVALID_ARG, "null argument");
        check_params(params);
        const bsm::PrecondTerms P = bsm::make_precond(p);
        BSM_REQUIRE(p->K == M(*x)->lay.K, BSMPS_ERR_INVALID_ARG, "precond K differs from the MPS");
        BSM_REQUIRE(M(*x)->lay.columns() == 1, BSMPS_ERR_INVALID_ARG,
                    "joint block MPS: use bsmps_eigensolve_joint_step");
        bsmps_step_info inf;
        bsmps_solver_state st = *state;
        bsm::MpsPtr r = bsm::eigensolve_step(c, W->W, P, *params, st, M(*x), inf);
        c->sync();
        *state = st;
        *info = inf;
        bsmps_mps old = *x;
        *x = wrap(std::move(r));
        delete old;
    });
}

}  // extern "C"
