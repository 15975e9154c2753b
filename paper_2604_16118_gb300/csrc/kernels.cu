// Device kernels: block scatter/copy, segmented FP64 grouped GEMM, batched
// Householder QR and batched one-sided Jacobi SVD for the small dense blocks of
// a block-sparse MPS.  All arithmetic is float64.
#include <cfloat>
#include <cmath>
#include <cstring>

#include "dense_dev.cuh"
#include "kernels.h"

namespace bsm {
namespace {

using dev::block_sum;
using dev::kThreads;
using dev::kWarps;
using dev::warp_sum;

constexpr int64_t kCopyChunk = 16384;

struct CopyChunk {
    int task;
    int64_t beg, end;
};

__global__ void __launch_bounds__(kThreads) k_copy(const CopyTask* __restrict__ tasks,
                                                   const CopyChunk* __restrict__ chunks) {
    const CopyChunk ch = chunks[blockIdx.x];
    const CopyTask tk = tasks[ch.task];
    for (int64_t e = ch.beg + threadIdx.x; e < ch.end; e += blockDim.x) {
        const int i = (int)(e / tk.cols), j = (int)(e % tk.cols);
        const int64_t si = tk.src_cm ? (int64_t)j * tk.src_ld + i : (int64_t)i * tk.src_ld + j;
        const int64_t di = tk.dst_cm ? (int64_t)j * tk.dst_ld + i : (int64_t)i * tk.dst_ld + j;
        const double v = tk.f * tk.src[si];
        if (tk.accumulate)
            tk.dst[di] += v;
        else
            tk.dst[di] = v;
    }
}

struct GemmTile {
    int out, m0, n0;
};

constexpr int kTile = dev::kGemmTile;
constexpr int kSmallGemmThreads = 128;

// 32 x 32 output tile per CTA; thread (ty, tx) owns rows ty + 8 r (r < 4), column tx.
__global__ void __launch_bounds__(kThreads) k_gemm(const GemmOut* __restrict__ outs,
                                                   const GemmIn* __restrict__ ins,
                                                   const GemmTile* __restrict__ tiles) {
    __shared__ double As[kTile][kTile + 1];   // [k][m]
    __shared__ double Bs[kTile][kTile + 1];   // [k][n]
    const GemmTile tl = tiles[blockIdx.x];
    const GemmOut o = outs[tl.out];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = o.beg; c < o.end; ++c) dev::gemm_tile_accumulate(ins[c], o.M, o.N, tl.m0, tl.n0, As, Bs, acc);
    const int gn = tl.n0 + tx;
    if (gn >= o.N) return;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gm = tl.m0 + ty + 8 * r;
        if (gm < o.M) {
            double* cp = o.C + (int64_t)gm * o.ldc + gn;
            *cp = o.beta == 0.0 ? acc[r] : o.beta * (*cp) + acc[r];
        }
    }
}

// Small outputs (M, N <= 32): one CTA per output, one thread per output
// element, the K loop reading A and B directly, so that no FP64 instruction is
// spent on tile padding.
__global__ void __launch_bounds__(kSmallGemmThreads) k_gemm_small(const GemmOut* __restrict__ outs,
                                                                  const GemmIn* __restrict__ ins,
                                                                  const int* __restrict__ ids) {
    const GemmOut o = outs[ids[blockIdx.x]];
    const int n_el = o.M * o.N;
    for (int e = threadIdx.x; e < n_el; e += kSmallGemmThreads) {
        const int m = e / o.N, n = e % o.N;
        double acc = 0.0;
        for (int c = o.beg; c < o.end; ++c) {
            const GemmIn in = ins[c];
            double part = 0.0;
            if (in.transA)
                part = dev::dot_global<false, false>(in.A + m, in.lda, in.B + n, in.ldb, in.K, 0.0);
            else
                part = dev::dot_global<false, false>(in.A + (int64_t)m * in.lda, 1, in.B + n, in.ldb, in.K, 0.0);
            acc = fma(in.alpha, part, acc);
        }
        double* cp = o.C + (int64_t)m * o.ldc + n;
        *cp = o.beta == 0.0 ? acc : o.beta * (*cp) + acc;
    }
}

// Householder QR, one CTA per matrix; the working set (A, Q, tau) lives in
// shared memory when it fits (smem = 1), else in global memory.  Reflector
// H = I - tau v v^T with v_j = 1, beta = -sign(alpha) ||x||,
// tau = (beta - alpha)/beta, v = x/(alpha - beta).
__global__ void __launch_bounds__(kThreads) k_qr(const QrTask* __restrict__ tasks) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ double sh[2];
    const QrTask tk = tasks[blockIdx.x];
    const int M = tk.M, N = tk.N, k = M < N ? M : N;
    double* A = tk.smem ? sm : tk.A;
    double* Q = tk.smem ? sm + (int64_t)M * N : tk.Q;
    double* tau = tk.smem ? sm + (int64_t)M * N + (int64_t)M * k : tk.tau;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (tk.smem) {
        for (int64_t e = threadIdx.x; e < (int64_t)M * N; e += kThreads) A[e] = tk.A[e];
        __syncthreads();
    }
    dev::householder(A, tau, M, N, red, sh);
    // R (k x N row-major) from the upper trapezoid
    for (int64_t e = threadIdx.x; e < (int64_t)k * N; e += kThreads) {
        const int r = (int)(e / N), c = (int)(e % N);
        tk.R[e] = c >= r ? A[(int64_t)c * M + r] : 0.0;
    }
    dev::form_q(A, tau, Q, M, k);
    // diag(R) >= 0 (R is in global memory; every thread sees the final R after the barrier)
    for (int j = warp; j < k; j += kWarps) {
        const double rjj = A[(int64_t)j * M + j];
        if (rjj < 0.0) {
            for (int c = lane; c < N; c += 32) tk.R[(int64_t)j * N + c] = -tk.R[(int64_t)j * N + c];
            for (int i = lane; i < M; i += 32) Q[(int64_t)j * M + i] = -Q[(int64_t)j * M + i];
        }
    }
    if (tk.smem) {
        __syncthreads();
        for (int64_t e = threadIdx.x; e < (int64_t)M * k; e += kThreads) tk.Q[e] = Q[e];
    }
}

constexpr int kSmemJacobiMax = 110;   // 2 k^2 doubles <= 193 KB of shared memory

// One-sided Jacobi task on a k x k matrix G (column-major, overwritten by the
// rotated columns) with the accumulated rotations in V (column-major).

// One-sided Jacobi (dev::jacobi), one CTA per matrix, in shared memory when k <= kSmemJacobiMax.
__global__ void __launch_bounds__(kThreads) k_jacobi(const JacTask* __restrict__ tasks) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ int s_rot;
    const JacTask tk = tasks[blockIdx.x];
    const int k = tk.k;
    double* G = tk.smem ? sm : tk.G;
    double* V = tk.smem ? sm + (int64_t)k * k : tk.V;
    if (tk.smem) {
        for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += kThreads) G[e] = tk.G[e];
        __syncthreads();
    }
    dev::jacobi(G, V, tk.Sraw, k, red, &s_rot);
    if (tk.smem) {
        for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += kThreads) {
            tk.G[e] = G[e];
            tk.V[e] = V[e];
        }
    }
}

// Assemble the SVD of M (M x N) from QR + Jacobi of the triangular factor:
// tall (M >= N): M = Q R, R^T = G, G V = U' S  =>  U = Q V, Vt = U'^T;
// wide (M < N):  M^T = Q R, R^T = G, G V = U' S => U = U', Vt = (Q V)^T.
// QVt = (Q V)^T (k x len, row-major) comes from a grouped GEMM.
struct SvdFin {
    const double* G;
    const double* QVt;
    const double* Sraw;
    double* S;
    double* US;
    double* Vt;
    int* perm;
    int M, N, k, len, wide;
};

__global__ void __launch_bounds__(kThreads) k_svd_finalize(const SvdFin* __restrict__ tasks) {
    const SvdFin tk = tasks[blockIdx.x];
    dev::svd_assemble(tk.G, tk.QVt, tk.Sraw, tk.perm, tk.S, tk.US, tk.Vt, tk.M, tk.N, tk.k, tk.len, tk.wide, tk.k, tk.N);
}

__global__ void __launch_bounds__(kThreads) k_sumsq(const double* const* __restrict__ xs,
                                                    const int64_t* __restrict__ ns,
                                                    double* __restrict__ out) {
    __shared__ double red[33];
    const double* x = xs[blockIdx.x];
    const int64_t n = ns[blockIdx.x];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kThreads) s += x[i] * x[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}


// Every kernel of the library prefers the same L1/shared-memory split (maximum
// shared memory), so consecutive launches never wait for the SM to re-partition.
void configure_carveout() {
    static bool done = false;
    if (done) return;
    const int carve = cudaSharedmemCarveoutMaxShared;
    BSM_CUDA(cudaFuncSetAttribute(k_copy, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    BSM_CUDA(cudaFuncSetAttribute(k_gemm, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    BSM_CUDA(cudaFuncSetAttribute(k_qr, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    BSM_CUDA(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    BSM_CUDA(cudaFuncSetAttribute(k_svd_finalize, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    BSM_CUDA(cudaFuncSetAttribute(k_sumsq, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    done = true;
}

}  // namespace

void check_launch(Context* ctx) {
    ctx->launches++;
    BSM_CUDA(cudaGetLastError());
}

cudaEvent_t Context::take_event() {
    cudaEvent_t e;
    if (!event_pool.empty()) {
        e = event_pool.back();
        event_pool.pop_back();
    } else {
        BSM_CUDA(cudaEventCreate(&e));
    }
    return e;
}

void Context::prof_begin(cudaEvent_t* e0) {
    *e0 = take_event();
    BSM_CUDA(cudaEventRecord(*e0, stream));
}

void Context::prof_end(int kind, double fl, double by, cudaEvent_t e0) {
    cudaEvent_t e1 = take_event();
    BSM_CUDA(cudaEventRecord(e1, stream));
    prof.push_back({kind, fl, by, e0, e1});
}

struct ZeroChunk {
    double* p;
    int64_t n;
};

__global__ void __launch_bounds__(kThreads) k_zero(const ZeroChunk* __restrict__ chunks) {
    const ZeroChunk c = chunks[blockIdx.x];
    for (int64_t e = threadIdx.x; e < c.n; e += kThreads) c.p[e] = 0.0;
}

void launch_zero(Context* ctx, const std::vector<double*>& ptr, const std::vector<int64_t>& n, int kind) {
    std::vector<ZeroChunk> chunks;
    for (size_t i = 0; i < ptr.size(); ++i)
        for (int64_t b = 0; b < n[i]; b += kCopyChunk) chunks.push_back({ptr[i] + b, std::min(n[i] - b, kCopyChunk)});
    if (chunks.empty()) return;
    configure_carveout();
    Scratch s(ctx);
    const ZeroChunk* d = s.up(chunks);
    ProfScope ps(ctx, kind, 0.0, 8.0 * [&] {
        double t = 0.0;
        for (int64_t v : n) t += (double)v;
        return t;
    }());
    k_zero<<<(unsigned)chunks.size(), kThreads, 0, ctx->stream>>>(d);
    check_launch(ctx);
    ps.done();
}

void launch_copy(Context* ctx, const std::vector<CopyTask>& tasks, int kind) {
    if (tasks.empty()) return;
    configure_carveout();
    std::vector<CopyChunk> chunks;
    for (int i = 0; i < (int)tasks.size(); ++i) {
        const int64_t n = (int64_t)tasks[i].rows * tasks[i].cols;
        for (int64_t b = 0; b < n; b += kCopyChunk) chunks.push_back({i, b, std::min(n, b + kCopyChunk)});
    }
    if (chunks.empty()) return;
    double by = 0.0;
    for (const CopyTask& t : tasks) by += (t.accumulate ? 24.0 : 16.0) * t.rows * (double)t.cols;
    Scratch s(ctx);
    CopyTask* dt = s.up(tasks);
    CopyChunk* dc = s.up(chunks);
    ProfScope ps(ctx, kind, 0.0, by);
    k_copy<<<(unsigned)chunks.size(), kThreads, 0, ctx->stream>>>(dt, dc);
    check_launch(ctx);
    ps.done();
}


namespace {

// The FP64 grouped GEMM with outputs of max(M, N) <= small_max on the
// one-thread-per-entry kernel and the rest on 32 x 32 tiles (small_max <= 32).
void launch_gemm_fp64(Context* ctx, const std::vector<GemmOut>& outs, const std::vector<GemmIn>& ins, int kind,
                      int small_max) {
    configure_carveout();
    std::vector<GemmTile> tiles;
    std::vector<int> small, emulated;
    double fl = 0.0, by = 0.0;
    for (int o = 0; o < (int)outs.size(); ++o) {
        const GemmOut& g = outs[o];
        // outputs of at least 2^gemm_emulation_log2 flops with one untransposed
        // contribution (overwritten) go to the tensor-core FP64 emulation; the
        // emulation takes untransposed operands only (the sweeps' large R X and
        // U S X products are untransposed)
        if (ctx->gemm_emulation_log2 > 0 && g.end == g.beg + 1 && g.beta == 0.0 && !ins[g.beg].transA &&
            2.0 * g.M * (double)g.N * ins[g.beg].K >= std::ldexp(1.0, ctx->gemm_emulation_log2)) {
            emulated.push_back(o);
            continue;
        }
        if (std::max(g.M, g.N) <= small_max) {
            if (g.M > 0 && g.N > 0) small.push_back(o);
        } else {
            for (int m0 = 0; m0 < g.M; m0 += kTile)
                for (int n0 = 0; n0 < g.N; n0 += kTile) tiles.push_back({o, m0, n0});
        }
        for (int c = g.beg; c < g.end; ++c) {
            fl += 2.0 * g.M * g.N * (double)ins[c].K;
            by += 8.0 * ((double)g.M * ins[c].K + (double)ins[c].K * g.N);
        }
        by += 8.0 * g.M * (double)g.N * (g.beta == 0.0 ? 1.0 : 2.0);
    }
    if (!emulated.empty()) {
        std::vector<OzGemm> og;
        double efl = 0.0;
        for (int o : emulated) {
            const GemmOut& g = outs[o];
            const GemmIn& in = ins[g.beg];
            og.push_back({in.A, in.B, g.C, g.M, g.N, in.K, in.lda, in.ldb, g.ldc, in.alpha});
            efl += 2.0 * g.M * (double)g.N * in.K;
        }
        ProfScope pe(ctx, kind, efl, 0.0);
        launch_gemm_ozaki_group(ctx, og, 8);
        pe.done();
    }
    if (tiles.empty() && small.empty()) return;
    ctx->flops += fl;
    // one staged upload for all task arrays
    std::vector<unsigned char> pack;
    auto add = [&](const void* src, size_t bytes) {
        const size_t off = (pack.size() + 15) & ~size_t(15);
        pack.resize(off + bytes);
        if (bytes) std::memcpy(pack.data() + off, src, bytes);
        return off;
    };
    const size_t oo = add(outs.data(), outs.size() * sizeof(GemmOut));
    const size_t oi = add(ins.data(), ins.size() * sizeof(GemmIn));
    const size_t os = add(small.data(), small.size() * sizeof(int));
    const size_t ot = add(tiles.data(), tiles.size() * sizeof(GemmTile));
    Scratch s(ctx);
    unsigned char* d = s.up(pack);
    const GemmOut* d_o = (const GemmOut*)(d + oo);
    const GemmIn* d_i = (const GemmIn*)(d + oi);
    ProfScope ps(ctx, kind, fl, by);
    if (!small.empty()) {
        k_gemm_small<<<(unsigned)small.size(), kSmallGemmThreads, 0, ctx->stream>>>(d_o, d_i, (const int*)(d + os));
        check_launch(ctx);
    }
    if (!tiles.empty()) {
        k_gemm<<<(unsigned)tiles.size(), kThreads, 0, ctx->stream>>>(d_o, d_i, (const GemmTile*)(d + ot));
        check_launch(ctx);
    }
    ps.done();
}

// Size class of a contraction launch for the autotuner: the fractions of
// outputs with max(M, N) <= 8, <= 16, <= 32 (in quarters) and log2 of the flops.
int64_t gemm_size_class(const std::vector<GemmOut>& outs, const std::vector<GemmIn>& ins) {
    int64_t c8 = 0, c16 = 0, c32 = 0;
    double fl = 0.0;
    for (const GemmOut& g : outs) {
        const int mx = std::max(g.M, g.N);
        c8 += mx <= 8;
        c16 += mx <= 16;
        c32 += mx <= 32;
        for (int c = g.beg; c < g.end; ++c) fl += 2.0 * g.M * g.N * (double)ins[c].K;
    }
    const int64_t n = std::max<int64_t>((int64_t)outs.size(), 1);
    const int64_t q8 = 4 * c8 / n, q16 = 4 * c16 / n, q32 = 4 * c32 / n;
    const int64_t lf = fl > 1.0 ? (int64_t)std::log2(fl) : 0;
    return ((q8 * 5 + q16) * 5 + q32) * 64 + std::min<int64_t>(lf, 63);
}

}  // namespace

// The zip-up contraction (kind KK_APPLY) in FP64 is autotuned: the split
// between the one-thread-per-entry kernel and the 32 x 32 tiled kernel
// (small_max in {0, 8, 16, 32}) is chosen per context and size class by timing
// every candidate on the first launch of that class (the contraction overwrites
// its outputs, so the repeats change nothing) and kept for later launches.
void launch_gemm(Context* ctx, const std::vector<GemmOut>& outs, const std::vector<GemmIn>& ins, int kind) {
    if (outs.empty()) return;
    if (kind == KK_APPLY && ctx->apply_precision == BSMPS_PREC_TF32X3 && gemm_tf32x3_eligible(outs, ins)) {
        launch_gemm_tf32x3(ctx, outs, ins, kind);
        return;
    }
    if (kind != KK_APPLY || !ctx->autotune) {
        launch_gemm_fp64(ctx, outs, ins, kind, kTile);
        return;
    }
    for (const GemmOut& g : outs)
        if (g.beta != 0.0) {   // accumulating outputs cannot be repeated
            launch_gemm_fp64(ctx, outs, ins, kind, kTile);
            return;
        }
    const int64_t key = gemm_size_class(outs, ins);
    auto it = ctx->gemm_tuned.find(key);
    if (it != ctx->gemm_tuned.end() || ctx->rec) {
        // a graph being recorded takes the tuned split (its sizing run tuned every
        // class) and never times candidates
        launch_gemm_fp64(ctx, outs, ins, kind, it != ctx->gemm_tuned.end() ? it->second : kTile);
        return;
    }
    const int cand[4] = {0, 8, 16, 32};
    float best_ms = 0.0f;
    int best = kTile;
    const bool prof = ctx->profiling;
    ctx->profiling = false;   // tuning launches are not part of the profile
    cudaEvent_t e0 = ctx->take_event(), e1 = ctx->take_event();
    for (int c : cand) {
        BSM_CUDA(cudaEventRecord(e0, ctx->stream));
        launch_gemm_fp64(ctx, outs, ins, kind, c);
        BSM_CUDA(cudaEventRecord(e1, ctx->stream));
        BSM_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        BSM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (c == cand[0] || ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    ctx->event_pool.push_back(e0);
    ctx->event_pool.push_back(e1);
    ctx->profiling = prof;
    ctx->gemm_tuned[key] = best;
    // the launch that counts (and is profiled)
    launch_gemm_fp64(ctx, outs, ins, kind, best);
}

constexpr size_t kSmemBudget = 220 * 1024;

void launch_qr(Context* ctx, const std::vector<QrTask>& tasks_in, int kind) {
    if (tasks_in.empty()) return;
    configure_carveout();
    double fl = 0.0, by = 0.0;
    std::vector<QrTask> small, large, clustered;
    size_t smem_max = 0;
    for (QrTask t : tasks_in) {
        if (qr_cluster_eligible(t.M, t.N)) {
            const double m = t.M, n = t.N, k = std::min(m, n);
            fl += 2.0 * m * n * k - (m + n) * k * k + 2.0 / 3.0 * k * k * k + 2.0 * m * k * k - 2.0 / 3.0 * k * k * k;
            by += 8.0 * (m * n + m * k + k * n);
            clustered.push_back(t);
            continue;
        }
        const double m = t.M, n = t.N, k = std::min(m, n);
        fl += 2.0 * m * n * k - (m + n) * k * k + 2.0 / 3.0 * k * k * k;   // factorisation
        fl += 2.0 * m * k * k - 2.0 / 3.0 * k * k * k;                     // forming Q
        by += 8.0 * (m * n + m * k + k * n);
        const size_t need = sizeof(double) * ((size_t)t.M * t.N + (size_t)t.M * std::min(t.M, t.N) +
                                              (size_t)std::min(t.M, t.N));
        if (need <= kSmemBudget) {
            t.smem = 1;
            small.push_back(t);
            smem_max = std::max(smem_max, need);
        } else {
            t.smem = 0;
            large.push_back(t);
        }
    }
    ctx->flops += fl;
    Scratch s(ctx);
    ProfScope ps(ctx, kind, fl, by);
    bool cluster_ran = false;
    if (!clustered.empty()) {
        cluster_ran = launch_qr_cluster(ctx, clustered, kind == KK_APPLY_QR);
        if (!cluster_ran) {
            for (QrTask t : clustered) {   // no cluster could be scheduled: one CTA per matrix
                const size_t need = sizeof(double) * ((size_t)t.M * t.N + (size_t)t.M * std::min(t.M, t.N) +
                                                      (size_t)std::min(t.M, t.N));
                t.smem = need <= kSmemBudget ? 1 : 0;
                if (t.smem) smem_max = std::max(smem_max, need);
                (t.smem ? small : large).push_back(t);
            }
        }
    }
    // the one-CTA QRs overlap the cluster QRs on the context's second stream:
    // their task lists are uploaded first, the fork follows, the join precedes
    // the release of s
    QrTask* d_small = small.empty() ? nullptr : s.up(small);
    QrTask* d_large = large.empty() ? nullptr : s.up(large);
    const bool overlap = cluster_ran && (d_small || d_large) && !ctx->profiling && !ctx->rec && !ctx->side_open;
    SideJoin guard(overlap ? ctx : nullptr);   // after s: joins before s releases the task lists
    const cudaStream_t st = overlap ? ctx->fork_side() : ctx->stream;
    if (d_small) {
        BSM_CUDA(cudaFuncSetAttribute(k_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
        k_qr<<<(unsigned)small.size(), kThreads, smem_max, st>>>(d_small);
        check_launch(ctx);
    }
    if (d_large) {
        k_qr<<<(unsigned)large.size(), kThreads, 0, st>>>(d_large);
        check_launch(ctx);
    }
    if (overlap) ctx->join_side();
    ps.done();
}

void launch_svd(Context* ctx, const std::vector<SvdTask>& tasks) {
    if (tasks.empty()) return;
    configure_carveout();
    Scratch s(ctx);
    // 1. Householder QR of M (tall) or M^T (wide): Q is len x k, R is k x k
    std::vector<QrTask> qr;
    std::vector<double*> Q(tasks.size()), R(tasks.size()), V(tasks.size()), Sraw(tasks.size()), QVt(tasks.size());
    std::vector<int*> perm(tasks.size());
    for (size_t i = 0; i < tasks.size(); ++i) {
        const SvdTask& t = tasks[i];
        const int k = std::min(t.M, t.N), len = std::max(t.M, t.N);
        Q[i] = s.dbl((size_t)len * k);
        R[i] = s.dbl((size_t)k * k);
        V[i] = s.dbl((size_t)k * k);
        Sraw[i] = s.dbl((size_t)k);
        QVt[i] = s.dbl((size_t)k * len);
        perm[i] = (int*)ctx->alloc(sizeof(int) * (size_t)k);
        s.ptrs.push_back(perm[i]);
        qr.push_back({t.G, Q[i], R[i], s.dbl((size_t)k), t.wide ? t.N : t.M, t.wide ? t.M : t.N});
    }
    launch_qr(ctx, qr);
    // 2. one-sided Jacobi on G = R^T (the row-major R is G column-major): one
    // thread-block cluster per matrix for kClusterJacobiMin <= k <= kClusterJacobiMax
    // (the FP64 units of several SMs on one matrix); one CTA in shared memory for
    // smaller k (and for k <= kSmemJacobiMax when no cluster can be scheduled);
    // beyond, across the grid (one CTA per matrix when the cooperative launch
    // cannot be resident)
    std::vector<JacTask> small, mid, large;
    std::vector<size_t> mid_i;
    double fl = 0.0, by = 0.0;
    for (size_t i = 0; i < tasks.size(); ++i) {
        const int k = std::min(tasks[i].M, tasks[i].N);
        JacTask jt{R[i], V[i], Sraw[i], k, 0};
        if (k >= kClusterJacobiMin && k <= kClusterJacobiMax) {
            mid.push_back(jt);
            mid_i.push_back(i);
        } else if (k <= kSmemJacobiMax)
            small.push_back(jt);
        else
            large.push_back(jt);
        fl += 54.0 * (double)k * k * k;   // nominal: 6 sweeps of k^2/2 pairs x 18k flops
        by += 8.0 * 3.0 * k * (double)k;
    }
    ctx->flops += fl;
    // 2a. FP32 preconditioning of the cluster tasks with k >= jacobi_precond_min:
    // P = the rotations of an FP32 one-sided Jacobi of G (orthogonal to ~1e-6),
    // Qp = the Q factor of P (FP64 Householder, orthogonal to FP64 rounding,
    // diag R >= 0 keeps it next to P), G <- G Qp.  The FP64 Jacobi below then
    // starts from nearly orthogonal columns and converges in a few sweeps
    // (quadratically), and V <- Qp V afterwards: G Qp V = U S exactly as before,
    // with every step that decides the result in FP64.
    struct Pre {
        size_t m;          // index in mid
        double *Qp, *V1;
    };
    std::vector<Pre> pre;
    if (ctx->jacobi_precond_min > 0 && !mid.empty()) {
        const double fl0 = ctx->flops;   // the preconditioner's work is not algorithmic work of the SVD
        std::vector<JacTask> pj;
        std::vector<double*> P;
        double pb = 0.0;
        for (size_t m = 0; m < mid.size(); ++m) {
            const int k = mid[m].k;
            if (k < ctx->jacobi_precond_min) continue;
            P.push_back(s.dbl((size_t)k * k));
            pj.push_back({mid[m].G, P.back(), nullptr, k, 0});
            pre.push_back({m, s.dbl((size_t)k * k), s.dbl((size_t)k * k)});
            pb += 16.0 * k * (double)k;
        }
        bool ok = pj.empty();
        if (!ok) {
            ProfScope ps(ctx, KK_SVD, 0.0, pb);
            ok = launch_jacobi_cluster_f32(ctx, pj);
            ps.done();
        }
        if (ok && !pre.empty()) {
            std::vector<QrTask> pq;
            for (size_t j = 0; j < pre.size(); ++j) {
                const int k = pj[j].k;
                pq.push_back({P[j], pre[j].Qp, s.dbl((size_t)k * k), s.dbl((size_t)k), k, k});
            }
            launch_qr(ctx, pq, KK_SVD);
            // G1 = G Qp (column-major): G1^T = Qp^T G^T, the buffers read row-major
            std::vector<GemmOut> go;
            std::vector<GemmIn> gi;
            for (Pre& pr : pre) {
                JacTask& jt = mid[pr.m];
                double* G1 = s.dbl((size_t)jt.k * jt.k);
                go.push_back({G1, jt.k, jt.k, jt.k, (int)gi.size(), (int)gi.size() + 1, 0.0});
                gi.push_back({pr.Qp, jt.G, jt.k, jt.k, jt.k, 0, 1.0});
                jt.G = G1;
                R[mid_i[pr.m]] = G1;   // the rotated G that step 4 reads
                // the cluster Jacobi rotates Qp's columns: V = Qp V1 without a product
                jt.V = pr.Qp;
                jt.v_given = 1;
            }
            launch_gemm(ctx, go, gi, KK_SVD);
        } else {
            pre.clear();
        }
        ctx->flops = fl0;
    }
    {
        ProfScope ps(ctx, KK_SVD, fl, by);
        if (!mid.empty() && launch_jacobi_cluster(ctx, mid)) {
            for (const Pre& pr : pre) V[mid_i[pr.m]] = pr.Qp;   // Qp V1, in place
            pre.clear();
        } else if (!mid.empty()) {
            // one CTA per matrix: those kernels start from the identity, so the
            // preconditioned tasks accumulate V1 and V = Qp V1 follows below
            for (size_t m = 0; m < mid.size(); ++m) mid[m].v_given = 0;
            for (const Pre& pr : pre) mid[pr.m].V = pr.V1;
            for (const JacTask& t : mid) (t.k <= kSmemJacobiMax ? small : large).push_back(t);
        }
        if (!small.empty()) {
            int kmax_small = 1;
            for (JacTask& t : small) {
                t.smem = 1;
                kmax_small = std::max(kmax_small, t.k);
            }
            JacTask* d = s.up(small);
            const size_t smem = sizeof(double) * 2 * (size_t)kmax_small * kmax_small;
            BSM_CUDA(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_jacobi<<<(unsigned)small.size(), kThreads, smem, ctx->stream>>>(d);
            check_launch(ctx);
        }
        if (!large.empty() && !launch_jacobi_grid(ctx, large)) {
            JacTask* d = s.up(large);
            k_jacobi<<<(unsigned)large.size(), kThreads, 0, ctx->stream>>>(d);
            check_launch(ctx);
        }
        ps.done();
    }
    if (!pre.empty()) {
        // V = Qp V1 (column-major): V^T = V1^T Qp^T
        const double fl0 = ctx->flops;
        std::vector<GemmOut> go;
        std::vector<GemmIn> gi;
        for (const Pre& pr : pre) {
            const int k = mid[pr.m].k;
            go.push_back({V[mid_i[pr.m]], k, k, k, (int)gi.size(), (int)gi.size() + 1, 0.0});
            gi.push_back({pr.V1, pr.Qp, k, k, k, 0, 1.0});
        }
        launch_gemm(ctx, go, gi, KK_SVD);
        ctx->flops = fl0;
    }
    // 3. (Q V)^T = V^T Q^T: A = V column-major read as V^T row-major, B = Q column-major = Q^T row-major
    std::vector<GemmOut> outs;
    std::vector<GemmIn> ins;
    for (size_t i = 0; i < tasks.size(); ++i) {
        const int k = std::min(tasks[i].M, tasks[i].N), len = std::max(tasks[i].M, tasks[i].N);
        outs.push_back({QVt[i], k, len, len, (int)ins.size(), (int)ins.size() + 1, 0.0});
        ins.push_back({V[i], Q[i], k, k, len, 0, 1.0});
    }
    launch_gemm(ctx, outs, ins);
    // 4. sort, assemble U S and V^T, sign convention
    std::vector<SvdFin> fin;
    double fb = 0.0;
    for (size_t i = 0; i < tasks.size(); ++i) {
        const SvdTask& t = tasks[i];
        const int k = std::min(t.M, t.N), len = std::max(t.M, t.N);
        fin.push_back({R[i], QVt[i], Sraw[i], t.S, t.US, t.Vt, perm[i], t.M, t.N, k, len, t.wide});
        fb += 8.0 * ((double)t.M * k + (double)k * t.N + 2.0 * k * (double)len);
    }
    SvdFin* d = s.up(fin);
    ProfScope ps(ctx, KK_SVD, 0.0, fb);
    k_svd_finalize<<<(unsigned)fin.size(), kThreads, 0, ctx->stream>>>(d);
    check_launch(ctx);
    ps.done();
}

void launch_sumsq(Context* ctx, const std::vector<const double*>& xs, const std::vector<int64_t>& ns,
                  double* out_dev) {
    if (xs.empty()) return;
    configure_carveout();
    Scratch s(ctx);
    const double** d_x = s.up(xs);
    int64_t* d_n = s.up(ns);
    double by = 0.0;
    for (int64_t n : ns) by += 8.0 * n;
    ProfScope ps(ctx, KK_SUMSQ, 2.0 * by / 8.0, by);
    k_sumsq<<<(unsigned)xs.size(), kThreads, 0, ctx->stream>>>(d_x, d_n, out_dev);
    check_launch(ctx);
    ps.done();
}

}  // namespace bsm
