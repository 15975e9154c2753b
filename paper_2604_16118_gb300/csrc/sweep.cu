// Fused per-site kernels of the truncation sweeps: each CTA owns one sector of
// the bond being orthogonalised or truncated and keeps its working set in
// shared memory, so one site costs one launch (left sweep) or two launches
// around the host's cut decision (right sweep).
#include <algorithm>
#include <cstring>

#include "dense_dev.cuh"
#include "kernels.h"

namespace bsm {
namespace {

using dev::kThreads;
using dev::kWarps;
using dev::nthreads;
using dev::nwarps;

constexpr size_t kSweepSmem = 220 * 1024;

size_t left_smem(int M, int N) {
    const size_t k = (size_t)std::min(M, N);
    return sizeof(double) * ((size_t)M * N + (size_t)M * k + k + k * (size_t)N);
}

size_t svd_smem(int M, int N) {
    const size_t k = (size_t)std::min(M, N), len = (size_t)std::max(M, N);
    return sizeof(double) * (2 * len * k + 2 * k * k + 3 * k);
}

__global__ void __launch_bounds__(kThreads) k_left_site(const LeftTask* __restrict__ tasks,
                                                        const LeftSrc* __restrict__ srcs,
                                                        const LeftX* __restrict__ xs) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ double sh[2];
    const LeftTask tk = tasks[blockIdx.x];
    const int M = tk.M, N = tk.N, k = tk.k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* A = sm;
    double* Q = A + (int64_t)M * N;
    double* tau = Q + (int64_t)M * k;
    double* R = tau + k;
    for (int s = tk.s_beg; s < tk.s_end; ++s) {
        const LeftSrc sr = srcs[s];
        for (int64_t e = threadIdx.x; e < (int64_t)sr.rows * N; e += nthreads()) {
            const int i = (int)(e / N), c = (int)(e % N);
            A[(int64_t)c * M + sr.r0 + i] = sr.src[e];
        }
    }
    __syncthreads();
    dev::householder(A, tau, M, N, red, sh);
    for (int64_t e = threadIdx.x; e < (int64_t)k * N; e += nthreads()) {
        const int r = (int)(e / N), c = (int)(e % N);
        R[e] = c >= r ? A[(int64_t)c * M + r] : 0.0;
    }
    dev::form_q(A, tau, Q, M, k);
    __syncthreads();
    for (int j = warp; j < k; j += nwarps()) {
        if (A[(int64_t)j * M + j] < 0.0) {
            for (int c = lane; c < N; c += 32) R[(int64_t)j * N + c] = -R[(int64_t)j * N + c];
            for (int i = lane; i < M; i += 32) Q[(int64_t)j * M + i] = -Q[(int64_t)j * M + i];
        }
    }
    __syncthreads();
    for (int s = tk.s_beg; s < tk.s_end; ++s) {
        const LeftSrc sr = srcs[s];
        for (int64_t e = threadIdx.x; e < (int64_t)sr.rows * k; e += nthreads()) {
            const int i = (int)(e / k), c = (int)(e % k);
            sr.dst[e] = Q[(int64_t)c * M + sr.r0 + i];
        }
    }
    for (int x = tk.x_beg; x < tk.x_end; ++x) {
        const LeftX lx = xs[x];
        for (int64_t e = threadIdx.x; e < (int64_t)k * lx.cols; e += nthreads()) {
            const int r = (int)(e / lx.cols), c = (int)(e % lx.cols);
            double acc = 0.0;
            for (int j = r; j < N; ++j) acc = fma(R[(int64_t)r * N + j], lx.X[(int64_t)j * lx.cols + c], acc);
            lx.dst[e] = acc;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_svd_site(const SvdSiteTask* __restrict__ tasks,
                                                       const SvdPart* __restrict__ parts) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ double sh[2];
    __shared__ int s_rot;
    const SvdSiteTask tk = tasks[blockIdx.x];
    const int M = tk.M, N = tk.N, k = tk.k, len = tk.len;
    double* B = sm;                               // QR input (len x k), later Q V
    double* Q = B + (int64_t)len * k;
    double* tau = Q + (int64_t)len * k;
    double* G = tau + k;
    double* V = G + (int64_t)k * k;
    double* Sraw = V + (int64_t)k * k;
    int* perm = (int*)(Sraw + k);
    for (int p = tk.p_beg; p < tk.p_end; ++p) {
        const SvdPart pt = parts[p];
        for (int64_t e = threadIdx.x; e < (int64_t)M * pt.cols; e += nthreads()) {
            const int i = (int)(e / pt.cols), c = pt.coff + (int)(e % pt.cols);
            if (tk.wide)
                B[(int64_t)i * N + c] = pt.src[e];      // A^T column-major
            else
                B[(int64_t)c * M + i] = pt.src[e];      // A column-major
        }
    }
    __syncthreads();
    dev::householder(B, tau, len, k, red, sh);
    // G = R^T (column-major): G(i, j) = R(j, i), nonzero for i >= j
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += nthreads()) {
        const int j = (int)(e / k), i = (int)(e % k);
        G[e] = i >= j ? B[(int64_t)i * len + j] : 0.0;
    }
    dev::form_q(B, tau, Q, len, k);
    __syncthreads();
    dev::jacobi(G, V, Sraw, k, red, &s_rot);
    for (int64_t e = threadIdx.x; e < (int64_t)len * k; e += nthreads()) {
        const int p = (int)(e / len), i = (int)(e % len);
        double acc = 0.0;
        for (int j = 0; j < k; ++j) acc = fma(Q[(int64_t)j * len + i], V[(int64_t)p * k + j], acc);
        B[e] = acc;
    }
    __syncthreads();
    dev::svd_assemble(G, B, Sraw, perm, tk.S, tk.US, tk.Vt, M, N, k, len, tk.wide, k, N);
}

__global__ void __launch_bounds__(kThreads) k_right_apply(const RTask* __restrict__ tasks,
                                                          const RCopy* __restrict__ copies,
                                                          const RGemm* __restrict__ gemms) {
    const RTask tk = tasks[blockIdx.x];
    for (int c = tk.c_beg; c < tk.c_end; ++c) {
        const RCopy rc = copies[c];
        for (int64_t e = threadIdx.x; e < (int64_t)rc.rows * rc.cols; e += nthreads()) {
            const int i = (int)(e / rc.cols), j = (int)(e % rc.cols);
            rc.dst[e] = rc.src[(int64_t)i * rc.src_ld + j];
        }
    }
    for (int g = tk.g_beg; g < tk.g_end; ++g) {
        const RGemm rg = gemms[g];
        for (int64_t e = threadIdx.x; e < (int64_t)rg.rows * rg.keep; e += nthreads()) {
            const int i = (int)(e / rg.keep), j = (int)(e % rg.keep);
            double acc = 0.0;
            for (int q = 0; q < rg.K; ++q) acc = fma(rg.X[(int64_t)i * rg.K + q], rg.US[(int64_t)q * rg.ldus + j], acc);
            rg.dst[e] = acc;
        }
    }
}

// Device-driven right sweep, one CTA per sector of bond b: the sector's matrix
// is formed from the left-orthogonal core-b blocks times the kept columns of
// the U S of bond b+1 (kept counts read from device memory), then QR, Jacobi
// and assembly as in k_svd_site into padded outputs.
__global__ void __launch_bounds__(kThreads) k_right_dyn(const DynTask* __restrict__ tasks,
                                                        const DynPart* __restrict__ parts) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ double sh[2];
    __shared__ int s_rot;
    __shared__ int s_cols[2];
    const DynTask tk = tasks[blockIdx.x];
    const int np = tk.p_end - tk.p_beg;
    if (threadIdx.x < 2) {
        int c = 0;
        if ((int)threadIdx.x < np) {
            const DynPart pt = parts[tk.p_beg + threadIdx.x];
            c = pt.keep ? *pt.keep : pt.xcols;
        }
        s_cols[threadIdx.x] = c;
    }
    __syncthreads();
    const int M = tk.M, N = s_cols[0] + s_cols[1];
    if (N == 0 || M == 0) {
        if (threadIdx.x == 0) *tk.kact = 0;
        return;
    }
    const int k = M < N ? M : N, len = M < N ? N : M, wide = M < N ? 1 : 0;
    double* B = sm;
    double* Q = B + (int64_t)len * k;
    double* tau = Q + (int64_t)len * k;
    double* G = tau + k;
    double* V = G + (int64_t)k * k;
    double* Sraw = V + (int64_t)k * k;
    int* perm = (int*)(Sraw + k);
    int coff = 0;
    for (int p = 0; p < np; ++p) {
        const DynPart pt = parts[tk.p_beg + p];
        const int cols = s_cols[p];
        for (int64_t e = threadIdx.x; e < (int64_t)M * cols; e += nthreads()) {
            const int i = (int)(e / cols), cc = (int)(e % cols), c = coff + cc;
            double v;
            if (pt.US) {
                v = 0.0;
                for (int q = 0; q < pt.xcols; ++q)
                    v = fma(pt.X[(int64_t)i * pt.xcols + q], pt.US[(int64_t)q * pt.ldus + cc], v);
            } else {
                v = pt.X[(int64_t)i * pt.xcols + cc];
            }
            if (wide)
                B[(int64_t)i * N + c] = v;
            else
                B[(int64_t)c * M + i] = v;
        }
        coff += cols;
    }
    __syncthreads();
    dev::householder(B, tau, len, k, red, sh);
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += nthreads()) {
        const int j = (int)(e / k), i = (int)(e % k);
        G[e] = i >= j ? B[(int64_t)i * len + j] : 0.0;
    }
    dev::form_q(B, tau, Q, len, k);
    __syncthreads();
    dev::jacobi(G, V, Sraw, k, red, &s_rot);
    for (int64_t e = threadIdx.x; e < (int64_t)len * k; e += nthreads()) {
        const int p = (int)(e / len), i = (int)(e % len);
        double acc = 0.0;
        for (int j = 0; j < k; ++j) acc = fma(Q[(int64_t)j * len + i], V[(int64_t)p * k + j], acc);
        B[e] = acc;
    }
    __syncthreads();
    dev::svd_assemble(G, B, Sraw, perm, tk.S, tk.US, tk.Vt, M, N, k, len, wide, tk.kpad, tk.ncols_pad);
    if (threadIdx.x == 0) *tk.kact = k;
}

// Pooled cut of one bond (one CTA): stable descending order with ties by
// (sector, index), then the sequential tolerance / cluster / cap rule; the
// products and sums are rounded individually (no contraction) so that the
// decisions equal the host rule.
__global__ void __launch_bounds__(kThreads) k_cut_dyn(const CutTask* __restrict__ tptr,
                                                      const CutSector* __restrict__ secs) {
    extern __shared__ double sm[];
    __shared__ int s_n;
    const CutTask tk = *tptr;
    double* val = sm;
    int* sec = (int*)(val + tk.cap_total);
    int* jj = sec + tk.cap_total;
    int* order = jj + tk.cap_total;
    int* off = order + tk.cap_total;   // n_sec + 1
    if (threadIdx.x == 0) {
        int o = 0;
        for (int i = 0; i < tk.n_sec; ++i) {
            off[i] = o;
            o += *secs[tk.s_beg + i].kact;
        }
        off[tk.n_sec] = o;
        s_n = o;
    }
    __syncthreads();
    const int n = s_n;
    for (int i = 0; i < tk.n_sec; ++i) {
        const int c = off[i + 1] - off[i];
        for (int j = threadIdx.x; j < c; j += nthreads()) {
            val[off[i] + j] = secs[tk.s_beg + i].S[j];
            sec[off[i] + j] = i;
            jj[off[i] + j] = j;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += nthreads()) {
        const double se = val[e];
        int rank = 0;
        for (int o = 0; o < n; ++o) {
            const double so = val[o];
            const bool before = so > se || (so == se && (sec[o] < sec[e] || (sec[o] == sec[e] && jj[o] < jj[e])));
            rank += before ? 1 : 0;
        }
        order[rank] = e;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double rtol = 1e-10;
        int keep = n;
        double acc = 0.0;
        while (keep > 0) {
            const double sv = val[order[keep - 1]];
            const double s2 = __dmul_rn(sv, sv);
            if (__dadd_rn(acc, s2) <= tk.tol2) {
                acc = __dadd_rn(acc, s2);
                keep -= 1;
            } else {
                break;
            }
        }
        while (keep > 0 && keep < n && val[order[keep]] >= __dmul_rn(val[order[keep - 1]], 1.0 - rtol)) keep += 1;
        double td = 0.0;
        for (int i = keep; i < n; ++i) td = __dadd_rn(td, __dmul_rn(val[order[i]], val[order[i]]));
        double cd = 0.0;
        if (tk.r_max > 0 && keep > tk.r_max) {
            int k2 = tk.r_max;
            while (k2 > 0 && val[order[k2]] >= __dmul_rn(val[order[k2 - 1]], 1.0 - rtol)) k2 -= 1;
            if (k2 == 0) k2 = tk.r_max;
            for (int i = k2; i < keep; ++i) cd = __dadd_rn(cd, __dmul_rn(val[order[i]], val[order[i]]));
            keep = k2;
        }
        for (int i = 0; i < tk.n_sec; ++i) tk.keep[i] = 0;
        for (int r = 0; r < keep; ++r) tk.keep[sec[order[r]]] += 1;
        tk.disc[0] = __dadd_rn(tk.disc[0], td);
        tk.disc[1] = __dadd_rn(tk.disc[1], cd);
    }
}

// All task arrays of one launch in one upload.
struct Pack {
    std::vector<unsigned char> host;
    template <class T>
    size_t add(const std::vector<T>& v) {
        const size_t off = (host.size() + 15) & ~size_t(15);
        host.resize(off + v.size() * sizeof(T));
        if (!v.empty()) std::memcpy(host.data() + off, v.data(), v.size() * sizeof(T));
        return off;
    }
};

unsigned char* upload_pack(Scratch& s, const Pack& p) {
    std::vector<unsigned char> h = p.host;
    if (h.empty()) h.push_back(0);
    return s.up(h);
}

// Warps per CTA: one per Jacobi pair of the largest problem, between 1 and 8.
int block_for(int kmax) { return 32 * std::max(1, std::min(8, (kmax + 1) / 2)); }

template <class F>
void allow_smem(F* kern) {
    static bool done = false;   // set once per process (the attributes are per function)
    if (!done) {
        BSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmem));
        BSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
        done = true;
    }
}

void count_launch(Context* ctx) {
    ctx->launches++;
    BSM_CUDA(cudaGetLastError());
}

struct Prof {
    Context* ctx;
    int kind;
    double fl, by;
    cudaEvent_t e0 = nullptr;
    Prof(Context* c, int k, double f, double b) : ctx(c), kind(k), fl(f), by(b) {
        if (ctx->profiling) ctx->prof_begin(&e0);
    }
    void done() {
        if (ctx->profiling) ctx->prof_end(kind, fl, by, e0);
    }
};

}  // namespace

bool left_site_fits(int M, int N, int64_t rx_fma) { return left_smem(M, N) <= kSweepSmem && rx_fma <= kFusedGemmMaxFma; }

size_t dyn_svd_smem(int M, int ncols_pad) { return svd_smem(M, ncols_pad); }

bool svd_site_fits(int M, int N) { return std::min(M, N) <= 96 && svd_smem(M, N) <= kSweepSmem; }

void launch_left_site(Context* ctx, const std::vector<LeftTask>& tasks, const std::vector<LeftSrc>& srcs,
                      const std::vector<LeftX>& xs) {
    if (tasks.empty()) return;
    size_t smem = 0;
    double fl = 0.0, by = 0.0;
    for (const LeftTask& t : tasks) {
        smem = std::max(smem, left_smem(t.M, t.N));
        const double m = t.M, n = t.N, k = t.k;
        fl += 2.0 * m * n * k - (m + n) * k * k + 2.0 / 3.0 * k * k * k + 2.0 * m * k * k - 2.0 / 3.0 * k * k * k;
        by += 8.0 * (m * n + m * k);
        for (int x = t.x_beg; x < t.x_end; ++x) {
            fl += 2.0 * k * n * xs[x].cols;
            by += 8.0 * (n + k) * xs[x].cols;
        }
    }
    ctx->flops += fl;
    Pack pk;
    const size_t ot = pk.add(tasks), os = pk.add(srcs), ox = pk.add(xs);
    Scratch s(ctx);
    unsigned char* d = upload_pack(s, pk);
    Prof pr(ctx, KK_QR, fl, by);
    allow_smem(k_left_site);
    int kmax = 1;
    for (const LeftTask& t : tasks) kmax = std::max(kmax, 2 * t.k);
    k_left_site<<<(unsigned)tasks.size(), block_for(kmax), smem, ctx->stream>>>((const LeftTask*)(d + ot),
                                                                        (const LeftSrc*)(d + os),
                                                                        (const LeftX*)(d + ox));
    count_launch(ctx);
    pr.done();
}

void launch_svd_site(Context* ctx, const std::vector<SvdSiteTask>& tasks, const std::vector<SvdPart>& parts) {
    if (tasks.empty()) return;
    size_t smem = 0;
    double fl = 0.0, by = 0.0;
    for (const SvdSiteTask& t : tasks) {
        smem = std::max(smem, svd_smem(t.M, t.N));
        const double k = t.k, len = t.len;
        fl += 2.0 * len * k * k - (len + k) * k * k + 2.0 / 3.0 * k * k * k + 2.0 * len * k * k -
              2.0 / 3.0 * k * k * k;                                   // QR and Q
        fl += 54.0 * k * k * k + 2.0 * len * k * k;                    // Jacobi (nominal) and Q V
        by += 8.0 * (2.0 * t.M * (double)t.N + t.M * k + k);
    }
    ctx->flops += fl;
    Pack pk;
    const size_t ot = pk.add(tasks), op = pk.add(parts);
    Scratch s(ctx);
    unsigned char* d = upload_pack(s, pk);
    Prof pr(ctx, KK_SVD, fl, by);
    allow_smem(k_svd_site);
    int kmax = 1;
    for (const SvdSiteTask& t : tasks) kmax = std::max(kmax, t.k);
    k_svd_site<<<(unsigned)tasks.size(), block_for(kmax), smem, ctx->stream>>>((const SvdSiteTask*)(d + ot),
                                                                       (const SvdPart*)(d + op));
    count_launch(ctx);
    pr.done();
}

void launch_right_apply(Context* ctx, const std::vector<RTask>& tasks, const std::vector<RCopy>& copies,
                        const std::vector<RGemm>& gemms) {
    if (tasks.empty()) return;
    double fl = 0.0, by = 0.0;
    for (const RCopy& c : copies) by += 16.0 * c.rows * (double)c.cols;
    for (const RGemm& g : gemms) {
        fl += 2.0 * g.rows * (double)g.K * g.keep;
        by += 8.0 * ((double)g.rows * g.K + (double)g.K * g.keep + (double)g.rows * g.keep);
    }
    ctx->flops += fl;
    Pack pk;
    const size_t ot = pk.add(tasks), oc = pk.add(copies), og = pk.add(gemms);
    Scratch s(ctx);
    unsigned char* d = upload_pack(s, pk);
    Prof pr(ctx, KK_GEMM, fl, by);
    allow_smem(k_right_apply);
    k_right_apply<<<(unsigned)tasks.size(), kThreads, 0, ctx->stream>>>(
        (const RTask*)(d + ot), (const RCopy*)(d + oc), (const RGemm*)(d + og));
    count_launch(ctx);
    pr.done();
}

}  // namespace bsm

namespace bsm {

int launch_right_dyn(Context* ctx, const std::vector<DynTask>& tasks, const std::vector<DynPart>& parts) {
    if (tasks.empty()) return -1;
    size_t smem = 0;
    int kmax = 1;
    double fl = 0.0, by = 0.0;
    for (const DynTask& t : tasks) {
        smem = std::max(smem, svd_smem(t.M, t.ncols_pad));
        kmax = std::max(kmax, t.kpad);
        const double k = t.kpad, len = std::max(t.M, t.ncols_pad);
        fl += 4.0 * len * k * k + 54.0 * k * k * k + 2.0 * len * k * k;   // nominal upper bound
        by += 8.0 * ((double)t.M * t.ncols_pad + t.M * k + k * t.ncols_pad);
    }
    Pack pk;
    const size_t ot = pk.add(tasks), op = pk.add(parts);
    Scratch s(ctx);
    unsigned char* d = upload_pack(s, pk);
    Prof pr(ctx, KK_SVD, fl, by);
    allow_smem(k_right_dyn);
    k_right_dyn<<<(unsigned)tasks.size(), block_for(kmax), smem, ctx->stream>>>((const DynTask*)(d + ot),
                                                                               (const DynPart*)(d + op));
    count_launch(ctx);
    pr.done();
    return ctx->profiling ? (int)ctx->prof.size() - 1 : -1;
}

void launch_cut(Context* ctx, const CutTask& task, const std::vector<CutSector>& secs) {
    Pack pk;
    const size_t ot = pk.add(std::vector<CutTask>{task}), os = pk.add(secs);
    Scratch s(ctx);
    unsigned char* d = upload_pack(s, pk);
    const size_t smem = sizeof(double) * (size_t)task.cap_total + sizeof(int) * (3 * (size_t)task.cap_total +
                                                                                 task.n_sec + 1);
    Prof pr(ctx, KK_SUMSQ, 0.0, 8.0 * task.cap_total);
    allow_smem(k_cut_dyn);
    k_cut_dyn<<<1, kThreads, smem, ctx->stream>>>((const CutTask*)(d + ot), (const CutSector*)(d + os));
    count_launch(ctx);
    pr.done();
}

}  // namespace bsm
