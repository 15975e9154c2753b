// Fused per-site kernels of the truncation sweeps: each CTA owns one sector of
// the bond being orthogonalised or truncated and keeps its working set in
// shared memory, so one site costs one launch (left sweep) or two launches
// around the host's cut decision (right sweep).
#include <algorithm>
#include <cstring>
#include <mutex>

#include "dense_dev.cuh"
#include "kernels.h"

namespace bsm {
namespace {

using dev::kThreads;
constexpr int kSweepThreads = 512;   // block size limit of the kernels sized by block_for()
using dev::kWarps;
using dev::nthreads;
using dev::nwarps;

constexpr size_t kSweepSmem = 220 * 1024;

size_t left_smem(int M, int N) {
    const size_t k = (size_t)std::min(M, N);
    return sizeof(double) * ((size_t)M * N + (size_t)M * k + k + k * (size_t)N);
}

// values, their squares, sector ids, order, and n_sec + 1 offsets
size_t cut_smem(const CutTask& c) {
    return sizeof(double) * 2 * (size_t)c.cap_total + sizeof(int) * (2 * (size_t)c.cap_total + c.n_sec + 1);
}

size_t svd_smem(int M, int N) {
    const size_t k = (size_t)std::min(M, N), len = (size_t)std::max(M, N);
    return sizeof(double) * (2 * len * k + 2 * k * k + 3 * k);
}

// Global loads of data that other CTAs of the same launch may have written
// (persistent sweeps) go through L2; the per-site kernels use plain loads.
template <bool CG>
__device__ __forceinline__ double ldd(const double* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}
template <bool CG>
__device__ __forceinline__ int ldi(const int* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// One sector stack of a left-sweep site: gather, Householder QR with
// diag(R) >= 0, Q scattered to the new core t, R X written to the new core t+1.
// Rank-1 sector stack of the left sweep (A: M x N column-major, min(M, N) = 1)
// in closed form, diag(R) >= 0 as in the general path: a column x gives
// Q = x / ||x||, R = ||x|| (Q = e_0, R = 0 for x = 0); a row x gives Q = [sgn],
// R = sgn x with sgn = -1 exactly when x_0 < 0.
template <bool CG>
__device__ void left_rank1(const LeftTask& tk, const LeftSrc* __restrict__ srcs, const LeftX* __restrict__ xs,
                           const double* A, double* red) {
    const int M = tk.M, N = tk.N;
    if (N == 1) {
        double s = 0.0;
        for (int i = threadIdx.x; i < M; i += nthreads()) s = fma(A[i], A[i], s);
        s = dev::block_sum(s, red);
        const double f = s > 0.0 ? rsqrt(s) : 0.0;   // 1/r
        const double r = s * f;
        for (int si = tk.s_beg; si < tk.s_end; ++si) {
            const LeftSrc sr = srcs[si];
            for (int i = threadIdx.x; i < sr.rows; i += nthreads())
                sr.dst[i] = r > 0.0 ? A[sr.r0 + i] * f : (sr.r0 + i == 0 ? 1.0 : 0.0);
        }
        for (int x = tk.x_beg; x < tk.x_end; ++x) {
            const LeftX lx = xs[x];
            for (int c = threadIdx.x; c < lx.cols; c += nthreads()) lx.dst[c] = r * ldd<CG>(lx.X + c);
        }
        return;
    }
    // M == 1: one row of N entries
    const double sgn = A[0] < 0.0 ? -1.0 : 1.0;
    if (threadIdx.x == 0) srcs[tk.s_beg].dst[0] = sgn;
    for (int x = tk.x_beg; x < tk.x_end; ++x) {
        const LeftX lx = xs[x];
        for (int c = threadIdx.x; c < lx.cols; c += nthreads()) {
            double acc = 0.0;
            acc = sgn * dev::dot_global<false, CG>(A, 1, lx.X + c, lx.cols, N, 0.0);
            lx.dst[c] = acc;
        }
    }
}

template <bool CG>
__device__ void left_body(const LeftTask& tk, const LeftSrc* __restrict__ srcs, const LeftX* __restrict__ xs,
                          double* sm, double* red, double* sh) {
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
            A[(int64_t)c * M + sr.r0 + i] = ldd<CG>(sr.src + e);
        }
    }
    __syncthreads();
    if (M <= N) {
        // a stack with no more rows than columns is orthogonalised by Q = I:
        // the new core holds the rows of the identity, R = A carries the block
        // to the next site (any exact orthogonalisation serves the sweep: the
        // SVD sweep that follows fixes the gauge)
        for (int s = tk.s_beg; s < tk.s_end; ++s) {
            const LeftSrc sr = srcs[s];
            for (int64_t e = threadIdx.x; e < (int64_t)sr.rows * M; e += nthreads()) {
                const int i = (int)(e / M), c = (int)(e % M);
                sr.dst[e] = sr.r0 + i == c ? 1.0 : 0.0;
            }
        }
        for (int x = tk.x_beg; x < tk.x_end; ++x) {
            const LeftX lx = xs[x];
            for (int64_t e = threadIdx.x; e < (int64_t)M * lx.cols; e += nthreads()) {
                const int r = (int)(e / lx.cols), c = (int)(e % lx.cols);
                lx.dst[e] = dev::dot_global<false, CG>(A + r, M, lx.X + c, lx.cols, N, 0.0);
            }
        }
        return;
    }
    if (k == 1) {
        left_rank1<CG>(tk, srcs, xs, A, red);
        return;
    }
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
            acc = dev::dot_global<false, CG>(R + (int64_t)r * N + r, 1, lx.X + (int64_t)r * lx.cols + c, lx.cols, N - r, acc);
            lx.dst[e] = acc;
        }
    }
}

__global__ void __launch_bounds__(kSweepThreads) k_left_site(const LeftTask* __restrict__ tasks,
                                                        const LeftSrc* __restrict__ srcs,
                                                        const LeftX* __restrict__ xs) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ double sh[2];
    left_body<false>(tasks[blockIdx.x], srcs, xs, sm, red, sh);
}

__global__ void __launch_bounds__(kSweepThreads) k_svd_site(const SvdSiteTask* __restrict__ tasks,
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
// Index of the largest |v[c]|, c < n (ties: the smallest index), known to
// every thread.  red: 33 shared doubles.
__device__ __forceinline__ int block_argmax_abs(const double* v, int n, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long best = -1;
    int bi = 0;
    for (int c = threadIdx.x; c < n; c += nthreads()) {
        const long long a = dev::abs_key(v[c]);
        if (a > best) {
            best = a;
            bi = c;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    if (nwarps() == 1) return __shfl_sync(0xffffffffu, bi, 0);
    long long* rk = (long long*)red;   // 8 keys, then 8 indices
    __syncthreads();
    if (lane == 0) {
        rk[w] = best;
        rk[16 + w] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long b = rk[0];
        long long i = rk[16];
        for (int u = 1; u < nwarps(); ++u) {
            if (rk[u] > b || (rk[u] == b && rk[16 + u] < i)) {
                b = rk[u];
                i = rk[16 + u];
            }
        }
        rk[32] = i;
    }
    __syncthreads();
    return (int)rk[32];
}

// Rank-1 sector of the right sweep (a single row or column v, length len):
// the SVD in closed form with the conventions of the general path.  A column
// (M x 1) gives US = v, Vt = [1]; a row (1 x N) gives Vt = sgn v / sigma and
// US = sgn sigma, sgn making the largest |entry| of the Vt row positive.  A
// zero vector gives S = 0 (a value every cut discards).
__device__ void right_rank1(const DynTask& tk, const double* v, int len, int wide, double* red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < len; i += nthreads()) s = fma(v[i], v[i], s);
    s = dev::block_sum(s, red);
    const double rs = s > 0.0 ? rsqrt(s) : 0.0;   // 1/sigma
    const double sigma = s * rs;
    if (!wide) {
        for (int i = threadIdx.x; i < len; i += nthreads()) tk.US[(int64_t)i * tk.kpad] = sigma > 0.0 ? v[i] : 0.0;
        if (threadIdx.x == 0) {
            tk.Vt[0] = sigma > 0.0 ? 1.0 : 0.0;
            tk.S[0] = sigma;
            *tk.kact = 1;
        }
        return;
    }
    const int im = block_argmax_abs(v, len, red);
    const double sgn = v[im] < 0.0 ? -1.0 : 1.0;
    const double f = sgn * rs;
    for (int c = threadIdx.x; c < len; c += nthreads()) tk.Vt[c] = sigma > 0.0 ? v[c] * f : (c == 0 ? 1.0 : 0.0);
    if (threadIdx.x == 0) {
        tk.US[0] = sgn * sigma;
        tk.S[0] = sigma;
        *tk.kact = 1;
    }
}

template <bool CG>
__device__ void right_body(const DynTask& tk, double* sm, double* red,
                           double* sh, int* s_rot, int* s_cols) {
    const int np = tk.p_end - tk.p_beg;
    if (threadIdx.x < 2) {
        int c = 0;
        if ((int)threadIdx.x < np) {
            const DynPart& pt = tk.part[threadIdx.x];
            c = pt.keep ? ldi<CG>(pt.keep) : pt.xcols;
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
        const DynPart& pt = tk.part[p];
        const int cols = s_cols[p];
        for (int64_t e = threadIdx.x; e < (int64_t)M * cols; e += nthreads()) {
            const int i = (int)(e / cols), cc = (int)(e % cols), c = coff + cc;
            double v;
            if (pt.US) {
                v = 0.0;
                v = dev::dot_global<CG, CG>(pt.X + (int64_t)i * pt.xcols, 1, pt.US + cc, pt.ldus, pt.xcols, 0.0);
            } else {
                v = ldd<CG>(pt.X + (int64_t)i * pt.xcols + cc);
            }
            if (wide)
                B[(int64_t)i * N + c] = v;
            else
                B[(int64_t)c * M + i] = v;
        }
        coff += cols;
    }
    __syncthreads();
    if (k == 1) {
        right_rank1(tk, B, len, wide, red);
        return;
    }
    if (len <= 32 && k <= 16) {
        // small sector: one-sided Jacobi directly on B (no QR step)
        double* Vd = B + (int64_t)len * k;
        double* Sr = Vd + (int64_t)k * k;
        double* rinv = Sr + k;
        int* prm = (int*)(rinv + k);
        dev::jacobi_direct(B, Vd, Sr, len, k, red, s_rot);
        dev::svd_assemble_direct(B, Vd, Sr, rinv, prm, tk.S, tk.US, tk.Vt, M, N, k, len, wide, tk.kpad,
                                 tk.ncols_pad);
        __syncthreads();
        if (threadIdx.x == 0) *tk.kact = k;
        return;
    }
    dev::householder(B, tau, len, k, red, sh);
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += nthreads()) {
        const int j = (int)(e / k), i = (int)(e % k);
        G[e] = i >= j ? B[(int64_t)i * len + j] : 0.0;
    }
    dev::form_q(B, tau, Q, len, k);
    __syncthreads();
    dev::jacobi(G, V, Sraw, k, red, s_rot);
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

__global__ void __launch_bounds__(kSweepThreads) k_right_dyn(const DynTask* __restrict__ tasks) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ double sh[2];
    __shared__ int s_rot;
    __shared__ int s_cols[2];
    right_body<false>(tasks[blockIdx.x], sm, red, sh, &s_rot, s_cols);
}

// Pooled cut of one bond (one CTA): stable descending order with ties by
// (sector, index), then the sequential tolerance / cluster / cap rule; the
// products and sums are rounded individually (no contraction) so that the
// decisions equal the host rule.
template <bool CG>
__device__ void cut_body(const CutTask& tk, const CutSector* __restrict__ secs, double* sm, int* s_n_ptr) {
    int& s_n = *s_n_ptr;
    double* val = sm;
    double* sq = val + tk.cap_total;   // squares in sorted order
    int* sec = (int*)(sq + tk.cap_total);
    int* order = sec + tk.cap_total;
    int* off = order + tk.cap_total;   // n_sec + 1 (later: kept counts per sector)
    // counts of all sectors in parallel, then their offsets
    for (int i = threadIdx.x; i < tk.n_sec; i += nthreads()) off[i + 1] = ldi<CG>(secs[tk.s_beg + i].kact);
    __syncthreads();
    if (threadIdx.x == 0) {
        off[0] = 0;
        for (int i = 0; i < tk.n_sec; ++i) off[i + 1] += off[i];
        s_n = off[tk.n_sec];
    }
    __syncthreads();
    const int n = s_n;
    // every singular value in parallel (its sector by binary search over the offsets)
    for (int e = threadIdx.x; e < n; e += nthreads()) {
        int lo = 0, hi = tk.n_sec - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        val[e] = ldd<CG>(secs[tk.s_beg + lo].S + (e - off[lo]));
        sec[e] = lo;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += nthreads()) {
        const double ve = val[e];
        const long long se = dev::nonneg_key(ve);
        int rank = 0;
        for (int o = 0; o < n; ++o) {
            const long long so = dev::nonneg_key(val[o]);
            // entries are stored sector by sector and index by index, so ties
            // in value are ordered by position
            rank += (so > se || (so == se && o < e)) ? 1 : 0;
        }
        order[rank] = e;
        sq[rank] = __dmul_rn(ve, ve);
    }
    __syncthreads();
    __shared__ int s_keep;
    if (threadIdx.x == 0) {
        const double rtol = 1e-10;
        int keep = n;
        double acc = 0.0;
        while (keep > 0) {
            const double na = __dadd_rn(acc, sq[keep - 1]);
            if (na <= tk.tol2) {
                acc = na;
                keep -= 1;
            } else {
                break;
            }
        }
        const int keep0 = keep;
        while (keep > 0 && keep < n && val[order[keep]] >= __dmul_rn(val[order[keep - 1]], 1.0 - rtol)) keep += 1;
        double td = acc;   // discarded squares, summed from the smallest
        if (keep != keep0) {
            td = 0.0;
            for (int i = n - 1; i >= keep; --i) td = __dadd_rn(td, sq[i]);
        }
        double cd = 0.0;
        if (tk.r_max > 0 && keep > tk.r_max) {
            int k2 = tk.r_max;
            while (k2 > 0 && val[order[k2]] >= __dmul_rn(val[order[k2 - 1]], 1.0 - rtol)) k2 -= 1;
            if (k2 == 0) k2 = tk.r_max;
            for (int i = k2; i < keep; ++i) cd = __dadd_rn(cd, sq[i]);
            keep = k2;
        }
        tk.disc[0] = __dadd_rn(tk.disc[0], td);
        tk.disc[1] = __dadd_rn(tk.disc[1], cd);
        s_keep = keep;
    }
    for (int i = threadIdx.x; i < tk.n_sec; i += nthreads()) off[i] = 0;
    __syncthreads();
    const int keep = s_keep;
    for (int r = threadIdx.x; r < keep; r += nthreads()) atomicAdd(&off[sec[order[r]]], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < tk.n_sec; i += nthreads()) tk.keep[i] = off[i];
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_cut_dyn(const CutTask* __restrict__ tptr,
                                                      const CutSector* __restrict__ secs) {
    extern __shared__ double sm[];
    __shared__ int s_n;
    cut_body<false>(*tptr, secs, sm, &s_n);
}

// ---- persistent sweeps: one cooperative launch per sweep ----
//
// Every CTA of the grid is resident (cooperative launch), the sites are
// phases, and a phase ends when all CTAs have arrived; the last CTA to arrive
// runs the phase's serial tail (the pooled cut of the right sweep) before it
// releases the others.  Waits are bounded by the global timer: a CTA that
// waits longer than kWaitLimitNs sets gs->err and every CTA returns.

constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // 1 s

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Phase p ends: every CTA arrives at a monotonic counter (acquire-release at
// GPU scope, so the CTA's writes before the barrier are visible to every CTA
// after it); the last CTA to arrive releases the phase, the others poll with
// acquire loads.  Returns false when the wait gave up (error word set).
__device__ bool phase_end(GridSync* gs, unsigned int p, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t;
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(t) : "l"(&gs->arrive) : "memory");
        if (t == (p + 1) * gridDim.x - 1) {
            asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(&gs->release), "r"(p + 1) : "memory");
            *s_flag = 2;
        } else {
            const unsigned long long t0 = global_ns();
            int ok = 1;
            for (;;) {
                unsigned int r;
                asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(r) : "l"(&gs->release) : "memory");
                if (r >= p + 1) break;
                if (*(volatile int*)&gs->err) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > kWaitLimitNs) {
                    atomicExch(&gs->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
            *s_flag = ok ? 2 : 3;
        }
    }
    __syncthreads();
    return *s_flag == 2;
}

__global__ void __launch_bounds__(kSweepThreads) k_left_sweep(const LeftTask* __restrict__ tasks,
                                                         const LeftSrc* __restrict__ srcs,
                                                         const LeftX* __restrict__ xs,
                                                         const int* __restrict__ phase_beg, int n_phase,
                                                         GridSync* gs) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ double sh[2];
    __shared__ int s_flag;
    for (int p = 0; p < n_phase; ++p) {
        for (int ti = phase_beg[p] + (int)blockIdx.x; ti < phase_beg[p + 1]; ti += (int)gridDim.x) {
            __syncthreads();
            left_body<true>(tasks[ti], srcs, xs, sm, red, sh);
        }
        if (p + 1 < n_phase && !phase_end(gs, (unsigned)p, &s_flag)) return;
    }
}

// cp.async of 16 bytes (global -> shared), completed by cp_async_wait_all.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// phase_beg (n_phase + 1 ints) is staged in shared memory behind the body's
// working set (offset pb_off bytes); the descriptor of a CTA's first task of
// phase p + 1 is copied asynchronously while phase p runs.
__global__ void __launch_bounds__(kSweepThreads) k_right_sweep(const DynTask* __restrict__ tasks,
                                                          const int* __restrict__ phase_beg,
                                                          const CutTask* __restrict__ cuts,
                                                          const CutSector* __restrict__ secs, int n_phase,
                                                          int pb_off, GridSync* gs) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ double sh[2];
    __shared__ int s_rot;
    __shared__ int s_cols[2];
    __shared__ int s_n;
    __shared__ int s_flag;
    __shared__ DynTask s_task[2];
    int* pb = (int*)((char*)sm + pb_off);
    for (int i = threadIdx.x; i <= n_phase; i += nthreads()) pb[i] = phase_beg[i];
    __syncthreads();
    constexpr int kChunks = (int)(sizeof(DynTask) / 16);
    auto prefetch = [&](int p) {
        if (p < n_phase) {
            const int ti = pb[p] + (int)blockIdx.x;
            if (ti < pb[p + 1] && (int)threadIdx.x < kChunks)
                cp_async16((char*)&s_task[p & 1] + 16 * threadIdx.x, (const char*)(tasks + ti) + 16 * threadIdx.x);
        }
        cp_async_commit();
    };
    prefetch(0);
    for (int p = 0; p < n_phase; ++p) {
        cp_async_wait_all();
        __syncthreads();
        prefetch(p + 1);
        for (int ti = pb[p] + (int)blockIdx.x; ti < pb[p + 1]; ti += (int)gridDim.x) {
            __syncthreads();
            const bool first = ti == pb[p] + (int)blockIdx.x;
            const DynTask& tk = first ? s_task[p & 1] : tasks[ti];
            right_body<true>(tk, sm, red, sh, &s_rot, s_cols);
            // the CTA that completes the last task of this truncation's bond runs its cut
            __syncthreads();
            const CutTask& ct = cuts[tk.cut];
            if (ct.n_tasks == 1) {
                // the only sector of this truncation's bond: its own CTA cuts
                cut_body<true>(ct, secs, sm, &s_n);
            } else {
                if (threadIdx.x == 0) {
                    unsigned int old;
                    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;"
                                 : "=r"(old)
                                 : "l"((unsigned int*)ct.done)
                                 : "memory");
                    s_flag = (int)old == ct.n_tasks - 1 ? 1 : 0;
                }
                __syncthreads();
                if (s_flag) cut_body<true>(ct, secs, sm, &s_n);
            }
        }
        if (p + 1 < n_phase && !phase_end(gs, (unsigned)p, &s_flag)) {
            cp_async_wait_all();
            return;
        }
    }
    cp_async_wait_all();
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
// One warp per column pair of a Jacobi round (k/2 pairs), at most max_warps
// (<= kSweepThreads / 32; the block argmax keeps 16 keys in red[]).  The SVD
// kernels take up to 16 warps; the QR kernels keep 8, where more warps only
// lengthen the barriers between reflectors.
int block_for(int kmax, int max_warps = 8) { return 32 * std::max(1, std::min(max_warps, (kmax + 1) / 2)); }
constexpr int kSvdWarps = kSweepThreads / 32;

// The attributes are per function and per process: set them once per kernel.
template <class F>
void allow_smem(F* kern) {
    static std::mutex mu;
    static std::vector<const void*> done;
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(done.begin(), done.end(), (const void*)kern) != done.end()) return;
    BSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmem));
    BSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared));
    done.push_back((const void*)kern);
}

// Largest grid of `kern` whose CTAs are all resident at once (0: none).
template <class F>
int coresident_ctas(F* kern, int threads, size_t smem) {
    int per_sm = 0, dev = 0, nsm = 0;
    BSM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    BSM_CUDA(cudaGetDevice(&dev));
    BSM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    return per_sm * nsm;
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


// Environment sweep: every phase is a set of independent output tiles of
// grouped GEMMs whose inputs may have been written in earlier phases (loads go
// through L2); one thread per output entry, the K loop reading A and B
// directly so that no FP64 instruction is spent on padding.
constexpr int kEnvThreads = 128;

// One phase boundary between two CTAs; CTA skip_cta returns without arriving.
__global__ void k_grid_wait_check(int skip_cta, GridSync* gs) {
    __shared__ int s_flag;
    if ((int)blockIdx.x == skip_cta) return;
    phase_end(gs, 0u, &s_flag);
}

__global__ void __launch_bounds__(kEnvThreads) k_env_sweep_t(const EnvOutT* __restrict__ outs,
                                                             const EnvInT* __restrict__ ins,
                                                             const EnvTileT* __restrict__ tiles,
                                                             const int* __restrict__ phase_beg, int n_phase,
                                                             const EnvGroupPhase* __restrict__ gph,
                                                             const EnvMemberFac* __restrict__ mfac,
                                                             const double* __restrict__ ftab, int K,
                                                             const double* b0, const double* b1, const double* b2,
                                                             const double* b3,
                                                             const double* const* __restrict__ finals,
                                                             const int* __restrict__ final_beg, int n_prob,
                                                             double* __restrict__ res, GridSync* gs) {
    __shared__ int s_flag;
    const double* bases[4] = {b0, b1, b2, b3};
    for (int p = 0; p < n_phase; ++p) {
        for (int ti = phase_beg[p] + (int)blockIdx.x; ti < phase_beg[p + 1]; ti += (int)gridDim.x) {
            const EnvTileT tl = tiles[ti];
            const EnvOutT o = outs[tl.out];
            const EnvGroupPhase g = gph[o.gp];
            const EnvMemberFac mf = mfac[g.mem_beg + tl.member];
            const int64_t mem = tl.member;
            double* C = const_cast<double*>(bases[o.cbuf]) + g.base[o.cbuf] + mem * g.stride[o.cbuf] + o.coff;
            const int tm = min(32, o.M - tl.m0), tn = min(32, o.N - tl.n0);
            for (int e = threadIdx.x; e < tm * tn; e += kEnvThreads) {
                const int m = tl.m0 + e / tn, n = tl.n0 + e % tn;
                double acc = 0.0;
                for (int c = o.beg; c < o.end; ++c) {
                    const EnvInT in = ins[c];
                    const double* A = in.abuf < 0 ? in.A : bases[in.abuf] + g.base[in.abuf] + mem * g.stride[in.abuf] + in.aoff;
                    const double* B = in.bbuf < 0 ? in.B : bases[in.bbuf] + g.base[in.bbuf] + mem * g.stride[in.bbuf] + in.boff;
                    double alpha = in.w;
                    if (in.so >= 0) {
                        alpha += in.shift_flag ? g.shift : 0.0;
                        const int ra = mf.row[in.so], rb = mf.row[2 + in.si];
                        if (ra >= 0) alpha *= ftab[(int64_t)ra * K + in.site];
                        if (rb >= 0) alpha *= ftab[(int64_t)rb * K + in.site];
                    }
                    double part;
                    if (in.transA)
                        part = dev::dot_global<true, true>(A + m, in.lda, B + n, in.ldb, in.K, 0.0);
                    else
                        part = dev::dot_global<true, true>(A + (int64_t)m * in.lda, 1, B + n, in.ldb, in.K, 0.0);
                    acc = fma(alpha, part, acc);
                }
                C[(int64_t)m * o.ldc + n] = acc;
            }
        }
        if (!phase_end(gs, (unsigned)p, &s_flag)) return;
    }
    if (blockIdx.x == 0)
        for (int q = threadIdx.x; q < n_prob; q += kEnvThreads) {
            double sum = 0.0;
            for (int i = final_beg[q]; i < final_beg[q + 1]; ++i) sum += __ldcg(finals[i]);
            res[q] = sum;
        }
}


// ---- one-sided Jacobi of large matrices across the grid ----
//
// The cyclic round-robin ordering of dev::jacobi rotates, in every round, k/2
// disjoint column pairs of a matrix.  Here the pairs of all unfinished
// matrices of a round are spread over every warp of the grid (one pair per
// warp at a time), and a grid-wide phase ends each round: columns are disjoint
// within a round, so nothing else needs ordering.  Same rotation formula and
// stopping rules as dev::jacobi; G and V live in global memory and are read
// through L2 (other SMs wrote them in earlier rounds).  A sweep without a
// rotation finishes a matrix; the flags of a sweep are read after its last
// round by every CTA, so all CTAs take the same decisions and run the same
// number of phases.
constexpr int kJacGridMaxTasks = 64;

__device__ __forceinline__ void jg_locate(const JacTask* tasks, int n_tasks, const unsigned char* done, int round,
                                          int u, int* t_out, int* pi_out) {
    int base = 0;
    for (int t = 0; t < n_tasks; ++t) {
        const int k = tasks[t].k, n2 = k + (k & 1);
        if (done[t] || round >= n2 - 1) continue;
        if (u < base + n2 / 2) {
            *t_out = t;
            *pi_out = u - base;
            return;
        }
        base += n2 / 2;
    }
    *t_out = -1;
}

__global__ void __launch_bounds__(kThreads) k_jacobi_grid(const JacTask* __restrict__ tasks, int n_tasks,
                                                          double* __restrict__ fro, int* __restrict__ rot_flags,
                                                          GridSync* gs, int* dev_err) {
    __shared__ int s_flag;
    __shared__ unsigned char s_done[kJacGridMaxTasks];
    const int lane = threadIdx.x & 31;
    const int wpb = kThreads / 32;
    const int gwarp = (int)blockIdx.x * wpb + (int)(threadIdx.x >> 5);
    const int nwarp = (int)gridDim.x * wpb;
    unsigned int ph = 0;
    // V = I and ||G||_F^2 of every matrix
    for (int t = 0; t < n_tasks; ++t) {
        const int k = tasks[t].k;
        const int64_t kk = (int64_t)k * k;
        double f = 0.0;
        for (int64_t e = (int64_t)gwarp * 32 + lane; e < kk; e += (int64_t)nwarp * 32) {
            const double v = tasks[t].G[e];
            f += v * v;
            tasks[t].V[e] = (e % k) == (e / k) ? 1.0 : 0.0;
        }
        f = dev::warp_sum(f);
        if (lane == 0 && f != 0.0) atomicAdd(&fro[t], f);
    }
    if ((int)threadIdx.x < n_tasks) s_done[threadIdx.x] = tasks[threadIdx.x].k <= 1;
    if (!phase_end(gs, ph++, &s_flag)) {
        if (threadIdx.x == 0) atomicOr(dev_err, 1);
        return;
    }
    int n2max = 0, total_cols = 0;
    for (int t = 0; t < n_tasks; ++t) {
        n2max = max(n2max, tasks[t].k + (tasks[t].k & 1));
        total_cols += tasks[t].k;
    }
    for (int sweep = 0; sweep < dev::kMaxSweeps; ++sweep) {
        for (int round = 0; round < n2max - 1; ++round) {
            int U = 0;
            for (int t = 0; t < n_tasks; ++t) {
                const int n2 = tasks[t].k + (tasks[t].k & 1);
                if (!s_done[t] && round < n2 - 1) U += n2 / 2;
            }
            for (int u = gwarp; u < U; u += nwarp) {
                int t, pi;
                jg_locate(tasks, n_tasks, s_done, round, u, &t, &pi);
                if (t < 0) continue;
                const int k = tasks[t].k, n2 = k + (k & 1);
                int p = dev::rr_player(pi, round, n2), q = dev::rr_player(n2 - 1 - pi, round, n2);
                if (p >= k || q >= k) continue;
                if (p > q) {
                    const int tmp = p;
                    p = q;
                    q = tmp;
                }
                double* Gp = tasks[t].G + (int64_t)p * k;
                double* Gq = tasks[t].G + (int64_t)q * k;
                double a = 0.0, b = 0.0, g = 0.0;
                for (int i = lane; i < k; i += 32) {
                    const double xp = __ldcg(Gp + i), xq = __ldcg(Gq + i);
                    a += xp * xp;
                    b += xq * xq;
                    g += xp * xq;
                }
                a = dev::warp_sum(a);
                b = dev::warp_sum(b);
                g = dev::warp_sum(g);
                const double tol = (double)k * DBL_EPSILON;
                const double tiny2 = tol * tol * __ldcg(&fro[t]);
                if (g != 0.0 && fabs(g) > tol * sqrt(a * b) && fmin(a, b) > tiny2) {
                    const double zeta = (b - a) / (2.0 * g);
                    const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double c = 1.0 / sqrt(1.0 + tt * tt), sn = c * tt;
                    double* Vp = tasks[t].V + (int64_t)p * k;
                    double* Vq = tasks[t].V + (int64_t)q * k;
                    for (int i = lane; i < k; i += 32) {
                        const double xp = __ldcg(Gp + i), xq = __ldcg(Gq + i);
                        Gp[i] = c * xp - sn * xq;
                        Gq[i] = sn * xp + c * xq;
                        const double vp = __ldcg(Vp + i), vq = __ldcg(Vq + i);
                        Vp[i] = c * vp - sn * vq;
                        Vq[i] = sn * vp + c * vq;
                    }
                    if (lane == 0) rot_flags[t * dev::kMaxSweeps + sweep] = 1;
                }
            }
            if (!phase_end(gs, ph++, &s_flag)) {
                if (threadIdx.x == 0) atomicOr(dev_err, 1);
                return;
            }
        }
        if ((int)threadIdx.x < n_tasks && !s_done[threadIdx.x])
            s_done[threadIdx.x] = __ldcg(&rot_flags[threadIdx.x * dev::kMaxSweeps + sweep]) == 0;
        __syncthreads();
        bool all = true;
        for (int t = 0; t < n_tasks; ++t) all = all && s_done[t];
        if (all) break;
    }
    // column norms of the rotated G
    for (int u = gwarp; u < total_cols; u += nwarp) {
        int t = 0, base = 0;
        while (u >= base + tasks[t].k) {
            base += tasks[t].k;
            ++t;
        }
        const int k = tasks[t].k, j = u - base;
        const double* Gj = tasks[t].G + (int64_t)j * k;
        double a = 0.0;
        for (int i = lane; i < k; i += 32) {
            const double x = __ldcg(Gj + i);
            a += x * x;
        }
        a = dev::warp_sum(a);
        if (lane == 0) tasks[t].Sraw[j] = sqrt(a);
    }
}

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
        if (t.M > t.N)   // stacks with M <= N take Q = I
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

void launch_svd_site(Context* ctx, const std::vector<SvdSiteTask>& tasks, const std::vector<SvdPart>& parts,
                     Scratch& keep, bool on_side) {
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
    unsigned char* d = upload_pack(keep, pk);
    on_side = on_side && !ctx->profiling;   // profiled launches stay on the context stream
    Prof pr(ctx, KK_SVD, fl, by);
    allow_smem(k_svd_site);
    int kmax = 1;
    for (const SvdSiteTask& t : tasks) kmax = std::max(kmax, t.k);
    const cudaStream_t st = on_side ? ctx->fork_side() : ctx->stream;
    k_svd_site<<<(unsigned)tasks.size(), block_for(kmax, kSvdWarps), smem, st>>>((const SvdSiteTask*)(d + ot),
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

// Copies of each task's parts into the task (a sector has at most two: sigma 0 and 1).
std::vector<DynTask> with_parts(const std::vector<DynTask>& tasks, const std::vector<DynPart>& parts) {
    std::vector<DynTask> out = tasks;
    for (DynTask& t : out) {
        BSM_REQUIRE(t.p_end - t.p_beg >= 0 && t.p_end - t.p_beg <= 2, BSMPS_ERR_INVALID_ARG,
                    "a sector has at most two parts");
        for (int i = 0; i < t.p_end - t.p_beg; ++i) t.part[i] = parts[t.p_beg + i];
    }
    return out;
}

int launch_right_dyn(Context* ctx, const std::vector<DynTask>& tasks_in, const std::vector<DynPart>& parts) {
    if (tasks_in.empty()) return -1;
    const std::vector<DynTask> tasks = with_parts(tasks_in, parts);
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
    const size_t ot = pk.add(tasks);
    Scratch s(ctx);
    unsigned char* d = upload_pack(s, pk);
    Prof pr(ctx, KK_SVD, fl, by);
    allow_smem(k_right_dyn);
    k_right_dyn<<<(unsigned)tasks.size(), block_for(kmax, kSvdWarps), smem, ctx->stream>>>((const DynTask*)(d + ot));
    count_launch(ctx);
    pr.done();
    return ctx->profiling ? (int)ctx->prof.size() - 1 : -1;
}

void launch_cut(Context* ctx, const CutTask& task, const std::vector<CutSector>& secs) {
    Pack pk;
    const size_t ot = pk.add(std::vector<CutTask>{task}), os = pk.add(secs);
    Scratch s(ctx);
    unsigned char* d = upload_pack(s, pk);
    const size_t smem = cut_smem(task);
    Prof pr(ctx, KK_SUMSQ, 0.0, 8.0 * task.cap_total);
    allow_smem(k_cut_dyn);
    k_cut_dyn<<<1, kThreads, smem, ctx->stream>>>((const CutTask*)(d + ot), (const CutSector*)(d + os));
    count_launch(ctx);
    pr.done();
}

bool launch_left_sweep(Context* ctx, const std::vector<LeftTask>& tasks, const std::vector<LeftSrc>& srcs,
                       const std::vector<LeftX>& xs, const std::vector<int>& phase_beg, GridSync* gs) {
    const int n_phase = (int)phase_beg.size() - 1;
    if (n_phase <= 0 || tasks.empty()) return false;
    size_t smem = 0;
    int kmax = 1, maxt = 1;
    double fl = 0.0, by = 0.0;
    for (const LeftTask& t : tasks) {
        smem = std::max(smem, left_smem(t.M, t.N));
        kmax = std::max(kmax, 2 * t.k);
        const double m = t.M, n = t.N, k = t.k;
        if (t.M > t.N)   // stacks with M <= N take Q = I
            fl += 2.0 * m * n * k - (m + n) * k * k + 2.0 / 3.0 * k * k * k + 2.0 * m * k * k - 2.0 / 3.0 * k * k * k;
        by += 8.0 * (m * n + m * k);
        for (int x = t.x_beg; x < t.x_end; ++x) {
            fl += 2.0 * k * n * xs[x].cols;
            by += 8.0 * (n + k) * xs[x].cols;
        }
    }
    for (int p = 0; p < n_phase; ++p) maxt = std::max(maxt, phase_beg[p + 1] - phase_beg[p]);
    const int threads = block_for(kmax);
    allow_smem(k_left_sweep);
    const int cap = coresident_ctas(k_left_sweep, threads, smem);
    if (cap <= 0) return false;
    const int grid = std::min(maxt, cap);
    ctx->flops += fl;
    Pack pk;
    const size_t ot = pk.add(tasks), os = pk.add(srcs), ox = pk.add(xs), op = pk.add(phase_beg);
    Scratch s(ctx);
    unsigned char* d = upload_pack(s, pk);
    const LeftTask* a0 = (const LeftTask*)(d + ot);
    const LeftSrc* a1 = (const LeftSrc*)(d + os);
    const LeftX* a2 = (const LeftX*)(d + ox);
    const int* a3 = (const int*)(d + op);
    int a4 = n_phase;
    GridSync* a5 = gs;
    void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5};
    Prof pr(ctx, KK_QR, fl, by);
    BSM_CUDA(cudaLaunchCooperativeKernel((const void*)k_left_sweep, dim3(grid), dim3(threads), args, smem,
                                         ctx->stream));
    count_launch(ctx);
    pr.done();
    return true;
}

bool launch_right_sweep(Context* ctx, const std::vector<DynTask>& tasks_in, const std::vector<DynPart>& parts,
                        const std::vector<int>& phase_beg, const std::vector<CutTask>& cuts,
                        const std::vector<CutSector>& secs, GridSync* gs, int* prof_idx) {
    *prof_idx = -1;
    const int n_phase = (int)phase_beg.size() - 1;
    if (n_phase <= 0 || cuts.empty()) return false;
    const std::vector<DynTask> tasks = with_parts(tasks_in, parts);
    size_t smem = 0;
    int kmax = 1, maxt = 1;
    double by = 0.0;
    for (const DynTask& t : tasks) {
        smem = std::max(smem, svd_smem(t.M, t.ncols_pad));
        kmax = std::max(kmax, t.kpad);
        by += 8.0 * ((double)t.M * t.ncols_pad + (double)t.M * t.kpad + (double)t.kpad * t.ncols_pad);
    }
    for (const CutTask& c : cuts) smem = std::max(smem, cut_smem(c));
    for (int p = 0; p < n_phase; ++p) maxt = std::max(maxt, phase_beg[p + 1] - phase_beg[p]);
    const size_t pb_off = (smem + 15) & ~size_t(15);   // phase_beg staged behind the working set
    smem = pb_off + sizeof(int) * (size_t)(n_phase + 1);
    if (smem > kSweepSmem) return false;
    const int threads = block_for(kmax, kSvdWarps);
    allow_smem(k_right_sweep);
    const int cap = coresident_ctas(k_right_sweep, threads, smem);
    if (cap <= 0) return false;
    const int grid = std::min(maxt, cap);
    Pack pk;
    const size_t ot = pk.add(tasks), oph = pk.add(phase_beg), oc = pk.add(cuts), os = pk.add(secs);
    Scratch s(ctx);
    unsigned char* d = upload_pack(s, pk);
    const DynTask* a0 = (const DynTask*)(d + ot);
    const int* a1 = (const int*)(d + oph);
    const CutTask* a2 = (const CutTask*)(d + oc);
    const CutSector* a3 = (const CutSector*)(d + os);
    int a4 = n_phase;
    int a5 = (int)pb_off;
    GridSync* a6 = gs;
    void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6};
    Prof pr(ctx, KK_SVD, 0.0, by);   // flops entered by the caller once the ranks are known
    BSM_CUDA(cudaLaunchCooperativeKernel((const void*)k_right_sweep, dim3(grid), dim3(threads), args, smem,
                                         ctx->stream));
    count_launch(ctx);
    pr.done();
    if (ctx->profiling) *prof_idx = (int)ctx->prof.size() - 1;
    return true;
}

int check_grid_wait(Context* ctx, int skip_cta) {
    Scratch s(ctx);
    GridSync* gs = (GridSync*)ctx->alloc(sizeof(GridSync));
    s.ptrs.push_back(gs);
    BSM_CUDA(cudaMemsetAsync(gs, 0, sizeof(GridSync), ctx->stream));
    int a0 = skip_cta;
    GridSync* a1 = gs;
    void* args[] = {&a0, &a1};
    BSM_CUDA(cudaLaunchCooperativeKernel((const void*)k_grid_wait_check, dim3(2), dim3(32), args, 0, ctx->stream));
    count_launch(ctx);
    GridSync h;
    BSM_CUDA(cudaMemcpyAsync(&h, gs, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    ctx->sync();
    return h.err;
}

bool launch_env_sweep_t(Context* ctx, const std::vector<EnvOutT>& outs, const std::vector<EnvInT>& ins,
                        const std::vector<EnvTileT>& tiles, const std::vector<int>& phase_beg,
                        const std::vector<EnvGroupPhase>& gph, const std::vector<EnvMemberFac>& mfac,
                        const std::vector<double>& ftab, int K, double* const base[4],
                        const std::vector<const double*>& finals, const std::vector<int>& final_beg, double* res,
                        GridSync* gs) {
    const int n_phase = (int)phase_beg.size() - 1;
    const int n_prob = (int)final_beg.size() - 1;
    if (n_phase <= 0 || n_prob <= 0) return false;
    int maxt = 1;
    for (int p = 0; p < n_phase; ++p) maxt = std::max(maxt, phase_beg[p + 1] - phase_beg[p]);
    double fl = 0.0, by = 0.0;
    std::vector<int> tiles_of(outs.size(), 0);   // flops per output template times its members
    for (const EnvTileT& t : tiles)
        if (t.m0 == 0 && t.n0 == 0) tiles_of[t.out] += 1;
    for (size_t o = 0; o < outs.size(); ++o)
        for (int c = outs[o].beg; c < outs[o].end; ++c) {
            fl += 2.0 * outs[o].M * outs[o].N * (double)ins[c].K * tiles_of[o];
            by += 8.0 * ((double)outs[o].M * ins[c].K + (double)ins[c].K * outs[o].N) * tiles_of[o];
        }
    const int cap = coresident_ctas(k_env_sweep_t, kEnvThreads, 0);
    if (cap <= 0) return false;
    const int grid = std::min(maxt, cap);
    ctx->flops += fl;
    Pack pk;
    const size_t oo = pk.add(outs), oi = pk.add(ins), ot = pk.add(tiles), op = pk.add(phase_beg), og = pk.add(gph),
                 om = pk.add(mfac), of = pk.add(ftab), ofi = pk.add(finals), ob = pk.add(final_beg);
    Scratch s(ctx);
    unsigned char* d = upload_pack(s, pk);
    const EnvOutT* a0 = (const EnvOutT*)(d + oo);
    const EnvInT* a1 = (const EnvInT*)(d + oi);
    const EnvTileT* a2 = (const EnvTileT*)(d + ot);
    const int* a3 = (const int*)(d + op);
    int a4 = n_phase;
    const EnvGroupPhase* a5 = (const EnvGroupPhase*)(d + og);
    const EnvMemberFac* a6 = (const EnvMemberFac*)(d + om);
    const double* a7 = ftab.empty() ? nullptr : (const double*)(d + of);
    int a8 = K;
    const double* a9 = base[0];
    const double* a10 = base[1];
    const double* a11 = base[2];
    const double* a12 = base[3];
    const double* const* a13 = (const double* const*)(d + ofi);
    const int* a14 = (const int*)(d + ob);
    int a15 = n_prob;
    double* a16 = res;
    GridSync* a17 = gs;
    void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8, &a9, &a10, &a11, &a12, &a13, &a14, &a15, &a16, &a17};
    Prof pr(ctx, KK_GEMM, fl, by);
    BSM_CUDA(cudaLaunchCooperativeKernel((const void*)k_env_sweep_t, dim3(grid), dim3(kEnvThreads), args, 0,
                                         ctx->stream));
    count_launch(ctx);
    pr.done();
    return true;
}

bool launch_jacobi_grid(Context* ctx, const std::vector<JacTask>& tasks_in) {
    const int cap = coresident_ctas(k_jacobi_grid, kThreads, 0);
    if (cap <= 0) return false;   // decided before any batch is launched
    int dev = 0, nsm = 0;
    BSM_CUDA(cudaGetDevice(&dev));
    BSM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    for (size_t b = 0; b < tasks_in.size(); b += kJacGridMaxTasks) {
        const std::vector<JacTask> tasks(tasks_in.begin() + b,
                                         tasks_in.begin() + std::min(tasks_in.size(), b + kJacGridMaxTasks));
        const int n = (int)tasks.size();
        int pairs = 0;
        for (const JacTask& t : tasks) pairs += (t.k + (t.k & 1)) / 2;
        // one warp per pair of the first round, at most one CTA per SM (fewer
        // arrivals per grid-wide wait)
        const int grid = std::max(1, std::min({cap, nsm, (pairs + kThreads / 32 - 1) / (kThreads / 32)}));
        Scratch s(ctx);
        const JacTask* d_t = s.up(tasks);
        double* fro = s.dbl((size_t)n);
        int* flags = (int*)ctx->alloc(sizeof(int) * (size_t)n * dev::kMaxSweeps);
        s.ptrs.push_back(flags);
        GridSync* gs = (GridSync*)ctx->alloc(sizeof(GridSync));
        s.ptrs.push_back(gs);
        BSM_CUDA(cudaMemsetAsync(fro, 0, sizeof(double) * n, ctx->stream));
        BSM_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)n * dev::kMaxSweeps, ctx->stream));
        BSM_CUDA(cudaMemsetAsync(gs, 0, sizeof(GridSync), ctx->stream));
        int* err = ctx->err_word();
        int a1 = n;
        void* args[] = {(void*)&d_t, &a1, &fro, &flags, &gs, &err};
        BSM_CUDA(cudaLaunchCooperativeKernel((const void*)k_jacobi_grid, dim3(grid), dim3(kThreads), args, 0,
                                             ctx->stream));
        count_launch(ctx);
    }
    return true;
}

}  // namespace bsm

