// Block-cooperative dense FP64 routines (one CTA of kThreads threads works on
// one small matrix): reductions, Householder QR, one-sided Jacobi and the SVD
// assembly used by the truncation kernels.
#pragma once

#include <cfloat>
#include <cstdint>

namespace bsm {
namespace dev {

constexpr int kThreads = 256;            // default block size of the batched kernels
constexpr int kWarps = kThreads / 32;
constexpr int kMaxSweeps = 40;

// The routines below work with any block size that is a multiple of 32
// (callers size small problems down to fewer warps).
__device__ __forceinline__ int nthreads() { return (int)blockDim.x; }
__device__ __forceinline__ int nwarps() { return (int)(blockDim.x >> 5); }

// One 32 x 32 output tile of a grouped FP64 GEMM, accumulated over one
// contribution alpha op(A) B (op(A): M x K, transA selects A^T stored K x M):
// the thread (ty, tx) of a 256-thread CTA owns rows m0 + ty + 8 r (r < 4) and
// column n0 + tx.  The K loop stages 32 x 32 chunks of op(A) and B in shared
// memory (As[k][m], Bs[k][n]); only the valid part of a chunk and the rows
// below M issue FP64 instructions.  In: any struct with A, B, K, lda, ldb,
// transA and alpha.
constexpr int kGemmTile = 32;
template <class In>
__device__ __forceinline__ void gemm_tile_accumulate(const In& in, int M, int N, int m0, int n0,
                                                     double (*As)[kGemmTile + 1], double (*Bs)[kGemmTile + 1],
                                                     double acc[4]) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k0 = 0; k0 < in.K; k0 += kGemmTile) {
        for (int idx = threadIdx.x; idx < kGemmTile * kGemmTile; idx += kThreads) {
            int mm, kk;
            if (in.transA) {
                kk = idx / kGemmTile;
                mm = idx % kGemmTile;
            } else {
                mm = idx / kGemmTile;
                kk = idx % kGemmTile;
            }
            const int gm = m0 + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < M && gk < in.K)
                v = in.transA ? in.A[(int64_t)gk * in.lda + gm] : in.A[(int64_t)gm * in.lda + gk];
            As[kk][mm] = in.alpha * v;
        }
        for (int idx = threadIdx.x; idx < kGemmTile * kGemmTile; idx += kThreads) {
            const int kk = idx / kGemmTile, nn = idx % kGemmTile;
            const int gk = k0 + kk, gn = n0 + nn;
            Bs[kk][nn] = (gk < in.K && gn < N) ? in.B[(int64_t)gk * in.ldb + gn] : 0.0;
        }
        __syncthreads();
        const int kk_end = min(kGemmTile, in.K - k0);
        for (int kk = 0; kk < kk_end; ++kk) {
            const double b = Bs[kk][tx];
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (m0 + ty + 8 * r < M) acc[r] = fma(As[kk][ty + 8 * r], b, acc[r]);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the block; every thread gets the result (red: 33 shared doubles)
__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    if (blockDim.x == 32) return v;   // one warp: no shared-memory stage
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Sum within aligned segments of S lanes (S a power of two, S <= 32); every
// lane of a segment receives its segment's sum.
__device__ __forceinline__ double seg_sum(double v, int S) {
    for (int o = S >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// acc + sum_{k < n} a[k sa] b[k sb] with the global loads issued eight terms
// at a time, so that a dot product of length n waits for about n/8 memory
// round trips instead of n.  CGA / CGB: loads of a / b through L2 (global
// data written by other CTAs of the same launch); otherwise plain loads (which
// also serve shared-memory operands).
template <bool CGA, bool CGB>
__device__ __forceinline__ double dot_global(const double* a, int64_t sa, const double* b, int64_t sb, int n,
                                             double acc) {
    for (int k0 = 0; k0 < n; k0 += 8) {
        double x[8], y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + u;
            if (k < n) {
                if constexpr (CGA) x[u] = __ldcg(a + (int64_t)k * sa);
                else x[u] = a[(int64_t)k * sa];
                if constexpr (CGB) y[u] = __ldcg(b + (int64_t)k * sb);
                else y[u] = b[(int64_t)k * sb];
            } else {
                x[u] = 0.0;
                y[u] = 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (k0 + u < n) acc = fma(x[u], y[u], acc);
    }
    return acc;
}

__device__ __forceinline__ int pow2_at_least(int n) {
    int s = 1;
    while (s < n) s <<= 1;
    return s;
}

// Householder reflector of the column (alpha, x) with ||x||^2 = s > 0:
// beta = -sign(alpha) n with n = ||(alpha, x)||, tau = (beta - alpha)/beta =
// 1 + |alpha|/n and scale = 1/(alpha - beta) = sign(alpha)/(|alpha| + n).
// On this GPU an FP64 square root or division costs about ten dependent FP64
// instructions; both quotients come from reciprocal square roots instead
// (1/n = rsqrt(n^2), 1/q = rsqrt(q)^2).
__device__ __forceinline__ void reflector(double alpha, double s, double* beta, double* tau, double* scale) {
    const double w = fma(alpha, alpha, s);
    const double rn = rsqrt(w);
    const double n = w * rn;
    const double aa = fabs(alpha);
    const double rq = rsqrt(aa + n);
    *beta = alpha >= 0.0 ? -n : n;
    *tau = fma(aa, rn, 1.0);
    *scale = (alpha >= 0.0 ? rq : -rq) * rq;
}

// householder() for M <= 32 rows: lanes are rows within aligned segments of
// S = pow2_at_least(M) lanes, so one warp instruction serves 32/S columns of
// the trailing update; every warp forms the reflector itself (no broadcast
// through shared memory), and the column's scaled v is stored after the
// barrier that ends the column.
__device__ __forceinline__ void householder_small(double* A, double* tau, int M, int N) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = nwarps();
    const int k = M < N ? M : N;
    const int S = pow2_at_least(M), G = 32 / S;
    const int i = lane % S, sg = lane / S;
    for (int j = 0; j < k; ++j) {
        const double xi = i < M ? A[(int64_t)j * M + i] : 0.0;
        const double s = seg_sum((i > j && i < M) ? xi * xi : 0.0, S);
        const double alpha = A[(int64_t)j * M + j];
        double tj = 0.0, scale = 0.0, beta = alpha;
        if (s != 0.0) reflector(alpha, s, &beta, &tj, &scale);
        if (tj != 0.0) {
            const double vi = (i > j && i < M) ? xi * scale : (i == j ? 1.0 : 0.0);
            for (int c0 = j + 1 + warp * G; c0 < N; c0 += nw * G) {
                const int c = c0 + sg;
                const bool own = c < N && i < M && i >= j;
                const double aic = own ? A[(int64_t)c * M + i] : 0.0;
                const double w = seg_sum(own ? vi * aic : 0.0, S);
                if (own) A[(int64_t)c * M + i] = fma(-(tj * w), vi, aic);
            }
        }
        __syncthreads();
        if (warp == 0 && sg == 0) {
            if (tj != 0.0) {
                if (i > j && i < M) A[(int64_t)j * M + i] = xi * scale;
                if (i == j) A[(int64_t)j * M + j] = beta;
            }
            if (i == 0) tau[j] = tj;
        }
    }
    __syncthreads();
}

// form_q() for M <= 32 rows (segment layout as in householder_small).
__device__ __forceinline__ void form_q_small(const double* A, const double* tau, double* Q, int M, int k) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = nwarps();
    const int S = pow2_at_least(M), G = 32 / S;
    const int i = lane % S, sg = lane / S;
    for (int64_t e = threadIdx.x; e < (int64_t)M * k; e += nthreads()) {
        const int r = (int)(e % M), c = (int)(e / M);
        Q[e] = r == c ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = k - 1; j >= 0; --j) {
        const double tj = tau[j];
        if (tj == 0.0) continue;
        const double vi = (i > j && i < M) ? A[(int64_t)j * M + i] : (i == j ? 1.0 : 0.0);
        for (int c0 = j + warp * G; c0 < k; c0 += nw * G) {
            const int c = c0 + sg;
            const bool own = c < k && i < M && i >= j;
            const double qic = own ? Q[(int64_t)c * M + i] : 0.0;
            const double w = seg_sum(own ? vi * qic : 0.0, S);
            if (own) Q[(int64_t)c * M + i] = fma(-(tj * w), vi, qic);
        }
        __syncthreads();
    }
}

// Householder factorisation of A (M x N, column-major, ld M) in place: R in the
// upper trapezoid, v_j below the diagonal (v_j = 1 implicit), tau[j].
// H = I - tau v v^T, beta = -sign(alpha) ||x||, tau = (beta - alpha)/beta,
// v = x/(alpha - beta).  sh: 2 shared doubles.
__device__ __forceinline__ void householder(double* A, double* tau, int M, int N, double* red, double* sh) {
    if (M <= 32) {
        householder_small(A, tau, M, N);
        return;
    }
    const int k = M < N ? M : N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < k; ++j) {
        double s = 0.0;
        for (int i = j + 1 + threadIdx.x; i < M; i += nthreads()) {
            const double v = A[(int64_t)j * M + i];
            s += v * v;
        }
        s = block_sum(s, red);
        if (threadIdx.x == 0) {
            const double alpha = A[(int64_t)j * M + j];
            if (s == 0.0) {
                sh[0] = 0.0;
                sh[1] = 0.0;
            } else {
                const double nrm = sqrt(alpha * alpha + s);
                const double beta = alpha >= 0.0 ? -nrm : nrm;
                sh[0] = (beta - alpha) / beta;
                sh[1] = 1.0 / (alpha - beta);
                A[(int64_t)j * M + j] = beta;
            }
            tau[j] = sh[0];
        }
        __syncthreads();
        const double tj = sh[0], scale = sh[1];
        if (tj != 0.0) {
            for (int i = j + 1 + threadIdx.x; i < M; i += nthreads()) A[(int64_t)j * M + i] *= scale;
            __syncthreads();
            for (int c = j + 1 + warp; c < N; c += nwarps()) {
                // read A(j, c) before the warp-synchronous reduction: lane 0 rewrites it after
                const double a_jc = A[(int64_t)c * M + j];
                double w = 0.0;
                for (int i = j + 1 + lane; i < M; i += 32) w += A[(int64_t)j * M + i] * A[(int64_t)c * M + i];
                w = warp_sum(w) + a_jc;
                const double tw = tj * w;
                if (lane == 0) A[(int64_t)c * M + j] -= tw;
                for (int i = j + 1 + lane; i < M; i += 32) A[(int64_t)c * M + i] -= tw * A[(int64_t)j * M + i];
            }
        }
        __syncthreads();
    }
}

// Q (M x k, column-major) = H_0 ... H_{k-1} applied to the first k columns of I.
__device__ __forceinline__ void form_q(const double* A, const double* tau, double* Q, int M, int k) {
    if (M <= 32) {
        form_q_small(A, tau, Q, M, k);
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t e = threadIdx.x; e < (int64_t)M * k; e += nthreads()) {
        const int i = (int)(e % M), c = (int)(e / M);
        Q[e] = i == c ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = k - 1; j >= 0; --j) {
        const double tj = tau[j];
        if (tj == 0.0) continue;
        for (int c = j + warp; c < k; c += nwarps()) {
            const double q_jc = Q[(int64_t)c * M + j];
            double w = 0.0;
            for (int i = j + 1 + lane; i < M; i += 32) w += A[(int64_t)j * M + i] * Q[(int64_t)c * M + i];
            w = warp_sum(w) + q_jc;
            const double tw = tj * w;
            if (lane == 0) Q[(int64_t)c * M + j] -= tw;
            for (int i = j + 1 + lane; i < M; i += 32) Q[(int64_t)c * M + i] -= tw * A[(int64_t)j * M + i];
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int rr_player(int pos, int round, int n2) {
    if (pos == 0) return 0;
    int v = pos - 1 + round;   // < 2 (n2 - 1) for round < n2 - 1
    if (v >= n2 - 1) v -= n2 - 1;
    return v + 1;
}

// Order of non-negative doubles through their bit patterns (integer compares
// instead of FP64 ones).
__device__ __forceinline__ long long nonneg_key(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ long long abs_key(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffLL; }

// sqrt(x) for x >= 0 from one reciprocal square root (about 2/3 of the cost of
// an FP64 square root here); 1 ulp-level accuracy.
__device__ __forceinline__ double sqrt_via_rsqrt(double x) { return x > 0.0 ? x * rsqrt(x) : 0.0; }

// Rotation (c, s) that makes the columns with squared norms a, b and inner
// product g orthogonal: with d = b - a, t = sign(zeta) 2|g| / (|d| + sqrt(d^2
// + 4 g^2)) equals sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) for zeta = d/(2g)
// (sign(zeta) = +1 at d = 0), c = 1/sqrt(1 + t^2), s = c t.
__device__ __forceinline__ void jacobi_rotation(double a, double b, double g, double* c, double* s) {
    const double d = b - a;
    const double r = sqrt(fma(d, d, 4.0 * g * g));
    const double sz = (d == 0.0 || (d > 0.0) == (g > 0.0)) ? 1.0 : -1.0;
    const double t = sz * (2.0 * fabs(g)) / (fabs(d) + r);
    *c = rsqrt(fma(t, t, 1.0));
    *s = *c * t;
}

// jacobi_rotation() with the angle taken in FP32: d = b - a and 2g are
// brought into FP32 range (scaled by a power of two when needed), t is formed
// in FP32, and c = rsqrt(1 + t^2), s = c t in FP64, so that c^2 + s^2 = 1
// within FP64 rounding.  The rotation is orthogonal in FP64 and only its angle
// carries the FP32 error, which leaves |g'| ~ 1e-7 |g| for the next sweep.
__device__ __forceinline__ void jacobi_rotation_fast(double a, double b, double g, double* c, double* s) {
    const double d = b - a, g2 = g + g;
    const int ed = (__double2hiint(d) >> 20) & 0x7ff, eg = (__double2hiint(g2) >> 20) & 0x7ff;
    const int e = ed > eg ? ed : eg;
    if (e < 2 || e > 2045) {   // zero, subnormal or non-finite scale: exact formula
        jacobi_rotation(a, b, g, c, s);
        return;
    }
    float df, gf;
    if (e >= 1023 - 60 && e <= 1023 + 60) {   // squares stay normal in FP32
        df = __double2float_rn(d);
        gf = __double2float_rn(g2);
    } else {
        const double sc = __hiloint2double((2046 - e) << 20, 0);   // 2^(1023 - e)
        df = __double2float_rn(d * sc);
        gf = __double2float_rn(g2 * sc);
    }
    // the angle only needs FP32 accuracy: hardware reciprocal square root and
    // fast division (the larger of |df|, |gf| is at least 2^-60, so both are in range)
    const float w = fmaf(df, df, gf * gf);
    const float r = w * rsqrtf(w);
    const float sz = (df == 0.0f || ((df > 0.0f) == (gf > 0.0f))) ? 1.0f : -1.0f;
    const double t = (double)(sz * __fdividef(fabsf(gf), fabsf(df) + r));
    const double cd = rsqrt(fma(t, t, 1.0));
    *c = cd;
    *s = cd * t;
}

// jacobi() for k <= 16: one round-robin pair per warp; the pair's three inner
// products are formed in aligned lane segments of S = pow2_at_least(k) lanes
// (S <= 8: a, b, g in three segments of one register; S = 16: a | b in one
// register, g in another), and the rotation of the G and V columns runs with
// lanes [0, S) on G and [S, 2S) on V.
__device__ __forceinline__ void jacobi_small(double* G, double* V, double* Sraw, int k, double* red, int* s_rot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double f = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += nthreads()) {
        const double v = G[e];
        f += v * v;
        V[e] = (e % k) == (e / k) ? 1.0 : 0.0;
    }
    f = block_sum(f, red);
    const double tol = (double)k * DBL_EPSILON;
    const double tol2 = tol * tol, tiny2 = tol2 * f;
    const int n2 = k + (k & 1);
    const int S = pow2_at_least(k);
    const int i = lane % S, sg = lane / S;
    for (int sweep = 0; sweep < kMaxSweeps && k > 1; ++sweep) {
        if (threadIdx.x == 0) *s_rot = 0;
        __syncthreads();
        for (int round = 0; round < n2 - 1; ++round) {
            for (int pi = warp; pi < n2 / 2; pi += nwarps()) {
                int p = rr_player(pi, round, n2), q = rr_player(n2 - 1 - pi, round, n2);
                if (p >= k || q >= k) continue;
                if (p > q) {
                    const int tmp = p;
                    p = q;
                    q = tmp;
                }
                const double xp = i < k ? G[(int64_t)p * k + i] : 0.0;
                const double xq = i < k ? G[(int64_t)q * k + i] : 0.0;
                double a, b, g;
                if (S <= 8) {
                    // segment 0: xp xp, 1: xq xq, 2: xp xq (segment 3 idle)
                    const double u = sg == 1 ? xq : xp, w = sg == 0 ? xp : xq;
                    const double prod = seg_sum(sg < 3 ? u * w : 0.0, S);
                    a = __shfl_sync(0xffffffffu, prod, 0);
                    b = __shfl_sync(0xffffffffu, prod, S);
                    g = __shfl_sync(0xffffffffu, prod, 2 * S);
                } else {
                    const double u = sg == 0 ? xp : xq;
                    const double ab = seg_sum(u * u, 16);
                    const double pg = seg_sum(xp * xq, 16);
                    a = __shfl_sync(0xffffffffu, ab, 0);
                    b = __shfl_sync(0xffffffffu, ab, 16);
                    g = __shfl_sync(0xffffffffu, pg, 0);
                }
                if (g * g > tol2 * (a * b) && nonneg_key(a) > nonneg_key(tiny2) &&
                    nonneg_key(b) > nonneg_key(tiny2)) {
                    double c, s;
                    jacobi_rotation_fast(a, b, g, &c, &s);
                    if (lane < 2 * S && i < k) {
                        double* X = lane < S ? G : V;
                        const double vp = X[(int64_t)p * k + i], vq = X[(int64_t)q * k + i];
                        X[(int64_t)p * k + i] = c * vp - s * vq;
                        X[(int64_t)q * k + i] = s * vp + c * vq;
                    }
                    if (lane == 0) *s_rot = 1;
                }
            }
            __syncthreads();
        }
        const int rot = *s_rot;
        __syncthreads();
        if (!rot) break;
    }
    // column norms: 32/S columns per warp instruction
    const int Gc = 32 / S;
    for (int j0 = warp * Gc; j0 < k; j0 += nwarps() * Gc) {
        const int j = j0 + sg;
        const double x = (j < k && i < k) ? G[(int64_t)j * k + i] : 0.0;
        const double a = seg_sum(x * x, S);
        if (j < k && i == 0) Sraw[j] = sqrt_via_rsqrt(a);
    }
    __syncthreads();
}

// One-sided Jacobi directly on B (rows x k, column-major, rows <= 32, k <=
// 16) with the rotations accumulated in V (k x k): no QR step.  One pair per
// warp; the pair's inner products reduce in aligned segments of S =
// pow2_at_least(rows) lanes.  Threshold |g| > tol sqrt(a b) with tol = rows
// eps, columns below the numerical-zero level (rows eps)^2 ||B||_F^2 are left
// alone.  Sraw: column norms of the result.
__device__ __forceinline__ void jacobi_direct(double* B, double* V, double* Sraw, int rows, int k, double* red,
                                              int* s_rot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double f = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)rows * k; e += nthreads()) {
        const double v = B[e];
        f += v * v;
    }
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += nthreads()) V[e] = (e % k) == (e / k) ? 1.0 : 0.0;
    f = block_sum(f, red);
    const double tol = (double)rows * DBL_EPSILON;
    const double tol2 = tol * tol, tiny2 = tol2 * f;
    const int n2 = k + (k & 1);
    const int S = pow2_at_least(rows);
    const int i = lane % S, sg = lane / S;
    for (int sweep = 0; sweep < kMaxSweeps && k > 1; ++sweep) {
        if (threadIdx.x == 0) *s_rot = 0;
        __syncthreads();
        for (int round = 0; round < n2 - 1; ++round) {
            for (int pi = warp; pi < n2 / 2; pi += nwarps()) {
                int p = rr_player(pi, round, n2), q = rr_player(n2 - 1 - pi, round, n2);
                if (p >= k || q >= k) continue;
                if (p > q) {
                    const int tmp = p;
                    p = q;
                    q = tmp;
                }
                const double xp = i < rows ? B[(int64_t)p * rows + i] : 0.0;
                const double xq = i < rows ? B[(int64_t)q * rows + i] : 0.0;
                double a, b, g;
                if (S <= 8) {
                    const double u = sg == 1 ? xq : xp, w = sg == 0 ? xp : xq;
                    const double prod = seg_sum(sg < 3 ? u * w : 0.0, S);
                    a = __shfl_sync(0xffffffffu, prod, 0);
                    b = __shfl_sync(0xffffffffu, prod, S);
                    g = __shfl_sync(0xffffffffu, prod, 2 * S);
                } else if (S == 16) {
                    const double u = sg == 0 ? xp : xq;
                    const double ab = seg_sum(u * u, 16);
                    const double pg = seg_sum(xp * xq, 16);
                    a = __shfl_sync(0xffffffffu, ab, 0);
                    b = __shfl_sync(0xffffffffu, ab, 16);
                    g = __shfl_sync(0xffffffffu, pg, 0);
                } else {
                    a = warp_sum(xp * xp);
                    b = warp_sum(xq * xq);
                    g = warp_sum(xp * xq);
                }
                if (g * g > tol2 * (a * b) && nonneg_key(a) > nonneg_key(tiny2) &&
                    nonneg_key(b) > nonneg_key(tiny2)) {
                    double c, s;
                    jacobi_rotation_fast(a, b, g, &c, &s);
                    if (S <= 16) {
                        // lanes [0, S): rows of B; lanes [S, 2S): rows of V (k <= rows <= S)
                        const bool onB = lane < S;
                        if ((onB && i < rows) || (!onB && lane < 2 * S && i < k)) {
                            double* X = onB ? B : V;
                            const int ld = onB ? rows : k;
                            const double vp = X[(int64_t)p * ld + i], vq = X[(int64_t)q * ld + i];
                            X[(int64_t)p * ld + i] = c * vp - s * vq;
                            X[(int64_t)q * ld + i] = s * vp + c * vq;
                        }
                    } else {
                        if (lane < rows) {
                            B[(int64_t)p * rows + lane] = c * xp - s * xq;
                            B[(int64_t)q * rows + lane] = s * xp + c * xq;
                        }
                        if (lane < k) {
                            const double vp = V[(int64_t)p * k + lane], vq = V[(int64_t)q * k + lane];
                            V[(int64_t)p * k + lane] = c * vp - s * vq;
                            V[(int64_t)q * k + lane] = s * vp + c * vq;
                        }
                    }
                    if (lane == 0) *s_rot = 1;
                }
            }
            __syncthreads();
        }
        const int rot = *s_rot;
        __syncthreads();
        if (!rot) break;
    }
    const int Gc = 32 / S;
    for (int j0 = warp * Gc; j0 < k; j0 += nwarps() * Gc) {
        const int j = j0 + sg;
        const double x = (j < k && i < rows) ? B[(int64_t)j * rows + i] : 0.0;
        const double a = seg_sum(x * x, S);
        if (j < k && i == 0) Sraw[j] = sqrt_via_rsqrt(a);
    }
    __syncthreads();
}

// SVD factors from jacobi_direct (B V = U diag(Sraw), B = M for a tall M, B =
// M^T for a wide M): tall: US = columns of B, Vt = rows V^T; wide: US = V
// diag(S), Vt = (B diag(1/S))^T.  Order, tie rule and sign rule as in
// svd_assemble.  rinv: k scratch doubles, perm: k ints.
__device__ __forceinline__ void svd_assemble_direct(const double* B, const double* V, const double* Sraw,
                                                    double* rinv, int* perm, double* S, double* US, double* Vt,
                                                    int M, int N, int k, int rows, int wide, int ldus, int ldvt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < k; i += nthreads()) {
        const double si = Sraw[i];
        const long long ki = nonneg_key(si);
        int rank = 0;
        for (int j = 0; j < k; ++j) {
            const long long kj = nonneg_key(Sraw[j]);
            rank += (kj > ki || (kj == ki && j < i)) ? 1 : 0;
        }
        perm[rank] = i;
        if (wide) {
            const double r = rsqrt(si);
            rinv[i] = si > 0.0 ? r * r : 0.0;
        }
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)M * k; e += nthreads()) {
        const int i = (int)(e / k), r = (int)(e % k);
        const int p = perm[r];
        US[(int64_t)i * ldus + r] = wide ? V[(int64_t)p * k + i] * Sraw[p] : B[(int64_t)p * rows + i];
    }
    for (int64_t e = threadIdx.x; e < (int64_t)k * N; e += nthreads()) {
        const int r = (int)(e / N), c = (int)(e % N);
        const int p = perm[r];
        Vt[(int64_t)r * ldvt + c] = wide ? B[(int64_t)p * rows + c] * rinv[p] : V[(int64_t)p * k + c];
    }
    for (int r = threadIdx.x; r < k; r += nthreads()) S[r] = Sraw[perm[r]];
    __syncthreads();
    for (int r = warp; r < k; r += nwarps()) {
        long long best = -1;
        int bi = 0;
        for (int c = lane; c < N; c += 32) {
            const long long a = abs_key(Vt[(int64_t)r * ldvt + c]);
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
        if (Vt[(int64_t)r * ldvt + bi] < 0.0) {
            for (int c = lane; c < N; c += 32) Vt[(int64_t)r * ldvt + c] = -Vt[(int64_t)r * ldvt + c];
            for (int i = lane; i < M; i += 32) US[(int64_t)i * ldus + r] = -US[(int64_t)i * ldus + r];
        }
    }
}

// One-sided (Hestenes) Jacobi on the columns of G (k x k, column-major) with the
// rotations accumulated in V (initialised here), parallel round-robin pair
// order.  zeta = (b - a)/(2 g), t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2)),
// c = 1/sqrt(1 + t^2), s = c t.  A pair is rotated while |g| > k eps sqrt(a b)
// and both columns are above the numerical-zero level k eps ||G||_F; a sweep
// without rotations ends the iteration.  Sraw: column norms of the result.
__device__ __forceinline__ void jacobi(double* G, double* V, double* Sraw, int k, double* red, int* s_rot) {
    if (k <= 16) {
        jacobi_small(G, V, Sraw, k, red, s_rot);
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double f = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += nthreads()) {
        const double v = G[e];
        f += v * v;
        V[e] = (e % k) == (e / k) ? 1.0 : 0.0;
    }
    f = block_sum(f, red);
    const double tol = (double)k * DBL_EPSILON;
    const double tiny2 = tol * tol * f;
    const int n2 = k + (k & 1);
    for (int sweep = 0; sweep < kMaxSweeps && k > 1; ++sweep) {
        if (threadIdx.x == 0) *s_rot = 0;
        __syncthreads();
        for (int round = 0; round < n2 - 1; ++round) {
            for (int pi = warp; pi < n2 / 2; pi += nwarps()) {
                int p = rr_player(pi, round, n2), q = rr_player(n2 - 1 - pi, round, n2);
                if (p >= k || q >= k) continue;
                if (p > q) {
                    const int tmp = p;
                    p = q;
                    q = tmp;
                }
                double a = 0.0, b = 0.0, g = 0.0;
                for (int i = lane; i < k; i += 32) {
                    const double xp = G[(int64_t)p * k + i], xq = G[(int64_t)q * k + i];
                    a += xp * xp;
                    b += xq * xq;
                    g += xp * xq;
                }
                a = warp_sum(a);
                b = warp_sum(b);
                g = warp_sum(g);
                if (g != 0.0 && fabs(g) > tol * sqrt(a * b) && fmin(a, b) > tiny2) {
                    const double zeta = (b - a) / (2.0 * g);
                    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                    for (int i = lane; i < k; i += 32) {
                        const double xp = G[(int64_t)p * k + i], xq = G[(int64_t)q * k + i];
                        G[(int64_t)p * k + i] = c * xp - s * xq;
                        G[(int64_t)q * k + i] = s * xp + c * xq;
                        const double vp = V[(int64_t)p * k + i], vq = V[(int64_t)q * k + i];
                        V[(int64_t)p * k + i] = c * vp - s * vq;
                        V[(int64_t)q * k + i] = s * vp + c * vq;
                    }
                    if (lane == 0) *s_rot = 1;
                }
            }
            __syncthreads();
        }
        const int rot = *s_rot;
        __syncthreads();
        if (!rot) break;
    }
    for (int j = warp; j < k; j += nwarps()) {
        double a = 0.0;
        for (int i = lane; i < k; i += 32) {
            const double x = G[(int64_t)j * k + i];
            a += x * x;
        }
        a = warp_sum(a);
        if (lane == 0) Sraw[j] = sqrt(a);
    }
    __syncthreads();
}

// SVD of an M x N matrix from QR + Jacobi of its k x k triangular factor:
// tall (M >= N): M = Q R, R^T = G, G V = U' S  =>  U = Q V, Vt = U'^T;
// wide (M < N):  M^T = Q R, R^T = G, G V = U' S => U = U', Vt = (Q V)^T.
// QV: column-major len x k (QV[p*len + i] = (Q V)(i, p)).  Writes S (k,
// descending, ties by index), US = U diag(S) (M x k row-major) and Vt (k x N
// row-major, row strides ldus / ldvt) with the largest-|.| entry of every Vt
// row positive.  perm: k ints.
__device__ __forceinline__ void svd_assemble(const double* G, const double* QV, const double* Sraw, int* perm,
                                             double* S, double* US, double* Vt, int M, int N, int k, int len,
                                             int wide, int ldus, int ldvt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < k; i += nthreads()) {
        const double si = Sraw[i];
        int rank = 0;
        for (int j = 0; j < k; ++j) {
            const double sj = Sraw[j];
            rank += (sj > si || (sj == si && j < i)) ? 1 : 0;
        }
        perm[rank] = i;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)M * k; e += nthreads()) {
        const int i = (int)(e / k), r = (int)(e % k);
        const int p = perm[r];
        US[(int64_t)i * ldus + r] = wide ? G[(int64_t)p * k + i] : Sraw[p] * QV[(int64_t)p * len + i];
    }
    for (int64_t e = threadIdx.x; e < (int64_t)k * N; e += nthreads()) {
        const int r = (int)(e / N), c = (int)(e % N);
        const int p = perm[r];
        double v;
        if (wide) {
            v = QV[(int64_t)p * len + c];
        } else {
            const double sp = Sraw[p];
            v = sp > 0.0 ? G[(int64_t)p * k + c] / sp : 0.0;
        }
        Vt[(int64_t)r * ldvt + c] = v;
    }
    for (int r = threadIdx.x; r < k; r += nthreads()) S[r] = Sraw[perm[r]];
    __syncthreads();
    for (int r = warp; r < k; r += nwarps()) {
        double best = -1.0;
        int bi = 0;
        for (int c = lane; c < N; c += 32) {
            const double a = fabs(Vt[(int64_t)r * ldvt + c]);
            if (a > best) {
                best = a;
                bi = c;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (Vt[(int64_t)r * ldvt + bi] < 0.0) {
            for (int c = lane; c < N; c += 32) Vt[(int64_t)r * ldvt + c] = -Vt[(int64_t)r * ldvt + c];
            for (int i = lane; i < M; i += 32) US[(int64_t)i * ldus + r] = -US[(int64_t)i * ldus + r];
        }
    }
}

}  // namespace dev
}  // namespace bsm
