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

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the block; every thread gets the result (red: 33 shared doubles)
__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
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

// Householder factorisation of A (M x N, column-major, ld M) in place: R in the
// upper trapezoid, v_j below the diagonal (v_j = 1 implicit), tau[j].
// H = I - tau v v^T, beta = -sign(alpha) ||x||, tau = (beta - alpha)/beta,
// v = x/(alpha - beta).  sh: 2 shared doubles.
__device__ __forceinline__ void householder(double* A, double* tau, int M, int N, double* red, double* sh) {
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
    return pos == 0 ? 0 : ((pos - 1 + round) % (n2 - 1)) + 1;
}

// One-sided (Hestenes) Jacobi on the columns of G (k x k, column-major) with the
// rotations accumulated in V (initialised here), parallel round-robin pair
// order.  zeta = (b - a)/(2 g), t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2)),
// c = 1/sqrt(1 + t^2), s = c t.  A pair is rotated while |g| > k eps sqrt(a b)
// and both columns are above the numerical-zero level k eps ||G||_F; a sweep
// without rotations ends the iteration.  Sraw: column norms of the result.
__device__ __forceinline__ void jacobi(double* G, double* V, double* Sraw, int k, double* red, int* s_rot) {
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
