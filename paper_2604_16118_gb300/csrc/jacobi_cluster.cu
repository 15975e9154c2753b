// One-sided Jacobi of a k x k matrix G (k up to kClusterJacobiMax) on one
// thread-block cluster of C CTAs (C = 16, else 8), in a block-cyclic ordering.
//
// The k columns form 2C blocks of b = ceil(k / 2C) columns.  A sweep is a
// round-robin tournament of the blocks by the circle method (position 0 keeps
// block 0, positions 1 .. 2C-1 rotate by one per step; 2C - 1 steps).  In a step
// CTA c holds the blocks at positions c and 2C-1-c in its shared memory and
// rotates every column pair between them in local rounds (round r pairs column
// j of the first block with column (j + r) mod B of the second, one warp per
// pair, __syncthreads between rounds); in the first step of a sweep it also
// rotates the pairs inside both blocks (the round-robin ordering of
// dev::jacobi).  One cluster barrier ends a step; then every CTA pulls the two
// blocks of its next positions from the other CTAs' shared memory into its
// second buffer.  So a sweep still meets every pair of columns once, with 2C
// cluster barriers instead of one per round of k / 2 pairs, and the rotations
// read and write the CTA's own shared memory.  The accumulated rotations V
// (k x k) stay in global memory (L2-resident, read with __ldcg because another
// CTA of the cluster wrote them in an earlier step).
//
// A pair rotates while g^2 > (k eps)^2 a b and min(a, b) > (k eps)^2 ||G||_F^2
// (the stopping rule of dev::jacobi without its square root), by the rotation
// of dev::jacobi_rotation_fast (angle in FP32, c and s in FP64 with
// c^2 + s^2 = 1 to FP64 rounding); a sweep without a rotation ends the
// iteration (at most dev::kMaxSweeps sweeps).  On this GPU an SM retires one
// FP64 warp instruction per 16 cycles, so one CTA's Jacobi is bound by its SM's
// FP64 rate: the cluster brings the FP64 units of C SMs to one matrix.  Every
// CTA takes the same decisions (the rotation flags and ||G||_F^2 are combined
// in a fixed order), so all of them pass the same barriers.
#include <cooperative_groups.h>

#include <algorithm>

#include "dense_dev.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace bsm {
namespace {

constexpr int kClusterThreads = 512;
constexpr int kClusterWarps = kClusterThreads / 32;
constexpr size_t kClusterSmemMax = 225 * 1024;

// Slot strides, in elements, rounded up to 16 bytes so that blocks move between
// the CTAs' shared memories in 16-byte units: FP64 slot = b columns of G; FP32
// slot = b columns of G, then b columns of V, each part 16-byte aligned.
__host__ __device__ __forceinline__ size_t slot_f64(int b, int k) { return ((size_t)b * k + 1) & ~size_t(1); }
__host__ __device__ __forceinline__ size_t part_f32(int b, int k) { return ((size_t)b * k + 3) & ~size_t(3); }

// shared memory of one CTA: two buffers of two block slots
size_t cluster_smem(int k, int ctas, bool f32) {
    const int b = (k + 2 * ctas - 1) / (2 * ctas);
    return f32 ? 4 * 2 * part_f32(b, k) * sizeof(float) : 4 * slot_f64(b, k) * sizeof(double);
}

// Copy n16 16-byte units from src (another CTA's shared memory) to dst, with
// four loads in flight per thread; both 16-byte aligned.
__device__ __forceinline__ void pull16(float4* __restrict__ dst, const float4* __restrict__ src, int n16) {
    constexpr int T = kClusterThreads;
    int e = threadIdx.x;
    for (; e + 3 * T < n16; e += 4 * T) {
        const float4 v0 = src[e], v1 = src[e + T], v2 = src[e + 2 * T], v3 = src[e + 3 * T];
        dst[e] = v0;
        dst[e + T] = v1;
        dst[e + 2 * T] = v2;
        dst[e + 3 * T] = v3;
    }
    for (; e < n16; e += T) dst[e] = src[e];
}

// Block at tournament position p in step s (n2m1 = 2C - 1; position 0 fixed).
__device__ __forceinline__ int block_at(int p, int s, int n2m1) {
    return p == 0 ? 0 : (p - 1 + s) % n2m1 + 1;
}
// Position of block beta in step s (the inverse of block_at).
__device__ __forceinline__ int pos_of(int beta, int s, int n2m1) {
    return beta == 0 ? 0 : ((beta - 1 - s) % n2m1 + n2m1) % n2m1 + 1;
}

// One warp: rotate columns Gp, Gq (shared memory) and columns gp, gq of V.
__device__ __forceinline__ void rotate_pair(double* Gp, double* Gq, double* __restrict__ V, int gp, int gq, int k,
                                            double tol2, double tiny2, int lane, int* s_rot) {
    double a = 0.0, b = 0.0, g = 0.0;
    for (int i = lane; i < k; i += 32) {
        const double xp = Gp[i], xq = Gq[i];
        a += xp * xp;
        b += xq * xq;
        g += xp * xq;
    }
    a = dev::warp_sum(a);
    b = dev::warp_sum(b);
    g = dev::warp_sum(g);
    if (g * g > tol2 * (a * b) && fmin(a, b) > tiny2) {
        double c, sn;
        dev::jacobi_rotation_fast(a, b, g, &c, &sn);
        double* Vp = V + (int64_t)gp * k;
        double* Vq = V + (int64_t)gq * k;
        for (int i = lane; i < k; i += 32) {
            const double xp = Gp[i], xq = Gq[i];
            Gp[i] = c * xp - sn * xq;
            Gq[i] = sn * xp + c * xq;
            const double vp = __ldcg(Vp + i), vq = __ldcg(Vq + i);
            Vp[i] = c * vp - sn * vq;
            Vq[i] = sn * vp + c * vq;
        }
        if (lane == 0) *s_rot = 1;
    }
}

template <int C>
__global__ void __launch_bounds__(kClusterThreads) k_jacobi_cluster(const JacTask* __restrict__ tasks) {
    extern __shared__ double jc_smem[];
    __shared__ double s_part[C];     // CTA 0's slots: partial ||G||^2 of every CTA
    __shared__ int s_flag[2][C];     // CTA 0's slots: rotation flags, by sweep parity
    __shared__ int s_rot;            // this CTA rotated in the current sweep
    __shared__ double red[33];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const JacTask tk = tasks[blockIdx.x / C];
    const int k = tk.k;
    constexpr int nblk = 2 * C, n2m1 = 2 * C - 1;
    const int b = (k + nblk - 1) / nblk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // slot sl of buffer buf: b columns of k rows
    const size_t sstride = slot_f64(b, k);
    auto slot = [&](int buf, int sl) { return jc_smem + (size_t)(buf * 2 + sl) * sstride; };
    auto bcols = [&](int beta) { return max(0, min(b, k - beta * b)); };
    // step 0: CTA c holds blocks c (slot 0) and 2C-1-c (slot 1); load them, set
    // their columns of V to the identity, partial ||G||_F^2
    double f = 0.0;
    for (int sl = 0; sl < 2; ++sl) {
        const int beta = sl == 0 ? rank : nblk - 1 - rank;
        const int nc = bcols(beta);
        double* dst = slot(0, sl);
        const int64_t off = (int64_t)beta * b * k;
        for (int64_t e = threadIdx.x; e < (int64_t)nc * k; e += kClusterThreads) {
            const double v = tk.G[off + e];
            dst[e] = v;
            f += v * v;
            const int j = (int)(e / k), i = (int)(e % k);
            if (!tk.v_given) tk.V[off + e] = i == beta * b + j ? 1.0 : 0.0;
        }
    }
    f = dev::block_sum(f, red);
    double* part0 = cluster.map_shared_rank(s_part, 0);
    if (threadIdx.x == 0) {
        part0[rank] = f;
        s_rot = 0;
    }
    cluster.sync();
    double fro = 0.0;
    for (int c = 0; c < C; ++c) fro += part0[c];
    const double tol = (double)k * DBL_EPSILON;
    const double tol2 = tol * tol, tiny2 = tol2 * fro;
    int* flag0 = cluster.map_shared_rank(&s_flag[0][0], 0);
    int gstep = 0;   // steps taken: buffer gstep & 1 holds the current blocks
    for (int sweep = 0; sweep < dev::kMaxSweeps && k > 1; ++sweep) {
        for (int s = 0; s < n2m1; ++s, ++gstep) {
            const int cur = gstep & 1;
            const int bL = block_at(rank, s, n2m1), bR = block_at(nblk - 1 - rank, s, n2m1);
            const int nL = bcols(bL), nR = bcols(bR);
            double* L = slot(cur, 0);
            double* R = slot(cur, 1);
            if (s == 0) {
                // pairs inside each block: round-robin over nb2 players per block
                const int nb = max(nL, nR), nb2 = nb + (nb & 1), half = nb2 / 2;
                for (int round = 0; round < nb2 - 1; ++round) {
                    for (int u = warp; u < nb2; u += kClusterWarps) {
                        const int pi = u % half, side = u / half;
                        int p = dev::rr_player(pi, round, nb2), q = dev::rr_player(nb2 - 1 - pi, round, nb2);
                        if (p > q) {
                            const int t = p;
                            p = q;
                            q = t;
                        }
                        if (q >= (side == 0 ? nL : nR)) continue;
                        double* X = side == 0 ? L : R;
                        const int c0 = (side == 0 ? bL : bR) * b;
                        rotate_pair(X + (size_t)p * k, X + (size_t)q * k, tk.V, c0 + p, c0 + q, k, tol2, tiny2, lane,
                                    &s_rot);
                    }
                    __syncthreads();
                }
            }
            // pairs between the two blocks
            const int B = max(nL, nR);
            for (int r = 0; r < B; ++r) {
                for (int j = warp; j < B; j += kClusterWarps) {
                    const int q = (j + r) % B;
                    if (j >= nL || q >= nR) continue;
                    rotate_pair(L + (size_t)j * k, R + (size_t)q * k, tk.V, bL * b + j, bR * b + q, k, tol2, tiny2,
                                lane, &s_rot);
                }
                __syncthreads();
            }
            cluster.sync();
            // pull the blocks of the next step's positions into the other buffer
            const int s1 = s + 1 == n2m1 ? 0 : s + 1;
            for (int sl = 0; sl < 2; ++sl) {
                const int beta = block_at(sl == 0 ? rank : nblk - 1 - rank, s1, n2m1);
                const int hp = pos_of(beta, s, n2m1);   // its position in this step
                const int holder = hp < C ? hp : nblk - 1 - hp;
                const double* src = cluster.map_shared_rank(slot(cur, hp < C ? 0 : 1), holder);
                pull16((float4*)slot(cur ^ 1, sl), (const float4*)src, (bcols(beta) * k + 1) / 2);
            }
            __syncthreads();
        }
        // combine the CTAs' rotation flags in CTA 0's slots (parity-indexed, so the
        // slots of one sweep are never reset while another CTA still reads them)
        const int par = sweep & 1;
        if (threadIdx.x == 0) {
            flag0[par * C + rank] = s_rot;
            s_rot = 0;
        }
        cluster.sync();
        int rot = 0;
        for (int c = 0; c < C; ++c) rot |= flag0[par * C + c];
        if (!rot) break;
    }
    // the current blocks (step gstep mod 2C-1 of the tournament) back to global
    // memory, with the column norms
    const int cur = gstep & 1, s_now = gstep % n2m1;
    for (int sl = 0; sl < 2; ++sl) {
        const int beta = block_at(sl == 0 ? rank : nblk - 1 - rank, s_now, n2m1);
        const int nc = bcols(beta);
        const double* X = slot(cur, sl);
        for (int j = warp; j < nc; j += kClusterWarps) {
            double a = 0.0;
            for (int i = lane; i < k; i += 32) a += X[(size_t)j * k + i] * X[(size_t)j * k + i];
            a = dev::warp_sum(a);
            if (lane == 0) tk.Sraw[beta * b + j] = sqrt(a);
        }
        const int64_t off = (int64_t)beta * b * k;
        for (int64_t e = threadIdx.x; e < (int64_t)nc * k; e += kClusterThreads) tk.G[off + e] = X[e];
    }
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
}

// One-sided Jacobi in FP32 of the k x k FP64 matrix G, as a preconditioner:
// the same block-cyclic tournament as k_jacobi_cluster, with G (scaled by a
// power of two to ||G||_F ~ 1, rounded to FP32) and the accumulated rotations
// V both in the CTAs' shared memory (a block moves with its columns of V).
// FP32 arithmetic runs at 64 times the FP64 rate of this GPU.  A pair rotates
// while |g| > tol sqrt(a) sqrt(b), tol = 4 sqrt(k) eps_32 (above the rounding
// noise of the FP32 inner products), and min(a, b) > 1e-36 (of ||G||_F^2 ~ 1):
// floating point resolves the small columns of a graded G relative to their
// own norms, so they are rotated too, which leaves the FP64 Jacobi only the
// last quadratic sweeps at every scale.  The rotation is that of
// dev::jacobi_rotation_fast in FP32, with d = b - a and 2g scaled by their
// larger magnitude so that no square underflows.  A sweep that rotates at most
// 1/32 of the pairs ends the iteration (at most kMaxSweepsF32).  Output: tk.V = the FP32 V as
// FP64 (orthogonal to about 1e-6); tk.G is read only; tk.Sraw unused.
constexpr int kMaxSweepsF32 = 20;

__device__ __forceinline__ void rotate_pair_f32(float* Gp, float* Gq, float* Vp, float* Vq, int k, float tol,
                                                int lane, int* s_rot) {
    float a = 0.0f, b = 0.0f, g = 0.0f;
    for (int i = lane; i < k; i += 32) {
        const float xp = Gp[i], xq = Gq[i];
        a = fmaf(xp, xp, a);
        b = fmaf(xq, xq, b);
        g = fmaf(xp, xq, g);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        g += __shfl_xor_sync(0xffffffffu, g, o);
    }
    if (fabsf(g) > tol * sqrtf(a) * sqrtf(b) && fminf(a, b) > 1e-36f) {
        // t = tan of the angle, the smaller root of t^2 + 2 zeta t - 1 = 0 with
        // zeta = (b - a) / 2g; c = 1 / sqrt(1 + t^2), s = c t
        const float d = b - a, g2 = g + g;
        const float m = fmaxf(fabsf(d), fabsf(g2));   // > 0 (g != 0)
        const float dn = d / m, gn = g2 / m;
        const float r = sqrtf(fmaf(dn, dn, gn * gn));
        const float sz = (d == 0.0f || ((d > 0.0f) == (g2 > 0.0f))) ? 1.0f : -1.0f;
        const float t = sz * __fdividef(fabsf(gn), fabsf(dn) + r);
        const float c = rsqrtf(fmaf(t, t, 1.0f)), sn = c * t;
        for (int i = lane; i < k; i += 32) {
            const float xp = Gp[i], xq = Gq[i];
            Gp[i] = c * xp - sn * xq;
            Gq[i] = sn * xp + c * xq;
            const float vp = Vp[i], vq = Vq[i];
            Vp[i] = c * vp - sn * vq;
            Vq[i] = sn * vp + c * vq;
        }
        if (lane == 0) atomicAdd(s_rot, 1);
    }
}

template <int C>
__global__ void __launch_bounds__(kClusterThreads) k_jacobi_cluster_f32(const JacTask* __restrict__ tasks) {
    extern __shared__ float jf_smem[];
    __shared__ double s_part[C];
    __shared__ int s_flag[2][C];
    __shared__ int s_rot;
    __shared__ double red[33];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const JacTask tk = tasks[blockIdx.x / C];
    const int k = tk.k;
    constexpr int nblk = 2 * C, n2m1 = 2 * C - 1;
    const int b = (k + nblk - 1) / nblk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // slot sl of buffer buf: b columns of G, then b columns of V (k rows each)
    const size_t vpart = part_f32(b, k);   // offset of the V columns in a slot
    auto slot = [&](int buf, int sl) { return jf_smem + (size_t)(buf * 2 + sl) * 2 * vpart; };
    auto bcols = [&](int beta) { return max(0, min(b, k - beta * b)); };
    double f = 0.0;
    for (int sl = 0; sl < 2; ++sl) {
        const int beta = sl == 0 ? rank : nblk - 1 - rank;
        const int64_t off = (int64_t)beta * b * k;
        for (int64_t e = threadIdx.x; e < (int64_t)bcols(beta) * k; e += kClusterThreads) {
            const double v = tk.G[off + e];
            f += v * v;
        }
    }
    f = dev::block_sum(f, red);
    double* part0 = cluster.map_shared_rank(s_part, 0);
    if (threadIdx.x == 0) {
        part0[rank] = f;
        s_rot = 0;
    }
    cluster.sync();
    double fro = 0.0;
    for (int c = 0; c < C; ++c) fro += part0[c];
    int ex = 0;
    if (fro > 0.0) frexp(sqrt(fro), &ex);
    const double sc = ldexp(1.0, -ex);   // exact power of two: ||sc G||_F in [1/2, 1)
    for (int sl = 0; sl < 2; ++sl) {
        const int beta = sl == 0 ? rank : nblk - 1 - rank;
        const int nc = bcols(beta);
        const int64_t off = (int64_t)beta * b * k;
        float* dst = slot(0, sl);
        for (int64_t e = threadIdx.x; e < (int64_t)nc * k; e += kClusterThreads) {
            dst[e] = (float)(tk.G[off + e] * sc);
            const int j = (int)(e / k), i = (int)(e % k);
            dst[vpart + e] = i == beta * b + j ? 1.0f : 0.0f;
        }
    }
    __syncthreads();
    const float tol = 4.0f * sqrtf((float)k) * FLT_EPSILON;
    int* flag0 = cluster.map_shared_rank(&s_flag[0][0], 0);
    int gstep = 0;
    for (int sweep = 0; sweep < kMaxSweepsF32 && k > 1; ++sweep) {
        for (int s = 0; s < n2m1; ++s, ++gstep) {
            const int cur = gstep & 1;
            const int bL = block_at(rank, s, n2m1), bR = block_at(nblk - 1 - rank, s, n2m1);
            const int nL = bcols(bL), nR = bcols(bR);
            float* L = slot(cur, 0);
            float* R = slot(cur, 1);
            float* LV = L + vpart;
            float* RV = R + vpart;
            if (s == 0) {
                const int nb = max(nL, nR), nb2 = nb + (nb & 1), half = nb2 / 2;
                for (int round = 0; round < nb2 - 1; ++round) {
                    for (int u = warp; u < nb2; u += kClusterWarps) {
                        const int pi = u % half, side = u / half;
                        int p = dev::rr_player(pi, round, nb2), q = dev::rr_player(nb2 - 1 - pi, round, nb2);
                        if (p > q) {
                            const int t = p;
                            p = q;
                            q = t;
                        }
                        if (q >= (side == 0 ? nL : nR)) continue;
                        float* X = side == 0 ? L : R;
                        float* XV = side == 0 ? LV : RV;
                        rotate_pair_f32(X + (size_t)p * k, X + (size_t)q * k, XV + (size_t)p * k, XV + (size_t)q * k,
                                        k, tol, lane, &s_rot);
                    }
                    __syncthreads();
                }
            }
            const int B = max(nL, nR);
            for (int r = 0; r < B; ++r) {
                for (int j = warp; j < B; j += kClusterWarps) {
                    const int q = (j + r) % B;
                    if (j >= nL || q >= nR) continue;
                    rotate_pair_f32(L + (size_t)j * k, R + (size_t)q * k, LV + (size_t)j * k, RV + (size_t)q * k, k,
                                    tol, lane, &s_rot);
                }
                __syncthreads();
            }
            cluster.sync();
            const int s1 = s + 1 == n2m1 ? 0 : s + 1;
            for (int sl = 0; sl < 2; ++sl) {
                const int beta = block_at(sl == 0 ? rank : nblk - 1 - rank, s1, n2m1);
                const int hp = pos_of(beta, s, n2m1);
                const int holder = hp < C ? hp : nblk - 1 - hp;
                const float* src = cluster.map_shared_rank(slot(cur, hp < C ? 0 : 1), holder);
                float* dst = slot(cur ^ 1, sl);
                const int n16 = (bcols(beta) * k + 3) / 4;
                pull16((float4*)dst, (const float4*)src, n16);
                pull16((float4*)(dst + vpart), (const float4*)(src + vpart), n16);
            }
            __syncthreads();
        }
        // rotation counts of the sweep; a sweep that rotated at most 1/32 of the
        // pairs ends the FP32 iteration (the FP64 Jacobi takes the rest)
        const int par = sweep & 1;
        if (threadIdx.x == 0) {
            flag0[par * C + rank] = s_rot;
            s_rot = 0;
        }
        cluster.sync();
        int64_t rot = 0;
        for (int c = 0; c < C; ++c) rot += flag0[par * C + c];
        if (32 * rot <= (int64_t)k * (k - 1) / 2) break;
    }
    const int cur = gstep & 1, s_now = gstep % n2m1;
    for (int sl = 0; sl < 2; ++sl) {
        const int beta = block_at(sl == 0 ? rank : nblk - 1 - rank, s_now, n2m1);
        const float* XV = slot(cur, sl) + vpart;
        const int64_t off = (int64_t)beta * b * k;
        for (int64_t e = threadIdx.x; e < (int64_t)bcols(beta) * k; e += kClusterThreads) tk.V[off + e] = XV[e];
    }
    cluster.sync();
}

// One launch of a C-CTA kernel (the FP64 Jacobi, or the FP32 one when f32);
// false (nothing launched) when such clusters cannot be scheduled.
template <int C>
bool launch_cluster_size(Context* ctx, const std::vector<JacTask>& tasks, int kmax, bool f32 = false) {
    const size_t smem = cluster_smem(kmax, C, f32);
    if (smem > kClusterSmemMax) return false;
    void (*kern)(const JacTask*) = f32 ? k_jacobi_cluster_f32<C> : k_jacobi_cluster<C>;
    static bool attr[2] = {false, false};
    if (!attr[f32]) {
        BSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusterSmemMax));
        if (C > 8) BSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        attr[f32] = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(tasks.size() * C));
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr_l[1];
    attr_l[0].id = cudaLaunchAttributeClusterDimension;
    attr_l[0].val.clusterDim.x = C;
    attr_l[0].val.clusterDim.y = 1;
    attr_l[0].val.clusterDim.z = 1;
    cfg.attrs = attr_l;
    cfg.numAttrs = 1;
    int n_clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&n_clusters, kern, &cfg) != cudaSuccess || n_clusters < 1) {
        (void)cudaGetLastError();
        return false;
    }
    Scratch s(ctx);
    const JacTask* d = s.up(tasks);
    BSM_CUDA(cudaLaunchKernelEx(&cfg, kern, d));
    check_launch(ctx);
    return true;
}

}  // namespace

// Tasks with k <= kClusterJacobiMax, one cluster each: 16 CTAs per cluster when
// such clusters can be scheduled (more FP64 units per matrix), else 8; false
// (nothing launched) when neither can.
bool launch_jacobi_cluster(Context* ctx, const std::vector<JacTask>& tasks) {
    if (tasks.empty()) return true;
    int kmax = 0;
    for (const JacTask& t : tasks) kmax = std::max(kmax, t.k);
    if (kmax > kClusterJacobiMax) return false;
    return launch_cluster_size<16>(ctx, tasks, kmax) || launch_cluster_size<8>(ctx, tasks, kmax);
}

// The FP32 preconditioning Jacobi (k_jacobi_cluster_f32) of the same tasks, on
// 8-CTA clusters first: the FP32 sweeps are bound by round latency, not by the
// arithmetic of the SMs, and 8 CTAs halve the tournament steps (cluster
// barriers and block pulls) per sweep (measured: full-rank step 12.23 -> 11.86 s).
bool launch_jacobi_cluster_f32(Context* ctx, const std::vector<JacTask>& tasks) {
    if (tasks.empty()) return true;
    int kmax = 0;
    for (const JacTask& t : tasks) kmax = std::max(kmax, t.k);
    if (kmax > kClusterJacobiMax) return false;
    return launch_cluster_size<8>(ctx, tasks, kmax, true) || launch_cluster_size<16>(ctx, tasks, kmax, true);
}

}  // namespace bsm
