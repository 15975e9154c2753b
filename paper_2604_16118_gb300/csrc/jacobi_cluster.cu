// One-sided Jacobi of a k x k matrix (k up to kClusterJacobiMax) on one
// thread-block cluster: the columns of G and of the rotation accumulator V are
// spread over the shared memories of the cluster's CTAs (CTA c holds columns
// c kc .. c kc + kc - 1, kc = ceil(k / C), C = 16 or 8), every warp of the cluster takes the
// column pairs of a round (the cyclic round-robin ordering of dev::jacobi) and
// reads / writes the partner columns through distributed shared memory, and a
// round ends at the cluster's hardware barrier instead of a grid-wide wait.
// A pair rotates while g^2 > (k eps)^2 a b and min(a, b) > (k eps)^2 ||G||_F^2
// (the stopping rule of dev::jacobi without its square root), by the rotation
// of dev::jacobi_rotation_fast (angle in FP32, c and s in FP64 with
// c^2 + s^2 = 1 to FP64 rounding); a sweep without a rotation ends the
// iteration (at most dev::kMaxSweeps sweeps).  On this GPU an SM retires one
// FP64 warp instruction per 16 cycles, so one CTA's Jacobi is bound by its SM's
// FP64 rate: the cluster brings the FP64 units of kClusterCtas SMs to one
// matrix.  Every CTA reaches the same decisions (the rotation flags and
// ||G||_F^2 are combined in a fixed order), so all of them pass the same
// barriers.
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

size_t cluster_smem(int k, int ctas) {
    const size_t kc = (size_t)(k + ctas - 1) / ctas;
    return 2 * kc * (size_t)k * sizeof(double);
}

template <int kClusterCtas>
__global__ void __launch_bounds__(kClusterThreads) k_jacobi_cluster(const JacTask* __restrict__ tasks) {
    extern __shared__ double jc_smem[];
    __shared__ double s_part[kClusterCtas];     // CTA 0's slots: partial ||G||^2 of every CTA
    __shared__ int s_flag[2][kClusterCtas];     // CTA 0's slots: rotation flags, by sweep parity
    __shared__ int s_rot;                       // this CTA rotated in the current sweep
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const JacTask tk = tasks[blockIdx.x / kClusterCtas];
    const int k = tk.k;
    const int kc = (k + kClusterCtas - 1) / kClusterCtas;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* Gl = jc_smem;                      // local columns: Gl[(p - rank kc) k + i]
    double* Vl = jc_smem + (size_t)kc * k;
    const int c_beg = rank * kc, c_end = min(k, c_beg + kc);
    // load the CTA's columns of G, V = I, partial ||G||_F^2
    double f = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)(c_end - c_beg) * k; e += kClusterThreads) {
        const int j = (int)(e / k), i = (int)(e % k);
        const double v = tk.G[(int64_t)(c_beg + j) * k + i];
        Gl[e] = v;
        Vl[e] = (i == c_beg + j) ? 1.0 : 0.0;
        f += v * v;
    }
    __shared__ double red[33];
    f = dev::block_sum(f, red);
    double* part0 = cluster.map_shared_rank(s_part, 0);
    if (threadIdx.x == 0) {
        part0[rank] = f;
        s_rot = 0;
    }
    cluster.sync();
    double fro = 0.0;
    for (int c = 0; c < kClusterCtas; ++c) fro += part0[c];
    const double tol = (double)k * DBL_EPSILON;
    const double tol2 = tol * tol, tiny2 = tol2 * fro;
    const int n2 = k + (k & 1);
    int* flag0 = cluster.map_shared_rank(&s_flag[0][0], 0);
    auto colG = [&](int p) -> double* {
        return cluster.map_shared_rank(Gl + (size_t)(p % kc) * k, p / kc);
    };
    auto colV = [&](int p) -> double* {
        return cluster.map_shared_rank(Vl + (size_t)(p % kc) * k, p / kc);
    };
    const int gw = rank * kClusterWarps + warp, nw = kClusterCtas * kClusterWarps;
    for (int sweep = 0; sweep < dev::kMaxSweeps && k > 1; ++sweep) {
        for (int round = 0; round < n2 - 1; ++round) {
            for (int pi = gw; pi < n2 / 2; pi += nw) {
                int p = dev::rr_player(pi, round, n2), q = dev::rr_player(n2 - 1 - pi, round, n2);
                if (p >= k || q >= k) continue;
                if (p > q) {
                    const int tmp = p;
                    p = q;
                    q = tmp;
                }
                double* Gp = colG(p);
                double* Gq = colG(q);
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
                    double* Vp = colV(p);
                    double* Vq = colV(q);
                    for (int i = lane; i < k; i += 32) {
                        const double xp = Gp[i], xq = Gq[i];
                        Gp[i] = c * xp - sn * xq;
                        Gq[i] = sn * xp + c * xq;
                        const double vp = Vp[i], vq = Vq[i];
                        Vp[i] = c * vp - sn * vq;
                        Vq[i] = sn * vp + c * vq;
                    }
                    if (lane == 0) s_rot = 1;
                }
            }
            cluster.sync();
        }
        // combine the CTAs' rotation flags in CTA 0's slots (parity-indexed, so the
        // slots of one sweep are never reset while another CTA still reads them)
        const int par = sweep & 1;
        if (threadIdx.x == 0) {
            flag0[par * kClusterCtas + rank] = s_rot;
            s_rot = 0;
        }
        cluster.sync();
        int rot = 0;
        for (int c = 0; c < kClusterCtas; ++c) rot |= flag0[par * kClusterCtas + c];
        if (!rot) break;
    }
    // column norms of the rotated G, then G and V back to global memory
    for (int j = c_beg + warp; j < c_end; j += kClusterWarps) {
        const double* Gj = Gl + (size_t)(j - c_beg) * k;
        double a = 0.0;
        for (int i = lane; i < k; i += 32) a += Gj[i] * Gj[i];
        a = dev::warp_sum(a);
        if (lane == 0) tk.Sraw[j] = sqrt(a);
    }
    for (int64_t e = threadIdx.x; e < (int64_t)(c_end - c_beg) * k; e += kClusterThreads) {
        tk.G[(int64_t)c_beg * k + e] = Gl[e];
        tk.V[(int64_t)c_beg * k + e] = Vl[e];
    }
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
}

// One launch of the C-CTA kernel; false (nothing launched) when such clusters
// cannot be scheduled.
template <int C>
bool launch_cluster_size(Context* ctx, const std::vector<JacTask>& tasks, int kmax) {
    const size_t smem = cluster_smem(kmax, C);
    if (smem > kClusterSmemMax) return false;
    static bool attr = false;
    if (!attr) {
        BSM_CUDA(cudaFuncSetAttribute(k_jacobi_cluster<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kClusterSmemMax));
        if (C > 8) BSM_CUDA(cudaFuncSetAttribute(k_jacobi_cluster<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        attr = true;
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
    if (cudaOccupancyMaxActiveClusters(&n_clusters, k_jacobi_cluster<C>, &cfg) != cudaSuccess || n_clusters < 1) {
        (void)cudaGetLastError();
        return false;
    }
    Scratch s(ctx);
    const JacTask* d = s.up(tasks);
    BSM_CUDA(cudaLaunchKernelEx(&cfg, k_jacobi_cluster<C>, d));
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

}  // namespace bsm
