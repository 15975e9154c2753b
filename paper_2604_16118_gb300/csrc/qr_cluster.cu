// Householder QR of one M x N matrix on one thread-block cluster: the columns of
// A and of Q are spread cyclically over the shared memories of the cluster's
// CTAs (column p on CTA p mod C), so the trailing updates of a column use the
// FP64 units of C SMs (one SM retires one FP64 warp instruction per 16 cycles
// on this GPU, which bounds a one-CTA QR).
//
// Column j: its owner forms the reflector H_j = I - tau v v^T (v_j = 1,
// beta = -sign(alpha) ||x||, the reflector() of dev::householder_small) and
// scales v in place; after one cluster barrier every CTA copies v_j and tau_j
// from the owner's shared memory and applies H_j to its own columns p > j.
// Q = H_0 ... H_{k-1} applied to the first k columns of I is formed
// afterwards by every CTA for its own Q columns without further barriers (the
// reflectors no longer change).  diag(R) >= 0: row j of R and column j of Q
// change sign when beta_j < 0.  Output as QrTask of k_qr: Q (M x k,
// column-major), R (k x N, row-major).
#include <cooperative_groups.h>

#include <algorithm>

#include "dense_dev.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace bsm {
namespace {

constexpr int kQcThreads = 512;
constexpr int kQcWarps = kQcThreads / 32;
constexpr size_t kQcSmemMax = 220 * 1024;

// shared memory of one CTA: its A and Q columns, one copy of v, tau and beta of every column
size_t qc_smem(int M, int N, int C) {
    const int k = std::min(M, N);
    const size_t na = (size_t)(N + C - 1) / C, nq = (size_t)(k + C - 1) / C;
    return sizeof(double) * ((na + nq + 1) * (size_t)M + 2 * (size_t)k);
}

template <int C>
__global__ void __launch_bounds__(kQcThreads) k_qr_cluster(const QrTask* __restrict__ tasks) {
    extern __shared__ double qc_sm[];
    __shared__ double red[33];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const QrTask tk = tasks[blockIdx.x / C];
    const int M = tk.M, N = tk.N, k = M < N ? M : N;
    const int na = (N + C - 1) / C, nq = (k + C - 1) / C;
    double* Al = qc_sm;                          // local column lp = global column rank + lp C
    double* Ql = Al + (size_t)na * M;
    double* vb = Ql + (size_t)nq * M;            // copy of the current reflector
    double* taus = vb + M;                       // tau_j of the columns this CTA owns (by j)
    double* betas = taus + k;                    // R(j, j) before the sign rule, owned columns
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_loc = rank < N ? (N - 1 - rank) / C + 1 : 0;
    for (int64_t e = threadIdx.x; e < (int64_t)n_loc * M; e += kQcThreads) {
        const int lp = (int)(e / M), i = (int)(e % M);
        Al[e] = tk.A[(int64_t)(rank + lp * C) * M + i];
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        const int owner = j % C;
        if (rank == owner) {
            double* col = Al + (size_t)(j / C) * M;
            double s = 0.0;
            for (int i = j + 1 + threadIdx.x; i < M; i += kQcThreads) s += col[i] * col[i];
            s = dev::block_sum(s, red);
            const double alpha = col[j];
            double tj = 0.0, scale = 0.0, beta = alpha;
            if (s != 0.0) dev::reflector(alpha, s, &beta, &tj, &scale);
            if (tj != 0.0)
                for (int i = j + 1 + threadIdx.x; i < M; i += kQcThreads) col[i] *= scale;
            __syncthreads();
            if (threadIdx.x == 0) {
                col[j] = beta;
                taus[j] = tj;
                betas[j] = beta;
            }
        }
        cluster.sync();
        const double* ocol = cluster.map_shared_rank(Al + (size_t)(j / C) * M, owner);
        const double tj = *cluster.map_shared_rank(taus + j, owner);
        if (tj != 0.0) {
            for (int i = j + 1 + threadIdx.x; i < M; i += kQcThreads) vb[i] = ocol[i];
            __syncthreads();
            // local columns p > j
            const int lp0 = (j + 1 - rank + C - 1) / C > 0 ? (j + 1 - rank + C - 1) / C : 0;
            for (int lp = lp0 + warp; lp < n_loc; lp += kQcWarps) {
                double* a = Al + (size_t)lp * M;
                const double a_j = a[j];
                double w = 0.0;
                for (int i = j + 1 + lane; i < M; i += 32) w += vb[i] * a[i];
                w = dev::warp_sum(w) + a_j;
                const double tw = tj * w;
                if (lane == 0) a[j] = a_j - tw;
                for (int i = j + 1 + lane; i < M; i += 32) a[i] -= tw * vb[i];
            }
        }
        __syncthreads();
    }
    // Q: this CTA's columns p < k (p = rank + lq C), from the identity, reflectors backwards
    const int q_loc = rank < k ? (k - 1 - rank) / C + 1 : 0;
    for (int64_t e = threadIdx.x; e < (int64_t)q_loc * M; e += kQcThreads) {
        const int lq = (int)(e / M), i = (int)(e % M);
        Ql[e] = i == rank + lq * C ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = k - 1; j >= 0; --j) {
        const int owner = j % C;
        const double tj = *cluster.map_shared_rank(taus + j, owner);
        if (tj == 0.0) continue;
        const double* ocol = cluster.map_shared_rank(Al + (size_t)(j / C) * M, owner);
        for (int i = j + 1 + threadIdx.x; i < M; i += kQcThreads) vb[i] = ocol[i];
        __syncthreads();
        const int lq0 = (j - rank + C - 1) / C > 0 ? (j - rank + C - 1) / C : 0;
        for (int lq = lq0 + warp; lq < q_loc; lq += kQcWarps) {
            double* q = Ql + (size_t)lq * M;
            const double q_j = q[j];
            double w = 0.0;
            for (int i = j + 1 + lane; i < M; i += 32) w += vb[i] * q[i];
            w = dev::warp_sum(w) + q_j;
            const double tw = tj * w;
            if (lane == 0) q[j] = q_j - tw;
            for (int i = j + 1 + lane; i < M; i += 32) q[i] -= tw * vb[i];
        }
        __syncthreads();
    }
    // R (row-major k x N) from this CTA's A columns and Q columns, with the sign rule
    for (int64_t e = threadIdx.x; e < (int64_t)n_loc * k; e += kQcThreads) {
        const int lp = (int)(e / k), r = (int)(e % k);
        const int c = rank + lp * C;
        const double sg = *cluster.map_shared_rank(betas + r, r % C) < 0.0 ? -1.0 : 1.0;
        tk.R[(int64_t)r * N + c] = c >= r ? sg * Al[(size_t)lp * M + r] : 0.0;
    }
    for (int64_t e = threadIdx.x; e < (int64_t)q_loc * M; e += kQcThreads) {
        const int lq = (int)(e / M), i = (int)(e % M);
        const int p = rank + lq * C;
        tk.Q[(int64_t)p * M + i] = (betas[p] < 0.0 ? -1.0 : 1.0) * Ql[e];
    }
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
}

template <int C>
bool launch_qc(Context* ctx, const std::vector<QrTask>& tasks) {
    size_t smem = 0;
    for (const QrTask& t : tasks) smem = std::max(smem, qc_smem(t.M, t.N, C));
    if (smem > kQcSmemMax) return false;
    static bool attr = false;
    if (!attr) {
        BSM_CUDA(cudaFuncSetAttribute(k_qr_cluster<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQcSmemMax));
        if (C > 8) BSM_CUDA(cudaFuncSetAttribute(k_qr_cluster<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(tasks.size() * C));
    cfg.blockDim = dim3(kQcThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n_clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&n_clusters, k_qr_cluster<C>, &cfg) != cudaSuccess || n_clusters < 1) {
        (void)cudaGetLastError();
        return false;
    }
    Scratch s(ctx);
    const QrTask* d = s.up(tasks);
    BSM_CUDA(cudaLaunchKernelEx(&cfg, k_qr_cluster<C>, d));
    check_launch(ctx);
    return true;
}

}  // namespace

bool qr_cluster_eligible(int M, int N) {
    const int k = std::min(M, N);
    return k >= kClusterQrMin && qc_smem(M, N, 16) <= kQcSmemMax;
}

bool launch_qr_cluster(Context* ctx, const std::vector<QrTask>& tasks, bool narrow_on_8) {
    if (tasks.empty()) return true;
    int nmax = 0;
    for (const QrTask& t : tasks) nmax = std::max(nmax, std::min(t.M, t.N));
    if (narrow_on_8 && nmax <= kClusterNarrowMax && launch_qc<8>(ctx, tasks)) return true;
    return launch_qc<16>(ctx, tasks) || launch_qc<8>(ctx, tasks);
}

}  // namespace bsm
