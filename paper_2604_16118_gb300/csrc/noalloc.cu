// Allocation-free inner product <a, O b>: the environment contraction of
// bsmps_dot with every temporary (environment blocks, intermediate products and
// the kernel task lists) placed in one file-scope device array instead of
// memory obtained from the allocator.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "dense_dev.cuh"
#include "ops.h"

namespace bsm {
namespace {

// 32 MiB of scratch, 256-byte aligned; held by every device that loads the library.
constexpr size_t kNaBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

constexpr int kNaThreads = dev::kThreads;
constexpr int kNaTile = dev::kGemmTile;

struct NaOut {
    int64_t c;         // output offset (doubles) into the scratch
    int M, N;
    int beg, end;
};

struct NaIn {
    const double* A;   // absolute device pointers (MPS cores or scratch)
    const double* B;
    int K, lda, ldb, transA;
    double alpha;
};

struct NaTile {
    int out, m0, n0;
};

// The grouped GEMM of the environment sweep with its outputs and task lists in
// the scratch: C = sum over contributions alpha op(A) B, C row-major M x N
// (ld N); the tile loop is the one of the library's grouped GEMM.
__global__ void __launch_bounds__(kNaThreads) k_gemm_noalloc(double* __restrict__ base,
                                                            const NaOut* __restrict__ outs,
                                                            const NaIn* __restrict__ ins,
                                                            const NaTile* __restrict__ tiles) {
    __shared__ double As[kNaTile][kNaTile + 1];
    __shared__ double Bs[kNaTile][kNaTile + 1];
    const NaTile tl = tiles[blockIdx.x];
    const NaOut o = outs[tl.out];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = o.beg; c < o.end; ++c) dev::gemm_tile_accumulate(ins[c], o.M, o.N, tl.m0, tl.n0, As, Bs, acc);
    const int gn = tl.n0 + tx;
    if (gn >= o.N) return;
    for (int r = 0; r < 4; ++r) {
        const int gm = tl.m0 + ty + 8 * r;
        if (gm < o.M) base[o.c + (int64_t)gm * o.N + gn] = acc[r];
    }
}

// sum of the final 1x1 environment blocks into base[dst]
__global__ void k_sum_noalloc(double* __restrict__ base, const int64_t* __restrict__ src, int n, int64_t dst) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += base[src[i]];
        base[dst] = s;
    }
}

// Device address of the scratch, resolved once per device (with that device current).
std::mutex g_na_mutex;
std::map<int, double*> g_na_base;

double* scratch_base(int device) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    auto it = g_na_base.find(device);
    if (it != g_na_base.end()) return it->second;
    void* p = nullptr;
    BSM_CUDA(cudaGetSymbolAddress(&p, g_na_scratch));
    g_na_base[device] = (double*)p;
    return (double*)p;
}

// Bump layout of the scratch (offsets in bytes, 256-byte aligned).
struct Bump {
    size_t used = 0;
    size_t take(size_t bytes) {
        const size_t off = (used + 255) & ~size_t(255);
        used = off + bytes;
        return off;
    }
};

}  // namespace

// Same contraction as op_dot_batch for one problem; returns the status through
// exceptions like the other operations.
double op_dot_noalloc(Context* ctx, const Mps* a, const Mps* b, const Mpo* W, double shift) {
    const Layout& A = a->lay;
    const Layout& B = b->lay;
    BSM_REQUIRE(same_space(A, B), BSMPS_ERR_INVALID_ARG, "dot of MPS of different spaces");
    const int K = A.K;
    Mpo ident;
    if (!W) {
        ident.K = K;
        ident.species = A.species;
        ident.charges.assign(K + 1, std::vector<Charge>(1, Charge{0, 0}));
        ident.entries.assign(K, {{0, 0, 0, 0, 1.0}, {0, 0, 1, 1, 1.0}});
    } else {
        BSM_REQUIRE(W->K == K && W->species == A.species, BSMPS_ERR_INVALID_ARG,
                    "MPO and MPS act on different sites");
    }
    const Mpo& O = W ? *W : ident;
    double* base = scratch_base(ctx->device);
    unsigned char* bytes = (unsigned char*)base;

    struct Env {
        int c, ia, ib, rows, cols;
        int64_t off;   // doubles, into the scratch
    };
    auto lookup = [](const Layout& L, int t) {
        std::vector<int> idx(L.bonds[t].q.size() * 2, -1);
        for (int i = 0; i < (int)L.blocks[t].size(); ++i) idx[L.blocks[t][i].li * 2 + L.blocks[t][i].sigma] = i;
        return idx;
    };
    // two environment regions alternate between sites; region 0 starts with [[1]]
    std::vector<Env> E;
    size_t region_off[2] = {0, 0};
    size_t region_cap = 0;
    // first pass on the host: size of the largest environment, T and task set
    size_t need_env = 8, need_site = 0;
    {
        std::vector<std::tuple<int, int, int, int, int>> cur;   // c, ia, ib, rows, cols
        if (!A.bonds[0].q.empty() && !B.bonds[0].q.empty()) cur.push_back({0, 0, 0, 1, 1});
        for (int t = 0; t < K; ++t) {
            const std::vector<int> al = lookup(A, t), bl = lookup(B, t);
            size_t tsz = 0, ntask = 0, ntile = 0;
            std::map<std::tuple<int, int, int>, int> outs;
            std::map<int, std::vector<int>> by_chan;
            for (int e = 0; e < (int)cur.size(); ++e) by_chan[std::get<0>(cur[e])].push_back(e);
            for (int e = 0; e < (int)cur.size(); ++e)
                for (int si = 0; si < 2; ++si) {
                    const int bb = bl[std::get<2>(cur[e]) * 2 + si];
                    if (bb < 0) continue;
                    tsz += (size_t)std::get<3>(cur[e]) * B.blocks[t][bb].cols;
                    ntask++;
                    ntile += ((std::get<3>(cur[e]) + 31) / 32) * ((B.blocks[t][bb].cols + 31) / 32);
                }
            for (const MpoEntry& me : O.entries[t]) {
                auto it = by_chan.find(me.a);
                if (it == by_chan.end()) continue;
                for (int e : it->second) {
                    const int ab = al[std::get<1>(cur[e]) * 2 + me.so], bb = bl[std::get<2>(cur[e]) * 2 + me.si];
                    if (ab < 0 || bb < 0) continue;
                    outs[{me.b, A.blocks[t][ab].ri, B.blocks[t][bb].ri}]++;
                    ntask++;
                }
            }
            std::vector<std::tuple<int, int, int, int, int>> nxt;
            size_t esz = 0;
            for (auto& kv : outs) {
                const int ra = std::get<1>(kv.first), rb = std::get<2>(kv.first);
                const int r = A.bonds[t + 1].dim[ra], c = B.bonds[t + 1].dim[rb];
                nxt.push_back({std::get<0>(kv.first), ra, rb, r, c});
                esz += (size_t)r * c;
                ntile += ((r + 31) / 32) * ((c + 31) / 32);
            }
            need_env = std::max(need_env, esz * 8 + 256 * nxt.size() + 256);
            need_site = std::max(need_site, tsz * 8 + 256 * (ntask + 8) +
                                                (ntask + outs.size() + cur.size() * 2) *
                                                    (sizeof(NaIn) + sizeof(NaOut)) +
                                                ntile * sizeof(NaTile) + 4096);
            cur.swap(nxt);
        }
    }
    region_cap = need_env;
    Bump bump;
    region_off[0] = bump.take(region_cap);
    region_off[1] = bump.take(region_cap);
    const size_t site_off = bump.take(need_site);
    const size_t result_off = bump.take(64 + 8 * 1024);
    BSM_REQUIRE(bump.used <= kNaBytes, BSMPS_ERR_RANK_CAP,
                "bsmps_dot_noalloc: the contraction needs " + std::to_string(bump.used) +
                    " bytes of scratch, above the fixed maximum of " + std::to_string(kNaBytes) + " bytes");

    // [[1]] in region 0
    {
        const double one = 1.0;
        BSM_CUDA(cudaMemcpyAsync(bytes + region_off[0], &one, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    }
    if (!A.bonds[0].q.empty() && !B.bonds[0].q.empty()) E.push_back({0, 0, 0, 1, 1, (int64_t)(region_off[0] / 8)});
    int region = 0;
    for (int t = 0; t < K; ++t) {
        const std::vector<int> al = lookup(A, t), bl = lookup(B, t);
        size_t cursor = site_off;
        auto take = [&](size_t by) {
            const size_t off = (cursor + 255) & ~size_t(255);
            cursor = off + by;
            return off;
        };
        // T blocks
        struct TB {
            int env, sigma, rows, cols;
            int64_t off;
        };
        std::vector<TB> T;
        std::vector<std::array<int, 2>> tidx(E.size(), {-1, -1});
        for (int e = 0; e < (int)E.size(); ++e)
            for (int si = 0; si < 2; ++si) {
                const int bb = bl[E[e].ib * 2 + si];
                if (bb < 0) continue;
                tidx[e][si] = (int)T.size();
                const int cols = B.blocks[t][bb].cols;
                T.push_back({e, si, E[e].rows, cols, (int64_t)(take((size_t)E[e].rows * cols * 8) / 8)});
            }
        std::map<int, std::vector<int>> by_chan;
        for (int e = 0; e < (int)E.size(); ++e) by_chan[E[e].c].push_back(e);
        std::map<std::tuple<int, int, int>, std::vector<std::tuple<int, int, double>>> contrib;
        for (int ei = 0; ei < (int)O.entries[t].size(); ++ei) {
            const MpoEntry& me = O.entries[t][ei];
            auto it = by_chan.find(me.a);
            if (it == by_chan.end()) continue;
            double w = me.w;
            if (W && t == 0 && (ei == W->shift_entry[0] || ei == W->shift_entry[1])) w += shift;
            for (int e : it->second) {
                const int ab = al[E[e].ia * 2 + me.so];
                const int ti = tidx[e][me.si];
                if (ab < 0 || ti < 0) continue;
                const int bb = bl[E[e].ib * 2 + me.si];
                contrib[{me.b, A.blocks[t][ab].ri, B.blocks[t][bb].ri}].push_back({ti, ab, w});
            }
        }
        // stage 1: T = E X_b
        std::vector<NaOut> o1;
        std::vector<NaIn> i1;
        std::vector<NaTile> t1;
        for (const TB& tb : T) {
            const Env& eb = E[tb.env];
            const Block& bk = B.blocks[t][bl[eb.ib * 2 + tb.sigma]];
            for (int m0 = 0; m0 < tb.rows; m0 += kNaTile)
                for (int n0 = 0; n0 < tb.cols; n0 += kNaTile) t1.push_back({(int)o1.size(), m0, n0});
            o1.push_back({tb.off, tb.rows, tb.cols, (int)i1.size(), (int)i1.size() + 1});
            i1.push_back({base + eb.off, b->core[t] + bk.off, eb.cols, eb.cols, bk.cols, 0, 1.0});
        }
        // stage 2: E' = sum w X_a^T T into the other region
        const int nreg = 1 - region;
        size_t ecur = region_off[nreg];
        std::vector<Env> En;
        std::vector<NaOut> o2;
        std::vector<NaIn> i2;
        std::vector<NaTile> t2;
        for (auto& kv : contrib) {
            const int d = std::get<0>(kv.first), ra = std::get<1>(kv.first), rb = std::get<2>(kv.first);
            const int r = A.bonds[t + 1].dim[ra], c = B.bonds[t + 1].dim[rb];
            const size_t off = (ecur + 255) & ~size_t(255);
            ecur = off + (size_t)r * c * 8;
            BSM_REQUIRE(ecur <= region_off[nreg] + region_cap, BSMPS_ERR_RANK_CAP,
                        "bsmps_dot_noalloc: environment region overflow");
            En.push_back({d, ra, rb, r, c, (int64_t)(off / 8)});
            const int beg = (int)i2.size();
            for (auto& ct : kv.second) {
                const TB& tb = T[std::get<0>(ct)];
                const Block& ab = A.blocks[t][std::get<1>(ct)];
                i2.push_back({a->core[t] + ab.off, base + tb.off, ab.rows, ab.cols, tb.cols, 1, std::get<2>(ct)});
            }
            for (int m0 = 0; m0 < r; m0 += kNaTile)
                for (int n0 = 0; n0 < c; n0 += kNaTile) t2.push_back({(int)o2.size(), m0, n0});
            o2.push_back({(int64_t)(off / 8), r, c, beg, (int)i2.size()});
        }
        // task lists into the scratch (after the T blocks of this site): every
        // offset is laid out and checked against the site region before any copy
        const void* srcs[6] = {o1.data(), i1.data(), t1.data(), o2.data(), i2.data(), t2.data()};
        const size_t lens[6] = {o1.size() * sizeof(NaOut), i1.size() * sizeof(NaIn), t1.size() * sizeof(NaTile),
                                o2.size() * sizeof(NaOut), i2.size() * sizeof(NaIn), t2.size() * sizeof(NaTile)};
        size_t offs[6];
        for (int q = 0; q < 6; ++q) offs[q] = take(lens[q]);
        BSM_REQUIRE(cursor <= site_off + need_site, BSMPS_ERR_RANK_CAP, "bsmps_dot_noalloc: site region overflow");
        for (int q = 0; q < 6; ++q)
            if (lens[q] > 0)
                BSM_CUDA(cudaMemcpyAsync(bytes + offs[q], srcs[q], lens[q], cudaMemcpyHostToDevice, ctx->stream));
        const size_t po1 = offs[0], pi1 = offs[1], pt1 = offs[2], po2 = offs[3], pi2 = offs[4], pt2 = offs[5];
        if (!t1.empty()) {
            k_gemm_noalloc<<<(unsigned)t1.size(), kNaThreads, 0, ctx->stream>>>(
                base, (const NaOut*)(bytes + po1), (const NaIn*)(bytes + pi1), (const NaTile*)(bytes + pt1));
            ctx->launches++;
            BSM_CUDA(cudaGetLastError());
        }
        if (!t2.empty()) {
            k_gemm_noalloc<<<(unsigned)t2.size(), kNaThreads, 0, ctx->stream>>>(
                base, (const NaOut*)(bytes + po2), (const NaIn*)(bytes + pi2), (const NaTile*)(bytes + pt2));
            ctx->launches++;
            BSM_CUDA(cudaGetLastError());
        }
        E.swap(En);
        region = nreg;
    }
    // sum of the final 1x1 blocks; the result slot is overwritten, never accumulated
    std::vector<int64_t> src;
    for (const Env& e : E) src.push_back(e.off);
    const size_t psrc = result_off + 64;
    BSM_REQUIRE(src.size() <= 1024, BSMPS_ERR_RANK_CAP, "bsmps_dot_noalloc: too many final blocks");
    if (!src.empty())
        BSM_CUDA(cudaMemcpyAsync(bytes + psrc, src.data(), src.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    k_sum_noalloc<<<1, 32, 0, ctx->stream>>>(base, (const int64_t*)(bytes + psrc), (int)src.size(),
                                            (int64_t)(result_off / 8));
    ctx->launches++;
    BSM_CUDA(cudaGetLastError());
    double out = 0.0;
    BSM_CUDA(cudaMemcpyAsync(&out, bytes + result_off, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    BSM_CUDA(cudaStreamSynchronize(ctx->stream));
    return out;
}

size_t noalloc_capacity_bytes() { return kNaBytes; }

}  // namespace bsm
