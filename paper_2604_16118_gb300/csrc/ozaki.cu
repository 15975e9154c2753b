// FP64 matrix product emulated on bf16 tensor cores by exact integer slice
// products (the Ozaki scheme: Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59
// (2012); integer slices as in Uchino, Ozaki, Imamura 2024).  Not part of the
// paper: an FP64 path for the large contractions of the solver.
//
// Row i of A is scaled by 2^-e_i (e_i the smallest integer with
// max_j |a_ij| < 2^e_i), column j of B by 2^-f_j; the scaled values are cut
// into S digits of 7 bits plus sign (d = trunc(r 2^7), r <- r 2^7 - d), each an
// integer in [-127, 127] and exact in bf16.  C = sum over slice pairs (p, q)
// with p + q = d <= S + 1 of 2^{e_i + f_j - 7d} A_p B_q.  A slice product sums
// integers below 2^14; the pairs of one d (at most 8) over 128 values of k stay
// below 2^24, so the FP32 accumulator of the tensor-core product (tcgen05.mma
// kind::f16, BF16 operands, accumulators in tensor memory) is exact, the
// diagonals are combined exactly in 64-bit integers, and only the FP64
// recombination rounds.
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.h"
#include "tc_common.cuh"

namespace bsm {
namespace {

void launched(Context* ctx) {
    ctx->launches++;
    BSM_CUDA(cudaGetLastError());
}

// One row of op(A) or one column of B: its exponent and its digit slices.
struct OzRow {
    const double* src;
    int64_t stride;        // element k at src[k * stride]
    int len, Kp;           // K and K rounded up to 16
    int* exp;
    __nv_bfloat16* dst;    // slice 0 of the row; slice p at dst + p * slice_stride
    int64_t slice_stride;
};

// One warp per row: e = the smallest integer with max |x| < 2^e, then the S
// digits of x 2^-e (d = trunc(r 2^7), r <- r 2^7 - d, exact), zeros for k >= K.
__global__ void k_oz_rows(const OzRow* __restrict__ rows, int n_rows, int S) {
    const int lane = threadIdx.x & 31;
    const int w = (int)blockIdx.x * (blockDim.x >> 5) + (int)(threadIdx.x >> 5);
    if (w >= n_rows) return;
    const OzRow rw = rows[w];
    double mx = 0.0;
    for (int k = lane; k < rw.len; k += 32) mx = fmax(mx, fabs(rw.src[(int64_t)k * rw.stride]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int ex = 0;
    if (mx > 0.0) frexp(mx, &ex);   // mx = m 2^ex, 0.5 <= m < 1
    if (lane == 0) *rw.exp = ex;
    for (int k = lane; k < rw.Kp; k += 32) {
        double rem = k < rw.len ? ldexp(rw.src[(int64_t)k * rw.stride], -ex) : 0.0;
        for (int p = 0; p < S; ++p) {
            rem *= 128.0;                 // exact (power of two)
            const double d = trunc(rem);
            rem -= d;                     // exact
            rw.dst[p * rw.slice_stride + k] = __double2bfloat16(d);   // |d| <= 127: exact
        }
    }
}

// 16-byte asynchronous copy global -> shared; src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp16(void* smem, const void* gmem, int src_bytes) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(a), "l"(gmem), "r"(src_bytes));
}

constexpr int kOzKStep = 32;       // Kp is a multiple of this (slice rows padded with zeros)
constexpr int kOzMaxS = 8;
constexpr int kOzM = 128;          // tile rows: the M of one tcgen05.mma (cta_group::1)
constexpr int kOzN = 64;           // tile columns: its N, and the tensor-memory columns of one diagonal
constexpr int kOzK = 16;           // k values per staged chunk: the K of one kind::f16 MMA
constexpr int kOzThreads = 128;    // warp w reads tensor-memory lanes 32 w .. 32 w + 31
constexpr int kOzSbo = 8 * kOzK * 2;                  // bytes between 8-row groups of a slice tile
constexpr int kOzSliceA = kOzM * kOzK * 2;            // bytes of one A slice tile (128 x 16 bf16)
constexpr int kOzSliceB = kOzN * kOzK * 2;            // bytes of one B slice tile (64 x 16 bf16)
constexpr uint32_t kOzIdesc = tc::idesc_bf16(kOzM, kOzN);

// byte offset of (row r, k) in a K-major slice tile without swizzle: 8-row x
// 16-byte core matrices, the two core matrices of a row group along k 128
// bytes apart, row groups kOzSbo bytes apart
__device__ __forceinline__ uint32_t oz_off(int r, int k) {
    return (uint32_t)((r >> 3) * kOzSbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// One product of a group, C = alpha op(A) B, with its slices and exponents.
struct OzProd {
    double* C;
    int M, N, Kp, ldc;
    double alpha;
    int64_t a_off, b_off;   // slice 0 of op(A) (M x Kp) and of B^T (N x Kp) in the slice buffers
    int e_off, f_off;       // row exponents of op(A), column exponents of B
};

struct OzTile {
    int prod, m0, n0;
};

// C (M x N, row-major, ldc) = alpha sum_d 2^{e_i + f_j - 7(d + 2)} sum_{p + q = d + 2} A_p B_q
// (slices numbered from 1).  One CTA per 128 x 64 output tile:
//  - k chunks of 16 values of every A and B slice are staged by cp.async into
//    two buffers (the next chunk loads while the tensor cores work on this one);
//  - one thread issues one tcgen05.mma.kind::f16 (BF16 operands, FP32
//    accumulation) per slice pair (p, q), p + q <= S + 1, into the tensor-memory
//    accumulator of its diagonal d (64 columns each) and commits the chunk to
//    the buffer's mbarrier;
//  - every 128 values of k (where the FP32 sums of integer slice products are
//    still exact) the warps read the accumulators with tcgen05.ld and combine
//    the diagonals exactly in two 64-bit integers (four diagonals each: below
//    2^46); the leading group is summed exactly in a 64-bit integer in shared
//    memory over all of k, the trailing one (2^-28 of its weight) in FP64; the
//    next chunk restarts the tensor-memory sums.  The shared accumulators of
//    (row r, column c) sit at r 64 + (c xor (r mod 32)), so the 32 rows a warp
//    updates together fall on distinct banks.
// Every mbarrier wait is bounded; a CTA that gives up sets *err, waits
// boundedly for its MMAs, frees its tensor memory and returns.
template <int S>
__global__ void __launch_bounds__(kOzThreads) k_oz_gemm(const OzProd* __restrict__ prods,
                                                        const OzTile* __restrict__ tiles,
                                                        const __nv_bfloat16* __restrict__ Aslices,
                                                        const __nv_bfloat16* __restrict__ Bslices,
                                                        const int* __restrict__ exps, int* err) {
    constexpr uint32_t kCols = S * kOzN <= 64 ? 64 : S * kOzN <= 128 ? 128 : S * kOzN <= 256 ? 256 : 512;
    constexpr int kBuf = S * (kOzSliceA + kOzSliceB);
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int gave_up;
    unsigned char* base = (unsigned char*)(((uintptr_t)oz_smem + 1023) & ~(uintptr_t)1023);
    long long* acc0 = (long long*)(base + 2 * kBuf);    // exact sums of the leading group (weight 2^-35)
    double* acc1 = (double*)(acc0 + kOzM * kOzN);        // sums of the trailing group, already scaled
    auto sw = [](int r, int c) { return r * kOzN + (c ^ (r & 31)); };
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const OzTile tl = tiles[blockIdx.x];
    const OzProd pd = prods[tl.prod];
    const int M = pd.M, N = pd.N, Kp = pd.Kp;
    const __nv_bfloat16* As = Aslices + pd.a_off;
    const __nv_bfloat16* Bs = Bslices + pd.b_off;
    const int64_t sa = (int64_t)M * Kp, sb = (int64_t)N * Kp;
    const uint32_t bar0 = tc::smem_addr(&bar[0]), bar1 = tc::smem_addr(&bar[1]);
    if (tid == 0) {
        gave_up = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    for (int e = tid; e < kOzM * kOzN; e += kOzThreads) {
        acc0[e] = 0;
        acc1[e] = 0.0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::smem_addr(&tmem_slot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    // stage chunk c (k = 16 c .. 16 c + 15) of every slice into buffer b
    auto stage = [&](int b, int c) {
        unsigned char* bb = base + b * kBuf;
        const int k0 = c * kOzK;
        constexpr int nA = S * kOzM * 2, nB = S * kOzN * 2;   // 16-byte pieces
        for (int i = tid; i < nA + nB; i += kOzThreads) {
            const bool isB = i >= nA;
            const int j = isB ? i - nA : i;
            const int R = isB ? kOzN : kOzM;
            const int p = j / (R * 2), r = (j / 2) % R, piece = j & 1;
            const int row = (isB ? tl.n0 : tl.m0) + r;
            const bool ok = row < (isB ? N : M);
            const __nv_bfloat16* src = (isB ? Bs + p * sb : As + p * sa) + (ok ? (int64_t)row * Kp + k0 + piece * 8 : 0);
            unsigned char* dst = bb + (isB ? S * kOzSliceA + p * kOzSliceB : p * kOzSliceA) + oz_off(r, piece * 8);
            cp16(dst, src, ok ? 16 : 0);
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };
    const int n_chunks = Kp / kOzK;
    constexpr int kFlushChunks = 128 / kOzK;   // exact FP32 sums cover 128 values of k
    uint32_t fresh = (1u << S) - 1u;           // diagonals whose next MMA starts a new sum (thread 0)
    int last = -1;                             // last committed chunk
    if (n_chunks > 0) stage(0, 0);
    for (int c = 0; c < n_chunks; ++c) {
        const int buf = c & 1;
        if (c + 1 < n_chunks) {
            if (c >= 1) {
                // the MMAs of chunk c - 1 read the buffer the next chunk goes to
                if (!tc::mbar_wait(buf ? bar0 : bar1, ((c - 1) >> 1) & 1)) {
                    if (tid == 0) atomicExch(&gave_up, 1);
                }
                __syncthreads();
                if (gave_up) break;
            }
            stage(buf ^ 1, c + 1);
            asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        // the copies of this thread landed; make every thread's copies visible to
        // the tensor cores' (async) proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sA = tc::smem_addr(base + buf * kBuf), sB = sA + S * kOzSliceA;
#pragma unroll
            for (int p = 1; p <= S; ++p)
#pragma unroll
                for (int q = 1; p + q <= S + 1; ++q) {
                    const int d = p + q - 2;
                    tc::mma_bf16(tmem + (uint32_t)(d * kOzN), tc::desc_sbo(sA + (p - 1) * kOzSliceA, kOzSbo),
                                 tc::desc_sbo(sB + (q - 1) * kOzSliceB, kOzSbo), kOzIdesc, (fresh >> d) & 1u ? 0u : 1u);
                    fresh &= ~(1u << d);
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             buf ? bar1 : bar0)
                         : "memory");
        }
        last = c;
        if ((c + 1) % kFlushChunks == 0 || c + 1 == n_chunks) {
            // the sums of this group of chunks: wait for its last commit (which
            // covers every earlier MMA of the issuing thread)
            if (!tc::mbar_wait(buf ? bar1 : bar0, (c >> 1) & 1)) {
                if (tid == 0) atomicExch(&gave_up, 1);
            }
            __syncthreads();
            if (gave_up) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int r = warp * 32 + lane;
            for (int c0 = 0; c0 < kOzN; c0 += 16) {
                long long i0[16], i1[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) i0[j] = i1[j] = 0;
#pragma unroll
                for (int d = 0; d < S; ++d) {
                    uint32_t v[16];
                    tc::ld_32x32b_x16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(d * kOzN + c0), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const long long x = __float2int_rz(__uint_as_float(v[j]));   // an exact integer below 2^24
                        if (d < 4)
                            i0[j] += x << (7 * (3 - d));
                        else
                            i1[j] += x << (7 * (7 - d));
                    }
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    // diagonal d carries 2^-7(d + 2): group 0 (d <= 3) 2^-35 i0, group 1 (d >= 4) 2^-63 i1
                    const int idx = sw(r, c0 + j);
                    acc0[idx] += i0[j];
                    if (S > 4) acc1[idx] = fma((double)i1[j], 0x1p-63, acc1[idx]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            if (tid == 0) fresh = (1u << S) - 1u;
        }
    }
    if (!gave_up) {
        const int* e = exps + pd.e_off;
        const int* f = exps + pd.f_off;
        for (int idx = tid; idx < kOzM * kOzN; idx += kOzThreads) {
            const int rr = idx / kOzN, cc = idx % kOzN;
            const int gr = tl.m0 + rr, gc = tl.n0 + cc;
            if (gr < M && gc < N) {
                const int a = sw(rr, cc);
                const double v = fma((double)acc0[a], 0x1p-35, acc1[a]);
                pd.C[(int64_t)gr * pd.ldc + gc] = pd.alpha * ldexp(ldexp(v, e[gr]), f[gc]);
            }
        }
    } else {
        if (tid == 0) atomicExch(err, 1);
        asm volatile("cp.async.wait_group 0;\n" ::);
        // MMAs may still be in flight: a bounded wait for the last commit before
        // the tensor memory they write is released
        if (last >= 0) tc::mbar_wait((last & 1) ? bar1 : bar0, (last >> 1) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

template <int S>
void launch_oz_gemm(Context* ctx, int n_tiles, const OzProd* prods, const OzTile* tiles, const __nv_bfloat16* As,
                    const __nv_bfloat16* Bs, const int* exps) {
    const size_t smem = 2 * (size_t)S * (kOzSliceA + kOzSliceB) + 16 * (size_t)kOzM * kOzN + 1024;
    static bool attr = false;
    if (!attr) {
        BSM_CUDA(cudaFuncSetAttribute(k_oz_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    k_oz_gemm<S><<<n_tiles, kOzThreads, smem, ctx->stream>>>(prods, tiles, As, Bs, exps, ctx->err_word());
}

}  // namespace

void launch_gemm_ozaki_group(Context* ctx, const std::vector<OzGemm>& gs, int S) {
    BSM_REQUIRE(S >= 1 && S <= kOzMaxS, BSMPS_ERR_INVALID_ARG, "emulated GEMM: 1 <= slices <= 8");
    std::vector<OzProd> prods;
    std::vector<OzTile> tiles;
    int64_t a_tot = 0, b_tot = 0;
    int ex_tot = 0;
    double fl = 0.0;
    for (const OzGemm& g : gs) {
        BSM_REQUIRE(g.M >= 0 && g.N >= 0 && g.K >= 0, BSMPS_ERR_INVALID_ARG, "emulated GEMM: sizes >= 0");
        // the exact 64-bit sum of the leading diagonals (below 2^46 per 128 values of k) stays below 2^63
        BSM_REQUIRE(g.K < (1 << 24), BSMPS_ERR_INVALID_ARG, "emulated GEMM: K < 2^24");
        if (g.M == 0 || g.N == 0) continue;
        const int Kp = (g.K + kOzKStep - 1) / kOzKStep * kOzKStep;
        OzProd pd{g.C, g.M, g.N, Kp, g.ldc, g.alpha, a_tot, b_tot, ex_tot, ex_tot + g.M};
        a_tot += (int64_t)S * g.M * Kp;
        b_tot += (int64_t)S * g.N * Kp;
        ex_tot += g.M + g.N;
        for (int m0 = 0; m0 < g.M; m0 += kOzM)
            for (int n0 = 0; n0 < g.N; n0 += kOzN) tiles.push_back({(int)prods.size(), m0, n0});
        prods.push_back(pd);
        fl += 2.0 * g.M * (double)g.N * g.K;
    }
    if (prods.empty()) return;
    Scratch s(ctx);
    __nv_bfloat16* As = (__nv_bfloat16*)ctx->alloc(sizeof(__nv_bfloat16) * (size_t)(a_tot + 8));
    s.ptrs.push_back(As);
    __nv_bfloat16* Bs = (__nv_bfloat16*)ctx->alloc(sizeof(__nv_bfloat16) * (size_t)(b_tot + 8));
    s.ptrs.push_back(Bs);
    int* exps = (int*)ctx->alloc(sizeof(int) * (size_t)ex_tot);
    s.ptrs.push_back(exps);
    // rows of op(A) and columns of B, with their exponent slots and slice rows
    std::vector<OzRow> rows;
    size_t pi = 0;
    for (const OzGemm& g : gs) {
        if (g.M == 0 || g.N == 0) continue;
        const OzProd& pd = prods[pi++];
        for (int r = 0; r < g.M; ++r)
            rows.push_back({g.A + (int64_t)r * g.lda, 1, g.K, pd.Kp,
                            exps + pd.e_off + r, As + pd.a_off + (int64_t)r * pd.Kp, (int64_t)g.M * pd.Kp});
        for (int c = 0; c < g.N; ++c)
            rows.push_back({g.B + c, (int64_t)g.ldb, g.K, pd.Kp, exps + pd.f_off + c, Bs + pd.b_off + (int64_t)c * pd.Kp,
                            (int64_t)g.N * pd.Kp});
    }
    const OzRow* d_rows = s.up(rows);
    const OzProd* d_prods = s.up(prods);
    const OzTile* d_tiles = s.up(tiles);
    k_oz_rows<<<((int)rows.size() + 7) / 8, 256, 0, ctx->stream>>>(d_rows, (int)rows.size(), S);
    launched(ctx);
    const int nt = (int)tiles.size();
    switch (S) {
        case 1: launch_oz_gemm<1>(ctx, nt, d_prods, d_tiles, As, Bs, exps); break;
        case 2: launch_oz_gemm<2>(ctx, nt, d_prods, d_tiles, As, Bs, exps); break;
        case 3: launch_oz_gemm<3>(ctx, nt, d_prods, d_tiles, As, Bs, exps); break;
        case 4: launch_oz_gemm<4>(ctx, nt, d_prods, d_tiles, As, Bs, exps); break;
        case 5: launch_oz_gemm<5>(ctx, nt, d_prods, d_tiles, As, Bs, exps); break;
        case 6: launch_oz_gemm<6>(ctx, nt, d_prods, d_tiles, As, Bs, exps); break;
        case 7: launch_oz_gemm<7>(ctx, nt, d_prods, d_tiles, As, Bs, exps); break;
        default: launch_oz_gemm<8>(ctx, nt, d_prods, d_tiles, As, Bs, exps); break;
    }
    launched(ctx);
    ctx->flops += fl;
}

void launch_gemm_ozaki(Context* ctx, int M, int N, int K, const double* A, int lda, const double* B, int ldb,
                       double* C, int ldc, int S, double alpha) {
    launch_gemm_ozaki_group(ctx, {OzGemm{A, B, C, M, N, K, lda, ldb, ldc, alpha}}, S);
}

}  // namespace bsm
