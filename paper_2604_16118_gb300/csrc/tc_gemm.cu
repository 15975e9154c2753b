// Grouped FP64-in / FP64-out GEMM on the 5th-generation tensor cores in split
// precision (3xTF32): every operand value v (scaled by its contribution's alpha)
// is split into v_hi (its leading 11 significant bits) and v_lo = tf32(v - v_hi),
// by integer operations on the FP64 bit pattern, and a tile accumulates
// A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 in tensor memory (the A_lo B_lo term,
// below 2^-21 relative, is dropped).  The relative error of an entry is a few
// units of 2^-21 times sum_k |a_ik| |b_kj| plus the FP32 accumulation error.
//
// Every row i of a tile is scaled by 2^-e_i and every column j by 2^-f_j before
// the split, with e_i (f_j) the exponent of the largest |alpha a_ik| (|b_kj|)
// over all contributions of the output: the scaling is exact, keeps every
// operand in TF32's range whatever the magnitudes of the FP64 data (MPS blocks
// can carry factors far outside the FP32 range), and is undone in FP64 when the
// tile is stored (C_ij = acc_ij 2^(e_i + f_j)).
//
// One CTA computes one 128 x 64 output tile of one grouped-GEMM output: 4 warps
// stage 32-wide k chunks of every contribution in shared memory (FP64 loads,
// split, canonical K-major layout without swizzle), one thread issues the
// tcgen05.mma instructions and commits them to an mbarrier, and at the end the
// four warps read their 32 accumulator lanes with tcgen05.ld.  Every wait on the
// mbarrier is bounded by the global timer; a CTA that gives up sets the device
// error word, waits (bounded) for its own MMAs, frees its tensor memory and
// returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.h"
#include "tc_common.cuh"

namespace bsm {
namespace {

constexpr int kTcM = 128;         // rows of a tile: the M of one tcgen05.mma (cta_group::1)
constexpr int kTcN = 64;          // columns of a tile: the N of one tcgen05.mma, also the TMEM columns
constexpr int kTcK = 32;          // k values per staged chunk (4 MMAs of K = 8 for tf32)
constexpr int kTcThreads = 128;   // warp w reads TMEM lanes 32 w .. 32 w + 31
constexpr int kTcOperandBytes = (2 * kTcM + 2 * kTcN) * kTcK * 4;   // A_hi, A_lo, B_hi, B_lo

struct TcTile {
    int out, m0, n0;
};

constexpr uint32_t kTcIdesc = tc::idesc_tf32(kTcM, kTcN);
using tc::global_ns;
using tc::mbar_wait;
using tc::smem_addr;
using tc::tf32_bits;

__device__ __forceinline__ uint32_t tc_off(int r, int k) { return tc::off(r, k); }
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) { return tc::desc(saddr); }

// v 2^-sc for the FP64 value with bit pattern `bits`, split into TF32 parts
// (FP32 bit patterns) by integer operations only (this GPU's FP64 pipe retires
// one warp instruction per 16 cycles per SM): hi = the leading 11 significant
// bits (truncated), lo = the rest rounded to TF32, so |v 2^-sc - hi - lo| <=
// 2^-22 |v 2^-sc|.  The scaling is an exponent subtraction (exact); a scaled
// value below FP32's normal range (2^-126 of a row or column maximum brought
// to [1, 2)) becomes 0, as do FP64 zeros and subnormals.
__device__ __forceinline__ void split_scaled(unsigned long long bits, int sc, uint32_t* hi, uint32_t* lo) {
    const uint32_t sign = (uint32_t)(bits >> 32) & 0x80000000u;
    const int e = (int)((bits >> 52) & 0x7ff);
    const int E = e - 1023 - sc;
    if (e == 0 || E < -126) {
        *hi = *lo = 0u;
        return;
    }
    const unsigned long long m = bits & 0xFFFFFFFFFFFFFull;   // 52 fraction bits
    *hi = sign | ((uint32_t)(E + 127) << 23) | ((uint32_t)(m >> 42) << 13);
    const unsigned long long r = m & ((1ull << 42) - 1);      // value r 2^(E - 52)
    if (r == 0ull) {
        *lo = 0u;
        return;
    }
    const int lz = __clzll((long long)r);                      // leading one at bit 63 - lz
    const int El = E - 52 + (63 - lz);
    if (El < -126) {
        *lo = 0u;
        return;
    }
    const uint32_t frac = (uint32_t)((r << (lz + 1)) >> 41);   // the 23 bits after the leading one
    *lo = (((sign | ((uint32_t)(El + 127) << 23) | frac) + 0x1000u) & 0xFFFFE000u);
}

// acc 2^sh in FP64 from the FP32 accumulator bits by exponent arithmetic, with
// ldexp only for FP32 subnormals and results outside the FP64 normal range.
__device__ __forceinline__ double scale_out(uint32_t a, int sh) {
    const int e = (int)((a >> 23) & 0xff);
    if (e == 0 || e == 255) return ldexp((double)__uint_as_float(a), sh);
    const int E = e - 127 + sh + 1023;
    if (E <= 0 || E >= 2047) return ldexp((double)__uint_as_float(a), sh);
    const unsigned long long b = ((unsigned long long)(a & 0x80000000u) << 32) | ((unsigned long long)E << 52) |
                                 ((unsigned long long)(a & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}

// Exponent e with 2^-e x in [1, 2) for the largest magnitude x given by its bit
// pattern (0 for x = 0: such rows and columns hold zeros only).
__device__ __forceinline__ int pow2_exponent(unsigned long long bits) {
    if (bits == 0ull) return 0;
    return (int)((bits >> 52) & 0x7ff) - 1023;
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    tc::mma_tf32(tmem, adesc, bdesc, kTcIdesc, accumulate);
}

__global__ void __launch_bounds__(kTcThreads) k_gemm_tf32x3(const GemmOut* __restrict__ outs,
                                                           const GemmIn* __restrict__ ins,
                                                           const TcTile* __restrict__ tiles, int* err) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int gave_up;
    __shared__ unsigned long long row_max[kTcM], col_max[kTcN];
    __shared__ int row_sc[kTcM], col_sc[kTcN];
    unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem + 1023) & ~(uintptr_t)1023);
    unsigned char* a_hi = base;
    unsigned char* a_lo = a_hi + kTcM * kTcK * 4;
    unsigned char* b_hi = a_lo + kTcM * kTcK * 4;
    unsigned char* b_lo = b_hi + kTcN * kTcK * 4;
    const TcTile tl = tiles[blockIdx.x];
    const GemmOut o = outs[tl.out];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar_a = smem_addr(&bar);

    if (threadIdx.x == 0) {
        gave_up = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // row and column scales: largest magnitudes (as ordered bit patterns of
    // non-negative doubles) over every contribution, then powers of two
    for (int r = threadIdx.x; r < kTcM; r += kTcThreads) row_max[r] = 0ull;
    for (int c = threadIdx.x; c < kTcN; c += kTcThreads) col_max[c] = 0ull;
    __syncthreads();
    // magnitudes compared as integers (the bit patterns of non-negative doubles
    // are ordered like their values)
    constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
    for (int c = o.beg; c < o.end; ++c) {
        const GemmIn in = ins[c];
        const double aa = fabs(in.alpha);
        const unsigned long long* Ab = (const unsigned long long*)in.A;
        const unsigned long long* Bb = (const unsigned long long*)in.B;
        for (int r = warp; r < kTcM; r += kTcThreads / 32) {
            const int gm = tl.m0 + r;
            if (gm >= o.M) break;
            unsigned long long mx = 0ull;
            for (int k = lane; k < in.K; k += 32) mx = max(mx, Ab[(int64_t)gm * in.lda + k] & kAbs);
            for (int d = 16; d > 0; d >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
            const double mxa = __longlong_as_double((long long)mx) * aa;
            if (lane == 0 && mxa > 0.0) atomicMax(&row_max[r], (unsigned long long)__double_as_longlong(mxa));
        }
        for (int n = threadIdx.x; n < kTcN; n += kTcThreads) {
            const int gn = tl.n0 + n;
            if (gn >= o.N) continue;
            unsigned long long mx = 0ull;
            for (int k = 0; k < in.K; ++k) mx = max(mx, Bb[(int64_t)k * in.ldb + gn] & kAbs);
            if (mx > 0ull) atomicMax(&col_max[n], mx);
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < kTcM; r += kTcThreads) row_sc[r] = pow2_exponent(row_max[r]);
    for (int c = threadIdx.x; c < kTcN; c += kTcThreads) col_sc[c] = pow2_exponent(col_max[c]);
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(kTcN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;

    uint32_t n_commits = 0;
    for (int c = o.beg; c < o.end; ++c) {
        const GemmIn in = ins[c];
        for (int k0 = 0; k0 < in.K; k0 += kTcK) {
            // the chunk before this one must have been consumed by the tensor cores
            if (n_commits > 0) {
                if (!mbar_wait(bar_a, (n_commits - 1) & 1)) {
                    if (threadIdx.x == 0) atomicExch(&gave_up, 1);
                }
                __syncthreads();
                if (gave_up) goto finish;
            }
            // A: rows m0 .. m0 + 127, k0 .. k0 + 31 (alpha folded in), split into hi / lo
            for (int idx = threadIdx.x; idx < kTcM * kTcK; idx += kTcThreads) {
                const int r = idx / kTcK, k = idx % kTcK;
                const int gm = tl.m0 + r, gk = k0 + k;
                uint32_t hi = 0u, lo = 0u;
                if (gm < o.M && gk < in.K)
                    split_scaled((unsigned long long)__double_as_longlong(in.alpha * in.A[(int64_t)gm * in.lda + gk]),
                                 row_sc[r], &hi, &lo);
                const uint32_t off = tc_off(r, k);
                *(uint32_t*)(a_hi + off) = hi;
                *(uint32_t*)(a_lo + off) = lo;
            }
            // B: k0 .. k0 + 31 x columns n0 .. n0 + 63, stored K-major (row = column n)
            for (int idx = threadIdx.x; idx < kTcN * kTcK; idx += kTcThreads) {
                const int k = idx / kTcN, n = idx % kTcN;
                const int gk = k0 + k, gn = tl.n0 + n;
                uint32_t hi = 0u, lo = 0u;
                if (gk < in.K && gn < o.N)
                    split_scaled(((const unsigned long long*)in.B)[(int64_t)gk * in.ldb + gn], col_sc[n], &hi, &lo);
                const uint32_t off = tc_off(n, k);
                *(uint32_t*)(b_hi + off) = hi;
                *(uint32_t*)(b_lo + off) = lo;
            }
            // generic-proxy writes become visible to the tensor cores' (async) proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sa_hi = smem_addr(a_hi), sa_lo = smem_addr(a_lo);
                const uint32_t sb_hi = smem_addr(b_hi), sb_lo = smem_addr(b_lo);
                for (int kk = 0; kk < kTcK / 8; ++kk) {
                    const uint32_t step = (uint32_t)kk * 256u;   // two core matrices along k per MMA
                    const uint32_t first = (n_commits == 0 && kk == 0) ? 0u : 1u;
                    tc_mma(tmem, tc_desc(sa_lo + step), tc_desc(sb_hi + step), first);
                    tc_mma(tmem, tc_desc(sa_hi + step), tc_desc(sb_lo + step), 1u);
                    tc_mma(tmem, tc_desc(sa_hi + step), tc_desc(sb_hi + step), 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 bar_a)
                             : "memory");
            }
            ++n_commits;
        }
    }
    if (n_commits > 0) {
        if (!mbar_wait(bar_a, (n_commits - 1) & 1)) {
            if (threadIdx.x == 0) atomicExch(&gave_up, 1);
        }
        __syncthreads();
        if (gave_up) goto finish;
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    {
        // warp w holds rows m0 + 32 w + lane of the tile
        const int row = tl.m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < kTcN; c0 += 16) {
            uint32_t v[16];
            if (n_commits > 0) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                    "%12, %13, %14, %15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0u;
            }
            if (row < o.M) {
                double* cr = o.C + (int64_t)row * o.ldc;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = tl.n0 + c0 + j;
                    const double acc = scale_out(v[j], row_sc[warp * 32 + lane] + col_sc[c0 + j]);
                    if (col < o.N) cr[col] = o.beta == 0.0 ? acc : o.beta * cr[col] + acc;
                }
            }
        }
    }
finish:
    if (gave_up) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        // MMAs of this CTA may still be in flight: give them a bounded wait before
        // the tensor memory they write is released
        if (n_commits > 0) mbar_wait(bar_a, (n_commits - 1) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN));
}

}  // namespace

bool gemm_tf32x3_eligible(const std::vector<GemmOut>& outs, const std::vector<GemmIn>& ins) {
    for (const GemmOut& g : outs)
        for (int c = g.beg; c < g.end; ++c)
            if (ins[c].transA) return false;
    return true;
}

void launch_gemm_tf32x3(Context* ctx, const std::vector<GemmOut>& outs, const std::vector<GemmIn>& ins, int kind) {
    if (outs.empty()) return;
    std::vector<TcTile> tiles;
    double fl = 0.0, by = 0.0;
    for (int o = 0; o < (int)outs.size(); ++o) {
        const GemmOut& g = outs[o];
        if (g.M <= 0 || g.N <= 0) continue;
        for (int m0 = 0; m0 < g.M; m0 += kTcM)
            for (int n0 = 0; n0 < g.N; n0 += kTcN) tiles.push_back({o, m0, n0});
        for (int c = g.beg; c < g.end; ++c) {
            BSM_REQUIRE(!ins[c].transA, BSMPS_ERR_INVALID_ARG, "split-precision GEMM: untransposed operands only");
            fl += 2.0 * g.M * g.N * (double)ins[c].K;
            by += 8.0 * ((double)g.M * ins[c].K + (double)ins[c].K * g.N);
        }
        by += 8.0 * g.M * (double)g.N * (g.beta == 0.0 ? 1.0 : 2.0);
    }
    if (tiles.empty()) return;
    ctx->flops += fl;
    Scratch s(ctx);
    const GemmOut* d_outs = s.up(outs);
    const GemmIn* d_ins = ins.empty() ? nullptr : s.up(ins);
    const TcTile* d_tiles = s.up(tiles);
    const int smem = kTcOperandBytes + 1024;   // room to align the operand tiles to 1024 bytes
    static bool attr_set = false;
    if (!attr_set) {
        BSM_CUDA(cudaFuncSetAttribute(k_gemm_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_set = true;
    }
    ProfScope ps(ctx, kind, fl, by);
    k_gemm_tf32x3<<<(unsigned)tiles.size(), kTcThreads, smem, ctx->stream>>>(d_outs, d_ins, d_tiles,
                                                                             ctx->err_word());
    check_launch(ctx);
    ps.done();
}

}  // namespace bsm
