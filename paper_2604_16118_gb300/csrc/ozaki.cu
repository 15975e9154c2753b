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
// below 2^24, so the FP32 accumulator of the tensor-core product is exact and
// only the FP64 recombination rounds.
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.h"

namespace bsm {
namespace {

constexpr int kOzTile = 64;      // output tile per CTA (64 x 64)
constexpr int kOzChunk = 128;    // k values per exact FP32 accumulation
constexpr int kOzThreads = 128;  // 4 warps, 2 x 2 warp tiles of 32 x 32

void launched(Context* ctx) {
    ctx->launches++;
    BSM_CUDA(cudaGetLastError());
}

// e_i of every row of the row-major M x K matrix A: one warp per row.
__global__ void k_oz_row_exp(const double* __restrict__ A, int M, int K, int lda, int* __restrict__ e) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= M) return;
    double mx = 0.0;
    for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(A[(int64_t)row * lda + k]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
        int ex = 0;
        if (mx > 0.0) frexp(mx, &ex);   // mx = m 2^ex, 0.5 <= m < 1
        e[row] = ex;
    }
}

// f_j of every column of the row-major K x N matrix B: one thread per column.
__global__ void k_oz_col_exp(const double* __restrict__ B, int K, int N, int ldb, int* __restrict__ f) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= N) return;
    double mx = 0.0;
    for (int k = 0; k < K; ++k) mx = fmax(mx, fabs(B[(int64_t)k * ldb + col]));
    int ex = 0;
    if (mx > 0.0) frexp(mx, &ex);
    f[col] = ex;
}

// Digits of A (row scale e) into S bf16 slices, each M x Kp row-major; or of B
// (column scale f) into S slices stored transposed, N x Kp.  k >= K: zeros.
__global__ void k_oz_split(const double* __restrict__ X, int rows, int cols, int ld, int trans,
                           const int* __restrict__ ex, int S, int Kp, __nv_bfloat16* __restrict__ out,
                           int64_t slice_stride) {
    // output element (r, k): r < rows_out, k < Kp (rows_out = rows of A or columns of B)
    const int64_t n = (int64_t)(trans ? cols : rows) * Kp;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / Kp), k = (int)(idx % Kp);
        double v = 0.0;
        if (!trans) {
            if (k < cols) v = X[(int64_t)r * ld + k];   // A: row r, column k
        } else {
            if (k < rows) v = X[(int64_t)k * ld + r];   // B: row k, column r
        }
        double rem = ldexp(v, -ex[r]);
        for (int p = 0; p < S; ++p) {
            rem *= 128.0;                 // exact (power of two)
            const double d = trunc(rem);
            rem -= d;                     // exact
            out[p * slice_stride + idx] = __double2bfloat16(d);   // |d| <= 127: exact
        }
    }
}

__device__ __forceinline__ unsigned ld_pair(const __nv_bfloat16* base, int64_t off, bool ok) {
    return ok ? *reinterpret_cast<const unsigned*>(base + off) : 0u;
}

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], const unsigned b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C (M x N, row-major, ldc) = sum_d 2^{e_i + f_j - 7d} sum_{p + q = d} A_p B_q.
// Fragment layouts of m16n8k16 (g = lane / 4, t = lane % 4): A rows g and g+8,
// k pairs 2t and 2t+8; B columns g, k pairs 2t and 2t+8; C rows g and g+8,
// columns 2t, 2t+1.
__global__ void __launch_bounds__(kOzThreads) k_oz_gemm(const __nv_bfloat16* __restrict__ As,
                                                        const __nv_bfloat16* __restrict__ Bs, int64_t sa,
                                                        int64_t sb, const int* __restrict__ e,
                                                        const int* __restrict__ f, int M, int N, int Kp, int S,
                                                        double* __restrict__ C, int ldc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * kOzTile + (warp >> 1) * 32;
    const int n0 = blockIdx.x * kOzTile + (warp & 1) * 32;
    double acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[i][j][v] = 0.0;
    for (int d = 2; d <= S + 1; ++d) {
        const int p_lo = d - S > 1 ? d - S : 1, p_hi = d - 1 < S ? d - 1 : S;
        const double w = ldexp(1.0, -7 * d);
        for (int k0 = 0; k0 < Kp; k0 += kOzChunk) {
            float c32[2][4][4];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int v = 0; v < 4; ++v) c32[i][j][v] = 0.f;
            const int k1 = k0 + kOzChunk < Kp ? k0 + kOzChunk : Kp;
            for (int kk = k0; kk < k1; kk += 16) {
                for (int p = p_lo; p <= p_hi; ++p) {
                    const __nv_bfloat16* Ap = As + (int64_t)(p - 1) * sa;
                    const __nv_bfloat16* Bq = Bs + (int64_t)(d - p - 1) * sb;
                    unsigned a[2][4], b[4][2];
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int r0 = m0 + i * 16 + g, r1 = r0 + 8;
                        a[i][0] = ld_pair(Ap, (int64_t)r0 * Kp + kk + 2 * t, r0 < M);
                        a[i][1] = ld_pair(Ap, (int64_t)r1 * Kp + kk + 2 * t, r1 < M);
                        a[i][2] = ld_pair(Ap, (int64_t)r0 * Kp + kk + 2 * t + 8, r0 < M);
                        a[i][3] = ld_pair(Ap, (int64_t)r1 * Kp + kk + 2 * t + 8, r1 < M);
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int cn = n0 + j * 8 + g;
                        b[j][0] = ld_pair(Bq, (int64_t)cn * Kp + kk + 2 * t, cn < N);
                        b[j][1] = ld_pair(Bq, (int64_t)cn * Kp + kk + 2 * t + 8, cn < N);
                    }
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) mma_bf16(c32[i][j], a[i], b[j]);
                }
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[i][j][v] += (double)c32[i][j][v] * w;
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int r = m0 + i * 16 + g + (v >= 2 ? 8 : 0);
                const int c = n0 + j * 8 + 2 * t + (v & 1);
                if (r < M && c < N) C[(int64_t)r * ldc + c] = ldexp(ldexp(acc[i][j][v], e[r]), f[c]);
            }
}

}  // namespace

void launch_gemm_ozaki(Context* ctx, int M, int N, int K, const double* A, int lda, const double* B, int ldb,
                       double* C, int ldc, int S) {
    BSM_REQUIRE(M >= 0 && N >= 0 && K >= 0 && S >= 1 && S <= 8, BSMPS_ERR_INVALID_ARG,
                "emulated GEMM: sizes >= 0 and 1 <= slices <= 8");
    if (M == 0 || N == 0) return;
    const int Kp = (K + 15) / 16 * 16;
    Scratch s(ctx);
    int* e = (int*)ctx->alloc(sizeof(int) * (size_t)M);
    s.ptrs.push_back(e);
    int* f = (int*)ctx->alloc(sizeof(int) * (size_t)N);
    s.ptrs.push_back(f);
    const int64_t sa = (int64_t)M * Kp, sb = (int64_t)N * Kp;
    __nv_bfloat16* As = (__nv_bfloat16*)ctx->alloc(sizeof(__nv_bfloat16) * (size_t)(sa * S + 2));
    s.ptrs.push_back(As);
    __nv_bfloat16* Bs = (__nv_bfloat16*)ctx->alloc(sizeof(__nv_bfloat16) * (size_t)(sb * S + 2));
    s.ptrs.push_back(Bs);
    if (K == 0) {
        for (int r = 0; r < M; ++r) BSM_CUDA(cudaMemsetAsync(C + (int64_t)r * ldc, 0, sizeof(double) * N, ctx->stream));
        return;
    }
    k_oz_row_exp<<<(M + 7) / 8, 256, 0, ctx->stream>>>(A, M, K, lda, e);
    launched(ctx);
    k_oz_col_exp<<<(N + 127) / 128, 128, 0, ctx->stream>>>(B, K, N, ldb, f);
    launched(ctx);
    const int blocks_a = (int)std::min<int64_t>((sa + 255) / 256, 152 * 16);
    k_oz_split<<<blocks_a, 256, 0, ctx->stream>>>(A, M, K, lda, 0, e, S, Kp, As, sa);
    launched(ctx);
    const int blocks_b = (int)std::min<int64_t>((sb + 255) / 256, 152 * 16);
    k_oz_split<<<blocks_b, 256, 0, ctx->stream>>>(B, K, N, ldb, 1, f, S, Kp, Bs, sb);
    launched(ctx);
    dim3 grid((N + kOzTile - 1) / kOzTile, (M + kOzTile - 1) / kOzTile);
    k_oz_gemm<<<grid, kOzThreads, 0, ctx->stream>>>(As, Bs, sa, sb, e, f, M, N, Kp, S, C, ldc);
    launched(ctx);
    ctx->flops += 2.0 * M * (double)N * K;
}

}  // namespace bsm
