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

__device__ __forceinline__ void mma_bf16(float c[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
    // a pure function of registers: the compiler may schedule it freely
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(unsigned r[4], const void* smem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// 16-byte asynchronous copy global -> shared; src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp16(void* smem, const void* gmem, int src_bytes) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(a), "l"(gmem), "r"(src_bytes));
}

constexpr int kOzKStep = 32;                                // values of k per staged buffer (two k16 steps)
constexpr int kOzPitch = 40;                                // bf16 per staged row (80 B: ldmatrix rows on distinct banks)
constexpr int kOzMaxS = 8;
constexpr int kOzStage = 2 * kOzMaxS * kOzTile * kOzPitch;  // bf16 of A and B slices for one staged step
constexpr int kOzWarps = 16;                                // 4 x 4 warp tiles of 16 x 16

// C (M x N, row-major, ldc) = sum_d 2^{e_i + f_j - 7d} sum_{p + q = d} A_p B_q.
// Per k16 step all slices of the CTA's 64 x 64 tile are staged in shared memory
// (double-buffered cp.async); each warp owns a 16 x 16 output tile and keeps
// one FP32 accumulator per d, flushed to FP64 every kOzChunk values of k.
// Fragment layouts of m16n8k16 (g = lane / 4, t = lane % 4): C rows g, g+8,
// columns 2t, 2t+1.
// Slice pairs (p, q), p + q <= S + 1, ordered by p then q: consecutive pairs
// accumulate into different d = p + q (independent tensor-core chains) and share
// the fragment of A_p.  abuf: which of two A fragment registers holds A_p.
template <int S>
struct OzPairs {
    int p[S * (S + 1) / 2], q[S * (S + 1) / 2], abuf[S * (S + 1) / 2];
    constexpr OzPairs() : p(), q(), abuf() {
        int i = 0;
        for (int pp = 1; pp <= S; ++pp)
            for (int qq = 1; pp + qq <= S + 1; ++qq) {
                p[i] = pp;
                q[i] = qq;
                abuf[i] = (pp - 1) & 1;
                ++i;
            }
    }
};

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

template <int S>
__global__ void __launch_bounds__(kOzWarps * 32) k_oz_gemm(const OzProd* __restrict__ prods,
                                                           const OzTile* __restrict__ tiles,
                                                           const __nv_bfloat16* __restrict__ Aslices,
                                                           const __nv_bfloat16* __restrict__ Bslices,
                                                           const int* __restrict__ exps) {
    constexpr int NP = S * (S + 1) / 2;
    constexpr OzPairs<S> PR{};
    extern __shared__ __align__(16) __nv_bfloat16 sm_oz[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const OzTile tl = tiles[blockIdx.x];
    const OzProd pd = prods[tl.prod];
    const int M = pd.M, N = pd.N, Kp = pd.Kp, ldc = pd.ldc;
    const double alpha = pd.alpha;
    double* __restrict__ C = pd.C;
    const __nv_bfloat16* As = Aslices + pd.a_off;
    const __nv_bfloat16* Bs = Bslices + pd.b_off;
    const int64_t sa = (int64_t)M * Kp, sb = (int64_t)N * Kp;
    const int* e = exps + pd.e_off;
    const int* f = exps + pd.f_off;
    const int mt = tl.m0, nt = tl.n0;
    const int wm = (warp >> 2) * 16, wn = (warp & 3) * 16;
    // staging of the kOzKStep values of k starting at kk into buffer b
    constexpr int kChunks = kOzKStep / 8;   // 16-byte pieces per staged row
    auto stage = [&](int b, int kk) {
        __nv_bfloat16* base = sm_oz + b * kOzStage;
        constexpr int n_copies = 2 * S * kOzTile * kChunks;
        for (int i = tid; i < n_copies; i += kOzWarps * 32) {
            const int which = i / (S * kOzTile * kChunks);            // 0: A, 1: B
            const int rem = i - which * S * kOzTile * kChunks;
            const int p = rem / (kOzTile * kChunks), r = (rem / kChunks) % kOzTile, piece = rem % kChunks;
            const int row = (which ? nt : mt) + r;
            const bool ok = row < (which ? N : M);
            const __nv_bfloat16* src = (which ? Bs + p * sb : As + p * sa) + (ok ? (int64_t)row * Kp + kk + piece * 8 : 0);
            __nv_bfloat16* dst = base + ((which * kOzMaxS + p) * kOzTile + r) * kOzPitch + piece * 8;
            cp16(dst, src, ok ? 16 : 0);
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };
    float c32[S][2][4];
    double acc[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[j][v] = 0.0;
#pragma unroll
    for (int d = 0; d < S; ++d)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int v = 0; v < 4; ++v) c32[d][j][v] = 0.f;
    const int nk = Kp / kOzKStep;
    // ldmatrix row addresses: A rows wm + lane % 16, k half lane / 16;
    // B rows (columns of B) wn + lane % 8 + (lane / 16) 8, k half (lane / 8) % 2
    const int a_off = (wm + (lane & 15)) * kOzPitch + (lane >> 4) * 8;
    const int b_off = (wn + (lane & 7) + (lane >> 4) * 8) * kOzPitch + ((lane >> 3) & 1) * 8;
    if (nk > 0) stage(0, 0);
    for (int step = 0; step < nk; ++step) {
        if (step + 1 < nk) {
            stage((step + 1) & 1, (step + 1) * kOzKStep);
            asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        __syncthreads();
#pragma unroll 1
        for (int kh = 0; kh < kOzKStep / 16; ++kh) {
        const __nv_bfloat16* base = sm_oz + (step & 1) * kOzStage + kh * 16;
        // fragments of pair i + 1 are loaded before the products of pair i; the
        // fragment of A_p is loaded once per p
        unsigned a[2][4], b[2][4];
        ldsm_x4(a[PR.abuf[0]], base + (PR.p[0] - 1) * kOzTile * kOzPitch + a_off);
        ldsm_x4(b[0], base + (kOzMaxS + PR.q[0] - 1) * kOzTile * kOzPitch + b_off);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const int bc = i & 1, ac = PR.abuf[i];
            if (i + 1 < NP) {
                if (PR.p[i + 1] != PR.p[i])
                    ldsm_x4(a[PR.abuf[i + 1]], base + (PR.p[i + 1] - 1) * kOzTile * kOzPitch + a_off);
                ldsm_x4(b[bc ^ 1], base + (kOzMaxS + PR.q[i + 1] - 1) * kOzTile * kOzPitch + b_off);
            }
            const int d = PR.p[i] + PR.q[i] - 2;
            mma_bf16(c32[d][0], a[ac][0], a[ac][1], a[ac][2], a[ac][3], b[bc][0], b[bc][1]);
            mma_bf16(c32[d][1], a[ac][0], a[ac][1], a[ac][2], a[ac][3], b[bc][2], b[bc][3]);
        }
        }
        // exact FP32 sums cover at most kOzChunk values of k: flush to FP64
        if ((step + 1) % (kOzChunk / kOzKStep) == 0 || step + 1 == nk) {
#pragma unroll
            for (int d = 0; d < S; ++d) {
                const double w = ldexp(1.0, -7 * (d + 2));
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        acc[j][v] = fma((double)c32[d][j][v], w, acc[j][v]);
                        c32[d][j][v] = 0.f;
                    }
            }
        }
        __syncthreads();   // the buffer read here is refilled by the next step's stage
    }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = mt + wm + g + (v >= 2 ? 8 : 0);
            const int c = nt + wn + j * 8 + 2 * t + (v & 1);
            if (r < M && c < N) C[(int64_t)r * ldc + c] = alpha * ldexp(ldexp(acc[j][v], e[r]), f[c]);
        }
}

template <int S>
void launch_oz_gemm(Context* ctx, int n_tiles, size_t smem, const OzProd* prods, const OzTile* tiles,
                    const __nv_bfloat16* As, const __nv_bfloat16* Bs, const int* exps) {
    static bool attr = false;
    if (!attr) {
        BSM_CUDA(cudaFuncSetAttribute(k_oz_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        BSM_CUDA(cudaFuncSetAttribute(k_oz_gemm<S>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
        attr = true;
    }
    k_oz_gemm<S><<<n_tiles, kOzWarps * 32, smem, ctx->stream>>>(prods, tiles, As, Bs, exps);
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
        if (g.M == 0 || g.N == 0) continue;
        const int Kp = (g.K + kOzKStep - 1) / kOzKStep * kOzKStep;
        OzProd pd{g.C, g.M, g.N, Kp, g.ldc, g.alpha, a_tot, b_tot, ex_tot, ex_tot + g.M};
        a_tot += (int64_t)S * g.M * Kp;
        b_tot += (int64_t)S * g.N * Kp;
        ex_tot += g.M + g.N;
        for (int m0 = 0; m0 < g.M; m0 += kOzTile)
            for (int n0 = 0; n0 < g.N; n0 += kOzTile) tiles.push_back({(int)prods.size(), m0, n0});
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
    const size_t smem = sizeof(__nv_bfloat16) * 2 * (size_t)kOzStage;
    const int nt = (int)tiles.size();
    switch (S) {
        case 1: launch_oz_gemm<1>(ctx, nt, smem, d_prods, d_tiles, As, Bs, exps); break;
        case 2: launch_oz_gemm<2>(ctx, nt, smem, d_prods, d_tiles, As, Bs, exps); break;
        case 3: launch_oz_gemm<3>(ctx, nt, smem, d_prods, d_tiles, As, Bs, exps); break;
        case 4: launch_oz_gemm<4>(ctx, nt, smem, d_prods, d_tiles, As, Bs, exps); break;
        case 5: launch_oz_gemm<5>(ctx, nt, smem, d_prods, d_tiles, As, Bs, exps); break;
        case 6: launch_oz_gemm<6>(ctx, nt, smem, d_prods, d_tiles, As, Bs, exps); break;
        case 7: launch_oz_gemm<7>(ctx, nt, smem, d_prods, d_tiles, As, Bs, exps); break;
        default: launch_oz_gemm<8>(ctx, nt, smem, d_prods, d_tiles, As, Bs, exps); break;
    }
    launched(ctx);
    ctx->flops += fl;
}

void launch_gemm_ozaki(Context* ctx, int M, int N, int K, const double* A, int lda, const double* B, int ldb,
                       double* C, int ldc, int S, double alpha) {
    launch_gemm_ozaki_group(ctx, {OzGemm{A, B, C, M, N, K, lda, ldb, ldc, alpha}}, S);
}

}  // namespace bsm
