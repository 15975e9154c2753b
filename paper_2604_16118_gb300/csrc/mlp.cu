// Small multilayer perceptron for the learned preconditioner controller:
// ReLU hidden layers, linear output, BF16 weights (rounded from FP32 master
// weights after every update), mean-squared-error loss and Adam updates of the
// masters.  Every product of the forward and backward passes runs on the
// 5th-generation tensor cores (tcgen05.mma kind::tf32, FP32 accumulation in
// tensor memory): the BF16 weights are exact in TF32, and the activations and
// back-propagated errors enter the products rounded to TF32 (nearest, ties
// away from zero).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <vector>

#include "ops.h"
#include "tc_common.cuh"

struct bsmps_mlp_s {
    bsm::Context* ctx;
    std::vector<int> widths;          // n_layers + 1
    std::vector<int64_t> w_off, b_off; // offsets into the flat parameter vector
    int64_t n_params = 0;
    float* master = nullptr;          // FP32 parameters (device)
    __nv_bfloat16* wbf = nullptr;     // BF16 copy of the parameters (device)
    float* m1 = nullptr;              // Adam first moment
    float* m2 = nullptr;              // Adam second moment
    float* grad = nullptr;
    int64_t step = 0;
};

namespace bsm {
namespace {

constexpr int kT = 256;

// One product of the network on the tensor cores:
//     C(m, n) = epi( sum_k a(m, k) b(n, k) ),   m < M, n < N, k < K,
// a and b read through element strides from FP32 or BF16 arrays and rounded to
// TF32; epi adds bias[n] (BF16) and applies ReLU, or keeps the entry only where
// mask(m, n) > 0 (the derivative of the ReLU that produced mask), else nothing.
struct MlpGemm {
    const void* A;
    int64_t sam, sak;
    int a_bf16;
    const void* B;
    int64_t sbn, sbk;
    int b_bf16;
    float* C;
    int64_t scm, scn;
    const __nv_bfloat16* bias;
    const float* mask;
    int relu;
    int M, N, K;
};

constexpr int kMlpM = 128;         // rows of a tile (the M of one tcgen05.mma)
constexpr int kMlpN = 64;          // columns of a tile (its N, and the tensor-memory columns)
constexpr int kMlpK = 32;          // k values per staged chunk (4 MMAs of K = 8)
constexpr int kMlpThreads = 128;   // warp w reads tensor-memory lanes 32 w .. 32 w + 31
constexpr uint32_t kMlpIdesc = tc::idesc_tf32(kMlpM, kMlpN);

__device__ __forceinline__ float mlp_load(const void* p, int bf16, int64_t i) {
    return bf16 ? __bfloat162float(((const __nv_bfloat16*)p)[i]) : ((const float*)p)[i];
}

// One CTA per 128 x 64 output tile and k range (blockIdx.z of gridDim.z, each
// a multiple of 32 long): 4 warps stage 32-wide k chunks of a and b in the
// canonical K-major layout (the index order follows whichever of the two
// strides is 1, so the loads coalesce) into two buffers, so that staging chunk
// i + 1 overlaps the MMAs of chunk i; one thread issues the MMAs and commits
// them to the buffer's mbarrier (bounded waits; a CTA that gives up sets *err,
// waits boundedly for its MMAs and frees its tensor memory).  With one k range
// the epilogue (tcgen05.ld) applies bias / ReLU / mask and stores C; with
// several, every CTA stores its raw tile to part[z] and k_mlp_reduce sums the
// ranges in order and applies the epilogue.
__global__ void __launch_bounds__(kMlpThreads) k_mlp_gemm_tc(const MlpGemm g, int k_len, float* part, int* err) {
    extern __shared__ __align__(1024) unsigned char mlp_smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int gave_up;
    unsigned char* base = (unsigned char*)(((uintptr_t)mlp_smem + 1023) & ~(uintptr_t)1023);
    constexpr int kBuf = (kMlpM + kMlpN) * kMlpK * 4;
    const int m0 = blockIdx.x * kMlpM, n0 = blockIdx.y * kMlpN;
    const int kb = blockIdx.z * k_len, ke = min(g.K, kb + k_len);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = tc::smem_addr(&bar[0]), bar1 = tc::smem_addr(&bar[1]);
    if (threadIdx.x == 0) {
        gave_up = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::smem_addr(&tmem_slot)),
                     "r"(kMlpN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    int n_chunks = 0;   // chunks committed; chunk i used buffer i & 1 and is commit i >> 1 of its mbarrier
    for (int k0 = kb; k0 < ke; k0 += kMlpK, ++n_chunks) {
        const int buf = n_chunks & 1;
        if (n_chunks >= 2) {
            // the MMAs of chunk n_chunks - 2 (the last user of this buffer) are done
            if (!tc::mbar_wait(buf ? bar1 : bar0, ((n_chunks - 2) >> 1) & 1)) {
                if (threadIdx.x == 0) atomicExch(&gave_up, 1);
            }
            __syncthreads();
            if (gave_up) break;
        }
        unsigned char* a_s = base + buf * kBuf;
        unsigned char* b_s = a_s + kMlpM * kMlpK * 4;
        for (int idx = threadIdx.x; idx < kMlpM * kMlpK; idx += kMlpThreads) {
            const int r = g.sak == 1 ? idx / kMlpK : idx % kMlpM;
            const int k = g.sak == 1 ? idx % kMlpK : idx / kMlpM;
            const int gm = m0 + r, gk = k0 + k;
            const float v = (gm < g.M && gk < ke) ? mlp_load(g.A, g.a_bf16, gm * g.sam + gk * g.sak) : 0.0f;
            *(uint32_t*)(a_s + tc::off(r, k)) = tc::tf32_bits(v);
        }
        for (int idx = threadIdx.x; idx < kMlpN * kMlpK; idx += kMlpThreads) {
            const int n = g.sbk == 1 ? idx / kMlpK : idx % kMlpN;
            const int k = g.sbk == 1 ? idx % kMlpK : idx / kMlpN;
            const int gn = n0 + n, gk = k0 + k;
            const float v = (gn < g.N && gk < ke) ? mlp_load(g.B, g.b_bf16, gn * g.sbn + gk * g.sbk) : 0.0f;
            *(uint32_t*)(b_s + tc::off(n, k)) = tc::tf32_bits(v);
        }
        // generic-proxy writes become visible to the tensor cores' (async) proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = tc::smem_addr(a_s), sb = tc::smem_addr(b_s);
            for (int kk = 0; kk < kMlpK / 8; ++kk) {
                const uint32_t step = (uint32_t)kk * 256u;   // two core matrices along k per MMA
                tc::mma_tf32(tmem, tc::desc(sa + step), tc::desc(sb + step), kMlpIdesc,
                             (n_chunks == 0 && kk == 0) ? 0u : 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             buf ? bar1 : bar0)
                         : "memory");
        }
    }
    // the last chunk's commit covers every earlier MMA of this thread
    const int last = n_chunks - 1;
    if (!gave_up && n_chunks > 0) {
        if (!tc::mbar_wait((last & 1) ? bar1 : bar0, (last >> 1) & 1)) {
            if (threadIdx.x == 0) atomicExch(&gave_up, 1);
        }
        __syncthreads();
        if (!gave_up) asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (!gave_up) {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < kMlpN; c0 += 16) {
            uint32_t v[16];
            if (n_chunks > 0) {
                tc::ld_32x32b_x16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0u;
            }
            if (row < g.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col >= g.N) continue;
                    float acc = __uint_as_float(v[j]);
                    if (part) {
                        part[((int64_t)blockIdx.z * g.M + row) * g.N + col] = acc;
                        continue;
                    }
                    if (g.bias) acc += __bfloat162float(g.bias[col]);
                    if (g.relu) acc = fmaxf(acc, 0.0f);
                    const int64_t ci = row * g.scm + col * g.scn;
                    if (g.mask && !(g.mask[ci] > 0.0f)) acc = 0.0f;
                    g.C[ci] = acc;
                }
            }
        }
    } else {
        if (threadIdx.x == 0) atomicExch(err, 1);
        // MMAs of this CTA may still be in flight: a bounded wait for the last
        // commit before the tensor memory they write is released
        if (n_chunks > 0) tc::mbar_wait((last & 1) ? bar1 : bar0, (last >> 1) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMlpN));
}

// C(m, n) = epi( sum_z part[z](m, n) ), the k ranges summed in order.
__global__ void k_mlp_reduce(const MlpGemm g, const float* __restrict__ part, int n_parts) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)g.M * g.N) return;
    const int m = (int)(e / g.N), n = (int)(e % g.N);
    float acc = 0.0f;
    for (int z = 0; z < n_parts; ++z) acc += part[(int64_t)z * g.M * g.N + e];
    if (g.bias) acc += __bfloat162float(g.bias[n]);
    if (g.relu) acc = fmaxf(acc, 0.0f);
    const int64_t ci = m * g.scm + n * g.scn;
    if (g.mask && !(g.mask[ci] > 0.0f)) acc = 0.0f;
    g.C[ci] = acc;
}

// dY of the loss 1/(B out) sum (Y - T)^2, and the per-element squared error.
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                      float* __restrict__ sq, int n, float scale) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float d = Y[e] - T[e];
    dY[e] = 2.0f * scale * d;
    sq[e] = d * d;
}

// db[o] = sum_b dY[b, o] (TF32-rounded dY, as the weight-gradient product reads it), one CTA per o.
__global__ void k_mlp_bgrad(const float* __restrict__ dY, float* __restrict__ db, int B, int out) {
    __shared__ float red[32];
    const int o = blockIdx.x;
    float acc = 0.0f;
    for (int b = threadIdx.x; b < B; b += blockDim.x)
        acc += __uint_as_float(tc::tf32_bits(dY[(int64_t)b * out + o]));
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
        if (threadIdx.x == 0) db[o] = acc;
    }
}

// Adam (beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on the FP32 masters, then the BF16 copy.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, __nv_bfloat16* __restrict__ pb, int64_t n, float lr, float c1,
                       float c2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gg = g[e];
    const float a = 0.9f * m1[e] + 0.1f * gg;
    const float v = 0.999f * m2[e] + 0.001f * gg * gg;
    m1[e] = a;
    m2[e] = v;
    const float q = p[e] - lr * (a / c1) / (sqrtf(v / c2) + 1e-8f);
    p[e] = q;
    pb[e] = __float2bfloat16_rn(q);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) pb[e] = __float2bfloat16_rn(p[e]);
}

unsigned grid(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

void done(Context* ctx) {
    ctx->launches++;
    BSM_CUDA(cudaGetLastError());
}

struct Acts {
    std::vector<float*> h;   // h[0] = input, h[l+1] = output of layer l
};

// One product: tiles of 128 x 64; the k range split over gridDim.z CTAs per
// tile (partials reduced in order by k_mlp_reduce) when the tiles alone would
// leave most SMs idle.
void launch_mlp_gemm(Context* ctx, const MlpGemm& g, Scratch& s) {
    if (g.M <= 0 || g.N <= 0) return;
    const int smem = 2 * (kMlpM + kMlpN) * kMlpK * 4 + 1024;   // two buffers, aligned to 1024 bytes
    static bool attr = false;
    if (!attr) {
        BSM_CUDA(cudaFuncSetAttribute(k_mlp_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = true;
    }
    const int64_t tiles = (int64_t)((g.M + kMlpM - 1) / kMlpM) * ((g.N + kMlpN - 1) / kMlpN);
    const int chunks = (g.K + kMlpK - 1) / kMlpK;
    int splits = 1;
    while (tiles * splits < 2 * 148 && chunks / (splits * 2) >= 4) splits *= 2;
    const int k_len = ((chunks + splits - 1) / splits) * kMlpK;
    splits = std::max(1, (g.K + k_len - 1) / k_len);
    float* part = splits > 1 ? (float*)s.dbl(((size_t)splits * g.M * g.N + 1) / 2) : nullptr;
    const dim3 grid_tc((unsigned)((g.M + kMlpM - 1) / kMlpM), (unsigned)((g.N + kMlpN - 1) / kMlpN),
                       (unsigned)splits);
    const double fl = 2.0 * g.M * (double)g.N * g.K;
    const double by = 4.0 * ((double)g.M * g.K + (double)g.N * g.K + (double)g.M * g.N);
    ProfScope ps(ctx, KK_MLP, fl, by);
    k_mlp_gemm_tc<<<grid_tc, kMlpThreads, smem, ctx->stream>>>(g, k_len, part, ctx->err_word());
    done(ctx);
    if (part) {
        k_mlp_reduce<<<grid((int64_t)g.M * g.N), kT, 0, ctx->stream>>>(g, part, splits);
        done(ctx);
    }
    ps.done();
}

// forward pass of a batch already on the device; returns the activations
Acts forward(Context* ctx, bsmps_mlp_s* net, const float* x_dev, int B, Scratch& s) {
    const int nl = (int)net->widths.size() - 1;
    Acts a;
    a.h.push_back(const_cast<float*>(x_dev));
    for (int l = 0; l < nl; ++l) {
        const int in = net->widths[l], out = net->widths[l + 1];
        float* y = (float*)s.dbl(((size_t)B * out + 1) / 2 + 1);
        // Y[b, o] = sum_i X[b, i] W[o, i] + bias[o]: a = X (B x in), b(n = o, k = i) = W[o, i]
        MlpGemm g{a.h.back(), in, 1, 0, net->wbf + net->w_off[l], in, 1, 1, y, out, 1,
                  net->wbf + net->b_off[l], nullptr, l + 1 < nl ? 1 : 0, B, out, in};
        launch_mlp_gemm(ctx, g, s);
        a.h.push_back(y);
    }
    return a;
}

// loss and gradient into net->grad (device)
float loss_grad(Context* ctx, bsmps_mlp_s* net, const float* x_host, const float* t_host, int B) {
    const int nl = (int)net->widths.size() - 1;
    const int in0 = net->widths[0], outL = net->widths[nl];
    Scratch s(ctx);
    std::vector<float> xv(x_host, x_host + (size_t)B * in0), tv(t_host, t_host + (size_t)B * outL);
    float* xd = s.up(xv);
    float* td = s.up(tv);
    Acts a = forward(ctx, net, xd, B, s);
    const int n = B * outL;
    float* dY = (float*)s.dbl((size_t)n / 2 + 1);
    float* sq = (float*)s.dbl((size_t)n / 2 + 1);
    k_mse<<<grid(n), kT, 0, ctx->stream>>>(a.h.back(), td, dY, sq, n, 1.0f / (float)n);
    done(ctx);
    for (int l = nl - 1; l >= 0; --l) {
        const int in = net->widths[l], out = net->widths[l + 1];
        // dW[o, i] = sum_b dY[b, o] X[b, i]: a(m = o, k = b) = dY[b, o], b(n = i, k = b) = X[b, i]
        MlpGemm gw{dY, 1, out, 0, a.h[l], 1, in, 0, net->grad + net->w_off[l], in, 1, nullptr, nullptr, 0,
                   out, in, B};
        launch_mlp_gemm(ctx, gw, s);
        k_mlp_bgrad<<<(unsigned)out, kT, 0, ctx->stream>>>(dY, net->grad + net->b_off[l], B, out);
        done(ctx);
        if (l > 0) {
            // dX[b, i] = (sum_o dY[b, o] W[o, i]) [X[b, i] > 0]: a = dY (B x out), b(n = i, k = o) = W[o, i]
            float* dX = (float*)s.dbl(((size_t)B * in) / 2 + 1);
            MlpGemm gx{dY, out, 1, 0, net->wbf + net->w_off[l], 1, in, 1, dX, in, 1, nullptr, a.h[l], 0, B, in, out};
            launch_mlp_gemm(ctx, gx, s);
            dY = dX;
        }
    }
    std::vector<float> sh((size_t)n);
    BSM_CUDA(cudaMemcpyAsync(sh.data(), sq, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->sync();
    double acc = 0.0;
    for (float v : sh) acc += v;
    return (float)(acc / n);
}

}  // namespace
}  // namespace bsm

namespace {
bsmps_status mlp_guard(bsm::Context* ctx, const std::function<void()>& f) {
    try {
        f();
        return BSMPS_OK;
    } catch (const bsm::Error& e) {
        if (ctx) ctx->last_error = e.what();
        return e.code;
    } catch (const std::exception& e) {
        if (ctx) ctx->last_error = e.what();
        return BSMPS_ERR_INVALID_ARG;
    }
}

bsm::Context* ctx_of(bsmps_mlp m) {
    if (!m || !m->ctx) throw bsm::Error(BSMPS_ERR_INVALID_ARG, "null MLP handle");
    BSM_CUDA(cudaSetDevice(m->ctx->device));
    (void)cudaGetLastError();   // a stale error left by another caller is not this call's
    return m->ctx;
}
}  // namespace

namespace bsm {
Context* context_of(bsmps_ctx ctx);
}

extern "C" {

bsmps_status bsmps_mlp_create(bsmps_ctx c, int n_layers, const int* widths, const float* params, int64_t n_params,
                              bsmps_mlp* out) {
    bsm::Context* ctx = nullptr;
    bsmps_status st = mlp_guard(nullptr, [&] { ctx = bsm::context_of(c); });
    if (st != BSMPS_OK) return st;
    bsmps_mlp_s* net = nullptr;
    st = mlp_guard(ctx, [&] {
        BSM_REQUIRE(n_layers >= 1 && n_layers <= 16 && widths && params && out, BSMPS_ERR_INVALID_ARG,
                    "mlp_create: 1..16 layers, widths, params and out required");
        net = new bsmps_mlp_s;
        net->ctx = ctx;
        int64_t off = 0;
        for (int l = 0; l <= n_layers; ++l) {
            BSM_REQUIRE(widths[l] > 0 && widths[l] <= 4096, BSMPS_ERR_INVALID_ARG, "mlp_create: width out of range");
            net->widths.push_back(widths[l]);
        }
        for (int l = 0; l < n_layers; ++l) {
            net->w_off.push_back(off);
            off += (int64_t)widths[l] * widths[l + 1];
            net->b_off.push_back(off);
            off += widths[l + 1];
        }
        net->n_params = off;
        BSM_REQUIRE(n_params == off, BSMPS_ERR_INVALID_ARG, "mlp_create: params must hold every weight and bias");
        BSM_CUDA(cudaMalloc(&net->master, sizeof(float) * off));
        BSM_CUDA(cudaMalloc(&net->wbf, sizeof(__nv_bfloat16) * off));
        BSM_CUDA(cudaMalloc(&net->m1, sizeof(float) * off));
        BSM_CUDA(cudaMalloc(&net->m2, sizeof(float) * off));
        BSM_CUDA(cudaMalloc(&net->grad, sizeof(float) * off));
        BSM_CUDA(cudaMemcpy(net->master, params, sizeof(float) * off, cudaMemcpyHostToDevice));
        BSM_CUDA(cudaMemset(net->m1, 0, sizeof(float) * off));
        BSM_CUDA(cudaMemset(net->m2, 0, sizeof(float) * off));
        bsm::k_to_bf16<<<bsm::grid(off), bsm::kT, 0, ctx->stream>>>(net->master, net->wbf, off);
        bsm::done(ctx);
        ctx->sync();
        *out = net;
        net = nullptr;
    });
    if (net) {
        cudaFree(net->master);
        cudaFree(net->wbf);
        cudaFree(net->m1);
        cudaFree(net->m2);
        cudaFree(net->grad);
        delete net;
    }
    return st;
}

bsmps_status bsmps_mlp_num_params(bsmps_mlp m, int64_t* n) {
    if (!m || !n) return BSMPS_ERR_INVALID_ARG;
    *n = m->n_params;
    return BSMPS_OK;
}

bsmps_status bsmps_mlp_get_params(bsmps_mlp m, float* params) {
    return mlp_guard(m ? m->ctx : nullptr, [&] {
        bsm::Context* ctx = ctx_of(m);
        BSM_REQUIRE(params, BSMPS_ERR_INVALID_ARG, "null out");
        BSM_CUDA(cudaMemcpyAsync(params, m->master, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost, ctx->stream));
        ctx->sync();
    });
}

bsmps_status bsmps_mlp_forward(bsmps_mlp m, const float* x, int B, float* y) {
    return mlp_guard(m ? m->ctx : nullptr, [&] {
        bsm::Context* ctx = ctx_of(m);
        BSM_REQUIRE(x && y && B > 0, BSMPS_ERR_INVALID_ARG, "mlp_forward: x, y and B > 0 required");
        bsm::Scratch s(ctx);
        std::vector<float> xv(x, x + (size_t)B * m->widths[0]);
        float* xd = s.up(xv);
        bsm::Acts a = bsm::forward(ctx, m, xd, B, s);
        const int out = m->widths.back();
        BSM_CUDA(cudaMemcpyAsync(y, a.h.back(), sizeof(float) * B * out, cudaMemcpyDeviceToHost, ctx->stream));
        ctx->sync();
    });
}

bsmps_status bsmps_mlp_loss_grad(bsmps_mlp m, const float* x, const float* t, int B, float* loss, float* grad) {
    return mlp_guard(m ? m->ctx : nullptr, [&] {
        bsm::Context* ctx = ctx_of(m);
        BSM_REQUIRE(x && t && B > 0, BSMPS_ERR_INVALID_ARG, "mlp_loss_grad: x, t and B > 0 required");
        const float l = bsm::loss_grad(ctx, m, x, t, B);
        if (loss) *loss = l;
        if (grad) {
            BSM_CUDA(cudaMemcpyAsync(grad, m->grad, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost, ctx->stream));
            ctx->sync();
        }
    });
}

bsmps_status bsmps_mlp_train_step(bsmps_mlp m, const float* x, const float* t, int B, float lr, float* loss) {
    return mlp_guard(m ? m->ctx : nullptr, [&] {
        bsm::Context* ctx = ctx_of(m);
        BSM_REQUIRE(x && t && B > 0 && lr > 0.0f, BSMPS_ERR_INVALID_ARG, "mlp_train_step: bad argument");
        const float l = bsm::loss_grad(ctx, m, x, t, B);
        m->step += 1;
        const float c1 = 1.0f - std::pow(0.9f, (float)m->step);
        const float c2 = 1.0f - std::pow(0.999f, (float)m->step);
        bsm::k_adam<<<bsm::grid(m->n_params), bsm::kT, 0, ctx->stream>>>(m->master, m->grad, m->m1, m->m2, m->wbf,
                                                                          m->n_params, lr, c1, c2);
        bsm::done(ctx);
        if (loss) *loss = l;
    });
}

bsmps_status bsmps_mlp_destroy(bsmps_mlp m) {
    if (!m) return BSMPS_ERR_INVALID_ARG;
    cudaSetDevice(m->ctx->device);
    cudaFree(m->master);
    cudaFree(m->wbf);
    cudaFree(m->m1);
    cudaFree(m->m2);
    cudaFree(m->grad);
    delete m;
    return BSMPS_OK;
}

}  // extern "C"
