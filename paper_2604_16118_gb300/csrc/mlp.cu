// Small multilayer perceptron for the learned preconditioner controller:
// ReLU hidden layers, linear output, BF16 weights for the forward and backward
// products (rounded from FP32 master weights after every update), FP32
// accumulation, mean-squared-error loss and Adam updates of the masters.
#include <cuda_bf16.h>

#include <cmath>
#include <functional>
#include <vector>

#include "ops.h"

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

// Y[b, o] = act( sum_i X[b, i] W[o, i] + bias[o] ), W bf16 (out x in), FP32 accumulate.
__global__ void k_mlp_fwd(const float* __restrict__ X, const __nv_bfloat16* __restrict__ W,
                          const __nv_bfloat16* __restrict__ bias, float* __restrict__ Y, int B, int in, int out,
                          int relu) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * out) return;
    const int b = (int)(e / out), o = (int)(e % out);
    float acc = __bfloat162float(bias[o]);
    const float* x = X + (int64_t)b * in;
    const __nv_bfloat16* w = W + (int64_t)o * in;
    for (int i = 0; i < in; ++i) acc = fmaf(x[i], __bfloat162float(w[i]), acc);
    Y[e] = relu ? fmaxf(acc, 0.0f) : acc;
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

// dW[o, i] = sum_b dY[b, o] X[b, i];  db[o] = sum_b dY[b, o]
__global__ void k_mlp_wgrad(const float* __restrict__ dY, const float* __restrict__ X, float* __restrict__ dW,
                            float* __restrict__ db, int B, int in, int out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)out * (in + 1)) return;
    const int o = (int)(e / (in + 1)), i = (int)(e % (in + 1));
    float acc = 0.0f;
    if (i < in) {
        for (int b = 0; b < B; ++b) acc = fmaf(dY[(int64_t)b * out + o], X[(int64_t)b * in + i], acc);
        dW[(int64_t)o * in + i] = acc;
    } else {
        for (int b = 0; b < B; ++b) acc += dY[(int64_t)b * out + o];
        db[o] = acc;
    }
}

// dX[b, i] = (sum_o dY[b, o] W[o, i]) * [X[b, i] > 0]   (X is the ReLU output feeding the layer)
__global__ void k_mlp_xgrad(const float* __restrict__ dY, const __nv_bfloat16* __restrict__ W,
                            const float* __restrict__ Xact, float* __restrict__ dX, int B, int in, int out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * in) return;
    const int b = (int)(e / in), i = (int)(e % in);
    float acc = 0.0f;
    for (int o = 0; o < out; ++o) acc = fmaf(dY[(int64_t)b * out + o], __bfloat162float(W[(int64_t)o * in + i]), acc);
    dX[e] = Xact[e] > 0.0f ? acc : 0.0f;
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

// forward pass of a batch already on the device; returns the activations
Acts forward(Context* ctx, bsmps_mlp_s* net, const float* x_dev, int B, Scratch& s) {
    const int nl = (int)net->widths.size() - 1;
    Acts a;
    a.h.push_back(const_cast<float*>(x_dev));
    for (int l = 0; l < nl; ++l) {
        const int in = net->widths[l], out = net->widths[l + 1];
        float* y = (float*)s.dbl(((size_t)B * out + 1) / 2 + 1);
        k_mlp_fwd<<<grid((int64_t)B * out), kT, 0, ctx->stream>>>(a.h.back(), net->wbf + net->w_off[l],
                                                                   net->wbf + net->b_off[l], y, B, in, out,
                                                                   l + 1 < nl ? 1 : 0);
        done(ctx);
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
        k_mlp_wgrad<<<grid((int64_t)out * (in + 1)), kT, 0, ctx->stream>>>(dY, a.h[l], net->grad + net->w_off[l],
                                                                           net->grad + net->b_off[l], B, in, out);
        done(ctx);
        if (l > 0) {
            float* dX = (float*)s.dbl(((size_t)B * in) / 2 + 1);
            k_mlp_xgrad<<<grid((int64_t)B * in), kT, 0, ctx->stream>>>(dY, net->wbf + net->w_off[l], a.h[l], dX, B,
                                                                      in, out);
            done(ctx);
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
