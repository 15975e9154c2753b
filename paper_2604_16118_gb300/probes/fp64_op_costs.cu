// Cost of dependent FP64 operations on one warp, with all 32 lanes active and
// with one lane active, and with 4 and 8 warps per CTA (one CTA).  A
// standalone program, not part of the library:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_op_costs fp64_op_costs.cu && ./fp64_op_costs
// It prints clock cycles per operation of a dependent chain (4 x 256 ops).
#include <cstdio>
#include <cuda_runtime.h>

constexpr int kIters = 256;
__device__ double g_sink[1024];
__device__ long long g_cycles[64];

template <int OP>
__device__ __forceinline__ double step(double x, double a, double b) {
    if (OP == 0) return fma(x, a, b);
    if (OP == 1) return x + a;
    if (OP == 2) return x * a;
    if (OP == 3) return sqrt(x + b);
    if (OP == 4) return a / (x + b);
    if (OP == 5) return rsqrt(x + b);
    if (OP == 6) return x + __shfl_xor_sync(0xffffffffu, x, 1) * a;   // needs all lanes
    if (OP == 7) return (double)(float)x * a + b;                     // conversion round trip
    return x;
}

template <int OP>
__global__ void k_chain(int active_lanes, int slot) {
    double x = 1.0 + threadIdx.x * 1e-3, a = 0.999999, b = 1e-7;
    __syncwarp();
    const long long t0 = clock64();
    if ((int)(threadIdx.x & 31) < active_lanes) {
#pragma unroll 1
        for (int i = 0; i < kIters; ++i) {
            x = step<OP>(x, a, b);
            x = step<OP>(x, a, b);
            x = step<OP>(x, a, b);
            x = step<OP>(x, a, b);
        }
    }
    __syncwarp();
    const long long t1 = clock64();
    g_sink[threadIdx.x] = x;
    if (threadIdx.x == 0) g_cycles[slot] = t1 - t0;
}

__global__ void k_f32_chain(int slot) {
    float x = 1.0f + threadIdx.x, a = 0.999f, b = 1e-3f;
    const long long t0 = clock64();
#pragma unroll 1
    for (int i = 0; i < kIters; ++i) {
        x = fmaf(x, a, b);
        x = fmaf(x, a, b);
        x = fmaf(x, a, b);
        x = fmaf(x, a, b);
    }
    const long long t1 = clock64();
    g_sink[threadIdx.x] = x;
    if (threadIdx.x == 0) g_cycles[slot] = t1 - t0;
}

int main() {
    const char* names[] = {"dfma", "dadd", "dmul", "dsqrt", "ddiv", "drsqrt", "shfl+dfma", "cvt f64-f32-f64"};
    void (*ks[8])(int, int) = {k_chain<0>, k_chain<1>, k_chain<2>, k_chain<3>,
                               k_chain<4>, k_chain<5>, k_chain<6>, k_chain<7>};
    for (int op = 0; op < 8; ++op)
        for (int cfg = 0; cfg < 4; ++cfg) {
            if (op == 6 && cfg == 1) continue;   // a full-mask shuffle needs every lane
            const int lanes = cfg == 1 ? 1 : 32, warps = cfg == 2 ? 4 : (cfg == 3 ? 8 : 1);
            for (int rep = 0; rep < 2; ++rep) ks[op]<<<1, 32 * warps>>>(lanes, op * 4 + cfg);
        }
    for (int rep = 0; rep < 2; ++rep) k_f32_chain<<<1, 32>>>(40);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        printf("error: %s\n", cudaGetErrorString(e));
        return 1;
    }
    long long h[64] = {0};
    cudaMemcpyFromSymbol(h, g_cycles, sizeof(h));
    const double n = 4.0 * kIters;
    printf("cycles per dependent op: 1 warp/32 lanes, 1 warp/1 lane, 4 warps, 8 warps\n");
    for (int op = 0; op < 8; ++op)
        printf("%-16s %8.1f %8.1f %8.1f %8.1f\n", names[op], h[op * 4] / n, h[op * 4 + 1] / n, h[op * 4 + 2] / n,
               h[op * 4 + 3] / n);
    printf("f32 fma chain    %8.1f\n", h[40] / n);
    return 0;
}
