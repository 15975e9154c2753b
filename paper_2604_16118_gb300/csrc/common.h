// Internal structures of the block-sparse MPS library (host side).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/bsmps.h"

namespace bsm {

struct Error : public std::runtime_error {
    bsmps_status code;
    Error(bsmps_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define BSM_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            throw ::bsm::Error(e_ == cudaErrorMemoryAllocation ? BSMPS_ERR_OOM            \
                                                               : BSMPS_ERR_CUDA,          \
                               std::string(#call) + ": " + cudaGetErrorString(e_));       \
        }                                                                                 \
    } while (0)

#define BSM_REQUIRE(cond, code, msg)                              \
    do {                                                          \
        if (!(cond)) throw ::bsm::Error((code), (msg));           \
    } while (0)

struct Charge {
    int q0 = 0, q1 = 0;
    bool operator<(const Charge& o) const { return q0 != o.q0 ? q0 < o.q0 : q1 < o.q1; }
    bool operator==(const Charge& o) const { return q0 == o.q0 && q1 == o.q1; }
    bool operator!=(const Charge& o) const { return !(*this == o); }
    Charge operator+(const Charge& o) const { return {q0 + o.q0, q1 + o.q1}; }
    Charge operator-(const Charge& o) const { return {q0 - o.q0, q1 - o.q1}; }
};

inline Charge site_delta(int species, int sigma) {
    return species == 0 ? Charge{sigma, 0} : Charge{0, sigma};
}

// Sectors of one bond, ascending by charge.
struct Bond {
    std::vector<Charge> q;
    std::vector<int> dim;
    int find(const Charge& c) const;   // index or -1
    int total() const;
};

// One dense block of a core: left sector index li (bond t), right sector ri
// (bond t+1), occupation sigma; row-major rows x cols at offset off in the core.
struct Block {
    int li, ri, sigma, rows, cols;
    int64_t off;
};

struct Layout {
    int K = 0;
    std::vector<int> species;          // per site
    Charge target;
    std::vector<Bond> bonds;           // K+1
    std::vector<std::vector<Block>> blocks;   // per site, layout order
    std::vector<int64_t> core_size;    // per site (entries)
    void rebuild_blocks();             // from bonds
    int64_t total() const;
    int block_index(int t, int li, int sigma) const;  // -1 if absent
    // Represented vectors: the dimension of the last bond (1 for a plain MPS,
    // D for a joint block MPS whose column index follows the last site, Sec. 6.2).
    int columns() const { return bonds.empty() || bonds.back().q.empty() ? 1 : bonds.back().dim[0]; }
};

std::vector<int> species_of(int n_orb, int spin);
std::vector<std::vector<Charge>> valid_sectors(const std::vector<int>& species, Charge target);
// D > 1: a joint block MPS of D columns (right counts times D, last bond D wide).
Layout default_layout(const std::vector<int>& species, Charge target, int r_max, int D = 1);
Layout e1_layout(const std::vector<int>& species, Charge target);
// Joint block MPS of the unit vectors given by D occupation strings (occ: D x K
// bytes, row i = vector i): every vector owns one index per inner bond, in
// order of i; values (one 1 per vector and site) written to *values.
Layout determinant_layout(const std::vector<int>& species, Charge target, const unsigned char* occ, int D,
                          std::vector<double>* values);
void check_layout(const Layout& L);

// MPO: per site a sorted list of entries; per bond channel charges.
struct MpoEntry {
    int a, b, so, si;
    double w;
};

struct Mpo {
    int K = 0;
    std::vector<int> species;
    std::vector<std::vector<Charge>> charges;     // per bond, per channel
    std::vector<std::vector<MpoEntry>> entries;   // per site, sorted (a, b, so, si)
    int shift_entry[2] = {-1, -1};                // site-0 entries (I->F, s, s)
    int ident_last = -1;                          // identity channel I on bond K-1
    int bond_dim(int b) const { return (int)charges[b].size(); }
};

Mpo build_mpo(int n_orb, const double* h, const double* eri, int spin, int n_particles,
              double gamma, double compress_tol);

struct Context;

// Device MPS: one device buffer per core (row-major blocks in layout order).
struct Mps {
    Context* ctx = nullptr;
    Layout lay;
    std::vector<double*> core;   // device pointers (nullptr when the core is empty)
    bool owns_cores = true;      // false: the cores belong to a recorded graph's arena
    ~Mps();
};

// Memory of a recorded CUDA graph (bsmps_plan): while a context records, its
// device requests are carved from dev (never recycled, so every buffer keeps
// the address the graph's launches were captured with) and its task lists are
// staged in host (pinned, read by the graph's copy nodes at every launch).
struct PlanArena {
    char* dev = nullptr;
    size_t dev_cap = 0, dev_used = 0;
    unsigned char* host = nullptr;
    size_t host_cap = 0, host_used = 0;
    bool owns(const void* p) const { return p >= dev && p < dev + dev_cap; }
};

// Per-launch record of the optional profiler (events resolved on query).
struct ProfRec {
    int kind;
    double flops, bytes;
    cudaEvent_t e0, e1;
};

// KK_APPLY: the contraction stage of the zip-up MPO application (grouped GEMM);
// KK_APPLY_QR: the zip-up's own factorisation launches (zeroing, gathers, QR)
enum KernelKind { KK_COPY = 0, KK_GEMM = 1, KK_QR = 2, KK_SVD = 3, KK_SUMSQ = 4, KK_APPLY = 5, KK_APPLY_QR = 6,
                  KK_MLP = 7, KK_COUNT = 8 };

struct Context {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    int64_t launches = 0;
    int64_t alloc_calls = 0;         // requests served by alloc()
    size_t alloc_bytes = 0;          // bytes requested from alloc() (256-byte granules), running total
    size_t upload_bytes = 0;         // bytes staged by upload_raw() (256-byte granules), running total
    PlanArena* rec = nullptr;        // set while a graph is being recorded
    // A second stream for independent launches of one sweep step: work forked
    // onto it after an event on `stream`, joined back by an event before the
    // step's results are read; every buffer it touches is allocated before the
    // fork and released after the join (the allocator orders reuse by `stream`).
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    bool side_open = false;          // forked and not yet joined
    cudaStream_t fork_side() {
        if (!side) {
            BSM_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
            BSM_CUDA(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
            BSM_CUDA(cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming));
        }
        BSM_CUDA(cudaEventRecord(fork_ev, stream));
        BSM_CUDA(cudaStreamWaitEvent(side, fork_ev, 0));
        side_open = true;
        return side;
    }
    void join_side() {
        BSM_CUDA(cudaEventRecord(join_ev, side));
        BSM_CUDA(cudaStreamWaitEvent(stream, join_ev, 0));
        side_open = false;
    }
    double flops = 0.0;              // algorithmic FP64 flops issued (running total)
    bool profiling = false;
    int gemm_emulation_log2 = 0;     // block products >= 2^this flops on the tensor cores (0: never)
    int apply_precision = BSMPS_PREC_FP64;   // arithmetic of the zip-up contraction stage
    bool autotune = true;                    // autotune the FP64 zip-up contraction (launch_gemm)
    int jacobi_precond_min = 48;             // cluster Jacobi from this k on starts from an FP32 Jacobi (0: never)
    std::map<int64_t, int> gemm_tuned;       // size class -> chosen split between the two GEMM kernels
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> event_pool;
    cudaEvent_t take_event();
    void prof_begin(cudaEvent_t* e0);
    void prof_end(int kind, double flops, double bytes, cudaEvent_t e0);
    // pinned staging ring for task uploads (a copy from pageable memory can
    // make the host wait for the stream): two halves, filled in turn; an event
    // recorded when a half is left gates its reuse
    static constexpr size_t kRingBytes = 8u << 20;
    unsigned char* ring_host = nullptr;
    size_t ring_head = 0;
    int ring_half = 0;
    cudaEvent_t half_ev[2] = {nullptr, nullptr};
    bool half_pending[2] = {false, false};
    void* upload_raw(const void* src, size_t bytes);
    void release_ring();
    // Device memory: a caching sub-allocator over the stream-ordered pool.
    // Blocks are rounded up to a power of two and recycled on this context's
    // stream; stream order makes a block freed after the work that uses it
    // safe for any later work, so alloc and free need no CUDA call once the
    // cache is warm.
    static constexpr int kMaxClass = 26;                 // 64 MiB; larger blocks bypass the cache
    static constexpr size_t kCacheCap = size_t(4) << 30;
    std::vector<std::vector<void*>> free_blocks = std::vector<std::vector<void*>>(kMaxClass + 1);
    std::unordered_map<void*, int> block_class;
    size_t cached_bytes = 0;
    void* alloc(size_t bytes);
    void free(void* p);
    void release_cache();
    template <class T>
    T* upload(const std::vector<T>& v) {
        if (v.empty()) return nullptr;
        return (T*)upload_raw(v.data(), v.size() * sizeof(T));
    }
    // Device error word of bounded grid-wide waits in kernels whose results the
    // host does not read back at once; checked (and cleared) by sync().
    int* dev_err = nullptr;
    bool dev_err_armed = false;
    int* err_word() {
        if (!dev_err) {
            BSM_CUDA(cudaMalloc(&dev_err, sizeof(int)));
            BSM_CUDA(cudaMemsetAsync(dev_err, 0, sizeof(int), stream));
        }
        dev_err_armed = true;
        return dev_err;
    }
    void sync() {
        BSM_CUDA(cudaStreamSynchronize(stream));
        half_pending[0] = half_pending[1] = false;   // every staged copy has completed
        if (dev_err_armed) {
            dev_err_armed = false;
            int h = 0;
            BSM_CUDA(cudaMemcpy(&h, dev_err, sizeof(int), cudaMemcpyDeviceToHost));
            if (h) {
                BSM_CUDA(cudaMemset(dev_err, 0, sizeof(int)));
                throw Error(BSMPS_ERR_TIMEOUT, "a grid-wide wait of a factorisation gave up");
            }
        }
    }
};

// Joins the context's second stream back into its stream when the scope ends
// with the fork still open (an error unwinding between fork and join): work
// released after this point in stream order then also waits for the side
// stream's kernels.  Constructed with the context only by the scope that forks
// (nullptr otherwise, so that a nested scope never joins an outer fork); a
// no-op after an explicit join_side().
struct SideJoin {
    Context* ctx;
    explicit SideJoin(Context* c) : ctx(c) {}
    ~SideJoin() {
        if (ctx && ctx->side_open) {
            cudaEventRecord(ctx->join_ev, ctx->side);
            cudaStreamWaitEvent(ctx->stream, ctx->join_ev, 0);
            ctx->side_open = false;
        }
    }
};

// RAII bracket of one launch for the optional profiler.
struct ProfScope {
    Context* ctx;
    int kind;
    double flops, bytes;
    cudaEvent_t e0 = nullptr;
    ProfScope(Context* c, int k, double f, double b) : ctx(c), kind(k), flops(f), bytes(b) {
        if (ctx->profiling) ctx->prof_begin(&e0);
    }
    void done() {
        if (ctx->profiling) ctx->prof_end(kind, flops, bytes, e0);
    }
};

// RAII holder for temporary device allocations of one operation.
struct Scratch {
    Context* ctx;
    std::vector<void*> ptrs;
    explicit Scratch(Context* c) : ctx(c) {}
    ~Scratch() {
        for (void* p : ptrs) ctx->free(p);
    }
    template <class T>
    T* up(const std::vector<T>& v) {
        T* p = ctx->upload(v);
        if (p) ptrs.push_back(p);
        return p;
    }
    double* dbl(size_t n) {
        if (n == 0) return nullptr;
        double* p = (double*)ctx->alloc(n * sizeof(double));
        ptrs.push_back(p);
        return p;
    }
};

Mps* new_mps(Context* ctx, const Layout& L, bool zero);   // allocates cores

}  // namespace bsm
