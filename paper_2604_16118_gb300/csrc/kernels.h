// Device kernels of the block-sparse MPS library and their task descriptors.
#pragma once

#include <vector>

#include "common.h"

namespace bsm {

// dst(i, j) (+)= f * src(i, j) for a rows x cols block; each side row-major
// (element (i,j) at i*ld + j) or column-major (at j*ld + i).
struct CopyTask {
    const double* src;
    double* dst;
    int rows, cols;
    int src_ld, dst_ld;
    int src_cm, dst_cm;
    int accumulate;
    double f;
};

// One output C (M x N, row-major, ldc) = beta*C + sum over its contributions
// alpha * op(A) * B with op(A) = A (M x K, row-major lda) or A^T (A stored
// K x M row-major lda); B is K x N row-major (ldb).
struct GemmOut {
    double* C;
    int M, N, ldc;
    int beg, end;       // contribution range
    double beta;
};

struct GemmIn {
    const double* A;
    const double* B;
    int K, lda, ldb;
    int transA;
    double alpha;
};

// Householder QR of a column-major M x N matrix A (destroyed): Q (M x k,
// column-major) and R (k x N, row-major), k = min(M, N), diag(R) >= 0.
struct QrTask {
    double* A;
    double* Q;
    double* R;
    double* tau;
    int M, N;
    int smem = 0;     // set by launch_qr
};

// SVD of an M x N matrix A, k = min(M, N), given in G: A column-major when
// M >= N ("tall"), A row-major (= A^T column-major) when M < N ("wide"); G is
// destroyed.  Householder QR of A (tall) or A^T (wide), one-sided Jacobi on the
// k x k triangular factor, then assembly.  Outputs: S (k, descending),
// US = U diag(S) (M x k, row-major), Vt (k x N, row-major); the largest-|.|
// entry of every row of Vt is positive.
struct SvdTask {
    double* G;
    double* V;        // unused (kept for layout compatibility)
    double* S;
    double* US;
    double* Vt;
    int M, N;
    int wide;
};

// One-sided Jacobi of the k x k matrix G (column-major, destroyed): V (k x k,
// column-major) accumulates the rotations, Sraw receives the column norms of
// the rotated G (unsorted).
struct JacTask {
    double* G;
    double* V;
    double* Sraw;
    int k;
    int smem;        // 1: iterate in shared memory (one CTA per matrix)
    int v_given = 0; // 1: V holds the starting columns (the cluster kernel rotates them
                     // instead of the identity); the other Jacobi kernels ignore it
};

// Jacobi of several large matrices in one cooperative launch: the disjoint
// column pairs of every round are spread over all warps of the grid, rounds are
// separated by bounded grid-wide waits (a timeout sets the context's device
// error word, raised at the next sync).  Returns false when no grid can be
// resident (the caller then runs one CTA per matrix).
bool launch_jacobi_grid(Context* ctx, const std::vector<JacTask>& tasks);
// Jacobi of matrices with k <= kClusterJacobiMax, one thread-block cluster of 16
// (else 8) CTAs per matrix in a block-cyclic ordering: every CTA rotates the
// pairs of the two column blocks it holds in its own shared memory, and the
// blocks move between the CTAs' shared memories at a cluster barrier per
// tournament step (csrc/jacobi_cluster.cu).  Returns false, with nothing
// launched, when such a cluster cannot be scheduled.
constexpr int kClusterJacobiMax = 336;
// Jacobi problems from this size on go to the cluster kernel: below it one SM's
// FP64 units suffice for the latency of a round.
constexpr int kClusterJacobiMin = 32;
bool launch_jacobi_cluster(Context* ctx, const std::vector<JacTask>& tasks);
// FP32 one-sided Jacobi of the same tasks as a preconditioner: reads G (FP64,
// unchanged), writes to V the accumulated FP32 rotations as FP64 (orthogonal to
// about 1e-6); Sraw unused.  Returns false, with nothing launched, when no
// cluster can be scheduled.
bool launch_jacobi_cluster_f32(Context* ctx, const std::vector<JacTask>& tasks);

// C (M x N) = alpha op(A) B, op(A) = A (M x K) or A^T (A stored K x M), B
// (K x N), all row-major FP64 on the device with leading dimensions, emulated by
// S (1..8) bf16 integer slices per factor on the tensor cores (Ozaki scheme);
// stream-ordered, no synchronisation.
void launch_gemm_ozaki(Context* ctx, int M, int N, int K, const double* A, int lda, const double* B, int ldb,
                       double* C, int ldc, int S, double alpha = 1.0);
// Several such products in one exponent/split launch and one GEMM launch
// (a tile list over all products).
// One untransposed product C = alpha A B (row-major, leading dimensions given).
struct OzGemm {
    const double* A;
    const double* B;
    double* C;
    int M, N, K, lda, ldb, ldc;
    double alpha;
};
void launch_gemm_ozaki_group(Context* ctx, const std::vector<OzGemm>& gs, int S);

void launch_copy(Context* ctx, const std::vector<CopyTask>& tasks, int kind = KK_COPY);
// Sets n[i] doubles at ptr[i] to zero, all regions in one launch.
void launch_zero(Context* ctx, const std::vector<double*>& ptr, const std::vector<int64_t>& n,
                 int kind = KK_COPY);
// Counts a launch and raises the launch error, if any.
void check_launch(Context* ctx);
// The same grouped GEMM on the tensor cores in split precision (3xTF32, FP32
// accumulation in tensor memory; csrc/tc_gemm.cu); untransposed operands only.
bool gemm_tf32x3_eligible(const std::vector<GemmOut>& outs, const std::vector<GemmIn>& ins);
void launch_gemm_tf32x3(Context* ctx, const std::vector<GemmOut>& outs, const std::vector<GemmIn>& ins, int kind);
// kind: the profiler's record of the launch (KK_GEMM, or KK_APPLY for the zip-up
// contraction, which runs as launch_gemm_tf32x3 when the context's apply
// precision is BSMPS_PREC_TF32X3)
void launch_gemm(Context* ctx, const std::vector<GemmOut>& outs, const std::vector<GemmIn>& ins,
                 int kind = KK_GEMM);
void launch_qr(Context* ctx, const std::vector<QrTask>& tasks, int kind = KK_QR);
// Householder QR of one matrix on a thread-block cluster (csrc/qr_cluster.cu),
// same output as a QrTask of launch_qr; used by launch_qr for matrices with
// min(M, N) >= kClusterQrMin whose columns fit the cluster's shared memory.
constexpr int kClusterQrMin = 48;
// Zip-up QR launches whose widest factor (min(M, N)) is at most this run on
// 8-CTA clusters: more columns per CTA, and SMs left for the other clusters of
// the launch (measured: the zip-up's factorisation 243 -> 208 ms per two
// full-rank steps; the truncation's QRs and the Jacobi were slower on 8).
constexpr int kClusterNarrowMax = 128;
bool qr_cluster_eligible(int M, int N);
bool launch_qr_cluster(Context* ctx, const std::vector<QrTask>& tasks, bool narrow_on_8 = false);
void launch_svd(Context* ctx, const std::vector<SvdTask>& tasks);
// out[i] = sum of squares of x[0..n) for a list of (x, n) segments
void launch_sumsq(Context* ctx, const std::vector<const double*>& xs, const std::vector<int64_t>& ns,
                  double* out_dev);

}  // namespace bsm

namespace bsm {

// ---- fused per-site kernels of the truncation sweeps (csrc/sweep.cu) ----

// Left sweep, one CTA per right sector m of bond t+1: gather the blocks of
// core t that end in m (rows stacked in layout order, r0 = row offset) into
// M x N, Householder QR (diag R >= 0), write Q's rows into the new core-t
// blocks (rows x k) and R X into the new core-(t+1) blocks (k x cols).
struct LeftSrc {
    const double* src;
    double* dst;
    int rows, r0;
};
struct LeftX {
    const double* X;
    double* dst;
    int cols;
};
struct LeftTask {
    int M, N, k;
    int s_beg, s_end, x_beg, x_end;
};
bool left_site_fits(int M, int N, int64_t rx_fma);
void launch_left_site(Context* ctx, const std::vector<LeftTask>& tasks, const std::vector<LeftSrc>& srcs,
                      const std::vector<LeftX>& xs);

// Right sweep, one CTA per left sector n of bond t: gather [X_t(n,0) | X_t(n,1)]
// (parts at column offsets), QR of it (tall) or of its transpose (wide), one-sided
// Jacobi on the triangular factor, and the assembled S, U S, V^T (as SvdTask).
struct SvdPart {
    const double* src;
    int cols, coff;
};
struct SvdSiteTask {
    int M, N, k, len, wide;
    int p_beg, p_end;
    double* S;
    double* US;
    double* Vt;
};
bool svd_site_fits(int M, int N);
// keep: holds the uploaded task lists (the caller releases it after any join);
// on_side: the kernel runs on the context's second stream, forked after the
// uploads (the caller joins before reading the results).
void launch_svd_site(Context* ctx, const std::vector<SvdSiteTask>& tasks, const std::vector<SvdPart>& parts,
                     Scratch& keep, bool on_side = false);

// After the cut of bond t, one CTA per kept sector n: copy the kept V^T rows into
// the new core-t blocks and multiply the core-(t-1) blocks ending in n by the
// kept columns of U S (rows x K times K x keep, US row stride ldus).
struct RCopy {
    const double* src;
    double* dst;
    int rows, cols, src_ld;
};
struct RGemm {
    const double* X;
    const double* US;
    double* dst;
    int rows, K, keep, ldus;
};
struct RTask {
    int c_beg, c_end, g_beg, g_end;
};
constexpr int64_t kFusedGemmMaxFma = 1 << 17;
void launch_right_apply(Context* ctx, const std::vector<RTask>& tasks, const std::vector<RCopy>& copies,
                        const std::vector<RGemm>& gemms);

}  // namespace bsm

namespace bsm {

// ---- device-driven right sweep (no host round trip per bond) ----

// One sigma part of a sector's matrix at bond b: the left-orthogonal core-b
// block X (rows x xcols, row-major) times the kept columns of U S of bond b+1
// (US: xcols x ldus row-major, *keep kept columns; US == nullptr: identity).
struct DynPart {
    const double* X;
    int xcols;
    const double* US;
    int ldus;
    const int* keep;
};
// One sector of bond b: SVD of [part_0 | part_1] into padded outputs
// (S: kpad, US: rows x kpad, Vt: kpad x ncols_pad); *kact receives the rank.
struct alignas(16) DynTask {
    int M, kpad, ncols_pad;
    int p_beg, p_end;
    double* S;
    double* US;
    double* Vt;
    int* kact;
    int cut;           // index of the cut of this task's truncation and bond
    DynPart part[2];   // copies of parts[p_beg .. p_end), filled by the launchers
};
// Cut of one bond: the singular values of its sectors (sector i: S[i] with
// *kact[i] values) pooled and cut exactly as choose_cut; keep[i] receives the
// kept counts, disc[0] / disc[1] accumulate the squared norms discarded by the
// tolerance / the cap.
struct CutSector {
    const double* S;
    const int* kact;
};
struct CutTask {
    int n_sec, s_beg, cap_total, r_max;
    double tol2;
    int* keep;
    double* disc;
    int n_tasks;   // SVD tasks of this truncation and bond (persistent sweep)
    int* done;     // their completion counter (zeroed before the launch)
};
size_t dyn_svd_smem(int M, int ncols_pad);
// returns the index of its profiler record (-1 when not profiling) so that the
// caller can enter the algorithmic flops once the ranks are known
int launch_right_dyn(Context* ctx, const std::vector<DynTask>& tasks, const std::vector<DynPart>& parts);
void launch_cut(Context* ctx, const CutTask& task, const std::vector<CutSector>& secs);

// ---- persistent sweeps (one cooperative launch per sweep) ----

// Phase bookkeeping of one persistent launch (16 bytes, zeroed before the
// launch).  err != 0 after the launch: a bounded wait gave up and the sweep's
// outputs are invalid.
struct GridSync {
    unsigned int arrive, release;
    int err, pad;
};
// Left sweep: phase p runs tasks[phase_beg[p] .. phase_beg[p+1]) (site p);
// the sources of phase p > 0 are the R X outputs of phase p-1.  Returns false
// (nothing launched) when the grid cannot be co-resident.
bool launch_left_sweep(Context* ctx, const std::vector<LeftTask>& tasks, const std::vector<LeftSrc>& srcs,
                       const std::vector<LeftX>& xs, const std::vector<int>& phase_beg, GridSync* gs);
// Right sweep: phase p runs its SVD tasks; the CTA that completes the last
// task of a truncation in the phase runs that truncation's cut (tasks[i].cut).
// *prof_idx: the profiler record (-1 when not profiling).
bool launch_right_sweep(Context* ctx, const std::vector<DynTask>& tasks, const std::vector<DynPart>& parts,
                        const std::vector<int>& phase_beg, const std::vector<CutTask>& cuts,
                        const std::vector<CutSector>& secs, GridSync* gs, int* prof_idx);

// ---- environment sweep of a batch of inner products (one cooperative launch) ----

// Two-CTA cooperative kernel meeting at one phase boundary; CTA skip_cta (if
// >= 0) never arrives.  Returns the error word of the wait (1: a wait gave up).
int check_grid_wait(Context* ctx, int skip_cta);

// ---- environment sweep with structures shared by groups of problems ----
//
// Problems with the same MPS pair and operator share every block structure;
// an output or input refers to a buffer (0: T, 1 / 2: E ping-pong, 3: the 1x1
// block [1]) by a relative offset, and member m of the output's group finds its
// copy at base[buf] + gp.base[buf] + m gp.stride[buf] + offset.
struct EnvGroupPhase {
    int64_t base[4], stride[4];
    int mem_beg, n_mem;   // members: member_fac[mem_beg .. mem_beg + n_mem)
    double shift;         // added to the weight of inputs with shift_flag
};
struct EnvOutT {
    int M, N, ldc, beg, end;
    int gp;    // its group-phase entry
    int cbuf;
    int64_t coff;
};
struct EnvInT {
    const double* A;   // real pointer when abuf < 0
    const double* B;   // real pointer when bbuf < 0
    int64_t aoff, boff;
    int abuf, bbuf;
    int K, lda, ldb, transA;
    double w;
    int shift_flag;
    int so, si;        // factor rows: fa[so], fb[si] of the member (so < 0: no factors)
    int site;
};
struct EnvTileT {
    int out, m0, n0, member;
};
// rows of the factor table (K doubles each) per member: fa0, fa1, fb0, fb1 (-1: 1.0)
struct EnvMemberFac {
    int row[4];
};
bool launch_env_sweep_t(Context* ctx, const std::vector<EnvOutT>& outs, const std::vector<EnvInT>& ins,
                        const std::vector<EnvTileT>& tiles, const std::vector<int>& phase_beg,
                        const std::vector<EnvGroupPhase>& gph, const std::vector<EnvMemberFac>& mfac,
                        const std::vector<double>& ftab, int K, double* const base[4],
                        const std::vector<const double*>& finals, const std::vector<int>& final_beg, double* res,
                        GridSync* gs);

}  // namespace bsm
