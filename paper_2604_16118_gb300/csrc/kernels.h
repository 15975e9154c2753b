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

void launch_copy(Context* ctx, const std::vector<CopyTask>& tasks);
void launch_gemm(Context* ctx, const std::vector<GemmOut>& outs, const std::vector<GemmIn>& ins);
void launch_qr(Context* ctx, const std::vector<QrTask>& tasks);
void launch_svd(Context* ctx, const std::vector<SvdTask>& tasks);
// out[i] = sum of squares of x[0..n) for a list of (x, n) segments
void launch_sumsq(Context* ctx, const std::vector<const double*>& xs, const std::vector<int64_t>& ns,
                  double* out_dev);

}  // namespace bsm
