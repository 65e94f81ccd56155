// FP64 matrix products on the BF16 tensor cores by error-free splitting
// (ozaki.cu): the scheme of Ozaki, Ogita, Oishi and Rump (2012), with the
// slice products on the tcgen05 engine's Gram mode.
#pragma once
#include <vector>

#include "kfac_internal.cuh"

// C = A B with A (M x K), B (K x N) and C (M x N) row-major FP64 matrices with
// leading dimensions lda, ldb, ldc (elements) (times alpha); K <= OZ_MAX_K.  ta: the memory
// at A holds A^T (K x M, row-major); tb: the memory at B holds B^T (N x K).
struct OzGemm {
    const double* A;
    long long lda;
    const double* B;
    long long ldb;
    double* C;
    long long ldc;
    int M, N, K;
    bool ta = false, tb = false;
    double alpha = 1.0;              // C = alpha A B, alpha a power of two or its negative
};

constexpr int OZ_MAX_K = 4096;

struct OzPlan;

// A plan for a fixed list of products (the pointers are fixed; the values may
// change between runs): the slice buffers, the partial sums and the member
// tables of the grouped Gram launches, all allocated here.  status: the word
// the Gram kernels latch KFAC_TIMEOUT into.
kfac_status_t oz_plan_create(const std::vector<OzGemm>& gemms, int* status, OzPlan** out);
// Every product of the plan on s: exponents, slices, one grouped Gram launch
// per slice level, the FP64 combination.  Launches are counted on h.
kfac_status_t oz_run(kfac_pinn_handle* h, OzPlan* p, cudaStream_t s);
void oz_plan_free(OzPlan* p);
