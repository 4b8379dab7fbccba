// CG vector-kernel launchers (float32 vectors, float64 scalars).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace lsm {

// Fixed reduction grid: partial-sum arrays have exactly this many entries.
constexpr int kRedBlocks = 296;

struct CgState {
    double gamma[2];  // s.z of the current and the next iterate (slots alternate); z = s unpreconditioned
    double alpha, beta, delta;
    double bb;        // ||A_k^T d_k||^2
    double ss[2];     // ||s||^2 matching gamma's slots (the stopping rule's numerator)
    int breakdown;
    int pad;
};

cudaError_t cg_reduce_image(const float* part, int nparts, int n, const float* m, float lam, int acc, float* out,
                            double* ss_part, cudaStream_t st, const float* minv = nullptr, double* sz_part = nullptr);
cudaError_t cg_norm2_c64(const float2* q, size_t n2, double* part, cudaStream_t st);
cudaError_t cg_residual(const float2* d, const float2* q, float2* r, size_t n2, cudaStream_t st);
cudaError_t cg_update_mr(float* m, const float* p, int n, float2* r, const float2* q, size_t n2,
                         const double* qq_part, const double* pp_part, double lam, CgState* state, int gi,
                         cudaStream_t st);
cudaError_t cg_update_p(float* p, const float* s, int n, const double* ss_part, int first, CgState* state,
                        int gi_old, int gi_new, double* pp_part, cudaStream_t st, const float* minv = nullptr,
                        const double* sz_part = nullptr);
// Diagonal source-illumination preconditioner of the window whose source wavefields fill the ring:
// illum = sum over the ring's slots and frequencies of |S_j(x)|^2; minv = 1 / (illum + eps max illum).
constexpr int kIllumBlocks = 512;
cudaError_t cg_illumination(const float2* S, int rows, int n, float* illum, float* block_max, cudaStream_t st);
cudaError_t cg_precond_finalize(const float* illum, int n, const float* block_max, double eps, float* minv,
                                cudaStream_t st);
cudaError_t cg_store_sum(const double* part, CgState* state, cudaStream_t st);
cudaError_t cg_zero_state(CgState* state, cudaStream_t st);

}  // namespace lsm
