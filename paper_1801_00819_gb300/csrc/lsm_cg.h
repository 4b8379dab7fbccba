// CG vector-kernel launchers (float32 vectors, float64 scalars).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace lsm {

// Fixed reduction grid: partial-sum arrays have exactly this many entries.
constexpr int kRedBlocks = 296;
// cg_reduce_image runs on a grid of its own size; its partial sums (ss_part, sz_part, and the ones
// cg_store_sum and cg_update_p read back) have exactly kImgRedBlocks entries.
constexpr int kImgRedBlocks = 512;

struct CgState {
    double gamma[2];  // s.z of the current and the next iterate (slots alternate); z = s unpreconditioned
    double alpha, beta, delta;
    double bb;        // ||A_k^T d_k||^2
    double ss[2];     // ||s||^2 matching gamma's slots (the stopping rule's numerator)
    int breakdown;
    // device-driven iteration loop (CUDA-graph CG): slot of the current gamma, iterations done,
    // iteration limit, tolerance, and the stopping-rule ratios before the first / after the last
    // iteration
    int gi;
    int iter, max_iter;
    double tol, rel0, rel;
};

// With p and state given (a CG iteration whose sweeps fold in the vector work), m += alpha p is
// applied before s = sum - lambda m and m is written back; alpha is read from the state.  With
// discard_part the partial planes are dead once read: their L2 lines are invalidated without a
// write-back (the partials a sweep has just written, still in L2, then never reach HBM).
cudaError_t cg_reduce_image(const float* part, int nparts, int n, float* m, float lam, int acc, float* out,
                            double* ss_part, cudaStream_t st, const float* minv = nullptr, double* sz_part = nullptr,
                            const float* p = nullptr, const CgState* state = nullptr, bool discard_part = false);
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
// *out = the sum of n partials in a fixed order (one block)
cudaError_t cg_sum_partials(const double* part, int n, double* out, cudaStream_t st);

// Device-driven CG loop.  gi = -1 in cg_update_mr / cg_update_p means "the slot in state->gi"
// (cg_update_p then writes slot state->gi ^ 1); cg_loop_setup resets the loop counters and stores
// the window's first shot for the sweeps' shot0_dev; cg_loop_test (one thread) advances the loop
// when `advance` is set (flips state->gi, counts the iteration), evaluates the stopping rule
// ||s|| / ||A_k^T d_k|| <= tol, the iteration limit and the breakdown flag, and sets the conditional
// handle of the enclosing WHILE node to 1 to continue or 0 to stop.
// With `halt` given and set, the window gets no iterations (a whole-solve graph after a breakdown).
cudaError_t cg_loop_setup(CgState* state, int* shot0_dev, int shot0, int max_iter, double tol, cudaStream_t st,
                          const int* halt = nullptr);
cudaError_t cg_loop_test(CgState* state, cudaGraphConditionalHandle handle, int advance, cudaStream_t st);
// kernel-node parameters of cg_loop_test for explicit graph construction (args must outlive the call)
void cg_loop_test_node_params(cudaKernelNodeParams* kp, void** args);
cudaError_t cg_zero_state(CgState* state, cudaStream_t st);

// One window's outcome, written on the device at the end of its CG loop (whole-solve graphs, where
// the host reads every window's outcome once, after the last window).
struct WindowRecord {
    int iters, breakdown;
    double rel0, rel;
};
// rec <- the state's iteration count, stopping ratios and breakdown flag; a breakdown also sets *halt
cudaError_t cg_record_window(const CgState* state, WindowRecord* rec, int* halt, cudaStream_t st);

}  // namespace lsm
