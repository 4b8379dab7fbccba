// Internal host-side declarations shared by the C-ABI layer and the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>

namespace lsm {

struct CgState;  // lsm_cg.h

enum SweepMode { MODE_SOURCE = 0, MODE_ADJOINT = 1, MODE_FORWARD = 2 };

// Arguments of one depth sweep over the (shot, frequency) items of shots [shot0, shot0+nshots).
// Item index = iw * nshots + (shot - shot0), so consecutive items share a frequency and read the
// same coefficient rows.  The source wavefield of shot s lives in ring slot s % ring.
struct SweepArgs {
    int nx, nz, nw, nrec;
    int shot0, nshots, ring;
    int rec_identity;              // 1: receivers at every column in order
    int wslots;                    // staging slots: most frequencies any block's items span
    const int* src_ix;             // device [ns]
    const int* rec_ix;             // device [ns][nrec] (unused when rec_identity)
    const float2* wavelet;         // device [nw]
    const float2* phi;             // device [nw][nz][nx]: Phi_j / nx in the FFT's output order
    const float2* dss;             // device [nw][nz][nx]: split-step factor D_j(x)
    float2* S;                     // device [ring][nw][nz][nx]: source wavefield cache
    const float2* din;             // adjoint input [nshots][nw][nrec]
    float2* dout;                  // forward output [nshots][nw][nrec]
    const float* m;                // forward model [nz][nx]
    float* part;                   // adjoint per-block partial images [grid][nz][nx]
    const int* shot0_dev;          // if set, shot0 is read from this device int (graph-replayed
                                   // CG iterations, whose window start changes between launches)
    // CG vector work folded into the sweeps of one CG iteration (all null / 0 outside it):
    double* qq_part;               // forward: one partial sum of |q|^2 over the recorded data per block
    float2* r_io;                  // adjoint: the residual r, updated in place to r - alpha q while it
                                   // is injected (replaces din)
    const float2* dq;              // adjoint: q = A p of this iteration, [nshots][nw][nrec]
    const double* qq_in;           // adjoint: the forward sweep's |q|^2 partials (nqq entries)
    const double* pp_in;           // adjoint: ||p||^2 partials (npp entries)
    int nqq, npp;
    int cg_gi;                     // slot of the current gamma in cg; -1: cg->gi (device-driven loop)
    double lam;                    // Tikhonov weight lambda
    CgState* cg;                   // gamma (read); delta, alpha and the breakdown flag (block 0 writes)
    int* dev_err;                  // set to 1 by a kernel whose bounded wait on the tensor core ran out
    int V;                         // FFT tile (points per thread) of the register-FFT sweeps; 0: default
};

// Arguments of the gradient kernel (lsm_grad.cuh) over the items of shots [shot0, shot0+nshots).
struct GradArgs {
    int nx, nz, nw, nrec;
    int shot0, nshots;
    int rec_identity;
    int ckpt_every;                // depth checkpoint stride of S and R
    int wslots;                    // staging slots: most frequencies any block's items span
    float dz;
    const int* src_ix;
    const int* rec_ix;
    const float2* wavelet;
    const float* freq_hz;          // device [nw]
    const float2* phi;             // coefficient tables in the order of Plan<nx, gradient_points_per_thread(nx)>
    const float2* dss;
    const float* m;                // [nz][nx]
    const float2* g;               // dL/dRe d + i dL/dIm d, [nshots][nw][nrec]
    float2* ckpt;                  // [items][2][ceil(nz/c)][nx]
    float2* seg;                   // [items][2c+1][nx]
    float2* park;                  // [items][2][nx]: U and mu while the other is in registers
    float* part_m;                 // [blocks][nz][nx]
    float* part_s;                 // [blocks][nz][nx]
    float2* dout;                  // optional modelled data [nshots][nw][nrec]
};

struct TableArgs {
    int V;                   // FFT tile whose register order the Phi table follows; 0: default
    int nx, nz, nw;
    float dx, dz;
    const float* slowness;   // [nz][nx]
    const double* sref;      // [nz]
    const float* freq_hz;    // [nw]
    float2* phi;
    float2* dss;
};

// Launch geometry of a sweep: grid.x blocks of `warps` warps whose items span at most `wslots`
// frequencies, with `smem` bytes of dynamic shared memory.
struct SweepShape {
    int blocks;
    int warps;
    int wslots;
    size_t smem;
};

bool nx_supported(int nx);
// Block count of the adjoint sweep for this many items (partial images to reduce).
SweepShape sweep_shape(int nx, int mode, int nshots, int nw, int num_sms);
cudaError_t launch_tables(const TableArgs& a, cudaStream_t st);
cudaError_t launch_sweep(int mode, const SweepArgs& a, const SweepShape& shape, cudaStream_t st);

// Per-nx entry points, one translation unit (sweep_n<nx>.cu) per supported nx.
struct NxOps {
    int nx;
    int points_per_thread;        // V of the sweep kernels
    bool has_gradient;            // lsm_born_gradient's kernel exists for this nx
    cudaError_t (*tables)(const TableArgs& a, cudaStream_t st);
    cudaError_t (*sweep)(int mode, const SweepArgs& a, const SweepShape& shape, cudaStream_t st);
    int (*max_warps)(int mode);
    size_t (*smem)(int mode, int warps, int wslots);
    cudaError_t (*tables_grad)(const TableArgs& a, cudaStream_t st);
    cudaError_t (*gradient)(const GradArgs& a, const SweepShape& shape, cudaStream_t st);
    int (*gradient_max_warps)();
    bool has_tc;                  // tensor-core transform variants exist for this nx
    cudaError_t (*tables_natural)(const TableArgs& a, cudaStream_t st);
    cudaError_t (*tc_sweep)(int mode, int prec, const SweepArgs& a, const SweepShape& shape, cudaStream_t st);
    size_t (*tc_smem)(int mode, int warps);
    size_t (*gradient_smem)(int warps, int wslots);
    bool has_tc5;                 // tcgen05 transform variants exist for this nx
    size_t (*tc5_smem)(int wslots);  // their dynamic shared memory per CTA (wslots 0: rows unstaged)
    int tc5_items;                // their (shot, frequency) items per CTA
    int tc5_threads;              // and threads per CTA
    const NxOps* alt;             // the sweeps with the alternative FFT tile (only tables, sweep,
                                  // max_warps and smem set), or nullptr
};
// Dynamic shared memory a tcgen05 sweep CTA may take: the 227 KB opt-in limit less a margin for
// the kernel's static shared memory.
constexpr size_t kTc5MaxDynSmem = 227 * 1024 - 1024;

// The operations for nx, or nullptr when nx is not supported.
const NxOps* nx_ops(int nx);

// Points per thread of the sweep kernels: 16 for power-of-two nx below 512 and 32 from 512; for
// nx = q 2^a (q = 3, 5, 7), 8 q (4 q when q = 7), doubled until at most 32 threads share a line.
constexpr int odd_factor(int n) {
    while (n > 1 && n % 2 == 0) n /= 2;
    return n;
}
constexpr int points_per_thread(int nx) {
    const int q = odd_factor(nx);
    if (q == 1) return nx >= 512 ? 32 : 16;
    int v = q == 7 ? 4 * q : 8 * q;
    while (nx / v > 32) v *= 2;
    return v;
}

// The alternative FFT tile of the sweep kernels: half the points per thread (twice the threads per
// (shot, frequency) item) where that plan exists -- V/2 a multiple of the odd factor with at least two
// power-of-two points left, and at most 32 threads per item; 0 where it does not (nx = 768, 896, 1024).
// At nx = 512 it is the pair plan (32 x 16 with each 32-point first-stage DFT shared by two lanes).
constexpr int alt_points_per_thread(int nx) {
    const int q = odd_factor(nx);
    const int v = points_per_thread(nx) / 2;
    if (v < 2 || v % q != 0 || v / q < 2 || nx % v != 0 || nx / v > 32) return 0;
    return v;
}

// Points per thread of the gradient kernel (two wavefields in registers at a time): 32 from 512
// columns (32 x 16 and 32 x 32 plans), 16 below.
constexpr int gradient_points_per_thread(int nx) { return nx >= 512 ? 32 : 16; }
bool gradient_nx_supported(int nx);
SweepShape gradient_shape(int nx, int nshots, int nw, int num_sms);
cudaError_t launch_tables_grad(const TableArgs& a, cudaStream_t st);
cudaError_t launch_gradient(const GradArgs& a, const SweepShape& shape, cudaStream_t st);

void count_launch(int n = 1);

// Runs a set-up call once per device (thread safe): kernel attributes are per device.
struct DeviceOnce {
    std::mutex mu;
    uint64_t done = 0;
    template <class F>
    cudaError_t run(F&& f) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        const uint64_t bit = dev < 64 ? (uint64_t)1 << dev : 0;
        std::lock_guard<std::mutex> lock(mu);
        if (bit && (done & bit)) return cudaSuccess;
        e = f();
        if (e == cudaSuccess) done |= bit;
        return e;
    }
};

// Per-launch event timing (lsm_profile_start / lsm_profile_stop).  Construct a ProfScope right
// before a launch and destroy it right after; both ends record an event on the launch stream
// when profiling is on.
enum KernelClass { KC_TABLES = 0, KC_SOURCE = 1, KC_ADJOINT = 2, KC_FORWARD = 3, KC_VECTOR = 4, KC_GRADIENT = 5 };
void profile_mark(int cls, cudaStream_t st, bool begin);
struct ProfScope {
    int cls;
    cudaStream_t st;
    ProfScope(int c, cudaStream_t s) : cls(c), st(s) { profile_mark(cls, st, true); }
    ~ProfScope() { profile_mark(cls, st, false); }
};

}  // namespace lsm
