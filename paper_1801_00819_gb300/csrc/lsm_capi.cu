// C ABI of the block-row recursive least-squares migration library (see include/lsm.h).
//
// Host side: argument validation, workspace carving, per-call upload of the host geometry and
// frequency arrays, launch geometry, and the sliding-window CG driver (block-row section,
// Eq. 10 and Eq. 11).  Every arithmetic step of the operator and of CG runs in the kernels of
// lsm_sweep.cuh and lsm_cg.cu; the host only sequences them and reads one small state struct
// per CG iteration (host-driven loop) or per window (graph-replayed loop, where the stopping rule
// is tested on the device).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/lsm.h"
#include "lsm_cg.h"
#include "lsm_internal.h"

namespace lsm {

static std::atomic<unsigned long long> g_launches{0};
// While this thread captures a CG iteration into a graph, launches are counted per replay (the
// captured count times the iterations run) and no profiling events are recorded (a conditional
// node's body may hold kernels only).
static thread_local bool g_capturing = false;
static thread_local int g_captured_launches = 0;
void count_launch(int n) {
    if (g_capturing) {
        g_captured_launches += n;
        return;
    }
    g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed);
}

struct ProfRecord {
    int cls;
    cudaEvent_t begin, end;
};
static std::atomic<bool> g_prof_on{false};
static std::atomic<unsigned> g_prof_mask{~0u};  // kernel classes timed while profiling is on
static std::mutex g_prof_mu;  // guards g_prof and g_event_pool
static std::vector<ProfRecord> g_prof;
static std::vector<cudaEvent_t> g_event_pool;
static thread_local cudaEvent_t g_pending_begin = nullptr;

static cudaEvent_t pooled_event() {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// whether lsm_profile_start(_classes) is timing the A or A^T sweeps (they cannot be timed inside a
// graph's conditional body)
static bool profiling_sweeps() {
    return g_prof_on && (g_prof_mask.load(std::memory_order_relaxed) & ((1u << KC_ADJOINT) | (1u << KC_FORWARD)));
}

void profile_mark(int cls, cudaStream_t st, bool begin) {
    if (!g_prof_on || g_capturing || !((g_prof_mask.load(std::memory_order_relaxed) >> cls) & 1u)) return;
    if (begin) {
        g_pending_begin = pooled_event();
        if (g_pending_begin) cudaEventRecord(g_pending_begin, st);
    } else {
        cudaEvent_t e = pooled_event();
        if (e && g_pending_begin) {
            cudaEventRecord(e, st);
            std::lock_guard<std::mutex> lock(g_prof_mu);
            g_prof.push_back({cls, g_pending_begin, e});
        }
        g_pending_begin = nullptr;
    }
}

#define LSM_NX_LIST(X)                                                                       \
    X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(48) X(96) X(192) X(384) X(768) X(80) X(160) \
    X(320) X(640) X(112) X(224) X(448) X(896)
#define LSM_DECLARE_OPS(NN) extern const NxOps kNxOps_##NN;
LSM_NX_LIST(LSM_DECLARE_OPS)
#undef LSM_DECLARE_OPS

const NxOps* nx_ops(int nx) {
#define LSM_MATCH_OPS(NN) \
    if (nx == NN) return &kNxOps_##NN;
    LSM_NX_LIST(LSM_MATCH_OPS)
#undef LSM_MATCH_OPS
    return nullptr;
}

bool nx_supported(int nx) { return nx_ops(nx) != nullptr; }

// The register-FFT sweeps of nx with V points per thread (0: the default tile), or nullptr.
const NxOps* fft_ops(int nx, int V) {
    const NxOps* ops = nx_ops(nx);
    if (!ops || V == 0 || V == ops->points_per_thread) return ops;
    return ops->alt && ops->alt->points_per_thread == V ? ops->alt : nullptr;
}

// ------------------------------------------------------------------ launch shapes and their tuning
// A launch shape is the number of warps per block (items per block = warps x items per warp); the
// heuristic spreads a launch's warps evenly over the SMs.  lsm_autotune measures the alternatives
// and records the fastest per (device, nx, sweep mode, transform, FFT tile, shots, frequencies);
// launches use a recorded shape, the workspace layout always the heuristic one (the tuner never picks
// an adjoint shape with more blocks, i.e. more partial images, than the heuristic's).  For the
// register FFTs it also picks the FFT tile (points per thread) of a problem: the default or, where
// one exists, the alternative with half the points per thread (twice the threads per item).  The
// tile fixes the coefficient tables' order, so a call builds its tables for the recorded tile and
// every sweep of the call uses it.
struct TuneKey {
    int dev, nx, mode, transform, V, nshots, nw;
    bool operator<(const TuneKey& o) const {
        return std::tie(dev, nx, mode, transform, V, nshots, nw) <
               std::tie(o.dev, o.nx, o.mode, o.transform, o.V, o.nshots, o.nw);
    }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, int> g_tune;
struct TileKey {
    int dev, nx, nshots, nw;
    bool operator<(const TileKey& o) const {
        return std::tie(dev, nx, nshots, nw) < std::tie(o.dev, o.nx, o.nshots, o.nw);
    }
};
static std::map<TileKey, int> g_tile;  // guarded by g_tune_mu

static int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
    return dev;
}
static TuneKey tune_key(int nx, int mode, int transform, int nshots, int nw, int V = 0) {
    return TuneKey{current_device(), nx, mode, transform, V, nshots, nw};
}
static int tuned_warps(int nx, int mode, int transform, int nshots, int nw, int V = 0) {
    const TuneKey k = tune_key(nx, mode, transform, nshots, nw, V);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(k);
    return it == g_tune.end() ? 0 : it->second;
}
// the FFT tile recorded for calls over nshots shots of this problem (0: the default)
static int chosen_tile(int nx, int nshots, int nw) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tile.find(TileKey{current_device(), nx, nshots, nw});
    return it == g_tile.end() ? 0 : it->second;
}

// Checkpoint stride of the gradient sweep (lsm_born_gradient): S and R are kept every c-th depth
// and recomputed segment by segment, so the arithmetic is the same for every c; c sets how many
// checkpoint and segment rows each item keeps, and with them the memory traffic.
// lsm_autotune_gradient times the candidates and records the fastest per (device, nx, nz, shots,
// frequencies); the layout reserves room for the largest candidate's rows.
static const int kCkptStrides[] = {8, 16, 32};
struct CkptKey {
    int dev, nx, nz, nshots, nw;
    bool operator<(const CkptKey& o) const {
        return std::tie(dev, nx, nz, nshots, nw) < std::tie(o.dev, o.nx, o.nz, o.nshots, o.nw);
    }
};
struct GradTune {
    int stride, warps;  // checkpoint stride; warps per block (0: the heuristic's)
};
static std::map<CkptKey, GradTune> g_ckpt_tune;  // guarded by g_tune_mu
static CkptKey ckpt_key(int nx, int nz, int nshots, int nw) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
    return CkptKey{dev, nx, nz, nshots, nw};
}
static int ckpt_stride(int nx, int nz, int nshots, int nw) {
    const CkptKey k = ckpt_key(nx, nz, nshots, nw);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_ckpt_tune.find(k);
    return std::min(it == g_ckpt_tune.end() ? LSM_CHECKPOINT_EVERY : it->second.stride, nz);
}
static int tuned_gradient_warps(int nx, int nz, int nshots, int nw) {
    const CkptKey k = ckpt_key(nx, nz, nshots, nw);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_ckpt_tune.find(k);
    return it == g_ckpt_tune.end() ? 0 : it->second.warps;
}
// rows of nx complex values one item keeps at stride c: S and R checkpoints, the segment's S rows
// (c + 1) and R rows (c), and two parking rows (U and mu)
static size_t ckpt_rows(int c, int nz) {
    c = std::min(c, nz);
    return 2 * (size_t)((nz + c - 1) / c) + 2 * (size_t)c + 1 + 2;
}

// most warps per block a sweep of this mode can take (registers, shared memory)
static int sweep_max_warps(int nx, int mode, int nshots, int nw, int tile = 0) {
    const NxOps* ops = fft_ops(nx, tile);
    const int V = ops->points_per_thread;
    const int ipw = 32 / (nx / V);
    auto wslots_of = [&](int w) { return std::min(nw, (w * ipw + nshots - 1) / nshots + 1); };
    int maxw = std::min(V >= 24 ? 8 : 16, ops->max_warps(mode));
    while (maxw > 1 && ops->smem(mode, maxw, wslots_of(maxw)) > 227 * 1024) --maxw;
    return maxw;
}

static SweepShape sweep_shape_for(int nx, int mode, int nshots, int nw, int warps, int tile = 0) {
    const NxOps* ops = fft_ops(nx, tile);
    const int ipw = 32 / (nx / ops->points_per_thread);
    const int warps_total = (nshots * nw + ipw - 1) / ipw;
    SweepShape s;
    s.warps = warps;
    s.blocks = (warps_total + warps - 1) / warps;
    s.wslots = std::min(nw, (warps * ipw + nshots - 1) / nshots + 1);
    s.smem = ops->smem(mode, warps, s.wslots);
    return s;
}

SweepShape sweep_shape_heuristic(int nx, int mode, int nshots, int nw, int num_sms, int tile = 0) {
    const int ipw = 32 / (nx / fft_ops(nx, tile)->points_per_thread);
    const int warps_total = (nshots * nw + ipw - 1) / ipw;
    int warps = (warps_total + num_sms - 1) / num_sms;
    warps = std::max(1, std::min(warps, sweep_max_warps(nx, mode, nshots, nw, tile)));
    return sweep_shape_for(nx, mode, nshots, nw, warps, tile);
}

SweepShape sweep_shape(int nx, int mode, int nshots, int nw, int num_sms, int tile = 0) {
    const int w = tuned_warps(nx, mode, 0, nshots, nw, tile);
    if (w > 0) return sweep_shape_for(nx, mode, nshots, nw, w, tile);
    return sweep_shape_heuristic(nx, mode, nshots, nw, num_sms, tile);
}

bool gradient_nx_supported(int nx) {
    const NxOps* ops = nx_ops(nx);
    return ops && ops->has_gradient;
}

// gradient launch with `warps` warps per block (at most the heuristic's, so shared memory fits)
static SweepShape gradient_shape_for(int nx, int nshots, int nw, int warps) {
    const NxOps* ops = nx_ops(nx);
    const int V = gradient_points_per_thread(nx);
    const int ipw = 32 / (nx / V);
    const int warps_total = (nshots * nw + ipw - 1) / ipw;
    SweepShape s;
    s.warps = warps;
    s.blocks = (warps_total + warps - 1) / warps;
    s.wslots = std::min(nw, (warps * ipw + nshots - 1) / nshots + 1);
    s.smem = ops->gradient_smem(warps, s.wslots);
    return s;
}

// the heuristic: a launch's warps spread evenly over the SMs, within the register and shared-memory
// limits of one block
SweepShape gradient_shape(int nx, int nshots, int nw, int num_sms) {
    const NxOps* ops = nx_ops(nx);
    const int V = gradient_points_per_thread(nx);
    const int ipw = 32 / (nx / V);
    const int warps_total = (nshots * nw + ipw - 1) / ipw;
    int maxw = std::min(8, ops->gradient_max_warps());
    while (maxw > 1 && gradient_shape_for(nx, nshots, nw, maxw).smem > 227 * 1024) --maxw;
    int warps = (warps_total + num_sms - 1) / num_sms;
    warps = std::max(1, std::min(warps, maxw));
    return gradient_shape_for(nx, nshots, nw, warps);
}

// lsm_autotune_gradient's warps-per-block candidates: the heuristic's and up to two fewer (more,
// smaller blocks even out the last round of blocks); the layout keeps partial images for the
// smallest
static int gradient_min_warps(int nx, int nshots, int nw, int num_sms) {
    return std::max(1, gradient_shape(nx, nshots, nw, num_sms).warps - 2);
}

// the shape lsm_born_gradient launches: a recorded one, else the heuristic
static SweepShape gradient_launch_shape(int nx, int nz, int nshots, int nw, int num_sms) {
    const int w = tuned_gradient_warps(nx, nz, nshots, nw);
    return w > 0 ? gradient_shape_for(nx, nshots, nw, w) : gradient_shape(nx, nshots, nw, num_sms);
}

// tensor-core variants: one item per warp, up to 7 warps per block (two blocks per SM)
static SweepShape tc_shape_for(int nx, int mode, int nshots, int nw, int warps) {
    const int nitems = nshots * nw;
    SweepShape s;
    s.warps = warps;
    s.blocks = (nitems + warps - 1) / warps;
    s.wslots = 0;
    s.smem = nx_ops(nx)->tc_smem(mode, warps);
    return s;
}

SweepShape tc_shape_heuristic(int nx, int mode, int nshots, int nw, int num_sms) {
    const int per_sm = nx > 512 ? 1 : 2;  // blocks an SM holds (shared memory, registers)
    int warps = (nshots * nw + per_sm * num_sms - 1) / (per_sm * num_sms);
    warps = std::max(1, std::min(warps, 7));
    return tc_shape_for(nx, mode, nshots, nw, warps);
}

// tcgen05 variants: a fixed shape per width (items and threads per CTA); a CTA whose frequencies'
// staged Phi and D rows would not fit its shared memory reads them from global memory (wslots 0)
static bool is_tc5(int transform) {
    return transform == LSM_TRANSFORM_DFT_FP16X3_TCGEN05 || transform == LSM_TRANSFORM_DFT_BF16X3_TCGEN05;
}
static SweepShape tc5_shape(int nx, int nshots, int nw) {
    const NxOps* ops = nx_ops(nx);
    const int items = ops->tc5_items;
    SweepShape s;
    s.warps = ops->tc5_threads / 32;
    s.blocks = (nshots * nw + items - 1) / items;
    s.wslots = std::min(nw, (items + nshots - 1) / nshots + 1);  // frequencies a CTA's items can span
    s.smem = ops->tc5_smem(s.wslots);
    if (s.smem > kTc5MaxDynSmem) {
        s.wslots = 0;
        s.smem = ops->tc5_smem(0);
    }
    return s;
}

SweepShape tc_shape(int nx, int mode, int nshots, int nw, int num_sms, int transform) {
    if (is_tc5(transform)) return tc5_shape(nx, nshots, nw);
    const int w = tuned_warps(nx, mode, transform, nshots, nw);
    if (w > 0) return tc_shape_for(nx, mode, nshots, nw, w);
    return tc_shape_heuristic(nx, mode, nshots, nw, num_sms);
}

cudaError_t launch_tables_grad(const TableArgs& a, cudaStream_t st) { return nx_ops(a.nx)->tables_grad(a, st); }
cudaError_t launch_gradient(const GradArgs& a, const SweepShape& sh, cudaStream_t st) {
    return nx_ops(a.nx)->gradient(a, sh, st);
}
cudaError_t launch_tables(const TableArgs& a, cudaStream_t st) { return fft_ops(a.nx, a.V)->tables(a, st); }
cudaError_t launch_sweep(int mode, const SweepArgs& a, const SweepShape& sh, cudaStream_t st) {
    return fft_ops(a.nx, a.V)->sweep(mode, a, sh, st);
}

// s_ref(z_j) = mean over x of s(x, z_j), summed in float64 (Examples section: split-step
// reference slowness per depth row)
__global__ void reference_slowness_kernel(const float* __restrict__ s, int nx, int nz, double* __restrict__ sref) {
    __shared__ double sh[32];
    const int j = blockIdx.x;
    if (j >= nz) return;
    double acc = 0.0;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) acc += (double)s[(size_t)j * nx + x];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
        sref[j] = tot / (double)nx;
    }
}

}  // namespace lsm

using namespace lsm;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int num_sms_current() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 152;
    }
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return 152;
    }
    return n;
}

struct Layout {
    // offsets in bytes from the workspace base
    size_t src, rec, freq, wav, sref, phi, dss, S, part;
    size_t p, s, r, q, qq, pp, ss, state;
    size_t ckpt, part_s, tune_m, tune_g;  // gradient op
    size_t illum, minv, bmax, sz;  // preconditioned solve
    size_t ctrl;                   // solve: window start read by graph-replayed sweeps
    size_t err;                    // int: set by a tcgen05 sweep whose bounded wait ran out
    size_t img, qqt;               // sharded solve: local image, all-reduced ||q||^2
    size_t wrec, halt;             // whole-solve graph: per-window records, breakdown halt flag
    size_t total;
    int ring, nparts;
};

bool rec_is_identity(const lsm_grid* g, const lsm_geom* geo) { return geo->rec_ix == nullptr; }

Layout make_layout(const lsm_grid* g, const lsm_geom* geo, const lsm_freqs* f, int nshots, int op, int num_sms) {
    Layout L{};
    const size_t nx = (size_t)g->nx, nz = (size_t)g->nz, nw = (size_t)f->nw;
    const size_t plane = nz * nx;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    L.src = take((size_t)geo->ns * sizeof(int));
    L.rec = take(rec_is_identity(g, geo) ? 0 : (size_t)geo->ns * geo->nrec * sizeof(int));
    L.freq = take(nw * sizeof(float));
    L.wav = take(nw * sizeof(float2));
    L.sref = take(nz * sizeof(double));
    L.phi = take(nw * plane * sizeof(float2));
    L.dss = take(nw * plane * sizeof(float2));
    L.ring = nshots;
    L.S = take((size_t)nshots * nw * plane * sizeof(float2));
    L.nparts = 0;
    if (op == LSM_OP_ADJOINT || op == LSM_OP_SOLVE) {
        const SweepShape sh = sweep_shape_heuristic(g->nx, MODE_ADJOINT, nshots, (int)nw, num_sms);
        L.nparts = sh.blocks;
        if (const NxOps* alt = nx_ops(g->nx)->alt)
            L.nparts = std::max(L.nparts, sweep_shape_heuristic(g->nx, MODE_ADJOINT, nshots, (int)nw, num_sms,
                                                                alt->points_per_thread).blocks);
        if (nx_ops(g->nx)->has_tc)
            L.nparts = std::max(L.nparts, tc_shape_heuristic(g->nx, MODE_ADJOINT, nshots, (int)nw, num_sms).blocks);
        if (nx_ops(g->nx)->has_tc5) L.nparts = std::max(L.nparts, tc5_shape(g->nx, nshots, (int)nw).blocks);
    } else if (op == LSM_OP_GRADIENT) {
        L.nparts = gradient_shape_for(g->nx, nshots, (int)nw, gradient_min_warps(g->nx, nshots, (int)nw, num_sms)).blocks;
    }
    L.part = take((size_t)L.nparts * plane * sizeof(float));
    if (op == LSM_OP_GRADIENT) {
        const size_t items = (size_t)nshots * nw;
        size_t rows = ckpt_rows(LSM_CHECKPOINT_EVERY, (int)nz);
        for (int c : kCkptStrides) rows = std::max(rows, ckpt_rows(c, (int)nz));
        L.part_s = take((size_t)L.nparts * plane * sizeof(float));
        L.ckpt = take(items * rows * nx * sizeof(float2));  // checkpoints, then segments (per stride)
        L.ss = take(kImgRedBlocks * sizeof(double));
        L.tune_m = take(plane * sizeof(float));  // lsm_autotune_gradient's zero inputs
        L.tune_g = take(items * geo->nrec * sizeof(float2));
    }
    if (op == LSM_OP_SOLVE) {
        const size_t nd = (size_t)nshots * nw * geo->nrec;
        L.p = take(plane * sizeof(float));
        L.s = take(plane * sizeof(float));
        L.r = take(nd * sizeof(float2));
        L.q = take(nd * sizeof(float2));
        // |q|^2 partials: one per block of the CG iteration's forward sweep (at most one per item)
        L.qq = take(std::max((size_t)kRedBlocks, (size_t)nshots * nw) * sizeof(double));
        L.pp = take(kRedBlocks * sizeof(double));
        L.ss = take(kImgRedBlocks * sizeof(double));
        L.state = take(sizeof(CgState));
        L.ctrl = take(sizeof(int));
        L.illum = take(plane * sizeof(float));
        L.minv = take(plane * sizeof(float));
        L.bmax = take(kIllumBlocks * sizeof(float));
        L.sz = take(kImgRedBlocks * sizeof(double));
        L.img = take(plane * sizeof(float));  // sharded solve: this rank's image before the all-reduce
        L.qqt = take(sizeof(double));         // sharded solve: ||q||^2 summed over the ranks
        // whole-solve graph: every window's outcome (at most ns + 1 windows) and the halt flag
        L.wrec = take((size_t)(geo->ns + 1) * sizeof(WindowRecord));
        L.halt = take(sizeof(int));
    } else if (op == LSM_OP_ADJOINT) {
        L.ss = take(kImgRedBlocks * sizeof(double));
    }
    L.err = take(sizeof(int));
    L.total = off;
    return L;
}

bool aligned16(const void* p) { return p != nullptr && ((uintptr_t)p & 15u) == 0; }

int validate_common(const lsm_grid* g, const lsm_freqs* f, const lsm_geom* geo) {
    if (!g || !f || !geo) return LSM_ERR_ARG;
    if (g->nz < 1 || g->nx < 1) return LSM_ERR_ARG;
    if (!nx_supported(g->nx)) return LSM_ERR_UNSUPPORTED_NX;
    if (!(g->dx > 0.f) || !(g->dz > 0.f) || !std::isfinite(g->dx) || !std::isfinite(g->dz)) return LSM_ERR_ARG;
    if (f->nw < 1 || !f->freq_hz || !f->wavelet) return LSM_ERR_ARG;
    for (int i = 0; i < f->nw; ++i) {
        if (!std::isfinite(f->freq_hz[i]) || f->freq_hz[i] < 0.f) return LSM_ERR_ARG;
        if (!std::isfinite(f->wavelet[2 * i]) || !std::isfinite(f->wavelet[2 * i + 1])) return LSM_ERR_ARG;
    }
    if (geo->ns < 1 || !geo->src_ix || geo->nrec < 1) return LSM_ERR_ARG;
    for (int i = 0; i < geo->ns; ++i)
        if (geo->src_ix[i] < 0 || geo->src_ix[i] >= g->nx) return LSM_ERR_ARG;
    if (!geo->rec_ix) {
        if (geo->nrec != g->nx) return LSM_ERR_ARG;
    } else {
        const size_t n = (size_t)geo->ns * geo->nrec;
        for (size_t i = 0; i < n; ++i)
            if (geo->rec_ix[i] < 0 || geo->rec_ix[i] >= g->nx) return LSM_ERR_ARG;
    }
    // item and index arithmetic in the kernels uses 32-bit item counts
    if ((double)geo->ns * f->nw > 1.0e9 || (double)g->nz * g->nx > 1.0e9) return LSM_ERR_ARG;
    return LSM_OK;
}

#define LSM_CHECK(expr)                       \
    do {                                      \
        cudaError_t e_ = (expr);              \
        if (e_ != cudaSuccess) return LSM_ERR_CUDA; \
    } while (0)

// Upload geometry / frequencies and build s_ref and the coefficient tables in the workspace.
enum TableOrder { TABLES_SWEEP = 0, TABLES_GRADIENT = 1, TABLES_NATURAL = 2 };

int prepare(const lsm_grid* g, const float* slowness, const lsm_freqs* f, const lsm_geom* geo, const Layout& L,
            char* ws, cudaStream_t st, const double* sref_override = nullptr, int table_order = TABLES_SWEEP,
            int tile = 0) {
    const size_t nw = (size_t)f->nw;
    // one staging copy of all host arrays (layout identical to the workspace prefix)
    const size_t head = L.sref;
    std::vector<char> host(head, 0);
    std::memcpy(host.data() + L.src, geo->src_ix, (size_t)geo->ns * sizeof(int));
    if (geo->rec_ix) std::memcpy(host.data() + L.rec, geo->rec_ix, (size_t)geo->ns * geo->nrec * sizeof(int));
    std::memcpy(host.data() + L.freq, f->freq_hz, nw * sizeof(float));
    std::memcpy(host.data() + L.wav, f->wavelet, nw * sizeof(float2));
    LSM_CHECK(cudaMemcpyAsync(ws, host.data(), head, cudaMemcpyHostToDevice, st));
    LSM_CHECK(cudaMemsetAsync(ws + L.err, 0, sizeof(int), st));
    if (sref_override) {
        LSM_CHECK(cudaMemcpyAsync(ws + L.sref, sref_override, (size_t)g->nz * sizeof(double), cudaMemcpyDeviceToDevice,
                                  st));
    } else {
        {
            ProfScope prof_(KC_TABLES, st);
            reference_slowness_kernel<<<g->nz, 256, 0, st>>>(slowness, g->nx, g->nz,
                                                             reinterpret_cast<double*>(ws + L.sref));
        }
        count_launch();
        LSM_CHECK(cudaGetLastError());
    }
    TableArgs ta;
    ta.V = tile;
    ta.nx = g->nx;
    ta.nz = g->nz;
    ta.nw = f->nw;
    ta.dx = g->dx;
    ta.dz = g->dz;
    ta.slowness = slowness;
    ta.sref = reinterpret_cast<const double*>(ws + L.sref);
    ta.freq_hz = reinterpret_cast<const float*>(ws + L.freq);
    ta.phi = reinterpret_cast<float2*>(ws + L.phi);
    ta.dss = reinterpret_cast<float2*>(ws + L.dss);
    if (table_order == TABLES_GRADIENT)
        LSM_CHECK(launch_tables_grad(ta, st));
    else if (table_order == TABLES_NATURAL)
        LSM_CHECK(nx_ops(g->nx)->tables_natural(ta, st));
    else
        LSM_CHECK(launch_tables(ta, st));
    return LSM_OK;
}

SweepArgs base_args(const lsm_grid* g, const lsm_freqs* f, const lsm_geom* geo, const Layout& L, char* ws,
                    int tile = 0) {
    SweepArgs a{};
    a.V = tile;
    a.nx = g->nx;
    a.nz = g->nz;
    a.nw = f->nw;
    a.nrec = geo->nrec;
    a.ring = L.ring;
    a.rec_identity = geo->rec_ix == nullptr ? 1 : 0;
    a.src_ix = reinterpret_cast<const int*>(ws + L.src);
    a.rec_ix = geo->rec_ix ? reinterpret_cast<const int*>(ws + L.rec) : nullptr;
    a.wavelet = reinterpret_cast<const float2*>(ws + L.wav);
    a.phi = reinterpret_cast<const float2*>(ws + L.phi);
    a.dss = reinterpret_cast<const float2*>(ws + L.dss);
    a.S = reinterpret_cast<float2*>(ws + L.S);
    a.part = reinterpret_cast<float*>(ws + L.part);
    a.dev_err = reinterpret_cast<int*>(ws + L.err);
    return a;
}

// transform: 0 = register FFT (FP32); otherwise the tensor-core precision variant (TcPrecision)
cudaError_t launch_any(int mode, int transform, SweepArgs& a, int n, int num_sms, cudaStream_t st, int* blocks) {
    if (transform == 0) {
        const SweepShape sh = sweep_shape(a.nx, mode, n, a.nw, num_sms, a.V);
        a.wslots = sh.wslots;
        if (blocks) *blocks = sh.blocks;
        return launch_sweep(mode, a, sh, st);
    }
    const SweepShape sh = tc_shape(a.nx, mode, n, a.nw, num_sms, transform);
    a.wslots = sh.wslots;
    if (blocks) *blocks = sh.blocks;
    return nx_ops(a.nx)->tc_sweep(mode, transform, a, sh, st);
}

// Source wavefields of shots [shot0, shot0 + n) into their ring slots.
cudaError_t run_source(SweepArgs a, int shot0, int n, int num_sms, cudaStream_t st, int transform = 0) {
    a.shot0 = shot0;
    a.nshots = n;
    return launch_any(MODE_SOURCE, transform, a, n, num_sms, st, nullptr);
}

cudaError_t run_forward(SweepArgs a, int shot0, int n, const float* m, float2* dout, int num_sms, cudaStream_t st,
                        int transform = 0, int* blocks = nullptr) {
    a.shot0 = shot0;
    a.nshots = n;
    a.m = m;
    a.dout = dout;
    return launch_any(MODE_FORWARD, transform, a, n, num_sms, st, blocks);
}

// Adjoint sweep into the block partial images; returns the number of partials in *nparts.
cudaError_t run_adjoint(SweepArgs a, int shot0, int n, const float2* din, int num_sms, cudaStream_t st, int* nparts,
                        int transform = 0) {
    a.shot0 = shot0;
    a.nshots = n;
    a.din = din;
    return launch_any(MODE_ADJOINT, transform, a, n, num_sms, st, nparts);
}

// The lateral transform selected by the options of an _ex entry point, and its requirements.
int transform_of(const lsm_solve_options* o, const lsm_grid* g, const lsm_geom* geo, int* transform) {
    *transform = o ? o->transform : LSM_TRANSFORM_FFT;
    if (*transform == LSM_TRANSFORM_FFT) return LSM_OK;
    if (is_tc5(*transform)) {
        if (!nx_ops(g->nx)->has_tc5) return LSM_ERR_UNSUPPORTED_NX;
        if (geo->rec_ix) return LSM_ERR_ARG;  // receivers at every column
        return LSM_OK;
    }
    if (*transform != LSM_TRANSFORM_DFT_BF16X3 && *transform != LSM_TRANSFORM_DFT_FP16X3 &&
        *transform != LSM_TRANSFORM_DFT_BF16X1)
        return LSM_ERR_ARG;
    if (!nx_ops(g->nx)->has_tc) return LSM_ERR_UNSUPPORTED_NX;
    if (geo->rec_ix) return LSM_ERR_ARG;  // the tensor-core variants take receivers at every column
    return LSM_OK;
}

}  // namespace

extern "C" {

size_t lsm_workspace_bytes(const lsm_grid* grid, const lsm_geom* geom, const lsm_freqs* freqs, int nshots, int op) {
    if (validate_common(grid, freqs, geom) != LSM_OK) return 0;
    if (nshots < 1 || nshots > geom->ns) return 0;
    if (op != LSM_OP_FORWARD && op != LSM_OP_ADJOINT && op != LSM_OP_SOLVE && op != LSM_OP_GRADIENT) return 0;
    return make_layout(grid, geom, freqs, nshots, op, num_sms_current()).total;
}

int lsm_forward(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs, const lsm_geom* geom,
                const float* m, float* d_out, int shot0, int nshots, void* workspace, size_t workspace_bytes,
                void* stream) {
    return lsm_forward_ex(grid, slowness, freqs, geom, m, d_out, shot0, nshots, workspace, workspace_bytes, stream,
                          nullptr);
}

int lsm_forward_ex(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs, const lsm_geom* geom,
                   const float* m, float* d_out, int shot0, int nshots, void* workspace, size_t workspace_bytes,
                   void* stream, const lsm_solve_options* options) {
    int rc = validate_common(grid, freqs, geom);
    if (rc != LSM_OK) return rc;
    int transform = 0;
    rc = transform_of(options, grid, geom, &transform);
    if (rc != LSM_OK) return rc;
    if (!aligned16(slowness) || !aligned16(m) || !aligned16(d_out) || !aligned16(workspace)) return LSM_ERR_ARG;
    if (shot0 < 0 || nshots < 1 || shot0 > geom->ns - nshots) return LSM_ERR_ARG;
    const int nsm = num_sms_current();
    const Layout L = make_layout(grid, geom, freqs, nshots, LSM_OP_FORWARD, nsm);
    if (workspace_bytes < L.total) return LSM_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    const int tile = transform ? 0 : chosen_tile(grid->nx, nshots, freqs->nw);
    rc = prepare(grid, slowness, freqs, geom, L, ws, st, nullptr, transform ? TABLES_NATURAL : TABLES_SWEEP, tile);
    if (rc != LSM_OK) return rc;
    SweepArgs a = base_args(grid, freqs, geom, L, ws, tile);
    LSM_CHECK(run_source(a, shot0, nshots, nsm, st, transform));
    LSM_CHECK(run_forward(a, shot0, nshots, m, reinterpret_cast<float2*>(d_out), nsm, st, transform));
    return LSM_OK;
}

int lsm_adjoint(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs, const lsm_geom* geom,
                const float* d, float* m_out, int shot0, int nshots, int accumulate, void* workspace,
                size_t workspace_bytes, void* stream) {
    return lsm_adjoint_ex(grid, slowness, freqs, geom, d, m_out, shot0, nshots, accumulate, workspace,
                          workspace_bytes, stream, nullptr);
}

int lsm_adjoint_ex(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs, const lsm_geom* geom,
                   const float* d, float* m_out, int shot0, int nshots, int accumulate, void* workspace,
                   size_t workspace_bytes, void* stream, const lsm_solve_options* options) {
    int rc = validate_common(grid, freqs, geom);
    if (rc != LSM_OK) return rc;
    int transform = 0;
    rc = transform_of(options, grid, geom, &transform);
    if (rc != LSM_OK) return rc;
    if (!aligned16(slowness) || !aligned16(d) || !aligned16(m_out) || !aligned16(workspace)) return LSM_ERR_ARG;
    if (shot0 < 0 || nshots < 1 || shot0 > geom->ns - nshots) return LSM_ERR_ARG;
    const int nsm = num_sms_current();
    const Layout L = make_layout(grid, geom, freqs, nshots, LSM_OP_ADJOINT, nsm);
    if (workspace_bytes < L.total) return LSM_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    const int tile = transform ? 0 : chosen_tile(grid->nx, nshots, freqs->nw);
    rc = prepare(grid, slowness, freqs, geom, L, ws, st, nullptr, transform ? TABLES_NATURAL : TABLES_SWEEP, tile);
    if (rc != LSM_OK) return rc;
    SweepArgs a = base_args(grid, freqs, geom, L, ws, tile);
    LSM_CHECK(run_source(a, shot0, nshots, nsm, st, transform));
    int nparts = 0;
    LSM_CHECK(run_adjoint(a, shot0, nshots, reinterpret_cast<const float2*>(d), nsm, st, &nparts, transform));
    LSM_CHECK(cg_reduce_image(a.part, nparts, grid->nx * grid->nz, nullptr, 0.f, accumulate ? 1 : 0, m_out,
                              reinterpret_cast<double*>(ws + L.ss), st, nullptr, nullptr, nullptr, nullptr, true));
    return LSM_OK;
}

// ------------------------------------------------------------------ allocation-free adjoint
//
// Scratch for lsm_adjoint_static: a fixed file-scope device array instead of a caller-provided
// workspace.  Every GPU that loads this library holds these LSM_STATIC_SCRATCH_BYTES until the
// process exits.  Host code must not hand `g_static_scratch` itself to a kernel (on the host it
// names a stand-in, not device memory): the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[LSM_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device for work issued to `st`.  The address
// is looked up again on every call made outside a stream capture (so a device reset, after which the
// module and its array are loaded anew, is picked up) and cached per device; a call made while `st`
// is being captured uses the cached address, so the first call on a device must come before any
// capture.
int static_scratch_address(cudaStream_t st, void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return LSM_ERR_CUDA;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return LSM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return LSM_ERR_CUDA;
        }
        g_static_ptr[dev] = p;
    } else if (!g_static_ptr[dev]) {
        return LSM_ERR_CUDA;  // no address looked up outside a capture yet
    }
    *out = g_static_ptr[dev];
    return LSM_OK;
}

}  // namespace

int lsm_adjoint_static(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs, const lsm_geom* geom,
                       const float* d, float* m_out, int shot0, int nshots, int accumulate, void* stream) {
    int rc = validate_common(grid, freqs, geom);
    if (rc != LSM_OK) return rc;
    if (!aligned16(slowness) || !aligned16(d) || !aligned16(m_out)) return LSM_ERR_ARG;
    if (shot0 < 0 || nshots < 1 || shot0 > geom->ns - nshots) return LSM_ERR_ARG;
    const int nsm = num_sms_current();
    const Layout L = make_layout(grid, geom, freqs, nshots, LSM_OP_ADJOINT, nsm);
    if (L.total > (size_t)LSM_STATIC_SCRATCH_BYTES) return LSM_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    void* base = nullptr;
    rc = static_scratch_address(st, &base);
    if (rc != LSM_OK) return rc;
    char* ws = static_cast<char*>(base);
    // the same set-up as lsm_adjoint: the host arrays are first copied into a host buffer owned by
    // this call (so the caller may change or free them as soon as the call returns), then the
    // reference slowness and the coefficient tables are built in the scratch
    const int tile = chosen_tile(grid->nx, nshots, freqs->nw);
    rc = prepare(grid, slowness, freqs, geom, L, ws, st, nullptr, TABLES_SWEEP, tile);
    if (rc != LSM_OK) return rc;
    // every scratch region below is fully written before it is read: nothing needs clearing
    SweepArgs a = base_args(grid, freqs, geom, L, ws, tile);
    LSM_CHECK(run_source(a, shot0, nshots, nsm, st));
    int nparts = 0;
    LSM_CHECK(run_adjoint(a, shot0, nshots, reinterpret_cast<const float2*>(d), nsm, st, &nparts));
    LSM_CHECK(cg_reduce_image(a.part, nparts, grid->nx * grid->nz, nullptr, 0.f, accumulate ? 1 : 0, m_out,
                              reinterpret_cast<double*>(ws + L.ss), st, nullptr, nullptr, nullptr, nullptr, true));
    return LSM_OK;
}

// Arguments of the gradient kernel over shots [shot0, shot0 + nshots) at checkpoint stride c: the
// checkpoint rows of every item, then its segment rows, in the layout's gradient region.
static GradArgs grad_args(const lsm_grid* grid, const lsm_freqs* freqs, const lsm_geom* geom, const Layout& L,
                          char* ws, int shot0, int nshots, int c) {
    GradArgs ga{};
    ga.nx = grid->nx;
    ga.nz = grid->nz;
    ga.nw = freqs->nw;
    ga.nrec = geom->nrec;
    ga.shot0 = shot0;
    ga.nshots = nshots;
    ga.rec_identity = geom->rec_ix == nullptr ? 1 : 0;
    ga.ckpt_every = c;
    ga.dz = grid->dz;
    ga.src_ix = reinterpret_cast<const int*>(ws + L.src);
    ga.rec_ix = geom->rec_ix ? reinterpret_cast<const int*>(ws + L.rec) : nullptr;
    ga.wavelet = reinterpret_cast<const float2*>(ws + L.wav);
    ga.freq_hz = reinterpret_cast<const float*>(ws + L.freq);
    ga.phi = reinterpret_cast<const float2*>(ws + L.phi);
    ga.dss = reinterpret_cast<const float2*>(ws + L.dss);
    const size_t items = (size_t)nshots * freqs->nw;
    const size_t ncp = (size_t)((grid->nz + c - 1) / c);
    ga.ckpt = reinterpret_cast<float2*>(ws + L.ckpt);
    ga.seg = ga.ckpt + items * 2 * ncp * grid->nx;
    ga.park = ga.seg + items * (2 * (size_t)std::min(c, grid->nz) + 1) * grid->nx;
    ga.part_m = reinterpret_cast<float*>(ws + L.part);
    ga.part_s = reinterpret_cast<float*>(ws + L.part_s);
    return ga;
}

int lsm_born_gradient(const lsm_grid* grid, const float* slowness, const double* sref, const lsm_freqs* freqs,
                      const lsm_geom* geom, const float* m, const float* g, float* d_out, float* grad_m, float* grad_s,
                      int shot0, int nshots, void* workspace, size_t workspace_bytes, void* stream) {
    int rc = validate_common(grid, freqs, geom);
    if (rc != LSM_OK) return rc;
    if (!aligned16(slowness) || !aligned16(m) || !aligned16(workspace)) return LSM_ERR_ARG;
    if (sref && ((uintptr_t)sref & 7u)) return LSM_ERR_ARG;
    if (g && !aligned16(g)) return LSM_ERR_ARG;
    if (d_out && !aligned16(d_out)) return LSM_ERR_ARG;
    if (grad_m && !aligned16(grad_m)) return LSM_ERR_ARG;
    if (grad_s && !aligned16(grad_s)) return LSM_ERR_ARG;
    if (!g && !d_out) return LSM_ERR_ARG;
    if (shot0 < 0 || nshots < 1 || shot0 > geom->ns - nshots) return LSM_ERR_ARG;
    if (g && !gradient_nx_supported(grid->nx)) return LSM_ERR_UNSUPPORTED_NX;
    const int nsm = num_sms_current();
    const Layout L = make_layout(grid, geom, freqs, nshots, LSM_OP_GRADIENT, nsm);
    if (workspace_bytes < L.total) return LSM_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    if (!g) {
        // modelling only: the sweep kernels with the given reference slowness
        rc = prepare(grid, slowness, freqs, geom, L, ws, st, sref, TABLES_SWEEP);
        if (rc != LSM_OK) return rc;
        SweepArgs a = base_args(grid, freqs, geom, L, ws);
        LSM_CHECK(run_source(a, shot0, nshots, nsm, st));
        LSM_CHECK(run_forward(a, shot0, nshots, m, reinterpret_cast<float2*>(d_out), nsm, st));
        return LSM_OK;
    }
    rc = prepare(grid, slowness, freqs, geom, L, ws, st, sref, TABLES_GRADIENT);
    if (rc != LSM_OK) return rc;
    GradArgs ga = grad_args(grid, freqs, geom, L, ws, shot0, nshots,
                            ckpt_stride(grid->nx, grid->nz, nshots, freqs->nw));
    ga.m = m;
    ga.g = reinterpret_cast<const float2*>(g);
    ga.dout = reinterpret_cast<float2*>(d_out);
    const SweepShape sh = gradient_launch_shape(grid->nx, grid->nz, nshots, freqs->nw, nsm);
    ga.wslots = sh.wslots;
    LSM_CHECK(launch_gradient(ga, sh, st));
    const int n = grid->nx * grid->nz;
    double* ssp = reinterpret_cast<double*>(ws + L.ss);
    if (grad_m) LSM_CHECK(cg_reduce_image(ga.part_m, sh.blocks, n, nullptr, 0.f, 0, grad_m, ssp, st));
    if (grad_s) LSM_CHECK(cg_reduce_image(ga.part_s, sh.blocks, n, nullptr, 0.f, 0, grad_s, ssp, st));
    return LSM_OK;
}

// ------------------------------------------------------------------ lsm_autotune

// Mean time of `reps` launches of one sweep shape (after one untimed launch), in ms.
static cudaError_t time_shape(int mode, int transform, SweepArgs a, const SweepShape& sh, cudaStream_t st,
                              cudaEvent_t e0, cudaEvent_t e1, int reps, double* ms) {
    auto launch = [&]() -> cudaError_t {
        a.wslots = sh.wslots;
        if (transform == 0) return launch_sweep(mode, a, sh, st);
        return nx_ops(a.nx)->tc_sweep(mode, transform, a, sh, st);
    };
    cudaError_t e = launch();
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(e0, st)) != cudaSuccess) return e;
    for (int i = 0; i < reps; ++i)
        if ((e = launch()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return e;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
    float t = 0.f;
    if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) return e;
    *ms = (double)t / reps;
    return cudaSuccess;
}

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

int lsm_autotune(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs, const lsm_geom* geom,
                 int nshots, const lsm_solve_options* options, void* workspace, size_t workspace_bytes, void* stream,
                 lsm_tune_report* report) {
    int rc = validate_common(grid, freqs, geom);
    if (rc != LSM_OK) return rc;
    if (!aligned16(slowness) || !aligned16(workspace)) return LSM_ERR_ARG;
    if (nshots < 1 || nshots > geom->ns) return LSM_ERR_ARG;
    int transform = 0;
    rc = transform_of(options, grid, geom, &transform);
    if (rc != LSM_OK) return rc;
    const int nsm = num_sms_current();
    const Layout L = make_layout(grid, geom, freqs, nshots, LSM_OP_SOLVE, nsm);
    if (workspace_bytes < L.total) return LSM_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    const int nx = grid->nx, nw = freqs->nw;
    // FFT tiles to try: the default, and the alternative where one exists (register FFTs only)
    int tiles[2] = {0, 0};
    int ntiles = 1;
    if (transform == 0 && nx_ops(nx)->alt) tiles[ntiles++] = nx_ops(nx)->alt->points_per_thread;
    // forget earlier choices for this problem, so that the set-up below runs the heuristic shapes
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (int ti = 0; ti < ntiles; ++ti)
            for (int mode = 0; mode < 3; ++mode) g_tune.erase(tune_key(nx, mode, transform, nshots, nw, tiles[ti]));
        if (transform == 0) g_tile.erase(TileKey{current_device(), nx, nshots, nw});
    }
    EventPair ev;
    LSM_CHECK(cudaEventCreate(&ev.a));
    LSM_CHECK(cudaEventCreate(&ev.b));
    const int modes[3] = {MODE_SOURCE, MODE_ADJOINT, MODE_FORWARD};
    lsm_tune_entry entries[2][3] = {};
    double tile_ms[2] = {0.0, 0.0};  // best A + best A^T of each tile
    for (int ti = 0; ti < ntiles; ++ti) {
        const int tile = tiles[ti];
        rc = prepare(grid, slowness, freqs, geom, L, ws, st, nullptr, transform ? TABLES_NATURAL : TABLES_SWEEP,
                     tile);
        if (rc != LSM_OK) return rc;
        SweepArgs a = base_args(grid, freqs, geom, L, ws, tile);
        a.shot0 = 0;
        a.nshots = nshots;
        a.m = reinterpret_cast<const float*>(ws + L.p);
        a.dout = reinterpret_cast<float2*>(ws + L.q);
        a.din = reinterpret_cast<const float2*>(ws + L.r);
        const size_t nd = (size_t)nshots * nw * geom->nrec;
        LSM_CHECK(cudaMemsetAsync(ws + L.p, 0, (size_t)nx * grid->nz * sizeof(float), st));
        LSM_CHECK(cudaMemsetAsync(ws + L.r, 0, nd * sizeof(float2), st));
        LSM_CHECK(run_source(a, 0, nshots, nsm, st, transform));  // the ring the A and A^T sweeps read
        for (int mi = 0; mi < 3; ++mi) {
            const int mode = modes[mi];
            if (is_tc5(transform)) {
                // one fixed launch shape: timed for the report, nothing recorded
                const SweepShape sh = tc5_shape(nx, nshots, nw);
                double ms = 0.0;
                LSM_CHECK(time_shape(mode, transform, a, sh, st, ev.a, ev.b, 3, &ms));
                entries[ti][mi] = lsm_tune_entry{sh.warps, sh.warps, 1, ms, ms};
                continue;
            }
            const SweepShape h = transform ? tc_shape_heuristic(nx, mode, nshots, nw, nsm)
                                           : sweep_shape_heuristic(nx, mode, nshots, nw, nsm, tile);
            const int maxw = transform ? 7 : sweep_max_warps(nx, mode, nshots, nw, tile);
            // the adjoint keeps at most the heuristic's number of blocks (partial images in the layout)
            const int minw = mode == MODE_ADJOINT ? h.warps : 1;
            int best_w = h.warps, ncand = 0;
            double best_ms = 0.0, h_ms = 0.0;
            for (int w = minw; w <= maxw; ++w) {
                const SweepShape sh = transform ? tc_shape_for(nx, mode, nshots, nw, w)
                                                : sweep_shape_for(nx, mode, nshots, nw, w, tile);
                if (sh.smem > 227 * 1024) continue;
                double ms = 0.0;
                LSM_CHECK(time_shape(mode, transform, a, sh, st, ev.a, ev.b, 3, &ms));
                ++ncand;
                if (w == h.warps) h_ms = ms;
                if (ncand == 1 || ms < best_ms) {
                    best_ms = ms;
                    best_w = w;
                }
            }
            {
                std::lock_guard<std::mutex> lock(g_tune_mu);
                g_tune[tune_key(nx, mode, transform, nshots, nw, tile)] = best_w;
            }
            entries[ti][mi] = lsm_tune_entry{best_w, h.warps, ncand, best_ms, h_ms};
            if (mode != MODE_SOURCE) tile_ms[ti] += best_ms;
        }
    }
    int pick = 0;
    if (ntiles > 1 && tile_ms[1] < tile_ms[0]) pick = 1;
    if (transform == 0) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tile[TileKey{current_device(), nx, nshots, nw}] = tiles[pick];
    }
    if (report) {
        report->source = entries[pick][0];
        report->adjoint = entries[pick][1];
        report->forward = entries[pick][2];
        report->points_per_thread = tiles[pick] ? tiles[pick] : nx_ops(nx)->points_per_thread;
        report->default_points_per_thread = nx_ops(nx)->points_per_thread;
        report->tiles = ntiles;
        report->tile_ms = tile_ms[pick];
        report->default_tile_ms = tile_ms[0];
    }
    LSM_CHECK(cudaStreamSynchronize(st));
    return LSM_OK;
}

int lsm_set_fft_tile(int nx, int nshots, int nw, int points_per_thread) {
    const NxOps* ops = nx_ops(nx);
    if (!ops) return LSM_ERR_UNSUPPORTED_NX;
    if (nshots < 1 || nw < 1) return LSM_ERR_ARG;
    const NxOps* t = fft_ops(nx, points_per_thread);
    if (!t) return LSM_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tile[TileKey{current_device(), nx, nshots, nw}] = t == ops ? 0 : points_per_thread;
    return LSM_OK;
}

int lsm_fft_tiles(int nx, int* tiles, int cap) {
    const NxOps* ops = nx_ops(nx);
    if (!ops) return 0;
    int n = 0;
    if (tiles && cap > n) tiles[n] = ops->points_per_thread;
    ++n;
    if (ops->alt) {
        if (tiles && cap > n) tiles[n] = ops->alt->points_per_thread;
        ++n;
    }
    return n;
}

int lsm_tcgen05_shape(int nx, int nshots, int nw, int* items, int* threads, int* blocks, int* wslots,
                      size_t* smem_bytes) {
    const NxOps* ops = nx_ops(nx);
    if (!ops || !ops->has_tc5) return LSM_ERR_UNSUPPORTED_NX;
    if (nshots < 1 || nw < 1) return LSM_ERR_ARG;
    const SweepShape sh = tc5_shape(nx, nshots, nw);
    if (items) *items = ops->tc5_items;
    if (threads) *threads = sh.warps * 32;
    if (blocks) *blocks = sh.blocks;
    if (wslots) *wslots = sh.wslots;
    if (smem_bytes) *smem_bytes = sh.smem;
    return LSM_OK;
}

void lsm_autotune_reset(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
    g_tile.clear();
    g_ckpt_tune.clear();
}

int lsm_autotune_gradient(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs, const lsm_geom* geom,
                          int nshots, void* workspace, size_t workspace_bytes, void* stream,
                          lsm_ckpt_tune_report* report) {
    int rc = validate_common(grid, freqs, geom);
    if (rc != LSM_OK) return rc;
    if (!aligned16(slowness) || !aligned16(workspace)) return LSM_ERR_ARG;
    if (nshots < 1 || nshots > geom->ns) return LSM_ERR_ARG;
    if (!gradient_nx_supported(grid->nx)) return LSM_ERR_UNSUPPORTED_NX;
    const int nsm = num_sms_current();
    const Layout L = make_layout(grid, geom, freqs, nshots, LSM_OP_GRADIENT, nsm);
    if (workspace_bytes < L.total) return LSM_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    const int nx = grid->nx, nz = grid->nz, nw = freqs->nw;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_ckpt_tune.erase(ckpt_key(nx, nz, nshots, nw));
    }
    rc = prepare(grid, slowness, freqs, geom, L, ws, st, nullptr, TABLES_GRADIENT);
    if (rc != LSM_OK) return rc;
    LSM_CHECK(cudaMemsetAsync(ws + L.tune_m, 0, (size_t)nx * nz * sizeof(float), st));
    LSM_CHECK(cudaMemsetAsync(ws + L.tune_g, 0, (size_t)nshots * nw * geom->nrec * sizeof(float2), st));
    const SweepShape h = gradient_shape(nx, nshots, nw, nsm);
    const int wmin = gradient_min_warps(nx, nshots, nw, nsm);
    EventPair ev;
    LSM_CHECK(cudaEventCreate(&ev.a));
    LSM_CHECK(cudaEventCreate(&ev.b));
    const int def = std::min(LSM_CHECKPOINT_EVERY, nz);
    int strides[sizeof(kCkptStrides) / sizeof(int) + 1];
    int nstrides = 0;
    for (int i = 0; i <= (int)(sizeof(kCkptStrides) / sizeof(int)); ++i) {
        // the default first, then the candidates (strides above nz act as nz and are timed once)
        const int c = std::min(i == 0 ? LSM_CHECKPOINT_EVERY : kCkptStrides[i - 1], nz);
        bool seen = false;
        for (int k = 0; k < nstrides; ++k) seen = seen || strides[k] == c;
        if (!seen) strides[nstrides++] = c;
    }
    GradTune best{def, h.warps};
    int ncand = 0;
    double best_ms = 0.0, def_ms = 0.0;
    for (int w = h.warps; w >= wmin; --w) {
        const SweepShape sh = gradient_shape_for(nx, nshots, nw, w);
        for (int k = 0; k < nstrides; ++k) {
            const int c = strides[k];
            GradArgs ga = grad_args(grid, freqs, geom, L, ws, 0, nshots, c);
            ga.m = reinterpret_cast<const float*>(ws + L.tune_m);
            ga.g = reinterpret_cast<const float2*>(ws + L.tune_g);
            ga.wslots = sh.wslots;
            LSM_CHECK(launch_gradient(ga, sh, st));  // untimed first launch
            LSM_CHECK(cudaEventRecord(ev.a, st));
            constexpr int reps = 3;
            for (int r = 0; r < reps; ++r) LSM_CHECK(launch_gradient(ga, sh, st));
            LSM_CHECK(cudaEventRecord(ev.b, st));
            LSM_CHECK(cudaEventSynchronize(ev.b));
            float t = 0.f;
            LSM_CHECK(cudaEventElapsedTime(&t, ev.a, ev.b));
            const double ms = (double)t / reps;
            ++ncand;
            if (c == def && w == h.warps) def_ms = ms;
            if (ncand == 1 || ms < best_ms) {
                best_ms = ms;
                best = GradTune{c, w};
            }
        }
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_ckpt_tune[ckpt_key(nx, nz, nshots, nw)] = best;
    }
    if (report) {
        report->stride = best.stride;
        report->default_stride = def;
        report->warps = best.warps;
        report->default_warps = h.warps;
        report->candidates = ncand;
        report->ms = best_ms;
        report->default_ms = def_ms;
    }
    LSM_CHECK(cudaStreamSynchronize(st));
    return LSM_OK;
}

int lsm_num_windows(int ns, int K, int slide) {
    if (ns < 1 || K < 1 || K > ns || slide < 1) return 0;
    const int regular = (ns - K) / slide + 1;
    const int last = (regular - 1) * slide;
    return regular + (last + K < ns ? 1 : 0);
}

static int window_start(int k, int ns, int K, int slide) {
    const int regular = (ns - K) / slide + 1;
    return k < regular ? k * slide : ns - K;
}

// The CG iterations of a window as one CUDA graph: a test node (cg_loop_test without advance)
// followed by a conditional WHILE node whose body is one iteration -- q = A p, ||q||^2, the m and r
// updates, s = A^T r - lambda m, the p update -- and the advancing test.  The sweeps read the
// window start from the workspace (shot0_dev), so one instantiation serves every window of a call.
struct CgGraph {
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int body_launches = 0;
    bool capturing = false;
    CgGraph() = default;
    CgGraph(const CgGraph&) = delete;
    CgGraph& operator=(const CgGraph&) = delete;
    ~CgGraph() {
        if (capturing) {
            cudaGraph_t body = nullptr;  // owned by the conditional node
            cudaStreamEndCapture(cs, &body);
            g_capturing = false;
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
    }
};

// A window solve sharded over ranks by frequency: every rank runs the operator on its own
// frequencies and the hooks sum, over the ranks, the images of A^T and ||q||^2 (the only places where
// a sum over (shot, frequency) items meets the model-space vectors, which every rank keeps whole).
struct ShardHooks {
    lsm_allreduce_fn fn;
    void* ctx;
    float* img;        // [nz][nx] this rank's image before the sum
    double* qq_total;  // ||q||^2 of this rank's items, then of all ranks' items
};

static cudaError_t shard_sum(const ShardHooks* h, void* buf, size_t count, int is_double, cudaStream_t st) {
    return h->fn(h->ctx, buf, count, is_double, st) == 0 ? cudaSuccess : cudaErrorUnknown;
}

// s = A^T(...) - lambda m over all ranks from this rank's block partial images: the partials are
// summed into the rank's image, the images are summed over the ranks, and the rest of the reduction
// (m += alpha p when p and state are given, s = image - lambda m, the ||s||^2 partials) runs on the
// sum as a single partial.
static cudaError_t shard_reduce_image(const ShardHooks* h, const float* part, int nparts, int n, float* m, float lam,
                                      float* s, double* ss, cudaStream_t st, const float* minv, double* sz,
                                      const float* p = nullptr, const CgState* state = nullptr) {
    cudaError_t e = cg_reduce_image(part, nparts, n, nullptr, 0.f, 0, h->img, nullptr, st);
    if (e == cudaSuccess) e = shard_sum(h, h->img, (size_t)n, 0, st);
    if (e == cudaSuccess) e = cg_reduce_image(h->img, 1, n, m, lam, 0, s, ss, st, minv, sz, p, state);
    return e;
}

struct CgVectors {
    float *m, *p, *s;
    float2 *r, *q;
    double *qq, *pp, *ss, *sz;
    const float* minv;
    CgState* state;
    size_t nd;
    int n;
    double lambda;
    const ShardHooks* shard;  // null: one rank
};

// One CG iteration after a window's set-up (Eq. 11): q = A p; alpha = gamma / (||q||^2 + lambda
// ||p||^2); m += alpha p; r -= alpha q; s = A^T r - lambda m; beta; p = s (or M^-1 s) + beta p.
// gi is the current gamma slot (-1: the state's, for the device-driven loop; cg_update_p then
// writes slot state->gi ^ 1).  With the register-FFT sweeps the vector work rides in the sweeps
// and the image reduction: the forward sweep emits the |q|^2 partials, the adjoint sweep forms alpha
// and applies r -= alpha q as it loads r, and the reduction applies m += alpha p, so an iteration
// is four launches.  The tensor-core transforms run the separate vector kernels (six launches).
static cudaError_t cg_iteration(SweepArgs a, int start, int K, int nsm, int transform, const CgVectors& v, int gi,
                                cudaStream_t st) {
    int nparts = 0;
    cudaError_t e;
    if (transform == 0) {
        int nqq = 0;
        SweepArgs af = a;
        af.qq_part = v.qq;
        e = run_forward(af, start, K, v.p, v.q, nsm, st, 0, &nqq);
        SweepArgs aa = a;
        aa.r_io = v.r;
        aa.dq = v.q;
        aa.qq_in = v.qq;
        aa.nqq = nqq;
        if (v.shard) {  // alpha needs ||q||^2 over every rank's items
            if (e == cudaSuccess) e = cg_sum_partials(v.qq, nqq, v.shard->qq_total, st);
            if (e == cudaSuccess) e = shard_sum(v.shard, v.shard->qq_total, 1, 1, st);
            aa.qq_in = v.shard->qq_total;
            aa.nqq = 1;
        }
        aa.pp_in = v.pp;
        aa.npp = kRedBlocks;
        aa.cg_gi = gi;
        aa.lam = v.lambda;
        aa.cg = v.state;
        if (e == cudaSuccess) e = run_adjoint(aa, start, K, nullptr, nsm, st, &nparts, 0);
        if (e == cudaSuccess && v.shard)
            e = shard_reduce_image(v.shard, a.part, nparts, v.n, v.m, (float)v.lambda, v.s, v.ss, st, v.minv, v.sz, v.p,
                                   v.state);
        else if (e == cudaSuccess)
            e = cg_reduce_image(a.part, nparts, v.n, v.m, (float)v.lambda, 0, v.s, v.ss, st, v.minv, v.sz, v.p,
                                v.state, true);
    } else {
        e = run_forward(a, start, K, v.p, v.q, nsm, st, transform);
        if (e == cudaSuccess) e = cg_norm2_c64(v.q, v.nd, v.qq, st);
        if (e == cudaSuccess) e = cg_update_mr(v.m, v.p, v.n, v.r, v.q, v.nd, v.qq, v.pp, v.lambda, v.state, gi, st);
        if (e == cudaSuccess) e = run_adjoint(a, start, K, v.r, nsm, st, &nparts, transform);
        if (e == cudaSuccess)
            e = cg_reduce_image(a.part, nparts, v.n, v.m, (float)v.lambda, 0, v.s, v.ss, st, v.minv, v.sz);
    }
    if (e == cudaSuccess)
        e = cg_update_p(v.p, v.s, v.n, v.ss, 0, v.state, gi, gi < 0 ? -1 : gi ^ 1, v.pp, st, v.minv, v.sz);
    return e;
}

static int build_cg_graph(CgGraph& G, SweepArgs a, int K, int nsm, int transform, const CgVectors& v) {
    LSM_CHECK(cudaStreamCreateWithFlags(&G.cs, cudaStreamNonBlocking));
    LSM_CHECK(cudaGraphCreate(&G.graph, 0));
    cudaGraphConditionalHandle handle = 0;
    LSM_CHECK(cudaGraphConditionalHandleCreate(&handle, G.graph, 0, cudaGraphCondAssignDefault));
    CgState* state = v.state;
    int no_advance = 0;
    void* test_args[] = {&state, &handle, &no_advance};
    cudaKernelNodeParams kp;
    cg_loop_test_node_params(&kp, test_args);
    cudaGraphNode_t test0 = nullptr, loop = nullptr;
    LSM_CHECK(cudaGraphAddKernelNode(&test0, G.graph, nullptr, 0, &kp));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    LSM_CHECK(cudaGraphAddNode(&loop, G.graph, &test0, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];

    LSM_CHECK(cudaStreamBeginCaptureToGraph(G.cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    G.capturing = true;
    g_capturing = true;
    g_captured_launches = 0;
    cudaError_t e = cg_iteration(a, 0, K, nsm, transform, v, -1, G.cs);
    if (e == cudaSuccess) e = cg_loop_test(v.state, handle, 1, G.cs);
    g_capturing = false;
    G.body_launches = g_captured_launches;
    cudaGraph_t out = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(G.cs, &out);
    G.capturing = false;
    if (e != cudaSuccess || e_end != cudaSuccess) return LSM_ERR_CUDA;
    LSM_CHECK(cudaGraphInstantiate(&G.exec, G.graph, 0));
    return LSM_OK;
}

// One line's prepared sliding-window solve: its arguments, workspace layout and device vectors.
struct SolveCtx {
    const lsm_grid* grid = nullptr;
    const lsm_freqs* freqs = nullptr;
    const lsm_geom* geom = nullptr;
    const float2* dall = nullptr;
    double lambda = 0.0, cg_tol = 0.0, precond_eps = 0.0;
    int K = 0, slide = 0, max_iter = 0, first = 0, last = 0;
    float* m = nullptr;
    lsm_window_stats* stats = nullptr;
    int stats_cap = 0;
    Layout L{};
    char* ws = nullptr;
    SweepArgs a{};
    int transform = 0, nsm = 0, n = 0, graph_opt = 0;
    size_t nd = 0, shot_stride = 0;
    float *p = nullptr, *s = nullptr, *minv = nullptr;
    float2 *r = nullptr, *q = nullptr;
    double *qq = nullptr, *pp = nullptr, *ss = nullptr, *sz = nullptr;
    CgState* state = nullptr;
    int* shot0_dev = nullptr;
    WindowRecord* wrec = nullptr;
    int* halt = nullptr;
};

// Argument checks, the coefficient tables and the device vectors of one line's solve; c.first ==
// c.last when the call has no window to solve.  `sharded`: the caller sums A^T images and ||q||^2
// over ranks (plain CG, FP32 FFT transforms, host-driven loop).
static int solve_init(SolveCtx& c, const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs,
                      const lsm_geom* geom, const float* d, double lambda, int K, int slide, double cg_tol,
                      int max_iter, int first_window, int n_windows, float* m_inout, lsm_window_stats* stats,
                      int stats_cap, void* workspace, size_t workspace_bytes, cudaStream_t st,
                      const lsm_solve_options* options, bool sharded) {
    int rc = validate_common(grid, freqs, geom);
    if (rc != LSM_OK) return rc;
    if (!aligned16(slowness) || !aligned16(d) || !aligned16(m_inout) || !aligned16(workspace)) return LSM_ERR_ARG;
    if (!std::isfinite(lambda) || lambda < 0.0 || !std::isfinite(cg_tol) || cg_tol < 0.0 || max_iter < 0)
        return LSM_ERR_ARG;
    const int precond = options ? options->preconditioner : LSM_PRECOND_NONE;
    c.precond_eps = options ? options->precond_eps : 0.0;
    if (precond != LSM_PRECOND_NONE && precond != LSM_PRECOND_ILLUMINATION) return LSM_ERR_ARG;
    if (precond == LSM_PRECOND_ILLUMINATION && !(c.precond_eps > 0.0 && std::isfinite(c.precond_eps)))
        return LSM_ERR_ARG;
    rc = transform_of(options, grid, geom, &c.transform);
    if (rc != LSM_OK) return rc;
    if (sharded && (c.transform != 0 || precond != LSM_PRECOND_NONE)) return LSM_ERR_ARG;
    c.graph_opt = options ? options->cuda_graph : 0;
    if (c.graph_opt > LSM_CUDA_GRAPH_SOLVE) return LSM_ERR_ARG;
    const int ns = geom->ns;
    const int nwin = lsm_num_windows(ns, K, slide);
    if (nwin == 0) return LSM_ERR_ARG;
    if (first_window < 0 || first_window > nwin) return LSM_ERR_ARG;
    if (stats_cap < 0 || (stats_cap > 0 && !stats)) return LSM_ERR_ARG;
    c.grid = grid;
    c.freqs = freqs;
    c.geom = geom;
    c.dall = reinterpret_cast<const float2*>(d);
    c.lambda = lambda;
    c.cg_tol = cg_tol;
    c.K = K;
    c.slide = slide;
    c.max_iter = max_iter;
    c.first = first_window;
    c.last = n_windows <= 0 ? nwin : std::min(nwin, first_window + n_windows);
    c.m = m_inout;
    c.stats = stats;
    c.stats_cap = stats_cap;
    c.nsm = num_sms_current();
    c.L = make_layout(grid, geom, freqs, K, LSM_OP_SOLVE, c.nsm);
    if (workspace_bytes < c.L.total) return LSM_ERR_WORKSPACE;
    if (c.first == c.last) return LSM_OK;

    c.ws = static_cast<char*>(workspace);
    const int tile = c.transform ? 0 : chosen_tile(grid->nx, K, freqs->nw);
    rc = prepare(grid, slowness, freqs, geom, c.L, c.ws, st, nullptr, c.transform ? TABLES_NATURAL : TABLES_SWEEP,
                 tile);
    if (rc != LSM_OK) return rc;
    c.a = base_args(grid, freqs, geom, c.L, c.ws, tile);
    char* ws = c.ws;
    const Layout& L = c.L;
    c.n = grid->nx * grid->nz;
    c.nd = (size_t)K * freqs->nw * geom->nrec;
    c.shot_stride = (size_t)freqs->nw * geom->nrec;
    c.p = reinterpret_cast<float*>(ws + L.p);
    c.s = reinterpret_cast<float*>(ws + L.s);
    c.r = reinterpret_cast<float2*>(ws + L.r);
    c.q = reinterpret_cast<float2*>(ws + L.q);
    c.qq = reinterpret_cast<double*>(ws + L.qq);
    c.pp = reinterpret_cast<double*>(ws + L.pp);
    c.ss = reinterpret_cast<double*>(ws + L.ss);
    c.state = reinterpret_cast<CgState*>(ws + L.state);
    c.shot0_dev = reinterpret_cast<int*>(ws + L.ctrl);
    c.wrec = reinterpret_cast<WindowRecord*>(ws + L.wrec);
    c.halt = reinterpret_cast<int*>(ws + L.halt);
    c.minv = precond == LSM_PRECOND_ILLUMINATION ? reinterpret_cast<float*>(ws + L.minv) : nullptr;
    c.sz = c.minv ? reinterpret_cast<double*>(ws + L.sz) : nullptr;
    return LSM_OK;
}

// The set-up of window k (Eq. 10, Eq. 11): the source wavefields of the shots that enter the window
// (the rank-`slide` update of the ring; prev_start is the previous window's first shot, -1 for none),
// the illumination preconditioner when asked, b = A_k^T d_k and ||b||^2, r = d_k - A_k m,
// s = A_k^T r - lambda m, p = s (or M^-1 s) and gamma (slot 0).  *start_out: the window's first shot.
static cudaError_t window_setup(const SolveCtx& c, int k, int prev_start, const ShardHooks* shard, cudaStream_t st,
                                int* start_out) {
    const int start = window_start(k, c.geom->ns, c.K, c.slide);
    *start_out = start;
    const float2* dk = c.dall + (size_t)start * c.shot_stride;
    const int new_from = prev_start < 0 ? start : std::max(start, prev_start + c.K);
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
        return e == cudaSuccess;
    };
    if (new_from < start + c.K && !ok(run_source(c.a, new_from, start + c.K - new_from, c.nsm, st, c.transform)))
        return e;
    if (c.minv) {
        // the ring now holds exactly this window's source wavefields
        float* illum = reinterpret_cast<float*>(c.ws + c.L.illum);
        float* bmax = reinterpret_cast<float*>(c.ws + c.L.bmax);
        if (!ok(cg_illumination(c.a.S, c.K * c.freqs->nw, c.n, illum, bmax, st))) return e;
        if (!ok(cg_precond_finalize(illum, c.n, bmax, c.precond_eps, c.minv, st))) return e;
    }
    int nparts = 0;
    const float lamf = (float)c.lambda;
    if (!ok(cg_zero_state(c.state, st))) return e;
    // b = A_k^T d_k  ->  ||b||^2
    if (!ok(run_adjoint(c.a, start, c.K, dk, c.nsm, st, &nparts, c.transform))) return e;
    if (shard) ok(shard_reduce_image(shard, c.a.part, nparts, c.n, nullptr, 0.f, c.s, c.ss, st, nullptr, nullptr));
    else ok(cg_reduce_image(c.a.part, nparts, c.n, nullptr, 0.f, 0, c.s, c.ss, st, nullptr, nullptr, nullptr, nullptr,
                            true));
    if (!ok(cg_store_sum(c.ss, c.state, st))) return e;
    // r = d_k - A_k m
    if (!ok(run_forward(c.a, start, c.K, c.m, c.q, c.nsm, st, c.transform))) return e;
    if (!ok(cg_residual(dk, c.q, c.r, c.nd, st))) return e;
    // s = A_k^T r - lambda m ; p = s ; gamma = ||s||^2
    if (!ok(run_adjoint(c.a, start, c.K, c.r, c.nsm, st, &nparts, c.transform))) return e;
    if (shard) ok(shard_reduce_image(shard, c.a.part, nparts, c.n, c.m, lamf, c.s, c.ss, st, c.minv, c.sz));
    else ok(cg_reduce_image(c.a.part, nparts, c.n, c.m, lamf, 0, c.s, c.ss, st, c.minv, c.sz, nullptr, nullptr, true));
    if (e != cudaSuccess) return e;
    ok(cg_update_p(c.p, c.s, c.n, c.ss, 1, c.state, 1, 0, c.pp, st, c.minv, c.sz));
    return e;
}

static CgVectors cg_vectors(const SolveCtx& c, const ShardHooks* shard) {
    return CgVectors{c.m, c.p, c.s, c.r, c.q, c.qq, c.pp, c.ss, c.sz, c.minv, c.state, c.nd, c.n, c.lambda, shard};
}

// The sliding-window solve of one prepared line, window after window, with the host-driven CG loop
// or each window's CG iterations as one CUDA graph; `shard` set: this rank's share of a solve
// sharded by frequency (host-driven loop).
static int window_loop(SolveCtx& c, cudaStream_t st, const ShardHooks* shard) {
    // cuda_graph > 0: graph; < 0: host-driven loop; 0: graph unless the sweeps are being event-timed
    const bool use_graph = !shard && (c.graph_opt > 0 || (c.graph_opt == 0 && !profiling_sweeps()));
    CgGraph graph;
    int prev_start = -1;
    for (int k = c.first; k < c.last; ++k) {
        const auto t0 = std::chrono::steady_clock::now();
        int start = 0;
        LSM_CHECK(window_setup(c, k, prev_start, shard, st, &start));
        prev_start = start;
        CgState hs;
        double rel = 0.0, rel0 = 0.0;
        int nfwd = 1, nadj = 2, it = 0, gi = 0;
        bool broke = false;
        if (use_graph) {
            // the iterations run on the device; the host waits once for the window
            if (!graph.exec) {
                SweepArgs ag = c.a;
                ag.shot0_dev = c.shot0_dev;
                const int rc = build_cg_graph(graph, ag, c.K, c.nsm, c.transform, cg_vectors(c, nullptr));
                if (rc != LSM_OK) return rc;
            }
            LSM_CHECK(cg_loop_setup(c.state, c.shot0_dev, start, c.max_iter, c.cg_tol, st));
            LSM_CHECK(cudaGraphLaunch(graph.exec, st));
            LSM_CHECK(cudaMemcpyAsync(&hs, c.state, sizeof(CgState), cudaMemcpyDeviceToHost, st));
            LSM_CHECK(cudaStreamSynchronize(st));
            it = hs.iter;
            rel0 = hs.rel0;
            rel = hs.rel;
            broke = hs.breakdown != 0;
            nfwd += it;
            nadj += it;
            count_launch(1 + graph.body_launches * it);
        } else {
            LSM_CHECK(cudaMemcpyAsync(&hs, c.state, sizeof(CgState), cudaMemcpyDeviceToHost, st));
            LSM_CHECK(cudaStreamSynchronize(st));
            const double bnorm = std::sqrt(hs.bb);
            rel = bnorm > 0.0 ? std::sqrt(hs.ss[gi]) / bnorm : 0.0;
            rel0 = rel;
            broke = hs.breakdown != 0;
            const CgVectors v = cg_vectors(c, shard);
            while (!broke && it < c.max_iter && !(rel <= c.cg_tol)) {
                LSM_CHECK(cg_iteration(c.a, start, c.K, c.nsm, c.transform, v, gi, st));
                gi ^= 1;
                ++nfwd;
                ++nadj;
                ++it;
                LSM_CHECK(cudaMemcpyAsync(&hs, c.state, sizeof(CgState), cudaMemcpyDeviceToHost, st));
                LSM_CHECK(cudaStreamSynchronize(st));
                broke = hs.breakdown != 0;
                rel = bnorm > 0.0 ? std::sqrt(hs.ss[gi]) / bnorm : 0.0;
            }
        }
        const auto t1 = std::chrono::steady_clock::now();
        if (c.transform != 0) {
            // a tcgen05 sweep whose bounded wait on the tensor core ran out leaves NaN and this flag
            int err = 0;
            LSM_CHECK(cudaMemcpyAsync(&err, c.ws + c.L.err, sizeof(int), cudaMemcpyDeviceToHost, st));
            LSM_CHECK(cudaStreamSynchronize(st));
            if (err) return LSM_ERR_TIMEOUT;
        }
        const int idx = k - c.first;
        if (idx < c.stats_cap) {
            c.stats[idx].start = start;
            c.stats[idx].iters = it;
            c.stats[idx].rel_res0 = rel0;
            c.stats[idx].rel_res = rel;
            c.stats[idx].n_forward = nfwd;
            c.stats[idx].n_adjoint = nadj;
            c.stats[idx].ms = std::chrono::duration<float, std::milli>(t1 - t0).count();
        }
        if (broke) return LSM_ERR_BREAKDOWN;
    }
    return LSM_OK;
}

// Whole solves as one CUDA graph (cuda_graph = LSM_CUDA_GRAPH_SOLVE): per line a chain of windows --
// the window's set-up launches (a child graph), the loop test and a conditional WHILE node whose body
// is one CG iteration and the advancing test, then a node that records the window's outcome in the
// workspace -- and the lines as independent branches of the same graph, so one launch runs every
// window of every line with no host thread and no host wait in between.  The kernels of each window,
// and their order, are those of the per-window graph, so results and iteration counts are identical.
struct SolveGraph {
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    SolveGraph() = default;
    SolveGraph(const SolveGraph&) = delete;
    SolveGraph& operator=(const SolveGraph&) = delete;
    ~SolveGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
    }
};

// Launches issued by `fn(stream)` recorded as a new graph (owned by the caller); *launches counts them.
static int capture_new_graph(cudaStream_t cs, cudaGraph_t* out, int* launches,
                             const std::function<cudaError_t(cudaStream_t)>& fn) {
    *out = nullptr;
    LSM_CHECK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    g_captured_launches = 0;
    const cudaError_t e = fn(cs);
    g_capturing = false;
    if (launches) *launches = g_captured_launches;
    cudaGraph_t g = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess || e_end != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return LSM_ERR_CUDA;
    }
    *out = g;
    return LSM_OK;
}

// `sub` added to `top` as a child-graph node after `dep` (none when null); `sub` is destroyed.
static int add_child(cudaGraph_t top, cudaGraph_t sub, cudaGraphNode_t dep, cudaGraphNode_t* node) {
    const cudaError_t e = cudaGraphAddChildGraphNode(node, top, dep ? &dep : nullptr, dep ? 1 : 0, sub);
    cudaGraphDestroy(sub);
    return e == cudaSuccess ? LSM_OK : LSM_ERR_CUDA;
}

struct ChainLaunches {
    std::vector<int> setup;  // per window: set-up launches (with the loop set-up)
    int body = 0;            // launches of one CG iteration with its test
};

static int add_solve_chain(SolveGraph& G, SolveCtx& c, ChainLaunches& nl) {
    SweepArgs ag = c.a;
    ag.shot0_dev = c.shot0_dev;
    const CgVectors v = cg_vectors(c, nullptr);
    cudaGraphNode_t prev = nullptr;
    int prev_start = -1;
    for (int k = c.first; k < c.last; ++k) {
        // (1) set-up of the window (before the first one, the halt flag is cleared)
        cudaGraph_t sub = nullptr;
        int start = 0, nset = 0;
        int rc = capture_new_graph(G.cs, &sub, &nset, [&](cudaStream_t cs) {
            cudaError_t e = k == c.first ? cudaMemsetAsync(c.halt, 0, sizeof(int), cs) : cudaSuccess;
            if (e == cudaSuccess) e = window_setup(c, k, prev_start, nullptr, cs, &start);
            if (e == cudaSuccess) e = cg_loop_setup(c.state, c.shot0_dev, start, c.max_iter, c.cg_tol, cs, c.halt);
            return e;
        });
        if (rc != LSM_OK) return rc;
        nl.setup.push_back(nset);
        cudaGraphNode_t n_setup = nullptr;
        rc = add_child(G.graph, sub, prev, &n_setup);
        if (rc != LSM_OK) return rc;
        prev_start = start;
        // (2) the CG iterations: the loop test, then WHILE { one iteration; the advancing test }
        cudaGraphConditionalHandle handle = 0;
        LSM_CHECK(cudaGraphConditionalHandleCreate(&handle, G.graph, 0, cudaGraphCondAssignDefault));
        CgState* state = c.state;
        int no_advance = 0;
        void* test_args[] = {&state, &handle, &no_advance};
        cudaKernelNodeParams kp;
        cg_loop_test_node_params(&kp, test_args);
        cudaGraphNode_t test0 = nullptr, loop = nullptr;
        LSM_CHECK(cudaGraphAddKernelNode(&test0, G.graph, &n_setup, 1, &kp));
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        LSM_CHECK(cudaGraphAddNode(&loop, G.graph, &test0, nullptr, 1, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];  // owned by the conditional node
        LSM_CHECK(cudaStreamBeginCaptureToGraph(G.cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        g_capturing = true;
        g_captured_launches = 0;
        cudaError_t e = cg_iteration(ag, 0, c.K, c.nsm, c.transform, v, -1, G.cs);
        if (e == cudaSuccess) e = cg_loop_test(c.state, handle, 1, G.cs);
        g_capturing = false;
        nl.body = g_captured_launches;
        cudaGraph_t captured = nullptr;
        const cudaError_t e_end = cudaStreamEndCapture(G.cs, &captured);
        if (e != cudaSuccess || e_end != cudaSuccess) return LSM_ERR_CUDA;
        // (3) the window's outcome (a breakdown halts the later windows: they run no iterations)
        WindowRecord* rec = c.wrec + (k - c.first);
        rc = capture_new_graph(G.cs, &sub, nullptr,
                               [&](cudaStream_t cs) { return cg_record_window(c.state, rec, c.halt, cs); });
        if (rc != LSM_OK) return rc;
        rc = add_child(G.graph, sub, loop, &prev);
        if (rc != LSM_OK) return rc;
    }
    return LSM_OK;
}

// Prepared solves run as one graph launch on `st`; every line's statistics are filled and its status
// written to status[i].
static int run_solve_graph(const std::vector<SolveCtx*>& lines, cudaStream_t st, std::vector<int>& status) {
    SolveGraph G;
    LSM_CHECK(cudaStreamCreateWithFlags(&G.cs, cudaStreamNonBlocking));
    LSM_CHECK(cudaGraphCreate(&G.graph, 0));
    std::vector<ChainLaunches> nl(lines.size());
    for (size_t i = 0; i < lines.size(); ++i) {
        const int rc = add_solve_chain(G, *lines[i], nl[i]);
        if (rc != LSM_OK) return rc;
    }
    LSM_CHECK(cudaGraphInstantiate(&G.exec, G.graph, 0));
    LSM_CHECK(cudaGraphLaunch(G.exec, st));
    LSM_CHECK(cudaStreamSynchronize(st));
    for (size_t i = 0; i < lines.size(); ++i) {
        SolveCtx& c = *lines[i];
        const int nwin = c.last - c.first;
        std::vector<WindowRecord> rec((size_t)nwin);
        LSM_CHECK(cudaMemcpy(rec.data(), c.wrec, (size_t)nwin * sizeof(WindowRecord), cudaMemcpyDeviceToHost));
        int err = 0;
        if (c.transform != 0) LSM_CHECK(cudaMemcpy(&err, c.ws + c.L.err, sizeof(int), cudaMemcpyDeviceToHost));
        int rc = err ? LSM_ERR_TIMEOUT : LSM_OK;
        for (int w = 0; w < nwin; ++w) {
            count_launch(nl[i].setup[(size_t)w] + 2 + nl[i].body * rec[(size_t)w].iters);
            if (rc != LSM_OK) continue;
            if (w < c.stats_cap) {
                lsm_window_stats& s = c.stats[w];
                s.start = window_start(c.first + w, c.geom->ns, c.K, c.slide);
                s.iters = rec[(size_t)w].iters;
                s.rel_res0 = rec[(size_t)w].rel0;
                s.rel_res = rec[(size_t)w].rel;
                s.n_forward = 1 + s.iters;
                s.n_adjoint = 2 + s.iters;
                s.ms = 0.f;  // the windows of a whole-solve graph are not timed one by one
            }
            if (rec[(size_t)w].breakdown) rc = LSM_ERR_BREAKDOWN;
        }
        status[i] = rc;
    }
    return LSM_OK;
}

int rls_window_solve_ex(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs, const lsm_geom* geom,
                        const float* d, double lambda, int K, int slide, double cg_tol, int max_iter,
                        int first_window, int n_windows, float* m_inout, lsm_window_stats* stats, int stats_cap,
                        void* workspace, size_t workspace_bytes, void* stream, const lsm_solve_options* options) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    SolveCtx c;
    int rc = solve_init(c, grid, slowness, freqs, geom, d, lambda, K, slide, cg_tol, max_iter, first_window,
                        n_windows, m_inout, stats, stats_cap, workspace, workspace_bytes, st, options, false);
    if (rc != LSM_OK || c.first == c.last) return rc;
    if (c.graph_opt == LSM_CUDA_GRAPH_SOLVE) {
        std::vector<int> status(1, LSM_OK);
        rc = run_solve_graph({&c}, st, status);
        return rc != LSM_OK ? rc : status[0];
    }
    return window_loop(c, st, nullptr);
}

int rls_window_solve_sharded(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs,
                             const lsm_geom* geom, const float* d, double lambda, int K, int slide, double cg_tol,
                             int max_iter, int first_window, int n_windows, float* m_inout, lsm_window_stats* stats,
                             int stats_cap, void* workspace, size_t workspace_bytes, void* stream,
                             lsm_allreduce_fn allreduce, void* allreduce_ctx) {
    if (!allreduce) return LSM_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    SolveCtx c;
    const int rc = solve_init(c, grid, slowness, freqs, geom, d, lambda, K, slide, cg_tol, max_iter, first_window,
                              n_windows, m_inout, stats, stats_cap, workspace, workspace_bytes, st, nullptr, true);
    if (rc != LSM_OK || c.first == c.last) return rc;
    ShardHooks hooks{allreduce, allreduce_ctx, reinterpret_cast<float*>(c.ws + c.L.img),
                     reinterpret_cast<double*>(c.ws + c.L.qqt)};
    return window_loop(c, st, &hooks);
}

int rls_window_solve(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs, const lsm_geom* geom,
                     const float* d, double lambda, int K, int slide, double cg_tol, int max_iter, int first_window,
                     int n_windows, float* m_inout, lsm_window_stats* stats, int stats_cap, void* workspace,
                     size_t workspace_bytes, void* stream) {
    return rls_window_solve_ex(grid, slowness, freqs, geom, d, lambda, K, slide, cg_tol, max_iter, first_window,
                               n_windows, m_inout, stats, stats_cap, workspace, workspace_bytes, stream, nullptr);
}

int rls_multi_line_solve(lsm_line* lines, int nlines, const lsm_solve_options* options) {
    if (!lines || nlines < 1) return LSM_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return LSM_ERR_CUDA;
    }
    if (options && options->cuda_graph == LSM_CUDA_GRAPH_SOLVE) {
        // every line prepared on its own stream, then all of them in one graph launched on the first
        std::vector<SolveCtx> ctx((size_t)nlines);
        std::vector<SolveCtx*> todo;
        std::vector<int> idx;
        for (int i = 0; i < nlines; ++i) {
            lsm_line& l = lines[i];
            cudaStream_t st = reinterpret_cast<cudaStream_t>(l.stream);
            l.status = solve_init(ctx[(size_t)i], &l.grid, l.slowness, &l.freqs, &l.geom, l.d, l.lambda, l.K, l.slide,
                                  l.cg_tol, l.max_iter, 0, 0, l.m_inout, l.stats, l.stats_cap, l.workspace,
                                  l.workspace_bytes, st, options, false);
            if (l.status == LSM_OK && cudaStreamSynchronize(st) != cudaSuccess) l.status = LSM_ERR_CUDA;
            if (l.status == LSM_OK && ctx[(size_t)i].first < ctx[(size_t)i].last) {
                todo.push_back(&ctx[(size_t)i]);
                idx.push_back(i);
            }
        }
        if (!todo.empty()) {
            std::vector<int> status(todo.size(), LSM_OK);
            const int rc = run_solve_graph(todo, reinterpret_cast<cudaStream_t>(lines[0].stream), status);
            for (size_t j = 0; j < todo.size(); ++j) lines[idx[j]].status = rc != LSM_OK ? rc : status[j];
        }
    } else {
        auto solve_line = [&](int i) {
            lsm_line& l = lines[i];
            if (cudaSetDevice(dev) != cudaSuccess) {
                cudaGetLastError();
                l.status = LSM_ERR_CUDA;
                return;
            }
            l.status = rls_window_solve_ex(&l.grid, l.slowness, &l.freqs, &l.geom, l.d, l.lambda, l.K, l.slide,
                                           l.cg_tol, l.max_iter, 0, 0, l.m_inout, l.stats, l.stats_cap, l.workspace,
                                           l.workspace_bytes, l.stream, options);
        };
        std::vector<std::thread> workers;
        workers.reserve((size_t)nlines);
        for (int i = 1; i < nlines; ++i) workers.emplace_back(solve_line, i);
        solve_line(0);
        for (auto& w : workers) w.join();
    }
    for (int i = 0; i < nlines; ++i)
        if (lines[i].status != LSM_OK) return lines[i].status;
    return LSM_OK;
}

const char* lsm_status_string(int status) {
    switch (status) {
        case LSM_OK: return "ok";
        case LSM_ERR_ARG: return "invalid argument";
        case LSM_ERR_CUDA: return "CUDA error";
        case LSM_ERR_WORKSPACE: return "workspace too small";
        case LSM_ERR_BREAKDOWN: return "CG breakdown (step length undefined)";
        case LSM_ERR_TIMEOUT: return "device wait timed out";
        case LSM_ERR_UNSUPPORTED_NX:
            return "unsupported nx: 16, 32, 64, 128, 256, 512, 1024, 48, 96, 192, 384, 768, 80, 160, 320, 640, "
                   "112, 224, 448, 896 (gradients: powers of two up to 512)";
        default: return "unknown status";
    }
}

unsigned long long lsm_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void lsm_profile_start(void) { lsm_profile_start_classes(~0u); }

void lsm_profile_start_classes(unsigned class_mask) {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    g_prof_mask = class_mask;
    for (auto& r : g_prof) {
        g_event_pool.push_back(r.begin);
        g_event_pool.push_back(r.end);
    }
    g_prof.clear();
    g_prof_on = true;
}

int lsm_profile_stop(lsm_profile* out) {
    g_prof_on = false;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    if (out) std::memset(out, 0, sizeof(*out));
    int rc = LSM_OK;
    for (auto& r : g_prof) {
        if (cudaEventSynchronize(r.end) != cudaSuccess) {
            rc = LSM_ERR_CUDA;
            continue;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.begin, r.end) != cudaSuccess) {
            rc = LSM_ERR_CUDA;
            continue;
        }
        if (out && r.cls >= 0 && r.cls < LSM_NUM_KCLASSES) {
            out->launches[r.cls] += 1;
            out->ms[r.cls] += ms;
        }
    }
    cudaGetLastError();
    for (auto& r : g_prof) {
        g_event_pool.push_back(r.begin);
        g_event_pool.push_back(r.end);
    }
    g_prof.clear();
    return rc;
}

}  // extern "C"
