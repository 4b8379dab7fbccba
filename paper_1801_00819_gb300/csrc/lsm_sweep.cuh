// Depth-sweep kernels of the shot-profile split-step operator (Eq. 1, Eq. 2; Examples section).
//
// One (shot, frequency) item is held in registers by T = N / V threads for the whole depth loop;
// a warp holds 32 / T items and a block `ipb` consecutive items in frequency-major order, so a
// block's items span only a few frequencies.  Per depth row j every item runs one step
//   P_j u   = D_j . F^-1 (Phi_j . F u)                    (source and forward sweeps)
//   P_j^H u = F^-1 (conj(Phi_j) . F (conj(D_j) . u))      (adjoint sweep)
// with Phi_j (already divided by nx and stored in the FFT's output order) and D_j taken from
// precomputed coefficient tables shared by every shot at that frequency.  The block stages the
// Phi and D rows of its frequencies for the next depth (and, in the forward sweep, the model row)
// into double-buffered shared memory with cp.async while it computes the current depth, and each
// item requests its next source-wavefield row into registers one step early, so no global-memory
// latency sits on the critical path of a step.  One block barrier per depth hands the staged
// buffers over.
//
//   MODE_SOURCE : S_0 = W(w) delta(x - x_s); store S_j, S_{j+1} = P_j S_j.
//   MODE_ADJOINT: R_0 = injected data; image_j += Re conj(S_j) R_j; R_{j+1} = P_j^H R_j.
//                 The block sums its items' image rows every depth and writes one partial row
//                 per block; a separate pass adds the partials in a fixed order, so the image is
//                 deterministic.
//   MODE_FORWARD: U <- P_j U_{j+1} + S_j m_j from j = nz-1 up to 0; record U_0.
#pragma once

#include "lsm_async.cuh"
#include "lsm_cg.h"
#include "lsm_fft.cuh"
#include "lsm_grad.cuh"
#include "lsm_internal.h"
#include "lsm_tc.cuh"
#include "lsm_tc5.cuh"

namespace lsm {

// ------------------------------------------------------------------ one depth step

// a natural-order row (S, data) into the register layout
template <int N, int V>
__device__ __forceinline__ void load_row(float2 (&v)[V], const float2* __restrict__ row, int t, bool ok) {
    using P = Plan<N, V>;
#pragma unroll
    for (int r = 0; r < V; ++r) v[r] = ok ? __ldcs(row + P::xpos(t, r)) : make_float2(0.f, 0.f);
}

// w[0] = sum of w[0 .. H) as a fixed tree: halves of ceil(H/2) are added elementwise until one remains
template <int H, int V>
__device__ __forceinline__ void tree_sum(float (&w)[V]) {
    if constexpr (H > 1) {
        constexpr int HALF = (H + 1) / 2;
#pragma unroll
        for (int r = 0; r < H - HALF; ++r) w[r] += w[r + HALF];
        tree_sum<HALF, V>(w);
    }
}

// sum of part[0 .. n) in a fixed order (thread i takes entries i, i + blockDim, ...; then a fixed
// shuffle tree and the warps in order), returned to every thread of the block; sh: blockDim / 32
// doubles of shared scratch, free on entry
__device__ __forceinline__ double sweep_sum_partials(const double* __restrict__ part, int n, double* sh) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();  // the scratch's previous readers are done
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
    return tot;
}

// Whether a step issues the caller's loads for the step (mid) once its first stage has parked the
// thread's registers in shared memory: two-stage plans of 1024 points, whose steps are long enough
// to hide the loads' latency from there.
template <int N, int V>
constexpr bool step_loads_mid() {
    return Plan<N, V>::NS == 2 && Plan<N, V>::NB(0) == 1 && N >= 1024;
}

// phi, dss: this depth's rows staged in shared memory; mid(): see step_loads_mid (otherwise the
// caller issues its loads before the step and passes a no-op)
template <int N, int V, class Mid>
__device__ __forceinline__ void step_down(float2 (&v)[V], const Twiddles<N, V>& tw, float2* buf, int t,
                                          const float2* phi, const float2* dss, Mid&& mid) {
    constexpr int T = Plan<N, V>::T;
    if constexpr (pair_plan<N, V>()) {
        phase_shift_pair<false>(v, tw, buf, t, phi, mid);
    } else if constexpr (Plan<N, V>::NS == 2 && Plan<N, V>::NB(0) == 1) {
        phase_shift_two_stage<N, V, false, true>(v, tw, buf, t, phi, mid);
    } else {
        mid();
        fft_forward<N, V>(v, tw, buf, t);
#pragma unroll
        for (int r = 0; r < V; ++r) v[r] = cmul(v[r], phi[t + T * r]);
        fft_inverse<N, V>(v, tw, buf, t);
    }
#pragma unroll
    for (int r = 0; r < V; ++r) v[r] = cmul(v[r], dss[Plan<N, V>::xpos(t, r)]);
}

// mid(): the adjoint sweep's load of the next source row, issued inside the step where
// step_loads_mid holds (A^T at 1024 x 512: 2.71 -> 2.63 ms) and before it otherwise, which leaves the
// whole step to hide its latency (at 512 and 256 points the later load measured 5 and 15 % slower).
template <int N, int V, class Mid>
__device__ __forceinline__ void step_down_adjoint(float2 (&v)[V], const Twiddles<N, V>& tw, float2* buf, int t,
                                                  const float2* phi, const float2* dss, Mid&& mid) {
    constexpr int T = Plan<N, V>::T;
    constexpr bool kTwoStage = Plan<N, V>::NS == 2 && Plan<N, V>::NB(0) == 1;
    constexpr bool kLoadMid = step_loads_mid<N, V>();
    if constexpr (!kLoadMid) mid();
#pragma unroll
    for (int r = 0; r < V; ++r) v[r] = cmulc(v[r], dss[Plan<N, V>::xpos(t, r)]);
    if constexpr (pair_plan<N, V>()) {
        phase_shift_pair<true>(v, tw, buf, t, phi, [] {});
    } else if constexpr (kLoadMid) {
        phase_shift_two_stage<N, V, true, true>(v, tw, buf, t, phi, mid);
    } else if constexpr (kTwoStage) {
        phase_shift_two_stage<N, V, true, false>(v, tw, buf, t, phi, [] {});
    } else {
        fft_forward<N, V>(v, tw, buf, t);
#pragma unroll
        for (int r = 0; r < V; ++r) v[r] = cmulc(v[r], phi[t + T * r]);
        fft_inverse<N, V>(v, tw, buf, t);
    }
}

// ------------------------------------------------------------------ shared-memory layout

// Threads per block the kernel is compiled for: 24 or more points per thread need up to ~250
// registers, which leaves room for 8 warps per SM; 16 points per thread fit 16 warps at 128
// registers, except with 32 threads per item and 16 to 20 points per thread: the pair plan (the
// alternative tile at nx = 512) is compiled for 14 warps, one block per SM for a window whose items
// fill 13 to 14 warps per SM, at 128 registers (a register-file quarter then holds four warps), and
// the alternative tile at 640, a deeper plan whose twiddles need more registers, for 12 warps at up
// to 168 registers.
template <int N, int V>
constexpr int sweep_max_threads() {
    return V >= 24 ? 256 : pair_plan<N, V>() ? 448 : (V >= 16 && N / V == 32 ? 384 : 512);
}

// Image rows of the adjoint: each warp writes SPW rows per depth (its items' imaging terms; with
// more than two items per warp they are first summed pairwise by shuffles), at a row stride of
// SLAB floats that puts a warp's two rows on different banks.
template <int N, int V>
struct ImageRows {
    static constexpr int T = Plan<N, V>::T;
    static constexpr int IPW = 32 / T;
    static constexpr int SPW = IPW >= 2 ? 2 : 1;
    static constexpr int SLAB = N + (SPW > 1 ? (T >= 4 ? T : 4) : 0);
    static_assert(SLAB % 4 == 0, "image rows are summed as float4");
};

// Depth rows per staging buffer: the source sweep stages the coefficient rows of two depth steps at
// a time, so its blocks meet at a barrier every other step (0.91 -> 0.86 ms on a 512 x 256 window
// of 16 shots x 128 frequencies); the forward sweep measured no gain from it, and the adjoint sums
// its image rows across the block at every depth.  Above 512 columns the doubled staging would
// leave room for only half the warps per block, so the source sweep stages one step at a time.
constexpr int stage_depths(int mode, int n) { return mode == MODE_SOURCE && n <= 512 ? 2 : 1; }

// Bytes of dynamic shared memory for a block of `warps` warps whose items span at most `wslots`
// frequencies (mirrored on the host by sweep_shape): per-item exchange buffers, the block's
// double-buffered staging of [depth steps][wslots][Phi row, D row] plus one model row per step,
// and the adjoint's double-buffered image rows.
template <int N, int V>
constexpr size_t sweep_smem_bytes(int warps, int wslots, int mode) {
    const bool adjoint = mode == MODE_ADJOINT;
    using IR = ImageRows<N, V>;
    return (size_t)Plan<N, V>::TAB * sizeof(float2) +
           (size_t)warps * (32 / Plan<N, V>::T) * Plan<N, V>::BUF * sizeof(float2) +
           2 * (size_t)stage_depths(mode, N) * ((size_t)wslots * 2 * N * sizeof(float2) + (size_t)N * sizeof(float)) +
           (adjoint ? (size_t)2 * warps * IR::SPW * IR::SLAB * sizeof(float) : 0);
}

template <int N, int V, int MODE>
__global__ void __launch_bounds__(sweep_max_threads<N, V>()) sweep_kernel(const SweepArgs a) {
    using P = Plan<N, V>;
    constexpr int T = P::T;
    constexpr int IPW = 32 / T;
    extern __shared__ float4 smem_f4[];
    float2* const tab = reinterpret_cast<float2*>(smem_f4);  // twiddle table (mixed-radix plans)
    float2* smem = tab + P::TAB;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int t = lane % T;
    const int sub = lane / T;
    const int ipb = nwarps * IPW;
    const int nitems = a.nshots * a.nw;
    // items are frequency-major: item = iw * nshots + ishot
    const int item = blockIdx.x * ipb + warp * IPW + sub;
    const bool ok = item < nitems;
    const int w_first = min(blockIdx.x * ipb, nitems - 1) / a.nshots;
    const int w_last = (min((blockIdx.x + 1) * ipb, nitems) - 1) / a.nshots;
    const int nslots = w_last - w_first + 1;  // <= a.wslots
    const int iw = ok ? item / a.nshots : w_first;
    const int ishot = ok ? item - iw * a.nshots : 0;
    const int shot = (a.shot0_dev ? __ldg(a.shot0_dev) : a.shot0) + ishot;
    const int slot = shot % a.ring;
    const int wslot = iw - w_first;
    const int nz = a.nz;

    // shared memory: exchange buffers | staging [2][DEP][wslots][2][N] float2 + [2][DEP][N] float |
    // images.  Depth step k (0 .. nz-2) reads staging buffer (k / DEP) % 2, slot k % DEP.
    constexpr int DEP = stage_depths(MODE, N);
    float2* buf = smem + (warp * IPW + sub) * P::BUF;
    float2* stage = smem + ipb * P::BUF;
    const int stage_buf = a.wslots * 2 * N;  // float2 per staging slot (coefficients)
    float* mstage = reinterpret_cast<float*>(stage + 2 * DEP * stage_buf);  // [2][DEP][N]
    float* img = mstage + 2 * DEP * N;                                        // [2][nwarps * SPW][SLAB]

    Twiddles<N, V> tw;
    init_twiddles<N, V>(tw, t, tab);
    if constexpr (P::TW_SMEM) __syncthreads();

    float2* Sitem = a.S + ((size_t)slot * a.nw + iw) * (size_t)nz * N;
    float2 v[V];

    // the whole block stages the Phi and D rows of depth `row` for its frequencies into
    // staging slot b (and the model row when asked), as one cp.async group per thread
    auto stage_rows = [&](int row, int b, bool with_model) {
        constexpr int CH = N / 2;  // 16-byte chunks per complex row
        float2* dst = stage + b * stage_buf;
        const int total = nslots * 2 * CH;
        // the coefficient rows are read once per launch: evict-first in L2, so that they do not
        // push out the partial image rows the image reduction reads back after the adjoint sweep
        const unsigned long long pol = l2_evict_first_policy();
        for (int c = threadIdx.x; c < total; c += blockDim.x) {
            const int sl = c / (2 * CH);
            const int rem = c - sl * 2 * CH;
            const int which = rem / CH;
            const int ch = rem - which * CH;
            const float2* src = (which ? a.dss : a.phi) + ((size_t)(w_first + sl) * nz + row) * N + 2 * ch;
            cp_async16_stream(dst + (sl * 2 + which) * N + 2 * ch, src, pol);
        }
        if (with_model) {
            for (int c = threadIdx.x; c < N / 4; c += blockDim.x)
                cp_async16(mstage + b * N + 4 * c, a.m + (size_t)row * N + 4 * c);
        }
        cp_async_commit();
    };
    auto phi_of = [&](int b) -> const float2* { return stage + b * stage_buf + (wslot * 2) * N; };
    auto dss_of = [&](int b) -> const float2* { return stage + b * stage_buf + (wslot * 2 + 1) * N; };
    auto slot_of = [&](int k) { return ((k / DEP) & 1) * DEP + k % DEP; };  // staging slot of step k

    if constexpr (MODE == MODE_SOURCE) {
        const int xs = ok ? __ldg(a.src_ix + shot) : -1;
        const float2 w = ok ? __ldg(a.wavelet + iw) : make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < V; ++r) v[r] = (P::xpos(t, r) == xs) ? w : make_float2(0.f, 0.f);
        // step k propagates with row k; steps are staged DEP at a time, one group ahead
        for (int k = 0; k < DEP && k + 1 < nz; ++k) stage_rows(k, slot_of(k), false);
        for (int j = 0; j < nz; ++j) {
            if (ok) {
                float2* row = Sitem + (size_t)j * N;
#pragma unroll
                for (int r = 0; r < V; ++r) __stcs(row + P::xpos(t, r), v[r]);
            }
            if (j + 1 < nz) {
                if (j % DEP == 0) {
                    cp_async_wait_all();
                    __syncthreads();
                    for (int k = j + DEP; k < j + 2 * DEP && k + 1 < nz; ++k) stage_rows(k, slot_of(k), false);
                }
                step_down<N, V>(v, tw, buf, t, phi_of(slot_of(j)), dss_of(slot_of(j)), [] {});
            }
        }
    } else if constexpr (MODE == MODE_ADJOINT) {
        // Inside a CG iteration the residual update r <- r - alpha q (alpha = gamma / (||q||^2 +
        // lambda ||p||^2), Eq. 11) is applied here, as each item loads its data: every block forms
        // alpha from the same partial sums in the same order; a non-positive or non-finite
        // denominator sets the breakdown flag and leaves r as it is.
        const size_t drow_off = ((size_t)ishot * a.nw + iw) * a.nrec;
        float alpha = 0.f;
        bool upd = false;
        float2 qv[V];
        if (a.r_io && a.rec_identity) {
            // r and q are requested before alpha is formed, so their latency hides behind it (and
            // no store to r sits between two loads)
#pragma unroll
            for (int r = 0; r < V; ++r) {
                v[r] = ok ? __ldcs(a.r_io + drow_off + P::xpos(t, r)) : make_float2(0.f, 0.f);
                qv[r] = ok ? __ldcs(a.dq + drow_off + P::xpos(t, r)) : make_float2(0.f, 0.f);
            }
        }
        if (a.r_io) {
            double* sh = reinterpret_cast<double*>(stage);  // scratch until staging starts below
            const double qq = sweep_sum_partials(a.qq_in, a.nqq, sh);
            const double pp = sweep_sum_partials(a.pp_in, a.npp, sh);
            const int gi = a.cg_gi < 0 ? a.cg->gi : a.cg_gi;
            const double gamma = a.cg->gamma[gi];
            const double delta = qq + a.lam * pp;
            const bool bad = !(delta > 0.0) || !isfinite(delta) || !isfinite(gamma);
            const double al = bad ? 0.0 : gamma / delta;
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                a.cg->delta = delta;
                a.cg->alpha = al;
                if (bad) a.cg->breakdown = 1;
            }
            alpha = (float)al;
            upd = !bad;
            __syncthreads();  // every thread has read the scratch
        }
        if (nz > 1) stage_rows(0, 0, false);
        // R_0: data injected at the receivers
        const float2* drow = a.r_io ? nullptr : a.din + drow_off;
        auto r_updated = [&](int rr) -> float2 {  // r[rr] - alpha q[rr], stored back
            float2 x = a.r_io[drow_off + rr];
            if (upd) {
                const float2 y = a.dq[drow_off + rr];
                x.x = fmaf(-alpha, y.x, x.x);
                x.y = fmaf(-alpha, y.y, x.y);
                a.r_io[drow_off + rr] = x;
            }
            return x;
        };
        if (a.rec_identity) {
            if (a.r_io) {
                if (upd && ok) {
#pragma unroll
                    for (int r = 0; r < V; ++r) {
                        v[r].x = fmaf(-alpha, qv[r].x, v[r].x);
                        v[r].y = fmaf(-alpha, qv[r].y, v[r].y);
                        __stcs(a.r_io + drow_off + P::xpos(t, r), v[r]);
                    }
                }
            } else {
                load_row<N, V>(v, drow, t, ok);
            }
        } else {
            __syncwarp();
            for (int x = t; x < P::BUF; x += T) buf[x] = make_float2(0.f, 0.f);
            __syncwarp();
            if (ok) {
                const int* rix = a.rec_ix + (size_t)shot * a.nrec;
                for (int rr = t; rr < a.nrec; rr += T) {
                    const float2 dv = a.r_io ? r_updated(rr) : __ldg(drow + rr);
                    const int x = P::phys(__ldg(rix + rr));
                    atomicAdd(&buf[x].x, dv.x);
                    atomicAdd(&buf[x].y, dv.y);
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < V; ++r) v[r] = buf[P::phys(P::xpos(t, r))];
        }
        float* part = a.part + (size_t)blockIdx.x * nz * N;
        // s holds S_j; the row of depth j+1 is requested after the image rows of depth j are
        // summed, right before the propagation step that hides its HBM latency
        float2 s[V];
        load_row<N, V>(s, Sitem, t, ok);
        for (int j = 0; j < nz; ++j) {
            float c[V];
#pragma unroll
            for (int r = 0; r < V; ++r) c[r] = fmaf(s[r].x, v[r].x, s[r].y * v[r].y);
            using IR = ImageRows<N, V>;
            // with more than two items per warp, sum the items of equal parity (lanes with equal
            // t hold equal x); the two remaining groups write one image row each
#pragma unroll
            for (int off = 2 * T; off < 32; off <<= 1) {
#pragma unroll
                for (int r = 0; r < V; ++r) c[r] += __shfl_xor_sync(0xffffffffu, c[r], off);
            }
            if (sub < IR::SPW) {
                float* slab = img + ((size_t)(j & 1) * nwarps * IR::SPW + warp * IR::SPW + sub) * IR::SLAB;
#pragma unroll
                for (int r = 0; r < V; ++r) slab[P::xpos(t, r)] = c[r];
            }
            if (j + 1 < nz) cp_async_wait_all();
            __syncthreads();  // image rows of depth j and staged rows of depth j are visible
            if (j + 2 < nz) stage_rows(j + 1, (j + 1) & 1, false);
            {
                // the block's partial row: the image rows summed in a fixed order, four columns a thread,
                // stored evict-last in L2 so that the image reduction launched next finds it there
                const int nslab = nwarps * IR::SPW;
                const float4* rows4 = reinterpret_cast<const float4*>(img + (size_t)(j & 1) * nslab * IR::SLAB);
                float4* prow = reinterpret_cast<float4*>(part + (size_t)j * N);
                for (int x4 = threadIdx.x; x4 < N / 4; x4 += blockDim.x) {
                    float4 acc = rows4[x4];
                    for (int w = 1; w < nslab; ++w) {
                        const float4 u4 = rows4[w * (IR::SLAB / 4) + x4];
                        acc.x += u4.x;
                        acc.y += u4.y;
                        acc.z += u4.z;
                        acc.w += u4.w;
                    }
                    st_global_keep_l2(prow + x4, acc);
                }
            }
            if (j + 1 < nz) {
                // S_{j+1} is requested with the propagation step so that its HBM latency hides
                // behind it
                step_down_adjoint<N, V>(v, tw, buf, t, phi_of(j & 1), dss_of(j & 1),
                                        [&] { load_row<N, V>(s, Sitem + (size_t)(j + 1) * N, t, ok); });
            }
        }
    } else {  // MODE_FORWARD
#pragma unroll
        for (int r = 0; r < V; ++r) v[r] = make_float2(0.f, 0.f);
        // step k (k = 0 .. nz-2) propagates with row j = nz-2-k and then adds model row j, both
        // from staging slot slot_of(k); the deepest model row is staged on its own into the
        // first slot of buffer 1, which the steps of that buffer only overwrite after a barrier
        for (int c = threadIdx.x; c < N / 4; c += blockDim.x)
            cp_async16(mstage + DEP * N + 4 * c, a.m + (size_t)(nz - 1) * N + 4 * c);
        cp_async_commit();
        for (int k = 0; k < DEP && k + 1 < nz; ++k) stage_rows(nz - 2 - k, slot_of(k), true);
        for (int j = nz - 1; j >= 0; --j) {
            // request S_j before (or, see step_loads_mid, during) propagating U_{j+1} so the load
            // overlaps the step
            float2 s[V];
            auto load_s = [&] { load_row<N, V>(s, Sitem + (size_t)j * N, t, ok); };
            const int k = nz - 2 - j;  // -1 for the deepest row, which is not propagated
            if (!step_loads_mid<N, V>() || k < 0) load_s();
            if (k < 0 || k % DEP == 0) {
                cp_async_wait_all();
                __syncthreads();
            }
            const float* mrow;
            if (k >= 0) {
                if (k % DEP == 0) {
                    for (int k2 = k + DEP; k2 < k + 2 * DEP && k2 + 1 < nz; ++k2)
                        stage_rows(nz - 2 - k2, slot_of(k2), true);
                }
                if constexpr (step_loads_mid<N, V>())
                    step_down<N, V>(v, tw, buf, t, phi_of(slot_of(k)), dss_of(slot_of(k)), load_s);
                else
                    step_down<N, V>(v, tw, buf, t, phi_of(slot_of(k)), dss_of(slot_of(k)), [] {});
                mrow = mstage + slot_of(k) * N;
            } else {
                mrow = mstage + DEP * N;
            }
#pragma unroll
            for (int r = 0; r < V; ++r) {
                const float mm = mrow[P::xpos(t, r)];
                v[r].x = fmaf(s[r].x, mm, v[r].x);
                v[r].y = fmaf(s[r].y, mm, v[r].y);
            }
        }
        float2* orow = a.dout + ((size_t)ishot * a.nw + iw) * a.nrec;
        if (a.rec_identity) {
            if (ok) {
#pragma unroll
                for (int r = 0; r < V; ++r) orow[P::xpos(t, r)] = v[r];
            }
        } else {
            __syncwarp();
#pragma unroll
            for (int r = 0; r < V; ++r) buf[P::phys(P::xpos(t, r))] = v[r];
            __syncwarp();
            if (ok) {
                const int* rix = a.rec_ix + (size_t)shot * a.nrec;
                for (int rr = t; rr < a.nrec; rr += T) orow[rr] = buf[P::phys(__ldg(rix + rr))];
            }
        }
        if (a.qq_part) {
            // the block's partial sum of |q|^2 over the data it recorded (the CG step length's
            // denominator), in a fixed order: each thread's elements, a shuffle tree, warps in order
            // (a thread's own |q|^2 terms are added as a float32 tree -- relative error at most
            // ceil(log2 V) 2^-24, V <= 56 -- because float64 arithmetic is slow on this part; the sums
            // across threads and warps are float64)
            double e = 0.0;
            if (ok) {
                if (a.rec_identity) {
                    float w[V];
#pragma unroll
                    for (int r = 0; r < V; ++r) w[r] = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
                    tree_sum<V, V>(w);
                    e = (double)w[0];
                } else {
                    const int* rix = a.rec_ix + (size_t)shot * a.nrec;
                    for (int rr = t; rr < a.nrec; rr += T) {
                        const float2 u = buf[P::phys(__ldg(rix + rr))];
                        e += (double)u.x * u.x + (double)u.y * u.y;
                    }
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
            double* sh = reinterpret_cast<double*>(stage);
            cp_async_wait_all();
            __syncthreads();  // every warp is past its last staged row
            if (lane == 0) sh[warp] = e;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int w = 0; w < nwarps; ++w) tot += sh[w];
                a.qq_part[blockIdx.x] = tot;
            }
        }
    }
}

// Coefficient tables for every (frequency, depth row): Phi_j / nx in the FFT output order of
// Plan<N, V>, and D_j in natural order.  Phase arguments are formed in float64 and reduced to
// [-pi, pi] before the float32 sin / cos.
template <int N, int V, bool NATURAL = false>
__global__ void tables_kernel(const TableArgs a) {
    using P = Plan<N, V>;
    const size_t total = (size_t)a.nw * a.nz * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(idx % N);
        const size_t row = idx / N;
        const int j = (int)(row % a.nz);
        const int iw = (int)(row / a.nz);
        const double omega = 2.0 * kPi * (double)a.freq_hz[iw];
        const double sref = a.sref[j];
        // phase shift at the frequency held by table slot p = r T + t
        {
            const int t = p % P::T, r = p / P::T;
            const int k = NATURAL ? p : P::freq_of_position(P::position_of(t, r));
            const int kk = k < N / 2 ? k : k - N;
            const double kx = fabs(2.0 * kPi * (double)kk / ((double)N * (double)a.dx));
            const double ws = omega * sref;
            const double kz2 = (ws - kx) * (ws + kx);
            float2 ph;
            if (kz2 >= 0.0) {
                double arg = sqrt(kz2) * (double)a.dz;
                arg = remainder(arg, 2.0 * kPi);
                float sn, cs;
                sincosf((float)arg, &sn, &cs);
                ph = make_float2(cs / (float)N, sn / (float)N);
            } else {
                ph = make_float2((float)(exp(-sqrt(-kz2) * (double)a.dz) / (double)N), 0.f);
            }
            a.phi[idx] = ph;
        }
        // split-step correction at column x = p
        {
            const double ds = (double)a.slowness[(size_t)j * N + p] - sref;
            double arg = omega * ds * (double)a.dz;
            arg = remainder(arg, 2.0 * kPi);
            float sn, cs;
            sincosf((float)arg, &sn, &cs);
            a.dss[idx] = make_float2(cs, sn);
        }
    }
}

template <int N, int VV = points_per_thread(N)>
struct Dispatch {
    static constexpr int V = VV;

    static cudaError_t tables(const TableArgs& a, cudaStream_t st) {
        const size_t total = (size_t)a.nw * a.nz * N;
        size_t blocks = (total + 255) / 256;
        if (blocks > 65535u * 8u) blocks = 65535u * 8u;
        ProfScope prof_(KC_TABLES, st);
        tables_kernel<N, V><<<(unsigned)blocks, 256, 0, st>>>(a);
        count_launch();
        return cudaGetLastError();
    }

    template <int MODE>
    static cudaError_t sweep(const SweepArgs& a, const SweepShape& sh, cudaStream_t st) {
        static DeviceOnce configured;
        cudaError_t e = configured.run([] {
            return cudaFuncSetAttribute(sweep_kernel<N, V, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        227 * 1024);
        });
        if (e != cudaSuccess) return e;
        if (sh.smem != sweep_smem_bytes<N, V>(sh.warps, a.wslots, MODE)) return cudaErrorInvalidValue;
        ProfScope prof_(MODE == MODE_SOURCE ? KC_SOURCE : MODE == MODE_ADJOINT ? KC_ADJOINT : KC_FORWARD, st);
        sweep_kernel<N, V, MODE><<<sh.blocks, sh.warps * 32, sh.smem, st>>>(a);
        count_launch();
        return cudaGetLastError();
    }

    static cudaError_t sweep_any(int mode, const SweepArgs& a, const SweepShape& sh, cudaStream_t st) {
        switch (mode) {
            case MODE_SOURCE: return sweep<MODE_SOURCE>(a, sh, st);
            case MODE_ADJOINT: return sweep<MODE_ADJOINT>(a, sh, st);
            default: return sweep<MODE_FORWARD>(a, sh, st);
        }
    }

    template <int MODE>
    static int max_warps_mode() {
        cudaFuncAttributes attr;
        if (cudaFuncGetAttributes(&attr, sweep_kernel<N, V, MODE>) != cudaSuccess) {
            cudaGetLastError();
            return sweep_max_threads<N, V>() / 32;
        }
        int w = attr.maxThreadsPerBlock / 32;
        return w < 1 ? 1 : w;
    }
    static int max_warps(int mode) {
        switch (mode) {
            case MODE_SOURCE: return max_warps_mode<MODE_SOURCE>();
            case MODE_ADJOINT: return max_warps_mode<MODE_ADJOINT>();
            default: return max_warps_mode<MODE_FORWARD>();
        }
    }

    // tensor-core transform variants (every supported nx: N = 16 R2, columns padded to a multiple of 8)
    static constexpr bool kTc = N % 16 == 0 && N <= 1024;

    static cudaError_t tables_natural(const TableArgs& a, cudaStream_t st) {
        const size_t total = (size_t)a.nw * a.nz * N;
        size_t blocks = (total + 255) / 256;
        if (blocks > 65535u * 8u) blocks = 65535u * 8u;
        ProfScope prof_(KC_TABLES, st);
        tables_kernel<N, V, true><<<(unsigned)blocks, 256, 0, st>>>(a);
        count_launch();
        return cudaGetLastError();
    }

    template <int PREC, int MODE>
    static cudaError_t tc_launch(const SweepArgs& a, const SweepShape& sh, cudaStream_t st) {
        if constexpr (kTc) {
            static DeviceOnce configured;
            cudaError_t e = configured.run([] {
                return cudaFuncSetAttribute(tc_sweep_kernel<N, PREC, MODE>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
            });
            if (e != cudaSuccess) return e;
            if (sh.smem != tc_smem_bytes<N>(sh.warps, MODE == MODE_ADJOINT)) return cudaErrorInvalidValue;
            ProfScope prof_(MODE == MODE_SOURCE ? KC_SOURCE : MODE == MODE_ADJOINT ? KC_ADJOINT : KC_FORWARD, st);
            tc_sweep_kernel<N, PREC, MODE><<<sh.blocks, sh.warps * 32, sh.smem, st>>>(a);
            count_launch();
            return cudaGetLastError();
        } else {
            return cudaErrorNotSupported;
        }
    }

    template <int PREC>
    static cudaError_t tc_mode(int mode, const SweepArgs& a, const SweepShape& sh, cudaStream_t st) {
        switch (mode) {
            case MODE_SOURCE: return tc_launch<PREC, MODE_SOURCE>(a, sh, st);
            case MODE_ADJOINT: return tc_launch<PREC, MODE_ADJOINT>(a, sh, st);
            default: return tc_launch<PREC, MODE_FORWARD>(a, sh, st);
        }
    }

    // tcgen05 transform variants (nx = 128, 256, 512, 1024): 8 items per CTA (16 at nx = 128), 128
    // threads (256 at nx = 1024)
    static constexpr bool kTc5 = tc5_width(N);

    template <int PREC, int MODE>
    static cudaError_t tc5_launch(const SweepArgs& a, const SweepShape& sh, cudaStream_t st) {
        if constexpr (kTc5) {
            using S5 = Tc5Shape<N>;
            static DeviceOnce configured;
            cudaError_t e = configured.run([] {
                return cudaFuncSetAttribute(tc5_sweep_kernel<N, PREC, MODE>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTc5MaxDynSmem);
            });
            if (e != cudaSuccess) return e;
            if (sh.smem != tc5_smem_bytes<N>(a.wslots) || sh.smem > kTc5MaxDynSmem || sh.warps != S5::THREADS / 32)
                return cudaErrorInvalidValue;
            ProfScope prof_(MODE == MODE_SOURCE ? KC_SOURCE : MODE == MODE_ADJOINT ? KC_ADJOINT : KC_FORWARD, st);
            tc5_sweep_kernel<N, PREC, MODE><<<sh.blocks, S5::THREADS, sh.smem, st>>>(a);
            count_launch();
            return cudaGetLastError();
        } else {
            return cudaErrorNotSupported;
        }
    }

    template <int PREC>
    static cudaError_t tc5_mode(int mode, const SweepArgs& a, const SweepShape& sh, cudaStream_t st) {
        switch (mode) {
            case MODE_SOURCE: return tc5_launch<PREC, MODE_SOURCE>(a, sh, st);
            case MODE_ADJOINT: return tc5_launch<PREC, MODE_ADJOINT>(a, sh, st);
            default: return tc5_launch<PREC, MODE_FORWARD>(a, sh, st);
        }
    }

    static cudaError_t tc_sweep(int mode, int prec, const SweepArgs& a, const SweepShape& sh, cudaStream_t st) {
        switch (prec) {
            case PREC_BF16X3: return tc_mode<PREC_BF16X3>(mode, a, sh, st);
            case PREC_FP16X3: return tc_mode<PREC_FP16X3>(mode, a, sh, st);
            case PREC_BF16X1: return tc_mode<PREC_BF16X1>(mode, a, sh, st);
            case PREC_FP16X3_TC5: return tc5_mode<PREC_FP16X3_TC5>(mode, a, sh, st);
            case PREC_BF16X3_TC5: return tc5_mode<PREC_BF16X3_TC5>(mode, a, sh, st);
            default: return cudaErrorInvalidValue;
        }
    }

    static size_t tc5_smem(int wslots) {
        if constexpr (kTc5) return tc5_smem_bytes<N>(wslots);
        else return 0;
    }
    static constexpr int tc5_items() {
        if constexpr (kTc5) return Tc5Shape<N>::ITEMS;
        else return 0;
    }
    static constexpr int tc5_threads() {
        if constexpr (kTc5) return Tc5Shape<N>::THREADS;
        else return 0;
    }

    static size_t tc_smem(int mode, int warps) {
        if constexpr (kTc) return tc_smem_bytes<N>(warps, mode == MODE_ADJOINT);
        return 0;
    }

    // gradient kernel: 16 points per thread, so nx <= 512
    static constexpr int VG = gradient_points_per_thread(N);
    static constexpr bool kGrad = (N & (N - 1)) == 0 && N >= VG && N / VG <= 32;

    static cudaError_t tables_grad(const TableArgs& a, cudaStream_t st) {
        if constexpr (kGrad) {
            const size_t total = (size_t)a.nw * a.nz * N;
            size_t blocks = (total + 255) / 256;
            if (blocks > 65535u * 8u) blocks = 65535u * 8u;
            ProfScope prof_(KC_TABLES, st);
            tables_kernel<N, VG><<<(unsigned)blocks, 256, 0, st>>>(a);
            count_launch();
            return cudaGetLastError();
        } else {
            return cudaErrorNotSupported;
        }
    }

    static cudaError_t gradient(const GradArgs& a, const SweepShape& sh, cudaStream_t st) {
        if constexpr (kGrad) {
            static DeviceOnce configured;
            cudaError_t e = configured.run([] {
                return cudaFuncSetAttribute(gradient_kernel<N, VG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            227 * 1024);
            });
            if (e != cudaSuccess) return e;
            if (sh.smem != gradient_smem_bytes<N, VG>(sh.warps, a.wslots)) return cudaErrorInvalidValue;
            ProfScope prof_(KC_GRADIENT, st);
            gradient_kernel<N, VG><<<sh.blocks, sh.warps * 32, sh.smem, st>>>(a);
            count_launch();
            return cudaGetLastError();
        } else {
            return cudaErrorNotSupported;
        }
    }

    static size_t gradient_smem(int warps, int wslots) {
        if constexpr (kGrad) return gradient_smem_bytes<N, VG>(warps, wslots);
        else return 0;
    }

    static int gradient_max_warps() {
        if constexpr (kGrad) {
            cudaFuncAttributes attr;
            if (cudaFuncGetAttributes(&attr, gradient_kernel<N, VG>) != cudaSuccess) {
                cudaGetLastError();
                return 8;
            }
            const int w = attr.maxThreadsPerBlock / 32;
            return w < 1 ? 1 : (w > 8 ? 8 : w);
        } else {
            return 1;
        }
    }
};

}  // namespace lsm

#define LSM_DEFINE_N(NN)                                                                          \
    namespace lsm {                                                                               \
    static cudaError_t tables_##NN(const TableArgs& a, cudaStream_t st) { return Dispatch<NN>::tables(a, st); } \
    static cudaError_t sweep_##NN(int mode, const SweepArgs& a, const SweepShape& sh, cudaStream_t st) {      \
        return Dispatch<NN>::sweep_any(mode, a, sh, st);                                          \
    }                                                                                             \
    static int max_warps_##NN(int mode) { return Dispatch<NN>::max_warps(mode); }                 \
    static size_t smem_##NN(int mode, int warps, int wslots) {                                    \
        return sweep_smem_bytes<NN, Dispatch<NN>::V>(warps, wslots, mode);        \
    }                                                                                             \
    static cudaError_t tables_grad_##NN(const TableArgs& a, cudaStream_t st) {                    \
        return Dispatch<NN>::tables_grad(a, st);                                                  \
    }                                                                                             \
    static cudaError_t gradient_##NN(const GradArgs& a, const SweepShape& sh, cudaStream_t st) {  \
        return Dispatch<NN>::gradient(a, sh, st);                                                 \
    }                                                                                             \
    static int gradient_max_warps_##NN() { return Dispatch<NN>::gradient_max_warps(); }           \
    static cudaError_t tables_natural_##NN(const TableArgs& a, cudaStream_t st) {                 \
        return Dispatch<NN>::tables_natural(a, st);                                               \
    }                                                                                             \
    static cudaError_t tc_sweep_##NN(int mode, int prec, const SweepArgs& a, const SweepShape& sh,  \
                                     cudaStream_t st) {                                           \
        return Dispatch<NN>::tc_sweep(mode, prec, a, sh, st);                                     \
    }                                                                                             \
    static size_t tc_smem_##NN(int mode, int warps) { return Dispatch<NN>::tc_smem(mode, warps); } \
    static size_t gradient_smem_##NN(int warps, int wslots) {                                     \
        return Dispatch<NN>::gradient_smem(warps, wslots);                                        \
    }                                                                                             \
    using DispatchAlt_##NN = Dispatch<NN, alt_points_per_thread(NN) ? alt_points_per_thread(NN) : points_per_thread(NN)>; \
    static cudaError_t alt_tables_##NN(const TableArgs& a, cudaStream_t st) { return DispatchAlt_##NN::tables(a, st); } \
    static cudaError_t alt_sweep_##NN(int mode, const SweepArgs& a, const SweepShape& sh, cudaStream_t st) { \
        return DispatchAlt_##NN::sweep_any(mode, a, sh, st);                                      \
    }                                                                                             \
    static int alt_max_warps_##NN(int mode) { return DispatchAlt_##NN::max_warps(mode); }         \
    static size_t alt_smem_##NN(int mode, int warps, int wslots) {                                \
        return sweep_smem_bytes<NN, DispatchAlt_##NN::V>(warps, wslots, mode);                    \
    }                                                                                             \
    static const NxOps kNxOpsAlt_##NN = {NN, DispatchAlt_##NN::V, false, alt_tables_##NN, alt_sweep_##NN, \
                                         alt_max_warps_##NN, alt_smem_##NN, nullptr, nullptr, nullptr, false, \
                                         nullptr, nullptr, nullptr, nullptr, false, nullptr, 0, 0, nullptr}; \
    extern const NxOps kNxOps_##NN = {NN, Dispatch<NN>::V, Dispatch<NN>::kGrad, tables_##NN, sweep_##NN,        \
                                      max_warps_##NN, smem_##NN, tables_grad_##NN, gradient_##NN,  \
                                      gradient_max_warps_##NN, Dispatch<NN>::kTc, tables_natural_##NN, \
                                      tc_sweep_##NN, tc_smem_##NN, gradient_smem_##NN,            \
                                      Dispatch<NN>::kTc5, Dispatch<NN>::tc5_smem,                  \
                                      Dispatch<NN>::tc5_items(), Dispatch<NN>::tc5_threads(),      \
                                      alt_points_per_thread(NN) ? &kNxOpsAlt_##NN : nullptr};       \
    }
