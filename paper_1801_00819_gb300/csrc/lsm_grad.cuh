// Gradients of a real loss L(d), d = A(s) m, with respect to the model m and the slowness s, for
// the shot-profile split-step operator (Eq. 1) with the reference slowness held fixed.  Given
// g = dL/dRe(d) + i dL/dIm(d) at the receivers, per (shot, w) item:
//   R_0 = injected g, R_{j+1} = P_j^H R_j                      (adjoint wavefield, top-down)
//   U_{nz-1} = S_{nz-1} m_{nz-1}, U_j = S_j m_j + P_j U_{j+1}  (scattered field, bottom-up)
//   mu_{nz} = 0, mu_j = m_j R_j + P_j^H mu_{j+1}               (source-side adjoint, bottom-up)
//   dL/dm_j += Re conj(S_j) R_j
//   dL/ds_j += Re i w dz [conj(R_j) P_j U_{j+1} + conj(mu_{j+1}) S_{j+1}]
// The source and adjoint wavefields run top-down but are needed bottom-up, so phase 1 sweeps them
// down once and keeps only every `c`-th depth (checkpoints); phase 2 walks the depth segments from
// the bottom, recomputes each segment's S and R rows from their checkpoints into a small per-item
// buffer, and runs the U and mu recursions in registers.  Per-depth gradient rows are summed over
// the block's items and written as block partials (reduced later in a fixed order).  The Phi and D
// rows of each depth are staged once per block (for the few frequencies its items span) into
// double-buffered shared memory with cp.async, and both wavefields of a loop step read them there.
#pragma once

#include "lsm_async.cuh"
#include "lsm_fft.cuh"
#include "lsm_internal.h"

namespace lsm {

// one propagation step in registers; phi and dss point at the staged rows in shared memory
template <int N, int V, bool ADJ>
__device__ __forceinline__ void grad_step(float2 (&v)[V], const Twiddles<N, V>& tw, float2* buf, int t,
                                          const float2* __restrict__ phi, const float2* __restrict__ dss) {
    constexpr int T = Plan<N, V>::T;
    if (ADJ) {
#pragma unroll
        for (int r = 0; r < V; ++r) v[r] = cmulc(v[r], dss[Plan<N, V>::xpos(t, r)]);
    }
    fft_forward<N, V>(v, tw, buf, t);
#pragma unroll
    for (int r = 0; r < V; ++r) v[r] = ADJ ? cmulc(v[r], phi[t + T * r]) : cmul(v[r], phi[t + T * r]);
    fft_inverse<N, V>(v, tw, buf, t);
    if (!ADJ) {
#pragma unroll
        for (int r = 0; r < V; ++r) v[r] = cmul(v[r], dss[Plan<N, V>::xpos(t, r)]);
    }
}

template <int N, int V>
__device__ __forceinline__ void grad_store(float2* __restrict__ row, const float2 (&v)[V], int t, bool ok) {
    constexpr int T = Plan<N, V>::T;
    if (ok) {
#pragma unroll
        for (int r = 0; r < V; ++r) row[t + T * r] = v[r];
    }
}

template <int N, int V>
__device__ __forceinline__ void grad_load(float2 (&v)[V], const float2* __restrict__ row, int t, bool ok) {
    constexpr int T = Plan<N, V>::T;
#pragma unroll
    for (int r = 0; r < V; ++r) v[r] = ok ? row[t + T * r] : make_float2(0.f, 0.f);
}

// dynamic shared memory: exchange buffers + [2 buffers][2 images][warps][N] floats + staged
// coefficient rows [2 buffers][wslots][Phi, D][N] float2 (mirrored on the host by gradient_shape)
template <int N, int V>
constexpr size_t gradient_smem_bytes(int warps, int wslots) {
    return (size_t)warps * (32 / Plan<N, V>::T) * Plan<N, V>::BUF * sizeof(float2) +
           (size_t)2 * 2 * warps * N * sizeof(float) + (size_t)2 * wslots * 2 * N * sizeof(float2);
}

template <int N, int V>
__global__ void __launch_bounds__(256) gradient_kernel(const GradArgs a) {
    using P = Plan<N, V>;
    static_assert(P::R0 == V && !P::TW_SMEM, "power-of-two plans: register r holds column t + T r");
    constexpr int T = P::T;
    constexpr int IPW = 32 / T;
    extern __shared__ float4 smem_f4[];
    float2* smem = reinterpret_cast<float2*>(smem_f4);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int t = lane % T;
    const int sub = lane / T;
    const int ipb = nwarps * IPW;
    const int nitems = a.nshots * a.nw;
    const int item = blockIdx.x * ipb + warp * IPW + sub;
    const bool ok = item < nitems;
    // items are frequency-major: the block's items span frequencies w_first .. w_last
    const int w_first = min(blockIdx.x * ipb, nitems - 1) / a.nshots;
    const int w_last = (min((blockIdx.x + 1) * ipb, nitems) - 1) / a.nshots;
    const int nslots = w_last - w_first + 1;  // <= a.wslots
    const int iw = ok ? item / a.nshots : w_first;
    const int ishot = ok ? item - iw * a.nshots : 0;
    const int shot = a.shot0 + ishot;
    const int nz = a.nz;
    const int c = a.ckpt_every;
    const int ncp = (nz + c - 1) / c;
    float2* buf = smem + (warp * IPW + sub) * P::BUF;
    float* img = reinterpret_cast<float*>(smem + ipb * P::BUF);  // [2][2][nwarps][N]
    float2* stage = reinterpret_cast<float2*>(img + 4 * nwarps * N);  // [2][wslots][2][N]
    const int stage_buf = a.wslots * 2 * N;
    const int wslot = iw - w_first;

    Twiddles<N, V> tw;
    init_twiddles<N, V>(tw, t);

    // the whole block stages the Phi and D rows of depth `row` for its frequencies into buffer b,
    // one cp.async group per thread
    auto stage_row = [&](int row, int b) {
        constexpr int CH = N / 2;  // 16-byte chunks per complex row
        float2* dst = stage + b * stage_buf;
        for (int q = threadIdx.x; q < nslots * 2 * CH; q += blockDim.x) {
            const int sl = q / (2 * CH);
            const int rem = q - sl * 2 * CH;
            const int which = rem / CH;
            const int ch = rem - which * CH;
            const float2* src = (which ? a.dss : a.phi) + ((size_t)(w_first + sl) * nz + row) * N + 2 * ch;
            cp_async16(dst + (sl * 2 + which) * N + 2 * ch, src);
        }
        cp_async_commit();
    };
    auto phi_s = [&](int b) -> const float2* { return stage + b * stage_buf + (wslot * 2) * N; };
    auto dss_s = [&](int b) -> const float2* { return stage + b * stage_buf + (wslot * 2 + 1) * N; };
    const size_t slot = ok ? (size_t)item : 0;
    float2* Sck = a.ckpt + slot * 2 * ncp * N;
    float2* Rck = Sck + (size_t)ncp * N;
    float2* Sseg = a.seg + slot * (2 * c + 1) * N;
    float2* Rseg = Sseg + (size_t)(c + 1) * N;
    const float wdz = 2.0f * (float)kPi * (ok ? __ldg(a.freq_hz + iw) : 0.f) * a.dz;

    // ---------------- phase 1: S and R down, checkpoints every c depths
    {
        float2 S[V], R[V];
        const int xs = ok ? __ldg(a.src_ix + shot) : -1;
        const float2 w = ok ? __ldg(a.wavelet + iw) : make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < V; ++r) S[r] = (t + T * r == xs) ? w : make_float2(0.f, 0.f);
        const float2* grow = a.g + ((size_t)ishot * a.nw + iw) * a.nrec;
        if (a.rec_identity) {
            grad_load<N, V>(R, grow, t, ok);
        } else {
            __syncwarp();
            for (int x = t; x < P::BUF; x += T) buf[x] = make_float2(0.f, 0.f);
            __syncwarp();
            if (ok) {
                const int* rix = a.rec_ix + (size_t)shot * a.nrec;
                for (int rr = t; rr < a.nrec; rr += T) {
                    const float2 dv = __ldg(grow + rr);
                    const int x = P::phys(__ldg(rix + rr));
                    atomicAdd(&buf[x].x, dv.x);
                    atomicAdd(&buf[x].y, dv.y);
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < V; ++r) R[r] = buf[P::phys(t + T * r)];
        }
        // step j reads buffer j % 2; the rows of step j + 1 are staged while step j runs
        if (nz > 1) stage_row(0, 0);
        for (int j = 0; j < nz; ++j) {
            if (j % c == 0) {
                grad_store<N, V>(Sck + (size_t)(j / c) * N, S, t, ok);
                grad_store<N, V>(Rck + (size_t)(j / c) * N, R, t, ok);
            }
            if (j + 1 < nz) {
                cp_async_wait_all();
                __syncthreads();  // rows of step j visible; every warp is done with step j - 1
                if (j + 2 < nz) stage_row(j + 1, (j + 1) & 1);
                grad_step<N, V, false>(S, tw, buf, t, phi_s(j & 1), dss_s(j & 1));
                grad_step<N, V, true>(R, tw, buf, t, phi_s(j & 1), dss_s(j & 1));
            }
        }
    }

    // ---------------- phase 2: segments bottom-up.  Per segment the S and R rows are recomputed
    // into the item's segment buffer, then two passes run up the segment: U (with dL/dm and the
    // conj(R_j) P_j U_{j+1} term of dL/ds), then mu (the conj(mu_{j+1}) S_{j+1} term).  Only one of
    // U and mu is in registers at a time; the other waits in the item's two parking rows.
    float2 U[V];
#pragma unroll
    for (int r = 0; r < V; ++r) U[r] = make_float2(0.f, 0.f);
    float2* Upark = a.park + slot * 2 * N;
    float2* Mpark = Upark + N;
    grad_store<N, V>(Mpark, U, t, ok);  // mu below the deepest row: zero
    int depth_count = 0;  // image-row buffer parity
    // the block's rows of a gradient summed in warp order and written (or, add_to, added) to its
    // partial row of depth j, four columns a thread
    auto block_sum = [&](int b, int which, float* part, int j, bool add_to) {
        const float4* rows = reinterpret_cast<const float4*>(img + (size_t)(b * 2 + which) * nwarps * N);
        float4* prow = reinterpret_cast<float4*>(part + ((size_t)blockIdx.x * nz + j) * N);
        for (int x4 = threadIdx.x; x4 < N / 4; x4 += blockDim.x) {
            float4 acc = rows[x4];
            for (int w2 = 1; w2 < nwarps; ++w2) {
                const float4 u4 = rows[w2 * (N / 4) + x4];
                acc.x += u4.x; acc.y += u4.y; acc.z += u4.z; acc.w += u4.w;
            }
            if (add_to) {
                const float4 p4 = prow[x4];
                acc.x += p4.x; acc.y += p4.y; acc.z += p4.z; acc.w += p4.w;
            }
            prow[x4] = acc;
        }
    };
    // one gradient row per warp: the items of equal t summed by shuffles, then lane group 0 writes
    auto warp_row = [&](float (&gv)[V], float* slab) {
#pragma unroll
        for (int off = T; off < 32; off <<= 1) {
#pragma unroll
            for (int r = 0; r < V; ++r) gv[r] += __shfl_xor_sync(0xffffffffu, gv[r], off);
        }
        if (sub == 0) {
#pragma unroll
            for (int r = 0; r < V; ++r) slab[t + T * r] = ok ? gv[r] : 0.f;
        }
    };
    for (int seg = ncp - 1; seg >= 0; --seg) {
        const int j0 = seg * c;
        const int j1 = min(j0 + c, nz);
        {
            // S rows j0 .. jmax (jmax = j1 when a deeper row exists, for S_{j+1} at j = j1 - 1);
            // step j reads buffer (j - j0) % 2
            const int jmax = j1 < nz ? j1 : nz - 1;
            float2 S[V];
            grad_load<N, V>(S, Sck + (size_t)seg * N, t, ok);
            __syncthreads();  // every warp is done with the staging buffers of the previous loop
            if (j0 < jmax) stage_row(j0, 0);
            for (int j = j0; j <= jmax; ++j) {
                grad_store<N, V>(Sseg + (size_t)(j - j0) * N, S, t, ok);
                if (j < jmax) {
                    const int b = (j - j0) & 1;
                    cp_async_wait_all();
                    __syncthreads();
                    if (j + 1 < jmax) stage_row(j + 1, b ^ 1);
                    grad_step<N, V, false>(S, tw, buf, t, phi_s(b), dss_s(b));
                }
            }
        }
        {
            // R rows j0 .. j1 - 1
            float2 R[V];
            grad_load<N, V>(R, Rck + (size_t)seg * N, t, ok);
            __syncthreads();
            if (j0 + 1 < j1) stage_row(j0, 0);
            for (int j = j0; j < j1; ++j) {
                grad_store<N, V>(Rseg + (size_t)(j - j0) * N, R, t, ok);
                if (j + 1 < j1) {
                    const int b = (j - j0) & 1;
                    cp_async_wait_all();
                    __syncthreads();
                    if (j + 2 < j1) stage_row(j + 1, b ^ 1);
                    grad_step<N, V, true>(R, tw, buf, t, phi_s(b), dss_s(b));
                }
            }
        }
        // each pass: row j of step j is in buffer (j1 - 1 - j) % 2; rows j1 - 1 and j1 - 2 are
        // staged up front, and row j - 2 replaces row j once every warp is past step j
        auto stage_pass = [&]() {
            __syncthreads();
            stage_row(j1 - 1, 0);
            if (j1 - 2 >= j0) stage_row(j1 - 2, 1);
            cp_async_wait_all();
            __syncthreads();
        };
        // pass U: U_j = S_j m_j + P_j U_{j+1}; dL/dm_j = Re conj(S_j) R_j; dL/ds_j gets
        // Re(i w dz conj(R_j) P_j U_{j+1}) = -w dz Im(conj(R_j) P_j U_{j+1})
        stage_pass();
        for (int j = j1 - 1; j >= j0; --j, ++depth_count) {
            const float* mrow = a.m + (size_t)j * N;
            const int bj = (j1 - 1 - j) & 1;
            if (j + 1 < nz) grad_step<N, V, false>(U, tw, buf, t, phi_s(bj), dss_s(bj));
            float gs[V], gm[V];
            const float2* Rrow = Rseg + (size_t)(j - j0) * N;
            const float2* Srow = Sseg + (size_t)(j - j0) * N;
#pragma unroll
            for (int r = 0; r < V; ++r) {
                const float2 Rj = ok ? Rrow[t + T * r] : make_float2(0.f, 0.f);
                const float2 Sj = ok ? Srow[t + T * r] : make_float2(0.f, 0.f);
                const float mm = __ldg(mrow + t + T * r);
                gs[r] = -wdz * fmaf(Rj.x, U[r].y, -Rj.y * U[r].x);
                gm[r] = fmaf(Sj.x, Rj.x, Sj.y * Rj.y);
                U[r].x = fmaf(Sj.x, mm, U[r].x);
                U[r].y = fmaf(Sj.y, mm, U[r].y);
            }
            const int b = depth_count & 1;
            warp_row(gm, img + ((size_t)(b * 2 + 0) * nwarps + warp) * N);
            warp_row(gs, img + ((size_t)(b * 2 + 1) * nwarps + warp) * N);
            cp_async_wait_all();
            __syncthreads();  // gradient rows visible; row j - 1 staged and visible; every warp is past step j
            if (j - 2 >= j0) stage_row(j - 2, bj);
            block_sum(b, 0, a.part_m, j, false);
            block_sum(b, 1, a.part_s, j, false);
        }
        // pass mu: mu_j = m_j R_j + P_j^H mu_{j+1}; dL/ds_j gets -w dz Im(conj(mu_{j+1}) S_{j+1}),
        // added to the partial row pass U wrote
        grad_store<N, V>(Upark, U, t, ok);
        {
            float2 mu[V];
            grad_load<N, V>(mu, Mpark, t, ok);
            stage_pass();
            for (int j = j1 - 1; j >= j0; --j, ++depth_count) {
                const float* mrow = a.m + (size_t)j * N;
                const int bj = (j1 - 1 - j) & 1;
                float gs[V];
                if (j + 1 < nz) {
                    const float2* S1row = Sseg + (size_t)(j + 1 - j0) * N;
#pragma unroll
                    for (int r = 0; r < V; ++r) {
                        const float2 S1 = ok ? S1row[t + T * r] : make_float2(0.f, 0.f);
                        gs[r] = -wdz * fmaf(mu[r].x, S1.y, -mu[r].y * S1.x);
                    }
                    grad_step<N, V, true>(mu, tw, buf, t, phi_s(bj), dss_s(bj));
                } else {
#pragma unroll
                    for (int r = 0; r < V; ++r) {
                        gs[r] = 0.f;
                        mu[r] = make_float2(0.f, 0.f);
                    }
                }
                const float2* Rrow = Rseg + (size_t)(j - j0) * N;
#pragma unroll
                for (int r = 0; r < V; ++r) {
                    const float2 Rj = ok ? Rrow[t + T * r] : make_float2(0.f, 0.f);
                    const float mm = __ldg(mrow + t + T * r);
                    mu[r].x = fmaf(mm, Rj.x, mu[r].x);
                    mu[r].y = fmaf(mm, Rj.y, mu[r].y);
                }
                const int b = depth_count & 1;
                warp_row(gs, img + ((size_t)(b * 2 + 1) * nwarps + warp) * N);
                cp_async_wait_all();
                __syncthreads();
                if (j - 2 >= j0) stage_row(j - 2, bj);
                block_sum(b, 1, a.part_s, j, true);
            }
            grad_store<N, V>(Mpark, mu, t, ok);
        }
        grad_load<N, V>(U, Upark, t, ok);
    }
    // U now holds U_0: the modelled data of this item
    if (a.dout) {
        float2* orow = a.dout + ((size_t)ishot * a.nw + iw) * a.nrec;
        if (a.rec_identity) {
            grad_store<N, V>(orow, U, t, ok);
        } else {
            __syncwarp();
#pragma unroll
            for (int r = 0; r < V; ++r) buf[P::phys(t + T * r)] = U[r];
            __syncwarp();
            if (ok) {
                const int* rix = a.rec_ix + (size_t)shot * a.nrec;
                for (int rr = t; rr < a.nrec; rr += T) orow[rr] = buf[P::phys(__ldg(rix + rr))];
            }
        }
    }
}

}  // namespace lsm
