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

    // ---------------- phase 2: segments bottom-up
    float2 U[V], mu[V];
#pragma unroll
    for (int r = 0; r < V; ++r) U[r] = mu[r] = make_float2(0.f, 0.f);
    int depth_count = 0;  // barrier parity
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
        // phase 2 of the segment: row j of step j is in buffer (j1 - 1 - j) % 2; rows j1 - 1 and
        // j1 - 2 are staged up front, and row j - 2 replaces row j once every warp is past step j
        __syncthreads();
        stage_row(j1 - 1, 0);
        if (j1 - 2 >= j0) stage_row(j1 - 2, 1);
        cp_async_wait_all();
        __syncthreads();
        for (int j = j1 - 1; j >= j0; --j, ++depth_count) {
            const float* mrow = a.m + (size_t)j * N;
            // P_j U_{j+1} (zero at the deepest row)
            const int bj = (j1 - 1 - j) & 1;
            if (j + 1 < nz) grad_step<N, V, false>(U, tw, buf, t, phi_s(bj), dss_s(bj));
            float2 Rj[V];
            grad_load<N, V>(Rj, Rseg + (size_t)(j - j0) * N, t, ok);
            float gs[V], gm[V];
#pragma unroll
            for (int r = 0; r < V; ++r) gs[r] = fmaf(Rj[r].x, U[r].y, -Rj[r].y * U[r].x);  // Im conj(R) PU
            if (j + 1 < nz) {
                float2 S1[V];
                grad_load<N, V>(S1, Sseg + (size_t)(j + 1 - j0) * N, t, ok);
#pragma unroll
                for (int r = 0; r < V; ++r) gs[r] += fmaf(mu[r].x, S1[r].y, -mu[r].y * S1[r].x);  // Im conj(mu) S1
            }
            {
                float2 Sj[V];
                grad_load<N, V>(Sj, Sseg + (size_t)(j - j0) * N, t, ok);
#pragma unroll
                for (int r = 0; r < V; ++r) {
                    const float mm = __ldg(mrow + t + T * r);
                    gm[r] = fmaf(Sj[r].x, Rj[r].x, Sj[r].y * Rj[r].y);
                    U[r].x = fmaf(Sj[r].x, mm, U[r].x);
                    U[r].y = fmaf(Sj[r].y, mm, U[r].y);
                }
            }
            // Re(i z) = -Im(z)
#pragma unroll
            for (int r = 0; r < V; ++r) gs[r] = -wdz * gs[r];
            // mu_j = m_j R_j + P_j^H mu_{j+1}
            if (j + 1 < nz) {
                grad_step<N, V, true>(mu, tw, buf, t, phi_s(bj), dss_s(bj));
            } else {
#pragma unroll
                for (int r = 0; r < V; ++r) mu[r] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int r = 0; r < V; ++r) {
                const float mm = __ldg(mrow + t + T * r);
                mu[r].x = fmaf(mm, Rj[r].x, mu[r].x);
                mu[r].y = fmaf(mm, Rj[r].y, mu[r].y);
            }
            // sum both gradient rows over the block's items
#pragma unroll
            for (int off = T; off < 32; off <<= 1) {
#pragma unroll
                for (int r = 0; r < V; ++r) {
                    gm[r] += __shfl_xor_sync(0xffffffffu, gm[r], off);
                    gs[r] += __shfl_xor_sync(0xffffffffu, gs[r], off);
                }
            }
            const int b = depth_count & 1;
            float* slab_m = img + ((size_t)(b * 2 + 0) * nwarps + warp) * N;
            float* slab_s = img + ((size_t)(b * 2 + 1) * nwarps + warp) * N;
            if (sub == 0) {
#pragma unroll
                for (int r = 0; r < V; ++r) {
                    slab_m[t + T * r] = ok ? gm[r] : 0.f;
                    slab_s[t + T * r] = ok ? gs[r] : 0.f;
                }
            }
            cp_async_wait_all();
            __syncthreads();  // image rows visible; row j - 1 staged and visible; every warp is past step j
            if (j - 2 >= j0) stage_row(j - 2, bj);
            {
                // the block's partial rows: the warps' rows summed in warp order, four columns a thread
                const float4* rows_m = reinterpret_cast<const float4*>(img + (size_t)(b * 2 + 0) * nwarps * N);
                const float4* rows_s = reinterpret_cast<const float4*>(img + (size_t)(b * 2 + 1) * nwarps * N);
                float4* pm = reinterpret_cast<float4*>(a.part_m + ((size_t)blockIdx.x * nz + j) * N);
                float4* ps = reinterpret_cast<float4*>(a.part_s + ((size_t)blockIdx.x * nz + j) * N);
                for (int x4 = threadIdx.x; x4 < N / 4; x4 += blockDim.x) {
                    float4 am = rows_m[x4], as = rows_s[x4];
                    for (int w2 = 1; w2 < nwarps; ++w2) {
                        const float4 um = rows_m[w2 * (N / 4) + x4], us = rows_s[w2 * (N / 4) + x4];
                        am.x += um.x; am.y += um.y; am.z += um.z; am.w += um.w;
                        as.x += us.x; as.y += us.y; as.z += us.z; as.w += us.w;
                    }
                    pm[x4] = am;
                    ps[x4] = as;
                }
            }
        }
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
