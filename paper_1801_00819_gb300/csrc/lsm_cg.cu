// CG vector kernels for the per-window normal equations (A_k^T A_k + lambda I) m = A_k^T d_k
// (Eq. 10), iterated from the previous window's image (Eq. 11).  Vectors are float32 (model:
// float [nz*nx]; data: complex64 [K*nw*nrec]); every inner product, the step length alpha and
// beta are float64.  Inner products are formed as per-block partial sums over a fixed grid and
// added in block order by whichever kernel consumes them, so every scalar is deterministic.
#include <cuda_runtime.h>

#include <cstdint>

#include "lsm_cg.h"
#include "lsm_internal.h"

namespace lsm {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
    }
    return tot;  // valid in thread 0
}

// every thread gets sum(part[0..n)) in a fixed order
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int n, double* sh) {
    double v = 0.0;
    // fixed assignment: thread i adds elements i, i + blockDim, ... then a fixed tree
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
    double tot = block_sum(v, sh);
    if (threadIdx.x == 0) sh[32] = tot;
    __syncthreads();
    tot = sh[32];
    __syncthreads();
    return tot;
}

// out[i] = (acc ? out[i] : 0) + sum_c part[c][i] - lam * m[i];  partial sums of out[i]^2 and,
// when minv is given, of out[i]^2 minv[i] (s.z for preconditioned CG).  With pdir given, the CG
// iteration's model update m += alpha pdir (alpha from the state, skipped after a breakdown) is
// applied first and m is written back.  A block takes 64 float4
// columns at a time and gives each column four threads: thread group q sums partials q, q + 4, ...
// with four accumulators (sixteen loads in flight per column), and the four group sums are added in
// a fixed order, so the result is deterministic.
constexpr int kImgCols = 64;                       // float4 columns per block and pass
constexpr int kImgGroups = kRedThreads / kImgCols;  // threads per column
__global__ void __launch_bounds__(kRedThreads) reduce_image_kernel(const float* __restrict__ part, int nparts, int n4,
                                                               float* __restrict__ m, float lam, int acc,
                                                               float* __restrict__ out, double* __restrict__ ss_part,
                                                               const float* __restrict__ minv,
                                                               double* __restrict__ sz_part,
                                                              const float* __restrict__ pdir,
                                                              const CgState* __restrict__ st, int discard) {
    __shared__ double sh[40];
    __shared__ float4 grp_sum[kImgGroups - 1][kImgCols];
    const float4* p4 = reinterpret_cast<const float4*>(part);
    float4* m4 = reinterpret_cast<float4*>(m);
    const float4* d4 = reinterpret_cast<const float4*>(pdir);
    const bool mupd = pdir && st->breakdown == 0;
    const float alpha = mupd ? (float)st->alpha : 0.f;
    const float4* w4 = reinterpret_cast<const float4*>(minv);
    float4* o4 = reinterpret_cast<float4*>(out);
    const int col = threadIdx.x % kImgCols, grp = threadIdx.x / kImgCols;
    double ss = 0.0, sz = 0.0;
    for (int base = blockIdx.x * kImgCols; base < n4; base += gridDim.x * kImgCols) {  // uniform per block
        const int i = base + col;
        constexpr int U = 4;  // accumulators (loads in flight) per thread; 8 measured no faster
        float4 a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) a[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < n4) {
            int c = grp;
            for (; c + (U - 1) * kImgGroups < nparts; c += U * kImgGroups) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float4 q = __ldcs(p4 + (size_t)(c + u * kImgGroups) * n4 + i);
                    a[u].x += q.x; a[u].y += q.y; a[u].z += q.z; a[u].w += q.w;
                }
            }
            for (; c < nparts; c += kImgGroups) {
                const float4 q = __ldcs(p4 + (size_t)c * n4 + i);
                a[0].x += q.x; a[0].y += q.y; a[0].z += q.z; a[0].w += q.w;
            }
        }
#pragma unroll
        for (int h = U / 2; h > 0; h >>= 1) {
#pragma unroll
            for (int u = 0; u < h; ++u) {
                a[u].x += a[u + h].x; a[u].y += a[u + h].y; a[u].z += a[u + h].z; a[u].w += a[u + h].w;
            }
        }
        if (grp > 0) grp_sum[grp - 1][col] = a[0];
        __syncthreads();
        if (grp == 0 && i < n4) {
            float4 s = acc ? o4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            s.x += a[0].x; s.y += a[0].y; s.z += a[0].z; s.w += a[0].w;
#pragma unroll
            for (int q = 0; q < kImgGroups - 1; ++q) {
                const float4 b = grp_sum[q][col];
                s.x += b.x; s.y += b.y; s.z += b.z; s.w += b.w;
            }
            if (m) {
                float4 mm = m4[i];
                if (mupd) {
                    const float4 y = d4[i];
                    mm.x = fmaf(alpha, y.x, mm.x); mm.y = fmaf(alpha, y.y, mm.y);
                    mm.z = fmaf(alpha, y.z, mm.z); mm.w = fmaf(alpha, y.w, mm.w);
                    m4[i] = mm;
                }
                s.x = fmaf(-lam, mm.x, s.x); s.y = fmaf(-lam, mm.y, s.y);
                s.z = fmaf(-lam, mm.z, s.z); s.w = fmaf(-lam, mm.w, s.w);
            }
            o4[i] = s;
            ss += (double)s.x * s.x + (double)s.y * s.y + (double)s.z * s.z + (double)s.w * s.w;
            if (minv) {
                const float4 w = w4[i];
                sz += (double)s.x * s.x * w.x + (double)s.y * s.y * w.y + (double)s.z * s.z * w.z +
                      (double)s.w * s.w * w.w;
            }
        }
        __syncthreads();  // grp_sum is rewritten by the next pass
        if (discard && (col & 7) == 0 && i < n4) {
            // every thread of the block has used its loads of this pass (barrier above), so the
            // partial rows are dead: their L2 lines are dropped without being written back to HBM
            // (i is a multiple of 8 float4, and the host checked that every line starts on 128 bytes)
            for (int c = grp; c < nparts; c += kImgGroups)
                asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(p4 + (size_t)c * n4 + i) : "memory");
        }
    }
    const double tot = block_sum(ss, sh);
    if (threadIdx.x == 0 && ss_part) ss_part[blockIdx.x] = tot;
    if (minv) {
        const double tz = block_sum(sz, sh);
        if (threadIdx.x == 0 && sz_part) sz_part[blockIdx.x] = tz;
    }
}

// partial sums of |q|^2 over a complex vector of n2 float2 pairs (processed as float4)
__global__ void __launch_bounds__(kRedThreads) norm2_c64_kernel(const float2* __restrict__ q, size_t n2,
                                                            double* __restrict__ part) {
    __shared__ double sh[40];
    const float4* q4 = reinterpret_cast<const float4*>(q);
    const size_t n4 = n2 / 2;
    double acc = 0.0;
#pragma unroll 4
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = q4[i];
        acc += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + (double)v.w * v.w;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (n2 & 1)) {
        const float2 v = q[n2 - 1];
        acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// r = d - q  (data space)
__global__ void residual_kernel(const float2* __restrict__ d, const float2* __restrict__ q, float2* __restrict__ r,
                                size_t n2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
        const float2 a = d[i], b = q[i];
        r[i] = make_float2(a.x - b.x, a.y - b.y);
    }
}

// delta = ||q||^2 + lam ||p||^2, alpha = gamma / delta; m += alpha p; r -= alpha q.
// A non-positive or non-finite delta sets the breakdown flag and leaves m and r untouched.
__global__ void __launch_bounds__(kRedThreads) update_mr_kernel(float* __restrict__ m, const float* __restrict__ p, int n4,
                                                            float2* __restrict__ r, const float2* __restrict__ q,
                                                            size_t n2, const double* __restrict__ qq_part,
                                                            const double* __restrict__ pp_part, int nred, double lam,
                                                            CgState* st, int gi) {
    __shared__ double sh[40];
    const double qq = sum_partials(qq_part, nred, sh);
    const double pp = sum_partials(pp_part, nred, sh);
    const double delta = qq + lam * pp;
    const double gamma = st->gamma[gi < 0 ? st->gi : gi];
    const bool bad = !(delta > 0.0) || !isfinite(delta) || !isfinite(gamma);
    const double alpha = bad ? 0.0 : gamma / delta;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->delta = delta;
        st->alpha = alpha;
        if (bad) st->breakdown = 1;
    }
    if (bad) return;
    const float a = (float)alpha;
    float4* m4 = reinterpret_cast<float4*>(m);
    const float4* p4 = reinterpret_cast<const float4*>(p);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x) {
        float4 x = m4[i];
        const float4 y = p4[i];
        x.x = fmaf(a, y.x, x.x); x.y = fmaf(a, y.y, x.y); x.z = fmaf(a, y.z, x.z); x.w = fmaf(a, y.w, x.w);
        m4[i] = x;
    }
    float4* r4 = reinterpret_cast<float4*>(r);
    const float4* q4 = reinterpret_cast<const float4*>(q);
    const size_t h4 = n2 / 2;
#pragma unroll 4
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < h4; i += (size_t)gridDim.x * blockDim.x) {
        float4 x = r4[i];
        const float4 y = q4[i];
        x.x = fmaf(-a, y.x, x.x); x.y = fmaf(-a, y.y, x.y); x.z = fmaf(-a, y.z, x.z); x.w = fmaf(-a, y.w, x.w);
        r4[i] = x;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (n2 & 1)) {
        float2 x = r[n2 - 1];
        const float2 y = q[n2 - 1];
        r[n2 - 1] = make_float2(fmaf(-a, y.x, x.x), fmaf(-a, y.y, x.y));
    }
}

// gamma_new = s.z (z = minv s, or z = s); beta = first ? 0 : gamma_new / gamma_old; p = z + beta p;
// partials of ||p||^2.  Reads gamma[gi_old] and writes gamma[gi_new] and ss[gi_new] (distinct
// slots, so blocks never race).
__global__ void __launch_bounds__(kRedThreads) update_p_kernel(float* __restrict__ p, const float* __restrict__ s, int n4,
                                                           const double* __restrict__ ss_part, int nred, int first,
                                                           CgState* st, int gi_old, int gi_new,
                                                           double* __restrict__ pp_part, const float* __restrict__ minv,
                                                           const double* __restrict__ sz_part) {
    __shared__ double sh[40];
    if (gi_old < 0) {  // device-driven loop: slots from the state (cg_loop_test flips them afterwards)
        gi_old = st->gi;
        gi_new = gi_old ^ 1;
    }
    const double ssum = sum_partials(ss_part, nred, sh);
    const double gnew = minv ? sum_partials(sz_part, nred, sh) : ssum;
    const double gold = first ? 1.0 : st->gamma[gi_old];
    const double beta = first ? 0.0 : gnew / gold;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->gamma[gi_new] = gnew;
        st->ss[gi_new] = ssum;
        st->beta = beta;
        if (!isfinite(gnew) || !isfinite(ssum)) st->breakdown = 1;
    }
    const float b = (float)beta;
    float4* p4 = reinterpret_cast<float4*>(p);
    const float4* s4 = reinterpret_cast<const float4*>(s);
    const float4* w4 = reinterpret_cast<const float4*>(minv);
    double pp = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x) {
        float4 x = s4[i];
        if (minv) {
            const float4 w = w4[i];
            x.x *= w.x; x.y *= w.y; x.z *= w.z; x.w *= w.w;
        }
        float4 y = first ? make_float4(0.f, 0.f, 0.f, 0.f) : p4[i];
        y.x = fmaf(b, y.x, x.x); y.y = fmaf(b, y.y, x.y); y.z = fmaf(b, y.z, x.z); y.w = fmaf(b, y.w, x.w);
        p4[i] = y;
        pp += (double)y.x * y.x + (double)y.y * y.y + (double)y.z * y.z + (double)y.w * y.w;
    }
    const double tot = block_sum(pp, sh);
    if (threadIdx.x == 0) pp_part[blockIdx.x] = tot;
}

// illum[i] = sum over rows r of |S[r * n + i]|^2 (rows = ring slots x frequencies, each row one
// [nz][nx] plane); per-block maxima of illum
__global__ void __launch_bounds__(256) illumination_kernel(const float2* __restrict__ S, int rows, int n,
                                                           float* __restrict__ illum, float* __restrict__ block_max) {
    __shared__ float shm[8];
    float mx = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
        int r = 0;
        for (; r + 4 <= rows; r += 4) {
            const float2 a = __ldcs(S + (size_t)r * n + i), b = __ldcs(S + (size_t)(r + 1) * n + i);
            const float2 c = __ldcs(S + (size_t)(r + 2) * n + i), d = __ldcs(S + (size_t)(r + 3) * n + i);
            acc0 = fmaf(a.x, a.x, fmaf(a.y, a.y, acc0));
            acc1 = fmaf(b.x, b.x, fmaf(b.y, b.y, acc1));
            acc2 = fmaf(c.x, c.x, fmaf(c.y, c.y, acc2));
            acc3 = fmaf(d.x, d.x, fmaf(d.y, d.y, acc3));
        }
        for (; r < rows; ++r) {
            const float2 a = __ldcs(S + (size_t)r * n + i);
            acc0 = fmaf(a.x, a.x, fmaf(a.y, a.y, acc0));
        }
        const float v = (acc0 + acc1) + (acc2 + acc3);
        illum[i] = v;
        mx = fmaxf(mx, v);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m2 = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmaxf(m2, shm[w]);
        block_max[blockIdx.x] = m2;
    }
}

// minv = 1 / (illum + eps max illum); every block takes the maximum of the block maxima itself
__global__ void __launch_bounds__(256) precond_finalize_kernel(const float* __restrict__ illum, int n,
                                                               const float* __restrict__ block_max, int nblocks,
                                                               float eps, float* __restrict__ minv) {
    __shared__ float shm[8];
    float mx = 0.f;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) mx = fmaxf(mx, block_max[b]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mx;
    __syncthreads();
    float gmax = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) gmax = fmaxf(gmax, shm[w]);
    const float stab = gmax > 0.f ? eps * gmax : 1.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        minv[i] = 1.f / (illum[i] + stab);
}

// st->bb = sum of partials (||A^T d||^2)
__global__ void __launch_bounds__(kRedThreads) store_sum_kernel(const double* __restrict__ part, int nred, CgState* st) {
    __shared__ double sh[40];
    const double tot = sum_partials(part, nred, sh);
    if (threadIdx.x == 0) st->bb = tot;
}

// *out = sum of part[0 .. n) in the fixed order of sum_partials
__global__ void __launch_bounds__(kRedThreads) sum_to_kernel(const double* __restrict__ part, int n, double* out) {
    __shared__ double sh[40];
    const double tot = sum_partials(part, n, sh);
    if (threadIdx.x == 0) *out = tot;
}

__global__ void zero_state_kernel(CgState* st) {
    if (threadIdx.x == 0) {
        st->gamma[0] = st->gamma[1] = 0.0;
        st->alpha = st->beta = st->delta = st->bb = 0.0;
        st->ss[0] = st->ss[1] = 0.0;
        st->breakdown = 0;
        st->gi = 0;
        st->iter = st->max_iter = 0;
        st->tol = st->rel0 = st->rel = 0.0;
    }
}

__global__ void loop_setup_kernel(CgState* st, int* shot0_dev, int shot0, int max_iter, double tol,
                                  const int* halt) {
    if (threadIdx.x == 0) {
        st->gi = 0;
        st->iter = 0;
        st->max_iter = (halt && *halt) ? 0 : max_iter;
        st->tol = tol;
        *shot0_dev = shot0;
    }
}

// The stopping test of the window loop (same order and arithmetic as the host-driven loop):
// after an iteration the new gamma slot becomes current; rel = sqrt(ss[gi]) / sqrt(bb).
__global__ void loop_test_kernel(CgState* st, cudaGraphConditionalHandle handle, int advance) {
    if (threadIdx.x != 0) return;
    if (advance) {
        st->gi ^= 1;
        st->iter += 1;
    }
    const double bnorm = sqrt(st->bb);
    const double rel = bnorm > 0.0 ? sqrt(st->ss[st->gi]) / bnorm : 0.0;
    st->rel = rel;
    if (!advance) st->rel0 = rel;
    const bool cont = st->breakdown == 0 && st->iter < st->max_iter && !(rel <= st->tol);
    cudaGraphSetConditional(handle, cont ? 1u : 0u);
}

__global__ void record_window_kernel(const CgState* st, WindowRecord* rec, int* halt) {
    if (threadIdx.x == 0) {
        rec->iters = st->iter;
        rec->breakdown = st->breakdown;
        rec->rel0 = st->rel0;
        rec->rel = st->rel;
        if (st->breakdown) *halt = 1;
    }
}

// ------------------------------------------------------------------ launchers

cudaError_t cg_reduce_image(const float* part, int nparts, int n, float* m, float lam, int acc, float* out,
                            double* ss_part, cudaStream_t st, const float* minv, double* sz_part, const float* p,
                            const CgState* state, bool discard_part) {
    ProfScope prof_(KC_VECTOR, st);
    // lines are dropped only when each partial plane is a whole number of 128-byte lines from a
    // 128-byte boundary
    const int discard = discard_part && ((uintptr_t)part & 127u) == 0 && (n / 4) % 8 == 0 && n % 4 == 0;
    reduce_image_kernel<<<kImgRedBlocks, kRedThreads, 0, st>>>(part, nparts, n / 4, m, lam, acc, out, ss_part, minv,
                                                            sz_part, p, state, discard);
    count_launch();
    return cudaGetLastError();
}

cudaError_t cg_norm2_c64(const float2* q, size_t n2, double* part, cudaStream_t st) {
    ProfScope prof_(KC_VECTOR, st);
    norm2_c64_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(q, n2, part);
    count_launch();
    return cudaGetLastError();
}

cudaError_t cg_residual(const float2* d, const float2* q, float2* r, size_t n2, cudaStream_t st) {
    ProfScope prof_(KC_VECTOR, st);
    residual_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(d, q, r, n2);
    count_launch();
    return cudaGetLastError();
}

cudaError_t cg_update_mr(float* m, const float* p, int n, float2* r, const float2* q, size_t n2,
                         const double* qq_part, const double* pp_part, double lam, CgState* state, int gi,
                         cudaStream_t st) {
    ProfScope prof_(KC_VECTOR, st);
    update_mr_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(m, p, n / 4, r, q, n2, qq_part, pp_part, kRedBlocks, lam,
                                                          state, gi);
    count_launch();
    return cudaGetLastError();
}

cudaError_t cg_update_p(float* p, const float* s, int n, const double* ss_part, int first, CgState* state,
                        int gi_old, int gi_new, double* pp_part, cudaStream_t st, const float* minv,
                        const double* sz_part) {
    ProfScope prof_(KC_VECTOR, st);
    update_p_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(p, s, n / 4, ss_part, kImgRedBlocks, first, state, gi_old,
                                                         gi_new, pp_part, minv, sz_part);
    count_launch();
    return cudaGetLastError();
}

cudaError_t cg_store_sum(const double* part, CgState* state, cudaStream_t st) {
    ProfScope prof_(KC_VECTOR, st);
    store_sum_kernel<<<1, kRedThreads, 0, st>>>(part, kImgRedBlocks, state);
    count_launch();
    return cudaGetLastError();
}

cudaError_t cg_sum_partials(const double* part, int n, double* out, cudaStream_t st) {
    ProfScope prof_(KC_VECTOR, st);
    sum_to_kernel<<<1, kRedThreads, 0, st>>>(part, n, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t cg_zero_state(CgState* state, cudaStream_t st) {
    ProfScope prof_(KC_VECTOR, st);
    zero_state_kernel<<<1, 32, 0, st>>>(state);
    count_launch();
    return cudaGetLastError();
}

cudaError_t cg_loop_setup(CgState* state, int* shot0_dev, int shot0, int max_iter, double tol, cudaStream_t st,
                          const int* halt) {
    ProfScope prof_(KC_VECTOR, st);
    loop_setup_kernel<<<1, 32, 0, st>>>(state, shot0_dev, shot0, max_iter, tol, halt);
    count_launch();
    return cudaGetLastError();
}

cudaError_t cg_record_window(const CgState* state, WindowRecord* rec, int* halt, cudaStream_t st) {
    ProfScope prof_(KC_VECTOR, st);
    record_window_kernel<<<1, 32, 0, st>>>(state, rec, halt);
    count_launch();
    return cudaGetLastError();
}

cudaError_t cg_loop_test(CgState* state, cudaGraphConditionalHandle handle, int advance, cudaStream_t st) {
    ProfScope prof_(KC_VECTOR, st);
    loop_test_kernel<<<1, 32, 0, st>>>(state, handle, advance);
    count_launch();
    return cudaGetLastError();
}

void cg_loop_test_node_params(cudaKernelNodeParams* kp, void** args) {
    *kp = cudaKernelNodeParams{};
    kp->func = reinterpret_cast<void*>(loop_test_kernel);
    kp->gridDim = dim3(1);
    kp->blockDim = dim3(32);
    kp->sharedMemBytes = 0;
    kp->kernelParams = args;
    kp->extra = nullptr;
}

cudaError_t cg_illumination(const float2* S, int rows, int n, float* illum, float* block_max, cudaStream_t st) {
    ProfScope prof_(KC_VECTOR, st);
    illumination_kernel<<<kIllumBlocks, 256, 0, st>>>(S, rows, n, illum, block_max);
    count_launch();
    return cudaGetLastError();
}

cudaError_t cg_precond_finalize(const float* illum, int n, const float* block_max, double eps, float* minv,
                                cudaStream_t st) {
    ProfScope prof_(KC_VECTOR, st);
    precond_finalize_kernel<<<kRedBlocks, 256, 0, st>>>(illum, n, block_max, kIllumBlocks, (float)eps, minv);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lsm
