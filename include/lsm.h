/*
 * lsm.h - C ABI of the GB300 block-row recursive least-squares migration library.
 *
 * The library applies the 2D shot-profile split-step Fourier de-migration operator A
 * (Eq. 1: d = A m + n), its adjoint A^T (Eq. 2: migration with the cross-correlation imaging
 * condition), and solves the damped least-squares problem (Eq. 3) on sliding windows of shots
 * with CG on each window's normal equations (A_k^T A_k + lambda I) m = A_k^T d_k (Eq. 10),
 * warm-started from the previous window's image (Eq. 11).  The operator is the one the paper's
 * Examples section uses: one-way shot-profile propagation by phase shift in (w, kx) with the
 * split-step slowness correction in (w, x).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grid: nx lateral cells by nz depth rows, spacing dx, dz in metres.  nx is a power of two
 *    from 16 to 1024 or one of 48, 96, 192, 384, 768 (3 * 2^a), 80, 160, 320, 640 (5 * 2^a),
 *    112, 224, 448, 896 (7 * 2^a); the lateral transforms are exact mixed-radix FFTs of that
 *    length (no padding, the boundary stays periodic).  Depth row j sits at z = j dz; sources and receivers are at row 0.
 *  - Slowness: device float32 [nz][nx] in s/m (row j contiguous).  Model / image: device
 *    float32 [nz][nx].
 *  - Frequencies: host float32 freq_hz[nw] (Hz; w = 2 pi f) and host float32 wavelet[nw][2]
 *    (interleaved real, imaginary source spectrum W(w)).
 *  - Geometry: host int32 src_ix[ns] (source grid column of each shot) and host int32
 *    rec_ix[ns][nrec] (receiver grid columns of each shot); rec_ix may be NULL when
 *    nrec == nx, meaning receivers at every column in order.  All indices in [0, nx).
 *  - Data: device complex64 [shots][nw][nrec] stored as interleaved float32 pairs
 *    (receiver index fastest).
 *  - Operator conventions (readings of the paper, which does not spell them out):
 *    lateral DFT F u[k] = sum_x u[x] exp(-2 pi i k x / nx) with a 1/nx inverse;
 *    kx = 2 pi k/(nx dx) for k < nx/2 and 2 pi (k - nx)/(nx dx) otherwise;
 *    s_ref(j) = mean_x s(x, j); Phi_j = exp(+i kz dz), kz = sqrt(w^2 s_ref^2 - kx^2) on the
 *    propagating band and exp(-sqrt(kx^2 - w^2 s_ref^2) dz) on the evanescent one;
 *    D_j(x) = exp(+i w (s(x, j) - s_ref(j)) dz); one depth step P_j = D_j F^-1 Phi_j F.
 *    Source S_0 = W(w) delta(x - x_s), S_{j+1} = P_j S_j.
 *    A m = sum_j P_0 ... P_{j-1} (S_j m_j) sampled at the receivers.
 *    A^T d: m_j(x) = Re sum_{shots, w} conj(S_j(x)) R_j(x), R_0 = injected data,
 *    R_{j+1} = P_j^H R_j.  A and A^T are adjoint under <u, v> = Re sum conj(u) v.
 *  - Memory: every device pointer is owned by the caller and must be 16-byte aligned.  The
 *    library allocates no device memory: all scratch lives in a caller-provided workspace of at
 *    least lsm_workspace_bytes(...) bytes.  Host arrays are read during the call only.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    lsm_forward and lsm_adjoint are asynchronous on that stream.  rls_window_solve
 *    synchronises the stream once per window with the default graph-replayed CG loop (once per CG
 *    iteration with the host-driven loop, to test convergence) and before returning.
 *  - Errors: every entry point returns an LSM_* status; arguments are validated on the host
 *    before anything is launched.  A call that fails validation launches nothing and leaves
 *    outputs untouched.  No kernel in this library waits on another block or device; the only
 *    waits are the tcgen05 transforms' waits on their own tensor-core work, each bounded (about a
 *    second, LSM_ERR_TIMEOUT).
 *  - Thread safety: calls sharing a workspace must be serialised by the caller.
 */
#ifndef LSM_GB300_H
#define LSM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LSM_OK 0
#define LSM_ERR_ARG (-1)            /* invalid argument (null pointer, out-of-range value) */
#define LSM_ERR_CUDA (-2)           /* a CUDA runtime call or kernel launch failed */
#define LSM_ERR_WORKSPACE (-3)      /* workspace smaller than lsm_workspace_bytes() */
#define LSM_ERR_BREAKDOWN (-4)      /* CG step length undefined: q^T q + lambda p^T p <= 0 or
                                       not finite (e.g. non-finite input data) */
#define LSM_ERR_TIMEOUT (-5)        /* a bounded device wait expired (tcgen05 transforms) */
#define LSM_ERR_UNSUPPORTED_NX (-6) /* nx is not one of the supported widths (see Grid) */

#define LSM_OP_FORWARD 0
#define LSM_OP_ADJOINT 1
#define LSM_OP_SOLVE 2
#define LSM_OP_GRADIENT 3

/* default depth stride of the source / adjoint wavefield checkpoints kept by lsm_born_gradient
 * (lsm_autotune_gradient may record another one of 8, 16, 32) */
#define LSM_CHECKPOINT_EVERY 16

typedef struct {
    int nx, nz;     /* lateral cells, depth rows */
    float dx, dz;   /* spacing in metres (> 0) */
} lsm_grid;

typedef struct {
    int ns;              /* number of shots in the survey */
    const int* src_ix;   /* host [ns] source grid columns */
    int nrec;            /* receivers per shot */
    const int* rec_ix;   /* host [ns][nrec] receiver columns, or NULL for every column */
} lsm_geom;

typedef struct {
    int nw;                 /* number of frequencies */
    const float* freq_hz;   /* host [nw] */
    const float* wavelet;   /* host [nw][2] interleaved source spectrum */
} lsm_freqs;

typedef struct {
    int start;          /* first shot of the window */
    int iters;          /* CG iterations taken in this window */
    double rel_res0;    /* ||A^T(d - A m0) - lambda m0|| / ||A^T d|| at the warm start m0 */
    double rel_res;     /* same ratio at the window's final image */
    int n_forward;      /* applications of A in this window */
    int n_adjoint;      /* applications of A^T in this window */
    float ms;           /* wall time of the window (host clock, includes synchronisation) */
} lsm_window_stats;

/*
 * Workspace size in bytes for one call.
 *   op = LSM_OP_FORWARD / LSM_OP_ADJOINT: nshots = shots processed per call.
 *   op = LSM_OP_SOLVE: nshots = the window length K.
 *   op = LSM_OP_GRADIENT: nshots = shots per lsm_born_gradient call.
 * The size depends on the current device's multiprocessor count (152 is assumed when no
 * device is visible), so query it with the device that will run the call current.
 * Returns 0 for invalid arguments.
 */
size_t lsm_workspace_bytes(const lsm_grid* grid, const lsm_geom* geom, const lsm_freqs* freqs,
                           int nshots, int op);

/*
 * De-migration d = A m (Eq. 1 without the noise term) for shots shot0 .. shot0+nshots-1.
 *   slowness: device [nz][nx]; m: device [nz][nx];
 *   d_out: device complex64 [nshots][nw][nrec], overwritten.
 * Evaluated per (shot, w) by Horner's rule from the deepest row upward:
 *   U_{nz-1} = S_{nz-1} m_{nz-1}, U_j = S_j m_j + P_j U_{j+1}, d = U_0 at the receivers,
 * after computing and caching S_j for every depth in the workspace.
 */
int lsm_forward(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs,
                const lsm_geom* geom, const float* m, float* d_out, int shot0, int nshots,
                void* workspace, size_t workspace_bytes, void* stream);

/*
 * Migration m = A^T d (Eq. 2) for shots shot0 .. shot0+nshots-1.
 *   d: device complex64 [nshots][nw][nrec] (the data of those shots);
 *   m_out: device [nz][nx]; overwritten when accumulate == 0, added to otherwise.
 * The image is summed over shots and frequencies in a fixed order, so repeated calls with the
 * same inputs and workspace size give bitwise identical results.
 */
int lsm_adjoint(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs,
                const lsm_geom* geom, const float* d, float* m_out, int shot0, int nshots,
                int accumulate, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Modelling and gradients for differentiable use of d = A(s) m (Eq. 1), e.g. behind an autograd
 * function whose backward is the adjoint.  The reference slowness of the split-step operator is held
 * fixed: `sref` is a device float64 [nz] array (for example the row means of a background model),
 * or NULL for the row means of `slowness`.  Only the split-step factor D_j then depends on s, and
 * the derivatives follow the adjoint-state recursion
 *   R_0 = injected g, R_{j+1} = P_j^H R_j;  U_j = S_j m_j + P_j U_{j+1};
 *   mu_nz = 0, mu_j = m_j R_j + P_j^H mu_{j+1};
 *   grad_m_j = Re sum conj(S_j) R_j   (= A^T g, Eq. 2),
 *   grad_s_j = Re sum i w dz [conj(R_j) P_j U_{j+1} + conj(mu_{j+1}) S_{j+1}],
 * summed over the shots and frequencies.  S and R are swept down once keeping only every c-th
 * depth, and recomputed segment by segment while U and mu run up; c is LSM_CHECKPOINT_EVERY unless
 * lsm_autotune_gradient recorded a stride for this problem (the results do not depend on c).
 *   m: device float32 [nz][nx];
 *   g: device complex64 [nshots][nw][nrec], dL/dRe(d) + i dL/dIm(d) (the convention of PyTorch
 *      complex gradients), or NULL to only model d;
 *   d_out: device complex64 [nshots][nw][nrec] or NULL (required when g is NULL);
 *   grad_m, grad_s: device float32 [nz][nx] or NULL; overwritten.
 * Workspace: lsm_workspace_bytes(..., nshots, LSM_OP_GRADIENT).  Gradients need a power-of-two nx
 * from 16 to 1024 (LSM_ERR_UNSUPPORTED_NX otherwise); modelling supports every nx of lsm_forward.
 */
int lsm_born_gradient(const lsm_grid* grid, const float* slowness, const double* sref,
                      const lsm_freqs* freqs, const lsm_geom* geom, const float* m,
                      const float* g, float* d_out, float* grad_m, float* grad_s, int shot0,
                      int nshots, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Number of sliding windows of K shots with the given slide over ns shots: starts are
 * 0, slide, 2 slide, ... while start + K <= ns, plus a final window at ns - K when the regular
 * schedule stops short of the last shot.  Returns 0 for invalid arguments.
 */
int lsm_num_windows(int ns, int K, int slide);

/*
 * Block-row recursive least-squares migration (block-row section, Eq. 10 and Eq. 11).
 * Windows first_window .. first_window + n_windows - 1 (n_windows <= 0: all remaining) of the
 * schedule of lsm_num_windows are solved in order.  Each window k runs CG on
 *   (A_k^T A_k + lambda I) m = A_k^T d_k
 * starting from the image in m_inout (the previous window's result, Eq. 11), until
 *   ||A_k^T (d_k - A_k m) - lambda m|| / ||A_k^T d_k|| <= cg_tol
 * or max_iter iterations.  Dot products, step lengths and beta are float64 on the device; the
 * vectors are float32.  Moving the window drops the first `slide` shots and adds the next ones
 * (rank-`slide` downdate/update): only the added shots' source wavefields are computed.
 *   d: device complex64 [ns][nw][nrec] (the whole survey);
 *   lambda >= 0 (absolute); K in [1, ns]; slide >= 1; cg_tol >= 0; max_iter >= 0;
 *   m_inout: device [nz][nx], the warm start on entry and the last window's image on return;
 *   stats: host array of stats_cap entries (may be NULL), filled for each solved window.
 * Resuming with first_window = k and the image returned after window k-1 reproduces an
 * uninterrupted run bitwise.  Returns LSM_ERR_BREAKDOWN if a step length is undefined; m_inout
 * then holds the last finite iterate.
 */
int rls_window_solve(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs,
                     const lsm_geom* geom, const float* d, double lambda, int K, int slide,
                     double cg_tol, int max_iter, int first_window, int n_windows,
                     float* m_inout, lsm_window_stats* stats, int stats_cap,
                     void* workspace, size_t workspace_bytes, void* stream);

/*
 * Migration m = A^T d for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a packaging variant of lsm_adjoint for code that must not
 * call cudaMalloc or any allocating routine (for example a plug-in running inside a host process
 * that owns every device allocation, or a step that must not allocate once it is set up).  It takes
 * the same arguments as lsm_adjoint minus the workspace: its scratch (coefficient tables, source
 * wavefields, partial images) lives in one fixed static device array of LSM_STATIC_SCRATCH_BYTES,
 * which every GPU that loads the library keeps until the process exits.
 *  - The caller still owns and passes d and m_out; nothing is allocated, freed or resized.
 *  - Problems whose scratch (lsm_workspace_bytes(..., LSM_OP_ADJOINT)) exceeds
 *    LSM_STATIC_SCRATCH_BYTES are rejected with LSM_ERR_WORKSPACE before anything is launched.
 *  - Each call made outside a stream capture looks up the array's device address on the current
 *    device (cudaGetSymbolAddress) and remembers it; a call made while `stream` is being captured
 *    uses the remembered address, so make the first call on each device before any stream capture
 *    (and again after a device reset, which reloads the library's device code).
 *  - The host arrays (src_ix, rec_ix, freq_hz, wavelet) are copied into a host buffer owned by the
 *    call before it returns, like every other entry point does: the caller may change or free
 *    them, pinned or not, as soon as the call returns.
 *  - All calls share the one array and it keeps the last call's contents; every region is fully
 *    rewritten before it is read, so results do not depend on earlier calls.  Calls that overlap
 *    on the GPU (other streams, other host threads) race on the array: serialise them.
 */
#define LSM_STATIC_SCRATCH_BYTES (64u << 20)
int lsm_adjoint_static(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs,
                       const lsm_geom* geom, const float* d, float* m_out, int shot0, int nshots,
                       int accumulate, void* stream);

/*
 * Kernel timing for benchmarks.  Between lsm_profile_start() and lsm_profile_stop() every kernel
 * this library launches is bracketed by CUDA events recorded on the stream it is launched on;
 * lsm_profile_stop() waits for those events and reports, per kernel class, the number of launches
 * and the summed event time in milliseconds.  Timing adds two event records per launch.  Not
 * thread safe: profile one caller at a time.  lsm_profile_start_classes(mask) times only the
 * kernel classes whose bit (1 << LSM_KCLASS_...) is set in mask, so that a benchmark can time the
 * kernels it reports without adding event records around the others; lsm_profile_start() times
 * every class.
 */
#define LSM_KCLASS_TABLES 0   /* reference slowness and coefficient tables */
#define LSM_KCLASS_SOURCE 1   /* source-wavefield depth sweep */
#define LSM_KCLASS_ADJOINT 2  /* A^T depth sweep (imaging) */
#define LSM_KCLASS_FORWARD 3  /* A depth sweep */
#define LSM_KCLASS_VECTOR 4   /* image reduction and CG vector updates */
#define LSM_KCLASS_GRADIENT 5 /* lsm_born_gradient's checkpointed gradient sweep */
#define LSM_NUM_KCLASSES 6

typedef struct {
    unsigned long long launches[LSM_NUM_KCLASSES];
    double ms[LSM_NUM_KCLASSES];
} lsm_profile;

void lsm_profile_start(void);
void lsm_profile_start_classes(unsigned class_mask);
int lsm_profile_stop(lsm_profile* out);

/*
 * Solver options for rls_window_solve_ex.
 *   preconditioner: LSM_PRECOND_NONE, or LSM_PRECOND_ILLUMINATION for preconditioned CG with the
 *     diagonal source-illumination preconditioner of each window,
 *     M = sum_{shots in window, w} |S_j(x)|^2 + precond_eps * max (M^-1 applied to the model
 *     residual).  The paper asks for preconditioners that cluster the spectrum of each windowed
 *     Hessian (block-row section) without naming one; this is the reading.  The stopping rule stays
 *     the unpreconditioned ||A_k^T (d_k - A_k m) - lambda m|| / ||A_k^T d_k||.
 *   precond_eps: > 0, relative stabiliser (1e-2 is a good default).
 */
#define LSM_PRECOND_NONE 0
#define LSM_PRECOND_ILLUMINATION 1
/*
 *   transform: the lateral transforms of every depth step.
 *     LSM_TRANSFORM_FFT (0): register-resident FP32 FFTs (every supported nx).
 *     LSM_TRANSFORM_DFT_BF16X3, _FP16X3, _BF16X1: the transforms as DFT-matrix products on the
 *     tensor cores (four-step 16 x nx/16 factorisation, mma.sync with FP32 accumulation), with every
 *     FP32 operand split as hi + lo in bf16 (three products), in fp16 with the lo part scaled by
 *     2^11 (three products), or bf16 hi only (one product).  These are precision variants for
 *     every supported nx (for nx/16 not a multiple of 8 the 16 x nx/16 matrix is zero-padded to
 *     whole 8-column tiles) with receivers at every column (rec_ix NULL); LSM_ERR_ARG otherwise.
 */
/*
 *     LSM_TRANSFORM_DFT_FP16X3_TCGEN05, _BF16X3_TCGEN05: the same four-step DFT products, split FP16
 *     (lo scaled by 2^11, two accumulators) or split BF16 three-term, on the fifth-generation tensor
 *     cores: tcgen05.mma issued by one thread per CTA with 128-byte-swizzled operands in shared
 *     memory and FP32 accumulators in tensor memory, eight (shot, frequency) items per 128-thread
 *     CTA stacked as the MMAs' 128-row tiles (16 items at nx = 128; a 256-thread CTA at nx = 1024;
 *     lsm_tcgen05_shape gives the launch shape).  nx = 128, 256, 512 and 1024 (LSM_ERR_UNSUPPORTED_NX otherwise), receivers at every
 *     column.  Every wait of these kernels on the tensor core is bounded (about a second);
 *     one that runs out leaves NaN in the call's outputs, and rls_window_solve_ex then returns
 *     LSM_ERR_TIMEOUT.
 */
#define LSM_TRANSFORM_FFT 0
#define LSM_TRANSFORM_DFT_BF16X3 1
#define LSM_TRANSFORM_DFT_FP16X3 2
#define LSM_TRANSFORM_DFT_BF16X1 3
#define LSM_TRANSFORM_DFT_FP16X3_TCGEN05 4
#define LSM_TRANSFORM_DFT_BF16X3_TCGEN05 5
/*
 *   cuda_graph: LSM_CUDA_GRAPH_WINDOW (1) runs each window's CG iterations as one CUDA graph -- a
 *     conditional WHILE node whose body is one iteration (A, the vector updates, A^T, the stopping
 *     test evaluated on the device) -- so the host waits once per window instead of once per
 *     iteration.  The kernels and their order are those of the host-driven loop, so results and
 *     iteration counts are identical.  The graph is built once per call on a private stream; kernels
 *     inside it are not seen by lsm_profile_start / lsm_profile_stop.  LSM_CUDA_GRAPH_SOLVE (2) runs
 *     the whole call as one graph launch: every window's set-up launches, its loop test and WHILE
 *     node, and a node that records its outcome in the workspace, chained window after window (for
 *     rls_multi_line_solve: every line's chain as an independent branch of the same graph, launched
 *     once on lines[0].stream after each line's tables are built on its own stream), so the host
 *     waits once per call; same kernels, order, results and iteration counts again, window
 *     statistics as usual except `ms` = 0 (the windows are not timed one by one); after a window
 *     breaks down the later windows of that line run no iterations, and the call returns
 *     LSM_ERR_BREAKDOWN with statistics up to that window.  < 0 runs the host-driven loop (the host
 *     reads the stopping test back after every iteration).  0, the default (also for
 *     rls_window_solve and NULL options), runs the per-window graph unless lsm_profile_start /
 *     lsm_profile_start_classes is timing the A or A^T sweeps, which needs the host-driven loop.
 *     Values above 2: LSM_ERR_ARG.
 */
#define LSM_CUDA_GRAPH_WINDOW 1
#define LSM_CUDA_GRAPH_SOLVE 2
typedef struct {
    int preconditioner;
    double precond_eps;
    int transform;
    int cuda_graph;
} lsm_solve_options;

/* lsm_forward / lsm_adjoint with solver options (only `transform` applies; NULL: FP32 FFTs). */
int lsm_forward_ex(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs,
                   const lsm_geom* geom, const float* m, float* d_out, int shot0, int nshots,
                   void* workspace, size_t workspace_bytes, void* stream,
                   const lsm_solve_options* options);
int lsm_adjoint_ex(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs,
                   const lsm_geom* geom, const float* d, float* m_out, int shot0, int nshots,
                   int accumulate, void* workspace, size_t workspace_bytes, void* stream,
                   const lsm_solve_options* options);

/* rls_window_solve with options (options == NULL: plain CG, identical to rls_window_solve). */
int rls_window_solve_ex(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs,
                        const lsm_geom* geom, const float* d, double lambda, int K, int slide,
                        double cg_tol, int max_iter, int first_window, int n_windows,
                        float* m_inout, lsm_window_stats* stats, int stats_cap,
                        void* workspace, size_t workspace_bytes, void* stream,
                        const lsm_solve_options* options);

/*
 * One sliding-window solve sharded over several ranks (processes, typically one per GPU) by
 * frequency.  Inside a window the (shot, frequency) items of A and A^T are independent (Eq. 1,
 * Eq. 2), so each rank runs the operator on its own subset of the frequencies -- `freqs` and `d`
 * ([ns][nw_rank][nrec]) hold this rank's frequencies only -- while the model-space vectors (image,
 * CG directions) are kept whole on every rank.  Two sums over the ranks make the ranks' CG identical
 * (Eq. 10, Eq. 11): the image of every A^T (nz nx float32 values, once per CG iteration and twice
 * per window set-up) and ||q||^2 of every A (one float64 value per CG iteration), each through the
 * caller's callback
 *   allreduce(ctx, buf, count, is_double, stream): replace `count` float32 (is_double == 0) or
 *   float64 values at device address `buf` by their sum over the ranks, ordered on `stream`;
 *   return 0 on success (anything else ends the solve with LSM_ERR_CUDA).
 * Every rank must call with the same grid, slowness, geometry, lambda, K, slide, tolerance, limits
 * and image; the ranks then take the same iterations and return the same image (up to the order in
 * which the callback adds the ranks' values).  Plain CG with the FP32 FFT transforms and the
 * host-driven loop; the workspace is lsm_workspace_bytes(grid, geom, freqs, K, LSM_OP_SOLVE) for this
 * rank's frequencies.  Other arguments and results as for rls_window_solve.
 */
typedef int (*lsm_allreduce_fn)(void* ctx, void* buf, size_t count, int is_double, void* stream);
int rls_window_solve_sharded(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs,
                             const lsm_geom* geom, const float* d, double lambda, int K, int slide,
                             double cg_tol, int max_iter, int first_window, int n_windows,
                             float* m_inout, lsm_window_stats* stats, int stats_cap,
                             void* workspace, size_t workspace_bytes, void* stream,
                             lsm_allreduce_fn allreduce, void* allreduce_ctx);

/*
 * Several independent survey lines solved together (batching): each line is a complete
 * rls_window_solve_ex problem with its own grid (any supported nx), data, window length K, slide,
 * tolerance, image, statistics, workspace and stream.  The lines run concurrently, so small lines
 * overlap on the GPU instead of running one after another: by default one host worker thread per
 * line issues that line's kernels on that line's stream; with options->cuda_graph =
 * LSM_CUDA_GRAPH_SOLVE every window of every line is one graph launched once (see cuda_graph).  Every line's result is bitwise identical to solving it
 * alone with rls_window_solve_ex.  Streams must be distinct (and not the legacy default stream) for
 * the lines to overlap.  Fields are the arguments of rls_window_solve_ex; `status` receives the
 * line's return code.  Returns LSM_OK when every line succeeded, else the first failing line's
 * code.  The calling thread's current device is used for every line.
 */
typedef struct {
    lsm_grid grid;
    const float* slowness;
    lsm_freqs freqs;
    lsm_geom geom;
    const float* d;
    double lambda;
    int K, slide;
    double cg_tol;
    int max_iter;
    float* m_inout;
    lsm_window_stats* stats;
    int stats_cap;
    void* workspace;
    size_t workspace_bytes;
    void* stream;
    int status;
} lsm_line;

int rls_multi_line_solve(lsm_line* lines, int nlines, const lsm_solve_options* options);

/*
 * Launch-shape and FFT-tile autotuning (an implementation choice, not a step of the paper's method).
 * The depth sweeps run a fixed number of (shot, frequency) items per warp, and the number of warps
 * per block sets how many items share a block's staged coefficient rows and how the launch fills the
 * SMs; the default spreads a launch evenly over the SMs.  With the FP32 FFTs the FFT tile -- the
 * points of a line each thread holds -- is tuned too: every width but 768, 896 and 1024 also has a
 * compiled tile with half the default points per thread (twice the threads per item: a smaller or
 * deeper FFT plan, or at nx = 512 the same 32 x 16 stages with each 32-point first-stage DFT shared
 * by two lanes of the warp that holds the item).  lsm_autotune times, for each tile, every admissible number of warps per block for
 * the source, A^T and A sweeps of launches over `nshots` shots of this grid and frequency set (for a
 * solve: nshots = K), with the FP32 FFTs or, when options->transform selects one, the tensor-core DFT
 * products, and records the fastest shape per sweep and the tile whose best A plus best A^T is
 * fastest.  From then on every call on the current device with the same (nx, nshots, nw) builds its
 * coefficient tables for the recorded tile and every launch with the same (nx, mode, transform,
 * tile, nshots, nw) uses the recorded shape (process-wide, thread safe); results stay within the
 * same tolerances, but the FFT's rounding and A^T's sum over block partial images, and so their last
 * bits, follow the tile and the shape.  The A^T candidates never use more
 * blocks than the default, so lsm_workspace_bytes is unchanged.  Needs a workspace of
 * lsm_workspace_bytes(grid, geom, freqs, nshots, LSM_OP_SOLVE); runs shots [0, nshots) on
 * zero-valued inputs, overwrites the workspace, and returns after synchronising the stream.
 * `report` (may be NULL) receives, per sweep of the chosen tile, the chosen and the default warps per
 * block with their mean launch times in ms and the number of shapes timed, and the chosen and default
 * tiles with their A + A^T times.  lsm_autotune_reset forgets every recorded shape and tile.
 */
typedef struct {
    int warps, heuristic_warps, candidates;
    double ms, heuristic_ms;
} lsm_tune_entry;
typedef struct {
    lsm_tune_entry source, adjoint, forward;  /* of the chosen FFT tile */
    int points_per_thread;           /* the chosen FFT tile (register FFTs; the sweeps' own otherwise) */
    int default_points_per_thread;   /* the default tile */
    int tiles;                       /* FFT tiles timed (1 or 2) */
    double tile_ms, default_tile_ms; /* best A + best A^T launch times, chosen and default tile */
} lsm_tune_report;

int lsm_autotune(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs,
                 const lsm_geom* geom, int nshots, const lsm_solve_options* options,
                 void* workspace, size_t workspace_bytes, void* stream, lsm_tune_report* report);

/*
 * The FFT tiles compiled for width nx: writes up to `cap` of them (points per thread, the default
 * first) to `tiles` (may be NULL) and returns how many there are (1 or 2; 0 for an unsupported nx).
 * lsm_set_fft_tile records `points_per_thread` as the tile of calls over `nshots` shots of nx columns
 * and nw frequencies on the current device, as lsm_autotune would (LSM_ERR_ARG for a tile that is not
 * compiled for nx, LSM_ERR_UNSUPPORTED_NX for an unsupported nx).  Launch shapes of that tile not
 * tuned yet are the heuristic's.
 */
int lsm_fft_tiles(int nx, int* tiles, int cap);
int lsm_set_fft_tile(int nx, int nshots, int nw, int points_per_thread);

/*
 * Launch shape of the tcgen05 transform variants for a call over `nshots` shots of nx columns and
 * nw frequencies (host only; no device is touched): (shot, frequency) items per CTA, threads per
 * CTA, CTAs, frequency slots whose Phi and D rows a CTA stages in shared memory (0: the rows are
 * read from global memory because a CTA's frequencies would not fit its shared memory) and its
 * dynamic shared-memory bytes.  Any output pointer may be NULL.  LSM_ERR_UNSUPPORTED_NX for a width
 * without tcgen05 variants, LSM_ERR_ARG for nshots < 1 or nw < 1.
 */
int lsm_tcgen05_shape(int nx, int nshots, int nw, int* items, int* threads, int* blocks, int* wslots,
                      size_t* smem_bytes);

/*
 * Checkpoint stride and launch shape of lsm_born_gradient.  The gradient sweep keeps S and R at
 * every c-th depth and recomputes them segment by segment, so its arithmetic and its results are the
 * same for every c; c sets how many checkpoint and segment rows each (shot, frequency) item keeps
 * and how much of that traffic stays in L2.  The number of warps per block sets how evenly the
 * launch's blocks fill the SMs' last round.  lsm_autotune_gradient times the gradient kernel of a
 * launch over `nshots` shots of this grid and frequency set at c = LSM_CHECKPOINT_EVERY, 8, 16 and
 * 32 (strides above nz act as nz) and at the default number of warps per block and up to two fewer,
 * and records the fastest pair; from then on lsm_born_gradient calls on the current device with the
 * same (nx, nz, nshots, nw) use it.  lsm_workspace_bytes(..., LSM_OP_GRADIENT) already reserves
 * room for every candidate.  Needs a workspace of lsm_workspace_bytes(grid, geom, freqs, nshots,
 * LSM_OP_GRADIENT); runs shots [0, nshots) on zero-valued model and data-space gradient, overwrites
 * the workspace, and returns after synchronising the stream.  Gradients need a power-of-two nx from
 * 16 to 1024 (LSM_ERR_UNSUPPORTED_NX otherwise).  `report` (may be NULL) receives the chosen and the default
 * stride and warps per block, their mean launch times in ms and the number of pairs timed.  The
 * gradients do not depend on the stride; the warps per block change the block partition of the
 * image sums and so their last bits.  lsm_autotune_reset also forgets these choices.
 */
typedef struct {
    int stride, default_stride;
    int warps, default_warps;
    int candidates;
    double ms, default_ms;
} lsm_ckpt_tune_report;

int lsm_autotune_gradient(const lsm_grid* grid, const float* slowness, const lsm_freqs* freqs,
                          const lsm_geom* geom, int nshots, void* workspace, size_t workspace_bytes,
                          void* stream, lsm_ckpt_tune_report* report);
void lsm_autotune_reset(void);

/*
 * Measured FP32 arithmetic peak of the current device, in TFLOP/s (a measurement utility with no
 * counterpart in the paper: the depth sweeps are bound by the FP32 pipe, and their roofline is
 * reported against this).  Times, with CUDA events on `stream`, launches of a kernel whose threads
 * run independent chains of fused multiply-adds (eight 256-thread blocks per SM), once with scalar
 * FMA instructions and once with the paired FP32 FMA instructions of sm_100-class GPUs; each result
 * is the flop count (2 per FMA) over the fastest of five timed launches.  Synchronises the stream;
 * takes about 20 ms.  Returns LSM_ERR_ARG for NULL outputs, LSM_ERR_CUDA on a CUDA failure.
 */
int lsm_measure_fp32_peak(double* tflops_ffma, double* tflops_ffma2, void* stream);

/*
 * Self-check of the bounded device waits (a failure-handling check with no counterpart in the
 * paper).  Launches one block that waits on an mbarrier nothing arrives at, with the same bounded
 * wait the tcgen05 transforms use; the wait must give up after about a second and the kernel return
 * normally.  Returns LSM_ERR_TIMEOUT when it did (the expected outcome: the context stays usable),
 * LSM_OK if the wait completed, LSM_ERR_CUDA on a CUDA failure.  Synchronises the stream.
 */
int lsm_check_bounded_wait(void* stream);

/* Human-readable name of a status code (static string). */
const char* lsm_status_string(int status);

/* Number of kernels this library has launched in this process (monotonic counter). */
unsigned long long lsm_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* LSM_GB300_H */
