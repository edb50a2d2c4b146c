/*
 * bttb.h -- C ABI of the GB300 solver for two-level block-Toeplitz
 * Method-of-Moments systems  Z I = V  (Akerstedt et al., "Solver Performance
 * of Accelerated MoM for Connected Arrays", arXiv:2506.20350).
 *
 * The matrix (Sec. II-A, Eq. (Tblock) with L = 2) belongs to an nx x ny
 * array of identical cells with b basis functions each, N = nx*ny*b:
 *   Z[(m*b + p), (n*b + q)] = T[ix_m - ix_n, iy_m - iy_n][p][q],
 *   cell m = iy_m*nx + ix_m, offsets i in [-(nx-1), nx-1], j in [-(ny-1), ny-1].
 * Only the (2nx-1)(2ny-1) generator blocks T[i,j] (b x b) are stored
 * (Sec. II-C).  Products use the multilevel FFT of Sec. II-C / III-A:
 * zero-pad onto an mx x my cell grid (Eq. (xc2)), 2-D DFT over cells for every
 * basis index (Eq. (F2), App. B), per-bin b x b block product with the
 * spectrum of the first block column (Eq. (circL2), (multL)), inverse DFT and
 * crop.  mx, my are the smallest 5-smooth integers >= 2nx-1, 2ny-1; any grid
 * at least that large gives the same product (the padded slots hold zeros).
 *
 * Conventions for every entry point
 *  - Complex numbers are interleaved (re, im): BTTB_C128 = 2 x double,
 *    BTTB_C64 = 2 x float.
 *  - A vector holds element (ix, iy, p) at (iy*nx + ix)*b + p; column c of a
 *    multi-vector starts at c*ld elements.
 *  - Pointers are DEVICE pointers unless an argument or option says host.
 *    The caller owns every buffer it passes; the plan owns its spectrum copies
 *    and workspace and frees them in bttb_plan_destroy.
 *  - Functions never exit, abort or trap.  They return BTTB_OK (0), a soft
 *    outcome (> 0) or an error (< 0); bttb_last_error() gives a message.
 *    Device-side problems (a bounded wait that ran out, a non-finite norm)
 *    set a flag in the plan that the next synchronising call returns.
 *  - One plan per CUDA stream; a plan is not thread-safe.
 *
 * "FP64" below means a result within ~1e-14 relative of binary64.  On this
 * GPU the binary64 pipe is ~30x slower than the binary32 pipes, so the FP64
 * product and the Krylov vector work run in double-float arithmetic (an
 * unevaluated sum hi + lo of two binary32 numbers, 48-bit significand,
 * Dekker 1971 / Joldes-Muller-Popescu 2017) on the binary32 pipes, reading the
 * same 8 bytes per real number as binary64.  BTTB_MV_FP64_NATIVE keeps the
 * IEEE binary64 pipe for comparison.
 */
#ifndef BTTB_H
#define BTTB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bttb_plan_s *bttb_plan;

/* Storage type of a caller's vectors and generators. */
typedef enum { BTTB_C64 = 0, BTTB_C128 = 1 } bttb_dtype;

/* Arithmetic of a product.  Bit (1u << prec) of a plan's prec_mask asks the
 * plan to keep the spectrum copy that precision reads. */
typedef enum {
    BTTB_MV_FP64 = 0,        /* double-float spectrum (hi+lo planes) and arithmetic  */
    BTTB_MV_FP32 = 1,        /* binary32 spectrum (the hi plane) and arithmetic      */
    BTTB_MV_FP64_NATIVE = 2, /* binary64 spectrum copy, binary64 (DFMA) arithmetic   */
    BTTB_MV_TC_3XTF32 = 3,   /* binary32 FFT passes; with >= 16 columns the per-bin
                                GEMM runs on the tensor cores in 3xTF32 (each factor
                                split into a TF32 head and tail, three MMAs, binary32
                                accumulation: binary32-level accuracy): tcgen05 MMAs
                                with TMA-fed tiles for even b <= 64, warp-level MMAs
                                for odd b <= 64; otherwise as BTTB_MV_FP32.  Reads the
                                binary32 spectrum (hi plane).                         */
    BTTB_MV_TC_BF16X3 = 4    /* as BTTB_MV_TC_3XTF32 with each factor split into two
                                bfloat16 terms (split-BF16x3, tcgen05 for even b <= 64,
                                else as BTTB_MV_FP32): about 2^-17 relative error per
                                product term                                          */
} bttb_mv_prec;

typedef enum {
    BTTB_PC_NONE = 0,
    BTTB_PC_BLOCK_JACOBI = 1, /* P_K of Sec. III-B: LU of T[0,0] applied to every cell */
    BTTB_PC_LEARNED = 2       /* P_K^{-1} r + f(r), f the learned Fourier-domain
                                 correction attached with bttb_plan_set_learned      */
} bttb_precond;

enum {
    BTTB_OK = 0,
    BTTB_NOT_CONVERGED = 1,  /* soft: max_iters reached before tol                  */
    BTTB_BREAKDOWN = 2,      /* soft: Krylov space exhausted without reaching tol    */
    BTTB_ERR_INVALID_ARG = -1,
    BTTB_ERR_CUDA = -2,
    BTTB_ERR_OOM = -3,
    BTTB_ERR_NO_GENERATORS = -4,
    BTTB_ERR_TIMEOUT = -5,   /* a bounded device wait ran out (kernel returned early) */
    BTTB_ERR_NONFINITE = -6, /* NaN/Inf seen in a norm or in the generators           */
    BTTB_ERR_SINGULAR = -7   /* zero pivot in the block-Jacobi LU of T[0,0]            */
};

/*
 * Create a plan for an nx x ny array with b bases per cell.
 *   max_rhs   : largest nrhs a later call may pass (sizes the workspace).
 *   prec_mask : OR of (1u << bttb_mv_prec) for the precisions to support;
 *               0 means FP64 | FP32.
 *   cuda_stream: cudaStream_t (NULL = legacy default stream) on which every
 *               call of this plan is ordered.
 * Picks the FFT grid (mx, my).  Returns BTTB_ERR_INVALID_ARG for sizes < 1,
 * nx or ny > 1024, b > 256 or max_rhs > 4096; BTTB_ERR_OOM / _CUDA on failure.
 */
int bttb_plan_create(bttb_plan *out, int nx, int ny, int b, int max_rhs,
                     unsigned prec_mask, void *cuda_stream);

/* FFT grid chosen by the plan (either pointer may be NULL). */
int bttb_plan_grid(bttb_plan plan, int *mx, int *my);

/*
 * Load the generator blocks and compute their spectrum (Eq. (circL2),
 * (multL)): T[i,j] goes to cell slot (i mod mx, j mod my) of the zero grid,
 * and each of the b*b entries gets a 2-D DFT, in binary64 on the GPU.  The
 * plan then keeps the copies its prec_mask asks for, scaled by 1/(mx*my).
 *   gen        : T[i,j][p][q] at ((j+ny-1)*(2nx-1) + (i+nx-1))*b*b + p*b + q,
 *                p the observer basis (row), q the source basis (column).
 *   dtype      : storage type of gen.
 *   gen_is_host: nonzero if gen is a host pointer.
 * Synchronises the plan's stream; with a device pointer it first waits for all
 * work already queued on the device (gen may come from any stream).  The
 * caller may free gen on return.  Returns BTTB_ERR_NONFINITE if gen holds
 * NaN/Inf.
 */
int bttb_set_generators(bttb_plan plan, const void *gen, bttb_dtype dtype, int gen_is_host);

/*
 * y[:, c] = Z x[:, c] for c < nrhs (Eq. (multL) with padding and crop of
 * Eq. (xc2)).  x and y are device multi-vectors of type dtype with column
 * stride ld >= N elements; they must not overlap.  Stream-ordered on the
 * plan's stream; does not synchronise.  nrhs <= max_rhs.
 */
int bttb_matvec(bttb_plan plan, const void *x, void *y, int nrhs, long ld,
                bttb_dtype dtype, bttb_mv_prec prec);

/* GMRES options (Sec. III-C hands the product to restarted GMRES). */
typedef struct {
    double tol;          /* stop when ||V - Z I||_2 / ||V||_2 <= tol (per column) */
    int restart;         /* Krylov dimension m of GMRES(m), 1..200                */
    int max_iters;       /* total Arnoldi steps per column                         */
    bttb_precond pc;     /* right preconditioner (the residual stays the true one) */
    bttb_mv_prec inner;  /* precision of the products inside a restart cycle:
                            FP64 = plain GMRES; FP32 or TC_* = GMRES-IR (each
                            cycle's starting residual is recomputed with the FP64
                            product, Arnoldi/Givens stay FP64)                    */
    int use_x0;          /* nonzero: I holds the initial guess on entry            */
    int host_io;         /* nonzero: V and I are HOST pointers (complex128); the
                            library copies them in and out on the plan's stream  */
    double *history;     /* optional HOST array: true relative residual of column 0
                            at the start of each restart cycle                     */
    int history_len;     /* capacity of history                                    */
    int flags;           /* OR of BTTB_GMRES_* below; 0 = defaults                 */
} bttb_gmres_opts;

/* Each restart cycle (m Arnoldi steps, back substitution, update) runs as one
 * CUDA graph replayed per cycle; finished columns make the remaining kernels of
 * the cycle exit at once.  BTTB_GMRES_NO_GRAPH launches the same kernels from
 * the host instead, with one host synchronisation per step.
 *
 * BTTB_GMRES_GLOBAL (nrhs > 1): the global GMRES of Sec. III-C, Eq. (ZIVvec):
 * one Krylov space for vec(I) of the system (I (x) Z) vec(I) = vec(V), with
 * Frobenius inner products, instead of one Krylov space per column.  Every
 * column stays in the space until all columns meet tol (each cycle targets a
 * Frobenius residual of tol * min_c ||V_c||); every column reports the same
 * iteration count and its own true residual.  Default: one space per column,
 * converged columns masked.
 *
 * Orthogonalisation is classical Gram-Schmidt applied twice (CGS2).  Without a
 * preconditioner and with block-Jacobi (a fixed linear operator: plain right
 * preconditioning, x += P_K^{-1} Q y at the end of each cycle) the default is
 * its delayed form (the reorthogonalisation of v_j is merged into step j+1's
 * reduction: one reduction and one update over the basis per step, and the
 * residual estimate one step behind); the learned preconditioner runs flexible
 * GMRES with the two-pass form, which BTTB_GMRES_CGS2 selects everywhere. */
enum { BTTB_GMRES_NO_GRAPH = 1, BTTB_GMRES_GLOBAL = 2, BTTB_GMRES_CGS2 = 4 };

typedef struct {
    int status;          /* BTTB_OK, BTTB_NOT_CONVERGED or BTTB_BREAKDOWN          */
    int iters;           /* Arnoldi steps taken                                    */
    int cycles;          /* restart cycles taken                                   */
    double relres_true;  /* ||V - Z I|| / ||V|| with the FP64 product, at return   */
} bttb_col_result;

/*
 * Solve Z I[:, c] = V[:, c] for c < nrhs with restarted GMRES(m), the product
 * above, classical Gram-Schmidt applied twice and Givens rotations in FP64.
 * V and I are complex128 with column stride ld (device pointers unless
 * opts->host_io).  x0 = 0 unless use_x0.  out_host (nrhs entries, host) gets
 * the per-column outcome.  Synchronises the plan's stream.  Returns the worst
 * column status (an error < 0 takes precedence).
 */
int bttb_gmres_solve(bttb_plan plan, const void *V, void *I, int nrhs, long ld,
                     const bttb_gmres_opts *opts, bttb_col_result *out_host);

/*
 * z[:, c] = P_K^{-1} x[:, c] (Sec. III-B): every cell's b-block is solved with
 * one LU (partial pivoting, FP64) of the self block T[0,0].  Device
 * multi-vectors of type dtype, stream-ordered.  Needs bttb_set_generators.
 */
int bttb_block_jacobi_apply(bttb_plan plan, const void *x, void *z, int nrhs, long ld,
                            bttb_dtype dtype);

/*
 * Copy the stored spectrum of bin (ky, kx) -- the b x b block of
 * F[2] C_1[2] / (mx*my), entry (p, q) at p*b + q -- into host memory
 * (complex128).  Reads the binary64 copy if the plan keeps one, else the
 * double-float planes summed in binary64.  Synchronises the stream.
 */
int bttb_get_spectrum_bin(bttb_plan plan, int ky, int kx, double *out_host);

/*
 * Kernel timing.  While enabled, the plan brackets every launch of the block
 * product and of the FFT passes with CUDA events on its stream and counts
 * every kernel it launches.  bttb_profile(plan, 1) clears and starts,
 * bttb_profile(plan, 0) stops.  Inside captured GMRES cycles level 1 times only
 * the block product; bttb_profile(plan, 2) times every kernel that has a kind
 * (the extra event nodes serialise the graph, so level 2 is for breakdowns).  bttb_profile_read synchronises the stream and
 * fills *out for `which`:
 *   BTTB_K_BLOCK_PRODUCT, BTTB_K_FFT: summed event time (ms), launches, and
 *     algorithmic bytes (the bytes the operation must move: spectrum planes
 *     read, vectors read and written; padding zeros excluded);
 *   BTTB_K_ALL: launches of every kernel of the library (ms, bytes = 0);
 *   BTTB_K_BLOCK_PRODUCT_PREC + prec: the block product of one bttb_mv_prec.
 */
enum { BTTB_K_BLOCK_PRODUCT = 0, BTTB_K_FFT = 1, BTTB_K_ALL = 2, BTTB_K_BLOCK_PRODUCT_PREC = 16 };
typedef struct {
    double ms;
    long launches;
    double bytes;
} bttb_kernel_stats;
int bttb_profile(bttb_plan plan, int enable);
int bttb_profile_read(bttb_plan plan, int which, bttb_kernel_stats *out);

/*
 * FP64 (double-float) product y = Z x for callers that cannot allocate
 * device memory -- for example a plug-in whose host application reserves all
 * GPU memory at load time, or code running while a CUDA graph is captured.
 * Such callers cannot create a plan (a plan allocates its spectrum and
 * workspace).  The paper has no counterpart of this entry point.
 *
 * The caller passes the generator blocks (device, complex128, the layout of
 * bttb_set_generators), x and y (device, complex128, column stride ld >= N)
 * and a stream.  The spectrum of the generators, its FFT work buffers, the
 * twiddle tables and the product workspace are computed on every call inside
 * one fixed file-scope __device__ array of 64 MiB, which every GPU that loads
 * the library holds until the process exits.  No cudaMalloc, cudaFree or
 * allocating library routine is called.
 *   - Sizes whose scratch exceeds 64 MiB are rejected with
 *     BTTB_ERR_INVALID_ARG and a message giving the bytes needed (roughly:
 *     2*(mx*my*b*b*16) + 2*(mx*my*nrhs*b*16) bytes; the 4x4, b=12 array fits,
 *     the 30x30, b=60 array does not).
 *   - All calls on a device share the array and it keeps the last call's
 *     contents; each call rewrites every buffer before reading it.  Calls
 *     that overlap on the GPU (different streams or host threads) race on the
 *     array: serialise them.
 *   - The call returns BTTB_OK once its work is queued and never reads
 *     anything back, so it reports no device-side finding: non-finite
 *     generators give a non-finite y (bttb_set_generators would reject
 *     them), and a bounded pipeline wait that runs out leaves y unfinished.
 *     Check y where that matters.
 *   - The first call on a device looks up the array's address
 *     (cudaGetSymbolAddress, once per device, with that device current):
 *     make that first call before any stream capture begins.
 * Stream-ordered; does not synchronise.
 */
int bttb_matvec_noalloc(int nx, int ny, int b, const void *gen, const void *x, void *y, int nrhs, long ld,
                        void *cuda_stream);

/*
 * Batches of independent arrays of uneven sizes.  Array i has nx[i] x ny[i]
 * cells, b[i] bases per cell and up to nrhs[i] right-hand sides; it gets its
 * own plan (created with prec_mask) on its own CUDA stream owned by the batch;
 * the streams are blocking streams, ordered after work on the legacy default
 * stream, and a batch solve first waits for all work queued on the device.
 * A batch solve runs every array's GMRES concurrently: one host thread per
 * array drives that array's captured restart cycles on its stream, so the GPU
 * overlaps the arrays' kernels.  The paper solves one array at a time; the
 * batch is this library's extension for many arrays.
 */
typedef struct bttb_batch_s *bttb_batch;
int bttb_batch_create(bttb_batch *out, int count, const int *nx, const int *ny, const int *b, const int *nrhs,
                      unsigned prec_mask);
/* The plan of array `index` (owned by the batch; do not destroy it). */
int bttb_batch_plan(bttb_batch batch, int index, bttb_plan *out);
/* bttb_set_generators for array `index`. */
int bttb_batch_set_generators(bttb_batch batch, int index, const void *gen, bttb_dtype dtype, int gen_is_host);
/*
 * Autotuner: for every distinct FFT grid and block size (mx, my, b) in the
 * batch, tune one array of that shape as bttb_plan_autotune does for one
 * column (the form of the product and the FFT batch-chunk width, forms that
 * do not apply to plans in a batch left out) and give every array of that
 * shape the result.  chosen_out (host, count entries, may be NULL) receives
 * the width per array.  Needs the generators of the arrays to tune.
 */
int bttb_batch_autotune(bttb_batch batch, int reps, int *chosen_out);
/*
 * Solve every array: V[i], I[i] are device complex128 multi-vectors of array i
 * with nrhs[i] columns and column stride ld[i] (opts->host_io makes them host
 * pointers).  out_host receives sum(nrhs) results, array by array.  Returns the
 * worst status over the arrays; bttb_last_error names the first failing array.
 */
int bttb_batch_gmres_solve(bttb_batch batch, const void *const *V, void *const *I, const long *ld,
                           const bttb_gmres_opts *opts, bttb_col_result *out_host);
int bttb_batch_destroy(bttb_batch batch);

/*
 * Learned Fourier-domain correction to the block-Jacobi preconditioner P_K of
 * Sec. III-B.  The paper stops at P_K and the row preconditioner P_Z and notes
 * (Sec. V) that coupling more neighbouring elements may help; this object adds
 * a trained correction that sees the whole array through the 2-level DFT of
 * App. B.  For a column r:
 *   r^   = FFT2(pad r)/s, s = sqrt(mx*my)          (Eq. (xc2), App. B)
 *   h_k  = B_k r^_k                 per bin k, B_k complex rank x b
 *   g    = h + conv3(relu(conv2(relu(conv1(h)))))  3x3 circular convolutions over
 *          the (ky, kx) grid; h read as 2*rank real channels (2r = Re, 2r+1 = Im);
 *          conv1: 2*rank -> channels, conv2: channels -> channels,
 *          conv3: channels -> 2*rank, each with a bias
 *   z^_k = A_k g_k                  per bin k, A_k complex b x rank
 *   f(r) = crop(IFFT2_unnormalised(z^))/s
 *   M(r) = P_K^{-1} r + f(r)
 * Parameters are one binary32 vector (bttb_learned_param_count entries) in the
 * order B [bin][r][p] (re, im), A [bin][p][r] (re, im), W1 [co][ci][3][3], c1,
 * W2, c2, W3, c3; bin = ky*mx + kx.  Every kernel reads a bfloat16 copy of
 * them and accumulates in binary32.  Training minimises
 *   L = (1/n) sum_c ||M(r_c) - e_c||^2 / ||e_c||^2
 * over pairs (r_c, e_c) with Z e_c = r_c, by Adam on the binary32 master copy.
 * The object belongs to one plan (which needs the FP32 spectrum and a regular
 * T[0,0]); destroy it before the plan.
 *   rank in {8, 16, 32}; channels in {16, 32, 64}; 1 <= max_cols <= 256
 *   (largest ncols of any later call, and largest nrhs of a BTTB_PC_LEARNED
 *   solve).  Weights are initialised from `seed` (small A, B: f starts near 0).
 */
typedef struct bttb_learned_s *bttb_learned;
int bttb_learned_create(bttb_learned *out, bttb_plan plan, int rank, int channels, int max_cols,
                        unsigned long long seed);
/* Number of binary32 parameters. */
long bttb_learned_param_count(bttb_learned l);
/* Copy the binary32 parameters to (to_host != 0) or from a HOST array;
 * synchronises the plan's stream.  Loading refreshes the bfloat16 copy. */
int bttb_learned_params(bttb_learned l, float *host, int to_host);
/* z[:, c] = M(r[:, c]) for c < ncols: device multi-vectors of type dtype,
 * column stride ld >= N.  Stream-ordered, no synchronisation. */
int bttb_learned_apply(bttb_learned l, const void *r, void *z, int ncols, long ld, bttb_dtype dtype);
/* Loss and gradient for pairs (r, e): device complex64 multi-vectors with
 * column stride ld.  grad_host (HOST, param_count floats, may be NULL)
 * receives dL/dtheta (complex parameters: dL/dRe, dL/dIm); loss_host (may be
 * NULL) the loss.  Either output synchronises the plan's stream. */
int bttb_learned_gradients(bttb_learned l, const void *r, const void *e, int ncols, long ld, float *grad_host,
                           double *loss_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * minibatch (r, e), laid out as for bttb_learned_gradients. */
int bttb_learned_train_step(bttb_learned l, const void *r, const void *e, int ncols, long ld, float lr,
                            double *loss_host);
/* Attach (or, with l == NULL, detach) the object used by BTTB_PC_LEARNED. */
int bttb_plan_set_learned(bttb_plan plan, bttb_learned l);
int bttb_learned_destroy(bttb_learned l);

/*
 * Autotuner for one plan: times `reps` binary32 products of `nrhs` columns in
 * every form that applies (forms 1 to 4 of BTTB_DEBUG_PRODUCT_ROUTE, which
 * give the same bits; with forms 1 and 3, whose level-1 passes are strided,
 * each FFT batch-chunk width in {2, 4, 8, 16, 32, 64}) on the plan's stream
 * and keeps the fastest
 * form and width for every later call of the plan; then, if the plan keeps
 * the double-float spectrum, the fastest of those forms of the double-float
 * product.  They change the launch shapes only, not the result.
 * chosen_out (host, may be NULL)
 * receives the width.  Needs the generators; frees the plan's GMRES
 * workspace (it is rebuilt on the next solve).
 */
int bttb_plan_autotune(bttb_plan plan, int nrhs, int reps, int *chosen_out);

/*
 * Test hooks for the failure paths; the paper has no counterpart.  Nothing
 * here faults or hangs the GPU: every device pipeline wait is bounded, and the
 * injected fault is an mbarrier arrival that a kernel withholds, which the
 * same kernel supplies once its wait has run out, before it drains its copies
 * in flight and returns.
 *   BTTB_DEBUG_WAIT_LIMIT_NS (value in ns, 0 = the default of 2 s, at most
 *     60 s): bound of every pipeline wait in this plan's kernels.  Frees the
 *     plan's GMRES workspace (its captured cycles hold the old bound).
 *   BTTB_DEBUG_PRODUCT_ROUTE (value 0..4): the form of products of one to
 *     four columns, for comparisons; every form gives the product to the
 *     precision's tolerance.  0: automatic (the default); 1: four strided FFT
 *     passes around the block product; 2: the two-level FFT in one cluster
 *     kernel each way around the block product; 3: the level-1 passes around
 *     one cluster kernel that runs the level-2 transforms and the block
 *     product (b <= 128; b <= 64 for two to four columns); 4: all five steps
 *     as phases of one persistent kernel (one CTA per SM, cooperative launch,
 *     bounded grid barriers).  All four give the same bits.  Forms 3 and 4
 *     are double-float and binary32 only.  A form that does
 *     not fit the plan falls back to the automatic choice.  Frees the GMRES
 *     workspace.
 *   BTTB_DEBUG_ROUTE_TAKEN (value = (prec << 8) | nrhs): returns the form
 *     (1..4 as above) that a product of nrhs columns in precision prec takes
 *     on this plan; products of more than four columns take the strided
 *     passes (1).  Changes nothing.
 *   BTTB_DEBUG_FUSED_SHAPE (value = (Q << 16) | (prec << 8) | nrhs, prec
 *     FP64 or FP32, nrhs 1..4): with Q = 0 returns the cluster size (bits
 *     0-7) and ring depth (bits 8-15) of form 3 for that product, 0 if form 3
 *     does not fit; with Q in 1..8 returns how many clusters of that size the
 *     occupancy API lets run at once.  Changes nothing.
 *   BTTB_DEBUG_FUSED_CLUSTER (value 0..8): cluster size of form 3 (0: the
 *     largest size whose clusters are all resident at once, the default);
 *     with a size that does not fit, form 3 does not apply.  Frees the GMRES
 *     workspace.
 *   BTTB_DEBUG_WITHHOLD_ARRIVAL (value = a count, at most 1000): the next
 *     `value` launches of the block product for one to eight columns outside
 *     CUDA graph capture withhold the first arrival of one warp, so that
 *     warp's first wait runs out after the wait limit; the launch then sets
 *     the plan's device error word to TIMEOUT (reported by the next
 *     synchronising call that reads it, e.g. bttb_gmres_solve, as
 *     BTTB_ERR_TIMEOUT) and leaves the product unfinished.
 * Returns BTTB_OK (or the route for BTTB_DEBUG_ROUTE_TAKEN), and
 * BTTB_ERR_INVALID_ARG for an unknown hook or a value out of range.
 */
enum { BTTB_DEBUG_WAIT_LIMIT_NS = 1, BTTB_DEBUG_WITHHOLD_ARRIVAL = 2, BTTB_DEBUG_PRODUCT_ROUTE = 3,
       BTTB_DEBUG_ROUTE_TAKEN = 4, BTTB_DEBUG_FUSED_SHAPE = 5, BTTB_DEBUG_FUSED_CLUSTER = 6 };
int bttb_plan_debug(bttb_plan plan, int what, long long value);

/*
 * Bounds-checked build (libbttb_checked.so, compiled with -DBTTB_CHECKED=1;
 * the paper has no counterpart).  Its kernels check the global accesses of
 * the vector loads and stores, the bulk and asynchronous copies, the Arnoldi,
 * Givens and GEMM-epilogue accesses against the device buffers the library
 * allocated or was handed in its calls, the FFT stages' shared-memory
 * accesses against the CTA's shared memory, and the exchanges between the
 * CTAs of a cluster against their buffers' lengths; a failed check is
 * counted, its address recorded, and the access skipped (no fault).
 * bttb_check_report: returns 1 in the checked build with *hits (HOST, may be
 * NULL) the number of failed checks since load and *first_addr (HOST, may be
 * NULL) the first bad address (a shared-memory offset carries 0x5 in the top
 * four bits, an out-of-range index 0x6); returns 0 in the normal build (both
 * 0).  Synchronises the device.
 * bttb_check_probe: checked build only; reads one element past the end of a
 * buffer of its own through a checked load (the check skips it) and returns
 * BTTB_OK with *hits_added (HOST) the failed checks that read counted (1);
 * BTTB_ERR_INVALID_ARG in the normal build, where it launches nothing.
 */
int bttb_check_report(unsigned long long *hits, unsigned long long *first_addr);
int bttb_check_probe(unsigned long long *hits_added);

/* Bytes of device memory the plan holds (spectrum copies and workspace). */
size_t bttb_plan_workspace_bytes(bttb_plan plan);

/* Release everything the plan owns.  NULL is accepted. */
int bttb_plan_destroy(bttb_plan plan);

/* Message of the last error on this plan (plan may be NULL for errors of
 * bttb_plan_create).  Thread-local; never NULL. */
const char *bttb_last_error(bttb_plan plan);

#ifdef __cplusplus
}
#endif
#endif /* BTTB_H */
