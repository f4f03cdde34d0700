/*
 * bfgc.h - C ABI of the GB300 Gauss-Chebyshev bilateral filter library (libbfgc.so).
 *
 * Method: S. Ghosh and K. N. Chaudhury, "Fast and High-Quality Bilateral Filtering
 * Using Gauss-Chebyshev Approximation" (2016).  The Gaussian bilateral filter of
 * eq. (1) is approximated by replacing the range kernel with a Gaussian times a
 * degree-N polynomial whose coefficients come from a Chebyshev interpolation of
 * exp on [-mu, mu] (eqs. (16)-(19), Sec. III).  The filter then becomes
 *   1. per-pixel auxiliary images F_n, n = 0..N+1 (eq. (6), after centring eq. (17)),
 *   2. a bank of N+2 spatial Gaussian filterings (eq. (7)),
 *   3. a per-pixel ratio P/Q (eqs. (8)-(10)) and un-centring.
 *
 * Conventions for every entry point:
 *  - Images are single-channel float32, row-major, H rows by W columns, contiguous
 *    (element (y, x) at y*W + x).  Device pointers must be 16-byte aligned.
 *  - Pointers prefixed d_ are device memory, h_ host memory.  The caller owns every
 *    buffer (inputs, outputs, workspace); the library allocates no device buffers of its
 *    own, except the fixed module-scope scratch of bf_gc_forward_static and what the CUDA
 *    runtime keeps for the streams, events and graphs of the batch and streaming calls.
 *  - Device work is enqueued asynchronously on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream).  Argument errors are returned synchronously and
 *    nothing is enqueued.  Launch failures return BF_ERR_CUDA; faults during
 *    execution surface at the caller's next synchronisation.
 *  - Boundary: the image is extended by half-sample symmetry per axis
 *    (... f1 f0 | f0 f1 ... ), the paper's "extend the image outside I using
 *    symmetry" (Sec. I).  Window half-width R = ceil(3 sigma_s) (W = 3 sigma_s, Sec. I).
 *  - Intensity range [L, U] defaults to [0, 255] (Sec. II); values outside it are
 *    accepted (the polynomial is then extrapolated).
 */
#ifndef BFGC_H
#define BFGC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bf_gc_plan_s *bf_gc_plan_t;   /* opaque, host-owned */
typedef struct CUstream_st *bf_stream_t;     /* identical to cudaStream_t */

typedef enum {
    BF_OK = 0,
    BF_ERR_INVALID_ARG = 1,   /* bad size, sigma, pointer, alignment, option or state */
    BF_ERR_UNSUPPORTED = 2,   /* valid request the library does not implement (e.g. R too large for a form) */
    BF_ERR_NOMEM = 3,         /* host allocation failed */
    BF_ERR_CUDA = 4,          /* a CUDA runtime call or kernel launch failed */
    BF_ERR_TIMEOUT = 5,       /* a bounded device wait gave up (reported by bf_gc_diagnostics) */
    BF_ERR_RANGE = 6,         /* reserved: strict range checking */
    BF_ERR_WORKSPACE = 7      /* workspace pointer NULL, misaligned or smaller than required */
} bf_status;

/* ---- plan options (bf_gc_plan_set) --------------------------------------------------- */
enum {
    BF_OPT_FORM = 1,          /* value: BF_FORM_*                                  (default PLAIN) */
    BF_OPT_PRECISION = 2,     /* value: BF_PREC_*, storage of the filtered channels (default FP32) */
    BF_OPT_RANGE_L = 3,       /* value: L of the intensity range                   (default 0)     */
    BF_OPT_RANGE_U = 4,       /* value: U of the intensity range                   (default 255)   */
    BF_OPT_POLY = 5,          /* value: BF_POLY_*, choice of c_n                   (default CHEB)  */
    BF_OPT_SAVE_CHANNELS = 6, /* value: 1 = forward leaves the filtered channels in the workspace
                                 for bf_gc_backward to reuse; 0 = backward recomputes them.
                                 Plain form only: the other forms never hold the filtered
                                 channels as FP32 planes, and their backward recomputes them. */
    BF_OPT_TILE_W = 7,        /* value: row-pass kernel of the tensor-core form.  0 (default):
                                 Toeplitz operand in tensor memory, tiles of 128 output columns.
                                 64, 128 or 256: Toeplitz operand in shared memory, tiles of that
                                 many output columns (128 and 256 need ceil(R/16) <= 4, else
                                 BF_ERR_UNSUPPORTED).  The three widths give identical results;
                                 the default kernel sums the same products in another order. */
    BF_OPT_REFINE = 8,        /* value: 1 (default) = the exact forms recompute in FP64 the
                                 pixels their own arithmetic cannot resolve and take the
                                 division of eq. (10) there in FP64 (see bf_gc_diag); 0 = they
                                 decide on their own sums like the recursive form (guarded
                                 below 2^-17 Qa), with no second launch and no list in the
                                 workspace.  Where the fit converges nothing is refined; where
                                 it does not, up to a fifth of the pixels may be (BF16), each
                                 costing a (2R+1)^2 window in FP64. */
    BF_OPT_WAIT_US = 9,       /* value: bound, in microseconds, of one wait of a pipelined
                                 tensor-core kernel on another role (1 .. 1e7; default 1e6).  A
                                 wait that runs out sets a bit of bf_gc_diag.error_flags (then
                                 BF_ERR_TIMEOUT from bf_gc_diagnostics) and every role of the
                                 kernel returns; the output of that call is incomplete. */
    BF_OPT_STALL = 10         /* value: 0 (default).  For testing the bounded waits only: 1 = the
                                 tensor-core row pass never hands its first tile to the MMA
                                 issuer, 2 = the tensor-core column pass never loads its first
                                 stage, so that a wait runs out (BF_ERR_TIMEOUT) without any
                                 asynchronous copy or MMA left outstanding. */
};
enum {
    BF_FORM_PLAIN = 0,        /* 4 kernels: build F_n -> row filter -> column filter -> ratio; FP32 */
    BF_FORM_FUSED_TC = 1,     /* 2 kernels: (build + row filter) and (column filter + ratio), the
                                 spatial Gaussian as a banded Toeplitz product on tensor cores;
                                 channels stored as BF16 or FP16, FP32 accumulation */
    BF_FORM_RECURSIVE = 2,    /* recursive (IIR) stand-in for eq. (7), Young-van Vliet 1995 */
    BF_FORM_AUTO = 3,         /* chosen from R and the precision, and re-chosen when the precision
                                 changes (bf_gc_plan_info reports the choice): with BF16 / FP16
                                 storage the tensor-core form while R <= 128 (its limit), else the
                                 recursive form; with FP32 the fused form (BF_FORM_FUSED) while
                                 R <= BF_AUTO_FP32_EXACT_MAX_R, else the recursive form (whose cost does not grow with sigma_s;
                                 it approximates the Gaussian of eq. (7), 57-65 dB PSNR against the
                                 exact filter on 4K test images, instead of computing it exactly,
                                 so AUTO takes it only where the exact forms cost at least twice
                                 as much or do not exist) */
    BF_FORM_FUSED = 4         /* 2 kernels on the FP32 ALUs: (build + row filter) and (column filter
                                 + ratio); FP32 channel planes between them (C planes instead of the
                                 plain form's 2 C), the same results as PLAIN bit for bit.  Needs
                                 FP32 and R <= 173 (its shared-memory windows), else
                                 BF_ERR_UNSUPPORTED from bf_gc_workspace_size and
                                 bf_gc_forward. */
};
/* Largest window radius for which BF_FORM_AUTO keeps an exact form at FP32 (the fused form,
 * BF_FORM_FUSED).  AUTO keeps an exact form of eq. (7) while it costs at most twice the
 * recursive form, which is faster at large R but a different, less accurate filter (57-65 dB
 * against the exact one): on a GB300 at 4K, N = 20, the fused form costs 0.86 ms at R = 15,
 * 1.29 ms at R = 30, 3.34 ms at R = 87 and 4.99 ms at R = 141, the recursive form 2.3 - 2.6 ms
 * whatever R; twice the recursive cost is reached at R = 141 (sigma_s = 47). */
#define BF_AUTO_FP32_EXACT_MAX_R 140
/* Storage of the filtered channels (BF_OPT_PRECISION).  BF16 keeps 8 significant bits and
 * exceeds the 0.5 max-abs tolerance against the FP64 oracle at the paper's operating point
 * sigma_r = 30, N = 28 (0.67 measured on a test image; the high-degree terms of P and Q cancel
 * there); FP16 (11 bits, channels stored times 2^14) stays within it (0.27).  Prefer FP16 for
 * sigma_r <= 30 with N >= 20; BF16 is within 0.02 at sigma_r >= 40. */
enum { BF_PREC_FP32 = 0, BF_PREC_BF16 = 1, BF_PREC_FP16 = 2 };
enum {
    BF_POLY_CHEBYSHEV = 0,    /* c_n of eq. (19): Gauss-Chebyshev filter (GCF)          */
    BF_POLY_TAYLOR = 1        /* c_n = 1/n!: the Gauss-polynomial filter (GPF) of Sec. II */
};

#define BF_MAX_N 62           /* largest supported degree N (N + 2 <= 64 channels) */

/* Plan information (bf_gc_plan_info). */
typedef struct {
    int H, W, N, R, C;        /* C = N + 2 channels */
    int form, precision, poly;
    double sigma_s, sigma_r, L, U;
    double t_c;               /* (L + U) / 2, eq. (17) */
    double s_r;               /* (U - L) / 2: the centred image lies in [-s_r, s_r] */
    double mu;                /* (U - L)^2 / (4 sigma_r^2), Sec. III-B */
    double kappa;             /* max_n |c~_n|; the device uses c~_n / kappa */
    double fit_err;           /* max |g_r(t - tau) - approximate kernel| over a 129x129 grid of
                                 (t, tau) in [L, U]^2, evaluated in FP64 */
    double c[BF_MAX_N + 1];       /* c_n of eq. (19) (or 1/n!), n = 0..N */
    double c_tilde[BF_MAX_N + 1]; /* c~_n = mu^n c_n (the coefficients in u = (f - t_c)/s_r) */
} bf_gc_info;

/* Device-side diagnostics written by the last forward into its workspace.
 *
 * Division of eq. (10).  The paper assumes Q > 0; where the range-kernel fit has not
 * converged Q can vanish or change sign.  Reading taken here (the FP64 oracle takes the same):
 * with Qa = sum_n |c~_n u^n Fbar_n| (the sum of the absolute terms of Q), the output is the
 * input pixel when |Q| < 1e-12 Qa or Qa = 0 ("guarded"), else P/Q + t_c.  FP32 cannot
 * resolve Q at 1e-12 Qa, so the exact forms (PLAIN, FUSED, FUSED_TC) take that decision in
 * FP64: a pixel whose sums in the form's own arithmetic give |Q| < r Qa (r = 1e-3 with FP32
 * channels, 1/16 with BF16, 1/128 with FP16: above the storage's error in Q), a |Q| within
 * the underflow error of the stored channels, or non-finite values is recomputed from the
 * input image (eq. (7) as a window sum, the channels, P, Q and Qa): in FP64, where the guard
 * and the division are then taken ("refined"); with 16-bit channels first in FP32, which
 * settles the pixel when |Q| >= 1e-2 Qa there (the storage, not FP32, had been the limit).  Where the fit converges
 * no pixel comes near these thresholds and the refinement costs one empty launch.  The
 * RECURSIVE form (its spatial filter is an IIR, which a per-pixel window cannot reproduce)
 * decides on its FP32 sums: guarded when |Q| < 2^-17 Qa, the resolution of those sums. */
typedef struct {
    unsigned long long n_guarded;   /* pixels whose output is the input pixel (rule above) */
    unsigned long long n_illcond;   /* pixels divided with |Q| < 1e-3 Qa (in FP64 for the refined
                                       pixels of the exact forms); a conditioning diagnostic */
    unsigned int error_flags;       /* nonzero: a bounded wait in a pipelined kernel gave up and
                                       the output is incomplete.  Bit 0: column pass (one channel
                                       per step), bit 1: row pass with the Toeplitz operand in
                                       shared memory, bit 2: row pass with it in tensor memory,
                                       bit 3: column pass (channel pairs) */
    unsigned long long n_refined;   /* pixels recomputed from the input (exact forms; 0 for RECURSIVE) */
    unsigned long long n_refined_fp64; /* of those, the pixels recomputed and decided in FP64 (the
                                       rest, in the BF16 / FP16 forms, were resolved by an FP32
                                       recomputation: |Q| >= 1e-2 Qa there) */
} bf_gc_diag;

/* Create a plan for H x W images (Sec. III-B): fits, in FP64 on the host, the
 * Chebyshev interpolant of exp at the N+1 zeros of T_{N+1} on [-mu, mu] (eqs. (16),
 * (18)), converts it to monomials (eq. (19)) and derives the spatial taps.
 * H, W >= 1; sigma_s > 0; sigma_r > 0; 1 <= N <= BF_MAX_N.  Host only; no CUDA call.
 * *out receives the plan, or NULL on error. */
bf_status bf_gc_plan(int H, int W, double sigma_s, double sigma_r, int N, bf_gc_plan_t *out);

/* Change an option (BF_OPT_*) before first use; refits when L, U or the polynomial
 * change.  Returns BF_ERR_INVALID_ARG for an unknown option or value, or after the
 * plan has run a forward or backward. */
bf_status bf_gc_plan_set(bf_gc_plan_t plan, int option, double value);

/* Copy the plan's parameters and coefficients.  Host only. */
bf_status bf_gc_plan_info(bf_gc_plan_t plan, bf_gc_info *out);

/* Bytes of device workspace needed by bf_gc_forward and by bf_gc_backward for the
 * plan's current options.  Either pointer may be NULL.  Host only. */
bf_status bf_gc_workspace_size(bf_gc_plan_t plan, size_t *fwd_bytes, size_t *bwd_bytes);

/* Forward filter, eqs. (6)-(10) with centring (17): d_out = B_hat[d_f] (H x W).
 * d_ws: device workspace of at least the forward size, 256-byte aligned; its
 * contents on entry are ignored.  d_f and d_out must not overlap.  The division of
 * eq. (10) follows the rule given with bf_gc_diag (FP64 refinement of the pixels the form's
 * own arithmetic cannot resolve, in the exact forms; a second kernel launch).  The exact
 * forms need H * W < 2^32 (32-bit pixel indices in the refinement list), else
 * BF_ERR_UNSUPPORTED. */
bf_status bf_gc_forward(bf_gc_plan_t plan, const float *d_f, float *d_out, void *d_ws,
                        size_t ws_bytes, bf_stream_t stream);

/* Same as bf_gc_forward with host input and output: copies h_f to the device
 * staging buffer d_f, runs the forward into d_out, copies d_out back to h_out and
 * waits for the stream.  h_f / h_out should be page-locked for asynchronous copies. */
bf_status bf_gc_forward_host(bf_gc_plan_t plan, const float *h_f, float *h_out, float *d_f,
                             float *d_out, void *d_ws, size_t ws_bytes, bf_stream_t stream);

/* Streaming forward of `count` images of the plan's size held in host memory: h_out[i] =
 * B_hat[h_f[i]] (HOST arrays of host pointers; page-locked buffers for the copies to overlap).
 * Consecutive images overlap: while image i is filtered, image i + 1 is uploaded and image
 * i - 1 downloaded (three internal streams ordered by events, two device slots).  d_scratch:
 * 256-byte aligned device memory of at least bf_gc_stream_bytes bytes (two input and two
 * output images and one forward workspace), owned by the caller.  Work queued on `stream`
 * before the call comes first; the call returns when every output is in host memory.
 * Per-image diagnostics are not kept. */
bf_status bf_gc_stream_bytes(bf_gc_plan_t plan, size_t *bytes);
bf_status bf_gc_forward_host_stream(bf_gc_plan_t plan, int count, const float *const *h_f, float *const *h_out,
                                    void *d_scratch, size_t scratch_bytes, bf_stream_t stream);

/* Adjoint of the forward (not in the paper): given d_gout = dL/dB_hat, writes
 * d_gf = dL/df (H x W) and, if d_gsigma_r is not NULL, *d_gsigma_r = dL/dsigma_r
 * (one double on the device).  The derivative is that of the approximation,
 * including the dependence of mu and of the Chebyshev coefficients on sigma_r.
 * d_ws: workspace of at least the backward size.  With BF_OPT_SAVE_CHANNELS = 1 (plain
 * form) the filtered channels are NOT recomputed but read from d_ws: the caller must pass
 * the workspace of the last forward of this plan on the same d_f (allocated at the backward
 * size, which covers the forward's); the library cannot check this, and any other buffer
 * gives wrong gradients.  Without the option (or for the other forms) they are recomputed. */
bf_status bf_gc_backward(bf_gc_plan_t plan, const float *d_f, const float *d_gout, float *d_gf,
                         double *d_gsigma_r, void *d_ws, size_t ws_bytes, bf_stream_t stream);

/* Forward filter that allocates nothing and takes no workspace (the paper has no
 * counterpart; this is a deployment aid).
 *
 * Some callers cannot allocate device memory at the time they filter: a plug-in
 * running inside a host application that owns the device allocator, or a real-time
 * pipeline that forbids cudaMalloc after start-up because it may synchronise the
 * device.  This entry point runs the same forward as bf_gc_forward but uses a fixed
 * scratch area of BF_STATIC_SCRATCH_BYTES bytes kept in the library's own device
 * memory (a file-scope __device__ array: every GPU that loads the library holds it
 * until the process exits).  The caller still passes d_f and d_out.
 *  - If the plan's forward workspace (bf_gc_workspace_size) exceeds
 *    BF_STATIC_SCRATCH_BYTES, returns BF_ERR_WORKSPACE and enqueues nothing.
 *  - The first call on a device looks up the array's device address with that device
 *    current (the current device is used, and `stream` must belong to it); make that
 *    first call before any stream capture.
 *  - All calls share the one scratch area, which keeps the last call's contents (the
 *    forward rewrites all of it that it reads).  Calls whose execution overlaps on the
 *    GPU (other streams, other plans) race on it and give wrong results: order them.
 *  - Calls no allocation routine; bf_gc_diagnostics cannot read this scratch. */
#define BF_STATIC_SCRATCH_BYTES (64u << 20)
bf_status bf_gc_forward_static(bf_gc_plan_t plan, const float *d_f, float *d_out,
                               bf_stream_t stream);

/* Read back the diagnostics of the last forward that used d_ws (synchronises stream). */
bf_status bf_gc_diagnostics(bf_gc_plan_t plan, const void *d_ws, bf_gc_diag *out,
                            bf_stream_t stream);

void bf_gc_plan_destroy(bf_gc_plan_t plan);

/* ---- batches of independent images (a deployment aid; the paper filters one image at a
 * time).  Each image has its own plan (size, sigma_s, sigma_r, N and options), so a batch
 * may mix sizes and parameters.  The images are split over `branches` concurrent graph
 * branches (longest processing time first, by an estimate of each plan's work), each
 * branch with its own workspace slice, and the whole batch runs as one CUDA graph: small
 * images leave most SMs idle, and the branches fill them with other images' tiles. */
typedef struct bf_gc_batch_s *bf_gc_batch_t;

/* Host only, no CUDA call.  `plans` (count entries, 1 <= count <= 65536) are borrowed: they
 * must outlive the batch and are not modified, except that the first forward marks them
 * used (bf_gc_plan_set then refuses changes).  1 <= branches <= 64.  Plans with profiling
 * enabled are refused (BF_ERR_INVALID_ARG). */
bf_status bf_gc_batch_create(int count, const bf_gc_plan_t *plans, int branches, bf_gc_batch_t *out);

/* Persistent mode of a batch of tensor-core plans: bf_gc_batch_forward then runs ONE launch
 * of a batched row pass and ONE launch of a batched column pass over a device work list of
 * (image, tile) items (both captured in a CUDA graph), instead of per-image launches.  Every
 * plan must have form BF_FORM_FUSED_TC with the same precision (BF16 or FP16), the default
 * row-pass tile (BF_OPT_TILE_W 0) and R <= 64; otherwise BF_ERR_UNSUPPORTED.  Each image is
 * filtered at the batch's largest window block count a = ceil(R / 16) with its own taps (zero
 * beyond its R), so its result equals its own forward up to the FP32 summation order of the
 * banded products; the division of eq. (10) takes the FP32 guard (no FP64 refinement).  The
 * counters of all images (n_guarded, n_illcond, error_flags) land in the workspace header:
 * bf_gc_diagnostics with any of the batch's plans reads them.  Allocates the device work
 * list (a few KB per image) and a pinned host copy of it; 1 <= count <= 65536. */
bf_status bf_gc_batch_create_persistent(int count, const bf_gc_plan_t *plans, bf_gc_batch_t *out);

/* Workspace bytes for bf_gc_batch_forward: the sum over branches of the largest forward
 * workspace among the branch's images (each rounded up to 256 bytes); in persistent mode a
 * 256-byte header and every image's channel buffer.  Host only. */
bf_status bf_gc_batch_workspace_size(bf_gc_batch_t batch, size_t *bytes);

/* The branch (0 .. branches-1) of image i in branch_of[i] (count entries, may be NULL) and
 * the number of CUDA graphs captured so far in *captures (may be NULL).  Host only. */
bf_status bf_gc_batch_info(bf_gc_batch_t batch, int *branch_of, int *captures);

/* Forward of every image: d_out[i] = B_hat[d_f[i]].  d_f and d_out are HOST arrays of
 * `count` device pointers (16-byte aligned, else BF_ERR_INVALID_ARG before any launch; no
 * input overlapping an output); d_ws is a
 * 256-byte aligned device workspace of at least bf_gc_batch_workspace_size bytes.  The
 * first call, and any call whose pointers differ from the previous one, captures the
 * launches into a CUDA graph (on internal streams, thread-local capture mode); every call
 * then launches that graph on `stream`, so a repeated call costs one graph launch on the
 * host.  Per-image diagnostics are not kept (each branch reuses one diagnostics header);
 * use bf_gc_forward and bf_gc_diagnostics on a plan to inspect one image.  Persistent mode:
 * a call with new pointers also rewrites the device work list (tensor maps and pointers of
 * every image) through a pinned host copy, after synchronising `stream` once so that the
 * copy is free; repeated calls launch the captured graph only. */
bf_status bf_gc_batch_forward(bf_gc_batch_t batch, const float *const *d_f, float *const *d_out,
                              void *d_ws, size_t ws_bytes, bf_stream_t stream);

void bf_gc_batch_destroy(bf_gc_batch_t batch);

/* Kernel timing (a tracing aid, off by default).  While enabled, each forward and
 * backward of the plan records a CUDA event before every kernel it launches and one
 * after the last, on the caller's stream; bf_gc_profile_read waits for those events
 * and returns, per kernel name, the summed duration and the number of launches since
 * the last enable.  Enabling (or disabling) resets the totals. */
typedef struct {
    char name[32];
    double total_ms;
    unsigned long long launches;
} bf_kernel_time;

bf_status bf_gc_profile_enable(bf_gc_plan_t plan, int enable);
bf_status bf_gc_profile_read(bf_gc_plan_t plan, bf_kernel_time *out, int max_entries,
                             int *n_entries);

/* The exact Gaussian bilateral filter of eq. (1) by brute force over the
 * (2R+1)^2 window, FP32, used to measure the approximation's accuracy.
 * No workspace. */
bf_status bf_direct(int H, int W, double sigma_s, double sigma_r, const float *d_f,
                    float *d_out, bf_stream_t stream);

/* Input check (a diagnostic; the filter itself does not call it): the range-kernel fit covers
 * intensities in [L, U] only (Sec. III-B, the approximation interval is the centred dynamic
 * range).  Counts, over the H x W device image d_f (row-major, float32, no alignment needed),
 * the finite pixels outside [L, U] into d_counts[0] and the non-finite ones into
 * d_counts[1]: d_counts is a caller-owned device array of two unsigned 64-bit integers,
 * zeroed and then written in stream order (read them after the stream has reached that
 * point).  Nothing traps.  BF_ERR_INVALID_ARG for H < 1, W < 1, a NULL pointer, L > U or a
 * non-finite bound; BF_ERR_CUDA if the launch fails. */
bf_status bf_check_range(int H, int W, double L, double U, const float *d_f, unsigned long long *d_counts,
                         bf_stream_t stream);

const char *bf_status_string(bf_status s);
const char *bf_version(void);

/* The CUDA error code behind the last BF_ERR_CUDA returned to this thread (0 if none), and in
 * *name (may be NULL) its name as a static string.  Host only. */
int bf_last_cuda_error(const char **name);

#ifdef __cplusplus
}
#endif
#endif /* BFGC_H */
