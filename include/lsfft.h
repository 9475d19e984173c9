/*
 * lsfft.h - C ABI of the GB300 (sm_103a) FFT Lippmann-Schwinger solver for
 * two-phase periodic conductors.
 *
 * Method: G. W. Milton, "Substitution of subspace collections with
 * nonorthogonal subspaces to accelerate Fast Fourier Transform methods applied
 * to conducting composites" (arXiv 2001.08289).
 *
 *   Problem (Eq. J12, J13): sigma(x) = 1 + (sigma_1 - 1) chi(x) on a periodic grid;
 *   find E curl-free with mean e and J = sigma E divergence-free; the effective
 *   conductivity satisfies <J> = sigma_* <E> (isotropic case).
 *   Green projection Gamma_1 (Eq. J11, J45) applied per frequency.
 *   Schemes: Moulinec-Suquet (Eq. J0-0, J1), Eyre-Milton (Eq. J2), and both
 *   applied in the substituted space H'' (Eq. J27-J44: J42a for MS, J43 for EM),
 *   parameterised by the singularity interval [-beta, -alpha] of sigma_*(sigma_1)
 *   through t(sigma_1) of Eq. J3.
 *
 * Conventions shared by every entry point
 *   - Every function returns an lsfft_status (0 = success) unless stated.
 *   - Grids are d = 2 or 3 dimensional with n[a] points along axis a, where
 *     n[0] is the fastest-varying (x) axis.  Each n[a] is a power of two in
 *     [16, 8192] (3-D: [16, 512]); in LSFFT_FP64, n[0] <= 4096.
 *     N = n[0] n[1] (n[2]).
 *   - Phase masks are uint8[N], x fastest (index x + n0*(y + n1*z)); a non-zero
 *     byte marks phase 1 (conductivity sigma_1), zero marks the matrix (1).
 *   - Fields are complex, component-planar: field[c][z][y][x], c = 0..d-1
 *     (x, y, z components), interleaved (re, im) pairs of float (LSFFT_FP32)
 *     or double (LSFFT_FP64).
 *   - Objects returned through `out` pointers are owned by the caller and
 *     released with the matching lsfft_free_result / lsfft_destroy_grid.
 *   - All GPU work of a grid is issued on the CUDA stream given at creation;
 *     for NULL the grid creates and owns a non-blocking stream (the iteration
 *     is captured in CUDA graphs, which the legacy default stream does not
 *     allow).  lsfft_solve returns after its work has completed.  A grid must
 *     not be used from two host threads at once.
 *   - Argument errors are detected on the host before any launch and return
 *     LSFFT_EINVAL without touching device state.  CUDA failures return
 *     LSFFT_ECUDA; lsfft_last_error() gives the CUDA message.
 */
#ifndef LSFFT_H
#define LSFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LSFFT_OK = 0,
    LSFFT_EINVAL = 1,     /* invalid argument (checked before any launch)          */
    LSFFT_ENOMEM = 2,     /* device or host allocation failed                      */
    LSFFT_ENOTCONV = 3,   /* max_iter reached; result and history still returned   */
    LSFFT_EDIVERGED = 4,  /* non-finite sigma_k or field norm grew by 1e12          */
    LSFFT_ECUDA = 5       /* CUDA runtime error                                    */
} lsfft_status;

typedef enum { LSFFT_MS = 0, LSFFT_EM = 1, LSFFT_MS_SUB = 2, LSFFT_EM_SUB = 3 } lsfft_scheme;
typedef enum { LSFFT_FP32 = 0, LSFFT_FP64 = 1 } lsfft_precision;
/* Green symbol.  TRIG: Gamma(k) = k k^T/|k|^2 (Eq. J11) and Gamma = 0 at k = 0 and
 * wherever a component sits at the Nyquist index -n/2.  FD: projection onto
 * forward-difference gradients, u_a = exp(2 pi i k_a/n_a) - 1,
 * Gamma(k) = u u^H/|u|^2 (the resistor-network picture of the section
 * "Substitution at the level of the Hilbert space"). */
typedef enum { LSFFT_GREEN_TRIG = 0, LSFFT_GREEN_FD = 1 } lsfft_green;

typedef struct { double re, im; } lsfft_c128;

typedef struct lsfft_grid lsfft_grid;

typedef struct {
    int scheme;            /* lsfft_scheme                                                  */
    int precision;         /* lsfft_precision: arithmetic of fields and FFTs; reductions and
                              the scalar recurrence are FP64 in both                        */
    int green;             /* lsfft_green                                                   */
    int max_iter;          /* maximum number of updates, >= 1                               */
    int stop_consecutive;  /* K >= 1: stop once, K times in a row, both the relative change
                              of sigma_* and that of <|E|^2> are below tol                 */
    int check_every;       /* updates per CUDA-graph launch between host checks, >= 1       */
    double tol;            /* relative sigma_* change threshold (0 = run max_iter updates)  */
    double alpha, beta;    /* pole interval [-beta,-alpha], 0 < alpha < beta; *_SUB only    */
} lsfft_opts;

typedef struct {
    lsfft_c128 sigma_star;     /* sigma_* of the returned field: <J>.e / <E>.e              */
    lsfft_c128 sigma1;         /* the inclusion conductivity of the solve                   */
    lsfft_c128 mean_E[3];      /* <E> of the returned field (d entries used)               */
    lsfft_c128 mean_J[3];      /* <J> of the returned field                                */
    int iters;                 /* number of updates applied                                 */
    int status;                /* LSFFT_OK, LSFFT_ENOTCONV or LSFFT_EDIVERGED               */
    int hist_len;              /* iters + 1 entries: iterate k = 0..iters                   */
    double *hist_sigma_re;     /* host arrays of hist_len entries, owned by the result      */
    double *hist_sigma_im;
    double *hist_rel_change;   /* |sigma_k - sigma_{k-1}|/|sigma_k|; entry 0 is +inf        */
    double *hist_field_norm;   /* <|E_k|^2>                                                 */
    double solve_ms;           /* device time of the iteration (CUDA events), ms            */
    int64_t kernel_launches;   /* kernels this solve launched (no-op launches included)     */
    int packed;                /* 1 if the packed real layout was used: 2-D with every scheme
                                  coefficient real (real sigma_1, real reference medium); the
                                  state then holds the x-spectra of the two real components
                                  as two half-spectrum planes (E_device is complex as always);
                                  2 if, in addition, the split layout of long columns ran
                                  (lsfft_set_column_split)                                    */
    int precision;             /* precision of E_device                                     */
    int d;
    int64_t n[3];
    void *E_device;            /* complex [d][N] in `precision`, owned by the result        */
} lsfft_result;

/* Library version string, and the message of the last CUDA error seen on this
 * host thread ("" if none). */
const char *lsfft_version(void);
const char *lsfft_last_error(void);
const char *lsfft_strerror(int status);

/* Create a grid: copies the host phase mask (N bytes, 1 = inclusion) to the
 * device; the caller keeps its buffer.  `cuda_stream` is a cudaStream_t (may be
 * NULL).  Problem statement of the introduction and Eq. J12: two phases, matrix
 * conductivity 1, d = 2 or 3. */
int lsfft_create_grid(int d, const int64_t n[3], const uint8_t *phase_mask_host,
                      void *cuda_stream, lsfft_grid **out);

/* Same, with the mask already on the device (N bytes, device pointer; copied on
 * the grid's stream, so the caller must have finished writing it). */
int lsfft_create_grid_device(int d, const int64_t n[3], const uint8_t *phase_mask_device,
                             void *cuda_stream, lsfft_grid **out);

/* Release every device buffer of the grid (after the stream has drained). */
void lsfft_destroy_grid(lsfft_grid *grid);

/* Fill `opts` with defaults: MS, FP32, TRIG, max_iter 1000, K = 3,
 * check_every 8, tol 1e-6, alpha = beta = 0. */
void lsfft_default_opts(lsfft_opts *opts);

/* Solve Eq. J12/J13 for inclusion conductivity sigma_1 (complex) and applied
 * field e (d real components, not all zero) with the chosen scheme.
 * Returns LSFFT_OK, LSFFT_ENOTCONV or LSFFT_EDIVERGED with *out filled (the
 * result exists in all three cases), or an error code with *out = NULL.
 * Validation (EINVAL): scheme/precision/green out of range; max_iter < 1;
 * stop_consecutive < 1; check_every < 1; tol < 0 or non-finite; non-finite
 * sigma_1; e all zero; *_SUB with !(0 < alpha < beta) or sigma_1 = -alpha, -beta;
 * MS with sigma_1 = -1 (reference medium 0); EM with sigma_1 = 0. */
int lsfft_solve(lsfft_grid *grid, lsfft_c128 sigma1, const double *e,
                const lsfft_opts *opts, lsfft_result **out);

/* Copy the result's field E (complex [d][N] in the result's precision,
 * d*N*(8 or 16) bytes) to `dst`: a host pointer if dst_on_device == 0, else a
 * device pointer.  Synchronises the grid's stream. */
int lsfft_copy_field(const lsfft_result *res, void *dst, int dst_on_device);

/* Stream-ordered form of lsfft_copy_field: enqueue the copy of E on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream) and return
 * without waiting, so that the copy of one solve's field overlaps the next
 * solve on the grid's stream.  E is complete when lsfft_solve returns, so no
 * ordering against the grid's stream is needed.  The caller keeps `res` and
 * `dst` alive until the copy has completed on that stream (synchronise it, or
 * an event recorded after this call); a pageable host `dst` makes the copy
 * synchronous, pinned host memory lets it run on a copy engine.  EINVAL for a
 * null result, destination or field; ECUDA if the copy cannot be enqueued. */
int lsfft_copy_field_async(const lsfft_result *res, void *dst, int dst_on_device, void *cuda_stream);

/* Free the result's host history and device field.  Grid workspaces and result
 * fields come from a per-device stream-ordered memory pool that keeps freed
 * blocks for the next grid or solve (no unmap and remap of gigabyte buffers);
 * the pool returns its memory to the driver once no grid and no result is
 * alive. */
void lsfft_free_result(lsfft_result *res);

/* Convergence and stability of EM in H'' (Eq. J4, J43, J46) for sigma_1 and
 * [alpha, beta]: rate = |z| with z = (sqrt t - 1)/(sqrt t + 1), t = t(sigma_1) of
 * Eq. J3; limit = min(|z(t(0))|, |z(t(inf))|).  chi Gamma_1 chi always has the
 * eigenvalues 1 and 0 (poles at sigma_1 = 0 and -inf) on modes that carry no
 * weight for sigma_* but are excited by rounding; in H'' they sit at t(0) and
 * t(inf), so when rate > limit the iteration amplifies rounding noise by
 * rate/limit per step and the field diverges although sigma_* converges.  For
 * real sigma_1 > 0, rate < limit always; complex sigma_1 close to the slit can
 * violate it, and plain EM is then the safe choice.  EINVAL unless
 * 0 < alpha < beta < inf. */
int lsfft_substitution_rates(lsfft_c128 sigma1, double alpha, double beta, double *rate, double *limit);

/* The full d x d effective conductivity tensor (Eq. J13 read as a tensor
 * relation <J> = sigma_* <E>, with the paper's remark that the anisotropic case
 * follows the same way): d solves with the applied fields e_a = unit vectors,
 * then sigma_* = [<J>_1 ... <J>_d] [<E>_1 ... <E>_d]^-1, formed on the host in
 * FP64 by Gaussian elimination with partial pivoting.  At the fixed point
 * <E>_a = e_a and the product is [<J>]; for the Eyre-Milton type schemes,
 * whose iterates reach <E> = e only in the limit, it is the matrix analogue of
 * the scalar estimate <J>.e / <E>.e.
 * out: d*d lsfft_c128, row-major (out[i*d + j] = sigma_ij), host memory.
 * results: NULL, or d slots that receive the d solves' results (caller frees
 * each with lsfft_free_result); with NULL the results are freed here.
 * Returns what the worst solve returned: OK, ENOTCONV or EDIVERGED (out is
 * still written from the last iterates), or an error (EINVAL, ENOMEM, ECUDA:
 * out untouched, no result kept).  EINVAL also when [<E>] is singular. */
int lsfft_effective_tensor(lsfft_grid *grid, lsfft_c128 sigma1, const lsfft_opts *opts, lsfft_c128 *out,
                           lsfft_result **results);

/* Strided-pass layout of long 2-D columns (the paper has no counterpart; a
 * tuning control).  It applies to 2-D grids with n_x, n_y in {4096, 8192} whose
 * solves run FP32 fields with real coefficients (the packed real layout).
 * split = 1: the row pass works on row pairs (j, j + n_y/2) and applies the
 * first radix-2 step of every y-DFT (decimation in frequency), so the strided
 * pass transforms independent columns of n_y/2 points on one SM each.
 * split = 0 (default, measured faster at 4096^2 and 8192^2 on GB300): the
 * strided pass transforms whole columns on two-block clusters that exchange
 * half-transforms through distributed shared memory.  Both give the same
 * iterates up to rounding; lsfft_autotune measures both.  Takes effect from the next solve or
 * lsfft_prepare; waits for the grid's pending work.  EINVAL for a null grid. */
int lsfft_set_column_split(lsfft_grid *grid, int split);

/* Tuning of a grid's solve (the paper has no counterpart).  Candidates: the
 * number of updates per CUDA-graph launch between host checks (check_every in
 * {4, 8, 16, 32, 64}) and, where both exist (lsfft_set_column_split), the split
 * or cluster strided pass.  Each candidate runs `iters` updates of the given
 * problem (tol 0, after one untimed run that captures its graph) and is timed
 * with CUDA events on the grid's stream; the fastest is applied to the grid
 * (column split) and returned.  opts: the solve's options (scheme, precision,
 * Green symbol, alpha, beta; its check_every, tol and max_iter are ignored). */
typedef struct {
    int check_every;       /* updates per graph launch of the fastest candidate        */
    int column_split;      /* 1 split layout, 0 cluster pass (or the only layout)      */
    double ms_per_iter;    /* its device time per update, ms                           */
    int candidates;        /* configurations timed                                     */
} lsfft_tuning;
int lsfft_autotune(lsfft_grid *grid, lsfft_c128 sigma1, const double *e, const lsfft_opts *opts, int iters,
                   lsfft_tuning *out);

/* One solve of a batch: grid, sigma_1, applied field (d entries used), options. */
typedef struct {
    lsfft_grid *grid;
    lsfft_c128 sigma1;
    double e[3];
    lsfft_opts opts;
} lsfft_job;

/* Run many solves: jobs that share a grid run in their order on that grid's
 * stream, jobs on different grids run concurrently (one solve in flight per
 * grid, driven by a host scheduler that polls CUDA events instead of
 * blocking), e.g. a sweep of sigma_1 over microstructures of different sizes.
 * results[j] / statuses[j] receive what lsfft_solve would return for job j
 * (a result for OK, ENOTCONV, EDIVERGED; NULL otherwise).  The call returns
 * LSFFT_OK once every job has finished, or EINVAL (with nothing run) for null
 * arrays or a job without grid.  Grids must not be used elsewhere meanwhile. */
int lsfft_solve_batch(int njobs, const lsfft_job *jobs, lsfft_result **results, int *statuses);

/* Run a batch of solves in one persistent kernel launch (the batched sweep over
 * sigma_1 and microstructures of uneven sizes; section "Estimating the
 * parameters alpha and beta" for the alpha, beta per microstructure, Eq. J3
 * for complex sigma_1).  Every job: a 2-D grid with n_x, n_y powers of two in
 * [128, 1024], a two-phase medium (no lsfft_set_sigma_field), FP32 fields, any
 * scheme and Green symbol.  A device work queue hands out items (a few rows of
 * a row pass, a few columns of a strided pass) of every solve to the resident
 * blocks; the block that completes a solve's pass takes the solve to its next
 * pass (row pass -> FP64 finalize and stop rule -> strided pass -> row pass,
 * and the output pass once the stop rule fired), so solves of all sizes and
 * iteration counts progress side by side with no host involvement.  The
 * batch (descriptors in, the launch, results out) is one captured CUDA graph.
 * results[j] / statuses[j] as for lsfft_solve (complex layout fields, FP32);
 * each result's solve_ms is the device time of the whole batch and its
 * kernel_launches is 1.  Returns EINVAL (nothing run) if a job does not
 * qualify, ECUDA if a block of the launch found no work for two seconds while
 * solves remained (no result is kept), else OK. */
int lsfft_solve_sweep(int njobs, const lsfft_job *jobs, lsfft_result **results, int *statuses);

/* Per-voxel conductivity sigma(x) (complex, N entries, host or device
 * pointer; copied).  Subsequent solves on the grid use sigma(x) instead of the
 * two-phase 1 + (sigma_1 - 1) chi(x) of the mask, with the MS or EM scheme only
 * (the substituted schemes of Eq. J36-J44 need two phases: EINVAL) and
 * reference medium sigma0 (0 = automatic: (min + max)/2 of Re sigma for MS,
 * sqrt(min max) for EM).  The mask is kept for lsfft_gradient's d/d sigma_1.
 * sigma = NULL returns to the two-phase medium.  EINVAL for non-finite
 * entries. */
int lsfft_set_sigma_field(lsfft_grid *grid, const lsfft_c128 *sigma, int on_device, lsfft_c128 sigma0);

/* Fault injection for tests (the paper has no counterpart).  kind 1: the
 * strided passes of later solves on this grid announce 16 more bytes to each
 * TMA completion barrier than the copy delivers, and every barrier wait gives
 * up after 2e7 clock cycles instead of about two seconds: each wait runs out,
 * the kernel records a fault and completes, and lsfft_solve returns
 * LSFFT_ECUDA ("a bounded wait ... gave up") with no result; the GPU context
 * stays usable.  kind 0 restores normal operation.  Waits for any pending work
 * of the grid first.  EINVAL for a null grid or another kind. */
int lsfft_debug_inject(lsfft_grid *grid, int kind);

/* Gradient of sigma_* for the field of `res` (a result of this grid): the first
 * variation of the energy <sigma E.E> = sigma_* |e|^2 of Eq. J12/J13 (E.E
 * bilinear, no conjugation, so complex conductivities are covered) gives
 *   d sigma_* / d sigma(x) = E(x).E(x) / (N |e|^2),
 *   d sigma_* / d sigma_1  = sum_x chi(x) E(x).E(x) / (N |e|^2).
 * grad_device (complex [N] in the result's precision) receives the first, or
 * may be NULL; dsigma1 and energy (may be NULL) receive the second and the
 * variational estimate <sigma E.E> / |e|^2 of sigma_*.  Both formulas hold at
 * the converged field.  Synchronises the grid's stream. */
int lsfft_gradient(lsfft_grid *grid, const lsfft_result *res, const double *e, void *grad_device,
                   lsfft_c128 *dsigma1, lsfft_c128 *energy);

/* Diagnostics and benchmarking: set up the state of a solve (constants of
 * Eq. J1/J2/J3/J24, the initial field and one full update, exactly as
 * lsfft_solve starts) and return without further iterations.  Same arguments
 * and validation as lsfft_solve.  Synchronises the grid's stream. */
int lsfft_prepare(lsfft_grid *grid, lsfft_c128 sigma1, const double *e, const lsfft_opts *opts);

/* After lsfft_prepare: enqueue `count` launches of one pass kind on the grid's
 * stream and return without waiting.  kind 0: row pass (inverse x-DFT, scheme
 * update with its volume-average partial sums, forward x-DFT); kind 1: the
 * strided pass(es) of one update (2-D: y forward-Gamma-inverse; 3-D: y
 * forward, z forward-Gamma-inverse, y inverse); kind 2: both, i.e. one update
 * without the one-block FP64 finalize.  The passes keep iterating the prepared
 * state in place; no stop test runs.  Returns EINVAL for an unknown kind,
 * count < 0, or a grid without a prepared state (or whose last solve stopped). */
int lsfft_launch_passes(lsfft_grid *grid, int kind, int count);

/* Benchmarking: the FP32 FMA throughput of the current device, the ceiling
 * against which the arithmetic of the FFT passes is reported.  Runs a kernel
 * of 8 independent FMA chains per thread (`paired` = 1: the paired
 * fma.rn.f32x2 form, two FMAs per instruction) on every SM, `reps` timed
 * launches after one warm-up, and writes the best rate in TFLOP/s (2 flops
 * per FMA) to *tflops.  Synchronises the device's legacy stream.  EINVAL for a
 * null pointer or reps < 1; ECUDA on a CUDA error. */
int lsfft_fma_peak(int paired, int reps, double *tflops);

/* Estimate of the pole interval [-beta, -alpha] (section "Estimating the
 * parameters alpha and beta").  The singularities of sigma_*(sigma_1) are the
 * poles 1 - 1/m_n with m_n the eigenvalues of chi Gamma_1 chi weighted by
 * |u_n^H chi e|^2; `steps` Lanczos steps from chi e on the GPU (matrix-vector
 * products through the same FFT passes as the solver, FP64 recurrence
 * scalars) give the Gauss nodes theta_i and weights w_i of that spectral
 * measure, and alpha = 1/theta_max - 1, beta = 1/theta_min - 1 over nodes with
 * w_i > cutoff * sum(w) and theta_i > 1e-14.  nodes, weights (host, >= steps
 * doubles each) and n_nodes may be NULL.  Uses the grid's stream and
 * synchronises it; allocates three field-sized vectors for the duration.
 * EINVAL for bad arguments (steps outside [2, 4096], cutoff outside [0, 1), e
 * zero), ENOTCONV if no node passes the cutoff. */
int lsfft_lanczos_hull(lsfft_grid *grid, const double *e, int green, int precision, int steps, double cutoff,
                       double *alpha, double *beta, double *nodes, double *weights, int *n_nodes);

/* Host helper: Gauss quadrature of a Jacobi matrix (diagonal a[m],
 * off-diagonal b[m-1]): its eigenvalues nodes[m] and the squared first
 * components of its normalised eigenvectors first2[m] (implicit QL iteration).
 * EINVAL for bad arguments, ENOTCONV if the iteration stalls. */
int lsfft_tridiag_gauss(int m, const double *a, const double *b, double *nodes, double *first2);

/* Volume averages of a field without any device allocation.  The paper has
 * no counterpart: this is a utility for callers that cannot call cudaMalloc,
 * e.g. code that must not block (cudaMalloc/cudaFree may synchronise the
 * device), code whose device memory is owned by another allocator under a
 * fixed budget, or code running where allocation is not allowed.
 * Inputs (device pointers, not copied): E_device, a complex field [d][N] in
 * `precision` (the layout of lsfft_result.E_device); mask_device, uint8[N]
 * (non-zero = phase 1, conductivity sigma1; zero = conductivity 1); e, d host
 * doubles.  Output: out_device, 4*d + 3 doubles on the device:
 *   out[4c+0], out[4c+1]  Re, Im <E_c>      out[4c+2], out[4c+3]  Re, Im <J_c>
 *   out[4d] <|E|^2>      out[4d+1], out[4d+2]  Re, Im sigma_* = <J>.e / <E>.e
 * with J = sigma E: what lsfft_solve reports for its field under LSFFT_MS, whose
 * flux is sigma E at every iterate (the other schemes report their own flux
 * estimate, which equals sigma E at convergence).
 * The work is enqueued on cuda_stream (NULL = legacy default stream) and the
 * call returns without waiting.  Block partial sums live in one file-scope
 * __device__ array of 4096 x 16 doubles (512 KiB, held by every device that
 * loads the library until the process exits), so N must not exceed
 * 4096 * 65536 = 268,435,456 voxels (EINVAL otherwise).  Every call on a device
 * shares that array and leaves its partial sums in it; calls whose kernels
 * overlap on the GPU race, so serialise them (one stream, or events).  Every
 * call looks up the array's device address on the current device with
 * cudaGetSymbolAddress (it allocates nothing; looking it up each time keeps the
 * address valid across a device reset); the first call on a device, which may
 * also load the module there, should come before any stream capture.
 * sigma_* (out[4d+1], out[4d+2]) is NaN when <E>.e = 0.  Errors: EINVAL (null
 * pointer, d not in {2, 3}, unknown precision, n[a] < 1, N over the limit,
 * e zero or not finite), ECUDA (lookup failure, or a CUDA error seen right
 * after a launch, which may also stem from earlier work on the thread: it is
 * left pending for the caller); lsfft_noalloc_last_error() gives the message. */
int lsfft_field_averages_noalloc(int d, const int64_t n[3], const void *E_device, int precision,
                                 const uint8_t *mask_device, lsfft_c128 sigma1, const double *e,
                                 double *out_device, void *cuda_stream);
const char *lsfft_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LSFFT_H */
