/*
 * parareal.h -- C ABI of the GB300 Parareal library for the periodic 3-D
 * advection-diffusion problem u_t + a.grad u = nu(t) Lap u (Sec. 3,
 * Eq. adv_diff_eq of Arteaga, Ruprecht & Krause, arXiv:1409.8563).
 *
 * Method (Sec. 2.2, Eq. parareal):
 *     U^{k+1}[n+1] = G(U^{k+1}[n]) + F(U^k[n]) - G(U^k[n]),  n = 0..N_p-1,
 * with F = classical RK4 with step dt_fine (Sec. 2.3) on the fine grid, and G
 * = RK4 with step dt_coarse on the grid coarsened by coarse_factor (box
 * restriction, trilinear prolongation; the spatial coarsening of Sec. 2.2.2),
 * a periodic integer shift, or a learned convolution net.  The spatial
 * operator is the 7-point Laplacian of Sec. 2.3 times nu(t) plus centred
 * first differences for advection.  All time slices of an iteration advance
 * concurrently on one GPU.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - Fields are n^3 arrays, x fastest: index (z*n + y)*n + x, point x_i = i/n.
 * - A pointer argument is a device pointer when the accompanying `mem`
 *   argument is PARAREAL_MEM_DEVICE and a host pointer when it is
 *   PARAREAL_MEM_HOST.  Buffers are copied with cudaMemcpyAsync on the
 *   context stream.
 * - Caller-supplied buffers are borrowed for the duration of the call only:
 *   every call that reads or writes one synchronises the context stream
 *   before it returns (except parareal_diff_norms_noalloc, which is fully
 *   asynchronous).  The context owns all of its device workspace and frees it
 *   in parareal_destroy.
 * - Device work is ordered on the context stream (the stream passed to
 *   parareal_create; NULL = the legacy default stream).  Calls that return
 *   host scalars synchronise that stream.
 * - Every call returns a parareal_status.  Failures never throw across the
 *   ABI; the message of the last failure is available from
 *   parareal_last_error.  After PARAREAL_E_CUDA the context must be
 *   destroyed; after any other error it stays usable.
 * - Not thread-safe: one context must not be used by two host threads at
 *   once.  Distinct contexts are independent.
 */
#ifndef PARAREAL_H
#define PARAREAL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct parareal_ctx parareal_ctx;

typedef enum {
    PARAREAL_OK = 0,
    PARAREAL_W_MARGINAL = 1,   /* created; the stability pre-check found growth > 1 per
                                  step, accepted because allow_unstable was set */
    PARAREAL_E_INVALID = -1,   /* bad argument or configuration */
    PARAREAL_E_UNSTABLE = -2,  /* stability pre-check failed (see parareal_stability) */
    PARAREAL_E_NOMEM = -3,     /* device allocation failed */
    PARAREAL_E_CUDA = -4,      /* CUDA runtime error; destroy the context */
    PARAREAL_E_DIVERGED = -5,  /* NaN or Inf detected in the iterate */
    PARAREAL_E_TIMEOUT = -6,   /* a bounded device-side wait gave up */
    PARAREAL_E_STATE = -7      /* call out of order (e.g. iterate before set_problem) */
} parareal_status;

enum { PARAREAL_F32 = 0, PARAREAL_F64 = 1 };
enum { PARAREAL_MEM_DEVICE = 0, PARAREAL_MEM_HOST = 1 };

/* Stage times of nu(t) inside an RK4 step starting at t:
 * STAGE  = classical non-autonomous RK4 (t, t+dt/2, t+dt/2, t+dt);
 * FROZEN = nu(t) for all four stages. */
enum { PARAREAL_NU_STAGE = 0, PARAREAL_NU_FROZEN = 1 };

/* Coarse propagator kinds. */
enum {
    PARAREAL_COARSE_STENCIL = 0,  /* RK4 on the (coarsened) grid, 7-point / centred operator */
    PARAREAL_COARSE_LEARNED = 1,  /* shift + convolution net (parareal_set_coarse_model) */
    PARAREAL_COARSE_SHIFT = 2,    /* periodic integer shift only (the net set to zero) */
    PARAREAL_COARSE_EULER_UPWIND = 3  /* the paper's coarse propagator (Sec. 3.1, Algorithm 2):
                                         forward Euler at dt_coarse, 7-point Laplacian, first-order
                                         upwind advection, nu at the step start, same grid
                                         (coarse_factor must be 1) */
};

/* Spatial operator of the fine propagator F (always classical RK4 in time):
 * C2 = 7-point Laplacian and centred first differences (Sec. 2.3);
 * C4 = fourth-order centred differences, (-1,16,-30,16,-1)/(12h^2) and
 *      (1,-8,0,8,-1)/(12h) per axis, the paper's fine operator (Sec. 3.1).
 *      C4 runs on the per-stage kernels (no fused path). */
enum { PARAREAL_SCHEME_C2 = 0, PARAREAL_SCHEME_C4 = 1 };

/* Stopping rules for parareal_iterate. */
enum {
    PARAREAL_STOP_DIFF = 0,    /* max_n ||U^{k+1}[n]-U^k[n]||_inf / ||U^{k+1}[n]||_inf <= tol */
    PARAREAL_STOP_DEFECT = 1,  /* d^k of Eq. (defect) against parareal_set_reference <= tol */
    PARAREAL_STOP_NONE = 2     /* run exactly k_max iterations */
};

/* Residual kinds for parareal_residual. */
enum {
    PARAREAL_RES_DIFF_INF = 0, /* per slice ||U^{k+1}[n]-U^k[n]||_inf / ||U^{k+1}[n]||_inf, last iteration */
    PARAREAL_RES_DIFF_L2 = 1,  /* same with the 2-norm */
    PARAREAL_RES_FINE = 2,     /* per slice ||F(U[n-1]) - U[n]||_inf / ||U[n]||_inf (runs one fine sweep) */
    PARAREAL_RES_DEFECT = 3,   /* ||U[N_p]-ref||_inf/||ref||_inf at index N_p; others 0 */
    PARAREAL_RES_FINE_L2 = 4   /* as PARAREAL_RES_FINE with the 2-norm */
};

typedef struct {
    int n;                 /* grid edge; n^3 points; multiple of 4, 8..1024 */
    int n_slices;          /* N_p >= 1 */
    double T;              /* final time; slices are [n T/N_p, (n+1) T/N_p] */
    double dt_fine;        /* delta t; T/(N_p dt_fine) must be an integer N_f */
    double dt_coarse;      /* Delta t; T/(N_p dt_coarse) must be an integer N_c */
    int coarse_factor;     /* r >= 1 dividing n, n/r >= 4: G runs on (n/r)^3 */
    double a[3];           /* advection velocity (x, y, z) */
    double nu0, nu_amp, nu_omega;  /* nu(t) = nu0 (1 + nu_amp sin(nu_omega t)) */
    int fine_dtype;        /* PARAREAL_F32 or PARAREAL_F64: arithmetic of F and G */
    int nu_mode;           /* PARAREAL_NU_STAGE or PARAREAL_NU_FROZEN */
    int coarse_kind;       /* PARAREAL_COARSE_* */
    int allow_unstable;    /* nonzero: stability pre-check failures become a warning */
    int learned_skip;      /* PARAREAL_SKIP_*: the skip path of the learned propagator */
    int fine_scheme;       /* PARAREAL_SCHEME_*: spatial operator of F */
    int learned_act;       /* PARAREAL_ACT_*: the learned propagator's layers */
    int correction_form;   /* PARAREAL_CORRECTION_*: how Eq. (parareal) is evaluated */
    int learned_eval;      /* PARAREAL_EVAL_*: how a LINEAR learned propagator is evaluated */
    int coarse_transfer;   /* PARAREAL_TRANSFER_*: restriction / prolongation of a coarse-grid G */
    int pipeline_blocks;   /* 0: off.  B > 0: pipelined iterations, see below */
} parareal_config;

/* Pipelined iterations (pipeline_blocks = B > 0; Sec. 2.2 notes that the
 * fine propagations of the next iteration can start as soon as the serial
 * coarse sweep has produced their initial values).  While an iteration's
 * serial coarse sweep and corrections run on the context's stream, the next
 * iteration's fine sweep F(U^{k+1}[n]) runs on a second stream of the
 * context, in B blocks of consecutive slices, each launched as soon as the
 * corrections have made its slices final; the next iteration's corrections
 * wait only for the block they read.  F's results go to a second buffer, so
 * the iterates are bit for bit those of pipeline_blocks = 0.  The fine sweep
 * started for an iteration that the stopping rule then makes unnecessary is
 * cancelled (its remaining launches exit at once); every call returns with
 * the context's stream ordered after all of the context's work.  Needs the
 * FP32 fused fine sweep (fine_dtype F32, fine_scheme C2) and N_p >= 2; costs
 * a second (N_p+1) n^3 FP32 buffer.  Not for batch instances. */

/* Transfers between the fine grid and the coarse grid of the stencil coarse
 * propagator (coarse_factor r > 1; Sec. 2.2.2 notes that a coarse propagator
 * on a coarser mesh needs them and that their order matters):
 * BOX      box average over the r^3 fine points of a coarse cell, trilinear
 *          prolongation from the cell centroids (default);
 * SPECTRAL the Fourier modes both grids represent (|k_d| <= n/(2r) - 1 on
 *          every axis) are kept with their coefficients, all others are
 *          dropped, coarse point I on fine point I r; applied as separable
 *          real matrices along each axis, in the coarse propagator's
 *          precision.  Only with coarse_kind STENCIL and r > 1, and with
 *          n (n / r) elements of G's precision per transfer matrix at most
 *          160 KiB. */
enum { PARAREAL_TRANSFER_BOX = 0, PARAREAL_TRANSFER_SPECTRAL = 1 };

/* Layers of the learned coarse propagator (coarse_kind LEARNED / SHIFT):
 * GELU   the network as specified: GELU after the first three convolutions,
 *        biases, second input channel the constant nu(t_n)/nu0;
 * LINEAR identity activations, no biases, second input channel
 *        nu(t_n)/nu0 * Sk(u) (Sk the skip propagator): G is then linear in u,
 *        with a kernel that depends on nu(t_n). */
enum { PARAREAL_ACT_GELU = 0, PARAREAL_ACT_LINEAR = 1 };

/* Evaluation of a LINEAR learned propagator (learned_act LINEAR):
 * LAYERS   layer by layer: BF16 weights and activations, FP32 accumulation,
 *          the 16 -> 16 layers on the tensor cores;
 * COMPOSED the four linear layers composed into one 9x9x9 periodic
 *          cross-correlation per slice, K_0 + nu(t_n)/nu0 K_1 (built in FP64
 *          from the FP32 master weights whenever the model changes), applied
 *          with FP32 accumulation: the same linear operator in about a
 *          twentieth of the arithmetic.
 * POLYPHASE with the stencil skip on a coarsened grid (coarse_factor r in
 *          {2, 4, 8}, BOX transfers, n a multiple of 16): the composed kernel
 *          and the skip's trilinear prolongation folded into r^3 phase
 *          kernels on the coarse grid (4^3 taps each for r = 4, 3^3 for
 *          r = 8, 6^3 for r = 2; built in FP64, applied in G's precision with
 *          FP32 weights).  G's output then stays on the coarse grid, as the
 *          stencil propagator's does, and the correction prolongs the change
 *          of G's output through the phase kernels: G costs about what the
 *          stencil propagator costs.  The same linear operator as COMPOSED.
 *          No counterpart in the paper. */
enum { PARAREAL_EVAL_LAYERS = 0, PARAREAL_EVAL_COMPOSED = 1, PARAREAL_EVAL_POLYPHASE = 2 };

/* Evaluation of the correction (Eq. parareal):
 * STANDARD   U^{k+1}[n+1] = F(U^k[n]) + (G(U^{k+1}[n]) - G(U^k[n])), as printed;
 * DIFFERENCE U^{k+1}[n+1] = F(U^k[n]) + G(U^{k+1}[n] - U^k[n]), the same for a
 *            linear G (stencil, Euler/upwind, shift, or the LINEAR learned
 *            propagator; rejected for a GELU network).  Rounding in G then
 *            scales with the change of its input instead of with the field,
 *            so a G evaluated in low precision (BF16) does not put a floor
 *            under the defect.  No counterpart in the paper. */
enum { PARAREAL_CORRECTION_STANDARD = 0, PARAREAL_CORRECTION_DIFFERENCE = 1 };

/* Skip path of the learned coarse propagator (coarse_kind LEARNED / SHIFT):
 * SHIFT   G = S(u) + Net([S(u), nu/nu0]) on the grid n / coarse_factor;
 * STENCIL G = Gs(u) + Net([Gs(u), nu/nu0]) on the fine grid, Gs the stencil
 *         coarse propagator (RK4 on n / coarse_factor at dt_coarse, box
 *         restriction, trilinear prolongation): the net learns F - Gs. */
enum { PARAREAL_SKIP_SHIFT = 0, PARAREAL_SKIP_STENCIL = 1 };

/* Validate cfg, run the stability pre-check, allocate all device workspace
 * and return a context bound to `cuda_stream` (a cudaStream_t; NULL = default
 * stream) on the current device.  On failure *out is NULL. */
parareal_status parareal_create(const parareal_config *cfg, void *cuda_stream,
                                parareal_ctx **out);

/* Stability pre-check without allocation: the largest per-step amplification
 * max |R(dt lambda(k))| over all Fourier modes k of the fine and coarse grids
 * and over nu in [nu0(1-|amp|), nu0(1+|amp|)], where R is the RK4 polynomial
 * (1 + z for forward Euler) and lambda the symbol of the operator (the fine
 * scheme for F; 7-point/centred for the stencil G, 7-point/upwind for the
 * Euler G).  growth[0] = fine, growth[1] = coarse (stencil or Euler G, else
 * 0).  Returns E_UNSTABLE when either exceeds 1 + 1e-12 (the per-step value is
 * still written). */
parareal_status parareal_stability(const parareal_config *cfg, double *growth2);

/* Set u0 = U[0] (Algorithm 1, "Data: initial condition") and reset the
 * iteration: every U^0[n] is produced by the initial serial coarse run on the
 * next parareal_iterate.  u0: n^3 values of `dtype`; `mem` says where. */
parareal_status parareal_set_problem(parareal_ctx *ctx, const void *u0, int dtype, int mem);

/* Fine propagator on a batch of slices (the concurrent F evaluations of
 * Sec. 2.2): Fv[n+1] = F(U[n]) for n in [first_slice, first_slice + count).
 * All slices run in the same launches. */
parareal_status parareal_fine_sweep(parareal_ctx *ctx, int first_slice, int count);

/* Coarse propagator.  chain = 1: the serial start-up run (Algorithm 1,
 * initialisation) U[n+1] = G(U[n]) and Gold[n+1] = G(U[n]) for n = first..first+count-1
 * in order.  chain = 0: Gold[n+1] = G(U[n]) for every slice in the range, U unchanged. */
parareal_status parareal_coarse_sweep(parareal_ctx *ctx, int first_slice, int count, int chain);

/* Run Parareal iterations (Algorithm 1 loop body for all slices): fine sweep
 * over the slices not yet exact, then the serial coarse sweep with the
 * correction U^{k+1}[n+1] = F(U^k[n]) + (G(U^{k+1}[n]) - G(U^k[n])) and the
 * defect norms, until the stopping rule holds or k_max iterations ran.  The
 * first call after set_problem first runs the coarse start-up chain.
 * k_done (may be NULL) receives the number of iterations run by this call;
 * hist (may be NULL) receives 4 doubles per iteration: {max_n diff_inf,
 * max_n diff_l2, defect (or -1 without a reference), elapsed ms}. */
parareal_status parareal_iterate(parareal_ctx *ctx, int k_max, double tol, int stop_rule,
                                 int *k_done, double *hist);

/* The iterations of parareal_iterate, with the same arguments, results and
 * iterates (bit for bit), run as ONE CUDA graph launch with the stopping
 * test on the device instead of one host round trip per iteration.  The
 * graph (conditional nodes) is a WHILE loop whose pass selects, with a
 * SWITCH on the number K of slices already exact, the iteration body
 * captured for that K (Eq. parareal for slices K..N_p-1: batched fine
 * sweep, serial coarse sweep with corrections, norms), followed by a
 * one-thread kernel that applies the stopping rule to the norms and ends
 * the loop (Sec. 2.2.4 criteria).  No counterpart in the paper: its loop
 * runs on the host of each node.
 * - The first call captures N_p bodies and instantiates the graph (once per
 *   context); it is rebuilt when the launch shapes change (parareal_autotune)
 *   or a reference is set or cleared.  Weights of a learned propagator may
 *   change between calls.
 * - hist[4 i + 3] is device time (ms, %globaltimer) since the first
 *   iteration of the call started.
 * - The context must have been advanced only by parareal_iterate and this
 *   call since parareal_set_problem (else PARAREAL_E_STATE); kernel timing
 *   (parareal_profile) does not see the launches inside the graph.
 * - Synchronises the context stream.  Errors as parareal_iterate. */
parareal_status parareal_iterate_device(parareal_ctx *ctx, int k_max, double tol, int stop_rule,
                                        int *k_done, double *hist);

/* Per-slice residuals of the current iterate; per_slice_out receives
 * n_slices + 1 doubles (index 0 = u0, always 0). */
parareal_status parareal_residual(parareal_ctx *ctx, int kind, double *per_slice_out);

/* Reference solution u_fine(T) for the defect d^k (Eq. defect). */
parareal_status parareal_set_reference(parareal_ctx *ctx, const void *ref, int dtype, int mem);

/* Serial fine run of all slices (Eq. fine applied for n = 0..N_p-1) from u0;
 * writes u_fine(T) to dst (n^3 values of dtype, `mem` says where) and, when
 * `as_reference` is nonzero, also stores it as the defect reference. */
parareal_status parareal_serial_fine(parareal_ctx *ctx, void *dst, int dtype, int mem,
                                     int as_reference);

/* Copy U[slice] (0..n_slices) out of / into the context, converting to/from dtype. */
parareal_status parareal_get_slice(parareal_ctx *ctx, int slice, void *dst, int dtype, int mem);
parareal_status parareal_set_slice(parareal_ctx *ctx, int slice, const void *src, int dtype, int mem);

/* Apply F or G of time slice first_slice+i to count caller fields in place
 * of the context's iterate: dst[i] = P(src[i]) where src and dst hold count
 * consecutive n^3 fields of `dtype` in device memory.  which = 0: F, 1: G. */
parareal_status parareal_propagate(parareal_ctx *ctx, int which, const void *src, void *dst,
                                   int dtype, int first_slice, int count);

/* Learned coarse propagator (coarse_kind PARAREAL_COARSE_LEARNED; SHIFT is
 * the same propagator with every weight zero):
 *     G(u, t_n) = S(u) + Net([S(u), nu(t_n)/nu0])
 * on the grid n / coarse_factor (box restriction before, trilinear
 * prolongation after, when coarse_factor > 1).  S shifts periodically by
 * round(a_d * (T/N_p) * m) cells per axis, the transport of one slice.  Net:
 * 3x3x3 periodic convolutions 2 -> 16 -> 16 -> 16 -> 1 with GELU after the
 * first three; BF16 weights and activations, FP32 accumulation.  There is no
 * counterpart in the paper, whose G is a stencil (Algorithm 2).
 *
 * The model is PARAREAL_MODEL_PARAMS FP32 values, in this order (tap index
 * (dz+1)*9 + (dy+1)*3 + (dx+1)):
 *   W1[16][2][27] b1[16] W2[16][16][27] b2[16] W3[16][16][27] b3[16] W4[1][16][27] b4[1]
 * A new context starts with every value zero (G = S). */
#define PARAREAL_MODEL_PARAMS 15169

typedef struct {
    int epochs;                  /* passes over the pairs */
    int batch;                   /* pairs per Adam step (the remainder of an epoch is dropped) */
    double lr, beta1, beta2, eps;/* Adam */
    unsigned long long seed;     /* shuffling seed */
} parareal_train_config;

/* Copy the model in / out (w: PARAREAL_MODEL_PARAMS floats; `mem` says
 * where).  Setting a model resets the Adam moments and restarts the iteration
 * at the coarse start-up on the next parareal_iterate. */
parareal_status parareal_set_coarse_model(parareal_ctx *ctx, const float *w, int mem);
parareal_status parareal_get_coarse_model(parareal_ctx *ctx, float *w, int mem);

/* Training pairs from the fine propagator: ics holds n_ics FP32 fields
 * (device, n^3 each); for each the serial fine trajectory over all slices
 * gives pairs (u_n, F(u_n)), n = 0..N_p-1, written at pair index ic*N_p + n
 * of pairs_u / pairs_f (device, FP32, on the net's grid: (n/coarse_factor)^3
 * each with the SHIFT skip, n^3 with the STENCIL skip).  With the STENCIL skip
 * pairs_u holds the net's input Gs(u_n) instead of u_n.  pair_slice (host,
 * may be NULL) receives n for every pair. */
parareal_status parareal_make_pairs(parareal_ctx *ctx, const float *ics, int n_ics, float *pairs_u,
                                    float *pairs_f, int *pair_slice);

/* Train the model on n_pairs pairs (device FP32 fields on the net's grid;
 * pair_slice on the host gives the slice index of each pair) by Adam on the
 * mean squared error |G(u) - F(u)|^2 over all points of a batch.  loss_hist
 * (host, may be NULL) receives one mean loss per epoch.  Where the net's
 * grid edge is a multiple of 16, the 16 -> 16 layers' forward and both
 * gradients run on the tensor cores, whose completion waits are bounded:
 * PARAREAL_E_TIMEOUT if one gave up (checked after every epoch; the
 * context stays usable). */
parareal_status parareal_train_coarse(parareal_ctx *ctx, const float *pairs_u, const float *pairs_f,
                                      const int *pair_slice, int n_pairs,
                                      const parareal_train_config *tc, double *loss_hist);

/* One forward and backward pass without an update: the mean squared error
 * over `count` fields (device FP32, net grid) against `target`, and its
 * gradient (device, PARAREAL_MODEL_PARAMS floats).  slices: host, count ints.
 * PARAREAL_E_TIMEOUT as for parareal_train_coarse. */
parareal_status parareal_coarse_model_grad(parareal_ctx *ctx, const float *u, const float *target,
                                           const int *slices, int count, float *grad_out,
                                           double *loss);

/* Autotuner: times every compiled launch shape of the fine step kernel (tile
 * in x and y, one or two region rows per thread, z-march chunk, or the
 * per-stage path) on this context's batch
 * of slices and on a single field, and of the coarse step kernel on the
 * coarse grid, keeps the fastest of each, and appends them to `cache_path`
 * (JSON lines keyed by grid edge,
 * dtype, batch size and SM count; NULL = no cache).  A cached key is reused
 * without timing.  Uses the iterate as scratch: call before
 * parareal_set_problem.  ms2 (may be NULL): best fine / coarse ms per step
 * (-1 when taken from the cache). */
parareal_status parareal_autotune(parareal_ctx *ctx, const char *cache_path, double *ms2);

/* The launch shapes in use, each {path, tile_x, tile_y, z chunk}: the batched
 * fine sweep, the coarse steps, and one fine field at a time (serial fine
 * run, propagate).  Paths: 0 fused with one region row per thread, 1
 * per-stage, 2 fused with two rows per thread, 3 persistent (every step of a
 * sweep in one cooperative launch), 4 cluster (every step of a sweep in one
 * launch, each field held in the shared memory of one thread-block cluster;
 * tile_x and tile_y unused).  Paths 1, 3 and 4 give bitwise the same fields.
 * Any pointer may be NULL.  The environment variables PARAREAL_FINE_TILE,
 * PARAREAL_SERIAL_TILE, PARAREAL_COARSE_TILE and PARAREAL_PIPE_TILE
 * ("path,tile_x,tile_y,zchunk") set the shapes at parareal_create. */
parareal_status parareal_get_launch_shape(const parareal_ctx *ctx, int *fine4, int *coarse4,
                                          int *serial4);

/* The number of CTAs of the cluster that holds one n^3 field of `dtype`
 * (PARAREAL_F32 / PARAREAL_F64) in launch path 4, or 0 when the field does
 * not fit one cluster (four n^3 arrays, three of them with a ghost plane
 * below and above each CTA's planes, in at most 200 KiB of shared memory per
 * CTA; planes split evenly over up to 16 CTAs where the device schedules
 * 16-CTA clusters, else over up to 8).  No counterpart in the paper. */
int parareal_cluster_size(int dtype, int n);

/* Batches of independent problems of uneven sizes.  Each instance is a
 * context of its own (its own config, workspace and stream); one round of
 * the batch (the coarse start-up, or one iteration of every instance not yet
 * stopped) is one CUDA graph whose parallel branches are the instances.
 * There is no counterpart in the paper, which runs one problem. */
typedef struct parareal_batch parareal_batch;
/* cuda_stream: the stream rounds are captured on and launched in (NULL: the
 * batch creates a stream of its own; the legacy default stream cannot be
 * captured). */
parareal_status parareal_batch_create(const parareal_config *cfgs, int count, void *cuda_stream,
                                      parareal_batch **out);
parareal_status parareal_batch_set_problem(parareal_batch *b, int i, const void *u0, int dtype, int mem);
/* Serial fine run of every instance (concurrently); as_reference as in parareal_serial_fine. */
parareal_status parareal_batch_serial_fine(parareal_batch *b, int as_reference);
/* Up to k_max rounds; every instance stops on its own rule.  k_done and defect
 * (host, count entries each, may be NULL): iterations run and last d^k (-1 without reference). */
parareal_status parareal_batch_iterate(parareal_batch *b, int k_max, double tol, int stop_rule,
                                       int *k_done, double *defect);
/* Autotune once per distinct (n, n/coarse_factor, dtype, N_p); call before set_problem. */
parareal_status parareal_batch_autotune(parareal_batch *b, const char *cache_path);
/* How the fine sweeps of a round run.  mode 0 (default): each instance's own
 * batched launches, in its branch of the round's graph.  mode 1: ONE
 * persistent launch over a queue of every open instance's tile steps (all
 * steps, all slices, all tiles, in step order), with tile_x x tile_y tiles
 * and `rows` region rows per thread for every instance (a tile that reaches
 * past a grid's edge wraps and writes only its own points); CTAs take the
 * next tile step from a device counter, and a step of instance i waits
 * (bounded) until every tile of i's previous step is done.  The coarse
 * sweeps and corrections then run as the graph's per-instance branches.
 * In mode 1 every instance's own fine launches (its fine_sweep calls) take
 * the queue's tile shape too; its serial fine run keeps its shape when that
 * is a fused one and takes the queue's otherwise.  The fused tile step gives
 * every point the same arithmetic whatever the shape, so the reference and
 * the iterates share one arithmetic; an instance's iterates are then the
 * same, bit for bit, as in mode 0 with fused fine shapes.
 * mode 1 needs FP32 instances of the 7-point operator, at most 64, and one
 * of the compiled shapes (64x32 and 64x16 with one row per thread, 32x16,
 * 64x32 with two); parareal_batch_autotune then picks the shape by timing.
 * A queue wait that gives up makes parareal_batch_iterate return
 * PARAREAL_E_TIMEOUT.  No counterpart in the paper. */
parareal_status parareal_batch_set_fine_mode(parareal_batch *b, int mode, int tile_x, int tile_y,
                                             int rows);
/* mode4 = {mode, tile_x, tile_y, rows} of parareal_batch_set_fine_mode. */
parareal_status parareal_batch_get_fine_mode(const parareal_batch *b, int *mode4);
/* The context of instance i (owned by the batch; use it for get_slice etc.). */
parareal_ctx *parareal_batch_context(parareal_batch *b, int i);
long long parareal_batch_graph_launches(const parareal_batch *b);
const char *parareal_batch_last_error(const parareal_batch *b);
void parareal_batch_destroy(parareal_batch *b);

/* Kernel timing.  While enabled, the context records a pair of CUDA events
 * (on its stream) around every launch of the fine propagator's step kernel
 * and accumulates them; parareal_profile_read synchronises the stream and
 * returns the summed device time (ms), the number of timed launches and the
 * algorithmic bytes they moved (one read and one write of every field per
 * RK4 step), then clears the accumulators.  Enabling also clears them. */
parareal_status parareal_profile(parareal_ctx *ctx, int enable);
parareal_status parareal_profile_read(parareal_ctx *ctx, double *fine_ms, long long *fine_launches,
                                      double *fine_bytes);

/* Defect norms without any device allocation.
 *
 * a and b are caller-owned FP64 device arrays of `count` values; out5 is a
 * caller-owned device array of 5 doubles that receives max|a-b|, max|b|,
 * sum (a-b)^2, sum b^2 and 1.0 if some a-b is NaN or infinite (else 0.0):
 * the numbers behind the defect d^k = out5[0] / out5[1].  The paper has no
 * counterpart of this call.
 *
 * It exists for callers that cannot call cudaMalloc: code that records work
 * into a CUDA graph while stream capture is active (allocation cannot be
 * captured), code running inside a framework whose caching allocator owns the
 * device memory (a second allocator would fragment it or break its
 * accounting), and latency-critical loops that must not wait on the driver's
 * allocation lock.  The per-block partial sums go to a fixed scratch array
 * compiled into the library (640 KiB of device memory, held by every GPU that
 * loads the library until the process exits).
 *
 * - count must be at most PARAREAL_NOALLOC_MAX_COUNT; larger counts return
 *   PARAREAL_E_INVALID and launch nothing (message: parareal_noalloc_last_error).
 * - Asynchronous on cuda_stream (NULL = default stream): out5 is valid once
 *   that stream reaches this point.
 * - The first call on a device looks up the scratch array's device address
 *   (cudaGetSymbolAddress); make that first call before any stream capture.
 * - All calls share the one scratch array: calls that may overlap on the GPU
 *   (different streams, concurrent graph replays) race and must be ordered
 *   by the caller.  Each call overwrites every scratch entry it reads, so no
 *   clearing is needed between calls. */
#define PARAREAL_NOALLOC_MAX_COUNT 67108864LL
parareal_status parareal_diff_norms_noalloc(const double *a, const double *b, long long count,
                                            double *out5, void *cuda_stream);
const char *parareal_noalloc_last_error(void);

/* Checkpoint and resume of the iteration state (a fault-tolerance aid; no
 * counterpart in the paper).  parareal_save_state copies the iterate
 * U^k[0..N] (FP64), the stored coarse outputs G(U^k[n]), the reference
 * u_fine(T) if one is set, and the iteration count into a caller-owned host
 * buffer of at least *needed bytes (host NULL: only report *needed).
 * parareal_load_state restores such a buffer into a context created with the
 * same configuration (grid, slices, coarsening, precision, kind of G); the
 * next parareal_iterate then continues exactly, bitwise, where the saved
 * context would have.  A learned propagator's weights are not part of the
 * state (parareal_get/set_coarse_model), but a fingerprint of them is: with
 * a learned G, saving and loading need a model, and a state saved with other
 * weights is refused.  The per-slice changes reported by
 * parareal_residual(DIFF_*) read zero until the next iteration.  Both calls
 * synchronise the context stream.  Errors: PARAREAL_E_STATE (nothing to
 * save; learned G without a model, or with other weights than the saved
 * state's), PARAREAL_E_INVALID (buffer too small, not a saved state, or
 * another configuration). */
parareal_status parareal_save_state(parareal_ctx *ctx, void *host, size_t bytes, size_t *needed);
parareal_status parareal_load_state(parareal_ctx *ctx, const void *host, size_t bytes);

/* Failure-detection self-test.  Runs the bounded device-side wait of the
 * tensor-core layers (the learned propagator's wait for MMA completion) on a
 * barrier that nothing ever arrives on, in one single-warp kernel on
 * `cuda_stream` (NULL = the legacy default stream), and synchronises it.
 * Returns PARAREAL_E_TIMEOUT when the wait gave up as designed (after about
 * 2^18 tries), PARAREAL_OK if it did not (a broken wait), PARAREAL_E_CUDA on
 * a CUDA error.  Allocates one int of device memory for the flag.  The device
 * stays usable afterwards.  No counterpart in the paper. */
parareal_status parareal_selftest_timeout(void *cuda_stream);

/* Failure-detection self-test of the grid barrier of the persistent RK4
 * path (launch path 3: all steps of a sweep in one cooperative launch, the
 * blocks meeting at a grid barrier between stages).  One cooperative launch
 * of one block per SM in which block 0 leaves without arriving: every other
 * block's bounded wait (about 2^20 polls) gives up and sets the error flag,
 * which the host reads.  Returns PARAREAL_E_TIMEOUT when the waits gave up
 * as designed, PARAREAL_OK if they did not (a broken wait), PARAREAL_E_CUDA
 * on a CUDA error.  Allocates 16 bytes of device memory; the device stays
 * usable.  A context whose persistent launch gives up the same way reports
 * PARAREAL_E_TIMEOUT from the call that ran it and stays usable.  No
 * counterpart in the paper. */
parareal_status parareal_selftest_grid_barrier(void *cuda_stream);

/* Number of kernel launches this context issued so far (for reporting). */
long long parareal_launch_count(const parareal_ctx *ctx);

/* Message of the last failure of this context ("" if none); with ctx NULL,
 * the last failure of parareal_create on this thread. */
const char *parareal_last_error(const parareal_ctx *ctx);

/* Free all device workspace.  NULL is accepted. */
void parareal_destroy(parareal_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PARAREAL_H */
