/*
 * mase.h - C ABI of libmase: GB300-native multi-area weighted-least-squares
 * (WLS) power-system state estimation by boundary-condensed Gauss-Newton.
 *
 * Method (arXiv 2604.23175):
 *   - measurement model z = h(x) + e, WLS objective J = r^T W r,
 *     r = z - h(x), W = R^{-1}                      (Sec. 2.1, Eqs. meas_model, wls)
 *   - Gauss-Newton step G dx = H^T W r, G = H^T W H   (Sec. 2.1, Eq. gn_normal)
 *   - typed measurement templates evaluated without forming H
 *                                                    (Sec. 2.2, Eq. typed_meas; Sec. 4.1-4.2)
 *   - per-area blocks, Schur condensation S_b = G_bb - G_bi G_ii^{-1} G_ib,
 *     b_hat = b_b - G_bi G_ii^{-1} b_i              (Sec. 3.1-3.2, Eqs. block_normal, schur_defs)
 *   - coordinator S_Gamma = sum_k E_k^T S_b^k E_k, solve, scatter back,
 *     interior recovery                              (Sec. 3.2, Eqs. global_assembly, backsub;
 *                                                     Sec. 4.3-4.4)
 *
 * Conventions used by every entry point:
 *   - Bus indices are 0-based int32.  Angles are radians, per unit elsewhere.
 *   - State layout x[n_snap][2*n_bus] = (Vm[0..N), Va[0..N)) per snapshot.
 *     The slack angle is held at its value in x0 (0 for a flat start), so a
 *     snapshot has n = 2N - 1 unknowns.
 *   - Canonical measurement row order, m = 3N + 4L:
 *       Vm[N], Pinj[N], Qinj[N], Pf[L], Qf[L], Pt[L], Qt[L]
 *     "f" rows are measured at the from end of a branch, "t" rows at its to
 *     end; injections are positive into the network.
 *   - Branch model: pi equivalent, series admittance 1/(r + jx), total line
 *     charging b split b/2 at each end; no taps, no bus shunts.
 *   - Pointers to per-snapshot arrays (z, mask, x0, x_out) may point to host
 *     or device memory; the library asks the CUDA runtime which.  All other
 *     pointers are host pointers.  The caller keeps ownership of everything
 *     it passes; the library copies what it needs before returning.
 *   - Return value: MASE_OK (0), a negative error code, or MASE_NOT_CONVERGED
 *     (positive) from mase_solve.  mase_status_str() names each code and
 *     mase_last_error() gives the message of the last failure on this thread.
 *   - A handle is not re-entrant: do not call it from two threads at once.
 *     Distinct handles are independent.  Work is enqueued on the stream given
 *     in mase_options (NULL = the legacy default stream); calls return after
 *     their results are available to the caller.
 */
#ifndef MASE_H
#define MASE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define MASE_OK                 0
#define MASE_NOT_CONVERGED      1   /* some snapshot reached max_iter         */
#define MASE_EINVAL           (-1)  /* bad size, index, pointer or option     */
#define MASE_EUNOBSERVABLE    (-2)  /* non-positive pivot: G_ii or S_Gamma not SPD */
#define MASE_ENONFINITE       (-3)  /* NaN/Inf in inputs or iterates          */
#define MASE_EDEVICE          (-4)  /* CUDA error, out of device memory        */
#define MASE_ENOTREADY        (-5)  /* no measurements / no warm-start model  */

/* per-snapshot status codes written to mase_stats.status */
#define MASE_SNAP_CONVERGED     0
#define MASE_SNAP_MAX_ITER      1
#define MASE_SNAP_NOT_SPD       2
#define MASE_SNAP_NONFINITE     3
#define MASE_SNAP_DEVICE        4   /* a bounded device-side wait gave up      */

/* precision modes */
#define MASE_FP64   0   /* every step in FP64 (the plain comparator)               */
#define MASE_MIXED  1   /* FP32 gain, factor, Schur and solves; FP64 residual,
                           gradient H^T W r, assembly of b_hat, refinement of the
                           boundary solve and update                             */
/* start modes */
#define MASE_START_FLAT     0   /* Vm = 1, Va = 0                               */
#define MASE_START_X0       1   /* x0 given to mase_solve                        */
#define MASE_START_LEARNED  2   /* per-area MLP proposal (mase_warmstart_*),
                                   kept only where it lowers J below the flat start;
                                   a snapshot whose factor then breaks down is
                                   solved again from the flat start           */
/* schedule modes */
#define MASE_PER_AREA   0   /* one launch per area and stage, like per-area streams */
#define MASE_BATCHED    1   /* one launch per stage over every (area, snapshot)   */

typedef struct mase_handle mase_handle;

/* Network (Sec. 2.1 bus-branch model).  Arrays have n_branch entries. */
typedef struct {
    int32_t n_bus, n_branch, slack_bus;
    const int32_t *from_bus, *to_bus;   /* 0-based, from != to                    */
    const double *r, *x;                /* series resistance, reactance (p.u.)    */
    const double *b_charge;             /* total line charging (p.u.)             */
} mase_network;

/* Partition into K areas (Sec. 2.3).  area_of_bus[n_bus] in [0, n_area);
 * every area must own at least one bus. */
typedef struct {
    int32_t n_area;
    const int32_t *area_of_bus;
} mase_partition;

/* Measurements (Sec. 2.1, 4.1).  sigma[m] is shared by all snapshots
 * (W = diag(1/sigma^2)); mask[n_snap][m] (1 = present, 0 = masked, weight 0)
 * or NULL for all present; z[n_snap][m] or NULL to supply it later with
 * mase_set_measurements. */
typedef struct {
    int32_t n_snap;
    const double *z;
    const double *sigma;
    const uint8_t *mask;
} mase_measurements;

typedef struct {
    int32_t precision;   /* MASE_FP64 | MASE_MIXED                     */
    int32_t schedule;    /* MASE_PER_AREA | MASE_BATCHED               */
    int32_t use_graph;   /* 1: run the Gauss-Newton loop as one CUDA graph
                            with a device-side loop (no host round trip per
                            step); 0: launch each step from the host      */
    int32_t refine;      /* boundary refinement sweeps (MIXED), 0..8    */
    int32_t threads;     /* threads per CTA of the area kernels, 0=auto */
    int32_t device;      /* CUDA device ordinal                         */
    void   *stream;      /* cudaStream_t, NULL = default stream         */
    int32_t profile;     /* 1: step from the host (use_graph is ignored) and
                            time each stage's kernels with CUDA events on
                            the library's stream; mase_stats.stage_ms[0..3]
                            then hold those event times                  */
    int32_t wait_polls;  /* unsatisfied polls after which a device-side
                            dependency wait of the area factorisation gives
                            up (snapshot status MASE_SNAP_DEVICE); 0 = the
                            default (4194304 polls, about 0.2 s).  Small
                            values exist to exercise that error path.     */
    int32_t inner_iters; /* 0..8 local Gauss-Newton steps per area with the
                            boundary state held fixed before each condensed
                            step (Eq. local_wls); 0 = the exact condensed
                            step alone, whose iterates equal centralised GN */
    int32_t autotune;    /* 1 (default): with MASE_BATCHED, mase_create times
                            candidate launch configurations on the device (on
                            a synthetic flat-start problem, so it needs no
                            measurements) and keeps the fastest: the split of
                            the areas into concurrent launch classes by the
                            shared memory they need and the block size of
                            each class, the back-substitution block size and
                            the coordinator's form; mase_info reports them   */
    int32_t tensor_units;/* MASE_MIXED: factorisation update units whose source
                            panel has at least this many columns run on the
                            tensor cores as m16n8k8 TF32 MMAs with split
                            operands (3xTF32, FP32-accurate products);
                            0 = every unit on the FP32 pipes; -1 = the
                            default (see mase_default_options)           */
} mase_options;

/* Per-solve results.  Arrays are host arrays of n_snap entries supplied by
 * the caller (any may be NULL). */
typedef struct {
    int32_t *iters;       /* Gauss-Newton steps taken per snapshot              */
    int32_t *status;      /* MASE_SNAP_* per snapshot                           */
    double  *J;           /* r^T W r at the returned state, per snapshot        */
    double  *max_step;    /* max |dx| of the last step, per snapshot            */
    double   stage_ms[7]; /* where solve_ms went, in ms: [0] area kernel (evaluation,
                             accumulation, condensation; with inner_iters also the
                             inner steps' interior recoveries), [1] coordinator, [2] back-
                             substitution, [3] bookkeeping, each summed over the steps
                             from device clocks (first block start to last block end
                             of the stage's launches), or from CUDA events around the
                             stage's kernels with options.profile; [4] learned start (inference
                             and its objective test); [5] the rest outside the loop (reset,
                             state in/out, objective pass, result copies); [6] time
                             inside the loop outside the stages' kernels (launch gaps,
                             and the per-step host round trip when use_graph = 0).
                             The seven sum to solve_ms.                           */
    double   solve_ms;       /* wall time of the solve on the library's stream    */
    int32_t  total_launches; /* kernels launched by the solve                   */
    int32_t  steps;          /* Gauss-Newton steps run for the batch (max over snapshots),
                                the flat-start fallback's included              */
    int32_t  restarted;      /* snapshots of a learned start whose factor broke down
                                from the networks' proposal (non-positive pivot or
                                non-finite step) and were solved again from the flat
                                start; their iters include the failed attempt's */
} mase_stats;

/* Structural sizes of a handle (host-side setup results). */
typedef struct {
    int32_t n_bus, n_branch, n_area, n_snap, n_meas, n_state;
    int32_t n_boundary_bus, n_gamma;        /* |boundary buses|, dim x_Gamma   */
    int32_t max_area_vars, max_area_nb;     /* largest n_i + n_b, largest n_b   */
    int64_t factor_nnz;                     /* sum over areas of stored factor entries */
    int64_t local_flops, boundary_flops;    /* per snapshot and GN step (multiply-adds) */
    int64_t g_updates;                      /* gain-matrix scalar updates per snapshot */
    int32_t smem_bytes_max;                 /* largest per-area shared-memory need */
    int32_t areas_in_smem;                  /* areas whose factor fits shared memory */
    int64_t n_supernodes, n_units;          /* over all areas: supernodes, update column units */
    int32_t max_levels;                     /* deepest level schedule of an area */
    int32_t max_area_store;                 /* largest per-area factor storage (entries) */
    int32_t boundary_store;                 /* boundary-system factor storage (entries) */
    int32_t boundary_levels;                /* levels of the boundary factor */
    int64_t coord_S_elems;                  /* sum over areas of nb(k)(nb(k)+1)/2: packed
                                               Schur-block entries of one snapshot */
    int64_t coord_b_elems;                  /* sum over areas of nb(k): condensed rhs
                                               entries of one snapshot */
    /* launch configuration (chosen by the autotuner when options.autotune) */
    int32_t tuned;                          /* 1: measured at create */
    int32_t local_classes;                  /* concurrent launch classes of the area kernel */
    int32_t class_areas[4];                 /* areas in each class */
    int32_t class_threads[4];               /* threads per block of each class */
    int32_t class_smem[4];                  /* dynamic shared memory per block of each class */
    int32_t back_threads;                   /* threads per block of the back-substitution */
    int32_t coord_cluster;                  /* 1: coordinator on 2-block clusters */
    float   tune_local_ms[2];               /* area-kernel time of one step on the tuning problem:
                                               one launch for every area, and the chosen classes */
} mase_info;

/* Default options: MIXED, BATCHED, graph on, one FP64 refinement sweep of the
 * boundary solve, device 0.  (refine = 0 makes each Gauss-Newton step an
 * inexact Newton step; the FP64 residual and gradient still fix the
 * converged state.) */
void mase_default_options(mase_options *opt);

/* Build a handle: validates the inputs, runs the one-time symbolic setup
 * (boundary sets and selectors E_k, measurement templates and gain-matrix
 * slot maps, fill-reducing orderings and supernodal symbolic factors of every
 * area and of the boundary system; Sec. 4.1, 4.3) and allocates every device
 * buffer once (Sec. 5.1).  meas->n_snap fixes the batch size.
 * Errors: MASE_EINVAL (sizes, indices, from == to, sigma <= 0, empty area),
 * MASE_EDEVICE.  *out is set only on success. */
int mase_create(const mase_network *net, const mase_partition *part,
                const mase_measurements *meas, const mase_options *opt,
                mase_handle **out);

/* Replace z (and the mask if meas->mask != NULL) for the next solve.
 * meas->n_snap must equal the handle's batch size; sigma is ignored. */
int mase_set_measurements(mase_handle *h, const mase_measurements *meas);

/* Solve every snapshot of the batch by Gauss-Newton from the start given by
 * the handle's start mode: x0 (n_snap x 2N) is used when non-NULL, otherwise
 * a flat start (or the learned start after mase_set_start_mode).  Stops a
 * snapshot once max|dx| < tol (the step is applied) or after max_iter steps.
 * x_out (n_snap x 2N) receives the estimates.  Each Gauss-Newton step is the
 * condensed step of Eqs. block_normal, schur_defs, global_assembly and
 * backsub, equal to the centralised step of Eq. gn_normal.  Per-snapshot
 * results go to stats.  The return value is the code of the worst snapshot:
 * MASE_EDEVICE (a bounded device-side wait gave up), else MASE_EUNOBSERVABLE
 * (a non-positive pivot), else MASE_ENONFINITE, else MASE_NOT_CONVERGED
 * (max_iter reached), else MASE_OK.  Other errors: MASE_EINVAL (NULL handle,
 * max_iter outside 1..1000, tol < 0 or NaN), MASE_ENOTREADY (no measurements,
 * or a learned start without a model), MASE_EDEVICE (a CUDA error, or a
 * tensor-core wait of the learned start that ran out). */
int mase_solve(mase_handle *h, const double *x0, double tol, int32_t max_iter,
               double *x_out, mase_stats *stats);

/* Evaluate h(x) (Eq. typed_meas: voltage magnitudes, injections and flows
 * at both ends under the pi model) for n_snap states x[n_snap][2N]
 * (Vm then Va per snapshot) into z_out[n_snap][m] (canonical order).  Uses
 * the handle's network; n_snap is independent of the handle's batch size;
 * x and z_out host or device.  Errors: MASE_EINVAL (NULL pointers,
 * n_snap < 1), MASE_EDEVICE. */
int mase_measure(mase_handle *h, const double *x, int32_t n_snap, double *z_out);

/* Copy the structural information and autotuner choices filled by
 * mase_create into *info.  MASE_EINVAL for NULL arguments. */
int mase_get_info(const mase_handle *h, mase_info *info);

/* Choose the start mode used by mase_solve when x0 is NULL: MASE_START_FLAT
 * (or MASE_START_X0, which then also means flat) or MASE_START_LEARNED (a
 * later mase_solve returns MASE_ENOTREADY if no model is trained or loaded).
 * MASE_EINVAL for a NULL handle or another value. */
int mase_set_start_mode(mase_handle *h, int32_t start_mode);

/* Host-only: run the one-time symbolic setup of mase_create (Sec. 4.1, 4.3)
 * without touching a GPU and report its structural sizes (n_snap and
 * smem fields are left 0).  Errors: MASE_EINVAL (see mase_analyze_error). */
int mase_analyze(const mase_network *net, const mase_partition *part, mase_info *info);

/* Host-only consistency check of the symbolic setup: random gain terms are
 * scattered through the slot maps as the device accumulation does and the
 * supernodal schedule is run serially in FP64.  errors4 receives the maximum
 * relative errors {slot maps vs dense assembly, Schur blocks vs dense Schur
 * complements (Eq. schur_defs), area solves vs dense solves, boundary solve
 * vs dense solve}.  Returns MASE_EINVAL on a structural inconsistency. */
int mase_selfcheck(const mase_network *net, const mase_partition *part, uint64_t seed,
                   double *errors4);

/* Message of the last mase_analyze / mase_selfcheck failure on this thread. */
const char *mase_analyze_error(void);

/* Host-only: sizeof of mase_options, mase_stats, mase_info and
 * mase_warmstart_options as compiled into the library, so that bindings in
 * other languages can check their copies of these structs. */
void mase_abi_sizes(int64_t *sizes4);

/* Coordinator step without device allocation.  The paper has no counterpart:
 * this entry point serves callers that cannot call cudaMalloc when they need
 * the step - a host program whose device memory belongs to another allocator
 * (a framework's caching pool, or one pool carved out at start-up) that allows
 * no raw allocations beside it, or a latency-bound loop that must not take the
 * device-wide synchronisation cudaMalloc and cudaFree can imply.  Given the
 * condensed blocks of every area and snapshot it assembles S_Gamma and
 * b_hat_Gamma, factors, refines (MASE_MIXED handles) and solves, like the
 * coordinator inside mase_solve, and writes the boundary step.  It calls no
 * cudaMalloc, cudaFree or allocating library routine: its scratch (boundary
 * factor storage, the assembled copy used by the refinement, index tables and
 * per-snapshot status words) is one static device array of 64 MiB that every
 * GPU which loads the library holds until the process exits; requests needing
 * more return MASE_EINVAL with the required size in mase_last_error().  The
 * first call on a device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current.  All calls share the array
 * and it keeps the last call's contents: calls that overlap on the GPU (two
 * handles or threads at once) race.  Everything the step reads is rewritten by
 * each call.  The call returns after the step is complete.
 *
 * S_blocks (device, FP64, n_S elements): for area k = 0..K-1, then snapshot
 *   s = 0..S-1, the packed lower triangle (column-major: column c holds rows
 *   c..nb-1) of S_b^k(s), nb = nb(k) local boundary unknowns ordered by
 *   ascending bus id over the area's own boundary buses and the far terminals
 *   of its tie lines, Vm then Va per bus, the slack angle omitted.
 *   n_S must equal S * mase_info.coord_S_elems.
 * b_blocks (device, FP64, n_b elements): for k, then s, b_hat_b^k(s) [nb(k)]
 *   in that order; n_b must equal S * mase_info.coord_b_elems.
 * dx_gamma (device, FP64, n_dx = S * n_gamma elements) [S][n_gamma]: x_Gamma
 *   order = ascending boundary bus id, Vm then Va per bus, slack angle omitted.
 * Returns MASE_OK, MASE_EINVAL (null/host pointers, element counts that differ
 * from the handle's, size above the maximum), MASE_EUNOBSERVABLE (non-positive
 * pivot), MASE_ENONFINITE or MASE_EDEVICE. */
int mase_coordinator_noalloc(mase_handle *h, const double *S_blocks, int64_t n_S,
                             const double *b_blocks, int64_t n_b, double *dx_gamma, int64_t n_dx);

/* ---- learned warm start (not in the paper) ----------------------------------
 * One MLP per area maps the area's own measurement rows (normalised) to the
 * (Vm, Va) of its own buses: Linear -> GELU -> Linear -> GELU -> Linear -> GELU
 * -> Linear, hidden width `hidden`, GELU in its erf form.  Weights and
 * activations are BF16 with FP32 accumulation on the tensor cores; master
 * weights and AdamW moments are FP32.  With MASE_START_LEARNED, mase_solve
 * keeps the proposal per snapshot only where its objective J is below the
 * flat start's, so Gauss-Newton has the last word on the proposal. */
typedef struct {
    int32_t  hidden;        /* width of the three hidden layers, a multiple of 8 in
                               8..8192 (512)                                           */
    int32_t  epochs;        /* passes over the training set                            */
    int32_t  batch;         /* samples per AdamW step, multiple of 8                   */
    float    lr;            /* peak learning rate (cosine decay to 5 %)                 */
    float    weight_decay;  /* decoupled weight decay                                   */
    uint64_t seed;          /* weight initialisation and shuffling                      */
} mase_warmstart_options;

void mase_warmstart_default_options(mase_warmstart_options *opt);

/* Train the per-area networks on n samples: z[n][m] measurements (canonical
 * order) and x[n][2N] states the estimator produced for them; both host or
 * both device pointers.  mask[n][m] (1 = present, canonical order, the same
 * memory kind as z; NULL = every row present) marks rows absent from a
 * sample: an absent row enters neither the normalisation moments nor the
 * sample's features (it reads as the row's mean, as at inference), and the
 * magnitude skip of an absent voltage row falls back to that mean, so that
 * networks trained on masked samples see what they will see under the same
 * kind of drops.  final_loss (may be NULL) receives the mean normalised MSE
 * per area over the last epoch.  Replaces any earlier model.  MASE_EINVAL for
 * bad sizes or options, or for pointers of mixed memory kinds. */
int mase_warmstart_train(mase_handle *h, const double *z, const uint8_t *mask, const double *x,
                         int32_t n, const mase_warmstart_options *opt, double *final_loss);

/* The networks' proposal x_out[n_snap][2N] for the handle's current
 * measurements (slack angle 0), without Gauss-Newton.  x_out host or device.
 * MASE_ENOTREADY without a model or measurements, MASE_EINVAL for NULL
 * arguments, MASE_EDEVICE. */
int mase_warmstart_predict(mase_handle *h, double *x_out);

/* Save / load the trained networks (weights and normalisation) to a file; a
 * loaded file must match the handle's network and partition.  MASE_EINVAL for
 * NULL arguments, a file that cannot be opened, is not a warm-start file or
 * does not match; save returns MASE_ENOTREADY without a model. */
int mase_warmstart_save(const mase_handle *h, const char *path);
int mase_warmstart_load(mase_handle *h, const char *path);

/* One forward and backward pass of a single network with the training
 * kernels, for checking gradients: dims[5] = {d_in, H, H, H, d_out}
 * (n_layers = 4, H a multiple of 8); params packs W_l[out][in] then b_l for
 * l = 1..4 (FP32, host); X[batch][d_in], T[batch][d_out] (host).  loss gets
 * mean((Y - T)^2); grads has the layout of params.  MASE_EINVAL unless
 * n_layers = 4, batch >= 1 and the hidden widths are equal multiples of 8;
 * MASE_EDEVICE (including a tensor-core wait that ran out). */
int mase_mlp_check(const int32_t *dims, int32_t n_layers, int32_t batch, const float *params,
                   const float *X, const float *T, float *loss, float *grads);

/* The optimiser of the warm-start training on its own, for checking: the
 * library's AdamW kernel run `steps` times over n FP32 parameters w (host,
 * updated in place) with the gradients grads[steps][n] and learning rates
 * lr[steps] (host).  Moments start at zero; beta1 = 0.9, beta2 = 0.999,
 * eps = 1e-8 as in training; per step t: m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, w <- w (1 - lr wd) - lr (m / (1-b1^t)) /
 * (sqrt(v / (1-b2^t)) + eps).  m_out, v_out (FP32) and w_bf16_out (the BF16
 * copy the networks compute with, as raw bits) may be NULL.  MASE_EINVAL for
 * n < 1, steps < 1 or NULL lr, grads or w; MASE_EDEVICE. */
int mase_adamw_check(int64_t n, int32_t steps, const float *lr, float weight_decay,
                     const float *grads, float *w, float *m_out, float *v_out,
                     uint16_t *w_bf16_out);

/* Free the handle and every device buffer it owns (NULL is a no-op). */
void mase_destroy(mase_handle *h);
/* Name of a status code ("MASE_OK", "MASE_EINVAL", ...; "MASE_UNKNOWN" for
 * any other value); static storage. */
const char *mase_status_str(int code);
/* Message of the last failure on this thread of a call other than
 * mase_analyze and mase_selfcheck (those use mase_analyze_error); thread-local
 * storage, valid until the next failing call on the thread. */
const char *mase_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MASE_H */
