/*
 * fd_gb300.h -- C ABI of the GB300 forward-dynamics library.
 *
 * Forward dynamics qdd = FD(q, qdot, tau) of serial chains of revolute joints by
 * the three factorisations of M(q)^{-1} compared in Yang, Wu & Pan (arXiv
 * 1609.06779): ABIA (Section II-C), JSIIA (Section II-C) and CFA (Section III,
 * Algorithm 1, with the block tri-diagonal system solved by odd-even elimination,
 * Section IV, Algorithm 2). Every algorithm first computes the bias torque by
 * inverse dynamics (Eq. 2a-2d with qdd = 0, Eq. 4) and works on
 * tau_delta = tau - tau_bias.
 *
 * Conventions (fixed by this library; the paper leaves them open):
 *   twist V = (omega; v), wrench F = (n; f), both in the link's own frame;
 *   joint i joins link i-1 to link i (link 0 of a chain is attached to the fixed
 *   base): g_{i-1,i}(q_i) = (R0_i, p0_i) * exp([a_i; 0] q_i), S_i = (a_i; 0);
 *   gravity enters as the base acceleration (0; -g), g given in the base frame;
 *   no external wrench at the tip.
 *
 * Memory: arrays documented as "host" are read during the call and not retained.
 * Arrays documented as "device" must be device memory of the chain set's device.
 * Solves are asynchronous on the given CUDA stream (NULL = legacy default stream).
 * Errors: every call returns an fd_status; fd_last_error() returns a message
 * for the calling thread's last failing call. Arguments are validated before any
 * launch; numerical failures of a problem (a non-positive pivot, a non-finite
 * result) are written to the optional per-problem status array on the device.
 * There is no CPU fallback: without a usable CUDA device calls that need one
 * return FD_ERR_CUDA.
 */
#ifndef FD_GB300_H
#define FD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FD_ABI_VERSION 1

typedef struct fd_chain_s *fd_chain_t; /* a set of serial chains resident on one GPU */
typedef struct fd_batch_s *fd_batch_t; /* a batch plan: which chain each problem uses */

typedef enum fd_algo {
  FD_ABIA = 0,  /* articulated-body inertia factorisation (Section II-C) */
  FD_JSIIA = 1, /* joint-space inertia by ID columns + Cholesky (Section II-C) */
  FD_CFA = 2,   /* constraint force algorithm with OEE (Section III, Alg. 1-2) */
  FD_CFA_CR = 3, /* CFA with the block tri-diagonal system solved by block cyclic
                    reduction instead of OEE: about n row updates instead of
                    n ceil(log2 n), the same result (not in the paper's
                    experiments; the reduction OEE is a variant of, Section IV) */
  FD_CFA_HYBRID = 4, /* CFA with the hybrid partition / cyclic-reduction solve:
                       each lane eliminates the interior rows of its own run of
                       rows, block cyclic reduction solves the reduced system of
                       the runs' end rows across the lanes, each lane back-
                       substitutes its interior (not in the paper's experiments;
                       a partitioned form of the reductions of Section IV) */
  FD_ABIA_SCAN = 5 /* ABIA with the articulated-inertia recursion as a parallel
                      scan over the team's lanes (Section III holds the ABI
                      recursion to be serial up to a constant factor; this is
                      its associative form: the Riccati step on the constraint-
                      space compliance composes as a Schur complement of an SPD
                      block matrix). FP64 only, teams of 8 .. 256 lanes (no
                      split by length class); every lane does about five times
                      the serial work in n / team + log2 team steps */
} fd_algo;

#define FD_N_ALGOS 6

typedef enum fd_prec {
  FD_FP64 = 0,  /* states and all arithmetic in double */
  FD_FP32 = 1,  /* states and all arithmetic in float */
  FD_MIXED = 2  /* float states, joint transforms and inverse dynamics (the bias
                   torque); in double: CFA's blocks of A, R = -B tau_delta, the OEE
                   elimination and CalcAcc (from the double model copy), the
                   articulated-inertia recursion and the JSIIA Cholesky */
} fd_prec;

typedef enum fd_status {
  FD_OK = 0,
  FD_ERR_INVALID_ARG = 1, /* bad pointer, size, shape or model (nothing launched) */
  FD_ERR_NOT_SPD = 2,     /* a pivot that must be positive was not */
  FD_ERR_OOM = 3,         /* device allocation failed */
  FD_ERR_CUDA = 4,        /* a CUDA runtime call failed or no device */
  FD_ERR_TIMEOUT = 5,     /* a bounded wait ran out */
  FD_ERR_NUMERIC = 6,     /* a non-finite result */
  FD_ERR_BUSY = 7,        /* the request cannot be admitted now; retry */
  FD_ERR_UNSUPPORTED = 8  /* combination of options not built */
} fd_status;

/* Message of the calling thread's last failing call ("" if none). The pointer
 * stays valid until the next call on this thread. */
const char *fd_last_error(void);

/* FD_ABI_VERSION of the loaded library. */
int32_t fd_abi_version(void);

/*
 * fd_create_chain -- copy a set of chains to the device.
 *
 * The problem statement of Algorithm 1 (inputs tau, q, qdot; model J_i and the
 * joints' twists and frames). Chain k owns links link_offsets[k] ..
 * link_offsets[k+1]-1 of the packed host arrays:
 *   joint_axes       [L][3]  joint axis a_i in child frame i (normalised here;
 *                            a zero axis is FD_ERR_INVALID_ARG)
 *   link_frames      [L][12] home transform parent -> child: R row-major (9),
 *                            then p (3); R must be a rotation (|R^T R - I| < 1e-9)
 *   spatial_inertias [L][36] 6x6 spatial inertia J_i of link i at the origin of
 *                            frame i, (omega; v) order; symmetric positive
 *                            definite (Eq. 1), else FD_ERR_INVALID_ARG
 *   gravity          [3]     gravity vector in the base frame (e.g. 0, 0, -9.81)
 * n_chains >= 0; link_offsets [n_chains+1] non-decreasing from 0; a chain may
 * have zero links. All arrays are host memory and are not retained. The model is
 * re-expressed in link frames whose x axis is the joint axis (q-independent;
 * qdd does not depend on the choice of link frames) and stored in double and
 * float copies on `device`. Ownership of *out passes to the caller; free it
 * with fd_destroy_chain.
 */
fd_status fd_create_chain(int32_t n_chains, const int64_t *link_offsets,
                          const double *joint_axes, const double *link_frames,
                          const double *spatial_inertias, const double gravity[3],
                          int32_t device, fd_chain_t *out);

/*
 * fd_create_tree -- copy a set of kinematic trees (branched robots) to the
 * device (not in the paper, whose algorithms are stated for serial chains; its
 * future work names branched robots). Arrays as for fd_create_chain, plus
 * parents [L] (host): the parent of each link within its tree, -1 for a link
 * attached to the fixed base, else a link of the same tree with a smaller index
 * (0-based within the tree; a tree's links are numbered parents first, so a
 * tree may hold several branches and several links on the base). link_frames[i]
 * is the home transform from the parent's frame (or the base's) to link i's.
 * Otherwise FD_ERR_INVALID_ARG. A set of trees solves with FD_ABIA, FD_JSIIA
 * (fd_solve_batch, FD_FP64 or FD_FP32, one thread per tree: team 0 or 1) and
 * fd_inverse_dynamics; CFA, the ABI scan, the adjoint, the projected and static
 * solves return FD_ERR_UNSUPPORTED (CFA's system of Eq. cfa-eq2 is block
 * tri-diagonal only on a serial chain). parents[i] = i - 1 within every tree
 * gives the same model as fd_create_chain. Free it with fd_destroy_chain.
 */
fd_status fd_create_tree(int32_t n_trees, const int64_t *link_offsets, const int32_t *parents,
                         const double *joint_axes, const double *link_frames,
                         const double *spatial_inertias, const double gravity[3],
                         int32_t device, fd_chain_t *out);

/*
 * fd_tree_add_loops -- close a set of kinematic trees by revolute loop joints
 * (looped robots; not in the paper). Loop k joins a joint frame on link
 * link_a[k] (-1: the base) and one on link link_b[k] of tree loop_tree[k] (link
 * indices within the tree), turning about the frames' x axes: frame_a[k],
 * frame_b[k] [12] (host) are the frames' poses in those links' frames (R
 * row-major, then p) as given to fd_create_tree. The relative twist of the two
 * frames may only turn about x, so each loop adds five constraints G qd = 0;
 * forward dynamics then solves M qdd + G^T lam = tau - bias, G qdd = -gamma
 * (gamma the constraint's velocity product) with JSIIA's factor of M. At most
 * four loops a tree, whose constraints must be independent (else that problem's
 * status is FD_ERR_NOT_SPD); once per set, before or after fd_batch_create. A
 * set with loops solves with FD_JSIIA in FD_FP64 only; other algorithms and
 * fd_inverse_dynamics return FD_ERR_UNSUPPORTED. FD_ERR_INVALID_ARG for a set
 * of chains, bad indices, frames that are not rotations, or too many loops.
 */
fd_status fd_tree_add_loops(fd_chain_t chain, int32_t n_loops, const int32_t *loop_tree,
                            const int32_t *link_a, const int32_t *link_b, const double *frame_a,
                            const double *frame_b);

fd_status fd_destroy_chain(fd_chain_t chain);

/* Number of chains, total links and the longest chain's link count. */
fd_status fd_chain_info(fd_chain_t chain, int32_t *n_chains, int64_t *n_links,
                        int32_t *max_links);

/*
 * fd_batch_create -- plan a batch of n_problems forward-dynamics problems.
 *
 * Problem p uses chain chain_index[p] of `chain` (host array, may be NULL: then
 * n_problems must equal the number of chains and problem p uses chain p). The
 * problems' joint states are packed in problem order: problem p occupies
 * entries state_offset(p) .. state_offset(p) + n_p - 1 of every state array,
 * where state_offset is the prefix sum of the problems' link counts. The plan
 * holds device copies of this map and is reusable for any number of solves.
 */
fd_status fd_batch_create(fd_chain_t chain, int32_t n_problems, const int32_t *chain_index,
                          fd_batch_t *out);

/* Frees a batch plan. Allowed before or after fd_destroy_chain of its chain set;
 * solving with a plan whose chain set was destroyed is an error the library
 * cannot detect. */
fd_status fd_batch_destroy(fd_batch_t batch);

/* Total state entries (sum of the problems' link counts) of a batch. */
fd_status fd_batch_info(fd_batch_t batch, int32_t *n_problems, int64_t *n_state_links,
                        int32_t *max_links);

/*
 * Threads that cooperate on one problem ("team"): 0 lets the library choose
 * (the autotuned size if fd_autotune ran for this batch, algorithm and
 * precision, else a size that fills the GPU; for a batch whose chains fall
 * into several length classes -- ceil(log2 n) differs -- one launch whose grid
 * is split by class, each class with its own team of 1 .. 128 lanes: its
 * autotuned one, else the size that fills the GPU with that class alone;
 * see fd_batch_classes); otherwise a power of two from 1
 * (one thread per chain: serial recursions) through 32 (one warp per chain:
 * warp-shuffle scans and OEE levels across lanes) to 256 (one block per chain:
 * scans across warps through shared memory). FD_ABIA keeps its articulated-
 * inertia recursion serial over the links (the paper notes it cannot be
 * parallelised beyond a constant factor, Section III) and takes that constant
 * factor: team 1 runs one thread per problem, teams 8, 16 and 32 spread each
 * step's 6x6 update over six (team 8) or twelve lanes and run inverse dynamics
 * on component lanes (chains of up to 64 links) or as a scan; other sizes
 * return FD_ERR_UNSUPPORTED.
 */

/* Bytes of device workspace fd_solve_batch / fd_inverse_dynamics need for
 * (algo, prec, team). For fd_inverse_dynamics pass algo = -1. */
size_t fd_workspace_size(fd_batch_t batch, int32_t algo, fd_prec prec, int32_t team);

/*
 * fd_solve_batch -- qdd = FD(q, qdot, tau) for every problem of the batch.
 *
 * q, qdot, tau (inputs) and qddot (output) are device arrays of n_state_links
 * elements, double for FD_FP64 and float for FD_FP32 / FD_MIXED, packed as
 * fd_batch_create describes. workspace: device memory of at least
 * fd_workspace_size(batch, algo, prec, team) bytes, 256-byte aligned, owned by
 * the caller, contents need not be initialised and are garbage afterwards; it
 * must not be shared by solves that overlap on the GPU. status: optional device
 * int32 array [n_problems] receiving FD_OK, FD_ERR_NOT_SPD or FD_ERR_NUMERIC per
 * problem (valid once the stream reaches that point). Enqueues work on `stream`
 * (a cudaStream_t) and returns without synchronising. No device memory is
 * allocated by this call.
 */
fd_status fd_solve_batch(fd_batch_t batch, const void *q, const void *qdot, const void *tau,
                         void *qddot, fd_algo algo, fd_prec prec, int32_t team,
                         void *workspace, size_t workspace_bytes, int32_t *status,
                         void *stream);

/*
 * fd_inverse_dynamics -- tau = ID(q, qdot, qddot) with gravity (Eq. 2a-2d): the
 * twist and acceleration recursions (forward, block bi-diagonal) and the force
 * recursion (backward, transposed), each solved as a segmented prefix scan over
 * composed SE(3)-affine operators (Section II-B). Arrays and workspace as for
 * fd_solve_batch (workspace size: fd_workspace_size(batch, -1, prec, team));
 * prec FD_MIXED is treated as FD_FP32.
 */
fd_status fd_inverse_dynamics(fd_batch_t batch, const void *q, const void *qdot,
                              const void *qddot, void *tau, fd_prec prec, int32_t team,
                              void *workspace, size_t workspace_bytes, void *stream);

/*
 * General projections W for CFA (not in the paper's experiments: its conclusion
 * leaves the choice of the projection W of Eq. cfa-eq1 open, as a trade of speed
 * against accuracy). Any W_i (6x5, W_i^T S_i = 0, rank 5) is Wc_i Q_i with Wc_i
 * the library's own complement (e_2 .. e_6 of the link frame whose x axis is the
 * joint axis) and Q_i an invertible 5x5 matrix. The system of Eq. cfa-eq2 then
 * becomes A' = Q^T A Q, R' = Q^T R with Q = diag(Q_i), its solution
 * F_c' = Q^{-1} F_c, and qdd is the same up to rounding: only the numbers the
 * odd-even elimination works on change.
 */
typedef enum fd_projection {
  FD_PROJ_CANONICAL = 0,   /* Q_i = I: the blocks fd_solve_batch's CFA solves */
  FD_PROJ_GIVEN = 1,       /* Q_i given per link (fd_projection_to_canonical) */
  FD_PROJ_BLOCK_JACOBI = 2 /* Q_i = L_i^{-T} with D_i = L_i L_i^T: every diagonal
                              block of A' is the identity (state-dependent) */
} fd_projection;

/*
 * fd_projection_to_canonical -- Q_i of given projections W_i. Host only.
 *
 * joint_axes [n_links][3] as given to fd_create_chain; W [n_links][6][5]
 * row-major, W_i in link i's frame and (omega; v) order as for fd_create_chain;
 * Q [n_links][5][5] row-major receives Q_i. FD_ERR_INVALID_ARG for a NULL
 * array, n_links < 0, a zero axis, |S_i^T W_i| above 1e-9 max|W_i|, or a W_i
 * whose Q_i is singular to working precision (|det Q_i| at most 1e-12 times the
 * product of its column norms).
 */
fd_status fd_projection_to_canonical(int64_t n_links, const double *joint_axes, const double *W,
                                     double *Q);

/*
 * fd_solve_cfa_projected -- CFA (Algorithm 1 with odd-even elimination,
 * Algorithm 2) on the system of the projection `proj`.
 *
 * Arrays, workspace (fd_workspace_size of FD_CFA), status and stream as for
 * fd_solve_batch. prec: FD_FP64 or FD_FP32 (FD_MIXED: FD_ERR_UNSUPPORTED).
 * team: as for fd_solve_batch, except that team 0 takes one team for the whole
 * batch (the autotuned CFA team of a one-class batch, else the default that
 * fills the GPU; no split by length class). Q: device array [L][25] of double
 * indexed by the chain set's link (link_offsets of fd_create_chain), Q_i
 * row-major, required for FD_PROJ_GIVEN (else ignored, may be NULL); not
 * retained after the solve completes. FD_PROJ_CANONICAL runs fd_solve_batch's
 * FD_CFA kernel (bit for bit its result at the same team). In FP32 the solve
 * keeps fd_solve_batch's refinement passes, each with its own projection.
 */
fd_status fd_solve_cfa_projected(fd_batch_t batch, const void *q, const void *qdot,
                                 const void *tau, void *qddot, fd_prec prec, int32_t team,
                                 fd_projection proj, const double *Q, void *workspace,
                                 size_t workspace_bytes, int32_t *status, void *stream);

/*
 * fd_autotune -- pick the team size for (batch, algo, prec) by timing.
 *
 * The paper leaves the parallel schedule to the implementation. For a batch of
 * one length class this times every team size (1 .. 256, at most the longest
 * chain rounded up to a power of two; ABIA: 1, 8, 16, 32) whose workspace fits
 * in workspace_bytes, one warm-up and two timed solves each with CUDA events on
 * `stream`, and records the fastest in the batch plan. For a batch of several
 * length classes it does the same per class (teams up to 128), each class
 * launched alone, then refines the choice inside the whole launch (each class
 * in turn, longest first, tries its other teams with the others fixed and
 * keeps one that makes the whole launch at least 1% faster), and records one
 * team per class; *best_team (may be NULL) then receives 0. Later calls with team 0 use the recorded teams. Choices are
 * also kept in a process-wide cache keyed by GPU, algorithm, precision, length
 * class and ceil(log2) of the problem count; a cached entry is used without
 * timing (fd_autotune_cache_load / _save persist it; refined choices are kept
 * under a key of the whole batch's classes as well). Synchronises the stream.
 * Inputs as fd_solve_batch (qddot is overwritten).
 */
fd_status fd_autotune(fd_batch_t batch, fd_algo algo, fd_prec prec, const void *q,
                      const void *qdot, const void *tau, void *qddot, void *workspace,
                      size_t workspace_bytes, void *stream, int32_t *best_team);

/*
 * fd_batch_classes -- the length classes of a batch (not in the paper: the
 * schedule of a team-0 solve). Problems whose chains share ceil(log2 n) form a
 * class (n <= 1: one class); *n_classes receives their number, and for the
 * first min(max, *n_classes) classes, longest first, the shortest and longest
 * chain, the problem count and the team a team-0 solve of (algo, prec) gives
 * the class (algo -1: fd_inverse_dynamics). Output arrays are host memory and
 * may be NULL.
 */
fd_status fd_batch_classes(fd_batch_t batch, int32_t algo, fd_prec prec, int32_t max,
                           int32_t *n_classes, int32_t *min_len, int32_t *max_len,
                           int32_t *count, int32_t *team);

/*
 * The autotune cache (see fd_autotune): load merges the JSON file at `path`
 * into the process-wide cache (a missing file loads nothing; a malformed one is
 * FD_ERR_INVALID_ARG) and sets *n_loaded (may be NULL); save writes the whole
 * cache to `path` (through a temporary file renamed into place); clear empties
 * it. Host only; thread safe.
 */
fd_status fd_autotune_cache_load(const char *path, int32_t *n_loaded);
fd_status fd_autotune_cache_save(const char *path);
fd_status fd_autotune_cache_clear(void);

/*
 * fd_solve_adjoint -- reverse-mode derivatives of qdd = FD(q, qdot, tau).
 *
 * Not in the paper; it follows from ID(q, qdot, FD(q, qdot, tau)) = tau
 * (Eq. 2a-2d, Eq. 4): with lambda = M^{-1} qddot_bar, solved by the algorithm's
 * own factorisation of M^{-1} (ABIA, JSIIA or CFA),
 *   tau_bar  = lambda,
 *   q_bar    = -(d ID/d q)^T lambda,   qdot_bar = -(d ID/d qdot)^T lambda,
 *   mass_bar = -(d ID/d m)^T lambda    (link masses, centre of mass and
 *                                       rotational inertia about it held fixed),
 * with (d ID/d x)^T lambda computed by a reverse sweep of the inverse-dynamics
 * recursions (three forward and three backward segmented scans).
 * Inputs (device, n_state_links elements, dtype as fd_solve_batch): q, qdot,
 * tau, qddot (the forward result; may be NULL, then it is recomputed) and
 * qddot_bar. Outputs: q_bar, qdot_bar, tau_bar and mass_bar (may be NULL; needs
 * rigid-body inertias, else FD_ERR_UNSUPPORTED). workspace: at least
 * fd_adjoint_workspace_size(batch, algo, prec, team) bytes, 256-byte aligned.
 * status as for fd_solve_batch (for the solve with M). Asynchronous on stream.
 */
size_t fd_adjoint_workspace_size(fd_batch_t batch, fd_algo algo, fd_prec prec, int32_t team);

fd_status fd_solve_adjoint(fd_batch_t batch, const void *q, const void *qdot, const void *tau,
                           const void *qddot, const void *qddot_bar, void *q_bar,
                           void *qdot_bar, void *tau_bar, void *mass_bar, fd_algo algo,
                           fd_prec prec, int32_t team, void *workspace, size_t workspace_bytes,
                           int32_t *status, void *stream);

/*
 * fd_solve_cfa_static -- CFA forward dynamics that allocates nothing.
 *
 * The paper has no counterpart: this is a deployment variant of fd_solve_batch
 * with algo = FD_CFA. It is for callers that cannot call cudaMalloc (or any
 * allocating routine) when they solve: a control loop with a hard deadline, a
 * host callback or a framework that owns all device memory and forbids raw
 * allocations. Instead of a caller workspace it uses a scratch array of 32 MiB
 * compiled into the library as a file-scope device variable; every GPU that
 * loads the library holds that array until the process exits.
 *
 * Problem p is chain p of `chain` (no batch plan); q, qdot, tau (inputs) and
 * qddot (output) are device arrays of the chain set's total link count, packed
 * in chain order, double for FD_FP64 and float for FD_FP32 / FD_MIXED. team: a
 * power of two from 1 to 256, as for fd_solve_batch, or 0: one team for all
 * chains, the largest power of two not above 152 x 2048 / n_chains, capped at
 * the longest chain rounded up to a power of two (no split by length class);
 * the result equals fd_solve_batch's at the same team bit for bit. status as for
 * fd_solve_batch. Limit: the CFA workspace of all links must fit in 32 MiB
 * (FD_FP64: 1 824 bytes per link, about 18 000 links; FD_MIXED about 19 000;
 * FD_FP32 about 36 000); larger sets return FD_ERR_INVALID_ARG with the sizes
 * in fd_last_error().
 *
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (host side only; nothing is copied to the device); make
 * that first call before any stream capture. Every call shares the one array
 * and leaves its contents behind; nothing in it has to start at zero, but calls
 * whose kernels overlap on the GPU (other streams, other host threads) race on
 * it and must be serialised by the caller.
 */
fd_status fd_solve_cfa_static(fd_chain_t chain, const void *q, const void *qdot,
                              const void *tau, void *qddot, fd_prec prec, int32_t team,
                              int32_t *status, void *stream);

/*
 * fd_measure_fp64_peak -- the FP64 rate this GPU sustains (not in the paper: the
 * denominator of the FP64 kernels' roofline, which the FP64 pipe bounds). Runs
 * independent fused multiply-adds, eight chains per thread, four 128-thread
 * blocks per SM, `iters` steps per chain (about 2e5 take a few hundred
 * milliseconds on a GB300), timed with CUDA events on a stream of its own after
 * a shorter warm-up; *tflops receives 2 x FMAs / time in TFLOP/s and
 * *elapsed_ms (may be NULL) the timed kernel's duration. Synchronous.
 */
fd_status fd_measure_fp64_peak(int32_t device, int32_t iters, double *tflops,
                               double *elapsed_ms);

/* ------------------------------------------------------------------ serving
 *
 * A server owns one device allocation of mem_budget_bytes (its memory budget)
 * and a worker thread. Chain models are registered once and stay resident.
 * Requests name a model and carry their state; they are admitted in arrival
 * order as link slots and memory free up, and every tick the worker runs the
 * forward dynamics of all admitted requests, one launch per algorithm and length
 * class ("continuous batching": requests arriving while others are on the GPU
 * join the next tick), the adjoint over new FD+gradient requests, and the
 * rollouts' integration steps (one per tick for the longest chains, several for
 * shorter ones, by length class). Not in the paper (its experiments solve fixed
 * groups); built on the same kernels as fd_solve_batch and fd_solve_adjoint,
 * FP64 only, with teams and steps per tick set by a request's algorithm and
 * chain length alone, so its arithmetic does not depend on the mix.
 */
typedef struct fd_server_s *fd_server_t;

typedef enum fd_request_kind {
  FD_REQ_FD_GRAD = 0, /* qdd = FD(q, qdot, tau) and its adjoint for qddot_bar */
  FD_REQ_ROLLOUT = 1  /* `steps` semi-implicit Euler steps:
                         qdot += dt FD(q, qdot, tau_k); q += dt qdot */
} fd_request_kind;

#define FD_SERVE_PER_SIZE 1 /* flag: one launch per distinct chain length (the
                               static per-size batching baseline) */

typedef struct fd_request {
  int32_t kind;     /* fd_request_kind */
  int32_t algo;     /* FD_ABIA or FD_CFA */
  int32_t model_id; /* from fd_serve_add_model */
  int32_t steps;    /* FD_REQ_ROLLOUT: >= 1 */
  double dt;        /* FD_REQ_ROLLOUT: > 0 */
  const double *q;         /* host [n] initial joint positions */
  const double *qdot;      /* host [n] initial joint velocities */
  const double *tau;       /* host: [n] (FD_GRAD) or [steps][n] torques per step */
  const double *qddot_bar; /* host [n], FD_GRAD: cotangent of qdd */
} fd_request;

typedef struct fd_result {
  int32_t status;      /* FD_OK, FD_ERR_NOT_SPD or FD_ERR_NUMERIC */
  int32_t n_links;
  int32_t steps_done;
  int32_t pad;
  double submit_time;  /* fd_serve_clock() seconds */
  double done_time;    /* when the result reached host memory */
  /* caller buffers of n_links doubles, each may be NULL */
  double *q, *qdot;    /* ROLLOUT: final state */
  double *qddot;       /* FD_GRAD: qdd; ROLLOUT: qdd of the last step */
  double *q_bar, *qdot_bar, *tau_bar; /* FD_GRAD: the adjoint */
} fd_result;

typedef struct fd_serve_stats_t {
  uint64_t ticks, launches, completed, queued, active;
  int64_t link_slots_used, link_slots;
  double link_solves;  /* sum over ticks of the links of the requests solved */
  double busy_seconds; /* worker time spent in ticks */
} fd_serve_stats_t;

/* Monotonic clock (seconds) of the server's timestamps (CLOCK_MONOTONIC). */
double fd_serve_clock(void);

/* Creates a server on `device`: allocates mem_budget_bytes (>= 16 MiB) once and
 * starts the worker. gravity in the base frame. flags: 0 or FD_SERVE_PER_SIZE. */
fd_status fd_serve_create(int32_t device, size_t mem_budget_bytes, const double gravity[3],
                          int32_t flags, fd_server_t *out);

/* Registers a chain model (host arrays as fd_create_chain, one chain of
 * n_links links); it stays resident until fd_serve_remove_model. FD_ERR_OOM if
 * the model region of the budget is full. */
fd_status fd_serve_add_model(fd_server_t server, int32_t n_links, const double *joint_axes,
                             const double *link_frames, const double *spatial_inertias,
                             int32_t *model_id);

/* FD_ERR_BUSY while requests that use the model are pending. */
fd_status fd_serve_remove_model(fd_server_t server, int32_t model_id);

/* Queues a request (its host arrays are copied); *ticket identifies it.
 * FD_ERR_INVALID_ARG if it can never fit the budget, FD_ERR_BUSY if the queue
 * is full (retry later). */
fd_status fd_serve_submit(fd_server_t server, const fd_request *request, uint64_t *ticket);

/* FD_OK and the result (ticket released) if done; FD_ERR_BUSY if not yet. */
fd_status fd_serve_poll(fd_server_t server, uint64_t ticket, fd_result *out);

/* As fd_serve_poll, but waits at most timeout_ms; FD_ERR_TIMEOUT if not done. */
fd_status fd_serve_wait(fd_server_t server, uint64_t ticket, int32_t timeout_ms,
                        fd_result *out);

/* Releases up to `max` finished requests without copying their states:
 * tickets, submit and completion times and statuses (submit_times, statuses may
 * be NULL); *count receives how many. For load generators. */
fd_status fd_serve_drain(fd_server_t server, int32_t max, uint64_t *tickets,
                         double *submit_times, double *done_times, int32_t *statuses,
                         int32_t *count);

fd_status fd_serve_stats(fd_server_t server, fd_serve_stats_t *out);

/* Stops the worker (pending requests are dropped) and frees everything. */
fd_status fd_serve_destroy(fd_server_t server);

#ifdef __cplusplus
}
#endif

#endif /* FD_GB300_H */
