/*
 * otm.h -- C ABI of the GB300 explicit OTM material-point update.
 *
 * One explicit step of the Optimal Transportation Meshfree method (Kumar et al., "Parallel
 * multiphysics simulation for the stabilized OTM method", arXiv 2206.08772, Algorithm 1):
 *   1. lumped nodal mass and internal force           (Eq. 5, optional stabilisation Eq. 7-8)
 *   2. central-difference nodal update + contact       (Eq. 4, Eq. 6; Sec. 4.1 wall, Sec. 4.2 tool)
 *   3. material-point position, F, volume              (Eq. 9-13)
 *   4. J2 / Johnson-Cook thermo-plastic return map     (Sec. 4.1, Sec. 4.2)
 *   5. linked-cell support search                      (Algorithm 3)
 *   6. local max-ent shape functions and gradients     (Eq. 14, Newton for lambda)
 * all on one GPU in hand-written sm_103a kernels.
 *
 * Conventions
 *  - Every call returns OTM_OK (0) or a negative OTM_ERR_* code; nothing aborts the process.
 *  - Units are SI. Vectors are xyz triples. Symmetric tensors are 6-vectors in the order
 *    (xx, yy, zz, xy, yz, xz). Full tensors are row-major 3x3 (F[3*i+j] = F_ij).
 *  - Device memory: the library never allocates device memory. The caller passes one device
 *    workspace (size from otm_workspace_bytes) that must stay valid until otm_destroy; all
 *    state lives in it. The handle itself is a small host object.
 *  - Host memory: otm_init reads the caller's host arrays (copied to the workspace before it
 *    returns); otm_state copies into caller-owned host memory.
 *  - Streams: all work is enqueued on the stream given to otm_init (a cudaStream_t passed as
 *    void*; NULL = legacy default stream). Only otm_init, otm_step, otm_state and
 *    otm_error_detail synchronise that stream.
 *  - Fields come back in ascending ID order (erosion removes entries, never reorders them).
 *  - After an error the state is that of the failing step, partially updated (the oracle
 *    behaves the same way); otm_error_detail names the code and the smallest offending ID.
 *    otm_keep_last_good makes otm_step leave the state at the last good step instead.
 *  - Device reset: the library keeps two pieces of module data per device (the table of its
 *    FP64 exponential and the allocation-free search's scratch address), set up by the first
 *    call on that device. A reset of the device or of its primary context (cudaDeviceReset)
 *    discards module data: otm_init checks for that and sets the table up again, so a reset must
 *    be followed by otm_init before the stand-alone kernels are used; the allocation-free search
 *    is not supported after a reset in the same process.
 */
#ifndef OTM_H
#define OTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OTM_OK 0
#define OTM_ERR_ARG (-1)              /* bad argument, size or pointer */
#define OTM_ERR_CUDA (-2)             /* a CUDA runtime call failed */
#define OTM_ERR_WORKSPACE (-3)        /* workspace smaller than otm_workspace_bytes */
#define OTM_ERR_LME_NOCONV (-4)       /* Newton for lambda did not converge (point outside hull) */
#define OTM_ERR_JACOBIAN (-5)         /* det(dF) <= 0 or non-positive elastic stretch */
#define OTM_ERR_NONFINITE (-6)        /* NaN / Inf in positions or stresses */
#define OTM_ERR_RETURNMAP_NOCONV (-7) /* Johnson-Cook consistency iteration failed */
#define OTM_ERR_CAPACITY (-8)         /* support / influence / cell capacity exceeded */

#define OTM_PRECISION_FP64 0          /* every step in FP64 */
#define OTM_PRECISION_MIXED 1         /* FP32 force scatter, node update, pair rows' e = N d and
                                       * kinematics gather (x_p increment and G = sum du (x) N d);
                                       * the LME Newton's Hessian sums in double-float (FP32 pairs,
                                       * ~2^-47); the weights, N, Z, the residual, dF = 1 - G K, F
                                       * and the return map in FP64 */

#define OTM_FLAG_FIXED 1              /* node flag: displacement increment held at zero */

typedef struct otm_material {
    int32_t model;      /* 0: J2 with linear isotropic hardening (Sec. 4.1); 1: Johnson-Cook (Sec. 4.2) */
    int32_t fracture;   /* 1: Johnson-Cook fracture strain checked (erosion when allow_erode) */
    double E, nu, rho0;
    double sigma_y0, H;                 /* J2: initial yield stress, hardening modulus */
    double A, B, n, C, m, eps_dot0;     /* JC flow stress */
    double T_room, T_melt, chi, cp;     /* JC thermal softening, Taylor-Quinney, heat capacity */
    double d1, d2, d3, d4, d5;          /* JC fracture */
} otm_material;

typedef struct otm_params {
    double h;            /* characteristic nodal spacing (beta = gamma / h^2, Sec. 2.3) */
    double beta;         /* LME locality parameter */
    double rs2;          /* squared support radius: node in support iff |x_p - x_a|^2 <= rs2 */
    double cell_size;    /* linked-cell edge, >= sqrt(rs2)/2 (stencil +-2 cells) */
    double dt;           /* time step */
    double T0;           /* initial temperature */
    double newton_tol;   /* Newton stops when |sum N_a (x_p - x_a)| <= newton_tol * h */
    double eps_stab;     /* stabilisation penalty of Eq. 7 (0 = off) */
    int32_t max_newton;  /* Newton iteration limit */
    int32_t n_materials; /* 1..4 */
    int32_t precision;   /* OTM_PRECISION_FP64 or OTM_PRECISION_MIXED */
    int32_t wall;        /* 1: rigid frictionless plane (wall_p, wall_n) */
    int32_t tool;        /* 1: rigid moving cutting tool */
    int32_t allow_erode; /* 1: MPs meeting the fracture criterion are removed */
    double wall_p[3], wall_n[3];
    double tool_x0, tool_tip_y, tool_rake, tool_clear, tool_v, friction; /* angles in radians */
    int32_t max_support; /* per-MP support capacity (pair slots per MP), multiple of 32, <= 1024 */
    int32_t max_insert;  /* node slots reserved for node insertion over the run (0: insertion off);
                          * see otm_step for the insertion rule */
    otm_material mat[4];
} otm_params;

typedef struct otm_problem {
    int64_t n_nodes, n_mps;
    const double *node_x;        /* n_nodes x 3, initial positions */
    const double *node_du0;      /* n_nodes x 3, initial displacement increment (v0 * dt) */
    const uint8_t *node_flags;   /* n_nodes, OTM_FLAG_* bits */
    const double *mp_x;          /* n_mps x 3, initial positions */
    const double *mp_vol;        /* n_mps, initial volumes */
    const double *mp_mass;       /* n_mps, masses (constant) */
    const int32_t *mp_material;  /* n_mps, index into params.mat */
} otm_problem;

typedef struct otm_handle otm_handle;

/* Fields for otm_state (host copies, ID order). Sizes in bytes:
 *  NODE_X, NODE_DU, NODE_FORCE: 24 n_nodes   NODE_MASS: 8 n_nodes   NODE_FLAGS: n_nodes
 *  MP_X: 24 n_mps  F, DF: 72 n_mps  BE, SIGMA: 48 n_mps  VOL, EBAR, T, RATE: 8 n_mps
 *  LAMBDA: 24 n_mps  SUPPORT_COUNT, NEWTON_IT: 4 n_mps
 *  SUPPORT_IDS: 4 n_mps max_support (padded rows, row p holds SUPPORT_COUNT[p] IDs, ascending)
 *  SHAPE: 32 n_mps max_support (padded rows of (N, dN/dx, dN/dy, dN/dz); in the mixed path the
 *         gradients carry FP32 rounding: e = N d is formed in FP32 there)
 *  MP_GID, NODE_GID: 8 * count (original IDs of the surviving entries)
 *  KINV: 48 n_mps (J^-1 of each MP's last LME solve, xx yy zz xy yz xz: grad N_a = -J^-1 N_a d_a) */
enum {
    OTM_FIELD_NODE_X = 0, OTM_FIELD_NODE_DU = 1, OTM_FIELD_NODE_MASS = 2, OTM_FIELD_NODE_FORCE = 3,
    OTM_FIELD_MP_X = 4, OTM_FIELD_F = 5, OTM_FIELD_BE = 6, OTM_FIELD_SIGMA = 7, OTM_FIELD_VOL = 8,
    OTM_FIELD_EBAR = 9, OTM_FIELD_T = 10, OTM_FIELD_LAMBDA = 11, OTM_FIELD_SUPPORT_COUNT = 12,
    OTM_FIELD_SUPPORT_IDS = 13, OTM_FIELD_SHAPE = 14, OTM_FIELD_NEWTON_IT = 15, OTM_FIELD_RATE = 16,
    OTM_FIELD_DF = 17, OTM_FIELD_MP_GID = 18, OTM_FIELD_NODE_GID = 19, OTM_FIELD_NODE_FLAGS = 20,
    OTM_FIELD_KINV = 21
};

/* Bytes of device workspace needed for a problem of this size. */
int otm_workspace_bytes(int64_t n_nodes, int64_t n_mps, const otm_params *params, size_t *bytes);

/* Create a simulation: copy the host problem into the workspace, then build the initial
 * supports and shape functions (Algorithm 1, REQUIRE line: initial node and MP sets).
 * params is copied. workspace: device pointer, 256-byte aligned, ws_bytes >= required.
 * On success *out is a new handle (free with otm_destroy). */
int otm_init(const otm_problem *prob, const otm_params *params, void *stream, void *workspace,
             size_t ws_bytes, otm_handle **out);

/* Advance n_steps explicit steps (Algorithm 1, steps 1-6 each). Synchronises the stream at
 * the end and returns the first error raised by any kernel (later steps are skipped).
 *
 * Changes of the node and MP sets within a step (the paper adds and removes nodes and MPs,
 * Sec. 1 and Sec. 3.2, without a rule; these are the rules taken):
 *  - erosion (allow_erode): MPs that meet the Johnson-Cook fracture criterion (Sec. 4.2) leave
 *    after the constitutive update; nodes left in no support after the new search are removed.
 *  - insertion (max_insert > 0): an MP whose LME solve fails at its new position, from the warm
 *    start and again from lambda = 0, lies outside the hull of its support. A node is inserted
 *    one spacing h beyond it, away from the centroid c of its support nodes:
 *    x_new = x_p + h (x_p - c) / |x_p - c|, with increment du = x_p,n+1 - x_p,n (the MP's own
 *    increment) and no flags; IDs continue the node numbering in ascending MP ID. The search and
 *    LME then run once more for every MP; a failure there is OTM_ERR_LME_NOCONV. More than
 *    max_insert insertions over the run give OTM_ERR_CAPACITY.
 * Both keep every array in ascending ID order (stream compaction, appended IDs). */
int otm_step(otm_handle *h, int32_t n_steps);

/* Same as otm_step but does not synchronise at the end; errors are reported by
 * otm_error_detail. Problems that erode MPs or insert nodes still synchronise inside each step
 * (the host reads how many entries leave or arrive before it sizes the following launches). */
int otm_step_async(otm_handle *h, int32_t n_steps);

/* Keep the last good step. With buf set (caller-owned, 256-byte aligned, device or page-locked
 * host memory of at least otm_snapshot_bytes), otm_step and otm_step_async save the state into
 * buf before every step and synchronise after it; a step that raises an error is undone by
 * loading buf (the state after the last good step, shape functions regenerated bit for bit, as
 * otm_snapshot_load), the error stays recorded for otm_error_detail, and the call returns it.
 * Later steps then return the same error until otm_snapshot_load or otm_refresh clears it (the
 * caller's resume path: change the state, refresh, step on). Costs one snapshot copy and one
 * synchronisation per step. buf = NULL turns it off. OTM_ERR_ARG for a misaligned or short buf.
 * (Without it, the state after an error is that of the failing step, partially updated.) */
int otm_keep_last_good(otm_handle *h, void *buf, size_t bytes);

/* Current sizes (host-side view; exact after otm_step returns). */
int otm_counts(otm_handle *h, int64_t *n_nodes, int64_t *n_mps, int64_t *n_pairs, int64_t *step);

/* Copy one field to host memory (bytes must equal the field size). Synchronises the stream. */
int otm_state(otm_handle *h, int32_t field, void *host_dst, size_t bytes);

/* Copy selected rows of a per-MP or per-node field (rows: host array of n_rows indices; bytes
 * = n_rows x the field's row size). SUPPORT_IDS / SHAPE rows are ordered by node ID. Synchronises. */
int otm_state_rows(otm_handle *h, int32_t field, const int64_t *rows, int64_t n_rows, void *host_dst,
                   size_t bytes);

/* Overwrite one field from host memory (NODE_X, NODE_DU, MP_X, F, BE, SIGMA, VOL, EBAR, T,
 * LAMBDA). Supports and shape functions are rebuilt by otm_refresh. */
int otm_set_state(otm_handle *h, int32_t field, const void *host_src, size_t bytes);

/* Rebuild supports, shape functions and node-major lists from the current positions. */
int otm_refresh(otm_handle *h);

/* Topology freezing, for finite-difference checks of the adjoint (which holds the supports of
 * the differentiated trajectory fixed). With on != 0 the following steps skip the support
 * search: every step keeps the supports it starts with, and the LME solve (Eq. 14) runs at the
 * new positions over them. OTM_ERR_ARG for problems that erode MPs or insert nodes. */
int otm_freeze_topology(otm_handle *h, int32_t on);

/* One step (as otm_step) whose new supports are given instead of searched, so that a perturbed
 * run can replay the supports recorded from a base run step by step: counts (host, n_mps int32,
 * each 1..max_support) and ids (host, n_mps rows of max_support int32; row p holds counts[p]
 * node indices in [0, n_nodes), any order, the rest is ignored). OTM_ERR_ARG on a bad count or
 * index (nothing runs), OTM_ERR_CAPACITY if a node gets more than 65,535 influences; not for
 * problems that erode MPs or insert nodes. Synchronises. */
int otm_step_with_supports(otm_handle *h, const int32_t *counts, const int32_t *ids);

/* The current supports (Algorithm 3 output of the last step) as a compact CSR in caller-owned
 * DEVICE memory: offsets (n_mps + 1 int32; offsets[0] = 0, offsets[p+1] - offsets[p] = support
 * size of MP p) and ids (at least *n_pairs int32; MP p's row at ids[offsets[p]...], in the
 * library's own row order, i.e. linked-cell order, so that otm_step_with_supports_csr replays it
 * bit for bit). ids_cap: capacity of ids in entries; if the state has more pairs,
 * OTM_ERR_CAPACITY (offsets and *n_pairs are written, ids is not). Enqueued on the handle's
 * stream; synchronises once to read the pair count. */
int otm_supports_export(otm_handle *h, int32_t *offsets, int32_t *ids, int64_t ids_cap, int64_t *n_pairs);

/* otm_step_with_supports with the new supports given as a CSR in DEVICE memory (offsets:
 * n_mps + 1 int32, ids: ids_len int32, as written by otm_supports_export; any order within a
 * row). Before anything reads through them, a kernel checks every row: 0 <= offsets[p] and
 * offsets[p+1] <= ids_len, 1 <= offsets[p+1] - offsets[p] <= max_support, every ID in
 * [0, n_nodes); a violation gives OTM_ERR_ARG and nothing runs. The caller must provide n_mps + 1
 * readable offsets. Not for problems that erode MPs or insert nodes. Synchronises. */
int otm_step_with_supports_csr(otm_handle *h, const int32_t *offsets, const int32_t *ids, int64_t ids_len);

/* The linked-cell grid of Algorithm 3 (step 1) for the current node positions, rebuilt by this
 * call and copied to host memory: origin[3] = componentwise minimum of the node positions,
 * dims[3] = floor((max - min) / cell_size) + 1, *n_cells = their product; cell_start (optional,
 * n_cells + 1 int32, capacity cap_cells entries, else OTM_ERR_CAPACITY): the nodes of cell
 * c = (iz * dims[1] + iy) * dims[0] + ix are sorted[cell_start[c] .. cell_start[c+1]); sorted
 * (optional, n_nodes int32): node indices (ID order) ordered by (cell, index). A grid that
 * cannot be built returns its error (OTM_ERR_NONFINITE, OTM_ERR_CAPACITY), which then stays
 * recorded like a step's. Synchronises. */
int otm_grid_cells(otm_handle *h, double *origin, int32_t *dims, int64_t *n_cells, int32_t *cell_start,
                   int64_t cap_cells, int32_t *sorted);

/* First error recorded on the device: its code and the smallest offending ID. Synchronises. */
int otm_error_detail(otm_handle *h, int32_t *code, int64_t *first_id);

/* Launch statistics: kernels enqueued since otm_init. */
int otm_kernel_launches(otm_handle *h, int64_t *launches);

/* Phase timing: with timing on, every phase of a step is bracketed by CUDA events on the
 * library's stream. otm_phase_times synchronises, returns the summed milliseconds and the
 * number of timed launches of each phase since the previous call, and resets them. */
enum {
    OTM_PHASE_NODE_UPDATE = 0,   /* Eq. 4-6: segmented reduction, central difference, contact */
    OTM_PHASE_KINEMATICS = 1,    /* Eq. 9-13 */
    OTM_PHASE_RETURN_MAP = 2,    /* Sec. 4.1 / 4.2 */
    OTM_PHASE_GRID = 3,          /* Algorithm 3 step 1: linked-cell counting sort */
    OTM_PHASE_SEARCH = 4,        /* Algorithm 3 steps 2-3: supports, influence counts */
    OTM_PHASE_NODE_MAJOR = 5,    /* influence-list offsets (scan of the counts) */
    OTM_PHASE_LME = 6,           /* Eq. 14 + per-pair contributions in node-major order */
    OTM_PHASE_COMPACT = 7,       /* erosion (Sec. 4.2 fracture), orphan-node removal, node insertion */
    OTM_N_PHASES = 8
};
int otm_phase_timing(otm_handle *h, int32_t enable);
int otm_phase_times(otm_handle *h, double *ms, int64_t *launches);

void otm_destroy(otm_handle *h);

/* ---------------------------------------------------------------------------------------
 * Snapshots and the adjoint (reverse mode). The adjoint differentiates functions of the final
 * node positions with respect to the Johnson-Cook constants (A, B, n, C, m) of material 0 and
 * the initial nodal increments, with the supports, the wall-contact set and each return map's
 * elastic/plastic branch frozen at the trajectory being differentiated (no erosion). Paper:
 * Eq. 4-14 and Sec. 4 define the step; the adjoint is their transpose (LME by the implicit-
 * function theorem on sum N_a (x_p - x_a) = 0, the return map as isotropic tensor functions).
 * ------------------------------------------------------------------------------------- */

/* Bytes of one snapshot (caller-owned, 256-byte aligned; device memory or page-locked host
 * memory). */
int otm_snapshot_bytes(otm_handle *h, size_t *bytes);
/* Copy the complete state into / from a snapshot. Loading regenerates the shape functions and
 * node-major lists from the stored state, reproducing them exactly. A snapshot loads into any
 * handle made with the same problem sizes, max_support and max_insert, of either precision
 * (otherwise OTM_ERR_ARG); the FP32 increments are rebuilt from the FP64 ones. */
int otm_snapshot_save(otm_handle *h, void *dst);
int otm_snapshot_load(otm_handle *h, const void *src);

/* Bytes of the adjoint workspace (device memory, 256-byte aligned, caller-owned). */
int otm_adjoint_bytes(otm_handle *h, size_t *bytes);
/* Start a backward pass at the current (final) state: xbar_host (n_nodes x 3, host) is
 * d objective / d node positions; every other adjoint starts at zero. The handle must be an
 * FP64-path handle without erosion, insertion or stabilisation (otherwise OTM_ERR_ARG). */
int otm_adjoint_begin(otm_handle *h, void *adj_ws, size_t bytes, const double *xbar_host);
/* One backward step. Precondition: the handle holds state n (e.g. from otm_snapshot_load) and
 * the adjoint workspace holds the adjoint of state n+1. The call needs state n+1 and the node
 * masses and forces of step n: with next_snapshot NULL it recomputes step n (deterministic);
 * with next_snapshot a snapshot of state n+1 (device or page-locked host memory, as written by
 * otm_snapshot_save on this trajectory) it runs only the node update of step n and loads state
 * n+1, which is cheaper (no search, return map or Newton solve); when the previous call of the
 * same backward pass was the backward step of step n+1, the shape functions of state n+1 kept
 * from it are copied instead of solved again. Then it propagates the adjoint to state n. The
 * handle then holds state n+1 (its node-major contributions are regenerated by the next step). */
int otm_adjoint_step(otm_handle *h, void *adj_ws, const void *next_snapshot);
/* theta_bar[6] = d objective / d (A, B, n, C, m, s): the Johnson-Cook constants of material 0
 * and a scalar s on which the initial displacement increments depend, through du0_ds (host,
 * n_nodes x 3, optional: d(du_I at step 0)/ds; NULL gives theta_bar[5] = 0). For an impact
 * with du_0 = -v0 dt e_z on every node, du0_ds = (0, 0, -dt) per node makes theta_bar[5] the
 * derivative with respect to the impact velocity v0. The chain rule is applied once the backward
 * pass has reached step 0. dubar_host (n_nodes x 3, optional) = d objective / d (displacement
 * increments of the state the backward pass has reached). */
int otm_adjoint_result(otm_handle *h, void *adj_ws, const double *du0_ds, double *theta_bar,
                       double *dubar_host);

/* ---------------------------------------------------------------------------------------
 * Stand-alone kernels (device pointers, caller-owned; enqueued on `stream`, not synchronised)
 * With a point count of 0 the per-point arrays may be NULL and nothing is launched.
 * ------------------------------------------------------------------------------------- */

/* Bytes of scratch needed by otm_support_search for n_nodes nodes. */
int otm_search_scratch_bytes(int64_t n_nodes, size_t *bytes);

/* Linked-cell support search (Algorithm 3; support definition as in otm_params.rs2).
 * node_x: n_nodes x 3, mp_x: n_mps x 3 (device, FP64). Output: ids[p * max_support + k],
 * k < counts[p], ascending node IDs; counts[p] is the full support size (> max_support means
 * the row was truncated and status holds OTM_ERR_CAPACITY). Grid: origin = componentwise
 * node minimum, dims = floor((max - min)/cell_size) + 1 per axis. scratch: device memory of
 * otm_search_scratch_bytes; grid_out (optional, device): origin[3] doubles then dims[3] as
 * doubles. status (device int32, caller zeroes it): 0 or the first error code. */
int otm_support_search(const double *node_x, int64_t n_nodes, const double *mp_x, int64_t n_mps,
                       double rs2, double cell_size, int32_t max_support, int32_t *ids,
                       int32_t *counts, void *scratch, size_t scratch_bytes, double *grid_out,
                       int32_t *status, void *stream);

/* Allocation-free variant of otm_support_search, for callers that cannot allocate device
 * memory when they call (for instance a process whose device memory is already reserved by
 * another allocator, or a loop that must not take cudaMalloc's implicit synchronisation).
 * The paper has no counterpart: this is a deployment convenience, not part of the method.
 * Same arguments, outputs and status as otm_support_search minus the scratch buffer: the
 * scratch is a static 16 MiB device array inside the library, held by every GPU that loads it
 * until the process exits. n_nodes must be <= OTM_NOALLOC_MAX_NODES (else OTM_ERR_CAPACITY,
 * nothing launched). The first call on a device looks up that array's device address with the
 * device current (call it once before any stream capture). All calls share the one array and
 * it keeps the previous call's contents (every call re-initialises what it reads), so calls
 * whose work overlaps on the GPU -- on different streams or from different threads without
 * ordering -- race; serialise them on one stream. Allocates nothing. */
#define OTM_NOALLOC_MAX_NODES 65536
int otm_support_search_noalloc(const double *node_x, int64_t n_nodes, const double *mp_x, int64_t n_mps,
                               double rs2, double cell_size, int32_t max_support, int32_t *ids,
                               int32_t *counts, double *grid_out, int32_t *status, void *stream);

/* LME shape functions (Eq. 14) for n_mps points with given supports (ids/counts as produced
 * by otm_support_search). lambda (n_mps x 3, in: start, out: solution). shape: n_mps x
 * max_support x 4 doubles (N, dN/dx, dN/dy, dN/dz). iters (n_mps, optional). status: as above
 * (OTM_ERR_LME_NOCONV on failure). */
int otm_lme(const double *node_x, const double *mp_x, int64_t n_mps, const int32_t *ids,
            const int32_t *counts, int32_t max_support, double beta, double tol_abs,
            int32_t max_newton, double *lambda, double *shape, int32_t *iters, int32_t *status,
            void *stream);

/* Self-test of the library's internal FP64 exponential (table-driven after Tang, used for the
 * LME weights of Eq. 14). Its argument is scaled: y = f * 1024 / ln 2. Device arrays of n
 * doubles: mine[i] = internal exp of f_i = y[i] ln2/1024; ref[i] = CUDA's exp of the same f_i
 * (carried as a rounded product plus its error, so ref is accurate to about an ulp). The first
 * call on a device uploads the exponential's table (synchronous copy). */
int otm_exp_selftest(const double *y, int64_t n, double *mine, double *ref, void *stream);

/* Constitutive update (Sec. 4.1 / 4.2) of n_mps points: inputs dF (9), F_new (9, for J),
 * be (6, in/out), ebar, T (in/out); outputs sigma (6), rate, failed (uint8, optional). */
int otm_return_map(const otm_material *mat, double dt, int64_t n_mps, const double *dF,
                   const double *F_new, double *be, double *ebar, double *T, double *sigma,
                   double *rate, uint8_t *failed, int32_t *status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* OTM_H */
