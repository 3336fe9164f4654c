/*
 * ipc.h -- C ABI of the B300 MAS-PNCG library (libipc_b300.so).
 *
 * One implicit-Euler timestep minimises the incremental potential of the
 * paper's problem statement (Sec. 3.1, Eq. 1 without friction):
 *     E(x) = 1/2 (x - x~)^T M (x - x~) + h^2 Psi_SNH(x) + kappa sum_c b(d_c(x)),
 *     x~ = x^t + h v^t + h^2 M^-1 f_ext,
 * over vertex positions, with no intersection along the way, by the MAS-PNCG
 * iteration of Algorithm 1: multilevel additive Schwarz preconditioner
 * (Sec. 3.3) patched by the Sparse-Input Woodbury update (Sec. 4.1, Eq. 6-8),
 * the Hessian-aware 2D subspace step (Sec. 4.2, Eq. 9-10), the restart test
 * (Sec. 4.3, Eq. 11) and per-subdomain conservative CCD (Sec. 4.4; supplement
 * Sec. 3).  Every step of the path runs in CUDA kernels built for sm_103a on
 * one GPU; the host only sequences them.
 *
 * Conventions
 *  - Positions, velocities and every per-vertex vector are arrays of
 *    n_verts x 3 doubles (x0, y0, z0, x1, ...), row-major, in metres and
 *    seconds.  Tets are n_tets x 4 int32 vertex ids, positively oriented.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  All device work of a call is ordered on that stream;
 *    calls that return host data synchronise it before returning.
 *  - Host pointers belong to the caller and are only read (or written, for
 *    outputs) during the call.  The library owns all device memory of a
 *    scene; it obtains it through ipc_alloc_fns (or cudaMalloc) at
 *    ipc_scene_create and releases it in ipc_scene_destroy.
 *  - Return codes: IPC_OK (0) or a positive warning on success, a negative
 *    ipc_status on failure; ipc_last_error() describes the last failure of
 *    the calling thread.  After a failure the scene keeps its pre-call state
 *    where possible (ipc_step: the state of the last completed timestep).
 */
#ifndef IPC_B300_H
#define IPC_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ipc_status {
    IPC_OK = 0,
    IPC_NOT_CONVERGED = 1,   /* warning: iteration cap reached, step still taken */
    IPC_PENDING = 2,         /* serving: ticket not finished yet */
    IPC_ERR_INVALID = -1,    /* bad argument or mesh */
    IPC_ERR_INTERSECTING = -2, /* initial state has a contact at distance <= 0 */
    IPC_ERR_OOM = -3,        /* device allocation failed */
    IPC_ERR_NUMERIC = -4,    /* NaN / Inf met in the iteration */
    IPC_ERR_TIMEOUT = -5,    /* a device-side wait ran out of its budget */
    IPC_ERR_CUDA = -6,       /* CUDA runtime error */
    IPC_ERR_CAPACITY = -7    /* a contact / candidate buffer overflowed and
                                could not be grown */
} ipc_status;

typedef enum ipc_precision {
    IPC_PREC_FP64 = 0,       /* every quantity in FP64 (the plain method) */
    IPC_PREC_FP32 = 1,       /* FP32 bulk (gradient, H v, MAS blocks and
                                products); FP64 for positions, barrier
                                distances, CCD, the 2x2 and capacitance
                                solves and all reductions */
    IPC_PREC_BF16_MAS = 2    /* as IPC_PREC_FP32, with the MAS block factors
                                W' (B = W'^T W') stored in BF16 and applied
                                on the tensor cores (BF16 products, FP32
                                accumulation; the right-hand sides split into
                                BF16 high and low parts) */
} ipc_precision;

/* Scene description (host memory, copied at create). */
typedef struct ipc_scene_desc {
    int n_verts;
    const double* x_rest;    /* n_verts x 3: rest shape */
    const double* x0;        /* n_verts x 3: initial positions (NULL = x_rest) */
    const double* v0;        /* n_verts x 3: initial velocities (NULL = 0) */
    int n_tets;
    const int32_t* tets;     /* n_tets x 4 */
    const double* E;         /* n_tets Young's modulus [Pa] */
    const double* nu;        /* n_tets Poisson ratio */
    const double* rho;       /* n_tets density [kg/m^3] */
    double gravity[3];       /* f_ext / m */
    int has_ground;          /* static plane n . x = offset */
    double ground_normal[3];
    double ground_offset;
} ipc_scene_desc;

/* Solver parameters (see ipc_default_params). */
typedef struct ipc_params {
    double h;                /* timestep [s] */
    double dhat;             /* barrier activation distance [m] */
    double kappa;            /* barrier stiffness [kg] */
    double tol;              /* converged when max_v |z_v| <= tol * h * bbox_diag */
    double delta;            /* restart threshold on r_k, Eq. 11 (0.3) */
    double eps_rot_deg;      /* normal rotation threshold, Sec. 4.1.1 (25) */
    double ccd_shrink;       /* s in alpha_l = (1 - s) d0 / l_tight (0.1) */
    double eps_sing;         /* 2x2 singular test, relative (1e-12) */
    double eps_abs;          /* 2x2 singular test, absolute (1e-300) */
    int K;                   /* Woodbury vectors kept per subdomain (8, <= 16) */
    int iter_max;            /* PNCG iteration cap per timestep (10000) */
    int levels_max;          /* MAS levels including level 0 (6) */
    int ls_max;              /* energy-check trials (20) */
    int precision;           /* ipc_precision */
    int contact_capacity;    /* initial contact buffer size, 0 = automatic */
    int broad_phase;         /* 0 automatic: cached candidate-pair lists while
                                valid, hashed grid otherwise; 1 hashed grid for
                                every query; 2 cached lists for every query
                                (built at the query's own positions where
                                needed).  All three give the same contact and
                                CCD candidate sets. */
    int mas_mode;            /* MAS maintenance between restarts (Sec. 4.3 and
                                its ablation): 0 Sparse-Input Woodbury updates
                                (default); 1 full rebuild, every iteration
                                reassembles and reinverts the blocks at the
                                current positions and contacts (the PNCG
                                recurrence goes on: not a restart); 2 freeze,
                                the preconditioner and H_base of the last
                                restart serve unchanged; 3 3x3 block-Jacobi
                                preconditioning instead of MAS (the inverse
                                3x3 diagonal blocks of H_base, rebuilt at
                                restarts, frozen between them: the paper's
                                MAS-vs-Jacobi comparison, Sec. 5.1) */
    int ccd_mode;            /* 0 per-subdomain step bounds alpha_d (Sec. 4.4,
                                default); 1 one global step min_d alpha_d */
    int graphs;              /* 1 (default): the per-iteration launch sequences
                                (preconditioner, forms and direction; cached-
                                list CCD and first trial) replay as CUDA graphs,
                                captured the second time each configuration
                                occurs; 0: every kernel launched one by one.
                                Both run the same kernels on the same data. */
    double fp32_pivot_floor; /* FP32 bulk only: a block whose FP32 Cholesky
                                of the unit-diagonal scaled block meets a pivot
                                at or below this value (or a column entry
                                L_rk^2 > 1) is inverted again in FP64 with the
                                pivot rules (Sec. 4.2). Default 1e-6; 1 sends
                                every block to FP64. */
    int grid_pair_capacity;  /* entries of the scratch pair list (0: 16 per
                                surface primitive + 4096): the pairs a grid
                                query, an FP32 screen of a cached candidate
                                list, or a CCD verification pass hands on to
                                be tested in FP64 on full warps. Pairs beyond
                                it are tested where they were found instead:
                                same results, slower. */
    int wait_polls;          /* polls of each bounded wait of a CTA on its
                                bulk copy into shared memory (default 2^22,
                                far above any copy's latency). A wait that
                                runs out marks the call IPC_ERR_TIMEOUT; the
                                CTA then still drains its copy before it
                                exits. 0 makes every such wait report a
                                timeout without polling (a test of the error
                                path that needs no fault). */
    int apply_ctas;          /* CTAs per SM of the persistent MAS block apply;
                                0 (default): picked at ipc_scene_create by
                                timing the candidates (IPC_Q_APPLY_CTAS) */
} ipc_params;

/* Device allocator used for all scene memory; NULL functions = cudaMalloc. */
typedef struct ipc_alloc_fns {
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, void* ctx);
    void* ctx;
} ipc_alloc_fns;

/* Per-call statistics of ipc_step (summed over its timesteps, last values
 * for the state fields). */
typedef struct ipc_step_stats {
    int steps;
    int iters;               /* PNCG iterations */
    int restarts;            /* MAS rebuilds */
    int ls_halvings;         /* rejected energy-check trials */
    int ls_failures;         /* iterations with no accepted trial */
    int converged;           /* 1 if the last timestep converged */
    int n_contacts;          /* active contacts at the end */
    int ccd_fallbacks;       /* verification passes that fell back to uniform alpha */
    double energy;           /* E at the end of the last timestep */
    double min_dist;         /* smallest active contact distance at the end */
    double znorm;            /* last max_v |z_v| */
} ipc_step_stats;

typedef struct ipc_scene ipc_scene;

/* Defaults of the paper's constants; h, dhat and kappa must still be set. */
void ipc_default_params(ipc_params* p);

/* Build a scene: validates the mesh (ids in range, positive rest volumes),
 * extracts the boundary surface, computes lumped mass rho V / 4 and rest
 * shapes, builds the MAS hierarchy (32-vertex subdomains by greedy BFS over
 * mesh adjacency, supplement Sec. 1.2), allocates device state and copies
 * it up, and picks the block apply's launch configuration by timing (see
 * IPC_Q_APPLY_CTAS).  Fails with IPC_ERR_INTERSECTING if a contact of the initial state
 * has distance <= 0.  `alloc` may be NULL.  Its device work runs on the
 * legacy default stream and waits only for that stream, never for the whole
 * device, so it may run in one thread while other scenes step (and capture
 * CUDA graphs) on non-blocking streams in others, e.g. under ipc_server. */
int ipc_scene_create(const ipc_scene_desc* desc, const ipc_params* params,
                     const ipc_alloc_fns* alloc, ipc_scene** out);

/* Release a scene.  Waits for the scene's own stream and the legacy default
 * stream only: every call the caller queued for this scene on its own
 * streams (or submitted to a server) must have completed.  Other scenes may
 * go on stepping meanwhile. */
void ipc_scene_destroy(ipc_scene* s);

/* Advance n_steps timesteps (Algorithm 1 each).  `stats` may be NULL.
 * Returns IPC_OK, IPC_NOT_CONVERGED (some timestep hit iter_max) or an
 * error. */
int ipc_step(ipc_scene* s, int n_steps, void* stream, ipc_step_stats* stats);

/* Replace positions and velocities (checkpoint / resume).  x, v are host
 * arrays (on_device = 0) or device arrays (on_device = 1) of n_verts x 3
 * doubles.  v may be NULL (zero). */
int ipc_set_state(ipc_scene* s, const double* x, const double* v, int on_device, void* stream);

typedef enum ipc_query_kind {
    IPC_Q_POSITIONS = 0,     /* n_verts x 3 double */
    IPC_Q_VELOCITIES = 1,    /* n_verts x 3 double */
    IPC_Q_N_VERTS = 2,       /* int */
    IPC_Q_N_CONTACTS = 3,    /* int: active contacts at the current state */
    IPC_Q_SUBDOMAIN_ALPHA = 4, /* n_subdomains double: last CCD step sizes */
    IPC_Q_N_SUBDOMAINS = 5,  /* int */
    IPC_Q_TRACE_LEN = 6,     /* int: PNCG iterations of the last timestep */
    IPC_Q_TRACE = 7,         /* trace_len x ipc_iter_record */
    IPC_Q_SURFACE_COUNTS = 8,/* 3 int: surface verts, tris, edges */
    IPC_Q_LEVEL_MAP = 9,     /* per level: group and slot of each node (see
                                ipc_query_level) */
    IPC_Q_BBOX_DIAG = 10,    /* double */
    IPC_Q_N_BODIES = 11,     /* int: connected bodies of the mesh */
    IPC_Q_FP64_BLOCKS = 12,  /* int: subdomain blocks the last restart inverted
                                in FP64. FP32 bulk: the blocks whose FP32
                                factorisation would floor a pivot or raise one
                                (Sec. 4.2 inverse with the row-norm bound), 0
                                before the first restart; FP64 bulk: every
                                block. */
    IPC_Q_PIVOT_FIXES = 13,  /* int: blocks of the last restart whose final
                                (FP64) factorisation floored or raised a
                                pivot: 0 means every stored inverse is that of
                                a plain Cholesky factorisation */
    IPC_Q_APPLY_CTAS = 14    /* int: CTAs per SM of the persistent MAS block
                                apply, picked at ipc_scene_create by timing
                                the candidates the kernel's shared memory
                                allows on this scene's blocks (the project's
                                autotuner; results do not depend on it) */
} ipc_query_kind;

/* Copy a piece of state into host memory dst (dst_bytes long). */
int ipc_query(ipc_scene* s, int what, void* dst, size_t dst_bytes, void* stream);

/* Hierarchy inspection: number of levels, and for `level` the node count,
 * group count and, if non-NULL, group / slot of every node. */
int ipc_query_level(ipc_scene* s, int level, int* n_nodes, int* n_groups,
                    int* group_of_node, int* slot_of_node);

/* Surface inspection: sorted surface vertex ids, triangles (3 ids each) and
 * edges (2 ids each, a < b), all in lexicographic order. */
int ipc_query_surface(ipc_scene* s, int* verts, int* tris, int* edges);

/* Per-stage device time of the scene's ipc_step calls, measured with CUDA
 * events recorded on the step's stream around each stage, accumulated until
 * reset.  Stages: 0 restart (RebuildMAS), 1 classify + top-K, 2 MAS block
 * apply with Woodbury (Eq. 7), 3 quadratic forms and dots, 4 direction, 5
 * broad-phase choice and CCD, 6 trial evaluation (contacts, energy,
 * gradient), 7 other (predictor, restriction, prolongation).  ms[8] in
 * milliseconds, launches[8] stage executions.  Event pairs around short
 * stages also catch host launch gaps; ipc_profile_replay times a stage's
 * kernels alone. */
typedef struct ipc_profile {
    double ms[8];
    long long launches[8];
} ipc_profile;

/* enable != 0 starts timing (and resets the counters); 0 stops it. */
int ipc_profile_enable(ipc_scene* s, int enable);
int ipc_profile_read(ipc_scene* s, ipc_profile* out);

/* Replays the kernels of one stage on the scene's current state and returns
 * their mean device time per launch in *ms_mean.  Stages: 0 = the batched
 * inversion of the blocks assembled at the scene's last RebuildMAS (FP32
 * pass and FP64 redo of flagged blocks; it rewrites the same factors), 2 =
 * MAS block apply of level-0 and coarse blocks to the scene's gradient (no
 * Woodbury patch), 3 = the H~ quadratic forms (Eq. 6) of the scene's z and p
 * (the reduction kernel; the packing of z and p before it is not timed), 4 =
 * the level-0 apply with the Sparse-Input Woodbury update (Eq. 7) of the
 * scene's current contacts against its C_base (their classification and
 * top-K run once before, untimed).  If flush != NULL, flush_bytes of that
 * caller-owned device buffer (16-byte aligned) are read before every launch,
 * which evicts the stage's data from L2 without leaving dirty lines.  Two
 * loops run on `stream`: reps x (flush, stage) and reps x (flush); the result
 * is the difference of their CUDA-event times over reps (an event pair
 * resolves about 2 us here).  Overwrites the scene's z (stages 2, 4) and its
 * dot-product scalars; meant for use between timesteps.  IPC_ERR_INVALID for
 * another stage, reps < 1, or stage 0 before any RebuildMAS. */
int ipc_profile_replay(ipc_scene* s, int stage, int reps, void* flush, size_t flush_bytes, void* stream,
                       double* ms_mean);

/* Measured FMA throughput of the SM's SIMT pipes on the current device, in
 * TFLOP/s (2 flops per FMA): every thread of a grid that fills each SM runs 8
 * independent FMA chains; one launch of about target_ms is timed with CUDA
 * events after a calibration and a warm-up launch.  precision:
 * IPC_PREC_FP32 or IPC_PREC_FP64.  The denominator of an ALU-bound kernel's
 * roofline (the FP32 block inversion) beside lanes x 2 x clock.  Allocates
 * and frees one device buffer; synchronises the device.  IPC_ERR_INVALID for
 * another precision or target_ms outside (0, 1000]; IPC_ERR_CUDA on a CUDA
 * error. */
int ipc_profile_fma_peak(int precision, double target_ms, double* tflops);

/* Number of CUDA kernels this library has launched in the process so far
 * (all scenes, all calls). */
long long ipc_kernel_launches(void);

/* One record per PNCG iteration of the last timestep. */
typedef struct ipc_iter_record {
    int restart;
    int n_contacts;
    int n_update;            /* classified contacts with dS > 0 */
    int ls_halvings;
    double mu, nu;
    double gz, znorm;
    double energy_before, energy_after;
    double alpha_min, alpha_max;
    double r;
    double pmax;             /* max_v |p_v| of the direction */
    int ccd_passes;          /* per-subdomain verification passes, -1 = uniform fallback */
    int cached_pairs;        /* 1 if the broad phase used the cached candidate lists */
    int ccd_passes_body;     /* per-body verification passes, -1 = uniform fallback; when
                                the per-subdomain one fell back and this one did not,
                                the first energy-check trial was the per-body step */
    int pad_;                /* layout padding, 0 */
} ipc_iter_record;

/* ---- evaluation entry points (host arrays in and out) -------------------
 * They run single pieces of the path on the GPU at caller-given positions so
 * that each can be checked on its own. */

/* E(x) with x~ given (Eq. 1) and, if g != NULL, its gradient. */
int ipc_eval_energy_grad(ipc_scene* s, const double* x, const double* xtilde,
                         double* energy, double* g, void* stream);

/* Active contact set at x (ComputeConstraintSet of Algorithm 1): writes up
 * to cap records and the full count to *n.  type: 0 point-triangle, 1
 * edge-edge, 2 point-ground; ids: (vertex, surface tri), (edge, edge) with
 * the lower edge first, or (vertex, 0); verts: 4 vertex ids (-1 unused);
 * dist; k = kappa b''(d); grad12 = nabla d over the 4 verts. */
int ipc_eval_contacts(ipc_scene* s, const double* x, int cap, int* n, int* type,
                      int* ids, int* verts, double* dist, double* k, double* grad12,
                      void* stream);

/* z = P g with P rebuilt at x_base (RebuildMAS) and, if x_curr != NULL,
 * patched by the Woodbury update for the contacts at x_curr (Eq. 7-8). */
int ipc_eval_precond(ipc_scene* s, const double* x_base, const double* x_curr,
                     const double* g, double* z, void* stream);

/* (z^T H~ z, z^T H~ p, p^T H~ p) with H~ = H_base(x_base) + U U^T, U from
 * the contacts at x_curr (Eq. 6; supplement Eq. 13-18). */
int ipc_eval_forms(ipc_scene* s, const double* x_base, const double* x_curr,
                   const double* z, const double* p, double out[3], void* stream);

/* Per-subdomain conservative step sizes for direction p at x (supplement
 * Sec. 3); alpha has n_subdomains entries; *passes = verification passes
 * used, -1 if the uniform fallback was taken.  alpha_body (n_bodies entries)
 * and passes_body, if not NULL, receive the same for the grouping by
 * connected body that the energy check falls back to. */
int ipc_eval_ccd(ipc_scene* s, const double* x, const double* p, double* alpha,
                 int* passes, double* alpha_body, int* passes_body, void* stream);

/* ---- allocation-free preconditioner apply --------------------------------
 * No counterpart in the paper: a library entry point for callers that must
 * not allocate device memory during the call (a solver loop beside other
 * busy streams, where cudaMalloc / cudaFree can synchronise the device; a
 * process whose device memory belongs to another allocator).
 *
 * z = P_base g: the additive multilevel Schwarz preconditioner (Sec. 3.3)
 * as the scene's last RebuildMAS left it (its last restart inside ipc_step,
 * or the last ipc_eval_precond / ipc_eval_forms call), without the Woodbury
 * patch, on caller-owned DEVICE arrays.
 *  - g_dev, z_dev: 3 n_verts values each in the scene's bulk precision
 *    (double for IPC_PREC_FP64, float for IPC_PREC_FP32), on the scene's
 *    device, which must be current; they must not overlap.  z need not be
 *    initialised.  The call reads g and the scene, writes z and the static
 *    array below, and nothing of the scene.
 *  - The work is enqueued on `stream`; the call then waits for that stream
 *    (it reads the status of the bulk-copy waits back into host stack
 *    memory), so z is complete when it returns IPC_OK.
 *  - Scratch: a status record and the coarse residuals and solutions
 *    (levels >= 1) live in one static 256 KiB device array per device
 *    (align256(status) + 2 x align256(3 x coarse nodes x sizeof(value))
 *    bytes are used).  The status record is cleared at the start of every
 *    call, and every coarse value is written before it is read.  Calls that
 *    overlap in time on one device race on that array: order them on one
 *    stream or synchronise between them.
 *  - The first call on each device resolves the array's address
 *    (cudaGetSymbolAddress), which may load the library's device code on
 *    that device; make that first call before any stream capture begins.
 *    The address is kept for the life of the process: after a reset of the
 *    device (cudaDeviceReset) this entry point must not be called again.
 *  - Errors: IPC_ERR_INVALID for a null argument, a scene with no
 *    RebuildMAS yet, host or foreign-device arrays, overlapping g and z, or
 *    another device current; IPC_ERR_CAPACITY when the coarse levels need
 *    more than the static array (above roughly 1.7e5 vertices in FP64, twice
 *    that in FP32); IPC_ERR_TIMEOUT when a bounded wait on a bulk copy ran
 *    out (z is then not defined); IPC_ERR_CUDA if a launch fails.  Only
 *    error paths allocate (host memory for the message). */
int ipc_precond_apply_noalloc(ipc_scene* s, const void* g_dev, void* z_dev, void* stream);

const char* ipc_last_error(void);

/* ---- Serving: continuous batching of step requests over resident scenes
 *
 * No counterpart in the paper (the method steps one scene); this is the
 * request loop of a simulation service. Scenes are created by the caller
 * and stay resident on the device (positions, MAS hierarchy, contact sets);
 * a request asks for n_steps timesteps of one scene. The server runs up to
 * cfg.slots requests at once, each on its own CUDA stream and host thread,
 * so their kernels overlap on the device. A queued request is admitted, in
 * submission order among the admissible ones, when a slot is free, no other
 * request of the same scene is running (a scene's steps stay in order) and
 * the device has at least cfg.min_free_bytes free (cudaMemGetInfo), or when
 * nothing else is running. Every timestep computes exactly what ipc_step
 * computes alone. Cooperative launches of concurrent scenes are ordered on
 * the device (no two grids that need full residency wait on each other).
 *
 * alloc is accepted for interface symmetry with ipc_scene_create and unused:
 * the server allocates no device memory. Scenes must outlive the requests
 * that name them and must not be stepped, queried or destroyed by the
 * caller while a request of theirs is queued or running. */
typedef struct ipc_server ipc_server;
typedef struct ipc_server_cfg {
    int slots;               /* requests running at once (>= 1) */
    size_t min_free_bytes;   /* free device memory needed to admit a request */
} ipc_server_cfg;

/* Starts cfg->slots worker threads (each with a non-blocking stream on the
 * current device). Returns IPC_OK or IPC_ERR_INVALID / IPC_ERR_CUDA. */
int ipc_server_create(const ipc_server_cfg* cfg, const ipc_alloc_fns* alloc, ipc_server** out);

/* Queues n_steps timesteps of scene; *ticket identifies the request. */
int ipc_server_submit(ipc_server* srv, ipc_scene* scene, int n_steps, unsigned long long* ticket);

/* IPC_PENDING while the request is queued or running; otherwise the return
 * code of its ipc_step, with its statistics in *stats and the time from
 * submission to completion in *latency_ms (both nullable); the ticket is
 * then released. IPC_ERR_INVALID for an unknown ticket. */
int ipc_server_poll(ipc_server* srv, unsigned long long ticket, ipc_step_stats* stats, double* latency_ms);

/* As ipc_server_poll, but blocks until the request finishes or timeout_ms
 * passes (IPC_PENDING then). timeout_ms <= 0 or NaN does not block; values
 * above 1e12 (about 30 years) are capped there. */
int ipc_server_wait(ipc_server* srv, unsigned long long ticket, double timeout_ms, ipc_step_stats* stats,
                    double* latency_ms);

/* Finishes every queued and running request, stops the workers, frees the
 * server. */
void ipc_server_destroy(ipc_server* srv);

#ifdef __cplusplus
}
#endif
#endif
