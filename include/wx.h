/*
 * wx.h -- C ABI of the GB300 weather-step library (libwx.so).
 *
 * One time step of a structured-grid weather model, the data-parallel hot
 * path of the paper's reduced weather application (Sec. 3.1) and of its
 * production model's dynamics + column physics split (Sec. 2 and Sec. 5):
 *
 *   dynamics  phi* = phi + dt (kappa_h Lap_h phi + kappa_h Lap_z phi - div(v phi))
 *             for phi in {T, q}: 7-point finite-volume diffusion (paper Eq. 1,
 *             explicit Euler), zero flux through bottom and top (the paper's
 *             appendix diffusion listing uses 1-5d on the end levels),
 *             periodic in x and y (Sec. 3.1: "cyclic" KI/KJ boundaries), plus
 *             flux-form first-order upwind advection by C-grid face winds;
 *   physics   per column (Sec. 3.1: one thread per K column, K sequential,
 *             Sec. 2.1): implicit vertical diffusion (I - dt L_v) T** = T*
 *             by the Thomas algorithm, optical depth dtau_k =
 *             alpha_k dz_k q*_k / q_ref scanned from the top, heating
 *             H_k = S0 (exp(-tau_top,k) - exp(-tau_bot,k)) / dz_k,
 *             T^{n+1} = T** + dt H, q^{n+1} = q*.
 *
 * Conventions
 *  - Every call returns a status (WX_OK = 0, negative on error); nothing is
 *    thrown across the ABI.  wx_last_error() gives a message for the last
 *    failing call on a context.
 *  - Host arrays are FP64 and C order: 3D fields [nz][ny][nx], 2D fields
 *    [ny][nx], per-level arrays [nz].  An FP32 context rounds them once on
 *    load.
 *  - The library owns all device memory of a context (fields stay resident
 *    across steps, the paper's "data region", Sec. 3.2.2 and Sec. 5.1.3);
 *    arrays passed in are copied and remain owned by the caller.
 *  - Streams belong to the caller (a cudaStream_t passed as void*, NULL =
 *    legacy default stream).  wx_step is asynchronous; wx_sync waits and
 *    reports the device status word.
 *  - A context is used by one host thread at a time.
 */
#ifndef WX_H
#define WX_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wx_ctx wx_ctx;

/* storage / compute precision of a context */
enum {
    WX_F32 = 0,   /* FP32 fields, FP32 arithmetic                               */
    WX_F64 = 1,   /* FP64 fields, FP64 arithmetic                               */
    WX_MIXED = 2  /* FP32 fields; FP64 elimination on weakly dominant columns   */
};

/* status codes */
enum {
    WX_OK = 0,
    WX_EINVAL = -1,      /* bad argument                                       */
    WX_ENOMEM = -2,      /* device or host allocation failed                   */
    WX_ECUDA = -3,       /* a CUDA runtime call failed                         */
    WX_ECFL = -4,        /* parameters/winds violate the positivity bound      */
    WX_ENONFINITE = -5,  /* a step produced a non-finite value                 */
    WX_ETIMEOUT = -6,    /* a bounded device wait gave up                      */
    WX_ESTATE = -7,      /* call out of order (e.g. step before load)          */
    WX_EUNSUPPORTED = -8 /* size or option outside what this build supports    */
};

/* wx_params.flags */
enum {
    WX_ADVECTION = 1u, /* include the upwind advection term                    */
    WX_PHYSICS = 2u,   /* run the column physics (Thomas solve + radiation)    */
    WX_SUMS = 4u,      /* record FP64 mass/energy sums after every step        */
    WX_SURROGATE = 8u, /* column physics by the attached MLP, residual-checked */
    WX_RK3 = 16u       /* dynamics by three-stage Runge-Kutta (Wicker-Skamarock,
                          ASUCA's integrator, Sec. 2.1): phi1 = phi + dt/3 L(phi),
                          phi2 = phi + dt/2 L(phi1), phi3 = phi + dt L(phi2),
                          then the column physics on phi3; WX_F32 / WX_F64
                          only, excludes WX_SUMS and WX_SURROGATE; one more
                          field buffer on the device */
};

typedef struct {
    double dt;           /* time step (> 0)                                    */
    double h;            /* horizontal grid spacing (> 0)                      */
    double kappa_h;      /* diffusivity of the dynamics (>= 0)                 */
    double S0;           /* top-of-column radiative flux (>= 0)                */
    double q_ref;        /* optical-depth reference tracer value (> 0)         */
    double dd_threshold; /* WX_MIXED: columns whose dominance ratio
                            min_k |b_k|/(|a_k|+|c_k|) is below this run the
                            elimination in FP64 (<= 0 selects 1.1)             */
    const double *dz;        /* [nz] layer thickness (> 0), host               */
    const double *kappa_lev; /* [nz] vertical diffusivity profile (>= 0), host */
    const double *alpha;     /* [nz] absorber coefficient (>= 0), host         */
    const double *kappa_mult;/* [ny*nx] per-column multiplier (>= 0) or NULL   */
    unsigned flags;          /* WX_ADVECTION | WX_PHYSICS | WX_SUMS | WX_SURROGATE | WX_RK3 */
} wx_params;

/* Create a context for an nx x ny x nz grid (each >= 1; nz <= 256).
 * dtype is WX_F32, WX_F64 or WX_MIXED.  Allocates the resident fields.
 * Errors: WX_EINVAL, WX_EUNSUPPORTED, WX_ENOMEM, WX_ECUDA. */
int wx_create(int nx, int ny, int nz, int dtype, wx_ctx **out);

/* Copy and validate parameters (positivity of dt, h, q_ref, dz; the
 * explicit update's coefficients must be non-negative, checked against the
 * winds at the next wx_step -> WX_ECFL).  Computes the per-level tables on
 * the device.  May be called again between steps.  A WX_F64 context with a
 * kappa_mult field eliminates per column on the fly and keeps two values
 * per level of each column in shared memory: at most 174 levels
 * (WX_EUNSUPPORTED beyond). */
int wx_set_params(wx_ctx *c, const wx_params *p);

/* Load the state: T, q [nz][ny][nx], face winds U, V [ny][nx] (U on the
 * east face of cell (i,j), V on its north face).  src_is_device = 0: host
 * pointers; 1: device pointers (e.g. torch tensors).  FP64 in both cases.
 * Synchronous.  Resets the sums record. */
int wx_load_fields(wx_ctx *c, const double *T, const double *q,
                   const double *U, const double *V, int src_is_device);

/* Advance n_steps >= 0 steps on the caller's stream (asynchronous).  The
 * fields are updated out of place and the buffers swapped after each step
 * (paper appendix, time-integration listing).  Errors found on the host
 * (WX_ESTATE, WX_ECFL) are returned at once; device-side errors surface in
 * wx_sync. */
int wx_step(wx_ctx *c, int n_steps, void *cuda_stream);

/* Wait for the context's last stream and return the device status word as
 * a status (WX_ENONFINITE, WX_ETIMEOUT) or WX_OK.  Clears the word. */
int wx_sync(wx_ctx *c);

/* The state (T, q) alone in FP32 [nz][ny][nx], for WX_F32 / WX_MIXED
 * contexts (WX_EUNSUPPORTED for WX_F64): the values the context stores, so
 * half the bytes of wx_load_fields / wx_read_fields and no rounding.  The
 * winds must have been loaded by wx_load_fields (WX_ESTATE otherwise); they
 * are kept.  Loading resets the sums record like wx_load_fields.  Host
 * (src_is_device = 0) or device input; host output (either of T, q may be
 * NULL on read); synchronous. */
int wx_load_state_f32(wx_ctx *c, const float *T, const float *q, int src_is_device);
int wx_read_state_f32(wx_ctx *c, float *T, float *q);

/* The same two transfers enqueued on the caller's stream without waiting:
 * T and q must be pinned host memory (cudaHostAlloc or cudaHostRegister;
 * WX_EINVAL otherwise) and stay untouched until the stream has passed the
 * call; results are valid after the stream (or wx_sync) completes.  The
 * copies go through the context's device staging buffer in stream order.
 * Contexts on different streams overlap one's download with another's
 * upload (the host link has a copy engine each way). */
int wx_load_state_f32_async(wx_ctx *c, const float *T, const float *q, void *cuda_stream);
int wx_read_state_f32_async(wx_ctx *c, float *T, float *q, void *cuda_stream);

/* Copy the current state to host FP64 arrays T, q [nz][ny][nx] (either may
 * be NULL).  Synchronous; a checkpoint that wx_load_fields restores. */
int wx_read_fields(wx_ctx *c, double *T, double *q);

/* Same as wx_read_fields into device FP64 buffers. */
int wx_read_fields_device(wx_ctx *c, double *T, double *q, void *cuda_stream);

/* Sums recorded with WX_SUMS since the last load: mass_q[s] = h^2 sum q dz,
 * energy_T[s] = h^2 sum T dz after step s (FP64, deterministic order).
 * Copies up to max_steps of the most recent entries; *n_out gets the count.
 * Synchronous. */
int wx_get_sums(wx_ctx *c, double *mass_q, double *energy_T, int max_steps,
                int *n_out);

/* Column physics only (the per-column half of the step) on ncol >= 0
 * independent columns in device memory, in the context's storage type
 * (float for WX_F32/WX_MIXED, double for WX_F64):
 *   Tstar, qstar [ncol][nz] in; kappa_mult [ncol] in (NULL = 1);
 *   Tout [ncol][nz] out = T** + dt H;
 *   tend [ncol][2][nz] out or NULL: (H_k, (T**_k - T*_k)/dt).
 * Uses the context's per-level tables (wx_set_params first). Asynchronous. */
int wx_physics_columns(wx_ctx *c, const void *Tstar, const void *qstar,
                       const void *kappa_mult, void *Tout, void *tend,
                       long ncol, void *cuda_stream);

/* Grid and layout facts of a context (any out pointer may be NULL). */
int wx_info(const wx_ctx *c, int *nx, int *ny, int *nz, int *dtype,
            long *pitch_cells, long *device_bytes);

/* Launch configuration of the step kernel (the autotuner's knobs): tile
 * rows ty (1, 2, 4 or 8; a tile is 64 x ty columns), k-planes per TMA box
 * kb (2 or 4), ring slots stages (3..16), resident CTAs per SM (>= 1) and
 * an L2 bulk-prefetch distance in stages (0..64; 0 = off).  Rejected with
 * WX_EUNSUPPORTED when the shared-memory plan does not fit (ty = 1 with
 * kb = 4 is not built).  wx_get_step_config reads the current one (chosen
 * by a built-in heuristic until set). */
int wx_set_step_config(wx_ctx *c, int ty, int kb, int stages, int ctas_per_sm,
                       int prefetch);
int wx_get_step_config(const wx_ctx *c, int *ty, int *kb, int *stages,
                       int *ctas_per_sm, int *prefetch, int *smem_bytes);

/* The current T and q as device FP32 columns, T[col][k] and q[col][k] with
 * col = j*nx + i and k = 0 (bottom) .. nz-1, i.e. [nx*ny][nz] (an FP64
 * context rounds to FP32); either output may be NULL.  The column layout of
 * wx_physics_columns and the network's features.  Asynchronous on the
 * stream; WX_ESTATE before any load. */
int wx_read_columns_f32(wx_ctx *c, float *T, float *q, void *cuda_stream);

/* WX_MIXED: number of columns flagged for the FP64 elimination (dominance
 * ratio below dd_threshold), 0 for other contexts. */
int wx_flagged_columns(const wx_ctx *c, long *n_flagged);

/* Number of kernel launches the last wx_step issued. */
long wx_last_launches(const wx_ctx *c);

/* FP64 sums of caller-owned fields without any device allocation.  The
 * paper has no counterpart: this exists for callers that cannot allocate
 * device memory, such as plug-ins whose host application owns every device
 * byte through its own pool, or real-time loops that cannot accept the
 * implicit synchronisation, latency or possible failure of cudaMalloc.
 *   T, q     device arrays [nz][ny][nx], float (dtype WX_F32) or double
 *            (WX_F64);
 *   dz       device array [nz] of double (used at full FP64 precision for
 *            either dtype: FP32 fields are weighted by dz split into two
 *            floats with compensated products and sums);
 *   out      device array of 2 doubles: out[0] = h^2 sum q dz_k,
 *            out[1] = h^2 sum T dz_k (deterministic order).
 * Per-tile partial sums go to one fixed __device__ array inside the library
 * (1 MiB, held by each GPU that loads it until the process exits).  Limits:
 * at most 65536 tiles of 32x4 columns, and ny <= 4*65535 = 262140 (the tile
 * grid's row limit); larger grids are rejected with WX_EUNSUPPORTED.
 * Nothing has to be cleared between calls, but calls sharing that array
 * must not overlap on the GPU (they would race).  The first successful call
 * on a device looks up the array's address with that device current; make
 * it before any stream capture (a failed lookup is retried on the next
 * call).  Asynchronous on the stream.  Errors: WX_EINVAL, WX_EUNSUPPORTED,
 * WX_ECUDA; message in wx_sums_noalloc_error(). */
int wx_sums_noalloc(const void *T, const void *q, int dtype, int nx, int ny,
                    int nz, const double *dz, double h, double *out,
                    void *cuda_stream);

/* Message of the last failing wx_sums_noalloc call on this host thread. */
const char *wx_sums_noalloc_error(void);

/* Failure-detection self test: one kernel waits on a barrier that nothing
 * will complete, with the same bounded wait every kernel of the library
 * uses, limited to limit_ns (1 .. 2e9).  Returns WX_ETIMEOUT when the wait
 * gave up and reported it (the expected outcome), WX_OK if it completed;
 * waited_ns receives the device time spent waiting.  The CUDA context
 * stays usable either way.  WX_EINVAL for a zero or larger limit. */
int wx_selftest_wait_timeout(unsigned long long limit_ns,
                             unsigned long long *waited_ns);

/* ------------------------------------------- the paper's reduced application
 * The reduced weather application of Sec. 3.1 (Eq. 1, explicit Euler) with
 * the semantics of its appendix listings, for comparison with the paper's
 * own timings (Sec. 5.1): the state E[k][j][i], i in [0, nx+2), j in
 * [0, ny+2), k in [0, nz), includes a ghost ring that evolves by its own
 * two-neighbour rule; each step applies the physics (radiation added to
 * every level; Newtonian heat wells at the bottom and top levels) to every
 * column, then the diffusion (7-point interior rule, 1 - 5d at the bottom
 * and top levels, 1 - 2d two-neighbour rule on ghost rows and columns, the
 * corner columns taking the column rule), then swaps buffers. */
typedef struct wx_pf wx_pf;
/* nx, ny >= 1, nz >= 2; dtype WX_F64 (the paper's real(8)) or WX_F32.
 * The state starts at 0 K.  Parameters default to d = 0.1, radiation 0.1,
 * transfer 0.01, wells 330 K / 200 K.  WX_EINVAL, WX_EUNSUPPORTED,
 * WX_ENOMEM. */
int wx_pf_create(int nx, int ny, int nz, int dtype, wx_pf **out);
/* d = diffusion_velocity in [0, 1/6], transfer in [0, 1] (WX_ECFL
 * otherwise: the update stops being a convex combination). */
int wx_pf_set_params(wx_pf *p, double d, double radiation, double transfer,
                     double T_surf, double T_pbl);
/* Storage order on the device (WX_PF_IJK: i fastest, the default; WX_PF_KIJ:
 * k fastest, the paper's CPU order) and thread-block shape (block_x *
 * block_y threads, 32..512, a multiple of 32; default 32 x 8), for the
 * paper's storage-order and block-size experiments (Sec. 5.1.1, 5.1.4).
 * A loaded state is converted.  WX_EINVAL otherwise. */
enum { WX_PF_IJK = 0, WX_PF_KIJ = 1 };
int wx_pf_set_launch(wx_pf *p, int layout, int block_x, int block_y);
/* Copy the whole state in: FP64 [nz][ny+2][nx+2], host (src_is_device = 0)
 * or device memory; synchronous. */
int wx_pf_load(wx_pf *p, const double *E, int src_is_device);
/* Copy the state out to a host FP64 [nz][ny+2][nx+2] array (synchronises). */
int wx_pf_read(wx_pf *p, double *E);
/* n_steps >= 0 steps on the stream, one kernel launch each. */
int wx_pf_step(wx_pf *p, int n_steps, void *cuda_stream);
/* Wait for the last stream; WX_ENONFINITE if a step produced a non-finite
 * value since the last call. */
int wx_pf_sync(wx_pf *p);
long wx_pf_last_launches(const wx_pf *p);
void wx_pf_destroy(wx_pf *p);               /* NULL-safe */
const char *wx_pf_last_error(const wx_pf *p);

/* Autotune the step kernel's launch configuration for this context (grid,
 * dtype, options): candidate tile rows x planes per TMA box x ring slots x
 * CTAs per SM are each timed with CUDA events over a few steps on the
 * caller's stream, on a copy of the state that is restored afterwards, and
 * the fastest is applied.  cache_path (or NULL) names a text file that keeps
 * the winner per (GPU, dtype, options, grid); with force = 0 a cached entry
 * is applied without timing.  *best_ms (optional) gets its time per step.
 * Synchronous. */
int wx_tune(wx_ctx *c, const char *cache_path, int force, void *cuda_stream,
            double *best_ms);

/* ---------------------------------------------------------- ensembles
 * A batch of up to 16 member grids of uneven sizes (the same dtype and
 * options), stepped together: each step is ONE persistent launch of the
 * step kernel over the combined (member, tile) work list, followed by the
 * members' sums kernels when enabled.  Members are ordinary contexts owned
 * by the ensemble: set their parameters, load and read their fields with
 * the wx_* calls on wx_ens_member(e, i).  (The paper's ensemble context is
 * its many-GPU strong-scaling runs, Sec. 5.4; this batches independent
 * grids on one GPU.) */
typedef struct wx_ens wx_ens;

/* m in 1..16 members of sizes nx[i] x ny[i] x nz[i]; dtype WX_F32 or
 * WX_F64. */
int wx_ens_create(int m, const int *nx, const int *ny, const int *nz,
                  int dtype, wx_ens **out);
int wx_ens_size(const wx_ens *e);
/* Member i (owned by the ensemble; do not destroy it), NULL if out of range. */
wx_ctx *wx_ens_member(wx_ens *e, int i);
/* Advance every member n_steps >= 0 steps on the caller's stream.  With
 * use_graph = 1 the n_steps launches are captured once into a CUDA graph
 * (cached per step count, buffer parity, member state generation and
 * configuration) and replayed with one graph launch.  Members must share
 * their option flags and kappa_mult use (WX_EINVAL otherwise). */
int wx_ens_step(wx_ens *e, int n_steps, int use_graph, void *cuda_stream);
/* Wait for the last stream; WX_ETIMEOUT / WX_ENONFINITE as wx_sync. */
int wx_ens_sync(wx_ens *e);
/* One launch configuration for all members (see wx_set_step_config); it
 * must fit the member with the deepest columns. */
int wx_ens_set_step_config(wx_ens *e, int ty, int kb, int stages,
                           int ctas_per_sm, int prefetch);
int wx_ens_get_step_config(const wx_ens *e, int *ty, int *kb, int *stages,
                           int *ctas_per_sm, int *prefetch);
/* wx_tune for the whole batch (one configuration for the batched launch). */
int wx_ens_tune(wx_ens *e, const char *cache_path, int force,
                void *cuda_stream, double *best_ms);
/* Kernel launches the last wx_ens_step issued (per replay for graphs). */
long wx_ens_last_launches(const wx_ens *e);
void wx_ens_destroy(wx_ens *e);          /* NULL-safe; frees the members */
const char *wx_ens_last_error(const wx_ens *e);

/* ------------------------------------------ horizontal decomposition
 * The paper's multi-GPU layout of ASUCA (App. F decomposition table;
 * Sec. 5.4, the halo exchange's share of the strong-scaling runs): one
 * periodic nx x ny x nz grid split into px x py horizontal blocks (ASUCA
 * decomposes only in i and j, never in k).  Each block is a sub-domain
 * context with its own resident fields and ghost ring; a step is the step
 * kernel over every block (one launch over all blocks' tiles, like an
 * ensemble), then ONE halo-exchange launch that overwrites every block's
 * four depth-1 ghost strips (west and east
 * columns, south and north rows, for T and q at every level) from its
 * neighbours' edge lines.  Corners are not exchanged: the 7-point stencil
 * and the upwind fluxes never read them.  The blocks run as simulated
 * ranks on one GPU; the interior of every block is bit-for-bit the
 * undecomposed step's.  Sub-domain r = iy*px + ix covers columns
 * [xsplit[ix], xsplit[ix+1]) x [ysplit[iy], ysplit[iy+1]). */
typedef struct wx_dom wx_dom;

enum { WX_HALO_WEST = 0, WX_HALO_EAST = 1, WX_HALO_SOUTH = 2, WX_HALO_NORTH = 3 };

/* One ghost strip of a sub-domain: for every level and field, the ghost
 * line dst_line of sub-domain r (a column index -1 or nx_r for WEST/EAST, a
 * row index -1 or ny_r for SOUTH/NORTH, in r's local coordinates) receives
 * line src_line of sub-domain src (its last or first interior column or
 * row, in src's local coordinates); len cells (ny_r for columns, nx_r for
 * rows).  src == r where a block is its own periodic neighbour. */
typedef struct {
    int dir, src, src_line, dst_line, len;
} wx_halo_strip;

/* The four strips of sub-domain r (WEST, EAST, SOUTH, NORTH order) of a
 * px x py decomposition of an nx x ny grid.  xsplit[px+1] / ysplit[py+1]:
 * block boundaries, 0 = x_0 < x_1 < ... < x_px = nx (strictly increasing,
 * so blocks are >= 1 column wide), or NULL for the even split x_i =
 * floor(i nx / px).  Host-only bookkeeping (no CUDA call); the device
 * exchange is built from it.  WX_EINVAL for bad sizes or splits. */
int wx_dom_halo_plan(int nx, int ny, int px, int py, const int *xsplit,
                     const int *ysplit, int r, wx_halo_strip out[4]);

/* px * py in 1..16 blocks; dtype WX_F32, WX_F64 or WX_MIXED.  WX_EINVAL,
 * WX_EUNSUPPORTED, WX_ENOMEM, WX_ECUDA; message in wx_dom_last_error(NULL). */
int wx_dom_create(int nx, int ny, int nz, int dtype, int px, int py,
                  const int *xsplit, const int *ysplit, wx_dom **out);
/* Parameters of the whole grid (kappa_mult [ny*nx] is split per block).
 * WX_RK3 and WX_SURROGATE are refused (WX_EUNSUPPORTED). */
int wx_dom_set_params(wx_dom *d, const wx_params *p);
/* Host FP64 arrays of the whole grid: T, q [nz][ny][nx]; U, V [ny][nx].
 * Scatters them to the blocks (with each block's west/south face winds
 * from its neighbours) and runs the exchange once.  Synchronous. */
int wx_dom_load_fields(wx_dom *d, const double *T, const double *q,
                       const double *U, const double *V);
/* n_steps >= 0 steps on the caller's stream, 2 launches per step (plus the
 * blocks' side solves and sums kernels where enabled); asynchronous. */
int wx_dom_step(wx_dom *d, int n_steps, void *cuda_stream);
/* Wait for the last stream; WX_ETIMEOUT / WX_ENONFINITE as wx_sync. */
int wx_dom_sync(wx_dom *d);
/* Gathers the blocks' states into host FP64 arrays of the whole grid
 * (either may be NULL).  Synchronous. */
int wx_dom_read_fields(wx_dom *d, double *T, double *q);
/* The whole grid's FP64 sums per recorded step (WX_SUMS): each block's
 * recorded sums, added in block order r = 0, 1, ... (the 2-double
 * reduction a multi-GPU run would do across ranks).  As wx_get_sums. */
int wx_dom_get_sums(wx_dom *d, double *mass_q, double *energy_T,
                    int max_steps, int *n_out);
int wx_dom_size(const wx_dom *d);          /* px * py, 0 for NULL */
/* Block r (owned by the decomposition; read-only use: stepping it alone
 * would leave its ghost ring stale), NULL if out of range. */
wx_ctx *wx_dom_block(wx_dom *d, int r);
long wx_dom_last_launches(const wx_dom *d);
void wx_dom_destroy(wx_dom *d);            /* NULL-safe; frees the blocks */
const char *wx_dom_last_error(const wx_dom *d);

/* ----------------------------------------------- learned column physics
 * A small MLP surrogate of the column physics (232 -> 512 -> 512 -> 512 ->
 * 116, exact-erf GELU): BF16 weights and activations, FP32 accumulation in
 * tensor memory, hand-written tcgen05 GEMMs.  The paper has no learned
 * part; this follows the batched per-column interface of its physics
 * (Sec. 3.1: every K column is processed independently). */

/* C[M][N] = A[M][K] . B[N][K]^T on device BF16 operands (both K-major),
 * FP32 accumulation; M, N multiples of 128, K of 64.  epilogue:
 *   0  out (f32)  = C + bias (bias may be NULL)
 *   1  out (bf16) = GELU(C + bias), out2 (bf16) = C + bias (out2 may be
 *      NULL: the pre-activation is then not stored)
 *   2  out (bf16) = C * GELU'(aux), aux (bf16 [M][N]) = the saved C + bias
 *   3  out (bf16) = C + bias (bias may be NULL)
 * status: device word that receives WX_ETIMEOUT's bit on a bounded-wait
 * timeout.  Asynchronous on the stream. */
int wx_gemm_bf16(const void *A, const void *B, int M, int N, int K,
                 int epilogue, const float *bias, const void *aux, void *out,
                 void *out2, unsigned *status, void *cuda_stream);

/* Message of the last failing wx_gemm_bf16 / wx_mlp_* call on this thread. */
const char *wx_mlp_last_error(void);

/* The surrogate network.  Layer l maps fan_in(l) -> fan_out(l) with
 * (232, 512), (512, 512), (512, 512), (512, 116); weights are FP32 masters
 * with BF16 copies, [fan_out][fan_in] row-major on the host side of the
 * get/set calls.  Inputs x = [T*_k | q*_k | kappa_mult kappa_lev(k) |
 * alpha_k dz_k] (k = 0..57, bottom first) are normalised per feature;
 * outputs y = [H_k | (T**_k - T*_k)/dt] likewise, where T** is the implicit
 * vertical diffusion's result and H the radiative heating (Sec. 3.1's
 * column physics, Eq. 1).  On the device, a normalised input row is 512
 * BF16 values: the two-term expansion x = hi + lo of every feature,
 * hi = bf16(x) in [0, 232) and lo = bf16(x - hi) in [256, 488), zeros
 * elsewhere; the first layer applies its weights to both halves.  Outputs
 * are FP32 rows of 128 (116 used).  Row counts are multiples of 128. */
typedef struct wx_mlp wx_mlp;
/* Allocate a network whose training and activation buffers hold max_batch
 * rows (multiple of 128); weights zero, normalisation identity. */
int wx_mlp_create(int max_batch, wx_mlp **out);
void wx_mlp_destroy(wx_mlp *m);                    /* NULL-safe */
/* Host FP32 weights W[l] ([fan_out][fan_in]) and biases b[l] (4 each);
 * resets the Adam moments and step count. */
int wx_mlp_set_weights(wx_mlp *m, const float *const *W, const float *const *b);
int wx_mlp_get_weights(wx_mlp *m, float *const *W, float *const *b);
/* Gradients of the last wx_mlp_gradients / wx_mlp_train_step (host FP32,
 * same layout as the weights). */
int wx_mlp_get_grads(wx_mlp *m, float *const *dW, float *const *db);
/* Normalisation: host mean/std of the 232 inputs and of the 116 outputs. */
int wx_mlp_set_norm(wx_mlp *m, const float *mean_in, const float *std_in,
                    const float *mean_out, const float *std_out);
int wx_mlp_get_norm(wx_mlp *m, float *mean_in, float *std_in,
                    float *mean_out, float *std_out);
/* Per-level constants of the features: kappa_lev[58] and alpha*dz [58]
 * (host); nz must be 58 (WX_EUNSUPPORTED otherwise). */
int wx_mlp_set_levels(wx_mlp *m, int nz, const float *kappa_lev,
                      const float *alpha_dz);
/* Fit the normalisation to a training set on the device: T*, q* [ncol][58],
 * kappa_mult [ncol] (NULL = 1), tend [ncol][2][58] as written by
 * wx_physics_columns.  Per-feature mean and population standard deviation
 * in FP64 (floor 1e-6 |mean|).  Asynchronous. */
int wx_mlp_fit_norm(wx_mlp *m, const float *Ts, const float *qs,
                    const float *kappa_mult, const float *tend, long ncol,
                    void *cuda_stream);
/* Normalised BF16 input rows X [ceil128(ncol)][512] and, when tend and Yt
 * are given, FP32 target rows Yt [ceil128(ncol)][128] of device columns
 * (padding rows zero).  Asynchronous. */
int wx_mlp_prepare(wx_mlp *m, const float *Ts, const float *qs,
                   const float *kappa_mult, const float *tend, long ncol,
                   void *X, float *Yt, void *cuda_stream);
/* Normalised outputs Y [M][128] (FP32) of BF16 rows X [M][512]; any M that
 * is a multiple of 128 (processed in chunks of max_batch). */
int wx_mlp_forward(wx_mlp *m, const void *X, int M, float *Y,
                   void *cuda_stream);
/* Forward and backward of the mean-squared error over the 116 outputs of
 * M rows (M multiple of 128, <= max_batch): gradients into the network's
 * buffers; loss (device float or NULL) = the batch loss. */
int wx_mlp_gradients(wx_mlp *m, const void *X, const float *Yt, int M,
                     float *loss, void *cuda_stream);
/* wx_mlp_gradients followed by one Adam step (beta1 0.9, beta2 0.999,
 * eps 1e-8, bias-corrected) at learning rate lr on the FP32 masters; BF16
 * copies refreshed. */
int wx_mlp_train_step(wx_mlp *m, const void *X, const float *Yt, int M,
                      float lr, float *loss, void *cuda_stream);
/* WX_OK, or WX_ETIMEOUT if a bounded device wait of a GEMM gave up since the
 * last call (synchronises). */
int wx_mlp_status(wx_mlp *m);
/* Physical-unit outputs of M rows of normalised outputs Y [M][128]:
 * out[r][o] = Y[r][o] std_out[o] + mean_out[o] for the 116 outputs (out
 * [M][116], device FP32).  Asynchronous. */
int wx_mlp_denormalize(wx_mlp *m, const float *Y, long M, float *out,
                       void *cuda_stream);

/* Device data movement for the training driver (no arithmetic of the
 * method): element conversion of n values FP32 -> FP64 (to_f64 = 1) or
 * FP64 -> FP32 (0, round to nearest); and a row gather dst[r] = src[idx[r]]
 * of n rows of row_bytes bytes (a multiple of 16, both arrays 16-byte
 * aligned; idx device int32; an index outside [0, src_rows) gives a zero
 * row).  Asynchronous; WX_EINVAL for bad arguments, message in
 * wx_mlp_last_error(). */
int wx_convert(const void *src, void *dst, long n, int to_f64,
               void *cuda_stream);
int wx_gather_rows(const void *src, long src_rows, long row_bytes,
                   const int *idx, long n, void *dst, void *cuda_stream);

/* The training driver's minibatch order: out[0..n) = a permutation of
 * 0..n-1 (host memory, n <= 2^31 - 1), Fisher-Yates from the top with the
 * splitmix64 generator (Steele, Lea and Flood, OOPSLA 2014) seeded with
 * `seed`; draw r for position i is the high 64 bits of u * (i + 1) (Lemire's
 * multiply-shift, bias below (i + 1) / 2^64).  The same (n, seed) gives the
 * same permutation on every host.  Host only: no CUDA call.  WX_EINVAL for
 * n < 0, n > 2^31 - 1 or a NULL out with n > 0. */
int wx_permutation(long n, unsigned long long seed, int *out);

/* Attach (m != NULL) or detach (NULL) a trained network to an FP32 context
 * with nz = 58.  With WX_SURROGATE in the flags, each wx_step then runs the
 * dynamics, predicts the column physics with the network and accepts a
 * column's prediction only if both residuals stay within fallback_tol:
 *   rho_vd = ||A x - T*|| / ||A T* - T*||  (A = the implicit vertical-
 *            diffusion matrix of the column, x = T* + dt y_vd);
 *   rho_H  = |sum_k H_k dz_k - S0 (1 - exp(-tau_tot))| / (S0 (1 - exp(-tau_tot))).
 * Rejected columns are recomputed exactly (Thomas sweep and scan).  The
 * network must outlive the attachment; the context owns its own activation
 * buffers.  WX_SURROGATE excludes WX_SUMS. */
int wx_set_surrogate(wx_ctx *c, wx_mlp *m, double fallback_tol);
/* Columns the residual check sent to the exact path in the last step, or
 * nx*ny when the acceptance policy ran that step exactly (synchronises). */
int wx_surrogate_fallbacks(wx_ctx *c, long *n_fallback);
/* Acceptance policy of WX_SURROGATE steps (the paper has no learned part;
 * this keeps the method's exact physics as the fallback).  With
 * min_accept = 0 (the default) the network runs on every step.  With
 * min_accept in (0, 1], a step whose measured acceptance (columns accepted
 * / columns) falls below min_accept switches the following steps to the
 * exact fused step (dynamics and column physics in one kernel, as without
 * WX_SURROGATE); every probe_every exact steps the network is evaluated on
 * a band of probe_rows rows of the new state (the next band each time),
 * counting the columns its residual checks would accept, and an acceptance
 * of at least min_accept switches back to network steps.  A decision uses
 * the counts of the step two before it, read back through pinned memory:
 * no device synchronisation in the step, and the same sequence of steps
 * always takes the same decisions.  The policy's measurements restart at
 * every state load and at wx_set_surrogate.  min_accept in [0, 1],
 * probe_every >= 1, probe_rows >= 1 (clamped to ny), else WX_EINVAL. */
int wx_set_surrogate_policy(wx_ctx *c, double min_accept, int probe_every,
                            int probe_rows);

/* Free the context and its device memory.  NULL-safe. */
void wx_destroy(wx_ctx *c);

/* Message of the last failing call on c (or of the last failed wx_create
 * when c is NULL).  Valid until the next call on c. */
const char *wx_last_error(const wx_ctx *c);

#ifdef __cplusplus
}
#endif
#endif
