/*
 * bsq.h -- C ABI of the GB300 (sm_103a) extended Boussinesq solver with
 * variable-step third-order Adams-Bashforth time stepping
 * (Tavakkol, Son & Lynett, arXiv 1909.04153).
 *
 * One call advances a domain: the 2D Madsen-Sorensen equations (Sec. 2,
 * Eqs. 1-3) in the Wei-Kirby form (Sec. 3.1, Eqs. 6-15) on a uniform grid with
 * two ghost layers per side (Sec. 3.3), hyperbolic part by the central-upwind
 * scheme of Kurganov-Petrova (Sec. 3), dispersive part by central differences,
 * P and Q recovered from tridiagonal line systems (Eqs. 19-21), the step size
 * from the CFL rule (Eq. 22) with the lazy moving average (Eq. 47), and the
 * variable-step AB3 update (Eqs. 42-46).
 *
 * Conventions
 *   - Every call returns a bsq_status; no call aborts the process.
 *   - Inputs are copied; outputs go to caller-owned buffers.
 *   - Host arrays are row-major with x fastest: element (i, j) at i + j*nx.
 *   - A domain handle is not thread-safe; all its work runs on one CUDA stream.
 *   - The first error is sticky: later calls on that domain return it until
 *     bsq_destroy.
 *   - Waits for the device are bounded (bsq_params.timeout_s) and end with
 *     BSQ_ERR_TIMEOUT; no call spins forever.
 *   - The library allocates its device memory with cudaMalloc at bsq_create
 *     and frees it in bsq_destroy; bsq_advance and bsq_step_dt allocate nothing.
 */
#ifndef BSQ_H
#define BSQ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bsq_domain bsq_domain;

typedef enum {
    BSQ_OK = 0,
    BSQ_ERR_ARG = 1,        /* invalid argument or size */
    BSQ_ERR_OOM = 2,        /* device or host allocation failed */
    BSQ_ERR_CUDA = 3,       /* a CUDA runtime call failed */
    BSQ_ERR_NONFINITE = 4,  /* a non-finite value appeared in the state */
    BSQ_ERR_UNSTABLE = 5,   /* the CFL step fell below dt_min */
    BSQ_ERR_TIMEOUT = 6,    /* a bounded wait for the device ran out */
    BSQ_ERR_STATE = 7       /* call not valid in the current state */
} bsq_status;

enum { BSQ_FP32 = 0, BSQ_FP64 = 1 };

/* Boundary types per side (Sec. 3.3).  A sponge side is a reflective wall
 * with an absorbing band of width sponge_width inside the domain. */
enum { BSQ_BC_WALL = 0, BSQ_BC_SPONGE = 1, BSQ_BC_MAKER = 2 };

/* Sides, in this order, in bsq_boundary.type and sponge_width. */
enum { BSQ_WEST = 0, BSQ_EAST = 1, BSQ_SOUTH = 2, BSQ_NORTH = 3 };

/* Fields for bsq_read. ETA = h - d with h = max(w - b, 0), d = max(w_s - b, 0). */
enum { BSQ_FIELD_ETA = 0, BSQ_FIELD_P = 1, BSQ_FIELD_Q = 2, BSQ_FIELD_H = 3, BSQ_FIELD_W = 4 };

/* Cross-term forms for the time derivatives of F*(Q) and G*(P) (Eqs. 7-8).
 * EXTRAPOLATED: both extrapolated in time with the variable-step differences
 *   of Eqs. 44-46 inside Eq. 43, exactly as printed (Eqs. 17-18 at fixed step);
 *   unstable in 2D once the still depth exceeds about 1.5 grid cells.
 * SEQUENTIAL (default): G* as printed; Q^{n+1} is solved first and F* is
 *   evaluated at the new level from Q^{n+1}; stable at any depth. */
enum { BSQ_CROSS_EXTRAPOLATED = 0, BSQ_CROSS_SEQUENTIAL = 1 };

typedef struct {
    int nx, ny;            /* interior cells; 3 <= nx, ny <= 16384 */
    double dx, dy;         /* cell sizes (m) */
    double g;              /* gravity, 9.81 */
    double Bd;             /* dispersion coefficient B of Eqs. 2-3, 1/15 */
    double cfl;            /* target CFL of Eq. 22; 0: fixed steps of dt_init (constant-step
                              AB3, Eqs. 16-18: the weights of Eq. 42 at equal steps) */
    double ema_alpha;      /* alpha of Eq. 47 (0 < alpha <= 1) */
    double dt_init;        /* first step; <= 0: from Eq. 22 (with cfl = 0: every step) */
    double dt_min;         /* a CFL step below this is BSQ_ERR_UNSTABLE */
    double dt_max;         /* upper clamp; <= 0: none */
    double friction;       /* quadratic bottom friction factor f (f1 = f u |u|) */
    double theta;          /* generalized minmod parameter, 1 = minmod (Sec. 3.4) */
    double eps;            /* desingularisation epsilon; <= 0: max(dx,dy)^4 */
    double w_s;            /* still water elevation above the datum */
    double ramp_time;      /* wave maker ramp r(t) = tanh(3 t / ramp_time); <= 0: none */
    double timeout_s;      /* bound of each host wait for the device; <= 0: 600 s */
    int precision;         /* BSQ_FP32 or BSQ_FP64 */
    int kahan;             /* FP32: compensated accumulation of w, P, Q increments */
    int cross_mode;        /* BSQ_CROSS_* */
    int graph_steps;       /* steps per captured CUDA graph in bsq_advance; <= 0: 16 */
    int tune[8];           /* kernel shape knobs, 0 = default: [0], [1] reserved;
                              [2] x-solver: bit 1 registers only (no staging), bit 3 the
                              persistent solver with two staged rows (the double-precision
                              default where its rows fit), bit 4 one warp per row (the
                              single-precision default); [3] rows per warp of the
                              sliding-window RHS (16, 24, 32, 48, 64, 128; 16 selects the
                              one-column kernel, which takes 24 and 48 as 32; 128: 128-row
                              strips of the one-column kernel where it forms 8-row chunk
                              summaries itself, else 64; 0: by grid size); [4] x-solver elements per thread (4, 8, 16, 32);
                              [5] rows per y-line chunk (8, 16); [6] bit 0: the chunk
                              summaries by a kernel of their own instead of inside the RHS
                              kernel, bit 1: one column per lane in the single-precision RHS
                              kernel (instead of two, paired); [7] reserved */
} bsq_params;

/* Most wave-maker components a domain takes. */
#define BSQ_MAX_COMP 1024

typedef struct {
    int type[4];               /* BSQ_BC_* per side W, E, S, N */
    double sponge_width[4];    /* band width (m) of sponge sides */
    int n_comp;                /* wave-maker components (0 if no maker side; at most
                                  BSQ_MAX_COMP) */
    const double *amp;         /* amplitude (m) */
    const double *freq;        /* frequency (Hz) */
    const double *phase;       /* phase (rad) */
    const double *dir;         /* direction of travel (rad, 0 = +x) */
} bsq_boundary;

/* Fill *p with the defaults (g 9.81, Bd 1/15, cfl 0.125, alpha 0.1, theta 1,
 * FP32 with Kahan, sequential cross terms); nx, ny, dx, dy are left zero. */
void bsq_params_default(bsq_params *p);

/* Create a domain (Sec. 3.3 grid with two ghost layers per side).
 *   bed_corners: (nx+1)*(ny+1) bed elevations at cell corners, corner (i,j) at
 *                (i dx, j dy); mirrored outward for the ghost cells; copied.
 *   bnd:         boundary spec; NULL = walls on all sides; arrays copied.
 *   eta0, P0, Q0: nx*ny initial surface (eta = h - d) and fluxes, or NULL (0).
 *                The initial depth is h = max(d + eta0, 0).
 *   cuda_stream: cudaStream_t to run on; NULL = a stream the library creates.
 *   out:         receives the handle; owned by the caller until bsq_destroy.
 * Errors: BSQ_ERR_ARG (bad sizes, tridiagonal rows not diagonally dominant),
 * BSQ_ERR_OOM, BSQ_ERR_CUDA.  On error *out is NULL. */
bsq_status bsq_create(const bsq_params *p, const double *bed_corners, const bsq_boundary *bnd,
                      const double *eta0, const double *P0, const double *Q0,
                      void *cuda_stream, bsq_domain **out);

/* Advance with adaptive steps (Eqs. 22, 47; AB3 of Eqs. 42-46 after the Euler
 * start of Sec. 3.2.1) until t = t_end (the last step is clamped to land on
 * t_end) or max_steps more steps were taken (<= 0: no limit; then t_end must
 * be finite).  *steps_done (may be NULL) receives the number taken.  Runs
 * captured CUDA graphs of graph_steps steps and graphs of 1, 2, 4, ... steps
 * for the remainder (the domain's first call launches its steps one by one
 * while it captures the graphs): with max_steps it enqueues exactly max_steps
 * step slots, toward t_end about the steps the last step size says are left,
 * and slots past the end do no work.  Errors: BSQ_ERR_ARG, BSQ_ERR_NONFINITE,
 * BSQ_ERR_UNSTABLE, BSQ_ERR_TIMEOUT, BSQ_ERR_CUDA. */
bsq_status bsq_advance(bsq_domain *d, double t_end, long long max_steps, long long *steps_done);

/* Take n steps with the given step sizes dts[0..n-1] (host array, each > 0 and
 * finite) instead of the CFL rule of Eq. 22 and the moving average of Eq. 47:
 * replays a recorded dt sequence through the same update (Euler start of
 * Sec. 3.2.1, then the variable-step weights of Eqs. 42-46 for those steps).
 * The steps are launched one by one (no graph).  Errors: BSQ_ERR_ARG (NULL
 * dts with n > 0, n < 0, a step not > 0), BSQ_ERR_NONFINITE, BSQ_ERR_TIMEOUT,
 * BSQ_ERR_CUDA. */
bsq_status bsq_step_dt(bsq_domain *d, const double *dts, long long n);

/* Copy one field of the interior (BSQ_FIELD_*) to host_out (nx*ny doubles,
 * caller-owned, row-major with x fastest).  The state variables are those of
 * Eq. 5 (w, P = hu, Q = hv); ETA is h - d of Sec. 2 with h = max(w - b, 0)
 * and d = max(w_s - b, 0), H is h, W is w.  FP32 values are widened to
 * double.  Waits for the domain's stream (bounded).  Errors: BSQ_ERR_ARG
 * (NULL, unknown field), BSQ_ERR_TIMEOUT, BSQ_ERR_CUDA, the sticky error. */
bsq_status bsq_read(const bsq_domain *d, int field, double *host_out);

/* Copy one field of the interior to device memory dev_out (nx*ny elements of
 * the domain's precision, caller-owned), enqueued on the domain's stream. */
bsq_status bsq_read_device(const bsq_domain *d, int field, void *dev_out);

/* Simulated time t_n, steps taken n, the last step size dt_{n-1} (Eq. 22
 * with Eq. 47), the water volume sum(h) dx dy (conserved by the finite-volume
 * update of Sec. 3 in a closed basin) and the number of positivity clamps (w
 * raised to b after an update, keeping h >= 0 as Sec. 3.5 requires) so far.
 * Any pointer may be NULL.  Waits for the domain's stream (bounded).  Errors:
 * BSQ_ERR_ARG (NULL domain), BSQ_ERR_TIMEOUT, BSQ_ERR_CUDA. */
bsq_status bsq_info(const bsq_domain *d, double *t, long long *n, double *last_dt, double *mass,
                    long long *clamps);

/* Checkpoint: with buf NULL, *len receives the size needed.  Otherwise writes
 * the full state (fields, compensation terms, AB3 history, step sizes, time)
 * into buf (*len bytes available) and sets *len.  Restore puts it back into a
 * domain created with the same parameters; the continued run is bitwise the
 * same as one that was never interrupted. */
bsq_status bsq_checkpoint(const bsq_domain *d, void *buf, size_t *len);
bsq_status bsq_restore(bsq_domain *d, const void *buf, size_t len);

/* Release everything; NULL-safe. */
void bsq_destroy(bsq_domain *d);

/* Static text for a status code. */
const char *bsq_status_string(bsq_status s);

/* Device bytes held by the domain (state, history, scratch, static fields). */
size_t bsq_device_bytes(const bsq_domain *d);

/* Kernel timing: takes n_steps adaptive steps kernel by kernel (no graph),
 * with CUDA events recorded on the domain's stream around every launch, and
 * writes the mean duration (ms) of each kernel of the step to ms_out[k]
 * (ms_out holds at least 8 doubles); *n_kernels receives the number of
 * kernels and bsq_kernel_name(k) their names.  The steps are real steps:
 * the simulation advances by n_steps. */
bsq_status bsq_profile_kernels(bsq_domain *d, long long n_steps, double *ms_out, int *n_kernels);
const char *bsq_kernel_name(int k);

/* Measured FP64 fused multiply-add rate of the current device (TFLOP/s, 2
 * flops per FMA) from a short kernel of independent FMA chains (about 1 ms);
 * the roof for the double-precision path, which on this device is bound by
 * FP64 arithmetic, not memory.  Errors: BSQ_ERR_ARG, BSQ_ERR_CUDA. */
bsq_status bsq_fp64_fma_rate(double *tflops);

/* Kernel launches one step makes (each a node of the captured graphs);
 * 0 for a NULL handle. */
int bsq_launches_per_step(const bsq_domain *d);

/* ---- Batches: many domains advanced together (one launch per stage).
 *
 * The per-step update of every member is the single-domain one (Sec. 3, Eqs.
 * 5-22, 42-47), each member with its own adaptive dt, AB3 history, time and
 * limits: the batch only changes how the work is launched.  Every stage of a
 * step (ghost cells, RHS + combine, the three y-line launches, the x-line
 * solves) is one kernel launch over the blocks of all members, captured in
 * CUDA graphs of graph_steps steps; a member that has reached its t_end or
 * step limit (or failed) does no work in later steps while the others go on.
 * The batch does not own the domains: they stay valid handles (bsq_read,
 * bsq_info, bsq_checkpoint, bsq_advance on their own), must outlive the batch,
 * and must not be used on their own while a batch call runs.  x-lines use the
 * warp-per-row solver, so a member advanced alone gives the same result
 * bitwise when created with tune[2] = 16 (and otherwise the same result up to
 * rounding order). */
typedef struct bsq_batch bsq_batch;

/* Group n distinct domains of the same precision, Kahan setting and cross
 * mode, created with default tune[0], [1], [4], [5], rows of at most 6144
 * (FP32) / 3072 (FP64) cells and ny <= 2048.  cuda_stream: the stream batch
 * calls run on; NULL = a stream the library creates.  Builds the per-stage
 * block tables on the device.  Errors: BSQ_ERR_ARG (mixed or unsupported
 * members, a member in an error state, repeated handles), BSQ_ERR_OOM,
 * BSQ_ERR_CUDA.  On error *out is NULL. */
bsq_status bsq_batch_create(bsq_domain *const *domains, int n, void *cuda_stream, bsq_batch **out);

/* Advance every member d until its own t_end[d] (NULL: no time limit for all)
 * or max_steps more steps (<= 0: no step limit; then every t_end must be
 * finite).  steps_done (NULL or n entries) receives the steps each member took.
 * Waits (bounded) for each member's own stream first.  A member that fails
 * (BSQ_ERR_NONFINITE, BSQ_ERR_UNSTABLE) stops, keeps that status as its sticky
 * error, and the others finish; the first such status is returned.  Other
 * errors: BSQ_ERR_ARG, BSQ_ERR_TIMEOUT, BSQ_ERR_CUDA. */
bsq_status bsq_batch_advance(bsq_batch *b, const double *t_end, long long max_steps, long long *steps_done);

/* Autotuner of the batch's tile shapes: times every combination of RHS rows
 * per warp (64, 32), x-line elements per lane (8, 4; FP64: 4) and y-line rows
 * per chunk (8, 16) over steps_per_trial steps (plus one warm-up graph) on
 * the batch itself -- real steps: every member advances -- and keeps the
 * fastest.  choice (NULL or 3 ints) receives {rows, x elements, y rows}.  The
 * shapes change the rounding order of the line solves, not the method. */
bsq_status bsq_batch_autotune(bsq_batch *b, long long steps_per_trial, int *choice);

/* Replace the batch's members by n other domains (same rules as
 * bsq_batch_create; precision, Kahan setting and cross mode those of the
 * batch), keeping its stream, its buffers (grown when needed), its tile shapes
 * and its executable CUDA graph, which the next bsq_batch_advance updates in
 * place when the launch sequence allows it.  Waits for the batch's stream
 * first.  Errors: BSQ_ERR_ARG, BSQ_ERR_OOM, BSQ_ERR_CUDA; on error the batch
 * must be destroyed. */
bsq_status bsq_batch_reset(bsq_batch *b, bsq_domain *const *domains, int n);

/* Members of the batch; kernel launches per batched step. */
int bsq_batch_size(const bsq_batch *b);
int bsq_batch_launches_per_step(const bsq_batch *b);

/* Release the batch (not its domains); NULL-safe. */
void bsq_batch_destroy(bsq_batch *b);

/* Time and step count of the domain as of the end of its last advance call
 * (bsq_advance, bsq_step_dt or bsq_batch_advance; 0 after bsq_create), from
 * the host copy: no device work and no wait.  Returns the domain's status
 * (its sticky error, or the error its last advance ended with). */
bsq_status bsq_clock(const bsq_domain *d, double *t, long long *n);

/* Device bytes bsq_create allocates for these parameters with n_comp wave-
 * maker components (0 for sizes bsq_create rejects). */
size_t bsq_domain_bytes(const bsq_params *p, int n_comp);

/* ---- Serving: continuous batching of simulation requests.
 *
 * A request is a domain (same arguments as bsq_create) and an end time.
 * Submitted requests wait in a first-come-first-served queue on the host; a
 * poll admits requests while a slot is free and their device bytes
 * (bsq_domain_bytes) fit the budget next to those held, rebuilds the batch
 * when its membership changed, advances all running requests together by
 * steps_per_round steps (each with its own adaptive dt, Eqs. 22, 47), and
 * retires those that reached their end time.  A finished request keeps its
 * device memory (and its share of the budget) until bsq_server_release.
 * Every request's result is the same as when it is served alone.  One host
 * thread drives a server; calls are not thread-safe. */
typedef struct bsq_server bsq_server;

typedef struct {
    size_t hbm_budget;    /* device bytes all admitted requests may hold; 0: no limit */
    int max_slots;        /* requests advanced together at most; <= 0: 64 */
    int steps_per_round;  /* steps per bsq_server_poll; <= 0: 32 */
    int precision;        /* BSQ_FP32 or BSQ_FP64: every request's precision */
    int kahan;            /* FP32: every request's Kahan setting */
    void *cuda_stream;    /* stream of every request and batch; NULL: library streams */
} bsq_server_config;

enum { BSQ_REQ_PENDING = 0, BSQ_REQ_RUNNING = 1, BSQ_REQ_DONE = 2, BSQ_REQ_FAILED = 3 };

bsq_status bsq_server_create(const bsq_server_config *cfg, bsq_server **out);

/* Queue a request; the inputs are copied (host memory until admission).
 * Requests must use the server's precision and Kahan setting, the
 * sequential cross form, default tune, ny <= 2048 and rows the batched
 * x-solver holds; t_end > 0 finite; a request larger than the whole budget is
 * refused (BSQ_ERR_ARG).  *id receives the request id (> 0). */
bsq_status bsq_server_submit(bsq_server *s, const bsq_params *p, const double *bed_corners,
                             const bsq_boundary *bnd, const double *eta0, const double *P0, const double *Q0,
                             double t_end, long long *id);

/* One round: admit, advance, retire.  n_running / n_pending (may be NULL)
 * receive the counts after the round.  A request that fails (creation, or a
 * non-finite state) is finished as BSQ_REQ_FAILED with its status; the call
 * itself fails only for errors of the batch (BSQ_ERR_CUDA, BSQ_ERR_TIMEOUT). */
bsq_status bsq_server_poll(bsq_server *s, int *n_running, int *n_pending);

/* State (BSQ_REQ_*), simulated time and steps (as of the last poll) and
 * status of a request.  BSQ_ERR_ARG for an unknown or released id. */
bsq_status bsq_server_request(const bsq_server *s, long long id, int *state, double *t, long long *steps,
                              int *status);

/* Read a field of a finished request (as bsq_read); BSQ_ERR_STATE if it is
 * not BSQ_REQ_DONE. */
bsq_status bsq_server_read(const bsq_server *s, long long id, int field, double *host_out);

/* Free a finished (or failed) request's device memory and forget it;
 * BSQ_ERR_STATE while it is pending or running. */
bsq_status bsq_server_release(bsq_server *s, long long id);

/* Device bytes held by admitted, not yet released requests. */
size_t bsq_server_bytes_in_use(const bsq_server *s);

/* Release everything (queued requests, domains, the batch); NULL-safe. */
void bsq_server_destroy(bsq_server *s);

/* Allocation-free variant of the volume reduction that bsq_info's mass uses.
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc, such as an application that owns every byte of device memory
 * through its own pool or budget, or code whose stream another component may
 * be capturing into a CUDA graph, where a device allocation would fail or
 * disturb that owner.  It computes sum over cells of max(w - b, 0) * dx * dy
 * for caller-owned device arrays w and b (precision BSQ_FP32 or BSQ_FP64,
 * ny rows of nx values, rows pitch elements apart) and writes the double to
 * the caller's device pointer mass_dev, enqueued on cuda_stream (NULL = the
 * default stream); it does not wait for the result.
 *   - Scratch: the per-row partial sums live in a fixed file-scope device
 *     array of BSQ_NOALLOC_MAX_ROWS doubles (128 KiB), held on every device
 *     that loads the library until the process exits.  ny above that limit
 *     returns BSQ_ERR_ARG without touching the device.
 *   - Set-up: the first call on a device looks up the array's device address
 *     with that device current; make that first call before any stream
 *     capture begins.
 *   - All calls share the one array, and each call overwrites it, so calls
 *     that overlap on the GPU (different streams, or threads) race: order them.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.
 * Errors: BSQ_ERR_ARG (NULL pointer, bad sizes, ny too large), BSQ_ERR_CUDA. */
#define BSQ_NOALLOC_MAX_ROWS 16384
bsq_status bsq_mass_noalloc(int precision, const void *w_dev, const void *b_dev, int nx, int ny,
                            long long pitch, double dx, double dy, double *mass_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* BSQ_H */
