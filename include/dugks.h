/*
 * dugks.h -- C ABI of libdugks.so: the discrete unified gas-kinetic scheme
 * (DUGKS) time step for the conservative Allen-Cahn equation on a uniform,
 * periodic 2D D2Q9 grid, on one GB300 GPU (sm_103a).
 *
 * Method: Yang, Zhong & Zhuo, "Performance evaluation of high-order
 * reconstruction for discrete unified gas-kinetic scheme in tracking fluid
 * interfaces". Equation numbers below are the paper's.
 *
 * Conventions shared by every call:
 *  - Cells are unit squares (Sec. III: "cell size of unity"); cell (i, j) has its
 *    centre at (i + 1/2, j + 1/2); host arrays are row-major, x fastest, ny * nx.
 *  - D2Q9 velocities xi_k = e_k in the order (0,0),(1,0),(1,1),(0,1),(-1,1),
 *    (-1,0),(-1,-1),(0,-1),(1,-1); RT = 1/3; tau = M / RT; dt = cfl (Eq. (39)).
 *  - Every call returns a dugks_status_code. Errors of asynchronous device work are
 *    sticky: they are recorded in the context and returned by the next call
 *    that synchronises (dugks_read_phi, dugks_mass, dugks_save_state,
 *    dugks_status). After an error, dugks_last_error() describes it.
 *  - A context owns all of its device memory; every host pointer stays owned by
 *    the caller and is only read or written during the call. A context is used
 *    by one host thread at a time.
 *  - Nothing falls back to the CPU: without a usable CUDA device, dugks_create
 *    returns DUGKS_ECUDA.
 */
#ifndef DUGKS_H
#define DUGKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dugks_ctx dugks_ctx;

typedef enum {
    DUGKS_OK = 0,
    DUGKS_EINVAL = 1,      /* bad argument or parameter set */
    DUGKS_ENOMEM = 2,      /* device allocation failed */
    DUGKS_ECUDA = 3,       /* CUDA runtime error (message in dugks_last_error) */
    DUGKS_ETIMEOUT = 4,    /* a bounded device wait ran out */
    DUGKS_ENONFINITE = 5,  /* the field holds NaN or Inf */
    DUGKS_ESTATE = 6,      /* call not valid in the context's current state */
    DUGKS_EAGAIN = 7       /* the result is not ready yet: call again later */
} dugks_status_code;

enum { DUGKS_FP64 = 0, DUGKS_FP32 = 1, DUGKS_FP16F = 2 };
enum { DUGKS_UPWIND = 0, DUGKS_CENTRAL = 1 };
enum { DUGKS_VEL_UNIFORM = 0, DUGKS_VEL_ROTATION = 1, DUGKS_VEL_VORTEX = 2, DUGKS_VEL_FIELD = 3,
       DUGKS_VEL_DEFORM = 4 };

/* Problem statement (Sec. II-III): interface width W, mobility M, CFL number,
 * isotropic stencil order, face reconstruction, number of stages.
 *   nx, ny     cells, each >= 8.
 *   W > 0      interface width in cells (Eq. (3), (4)).
 *   M > 0      mobility of Eq. (1); tau = 3 M.
 *   cfl        in (0, 1]; dt = cfl.
 *   order      2, 3 or 4: derivative stencils and Taylor degree order - 1 of the
 *              upwind reconstruction Eq. (26); gradient order of Eq. (2). 5:
 *              DUGKS-T2S5 (Sec. III.A), the fifth-order reconstruction: the
 *              degree-4 tensor-product Lagrange interpolant on the 5 x 5 cells
 *              centred at the cell nearest to x_b - xi h (the paper prints no
 *              stencil), the gradient of order 4; upwind, two-stage, TMA-staged
 *              kernels only (dugks_set_variant(-1) and dugks_debug_faces refuse it).
 *   flux       DUGKS_UPWIND (Eq. (26)) or DUGKS_CENTRAL (Eq. (25)).
 *   stages     2: original two-stage DUGKS; 3: three-stage third-order DUGKS
 *              (Sec. II.B.2), which needs dt < 12 tau (Sec. III.A); 1: the
 *              streaming-collision discrete velocity method of Sec. II.B.1
 *              (Eqs. (8)-(14), the comparison scheme of the paper; flux unused,
 *              order = the Taylor degree + 1 of the streaming interpolation
 *              Eq. (12)), which at cfl = 1 is the lattice Boltzmann method
 *              (FP64 and FP32 storage).
 *   precision  DUGKS_FP64, DUGKS_FP32, or DUGKS_FP16F (FP32 arithmetic; f stored
 *              in half precision as the scaled deviation f_k - w_k phi, phi kept
 *              in FP32; two-stage only). FP32 and FP16F keep phi as an FP32 plane
 *              of its own and add each step's flux sum to it with unbiased
 *              stochastic rounding (uniform bits hashed from cell and step, so
 *              runs are deterministic); FP64 sums phi from the distribution.
 *   dtphiu     1 keeps the d(phi u)/dt term of the source Eq. (14b), evaluated
 *              by a backward difference over the last step; 0 drops it.
 *   phiA, phiB phase indicators (Eq. (3)), phiA != phiB; usually 1 and 0. */
typedef struct {
    int32_t nx, ny;
    double W, M, cfl;
    int32_t order, flux, stages, precision, dtphiu;
    double phiA, phiB;
} dugks_params;

/* Validates p, allocates the state on the current CUDA device and uploads phi0
 * (ny * nx doubles, host). cuda_stream is a cudaStream_t the context launches
 * on; NULL makes the context create and own a stream. The initial distribution
 * (f = f^eq, Omega = 0) is built on the device at the first dugks_step /
 * read / save after the velocity is set (default: uniform zero velocity).
 * Returns DUGKS_EINVAL (bad p, also stages == 3 with dt >= 12 tau, or FP16F
 * with stages == 3), DUGKS_ENOMEM or DUGKS_ECUDA; *out is NULL on error. */
int dugks_create(const dugks_params *p, const double *phi0_host, void *cuda_stream, dugks_ctx **out);

/* Sets the prescribed divergence-free velocity (Sec. II.A).
 *   UNIFORM  params = (ux, uy)
 *   ROTATION params = (cx, cy, omega): u = -omega (y - cy), v = omega (x - cx)
 *   VORTEX   params = (L, U, T): u = -U sin^2(pi x/L) sin(2 pi y/L) cos(pi t/T),
 *                                v =  U sin^2(pi y/L) sin(2 pi x/L) cos(pi t/T)
 *   FIELD    u_host, v_host = ny * nx cell-centre components (copied); a face
 *            takes the mean of its two cells.
 *   DEFORM   params = (L, U, T): the smoothed deformation of Sec. III.D,
 *            u = -U sin(4 pi x/L) sin(4 pi y/L) cos(pi t/T),
 *            v = -U cos(4 pi x/L) cos(4 pi y/L) cos(pi t/T).
 * Analytic fields are evaluated in the kernels at each point and time.
 * Allowed before the first step (it then defines the initial equilibrium) or
 * later (the new field applies from the next step). */
int dugks_set_velocity(dugks_ctx *c, int kind, const double *params, const double *u_host,
                       const double *v_host);

/* Enqueues nsteps >= 0 full time steps on the context's stream and returns
 * without waiting. Two-stage (Sec. II.B.2, the original DUGKS): one fused
 * kernel per step, which computes the cell moments, the source of Eq. (14b)
 * and bar f^+, the isotropic gradients of Eq. (2) and of the reconstruction,
 * bar f at x_b - xi h by Eqs. (24)-(26), the face phi, equilibrium, source
 * and original f of Eqs. (27)-(28), and the meso-flux update of Eq. (21), and
 * also writes per-tile FP64 mass partials. Three-stage (Eqs. (29)-(34)): two
 * kernels per step (steps (i)-(ii) and (iii)-(iv) of Sec. II.B.2). DVM
 * (stages = 1): one kernel per step, streaming (Eqs. (11a), (12)), phi of
 * Eq. (13), cell quantities at t + dt and the collision of Eq. (11b), with the
 * same per-tile mass partials. */
int dugks_step(dugks_ctx *c, int64_t nsteps);

/* Waits for the stream and writes phi = sum_k f_k (Eq. (30)) into out_host
 * (ny * nx doubles). */
int dugks_read_phi(dugks_ctx *c, double *out_host);

/* Enqueues phi into a device buffer dev_out of ny * nx elements of the
 * context's arithmetic type (double for FP64, float otherwise); no wait. */
int dugks_read_phi_device(dugks_ctx *c, void *dev_out);

/* Debug read-out of one step's face stage, for checking the path stage by
 * stage (two-stage scheme). For the current state at t_n it writes, for every
 * cell (x, y) and direction k (arrays of 9 * ny * nx doubles, index
 * (k * ny + y) * nx + x, caller-owned):
 *   fbar_E, fbar_N  bar f_k at the midpoint of the cell's east (x + 1) and north
 *                   (y + 1) face at t_n + dt/2, reconstructed from bar f^+ at
 *                   x_b - xi_k dt/2 (Eqs. (24)-(26), upwind or central);
 *   f_E, f_N        the original distribution at those faces, Eqs. (27)-(28).
 * The values come from the generic (plain) CUDA kernel in the context's
 * arithmetic type, widened to double; the context's state, step index and mass
 * do not change. Waits for the stream. DUGKS_EINVAL (not sticky) for a null
 * output or a three-stage context; DUGKS_ENOMEM (not sticky) if the 36 * ny * nx
 * doubles of device scratch cannot be allocated. */
int dugks_debug_faces(dugks_ctx *c, double *fbar_E, double *fbar_N, double *f_E, double *f_N);

/* Waits and returns the total mass sum phi over all cells, reduced in FP64 in
 * a fixed order (deterministic). DUGKS_ENONFINITE if it is NaN or Inf. */
int dugks_mass(dugks_ctx *c, double *out);

/* Enqueues the same reduction into dev_out (one double, device); no wait. */
int dugks_mass_device(dugks_ctx *c, double *dev_out);

/* Waits for the stream and returns the sticky status. */
int dugks_status(dugks_ctx *c);

/* Self-test of the device-side failure detection. Enqueues on the context's
 * stream one CTA that waits, with the same bounded mbarrier wait that guards the
 * step kernels' TMA copies, for 16 bytes that no copy ever delivers. After
 * max_polls polls (1 .. 1048576) the wait gives up, the kernel records a timeout
 * in the context's status word and returns: nothing faults, hangs or stays in
 * flight, and the device stays usable. The next dugks_status (and every later
 * call on this context) reports DUGKS_ETIMEOUT. DUGKS_EINVAL for a bad count. */
int dugks_selftest_wait_timeout(dugks_ctx *c, uint32_t max_polls);

/* Self-test of the allocation-failure paths, on the host only (process-wide;
 * the paper has no counterpart). After this call the next `skip` device
 * allocations of the library proceed and the `count` after them report
 * failure without asking the device; count = 0 disarms. An allocation that
 * fails inside dugks_create frees what was allocated and returns DUGKS_ENOMEM;
 * inside dugks_batch_add it returns DUGKS_ENOMEM and the batch stays usable.
 * DUGKS_EINVAL for a negative argument. */
int dugks_selftest_fail_allocs(int32_t skip, int32_t count);

/* Text of the last error; never NULL (empty when there was none). */
const char *dugks_last_error(const dugks_ctx *c);

/* Tile variant of the TMA-staged two-stage kernel (orders 2, 3), warps per CTA x
 * rows of cells per thread: 0 = 8 x 4 (FP64: 8 x 2), 1 = 16 x 1, 2 = 8 x 2,
 * 3 = 12 x 3, 4 = 8 x 3, 5 = 10 x 4 (a tile is 31 cells wide and warps x rows - 1
 * cells high). The default is 2 below 512 x 512 cells and 4 from there up; -1
 * selects the generic fused kernel (one thread per cell and stage, no TMA), the
 * plain comparison path. A tuning choice only: results agree to rounding.
 * Returns DUGKS_EINVAL for any other number. Order 4 and the three-stage
 * scheme have one TMA-staged tile shape each (orders 4-5, two-stage: 10 x 3, FP64
 * 8 x 2; three-stage: 8 x 2): any variant >= 0 selects it.
 * dugks_get_variant returns -1 when the context uses the generic kernel. */
int dugks_set_variant(dugks_ctx *c, int variant);
int dugks_get_variant(const dugks_ctx *c);

/* Number of steps taken since creation (or as restored by dugks_load_state). */
int64_t dugks_step_index(const dugks_ctx *c);

/* Checkpoint: raw device state (distribution planes, phi planes) in the
 * context's storage layout. dugks_state_bytes gives the size. save waits and
 * copies to host; load copies from host and sets the step index. The bytes
 * are only meaningful to a context created with the same dugks_params. */
size_t dugks_state_bytes(const dugks_ctx *c);
int dugks_save_state(dugks_ctx *c, void *host, size_t bytes, int64_t *step_index);
int dugks_load_state(dugks_ctx *c, const void *host, size_t bytes, int64_t step_index);

/* Frees everything; NULL-safe; waits for the context's outstanding work. */
void dugks_destroy(dugks_ctx *c);

/* ---- many grids per launch ------------------------------------------------
 * A batch advances many independent periodic grids of different sizes with one
 * launch per step: a work list of 31-cell-wide tiles of all grids is processed
 * by a grid-stride set of CTAs (the TMA-staged two-stage kernel), followed by a
 * per-grid FP64 mass and step-counter update. Each grid keeps its own step
 * counter on the device, so grids may join (dugks_batch_add) and leave
 * (dugks_batch_remove) between calls of dugks_batch_step, and a sequence of
 * steps is replayed as a CUDA graph. Every grid's result is bitwise the same
 * whatever else is in the batch. Two-stage scheme, orders 2 and 3 only.
 *
 * Add, step, retire, collect (without wait), fence, reached and remove queue
 * their device work on the batch's stream and return without waiting for it:
 * grid memory comes from a stream-ordered memory pool owned by the batch, host
 * data moves through pinned staging buffers, and whatever the stream may still
 * read is released only after it has passed. A server can therefore admit and
 * finish grids while earlier steps are still running; several batches on
 * streams of different priority share the GPU tile by tile when their kernels
 * run one CTA per tile (dugks_batch_set_ctas). The calls described as waiting
 * (read_phi, mass, status, set_variant, destroy) synchronise the stream. A
 * batch is not thread-safe: one host thread drives it. */
typedef struct dugks_batch dugks_batch;

/* Common parameters of all grids (nx, ny ignored; stages must be 2, order 2 or
 * 3). cuda_stream as in dugks_create. */
int dugks_batch_create(const dugks_params *common, void *cuda_stream, dugks_batch **out);

/* Device bytes one grid of nx * ny cells needs in a batch (admission control). */
size_t dugks_batch_grid_bytes(const dugks_params *common, int32_t nx, int32_t ny);

/* Adds a grid: phi0_host (ny * nx doubles), velocity kind UNIFORM, ROTATION or
 * VORTEX with its parameters (as dugks_set_velocity), and the number of steps
 * after which the grid stops advancing (target_steps < 0: unbounded). Queues
 * the initial equilibrium on the stream (no wait). *grid_id receives a
 * non-negative id. DUGKS_ENONFINITE (not sticky) for a field holding NaN or
 * Inf; DUGKS_ENOMEM (not sticky) if device or pinned host memory is not
 * available. */
int dugks_batch_add(dugks_batch *b, int32_t nx, int32_t ny, const double *phi0_host, int vel_kind,
                    const double *vel_params, int64_t target_steps, int32_t *grid_id);

/* Removes a grid: its device memory goes back to the batch's pool once the
 * steps queued before the call have run (no wait). A pending read-out of a
 * retiring grid is dropped. DUGKS_EINVAL for an unknown id. */
int dugks_batch_remove(dugks_batch *b, int32_t grid_id);

/* Finishing a grid without waiting. Freezes the grid where it stands (after the
 * steps already queued), queues the read-out of phi (ny * nx doubles, widened to
 * FP64 on the device) into a pinned host buffer owned by the batch, and returns
 * in *ticket the fence that follows the copy. The grid leaves the work list; its
 * id stays reserved until dugks_batch_collect or dugks_batch_remove. DUGKS_EINVAL
 * for an unknown or already retiring id; DUGKS_ENOMEM (not sticky) if no pinned
 * host memory is available. */
int dugks_batch_retire(dugks_batch *b, int32_t grid_id, uint64_t *ticket);

/* Result of a retired grid: if its read-out has completed (or wait != 0, after
 * waiting for it) copies phi into out_host (ny * nx doubles, row-major), frees
 * the grid as dugks_batch_remove does and returns DUGKS_OK. With wait == 0 and
 * the copy still in flight it returns DUGKS_EAGAIN and changes nothing.
 * DUGKS_EINVAL for an id that is not retiring. */
int dugks_batch_collect(dugks_batch *b, int32_t grid_id, double *out_host, int wait);

/* Fences: dugks_batch_fence records a point in the batch's stream and returns its
 * ticket (tickets increase by one per fence, retire's included); dugks_batch_reached
 * sets *done to 1 once the stream has passed it, else 0 (no wait). A caller
 * keeps the number of steps in flight bounded with them. DUGKS_EINVAL for a
 * ticket never issued. */
int dugks_batch_fence(dugks_batch *b, uint64_t *ticket);
int dugks_batch_reached(dugks_batch *b, uint64_t ticket, int32_t *done);

/* CTAs of the step kernel: 0 (default) as many as are resident on the GPU, each
 * striding over the work list; a negative value one CTA per tile, so that a
 * kernel of a higher-priority stream takes SMs as soon as tiles finish; a
 * positive value at most that many. DUGKS_EINVAL for a null batch. */
int dugks_batch_set_ctas(dugks_batch *b, int32_t ctas);

/* Enqueues nsteps steps of every grid that has not reached its target. */
int dugks_batch_step(dugks_batch *b, int64_t nsteps);

/* Steps taken by a grid (host mirror of its device counter). */
int64_t dugks_batch_step_index(const dugks_batch *b, int32_t grid_id);

/* Waits and copies phi (ny * nx doubles) of one grid to the host. */
int dugks_batch_read_phi(dugks_batch *b, int32_t grid_id, double *out_host);

/* Waits and returns one grid's mass (FP64, fixed-order sum). */
int dugks_batch_mass(dugks_batch *b, int32_t grid_id, double *out);

/* Tile variant of the batch kernel (0..5 as for dugks_set_variant; default 5 in
 * FP32, 4 otherwise);
 * waits for the stream and rebuilds the grid descriptors. */
int dugks_batch_set_variant(dugks_batch *b, int variant);

/* Cells of all grids that are still advancing. */
int64_t dugks_batch_active_cells(const dugks_batch *b);

/* Waits and returns the sticky status; text of the last error. */
int dugks_batch_status(dugks_batch *b);
const char *dugks_batch_last_error(const dugks_batch *b);

/* Frees everything (NULL-safe). */
void dugks_batch_destroy(dugks_batch *b);

/* Allocation-free FP64 sum of a device field. The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc where they need a mass:
 * hosts whose device memory is fully reserved by another allocator (a
 * framework's caching pool hands out no raw cudaMalloc memory), and
 * latency-critical loops that cannot take the implicit device synchronisation
 * of cudaMalloc and cudaFree. It runs the same reduction as dugks_mass_device
 * (one FP64 partial per 32 x 8 tile, then a fixed-order sum) with the partials
 * in a static device array of DUGKS_NOALLOC_MAX_TILES doubles (512 KiB), which
 * every GPU that loads the library holds until the process exits. It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   field    device pointer: ny rows of nx values, row stride pitch elements
 *   dtype    0 = double, 1 = float
 *   out_dev  device pointer to one double, written by the kernels
 *   cuda_stream  cudaStream_t to launch on (NULL = legacy default stream)
 * Returns DUGKS_EINVAL for bad arguments or when ceil(nx/32) * ceil(ny/8)
 * exceeds DUGKS_NOALLOC_MAX_TILES (e.g. more than 4096 x 4096 cells; any shape
 * within the limit is served, down to one tile column of 524288 rows), and
 * DUGKS_ECUDA when one of its own launches fails (an error left pending by
 * earlier work is neither reported nor cleared). It enqueues work and does not
 * wait. The first call on each device looks up the array's device address
 * (with that device current); make that first call before any stream capture.
 * Every call on a device shares the array: calls whose kernels may overlap on
 * the GPU (different streams without ordering) race and must be serialised by
 * the caller. Each call overwrites the entries it reads, so no clearing is
 * needed between calls. */
#define DUGKS_NOALLOC_MAX_TILES 65536
int dugks_field_mass_noalloc(const void *field, int dtype, int32_t nx, int32_t ny, int32_t pitch,
                             double *out_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
