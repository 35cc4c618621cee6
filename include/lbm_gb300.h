/*
 * lbm_gb300.h -- C ABI of the GB300 (sm_103a) D3Q27 lattice-Boltzmann solver
 * coupled to the actuator line model, the method of arxiv 2402.13171.
 *
 * One time step (Sec. 2.1 and 2.2 of the paper, in this order):
 *   1. blade kinematics at t = n (Algorithm 2, Line::update);
 *   2. trilinear sampling of rho and u at every blade element (Sec. 2.2);
 *   3. blade-element forces from tabulated polars (Sec. 2.2, element-force equation);
 *   4. regularisation of the element forces onto the lattice, f_eps = f (x) eta_eps (Sec. 2.2),
 *      with a Gaussian kernel or the discrete delta of Roma et al. (1999) the paper uses;
 *   5. pull streaming with boundary rules, and
 *   6. cumulant collision (Geier et al. 2015, Sec. 2.1) or BGK-Smagorinsky with Guo forcing
 *      (Sec. 2.1, lattice Boltzmann equation with source term).
 * Steps 5-6 run fused in one pass over the lattice, launched per time step
 * over the tiles around the rotors, then (where there are any) over the tiles
 * on a no-slip or free-slip face, then over the rest, each launch overlapping
 * the one before.  Steps 1-4 of step n+1 run inside the rotor launch of step n
 * as soon as the cells around the rotor are written, under the bulk launch,
 * so the actuator line adds no serial gap.
 *
 * Conventions shared by every call:
 *  - Lattice units: dx = dt = 1, c_s^2 = 1/3, relaxation rate omega = 1/(3 nu + 1/2).
 *  - Velocities q = (cz+1)*9 + (cy+1)*3 + (cx+1), cx, cy, cz in {-1, 0, 1};
 *    q = 13 is the rest population, opposite(q) = 26 - q.
 *  - Host field arrays are x fastest: scalar fields [nz][ny][nx], vector fields
 *    3 planes [3][nz][ny][nx], PDF fields 27 planes [27][nz][ny][nx].
 *  - Device PDFs are stored as offsets f_q - w_q from the lattice weights, in
 *    FP32, BF16 or FP16 (lbm_config.storage); collision arithmetic is FP32.
 *  - Every function returns an lbm_status.  The first error is sticky: every
 *    later call on the same context returns it until lbm_destroy.  No C++
 *    exception crosses this interface.  lbm_last_error() gives the message.
 *  - The context owns all device memory it allocates (through
 *    lbm_config.dev_alloc/dev_free if given, else cudaMalloc/cudaFree).  The
 *    caller owns every host array it passes; tables are copied.
 *  - Calls that return host data synchronise the context's stream; lbm_step
 *    only enqueues work.
 *  - Fault injection for tests, on the host only: the environment variable
 *    LBM_FAULT=alloc fails every device allocation (LBM_ERR_OOM), =capture
 *    every CUDA graph capture (LBM_ERR_CUDA), =step:N the lbm_step call that
 *    would run step N (LBM_ERR_CUDA, before it enqueues anything).  It is
 *    read at each check.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque handle of one lattice (one instance) */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = 1, /* bad pointer, size or value; the context stays usable */
    LBM_ERR_OOM = 2,         /* device allocation failed */
    LBM_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    LBM_ERR_NUMERIC = 4,     /* NaN/Inf seen by the diagnostic sums */
    LBM_ERR_TIMEOUT = 5,     /* a bounded device wait (the staged step's copy barriers, ~1 s) gave up */
    LBM_ERR_STATE = 6,       /* call not valid in the current state */
    LBM_ERR_UNSUPPORTED = 7  /* combination not built */
} lbm_status;

typedef enum { LBM_COLL_CUMULANT = 0, LBM_COLL_SRT_SMAGORINSKY = 1 } lbm_collision;
typedef enum { LBM_STORE_FP32 = 0, LBM_STORE_BF16 = 1, LBM_STORE_FP16 = 2 } lbm_storage;
typedef enum {
    LBM_BC_PERIODIC = 0,       /* source index wraps */
    LBM_BC_INFLOW_OUTFLOW = 1, /* x only: equilibrium inlet at x = 0 (rho = 1, lbm_inflow velocity),
                                  zero-gradient outlet at x = nx-1 */
    LBM_BC_NOSLIP = 2,         /* halfway bounce-back walls at -1/2 and n-1/2 */
    LBM_BC_FREESLIP = 3        /* specular (zero-shear) walls at -1/2 and n-1/2 */
} lbm_bc;

typedef struct {
    int nx, ny, nz;          /* cells; each in [1, 65535] */
    int collision;           /* lbm_collision */
    double nu;               /* lattice kinematic viscosity, > 0 */
    double smag_c;           /* Smagorinsky constant (SRT variant only) */
    int storage;             /* lbm_storage */
    int bc[3];               /* lbm_bc per axis */
    double body_force[3];    /* uniform body force density, added to the ALM force */
    unsigned long long seed; /* key of the inflow noise (splitmix64) */
    int diag_every;          /* FP64 mass/momentum sums every k steps (0 = off) */
    void* cuda_stream;       /* cudaStream_t to enqueue on; NULL = legacy default stream */
    void* (*dev_alloc)(size_t bytes, void* user); /* optional device allocator */
    void (*dev_free)(void* ptr, void* user);
    void* alloc_user;
    int tile_x, tile_y;      /* CTA tile (threads along x, rows along y); 0 = default 32 x 4;
                                tile_x a multiple of 32, tile_x * tile_y <= 256 */
    int tile_z;              /* planes per CTA, each thread marching through them; 0 = default 1; <= 64 */
    int staged;              /* kernel form of the step.  0 = direct loads; with 16-bit storage,
                                single-plane tiles and every nx of the batch even,
                                the tiles without a no-slip or free-slip face cell then take two cells
                                of a row per thread (32-bit words, the collision on f32x2 instructions
                                across the pair; bit for bit the one-cell results).
                                1 = persistent CTAs stage the 27 source rows of each 1-row tile in a
                                3-4 stage shared-memory ring filled by TMA bulk copies (needs
                                tile_y = tile_z = 1 and nx a multiple of 4 (FP32) or 8 (16-bit)).
                                2 = direct loads, one cell per thread everywhere */
    int inplace;             /* 1: one PDF array updated in place (AA pattern: even steps pull from the
                                neighbours and push into the slots they read, odd steps read and write a
                                cell's own slots), half the PDF memory, for every boundary rule and
                                rotors (the outlet keeps a copy of its last plane, 9 ny nz values per
                                step parity).  Needs single-plane direct tiles; the state read-out and
                                write calls (moments, probe, PDFs, state, init, inflow, step counter,
                                autotune) need an even step count, where the array equals the two-array
                                scheme's.  0 = two arrays */
} lbm_config;

typedef struct {
    int kind;          /* 0: uniform u_ref; 1: log law u_ref * ln(z_c/z0)/ln(z_ref/z0), z_c = z + 1/2 */
    double u_ref[3];
    double z0, z_ref;
    double noise_rel;  /* per component, per step and inlet column: + noise_rel * |u_ref| * xi,
                          xi uniform in [-1, 1) from splitmix64(seed, ((n*nz + z)*ny + y)*3 + a + 1) */
} lbm_inflow;

/* One rotor of n_blades straight blade lines (Sec. 2.2; kinematics of
 * Algorithm 2).  Rotor axis (cos yaw, sin yaw, 0); blade b at angle
 * theta0 + omega * n + 2 pi b / n_blades about it; element k at radius
 * (k + 1/2) R / n_elements, length R / n_elements, chord linear from
 * chord_root (r = 0) to chord_tip (r = R); alpha = phi - twist_k - pitch.
 * The polar table (alpha ascending, radians) is interpolated linearly and
 * clamped at its ends.  The force of element k is spread with the kernel
 * `regularisation` names:
 *   ALM_REG_GAUSSIAN: prod_a exp(-d_a^2 / eps^2) on |d_a| <= 3 eps, each axis
 *     renormalised to unit lattice sum (eps in [0.5, 5]);
 *   ALM_REG_ROMA: prod_a phi(d_a), Roma, Peskin and Berger's three-point
 *     delta on |d_a| <= 3/2, unit sum by construction (epsilon unused),
 * d = cell - element position.  With tip_loss = 1 each element force is
 * scaled by Glauert's tip-loss factor in Prandtl's form (Sec. 2.2),
 * F = (2/pi) arccos(exp(-B (R - r) / (2 r |sin phi|))), phi the inflow angle
 * (F = 1 where sin phi = 0).  The whole force support (hub +- (R + cut + 1),
 * cut = 3 eps or 3/2) must lie inside [1, n-2] on every axis. */
typedef enum { ALM_REG_GAUSSIAN = 0, ALM_REG_ROMA = 1 } alm_regularisation;

typedef struct {
    double hub[3];
    double radius;
    int n_blades, n_elements;
    double epsilon;       /* Gaussian width, cells (ALM_REG_GAUSSIAN) */
    double omega;         /* rotor speed, rad per step, positive about the axis */
    double yaw, pitch, theta0;
    double chord_root, chord_tip;
    const double* twist;  /* n_elements values or NULL (0) */
    int n_polar;          /* >= 2 */
    const double* alpha;
    const double* cl;
    const double* cd;
    int regularisation;   /* alm_regularisation; 0 (zero-initialised) = Gaussian */
    int tip_loss;         /* 1: Glauert tip-loss factor on the element forces, 0: none */
} alm_turbine_desc;

/* Create one lattice.  The state starts at f = feq(rho = 1, u = 0) until
 * lbm_set_inflow / lbm_init_fields set it; the step counter starts at 0.
 * Errors: INVALID_ARG (sizes, collision/storage/bc codes, nu <= 0), OOM, CUDA. */
lbm_status lbm_create(const lbm_config* cfg, lbm_ctx** out);

/* Create n lattices that step together: the same two launches per time step
 * cover all of them (the batched form of lbm_step).  cfgs[i] may differ in sizes, viscosity, inflow
 * and rotors, but collision, storage and cuda_stream must agree
 * (UNSUPPORTED otherwise).  out receives n handles; lbm_step on any of them
 * advances all n.  Each handle is destroyed with lbm_destroy; memory is freed
 * with the last one. */
lbm_status lbm_batch_create(int n, const lbm_config* cfgs, lbm_ctx** out);

/* Inflow of the x inlet (reading: the paper's validation runs are periodic).
 * Also sets the state to feq(rho = 1, u = mean inflow) everywhere and the
 * lagged ALM force to zero; the step counter is unchanged. */
lbm_status lbm_set_inflow(lbm_ctx* ctx, const lbm_inflow* inflow);

/* Set the state to feq(rho, u) + fneq (host arrays: rho [N] or NULL for 1,
 * u [3][N] or NULL for the mean inflow, fneq [27][N] or NULL for 0) and the
 * lagged ALM force to zero; the step counter is unchanged.  Synchronises. */
lbm_status lbm_init_fields(lbm_ctx* ctx, const double* rho, const double* u, const float* fneq);

/* Add a rotor (copied).  id_out receives its index within this lattice.
 * Errors: INVALID_ARG for a support outside [1, n-2], an unknown
 * regularisation or tip_loss code, bad epsilon (Gaussian), table or element
 * counts (at most 4096 elements per lattice). */
lbm_status alm_add_turbine(lbm_ctx* ctx, const alm_turbine_desc* desc, int* id_out);

/* Enqueue n_steps time steps on the stream: replays of captured 8- and 2-step
 * CUDA graphs (plain launches for an odd last step and on the legacy default
 * stream).  Errors from earlier steps surface here or at the
 * next synchronising call. */
lbm_status lbm_step(lbm_ctx* ctx, int n_steps);

/* Wait for the stream; report any device-side error. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* rho [N] and u [3][N] of the last collision: rho = sum f*, u = (sum c f* -
 * F/2)/rho with F the force of that collision (the velocity the collision
 * used).  Host arrays, caller-owned.  Synchronises. */
lbm_status lbm_get_moments(lbm_ctx* ctx, double* rho, double* u);

/* rho and u (as lbm_get_moments computes them) at n listed cells (linear
 * indices (z*ny + y)*nx + x, host array); rho [n] (may be NULL) and u [n][3]
 * are host, caller-owned.  For monitoring points and wake profiles without
 * copying whole fields.  Synchronises. */
lbm_status lbm_probe(lbm_ctx* ctx, const long long* cells, int n, double* rho, double* u);

/* Absolute populations f [27][N] (host, FP64) / overwrite them (the step
 * counter and the lagged ALM force are kept; the actuator line of the current
 * step is re-evaluated).  Conversion runs on the device, plane by plane, in a
 * reused staging buffer.  Synchronises.  For a bitwise resume use
 * lbm_get_state / lbm_set_state. */
lbm_status lbm_get_pdfs(lbm_ctx* ctx, double* f);
lbm_status lbm_set_pdfs(lbm_ctx* ctx, const double* f);

/* Checkpoint of one lattice, for a bitwise resume: everything a time step
 * reads that is not a descriptor -- the raw PDF array of the current step in
 * the storage type, each rotor's lagged force box (the ALM force of the last
 * collision, which the next sampling of Sec. 2.2 reads), the actuator-line
 * element buffers and FP64 rotor loads of both step parities, the inlet
 * ghost populations (the equilibria the x = 0 cells pull) of both parities,
 * the last diagnostic sums -- and the step counter, behind a header with the
 * lattice's shape.  The blob is
 * host memory owned by the caller: lbm_get_state_size gives its size,
 * lbm_get_state fills it, lbm_set_state restores it into a lattice of the
 * same sizes, storage, collision, boundary rules and rotors (INVALID_ARG
 * otherwise) and sets the step counter (for a batch: restore every member
 * from states taken at the same step).  A run resumed from it continues
 * bit for bit as the original.  In-place lattices need an even step count
 * (STATE otherwise).  get/set synchronise. */
lbm_status lbm_get_state_size(lbm_ctx* ctx, size_t* bytes);
lbm_status lbm_get_state(lbm_ctx* ctx, void* buf, size_t bytes);
lbm_status lbm_set_state(lbm_ctx* ctx, const void* buf, size_t bytes);

/* Bound of the staged step's waits on its own TMA copies, in SM clock cycles
 * (default 2^31, about 1 s; the bounded waits of Sec. 2.1's streaming are an
 * implementation matter, not the paper's).  A wait that passes it sets
 * LBM_ERR_TIMEOUT, reported by the next synchronising call; the kernel first
 * waits, with the default bound, for the copies it still has in flight.
 * Meant for tests of that error path: with a bound of 0 every wait gives up
 * before it looks, on copies that are valid and land a little later.
 * INVALID_ARG for a negative bound. */
lbm_status lbm_set_wait_limit(lbm_ctx* ctx, long long cycles);

/* Rotor thrust and torque (FP64 sums, Sec. 2.2) of the forces applied in the
 * last completed step; optionally the element blade forces and positions
 * (3 floats each, blade-major).  Synchronises. */
lbm_status alm_get_loads(lbm_ctx* ctx, int id, double* thrust, double* torque, float* elem_force, float* elem_pos);

/* The same thrust and torque, without waiting: enqueues a copy of the 2
 * doubles of the last enqueued step into thrust_torque on the lattice's
 * stream and returns.  thrust_torque (host, caller-owned) must stay valid
 * until the stream has passed the copy (lbm_sync, or an event the caller
 * records on the stream); from page-locked memory the copy is asynchronous,
 * so a serving loop can enqueue step n + 1 before it reads the loads of step
 * n.  Device errors surface at the next synchronising call.  Errors:
 * INVALID_ARG for a bad rotor id or a null output. */
lbm_status alm_get_loads_async(lbm_ctx* ctx, int id, double* thrust_torque);

/* Zero-copy loads: from the next launch on, the actuator-line evaluation of
 * step s also writes (thrust, torque) of every rotor t of this lattice into
 * host_ring[2 ((s mod ring_len) n_turb + t) + {0, 1}].  host_ring must be
 * page-locked host memory mapped into the device address space (cudaHostAlloc,
 * or a pinned torch tensor), of 2 n_turb ring_len doubles, owned by the caller
 * and valid until the sink is cleared (host_ring NULL or ring_len 0) or the
 * context is destroyed.  The loads of step s are evaluated during step s - 1,
 * so they are complete once that step's work has finished on the stream (an
 * event recorded behind it); ring_len >= 3 leaves a step's entry untouched
 * while the next two steps run.  Adding a rotor clears the sink.
 * Synchronises.  Errors: INVALID_ARG when host_ring is not mapped. */
lbm_status alm_set_loads_sink(lbm_ctx* ctx, double* host_ring, int ring_len);

/* FP64 sums [mass, momentum x, y, z] of the last diagnostic step (post-
 * collision state).  Synchronises; NUMERIC if NaN/Inf was seen. */
lbm_status lbm_get_diagnostics(lbm_ctx* ctx, double mass_mom[4], long long* at_step);

/* Completed-step counter n (also the key of the inflow noise and blade angle),
 * shared by all lattices of a batch.  lbm_set_step sets it (checkpoint
 * restore together with lbm_set_pdfs) and re-evaluates the actuator line for
 * step n.  Synchronises. */
lbm_status lbm_get_step(lbm_ctx* ctx, long long* step);
lbm_status lbm_set_step(lbm_ctx* ctx, long long step);

/* CTA tile of the step kernel and its form (see lbm_config.tile_* and staged:
 * 0 direct, paired cells where they apply; 1 staged rows; 2 direct, one cell
 * per thread); changing it rebuilds the work list.  Results do not depend on
 * the tile or the form.  INVALID_ARG for a bad shape or form. */
lbm_status lbm_set_tile(lbm_ctx* ctx, int tile_x, int tile_y, int tile_z, int staged);
lbm_status lbm_get_tile(lbm_ctx* ctx, int* tile_x, int* tile_y, int* tile_z, int* staged);

/* Autotuner: times the step kernel for a fixed set of CTA tiles (tile_x,
 * tile_y, tile_z, staged) on the current state of every lattice of the batch
 * (steps_per_candidate timed launches each, after 3 untimed ones), restoring
 * the state (PDFs, rotor force boxes, step counter) after every candidate, and
 * applies the fastest.  cache_path (or NULL): a text file of
 * "<gpu/collision/storage/lattices key> tile_x tile_y tile_z staged ms" lines; a
 * matching line is applied without timing, a new result is appended.
 * tile_out receives the tile, best_ms its mean launch time.  The last
 * diagnostic result may be overwritten.  Synchronises. */
lbm_status lbm_autotune(lbm_ctx* ctx, int steps_per_candidate, const char* cache_path, int tile_out[4],
                        double* best_ms);

/* Kernel timing: when enabled, lbm_step brackets every replay of its 8- or
 * 2-step graph (or a single step) with CUDA events on the lattice's stream, so
 * timing does not break up the replays; lbm_get_kernel_time returns the mean
 * device time per time step (ms, both launches of a step) and the number of
 * timed steps since enabling. */
lbm_status lbm_set_profiling(lbm_ctx* ctx, int enable);
lbm_status lbm_get_kernel_time(lbm_ctx* ctx, double* mean_ms, long long* steps);

/* Algorithmic bytes one time step moves per cell (27 loads + 27 stores of
 * the storage type) and the number of cells of one step (all lattices). */
lbm_status lbm_get_traffic_model(lbm_ctx* ctx, double* bytes_per_cell, long long* cells_per_step);

/* Kernel launches of one time step with the current tile and rotors: the
 * tiles around the rotors, then the tiles with a cell on a no-slip or
 * free-slip face, then the rest (each launch only where it has tiles; the
 * in-place scheme takes the last two together; staged rows are one launch).
 * Uploads pending descriptors first (stream-ordered).  Errors: INVALID_ARG
 * for a null output. */
lbm_status lbm_get_launches_per_step(lbm_ctx* ctx, int* launches);

/* Actuator-line evaluation for callers that cannot allocate device memory:
 * a real-time turbine-controller loop, or code embedded in another framework
 * that owns the memory pool, where cudaMalloc/cudaFree may synchronise the
 * device, take unbounded time or be forbidden.  The paper has no counterpart.
 * It is the same evaluation as a lattice's actuator line (kinematics,
 * trilinear sampling, blade-element forces, FP64 thrust and torque) for one
 * rotor at step `step` on a caller-owned field, with no lagged blade force
 * (only body_force enters the half-force shift of the sampled velocity).
 *   pdf_offsets  device, FP32 offsets f - w, [27][nz][ny][nx]; 27*nx*ny*nz < 2^31
 *   desc         as for alm_add_turbine; its support must lie inside [1, n-2]
 *   elem_force   device, 3 floats per element (blade-major): blade forces
 *   elem_pos     device, 3 floats per element, or NULL
 *   loads        device, 2 doubles: thrust, torque
 * Work is enqueued on cuda_stream (NULL = legacy default stream).  The rotor
 * descriptor and polar table are copied from pageable host memory, so the
 * call may wait for earlier work on that stream before it returns; the
 * outputs are complete once the stream has passed the call's work.  Nothing
 * is allocated: the scratch is one static
 * device block of about 180 KB that every GPU loading this library holds
 * until the process exits.  Limits: at most 1024 elements and 8192 polar
 * points (INVALID_ARG beyond, before anything is enqueued).  The first call
 * on a device looks up the block's address (make it before any stream
 * capture).  All calls share the block: calls that overlap on the GPU race.
 * Errors: INVALID_ARG (also for non-finite rotor inputs or body force, and
 * blade or element counts whose product exceeds the limit), CUDA. */
lbm_status alm_eval_static(const float* pdf_offsets, int nx, int ny, int nz, const double body_force[3],
                           const alm_turbine_desc* desc, long long step, float* elem_force, float* elem_pos,
                           double* loads, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Wake surrogate for warm starts.  Not part of the paper's method: a small
 * multilayer perceptron n_in -> width (x n_hidden, GELU) -> n_out, trained on
 * time-mean wake fields this solver produced, whose prediction initialises new
 * runs (lbm_init_fields).  Weights: FP32 masters for the optimiser (Adam),
 * BF16 copies in every product, FP32 accumulation.  Parameter vector layout
 * (FP32): for each layer, W [out][in] row-major then b [out].  Host arrays
 * are row-major [n][n_in] / [n][n_out].  Training is deterministic (fixed
 * reduction orders, counter-based minibatch sampling). */
typedef struct mlp_ctx mlp_ctx;

/* width, n_in, n_out <= 128; 1 <= n_hidden <= 16.  Parameters start at zero. */
lbm_status mlp_create(int n_in, int width, int n_hidden, int n_out, void* cuda_stream, mlp_ctx** out);
void mlp_destroy(mlp_ctx* m);
const char* mlp_last_error(const mlp_ctx* m);
int mlp_num_params(const mlp_ctx* m);
/* Set / read the FP32 parameters (set also resets the optimiser state). */
lbm_status mlp_set_params(mlp_ctx* m, const float* params);
lbm_status mlp_get_params(mlp_ctx* m, float* params);
/* y [n][n_out] = network(x [n][n_in]).  Synchronises. */
lbm_status mlp_forward(mlp_ctx* m, const float* x, int n, float* y);
/* Mean squared error over all outputs of the batch and its gradient w.r.t.
 * the parameters (grad may be NULL).  Synchronises. */
lbm_status mlp_loss_grad(mlp_ctx* m, const float* x, const float* target, int n, double* loss, float* grad);
/* Upload a training set, then run `steps` Adam steps (lr, beta = 0.9/0.999)
 * on minibatches of `batch` rows drawn with splitmix64(seed, step*batch + k + 1)
 * mod n.  last_loss: the MSE of the last minibatch (may be NULL). */
lbm_status mlp_set_data(mlp_ctx* m, const float* x, const float* target, int n);
lbm_status mlp_train(mlp_ctx* m, int steps, int batch, double lr, unsigned long long seed, double* last_loss);

const char* lbm_last_error(const lbm_ctx* ctx);
const char* lbm_status_string(lbm_status s);

/* Free the handle (and the batch's device memory with its last handle). NULL-safe. */
void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
