/*
 * lbm.h -- C ABI of the GB300 (sm_103a) phase-field WMRT lattice Boltzmann
 * library: the fused per-timestep update of the conservative Allen-Cahn
 * populations g and the pressure-based hydrodynamic populations f on D2Q9
 * and D3Q19 (arXiv 2505.12205, Sec. 3.2, Algorithms 1-3, App. A and B).
 *
 * Conventions shared by every entry point
 *  - Lattice units: dx = dt = c = 1, c_s^2 = 1/3; phi_L = 0 (light fluid),
 *    phi_H = 1 (heavy fluid).
 *  - Fields are float32 arrays [nz][ny][nx] with x fastest (nz = 1 in 2D).
 *    A velocity is D consecutive planes (u_x, u_y[, u_z]).  Populations are
 *    population-major [Q][nz][ny][nx] (Q = 9 or 19) in the velocity order of
 *    the momentum rows of eq:A1 (D2Q9) and eq:A2 (D3Q19).
 *  - Buffers passed in are owned by the caller; the library copies from or
 *    into them and never keeps a pointer.  When on_device is non-zero the
 *    pointers are CUDA device pointers of the context's device (for example
 *    torch.Tensor.data_ptr()); otherwise they are host pointers.
 *  - All work is enqueued on the context's stream.  lbm_step returns once
 *    its kernels are enqueued; calls that return data to the host
 *    synchronise the stream.
 *  - Every call returns an lbm_status.  Nothing aborts or exits; the text of
 *    the last error of a context is available from lbm_last_error.
 *  - There is no CPU fallback: without a CUDA device lbm_create fails with
 *    LBM_ERR_CUDA.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;   /* opaque; owns all device memory */

typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 } lbm_lattice;

/* Face conditions, App. B: periodic (eq:periodic_f/g/phi), halfway
 * bounce-back wall (eq:no_slip_f/g), velocity + phase-field inlet
 * (eq:velocity_boundary_distribution, eq:unknown_distribution_*), convective
 * outlet (eq:convective_f/g), free slip (eq:free_slip_f/g: specular
 * reflection, the population returns to the tangential neighbour with its
 * normal component reversed; over an edge of two slip faces both components
 * are reversed; a crossing of a wall as well bounces back).  The inlet is
 * allowed only on the low face and the outlet only on the high face of the
 * last axis (y in 2D, z in 3D).  The ghost phi of walls, slip faces and the
 * outlet is that of the adjacent node (zero normal gradient). */
typedef enum {
    LBM_BC_PERIODIC = 0,
    LBM_BC_WALL = 1,
    LBM_BC_INLET = 2,
    LBM_BC_OUTFLOW = 3,
    LBM_BC_FREESLIP = 4
} lbm_bc;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,      /* invalid argument or parameter */
    LBM_ERR_CUDA = -2,     /* a CUDA runtime call failed */
    LBM_ERR_OOM = -3,      /* device allocation failed */
    LBM_ERR_DIVERGED = -4, /* non-finite populations found by lbm_diag or by
                              the in-step check of lbm_step (diag_every) */
    LBM_ERR_TIMEOUT = -5,  /* a bounded iteration gave up (lbm_jet_stats) */
    LBM_ERR_STATE = -6     /* call out of order (e.g. step before init) */
} lbm_status;

/* Problem statement of Sec. 3 of the paper.
 *  lattice      lbm_lattice; nx, ny, nz grid (nz = 1 for D2Q9)
 *  bc[6]        lbm_bc of the faces -x, +x, -y, +y, -z, +z (z ignored in 2D)
 *  visc_model   0: dynamic viscosity linear in phi (eq:dynamic_viscosity),
 *                  tau = mu(phi) / (rho(phi) c_s^2), mu_X = rho_X tau_X c_s^2;
 *               1: relaxation time linear in phi (eq:relaxation_time)
 *  outlet_scheme the outlet speed U of the convective outlet
 *               (eq:velocity_options): 0 local u(x, N-1), 1 its maximum, 2 its
 *               average over the layer N-1
 *  storage      population storage format (arithmetic is float32 always):
 *               0 = float32;
 *               1 = 16-bit: f in float16 as (f_a / w_a - r_m) * storage_scale,
 *               r_m a reference of the node's plane m along the last axis
 *               (z in 3D, y in 2D): the plane's mean p* when lbm_init_fields
 *               gives the state, its mean f_0 / w_0 when lbm_set_populations
 *               gives a context its first state, kept after that; g in
 *               16-bit fixed point, q = rint((g_a / w_a + 1/2) * 65535 / 2)
 *               saturated to [0, 65535];
 *               2 = bfloat16: f as (f_a / w_a) * storage_scale, g as
 *               g_a / w_a - 1/2
 *  diag_every   steps between the in-step diagnostics of lbm_step (FP64
 *               sum of phi, finite check, Laplace pressure sums; Sec. 5.2,
 *               5.4); 0 = off
 *  layout       0: two copies of each population set (A/B: the step reads
 *               one and writes the other; the fastest step); 1: one copy,
 *               updated in place (AA pattern: steps alternate between writing
 *               each node's post-collision populations into its own opposite
 *               slots and reading/writing them at the neighbours), half the
 *               population memory; each step then forms phi in a separate
 *               pass first.  Both give the same results, bit for bit.
 *               lbm_advect_phase needs layout 0.
 *  rho_L, rho_H densities (eq:density_interpolation)
 *  tau_L, tau_H relaxation times, nu = tau c_s^2 (eq:kinematic_viscosity)
 *  mu_ratio     viscosity ratio mu_H / mu_L; when > 0 it replaces tau_L:
 *               tau_L = tau_H (rho_H / rho_L) / mu_ratio (mu_X = rho_X tau_X c_s^2)
 *  sigma, W     surface tension and interface width xi
 *               (eq:beta_kappa_relation)
 *  mobility     M = tau_phi c_s^2 (eq:mobility_relation)
 *  force[3]     body-force acceleration g; F_b = (rho - rho_ref) g
 *               (eq:gravity_force); force[2] is ignored in 2D
 *  rho_ref      reference density of the body force
 *  inlet_u      plug speed u_j along the inward normal of the inlet face
 *  inlet_center nozzle centre (x[, y]) in the inlet plane
 *  inlet_radius nozzle radius (2D: half width of the slot); the inlet
 *               profile is phi_in = 1/2 + 1/2 tanh(2 (R - r) / W), u_in = u_j
 *               for r < R and 0 elsewhere.
 */
typedef struct {
    int32_t lattice, nx, ny, nz;
    int32_t bc[6];
    int32_t visc_model;
    int32_t storage;
    int32_t outlet_scheme;
    int32_t diag_every;
    int32_t layout;
    int32_t reserved;       /* 0 */
    double rho_L, rho_H, tau_L, tau_H;
    double mu_ratio;
    double sigma, W, mobility;
    double force[3];
    double rho_ref;
    double inlet_u;
    double inlet_center[2];
    double inlet_radius;
    double storage_scale;   /* power-of-two scale of f in 16-bit storage;
                               0 = 2048 (a deviation f_a / w_a - r_m from
                               ~3e-8 to ~30 in float16 normal range) */
} lbm_params;

/* FP64 diagnostics of the current state (lbm_diag). */
typedef struct {
    double sum_phi;    /* sum of phi over all nodes (mass, Sec. 5.4) */
    double sum_p_in;   /* sum of p = p* rho c_s^2 over nodes with phi >= 1 - eps */
    double sum_p_out;  /* sum of p over nodes with phi <= eps */
    double max_speed;  /* max |u| */
    int64_t n_in, n_out;
    int32_t finite;    /* 1 if every population is finite */
    int32_t reserved;
    double dp_laplace; /* sum_p_in / n_in - sum_p_out / n_out (eq:laplace_law);
                          0 when either set is empty */
} lbm_diag_out;

/* Create a context: validate p, allocate the populations (2 sets x 2
 * buffers, or 1 buffer with layout 1, x Q values per node, rows padded to a
 * multiple of 32 nodes, 4 or 2 bytes per value by `storage`) on the current CUDA
 * device and bind the CUDA stream `stream` (a cudaStream_t; NULL = the legacy
 * default stream).  Errors: LBM_ERR_ARG (out == NULL, a parameter out of
 * range, unpaired periodic faces, inlet/outlet on another face, last axis
 * shorter than 4 with open faces, an inlet without the outlet on the
 * opposite face, W < 2, a negative diag_every, layout not 0 or 1),
 * LBM_ERR_CUDA (no device),
 * LBM_ERR_OOM.  On failure *out is NULL. */
int lbm_create(const lbm_params* p, void* stream, lbm_ctx** out);

/* Set the state to the equilibria of the given fields (eq:equilibrium,
 * eq:equilibrium_function): g_a = phi Gamma_a(u), f_a = p* w_a + Gamma_a(u)
 * - w_a.  phi: [N]; u: [D][N] or NULL (zero); pstar: [N] or NULL (zero),
 * p* = p / (rho c_s^2).  Host arrays that are page-locked (cudaHostAlloc,
 * cudaHostRegister, torch pin_memory) are read by the kernel in place; other
 * host arrays are copied to the device first.  Synchronises when on_device
 * is 0. */
int lbm_init_fields(lbm_ctx* ctx, const float* phi, const float* u, const float* pstar,
                    int on_device);

/* Advance nsteps >= 0 time steps (collision, streaming, boundary conditions
 * and macroscopic update of Algorithms 1-3, fused).  Asynchronous.  Runs of
 * 16 steps are replayed as one CUDA graph (captured on first use, kept until
 * lbm_destroy; not while kernel timing is on, nor after a capture was
 * refused, e.g. inside the caller's own global-mode stream capture), the rest
 * launched one by one; the results are the same either way.
 * With diag_every = k > 0, after every k-th step (counted from the last
 * lbm_init_fields / lbm_set_populations) the FP64 diagnostics of lbm_diag
 * (phase threshold 1e-3) run on the stream and lbm_step waits for them: when
 * a population is not finite it stops there and returns LBM_ERR_DIVERGED
 * (the state of that step stays readable; lbm_diag_last gives the record).
 * Errors: LBM_ERR_STATE before lbm_init_fields / lbm_set_populations;
 * LBM_ERR_CUDA when a launch or the graph capture fails; LBM_ERR_DIVERGED. */
int lbm_step(lbm_ctx* ctx, int64_t nsteps);

/* The record of the last in-step diagnostic of lbm_step (diag_every) and the
 * step count it was taken at (*step = -1 and *out zeroed if none yet).  Does
 * not touch the device. */
int lbm_diag_last(const lbm_ctx* ctx, lbm_diag_out* out, int64_t* step);

/* Macroscopic fields of the current state, computed with the same device
 * code as the step: phi [N], u [D][N] (eq:velocity_update), p [N]
 * (p = p* rho c_s^2).  Any output may be NULL.  Page-locked host outputs are
 * written by the kernel in place, other host outputs through a device copy.
 * Synchronises when on_device is 0. */
int lbm_get_fields(lbm_ctx* ctx, float* phi, float* u, float* p, int on_device);

/* Raw state (checkpoint): the post-streaming populations f and g, each
 * [Q][N] float32 (either may be NULL in lbm_get_populations), in the same
 * order whatever the layout.  With float32 storage lbm_set_populations
 * restores it exactly; with 16-bit storage the values are decoded to float32
 * and encoded again on restore: g (storage 1: fixed point) exactly, f to
 * within half a step of its 16-bit format (storage 1: where f_a / w_a lies
 * within ~2^-11 of the plane reference, float16 resolves more than the
 * float32 value carries, so a restart is not bit for bit).  The conversion
 * goes through a staging buffer of 4 N floats (allocated on first use).
 * Synchronises. */
int lbm_get_populations(lbm_ctx* ctx, float* f, float* g, int on_device);
int lbm_set_populations(lbm_ctx* ctx, const float* f, const float* g, int on_device);

/* FP64 reductions of the current state (deterministic order): sum phi, the
 * pressure sums inside (phi >= 1 - phase_eps) and outside (phi <= phase_eps)
 * for the Laplace test (eq:laplace_law), max |u| and a finite check.
 * Synchronises.  Returns LBM_ERR_DIVERGED (with *out filled) when a
 * population is not finite. */
int lbm_diag(lbm_ctx* ctx, double phase_eps, lbm_diag_out* out);

/* Kernel timing (tracing).  With enable != 0, lbm_step records CUDA events
 * on the context's stream around its kernels; lbm_get_timing synchronises,
 * returns the summed device time in milliseconds of (0) work before the main
 * kernel (0 with the single-pass step), (1) the fused collide-stream kernel,
 * (2) the face kernels (inlet, outlet) and the number of steps recorded, then
 * clears the record.  Timing is off by
 * default.  ms may not be NULL; it has room for 3 values. */
int lbm_set_timing(lbm_ctx* ctx, int enable);
int lbm_get_timing(lbm_ctx* ctx, double* ms, int64_t* nsteps);

/* lbm_diag without a context and without allocating: for callers that
 * cannot allocate device memory (code running where cudaMalloc is forbidden
 * or would bypass an allocator that must own every byte, e.g. a host
 * framework's caching allocator, a real-time loop, a plug-in that is only
 * handed buffers).  The paper has no counterpart; this is a library service.
 * p describes the grid and physics as for lbm_create (its storage field is
 * ignored); f and g are device pointers to float32 post-streaming populations
 * [Q][N] each (the layout of lbm_get_populations); out is a host pointer.
 * The same kernels as lbm_diag run on `stream` with their scratch (phi, the
 * inlet profile, the reduction partials) in one static device array of the
 * library: at most 2,097,152 nodes and, with an inlet face, 65,536
 * inlet-plane nodes (LBM_ERR_ARG beyond that).  The array (about 8.6 MB)
 * stays on every device that loads the library until exit.  The first call
 * on a device looks up the array's device address and keeps it for that
 * device's primary context (not valid after cudaDeviceReset or under another
 * driver context); make that call before any stream capture.  All calls
 * share the array and rewrite
 * everything they read, so results do not depend on earlier calls, but calls
 * that overlap on the GPU race.  Synchronises `stream`.  Errors as lbm_diag;
 * their text is returned by lbm_last_error(NULL). */
int lbm_diag_noalloc(const lbm_params* p, const float* f, const float* g, double phase_eps,
                     lbm_diag_out* out, void* stream);

/* Wait for all work enqueued on the context's stream. */
int lbm_sync(lbm_ctx* ctx);

/* Number of nodes N = nx*ny*nz and populations Q of a context. */
int lbm_shape(const lbm_ctx* ctx, int64_t* n_nodes, int32_t* q);

/* Text of the last error of ctx (never NULL; "" if none).  With ctx == NULL,
 * the last error of a failed lbm_create on this thread. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Free all device memory of ctx (after synchronising its stream). */
int lbm_destroy(lbm_ctx* ctx);

/* Advance only the phase field by nsteps in the prescribed velocity field
 * scale * u (u: D planes [nz][ny][nx], host or device per on_device): the
 * conservative Allen-Cahn step of eq:lbe_interface with the forcing term
 * eq:forcing_term and g^eq = phi Gamma(u), then streaming of g with the face
 * rules; f is left as it is.  This is the frozen-velocity mode of the
 * paper's circular interface in a shear flow (Sec. 5.3, eq:velocity_u,
 * eq:velocity_v).  Faces must be periodic, walls or free slip, and the
 * layout 0 (LBM_ERR_ARG otherwise).
 * With host u the call synchronises the stream. */
int lbm_advect_phase(lbm_ctx* ctx, const float* u, double scale, int64_t nsteps, int on_device);

/* Jet post-processing (Sec. 6: breakup length L_b and drop size d_e): the
 * liquid phi > threshold of the current state is split into connected
 * components (face neighbours, wrapped across periodic faces).  The largest
 * component touching the first plane of the last axis (the inlet side) is
 * the intact jet, and breakup_length is its extent along that axis (cells
 * from the plane to its farthest node, inclusive); every other component is
 * a drop, with equivalent diameter 2 sqrt(A / pi) (2D) or (6 V / pi)^(1/3)
 * (3D) from its cell count.  Up to max_drops drop volumes (cells, in no
 * particular order) are written to drop_volumes (may be NULL).  Allocates
 * 16 bytes per node of scratch on the first call; synchronises the stream. */
typedef struct {
    int32_t n_components;        /* liquid components */
    int32_t has_jet;             /* 1 if a component touches the first plane */
    double breakup_length;       /* cells; 0 without a jet */
    int32_t n_drops;             /* components other than the jet */
    int32_t truncated;           /* 1 if more drops than max_drops were found */
    double mean_drop_diameter;   /* cells; 0 without drops */
    double drop_volume;          /* total cells of the drops */
} lbm_jet_stats_out;

int lbm_jet_stats(lbm_ctx* ctx, double threshold, int32_t max_drops, double* drop_volumes, lbm_jet_stats_out* out);

/* Test hook: macroscopic update and collision of n independent cells with
 * the device code of the step (Algorithm 1 with eq:mrt_collision in moment
 * space).  Device pointers: f, g [n][Q] post-stream populations; phin
 * [n][Q] = phi(x + e_a) of each cell; fs, gs [n][Q] outputs; out [n][5] =
 * {phi, u_x, u_y, u_z, p} (may be NULL).  Uses the physical parameters of p;
 * the grid and faces of p are ignored.  Synchronises the stream. */
int lbm_collide_cells(const lbm_params* p, int64_t n, const float* f, const float* g,
                      const float* phin, float* fs, float* gs, float* out, void* stream);

/* ---------------------------------------------------------- batched sweeps
 *
 * A batch holds many independent cases of one lattice and one storage format
 * (float32 or float16), each with its own grid and physical parameters, and
 * advances all of them together: one time step of the batch is one time step
 * (the fused update of Algorithms 1-3) of every case.  Faces must be periodic
 * or walls (no inlet or outlet).  The cases are grouped into size classes by
 * nx; each class runs one persistent kernel per step over a device work list
 * of (case, tile segment) items, taken from a per-launch counter so that
 * items of unequal size balance themselves, and the classes run concurrently
 * on their own streams.  The steps are recorded once into CUDA graphs and
 * replayed.  A plan gives, per class, the tile width, the planes per work
 * item and the persistent blocks per SM; lbm_batch_tune measures candidate
 * plans on the batch itself and keeps the fastest.  Each case computes
 * exactly what a context of its own (lbm_create with the same parameters)
 * computes, bit for bit.
 *
 * The batch runs on `stream`; with stream == NULL it owns a blocking stream
 * (the legacy default stream cannot be recorded into a graph).  Calls that
 * return data synchronise that stream. */
typedef struct lbm_batch lbm_batch;   /* opaque; owns all device memory */

#define LBM_BATCH_MAX_CLASSES 8

typedef struct {
    int32_t nclasses;                           /* size classes in use */
    int32_t nx_max[LBM_BATCH_MAX_CLASSES];      /* class k holds cases with nx_max[k-1] < nx <= nx_max[k] */
    int32_t ncases[LBM_BATCH_MAX_CLASSES];      /* cases in the class */
    int32_t tile_x[LBM_BATCH_MAX_CLASSES];      /* tile width: 32, 64 or 128 (D2Q9), 32 (D3Q19, 32 x 8) */
    int32_t seglen[LBM_BATCH_MAX_CLASSES];      /* planes of the march axis per work item (>= 1) */
    int32_t blocks_per_sm[LBM_BATCH_MAX_CLASSES]; /* persistent blocks per SM (1 .. occupancy) */
    double ms_per_step[LBM_BATCH_MAX_CLASSES];  /* last measurement of lbm_batch_tune (0 if none) */
} lbm_batch_plan;

/* Create a batch of ncases cases from params[0 .. ncases-1] (each validated
 * like lbm_create; all with the same lattice and storage, storage 0 or 1,
 * faces periodic or wall, layout 0; diag_every is not used).  Allocates the populations of every case (two
 * buffers per set).  Returns LBM_ERR_ARG, LBM_ERR_CUDA or LBM_ERR_OOM on
 * failure (*out = NULL; text from lbm_batch_last_error(NULL)). */
int lbm_batch_create(const lbm_params* params, int32_t ncases, void* stream, lbm_batch** out);

/* Equilibrium initialisation of case c from its fields, as lbm_init_fields
 * (phi [nz][ny][nx]; u D planes or NULL; pstar or NULL). */
int lbm_batch_init_fields(lbm_batch* b, int32_t c, const float* phi, const float* u, const float* pstar,
                          int32_t on_device);

/* Advance every case by nsteps time steps (enqueued; returns at once).
 * LBM_ERR_STATE if a case has not been initialised. */
int lbm_batch_step(lbm_batch* b, int64_t nsteps);

/* Macroscopic fields of case c, as lbm_get_fields. */
int lbm_batch_get_fields(lbm_batch* b, int32_t c, float* phi, float* u, float* p, int32_t on_device);

/* FP64 diagnostics of case c, as lbm_diag. */
int lbm_batch_diag(lbm_batch* b, int32_t c, double phase_eps, lbm_diag_out* out);

/* Read or replace the plan.  set: each class's fields tile_x, seglen and
 * blocks_per_sm are checked (LBM_ERR_ARG when out of range); nclasses,
 * nx_max and ncases must equal those of the batch. */
int lbm_batch_get_plan(const lbm_batch* b, lbm_batch_plan* plan);
int lbm_batch_set_plan(lbm_batch* b, const lbm_batch_plan* plan);

/* Autotuner: for every class, time each candidate (tile width 32, 64, 128
 * for D2Q9; planes per item 4, 16, 64 for D2Q9 and 4, 8, 16, 32 for D3Q19;
 * blocks per SM: the occupancy and half of it) over trial_steps launches of
 * that class alone (one
 * step from the current state, repeated: the state is not advanced), keep
 * the fastest, and return the resulting plan (may be NULL).  Synchronises. */
int lbm_batch_tune(lbm_batch* b, int32_t trial_steps, lbm_batch_plan* plan);

/* Wait for the batch's queued work. */
int lbm_batch_sync(lbm_batch* b);

/* Last error text of b (never NULL); with b == NULL, that of the last failed
 * lbm_batch_create on this thread. */
const char* lbm_batch_last_error(const lbm_batch* b);

/* Free all device memory of b (after synchronising its stream). */
int lbm_batch_destroy(lbm_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
