/*
 * pflb.h -- C ABI of the GB300 phase-field lattice Boltzmann library.
 *
 * One time step advances the two D3Q19 population sets of the conservative
 * Allen-Cahn phase-field lattice Boltzmann method of "Capillary flow
 * simulation with the phase-field-based lattice Boltzmann solver"
 * (arXiv 2512.01032):
 *   h_i : phase-field populations, Eqs. 1-4 (with the local mobility
 *         correction of Eq. 4);
 *   g_i : hydrodynamic populations (the paper's g-bar), Eqs. 5-11 (filtered
 *         collision, force K_i with the chemical potential of Eq. 7);
 * with the central-difference gradient and Laplacian of Eq. 13, the
 * wettability ghosts of Eqs. 12-15 and the optimised friction model of
 * Sec. III A (tanh F(phi), free-slip band, hysteresis blend) at solid voxels.
 *
 * Conventions shared by every call:
 *   - Lattice units (the paper's Sec. I convention), T = 1/3.
 *   - Cells are indexed x fastest: cell = x + nx*(y + ny*z).  The box is
 *     periodic in x, y and z; walls are solid voxels.
 *   - The library owns all device memory of a lattice; the caller owns every
 *     host buffer.  Input arrays are copied before the call returns.
 *   - Every call returns a pflb_status; no exception crosses the ABI.  After
 *     a CUDA error the lattice is poisoned: later calls return
 *     PFLB_ERR_STATE.  pflb_last_error() gives a thread-local message.
 *   - Work is ordered on the CUDA stream given at creation (NULL = the
 *     legacy default stream).  pflb_step is asynchronous; pflb_read,
 *     pflb_diag and pflb_save synchronise that stream.
 */
#ifndef PFLB_H
#define PFLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pflb_lattice pflb_lattice;

typedef enum {
  PFLB_OK = 0,
  PFLB_ERR_ARG = 1,     /* invalid argument or parameter */
  PFLB_ERR_OOM = 2,     /* out of device memory, or a host allocation failed */
  PFLB_ERR_CUDA = 3,    /* a CUDA call failed, including no usable device (a lattice
                           that exists is poisoned) */
  PFLB_ERR_NAN = 4,     /* a diagnostic found non-finite fields */
  PFLB_ERR_TIMEOUT = 5, /* a bounded wait ran out */
  PFLB_ERR_BUDGET = 6,  /* request exceeds the memory budget */
  PFLB_ERR_STATE = 7    /* lattice poisoned by an earlier error */
} pflb_status;

/* Population storage.  The collision computes in FP64 for FP64 storage and
 * in FP32 otherwise.  FP16 stores each population divided by its lattice
 * weight, h_i / w_i and g_i / w_i (at rest these are phi and P/T, so every
 * stored value has the scale of a macroscopic field, clear of FP16's
 * subnormals); BF16, whose exponent range is FP32's, stores the value
 * itself.  Both 16-bit formats compensate the rounding of a cell's moving h
 * in its rest population so that total phi does not drift (bytes per cell
 * and step: 305 at FP32, 157 at FP16/BF16, 609 at FP64). */
enum { PFLB_STORAGE_FP64 = 0, PFLB_STORAGE_FP32 = 1, PFLB_STORAGE_FP16 = 2,
       PFLB_STORAGE_BF16 = 3 };

/* Fields for pflb_read. */
enum { PFLB_FIELD_PHI = 0, PFLB_FIELD_RHO = 1, PFLB_FIELD_P = 2,
       PFLB_FIELD_UX = 3, PFLB_FIELD_UY = 4, PFLB_FIELD_UZ = 5 };

/* Step kernels.  Every kind computes the same step; they differ in how the
 * populations reach the arithmetic:
 *   PFLB_KERNEL_PIPE (default): the fused z-marching pass with each thread's
 *     populations of the next planes copied into shared memory one plane
 *     ahead (cp.async in 16-byte chunks; 8-byte chunks at FP16/BF16 storage
 *     when nx is not a multiple of 8), 32 x 4 tiles, pair form of the
 *     collision, each block's wall nodes updated after its march (one
 *     launch per step); periodic x and nx a multiple of 4, otherwise
 *     PFLB_KERNEL_FUSED runs;
 *   PFLB_KERNEL_FUSED: one fused z-marching pass with direct loads;
 *   PFLB_KERNEL_TWOPASS: a phi pass followed by a per-cell pass;
 *   PFLB_KERNEL_FUSED_TMA: the fused pass with h staged through shared
 *     memory by TMA (FP32 storage, nx a multiple of 4 and nx >= 64;
 *     otherwise PFLB_KERNEL_FUSED runs). */
enum { PFLB_KERNEL_FUSED = 0, PFLB_KERNEL_TWOPASS = 1, PFLB_KERNEL_FUSED_TMA = 2,
       PFLB_KERNEL_PIPE = 3 };

/* Geometry, read during pflb_create only.
 *   solid       : host, nx*ny*nz bytes, nonzero = solid voxel.
 *   wall_normal : host, 3 doubles per cell (x,y,z), unit normal pointing into
 *                 the fluid, read at wall nodes (fluid cells with a solid
 *                 D3Q19 neighbour); NULL = estimate from the mask as the
 *                 normalised -sum_i w_i c_i [x + c_i solid].
 *   theta_deg   : host, one input contact angle per cell (degrees, measured
 *                 inside the phi = 1 phase), read at wall nodes; NULL = use
 *                 params.theta_deg everywhere.
 *   solid_frac  : host, one double per cell, or NULL (voxel walls).  Walls
 *                 that cut fluid cells (Sec. II B's volume-weighted sampling;
 *                 the offset walls of Sec. IV A): the solid volume fraction s
 *                 of each fluid cell, in [0, 1) (values on solid voxels are
 *                 ignored; a fluid value outside [0, 1) is PFLB_ERR_ARG).  A
 *                 cut cell (s > 0) stays a fluid cell (bounce-back acts only
 *                 at links into solid voxels); a fluid cell next to one is a
 *                 wall node that keeps a ghost for that link, and its CD
 *                 stencils take s_y ghost + (1 - s_y) phi(y) for the cut
 *                 neighbour y; a cut wall node samples phi as
 *                 (1 - s) phi(x) + s phi(x + c_n), c_n the axis direction
 *                 nearest its wall normal.  Wall normals are read at these
 *                 wall nodes too (NULL: the fraction-weighted mask). */
typedef struct {
  int nx, ny, nz;
  const uint8_t *solid;
  const double *wall_normal;
  const double *theta_deg;
  const double *solid_frac;
} pflb_geometry;

/* Model parameters (lattice units).
 *   sigma, W, M       : surface tension, interface width, mobility (Eqs. 1-7)
 *   rho_H, rho_L      : densities of the phi = 1 (heavy) and phi = 0 phases;
 *                       rho = rho_L + phi (rho_H - rho_L)
 *   nu_H, nu_L        : kinematic viscosities; tau = nu/T + 1/2 (Eq. 8)
 *   theta_deg         : default input contact angle (Sec. II B)
 *   Fex               : external body force (Eq. 6)
 *   gamma, phi_M, phi_m, D, eps : mobility correction constants (Eq. 4)
 *   blend             : hysteresis blend b: ghost = b old + (1-b) new
 *   band_lo, band_hi  : free-slip band on phi (Sec. III A)
 *   F_tilde, F_width  : optimised F(phi) = (tanh((phi-F_tilde)/F_width)+1)/2
 *   F_mode            : 0 = F(phi) = phi, 1 = optimised tanh F
 *   mobility_corr     : 1 = add delta-theta of Eq. 4
 *   free_slip         : 1 = specular reflection of edge links at flat
 *                       axis-aligned walls when phi at both wall nodes of
 *                       the link pair lies in the band
 *   storage           : PFLB_STORAGE_* */
typedef struct {
  double sigma, W, M, rho_H, rho_L, nu_H, nu_L, theta_deg;
  double Fex[3];
  double gamma, phi_M, phi_m, D, eps, blend, band_lo, band_hi, F_tilde, F_width;
  int F_mode, mobility_corr, free_slip, storage;
} pflb_params;

/* Diagnostics of the current state, accumulated in FP64 on the device.
 *   mass        : sum of phi over fluid cells
 *   n_heavy     : number of fluid cells with phi >= 0.5
 *   p_heavy/p_light : mean P over fluid cells with phi > 0.95 / phi < 0.05
 *   dp          : p_heavy - p_light (pressure jump)
 *   u_max       : max |u| over fluid cells
 *   region_mass : sum of phi over the box set by pflb_set_region
 *   cl_count, cl_mean[3], cl_m2[3] : wall nodes with 0.25 <= phi <= 0.75
 *                 (contact-line band): count, mean and mean square position
 *   kinetic     : sum of rho |u|^2 / 2
 *   nonfinite   : number of fluid cells with a non-finite phi, P or u
 *   front_x, rear_x : interface position along x (Sec. III C: the phi = 0.5
 *                 contour), over fluid cells of the region box whose +x
 *                 neighbour is fluid, linearly interpolated between the two:
 *                 front_x = the largest x at which phi falls through 0.5
 *                 going +x (the advancing front of liquid entering from low
 *                 x), rear_x = the smallest x at which phi rises through 0.5;
 *                 -1 where there is no such crossing.  On a periodic x axis a
 *                 crossing between x = nx-1 and x = 0 lies in [nx-1, nx). */
typedef struct {
  int64_t step;
  double mass, n_heavy, p_heavy, p_light, n_p_heavy, n_p_light, dp, u_max;
  double region_mass;
  double cl_count, cl_mean[3], cl_m2[3];
  double kinetic;
  double nonfinite;
  double front_x, rear_x;
} pflb_diag_t;

/* Fill p with the paper's defaults: gamma = -22.5, phi_M = 0.8,
 * phi_m = 0.2, D = 1e-4, eps = 1e-10 (Eq. 4); blend = 0.95, band
 * [0.5, 0.95], F_tilde = 0.1, F_width = 0.001 (Sec. III A); the remaining
 * physical values are those of the static-droplet case (sigma = 0.01,
 * W = 4, M = 0.02, rho ratio 1000, nu = 0.1), FP32 storage. */
void pflb_default_params(pflb_params *p);

/* Create a lattice from geometry and parameters.  Validates parameters
 * (dimensions >= 1 with nx*ny*nz < 2^31, W > 0, M > 0, nu > 0 so that
 * tau > 1/2, rho_L > 0,
 * rho_H > 0, 0 <= blend <= 1, storage known) and returns PFLB_ERR_ARG
 * otherwise.  cuda_stream: a cudaStream_t or NULL.  On success *out owns
 * all device memory (about 228 B/cell at FP32 storage); the state is
 * zero until an init call. */
pflb_status pflb_create(const pflb_geometry *geom, const pflb_params *params, void *cuda_stream,
                        pflb_lattice **out);

/* Initialise phi from the steady tanh profile of Eq. 12 and set the
 * equilibrium state (u = 0, P = P0, h = h_eq, g = g_eq with K_i from the
 * initial gradient, wetting ghosts = phi of the wall node); resets the
 * step counter.
 *   shape 0 (sphere): phi = (1 + tanh(2 (R - r)/W))/2, r = minimum-image
 *           distance from center (cell centres at integer coordinates);
 *   shape 1 (half space): phi = (1 + tanh(2 d/W))/2, d = (center - x).normal;
 *   shape 2 (slab): phi = (1 + tanh(2 (R - |d|)/W))/2.
 * normal may be NULL for shape 0.  phi is zero on solid cells.  The
 * initialisation runs asynchronously on the lattice stream (the host data is
 * copied before return). */
pflb_status pflb_init_tanh(pflb_lattice *L, int shape, const double center[3], double R,
                           const double normal[3], double P0);

/* Same from a host phi array (nx*ny*nz doubles; solid cells ignored). */
pflb_status pflb_init_phi(pflb_lattice *L, const double *phi_host, double P0);

/* Set the external body force F_ex of Eq. 6 for the following steps. */
pflb_status pflb_set_force(pflb_lattice *L, const double Fex[3]);

/* Box [lo, hi) (x0,x1,y0,y1,z0,z1) over which region_mass is summed. */
pflb_status pflb_set_region(pflb_lattice *L, const int box[6]);

/* Choose the step kernel and its launch shape: tile bx * by threads
 * (bx * by a multiple of 32 up to 256, 2 (bx+2) + 2 by <= bx * by; whole
 * warps, for the warp reductions of the diagnostics) marching lz planes in z
 * (the TMA kernel always uses 32 x 8 and takes only lz).  Defaults:
 * 32 x 4 and automatic lz.  Zeros keep the current values; lz = -1 returns
 * to the automatic choice, which minimises the launch's rounds of resident
 * blocks times the planes per block (plus its halo cost) over lz in
 * [2, 32], from the device's SM count and the kernel's occupancy. */
pflb_status pflb_set_kernel(pflb_lattice *L, int kind, int bx, int by, int lz);

/* Open x boundaries (Sec. IV A: "standard" Dirichlet pressure with Neumann
 * velocity and phi; velocity inlets).  The fluid cells of the planes x = 0
 * (lo) and x = nx-1 (hi) become boundary cells; both planes must be given
 * (NULL for both restores periodic x).  Each step, before the update, a
 * boundary state (phi_b, P_b, u_b) is formed per boundary cell:
 *   PFLB_XBC_PRESSURE: P_b = P; phi_b and u_b are those of the adjacent
 *     interior cell (x = 1 or nx-2) in bulk form (phi = sum h,
 *     rho u = sum c g + F/2);
 *   PFLB_XBC_VELOCITY: u_b = u and phi_b = phi; P_b = T sum g of the
 *     adjacent interior cell.
 * A boundary cell is not collided: its post-collision populations are the
 * equilibria h_i = phi_b Gamma_i(u_b), g_i = w_i P_b / T +
 * rho_b (Gamma_i(u_b) - w_i), streamed as usual (bounce-back at solid
 * links), and whatever streams into it is discarded.  Boundary cells carry
 * no diagnostics and read back their boundary state.  First-order accurate
 * (equilibrium boundary).  Lattices with open boundaries run the fused or
 * two-pass kernel (not the TMA one); in a batch their boundary states are
 * formed by one extra kernel per step over all such lattices. */
enum { PFLB_XBC_PRESSURE = 1, PFLB_XBC_VELOCITY = 2 };
typedef struct {
  int type;        /* PFLB_XBC_PRESSURE or PFLB_XBC_VELOCITY */
  double P;        /* pressure (pressure boundary) */
  double u[3];     /* velocity (velocity boundary) */
  double phi;      /* order parameter (velocity boundary) */
  int64_t ramp_steps; /* > 0: the given values are reached linearly over this many
                         steps from those in effect at the call (the rest state,
                         P = 0 and u = 0, when the boundaries were off); a function
                         of the step counter, so reads do not advance it */
} pflb_xbc;

pflb_status pflb_set_x_boundaries(pflb_lattice *L, const pflb_xbc *lo, const pflb_xbc *hi);

/* The launch shape in effect: out = {kind, bx, by, lz}. */
pflb_status pflb_get_kernel(const pflb_lattice *L, int out[4]);

/* Autotuner of the planes per block (no counterpart in the paper: a launch
 * parameter of this library's kernels).  For the kernel kind in effect it
 * times trial_steps steps at each of a fixed set of depths (the automatic
 * choice, 4, 6, 8, 10, 12, 16, 24, 32 planes, those not above nz) on the
 * lattice itself, keeps the fastest (as pflb_set_kernel with that lz) and
 * returns it in *lz_out if not NULL.  The trial steps are real steps: the
 * lattice advances by (trial_steps + 1) per depth tried.  Results do not
 * depend on the depth (the per-cell arithmetic is the same).  Synchronises
 * the lattice stream; not for use inside stream capture.  Errors:
 * PFLB_ERR_ARG (trial_steps < 1), PFLB_ERR_CUDA. */
pflb_status pflb_tune(pflb_lattice *L, int trial_steps, int *lz_out);

/* Advance nsteps time steps (asynchronous on the lattice stream). */
pflb_status pflb_step(pflb_lattice *L, int64_t nsteps);

/* Make pflb_step accumulate the diagnostics (pflb_diag_t) inside the step
 * kernel on every k-th step (step index divisible by k), at the cost of a
 * block reduction and a few FP64 atomics per block; 0 (the default) turns
 * this off.  The values describe the state each such step consumed. */
pflb_status pflb_set_diag_every(pflb_lattice *L, int k);

/* Diagnostics accumulated by the most recent step that computed them;
 * out->step is that step's index.  Synchronises.  PFLB_ERR_STATE if no step
 * has computed diagnostics since the last init; PFLB_ERR_NAN (with *out
 * filled) when a non-finite value was found. */
pflb_status pflb_last_diag(pflb_lattice *L, pflb_diag_t *out);

/* Asynchronous form of pflb_last_diag, for stepping loops that read every
 * step's diagnostics without stalling the GPU.  pflb_last_diag_async queues,
 * on the lattice stream, a copy of the raw accumulators of the most recent
 * diagnostic step (and the device error flag) into raw, caller host memory
 * that must stay valid until the matching wait (page-locked memory keeps the
 * call from blocking on the copy), and returns a ticket.  pflb_diag_wait
 * blocks until that copy has landed and decodes raw into out (status as
 * pflb_last_diag).  At most 16 reads per lattice may be outstanding; a
 * ticket is valid until 16 newer reads have been queued. */
typedef struct {
  double acc[32];
  int64_t step;
  int32_t err;
  int32_t pad;
} pflb_diag_raw_t;

pflb_status pflb_last_diag_async(pflb_lattice *L, pflb_diag_raw_t *raw, int64_t *ticket);
pflb_status pflb_diag_wait(pflb_lattice *L, int64_t ticket, const pflb_diag_raw_t *raw,
                           pflb_diag_t *out);

/* Advance nsteps >= 1 steps, the last of them accumulating diagnostics, and
 * return those (as pflb_last_diag; synchronises). */
pflb_status pflb_step_diag(pflb_lattice *L, int64_t nsteps, pflb_diag_t *out);

/* Advance nsteps steps asynchronously; with diag_last != 0 (then nsteps >= 1)
 * the last step accumulates diagnostics, read later with pflb_last_diag. */
pflb_status pflb_step_ex(pflb_lattice *L, int64_t nsteps, int diag_last);

/* Copy one macroscopic field of the current state (as the next step would
 * see it: phi = sum h, ghosts updated, P and u recovered) into host_out
 * (nx*ny*nz doubles; zero on solid cells).  Synchronises. */
pflb_status pflb_read(pflb_lattice *L, int field, double *host_out);

/* Diagnostics of the current state (synchronises).  Returns PFLB_ERR_NAN
 * (with *out filled) when a non-finite value was found, and
 * PFLB_ERR_TIMEOUT (lattice poisoned) when a bounded wait inside a step
 * kernel ran out; pflb_read and pflb_last_diag check the same flag. */
pflb_status pflb_diag(pflb_lattice *L, pflb_diag_t *out);

/* Number of steps taken since the last init. */
int64_t pflb_get_step(const pflb_lattice *L);

/* Bytes of device memory the lattice holds. */
int64_t pflb_device_bytes(const pflb_lattice *L);

/* Device memory a lattice of this geometry and storage would need (bytes),
 * counted from the mask without allocating (the lazily allocated field
 * output of pflb_read and the init scratch are not included); -1 on a bad
 * argument. */
int64_t pflb_estimate_bytes(const pflb_geometry *geom, int storage);

/* Checkpoint the full state (populations, wall buffers, ghosts, step) to a
 * file, and restore it into a lattice of identical geometry and storage.
 * A restored run continues bit for bit. */
pflb_status pflb_save(pflb_lattice *L, const char *path);
pflb_status pflb_load(pflb_lattice *L, const char *path);

/* Allocation-free field and diagnostic pass over caller-owned populations.
 * No counterpart in the paper: this serves callers that cannot allocate
 * device memory -- code whose device memory belongs to another allocator
 * (a framework's memory pool that must account for every byte) or that runs
 * in a latency-critical loop where cudaMalloc's implicit device
 * synchronisation is not acceptable.  It calls no cudaMalloc, cudaFree or
 * other allocating routine; its scratch (the phi field and the FP64
 * diagnostic accumulators) lives in file-scope device arrays sized for at
 * most 2^20 cells (about 4 MiB, held by every GPU that loads the library
 * until the process exits).
 *   nx, ny, nz : wall-free periodic lattice, nx*ny*nz <= 2^20, else
 *                PFLB_ERR_ARG with a message naming the limit.
 *   h_dev, g_dev : device, FP32, [19][N] each (direction-major, x fastest),
 *                slot i holding the population arriving in direction i (the
 *                layout pflb_save writes after an even number of steps).
 *   params     : model parameters (host, read during the call); storage
 *                must be PFLB_STORAGE_FP32, else PFLB_ERR_ARG.
 *   fields_dev : device, 6*N doubles (phi, rho, P, ux, uy, uz), or NULL.
 *   diag_out   : host, or NULL (at least one output); region_mass is the
 *                whole box, the contact-line fields are zero, front_x and
 *                rear_x are -1, step is -1.
 *   cuda_stream: stream to order the work on (NULL = legacy default); the
 *                call synchronises it when diag_out is given, and with
 *                diag_out given on a stream that is being captured it
 *                returns PFLB_ERR_ARG without enqueuing anything.
 * The first call on a device loads this entry point's device code on that
 * device (which is when the scratch is reserved) and looks up the scratch
 * addresses for it (cudaGetSymbolAddress with the device current); make that
 * first call before any stream capture.  Later calls allocate nothing.
 * Every call shares the same scratch, cleared at the start of each call:
 * calls that overlap on the GPU (different streams or threads) race and must
 * be serialised by the caller. */
pflb_status pflb_fields_noalloc(int nx, int ny, int nz, const float *h_dev, const float *g_dev,
                                const pflb_params *params, double *fields_dev,
                                pflb_diag_t *diag_out, void *cuda_stream);

/* ------------------------------------------------------------- batches
 * Many independent lattices (of any sizes) advanced together by persistent
 * kernels: a grid of (SMs x blocks per SM) blocks pulls work items -- one
 * per (lattice, tile column, chunk of z planes) -- from a device work list,
 * so small lattices that could not fill the GPU on their own share it.
 * Lattices that PFLB_KERNEL_PIPE can run (periodic x, nx a multiple of 4)
 * are marched by its pipelined per-cell code, 32 x 4
 * tiles with an automatic number of planes, their wall nodes by a second
 * small kernel; the others by the fused tile march with the launch shape
 * below.  No work item reads another lattice, so a lattice's result does
 * not depend on what it is batched with: it is bit-identical to the same
 * lattice in a batch of its own.  Against pflb_step on that lattice it
 * agrees to rounding (the two kernels are compiled separately and may
 * contract different multiply-adds).  Plain steps are replayed from a
 * captured CUDA graph of 16 steps.  The batch does not own the lattices;
 * they must outlive it, share one storage type, and appear once.  Work is
 * ordered on the batch stream (cuda_stream, or a stream the batch creates
 * when NULL), after and before the lattices' own streams. */
typedef struct pflb_batch pflb_batch;

pflb_status pflb_batch_create(pflb_lattice *const *lattices, int count, void *cuda_stream,
                              pflb_batch **out);

/* Launch shape of the fused tile march: bx * by threads per block (same
 * rules as pflb_set_kernel), lz planes per work item, blocks per SM (0 = as
 * many as fit, at most 4); zeros keep the current values (default
 * 32 x 4 x 16, 0). */
pflb_status pflb_batch_set_launch(pflb_batch *b, int bx, int by, int lz, int blocks_per_sm);

/* Autotuner: times trial_steps steps of each of a fixed set of launch shapes
 * on the batch itself (the steps are real steps of every lattice), keeps the
 * fastest and returns it in best (bx, by, lz, blocks per SM) if not NULL. */
pflb_status pflb_batch_tune(pflb_batch *b, int trial_steps, int best[4]);

/* Advance every lattice of the batch by nsteps (asynchronous).  With
 * diag_last != 0 the last step accumulates each lattice's diagnostics,
 * read afterwards with pflb_last_diag on that lattice. */
pflb_status pflb_batch_step(pflb_batch *b, int64_t nsteps, int diag_last);

/* Free the batch (not its lattices); NULL is ignored. */
void pflb_batch_destroy(pflb_batch *b);

/* ------------------------------------------------------------- serving
 * A native request server for many independent solves of the kind the
 * paper runs to find a critical (breakthrough) pressure (Sec. IV): each
 * request is a lattice, an initial state and a pressure ramp applied as a
 * body force, F_ex(t) = dir * beta(t) * p_ref / length with
 *   beta(t) = min(beta0 + dbeta * floor(t / ramp_every), beta_max),
 * run until breakthrough (the phi summed over the request's region box
 * exceeds threshold) or max_steps.  Continuous batching: every tick admits
 * queued requests in arrival order while their estimated device footprint
 * (pflb_estimate_bytes) fits the HBM budget (and the optional caps on
 * resident requests and cells), advances every resident request by
 * steps_per_tick steps (one persistent batch kernel per step, or one launch
 * per request in plain mode), checks each request's diagnostics once, and
 * retires the finished ones, freeing their memory.  Admission's host work
 * (building and uploading a new lattice) runs while the tick's steps run on
 * the GPU; admitted requests start at the next tick.
 * A request's trajectory does not depend on what it is batched with.
 * Latency = time from submit to the tick that finishes the request (host
 * steady clock).  Not thread-safe: one host thread drives a server. */
typedef struct pflb_server pflb_server;

typedef struct {
  size_t hbm_budget_bytes; /* admission limit on the sum of resident footprints */
  int storage;             /* population storage of every request (PFLB_STORAGE_*) */
  int steps_per_tick;      /* steps between breakthrough checks (>= 1) */
  int max_active;          /* resident request cap, 0 = budget only */
  int batched;             /* 1: one batch kernel per step; 0: one launch per request */
  int64_t max_active_cells;/* cap on the summed cells of resident requests, 0 = none (a
                              request larger than the cap still runs when it is alone) */
} pflb_server_config;

typedef struct {
  int init_shape;          /* pflb_init_tanh shape, centre, R and normal */
  double center[3];
  double R;
  double normal[3];
  double p_ref;            /* reference pressure (e.g. the capillary entry pressure) */
  double length;           /* length over which the ramp pressure acts */
  double dir[3];           /* unit force direction */
  double beta0, dbeta, beta_max;
  int64_t ramp_every;      /* multiple of steps_per_tick */
  int64_t max_steps;       /* multiple of steps_per_tick */
  int region[6];           /* breakthrough box x0,x1,y0,y1,z0,z1 */
  double threshold;        /* breakthrough when region_mass > threshold */
  int keep_phi;            /* keep the final phi field for pflb_server_fetch_phi */
  int drive;               /* 0: the ramp pressure as the body force above;
                              1: as a pressure difference across open x boundaries,
                              P = beta(t) p_ref at x = 0 and 0 at x = nx-1 (dir and
                              length unused), each change ramped over one tick
                              (from rest at admission) */
} pflb_solve_spec;

enum { PFLB_REQ_QUEUED = 0, PFLB_REQ_RUNNING = 1, PFLB_REQ_DONE = 2, PFLB_REQ_FAILED = 3,
       PFLB_REQ_REJECTED = 4 };

typedef struct {
  int state;               /* PFLB_REQ_* */
  int broke_through;       /* 1 if the region threshold was crossed */
  double beta;             /* ramp value at the finishing tick */
  int64_t steps;           /* steps run */
  double latency_s;        /* submit -> finish (0 until finished) */
  double queue_s;          /* submit -> admission */
  double region_mass, mass, u_max;  /* diagnostics of the last step */
} pflb_solve_result;

typedef struct {
  int64_t submitted, completed, failed, rejected, active, queued;
  double p50_s, p99_s, mean_s, max_s; /* latency percentiles of completed requests */
  double makespan_s;       /* first submit -> last completion */
  double solves_per_s;     /* completed / makespan_s */
  double cell_updates;     /* fluid-or-solid cells x steps advanced */
  size_t bytes_in_use, peak_bytes;
  int64_t ticks;
  double admit_s;          /* host time spent admitting (lattice build and upload) */
  double wait_s;           /* host time blocked on the GPU at the end of ticks */
  double retire_s;         /* host time spent checking and retiring requests */
} pflb_server_stats;

/* cuda_stream as pflb_create (NULL: the server creates its own). */
pflb_status pflb_server_create(const pflb_server_config *cfg, void *cuda_stream,
                               pflb_server **out);

/* Queue a request (the geometry arrays are copied).  A request whose
 * footprint alone exceeds the budget is REJECTED at once; the call still
 * returns PFLB_OK and a ticket (>= 1). */
pflb_status pflb_server_submit(pflb_server *s, const pflb_geometry *geom,
                               const pflb_params *params, const pflb_solve_spec *spec,
                               int64_t *ticket);

/* One tick: admit, advance, retire (synchronises once).  n_active (may be
 * NULL) receives the number of resident requests after the tick. */
pflb_status pflb_server_tick(pflb_server *s, int *n_active);

pflb_status pflb_server_poll(pflb_server *s, int64_t ticket, pflb_solve_result *out);

/* Copy the final phi (nx*ny*nz doubles, solids 0) of a finished request
 * submitted with keep_phi; n is the capacity of out in doubles. */
pflb_status pflb_server_fetch_phi(pflb_server *s, int64_t ticket, double *out, int64_t n);

pflb_status pflb_server_stats_get(pflb_server *s, pflb_server_stats *out);

/* Free the server and every resident lattice; NULL is ignored. */
void pflb_server_destroy(pflb_server *s);

/* Self-test of the failure-detection path (no counterpart in the paper).
 * Queues on the lattice's stream a kernel that waits, through the same
 * bounded-wait helper the staged step kernel uses for its TMA copies, on an
 * mbarrier that nothing completes; after `polls` polls (1 .. 2^20) the wait
 * gives up, raises the lattice's device error flag and the kernel returns,
 * so no fault occurs and the GPU context stays usable.  The lattice's next
 * synchronising call (pflb_read, pflb_last_diag, pflb_diag) then returns
 * PFLB_ERR_TIMEOUT and the lattice is poisoned (PFLB_ERR_STATE afterwards),
 * as after a real stalled copy.  Other lattices are unaffected. */
pflb_status pflb_selftest_wait_timeout(pflb_lattice *L, int64_t polls);

/* Free the lattice (synchronises its stream first).  NULL is ignored. */
void pflb_destroy(pflb_lattice *L);

/* Message of the last failing call on this thread ("" if none). */
const char *pflb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PFLB_H */
