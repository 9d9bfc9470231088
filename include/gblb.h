/*
 * gblb — RD3Q41 energy-conserving crystallographic lattice Boltzmann solver
 * for NVIDIA GB300 (sm_103a).  C ABI.
 *
 * Model (Kolluru, Atif, Namburi, Ansumali, arXiv:1909.08406):
 *   - 41 discrete velocities in five energy shells plus rest (Sec. IV,
 *     Table I): sc-1 (+-1,0,0), sc-2 (+-2,0,0), fcc-1 (+-1,+-1,0),
 *     bcc-1 (+-1,+-1,+-1), bcc-1/2 (+-1/2,+-1/2,+-1/2); w_0 = 1 - sum of the
 *     others and theta_0 = sum_i w_i c_ix^2 (Sec. III, Eq. allWeights).
 *   - bcc grid: two simple-cubic sub-lattices A (integer positions) and B
 *     (offset by (1/2,1/2,1/2)) (Sec. IV).  A grid of nx*ny*nz cells has
 *     2*nx*ny*nz nodes and is periodic in every direction.
 *   - discrete BGK update f_i(x + c_i, t + 1) = f_i + 2 beta (f_i^eq - f_i),
 *     beta = 1 / (2 tau + 1) (Sec. II), with the energy-conserving
 *     equilibrium of Sec. V, Eq. (feqGenU3): the rest-state equilibrium to
 *     O(eta^3), eta = theta/theta_0 - 1, times the velocity series with
 *     M_2, M_2', A_1, A_2.  M_2 and M_2' are evaluated exactly from the
 *     weights.  Unless LB_FLAG_PAPER_LITERAL is given, the equilibrium also
 *     carries the momentum projection f~_i c_i . dj / (rho theta) that
 *     makes momentum an exact collision invariant (the printed series
 *     misses it at O(u^3 eta^2)).
 *   - kinematic viscosity nu = tau theta_0; thermal diffusivity = nu
 *     (Prandtl number 1); isentropic sound speed sqrt(5 theta_0 / 3).
 *   - optional modes: the exact entropic equilibrium (LB_FLAG_ENTROPIC),
 *     kinetic walls normal to z (lb_set_walls), and the isothermal nonideal
 *     fluid with the van der Waals, Peng-Robinson type or Carnahan-Starling
 *     equation of state (lb_set_nonideal), each documented at its call.
 *
 * Array layouts (all C order, x fastest):
 *   scalar field   a[s][nz][ny][nx]            s = 0 (A), 1 (B)
 *   velocity       u[3][s][nz][ny][nx]         component-major
 *   populations    f[s][41][nz][ny][nx]        velocity order of lb_velocity_set
 * Scalar fields and populations crossing this interface are float64.
 *
 * Ownership: the context owns every device buffer it allocates (population
 * buffers, reduction partials, staging) and frees them in lb_destroy.  Caller
 * buffers stay the caller's: they are read or written during the call (or, for
 * device pointers, by work the call enqueues on the context's stream) and
 * never retained.  "on_device" != 0 means the pointer is device memory of the
 * context's GPU; 0 means host memory (pageable or pinned).
 *
 * Streams and errors: work is enqueued on the stream given to lb_init (NULL =
 * the legacy default stream).  Calls that return data to the host synchronise
 * that stream.  Every call returns an lb_status; lb_last_error gives a
 * message.  A device-side error word is set when a node's density or
 * temperature becomes non-positive or non-finite; it is sticky and is reported
 * as LB_ERR_UNSTABLE by lb_sync and every synchronising call.
 */
#ifndef GBLB_H
#define GBLB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_ERR_ARG = -1,      /* invalid argument (null pointer, size, enum)            */
    LB_ERR_OOM = -2,      /* device or host allocation failed                        */
    LB_ERR_CUDA = -3,     /* a CUDA runtime call failed (message in lb_last_error)   */
    LB_ERR_THETA0 = -4,   /* theta0 argument disagrees with the weights             */
    LB_ERR_UNSTABLE = -5, /* a node reached rho <= 0, theta <= 0 or a non-finite value */
    LB_ERR_TIMEOUT = -6,  /* a bounded device wait gave up                           */
    LB_ERR_STATE = -7     /* call not valid in the current state                    */
} lb_status;

typedef enum {
    LB_F64 = 0,      /* FP64 arithmetic, populations stored as FP64 f_i                 */
    LB_F32 = 1,      /* FP32 arithmetic, stored as FP32 h_i = f_i / w_i - 1              */
    LB_F32_S16F = 2, /* FP32 arithmetic, stored as FP16 2^8 h_i (round to nearest even) */
    LB_F32_S16B = 3  /* FP32 arithmetic, stored as BF16 h_i (round to nearest even)     */
} lb_precision;

#define LB_RD3Q41 41

/* lb_init flags */
#define LB_FLAG_PAPER_LITERAL 1u /* equilibrium exactly as printed (no momentum projection) */
#define LB_FLAG_STAGED 2u        /* start with LB_KERNEL_STAGED (see lb_set_step_kernel) */
/* Exact entropic equilibrium instead of the series (Eqs. (discreteentropiceq),
 * (fivelagrangemultipliersystem)): f^eq_i = w_i rho exp(-alpha - beta.c_i -
 * gamma c_i^2), the five multipliers solved per node by Newton's method (FP64
 * in LB_F64, else FP32), so mass, momentum and energy are exact collision
 * invariants for any u and theta.  The update then always runs
 * LB_KERNEL_DIRECT1; a node whose Newton residual stays above tolerance is
 * reported as LB_ERR_UNSTABLE.  Excludes LB_FLAG_PAPER_LITERAL; not for
 * lb_batch_init. */
#define LB_FLAG_ENTROPIC 4u
/* With LB_FLAG_ENTROPIC: the entropic path length (Sec. "Droplet Collision", the update with
 * alpha beta, alpha such that the dynamics obeys the H theorem).  The collision becomes
 * f' = f + alpha beta (f^eq - f), beta = 1 / (2 tau + 1), with alpha per node the nontrivial
 * root of H(f + alpha (f^eq - f)) = H(f), H(f) = sum_i f_i ln(f_i / w_i) (alpha = 2 is BGK).
 * Solved by Newton's method in the storage's compute type; alpha = 2 where f = f^eq or where no
 * root lies below the value at which a population reaches zero.  Needs LB_FLAG_ENTROPIC
 * (LB_ERR_ARG otherwise); lb_set_walls refuses it (LB_ERR_ARG); not for lb_batch_init. */
#define LB_FLAG_ENTROPIC_PATH 8u

typedef struct {
    int64_t nx, ny, nz; /* simple-cubic cells per axis, each >= 1; nodes = 2 nx ny nz */
} lb_grid;

/* Velocity set of the library, in its population order (pairs +c, -c at
 * indices 2k+1, 2k+2; index 0 is rest).  c2 receives 41*3 doubled components
 * 2 c_i (integers), w receives the 41 weights (Table I; w_0 derived).  Either
 * pointer may be NULL. */
lb_status lb_velocity_set(int *c2, double *w);

/* Reference temperature theta_0 = sum_i w_i c_ix^2 from the Table I weights. */
double lb_theta0(void);

/* Create a solver context.
 *   grid          cells per axis (each 1 .. 2^30, total nodes < 2^40)
 *   velocity_set  must be LB_RD3Q41
 *   theta0        <= 0: use the derived theta_0; otherwise it must equal the
 *                 derived value to 1e-12 relative, else LB_ERR_THETA0
 *   tau           mean free time, > 0 (beta = 1/(2 tau + 1)); +inf gives
 *                 beta = 0 (free streaming, collision is the identity)
 *   precision     lb_precision
 *   flags         LB_FLAG_* bits
 *   cuda_stream   cudaStream_t to enqueue on (NULL = legacy default stream)
 * Allocates two population buffers of 2*41*nodes/2 elements of the storage
 * type.  The populations are zero until lb_set_fields / lb_set_populations. */
lb_status lb_init(lb_ctx **out, lb_grid grid, int velocity_set, double theta0, double tau, lb_precision precision,
                  unsigned flags, void *cuda_stream);

/* Replace the stream the context enqueues on. */
lb_status lb_set_stream(lb_ctx *ctx, void *cuda_stream);

/* Set the populations to the equilibrium (Eq. feqGenU3) of the given fields:
 * rho[s][z][y][x], u[3][s][z][y][x], theta[s][z][y][x] (float64).  The stored
 * state is then the post-collision state at t = 0.  on_device = 0: host arrays.
 * Page-locked (pinned) host arrays are read by the kernel directly over the
 * host link; pageable ones are copied through a device staging buffer in
 * chunks.  Returns after the host arrays have been read. */
lb_status lb_set_fields(lb_ctx *ctx, const double *rho, const double *u, const double *theta, int on_device);

/* Advance n >= 0 time steps: each step streams (pull) and collides every node
 * in one fused kernel.  Asynchronous on the context's stream. */
lb_status lb_step(lb_ctx *ctx, int64_t n);

/* Node moments of the current state: rho, u = j/rho, theta = (<f,c^2>/rho - u^2)/3
 * (Sec. II), into caller arrays in the field layouts above.  Any output
 * pointer may be NULL.  Host outputs (on_device = 0) are complete on return;
 * page-locked ones are written by the kernel directly, pageable ones through
 * the staging buffer. */
lb_status lb_get_moments(lb_ctx *ctx, double *rho, double *u, double *theta, int on_device);

/* Global sums in FP64, deterministic order: out[0] = mass sum <f,1>,
 * out[1..3] = momentum sum <f,c>, out[4] = energy sum <f,c^2/2>.  out is host memory. */
lb_status lb_conserved(lb_ctx *ctx, double out[5]);
/* The same sums over the planes z0 <= z < z1 of both sub-lattices (a z slab's
 * interior); LB_ERR_ARG unless 0 <= z0 < z1 <= nz. */
lb_status lb_conserved_planes(lb_ctx *ctx, int64_t z0, int64_t z1, double out[5]);

/* z-slab decomposition over ranks (one process per GPU), the host side of
 * which is paper_1909_08406_gb300/decomp.py.  Rank r's context holds its slab
 * of nz_r planes plus LB_HALO planes below and above (lb_init with
 * nz = nz_r + 2 LB_HALO, nz_r >= LB_HALO), and the ordinary periodic update
 * steps it: its wrap touches only halo planes.  Before each step the halo
 * planes are refreshed from the neighbouring ranks' interiors, after which the
 * slab's interior update is identical to that of the whole grid.  An interior
 * node pulls population i from at most ceil(|c_iz|) cells away, so the halo
 * plane at distance d from the interior is read only through the populations
 * whose c_z points into the slab and for which (|2 c_z| + 1) / 2 >= d; only
 * those are sent (15 of the 82 plane-populations of each direction).
 * Messages are device buffers of lb_halo_bytes bytes, laid out
 * [entry][s][y][x] in the storage type, entries ordered by distance d = 1, 2,
 * then population index:
 *   lb_halo_pack(ctx, 1, buf)    the top interior planes, for rank + 1's lower halo
 *   lb_halo_pack(ctx, 0, buf)    the bottom interior planes, for rank - 1's upper halo
 *   lb_halo_unpack(ctx, 0, buf)  the lower halo, from rank - 1's pack of side 1
 *   lb_halo_unpack(ctx, 1, buf)  the upper halo, from rank + 1's pack of side 0
 * Both are enqueued on the context's stream (lb_set_stream) and return
 * without waiting.  LB_ERR_ARG for nz < 3 LB_HALO, a side other than 0 or 1,
 * or a buffer that is not device memory. */
#define LB_HALO 2
lb_status lb_halo_bytes(lb_ctx *ctx, int64_t *bytes);
lb_status lb_halo_pack(lb_ctx *ctx, int side, void *buf);
lb_status lb_halo_unpack(lb_ctx *ctx, int side, const void *buf);

/* The global sums of lb_conserved, for callers that cannot allocate device
 * memory (code running under a memory budget owned by another allocator, or
 * latency-critical loops that must not pay cudaMalloc's implicit device
 * synchronisation).  The paper has no counterpart; this is an interface
 * addition.  It needs no context and allocates nothing:
 *   populations  device pointer to stored populations in the raw layout of
 *                lb_get_state ([s][41][nz][ny][nx] of the storage type of
 *                `precision`, e.g. a copy made with lb_get_state on the device)
 *   grid         cells per axis; 2 * nz must not exceed 4096, else LB_ERR_ARG
 *   out          device pointer to 5 doubles (mass, momentum x/y/z, energy)
 *   cuda_stream  stream to enqueue on (NULL = legacy default stream)
 * Asynchronous: out is written by work enqueued on cuda_stream.  Its only
 * scratch is a fixed 160 KB array (4096 planes x 5 doubles) in the library's
 * device memory, which every GPU that loads the library holds until the
 * process exits.  The first call on each device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current; make that first
 * call before any stream capture.  The address is kept for the life of the
 * process; a device reset (cudaDeviceReset) or any other teardown of the
 * device's primary context invalidates it, so do not call this entry point
 * again after one.  All calls share the array: calls whose work overlaps on
 * the GPU race.  Each call writes every slot it reads, so no state carries
 * over between calls.  lb_conserved_noalloc_error returns the message of the
 * calling thread's last failed call (the message is kept per host thread). */
lb_status lb_conserved_noalloc(const void *populations, lb_grid grid, lb_precision precision, double *out,
                               void *cuda_stream);
const char *lb_conserved_noalloc_error(void);

/* Current (post-collision) populations as float64 f_i in the population
 * layout.  lb_set_populations stores them (rounded to the storage type). */
lb_status lb_get_populations(lb_ctx *ctx, double *f, int on_device);
lb_status lb_set_populations(lb_ctx *ctx, const double *f, int on_device);

/* Raw storage (checkpoint / restart): lb_state_bytes bytes, layout
 * [s][41][nz][ny][nx] of the storage type: f64 f_i; f32 h_i; f16 2^8 h_i;
 * bf16 h_i, with h_i = f_i/w_i - 1.  Restoring a saved state reproduces the
 * run bit for bit. */
int64_t lb_state_bytes(const lb_ctx *ctx);
/* The grid the context was created with (LB_ERR_ARG for a NULL argument). */
lb_status lb_get_grid(const lb_ctx *ctx, lb_grid *grid);
lb_status lb_get_state(lb_ctx *ctx, void *raw, int on_device);
lb_status lb_set_state(lb_ctx *ctx, const void *raw, int on_device);

/* Step kernels.  All compute the same update; they differ in how the 41
 * upwind values reach the registers:
 *   LB_KERNEL_DIRECT1  one node per thread, direct global loads
 *   LB_KERNEL_DIRECT2  two rows per thread, packed FP32x2 arithmetic (not FP64;
 *                      ny even, nx*ny*nz < 2^32)
 *   LB_KERNEL_DIRECT2R the same with a register budget for 4 CTAs per SM
 *   LB_KERNEL_STAGED   tiles of 128/256 x fetched by TMA bulk copies into a
 *                      shared-memory ring (not FP64; nx a multiple of 128 and
 *                      of 16 bytes)
 *   LB_KERNEL_WARPSPEC the staging done by one producer warp through a ring of
 *                      full/empty mbarriers, consumer warps updating two rows
 *                      per thread (not FP64; nx a multiple of 128, ny even)
 *   LB_KERNEL_DIRECT2X two x-adjacent nodes per thread, FP32x2 arithmetic,
 *                      32-bit paired loads and stores (FP16/BF16 storage; nx even)
 *   LB_KERNEL_DIRECT2XL the same over 2 rows per block, the next row's source
 *                      rows prefetched into L2 by bulk prefetches
 *   LB_KERNEL_AUTO     DIRECT2XL for 16-bit storage with nx even, else DIRECT2 where
 *                      it applies, else DIRECT1 (the default)
 * A request that does not apply to the grid falls back to one that does. */
#define LB_KERNEL_AUTO (-1)
#define LB_KERNEL_DIRECT1 0
#define LB_KERNEL_DIRECT2 1
#define LB_KERNEL_DIRECT2R 2
#define LB_KERNEL_STAGED 3
#define LB_KERNEL_WARPSPEC 4
#define LB_KERNEL_DIRECT2X 5
#define LB_KERNEL_DIRECT2XL 6

/* Kernel lb_step will run for this context (LB_KERNEL_DIRECT1 .. LB_KERNEL_DIRECT2XL;
 * with stochastic rounding on, the one that carries the stochastic store). */
int lb_step_variant(const lb_ctx *ctx);
/* Request a step kernel (LB_KERNEL_*). */
lb_status lb_set_step_kernel(lb_ctx *ctx, int kernel);
/* Autotuner: time every step kernel that applies to this grid for reps steps
 * (the state is not advanced), keep the fastest, report it and its ms per step. */
lb_status lb_tune(lb_ctx *ctx, int reps, int *kernel, double *ms_per_step);

/* Stochastic rounding of the BF16 store (LB_F32_S16B contexts; the rounding
 * of 16-bit storage is a choice the paper leaves open).  Round to nearest
 * rounds a slowly varying field the same way at every step, so its error adds
 * up coherently; an unbiased random rounding makes it a random walk instead.
 * With enable != 0, step t (t = 0 for the first lb_step after this call)
 * stores population i of node q (q = s nx ny nz + (z ny + y) nx + x, taken
 * mod 2^32) as the upper half of bits(h_i) + r, h_i the FP32 value and r 16
 * random bits, so the magnitude is rounded up with probability (lower half of
 * bits(h_i)) / 2^16.  r is the low (q even) or high (q odd) half of
 *   w_i = s_(i+1) ^ (s_(i+1) >> 16),  s_(i+1) = 1664525 s_i + 1013904223,
 *   s_0 = H(k_t ^ (q >> 1)),  k_t = H(H(lo32(seed) ^ H(hi32(seed))) + t),
 * all mod 2^32, i in the library's population order, H the 32-bit PCG hash
 * of Jarzynski and Olano (JCGT 9(3), 2020): with v = x * 747796405 +
 * 2891336453 and u = ((v >> ((v >> 28) + 4)) ^ v) * 277803737, H(x) = (u >> 22)
 * ^ u.  The step then always runs the x-pair kernel (nx even) or one node per
 * thread, whatever lb_set_step_kernel or lb_tune chose.  Requires BF16
 * storage and the series equilibrium with the momentum projection (no
 * LB_FLAG_PAPER_LITERAL or LB_FLAG_ENTROPIC: LB_ERR_ARG), and neither walls
 * nor the nonideal mode (LB_ERR_STATE; those refuse to start while it is on).
 * enable = 0 restores round to nearest.  A batch (lb_batch_step) refuses
 * members with it on (LB_ERR_STATE). */
lb_status lb_set_stochastic_rounding(lb_ctx *ctx, int enable, uint64_t seed);

/* Kinetic walls normal to z (Sec. "Viscous heat dissipation", which applies
 * the kinetic boundary condition of Ansumali and Karlin 2002 at the walls and
 * keeps the other two directions periodic).  With enable != 0 the grid is no
 * longer periodic in z: a bottom wall lies a quarter cell below the lowest
 * node plane (A nodes of z = 0) and a top wall a quarter cell above the
 * highest (B nodes of z = nz - 1), so the channel is nz cells high.  Each wall
 * is cut into the grid's cell columns (x, y).  Diffuse reflection, column by
 * column: every post-collision population that would stream through a wall
 * is absorbed by the column it lands in, and every population whose upwind
 * position lies beyond a wall arrives as rho_w f^eq_i(1, u_w, theta_w), the
 * model's equilibrium at the velocity and temperature of the column it comes
 * from, with rho_w the density that returns that column's absorbed mass.
 * Mass is conserved; momentum and energy are exchanged with the walls.
 *   bottom, top  {u_x, u_y, u_z, theta} of every column of each wall, host
 *                arrays read during the call; u_z must be 0, theta > 0
 * Requires nz >= 4 (LB_ERR_ARG otherwise).  enable = 0 restores the periodic
 * grid.  Each step then runs two small kernels besides the step kernel (the
 * columns' densities and the two outermost cell layers at each wall).  Walls
 * are not part of lb_get_state; a batch (lb_batch_step) refuses members with
 * walls (LB_ERR_STATE). */
lb_status lb_set_walls(lb_ctx *ctx, int enable, const double bottom[4], const double top[4]);
/* Walls as lb_set_walls, with a velocity and temperature per cell column:
 * bottom, top  host arrays [3][ny][nx]: u_x, u_y and theta of every column
 *              (finite, theta > 0), read during the call. */
lb_status lb_set_wall_columns(lb_ctx *ctx, const double *bottom, const double *top);
/* rho_w of every column of the bottom then the top wall in the last step (1 before the
 * first): host array [2][ny][nx].  LB_ERR_STATE without walls.  Synchronises the stream. */
lb_status lb_wall_density(lb_ctx *ctx, double *rho_w);

/* Equations of state of the nonideal fluid (the eos argument of lb_set_nonideal), at the
 * lattice temperature theta0, with Z(p) = (1 + p + p^2 - p^3) / (1 - p)^3, p = b rho / 4:
 *   van der Waals        p = rho theta0 / (1 - b rho) - a rho^2
 *                        (critical point: theta_c = 8a / (27b), rho_c = 1 / (3b))
 *   Peng-Robinson type   p = rho theta0 Z - a rho^2 / (1 + 2 b rho - b^2 rho^2), Eq. (cspreos)
 *                        (a = 1.851427622 theta_c / rho_c, b = 0.353748714 / rho_c)
 *   Carnahan-Starling    p = rho theta0 Z - a rho^2
 *                        (a = 1.3828652 theta_c / rho_c, b = 0.52177554 / rho_c: the roots of
 *                        dp/drho = d2p/drho2 = 0 at (rho_c, theta_c)) */
#define LB_EOS_VAN_DER_WAALS 1
#define LB_EOS_PENG_ROBINSON 2
#define LB_EOS_CARNAHAN_STARLING 3

/* The constants a, b of equation of state eos (LB_EOS_*) whose critical point is
 * (rho_c, theta_c = theta0 / theta_star), for the lattice temperature theta0 of
 * lb_theta0(): the relations listed above, the Carnahan-Starling packing
 * fraction solved by bisection to round-off.  Host only (no device, no context);
 * a and b are caller-owned outputs.  LB_ERR_ARG for an unknown eos, NULL
 * outputs, or theta_star, rho_c not positive and finite. */
lb_status lb_nonideal_constants(int eos, double theta_star, double rho_c, double *a, double *b);

/* Isothermal nonideal fluid (Sec. "Nonideal Fluids and two-phase flow"): with
 * eos != 0 (one of LB_EOS_*) each step adds the force of the paper's
 * momentum-conserving formulation, Eq. (gradientFinal), for that equation of
 * state at the lattice temperature theta0,
 *   rho g = -[rho d2 mu + mu d2 rho - eta d2 F - (1 - eta) d4 F + kappa d2_b I_ab]
 * (mu, F: the nonideal chemical potential and free energy, without the ideal
 * part theta0 rho (ln rho - 1) that the lattice carries, so that p = rho mu - F;
 * I_ab: the interfacial stress; d2, d4: the second- and fourth-order gradients
 * of the 15-velocity bcc stencil of Appendix A), and collides with the forcing
 * of Eq. (multiphaseEvolution), alpha = 2, at the equilibrium f^eq(rho, u,
 * theta0) (isothermal: the temperature moment is not kept).  u is then
 * sum f c / rho + g / 2 (lb_get_moments reports sum f c / rho).
 *   a >= 0, b > 0   the equation of state's constants (above)
 *   kappa >= 0      interfacial stiffness; eta in [0, 1]: weight of the second-order
 *                   gradient of F (the paper uses 1/2)
 * Densities must stay below the equation of state's singular density (1/b for
 * van der Waals, 4/b for Carnahan-Starling, (1 + sqrt2)/b for the Peng-Robinson
 * type).  Beyond it the van der Waals and Peng-Robinson logarithms give NaN,
 * which the step's state check reports as LB_ERR_UNSTABLE at the next
 * synchronising call; the Carnahan-Starling form is checked only for
 * rho > 0 and finite moments.  An eos outside LB_EOS_* gives LB_ERR_ARG.
 * Needs the projected series equilibrium (no LB_FLAG_PAPER_LITERAL or
 * LB_FLAG_ENTROPIC; LB_ERR_ARG), fewer than 2^31 cells (LB_ERR_ARG), and
 * neither walls nor stochastic rounding (LB_ERR_STATE).  Each step runs four kernels (density,
 * stencil fields, force, forced step); the work buffer holds 13 field values per node, 104 bytes
 * with FP64 storage and 52 otherwise.  A batch (lb_batch_step) refuses members with
 * it on (LB_ERR_STATE).  eos = 0 restores the energy-conserving update. */
lb_status lb_set_nonideal(lb_ctx *ctx, int eos, double a, double b, double kappa, double eta);

/* Number of time steps taken since the last lb_set_fields / lb_set_populations / lb_set_state. */
int64_t lb_time(const lb_ctx *ctx);

/* Wait for the context's stream; report the sticky device error word. */
lb_status lb_sync(lb_ctx *ctx);

lb_status lb_destroy(lb_ctx *ctx);

/* Message for the last failing call on ctx (or for a failing lb_init when ctx is NULL). */
const char *lb_last_error(const lb_ctx *ctx);

/* ------------------------------------------------------------------------
 * Batched sweep of independent simulations (uneven grids, per-simulation tau).
 * Not in the paper: many small simulations advanced in one launch so that
 * the GPU is filled.  Each simulation is an lb_ctx owned by the batch
 * (lb_batch_sim); use it with lb_set_fields / lb_get_moments / lb_conserved /
 * lb_get_populations, but never lb_destroy it or lb_step it alone.
 * ------------------------------------------------------------------------ */
typedef struct lb_batch lb_batch;

#define LB_BATCH_GRAPH 0      /* one batched launch per step, n steps replayed as one CUDA graph */
#define LB_BATCH_PERSISTENT 1 /* one cooperative launch for all n steps, grid barrier between steps */
#define LB_BATCH_SEQUENTIAL 2 /* each simulation stepped by its own launches (baseline) */

/* nsims simulations, grids[k] and tau[k] each; precision and flags as lb_init.  Each
 * simulation must have fewer than 2^31 nodes (LB_ERR_ARG otherwise). */
lb_status lb_batch_init(lb_batch **out, int nsims, const lb_grid *grids, const double *tau, lb_precision precision,
                        unsigned flags, void *cuda_stream);
int lb_batch_size(const lb_batch *b);
/* Context of simulation sim (0 <= sim < size), owned by the batch; NULL if out of range. */
lb_ctx *lb_batch_sim(lb_batch *b, int sim);
/* Autotuner.  For each of the two batched launch modes (LB_BATCH_GRAPH and
 * LB_BATCH_PERSISTENT, tuned separately) it times every tile shape (TX x-nodes
 * by RY rows per CTA, or RY = 0: TX consecutive entries of a simulation's
 * x-fastest node order, crossing row ends), with one and, where allowed, two
 * rows per thread, on this batch for reps steps each (the state is not
 * advanced), and keeps the fastest.  Reports the graph mode's shape and time
 * per step in ms (lb_batch_get_plan gives both modes').  Any output may be NULL. */
lb_status lb_batch_tune(lb_batch *b, int reps, int *tx, int *ry, double *ms_per_step);
/* Tile shape of the graph mode; lb_batch_set_tile sets it for both modes and accepts
 * (16,4) (16,8) (32,2) (32,4) (64,1) (64,2) (128,1) and the linear shapes (64,0) (128,0). */
lb_status lb_batch_get_tile(const lb_batch *b, int *tx, int *ry);
lb_status lb_batch_set_tile(lb_batch *b, int tx, int ry);
/* Rows updated per thread, for both modes: 1, or 2 (nodes (y, x) and (y + 1, x) with
 * packed FP32x2 arithmetic; FP32/FP16/BF16 storage with every simulation's ny even,
 * else LB_ERR_ARG).  Two is the default where allowed; lb_batch_tune may change it.
 * lb_batch_get_rows reports the graph mode's (-1 for NULL). */
lb_status lb_batch_set_rows(lb_batch *b, int rows_per_thread);
int lb_batch_get_rows(const lb_batch *b);
/* Tile shape and rows per thread of mode LB_BATCH_GRAPH or LB_BATCH_PERSISTENT (else
 * LB_ERR_ARG).  Any output may be NULL. */
lb_status lb_batch_get_plan(const lb_batch *b, int mode, int *tx, int *ry, int *rows_per_thread);
/* Advance every simulation by n steps in the given mode (LB_BATCH_*).  Asynchronous. */
lb_status lb_batch_step(lb_batch *b, int64_t n, int mode);
/* Cycle budget of each grid-barrier wait of the persistent mode (default 4e9) and, for
 * diagnostics, extra arrivals the barrier waits for (0 in normal use; > 0 makes every
 * wait run out, which must end in LB_ERR_TIMEOUT, never a hang). */
lb_status lb_batch_set_wait(lb_batch *b, long long limit_cycles, unsigned extra_arrivals);
/* Wait for the batch's work; reports LB_ERR_TIMEOUT / LB_ERR_UNSTABLE from the device error words. */
lb_status lb_batch_sync(lb_batch *b);
lb_status lb_batch_destroy(lb_batch *b);
const char *lb_batch_last_error(const lb_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* GBLB_H */
