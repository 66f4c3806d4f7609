/*
 * lbmd.h -- C ABI of the GB300 library for the fluctuating D3Q19 lattice
 * Boltzmann (LB) fluid with dissipative point-particle coupling of
 * Tretyakov & Duenweg, arXiv:1610.02733 ("An improved dissipative coupling
 * scheme for a system of Molecular Dynamics particles interacting with a
 * Lattice Boltzmann fluid"), variants A, B and C, with the Kremer-Grest
 * interactions of the paper's test system.
 *
 * The calls follow the paper's statement of the problem (Sec. 3, Fig. 2):
 * the fluid is advanced by LB steps of length tau_LB, the particles by m MD
 * steps of length dt = tau_LB / m per LB step.  A caller therefore issues
 *     m x lbmd_md_substep(), then 1 x lbmd_lb_step(), and repeats.
 *
 * Units: lattice units, lattice spacing a = 1 and tau_LB = 1.
 * Lattice: nx x ny x nz nodes at integer coordinates, periodic in every axis.
 * Node index: r = x + nx * (y + ny * z).
 * Populations in host arrays: f[i * N + r], i = 0..18 in the D3Q19 order
 *     c_0 = 0; c_1..6 = +x, -x, +y, -y, +z, -z;
 *     c_7..18 = (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1),
 *               (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1).
 *
 * Ownership: the context owns every device buffer it allocates in
 * lbmd_create; host arrays passed in are read during the call and not kept;
 * host arrays passed out are written during the call.  The "_device" calls
 * take device pointers that stay owned by the caller and are used in stream
 * order on the context's stream.
 *
 * Errors: every call returns an lbmd_status; nothing else crosses the ABI
 * (no exceptions, no exit).  A CUDA failure returns LBMD_ERR_CUDA and keeps
 * its message for lbmd_last_error().  lbmd_md_substep, lbmd_lb_step and
 * lbmd_run_cycles only enqueue work on the context's stream: they neither
 * allocate nor synchronise.  Calls documented as "synchronising" wait for the
 * stream.
 *
 * Randomness: every random number is drawn from Philox4x32-10 (Salmon et al.,
 * SC'11) keyed by params.seed: fluid noise at node r of LB step t uses the
 * counters (r, t, 0, q), q = 0, 1, two 16-bit variates per 32-bit output
 * word; the random force on particle p in MD step s uses (p, s, 1, 0), one
 * 32-bit variate per component.  Results are reproducible bit for bit.
 * The step counters are 32 bits wide in these counters: runs longer than
 * 2^32 LB steps (or MD steps) repeat their noise.
 */
#ifndef LBMD_H
#define LBMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lbmd_status {
    LBMD_OK = 0,
    LBMD_ERR_ARG = -1,       /* invalid argument or parameter */
    LBMD_ERR_CUDA = -2,      /* a CUDA call failed; see lbmd_last_error */
    LBMD_ERR_OOM = -3,       /* device or host allocation failed */
    LBMD_ERR_SEQUENCE = -4,  /* call out of the m-substeps-then-LB-step order */
    LBMD_ERR_NONFINITE = -5, /* an observable came out NaN or infinite */
    LBMD_ERR_CAPACITY = -6,  /* more particles or bonds than reserved */
    LBMD_ERR_RANGE = -7      /* node momentum left the fixed-point range */
} lbmd_status;

/* Variants of the coupling: A and B (Sec. 3); C (Sec. 4): after every MD step
 * the populations at the touched nodes take that step's momentum transfer
 * through the forcing part of the collision (local streaming velocity
 * u = (j + F/2)/rho, no relaxation, noise or streaming). */
enum { LBMD_VARIANT_A = 0, LBMD_VARIANT_B = 1, LBMD_VARIANT_C = 2 };
/* Storage and arithmetic.  FP32 / FP64: populations, node field and particles
 * in that precision.  FP16_DEV / BF16_DEV: populations stored as deviations
 * f_i - w_i rho0 in FP16 / BF16 (round to nearest), everything else as in
 * FP32, the LB arithmetic on the deviations (the mass moment is their sum);
 * the rounding of the stored deviations breaks exact mass and momentum
 * conservation at the level of their last bit (a random walk).  FP16_DEV_SR /
 * BF16_DEV_SR: the same storage, but the collision rounds each stored
 * deviation stochastically (up with probability equal to its distance from
 * the grid value below, in units of the grid step, resolved to 2^-16), with 16
 * bits of Philox4x32-10 under the context's seed: counter (node r, LB step,
 * 2, i / 8), word (i / 2) mod 4, low half for even i, for population i of the
 * post-collision state of node r.  Variants A and B only. */
enum {
    LBMD_FP32 = 0,
    LBMD_FP64 = 1,
    LBMD_FP16_DEV = 2,
    LBMD_BF16_DEV = 3,
    LBMD_FP16_DEV_SR = 4,
    LBMD_BF16_DEV_SR = 5
};
/* Where velocity Verlet evaluates the coupling force of Eq. (4).
 * START (default, the reading of Eq. (6): R, v and F_rand of the beginning of
 *   the MD step): F_c from R, v at the start of the step, used in both
 *   half-kicks; the transfer goes to the nodes around the start position.
 * HALF_STEP: after the first half-kick (with the previous step's F_c) and the
 *   drift, F_c from the half-step velocity and the node velocities at the new
 *   position, then the second half-kick; the transfer goes to the nodes around
 *   the new position.  The particle takes dt F_c in two halves (this step and
 *   the next), so fluid + particle momentum + dt/2 sum F_c is conserved.  In
 *   a bath at rest the full-step velocity then has exactly the temperature
 *   kT, where START gives kT / (1 - zeta dt / 2m). */
enum { LBMD_INTEGRATOR_START = 0, LBMD_INTEGRATOR_HALF_STEP = 1 };
/* How variant B hands each MD step's transfers to the nodes (Eqs. (7), (8)).
 * ROWS: a gather per lattice row over the particles re-ordered by row, after
 * a separate particle pass, plus atomics for the particles that left their
 * row (few atomics; pays off for many particles).  ATOMIC: every particle
 * adds its 8 corner transfers with integer atomics (one launch; pays off for
 * few particles).  TILES: the whole MD step in one pass over tiles of 4 x 4
 * lattice rows: a block stages the node records of its rows (and one more
 * row above in y and z) in shared memory, steps the particles of its rows,
 * sums their transfers to its rows in shared memory and hands those to the
 * rows above to the neighbouring tile through an edge accumulator; particles
 * that left their row go through atomics (needs the START integrator, no
 * bonds or Lennard-Jones forces, nx <= 512, ny and nz >= 6; otherwise ROWS is
 * used; measured slower than ROWS at 0.06 particles per node).  AUTO: ATOMIC
 * while there are fewer than LBMD_SPREAD_ATOMIC_PER_ROW particles per lattice
 * row (y, z) on average, ROWS above (measured crossover).  The transfers are
 * fixed-point integers, so all of them give bitwise the same results. */
enum { LBMD_SPREAD_AUTO = 0, LBMD_SPREAD_ROWS = 1, LBMD_SPREAD_ATOMIC = 2, LBMD_SPREAD_TILES = 3 };
/* Distribution of the random numbers of the thermal noise (fluid modes,
 * Sec. 2) and of the particles' random force (Eq. (4)); both have zero mean
 * and unit variance, which is all the fluctuation-dissipation balance needs.
 * UNIFORM (default): sqrt(12) (u - 1/2) from 16 (fluid) or 32 (particles)
 * bits of Philox4x32-10, no transcendental function, so any two
 * implementations agree to rounding.  GAUSS: standard normal variates by the
 * Box-Muller transform of pairs of Philox words (u = (h + 1/2) 2^-24 from the
 * top 24 bits h of a word; r = sqrt(-2 ln u1), (r cos 2 pi u2, r sin 2 pi u2)),
 * evaluated with the device's log and sincospi; the fluid takes four Philox
 * calls per node, counter (node, LB step, 0, q), q = 0..3, variates in mode
 * order k = 4..18, two per word pair; a particle takes one, (id, MD step, 1,
 * 0), words (x, y) and (z, w) for its three components.  GAUSS needs FP32 or
 * FP64 storage (LBMD_ERR_ARG otherwise). */
enum { LBMD_NOISE_UNIFORM = 0, LBMD_NOISE_GAUSS = 1 };
#define LBMD_SPREAD_ATOMIC_PER_ROW 10

typedef struct lbmd_params {
    int32_t nx, ny, nz;    /* lattice nodes per axis (periodic), each >= 2 */
    int32_t n_sub;         /* m = tau_LB / dt: MD steps per LB step, >= 1 (Sec. 3) */
    int32_t variant;       /* LBMD_VARIANT_A, _B (Sec. 3) or _C (Sec. 4) */
    int32_t precision;     /* LBMD_FP32, LBMD_FP64, LBMD_FP16_DEV, LBMD_BF16_DEV or their _SR forms */
    double rho0;           /* initial fluid density; the fluid starts at rest */
    double nu;             /* kinematic shear viscosity, > 0 */
    double nu_bulk;        /* bulk viscosity; < 0 selects relaxation factor 0 */
    double gamma_ghost;    /* relaxation factor of the 9 ghost modes, |g| < 1 */
    double kT;             /* temperature; 0 switches all noise off */
    double zeta;           /* particle friction coefficient of Eq. (4), >= 0 */
    double body_force[3];  /* uniform force density on the fluid */
    uint64_t seed;         /* Philox key */
    int64_t max_particles; /* capacity reserved at creation */
    int64_t max_bonds;     /* capacity reserved at creation */
    void *stream;          /* cudaStream_t to enqueue on (borrowed); NULL: the
                              context creates and owns a stream of its own */
    int32_t integrator;    /* LBMD_INTEGRATOR_START or LBMD_INTEGRATOR_HALF_STEP */
    int32_t spread;        /* variant B: LBMD_SPREAD_AUTO, _TILES, _ROWS or _ATOMIC */
    int32_t noise;         /* LBMD_NOISE_UNIFORM or LBMD_NOISE_GAUSS */
} lbmd_params;

typedef struct lbmd_ctx lbmd_ctx;

/* Observables, computed with FP64 reductions on the device (Sec. 3: the
 * particle temperature is the mean kinetic energy). */
typedef struct lbmd_observables_t {
    double mass;           /* sum over nodes of rho */
    double p_fluid[3];     /* fluid momentum incl. transfers not yet collided */
    double p_particles[3]; /* sum of m v */
    double kT_particles;   /* sum of m v^2 / (3 N_particles), k_B = 1 */
    double e_kin;          /* sum of m v^2 / 2 */
    int64_t lb_step;       /* LB steps done */
    int64_t md_step;       /* MD steps done */
} lbmd_observables_t;

/* Create a context: allocates populations (two buffers), the node field, the
 * momentum-transfer accumulator and particle storage on the current device,
 * and sets the fluid at rest, f_i = w_i rho0 (Sec. 2).
 * Momentum range: the node field holds the momentum density j (Eq. (2)) and
 * the particles' transfers (Eqs. (7), (8)) as integers in units of
 * 2^(e - 30) (FP32, FP16_DEV, BF16_DEV) or 2^(e - 56) (FP64) with
 * e = ceil(log2 rho0), so that transfers add up in any order to the same
 * bits.  Each component must stay below 2^(e + 1) (FP32) / 2^(e + 7) (FP64)
 * in magnitude: a node velocity of 2 / 128 lattice units at rho = rho0, far
 * beyond the lattice speed of sound (c_s^2 = 1/3) up to which an LB fluid is
 * valid at all.  A node whose momentum reaches half of that raises a sticky
 * range flag, which lbmd_observables reports as LBMD_ERR_RANGE.
 * Errors: LBMD_ERR_ARG for invalid parameters (rho0 outside [2^-60, 2^60]
 * among them), LBMD_ERR_OOM, LBMD_ERR_CUDA. */
lbmd_status lbmd_create(const lbmd_params *params, lbmd_ctx **out);

/* Free every resource of the context (synchronising).  NULL is accepted. */
lbmd_status lbmd_destroy(lbmd_ctx *ctx);

/* Append n particles (synchronising).  pos, vel: host arrays of 3n doubles
 * (x, y, z per particle; positions are wrapped into the box); mass: n doubles,
 * or NULL for mass 1.  Particle ids are assigned consecutively; the first is
 * written to *first_id_out if it is not NULL.
 * Errors: LBMD_ERR_CAPACITY beyond max_particles, LBMD_ERR_ARG for
 * non-finite input, mass <= 0, or zeta dt / mass >= 2 (where the explicit
 * friction step of a particle alone already diverges; the coupled system
 * can become unstable below that, see lbmd_observables' non-finite check). */
lbmd_status lbmd_add_particles(lbmd_ctx *ctx, int64_t n, const double *pos, const double *vel, const double *mass,
                               int64_t *first_id_out);

/* Append nb harmonic bonds U = (k/2)(|r| - r0)^2 between particle ids
 * pairs[2b], pairs[2b+1] (host array of 2 nb int64, ids must exist; each
 * particle may take part in at most 8 bonds).  Conservative force of Eq. (4),
 * synchronising.  Errors: LBMD_ERR_CAPACITY, LBMD_ERR_ARG. */
lbmd_status lbmd_add_bonds(lbmd_ctx *ctx, int64_t nb, const int64_t *pairs, double k, double r0);

/* Kinds of bonds (per bond, fixed when it is added). */
enum { LBMD_BOND_HARMONIC = 0, LBMD_BOND_FENE = 1 };

/* Append nb FENE springs U = -(k/2) R0^2 ln(1 - (r/R0)^2), the finitely
 * extensible bonds of the Kremer-Grest chains of Sec. 4 (standard model:
 * k = 30 epsilon / sigma^2, R0 = 1.5 sigma), between particle ids
 * pairs[2b], pairs[2b+1]; same storage, limits and behaviour as
 * lbmd_add_bonds (at most 8 bonds of any kind per particle, max_bonds in
 * total).  A spring stretched to r >= R0 has infinite energy: its force is
 * NaN, the particles' velocities become NaN and lbmd_observables reports
 * LBMD_ERR_NONFINITE.  Synchronising.  Errors: LBMD_ERR_ARG (ids, k < 0,
 * R0 <= 0), LBMD_ERR_CAPACITY. */
lbmd_status lbmd_add_fene_bonds(lbmd_ctx *ctx, int64_t nb, const int64_t *pairs, double k, double R0);

/* Largest max_particles with which Lennard-Jones forces can be switched on:
 * every particle interacts with every other one (all pairs, minimum image),
 * which costs O(N^2) per MD step. */
#define LBMD_MAX_LJ_PARTICLES 131072

/* Lennard-Jones forces between all particles (bonded ones included), the
 * monomer interaction of the Kremer-Grest model of Sec. 4:
 *     U(r) = 4 eps ((sigma/r)^12 - (sigma/r)^6) - U(r_cut)   for r < r_cut,
 *     0 beyond (the paper cuts at r_cut = 2^(7/6) sigma).
 * Part of the conservative force of Eq. (4), evaluated at the current
 * positions with the minimum image; velocity Verlet as for bonds.
 * r_cut = 0 switches the forces off.  Each box edge must be at least
 * 2 r_cut + 2 lattice spacings, and max_particles at most
 * LBMD_MAX_LJ_PARTICLES.  The per-particle sums run over particle ids in a
 * fixed order, so results are reproducible bit for bit.  Synchronising;
 * recomputes the conservative forces.  Errors: LBMD_ERR_ARG (eps < 0,
 * sigma <= 0, r_cut < 0, box too small), LBMD_ERR_CAPACITY. */
lbmd_status lbmd_set_lj(lbmd_ctx *ctx, double eps, double sigma, double r_cut);

/* Overwrite positions and velocities of all particles from host arrays of
 * 3 N doubles each in id order (either may be NULL to keep it).
 * Enqueues the host-to-device copies; the host arrays must stay valid until
 * the stream reaches them (pinned memory makes the copy asynchronous;
 * pageable memory makes it synchronous). */
lbmd_status lbmd_set_particles(lbmd_ctx *ctx, const double *pos, const double *vel);

/* One MD step of length dt = tau_LB / m (Sec. 3, Eqs. (4)-(8)):
 *   node velocities at the 8 corners of each particle's cell, trilinear
 *   interpolation u(R) (Eq. (5)); F = -zeta (v - u(R)) + F_rand (Eq. (4)),
 *   F_rand with variance 2 zeta kT / dt per component; Delta P = dt F with
 *   R, v, F_rand of the start of the step (Eq. (6)); velocity Verlet with
 *   that F held fixed; Delta j_k = -delta_k Delta P / a^3 to the 8 nodes
 *   (Eqs. (7), (8)).  With LBMD_INTEGRATOR_HALF_STEP, F is instead taken
 *   after the drift from the half-step velocity at the new position (see the
 *   integrator enum).  Conservative forces (bonds, Lennard-Jones) enter both
 *   half-kicks at the positions of the kick.
 * Variant A reads the node velocities of the last LB update; variant B reads
 * them updated by every earlier MD step since (Sec. 3); variant C moves each
 * MD step's transfers into the populations (Sec. 4).  All particles read
 * the nodes before any transfer of the same step is applied.
 * Enqueue only.  LBMD_ERR_SEQUENCE if m MD steps were already done since the
 * last LB step. */
lbmd_status lbmd_md_substep(lbmd_ctx *ctx);

/* One LB step (Eq. (3)): at every node the MRT collision with thermal noise
 * and the forcing term Delta'_i of the force density J_acc / tau_LB + g
 * (J_acc = the momentum the particles handed over since the last LB step),
 * then streaming; afterwards the node velocities are those of the new
 * populations.  Enqueue only.  LBMD_ERR_SEQUENCE unless exactly m MD steps
 * were done since the last LB step. */
lbmd_status lbmd_lb_step(lbmd_ctx *ctx);

/* Run n complete cycles (m MD steps + 1 LB step each) by replaying a CUDA
 * graph of one cycle, captured on first use.  Same results as the separate
 * calls.  Enqueue only (the first call also captures and instantiates the
 * graph).  LBMD_ERR_SEQUENCE unless called at a cycle boundary. */
lbmd_status lbmd_run_cycles(lbmd_ctx *ctx, int64_t n);

/* FP64 device reductions of the observables; synchronising; copies the
 * result to *out.  LBMD_ERR_NONFINITE if any of them is NaN or infinite;
 * LBMD_ERR_RANGE (out still filled) once any node's momentum density has
 * reached half the fixed-point range since creation or the last
 * lbmd_set_populations / lbmd_load_state (see lbmd_create): the state is no
 * longer valid. */
lbmd_status lbmd_observables(lbmd_ctx *ctx, lbmd_observables_t *out);

/* The post-stream moments (Eqs. (1), (2)) of a node row are computed inside
 * the LB step's collide kernel once the 27 blocks around the row have pushed
 * their populations; a block waits for them at most `polls` polls of 64 ns and
 * otherwise leaves the row to a follow-up kernel, which gives the same bits.
 * polls = -1 restores the default (2^20 polls, ~67 ms); 0 sends every row to
 * the follow-up kernel; small values make some rows time out.  Results do not
 * depend on it: it exists to exercise and measure the fallback.  Takes effect
 * from the next LB step (drops the captured cycle graphs).
 * Errors: LBMD_ERR_ARG for polls < -1. */
lbmd_status lbmd_set_moments_wait(lbmd_ctx *ctx, int32_t polls);

/* Rows (collide blocks of up to 256 nodes) whose fused moments timed out and
 * were computed by the follow-up kernel, summed over every LB step since
 * creation (synchronising). */
lbmd_status lbmd_moments_fallback_rows(lbmd_ctx *ctx, int64_t *rows);

/* Variant A (Sec. 3): where the MD steps of a cycle read the node velocities
 * frozen at the last LB step.  on = 1: a copy of the active nodes' compact
 * records, made by the post-stream moments (the transfers then go to the
 * records themselves); on = 0: the node field.  Results are the same bit for
 * bit; the default is the node field while it takes at most a quarter of the
 * device's L2 cache (its scattered reads stay on chip), the copy above.
 * Only at a cycle boundary; no effect for variants B and C.
 * Errors: LBMD_ERR_ARG (on not 0 or 1), LBMD_ERR_SEQUENCE (MD steps of the
 * cycle done), LBMD_ERR_CUDA. */
lbmd_status lbmd_set_frozen_copy(lbmd_ctx *ctx, int32_t on);

/* Synchronising accessors (host arrays, id order, FP64). */
/* populations f*_i after the last streaming step: 19 N doubles, [i][r] */
lbmd_status lbmd_get_populations(lbmd_ctx *ctx, double *out);
/* replace the populations (19 N doubles, [i][r]); recomputes the node field
 * and clears the pending transfer; only at a cycle boundary */
lbmd_status lbmd_set_populations(lbmd_ctx *ctx, const double *in);
/* node field as the particles see it: 4 N doubles (rho, j_x, j_y, j_z) per
 * node; variant A: j of the last LB update; variant B: that plus the
 * transfers since */
lbmd_status lbmd_get_node_field(lbmd_ctx *ctx, double *out);
/* momentum handed to the fluid since the last LB step: 3 N doubles */
lbmd_status lbmd_get_transfer(lbmd_ctx *ctx, double *out);
/* positions (wrapped into the box) and velocities, 3 N doubles each; either
 * may be NULL */
lbmd_status lbmd_get_particles(lbmd_ctx *ctx, double *pos, double *vel);

/* Stream-ordered device-pointer variant of lbmd_get_particles for callers
 * that keep particle data on the GPU (e.g. PyTorch tensors): pos, vel are
 * device arrays of 3 N doubles (either may be NULL).  Enqueue only. */
lbmd_status lbmd_get_particles_device(lbmd_ctx *ctx, double *pos, double *vel);

/* Asynchronous host accessors, for a caller that streams particle data in
 * and out while the cycles run (the paper has no counterpart).  Each call only
 * enqueues: the copies run on two streams of the context's own (one up, one
 * down), through two device staging buffers per direction used in turn, and
 * are ordered against the cycles on the context's stream by events, so an
 * upload overlaps the cycle before it and a download the cycle after it.
 * Results and checks equal those of the synchronising calls.
 *   lbmd_set_particles_async: as lbmd_set_particles; the host arrays are read
 *     after the call returns, so they must stay unchanged until
 *     lbmd_synchronize (or until a later synchronising call) -- pinned host
 *     memory, or the copy from pageable memory is made before returning.
 *   lbmd_get_particles_async: as lbmd_get_particles, at the point of the
 *     call in the context's stream order; pos / vel are written after the
 *     call returns and hold the values after lbmd_synchronize.
 *   lbmd_observables_async: as lbmd_observables, at the point of the call;
 *     *out is filled, and its checks (LBMD_ERR_RANGE, LBMD_ERR_NONFINITE,
 *     LBMD_ERR_CUDA for a device error) are reported, by lbmd_synchronize --
 *     or by the observables call after next, which reuses its slot and
 *     reports the checks of the one it completes; out must stay valid until
 *     then.
 *   lbmd_synchronize: waits for everything enqueued on the context's streams,
 *     completes the queued observables (oldest first) and returns the first
 *     failed check among them, else LBMD_OK.
 * The streams, events, 4 staging buffers of 6 max_particles doubles and 160 B
 * of pinned host memory are created on the first asynchronous call and freed
 * with the context.  Errors: LBMD_ERR_ARG, LBMD_ERR_CAPACITY, LBMD_ERR_OOM,
 * LBMD_ERR_CUDA. */
lbmd_status lbmd_set_particles_async(lbmd_ctx *ctx, const double *pos, const double *vel);
lbmd_status lbmd_get_particles_async(lbmd_ctx *ctx, double *pos, double *vel);
lbmd_status lbmd_observables_async(lbmd_ctx *ctx, lbmd_observables_t *out);
lbmd_status lbmd_synchronize(lbmd_ctx *ctx);

/* Counters and sizes. */
lbmd_status lbmd_get_counts(lbmd_ctx *ctx, int64_t *n_particles, int64_t *n_bonds, int64_t *lb_step,
                            int64_t *md_step, int32_t *substeps_done);

/* Saved state (checkpoint / resume; the paper has no counterpart).  At a
 * cycle boundary, the state of a context is its populations, its particles
 * (positions, velocities, the last coupling force, ids, masses), its bonds,
 * its Lennard-Jones parameters and the LB / MD step counters, which key the
 * Philox noise.  Saved in the device representation, so a context restored
 * from it continues bit for bit as the saved one would have.
 *   lbmd_state_size: bytes the state of this context takes now.
 *   lbmd_save_state: writes it to a host buffer of at least that many bytes;
 *     synchronising; LBMD_ERR_SEQUENCE unless at a cycle boundary,
 *     LBMD_ERR_CAPACITY if the buffer is too small.
 *   lbmd_load_state: restores it into a context created with the same
 *     parameters (capacities may differ) that has no particles yet;
 *     synchronising; LBMD_ERR_ARG for another context's parameters or a
 *     damaged buffer, LBMD_ERR_CAPACITY if the capacities are too small. */
lbmd_status lbmd_state_size(lbmd_ctx *ctx, int64_t *bytes);
lbmd_status lbmd_save_state(lbmd_ctx *ctx, void *buf, int64_t bytes);
lbmd_status lbmd_load_state(lbmd_ctx *ctx, const void *buf, int64_t bytes);

/* Particle momentum and kinetic energy of caller-owned device arrays, like the
 * p_particles / e_kin part of lbmd_observables, but without allocating any
 * device memory.  The paper has no counterpart: this is a service for callers
 * that cannot allocate -- code running while a framework captures the stream
 * into a CUDA graph and forbids allocation during capture, code inside a
 * framework whose caching allocator owns the device memory budget, or
 * latency-critical paths where cudaMalloc would be too slow or synchronise.
 *   vel   device, 3n doubles (v_x, v_y, v_z per particle)
 *   mass  device, n doubles, or NULL for mass 1
 *   out   device, 4 doubles: sum m v_x, sum m v_y, sum m v_z, sum m v^2
 *   stream  cudaStream_t to enqueue on (NULL: the default stream)
 * Enqueue only; the caller synchronises before reading out.  Scratch: one
 * fixed 32 KB __device__ array in the library, held by every GPU that loads
 * it until the process exits; n above 4194304 is rejected with
 * LBMD_ERR_CAPACITY.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current; make that first
 * call before any stream capture.  All calls on one device share that
 * device's array, and it keeps the last call's partial sums: calls that can
 * overlap on the GPU (e.g. issued on different streams) race, so the caller
 * must order them.  The looked-up address is kept for the life of the
 * process: after cudaDeviceReset (or any other teardown of the device's
 * primary context) the entry point must not be called on that device again.
 * Errors: LBMD_ERR_ARG,
 * LBMD_ERR_CAPACITY, LBMD_ERR_CUDA (message in lbmd_last_error(NULL)). */
lbmd_status lbmd_particle_sums_static(const double *vel, const double *mass, int64_t n, double *out, void *stream);

/* ---------------------------------------------------------------------------
 * Batched replicas.  Many independent periodic boxes advanced together: each
 * replica r is a complete problem of its own (lattice dims, particles,
 * friction zeta_r, m_r MD steps per LB step, variant, Philox key seed_r) and
 * evolves exactly as a context created by lbmd_create with those parameters
 * (shared: rho0, nu, nu_bulk, gamma_ghost, kT; no body force, no bonds).  The
 * paper's temperature experiment (Sec. 4: particle temperature against zeta,
 * m and dt in variants A and B) needs many such boxes.  Every replica makes
 * one MD step per "tick" and its LB step after every m_r-th tick; by
 * default the P = lcm(m_r) ticks of a period are captured once into a CUDA
 * graph and replayed (lbmd_batch_set_schedule selects one persistent launch
 * per call instead).  Block sizes are chosen by timing candidates on the batch
 * (lbmd_batch_tuning).  Explicit friction is unstable for zeta dt / m >~ 2:
 * a replica whose particle speed exceeds 1 (lattice units) or stops being
 * finite is flagged unstable and frozen rather than clamped
 * (lbmd_batch_unstable).
 * ------------------------------------------------------------------------- */
typedef struct lbmd_batch_params {
    int32_t n_replicas;            /* R >= 1 */
    const int32_t *dims;           /* 3R: nx, ny, nz of every replica, each in [2, 512] */
    const int32_t *n_sub;          /* R: m_r >= 1; lcm over replicas <= 256 */
    const int32_t *variant;        /* R: LBMD_VARIANT_A or LBMD_VARIANT_B */
    const double *zeta;            /* R: friction coefficient, >= 0 */
    const uint64_t *seed;          /* R: Philox key of the replica */
    const int32_t *max_particles;  /* R: particle capacity of the replica */
    int32_t precision;             /* LBMD_FP32 or LBMD_FP64 */
    double rho0, nu, nu_bulk, gamma_ghost, kT; /* as in lbmd_params, shared */
    void *stream;                  /* cudaStream_t (borrowed) or NULL: own stream */
} lbmd_batch_params;

typedef struct lbmd_batch lbmd_batch;

/* Create the batch (arrays of the params are read during the call); fluid at
 * rest in every replica; tunes the node kernels' block size (synchronising).
 * Errors: LBMD_ERR_ARG, LBMD_ERR_OOM, LBMD_ERR_CUDA. */
lbmd_status lbmd_batch_create(const lbmd_batch_params *params, lbmd_batch **out);
lbmd_status lbmd_batch_destroy(lbmd_batch *b);
/* Append n particles to replica r (ids continue from the replica's count;
 * host arrays pos, vel of 3n doubles, mass of n or NULL for 1; synchronising).
 * LBMD_ERR_CAPACITY beyond max_particles[r]. */
lbmd_status lbmd_batch_add_particles(lbmd_batch *b, int32_t replica, int64_t n, const double *pos,
                                     const double *vel, const double *mass);
/* Advance every replica by md_steps MD steps (each makes its LB step after
 * every m_r-th).  Enqueues only, except that the first call after particles
 * were added tunes the particle kernels (synchronising). */
lbmd_status lbmd_batch_run(lbmd_batch *b, int64_t md_steps);
/* Per replica, 5 doubles: sum m v^2, sum m v (x, y, z), particle count
 * (FP64 device reductions in a fixed order; synchronising). */
lbmd_status lbmd_batch_kinetic(lbmd_batch *b, double *out);
/* The same 5 R doubles written to caller-owned device memory in stream order
 * on the batch's stream (no synchronisation; for sampling during a run). */
lbmd_status lbmd_batch_kinetic_device(lbmd_batch *b, double *out);
/* Per replica: 1 if flagged unstable (frozen since), else 0 (synchronising). */
lbmd_status lbmd_batch_unstable(lbmd_batch *b, int32_t *out);
/* Replica accessors, as the single-box ones (synchronising, FP64 host arrays,
 * populations [i][r] of 19 N_r doubles, particles in id order). */
lbmd_status lbmd_batch_get_populations(lbmd_batch *b, int32_t replica, double *out);
/* only at the replica's cycle boundary (LBMD_ERR_SEQUENCE otherwise); recomputes
 * its node field and clears its pending transfers */
lbmd_status lbmd_batch_set_populations(lbmd_batch *b, int32_t replica, const double *in);
lbmd_status lbmd_batch_get_particles(lbmd_batch *b, int32_t replica, double *pos, double *vel);
lbmd_status lbmd_batch_get_counts(lbmd_batch *b, int32_t replica, int64_t *n_particles, int64_t *lb_step,
                                  int64_t *md_step);
/* The autotuner's choice and its timings of the 3 candidates (64, 128, 256):
 * nodes per work item of the LB kernels (a block has one more warp, which
 * prefetches the items), threads per block of the particle kernels; lb_ms
 * and particle_ms take 3 doubles each or NULL. */
lbmd_status lbmd_batch_tuning(lbmd_batch *b, int32_t *nodes_per_block, int32_t *particle_block, double *lb_ms,
                              double *particle_ms);
/* Cap on the number of blocks of the persistent LB kernels (each block works
 * through the work items b, b + G, b + 2G, ... of a tick, G = the grid size);
 * 0 = as many blocks as fit on the GPU at once (the default).  Results do not
 * depend on it; a small cap leaves SMs to other work on the device.
 * LBMD_ERR_ARG for a negative cap. */
lbmd_status lbmd_batch_set_lb_grid(lbmd_batch *b, int32_t max_blocks);
/* Schedule of lbmd_batch_run (Sec. 4's many-replica experiment; the paper
 * itself steps one box at a time).
 *   LBMD_BATCH_PERIOD_GRAPH (the default): per tick, one kernel per phase over
 *     every replica (particles, variant-B transfers, collide and moments of
 *     the due replicas); a period of lcm(m_r) ticks is captured in a CUDA
 *     graph and replayed.
 *   LBMD_BATCH_PERSISTENT: one launch per call, captured in a CUDA graph (one
 *     graph per distinct md_steps): a grid of thread-block clusters of
 *     cluster_blocks blocks of 256 threads, as many clusters as fit on the
 *     GPU; each cluster takes replicas one at a time, heaviest first, and
 *     runs all md_steps MD steps of the replica it holds, with cluster
 *     barriers between the phases of a tick.  No replica waits for another.
 * Both schedules run every node and particle through the same functions
 * and give the same results bit for bit, except for a replica flagged
 * unstable, whose frozen state differs (persistent: it stops at its
 * cluster's next barrier).  cluster_blocks: 0 = the autotuner's choice (timed
 * at creation over 1, 2, 4, 8 and 16 blocks on the rest state), else 1, 2, 4, 8
 * or 16 (16: a non-portable cluster size, where the device allows it).
 * Enqueued work is finished first (synchronising).  LBMD_ERR_ARG for an
 * unknown schedule or cluster size. */
#define LBMD_BATCH_PERIOD_GRAPH 0
#define LBMD_BATCH_PERSISTENT 1
lbmd_status lbmd_batch_set_schedule(lbmd_batch *b, int32_t schedule, int32_t cluster_blocks);
/* The persistent schedule's tuned cluster size and its timings (ms of one
 * period on the rest state) for 1, 2, 4, 8 and 16 blocks per cluster (ms: 5
 * doubles or NULL; 0 for a size that does not fit on the device). */
lbmd_status lbmd_batch_persistent_tuning(lbmd_batch *b, int32_t *cluster_blocks, double *ms);
void *lbmd_batch_stream(lbmd_batch *b);
const char *lbmd_batch_last_error(lbmd_batch *b);

/* ---------------------------------------------------------------------------
 * Adjoint (reverse-mode derivative) of the coupled step, variant B, for the
 * mean particle drag along x:
 *     L = (1 / (K m N_p)) sum over K cycles of m MD steps and N_p particles of
 *         the coupling force F_x of Eq. (4),
 * with respect to zeta and the initial particle positions.  The random
 * numbers are fixed by their Philox counters (kT = 0 or kT > 0), so the map
 * is deterministic; it is piecewise smooth (kinks where a particle crosses a
 * cell face).  The forward pass starts from the fluid at rest (f_i = w_i rho0)
 * and keeps the populations and particles of every LB step; the backward pass
 * recomputes each cycle's m MD steps from its checkpoint and runs the
 * hand-written adjoint kernels (transposed collision and streaming, moments,
 * interpolation, friction, velocity Verlet and transfers).  Ideal particles
 * of mass 1.
 * ------------------------------------------------------------------------- */
typedef struct lbmd_adjoint_params {
    int32_t nx, ny, nz;     /* periodic lattice, each >= 2 */
    int32_t n_sub;          /* m MD steps per LB step, >= 1 */
    int32_t n_particles;    /* N_p */
    int32_t n_cycles;       /* K LB steps of the forward pass */
    int32_t precision;      /* LBMD_FP32 or LBMD_FP64 */
    int32_t pad_;
    double rho0, nu, nu_bulk, gamma_ghost, kT; /* as in lbmd_params */
    double body_force[3];   /* uniform force density on the fluid */
    uint64_t seed;          /* Philox key */
    void *stream;           /* cudaStream_t (borrowed) or NULL: own stream */
} lbmd_adjoint_params;

typedef struct lbmd_adjoint lbmd_adjoint;

lbmd_status lbmd_adjoint_create(const lbmd_adjoint_params *params, lbmd_adjoint **out);
lbmd_status lbmd_adjoint_destroy(lbmd_adjoint *a);
/* Forward pass with friction zeta from N_p initial positions and velocities
 * (host arrays of 3 N_p doubles); writes L.  Synchronising. */
lbmd_status lbmd_adjoint_forward(lbmd_adjoint *a, double zeta, const double *pos0, const double *vel0, double *loss);
/* dL/dzeta and dL/dR0 (host array of 3 N_p doubles) of the last forward pass;
 * LBMD_ERR_SEQUENCE before any forward pass.  Synchronising. */
lbmd_status lbmd_adjoint_backward(lbmd_adjoint *a, double *dloss_dzeta, double *dloss_dpos0);
const char *lbmd_adjoint_last_error(lbmd_adjoint *a);

/* The cudaStream_t the context enqueues on. */
void *lbmd_stream(lbmd_ctx *ctx);

/* Message of the last error of this context (or of lbmd_create when ctx is
 * NULL); never NULL. */
const char *lbmd_last_error(lbmd_ctx *ctx);
const char *lbmd_status_string(lbmd_status s);

#ifdef __cplusplus
}
#endif
#endif /* LBMD_H */
