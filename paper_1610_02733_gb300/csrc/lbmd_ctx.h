// lbmd_ctx.h -- host-side context of the LB/MD library and the launchers the
// C-ABI layer calls.  Device memory layout (all on one GPU):
//
//   f[2]        populations, structure of arrays f[i * N + r], ping-pong:
//               f[cur] holds the post-stream populations f*.
//   node        node field, one 16-byte (FP32) / 32-byte (FP64) record per
//               node: rho* as bits and the momentum density j in fixed point.
//               Variant A: j* of the last LB update (frozen during the MD
//               steps).  Variant B: j* plus every transfer since.
//   jacc        variants A and C: the transfers since the last LB step (C:
//               since the last MD step), fixed point, 4 words per node.
//   Particles live in "slots".  Once per LB step they are re-ordered by
//   lattice row (y, z) of their cell, so that the particles a warp handles
//   touch neighbouring nodes (cache locality of the corner reads and
//   transfers).  Results do not depend on the order: every per-particle
//   quantity is keyed by the particle id, and transfers are integer sums.
//   pos4[2]     per slot: fractional position in its cell (x, y, z) and the
//               linear cell index (two buffers, current one pv: the
//               re-ordering and the tiled variant-B MD step write the other).
//   vel4[2]     per slot: velocity (x, y, z) and 1 / mass (same buffers).
//   fcons4[2]   per slot: bond force at the current positions.
//   pid[2]      per slot: particle id.   slot_of: per id, its slot.
//   fc4         per slot: coupling force F of the current MD step.
//   old4        variant B only: pos4 at the start of the current MD step.
//   bond_*      per particle id: up to LBMD_MAX_BONDS_PER_PARTICLE partner ids.
//   row_count   per lattice row: particle counts / offsets of the re-ordering.
//   row_start   first slot of every cell row after the re-ordering; slot_row
//               the row bucket of every slot (-1 for particles added since).
//   occw        variant B: the active nodes (corners of the particles' cells
//               at the last re-ordering), per row and 32-node word the bits
//               and the compact slot of the word's first active node.
//   cact        variant B: compact node records of the active nodes, two
//               buffers per active set (the current one `rec`; the tiled MD
//               step reads one and writes the other).  For an active node
//               the compact record, not `node`, is current between LB
//               updates; `node` is brought up to date from it only for the
//               observables and the host accessors.
//   arow        variant B, per active set: compact slot of every row's first
//               record (rows + 1 entries, the last the total).
//   ccw         per cell row and 32-cell word, the cells that hold a particle
//               at the last re-ordering (marked while counting the rows; the
//               active words are built from them).
#pragma once

#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>
#include <string>

#include "../../include/lbmd.h"
#include "lbmd_device.cuh"

#include <nvtx3/nvToolsExt.h>

// A named NVTX range around a C-ABI call (visible in Nsight tools, free
// otherwise): LBMD_TRACE("lbmd_md_substep");
struct LbmdTraceRange {
    explicit LbmdTraceRange(const char *name) { nvtxRangePushA(name); }
    ~LbmdTraceRange() { nvtxRangePop(); }
    LbmdTraceRange(const LbmdTraceRange &) = delete;
    LbmdTraceRange &operator=(const LbmdTraceRange &) = delete;
};
#define LBMD_TRACE(name) LbmdTraceRange lbmd_trace_range_(name)

#define LBMD_MAX_BONDS_PER_PARTICLE 8

struct LbCoeffs {
    double gamma_bulk, gamma_shear, gamma_ghost;
    double noise_amp[19];  // sqrt(mu b_k (1 - gamma_k^2)), multiplied by sqrt(rho) per node
    double body_force[3];
    int noisy;
};

// Relaxation factors and noise amplitudes of the collision operator (Sec. 2),
// one definition for the single box, the batched replicas and the adjoint:
// nu = (1 + g_s) / (6 (1 - g_s)), nu_b = (1 + g_b) / (9 (1 - g_b)) (g_b = 0
// for nu_b < 0), ghost factor as given; mode k >= 4 gets the amplitude
// sqrt(mu b_k (1 - g_k^2)) with mu = kT / (a^3 c_s^2) = 3 kT, the conserved
// modes 0-3 none.  The body force is left to the caller.
inline void lb_coefficients(double nu, double nu_bulk, double gamma_ghost, double kT, LbCoeffs &co) {
    co.gamma_shear = (6.0 * nu - 1.0) / (6.0 * nu + 1.0);
    co.gamma_bulk = nu_bulk < 0 ? 0.0 : (9.0 * nu_bulk - 1.0) / (9.0 * nu_bulk + 1.0);
    co.gamma_ghost = gamma_ghost;
    const double mu = 3.0 * kT;
    for (int k = 0; k < lbmd::Q; ++k) {
        const double g = k < 4 ? 1.0 : (k == 4 ? co.gamma_bulk : (k <= 9 ? co.gamma_shear : co.gamma_ghost));
        co.noise_amp[k] = k < 4 ? 0.0 : std::sqrt(mu * lbmd::BNORM(k) * (1.0 - g * g));
    }
    for (int d = 0; d < 3; ++d) co.body_force[d] = 0.0;
    co.noisy = kT > 0 ? 1 : 0;
}

// Unit of the fixed-point momentum density, 2^(e - scale_log2) with
// e = ceil(log2 rho0): |j| then stays representable up to a node velocity of
// 2 (FP32) / 128 (FP64) at rho = rho0 whatever rho0 is.  At rho0 = 1, e = 0
// (units 2^-30 / 2^-56).  False for rho0 outside [2^-60, 2^60].
struct FixUnit {
    int e;
    double scale, inv_scale;  // 2^(scale_log2 - e) and its inverse
};
inline bool fix_unit(double rho0, int scale_log2, FixUnit &u) {
    if (!(rho0 >= std::ldexp(1.0, -60) && rho0 <= std::ldexp(1.0, 60))) return false;
    int E = 0;
    const double m = std::frexp(rho0, &E);  // rho0 = m 2^E, m in [0.5, 1)
    u.e = m == 0.5 ? E - 1 : E;
    u.scale = std::ldexp(1.0, scale_log2 - u.e);
    u.inv_scale = std::ldexp(1.0, u.e - scale_log2);
    return true;
}

struct lbmd_ctx {
    lbmd_params p;
    int64_t N;
    cudaStream_t stream;
    bool own_stream;
    int cur;  // index of the population buffer that holds f*
    void *f[2];
    void *node;
    void *jacc;
    int pcur;  // index of the particle buffers in use (ids, forces)
    int pv;    // index of the position / velocity buffers in use
    void *pos4[2], *vel4[2], *fcons4[2];
    int32_t *pid[2];
    int32_t *slot_of;
    void *fc4[2], *old4;  // fc4 indexed by pcur: it carries the last F_c over steps (HALF_STEP)
    int32_t *row_count, *sort_rank, *chunk_total;
    int32_t *row_start;     // first slot of every cell row (ny*nz + 1 entries)
    int32_t *slot_row;      // per slot: the row bucket it belongs to, -1 if none
    int32_t *migrant_slot;  // variant B: slots that left their row bucket
    int32_t *migrant_count;
    // variant B, two sets by LB-step parity: the MD steps of LB cycle s use set
    // s & 1 (built at the end of cycle s - 1); the LB step of cycle s reads
    // set s & 1 and writes the new moments into set (s + 1) & 1
    uint2 *occw[2];      // (ny * nz) x active_words(nx) words
    uint32_t *ccw;       // (ny * nz) x active_words(nx): cells holding a particle, per cell row (re-ordering)
    void *cact[2];       // compact node records: two buffers of cact_cap each
    int32_t *arow[2];    // first compact slot of every row, ny * nz + 1 entries
    void *tile_table[2]; // per active set: the tiled MD step's table of every tile (md_tile.cu)
    void *edge_acc;      // tiled MD step: transfers into the rows above each tile, per compact slot (zero
                         // between MD steps)
    uint32_t *tile_flag; // tiled MD step: per tile, the MD step (+ 1) whose particles are done
    int32_t *late_rows;  // tiled MD step: rows left to the follow-up, two lists by MD-step parity
    int32_t *late_count;
    int64_t cact_cap;
    size_t node_bytes;   // bytes of one node record
    int rec;             // record buffer of the current set in use (0 after every LB step)
    // LB collide with fused post-stream moments: per collide block the LB step
    // (+1) it last pushed, and the rows whose moments the fallback computes
    uint32_t *blk_done;
    int32_t *lb_missed;    // count
    int32_t *missed_list;  // collide-block ids
    unsigned long long *missed_total;  // rows left to the fallback since creation
    int fuse_spin;         // polls of a collide block's wait (0: no fused moments)
    int sm_count;
    int gather_warps;  // warps per block of the variant B row gather
    bool a_frozen_copy;  // variant A: interpolate from a frozen copy of the compact records (else the node field)
    int32_t *bond_count, *bond_partner;
    double *bond_k, *bond_r0;
    uint8_t *bond_kind;  // LBMD_BOND_HARMONIC or LBMD_BOND_FENE per (id, bond)
    // Lennard-Jones between all particles (Kremer-Grest monomers); off while
    // lj_rc == 0
    double lj_eps, lj_sigma, lj_rc;
    // Verlet lists of the LJ forces: per id the ids within lj_rc +
    // LBMD_NB_SKIN, ascending, and the position at the build; a flag set once
    // any particle moved more than half the skin since (the lists are then not
    // used until the next re-ordering rebuilds them)
    int32_t *nb_list, *nb_count, *nb_invalid;
    void *nb_ref4;
    double *staging;   // device staging buffer for host <-> device conversions
    int64_t staging_len;
    double *red_partial;  // per-block partial sums of the observables, then an arrival counter
    double *red_out;      // final sums (8), then the range and device error flags
    // range guard of the fixed-point momentum: set (sticky) by the kernels
    // that write a node record whose momentum reaches half the range
    int32_t *range_flag;
    int32_t *dev_error;  // set by a kernel whose bounded wait gave up
    FixUnit fix;
    int red_blocks;
    unsigned long long *d_lb_step;  // LB step counter read by the kernels
    int64_t np, nb;
    int64_t lb_step, md_step;
    int sub_done;
    LbCoeffs co;
    double dt;
    // the asynchronous accessors (created on first use): uploads and
    // downloads on streams of their own through two device staging buffers
    // each, ordered against the context's stream by events
    bool async_ready;
    cudaStream_t up_stream, down_stream;
    cudaEvent_t in_ready[2], in_done[2], out_ready[2], out_done[2], obs_ready, obs_done[2];
    double *stage_in[2], *stage_out[2];
    int in_idx, out_idx;
    // queued observables: raw sums and flags in pinned host memory, and the
    // caller's structure they are finalised into (two slots, used in turn)
    double *obs_host;  // per slot: 8 sums, then the range flag and the device error flag
    lbmd_observables_t *obs_out[2];
    int64_t obs_np[2], obs_lb[2], obs_md[2];
    int obs_next;
    // captured cycles, keyed by the buffer state at the start of the cycle
    // (population buffer, LB step parity, particle buffers, position buffer),
    // each with the buffer state it leaves
    cudaGraphExec_t cycle_graph[16];
    int cycle_post[16][3];  // cur, pcur, pv after the cycle
    std::string err;
};

// The active-node set the MD steps of the current LB cycle use, and the one
// the coming LB step fills.
inline uint2 *active_words_now(const lbmd_ctx *c) { return c->occw[c->lb_step & 1]; }
inline void *active_records_now(const lbmd_ctx *c) {
    return static_cast<char *>(c->cact[c->lb_step & 1]) + (size_t)c->rec * c->cact_cap * c->node_bytes;
}
// the other record buffer of the current set (written by the tiled MD step)
inline void *active_records_other(const lbmd_ctx *c) {
    return static_cast<char *>(c->cact[c->lb_step & 1]) + (size_t)(c->rec ^ 1) * c->cact_cap * c->node_bytes;
}
inline uint2 *active_words_next(const lbmd_ctx *c) { return c->occw[(c->lb_step + 1) & 1]; }
inline void *active_records_next(const lbmd_ctx *c) { return c->cact[(c->lb_step + 1) & 1]; }
// Variants A and B keep the node records of the active nodes in compact
// arrays, which the MD steps add their transfers to (variant C updates the
// populations every MD step instead).  Variant B's MD steps also read them.
// Variant A's read the node velocities as the LB step left them: from the
// node field, which nobody writes between LB steps in A (transfers to
// inactive nodes go to J_acc), or -- when the node field is too large for the
// L2 cache, where its scattered reads cost more than a copy -- from the first
// buffer of the set, the transfers then going to the second buffer, which the
// moments fill with the same records.
inline bool compact_nodes(const lbmd_ctx *c) { return c->p.variant != LBMD_VARIANT_C; }
inline bool a_copy(const lbmd_ctx *c) { return c->p.variant == LBMD_VARIANT_A && c->a_frozen_copy; }
// the records the MD steps add transfers to (and the LB step reads)
inline void *active_records_acc(const lbmd_ctx *c) {
    return a_copy(c) ? static_cast<char *>(c->cact[c->lb_step & 1]) + (size_t)c->cact_cap * c->node_bytes
                     : active_records_now(c);
}
// the second buffer of set `set`, which the moments fill with the same records
// as the first (null unless variant A keeps a frozen copy)
inline void *active_records_copy(const lbmd_ctx *c, int set) {
    return a_copy(c) ? static_cast<char *>(c->cact[set]) + (size_t)c->cact_cap * c->node_bytes : nullptr;
}
inline void *pos_now(const lbmd_ctx *c) { return c->pos4[c->pv]; }
inline void *vel_now(const lbmd_ctx *c) { return c->vel4[c->pv]; }

// Default poll limit of a collide block's wait for its neighbour blocks
// before it leaves its row's fused moments to the follow-up kernel (64 ns per
// poll: about 67 ms, far above the few microseconds the lag needs).
constexpr int LBMD_DEFAULT_FUSE_SPIN = 1 << 20;

// Launchers, one per kernel family; each enqueues on ctx->stream and returns
// the launch status.
cudaError_t launch_lb_step(lbmd_ctx *ctx);
cudaError_t launch_node_moments(lbmd_ctx *ctx, bool count_step);
cudaError_t launch_forcing_update(lbmd_ctx *ctx);
cudaError_t launch_init_equilibrium(lbmd_ctx *ctx);
cudaError_t launch_md_substep(lbmd_ctx *ctx, int substep);
cudaError_t launch_bond_forces_only(lbmd_ctx *ctx);
// conservative forces present (bonds or Lennard-Jones)
inline bool has_cons(const lbmd_ctx *ctx) { return ctx->nb > 0 || ctx->lj_rc > 0.0; }
constexpr int LBMD_NB_MAX = 128;      // list entries per particle (more: that particle's block uses all pairs)
constexpr double LBMD_NB_SKIN = 0.5;  // lattice spacings beyond the cut-off
cudaError_t launch_nb_build(lbmd_ctx *ctx);
cudaError_t launch_observables(lbmd_ctx *ctx);
cudaError_t launch_populations_to_double(lbmd_ctx *ctx, int64_t first, int64_t count, double *dst);
cudaError_t launch_populations_from_double(lbmd_ctx *ctx, int64_t first, int64_t count, const double *src);
cudaError_t launch_node_field_to_double(lbmd_ctx *ctx, int64_t first, int64_t count, double *dst, bool transfer_only);
cudaError_t launch_particles_from_double(lbmd_ctx *ctx, int64_t first, int64_t count, const double *pos,
                                         const double *vel, const double *mass, bool set_pos, bool set_vel,
                                         bool set_mass);
cudaError_t launch_particles_to_double(lbmd_ctx *ctx, double *pos, double *vel);
cudaError_t launch_clear_transfer(lbmd_ctx *ctx);
cudaError_t launch_sort_particles(lbmd_ctx *ctx);
cudaError_t launch_active_set(lbmd_ctx *ctx);
cudaError_t launch_active_sync(lbmd_ctx *ctx);
cudaError_t setup_particle_kernels(lbmd_ctx *ctx);
// the tiled variant-B MD step (md_tile.cu)
bool md_tile_geometry(const lbmd_ctx *ctx);
int md_tile_count(const lbmd_ctx *ctx);
size_t md_tile_table_bytes(const lbmd_ctx *ctx);
size_t md_tile_edge_bytes(const lbmd_ctx *ctx);
int md_tile_late_cap(const lbmd_ctx *ctx);
cudaError_t md_tile_build_table(lbmd_ctx *ctx, int set);
bool md_tile_supported(const lbmd_ctx *ctx);
bool md_tile_expected_to_fit(const lbmd_ctx *ctx);
cudaError_t md_tile_setup_kernels(lbmd_ctx *ctx);

// message returned by lbmd_last_error(NULL) (calls without a context)
void lbmd_set_global_error(const std::string &msg);
