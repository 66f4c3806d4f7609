// lbmd_api.cu -- the C ABI declared in include/lbmd.h: context life cycle,
// the m-MD-steps-then-one-LB-step sequence of Sec. 3, CUDA-graph replay of
// whole cycles, observables and host accessors.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lbmd_ctx.h"

namespace {

thread_local std::string g_create_error;

lbmd_status fail(lbmd_ctx *ctx, lbmd_status s, const std::string &msg) {
    if (ctx)
        ctx->err = msg;
    else
        g_create_error = msg;
    return s;
}

lbmd_status cuda_fail(lbmd_ctx *ctx, cudaError_t e, const char *where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? LBMD_ERR_OOM : LBMD_ERR_CUDA, msg);
}

#define CK(ctx, call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

// bytes of one real of the node field and particle records (FP32 for the
// reduced-precision population forms)
size_t real_size(const lbmd_ctx *ctx) { return ctx->p.precision == LBMD_FP64 ? 8 : 4; }

// bytes of one stored population
size_t pop_size(const lbmd_ctx *ctx) {
    return ctx->p.precision == LBMD_FP64 ? 8 : (ctx->p.precision == LBMD_FP32 ? 4 : 2);
}

void free_all(lbmd_ctx *ctx) {
    void *bufs[] = {ctx->f[0],         ctx->f[1],          ctx->node,          ctx->jacc,
                    ctx->pos4[0],      ctx->pos4[1],       ctx->vel4[0],       ctx->vel4[1],
                    ctx->fcons4[0],    ctx->fcons4[1],     ctx->pid[0],        ctx->pid[1],
                    ctx->slot_of,      ctx->row_count,     ctx->sort_rank,     ctx->chunk_total,
                    ctx->row_start,    ctx->slot_row,      ctx->migrant_slot,  ctx->migrant_count,
                    ctx->fc4[0],       ctx->fc4[1],        ctx->old4,          ctx->bond_count,
                    ctx->bond_partner, ctx->bond_k,        ctx->bond_r0,       ctx->bond_kind,
                    ctx->staging,      ctx->red_partial,   ctx->red_out,       ctx->d_lb_step,
                    ctx->occw[0],      ctx->occw[1],       ctx->cact[0],       ctx->cact[1],
                    ctx->blk_done,     ctx->lb_missed,     ctx->missed_list,   ctx->nb_list,
                    ctx->nb_count,     ctx->nb_invalid,    ctx->nb_ref4,       ctx->range_flag,
                    ctx->missed_total, ctx->dev_error,     ctx->arow[0],       ctx->arow[1],
                    ctx->tile_table[0], ctx->tile_table[1], ctx->edge_acc,  ctx->tile_flag,
                    ctx->late_rows,    ctx->late_count, ctx->ccw};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (int b = 0; b < 2; ++b) {
        if (ctx->stage_in[b]) cudaFree(ctx->stage_in[b]);
        if (ctx->stage_out[b]) cudaFree(ctx->stage_out[b]);
        for (cudaEvent_t ev : {ctx->in_ready[b], ctx->in_done[b], ctx->out_ready[b], ctx->out_done[b], ctx->obs_done[b]})
            if (ev) cudaEventDestroy(ev);
    }
    if (ctx->obs_ready) cudaEventDestroy(ctx->obs_ready);
    if (ctx->obs_host) cudaFreeHost(ctx->obs_host);
    if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
    if (ctx->down_stream) cudaStreamDestroy(ctx->down_stream);
    for (int i = 0; i < 16; ++i)
        if (ctx->cycle_graph[i]) cudaGraphExecDestroy(ctx->cycle_graph[i]);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
}

bool is_finite_d(double x) { return std::isfinite(x); }

}  // namespace

void lbmd_set_global_error(const std::string &msg) { g_create_error = msg; }

extern "C" {

const char *lbmd_status_string(lbmd_status s) {
    switch (s) {
    case LBMD_OK: return "ok";
    case LBMD_ERR_ARG: return "invalid argument";
    case LBMD_ERR_CUDA: return "CUDA error";
    case LBMD_ERR_OOM: return "out of memory";
    case LBMD_ERR_SEQUENCE: return "call out of the MD/LB step sequence";
    case LBMD_ERR_NONFINITE: return "non-finite observable";
    case LBMD_ERR_CAPACITY: return "capacity exceeded";
    case LBMD_ERR_RANGE: return "node momentum beyond the fixed-point range";
    }
    return "unknown status";
}

const char *lbmd_last_error(lbmd_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void *lbmd_stream(lbmd_ctx *ctx) { return ctx ? (void *)ctx->stream : nullptr; }

lbmd_status lbmd_create(const lbmd_params *p, lbmd_ctx **out) {
    LBMD_TRACE("lbmd_create");
    if (!p || !out) return fail(nullptr, LBMD_ERR_ARG, "null argument");
    *out = nullptr;
    if (p->nx < 2 || p->ny < 2 || p->nz < 2) return fail(nullptr, LBMD_ERR_ARG, "lattice sides must be >= 2");
    if ((int64_t)p->nx * p->ny * p->nz > (int64_t)0x7fffffff)
        return fail(nullptr, LBMD_ERR_ARG, "more than 2^31-1 nodes");
    if (p->n_sub < 1) return fail(nullptr, LBMD_ERR_ARG, "n_sub must be >= 1");
    if (p->variant != LBMD_VARIANT_A && p->variant != LBMD_VARIANT_B && p->variant != LBMD_VARIANT_C)
        return fail(nullptr, LBMD_ERR_ARG, "variant must be A (0), B (1) or C (2)");
    if (p->precision < LBMD_FP32 || p->precision > LBMD_BF16_DEV_SR)
        return fail(nullptr, LBMD_ERR_ARG, "precision must be FP32, FP64, FP16_DEV, BF16_DEV or an _SR form");
    if ((p->precision == LBMD_FP16_DEV_SR || p->precision == LBMD_BF16_DEV_SR) && p->variant == LBMD_VARIANT_C)
        return fail(nullptr, LBMD_ERR_ARG, "stochastic rounding of the stored populations needs variant A or B");
    if (!(p->rho0 > 0) || !(p->nu > 0) || !is_finite_d(p->rho0) || !is_finite_d(p->nu))
        return fail(nullptr, LBMD_ERR_ARG, "rho0 and nu must be positive");
    FixUnit fix;
    if (!fix_unit(p->rho0, p->precision == LBMD_FP64 ? lbmd::Prec<double>::SCALE_LOG2 : lbmd::Prec<float>::SCALE_LOG2,
                  fix))
        return fail(nullptr, LBMD_ERR_ARG, "rho0 must lie in [2^-60, 2^60]");
    if (!(p->kT >= 0) || !is_finite_d(p->kT)) return fail(nullptr, LBMD_ERR_ARG, "kT must be >= 0");
    if (!(p->zeta >= 0) || !is_finite_d(p->zeta)) return fail(nullptr, LBMD_ERR_ARG, "zeta must be >= 0");
    if (!(std::fabs(p->gamma_ghost) < 1.0)) return fail(nullptr, LBMD_ERR_ARG, "|gamma_ghost| must be < 1");
    if (p->max_particles < 0 || p->max_bonds < 0 || p->max_particles > 0x7fffffffLL)
        return fail(nullptr, LBMD_ERR_ARG, "bad capacities");
    if ((int64_t)p->ny * p->nz > (int64_t)1024 * 1024)
        return fail(nullptr, LBMD_ERR_ARG, "ny * nz must not exceed 2^20 (particle re-ordering by row)");
    if (p->ny > 65535 || p->nz > 65535)
        return fail(nullptr, LBMD_ERR_ARG, "ny and nz must not exceed 65535 (one collide block row per (y, z))");
    if (p->nx > (p->precision == LBMD_FP64 ? 2048 : 4096))
        return fail(nullptr, LBMD_ERR_ARG, "nx must not exceed 4096 (FP32) / 2048 (FP64): row gather shared memory");
    for (int d = 0; d < 3; ++d)
        if (!is_finite_d(p->body_force[d])) return fail(nullptr, LBMD_ERR_ARG, "non-finite body force");
    if (p->integrator != LBMD_INTEGRATOR_START && p->integrator != LBMD_INTEGRATOR_HALF_STEP)
        return fail(nullptr, LBMD_ERR_ARG, "integrator must be START or HALF_STEP");
    if (p->noise != LBMD_NOISE_UNIFORM && p->noise != LBMD_NOISE_GAUSS)
        return fail(nullptr, LBMD_ERR_ARG, "noise must be LBMD_NOISE_UNIFORM or LBMD_NOISE_GAUSS");
    if (p->noise == LBMD_NOISE_GAUSS && p->precision != LBMD_FP32 && p->precision != LBMD_FP64)
        return fail(nullptr, LBMD_ERR_ARG, "normal variates need FP32 or FP64 storage");
    if (p->spread < LBMD_SPREAD_AUTO || p->spread > LBMD_SPREAD_TILES)
        return fail(nullptr, LBMD_ERR_ARG, "spread must be AUTO, ROWS, ATOMIC or TILES");

    lbmd_ctx *ctx = new (std::nothrow) lbmd_ctx();
    if (!ctx) return fail(nullptr, LBMD_ERR_OOM, "host allocation");
    ctx->p = *p;
    ctx->N = (int64_t)p->nx * p->ny * p->nz;
    ctx->dt = 1.0 / (double)p->n_sub;
    ctx->fix = fix;
    ctx->fuse_spin = LBMD_DEFAULT_FUSE_SPIN;
    lb_coefficients(p->nu, p->nu_bulk, p->gamma_ghost, p->kT, ctx->co);
    for (int d = 0; d < 3; ++d) ctx->co.body_force[d] = p->body_force[d];

    if (p->stream) {
        ctx->stream = (cudaStream_t)p->stream;
        ctx->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            lbmd_status s = cuda_fail(nullptr, e, "cudaStreamCreate");
            delete ctx;
            return s;
        }
        ctx->own_stream = true;
    }

    const int64_t N = ctx->N;
    const size_t rs = real_size(ctx);
    const size_t node_bytes = 4 * rs;  // int4 / longlong4 records
    const int64_t maxp = p->max_particles > 0 ? p->max_particles : 1;
    const int64_t chunk = (int64_t)1 << 22;
    ctx->staging_len = std::max<int64_t>(chunk, 9 * maxp);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    ctx->red_blocks = 4 * sms;
    ctx->sm_count = sms;
    // variant A's frozen node velocities: the node field while it takes at
    // most a quarter of the L2 cache (measured: at 64^3 A then runs 1.5 %
    // faster than B, at 256^3 11 % slower), else a copy of the compact records
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    ctx->a_frozen_copy = (double)N * (double)(4 * rs) > 0.25 * (double)l2;
    // active nodes: every particle makes at most the 8 corners of its cell
    // active
    ctx->cact_cap = std::min<int64_t>(N, 8 * maxp);
    const size_t occ_bytes = (size_t)p->ny * p->nz * (size_t)((p->nx + 31) / 32) * sizeof(uint2);
    const size_t arow_bytes = ((size_t)p->ny * p->nz + 1) * sizeof(int32_t);
    const bool compact = compact_nodes(ctx);  // variants A and B: compact records of the active nodes
    ctx->node_bytes = node_bytes;
    // the tiled MD step's tables and buffers, where the lattice suits it and
    // the spread mode asks for it
    const size_t table_bytes = md_tile_geometry(ctx) && p->spread == LBMD_SPREAD_TILES ? md_tile_table_bytes(ctx) : 0;
    // blocks of the LB collide (node kernels: rows of up to 256 nodes)
    const int bx = p->nx >= 256 ? 256 : (p->nx >= 128 ? 128 : (p->nx >= 64 ? 64 : 32));
    const int64_t n_lb_blocks = (int64_t)((p->nx + bx - 1) / bx) * p->ny * p->nz;

    struct Alloc {
        void **ptr;
        size_t bytes;
    } allocs[] = {
        {&ctx->f[0], (size_t)19 * N * pop_size(ctx)},
        {&ctx->f[1], (size_t)19 * N * pop_size(ctx)},
        {&ctx->node, (size_t)N * node_bytes},
        {&ctx->jacc, p->variant != LBMD_VARIANT_B ? (size_t)N * node_bytes : 0},
        {&ctx->pos4[0], (size_t)maxp * 4 * rs},
        {&ctx->pos4[1], (size_t)maxp * 4 * rs},
        {&ctx->vel4[0], (size_t)maxp * 4 * rs},
        {&ctx->vel4[1], (size_t)maxp * 4 * rs},
        {&ctx->fcons4[0], (size_t)maxp * 4 * rs},
        {&ctx->fcons4[1], (size_t)maxp * 4 * rs},
        {(void **)&ctx->pid[0], (size_t)maxp * sizeof(int32_t)},
        {(void **)&ctx->pid[1], (size_t)maxp * sizeof(int32_t)},
        {(void **)&ctx->slot_of, (size_t)maxp * sizeof(int32_t)},
        {(void **)&ctx->row_count, (size_t)p->ny * p->nz * sizeof(int32_t)},
        {(void **)&ctx->sort_rank, (size_t)maxp * sizeof(int32_t)},
        {(void **)&ctx->chunk_total, (size_t)1024 * sizeof(int32_t)},
        {(void **)&ctx->row_start, ((size_t)p->ny * p->nz + 1) * sizeof(int32_t)},
        {(void **)&ctx->slot_row, (size_t)maxp * sizeof(int32_t)},
        {(void **)&ctx->migrant_slot, (size_t)2 * maxp * sizeof(int32_t)},
        {(void **)&ctx->migrant_count, 2 * sizeof(int32_t)},
        {&ctx->fc4[0], (size_t)maxp * 4 * rs},
        {&ctx->fc4[1], (size_t)maxp * 4 * rs},
        {&ctx->old4, compact ? (size_t)maxp * 4 * rs : 0},
        {(void **)&ctx->occw[0], compact ? occ_bytes : 0},
        {(void **)&ctx->occw[1], compact ? occ_bytes : 0},
        {&ctx->cact[0], compact ? (size_t)2 * ctx->cact_cap * node_bytes : 0},
        {&ctx->cact[1], compact ? (size_t)2 * ctx->cact_cap * node_bytes : 0},
        {(void **)&ctx->arow[0], compact ? arow_bytes : 0},
        {(void **)&ctx->arow[1], compact ? arow_bytes : 0},
        {(void **)&ctx->ccw, compact ? occ_bytes / 2 : 0},
        {(void **)&ctx->dev_error, sizeof(int32_t)},
        {&ctx->tile_table[0], table_bytes},
        {&ctx->tile_table[1], table_bytes},
        {&ctx->edge_acc, table_bytes ? (size_t)ctx->cact_cap * md_tile_edge_bytes(ctx) : 0},
        {(void **)&ctx->tile_flag, table_bytes ? (size_t)md_tile_count(ctx) * sizeof(uint32_t) : 0},
        {(void **)&ctx->late_rows, table_bytes ? (size_t)2 * md_tile_late_cap(ctx) * sizeof(int32_t) : 0},
        {(void **)&ctx->late_count, table_bytes ? 2 * sizeof(int32_t) : 0},
        {(void **)&ctx->blk_done, (size_t)n_lb_blocks * sizeof(uint32_t)},
        {(void **)&ctx->lb_missed, sizeof(int32_t)},
        {(void **)&ctx->missed_list, (size_t)n_lb_blocks * sizeof(int32_t)},
        {(void **)&ctx->missed_total, sizeof(unsigned long long)},
        {(void **)&ctx->range_flag, sizeof(int32_t)},
        {(void **)&ctx->bond_count, (size_t)maxp * sizeof(int32_t)},
        {(void **)&ctx->bond_partner, (size_t)maxp * LBMD_MAX_BONDS_PER_PARTICLE * sizeof(int32_t)},
        {(void **)&ctx->bond_k, (size_t)maxp * LBMD_MAX_BONDS_PER_PARTICLE * sizeof(double)},
        {(void **)&ctx->bond_r0, (size_t)maxp * LBMD_MAX_BONDS_PER_PARTICLE * sizeof(double)},
        {(void **)&ctx->bond_kind, (size_t)maxp * LBMD_MAX_BONDS_PER_PARTICLE},
        {(void **)&ctx->staging, (size_t)ctx->staging_len * sizeof(double)},
        {(void **)&ctx->red_partial, (size_t)ctx->red_blocks * 8 * sizeof(double) + 16},  // + arrival counter
        {(void **)&ctx->red_out, 10 * sizeof(double)},
        {(void **)&ctx->d_lb_step, sizeof(unsigned long long)},
    };
    for (auto &a : allocs) {
        if (a.bytes == 0) continue;
        cudaError_t e = cudaMalloc(a.ptr, a.bytes);
        if (e != cudaSuccess) {
            lbmd_status s = cuda_fail(nullptr, e, "cudaMalloc");
            free_all(ctx);
            delete ctx;
            return s;
        }
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_lb_step, 0, sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->missed_total, 0, sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->range_flag, 0, sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dev_error, 0, sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctx->red_partial, 0, (size_t)ctx->red_blocks * 8 * sizeof(double) + 16, ctx->stream);
    if (e == cudaSuccess && ctx->edge_acc)
        e = cudaMemsetAsync(ctx->edge_acc, 0, (size_t)ctx->cact_cap * md_tile_edge_bytes(ctx), ctx->stream);
    if (e == cudaSuccess && ctx->tile_flag)
        e = cudaMemsetAsync(ctx->tile_flag, 0, (size_t)md_tile_count(ctx) * sizeof(uint32_t), ctx->stream);
    if (e == cudaSuccess && ctx->late_count) e = cudaMemsetAsync(ctx->late_count, 0, 2 * sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->bond_count, 0, (size_t)maxp * sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->bond_kind, 0, (size_t)maxp * LBMD_MAX_BONDS_PER_PARTICLE, ctx->stream);
    // no row buckets yet: every particle is spread as a migrant until the
    // first re-ordering
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctx->row_start, 0, ((size_t)p->ny * p->nz + 1) * sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->slot_row, 0xff, (size_t)maxp * sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->migrant_count, 0, 2 * sizeof(int32_t), ctx->stream);
    // no active nodes until the first re-ordering
    for (int s = 0; s < 2 && e == cudaSuccess; ++s)
        if (ctx->occw[s]) e = cudaMemsetAsync(ctx->occw[s], 0, occ_bytes, ctx->stream);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s)
        if (ctx->arow[s]) e = cudaMemsetAsync(ctx->arow[s], 0, arow_bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->blk_done, 0, (size_t)n_lb_blocks * sizeof(uint32_t), ctx->stream);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b)
        e = cudaMemsetAsync(ctx->fcons4[b], 0, (size_t)maxp * 4 * rs, ctx->stream);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b)
        e = cudaMemsetAsync(ctx->fc4[b], 0, (size_t)maxp * 4 * rs, ctx->stream);
    if (e == cudaSuccess && ctx->jacc) e = cudaMemsetAsync(ctx->jacc, 0, (size_t)N * node_bytes, ctx->stream);
    if (e == cudaSuccess) e = setup_particle_kernels(ctx);
    if (e == cudaSuccess) e = launch_init_equilibrium(ctx);
    if (e == cudaSuccess) e = launch_node_moments(ctx, false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        lbmd_status s = cuda_fail(nullptr, e, "initialisation");
        free_all(ctx);
        delete ctx;
        return s;
    }
    *out = ctx;
    return LBMD_OK;
}

lbmd_status lbmd_destroy(lbmd_ctx *ctx) {
    LBMD_TRACE("lbmd_destroy");
    if (!ctx) return LBMD_OK;
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
    return LBMD_OK;
}

static void drop_cycle_graphs(lbmd_ctx *ctx) {
    for (int i = 0; i < 16; ++i)
        if (ctx->cycle_graph[i]) {
            cudaGraphExecDestroy(ctx->cycle_graph[i]);
            ctx->cycle_graph[i] = nullptr;
        }
}

// The LJ neighbour lists, allocated when LJ forces are first switched on.
static lbmd_status ensure_nb_lists(lbmd_ctx *ctx) {
    if (ctx->nb_list) return LBMD_OK;
    const size_t maxp = (size_t)std::max<int64_t>(ctx->p.max_particles, 1);
    void *bufs[4] = {nullptr, nullptr, nullptr, nullptr};
    const size_t bytes[4] = {maxp * LBMD_NB_MAX * sizeof(int32_t), maxp * sizeof(int32_t), sizeof(int32_t),
                             maxp * 4 * real_size(ctx)};
    for (int k = 0; k < 4; ++k)
        if (cudaMalloc(&bufs[k], bytes[k]) != cudaSuccess) {
            for (int q = 0; q < 4; ++q)
                if (bufs[q]) cudaFree(bufs[q]);
            cudaGetLastError();
            return fail(ctx, LBMD_ERR_OOM, "Lennard-Jones neighbour lists");
        }
    ctx->nb_list = static_cast<int32_t *>(bufs[0]);
    ctx->nb_count = static_cast<int32_t *>(bufs[1]);
    ctx->nb_invalid = static_cast<int32_t *>(bufs[2]);
    ctx->nb_ref4 = bufs[3];
    return LBMD_OK;
}

// Positions changed outside the MD steps (or the lists were never built):
// the pair kernel uses all pairs until the next re-ordering rebuilds them.
static cudaError_t invalidate_nb_lists(lbmd_ctx *ctx) {
    if (!ctx->nb_invalid) return cudaSuccess;
    const int32_t one = 1;
    return cudaMemcpyAsync(ctx->nb_invalid, &one, sizeof(one), cudaMemcpyHostToDevice, ctx->stream);
}

lbmd_status lbmd_add_particles(lbmd_ctx *ctx, int64_t n, const double *pos, const double *vel, const double *mass,
                               int64_t *first_id_out) {
    LBMD_TRACE("lbmd_add_particles");
    if (!ctx) return LBMD_ERR_ARG;
    if (n < 0 || (n > 0 && (!pos || !vel))) return fail(ctx, LBMD_ERR_ARG, "bad particle arrays");
    if (ctx->np + n > ctx->p.max_particles) return fail(ctx, LBMD_ERR_CAPACITY, "max_particles exceeded");
    for (int64_t q = 0; q < 3 * n; ++q)
        if (!is_finite_d(pos[q]) || !is_finite_d(vel[q])) return fail(ctx, LBMD_ERR_ARG, "non-finite particle data");
    if (mass)
        for (int64_t q = 0; q < n; ++q)
            if (!(mass[q] > 0) || !is_finite_d(mass[q])) return fail(ctx, LBMD_ERR_ARG, "mass must be positive");
    // the explicit friction step multiplies the relative velocity by
    // 1 - zeta dt / m per MD step: at zeta dt / m >= 2 it grows without bound
    for (int64_t q = 0; q < (mass ? n : (n > 0 ? 1 : 0)); ++q)
        if (ctx->p.zeta * ctx->dt / (mass ? mass[q] : 1.0) >= 2.0)
            return fail(ctx, LBMD_ERR_ARG, "zeta dt / mass >= 2: the explicit friction step is unstable");
    if (first_id_out) *first_id_out = ctx->np;
    if (n == 0) return LBMD_OK;
    // stage in chunks through the device staging buffer (3 + 3 + 1 doubles each)
    const int64_t per = ctx->staging_len / 7;
    for (int64_t s = 0; s < n; s += per) {
        const int64_t c = std::min(per, n - s);
        double *dpos = ctx->staging, *dvel = ctx->staging + 3 * c, *dm = ctx->staging + 6 * c;
        CK(ctx, cudaMemcpyAsync(dpos, pos + 3 * s, 3 * c * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, cudaMemcpyAsync(dvel, vel + 3 * s, 3 * c * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        if (mass) CK(ctx, cudaMemcpyAsync(dm, mass + s, c * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, launch_particles_from_double(ctx, ctx->np + s, c, dpos, dvel, mass ? dm : nullptr, true, true, true));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    const size_t rs = real_size(ctx);
    CK(ctx, cudaMemsetAsync((char *)ctx->fcons4[ctx->pcur] + ctx->np * 4 * rs, 0, n * 4 * rs, ctx->stream));
    // new slots are in no row bucket until the next re-ordering
    CK(ctx, cudaMemsetAsync(ctx->slot_row + ctx->np, 0xff, n * sizeof(int32_t), ctx->stream));
    CK(ctx, cudaMemsetAsync((char *)ctx->fc4[ctx->pcur] + ctx->np * 4 * rs, 0, n * 4 * rs, ctx->stream));
    ctx->np += n;
    CK(ctx, invalidate_nb_lists(ctx));
    // re-order now, so that every particle sits in the row bucket of its cell
    // (the MD kernels of variant B walk the buckets; the active nodes stay
    // those of the last LB step until the next one)
    CK(ctx, launch_sort_particles(ctx));
    CK(ctx, md_tile_build_table(ctx, (int)(ctx->lb_step & 1)));
    if (has_cons(ctx)) CK(ctx, launch_bond_forces_only(ctx));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    drop_cycle_graphs(ctx);
    return LBMD_OK;
}

static lbmd_status add_bonds_of_kind(lbmd_ctx *ctx, int64_t nb, const int64_t *pairs, double k, double r0,
                                     uint8_t kind) {
    if (ctx->nb + nb > ctx->p.max_bonds) return fail(ctx, LBMD_ERR_CAPACITY, "max_bonds exceeded");
    if (nb == 0) return LBMD_OK;
    const int64_t np = ctx->np;
    const int M = LBMD_MAX_BONDS_PER_PARTICLE;
    std::vector<int32_t> count(np), partner((size_t)np * M);
    std::vector<double> bk((size_t)np * M), br((size_t)np * M);
    std::vector<uint8_t> kd((size_t)np * M);
    CK(ctx, cudaMemcpy(count.data(), ctx->bond_count, np * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CK(ctx, cudaMemcpy(partner.data(), ctx->bond_partner, (size_t)np * M * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CK(ctx, cudaMemcpy(bk.data(), ctx->bond_k, (size_t)np * M * sizeof(double), cudaMemcpyDeviceToHost));
    CK(ctx, cudaMemcpy(br.data(), ctx->bond_r0, (size_t)np * M * sizeof(double), cudaMemcpyDeviceToHost));
    CK(ctx, cudaMemcpy(kd.data(), ctx->bond_kind, (size_t)np * M, cudaMemcpyDeviceToHost));
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t i = pairs[2 * b], j = pairs[2 * b + 1];
        if (i < 0 || j < 0 || i >= np || j >= np || i == j) return fail(ctx, LBMD_ERR_ARG, "bond ids out of range");
        if (count[i] >= M || count[j] >= M) return fail(ctx, LBMD_ERR_CAPACITY, "more than 8 bonds on a particle");
        for (const int64_t e : {i, j}) {
            const size_t s = (size_t)e * M + count[e];
            partner[s] = (int32_t)(e == i ? j : i);
            bk[s] = k;
            br[s] = r0;
            kd[s] = kind;
            count[e]++;
        }
    }
    CK(ctx, cudaMemcpy(ctx->bond_count, count.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(ctx->bond_partner, partner.data(), (size_t)np * M * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(ctx->bond_k, bk.data(), (size_t)np * M * sizeof(double), cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(ctx->bond_r0, br.data(), (size_t)np * M * sizeof(double), cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(ctx->bond_kind, kd.data(), (size_t)np * M, cudaMemcpyHostToDevice));
    ctx->nb += nb;
    CK(ctx, launch_bond_forces_only(ctx));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    drop_cycle_graphs(ctx);
    return LBMD_OK;
}

lbmd_status lbmd_add_bonds(lbmd_ctx *ctx, int64_t nb, const int64_t *pairs, double k, double r0) {
    LBMD_TRACE("lbmd_add_bonds");
    if (!ctx) return LBMD_ERR_ARG;
    if (nb < 0 || (nb > 0 && !pairs) || !is_finite_d(k) || !is_finite_d(r0))
        return fail(ctx, LBMD_ERR_ARG, "bad bonds");
    return add_bonds_of_kind(ctx, nb, pairs, k, r0, LBMD_BOND_HARMONIC);
}

lbmd_status lbmd_add_fene_bonds(lbmd_ctx *ctx, int64_t nb, const int64_t *pairs, double k, double R0) {
    LBMD_TRACE("lbmd_add_fene_bonds");
    if (!ctx) return LBMD_ERR_ARG;
    if (nb < 0 || (nb > 0 && !pairs) || !is_finite_d(k) || !(k >= 0) || !is_finite_d(R0) || !(R0 > 0))
        return fail(ctx, LBMD_ERR_ARG, "bad FENE bonds");
    return add_bonds_of_kind(ctx, nb, pairs, k, R0, LBMD_BOND_FENE);
}

lbmd_status lbmd_set_lj(lbmd_ctx *ctx, double eps, double sigma, double r_cut) {
    LBMD_TRACE("lbmd_set_lj");
    if (!ctx) return LBMD_ERR_ARG;
    if (!is_finite_d(eps) || !(eps >= 0) || !is_finite_d(sigma) || !(sigma > 0) || !is_finite_d(r_cut) ||
        !(r_cut >= 0))
        return fail(ctx, LBMD_ERR_ARG, "bad Lennard-Jones parameters");
    if (r_cut > 0) {
        if (ctx->p.max_particles > LBMD_MAX_LJ_PARTICLES)
            return fail(ctx, LBMD_ERR_CAPACITY, "Lennard-Jones: max_particles above LBMD_MAX_LJ_PARTICLES");
        const int dims[3] = {ctx->p.nx, ctx->p.ny, ctx->p.nz};
        for (int d : dims)
            if ((double)d < 2.0 * r_cut + 2.0)
                return fail(ctx, LBMD_ERR_ARG, "Lennard-Jones: every box edge must be at least 2 r_cut + 2");
    }
    if (r_cut > 0) {
        const lbmd_status st = ensure_nb_lists(ctx);
        if (st != LBMD_OK) return st;
    }
    CK(ctx, invalidate_nb_lists(ctx));  // lists of the old parameters are void until the next build
    ctx->lj_eps = eps;
    ctx->lj_sigma = sigma;
    ctx->lj_rc = r_cut;
    if (ctx->np > 0 && has_cons(ctx)) CK(ctx, launch_bond_forces_only(ctx));
    if (ctx->np > 0 && !has_cons(ctx)) {
        const size_t rs = real_size(ctx);
        CK(ctx, cudaMemsetAsync(ctx->fcons4[ctx->pcur], 0, (size_t)ctx->np * 4 * rs, ctx->stream));
    }
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    drop_cycle_graphs(ctx);
    return LBMD_OK;
}

lbmd_status lbmd_set_particles(lbmd_ctx *ctx, const double *pos, const double *vel) {
    LBMD_TRACE("lbmd_set_particles");
    if (!ctx) return LBMD_ERR_ARG;
    const int64_t n = ctx->np;
    if (n == 0 || (!pos && !vel)) return LBMD_OK;
    if (6 * n > ctx->staging_len) return fail(ctx, LBMD_ERR_CAPACITY, "staging buffer too small");
    double *dpos = ctx->staging, *dvel = ctx->staging + 3 * n;
    if (pos) CK(ctx, cudaMemcpyAsync(dpos, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (vel) CK(ctx, cudaMemcpyAsync(dvel, vel, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, launch_particles_from_double(ctx, 0, n, dpos, dvel, nullptr, pos != nullptr, vel != nullptr, false));
    if (pos) CK(ctx, invalidate_nb_lists(ctx));
    if (pos && has_cons(ctx)) CK(ctx, launch_bond_forces_only(ctx));
    return LBMD_OK;
}

lbmd_status lbmd_md_substep(lbmd_ctx *ctx) {
    LBMD_TRACE("lbmd_md_substep");
    if (!ctx) return LBMD_ERR_ARG;
    if (ctx->sub_done >= ctx->p.n_sub) return fail(ctx, LBMD_ERR_SEQUENCE, "n_sub MD steps already done");
    CK(ctx, launch_md_substep(ctx, ctx->sub_done));
    ctx->sub_done += 1;
    ctx->md_step += 1;
    return LBMD_OK;
}

lbmd_status lbmd_lb_step(lbmd_ctx *ctx) {
    LBMD_TRACE("lbmd_lb_step");
    if (!ctx) return LBMD_ERR_ARG;
    if (ctx->sub_done != ctx->p.n_sub) return fail(ctx, LBMD_ERR_SEQUENCE, "LB step before n_sub MD steps");
    CK(ctx, launch_lb_step(ctx));
    ctx->sub_done = 0;
    ctx->lb_step += 1;
    return LBMD_OK;
}

lbmd_status lbmd_run_cycles(lbmd_ctx *ctx, int64_t n) {
    LBMD_TRACE("lbmd_run_cycles");
    if (!ctx || n < 0) return LBMD_ERR_ARG;
    if (ctx->sub_done != 0) return fail(ctx, LBMD_ERR_SEQUENCE, "run_cycles must start at a cycle boundary");
    for (int64_t c = 0; c < n; ++c) {
        // the launches of a cycle depend on the buffer state it starts from
        const int key = ctx->cur | (int)((ctx->lb_step & 1) << 1) | (ctx->pcur << 2) | (ctx->pv << 3);
        if (!ctx->cycle_graph[key]) {
            // capture one cycle starting from this state
            cudaGraph_t g = nullptr;
            CK(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            const int cur0 = ctx->cur, pcur0 = ctx->pcur, pv0 = ctx->pv, rec0 = ctx->rec;
            for (int s = 0; s < ctx->p.n_sub && e == cudaSuccess; ++s) e = launch_md_substep(ctx, s);
            if (e == cudaSuccess) e = launch_lb_step(ctx);
            // the launchers flipped the buffers during capture: keep the state
            // the cycle leaves, then restore the starting one
            ctx->cycle_post[key][0] = ctx->cur;
            ctx->cycle_post[key][1] = ctx->pcur;
            ctx->cycle_post[key][2] = ctx->pv;
            ctx->cur = cur0;
            ctx->pcur = pcur0;
            ctx->pv = pv0;
            ctx->rec = rec0;
            cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
            if (e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return cuda_fail(ctx, e, "capture");
            }
            if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ctx->cycle_graph[key], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                ctx->cycle_graph[key] = nullptr;
                return cuda_fail(ctx, e, "cudaGraphInstantiate");
            }
        }
        CK(ctx, cudaGraphLaunch(ctx->cycle_graph[key], ctx->stream));
        ctx->cur = ctx->cycle_post[key][0];
        ctx->pcur = ctx->cycle_post[key][1];
        ctx->pv = ctx->cycle_post[key][2];
        ctx->rec = 0;
        ctx->lb_step += 1;
        ctx->md_step += ctx->p.n_sub;
    }
    return LBMD_OK;
}

lbmd_status lbmd_observables(lbmd_ctx *ctx, lbmd_observables_t *out) {
    LBMD_TRACE("lbmd_observables");
    if (!ctx || !out) return LBMD_ERR_ARG;
    double h[10];  // 8 sums, the range flag, the device error flag
    if (ctx->async_ready)  // queued downloads still read the sums
        for (int s = 0; s < 2; ++s) CK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->obs_done[s], 0));
    CK(ctx, launch_observables(ctx));
    CK(ctx, cudaMemcpyAsync(h, ctx->red_out, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (h[9] != 0.0)
        return fail(ctx, LBMD_ERR_CUDA, "a kernel's bounded wait for its own bulk copies gave up: results are invalid");
    out->mass = h[0];
    for (int d = 0; d < 3; ++d) {
        out->p_fluid[d] = h[1 + d];
        out->p_particles[d] = h[4 + d];
    }
    out->e_kin = 0.5 * h[7];
    out->kT_particles = ctx->np > 0 ? h[7] / (3.0 * (double)ctx->np) : 0.0;
    out->lb_step = ctx->lb_step;
    out->md_step = ctx->md_step;
    for (int c = 0; c < 8; ++c)
        if (!is_finite_d(h[c])) return fail(ctx, LBMD_ERR_NONFINITE, "non-finite observable");
    if (h[8] != 0.0)
        return fail(ctx, LBMD_ERR_RANGE,
                    "a node's momentum density reached half the fixed-point range (|u| ~ 1 at rho0): the fluid "
                    "state is no longer valid");
    return LBMD_OK;
}

lbmd_status lbmd_set_moments_wait(lbmd_ctx *ctx, int32_t polls) {
    if (!ctx) return LBMD_ERR_ARG;
    if (polls < -1) return fail(ctx, LBMD_ERR_ARG, "polls must be >= -1");
    const int v = polls < 0 ? LBMD_DEFAULT_FUSE_SPIN : polls;
    if (v != ctx->fuse_spin) {
        ctx->fuse_spin = v;
        drop_cycle_graphs(ctx);  // the captured launches carry the old limit
    }
    return LBMD_OK;
}

lbmd_status lbmd_set_frozen_copy(lbmd_ctx *ctx, int32_t on) {
    if (!ctx) return LBMD_ERR_ARG;
    if (on != 0 && on != 1) return fail(ctx, LBMD_ERR_ARG, "on must be 0 or 1");
    if (ctx->sub_done != 0) return fail(ctx, LBMD_ERR_SEQUENCE, "set_frozen_copy only at a cycle boundary");
    if (ctx->p.variant != LBMD_VARIANT_A || (on != 0) == ctx->a_frozen_copy) return LBMD_OK;
    ctx->a_frozen_copy = on != 0;
    // at a cycle boundary the current set's records are those the moments
    // wrote: the copy starts as the same bytes
    if (ctx->a_frozen_copy)
        CK(ctx, cudaMemcpyAsync(active_records_acc(ctx), active_records_now(ctx),
                                (size_t)ctx->cact_cap * ctx->node_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    drop_cycle_graphs(ctx);  // the captured launches carry the old buffers
    return LBMD_OK;
}

lbmd_status lbmd_moments_fallback_rows(lbmd_ctx *ctx, int64_t *rows) {
    if (!ctx || !rows) return LBMD_ERR_ARG;
    unsigned long long v = 0;
    CK(ctx, cudaMemcpyAsync(&v, ctx->missed_total, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    *rows = (int64_t)v;
    return LBMD_OK;
}

lbmd_status lbmd_get_populations(lbmd_ctx *ctx, double *out) {
    LBMD_TRACE("lbmd_get_populations");
    if (!ctx || !out) return LBMD_ERR_ARG;
    const int64_t total = 19 * ctx->N;
    for (int64_t s = 0; s < total; s += ctx->staging_len) {
        const int64_t c = std::min(ctx->staging_len, total - s);
        CK(ctx, launch_populations_to_double(ctx, s, c, ctx->staging));
        CK(ctx, cudaMemcpyAsync(out + s, ctx->staging, c * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return LBMD_OK;
}

lbmd_status lbmd_set_populations(lbmd_ctx *ctx, const double *in) {
    LBMD_TRACE("lbmd_set_populations");
    if (!ctx || !in) return LBMD_ERR_ARG;
    if (ctx->sub_done != 0) return fail(ctx, LBMD_ERR_SEQUENCE, "set_populations only at a cycle boundary");
    const int64_t total = 19 * ctx->N;
    for (int64_t s = 0; s < total; s += ctx->staging_len) {
        const int64_t c = std::min(ctx->staging_len, total - s);
        CK(ctx, cudaMemcpyAsync(ctx->staging, in + s, c * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, launch_populations_from_double(ctx, s, c, ctx->staging));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    // a new fluid state: the range guard starts over
    CK(ctx, cudaMemsetAsync(ctx->range_flag, 0, sizeof(int32_t), ctx->stream));
    CK(ctx, launch_node_moments(ctx, false));
    CK(ctx, launch_clear_transfer(ctx));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return LBMD_OK;
}

static lbmd_status node_out(lbmd_ctx *ctx, double *out, bool transfer) {
    const int w = transfer ? 3 : 4;
    CK(ctx, launch_active_sync(ctx));
    const int64_t per = ctx->staging_len / w;
    for (int64_t s = 0; s < ctx->N; s += per) {
        const int64_t c = std::min(per, ctx->N - s);
        CK(ctx, launch_node_field_to_double(ctx, s, c, ctx->staging, transfer));
        CK(ctx, cudaMemcpyAsync(out + w * s, ctx->staging, w * c * sizeof(double), cudaMemcpyDeviceToHost,
                                ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return LBMD_OK;
}

lbmd_status lbmd_get_node_field(lbmd_ctx *ctx, double *out) {
    LBMD_TRACE("lbmd_get_node_field");
    if (!ctx || !out) return LBMD_ERR_ARG;
    return node_out(ctx, out, false);
}

lbmd_status lbmd_get_transfer(lbmd_ctx *ctx, double *out) {
    LBMD_TRACE("lbmd_get_transfer");
    if (!ctx || !out) return LBMD_ERR_ARG;
    return node_out(ctx, out, true);
}

lbmd_status lbmd_get_particles(lbmd_ctx *ctx, double *pos, double *vel) {
    LBMD_TRACE("lbmd_get_particles");
    if (!ctx) return LBMD_ERR_ARG;
    const int64_t n = ctx->np;
    if (n == 0 || (!pos && !vel)) return LBMD_OK;
    if (6 * n > ctx->staging_len) return fail(ctx, LBMD_ERR_CAPACITY, "staging buffer too small");
    double *dpos = ctx->staging, *dvel = ctx->staging + 3 * n;
    CK(ctx, launch_particles_to_double(ctx, pos ? dpos : nullptr, vel ? dvel : nullptr));
    if (pos) CK(ctx, cudaMemcpyAsync(pos, dpos, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (vel) CK(ctx, cudaMemcpyAsync(vel, dvel, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return LBMD_OK;
}

}  // extern "C"

namespace {

// the asynchronous accessors' streams, events and buffers, on first use
lbmd_status async_init(lbmd_ctx *ctx) {
    if (ctx->async_ready) return LBMD_OK;
    const size_t n6 = (size_t)6 * (size_t)std::max<int64_t>(ctx->p.max_particles, 1);
    if (!ctx->up_stream) CK(ctx, cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking));
    if (!ctx->down_stream) CK(ctx, cudaStreamCreateWithFlags(&ctx->down_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
        for (cudaEvent_t *ev : {&ctx->in_ready[b], &ctx->in_done[b], &ctx->out_ready[b], &ctx->out_done[b],
                                &ctx->obs_done[b]})
            if (!*ev) CK(ctx, cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
        if (!ctx->stage_in[b]) CK(ctx, cudaMalloc(&ctx->stage_in[b], n6 * sizeof(double)));
        if (!ctx->stage_out[b]) CK(ctx, cudaMalloc(&ctx->stage_out[b], n6 * sizeof(double)));
    }
    if (!ctx->obs_ready) CK(ctx, cudaEventCreateWithFlags(&ctx->obs_ready, cudaEventDisableTiming));
    if (!ctx->obs_host) CK(ctx, cudaHostAlloc((void **)&ctx->obs_host, 2 * 10 * sizeof(double), cudaHostAllocDefault));
    ctx->async_ready = true;
    return LBMD_OK;
}

// the observables of queued slot `s` (whose download is complete) into the
// caller's structure, with the checks of lbmd_observables
lbmd_status finalise_observables(lbmd_ctx *ctx, int s) {
    lbmd_observables_t *out = ctx->obs_out[s];
    ctx->obs_out[s] = nullptr;
    const double *h = ctx->obs_host + 10 * s;
    out->mass = h[0];
    for (int d = 0; d < 3; ++d) {
        out->p_fluid[d] = h[1 + d];
        out->p_particles[d] = h[4 + d];
    }
    out->e_kin = 0.5 * h[7];
    out->kT_particles = ctx->obs_np[s] > 0 ? h[7] / (3.0 * (double)ctx->obs_np[s]) : 0.0;
    out->lb_step = ctx->obs_lb[s];
    out->md_step = ctx->obs_md[s];
    if (h[9] != 0.0)
        return fail(ctx, LBMD_ERR_CUDA, "a kernel's bounded wait for its own bulk copies gave up: results are invalid");
    for (int c = 0; c < 8; ++c)
        if (!is_finite_d(h[c])) return fail(ctx, LBMD_ERR_NONFINITE, "non-finite observable");
    if (h[8] != 0.0)
        return fail(ctx, LBMD_ERR_RANGE,
                    "a node's momentum density reached half the fixed-point range (|u| ~ 1 at rho0): the fluid "
                    "state is no longer valid");
    return LBMD_OK;
}

}  // namespace

extern "C" {

lbmd_status lbmd_set_particles_async(lbmd_ctx *ctx, const double *pos, const double *vel) {
    LBMD_TRACE("lbmd_set_particles_async");
    if (!ctx) return LBMD_ERR_ARG;
    const int64_t n = ctx->np;
    if (n == 0 || (!pos && !vel)) return LBMD_OK;
    if (n > ctx->p.max_particles) return fail(ctx, LBMD_ERR_CAPACITY, "more particles than max_particles");
    const lbmd_status st = async_init(ctx);
    if (st != LBMD_OK) return st;
    const int b = ctx->in_idx;
    ctx->in_idx ^= 1;
    double *dpos = ctx->stage_in[b], *dvel = ctx->stage_in[b] + 3 * n;
    // the upload waits only for the conversion that last read this staging
    // buffer, so it can run beside the work already enqueued
    CK(ctx, cudaStreamWaitEvent(ctx->up_stream, ctx->in_done[b], 0));
    if (pos) CK(ctx, cudaMemcpyAsync(dpos, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->up_stream));
    if (vel) CK(ctx, cudaMemcpyAsync(dvel, vel, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->up_stream));
    CK(ctx, cudaEventRecord(ctx->in_ready[b], ctx->up_stream));
    CK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->in_ready[b], 0));
    CK(ctx, launch_particles_from_double(ctx, 0, n, dpos, dvel, nullptr, pos != nullptr, vel != nullptr, false));
    CK(ctx, cudaEventRecord(ctx->in_done[b], ctx->stream));
    if (pos) CK(ctx, invalidate_nb_lists(ctx));
    if (pos && has_cons(ctx)) CK(ctx, launch_bond_forces_only(ctx));
    return LBMD_OK;
}

lbmd_status lbmd_get_particles_async(lbmd_ctx *ctx, double *pos, double *vel) {
    LBMD_TRACE("lbmd_get_particles_async");
    if (!ctx) return LBMD_ERR_ARG;
    const int64_t n = ctx->np;
    if (n == 0 || (!pos && !vel)) return LBMD_OK;
    if (n > ctx->p.max_particles) return fail(ctx, LBMD_ERR_CAPACITY, "more particles than max_particles");
    const lbmd_status st = async_init(ctx);
    if (st != LBMD_OK) return st;
    const int b = ctx->out_idx;
    ctx->out_idx ^= 1;
    double *dpos = ctx->stage_out[b], *dvel = ctx->stage_out[b] + 3 * n;
    CK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->out_done[b], 0));  // its last download has read it
    CK(ctx, launch_particles_to_double(ctx, pos ? dpos : nullptr, vel ? dvel : nullptr));
    CK(ctx, cudaEventRecord(ctx->out_ready[b], ctx->stream));
    CK(ctx, cudaStreamWaitEvent(ctx->down_stream, ctx->out_ready[b], 0));
    if (pos) CK(ctx, cudaMemcpyAsync(pos, dpos, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->down_stream));
    if (vel) CK(ctx, cudaMemcpyAsync(vel, dvel, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->down_stream));
    CK(ctx, cudaEventRecord(ctx->out_done[b], ctx->down_stream));
    return LBMD_OK;
}

lbmd_status lbmd_observables_async(lbmd_ctx *ctx, lbmd_observables_t *out) {
    LBMD_TRACE("lbmd_observables_async");
    if (!ctx || !out) return LBMD_ERR_ARG;
    lbmd_status st = async_init(ctx);
    if (st != LBMD_OK) return st;
    const int s = ctx->obs_next, prev = s ^ 1;
    ctx->obs_next ^= 1;
    if (ctx->obs_out[s]) {  // the slot's previous observables: complete it first
        CK(ctx, cudaEventSynchronize(ctx->obs_done[s]));
        st = finalise_observables(ctx, s);
    }
    // the reduction overwrites the sums the previous slot's download reads
    CK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->obs_done[prev], 0));
    CK(ctx, launch_observables(ctx));
    CK(ctx, cudaEventRecord(ctx->obs_ready, ctx->stream));
    CK(ctx, cudaStreamWaitEvent(ctx->down_stream, ctx->obs_ready, 0));
    double *h = ctx->obs_host + 10 * s;
    CK(ctx, cudaMemcpyAsync(h, ctx->red_out, 10 * sizeof(double), cudaMemcpyDeviceToHost, ctx->down_stream));
    CK(ctx, cudaEventRecord(ctx->obs_done[s], ctx->down_stream));
    ctx->obs_out[s] = out;
    ctx->obs_np[s] = ctx->np;
    ctx->obs_lb[s] = ctx->lb_step;
    ctx->obs_md[s] = ctx->md_step;
    return st;
}

lbmd_status lbmd_synchronize(lbmd_ctx *ctx) {
    LBMD_TRACE("lbmd_synchronize");
    if (!ctx) return LBMD_ERR_ARG;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (!ctx->async_ready) return LBMD_OK;
    CK(ctx, cudaStreamSynchronize(ctx->up_stream));
    CK(ctx, cudaStreamSynchronize(ctx->down_stream));
    lbmd_status st = LBMD_OK;
    for (int k = 0; k < 2; ++k) {  // oldest first
        const int s = (ctx->obs_next + k) & 1;
        if (!ctx->obs_out[s]) continue;
        const lbmd_status r = finalise_observables(ctx, s);
        if (st == LBMD_OK) st = r;
    }
    return st;
}

lbmd_status lbmd_get_particles_device(lbmd_ctx *ctx, double *pos, double *vel) {
    if (!ctx) return LBMD_ERR_ARG;
    CK(ctx, launch_particles_to_double(ctx, pos, vel));
    return LBMD_OK;
}

lbmd_status lbmd_get_counts(lbmd_ctx *ctx, int64_t *n_particles, int64_t *n_bonds, int64_t *lb_step, int64_t *md_step,
                            int32_t *substeps_done) {
    if (!ctx) return LBMD_ERR_ARG;
    if (n_particles) *n_particles = ctx->np;
    if (n_bonds) *n_bonds = ctx->nb;
    if (lb_step) *lb_step = ctx->lb_step;
    if (md_step) *md_step = ctx->md_step;
    if (substeps_done) *substeps_done = ctx->sub_done;
    return LBMD_OK;
}

// ---------------------------------------------------------------------------
// Saved state: header, populations as stored, particle records as stored
// (slot order, with their ids), the bonds per particle id.  Everything is
// copied in the device representation, so a restored run continues bit for
// bit.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

struct StateHeader {
    char magic[8];
    int32_t version, nx, ny, nz, n_sub, variant, precision, integrator;
    double rho0, nu, nu_bulk, gamma_ghost, kT, zeta, body_force[3];
    uint64_t seed;
    int64_t np, nb, lb_step, md_step;
    double lj_eps, lj_sigma, lj_rc;
};
constexpr char STATE_MAGIC[8] = {'L', 'B', 'M', 'D', 'S', 'T', 'A', 'T'};

size_t align8(size_t b) { return (b + 7) & ~(size_t)7; }

// byte sizes of the sections for np particles
struct StateLayout {
    size_t pops, recs, pid, bonds, total;
};
StateLayout state_layout(const lbmd_ctx *ctx, int64_t np) {
    const int M = LBMD_MAX_BONDS_PER_PARTICLE;
    StateLayout L;
    L.pops = align8((size_t)19 * ctx->N * pop_size(ctx));
    L.recs = (size_t)3 * np * 4 * real_size(ctx);  // pos4, vel4, fc4
    L.pid = align8((size_t)np * sizeof(int32_t));
    L.bonds = align8((size_t)np * sizeof(int32_t)) + align8((size_t)np * M * sizeof(int32_t)) +
              (size_t)2 * np * M * sizeof(double) + align8((size_t)np * M);
    L.total = sizeof(StateHeader) + L.pops + L.recs + L.pid + L.bonds;
    return L;
}

}  // namespace

extern "C" {

lbmd_status lbmd_state_size(lbmd_ctx *ctx, int64_t *bytes) {
    if (!ctx || !bytes) return LBMD_ERR_ARG;
    *bytes = (int64_t)state_layout(ctx, ctx->np).total;
    return LBMD_OK;
}

lbmd_status lbmd_save_state(lbmd_ctx *ctx, void *buf, int64_t bytes) {
    LBMD_TRACE("lbmd_save_state");
    if (!ctx || !buf) return LBMD_ERR_ARG;
    if (ctx->sub_done != 0) return fail(ctx, LBMD_ERR_SEQUENCE, "save_state only at a cycle boundary");
    const StateLayout L = state_layout(ctx, ctx->np);
    if (bytes < (int64_t)L.total) return fail(ctx, LBMD_ERR_CAPACITY, "state buffer smaller than lbmd_state_size");
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, STATE_MAGIC, 8);
    h.version = 1;
    h.nx = ctx->p.nx;
    h.ny = ctx->p.ny;
    h.nz = ctx->p.nz;
    h.n_sub = ctx->p.n_sub;
    h.variant = ctx->p.variant;
    h.precision = ctx->p.precision;
    h.integrator = ctx->p.integrator;
    h.rho0 = ctx->p.rho0;
    h.nu = ctx->p.nu;
    h.nu_bulk = ctx->p.nu_bulk;
    h.gamma_ghost = ctx->p.gamma_ghost;
    h.kT = ctx->p.kT;
    h.zeta = ctx->p.zeta;
    for (int d = 0; d < 3; ++d) h.body_force[d] = ctx->p.body_force[d];
    h.seed = ctx->p.seed;
    h.np = ctx->np;
    h.nb = ctx->nb;
    h.lb_step = ctx->lb_step;
    h.md_step = ctx->md_step;
    h.lj_eps = ctx->lj_eps;
    h.lj_sigma = ctx->lj_sigma;
    h.lj_rc = ctx->lj_rc;
    char *o = static_cast<char *>(buf);
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    const int b = ctx->pcur, M = LBMD_MAX_BONDS_PER_PARTICLE;
    const size_t rb = (size_t)ctx->np * 4 * real_size(ctx), np = (size_t)ctx->np;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    CK(ctx, cudaMemcpy(o, ctx->f[ctx->cur], (size_t)19 * ctx->N * pop_size(ctx), cudaMemcpyDeviceToHost));
    o += L.pops;
    if (np) {
        CK(ctx, cudaMemcpy(o, pos_now(ctx), rb, cudaMemcpyDeviceToHost));
        CK(ctx, cudaMemcpy(o + rb, vel_now(ctx), rb, cudaMemcpyDeviceToHost));
        CK(ctx, cudaMemcpy(o + 2 * rb, ctx->fc4[b], rb, cudaMemcpyDeviceToHost));
        o += L.recs;
        CK(ctx, cudaMemcpy(o, ctx->pid[b], np * sizeof(int32_t), cudaMemcpyDeviceToHost));
        o += L.pid;
        CK(ctx, cudaMemcpy(o, ctx->bond_count, np * sizeof(int32_t), cudaMemcpyDeviceToHost));
        o += align8(np * sizeof(int32_t));
        CK(ctx, cudaMemcpy(o, ctx->bond_partner, np * M * sizeof(int32_t), cudaMemcpyDeviceToHost));
        o += align8(np * M * sizeof(int32_t));
        CK(ctx, cudaMemcpy(o, ctx->bond_k, np * M * sizeof(double), cudaMemcpyDeviceToHost));
        o += np * M * sizeof(double);
        CK(ctx, cudaMemcpy(o, ctx->bond_r0, np * M * sizeof(double), cudaMemcpyDeviceToHost));
        o += np * M * sizeof(double);
        CK(ctx, cudaMemcpy(o, ctx->bond_kind, np * M, cudaMemcpyDeviceToHost));
    }
    return LBMD_OK;
}

lbmd_status lbmd_load_state(lbmd_ctx *ctx, const void *buf, int64_t bytes) {
    LBMD_TRACE("lbmd_load_state");
    if (!ctx || !buf) return LBMD_ERR_ARG;
    if (bytes < (int64_t)sizeof(StateHeader)) return fail(ctx, LBMD_ERR_ARG, "state buffer too small");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, STATE_MAGIC, 8) != 0 || h.version != 1)
        return fail(ctx, LBMD_ERR_ARG, "not a saved lbmd state");
    const lbmd_params &p = ctx->p;
    bool same = h.nx == p.nx && h.ny == p.ny && h.nz == p.nz && h.n_sub == p.n_sub && h.variant == p.variant &&
                h.precision == p.precision && h.integrator == p.integrator && h.rho0 == p.rho0 && h.nu == p.nu &&
                h.nu_bulk == p.nu_bulk && h.gamma_ghost == p.gamma_ghost && h.kT == p.kT && h.zeta == p.zeta &&
                h.seed == p.seed;
    for (int d = 0; d < 3; ++d) same = same && h.body_force[d] == p.body_force[d];
    if (!same) return fail(ctx, LBMD_ERR_ARG, "saved state comes from other parameters");
    if (ctx->np != 0 || ctx->sub_done != 0)
        return fail(ctx, LBMD_ERR_SEQUENCE, "load_state needs a context without particles, at a cycle boundary");
    if (h.np < 0 || h.np > p.max_particles || h.nb < 0 || h.nb > p.max_bonds)
        return fail(ctx, LBMD_ERR_CAPACITY, "saved state needs more particles or bonds than reserved");
    const StateLayout L = state_layout(ctx, h.np);
    if (bytes < (int64_t)L.total) return fail(ctx, LBMD_ERR_ARG, "state buffer shorter than its header says");
    const int b = ctx->pcur, M = LBMD_MAX_BONDS_PER_PARTICLE;
    const size_t np = (size_t)h.np, rb = np * 4 * real_size(ctx);
    const char *in = static_cast<const char *>(buf) + sizeof(h);
    // the ids: a permutation of 0..np-1
    std::vector<int32_t> pid(np), slot_of(np, -1);
    std::memcpy(pid.data(), in + L.pops + L.recs, np * sizeof(int32_t));
    for (size_t s = 0; s < np; ++s) {
        if (pid[s] < 0 || (size_t)pid[s] >= np || slot_of[pid[s]] >= 0)
            return fail(ctx, LBMD_ERR_ARG, "saved state: particle ids are not a permutation");
        slot_of[pid[s]] = (int32_t)s;
    }
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    CK(ctx, cudaMemcpy(ctx->f[ctx->cur], in, (size_t)19 * ctx->N * pop_size(ctx), cudaMemcpyHostToDevice));
    in += L.pops;
    if (np) {
        CK(ctx, cudaMemcpy(pos_now(ctx), in, rb, cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(vel_now(ctx), in + rb, rb, cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(ctx->fc4[b], in + 2 * rb, rb, cudaMemcpyHostToDevice));
        in += L.recs;
        CK(ctx, cudaMemcpy(ctx->pid[b], pid.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(ctx->slot_of, slot_of.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice));
        in += L.pid;
        CK(ctx, cudaMemcpy(ctx->bond_count, in, np * sizeof(int32_t), cudaMemcpyHostToDevice));
        in += align8(np * sizeof(int32_t));
        CK(ctx, cudaMemcpy(ctx->bond_partner, in, np * M * sizeof(int32_t), cudaMemcpyHostToDevice));
        in += align8(np * M * sizeof(int32_t));
        CK(ctx, cudaMemcpy(ctx->bond_k, in, np * M * sizeof(double), cudaMemcpyHostToDevice));
        in += np * M * sizeof(double);
        CK(ctx, cudaMemcpy(ctx->bond_r0, in, np * M * sizeof(double), cudaMemcpyHostToDevice));
        in += np * M * sizeof(double);
        CK(ctx, cudaMemcpy(ctx->bond_kind, in, np * M, cudaMemcpyHostToDevice));
        // no row buckets until the next re-ordering; no migrants listed
        CK(ctx, cudaMemset(ctx->slot_row, 0xff, np * sizeof(int32_t)));
        CK(ctx, cudaMemset(ctx->migrant_count, 0, 2 * sizeof(int32_t)));
    }
    ctx->np = h.np;
    ctx->nb = h.nb;
    ctx->lb_step = h.lb_step;
    ctx->md_step = h.md_step;
    ctx->lj_eps = h.lj_eps;
    ctx->lj_sigma = h.lj_sigma;
    ctx->lj_rc = h.lj_rc;
    if (h.lj_rc > 0) {
        const lbmd_status st = ensure_nb_lists(ctx);
        if (st != LBMD_OK) return st;
    }
    CK(ctx, invalidate_nb_lists(ctx));
    const unsigned long long step = (unsigned long long)h.lb_step;
    CK(ctx, cudaMemcpy(ctx->d_lb_step, &step, sizeof(step), cudaMemcpyHostToDevice));
    // node field of the restored populations (no pending transfer at a cycle
    // boundary) and the conservative forces at the restored positions; the
    // range guard starts over
    CK(ctx, cudaMemset(ctx->range_flag, 0, sizeof(int32_t)));
    CK(ctx, launch_node_moments(ctx, false));
    CK(ctx, launch_clear_transfer(ctx));
    // every particle into the row bucket of its cell (see lbmd_add_particles)
    if (ctx->np > 0) CK(ctx, launch_sort_particles(ctx));
    CK(ctx, md_tile_build_table(ctx, (int)(ctx->lb_step & 1)));
    if (ctx->np > 0 && has_cons(ctx)) CK(ctx, launch_bond_forces_only(ctx));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    drop_cycle_graphs(ctx);
    return LBMD_OK;
}

}  // extern "C"
