// particles.cu -- the dissipative particle-fluid coupling of Sec. 3 on the GPU.
//
// couple_kernel (one thread per particle slot), one MD step of length dt:
//   * node velocities at the 8 corners of the particle's cell, trilinear
//     weights delta_k from the fractional position (Eq. (5));
//   * random force from Philox(id, md_step, 1, 0), friction against the
//     interpolated fluid velocity (Eq. (4)); Delta P = dt F (Eq. (6));
//   * velocity Verlet with F held fixed (second half-kick here for ideal
//     particles, in bond_kick_kernel when bonds exist);
//   * variant A: the transfer -delta_k Delta P (Eqs. (7), (8)) goes straight
//     into the accumulator J_acc, which no MD step reads;
//     variant B: the start-of-step position and F are kept for
//     spread_rows_kernel, which runs once every particle has read the node
//     field.
// Transfers are added as fixed-point integers with atomics, so the sum does
// not depend on the order of the particles (bitwise reproducible).
//
// Particle positions are stored as cell index + fractional offset in [0,1):
// the offset is exactly the interpolation coordinate, and its precision does
// not degrade with the box size.
//
// sort_*: once per LB step the particles are re-ordered by the lattice row
// (y, z) of their cell (counting sort: count, scan, scatter), so that a warp
// handles particles whose corner nodes lie in a few neighbouring rows.
#include "lbmd_ctx.h"
#include "lbmd_device.cuh"

namespace lbmd {

template <typename T>
struct PArgs {
    using P = Prec<T>;
    typename P::real4 *pos4, *vel4, *fc4, *old4, *fcons4;
    const int32_t *pid, *slot_of;
    typename P::node4 *node, *jacc;
    const int32_t *bond_count, *bond_partner;
    const double *bond_k, *bond_r0;
    int nx, ny, nz;
    int64_t np;
    T zeta, dt, half_dt, amp;
    uint32_t key0, key1;
    const unsigned long long *lb_step;
    int n_sub, substep, noisy;
    int variant;
    // variant B row-gather spreading
    const int32_t *row_start, *slot_row;
    int32_t *migrant_slot, *migrant_count;  // two lists of np_cap slots, two counters
    int64_t np_cap;
};

struct CellXYZ {
    int x, y, z;
};

__device__ __forceinline__ CellXYZ cell_xyz(int64_t cell, int nx, int ny) {
    const uint32_t c = (uint32_t)cell;
    const uint32_t row = c / (uint32_t)nx;
    CellXYZ r;
    r.x = (int)(c - row * (uint32_t)nx);
    r.z = (int)(row / (uint32_t)ny);
    r.y = (int)(row - (uint32_t)r.z * (uint32_t)ny);
    return r;
}

// The 8 corner nodes (k = ox + 2 oy + 4 oz) and trilinear weights of Eq. (5).
template <typename T>
__device__ __forceinline__ void corners(const CellXYZ &c, T fx, T fy, T fz, int nx, int ny, int nz, uint32_t idx[8],
                                        T delta[8]) {
    const int x1 = c.x + 1 == nx ? 0 : c.x + 1;
    const int y1 = c.y + 1 == ny ? 0 : c.y + 1;
    const int z1 = c.z + 1 == nz ? 0 : c.z + 1;
    const int X[2] = {c.x, x1}, Y[2] = {c.y, y1}, Z[2] = {c.z, z1};
    const T wx[2] = {T(1) - fx, fx}, wy[2] = {T(1) - fy, fy}, wz[2] = {T(1) - fz, fz};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int ox = k & 1, oy = (k >> 1) & 1, oz = (k >> 2) & 1;
        idx[k] = (uint32_t)X[ox] + (uint32_t)nx * ((uint32_t)Y[oy] + (uint32_t)ny * (uint32_t)Z[oz]);
        delta[k] = wx[ox] * wy[oy] * wz[oz];
    }
}

// Move a fractional coordinate by d and carry whole cells into the index.
template <typename T>
__device__ __forceinline__ void advance(T &frac, int &c, T d, int n) {
    T x = frac + d;
    T s = floor(x);
    x -= s;
    if (x >= T(1)) {  // a tiny negative offset rounded up to the next node
        x = T(0);
        s += T(1);
    }
    int cn = c + (int)s;
    cn %= n;
    if (cn < 0) cn += n;
    frac = x;
    c = cn;
}

template <typename T>
__device__ __forceinline__ void spread_to(typename Prec<T>::node4 *field, const uint32_t idx[8], const T delta[8], T dPx,
                                          T dPy, T dPz) {
    using P = Prec<T>;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        P::add_transfer(&field[idx[k]], P::to_fix(-delta[k] * dPx), P::to_fix(-delta[k] * dPy),
                        P::to_fix(-delta[k] * dPz));
}

// The variant is a run-time flag (one instruction sequence for both
// variants, as in the LB kernel).  At least 6 blocks of 256 threads per SM:
// the corner loads are scattered, so latency hiding needs many warps.
template <typename T, bool BONDS>
__global__ void __launch_bounds__(256, 6) couple_kernel(PArgs<T> a) {
    using P = Prec<T>;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const typename P::real4 R = a.pos4[p];
    typename P::real4 V = a.vel4[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.nx, a.ny);
    uint32_t idx[8];
    T delta[8];
    corners(c, R.x, R.y, R.z, a.nx, a.ny, a.nz, idx, delta);

    // fluid velocity at the particle, Eq. (5)
    T ux = T(0), uy = T(0), uz = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const typename P::node4 n = a.node[idx[k]];
        const T w = delta[k] / P::rho_of(n);
        ux += w * P::from_fix(P::jx_of(n));
        uy += w * P::from_fix(P::jy_of(n));
        uz += w * P::from_fix(P::jz_of(n));
    }
    // coupling force, Eq. (4) without the conservative part
    T Fx = -a.zeta * (V.x - ux), Fy = -a.zeta * (V.y - uy), Fz = -a.zeta * (V.z - uz);
    if (a.noisy) {
        const uint32_t md_step = (uint32_t)((*a.lb_step) * (unsigned long long)a.n_sub + (unsigned)a.substep);
        const U4 r = philox4x32_10(U4{(uint32_t)a.pid[p], md_step, 1u, 0u}, a.key0, a.key1);
        Fx += a.amp * unit_uniform<T>(r.x);
        Fy += a.amp * unit_uniform<T>(r.y);
        Fz += a.amp * unit_uniform<T>(r.z);
    }
    // velocity Verlet with F held fixed over the step
    const T hm = a.half_dt * V.w;  // V.w = 1 / mass
    T Gx = Fx, Gy = Fy, Gz = Fz;
    if (BONDS) {
        const typename P::real4 Fc = a.fcons4[p];
        Gx += Fc.x;
        Gy += Fc.y;
        Gz += Fc.z;
    }
    V.x += hm * Gx;
    V.y += hm * Gy;
    V.z += hm * Gz;
    T fx = R.x, fy = R.y, fz = R.z;
    int cx = c.x, cy = c.y, cz = c.z;
    advance(fx, cx, a.dt * V.x, a.nx);
    advance(fy, cy, a.dt * V.y, a.ny);
    advance(fz, cz, a.dt * V.z, a.nz);
    if (!BONDS) {
        V.x += hm * Fx;
        V.y += hm * Fy;
        V.z += hm * Fz;
    }
    a.pos4[p] = P::make_pos(fx, fy, fz, cx + (int64_t)a.nx * (cy + (int64_t)a.ny * cz));
    a.vel4[p] = V;
    if (BONDS || a.variant == LBMD_VARIANT_B) a.fc4[p] = P::make4(Fx, Fy, Fz, T(0));

    if (a.variant == LBMD_VARIANT_A) {
        // Newton's third law, Eqs. (7), (8): straight into J_acc
        spread_to<T>(a.jacc, idx, delta, a.dt * Fx, a.dt * Fy, a.dt * Fz);
    } else {
        a.old4[p] = R;
        // a particle whose cell row is no longer the row bucket it was sorted
        // into is spread separately, after the row gather; the two lists
        // alternate with the parity of the MD step
        if ((int32_t)((uint32_t)P::cell_of(R) / (uint32_t)a.nx) != a.slot_row[p]) {
            const int par = (int)((*a.lb_step * (unsigned long long)a.n_sub + (unsigned)a.substep) & 1ull);
            a.migrant_slot[(int64_t)par * a.np_cap + atomicAdd(a.migrant_count + par, 1)] = (int32_t)p;
        }
    }
}

__device__ __forceinline__ void fix_add(int32_t *a, int32_t v) { atomicAdd(a, v); }
__device__ __forceinline__ void fix_add(long long *a, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(a), (unsigned long long)v);
}

// Variant B, atomic-free: one warp per node row (y, z), four rows per block,
// rows in reverse order (the couple kernel touched the high rows last).  The
// row's nodes get transfers only from particles in the four cell rows
// (y - oy, z - oz), oy, oz in {0, 1}; with the particles bucketed by cell
// row, the warp reads those buckets, adds each particle's two contributions
// to this row (nodes x and x + 1, weight delta_k as in Eq. (5)) as
// fixed-point integers in shared memory, and then updates only the touched
// nodes of the row with plain loads and stores: no other warp writes this
// row.  Particles that left their bucket's row are skipped here and spread
// by migrant_spread_kernel.
constexpr int GATHER_WARPS = 4;

template <typename T>
__global__ void __launch_bounds__(32 * GATHER_WARPS) spread_rows_kernel(PArgs<T> a, int n_rows) {
    using P = Prec<T>;
    using fix = typename P::fix;
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    fix *acc = reinterpret_cast<fix *>(smem_raw) + (size_t)warp * 3 * a.nx;  // [nx][3] per warp
    const int g = blockIdx.x * GATHER_WARPS + warp;
    if (g >= n_rows) return;
    const int nrow = n_rows - 1 - g;
    const int y = nrow % a.ny, z = nrow / a.ny;
    for (int i = lane; i < 3 * a.nx; i += 32) acc[i] = 0;
    int32_t lo[4], len[4], crow[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int oy = q & 1, oz = q >> 1;
        const int cy = y - oy < 0 ? a.ny - 1 : y - oy;
        const int cz = z - oz < 0 ? a.nz - 1 : z - oz;
        crow[q] = cy + a.ny * cz;
        lo[q] = a.row_start[crow[q]];
        len[q] = a.row_start[crow[q] + 1] - lo[q];
    }
    __syncwarp();
    const int total = len[0] + len[1] + len[2] + len[3];
    for (int t = lane; t < total; t += 32) {
        int q = 0, off = t;
        while (off >= len[q]) {
            off -= len[q];
            ++q;
        }
        const int64_t p = lo[q] + off;
        const typename P::real4 R = a.old4[p];
        const uint32_t cell = (uint32_t)P::cell_of(R);
        const uint32_t row = cell / (uint32_t)a.nx;
        if ((int32_t)row != crow[q]) continue;  // migrant
        const int cx = (int)(cell - row * (uint32_t)a.nx);
        const int x1 = cx + 1 == a.nx ? 0 : cx + 1;
        const typename P::real4 F = a.fc4[p];
        const int oy = q & 1, oz = q >> 1;
        const T wx[2] = {T(1) - R.x, R.x};
        const T wy = oy ? R.y : T(1) - R.y;
        const T wz = oz ? R.z : T(1) - R.z;
        const T dPx = a.dt * F.x, dPy = a.dt * F.y, dPz = a.dt * F.z;
#pragma unroll
        for (int ox = 0; ox < 2; ++ox) {
            const T d = wx[ox] * wy * wz;  // the corner weight delta_k of Eq. (5)
            fix *ak = acc + 3 * (ox ? x1 : cx);
            fix_add(ak + 0, P::to_fix(-d * dPx));
            fix_add(ak + 1, P::to_fix(-d * dPy));
            fix_add(ak + 2, P::to_fix(-d * dPz));
        }
    }
    __syncwarp();
    typename P::node4 *rowp = a.node + (size_t)a.nx * nrow;
    for (int x = lane; x < a.nx; x += 32) {
        const fix dx = acc[3 * x], dy = acc[3 * x + 1], dz = acc[3 * x + 2];
        if (dx == 0 && dy == 0 && dz == 0) continue;
        P::add_transfer_plain(&rowp[x], dx, dy, dz);
    }
}

// Variant B: the migrants of this MD step, spread with atomics once the row
// gather is done.
template <typename T>
__global__ void __launch_bounds__(256) migrant_spread_kernel(PArgs<T> a) {
    using P = Prec<T>;
    const int par = (int)((*a.lb_step * (unsigned long long)a.n_sub + (unsigned)a.substep) & 1ull);
    const int n = a.migrant_count[par];
    // the other list serves the next MD step: empty it now (nobody uses it
    // during this one)
    if (blockIdx.x == 0 && threadIdx.x == 0) a.migrant_count[par ^ 1] = 0;
    const int32_t *list = a.migrant_slot + (int64_t)par * a.np_cap;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int64_t p = list[t];
        const typename P::real4 R = a.old4[p];
        const typename P::real4 F = a.fc4[p];
        const CellXYZ c = cell_xyz(P::cell_of(R), a.nx, a.ny);
        uint32_t idx[8];
        T delta[8];
        corners(c, R.x, R.y, R.z, a.nx, a.ny, a.nz, idx, delta);
        spread_to<T>(a.node, idx, delta, a.dt * F.x, a.dt * F.y, a.dt * F.z);
    }
}

// Harmonic bond forces at the current positions (minimum image), summed per
// particle over its partners in a fixed order; with KICK, also the second
// velocity-Verlet half-kick with the stored coupling force.
template <typename T, bool KICK>
__global__ void __launch_bounds__(256) bond_kick_kernel(PArgs<T> a) {
    using P = Prec<T>;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const typename P::real4 R = a.pos4[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.nx, a.ny);
    const int64_t id = a.pid[p];
    T Fx = T(0), Fy = T(0), Fz = T(0);
    const int nbond = a.bond_count[id];
    for (int b = 0; b < nbond; ++b) {
        const int64_t q = a.slot_of[a.bond_partner[id * LBMD_MAX_BONDS_PER_PARTICLE + b]];
        const typename P::real4 S = a.pos4[q];
        const CellXYZ d = cell_xyz(P::cell_of(S), a.nx, a.ny);
        T dx = T(d.x - c.x) + (S.x - R.x);
        T dy = T(d.y - c.y) + (S.y - R.y);
        T dz = T(d.z - c.z) + (S.z - R.z);
        dx -= T(a.nx) * rint(dx / T(a.nx));
        dy -= T(a.ny) * rint(dy / T(a.ny));
        dz -= T(a.nz) * rint(dz / T(a.nz));
        const T r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r > T(0)) {
            const T k = (T)a.bond_k[id * LBMD_MAX_BONDS_PER_PARTICLE + b];
            const T r0 = (T)a.bond_r0[id * LBMD_MAX_BONDS_PER_PARTICLE + b];
            const T mag = k * (r - r0) / r;
            Fx += mag * dx;
            Fy += mag * dy;
            Fz += mag * dz;
        }
    }
    a.fcons4[p] = P::make4(Fx, Fy, Fz, T(0));
    if (KICK) {
        typename P::real4 V = a.vel4[p];
        const typename P::real4 Fc = a.fc4[p];
        const T hm = a.half_dt * V.w;
        V.x += hm * (Fx + Fc.x);
        V.y += hm * (Fy + Fc.y);
        V.z += hm * (Fz + Fc.z);
        a.vel4[p] = V;
    }
}

// ---------------------------------------------------------------------------
// Re-ordering by lattice row.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
    sort_count_kernel(const typename Prec<T>::real4 *pos4, int64_t np, int nx, int32_t *row_count, int32_t *rank) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const uint32_t row = (uint32_t)Prec<T>::cell_of(pos4[p]) / (uint32_t)nx;
    rank[p] = atomicAdd(&row_count[row], 1);
}

// Block-wide exclusive scan of one value per thread (1024 threads).
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *total) {
    __shared__ int32_t warp_sum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sum[w] = x;
    __syncthreads();
    if (w == 0) {
        int32_t s = warp_sum[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        warp_sum[lane] = s;  // inclusive prefix of warp sums
    }
    __syncthreads();
    const int32_t before = w > 0 ? warp_sum[w - 1] : 0;
    if (total) *total = warp_sum[31];
    __syncthreads();
    return before + x - v;
}

// Level 1: each block of 1024 threads turns 1024 row counts into exclusive
// offsets within its chunk and records the chunk total.
__global__ void __launch_bounds__(1024) sort_chunk_scan_kernel(int32_t *row_count, int64_t n, int32_t *chunk_total) {
    const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    const int32_t v = i < n ? row_count[i] : 0;
    int32_t tot;
    const int32_t ex = block_exclusive_scan(v, &tot);
    if (i < n) row_count[i] = ex;
    if (threadIdx.x == 0) chunk_total[blockIdx.x] = tot;
}

// Level 2: block c adds the totals of chunks 0..c-1 to its 1024 offsets,
// giving the first slot of every row; row_start[n] = np closes the table.
__global__ void __launch_bounds__(1024) sort_finalize_kernel(const int32_t *row_offset, const int32_t *chunk_total,
                                                             int64_t n, int32_t *row_start, int32_t np) {
    int32_t before;
    const int32_t v = (int)threadIdx.x < (int)blockIdx.x ? chunk_total[threadIdx.x] : 0;
    block_exclusive_scan(v, &before);  // total of the first blockIdx.x chunks
    const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) row_start[i] = before + row_offset[i];
    if (i == n - 1) row_start[n] = np;
}

// Move every particle to row_start[row] + rank within the row.
template <typename T>
__global__ void __launch_bounds__(256)
    sort_scatter_kernel(const typename Prec<T>::real4 *pos_in, const typename Prec<T>::real4 *vel_in,
                        const typename Prec<T>::real4 *fcons_in, const int32_t *pid_in, typename Prec<T>::real4 *pos_out,
                        typename Prec<T>::real4 *vel_out, typename Prec<T>::real4 *fcons_out, int32_t *pid_out,
                        int32_t *slot_of, int32_t *slot_row, const int32_t *row_start, const int32_t *rank, int64_t np,
                        int nx, int bonds) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const typename Prec<T>::real4 R = pos_in[p];
    const uint32_t row = (uint32_t)Prec<T>::cell_of(R) / (uint32_t)nx;
    const int32_t dst = row_start[row] + rank[p];
    slot_row[dst] = (int32_t)row;
    pos_out[dst] = R;
    vel_out[dst] = vel_in[p];
    if (bonds) fcons_out[dst] = fcons_in[p];
    const int32_t id = pid_in[p];
    pid_out[dst] = id;
    slot_of[id] = dst;
}

// shared memory of the row gather: 3 fixed-point sums per node of a row
template <typename T>
static size_t gather_smem_bytes(const lbmd_ctx *ctx) {
    return (size_t)GATHER_WARPS * 3 * ctx->p.nx * sizeof(typename Prec<T>::fix);
}

// The row gather's shared memory grows with nx; allow more than the default
// 48 KB per block (up to 200 KB: nx <= 4096 in FP32, 2048 in FP64).
template <typename T>
static cudaError_t setup_t(lbmd_ctx *ctx) {
    const size_t smem = gather_smem_bytes<T>(ctx);
    if (smem > (size_t)200 * 1024) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(spread_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
static PArgs<T> make_pargs(lbmd_ctx *ctx, int substep) {
    using P = Prec<T>;
    const int b = ctx->pcur;
    PArgs<T> a;
    a.pos4 = static_cast<typename P::real4 *>(ctx->pos4[b]);
    a.vel4 = static_cast<typename P::real4 *>(ctx->vel4[b]);
    a.fcons4 = static_cast<typename P::real4 *>(ctx->fcons4[b]);
    a.pid = ctx->pid[b];
    a.slot_of = ctx->slot_of;
    a.fc4 = static_cast<typename P::real4 *>(ctx->fc4);
    a.old4 = static_cast<typename P::real4 *>(ctx->old4);
    a.node = static_cast<typename P::node4 *>(ctx->node);
    a.jacc = static_cast<typename P::node4 *>(ctx->jacc);
    a.bond_count = ctx->bond_count;
    a.bond_partner = ctx->bond_partner;
    a.bond_k = ctx->bond_k;
    a.bond_r0 = ctx->bond_r0;
    a.nx = ctx->p.nx;
    a.ny = ctx->p.ny;
    a.nz = ctx->p.nz;
    a.np = ctx->np;
    a.zeta = (T)ctx->p.zeta;
    a.dt = (T)ctx->dt;
    a.half_dt = (T)(0.5 * ctx->dt);
    a.amp = (T)sqrt(2.0 * ctx->p.zeta * ctx->p.kT / ctx->dt);
    a.key0 = (uint32_t)(ctx->p.seed & 0xffffffffu);
    a.key1 = (uint32_t)(ctx->p.seed >> 32);
    a.lb_step = ctx->d_lb_step;
    a.n_sub = ctx->p.n_sub;
    a.substep = substep;
    a.noisy = ctx->p.kT > 0.0 ? 1 : 0;
    a.variant = ctx->p.variant;
    a.row_start = ctx->row_start;
    a.slot_row = ctx->slot_row;
    a.migrant_slot = ctx->migrant_slot;
    a.migrant_count = ctx->migrant_count;
    a.np_cap = ctx->p.max_particles > 0 ? ctx->p.max_particles : 1;
    return a;
}

template <typename T>
static cudaError_t md_substep_t(lbmd_ctx *ctx, int substep) {
    if (ctx->np == 0) return cudaSuccess;
    PArgs<T> a = make_pargs<T>(ctx, substep);
    const unsigned blocks = (unsigned)((ctx->np + 255) / 256);
    const bool bonds = ctx->nb > 0;
    const bool B = ctx->p.variant == LBMD_VARIANT_B;
    cudaError_t e;
    if (bonds)
        couple_kernel<T, true><<<blocks, 256, 0, ctx->stream>>>(a);
    else
        couple_kernel<T, false><<<blocks, 256, 0, ctx->stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (bonds) {
        bond_kick_kernel<T, true><<<blocks, 256, 0, ctx->stream>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (B) {
        const int rows = (int)((int64_t)ctx->p.ny * ctx->p.nz);
        const unsigned gblocks = (unsigned)((rows + GATHER_WARPS - 1) / GATHER_WARPS);
        spread_rows_kernel<T><<<gblocks, 32 * GATHER_WARPS, gather_smem_bytes<T>(ctx), ctx->stream>>>(a, rows);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        migrant_spread_kernel<T><<<ctx->sm_count, 256, 0, ctx->stream>>>(a);
        e = cudaGetLastError();
    }
    return e;
}

template <typename T>
static cudaError_t bond_forces_t(lbmd_ctx *ctx) {
    if (ctx->np == 0) return cudaSuccess;
    PArgs<T> a = make_pargs<T>(ctx, 0);
    const unsigned blocks = (unsigned)((ctx->np + 255) / 256);
    bond_kick_kernel<T, false><<<blocks, 256, 0, ctx->stream>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t sort_t(lbmd_ctx *ctx) {
    using R4 = typename Prec<T>::real4;
    const int b = ctx->pcur, o = b ^ 1;
    const int64_t rows = (int64_t)ctx->p.ny * ctx->p.nz;
    cudaError_t e = cudaMemsetAsync(ctx->row_count, 0, (size_t)rows * sizeof(int32_t), ctx->stream);
    if (e != cudaSuccess) return e;
    if (ctx->np > 0) {
        const unsigned blocks = (unsigned)((ctx->np + 255) / 256);
        sort_count_kernel<T><<<blocks, 256, 0, ctx->stream>>>(static_cast<const R4 *>(ctx->pos4[b]), ctx->np,
                                                                ctx->p.nx, ctx->row_count, ctx->sort_rank);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int n_chunks = (int)((rows + 1023) / 1024);
        sort_chunk_scan_kernel<<<n_chunks, 1024, 0, ctx->stream>>>(ctx->row_count, rows, ctx->chunk_total);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        sort_finalize_kernel<<<n_chunks, 1024, 0, ctx->stream>>>(ctx->row_count, ctx->chunk_total, rows,
                                                                 ctx->row_start, (int32_t)ctx->np);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        sort_scatter_kernel<T><<<blocks, 256, 0, ctx->stream>>>(
            static_cast<const R4 *>(ctx->pos4[b]), static_cast<const R4 *>(ctx->vel4[b]),
            static_cast<const R4 *>(ctx->fcons4[b]), ctx->pid[b], static_cast<R4 *>(ctx->pos4[o]),
            static_cast<R4 *>(ctx->vel4[o]), static_cast<R4 *>(ctx->fcons4[o]), ctx->pid[o], ctx->slot_of,
            ctx->slot_row, ctx->row_start, ctx->sort_rank, ctx->np, ctx->p.nx, ctx->nb > 0 ? 1 : 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    ctx->pcur = o;
    return cudaSuccess;
}

}  // namespace lbmd

cudaError_t launch_md_substep(lbmd_ctx *ctx, int substep) {
    return ctx->p.precision == LBMD_FP64 ? lbmd::md_substep_t<double>(ctx, substep)
                                         : lbmd::md_substep_t<float>(ctx, substep);
}

cudaError_t launch_bond_forces_only(lbmd_ctx *ctx) {
    return ctx->p.precision == LBMD_FP64 ? lbmd::bond_forces_t<double>(ctx) : lbmd::bond_forces_t<float>(ctx);
}

cudaError_t setup_particle_kernels(lbmd_ctx *ctx) {
    return ctx->p.precision == LBMD_FP64 ? lbmd::setup_t<double>(ctx) : lbmd::setup_t<float>(ctx);
}

cudaError_t launch_sort_particles(lbmd_ctx *ctx) {
    return ctx->p.precision == LBMD_FP64 ? lbmd::sort_t<double>(ctx) : lbmd::sort_t<float>(ctx);
}
