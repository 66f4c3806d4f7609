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
//
// active_*: variant B, after each re-ordering: the corners of the particles'
// cells become the active nodes, numbered row by row into a compact array of
// node records (filled by the post-stream moments of the LB step).  Between
// LB updates the MD kernels read and update an active node through its
// compact record, which is about as large as the touched part of the lattice
// rather than the whole node field, and a node that is not active (one a
// particle reaches only after moving to another cell) through the node
// field, as before.
#include <algorithm>
#include <cmath>

#include "lbmd_ctx.h"
#include "lbmd_device.cuh"
#include "particle_core.cuh"
#include "particle_step.cuh"

// the tiled variant-B MD step (md_tile.cu)
namespace lbmd {
template <typename T>
struct PArgs;
}
template <typename T>
cudaError_t md_tile_step(lbmd_ctx *ctx, const lbmd::PArgs<T> &a);

namespace lbmd {

// One MD step, coupling force from the start of the step (integrator START):
// F = -zeta (v - u(R)) + F_rand with R, v of the beginning of the step
// (Eqs. (4)-(6)), velocity Verlet with F held over both half-kicks (the
// second one here for particles without conservative forces, in the bond /
// pair kernel otherwise), transfer around the start position.
// The variant is a run-time flag (one instruction sequence for both
// variants, as in the LB kernel).  At least 5 blocks of 256 threads per SM
// (3 in FP64): the corner loads are scattered, so latency hiding needs many
// warps.
template <typename T, bool BONDS>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 3) couple_kernel(PArgs<T> a) {
    using P = Prec<T>;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const typename P::real4 R = a.pos4[p];
    typename P::real4 V = a.vel4[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.fd_nx, a.fd_ny);
    T ux, uy, uz, Fx, Fy, Fz;
    interp_u(a, c, R.x, R.y, R.z, ux, uy, uz);
    coupling_force(a, p, V, ux, uy, uz, Fx, Fy, Fz);
    // velocity Verlet with F held fixed over the step
    const T hm = a.half_dt * V.w;  // V.w = 1 / mass
    T Gx = Fx, Gy = Fy, Gz = Fz;
    if (BONDS) {
        const typename P::real4 Fc = a.fcons4[p];
        Gx += Fc.x;
        Gy += Fc.y;
        Gz += Fc.z;
    }
    V.x = fma(hm, Gx, V.x);
    V.y = fma(hm, Gy, V.y);
    V.z = fma(hm, Gz, V.z);
    T fx = R.x, fy = R.y, fz = R.z;
    int cx = c.x, cy = c.y, cz = c.z;
    advance(fx, cx, a.dt, V.x, a.nx);
    advance(fy, cy, a.dt, V.y, a.ny);
    advance(fz, cz, a.dt, V.z, a.nz);
    if (!BONDS) {
        V.x = fma(hm, Fx, V.x);
        V.y = fma(hm, Fy, V.y);
        V.z = fma(hm, Fz, V.z);
    }
    if (BONDS) check_list_skin(a, p, CellXYZ{cx, cy, cz}, fx, fy, fz);
    a.pos4[p] = P::make_pos(fx, fy, fz, cx + (int64_t)a.nx * (cy + (int64_t)a.ny * cz));
    a.vel4[p] = V;
    if (BONDS || a.variant != LBMD_VARIANT_C) a.fc4[p] = P::make4(Fx, Fy, Fz, T(0));
    hand_over(a, p, R, c, Fx, Fy, Fz);
}

// One MD step, coupling force from the half-step velocity (integrator
// HALF_STEP): first half-kick with the previous step's F (kept in fc4) and
// the conservative force, drift, then F = -zeta (v_half - u(R')) + F_rand at
// the new position R', second half-kick (here without conservative forces,
// in the bond / pair kernel otherwise), transfer around R'.
template <typename T, bool BONDS>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 3) couple_half_kernel(PArgs<T> a) {
    using P = Prec<T>;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const typename P::real4 R = a.pos4[p];
    typename P::real4 V = a.vel4[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.fd_nx, a.fd_ny);
    const T hm = a.half_dt * V.w;  // V.w = 1 / mass
    typename P::real4 G = a.fc4[p];
    if (BONDS) {
        const typename P::real4 Fc = a.fcons4[p];
        G.x += Fc.x;
        G.y += Fc.y;
        G.z += Fc.z;
    }
    V.x = fma(hm, G.x, V.x);
    V.y = fma(hm, G.y, V.y);
    V.z = fma(hm, G.z, V.z);
    T fx = R.x, fy = R.y, fz = R.z;
    CellXYZ cn = c;
    advance(fx, cn.x, a.dt, V.x, a.nx);
    advance(fy, cn.y, a.dt, V.y, a.ny);
    advance(fz, cn.z, a.dt, V.z, a.nz);
    const typename P::real4 Rn = P::make_pos(fx, fy, fz, cn.x + (int64_t)a.nx * (cn.y + (int64_t)a.ny * cn.z));
    if (BONDS) check_list_skin(a, p, cn, fx, fy, fz);
    T ux, uy, uz, Fx, Fy, Fz;
    interp_u(a, cn, fx, fy, fz, ux, uy, uz);
    coupling_force(a, p, V, ux, uy, uz, Fx, Fy, Fz);
    if (!BONDS) {
        V.x = fma(hm, Fx, V.x);
        V.y = fma(hm, Fy, V.y);
        V.z = fma(hm, Fz, V.z);
    }
    a.pos4[p] = Rn;
    a.vel4[p] = V;
    a.fc4[p] = P::make4(Fx, Fy, Fz, T(0));
    hand_over(a, p, Rn, cn, Fx, Fy, Fz);
}


// Variants A and B, atomic-free: one warp per node row (y, z), four rows per block,
// rows in reverse order (the couple kernel touched the high rows last).  The
// row's nodes get transfers only from particles in the four cell rows
// (y - oy, z - oz), oy, oz in {0, 1}; with the particles bucketed by cell
// row, the warp reads those buckets and adds each particle's two
// contributions to this row (nodes x and x + 1, weight delta_k as in
// Eq. (5)) as fixed-point integers in shared memory, one entry per active
// node of the row; then it updates the row's compact records with plain
// loads and stores (no other warp writes them).  A contribution to an inactive node goes with atomics to the
// node field (B) or J_acc (A).  Particles that left their bucket's row are
// skipped here and spread by migrant_spread_kernel.
constexpr int GATHER_WARPS = 4;  // warps per block (fewer for very long rows)

// Shared-memory sums of the row gather: 3 per active node (odd stride, so
// the lanes' atomics spread over the banks), cleared with 16-byte stores; the
// per-warp area has room for 3 nx + 4 sums.
template <typename fix>
__host__ __device__ constexpr size_t acc_words(int nx) {
    return ((size_t)3 * nx + 4 + (16 / sizeof(fix)) - 1) / (16 / sizeof(fix)) * (16 / sizeof(fix));
}
template <typename fix>
__device__ __forceinline__ void acc_clear(fix *acc, int cnt, int lane) {
    constexpr int per = 16 / sizeof(fix);
    const int n4 = (3 * cnt + per - 1) / per;
    int4 *a4 = reinterpret_cast<int4 *>(acc);
    for (int k = lane; k < n4; k += 32) a4[k] = make_int4(0, 0, 0, 0);
}

// bytes of the active-word area of one block (rounded to 16)
__host__ __device__ inline size_t gather_occ_bytes(int warps, int W) {
    return ((size_t)warps * W * sizeof(uint2) + 15) & ~(size_t)15;
}

template <typename T>
__global__ void __launch_bounds__(32 * GATHER_WARPS) spread_rows_kernel(PArgs<T> a, int n_rows) {
    using P = Prec<T>;
    using fix = typename P::fix;
    using N4 = typename P::node4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = a.occ_words;
    // per warp: the row's active words (slots relative to the row's first),
    // then the sums of the active nodes
    uint2 *occ = reinterpret_cast<uint2 *>(smem_raw) + (size_t)warp * W;
    fix *acc = reinterpret_cast<fix *>(smem_raw + gather_occ_bytes(warps, W)) + (size_t)warp * acc_words<fix>(a.nx);
    const int g = blockIdx.x * warps + warp;
    if (g >= n_rows) return;
    const int nrow = n_rows - 1 - g;
    const int z = (int)fdiv((uint32_t)nrow, a.fd_ny), y = nrow - z * a.ny;
    // the four cell rows (y - oy, z - oz), q = oy + 2 oz, as one run of
    // total = e[4] particle entries: entry t belongs to row q with
    // e[q] <= t < e[q + 1], at slot lo[q] + t - e[q]
    const int ym = y == 0 ? a.ny - 1 : y - 1, zm = z == 0 ? a.nz - 1 : z - 1;
    const int c0 = y + a.ny * z, c1 = ym + a.ny * z, c2 = y + a.ny * zm, c3 = ym + a.ny * zm;
    const int lo0 = a.row_start[c0], lo1 = a.row_start[c1], lo2 = a.row_start[c2], lo3 = a.row_start[c3];
    const int e1 = a.row_start[c0 + 1] - lo0;
    const int e2 = e1 + a.row_start[c1 + 1] - lo1;
    const int e3 = e2 + a.row_start[c2 + 1] - lo2;
    const int total = e3 + a.row_start[c3 + 1] - lo3;
    const uint2 *wrow = a.occw + (size_t)nrow * W;
    const int base = (int)wrow[0].y;
    for (int w = lane; w < W; w += 32) {
        uint2 v = wrow[w];
        v.y -= (uint32_t)base;
        occ[w] = v;
    }
    const uint2 last = wrow[W - 1];
    const int cnt = (int)last.y - base + __popc(last.x);
    acc_clear(acc, cnt, lane);
    __syncwarp();
    N4 *rowp = a.inactive_acc + (size_t)a.nx * nrow;
    // entries in passes of 64, two per lane, both loaded before either is used
    for (int t0 = 0; t0 < total; t0 += 64) {
        typename P::real4 Rv[2], Fv[2];
        int crow[2];
        bool oyv[2], ozv[2], live[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = t0 + 32 * h + lane;
            live[h] = t < total;
            const bool b1 = t >= e1, b2 = t >= e2, b3 = t >= e3;
            const int slot0 = b3 ? lo3 - e3 : b2 ? lo2 - e2 : b1 ? lo1 - e1 : lo0;
            crow[h] = b3 ? c3 : b2 ? c2 : b1 ? c1 : c0;
            oyv[h] = b1 != b2 || b3;  // q = 1 or 3
            ozv[h] = b2;              // q = 2 or 3
            if (live[h]) {
                Rv[h] = a.old4[slot0 + t];
                Fv[h] = a.fc4[slot0 + t];
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!live[h]) continue;
            const typename P::real4 R = Rv[h], F = Fv[h];
            // cell x within the bucket's row; anything else is a migrant
            const int cx = (int)((uint32_t)P::cell_of(R) - (uint32_t)crow[h] * (uint32_t)a.nx);
            if ((uint32_t)cx >= (uint32_t)a.nx) continue;
            const int x1 = cx + 1 == a.nx ? 0 : cx + 1;
            const T wx[2] = {T(1) - R.x, R.x};
            const T wy = oyv[h] ? R.y : T(1) - R.y;
            const T wz = ozv[h] ? R.z : T(1) - R.z;
            const T sx = F.x * a.neg_scale_dt, sy = F.y * a.neg_scale_dt, sz = F.z * a.neg_scale_dt;
#pragma unroll
            for (int ox = 0; ox < 2; ++ox) {
                const T d = wx[ox] * wy * wz;  // the corner weight delta_k of Eq. (5)
                const int xn = ox ? x1 : cx;
                const fix vx = P::to_fix_neg(d, sx), vy = P::to_fix_neg(d, sy), vz = P::to_fix_neg(d, sz);
                const int sl = active_slot(occ[xn >> 5], xn);
                if (sl >= 0) {
                    fix *ak = acc + 3 * sl;
                    fix_add(ak + 0, vx);
                    fix_add(ak + 1, vy);
                    fix_add(ak + 2, vz);
                } else {
                    P::add_transfer(&rowp[xn], vx, vy, vz);
                }
            }
        }
    }
    __syncwarp();
    // write-back in passes of 128 nodes, the four records loaded together
    N4 *crec = a.cact_acc + base;
    for (int k0 = 0; k0 < cnt; k0 += 128) {
        N4 rec[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int k = k0 + 32 * h + lane;
            if (k < cnt) rec[h] = crec[k];
        }
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int k = k0 + 32 * h + lane;
            if (k >= cnt) continue;
            const fix dx = acc[3 * k], dy = acc[3 * k + 1], dz = acc[3 * k + 2];
            if (dx == 0 && dy == 0 && dz == 0) continue;
            P::add_transfer_reg(rec[h], dx, dy, dz);
            crec[k] = rec[h];
        }
    }
}

// Variant B: the migrants of this MD step, spread with atomics once the row
// gather is done (spread_particle_atomic, particle_step.cuh).  With `all`,
// every particle is spread this way and the row gather does not run
// (LBMD_SPREAD_ATOMIC).
template <typename T>
__global__ void __launch_bounds__(256) migrant_spread_kernel(PArgs<T> a, int all) {
    using P = Prec<T>;
    const int par = a.mig_par;
    const int n = all ? (int)a.np : a.migrant_count[par];
    // the other list serves the next MD step: empty it now (nobody uses it
    // during this one)
    if (blockIdx.x == 0 && threadIdx.x == 0) a.migrant_count[par ^ 1] = 0;
    const int32_t *list = a.migrant_slot + (int64_t)par * a.np_cap;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        spread_particle_atomic(a, all ? (int64_t)t : (int64_t)list[t]);
    }
}

template <typename T>
__device__ __forceinline__ T quiet_nan();
template <>
__device__ __forceinline__ float quiet_nan<float>() { return __int_as_float(0x7fc00000); }
template <>
__device__ __forceinline__ double quiet_nan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }

// Bond force on a particle from a partner at minimum-image separation d
// (partner minus particle), |d|^2 = r2: g d with
//   harmonic U = (k/2)(r - r0)^2               g = k (r - r0) / r   (0 at r = 0)
//   FENE     U = -(k/2) R0^2 ln(1 - (r/R0)^2)  g = k / (1 - (r/R0)^2), R0 = r0
// (Kremer-Grest springs, Sec. 4); a FENE bond at r >= R0 gives NaN.
template <typename T>
__device__ __forceinline__ T bond_gain(uint8_t kind, T k, T r0, T r2) {
    if (kind == LBMD_BOND_FENE) {
        const T x = r2 / (r0 * r0);
        return x < T(1) ? k / (T(1) - x) : quiet_nan<T>();
    }
    const T r = sqrt(r2);
    return r > T(0) ? k * (r - r0) / r : T(0);
}

// Minimum-image separation of the partner in slot q from a particle at
// (R, c), through the stored cell indices and offsets.
template <typename T>
__device__ __forceinline__ void bond_separation(const PArgs<T> &a, const typename Prec<T>::real4 &R, const CellXYZ &c,
                                                int64_t q, T &dx, T &dy, T &dz) {
    using P = Prec<T>;
    const typename P::real4 S = a.pos4[q];
    const CellXYZ d = cell_xyz(P::cell_of(S), a.fd_nx, a.fd_ny);
    dx = T(d.x - c.x) + (S.x - R.x);
    dy = T(d.y - c.y) + (S.y - R.y);
    dz = T(d.z - c.z) + (S.z - R.z);
    dx -= T(a.nx) * rint(dx / T(a.nx));
    dy -= T(a.ny) * rint(dy / T(a.ny));
    dz -= T(a.nz) * rint(dz / T(a.nz));
}

// Bond forces (harmonic or FENE) at the current positions (minimum image),
// summed per particle over its partners in a fixed order; with KICK, also
// the second velocity-Verlet half-kick with the stored coupling force.
template <typename T, bool KICK>
__global__ void __launch_bounds__(256) bond_kick_kernel(PArgs<T> a) {
    using P = Prec<T>;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const typename P::real4 R = a.pos4[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.fd_nx, a.fd_ny);
    const int64_t id = a.pid[p];
    T Fx = T(0), Fy = T(0), Fz = T(0);
    const int nbond = a.bond_count[id];
    for (int b = 0; b < nbond; ++b) {
        const int64_t e = id * LBMD_MAX_BONDS_PER_PARTICLE + b;
        T dx, dy, dz;
        bond_separation(a, R, c, a.slot_of[a.bond_partner[e]], dx, dy, dz);
        const T g = bond_gain(a.bond_kind[e], (T)a.bond_k[e], (T)a.bond_r0[e], dx * dx + dy * dy + dz * dz);
        Fx += g * dx;
        Fy += g * dy;
        Fz += g * dz;
    }
    a.fcons4[p] = P::make4(Fx, Fy, Fz, T(0));
    if (KICK) {
        typename P::real4 V = a.vel4[p];
        const typename P::real4 Fc = a.fc4[p];
        const T hm = a.half_dt * V.w;
        V.x = fma(hm, Fx + Fc.x, V.x);
        V.y = fma(hm, Fy + Fc.y, V.y);
        V.z = fma(hm, Fz + Fc.z, V.z);
        a.vel4[p] = V;
        // variant B, all atomics: every particle has read the nodes (couple
        // kernel), so the transfers can go in now
        if (a.kick_spreads) spread_particle_atomic(a, p);
    }
}


// Conservative forces with Lennard-Jones (Kremer-Grest monomers, Sec. 4):
// one warp per particle id i, eight per block.  The block stages the other
// particles in tiles of PairTile ids in shared memory (cell coordinates and
// offsets, decoded once per block instead of once per pair); the lanes then
// run over the tile (lane l takes ids l, l + 32, ...) and add the LJ force of
// every j within the cut-off,
//   F_i += g d,  g = -24 eps (2 t^2 - t) / r^2,  t = (sigma^2 / r^2)^3,
// d = R_j - R_i at the nearest image (cell offsets wrapped as integers, then
// the fractional offsets added: exact to the last bit of the offsets; every
// box edge is at least 2 r_cut + 2, so the nearest image is unique within
// the cut-off); lane b < n_bonds(i) adds bond b.  The lane sums are combined
// by a fixed butterfly, so the result does not depend on the slot order.
// With KICK, lane 0 also makes the second velocity-Verlet half-kick.
template <typename T>
struct PairTile {
    static constexpr int N = sizeof(T) == 4 ? 1024 : 512;  // 40 / 26 KB of shared memory
};

constexpr int PAIR_THREADS = 256;  // eight particles per block

template <typename T, bool KICK>
__global__ void __launch_bounds__(PAIR_THREADS) pair_kick_kernel(PArgs<T> a) {
    using P = Prec<T>;
    constexpr int TILE = PairTile<T>::N;
    __shared__ T s_f[3][TILE];
    __shared__ int s_c[3][TILE];
    __shared__ float4 s_abs[TILE];  // FP32 absolute positions, for the filter
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const bool live = i < a.np;
    const int64_t p = live ? a.slot_of[i] : 0;
    const typename P::real4 R = a.pos4[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.fd_nx, a.fd_ny);
    const float xi = (float)(T(c.x) + R.x), yi = (float)(T(c.y) + R.y), zi = (float)(T(c.z) + R.z);
    const float fnx = (float)a.nx, fny = (float)a.ny, fnz = (float)a.nz;
    const float inx = 1.0f / fnx, iny = 1.0f / fny, inz = 1.0f / fnz;
    T Fx = T(0), Fy = T(0), Fz = T(0);
    // Verlet lists when they hold every pair within the cut-off (no particle
    // moved more than half the skin since the build, no list overflowed in
    // this block).  Lane l takes the listed ids j = l (mod 32) in ascending
    // order: the same terms in the same order as the all-pairs loop below,
    // so both give the same bits.
    int use_all = a.nb_list == nullptr || *a.nb_invalid != 0;
    if (!use_all && live && a.nb_count[i] < 0) use_all = 1;
    use_all = __syncthreads_or(use_all);
    if (!use_all && live) {
        // the lanes evaluate 32 listed pairs at a time; each term then goes,
        // in list (= id) order, to the lane that owns its id (j mod 32)
        const int cnt = a.nb_count[i];
        const int32_t *L = a.nb_list + i * LBMD_NB_MAX;
        for (int e0 = 0; e0 < cnt; e0 += 32) {
            int32_t j = -1;
            T g = T(0), dx = T(0), dy = T(0), dz = T(0);
            if (e0 + lane < cnt) {
                j = L[e0 + lane];
                const typename P::real4 S = a.pos4[a.slot_of[j]];
                const CellXYZ d = cell_xyz(P::cell_of(S), a.fd_nx, a.fd_ny);
                dx = T(nearest_image(d.x - c.x, a.nx)) + (S.x - R.x);
                dy = T(nearest_image(d.y - c.y, a.ny)) + (S.y - R.y);
                dz = T(nearest_image(d.z - c.z, a.nz)) + (S.z - R.z);
                const T r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < a.lj_rc2) {  // beyond the cut-off: g = 0 adds nothing
                    const T s = a.lj_sig2 / r2;
                    const T t = s * s * s;
                    g = -a.lj_eps24 * (T(2) * t * t - t) / r2;
                }
            }
            const int m = cnt - e0 < 32 ? cnt - e0 : 32;
            for (int k = 0; k < m; ++k) {
                const int32_t jk = __shfl_sync(0xffffffffu, j, k);
                const T gk = __shfl_sync(0xffffffffu, g, k);
                const T xk = __shfl_sync(0xffffffffu, dx, k);
                const T yk = __shfl_sync(0xffffffffu, dy, k);
                const T zk = __shfl_sync(0xffffffffu, dz, k);
                if ((jk & 31) == lane) {
                    Fx += gk * xk;
                    Fy += gk * yk;
                    Fz += gk * zk;
                }
            }
        }
    }
    for (int64_t j0 = 0; use_all && j0 < a.np; j0 += TILE) {
        const int cnt = a.np - j0 < TILE ? (int)(a.np - j0) : TILE;
        __syncthreads();  // the previous tile is consumed
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const typename P::real4 S = a.pos4[a.slot_of[j0 + k]];
            const CellXYZ d = cell_xyz(P::cell_of(S), a.fd_nx, a.fd_ny);
            s_f[0][k] = S.x;
            s_f[1][k] = S.y;
            s_f[2][k] = S.z;
            s_c[0][k] = d.x;
            s_c[1][k] = d.y;
            s_c[2][k] = d.z;
            s_abs[k] = make_float4((float)(T(d.x) + S.x), (float)(T(d.y) + S.y), (float)(T(d.z) + S.z), 0.0f);
        }
        __syncthreads();
        if (!live) continue;
        for (int k = lane; k < cnt; k += 32) {
            // filter on FP32 absolute positions: a pair whose approximate
            // distance is beyond the cut-off plus the rounding margin is
            // beyond the cut-off (the exact test below would reject it too)
            const float4 A = s_abs[k];
            float ex = A.x - xi, ey = A.y - yi, ez = A.z - zi;
            ex -= fnx * rintf(ex * inx);
            ey -= fny * rintf(ey * iny);
            ez -= fnz * rintf(ez * inz);
            if (ex * ex + ey * ey + ez * ez >= a.lj_filter2) continue;
            const int ix = nearest_image(s_c[0][k] - c.x, a.nx);
            const int iy = nearest_image(s_c[1][k] - c.y, a.ny);
            const int iz = nearest_image(s_c[2][k] - c.z, a.nz);
            const T dx = T(ix) + (s_f[0][k] - R.x);
            const T dy = T(iy) + (s_f[1][k] - R.y);
            const T dz = T(iz) + (s_f[2][k] - R.z);
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (j0 + k != i && r2 < a.lj_rc2) {
                const T s = a.lj_sig2 / r2;
                const T t = s * s * s;
                const T g = -a.lj_eps24 * (T(2) * t * t - t) / r2;
                Fx += g * dx;
                Fy += g * dy;
                Fz += g * dz;
            }
        }
    }
    if (!live) return;  // whole warps, after the block's last barrier
    if (lane < a.bond_count[i]) {
        const int64_t e = i * LBMD_MAX_BONDS_PER_PARTICLE + lane;
        T dx, dy, dz;
        bond_separation(a, R, c, a.slot_of[a.bond_partner[e]], dx, dy, dz);
        const T g = bond_gain(a.bond_kind[e], (T)a.bond_k[e], (T)a.bond_r0[e], dx * dx + dy * dy + dz * dz);
        Fx += g * dx;
        Fy += g * dy;
        Fz += g * dz;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Fx += __shfl_xor_sync(0xffffffffu, Fx, off);
        Fy += __shfl_xor_sync(0xffffffffu, Fy, off);
        Fz += __shfl_xor_sync(0xffffffffu, Fz, off);
    }
    // variant B, all atomics: the couple kernel is done, so every particle
    // has read the nodes; lanes 0..7 hand over the 8 corner transfers
    if (KICK && a.kick_spreads && lane < 8) spread_corner_atomic(a, p, lane);
    if (lane != 0) return;
    a.fcons4[p] = P::make4(Fx, Fy, Fz, T(0));
    if (KICK) {
        typename P::real4 V = a.vel4[p];
        const typename P::real4 Fc = a.fc4[p];
        const T hm = a.half_dt * V.w;
        V.x = fma(hm, Fx + Fc.x, V.x);
        V.y = fma(hm, Fy + Fc.y, V.y);
        V.z = fma(hm, Fz + Fc.z, V.z);
        a.vel4[p] = V;
    }
}

// LJ Verlet lists, rebuilt after each re-ordering (rebuilding only voided
// lists made the all-pairs fallback frequent: the skin is then spent over
// several LB steps): one warp per slot q (particle i = pid[q]) builds i's
// list: the lanes run over the particles of the row buckets
// within ceil(r_list) rows in y and z (each distinct row once; the buckets'
// slot ranges are concatenated and shared out 32 at a time), keep the ids
// j != i closer than r_list = r_cut + skin, and write them in ascending order
// (each lane ranks its entries by counting the smaller ids).  A particle with
// more than LBMD_NB_MAX candidates gets count -1 (its block then uses all
// pairs).  The positions at the build are kept per id.
constexpr int NB_WARPS = 8;

template <typename T>
__global__ void __launch_bounds__(32 * NB_WARPS) nb_build_kernel(PArgs<T> a, T rlist2, int reach) {
    using P = Prec<T>;
    __shared__ int32_t s_ids[NB_WARPS][LBMD_NB_MAX];
    __shared__ int s_cnt[NB_WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * NB_WARPS + warp;
    if (q >= a.np) return;  // whole warps; no block barrier below
    const int32_t i = a.pid[q];
    const typename P::real4 R = a.pos4[q];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.fd_nx, a.fd_ny);
    if (lane == 0) {
        s_cnt[warp] = 0;
        const_cast<typename P::real4 *>(a.nb_ref4)[i] = R;
    }
    __syncwarp();
    const int ny_rows = 2 * reach + 1 < a.ny ? 2 * reach + 1 : a.ny;
    const int nz_rows = 2 * reach + 1 < a.nz ? 2 * reach + 1 : a.nz;
    const int y0 = 2 * reach + 1 < a.ny ? c.y - reach + a.ny : 0;
    const int z0 = 2 * reach + 1 < a.nz ? c.z - reach + a.nz : 0;
    const int nrows = ny_rows * nz_rows;
    for (int r0 = 0; r0 < nrows; r0 += 32) {
        // lane r: the slot range of candidate row r0 + r, and its offset in
        // the concatenation of the ranges
        int lo = 0, cnt = 0;
        if (r0 + lane < nrows) {
            const int ky = (r0 + lane) % ny_rows, kz = (r0 + lane) / ny_rows;
            const int row = (y0 + ky) % a.ny + a.ny * ((z0 + kz) % a.nz);
            lo = a.row_start[row];
            cnt = a.row_start[row + 1] - lo;
        }
        int incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        const int excl = incl - cnt;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            // the last row whose range starts at or before t
            int r = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int v = __shfl_sync(0xffffffffu, excl, r + step);
                if (v <= t) r += step;
            }
            const int lo_r = __shfl_sync(0xffffffffu, lo, r), ex_r = __shfl_sync(0xffffffffu, excl, r);
            if (t >= total) continue;
            const int sl = lo_r + (t - ex_r);
            const int32_t j = a.pid[sl];
            if (j == i) continue;
            const typename P::real4 S = a.pos4[sl];
            const CellXYZ d = cell_xyz(P::cell_of(S), a.fd_nx, a.fd_ny);
            const T dx = T(nearest_image(d.x - c.x, a.nx)) + (S.x - R.x);
            const T dy = T(nearest_image(d.y - c.y, a.ny)) + (S.y - R.y);
            const T dz = T(nearest_image(d.z - c.z, a.nz)) + (S.z - R.z);
            if (dx * dx + dy * dy + dz * dz < rlist2) {
                const int k = atomicAdd(&s_cnt[warp], 1);
                if (k < LBMD_NB_MAX) s_ids[warp][k] = j;
            }
        }
    }
    __syncwarp();
    const int cnt = s_cnt[warp];
    if (cnt > LBMD_NB_MAX) {
        if (lane == 0) const_cast<int32_t *>(a.nb_count)[i] = -1;
        return;
    }
    int32_t *L = const_cast<int32_t *>(a.nb_list) + (int64_t)i * LBMD_NB_MAX;
    for (int k = lane; k < cnt; k += 32) {
        const int32_t j = s_ids[warp][k];
        int rank = 0;
        for (int m = 0; m < cnt; ++m) rank += s_ids[warp][m] < j ? 1 : 0;
        L[rank] = j;
    }
    if (lane == 0) const_cast<int32_t *>(a.nb_count)[i] = cnt;
}

// after a build (or none): the lists hold every pair within the cut-off
__global__ void nb_validate_kernel(int32_t *invalid) { *invalid = 0; }

// ---------------------------------------------------------------------------
// Re-ordering by lattice row.
// ---------------------------------------------------------------------------
// Every particle's rank within its cell row and, with ccw, its cell marked in
// the row's occupancy words.  The particles come mostly in row order (the
// order of the last re-ordering), so the valid lanes of a warp form runs of
// equal rows (and of equal occupancy words): each run takes its ranks with one
// atomic on the row's count, and ORs its cells into a word with one atomic.
// The order within a row is free: every later sum is order-independent.
template <typename T>
__global__ void __launch_bounds__(256)
    sort_count_kernel(const typename Prec<T>::real4 *pos4, int64_t np, FastDiv fnx, int32_t *row_count, int32_t *rank,
                      uint32_t *ccw, int W) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned act = __ballot_sync(0xffffffffu, p < np);  // a prefix of the warp's lanes
    if (p >= np) return;
    const int lane = (int)(threadIdx.x & 31), nvalid = __popc(act);
    const unsigned upto = 0xffffffffu >> (31 - lane);  // lanes 0..lane
    const uint32_t cell = (uint32_t)Prec<T>::cell_of(pos4[p]);
    const uint32_t row = fdiv(cell, fnx);
    // runs of equal rows: the run's first lane takes the ranks
    const uint32_t row_prev = __shfl_up_sync(act, row, 1);
    const unsigned heads = __ballot_sync(act, lane == 0 || row_prev != row);
    const int head = 31 - __clz((int)(heads & upto));
    const unsigned after = heads & ~upto;
    const int next = after ? __ffs((int)after) - 1 : nvalid;
    int base = 0;
    if (lane == head) base = atomicAdd(&row_count[row], next - head);
    base = __shfl_sync(act, base, head);
    rank[p] = base + (lane - head);
    if (ccw) {
        const uint32_t cx = cell - row * fnx.d;
        const unsigned long long key = (unsigned long long)row * (unsigned)W + (cx >> 5);
        const unsigned long long key_prev = __shfl_up_sync(act, key, 1);
        const unsigned kheads = __ballot_sync(act, lane == 0 || key_prev != key);
        const unsigned kafter = kheads & ~upto;
        const int knext = kafter ? __ffs((int)kafter) - 1 : nvalid;
        // the run's cells ORed towards its first lane (segmented, log steps)
        uint32_t bits = 1u << (cx & 31);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_down_sync(act, bits, off);
            if (lane + off < knext) bits |= o;
        }
        if (kheads & (1u << lane)) atomicOr(&ccw[key], bits);
    }
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

// Move every particle to row_start[row] + rank within the row, with its
// conservative force (if any) and its last coupling force (integrator
// HALF_STEP, where it carries over to the next MD step).
template <typename T>
__global__ void __launch_bounds__(256)
    sort_scatter_kernel(const typename Prec<T>::real4 *pos_in, const typename Prec<T>::real4 *vel_in,
                        const typename Prec<T>::real4 *fcons_in, const typename Prec<T>::real4 *fc_in,
                        const int32_t *pid_in, typename Prec<T>::real4 *pos_out, typename Prec<T>::real4 *vel_out,
                        typename Prec<T>::real4 *fcons_out, typename Prec<T>::real4 *fc_out, int32_t *pid_out,
                        int32_t *slot_of, int32_t *slot_row, const int32_t *row_start, const int32_t *rank, int64_t np,
                        FastDiv fnx, int bonds, int carry_fc) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const typename Prec<T>::real4 R = pos_in[p];
    const uint32_t row = fdiv((uint32_t)Prec<T>::cell_of(R), fnx);
    const int32_t dst = row_start[row] + rank[p];
    slot_row[dst] = (int32_t)row;
    pos_out[dst] = R;
    vel_out[dst] = vel_in[p];
    if (bonds) fcons_out[dst] = fcons_in[p];
    if (carry_fc) fc_out[dst] = fc_in[p];
    const int32_t id = pid_in[p];
    pid_out[dst] = id;
    slot_of[id] = dst;
}

// ---------------------------------------------------------------------------
// Active nodes (variants A and B), rebuilt after each re-ordering.
// ---------------------------------------------------------------------------
// Level 0: node x of row (y, z) is active when a particle's cell has it as a
// corner, i.e. when cell x or x - 1 (periodic) of one of the four cell rows
// (y - oy, z - oz), oy, oz in {0, 1}, holds a particle.  A group of L lanes
// (L = min(32, W rounded up to a power of two)) builds one row's words from
// the cell-occupancy words ccw, with the in-row slot of each word's first
// active node (a scan over the group), and the row's count.
__global__ void __launch_bounds__(256)
    active_rows_kernel(const uint32_t *ccw, int nx, FastDiv fny, int nz, int W, int L, uint2 *occw, int32_t *row_count,
                       int n_rows) {
    const int lane = (int)(threadIdx.x & 31);
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nrow = gwarp * (32 / L) + lane / L, sub = lane % L;
    const bool valid = nrow < n_rows;
    const int ny = (int)fny.d;
    int cr[4] = {0, 0, 0, 0};
    if (valid) {
        const int z = (int)fdiv((uint32_t)nrow, fny), y = nrow - z * ny;
        const int ym = y == 0 ? ny - 1 : y - 1, zm = z == 0 ? nz - 1 : z - 1;
        cr[0] = y + ny * z;
        cr[1] = ym + ny * z;
        cr[2] = y + ny * zm;
        cr[3] = ym + ny * zm;
    }
    const int last = nx - 1;
    const uint32_t tail_mask = (nx & 31) ? ((1u << (nx & 31)) - 1u) : 0xffffffffu;
    int carry = 0;
    for (int w0 = 0; w0 < W; w0 += L) {  // uniform over the warp
        const int w = w0 + sub;
        uint32_t a = 0u;
        if (valid && w < W) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t *cw = ccw + (size_t)cr[c] * W;
                const uint32_t b = cw[w];
                // cell x - 1 of bit x: the previous word's top bit, or (w = 0)
                // the periodic neighbour x = nx - 1
                const uint32_t in = w > 0 ? (cw[w - 1] >> 31) : ((cw[last >> 5] >> (last & 31)) & 1u);
                a |= b | (b << 1) | in;
            }
            if (w == W - 1) a &= tail_mask;
        }
        const int cnt = __popc(a);
        int incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, off, L);
            if (off < L && sub >= off) incl += v;
        }
        if (valid && w < W) occw[(size_t)nrow * W + w] = make_uint2(a, (uint32_t)(carry + incl - cnt));
        carry += __shfl_sync(0xffffffffu, incl, L - 1, L);
    }
    if (valid && sub == 0) row_count[nrow] = carry;
}

// Level 2 (after sort_chunk_scan_kernel turned the row counts into offsets
// within chunks of 1024 rows): the first slot of every row added to the
// in-row slots of its words, one word per thread; block (c, s) takes slice s
// of chunk c's words.
constexpr int FINALIZE_SLICES = 4;
__global__ void __launch_bounds__(1024) active_finalize_kernel(const int32_t *row_offset, const int32_t *chunk_total,
                                                               int64_t n_rows, uint2 *occw, int W, int32_t *arow) {
    int32_t before;
    const int32_t v = (int)threadIdx.x < (int)blockIdx.x ? chunk_total[threadIdx.x] : 0;
    block_exclusive_scan(v, &before);  // total of the first blockIdx.x chunks
    const int64_t r0 = (int64_t)blockIdx.x * 1024, r1 = r0 + 1024 < n_rows ? r0 + 1024 : n_rows;
    const int64_t w_end = r1 * W;
    for (int64_t i = r0 * W + (int64_t)blockIdx.y * 1024 + threadIdx.x; i < w_end; i += FINALIZE_SLICES * 1024) {
        const int64_t row = i / W;
        const uint32_t b = (uint32_t)(before + row_offset[row]);
        uint2 wd = occw[i];
        wd.y += b;
        occw[i] = wd;
        if (i == row * W) arow[row] = (int32_t)b;  // the row's first compact slot
        if (row == n_rows - 1 && i == w_end - 1) arow[n_rows] = (int32_t)(wd.y + __popc(wd.x));  // closes the table
    }
}

// Node field entries of the active nodes brought up to date from their
// compact records (for the observables and the host accessors).
template <typename T>
__global__ void __launch_bounds__(256) active_sync_kernel(const uint2 *occw, const typename Prec<T>::node4 *cact,
                                                          typename Prec<T>::node4 *node, int64_t N, int nx, int W) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const int64_t row = r / nx;
    const int x = (int)(r - row * nx);
    const int sl = active_slot(occw[(size_t)row * W + (x >> 5)], x);
    if (sl >= 0) node[r] = cact[sl];
}

// shared memory of the row gather with `warps` warps per block: the rows'
// active words and the sums of up to nx active nodes per row
template <typename T>
static size_t gather_smem_bytes(const lbmd_ctx *ctx, int warps) {
    using fix = typename Prec<T>::fix;
    return gather_occ_bytes(warps, active_words(ctx->p.nx)) + (size_t)warps * acc_words<fix>(ctx->p.nx) * sizeof(fix);
}

// The row gather's shared memory grows with nx: as many warps per block (at
// most GATHER_WARPS) as fit in 200 KB, and the opt-in above the default
// 48 KB per block.
template <typename T>
static cudaError_t setup_t(lbmd_ctx *ctx) {
    int warps = GATHER_WARPS;
    while (warps > 1 && gather_smem_bytes<T>(ctx, warps) > (size_t)200 * 1024) --warps;
    const size_t smem = gather_smem_bytes<T>(ctx, warps);
    if (smem > (size_t)200 * 1024) return cudaErrorInvalidValue;
    ctx->gather_warps = warps;
    cudaError_t e = cudaFuncSetAttribute(spread_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return md_tile_setup_kernels(ctx);
}

template <typename T>
static PArgs<T> make_pargs(lbmd_ctx *ctx, int substep) {
    using P = Prec<T>;
    const int b = ctx->pcur;
    PArgs<T> a;
    a.pos4 = static_cast<typename P::real4 *>(pos_now(ctx));
    a.vel4 = static_cast<typename P::real4 *>(vel_now(ctx));
    a.fcons4 = static_cast<typename P::real4 *>(ctx->fcons4[b]);
    a.pid = ctx->pid[b];
    a.slot_of = ctx->slot_of;
    a.fc4 = static_cast<typename P::real4 *>(ctx->fc4[b]);
    a.old4 = static_cast<typename P::real4 *>(ctx->old4);
    a.node = static_cast<typename P::node4 *>(ctx->node);
    a.jacc = static_cast<typename P::node4 *>(ctx->jacc);
    a.bond_count = ctx->bond_count;
    a.bond_partner = ctx->bond_partner;
    a.bond_k = ctx->bond_k;
    a.bond_r0 = ctx->bond_r0;
    a.bond_kind = ctx->bond_kind;
    a.lj_eps24 = (T)(24.0 * ctx->lj_eps);
    a.lj_sig2 = (T)(ctx->lj_sigma * ctx->lj_sigma);
    a.lj_rc2 = (T)(ctx->lj_rc * ctx->lj_rc);
    {
        // |error| of an FP32 absolute coordinate <= max edge * 2^-24, of a
        // distance <= sqrt(3) * 2 of that (plus the float arithmetic); the
        // margin is a generous multiple of it
        const double edge = std::max(ctx->p.nx, std::max(ctx->p.ny, ctx->p.nz));
        const double margin = edge * std::ldexp(1.0, -18) + 1e-6;
        a.lj_filter2 = (float)((ctx->lj_rc + margin) * (ctx->lj_rc + margin));
    }
    const bool lists = ctx->lj_rc > 0.0 && ctx->nb_list;
    a.nb_list = lists ? ctx->nb_list : nullptr;
    a.nb_count = lists ? ctx->nb_count : nullptr;
    a.nb_invalid = lists ? ctx->nb_invalid : nullptr;
    a.nb_ref4 = lists ? static_cast<const typename P::real4 *>(ctx->nb_ref4) : nullptr;
    a.nb_half_skin2 = (T)(0.25 * LBMD_NB_SKIN * LBMD_NB_SKIN);
    a.nx = ctx->p.nx;
    a.ny = ctx->p.ny;
    a.nz = ctx->p.nz;
    a.fd_nx = make_fastdiv((uint32_t)ctx->p.nx);
    a.fd_ny = make_fastdiv((uint32_t)ctx->p.ny);
    a.np = ctx->np;
    a.zeta = (T)ctx->p.zeta;
    a.dt = (T)ctx->dt;
    a.half_dt = (T)(0.5 * ctx->dt);
    a.amp = (T)sqrt(2.0 * ctx->p.zeta * ctx->p.kT / ctx->dt);
    a.neg_scale_dt = (T)ctx->dt * -(T)ctx->fix.scale;
    a.fis = (T)ctx->fix.inv_scale;
    a.key0 = (uint32_t)(ctx->p.seed & 0xffffffffu);
    a.key1 = (uint32_t)(ctx->p.seed >> 32);
    a.lb_step = ctx->d_lb_step;
    a.n_sub = ctx->p.n_sub;
    a.substep = substep;
    a.mig_par = (int)((ctx->lb_step * ctx->p.n_sub + substep) & 1);
    a.noisy = ctx->p.kT > 0.0 ? 1 : 0;
    a.gauss = ctx->p.noise == LBMD_NOISE_GAUSS ? 1 : 0;
    a.variant = ctx->p.variant;
    a.row_start = ctx->row_start;
    a.slot_row = ctx->slot_row;
    a.migrant_slot = ctx->migrant_slot;
    a.migrant_count = ctx->migrant_count;
    a.np_cap = ctx->p.max_particles > 0 ? ctx->p.max_particles : 1;
    a.b_atomic = 0;
    a.kick_spreads = 0;
    a.occw = active_words_now(ctx);
    a.cact = static_cast<typename P::node4 *>(active_records_now(ctx));
    a.cact_acc = static_cast<typename P::node4 *>(active_records_acc(ctx));
    a.interp_compact = ctx->p.variant == LBMD_VARIANT_B || a_copy(ctx) ? 1 : 0;
    a.inactive_acc = ctx->p.variant == LBMD_VARIANT_A ? a.jacc : a.node;
    a.occ_words = active_words(ctx->p.nx);
    return a;
}

template <typename T>
static cudaError_t md_substep_t(lbmd_ctx *ctx, int substep) {
    if (ctx->np == 0) return cudaSuccess;
    PArgs<T> a = make_pargs<T>(ctx, substep);
    const unsigned blocks = (unsigned)((ctx->np + 255) / 256);
    const bool cons = has_cons(ctx);
    const bool B = compact_nodes(ctx);  // variants A and B: spreading into the compact records
    const bool atomic = B && (ctx->p.spread == LBMD_SPREAD_ATOMIC ||
                              (ctx->p.spread == LBMD_SPREAD_AUTO &&
                               ctx->np < (int64_t)LBMD_SPREAD_ATOMIC_PER_ROW * ctx->p.ny * ctx->p.nz));
    a.b_atomic = atomic ? 1 : 0;
    a.kick_spreads = atomic && cons ? 1 : 0;
    // the tiled step only on request: at the benchmark density it measured
    // slower than the separate particle pass and row gather
    const bool tiles = !atomic && md_tile_supported(ctx) && ctx->p.spread == LBMD_SPREAD_TILES;
    cudaError_t e;
    if (tiles) {
        // the whole MD step in one pass over tiles of rows (new positions,
        // velocities and records into the other buffers) and a short
        // follow-up (transfers across the periodic wrap, listed particles)
        if ((e = md_tile_step<T>(ctx, a)) != cudaSuccess) return e;
        ctx->pv ^= 1;
        ctx->rec ^= 1;
        return cudaSuccess;
    }
    if (ctx->p.integrator == LBMD_INTEGRATOR_HALF_STEP) {
        if (cons)
            couple_half_kernel<T, true><<<blocks, 256, 0, ctx->stream>>>(a);
        else
            couple_half_kernel<T, false><<<blocks, 256, 0, ctx->stream>>>(a);
    } else if (cons) {
        couple_kernel<T, true><<<blocks, 256, 0, ctx->stream>>>(a);
    } else {
        couple_kernel<T, false><<<blocks, 256, 0, ctx->stream>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (cons) {
        if (ctx->lj_rc > 0.0)
            pair_kick_kernel<T, true><<<(unsigned)((ctx->np + 7) / 8), PAIR_THREADS, 0, ctx->stream>>>(a);
        else
            bond_kick_kernel<T, true><<<blocks, 256, 0, ctx->stream>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (ctx->p.variant == LBMD_VARIANT_C) return launch_forcing_update(ctx);
    if (B) {
        if (atomic && cons) {
            // spread by the bond / pair kernel above
        } else if (atomic) {
            const unsigned sb = (unsigned)std::min<int64_t>(ctx->sm_count, (ctx->np + 255) / 256);
            migrant_spread_kernel<T><<<sb, 256, 0, ctx->stream>>>(a, 1);
        } else {
            const int rows = (int)((int64_t)ctx->p.ny * ctx->p.nz);
            const int gw = ctx->gather_warps;
            const unsigned gblocks = (unsigned)((rows + gw - 1) / gw);
            spread_rows_kernel<T><<<gblocks, 32 * gw, gather_smem_bytes<T>(ctx, gw), ctx->stream>>>(a, rows);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            migrant_spread_kernel<T><<<ctx->sm_count, 256, 0, ctx->stream>>>(a, 0);
        }
        e = cudaGetLastError();
    }
    return e;
}

template <typename T>
static cudaError_t bond_forces_t(lbmd_ctx *ctx) {
    if (ctx->np == 0) return cudaSuccess;
    PArgs<T> a = make_pargs<T>(ctx, 0);
    const unsigned blocks = (unsigned)((ctx->np + 255) / 256);
    if (ctx->lj_rc > 0.0)
        pair_kick_kernel<T, false><<<(unsigned)((ctx->np + 7) / 8), PAIR_THREADS, 0, ctx->stream>>>(a);
    else
        bond_kick_kernel<T, false><<<blocks, 256, 0, ctx->stream>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t sort_t(lbmd_ctx *ctx) {
    using R4 = typename Prec<T>::real4;
    const int b = ctx->pcur, o = b ^ 1;
    const int v = ctx->pv, vo = v ^ 1;  // position / velocity buffers
    const int64_t rows = (int64_t)ctx->p.ny * ctx->p.nz;
    const int W = active_words(ctx->p.nx);
    cudaError_t e = cudaMemsetAsync(ctx->row_count, 0, (size_t)rows * sizeof(int32_t), ctx->stream);
    if (e != cudaSuccess) return e;
    if (ctx->ccw && ctx->np > 0 &&
        (e = cudaMemsetAsync(ctx->ccw, 0, (size_t)rows * W * sizeof(uint32_t), ctx->stream)) != cudaSuccess)
        return e;
    if (ctx->np > 0) {
        const unsigned blocks = (unsigned)((ctx->np + 255) / 256);
        sort_count_kernel<T><<<blocks, 256, 0, ctx->stream>>>(static_cast<const R4 *>(ctx->pos4[v]), ctx->np,
                                                                make_fastdiv((uint32_t)ctx->p.nx), ctx->row_count,
                                                                ctx->sort_rank, ctx->ccw, W);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int n_chunks = (int)((rows + 1023) / 1024);
        sort_chunk_scan_kernel<<<n_chunks, 1024, 0, ctx->stream>>>(ctx->row_count, rows, ctx->chunk_total);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        sort_finalize_kernel<<<n_chunks, 1024, 0, ctx->stream>>>(ctx->row_count, ctx->chunk_total, rows,
                                                                 ctx->row_start, (int32_t)ctx->np);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        sort_scatter_kernel<T><<<blocks, 256, 0, ctx->stream>>>(
            static_cast<const R4 *>(ctx->pos4[v]), static_cast<const R4 *>(ctx->vel4[v]),
            static_cast<const R4 *>(ctx->fcons4[b]), static_cast<const R4 *>(ctx->fc4[b]), ctx->pid[b],
            static_cast<R4 *>(ctx->pos4[vo]), static_cast<R4 *>(ctx->vel4[vo]), static_cast<R4 *>(ctx->fcons4[o]),
            static_cast<R4 *>(ctx->fc4[o]), ctx->pid[o], ctx->slot_of, ctx->slot_row, ctx->row_start,
            ctx->sort_rank, ctx->np, make_fastdiv((uint32_t)ctx->p.nx), has_cons(ctx) ? 1 : 0,
            ctx->p.integrator == LBMD_INTEGRATOR_HALF_STEP ? 1 : 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    ctx->pcur = o;
    ctx->pv = vo;
    return cudaSuccess;
}

template <typename T>
static cudaError_t active_set_t(lbmd_ctx *ctx) {
    const int64_t rows = (int64_t)ctx->p.ny * ctx->p.nz;
    const int W = active_words(ctx->p.nx);
    uint2 *occw = active_words_next(ctx);  // built for the coming LB cycle
    int32_t *arow = ctx->arow[(ctx->lb_step + 1) & 1];
    if (ctx->np == 0) {
        cudaError_t e = cudaMemsetAsync(occw, 0, (size_t)rows * W * sizeof(uint2), ctx->stream);
        if (e != cudaSuccess) return e;
        return cudaMemsetAsync(arow, 0, (size_t)(rows + 1) * sizeof(int32_t), ctx->stream);
    }
    int L = 1;
    while (L < W && L < 32) L <<= 1;
    const int64_t warps = (rows + (32 / L) - 1) / (32 / L);
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    active_rows_kernel<<<blocks, 256, 0, ctx->stream>>>(ctx->ccw, ctx->p.nx, make_fastdiv((uint32_t)ctx->p.ny),
                                                        ctx->p.nz, W, L, occw, ctx->row_count, (int)rows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n_chunks = (int)((rows + 1023) / 1024);
    sort_chunk_scan_kernel<<<n_chunks, 1024, 0, ctx->stream>>>(ctx->row_count, rows, ctx->chunk_total);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    active_finalize_kernel<<<dim3(n_chunks, FINALIZE_SLICES), 1024, 0, ctx->stream>>>(ctx->row_count,
                                                                                      ctx->chunk_total, rows, occw,
                                                                                      W, arow);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t active_sync_t(lbmd_ctx *ctx) {
    using N4 = typename Prec<T>::node4;
    const unsigned blocks = (unsigned)((ctx->N + 255) / 256);
    active_sync_kernel<T><<<blocks, 256, 0, ctx->stream>>>(active_words_now(ctx),
                                                           static_cast<const N4 *>(active_records_now(ctx)),
                                                           static_cast<N4 *>(ctx->node), ctx->N, ctx->p.nx,
                                                           active_words(ctx->p.nx));
    return cudaGetLastError();
}

template <typename T>
static cudaError_t nb_build_t(lbmd_ctx *ctx) {
    if (ctx->np == 0 || !(ctx->lj_rc > 0.0) || !ctx->nb_list) return cudaSuccess;
    PArgs<T> a = make_pargs<T>(ctx, 0);
    const double rl = ctx->lj_rc + LBMD_NB_SKIN;
    nb_build_kernel<T><<<(unsigned)((ctx->np + NB_WARPS - 1) / NB_WARPS), 32 * NB_WARPS, 0, ctx->stream>>>(
        a, (T)(rl * rl), (int)std::ceil(rl));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    nb_validate_kernel<<<1, 1, 0, ctx->stream>>>(ctx->nb_invalid);
    return cudaGetLastError();
}

}  // namespace lbmd

cudaError_t launch_active_set(lbmd_ctx *ctx) {
    if (!compact_nodes(ctx)) return cudaSuccess;
    return ctx->p.precision == LBMD_FP64 ? lbmd::active_set_t<double>(ctx) : lbmd::active_set_t<float>(ctx);
}

cudaError_t launch_active_sync(lbmd_ctx *ctx) {
    if (ctx->p.variant != LBMD_VARIANT_B) return cudaSuccess;
    return ctx->p.precision == LBMD_FP64 ? lbmd::active_sync_t<double>(ctx) : lbmd::active_sync_t<float>(ctx);
}

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

cudaError_t launch_nb_build(lbmd_ctx *ctx) {
    return ctx->p.precision == LBMD_FP64 ? lbmd::nb_build_t<double>(ctx) : lbmd::nb_build_t<float>(ctx);
}

cudaError_t launch_sort_particles(lbmd_ctx *ctx) {
    return ctx->p.precision == LBMD_FP64 ? lbmd::sort_t<double>(ctx) : lbmd::sort_t<float>(ctx);
}
