// observe.cu -- FP64 reductions of the observables and the conversions
// between the device storage and the FP64 host arrays of the C ABI.
//
// Observables (mass, fluid momentum incl. pending transfers, particle
// momentum, sum of m v^2): every thread accumulates a fixed strided subset,
// each block reduces in a fixed tree order into one row of a partial-sum
// table in double precision, and a single block adds the rows in order.  The
// grid size is fixed per context, so the sums are bitwise reproducible.
//
// The FP64 pipes of this GPU issue a small fraction of the FP32 / integer
// rate, so the per-element work of the FP32 forms avoids them: the mass and
// the fluid momentum are summed in 64-bit integers (fixed point) up to the
// block totals, the particle sums in pairs of FP32 values, and FP32 values
// become doubles through their bit fields (exact, integer pipes).  Doubles
// are added only per block and in the final reduction.
#include "lbmd_ctx.h"
#include "lbmd_device.cuh"
#include "particle_core.cuh"
#include "convert.cuh"

namespace lbmd {

constexpr int RED_THREADS = 256;
constexpr int RED_COLS = 8;  // mass, pfx, pfy, pfz, ppx, ppy, ppz, sum m v^2

template <int NV>
__device__ __forceinline__ void block_reduce_store(double v[NV], double *row) {
    __shared__ double sh[NV][RED_THREADS];
#pragma unroll
    for (int c = 0; c < NV; ++c) sh[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int c = 0; c < NV; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) row[c] = sh[c][0];
    }
}

__device__ __forceinline__ double to_double(float v) { return exact_double(v); }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double cell_plus_fraction(uint32_t x, double f) { return (double)x + f; }

// Fixed-order block reduction of NV 64-bit integers: a butterfly within each
// warp, then thread 0 adds the warps' totals in warp order (integer sums are
// exact, so the order only matters for the doubles beside them).
template <int NV>
__device__ __forceinline__ void block_sum_ll(long long v[NV]) {
    __shared__ long long sh[RED_THREADS / 32][NV];
#pragma unroll
    for (int c = 0; c < NV; ++c)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], off);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) sh[threadIdx.x >> 5][c] = v[c];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            long long t = 0;
            for (int w = 0; w < RED_THREADS / 32; ++w) t += sh[w][c];
            v[c] = t;
        }
}

// ---------------------------------------------------------------------------
// Fluid sums.  FP64 records: rho and the fixed-point momentum (56 fraction
// bits) are added in doubles.  FP32 records: the momentum components are
// 32-bit fixed-point integers, added exactly in 64-bit integers; the density
// is added in 64-bit integers too, in units of 2^-u, u = 40 - e
// (e = ceil(log2 rho0)): every density of at least 2^(e - 17) is a whole
// number of units, so those sums are exact, and smaller ones lose their parts
// below one unit (2^(e - 40)).  Densities of 2^(e + 4) and more, infinite or
// NaN (an unstable fluid) go to a double sum beside it, which keeps them
// visible to the non-finite check; the integer terms stay below 2^44, so a
// block's totals fit 64 bits while it adds fewer than 2^19 nodes.
// ---------------------------------------------------------------------------
template <typename T>
struct FluidSums {
    using P = Prec<T>;
    double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    __device__ __forceinline__ void add(const typename P::node4 &n, int) {
        rho += P::rho_of(n);
        add_j(n);
    }
    __device__ __forceinline__ void add_j(const typename P::node4 &n) {
        jx += (double)P::jx_of(n);
        jy += (double)P::jy_of(n);
        jz += (double)P::jz_of(n);
    }
    __device__ __forceinline__ void store(double *row, double) {
        double v[4] = {rho, jx, jy, jz};
        block_reduce_store<4>(v, row);
    }
};
template <>
struct FluidSums<float> {
    using P = Prec<float>;
    long long q[4] = {0, 0, 0, 0};  // rho in units of 2^-u, then j in fixed-point units
    double big = 0.0;
    __device__ __forceinline__ void add(const P::node4 &n, int u) {
        const uint32_t b = __float_as_uint(P::rho_of(n));
        const int ex = (int)((b >> 23) & 0xffu);
        const int sh = ex - 150 + u;  // a normal density is m 2^(ex - 150), m < 2^24
        if (ex == 0xff || sh > 20) {
            big += (double)P::rho_of(n);
        } else if (ex != 0 && sh > -24) {
            const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
            const long long t = sh >= 0 ? (m << sh) : (m >> -sh);
            q[0] += (b >> 31) ? -t : t;
        }
        add_j(n);
    }
    __device__ __forceinline__ void add_j(const P::node4 &n) {
        q[1] += (long long)P::jx_of(n);
        q[2] += (long long)P::jy_of(n);
        q[3] += (long long)P::jz_of(n);
    }
    __device__ __forceinline__ void store(double *row, double unit) {
        double bsum = 0.0;
        if (__syncthreads_or(big != 0.0)) {  // rare: a fluid far from rho0
            double v[1] = {big};
            block_reduce_store<1>(v, row);
            __syncthreads();
            bsum = row[0];
        }
        block_sum_ll<4>(q);
        if (threadIdx.x == 0) {
            row[0] = (double)q[0] * unit + bsum;
            row[1] = (double)q[1];
            row[2] = (double)q[2];
            row[3] = (double)q[3];
        }
    }
};

// Variant B keeps the records of the active nodes in their compact array
// during a cycle: a node's current record is found through the active words
// (occw non-null), so no copy back is needed first.  Every thread issues the
// loads of U nodes before it adds any (memory-level parallelism), and the
// active-word lookups run one pass ahead of the record loads that depend on
// them, so a pass waits on one round trip to memory, not two.
template <typename T, int VARIANT>
__device__ __forceinline__ void observe_nodes(const typename Prec<T>::node4 *node, const typename Prec<T>::node4 *jacc,
                                              const uint2 *occw, const typename Prec<T>::node4 *cact, int W,
                                              FastDiv fnx, int64_t N, int mass_u, double mass_unit, double *row) {
    using P = Prec<T>;
    constexpr int U = VARIANT == LBMD_VARIANT_A ? (sizeof(T) == 8 ? 2 : 4) : (sizeof(T) == 8 ? 4 : 6);
    FluidSums<T> acc;
    const int64_t stride = (int64_t)gridDim.x * RED_THREADS;
    // active-word lookups of the pass starting at r0 (slot -1: inactive or beyond N)
    auto lookup = [&](int64_t r0, uint2 wd[U], int x[U]) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = r0 + u * stride;
            x[u] = -1;
            if (!occw || r >= N) continue;
            const uint32_t row = fdiv((uint32_t)r, fnx);
            x[u] = (int)((uint32_t)r - row * fnx.d);
            wd[u] = occw[(size_t)row * W + (x[u] >> 5)];
        }
    };
    int64_t r0 = (int64_t)blockIdx.x * RED_THREADS + threadIdx.x;
    uint2 wd[U];
    int x[U];
    lookup(r0, wd, x);
    for (; r0 < N; r0 += U * stride) {
        int sl[U];
#pragma unroll
        for (int u = 0; u < U; ++u) sl[u] = x[u] >= 0 ? active_slot(wd[u], x[u]) : -1;
        typename P::node4 n[U], J[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = r0 + u * stride;
            if (r >= N) continue;
            n[u] = sl[u] >= 0 ? cact[sl[u]] : node[r];
            if (VARIANT == LBMD_VARIANT_A) J[u] = jacc[r];
        }
        lookup(r0 + U * stride, wd, x);  // the next pass's words, in flight with this pass's records
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (r0 + u * stride >= N) continue;
            acc.add(n[u], mass_u);
            if (VARIANT == LBMD_VARIANT_A) acc.add_j(J[u]);
        }
    }
    // momenta stay in fixed-point units until the final scaling
    acc.store(row, mass_unit);
}

// ---------------------------------------------------------------------------
// Particle sums (momentum m v and m v^2).  FP64 velocities: doubles.  FP32
// velocities: every thread keeps each sum as an unevaluated pair hi + lo of
// FP32 values -- hi the running sum, lo the exact rounding errors of its
// additions (Knuth's two-sum) and of the products (FMA) -- about 44
// significant bits, on the FP32 pipes; m = 1/w is the pair of the rounded
// reciprocal and its residual.  A block combines the pairs in a fixed order
// and stores hi + lo as a double.
// ---------------------------------------------------------------------------
template <typename T>
struct ParticleSums {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    __device__ __forceinline__ void add(const typename Prec<T>::real4 &V) {
        const double m = V.w == T(1) ? 1.0 : 1.0 / (double)V.w;
        v[0] += m * V.x;
        v[1] += m * V.y;
        v[2] += m * V.z;
        v[3] += m * (V.x * V.x + V.y * V.y + V.z * V.z);
    }
    __device__ __forceinline__ void store(double *row) { block_reduce_store<4>(v, row); }
};
template <>
struct ParticleSums<float> {
    FF s[4];  // m v_x, m v_y, m v_z, m v^2
    __device__ __forceinline__ void add(const Prec<float>::real4 &V) { add_particle_moments(s, V.x, V.y, V.z, V.w); }
    __device__ __forceinline__ void store(double *row) {
        double v[4];
        ff_block_sum<RED_THREADS, 4>(s, v);
        if (threadIdx.x == 0)
#pragma unroll
            for (int c = 0; c < 4; ++c) row[c] = v[c];
    }
};

// particles are visited in id order (not slot order), so the sums do not
// depend on how the particles are currently arranged
template <typename T>
__device__ __forceinline__ void observe_particles(const typename Prec<T>::real4 *vel4, const int32_t *slot_of,
                                                  int64_t np, double *row) {
    ParticleSums<T> acc;
    const int64_t stride = (int64_t)gridDim.x * RED_THREADS;
    for (int64_t id0 = (int64_t)blockIdx.x * RED_THREADS + threadIdx.x; id0 < np; id0 += 4 * stride) {
        typename Prec<T>::real4 Vs[4];
        int32_t sl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) sl[u] = id0 + u * stride < np ? slot_of[id0 + u * stride] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (sl[u] >= 0) Vs[u] = vel4[sl[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (sl[u] >= 0) acc.add(Vs[u]);
    }
    acc.store(row);
}

// The observables in one launch: every block adds its share of the nodes and
// of the particles into its row of the partial-sum table; the last block to
// finish (an arrival counter behind the table, zero between launches) adds
// the rows in order -- one warp per column, lane l taking rows l, l + 32, ...
// (loads issued four rows ahead), then a fixed butterfly -- and writes the
// sums, then the range and device error flags as they stand at this point of
// the stream order, to out[0..9].
static_assert(RED_THREADS == 32 * RED_COLS, "the last block has one warp per column");
template <typename T, int VARIANT>
__global__ void __launch_bounds__(RED_THREADS, 4)
    observe_kernel(const typename Prec<T>::node4 *node, const typename Prec<T>::node4 *jacc, const uint2 *occw,
                   const typename Prec<T>::node4 *cact, int W, FastDiv fnx, int64_t N, int mass_u,
                   double mass_unit, const typename Prec<T>::real4 *vel4, const int32_t *slot_of, int64_t np,
                   double *partial, double inv_scale, const int32_t *range_flag, const int32_t *dev_error,
                   double *out) {
    double *row = partial + (int64_t)blockIdx.x * RED_COLS;
    observe_nodes<T, VARIANT>(node, jacc, occw, cact, W, fnx, N, mass_u, mass_unit, row);
    observe_particles<T>(vel4, slot_of, np, row + 4);
    unsigned *arrive = reinterpret_cast<unsigned *>(partial + (int64_t)gridDim.x * RED_COLS);
    __shared__ int last;
    if (threadIdx.x == 0) {
        __threadfence();  // this block's row before its arrival
        last = atomicAdd(arrive, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rows = (int)gridDim.x;
    double s = 0.0;
    int r = lane;
    for (; r + 96 < rows; r += 128) {
        double a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = __ldcg(&partial[(int64_t)(r + 32 * k) * RED_COLS + c]);
#pragma unroll
        for (int k = 0; k < 4; ++k) s += a[k];
    }
    for (; r < rows; r += 32) s += __ldcg(&partial[(int64_t)r * RED_COLS + c]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane != 0) return;
    if (c >= 1 && c <= 3) s *= inv_scale;  // fixed-point units -> momentum (a power of two: exact)
    out[c] = s;
    if (c == 0) {
        out[RED_COLS] = (double)*range_flag;
        out[RED_COLS + 1] = (double)*dev_error;
        *arrive = 0u;
    }
}

template <typename T>
static cudaError_t observables_t(lbmd_ctx *ctx) {
    using P = Prec<T>;
    const int B = ctx->red_blocks;
    const FastDiv fnx = make_fastdiv((uint32_t)ctx->p.nx);
    const int mass_u = 40 - ctx->fix.e;  // the FP32 mass sum's unit 2^-mass_u
    const double mass_unit = std::ldexp(1.0, -mass_u);
    const auto *vel = static_cast<const typename P::real4 *>(vel_now(ctx));
    if (ctx->p.variant == LBMD_VARIANT_B)
        observe_kernel<T, LBMD_VARIANT_B><<<B, RED_THREADS, 0, ctx->stream>>>(
            static_cast<const typename P::node4 *>(ctx->node), nullptr, active_words_now(ctx),
            static_cast<const typename P::node4 *>(active_records_now(ctx)), active_words(ctx->p.nx), fnx, ctx->N,
            mass_u, mass_unit, vel, ctx->slot_of, ctx->np, ctx->red_partial, ctx->fix.inv_scale, ctx->range_flag,
            ctx->dev_error, ctx->red_out);
    else  // variant A: the accumulating records of the active nodes (j* + J_acc), J_acc elsewhere; C: J_acc
        observe_kernel<T, LBMD_VARIANT_A><<<B, RED_THREADS, 0, ctx->stream>>>(
            static_cast<const typename P::node4 *>(ctx->node), static_cast<const typename P::node4 *>(ctx->jacc),
            compact_nodes(ctx) ? active_words_now(ctx) : nullptr,
            static_cast<const typename P::node4 *>(compact_nodes(ctx) ? active_records_acc(ctx) : nullptr),
            active_words(ctx->p.nx), fnx, ctx->N, mass_u, mass_unit, vel, ctx->slot_of, ctx->np, ctx->red_partial,
            ctx->fix.inv_scale, ctx->range_flag, ctx->dev_error, ctx->red_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conversions for the host accessors.
// ---------------------------------------------------------------------------
// populations [first, first + count) of the flat array f[i * N + r]; the
// base of the deviation storage w_i rho0 formed as the collision forms it
template <typename T>
__device__ __forceinline__ T pop_base(int64_t flat, int64_t N, double rho0) {
    const int i = (int)(flat / N);
    double w = 1.0 / 36.0;
    if (i == 0) w = 1.0 / 3.0;
    else if (i <= 6) w = 1.0 / 18.0;
    return T(w) * T(rho0);
}

template <typename T, typename S>
__global__ void pops_to_double_kernel(const S *f, int64_t first, int64_t count, int64_t N, double rho0,
                                      double *dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t k = first + t;
    dst[t] = (double)PopStore<S, T>::load(f + k, pop_base<T>(k, N, rho0));
}

template <typename T, typename S>
__global__ void pops_from_double_kernel(S *f, int64_t first, int64_t count, int64_t N, double rho0,
                                        const double *src) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t k = first + t;
    PopStore<S, T>::store(f + k, (T)src[t], pop_base<T>(k, N, rho0));
}

// node field (rho, j seen by the particles) or, with transfer_only, the
// pending transfer J_acc, for nodes [first, first + count)
template <typename T, typename S>
__global__ void node_to_double_kernel(const typename Prec<T>::node4 *node, const typename Prec<T>::node4 *jacc,
                                      const uint2 *occw, const typename Prec<T>::node4 *cacc, int W, int nx,
                                      const S *f, int64_t N, T rho0, T fs, T fis, int64_t first, int64_t count,
                                      double *dst, int transfer_only, int variant) {
    using P = Prec<T>;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t r = first + t;
    const typename P::node4 n = node[r];
    if (!transfer_only) {
        dst[4 * t + 0] = (double)P::rho_of(n);
        dst[4 * t + 1] = (double)P::from_fix(P::jx_of(n), fis);
        dst[4 * t + 2] = (double)P::from_fix(P::jy_of(n), fis);
        dst[4 * t + 3] = (double)P::from_fix(P::jz_of(n), fis);
        return;
    }
    const int sl = occw ? active_slot(occw[(size_t)(r / nx) * W + ((r % nx) >> 5)], (int)(r % nx)) : -1;
    if (sl >= 0 && variant == LBMD_VARIANT_A) {
        // variant A, active node: the accumulating record minus the frozen one
        const typename P::node4 c = cacc[sl];
        dst[3 * t + 0] = (double)P::from_fix(P::jx_of(c) - P::jx_of(n), fis);
        dst[3 * t + 1] = (double)P::from_fix(P::jy_of(c) - P::jy_of(n), fis);
        dst[3 * t + 2] = (double)P::from_fix(P::jz_of(c) - P::jz_of(n), fis);
    } else if (variant != LBMD_VARIANT_B) {
        const typename P::node4 J = jacc[r];
        dst[3 * t + 0] = (double)P::from_fix(P::jx_of(J), fis);
        dst[3 * t + 1] = (double)P::from_fix(P::jy_of(J), fis);
        dst[3 * t + 2] = (double)P::from_fix(P::jz_of(J), fis);
    } else {
        T fl[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) fl[i] = PopStore<S, T>::load(f + (int64_t)i * N + r, T(WEIGHT(i)) * rho0);
        T rho, jx, jy, jz;
        node_moments(fl, rho, jx, jy, jz);
        dst[3 * t + 0] = (double)P::from_fix(P::jx_of(n) - P::to_fix(jx, fs), fis);
        dst[3 * t + 1] = (double)P::from_fix(P::jy_of(n) - P::to_fix(jy, fs), fis);
        dst[3 * t + 2] = (double)P::from_fix(P::jz_of(n) - P::to_fix(jz, fs), fis);
    }
}

template <typename T>
__global__ void clear_transfer_kernel(typename Prec<T>::node4 *jacc, int64_t N) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    typename Prec<T>::node4 z;
    z.x = z.y = z.z = z.w = 0;
    jacc[r] = z;
}

// host FP64 particle arrays -> cell index + fractional offset, velocity, 1/m,
// for slots [first, first + count).  assign_ids: new particles, slot = id,
// source row t; otherwise the source row is the slot's particle id.
template <typename T>
__global__ void particles_from_double_kernel(typename Prec<T>::real4 *pos4, typename Prec<T>::real4 *vel4,
                                             int32_t *pid, int32_t *slot_of, int64_t first, int64_t count,
                                             const double *pos, const double *vel, const double *mass, int set_pos,
                                             int set_vel, int set_mass, int assign_ids, int nx, int ny, int nz) {
    using P = Prec<T>;
    // one thread per id: the FP64 host arrays are read in order (coalesced),
    // the device records written to their slots
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    int64_t src = t, p = first + t;
    if (assign_ids) {  // new particles: slot = id, the arrays hold the new ones only
        pid[p] = (int32_t)p;
        slot_of[p] = (int32_t)p;
    } else {  // existing particles: the arrays are indexed by id
        src = first + t;
        p = slot_of[src];
    }
    if (set_pos) pos4[p] = pos_from_host<T>(pos + 3 * src, nx, ny, nz);
    typename P::real4 V = vel4[p];
    if (set_vel) {
        V.x = to_storage(vel[3 * src + 0], T());
        V.y = to_storage(vel[3 * src + 1], T());
        V.z = to_storage(vel[3 * src + 2], T());
    }
    if (set_mass) V.w = (T)(1.0 / (mass ? mass[src] : 1.0));
    vel4[p] = V;
}

// device state -> FP64 arrays in id order
template <typename T>
__global__ void particles_to_double_kernel(const typename Prec<T>::real4 *pos4, const typename Prec<T>::real4 *vel4,
                                           const int32_t *slot_of, int64_t np, double *pos, double *vel, FastDiv fnx,
                                           FastDiv fny) {
    using P = Prec<T>;
    // one thread per id: the FP64 host arrays are written in order
    // (coalesced), the device records read from their slots (writing in slot
    // order instead, with coalesced reads and scattered 24-byte writes, made
    // the download and the cycle after it slower)
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= np) return;
    const int64_t p = slot_of[id];
    if (pos) {
        const typename P::real4 R = pos4[p];
        const uint32_t cell = (uint32_t)P::cell_of(R);  // < nx ny nz <= 2^32
        const uint32_t row = fdiv(cell, fnx), z = fdiv(row, fny);
        const uint32_t x = cell - row * fnx.d, y = row - z * fny.d;
        pos[3 * id + 0] = cell_plus_fraction(x, R.x);
        pos[3 * id + 1] = cell_plus_fraction(y, R.y);
        pos[3 * id + 2] = cell_plus_fraction(z, R.z);
    }
    if (vel) {
        const typename P::real4 V = vel4[p];
        vel[3 * id + 0] = to_double(V.x);
        vel[3 * id + 1] = to_double(V.y);
        vel[3 * id + 2] = to_double(V.z);
    }
}

inline unsigned nblocks(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace lbmd

using namespace lbmd;

cudaError_t launch_observables(lbmd_ctx *ctx) {
    return ctx->p.precision == LBMD_FP64 ? observables_t<double>(ctx) : observables_t<float>(ctx);
}

template <typename T, typename S>
static cudaError_t pops_to_double_t(lbmd_ctx *ctx, int64_t first, int64_t count, double *dst) {
    pops_to_double_kernel<T, S><<<nblocks(count), 256, 0, ctx->stream>>>(
        static_cast<const S *>(ctx->f[ctx->cur]), first, count, ctx->N, ctx->p.rho0, dst);
    return cudaGetLastError();
}

template <typename T, typename S>
static cudaError_t pops_from_double_t(lbmd_ctx *ctx, int64_t first, int64_t count, const double *src) {
    pops_from_double_kernel<T, S><<<nblocks(count), 256, 0, ctx->stream>>>(static_cast<S *>(ctx->f[ctx->cur]),
                                                                            first, count, ctx->N, ctx->p.rho0, src);
    return cudaGetLastError();
}

template <typename T, typename S>
static cudaError_t node_to_double_t(lbmd_ctx *ctx, int64_t first, int64_t count, double *dst, bool transfer_only) {
    using N4 = typename Prec<T>::node4;
    node_to_double_kernel<T, S><<<nblocks(count), 256, 0, ctx->stream>>>(
        static_cast<const N4 *>(ctx->node), static_cast<const N4 *>(ctx->jacc),
        compact_nodes(ctx) ? active_words_now(ctx) : nullptr,
        static_cast<const N4 *>(compact_nodes(ctx) ? active_records_acc(ctx) : nullptr), active_words(ctx->p.nx),
        ctx->p.nx, static_cast<const S *>(ctx->f[ctx->cur]), ctx->N, (T)ctx->p.rho0, (T)ctx->fix.scale,
        (T)ctx->fix.inv_scale, first, count, dst, transfer_only ? 1 : 0, ctx->p.variant);
    return cudaGetLastError();
}

#define LBMD_DISPATCH_POPS(ctx, FN, ...)                                                      \
    ((ctx)->p.precision == LBMD_FP64          ? FN<double, double>(__VA_ARGS__)               \
     : (ctx)->p.precision == LBMD_FP16_DEV    ? FN<float, __half>(__VA_ARGS__)                \
     : (ctx)->p.precision == LBMD_BF16_DEV    ? FN<float, __nv_bfloat16>(__VA_ARGS__)         \
     : (ctx)->p.precision == LBMD_FP16_DEV_SR ? FN<float, lbmd::half_sr>(__VA_ARGS__)         \
     : (ctx)->p.precision == LBMD_BF16_DEV_SR ? FN<float, lbmd::bf16_sr>(__VA_ARGS__)         \
                                              : FN<float, float>(__VA_ARGS__))

cudaError_t launch_populations_to_double(lbmd_ctx *ctx, int64_t first, int64_t count, double *dst) {
    if (count <= 0) return cudaSuccess;
    return LBMD_DISPATCH_POPS(ctx, pops_to_double_t, ctx, first, count, dst);
}

cudaError_t launch_populations_from_double(lbmd_ctx *ctx, int64_t first, int64_t count, const double *src) {
    if (count <= 0) return cudaSuccess;
    return LBMD_DISPATCH_POPS(ctx, pops_from_double_t, ctx, first, count, src);
}

cudaError_t launch_node_field_to_double(lbmd_ctx *ctx, int64_t first, int64_t count, double *dst,
                                        bool transfer_only) {
    if (count <= 0) return cudaSuccess;
    return LBMD_DISPATCH_POPS(ctx, node_to_double_t, ctx, first, count, dst, transfer_only);
}

cudaError_t launch_clear_transfer(lbmd_ctx *ctx) {
    if (ctx->p.variant == LBMD_VARIANT_B) return cudaSuccess;
    if (ctx->p.precision == LBMD_FP64)
        clear_transfer_kernel<double><<<nblocks(ctx->N), 256, 0, ctx->stream>>>(
            static_cast<Prec<double>::node4 *>(ctx->jacc), ctx->N);
    else
        clear_transfer_kernel<float><<<nblocks(ctx->N), 256, 0, ctx->stream>>>(
            static_cast<Prec<float>::node4 *>(ctx->jacc), ctx->N);
    return cudaGetLastError();
}

cudaError_t launch_particles_from_double(lbmd_ctx *ctx, int64_t first, int64_t count, const double *pos,
                                         const double *vel, const double *mass, bool set_pos, bool set_vel,
                                         bool set_mass) {
    if (count <= 0) return cudaSuccess;
    const int b = ctx->pcur;
    const int assign = set_mass ? 1 : 0;  // only lbmd_add_particles sets masses
    if (ctx->p.precision == LBMD_FP64)
        particles_from_double_kernel<double><<<nblocks(count), 256, 0, ctx->stream>>>(
            static_cast<Prec<double>::real4 *>(pos_now(ctx)), static_cast<Prec<double>::real4 *>(vel_now(ctx)),
            ctx->pid[b], ctx->slot_of, first, count, pos, vel, mass, set_pos, set_vel, set_mass, assign, ctx->p.nx,
            ctx->p.ny, ctx->p.nz);
    else
        particles_from_double_kernel<float><<<nblocks(count), 256, 0, ctx->stream>>>(
            static_cast<Prec<float>::real4 *>(pos_now(ctx)), static_cast<Prec<float>::real4 *>(vel_now(ctx)),
            ctx->pid[b], ctx->slot_of, first, count, pos, vel, mass, set_pos, set_vel, set_mass, assign, ctx->p.nx,
            ctx->p.ny, ctx->p.nz);
    return cudaGetLastError();
}

cudaError_t launch_particles_to_double(lbmd_ctx *ctx, double *pos, double *vel) {
    if (ctx->np <= 0) return cudaSuccess;
    const FastDiv fnx = make_fastdiv((uint32_t)ctx->p.nx), fny = make_fastdiv((uint32_t)ctx->p.ny);
    if (ctx->p.precision == LBMD_FP64)
        particles_to_double_kernel<double><<<nblocks(ctx->np), 256, 0, ctx->stream>>>(
            static_cast<const Prec<double>::real4 *>(pos_now(ctx)),
            static_cast<const Prec<double>::real4 *>(vel_now(ctx)), ctx->slot_of, ctx->np, pos, vel, fnx, fny);
    else
        particles_to_double_kernel<float><<<nblocks(ctx->np), 256, 0, ctx->stream>>>(
            static_cast<const Prec<float>::real4 *>(pos_now(ctx)),
            static_cast<const Prec<float>::real4 *>(vel_now(ctx)), ctx->slot_of, ctx->np, pos, vel, fnx, fny);
    return cudaGetLastError();
}
