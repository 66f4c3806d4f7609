// observe.cu -- FP64 reductions of the observables and the conversions
// between the device storage and the FP64 host arrays of the C ABI.
//
// Observables (mass, fluid momentum incl. pending transfers, particle
// momentum, sum of m v^2): every thread accumulates a fixed strided subset in
// double precision, each block reduces in a fixed tree order into one row of
// a partial-sum table, and a single block adds the rows in order.  The grid
// size is fixed per context, so the sums are bitwise reproducible.
#include "lbmd_ctx.h"
#include "lbmd_device.cuh"
#include "particle_core.cuh"

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

// Momentum sums in fixed-point units: FP32 records hold 32-bit integers,
// whose per-thread sums are exact in 64-bit integers (and exact again as
// doubles, being far below 2^53); FP64 records (56 fraction bits) are summed
// in doubles.
template <typename T>
struct MomentumSum {
    using type = double;
};
template <>
struct MomentumSum<float> {
    using type = long long;
};

// Variant B keeps the records of the active nodes in their compact array
// during a cycle: a node's current record is found through the active words
// (occw non-null), so no copy back is needed first.
template <typename T, int VARIANT>
__global__ void __launch_bounds__(RED_THREADS)
    observe_nodes_kernel(const typename Prec<T>::node4 *node, const typename Prec<T>::node4 *jacc,
                         const uint2 *occw, const typename Prec<T>::node4 *cact, int W, FastDiv fnx, int64_t N,
                         double *partial) {
    using P = Prec<T>;
    using M = typename MomentumSum<T>::type;
    double rho = 0.0;
    M jx = 0, jy = 0, jz = 0;
    const int64_t stride = (int64_t)gridDim.x * RED_THREADS;
    // four nodes per pass, all loaded before use (memory-level parallelism)
    for (int64_t r0 = (int64_t)blockIdx.x * RED_THREADS + threadIdx.x; r0 < N; r0 += 4 * stride) {
        typename P::node4 n[4], J[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t r = r0 + u * stride;
            if (r >= N) continue;
            if (occw) {
                const uint32_t row = fdiv((uint32_t)r, fnx);
                const int x = (int)((uint32_t)r - row * fnx.d);
                const int sl = active_slot(occw[(size_t)row * W + (x >> 5)], x);
                n[u] = sl >= 0 ? cact[sl] : node[r];
            } else {
                n[u] = node[r];
            }
            if (VARIANT == LBMD_VARIANT_A) J[u] = jacc[r];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (r0 + u * stride >= N) continue;
            rho += (double)P::rho_of(n[u]);
            jx += (M)P::jx_of(n[u]);
            jy += (M)P::jy_of(n[u]);
            jz += (M)P::jz_of(n[u]);
            if (VARIANT == LBMD_VARIANT_A) {
                jx += (M)P::jx_of(J[u]);
                jy += (M)P::jy_of(J[u]);
                jz += (M)P::jz_of(J[u]);
            }
        }
    }
    // momenta stay in fixed-point units until the final scaling
    double v[4] = {rho, (double)jx, (double)jy, (double)jz};
    block_reduce_store<4>(v, partial + (int64_t)blockIdx.x * RED_COLS);
}

// particles are visited in id order (not slot order), so the sums do not
// depend on how the particles are currently arranged
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
    observe_particles_kernel(const typename Prec<T>::real4 *vel4, const int32_t *slot_of, int64_t np,
                             double *partial) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
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
        for (int u = 0; u < 4; ++u) {
            if (sl[u] < 0) continue;
            const double m = 1.0 / (double)Vs[u].w;
            const double vx = Vs[u].x, vy = Vs[u].y, vz = Vs[u].z;
            v[0] += m * vx;
            v[1] += m * vy;
            v[2] += m * vz;
            v[3] += m * (vx * vx + vy * vy + vz * vz);
        }
    }
    block_reduce_store<4>(v, partial + (int64_t)blockIdx.x * RED_COLS + 4);
}

// one warp per column: lane l adds rows l, l + 32, ... in order, then a fixed
// butterfly combines the lanes; out[8], out[9] take the range and device
// error flags as they stand at this point of the stream order
template <typename T>
__global__ void __launch_bounds__(32 * RED_COLS) observe_final_kernel(const double *partial, int rows, double inv_scale,
                                                                      const int32_t *range_flag,
                                                                      const int32_t *dev_error, double *out) {
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        out[RED_COLS] = (double)*range_flag;
        out[RED_COLS + 1] = (double)*dev_error;
    }
    double s = 0.0;
    for (int r = lane; r < rows; r += 32) s += partial[(int64_t)r * RED_COLS + c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane != 0) return;
    if (c >= 1 && c <= 3) s *= inv_scale;  // fixed-point units -> momentum (a power of two: exact)
    out[c] = s;
}

template <typename T>
static cudaError_t observables_t(lbmd_ctx *ctx) {
    using P = Prec<T>;
    const int B = ctx->red_blocks;
    const FastDiv fnx = make_fastdiv((uint32_t)ctx->p.nx);
    if (ctx->p.variant == LBMD_VARIANT_B)
        observe_nodes_kernel<T, LBMD_VARIANT_B><<<B, RED_THREADS, 0, ctx->stream>>>(
            static_cast<const typename P::node4 *>(ctx->node), nullptr, active_words_now(ctx),
            static_cast<const typename P::node4 *>(active_records_now(ctx)), active_words(ctx->p.nx), fnx, ctx->N,
            ctx->red_partial);
    else  // variant A: the accumulating records of the active nodes (j* + J_acc), J_acc elsewhere; C: J_acc
        observe_nodes_kernel<T, LBMD_VARIANT_A><<<B, RED_THREADS, 0, ctx->stream>>>(
            static_cast<const typename P::node4 *>(ctx->node), static_cast<const typename P::node4 *>(ctx->jacc),
            compact_nodes(ctx) ? active_words_now(ctx) : nullptr,
            static_cast<const typename P::node4 *>(compact_nodes(ctx) ? active_records_acc(ctx) : nullptr),
            active_words(ctx->p.nx), fnx, ctx->N, ctx->red_partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    observe_particles_kernel<T><<<B, RED_THREADS, 0, ctx->stream>>>(
        static_cast<const typename P::real4 *>(vel_now(ctx)), ctx->slot_of, ctx->np, ctx->red_partial);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    observe_final_kernel<T><<<1, 32 * RED_COLS, 0, ctx->stream>>>(ctx->red_partial, B, ctx->fix.inv_scale,
                                                                   ctx->range_flag, ctx->dev_error, ctx->red_out);
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
    if (set_pos) pos4[p] = pos_from_double<T>(pos + 3 * src, nx, ny, nz);
    typename P::real4 V = vel4[p];
    if (set_vel) {
        V.x = (T)vel[3 * src + 0];
        V.y = (T)vel[3 * src + 1];
        V.z = (T)vel[3 * src + 2];
    }
    if (set_mass) V.w = (T)(1.0 / (mass ? mass[src] : 1.0));
    vel4[p] = V;
}

// device state -> FP64 arrays in id order
template <typename T>
__global__ void particles_to_double_kernel(const typename Prec<T>::real4 *pos4, const typename Prec<T>::real4 *vel4,
                                           const int32_t *slot_of, int64_t np, double *pos, double *vel, int nx,
                                           int ny) {
    using P = Prec<T>;
    // one thread per id: the FP64 host arrays are written in order
    // (coalesced), the device records read from their slots
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= np) return;
    const int64_t p = slot_of[id];
    if (pos) {
        const typename P::real4 R = pos4[p];
        const uint32_t cell = (uint32_t)P::cell_of(R);  // < nx ny nz <= 2^32
        const uint32_t nxy = (uint32_t)nx * (uint32_t)ny;
        const uint32_t z = cell / nxy, rem = cell - z * nxy, y = rem / (uint32_t)nx, x = rem - y * (uint32_t)nx;
        pos[3 * id + 0] = (double)x + (double)R.x;
        pos[3 * id + 1] = (double)y + (double)R.y;
        pos[3 * id + 2] = (double)z + (double)R.z;
    }
    if (vel) {
        const typename P::real4 V = vel4[p];
        vel[3 * id + 0] = (double)V.x;
        vel[3 * id + 1] = (double)V.y;
        vel[3 * id + 2] = (double)V.z;
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
    if (ctx->p.precision == LBMD_FP64)
        particles_to_double_kernel<double><<<nblocks(ctx->np), 256, 0, ctx->stream>>>(
            static_cast<const Prec<double>::real4 *>(pos_now(ctx)),
            static_cast<const Prec<double>::real4 *>(vel_now(ctx)), ctx->slot_of, ctx->np, pos, vel, ctx->p.nx,
            ctx->p.ny);
    else
        particles_to_double_kernel<float><<<nblocks(ctx->np), 256, 0, ctx->stream>>>(
            static_cast<const Prec<float>::real4 *>(pos_now(ctx)),
            static_cast<const Prec<float>::real4 *>(vel_now(ctx)),
            ctx->slot_of, ctx->np, pos, vel, ctx->p.nx, ctx->p.ny);
    return cudaGetLastError();
}
