// lb.cu -- the lattice Boltzmann update (Sec. 2, Eq. (3)) on the GPU.
//
// lb_collide_push: one thread per node.  Reads the 19 post-stream populations
// f*_i (coalesced structure-of-arrays loads), the momentum the particles
// handed over since the last LB step, and applies the MRT collision in moment
// space with thermal noise (Philox in registers) and the forcing term of the
// force density F = J_acc / tau_LB + g; the post-collision populations are
// pushed to the neighbours r + c_i in the other buffer.
//
// forcing_update_kernel (variant C): after every MD step, the transfer of
// that step enters the populations through the forcing part of the collision.
//
// node_moments_kernel: one thread per node.  Recomputes rho* and j* of the
// freshly streamed populations and writes the node field that the MD steps of
// the next LB cycle read (and, in variant B, update); in variant B also the
// compact record of every active node.
#include "lb_core.cuh"
#include "lbmd_ctx.h"
#include "lbmd_device.cuh"

namespace lbmd {

template <typename T, typename S>
struct LbArgs {
    const S *__restrict__ fin;
    S *__restrict__ fout;
    T rho0;  // reference density of the deviation storage
    typename Prec<T>::node4 *node;
    typename Prec<T>::node4 *jacc;
    const uint2 *occw;                     // variant B: active nodes
    const typename Prec<T>::node4 *cact;   // variant B: their compact records
    int occ_words;
    int nx, ny, nz;
    int64_t N;
    T gamma_bulk, gamma_shear, gamma_ghost;
    T amp16[Q];  // noise amplitude sqrt(mu b_k (1 - g_k^2)) times sqrt(12) 2^-16
    T g[3];
    uint32_t key0, key1;
    const unsigned long long *lb_step;
    int noisy;
    int variant;
};

// One thread per node; grid (ceil(nx / blockDim.x), ny, nz).  The variant is
// a run-time (warp-uniform) flag rather than a template parameter: both
// variants then execute one compiled instruction sequence, so at m = 1 they
// agree bit for bit, as the paper's algorithmic equivalence requires.
template <typename T, typename S, bool RELAX_FULL>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 3) lb_collide_push(LbArgs<T, S> a) {
    using P = Prec<T>;
    using St = PopStore<S, T>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const uint32_t r = (uint32_t)x + (uint32_t)a.nx * ((uint32_t)y + (uint32_t)a.ny * (uint32_t)z);
    T f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = St::load(a.fin + (size_t)i * a.N + r, T(WEIGHT(i)) * a.rho0);
    T rho, jx, jy, jz;
    node_moments(f, rho, jx, jy, jz);
    T Fx, Fy, Fz;
    if (a.variant == LBMD_VARIANT_B) {
        // node j = fix(j*) + sum of fixed-point transfers: the difference is
        // exactly the accumulated transfer J_acc (an active node's current
        // record is its compact one)
        const int sl = active_slot(a.occw[((size_t)y + (size_t)a.ny * z) * a.occ_words + (x >> 5)], x);
        const typename P::node4 n = sl >= 0 ? a.cact[sl] : a.node[r];
        Fx = P::from_fix(P::jx_of(n) - P::to_fix(jx));
        Fy = P::from_fix(P::jy_of(n) - P::to_fix(jy));
        Fz = P::from_fix(P::jz_of(n) - P::to_fix(jz));
    } else {
        const typename P::node4 J = a.jacc[r];
        Fx = P::from_fix(P::jx_of(J));
        Fy = P::from_fix(P::jy_of(J));
        Fz = P::from_fix(P::jz_of(J));
        typename P::node4 zero;
        zero.x = zero.y = zero.z = zero.w = 0;
        a.jacc[r] = zero;
    }
    Fx += a.g[0];
    Fy += a.g[1];
    Fz += a.g[2];
    collide<T, RELAX_FULL>(f, rho, jx, jy, jz, Fx, Fy, Fz, a, a.key0, a.key1, r, (uint32_t)(*a.lb_step));

    const int xm = x == 0 ? a.nx - 1 : x - 1, xp = x == a.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? a.ny - 1 : y - 1, yp = y == a.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? a.nz - 1 : z - 1, zp = z == a.nz - 1 ? 0 : z + 1;
    const int X[3] = {xm, x, xp}, Y[3] = {ym, y, yp}, Z[3] = {zm, z, zp};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const uint32_t t = (uint32_t)X[CX(i) + 1] +
                           (uint32_t)a.nx * ((uint32_t)Y[CY(i) + 1] + (uint32_t)a.ny * (uint32_t)Z[CZ(i) + 1]);
        St::store(a.fout + (size_t)i * a.N + t, f[i], T(WEIGHT(i)) * a.rho0);
    }
}

template <typename T, typename S>
__global__ void __launch_bounds__(256)
    node_moments_kernel(const S *__restrict__ f, typename Prec<T>::node4 *node, const uint2 *occw,
                        typename Prec<T>::node4 *cact, int occ_words, int64_t N, int nx, int ny, T rho0,
                        unsigned long long *lb_step, int count_step) {
    using P = Prec<T>;
    using St = PopStore<S, T>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (count_step && x == 0 && blockIdx.y == 0 && blockIdx.z == 0) *lb_step += 1ull;
    if (x >= nx) return;
    // planes in reverse order: the LB kernel wrote the high planes last, so
    // they are the ones still in L2
    const uint32_t z = gridDim.z - 1 - blockIdx.z;
    const uint32_t r = (uint32_t)x + (uint32_t)nx * ((uint32_t)blockIdx.y + (uint32_t)ny * z);
    T fl[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fl[i] = St::load(f + (size_t)i * N + r, T(WEIGHT(i)) * rho0);
    T rho, jx, jy, jz;
    node_moments(fl, rho, jx, jy, jz);
    const typename P::node4 rec = P::pack(rho, P::to_fix(jx), P::to_fix(jy), P::to_fix(jz));
    node[r] = rec;
    if (occw) {
        const int sl = active_slot(occw[((size_t)blockIdx.y + (size_t)ny * z) * occ_words + (x >> 5)], x);
        if (sl >= 0) cact[sl] = rec;
    }
}

// Variant C (Sec. 4): the momentum transfer F = J_acc of the MD step just
// done enters the populations through the forcing part of the collision
// alone: mass unchanged, momentum + F, stress modes + (1 + gamma) times the
// symmetric products of u = (j + F/2)/rho and F (as in collide()), ghost
// modes unchanged; then the node record is recomputed from the populations
// and J_acc is cleared.  Nodes without a transfer are left as they are.
template <typename T, typename S>
__global__ void __launch_bounds__(256) forcing_update_kernel(S *__restrict__ f, typename Prec<T>::node4 *node,
                                                             typename Prec<T>::node4 *jacc, int64_t N, T rho0,
                                                             T gamma_bulk, T gamma_shear) {
    using P = Prec<T>;
    using St = PopStore<S, T>;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const typename P::node4 J = jacc[r];
    if (P::jx_of(J) == 0 && P::jy_of(J) == 0 && P::jz_of(J) == 0) return;
    const T Fx = P::from_fix(P::jx_of(J)), Fy = P::from_fix(P::jy_of(J)), Fz = P::from_fix(P::jz_of(J));
    T fl[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fl[i] = St::load(f + (int64_t)i * N + r, T(WEIGHT(i)) * rho0);
    T rho, jx, jy, jz;
    node_moments(fl, rho, jx, jy, jz);
    const T ir = T(1) / rho;
    const T ux = (jx + T(0.5) * Fx) * ir, uy = (jy + T(0.5) * Fy) * ir, uz = (jz + T(0.5) * Fz) * ir;
    const T uF = ux * Fx + uy * Fy + uz * Fz;
    T dm[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) dm[k] = T(0);
    dm[1] = Fx;
    dm[2] = Fy;
    dm[3] = Fz;
    const T fb = T(1) + gamma_bulk, fs = T(1) + gamma_shear;
    dm[4] = fb * uF;
    dm[5] = fs * (T(3) * ux * Fx - uF);
    dm[6] = fs * (uy * Fy - uz * Fz);
    dm[7] = fs * T(0.5) * (ux * Fy + uy * Fx);
    dm[8] = fs * T(0.5) * (ux * Fz + uz * Fx);
    dm[9] = fs * T(0.5) * (uy * Fz + uz * Fy);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T acc = T(0);
#pragma unroll
        for (int k = 1; k <= 9; ++k) {
            const int e = EMODE(k, i);
            if (e != 0) acc += T(e) * dm[k] * T(INV_BNORM(k));
        }
        fl[i] += T(WEIGHT(i)) * acc;
        St::store(f + (int64_t)i * N + r, fl[i], T(WEIGHT(i)) * rho0);
    }
    node_moments(fl, rho, jx, jy, jz);
    node[r] = P::pack(rho, P::to_fix(jx), P::to_fix(jy), P::to_fix(jz));
    typename P::node4 zero;
    zero.x = zero.y = zero.z = zero.w = 0;
    jacc[r] = zero;
}

template <typename T, typename S>
__global__ void init_equilibrium_kernel(S *f, int64_t N, T rho0) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) PopStore<S, T>::store(f + (int64_t)i * N + r, T(WEIGHT(i)) * rho0, T(WEIGHT(i)) * rho0);
}

// Node kernels run one thread per node on a (x-blocks, ny, nz) grid.
static dim3 node_block(const lbmd_ctx *ctx) {
    const int bx = ctx->p.nx >= 256 ? 256 : (ctx->p.nx >= 128 ? 128 : (ctx->p.nx >= 64 ? 64 : 32));
    return dim3(bx, 1, 1);
}
static dim3 node_grid(const lbmd_ctx *ctx, dim3 block) {
    return dim3((ctx->p.nx + block.x - 1) / block.x, ctx->p.ny, ctx->p.nz);
}

template <typename T, typename S>
static cudaError_t lb_step_t(lbmd_ctx *ctx) {
    LbArgs<T, S> a;
    a.fin = static_cast<const S *>(ctx->f[ctx->cur]);
    a.fout = static_cast<S *>(ctx->f[ctx->cur ^ 1]);
    a.rho0 = (T)ctx->p.rho0;
    a.node = static_cast<typename Prec<T>::node4 *>(ctx->node);
    a.jacc = static_cast<typename Prec<T>::node4 *>(ctx->jacc);
    a.occw = ctx->occw;
    a.cact = static_cast<const typename Prec<T>::node4 *>(ctx->cact);
    a.occ_words = active_words(ctx->p.nx);
    a.nx = ctx->p.nx;
    a.ny = ctx->p.ny;
    a.nz = ctx->p.nz;
    a.N = ctx->N;
    a.gamma_bulk = (T)ctx->co.gamma_bulk;
    a.gamma_shear = (T)ctx->co.gamma_shear;
    a.gamma_ghost = (T)ctx->co.gamma_ghost;
    for (int k = 0; k < Q; ++k) a.amp16[k] = (T)(ctx->co.noise_amp[k] * 3.4641016151377544 * 1.52587890625e-05);
    for (int d = 0; d < 3; ++d) a.g[d] = (T)ctx->co.body_force[d];
    a.key0 = (uint32_t)(ctx->p.seed & 0xffffffffu);
    a.key1 = (uint32_t)(ctx->p.seed >> 32);
    a.lb_step = ctx->d_lb_step;
    a.noisy = ctx->co.noisy;
    a.variant = ctx->p.variant;
    const dim3 block = node_block(ctx), grid = node_grid(ctx, block);
    if (ctx->co.gamma_bulk == 0.0 && ctx->co.gamma_ghost == 0.0)
        lb_collide_push<T, S, true><<<grid, block, 0, ctx->stream>>>(a);
    else
        lb_collide_push<T, S, false><<<grid, block, 0, ctx->stream>>>(a);
    return cudaGetLastError();
}

template <typename T, typename S>
static cudaError_t node_moments_t(lbmd_ctx *ctx, bool count_step) {
    const dim3 block = node_block(ctx), grid = node_grid(ctx, block);
    const bool B = ctx->p.variant == LBMD_VARIANT_B;
    node_moments_kernel<T, S><<<grid, block, 0, ctx->stream>>>(
        static_cast<const S *>(ctx->f[ctx->cur]), static_cast<typename Prec<T>::node4 *>(ctx->node),
        B ? ctx->occw : nullptr, static_cast<typename Prec<T>::node4 *>(ctx->cact), active_words(ctx->p.nx), ctx->N,
        ctx->p.nx, ctx->p.ny, (T)ctx->p.rho0, ctx->d_lb_step, count_step ? 1 : 0);
    return cudaGetLastError();
}

template <typename T, typename S>
static cudaError_t forcing_update_t(lbmd_ctx *ctx) {
    const unsigned blocks = (unsigned)((ctx->N + 255) / 256);
    forcing_update_kernel<T, S><<<blocks, 256, 0, ctx->stream>>>(
        static_cast<S *>(ctx->f[ctx->cur]), static_cast<typename Prec<T>::node4 *>(ctx->node),
        static_cast<typename Prec<T>::node4 *>(ctx->jacc), ctx->N, (T)ctx->p.rho0, (T)ctx->co.gamma_bulk,
        (T)ctx->co.gamma_shear);
    return cudaGetLastError();
}

template <typename T, typename S>
static cudaError_t init_equilibrium_t(lbmd_ctx *ctx) {
    const unsigned blocks = (unsigned)((ctx->N + 255) / 256);
    init_equilibrium_kernel<T, S><<<blocks, 256, 0, ctx->stream>>>(static_cast<S *>(ctx->f[ctx->cur]), ctx->N,
                                                                    (T)ctx->p.rho0);
    return cudaGetLastError();
}

}  // namespace lbmd

// population storage per precision: FP32 and FP64 plain, FP16 / BF16 as
// deviations with FP32 arithmetic
#define LBMD_DISPATCH_POPS(ctx, FN, ...)                                                   \
    ((ctx)->p.precision == LBMD_FP64       ? FN<double, double>(__VA_ARGS__)               \
     : (ctx)->p.precision == LBMD_FP16_DEV ? FN<float, __half>(__VA_ARGS__)                \
     : (ctx)->p.precision == LBMD_BF16_DEV ? FN<float, __nv_bfloat16>(__VA_ARGS__)         \
                                           : FN<float, float>(__VA_ARGS__))

// One LB update: collide and stream, re-order the particles by row, rebuild
// the active nodes (variant B) and recompute the node field (and the active
// nodes' compact records) from the new populations.
cudaError_t launch_lb_step(lbmd_ctx *ctx) {
    cudaError_t e = LBMD_DISPATCH_POPS(ctx, lbmd::lb_step_t, ctx);
    if (e != cudaSuccess) return e;
    ctx->cur ^= 1;
    if ((e = launch_sort_particles(ctx)) != cudaSuccess) return e;
    if ((e = launch_active_set(ctx)) != cudaSuccess) return e;
    return launch_node_moments(ctx, true);
}

cudaError_t launch_node_moments(lbmd_ctx *ctx, bool count_step) {
    return LBMD_DISPATCH_POPS(ctx, lbmd::node_moments_t, ctx, count_step);
}

cudaError_t launch_init_equilibrium(lbmd_ctx *ctx) { return LBMD_DISPATCH_POPS(ctx, lbmd::init_equilibrium_t, ctx); }

cudaError_t launch_forcing_update(lbmd_ctx *ctx) { return LBMD_DISPATCH_POPS(ctx, lbmd::forcing_update_t, ctx); }
