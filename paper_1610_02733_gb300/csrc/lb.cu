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
// The post-stream moments rho* and j* of the freshly streamed populations
// (the node field the MD steps of the next LB cycle read and, in variant B,
// update, plus the compact record of every active node) are fused into
// lb_collide_push: a block computes them for the node row two planes back,
// once the 27 blocks around that row have pushed (per-block flags tagged with
// the LB step); moments_rest_kernel covers the rows the dataflow cannot
// reach.  node_moments_kernel computes them on their own (creation, replaced
// populations).
#include "lb_core.cuh"
#include "lbmd_ctx.h"
#include "lbmd_device.cuh"

namespace lbmd {

template <typename T, typename S>
struct LbArgs {
    const S *__restrict__ fin;
    S *__restrict__ fout;
    T rho_base;  // deviation storage: sum_i of the stored rest values w_i rho0
    typename Prec<T>::node4 *node;
    typename Prec<T>::node4 *jacc;
    const uint2 *occw;                     // variant B: active nodes of this cycle
    const typename Prec<T>::node4 *cact;   // variant B: their compact records
    const uint2 *occw_new;                 // variant B: active nodes of the next cycle
    typename Prec<T>::node4 *cact_new;     // ... whose records the fused moments write
    typename Prec<T>::node4 *cact_new2;    // variant A with a frozen copy: the same records again
    int occ_words;
    // fused post-stream moments (dataflow between collide blocks)
    uint32_t *blk_done;
    int32_t *missed, *missed_list;
    int spin;  // polls of the wait for the neighbour blocks (0: every row to the fallback)
    int nx, ny, nz;
    int64_t N;
    T fs, fis;            // fixed-point scale of the momentum density and its inverse
    int32_t *range_flag;  // set when a written record reaches half the fixed-point range
    T gamma_bulk, gamma_shear, gamma_ghost;
    T amp16[Q];  // noise amplitude sqrt(mu b_k (1 - g_k^2)) times sqrt(12) 2^-16
    T ampg[Q];   // the amplitude itself (normal variates)
    T g[3];
    uint32_t key0, key1;
    const unsigned long long *lb_step;
    int noisy;
    int variant;
};

// Range guard: a record whose momentum reaches half the fixed-point range
// raises the context's flag (the integer sums of later transfers could wrap).
template <typename T>
__device__ __forceinline__ typename Prec<T>::node4 guarded_record(T rho, T jx, T jy, T jz, T fs,
                                                                  int32_t *range_flag) {
    using P = Prec<T>;
    const typename P::fix ix = P::to_fix(jx, fs), iy = P::to_fix(jy, fs), iz = P::to_fix(jz, fs);
    if (P::beyond_half(ix) | P::beyond_half(iy) | P::beyond_half(iz)) atomicOr(range_flag, 1);
    return P::pack(rho, ix, iy, iz);
}

// Post-stream moments rho*, j* (Eqs. (1), (2)) of node (x, y, t): the node
// record and, for an active node of the coming cycle (variant B), its
// compact record.  The populations are read through L2 (ld.global.cg): they
// were written by other blocks of the same kernel.
template <typename T, typename S>
__device__ __forceinline__ void node_moments_at(const S *f, typename Prec<T>::node4 *node, const uint2 *occw,
                                                typename Prec<T>::node4 *cact, typename Prec<T>::node4 *cact2,
                                                int occ_words, int64_t N, int nx, int ny, T rho_base, T fs,
                                                int32_t *range_flag, int x, int y, int t) {
    using P = Prec<T>;
    using St = PopStore<S, T>;
    const uint32_t r = (uint32_t)x + (uint32_t)nx * ((uint32_t)y + (uint32_t)ny * (uint32_t)t);
    T fl[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fl[i] = St::arith_cg(f + (size_t)i * N + r);
    T rho, rho_m, jx, jy, jz;
    pop_moments<St::deviation>(fl, rho_base, rho, rho_m, jx, jy, jz);
    const typename P::node4 rec = guarded_record(rho, jx, jy, jz, fs, range_flag);
    node[r] = rec;
    if (occw) {
        const int sl = active_slot(occw[((size_t)y + (size_t)ny * t) * occ_words + (x >> 5)], x);
        if (sl >= 0) {
            cact[sl] = rec;
            if (cact2) cact2[sl] = rec;
        }
    }
}

// The moments of node row (block) b of the collide grid are computed, once
// its 27 neighbouring blocks (planes t - 1..t + 1) have pushed, by the block
// FUSE_LAG planes further on; rows of the first plane and of the last
// FUSE_LAG planes (whose neighbourhood wraps to later planes), and any row
// whose wait ran out, are left to moments_rest_kernel.
constexpr int FUSE_LAG = 2;
// The wait polls at most ctx->fuse_spin times (64 ns apart; default
// LBMD_DEFAULT_FUSE_SPIN, far above the few us the lag needs); a context can
// lower it (lbmd_set_moments_wait), down to 0, where every row goes to the
// fallback kernel.

// One thread per node; grid (ceil(nx / blockDim.x), ny, nz).  The variant is
// a run-time (warp-uniform) flag rather than a template parameter: both
// variants then execute one compiled instruction sequence, so at m = 1 they
// agree bit for bit, as the paper's algorithmic equivalence requires.
// Collide node (x, y, z) and push its post-collision populations to the
// neighbours r + c_i in the other buffer.
template <typename T, typename S, bool RELAX_FULL, bool GAUSS>
__device__ __forceinline__ void collide_push_node(const LbArgs<T, S> &a, int x, int y, int z,
                                                  unsigned long long step) {
    using P = Prec<T>;
    using St = PopStore<S, T>;
    const uint32_t r = (uint32_t)x + (uint32_t)a.nx * ((uint32_t)y + (uint32_t)a.ny * (uint32_t)z);
    T f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = St::arith(a.fin + (size_t)i * a.N + r);
    T rho, rho_m, jx, jy, jz;
    pop_moments<St::deviation>(f, a.rho_base, rho, rho_m, jx, jy, jz);
    T Fx, Fy, Fz;
    const int sl = a.occw ? active_slot(a.occw[((size_t)y + (size_t)a.ny * z) * a.occ_words + (x >> 5)], x) : -1;
    if (sl >= 0 || a.variant == LBMD_VARIANT_B) {
        // the record j = fix(j*) + sum of fixed-point transfers: the
        // difference is exactly the accumulated transfer J_acc (an active
        // node's record is its compact one -- variant A: the accumulating
        // copy; B: an inactive node's is the node field)
        const typename P::node4 n = sl >= 0 ? a.cact[sl] : a.node[r];
        Fx = P::from_fix(P::jx_of(n) - P::to_fix(jx, a.fs), a.fis);
        Fy = P::from_fix(P::jy_of(n) - P::to_fix(jy, a.fs), a.fis);
        Fz = P::from_fix(P::jz_of(n) - P::to_fix(jz, a.fs), a.fis);
    } else if (a.occw) {
        // variant A, inactive node: J_acc holds what migrants handed over
        // (rarely anything; cleared only where set)
        const typename P::node4 J = a.jacc[r];
        Fx = P::from_fix(P::jx_of(J), a.fis);
        Fy = P::from_fix(P::jy_of(J), a.fis);
        Fz = P::from_fix(P::jz_of(J), a.fis);
        if ((P::jx_of(J) | P::jy_of(J) | P::jz_of(J)) != 0) {
            typename P::node4 zero;
            zero.x = zero.y = zero.z = zero.w = 0;
            a.jacc[r] = zero;
        }
    } else {
        const typename P::node4 J = a.jacc[r];
        Fx = P::from_fix(P::jx_of(J), a.fis);
        Fy = P::from_fix(P::jy_of(J), a.fis);
        Fz = P::from_fix(P::jz_of(J), a.fis);
        typename P::node4 zero;
        zero.x = zero.y = zero.z = zero.w = 0;
        a.jacc[r] = zero;
    }
    Fx += a.g[0];
    Fy += a.g[1];
    Fz += a.g[2];
    collide<T, RELAX_FULL, LbArgs<T, S>, GAUSS>(f, rho, rho_m, jx, jy, jz, Fx, Fy, Fz, a, a.key0, a.key1, r,
                                                (uint32_t)step);

    const int xm = x == 0 ? a.nx - 1 : x - 1, xp = x == a.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? a.ny - 1 : y - 1, yp = y == a.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? a.nz - 1 : z - 1, zp = z == a.nz - 1 ? 0 : z + 1;
    const int X[3] = {xm, x, xp}, Y[3] = {ym, y, yp}, Z[3] = {zm, z, zp};
    if constexpr (St::stochastic) {
        // stochastic rounding of the stored deviations: 16 random bits per
        // population from Philox stream 2 of (node, LB step), population i
        // from call i / 8, word (i / 2) mod 4, low half for even i
        U4 rb{0u, 0u, 0u, 0u};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if ((i & 7) == 0) rb = philox4x32_10(U4{r, (uint32_t)step, 2u, (uint32_t)(i >> 3)}, a.key0, a.key1);
            const uint32_t w = ((i >> 1) & 3) == 0 ? rb.x : ((i >> 1) & 3) == 1 ? rb.y : ((i >> 1) & 3) == 2 ? rb.z : rb.w;
            const uint32_t t = (uint32_t)X[CX(i) + 1] +
                               (uint32_t)a.nx * ((uint32_t)Y[CY(i) + 1] + (uint32_t)a.ny * (uint32_t)Z[CZ(i) + 1]);
            St::store_arith_sr(a.fout + (size_t)i * a.N + t, f[i], (i & 1) ? w >> 16 : w & 0xffffu);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const uint32_t t = (uint32_t)X[CX(i) + 1] +
                               (uint32_t)a.nx * ((uint32_t)Y[CY(i) + 1] + (uint32_t)a.ny * (uint32_t)Z[CZ(i) + 1]);
            St::store_arith(a.fout + (size_t)i * a.N + t, f[i]);
        }
    }
}

// Resident blocks per SM the compiler plans registers for: 7 (32 registers)
// for the forms with full relaxation, uniform noise and FP32 or
// rounded-to-nearest 16-bit storage, measured faster than 6 (40 registers)
// despite their spills: FP32 cycle -0.8 %, FP16 / BF16 LB step -6.5 % /
// -4.3 %; the stochastic-rounding form measured slower at 7, and it and the
// Gaussian-noise and partial-relaxation forms keep 6 (3 in FP64).
template <typename T, typename S, bool RELAX_FULL, bool GAUSS>
constexpr int collide_min_blocks() {
    return sizeof(T) == 8 ? 3 : (RELAX_FULL && !GAUSS && !PopStore<S, T>::stochastic ? 7 : 6);
}

template <typename T, typename S, bool RELAX_FULL, bool GAUSS>
__global__ void __launch_bounds__(256, (collide_min_blocks<T, S, RELAX_FULL, GAUSS>())) lb_collide_push(LbArgs<T, S> a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    // the step counter, read before the fallback kernel advances it; it also
    // tags the blocks that have pushed
    const unsigned long long step = *a.lb_step;
    if (x < a.nx) collide_push_node<T, S, RELAX_FULL, GAUSS>(a, x, y, z, step);

    // fused post-stream moments: publish this block, then compute the
    // moments of the block FUSE_LAG planes back once its neighbourhood is in
    const uint32_t gx = gridDim.x, gy = gridDim.y;
    const uint32_t epoch = (uint32_t)step + 1u;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(&a.blk_done[blockIdx.x + gx * (blockIdx.y + gy * blockIdx.z)], epoch);
    }
    const int t = z - FUSE_LAG;
    if (t < 1) return;
    __shared__ int s_ok;
    if (threadIdx.x < 32) {
        bool ok = a.spin > 0;
        if (ok && threadIdx.x < 27) {
            const int dx = (int)threadIdx.x % 3 - 1, dy = ((int)threadIdx.x / 3) % 3 - 1;
            const int dz = (int)threadIdx.x / 9 - 1;
            const uint32_t xb = (blockIdx.x + gx + dx) % gx, yb = (uint32_t)((y + a.ny + dy) % a.ny);
            const volatile uint32_t *flag = a.blk_done + xb + gx * (yb + gy * (uint32_t)(t + dz));
            int polls = 0;
            while (*flag != epoch) {
                if (++polls > a.spin) {
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (threadIdx.x == 0) {
            __threadfence();
            s_ok = ok ? 1 : 0;
        }
    }
    __syncthreads();
    if (!s_ok) {
        if (threadIdx.x == 0) a.missed_list[atomicAdd(a.missed, 1)] = (int32_t)(blockIdx.x + gx * (y + gy * t));
        return;
    }
    if (x < a.nx)
        node_moments_at<T, S>(a.fout, a.node, a.occw_new, a.cact_new, a.cact_new2, a.occ_words, a.N, a.nx, a.ny,
                              a.rho_base, a.fs, a.range_flag, x, y, t);
}

// The moments the collide kernel left: node rows of plane 0 and of the last
// FUSE_LAG planes, and the rows whose wait ran out (counted into
// missed_total); then the LB step counter advances.
template <typename T, typename S>
__global__ void __launch_bounds__(256)
    moments_rest_kernel(const S *__restrict__ f, typename Prec<T>::node4 *node, const uint2 *occw,
                        typename Prec<T>::node4 *cact, typename Prec<T>::node4 *cact2, int occ_words, int64_t N,
                        int nx, int ny, int nz, T rho_base, T fs, int32_t *range_flag, const int32_t *missed, const int32_t *missed_list,
                        unsigned long long *missed_total, unsigned long long *lb_step) {
    const int gx = (nx + (int)blockDim.x - 1) / (int)blockDim.x;
    const int rows = gx * ny;
    // boundary planes: 0 and max(1, nz - FUSE_LAG) .. nz - 1
    const int first_tail = nz - FUSE_LAG > 1 ? nz - FUSE_LAG : 1;
    const int n_planes = 1 + (nz - first_tail);
    const int n_boundary = n_planes * rows;
    const int total = n_boundary + *missed;
    for (int i = blockIdx.x; i < total; i += gridDim.x) {
        int b;
        if (i < n_boundary) {
            const int k = i / rows;
            const int plane = k == 0 ? 0 : first_tail + (k - 1);
            b = i - k * rows + plane * rows;
        } else {
            b = missed_list[i - n_boundary];
        }
        const int xb = b % gx, rest = b / gx, y = rest % ny, t = rest / ny;
        const int x = xb * (int)blockDim.x + (int)threadIdx.x;
        if (x < nx)
            node_moments_at<T, S>(f, node, occw, cact, cact2, occ_words, N, nx, ny, rho_base, fs, range_flag, x, y,
                                  t);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *missed_total += (unsigned long long)*missed;
        *lb_step += 1ull;
    }
}

template <typename T, typename S>
__global__ void __launch_bounds__(256)
    node_moments_kernel(const S *__restrict__ f, typename Prec<T>::node4 *node, const uint2 *occw,
                        typename Prec<T>::node4 *cact, typename Prec<T>::node4 *cact2, int occ_words, int64_t N,
                        int nx, int ny, T rho_base, T fs, int32_t *range_flag) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    node_moments_at<T, S>(f, node, occw, cact, cact2, occ_words, N, nx, ny, rho_base, fs, range_flag, x, blockIdx.y,
                          blockIdx.z);
}

// Variant C (Sec. 4): the momentum transfer F = J_acc of the MD step just
// done enters the populations through the forcing part of the collision
// alone: mass unchanged, momentum + F, stress modes + (1 + gamma) times the
// symmetric products of u = (j + F/2)/rho and F (as in collide()), ghost
// modes unchanged; then the node record is recomputed from the populations
// and J_acc is cleared.  Nodes without a transfer are left as they are.
template <typename T, typename S>
__global__ void __launch_bounds__(256) forcing_update_kernel(S *__restrict__ f, typename Prec<T>::node4 *node,
                                                             typename Prec<T>::node4 *jacc, int64_t N, T rho_base,
                                                             T gamma_bulk, T gamma_shear, T fix_s, T fix_is,
                                                             int32_t *range_flag) {
    using P = Prec<T>;
    using St = PopStore<S, T>;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const typename P::node4 J = jacc[r];
    if (P::jx_of(J) == 0 && P::jy_of(J) == 0 && P::jz_of(J) == 0) return;
    const T Fx = P::from_fix(P::jx_of(J), fix_is), Fy = P::from_fix(P::jy_of(J), fix_is),
            Fz = P::from_fix(P::jz_of(J), fix_is);
    T fl[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fl[i] = St::arith(f + (int64_t)i * N + r);
    T rho, rho_m, jx, jy, jz;
    pop_moments<St::deviation>(fl, rho_base, rho, rho_m, jx, jy, jz);
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
        St::store_arith(f + (int64_t)i * N + r, fl[i]);
    }
    pop_moments<St::deviation>(fl, rho_base, rho, rho_m, jx, jy, jz);
    node[r] = guarded_record(rho, jx, jy, jz, fix_s, range_flag);
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

// Deviation storage: the density of the stored rest values, sum_i b_i with
// b_i = w_i rho0 formed in T as the kernels form it (0 for the plain forms,
// whose arithmetic is on the populations themselves).
template <typename T, typename S>
static T rest_density(const lbmd_ctx *ctx) {
    if (!PopStore<S, T>::deviation) return T(0);
    double sum = 0.0;
    for (int i = 0; i < Q; ++i) sum += (double)(T(WEIGHT(i)) * (T)ctx->p.rho0);
    return (T)sum;
}

template <typename T, typename S>
static cudaError_t lb_step_t(lbmd_ctx *ctx) {
    LbArgs<T, S> a;
    a.fin = static_cast<const S *>(ctx->f[ctx->cur]);
    a.fout = static_cast<S *>(ctx->f[ctx->cur ^ 1]);
    a.rho_base = rest_density<T, S>(ctx);
    a.node = static_cast<typename Prec<T>::node4 *>(ctx->node);
    a.jacc = static_cast<typename Prec<T>::node4 *>(ctx->jacc);
    const bool B = compact_nodes(ctx);  // variants A and B
    a.occw = B ? active_words_now(ctx) : nullptr;
    a.cact = static_cast<const typename Prec<T>::node4 *>(B ? active_records_acc(ctx) : nullptr);
    a.occw_new = B ? active_words_next(ctx) : nullptr;
    a.cact_new = static_cast<typename Prec<T>::node4 *>(B ? active_records_next(ctx) : nullptr);
    a.cact_new2 = static_cast<typename Prec<T>::node4 *>(active_records_copy(ctx, (int)((ctx->lb_step + 1) & 1)));
    a.occ_words = active_words(ctx->p.nx);
    a.blk_done = ctx->blk_done;
    a.missed = ctx->lb_missed;
    a.missed_list = ctx->missed_list;
    a.spin = ctx->fuse_spin;
    a.fs = (T)ctx->fix.scale;
    a.fis = (T)ctx->fix.inv_scale;
    a.range_flag = ctx->range_flag;
    a.nx = ctx->p.nx;
    a.ny = ctx->p.ny;
    a.nz = ctx->p.nz;
    a.N = ctx->N;
    a.gamma_bulk = (T)ctx->co.gamma_bulk;
    a.gamma_shear = (T)ctx->co.gamma_shear;
    a.gamma_ghost = (T)ctx->co.gamma_ghost;
    for (int k = 0; k < Q; ++k) {
        a.amp16[k] = (T)(ctx->co.noise_amp[k] * 3.4641016151377544 * 1.52587890625e-05);
        a.ampg[k] = (T)ctx->co.noise_amp[k];
    }
    for (int d = 0; d < 3; ++d) a.g[d] = (T)ctx->co.body_force[d];
    a.key0 = (uint32_t)(ctx->p.seed & 0xffffffffu);
    a.key1 = (uint32_t)(ctx->p.seed >> 32);
    a.lb_step = ctx->d_lb_step;
    a.noisy = ctx->co.noisy;
    a.variant = ctx->p.variant;
    const dim3 block = node_block(ctx), grid = node_grid(ctx, block);
    cudaError_t e = cudaMemsetAsync(ctx->lb_missed, 0, sizeof(int32_t), ctx->stream);
    if (e != cudaSuccess) return e;
    const bool full = ctx->co.gamma_bulk == 0.0 && ctx->co.gamma_ghost == 0.0;
    // normal variates: a kernel instance of its own (FP32 / FP64 storage),
    // so that the default one keeps its registers
    if constexpr (!PopStore<S, T>::deviation) {
        if (ctx->p.noise == LBMD_NOISE_GAUSS) {
            if (full)
                lb_collide_push<T, S, true, true><<<grid, block, 0, ctx->stream>>>(a);
            else
                lb_collide_push<T, S, false, true><<<grid, block, 0, ctx->stream>>>(a);
        }
    }
    if (ctx->p.noise != LBMD_NOISE_GAUSS) {
        if (full)
            lb_collide_push<T, S, true, false><<<grid, block, 0, ctx->stream>>>(a);
        else
            lb_collide_push<T, S, false, false><<<grid, block, 0, ctx->stream>>>(a);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the moments the collide kernel left, on the new populations
    moments_rest_kernel<T, S><<<2 * ctx->sm_count, block, 0, ctx->stream>>>(
        a.fout, a.node, a.occw_new, a.cact_new, a.cact_new2, a.occ_words, ctx->N, ctx->p.nx, ctx->p.ny, ctx->p.nz,
        a.rho_base,
        a.fs, ctx->range_flag, ctx->lb_missed, ctx->missed_list, ctx->missed_total, ctx->d_lb_step);
    return cudaGetLastError();
}

// node field (and the current active nodes' records) of the current
// populations, outside the LB step (creation, replaced populations)
template <typename T, typename S>
static cudaError_t node_moments_t(lbmd_ctx *ctx) {
    const dim3 block = node_block(ctx), grid = node_grid(ctx, block);
    const bool B = compact_nodes(ctx);  // variants A and B
    node_moments_kernel<T, S><<<grid, block, 0, ctx->stream>>>(
        static_cast<const S *>(ctx->f[ctx->cur]), static_cast<typename Prec<T>::node4 *>(ctx->node),
        B ? active_words_now(ctx) : nullptr,
        static_cast<typename Prec<T>::node4 *>(B ? active_records_now(ctx) : nullptr),
        static_cast<typename Prec<T>::node4 *>(active_records_copy(ctx, (int)(ctx->lb_step & 1))),
        active_words(ctx->p.nx), ctx->N, ctx->p.nx, ctx->p.ny, rest_density<T, S>(ctx), (T)ctx->fix.scale,
        ctx->range_flag);
    return cudaGetLastError();
}

template <typename T, typename S>
static cudaError_t forcing_update_t(lbmd_ctx *ctx) {
    const unsigned blocks = (unsigned)((ctx->N + 255) / 256);
    forcing_update_kernel<T, S><<<blocks, 256, 0, ctx->stream>>>(
        static_cast<S *>(ctx->f[ctx->cur]), static_cast<typename Prec<T>::node4 *>(ctx->node),
        static_cast<typename Prec<T>::node4 *>(ctx->jacc), ctx->N, rest_density<T, S>(ctx), (T)ctx->co.gamma_bulk,
        (T)ctx->co.gamma_shear, (T)ctx->fix.scale, (T)ctx->fix.inv_scale, ctx->range_flag);
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
#define LBMD_DISPATCH_POPS(ctx, FN, ...)                                                      \
    ((ctx)->p.precision == LBMD_FP64          ? FN<double, double>(__VA_ARGS__)               \
     : (ctx)->p.precision == LBMD_FP16_DEV    ? FN<float, __half>(__VA_ARGS__)                \
     : (ctx)->p.precision == LBMD_BF16_DEV    ? FN<float, __nv_bfloat16>(__VA_ARGS__)         \
     : (ctx)->p.precision == LBMD_FP16_DEV_SR ? FN<float, lbmd::half_sr>(__VA_ARGS__)         \
     : (ctx)->p.precision == LBMD_BF16_DEV_SR ? FN<float, lbmd::bf16_sr>(__VA_ARGS__)         \
                                              : FN<float, float>(__VA_ARGS__))

// One LB update: re-order the particles by row and build the active nodes of
// the coming cycle (variant B; the particles do not move during the LB
// step), then collide and stream with the post-stream moments fused in
// (node field and the new active nodes' compact records).
cudaError_t launch_lb_step(lbmd_ctx *ctx) {
    cudaError_t e = launch_sort_particles(ctx);
    if (e != cudaSuccess) return e;
    if ((e = launch_nb_build(ctx)) != cudaSuccess) return e;
    if ((e = launch_active_set(ctx)) != cudaSuccess) return e;
    if ((e = md_tile_build_table(ctx, (int)((ctx->lb_step + 1) & 1))) != cudaSuccess) return e;
    if ((e = LBMD_DISPATCH_POPS(ctx, lbmd::lb_step_t, ctx)) != cudaSuccess) return e;
    ctx->cur ^= 1;
    ctx->rec = 0;  // the moments wrote the next set's first record buffer
    return cudaSuccess;
}

cudaError_t launch_node_moments(lbmd_ctx *ctx, bool) { return LBMD_DISPATCH_POPS(ctx, lbmd::node_moments_t, ctx); }

cudaError_t launch_init_equilibrium(lbmd_ctx *ctx) { return LBMD_DISPATCH_POPS(ctx, lbmd::init_equilibrium_t, ctx); }

cudaError_t launch_forcing_update(lbmd_ctx *ctx) { return LBMD_DISPATCH_POPS(ctx, lbmd::forcing_update_t, ctx); }
