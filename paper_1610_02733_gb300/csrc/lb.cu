// lb.cu -- the lattice Boltzmann update (Sec. 2, Eq. (3)) on the GPU.
//
// lb_collide_push: one thread per node.  Reads the 19 post-stream populations
// f*_i (coalesced structure-of-arrays loads), the momentum the particles
// handed over since the last LB step, and applies the MRT collision in moment
// space with thermal noise (Philox in registers) and the forcing term of the
// force density F = J_acc / tau_LB + g; the post-collision populations are
// pushed to the neighbours r + c_i in the other buffer.
//
// node_moments_kernel: one thread per node.  Recomputes rho* and j* of the
// freshly streamed populations and writes the node field that the MD steps of
// the next LB cycle read (and, in variant B, update); in variant B also the
// compact record of every active node.
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

// Reciprocal norms 1/b_k, exact binary fractions.
__host__ __device__ constexpr double INV_BNORM(int k) {
    constexpr double t[Q] = {1.0, 3.0, 3.0, 3.0, 1.5, 0.75, 2.25, 9.0, 9.0, 9.0,
                             1.5, 1.5, 1.5, 4.5, 4.5, 4.5, 0.5, 0.75, 2.25};
    return t[k];
}

// The D3Q19 order pairs every moving velocity with its opposite:
// c_{2p+2} = -c_{2p+1}, p = 0..8.  Even modes (0, 4-9, 16-18) see only the
// pair sums s_p = f_{2p+1} + f_{2p+2}, odd modes (1-3, 10-15) only the
// differences d_p = f_{2p+1} - f_{2p+2}; the back-transform likewise returns
// an even part E_p and an odd part O_p with f_{2p+1} = w (E_p + O_p) and
// f_{2p+2} = w (E_p - O_p).  This halves the arithmetic of both transforms.
__host__ __device__ constexpr bool EVEN_MODE(int k) { return k == 0 || (k >= 4 && k <= 9) || k >= 16; }

// MRT collision with forcing and noise at one node; f holds f* on entry and
// f' on exit.
// 1/rho and sqrt(rho): IEEE in FP64; in FP32 both from one reciprocal square
// root (at most a few ulp, far below the FP32 path's tolerance)
__device__ __forceinline__ void rho_factors(double rho, double &inv, double &sq) {
    inv = 1.0 / rho;
    sq = sqrt(rho);
}
__device__ __forceinline__ void rho_factors(float rho, float &inv, float &sq) {
    const float r = rsqrtf(rho);
    inv = r * r;
    sq = rho * r;
}

// (h - 32767.5) for a 16-bit h, exactly: FP32 builds 2^23 + h from its bit
// pattern (no int-to-float conversion), removes 2^23 and then 32767.5 (both
// subtractions exact); FP64 converts.
__device__ __forceinline__ float centred16(uint32_t h, float) {
    return (__int_as_float((int)(0x4B000000u | h)) - 8388608.0f) - 32767.5f;
}
__device__ __forceinline__ double centred16(uint32_t h, double) { return (double)h - 32767.5; }

// RELAX_FULL: gamma_bulk = gamma_ghost = 0 (the default reading), so the
// bulk and ghost modes relax fully, m'_k = m^eq_k exactly, and their moments
// m_k need not be computed (gamma (m - m^eq) is +-0 for finite m).
template <typename T, typename S, bool RELAX_FULL>
__device__ __forceinline__ void collide(T f[Q], T rho, T jx, T jy, T jz, T Fx, T Fy, T Fz, const LbArgs<T, S> &a,
                                        uint32_t node, uint32_t step) {
    T inv_rho, sr;
    rho_factors(rho, inv_rho, sr);
    const T ux = (jx + T(0.5) * Fx) * inv_rho;
    const T uy = (jy + T(0.5) * Fy) * inv_rho;
    const T uz = (jz + T(0.5) * Fz) * inv_rho;
    const T uu = ux * ux + uy * uy + uz * uz;
    const T uF = ux * Fx + uy * Fy + uz * Fz;

    T s[9], d[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        s[p] = f[2 * p + 1] + f[2 * p + 2];
        d[p] = f[2 * p + 1] - f[2 * p + 2];
    }
    // non-conserved moments m_k = sum_i e_k(c_i) f_i, k = 4..18
    T m[Q];
#pragma unroll
    for (int k = 4; k < Q; ++k) {
        T acc = T(0);
        if (EVEN_MODE(k) && EMODE(k, 0) != 0) acc = T(EMODE(k, 0)) * f[0];
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            const int e = EMODE(k, 2 * p + 1);
            if (e != 0) acc += T(e) * (EVEN_MODE(k) ? s[p] : d[p]);
        }
        m[k] = acc;
    }
    // equilibria of the stress modes (ghost equilibria vanish)
    T meq[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) meq[k] = T(0);
    meq[4] = rho * uu;
    meq[5] = rho * (T(3) * ux * ux - uu);
    meq[6] = rho * (uy * uy - uz * uz);
    meq[7] = rho * ux * uy;
    meq[8] = rho * ux * uz;
    meq[9] = rho * uy * uz;

    T mp[Q];
    mp[0] = rho;
    mp[1] = jx + Fx;
    mp[2] = jy + Fy;
    mp[3] = jz + Fz;
#pragma unroll
    for (int k = 4; k < Q; ++k) {
        if (RELAX_FULL && (k == 4 || k >= 10)) {
            mp[k] = meq[k];
            continue;
        }
        const T gk = k == 4 ? a.gamma_bulk : (k <= 9 ? a.gamma_shear : a.gamma_ghost);
        mp[k] = meq[k] + gk * (m[k] - meq[k]);
    }
    const T fb = T(1) + a.gamma_bulk, fs = T(1) + a.gamma_shear;
    mp[4] += fb * uF;
    mp[5] += fs * (T(3) * ux * Fx - uF);
    mp[6] += fs * (uy * Fy - uz * Fz);
    mp[7] += fs * T(0.5) * (ux * Fy + uy * Fx);
    mp[8] += fs * T(0.5) * (ux * Fz + uz * Fx);
    mp[9] += fs * T(0.5) * (uy * Fz + uz * Fy);

    if (a.noisy) {
        // 15 variates from two Philox calls: two 16-bit halves per 32-bit
        // word, low half first, in mode order k = 4..18.  The variate
        // sqrt(12) ((h + 1/2) 2^-16 - 1/2) is (h - 32767.5) times
        // sqrt(12) 2^-16, folded into amp16[k] = amp[k] sqrt(12) 2^-16.
#pragma unroll
        for (uint32_t q = 0; q < 2; ++q) {
            const U4 r = philox4x32_10(U4{node, step, 0u, q}, a.key0, a.key1);
            const uint32_t bits[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int k = 4 + 8 * (int)q + t;
                const uint32_t h = (t & 1) ? (bits[t >> 1] >> 16) : (bits[t >> 1] & 0xffffu);
                if (k < Q) mp[k] += (a.amp16[k] * sr) * centred16(h, T(0));
            }
        }
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) mp[k] *= T(INV_BNORM(k));
    {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < Q; ++k)
            if (EVEN_MODE(k) && EMODE(k, 0) != 0) acc += T(EMODE(k, 0)) * mp[k];
        f[0] = T(WEIGHT(0)) * acc;
    }
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        T ev = T(0), od = T(0);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int e = EMODE(k, 2 * p + 1);
            if (e == 0) continue;
            if (EVEN_MODE(k))
                ev += T(e) * mp[k];
            else
                od += T(e) * mp[k];
        }
        const T w = T(WEIGHT(2 * p + 1));
        f[2 * p + 1] = w * (ev + od);
        f[2 * p + 2] = w * (ev - od);
    }
}

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
    collide<T, S, RELAX_FULL>(f, rho, jx, jy, jz, Fx, Fy, Fz, a, r, (uint32_t)(*a.lb_step));

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
