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
// the next LB cycle read (and, in variant B, update).
#include "lbmd_ctx.h"
#include "lbmd_device.cuh"

namespace lbmd {

template <typename T>
struct LbArgs {
    const T *__restrict__ fin;
    T *__restrict__ fout;
    typename Prec<T>::node4 *node;
    typename Prec<T>::node4 *jacc;
    int nx, ny, nz;
    int64_t N;
    T gamma_bulk, gamma_shear, gamma_ghost;
    T amp[Q];
    T g[3];
    uint32_t key0, key1;
    const unsigned long long *lb_step;
    int noisy;
};

// Reciprocal norms 1/b_k, exact binary fractions.
__host__ __device__ constexpr double INV_BNORM(int k) {
    constexpr double t[Q] = {1.0, 3.0, 3.0, 3.0, 1.5, 0.75, 2.25, 9.0, 9.0, 9.0,
                             1.5, 1.5, 1.5, 4.5, 4.5, 4.5, 0.5, 0.75, 2.25};
    return t[k];
}

// MRT collision with forcing and noise at one node; f holds f* on entry and
// f' on exit.
template <typename T>
__device__ __forceinline__ void collide(T f[Q], T rho, T jx, T jy, T jz, T Fx, T Fy, T Fz, const LbArgs<T> &a,
                                        uint32_t node, uint32_t step) {
    const T inv_rho = T(1) / rho;
    const T ux = (jx + T(0.5) * Fx) * inv_rho;
    const T uy = (jy + T(0.5) * Fy) * inv_rho;
    const T uz = (jz + T(0.5) * Fz) * inv_rho;
    const T uu = ux * ux + uy * uy + uz * uz;
    const T uF = ux * Fx + uy * Fy + uz * Fz;

    // non-conserved moments m_k = sum_i e_k(c_i) f_i, k = 4..18
    T m[Q];
#pragma unroll
    for (int k = 4; k < Q; ++k) {
        T acc = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (EMODE(k, i) != 0) acc += T(EMODE(k, i)) * f[i];
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
        const T sr = sqrt(rho);
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q) {
            const U4 r = philox4x32_10(U4{node, step, 0u, q}, a.key0, a.key1);
            const uint32_t bits[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int k = 4 + 4 * (int)q + t;
                if (k < Q) mp[k] += a.amp[k] * sr * unit_uniform<T>(bits[t]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) mp[k] *= T(INV_BNORM(k));
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < Q; ++k)
            if (EMODE(k, i) != 0) acc += T(EMODE(k, i)) * mp[k];
        f[i] = T(WEIGHT(i)) * acc;
    }
}

template <typename T, int VARIANT>
__global__ void __launch_bounds__(256) lb_collide_push(LbArgs<T> a) {
    using P = Prec<T>;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.N) return;
    T f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = a.fin[(int64_t)i * a.N + r];
    T rho, jx, jy, jz;
    node_moments(f, rho, jx, jy, jz);
    T Fx, Fy, Fz;
    if (VARIANT == LBMD_VARIANT_B) {
        // node j = fix(j*) + sum of fixed-point transfers: the difference is
        // exactly the accumulated transfer J_acc
        const typename P::node4 n = a.node[r];
        Fx = P::from_fix(n.y - P::to_fix(jx));
        Fy = P::from_fix(n.z - P::to_fix(jy));
        Fz = P::from_fix(n.w - P::to_fix(jz));
    } else {
        const typename P::node4 J = a.jacc[r];
        Fx = P::from_fix(J.y);
        Fy = P::from_fix(J.z);
        Fz = P::from_fix(J.w);
        typename P::node4 zero;
        zero.x = zero.y = zero.z = zero.w = 0;
        a.jacc[r] = zero;
    }
    Fx += a.g[0];
    Fy += a.g[1];
    Fz += a.g[2];
    collide(f, rho, jx, jy, jz, Fx, Fy, Fz, a, (uint32_t)r, (uint32_t)(*a.lb_step));

    const int64_t nxy = (int64_t)a.nx * a.ny;
    const int z = (int)(r / nxy);
    const int64_t rem = r - (int64_t)z * nxy;
    const int y = (int)(rem / a.nx);
    const int x = (int)(rem - (int64_t)y * a.nx);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int xn = x + CX(i), yn = y + CY(i), zn = z + CZ(i);
        xn = xn < 0 ? a.nx - 1 : (xn == a.nx ? 0 : xn);
        yn = yn < 0 ? a.ny - 1 : (yn == a.ny ? 0 : yn);
        zn = zn < 0 ? a.nz - 1 : (zn == a.nz ? 0 : zn);
        a.fout[(int64_t)i * a.N + xn + a.nx * ((int64_t)yn + (int64_t)a.ny * zn)] = f[i];
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
    node_moments_kernel(const T *__restrict__ f, typename Prec<T>::node4 *node, int64_t N, unsigned long long *lb_step,
                        int count_step) {
    using P = Prec<T>;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (count_step && r == 0) *lb_step += 1ull;
    if (r >= N) return;
    T fl[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fl[i] = f[(int64_t)i * N + r];
    T rho, jx, jy, jz;
    node_moments(fl, rho, jx, jy, jz);
    node[r] = P::pack(rho, P::to_fix(jx), P::to_fix(jy), P::to_fix(jz));
}

template <typename T>
__global__ void init_equilibrium_kernel(T *f, int64_t N, T rho0) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) f[(int64_t)i * N + r] = T(WEIGHT(i)) * rho0;
}

template <typename T>
static cudaError_t lb_step_t(lbmd_ctx *ctx) {
    LbArgs<T> a;
    a.fin = static_cast<const T *>(ctx->f[ctx->cur]);
    a.fout = static_cast<T *>(ctx->f[ctx->cur ^ 1]);
    a.node = static_cast<typename Prec<T>::node4 *>(ctx->node);
    a.jacc = static_cast<typename Prec<T>::node4 *>(ctx->jacc);
    a.nx = ctx->p.nx;
    a.ny = ctx->p.ny;
    a.nz = ctx->p.nz;
    a.N = ctx->N;
    a.gamma_bulk = (T)ctx->co.gamma_bulk;
    a.gamma_shear = (T)ctx->co.gamma_shear;
    a.gamma_ghost = (T)ctx->co.gamma_ghost;
    for (int k = 0; k < Q; ++k) a.amp[k] = (T)ctx->co.noise_amp[k];
    for (int d = 0; d < 3; ++d) a.g[d] = (T)ctx->co.body_force[d];
    a.key0 = (uint32_t)(ctx->p.seed & 0xffffffffu);
    a.key1 = (uint32_t)(ctx->p.seed >> 32);
    a.lb_step = ctx->d_lb_step;
    a.noisy = ctx->co.noisy;
    const unsigned blocks = (unsigned)((ctx->N + 255) / 256);
    if (ctx->p.variant == LBMD_VARIANT_B)
        lb_collide_push<T, LBMD_VARIANT_B><<<blocks, 256, 0, ctx->stream>>>(a);
    else
        lb_collide_push<T, LBMD_VARIANT_A><<<blocks, 256, 0, ctx->stream>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t node_moments_t(lbmd_ctx *ctx, bool count_step) {
    const unsigned blocks = (unsigned)((ctx->N + 255) / 256);
    node_moments_kernel<T><<<blocks, 256, 0, ctx->stream>>>(static_cast<const T *>(ctx->f[ctx->cur]),
                                                             static_cast<typename Prec<T>::node4 *>(ctx->node),
                                                             ctx->N, ctx->d_lb_step, count_step ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t init_equilibrium_t(lbmd_ctx *ctx) {
    const unsigned blocks = (unsigned)((ctx->N + 255) / 256);
    init_equilibrium_kernel<T><<<blocks, 256, 0, ctx->stream>>>(static_cast<T *>(ctx->f[ctx->cur]), ctx->N,
                                                                 (T)ctx->p.rho0);
    return cudaGetLastError();
}

}  // namespace lbmd

cudaError_t launch_lb_step(lbmd_ctx *ctx) {
    cudaError_t e = ctx->p.precision == LBMD_FP64 ? lbmd::lb_step_t<double>(ctx) : lbmd::lb_step_t<float>(ctx);
    if (e != cudaSuccess) return e;
    ctx->cur ^= 1;
    return launch_node_moments(ctx, true);
}

cudaError_t launch_node_moments(lbmd_ctx *ctx, bool count_step) {
    return ctx->p.precision == LBMD_FP64 ? lbmd::node_moments_t<double>(ctx, count_step)
                                         : lbmd::node_moments_t<float>(ctx, count_step);
}

cudaError_t launch_init_equilibrium(lbmd_ctx *ctx) {
    return ctx->p.precision == LBMD_FP64 ? lbmd::init_equilibrium_t<double>(ctx)
                                         : lbmd::init_equilibrium_t<float>(ctx);
}
