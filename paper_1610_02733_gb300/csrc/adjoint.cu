// adjoint.cu -- hand-written adjoint (reverse-mode derivative) of the coupled
// LB/MD step, variant B, for the mean particle drag along x:
//     L = (1 / (K m N_p)) sum over the K m MD steps and the N_p particles of
//         the coupling force F_x of Eq. (4),
// with respect to the friction coefficient zeta and the initial particle
// positions.  The random numbers are fixed by their Philox counters, so the
// map is deterministic (kT = 0 or kT > 0 alike); only the noise amplitudes
// depend on the inputs (sqrt(rho) in the fluid, sqrt(zeta) on the particles).
//
// Forward: K cycles (m MD steps + one LB step each) from the fluid at rest,
// keeping the populations and the particle state at the start of every cycle
// (checkpoint per LB step) and the drag of every particle and MD step.
// Backward, cycle by cycle from the last: recompute the cycle's m MD steps
// from its checkpoint, recording what the reverse steps need (positions,
// velocities, forces, the interpolated velocity and the 8 corner records),
// then
//   1. the adjoint of the LB step: pull the adjoint populations back along
//      the streaming (the transpose of the push), add the adjoint of the next
//      cycle's node moments (Eqs. (1), (2)), and apply the transposed
//      Jacobian of the collision in moment space (relaxation, equilibria and
//      forcing in u = (j + F/2)/rho, noise in sqrt(rho)); the force density
//      F = J_acc + g with J_acc = j_node - j* hands its adjoint to the node
//      momentum after the last MD step and (with a minus sign) to the
//      populations;
//   2. the adjoints of the MD steps, last first: per particle the transposed
//      velocity Verlet (F held over the step), friction (Eq. (4)), trilinear
//      interpolation (Eq. (5)) and transfer (Eqs. (7), (8)), then the
//      scatter of the node adjoints (momentum and density at the 8 corners)
//      with atomics, once every particle has read them;
//   3. the node adjoints at the start of the cycle are the adjoint of that
//      cycle's moments, folded into the pull of the previous cycle.
// The trilinear weights are piecewise linear in the position: the map has
// kinks where a particle crosses a cell face, and the derivative is that of
// the piece the particle is on.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lb_core.cuh"
#include "lbmd_ctx.h"
#include "lbmd_device.cuh"
#include "particle_core.cuh"

namespace lbmd {

template <typename T>
struct AdArgs {
    int nx, ny, nz, np, n_sub;
    int64_t N;
    FastDiv fd_nx, fd_ny;
    T zeta, dt, half_dt, amp, neg_scale_dt, norm;
    T fs, fis;  // fixed-point scale of the momentum density and its inverse
    uint32_t key0, key1;
    T g[3];
    // read by collide()
    T gamma_bulk, gamma_shear, gamma_ghost;
    T amp16[Q];
    int noisy;
    T gam[Q];  // relaxation factor per mode (0-3 unused)
};

// What the reverse MD step needs, per MD step of the cycle and particle.
template <typename T>
struct AdRec {
    typename Prec<T>::real4 *R, *V, *F, *U;  // start position (frac, cell), velocity (v, 1/m), force, u(R)
    typename Prec<T>::real4 *C;              // 8 per particle: (rho_k, j_k) of the corners
};

template <typename T>
__global__ void ad_init_kernel(T *f, int64_t N, T rho0) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) f[(int64_t)i * N + r] = T(WEIGHT(i)) * rho0;
}

template <typename T>
__global__ void ad_moments_kernel(const T *f, typename Prec<T>::node4 *node, int64_t N, T fs) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    T fl[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fl[i] = f[(int64_t)i * N + r];
    T rho, jx, jy, jz;
    node_moments(fl, rho, jx, jy, jz);
    using P = Prec<T>;
    node[r] = P::pack(rho, P::to_fix(jx, fs), P::to_fix(jy, fs), P::to_fix(jz, fs));
}

template <typename T>
__device__ __forceinline__ void node_xyz(const AdArgs<T> &a, int64_t r, int &x, int &y, int &z) {
    const uint32_t u = (uint32_t)r;
    const uint32_t row = fdiv(u, a.fd_nx);
    x = (int)(u - row * a.fd_nx.d);
    z = (int)fdiv(row, a.fd_ny);
    y = (int)(row - (uint32_t)z * a.fd_ny.d);
}

template <typename T>
__device__ __forceinline__ int64_t neighbour(const AdArgs<T> &a, int x, int y, int z, int i) {
    int xn = x + CX(i), yn = y + CY(i), zn = z + CZ(i);
    xn = xn < 0 ? a.nx - 1 : (xn == a.nx ? 0 : xn);
    yn = yn < 0 ? a.ny - 1 : (yn == a.ny ? 0 : yn);
    zn = zn < 0 ? a.nz - 1 : (zn == a.nz ? 0 : zn);
    return (int64_t)xn + (int64_t)a.nx * (yn + (int64_t)a.ny * zn);
}

// force density of the LB step at a node: J_acc + g, J_acc = j_node - fix(j*)
template <typename T>
__device__ __forceinline__ void node_force(const AdArgs<T> &a, const typename Prec<T>::node4 &n, T jx, T jy, T jz,
                                           T &Fx, T &Fy, T &Fz) {
    using P = Prec<T>;
    Fx = P::from_fix(P::jx_of(n) - P::to_fix(jx, a.fs), a.fis) + a.g[0];
    Fy = P::from_fix(P::jy_of(n) - P::to_fix(jy, a.fs), a.fis) + a.g[1];
    Fz = P::from_fix(P::jz_of(n) - P::to_fix(jz, a.fs), a.fis) + a.g[2];
}

// LB step of the forward pass: collide at every node and push into fout.
template <typename T, bool RELAX_FULL>
__global__ void __launch_bounds__(256) ad_collide_push(const T *fin, T *fout, const typename Prec<T>::node4 *node,
                                                       AdArgs<T> a, uint32_t step) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.N) return;
    int x, y, z;
    node_xyz(a, r, x, y, z);
    T f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = fin[(int64_t)i * a.N + r];
    T rho, jx, jy, jz, Fx, Fy, Fz;
    node_moments(f, rho, jx, jy, jz);
    node_force(a, node[r], jx, jy, jz, Fx, Fy, Fz);
    collide<T, RELAX_FULL>(f, rho, rho, jx, jy, jz, Fx, Fy, Fz, a, a.key0, a.key1, (uint32_t)r, step);
#pragma unroll
    for (int i = 0; i < Q; ++i) fout[(int64_t)i * a.N + neighbour(a, x, y, z, i)] = f[i];
}

// One MD step of every particle (Eqs. (4)-(6)); drag[p] = F_x; with a
// record, also what the reverse step needs.
template <typename T>
__global__ void __launch_bounds__(256) ad_couple(AdArgs<T> a, typename Prec<T>::real4 *pos4,
                                                 typename Prec<T>::real4 *vel4, typename Prec<T>::real4 *old4,
                                                 typename Prec<T>::real4 *fc4, const typename Prec<T>::node4 *node,
                                                 T *drag, AdRec<T> rec, uint32_t md_step) {
    using P = Prec<T>;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const typename P::real4 R = pos4[p];
    typename P::real4 V = vel4[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.fd_nx, a.fd_ny);
    uint32_t idx[8];
    T delta[8];
    corners(c, R.x, R.y, R.z, a.nx, a.ny, a.nz, idx, delta);
    T ux = T(0), uy = T(0), uz = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const typename P::node4 n = node[idx[k]];
        const T rho = P::rho_of(n), jx = P::from_fix(P::jx_of(n), a.fis), jy = P::from_fix(P::jy_of(n), a.fis),
                jz = P::from_fix(P::jz_of(n), a.fis);
        if (rec.C) rec.C[8 * p + k] = P::make4(rho, jx, jy, jz);
        const T w = delta[k] / rho;
        ux += w * jx;
        uy += w * jy;
        uz += w * jz;
    }
    T Fx = -a.zeta * (V.x - ux), Fy = -a.zeta * (V.y - uy), Fz = -a.zeta * (V.z - uz);
    if (a.amp != T(0)) {
        const U4 rnd = philox4x32_10(U4{(uint32_t)p, md_step, 1u, 0u}, a.key0, a.key1);
        Fx = fma(a.amp, unit_uniform<T>(rnd.x), Fx);
        Fy = fma(a.amp, unit_uniform<T>(rnd.y), Fy);
        Fz = fma(a.amp, unit_uniform<T>(rnd.z), Fz);
    }
    drag[p] = Fx;
    if (rec.R) {
        rec.R[p] = R;
        rec.V[p] = V;
        rec.F[p] = P::make4(Fx, Fy, Fz, T(0));
        rec.U[p] = P::make4(ux, uy, uz, T(0));
    }
    const T hm = a.half_dt * V.w;
    V.x = fma(hm, Fx, V.x);
    V.y = fma(hm, Fy, V.y);
    V.z = fma(hm, Fz, V.z);
    T fx = R.x, fy = R.y, fz = R.z;
    int cx = c.x, cy = c.y, cz = c.z;
    advance(fx, cx, a.dt, V.x, a.nx);
    advance(fy, cy, a.dt, V.y, a.ny);
    advance(fz, cz, a.dt, V.z, a.nz);
    V.x = fma(hm, Fx, V.x);
    V.y = fma(hm, Fy, V.y);
    V.z = fma(hm, Fz, V.z);
    pos4[p] = P::make_pos(fx, fy, fz, cx + (int64_t)a.nx * (cy + (int64_t)a.ny * cz));
    vel4[p] = V;
    old4[p] = R;
    fc4[p] = P::make4(Fx, Fy, Fz, T(0));
}

// Transfers of the MD step (Eqs. (7), (8)), after every particle read the nodes.
template <typename T>
__global__ void __launch_bounds__(256) ad_transfer(AdArgs<T> a, const typename Prec<T>::real4 *old4,
                                                   const typename Prec<T>::real4 *fc4,
                                                   typename Prec<T>::node4 *node) {
    using P = Prec<T>;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const typename P::real4 R = old4[p], F = fc4[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.fd_nx, a.fd_ny);
    uint32_t idx[8];
    T delta[8];
    corners(c, R.x, R.y, R.z, a.nx, a.ny, a.nz, idx, delta);
    spread_to<T>(node, idx, delta, F.x * a.neg_scale_dt, F.y * a.neg_scale_dt, F.z * a.neg_scale_dt);
}

// Adjoint of the LB step at node r.  gin_i = adjoint of f'_i(r): pulled from
// the next cycle's adjoint populations at r + c_i, plus the adjoint of that
// cycle's moments there.  Writes the adjoint of this cycle's f*(r) and, for
// the MD steps, the node adjoint (rho: 0, j: adjoint of F).
template <typename T>
__global__ void __launch_bounds__(128) ad_collide_adj(const T *fc, const typename Prec<T>::node4 *node_fin,
                                                      const T *fbar_next, const typename Prec<T>::real4 *nbar_next,
                                                      T *fbar, typename Prec<T>::real4 *nbar, AdArgs<T> a,
                                                      uint32_t step) {
    using P = Prec<T>;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.N) return;
    int x, y, z;
    node_xyz(a, r, x, y, z);
    T gin[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int64_t t = neighbour(a, x, y, z, i);
        const typename P::real4 nb = nbar_next[t];
        gin[i] = fbar_next[(int64_t)i * a.N + t] + nb.x + T(CX(i)) * nb.y + T(CY(i)) * nb.z + T(CZ(i)) * nb.w;
    }
    T f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = fc[(int64_t)i * a.N + r];
    T rho, jx, jy, jz, F[3];
    node_moments(f, rho, jx, jy, jz);
    node_force(a, node_fin[r], jx, jy, jz, F[0], F[1], F[2]);
    const T Pv[3] = {jx + T(0.5) * F[0], jy + T(0.5) * F[1], jz + T(0.5) * F[2]};
    const T ir = T(1) / rho;
    // adjoint of the post-collision modes: mb_k = (1/b_k) sum_i w_i e_k(c_i) gin_i
    T mb[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        T acc = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int e = EMODE(k, i);
            if (e != 0) acc += T(e * WEIGHT(i)) * gin[i];
        }
        mb[k] = acc * T(INV_BNORM(k));
    }
    // stress modes 4..9: m'_k = (1 - g_k) Q_k(P)/rho + g_k m_k + (1 + g_k) H_k(P, F)/rho (+ noise)
    T A[10], B[10];
#pragma unroll
    for (int k = 4; k <= 9; ++k) {
        A[k] = (T(1) - a.gam[k]) * mb[k];
        B[k] = (T(1) + a.gam[k]) * mb[k];
    }
    const T Px = Pv[0], Py = Pv[1], Pz = Pv[2], Fx = F[0], Fy = F[1], Fz = F[2];
    const T PP = Px * Px + Py * Py + Pz * Pz, PF = Px * Fx + Py * Fy + Pz * Fz;
    // numerators Q_k and H_k, and their gradients
    const T Qn = A[4] * PP + A[5] * (T(3) * Px * Px - PP) + A[6] * (Py * Py - Pz * Pz) + A[7] * Px * Py +
                 A[8] * Px * Pz + A[9] * Py * Pz;
    const T Hn = B[4] * PF + B[5] * (T(3) * Px * Fx - PF) + B[6] * (Py * Fy - Pz * Fz) +
                 B[7] * T(0.5) * (Px * Fy + Py * Fx) + B[8] * T(0.5) * (Px * Fz + Pz * Fx) +
                 B[9] * T(0.5) * (Py * Fz + Pz * Fy);
    T Pb[3], Fb[3];
    Pb[0] = A[4] * T(2) * Px + A[5] * T(4) * Px + A[7] * Py + A[8] * Pz;
    Pb[1] = A[4] * T(2) * Py - A[5] * T(2) * Py + A[6] * T(2) * Py + A[7] * Px + A[9] * Pz;
    Pb[2] = A[4] * T(2) * Pz - A[5] * T(2) * Pz - A[6] * T(2) * Pz + A[8] * Px + A[9] * Py;
    Pb[0] += B[4] * Fx + B[5] * T(2) * Fx + T(0.5) * (B[7] * Fy + B[8] * Fz);
    Pb[1] += B[4] * Fy - B[5] * Fy + B[6] * Fy + T(0.5) * (B[7] * Fx + B[9] * Fz);
    Pb[2] += B[4] * Fz - B[5] * Fz - B[6] * Fz + T(0.5) * (B[8] * Fx + B[9] * Fy);
    Fb[0] = B[4] * Px + B[5] * T(2) * Px + T(0.5) * (B[7] * Py + B[8] * Pz);
    Fb[1] = B[4] * Py - B[5] * Py + B[6] * Py + T(0.5) * (B[7] * Px + B[9] * Pz);
    Fb[2] = B[4] * Pz - B[5] * Pz - B[6] * Pz + T(0.5) * (B[8] * Px + B[9] * Py);
    for (int d = 0; d < 3; ++d) {
        Pb[d] *= ir;
        Fb[d] *= ir;
    }
    T rb = mb[0] - (Qn + Hn) * ir * ir;
    // noise sqrt(rho) a_k xi_k: d/drho = noise / (2 rho)
    if (a.noisy) {
        T inv_r, sr;
        rho_factors(rho, inv_r, sr);
        T nsum = T(0);
#pragma unroll
        for (uint32_t q = 0; q < 2; ++q) {
            const U4 rr = philox4x32_10(U4{(uint32_t)r, step, 0u, q}, a.key0, a.key1);
            const uint32_t bits[4] = {rr.x, rr.y, rr.z, rr.w};
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int k = 4 + 8 * (int)q + t;
                const uint32_t h = (t & 1) ? (bits[t >> 1] >> 16) : (bits[t >> 1] & 0xffffu);
                if (k < Q) nsum += mb[k] * ((a.amp16[k] * sr) * centred16(h, T(0)));
            }
        }
        rb += nsum * T(0.5) * ir;
    }
    // j-bar and F-bar: m'_{1..3} = j + F; P = j + F/2
    T jb[3], Fbt[3];
    for (int d = 0; d < 3; ++d) {
        jb[d] = mb[1 + d] + Pb[d];
        Fbt[d] = mb[1 + d] + Fb[d] + T(0.5) * Pb[d];
    }
    // populations: rho = sum f, j* = sum c f (also entering F = j_node - j* + g
    // with a minus sign), non-conserved modes m_k relaxed with g_k
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T v = rb + T(CX(i)) * (jb[0] - Fbt[0]) + T(CY(i)) * (jb[1] - Fbt[1]) + T(CZ(i)) * (jb[2] - Fbt[2]);
#pragma unroll
        for (int k = 4; k < Q; ++k) {
            const int e = EMODE(k, i);
            if (e != 0) v += T(e) * a.gam[k] * mb[k];
        }
        fbar[(int64_t)i * a.N + r] = v;
    }
    nbar[r] = P::make4(T(0), Fbt[0], Fbt[1], Fbt[2]);
}

// Adjoint of one MD step for every particle (reads the node adjoint after
// the step; writes the particle's scatter contributions).
template <typename T>
__global__ void __launch_bounds__(128) ad_particle_adj(AdArgs<T> a, AdRec<T> rec,
                                                       const typename Prec<T>::real4 *nbar,
                                                       typename Prec<T>::real4 *Rbar, typename Prec<T>::real4 *vbar,
                                                       typename Prec<T>::real4 *scat, T *zbar) {
    using P = Prec<T>;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const typename P::real4 R = rec.R[p], V = rec.V[p], F = rec.F[p], U = rec.U[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.fd_nx, a.fd_ny);
    uint32_t idx[8];
    T delta[8];
    corners(c, R.x, R.y, R.z, a.nx, a.ny, a.nz, idx, delta);
    typename P::real4 xb = Rbar[p], vb = vbar[p];
    const T im = V.w, dt = a.dt;
    // F-bar: through v' = v + (dt/m) F, x' = x + dt v + dt^2/(2m) F, the
    // transfers -dt delta_k F and the drag term of the loss
    T Fb[3] = {im * dt * vb.x + a.half_dt * im * dt * xb.x + a.norm, im * dt * vb.y + a.half_dt * im * dt * xb.y,
               im * dt * vb.z + a.half_dt * im * dt * xb.z};
    T jbk[8][3];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const typename P::real4 nb = nbar[idx[k]];
        jbk[k][0] = nb.y;
        jbk[k][1] = nb.z;
        jbk[k][2] = nb.w;
        Fb[0] -= dt * delta[k] * nb.y;
        Fb[1] -= dt * delta[k] * nb.z;
        Fb[2] -= dt * delta[k] * nb.w;
    }
    // positions: gradient of the weights delta_k(d) within the cell
    const T d[3] = {R.x, R.y, R.z};
    T gx = xb.x, gy = xb.y, gz = xb.z;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
        const T w0 = o[0] ? d[0] : T(1) - d[0], w1 = o[1] ? d[1] : T(1) - d[1], w2 = o[2] ? d[2] : T(1) - d[2];
        const T s0 = o[0] ? T(1) : T(-1), s1 = o[1] ? T(1) : T(-1), s2 = o[2] ? T(1) : T(-1);
        const typename P::real4 ck = rec.C[8 * p + k];
        const T irk = T(1) / ck.x;
        const T uF = (ck.y * Fb[0] + ck.z * Fb[1] + ck.w * Fb[2]) * irk;  // u_k . F-bar
        const T Fj = F.x * jbk[k][0] + F.y * jbk[k][1] + F.z * jbk[k][2];
        const T coef = a.zeta * uF - dt * Fj;
        gx += coef * s0 * w1 * w2;
        gy += coef * w0 * s1 * w2;
        gz += coef * w0 * w1 * s2;
        // node adjoints: j_k gets zeta delta_k / rho_k F-bar, rho_k gets
        // -zeta delta_k (u_k . F-bar) / rho_k
        const T sk = a.zeta * delta[k] * irk;
        scat[8 * p + k] = P::make4(-sk * uF, sk * Fb[0], sk * Fb[1], sk * Fb[2]);
    }
    // zeta: F = -zeta (v - u) + sqrt(zeta) (...) xi
    const T Fr[3] = {F.x + a.zeta * (V.x - U.x), F.y + a.zeta * (V.y - U.y), F.z + a.zeta * (V.z - U.z)};
    T zb = -(Fb[0] * (V.x - U.x) + Fb[1] * (V.y - U.y) + Fb[2] * (V.z - U.z));
    if (a.zeta > T(0)) zb += (Fb[0] * Fr[0] + Fb[1] * Fr[1] + Fb[2] * Fr[2]) / (T(2) * a.zeta);
    zbar[p] = zb;
    Rbar[p] = P::make4(gx, gy, gz, T(0));
    vbar[p] = P::make4(vb.x + dt * xb.x - a.zeta * Fb[0], vb.y + dt * xb.y - a.zeta * Fb[1],
                       vb.z + dt * xb.z - a.zeta * Fb[2], T(0));
}

__device__ __forceinline__ void atomic_addT(float *p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_addT(double *p, double v) { atomicAdd(p, v); }

template <typename T>
__global__ void __launch_bounds__(128) ad_scatter_adj(AdArgs<T> a, AdRec<T> rec,
                                                      const typename Prec<T>::real4 *scat,
                                                      typename Prec<T>::real4 *nbar) {
    using P = Prec<T>;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8 * a.np) return;
    const int p = t >> 3, k = t & 7;
    const typename P::real4 R = rec.R[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.fd_nx, a.fd_ny);
    uint32_t idx[8];
    T delta[8];
    corners(c, R.x, R.y, R.z, a.nx, a.ny, a.nz, idx, delta);
    const typename P::real4 s = scat[t];
    T *n = reinterpret_cast<T *>(&nbar[idx[k]]);
    atomic_addT(n + 0, s.x);
    atomic_addT(n + 1, s.y);
    atomic_addT(n + 2, s.z);
    atomic_addT(n + 3, s.w);
}

template <typename T>
__global__ void ad_particles_from_double(typename Prec<T>::real4 *pos4, typename Prec<T>::real4 *vel4,
                                         const double *pos, const double *vel, int np, int nx, int ny, int nz) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    pos4[p] = pos_from_double<T>(pos + 3 * p, nx, ny, nz);
    vel4[p] = Prec<T>::make4((T)vel[3 * p], (T)vel[3 * p + 1], (T)vel[3 * p + 2], T(1));
}

template <typename T>
__global__ void ad_to_double(const typename Prec<T>::real4 *v4, double *out, int np) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    out[3 * p] = (double)v4[p].x;
    out[3 * p + 1] = (double)v4[p].y;
    out[3 * p + 2] = (double)v4[p].z;
}

template <typename T>
__global__ void ad_to_double_scalar(const T *v, double *out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)v[i];
}

}  // namespace lbmd

using namespace lbmd;

struct lbmd_adjoint {
    lbmd_adjoint_params p{};
    int64_t N = 0;
    size_t rs = 4;  // bytes of a real
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    LbCoeffs co{};
    FixUnit fix{};  // fixed-point unit of the momentum density (from rho0)
    double zeta = 0.0;
    bool have_forward = false;
    // device
    void *fchk = nullptr;                    // (K + 1) x 19 N populations
    void *pchk = nullptr;                    // (K + 1) x 2 x np real4 (position, velocity)
    void *pos = nullptr, *vel = nullptr, *old = nullptr, *fc = nullptr;
    void *node = nullptr;                    // N node records
    void *drag = nullptr;                    // K m np
    void *rec = nullptr;                     // m x np x (4 + 8) real4
    void *fbar[2] = {nullptr, nullptr};      // 19 N each
    void *nbar[2] = {nullptr, nullptr};      // N real4 each
    void *Rbar = nullptr, *vbar = nullptr;   // np real4
    void *scat = nullptr;                    // 8 np real4
    void *zbar = nullptr;                    // K m np
    double *staging = nullptr;               // host-conversion scratch, 8 K m np doubles or more
    int64_t staging_len = 0;
    std::string err;
};

namespace {

std::mutex g_ad_mutex;
std::string g_ad_create_error;

lbmd_status afail(lbmd_adjoint *a, lbmd_status s, const std::string &msg) {
    if (a) {
        a->err = msg;
    } else {
        std::lock_guard<std::mutex> lock(g_ad_mutex);
        g_ad_create_error = msg;
    }
    return s;
}

#define ACK(a, call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return afail(a, e_ == cudaErrorMemoryAllocation ? LBMD_ERR_OOM : LBMD_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

void free_ad(lbmd_adjoint *a) {
    void *bufs[] = {a->fchk, a->pchk, a->pos,  a->vel,  a->old,  a->fc,  a->node,    a->drag,    a->rec,
                    a->fbar[0], a->fbar[1], a->nbar[0], a->nbar[1], a->Rbar, a->vbar, a->scat, a->zbar,
                    a->staging};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (a->own_stream && a->stream) cudaStreamDestroy(a->stream);
}

template <typename T>
AdArgs<T> make_args(const lbmd_adjoint *ad) {
    AdArgs<T> a;
    const lbmd_adjoint_params &p = ad->p;
    a.nx = p.nx;
    a.ny = p.ny;
    a.nz = p.nz;
    a.np = p.n_particles;
    a.n_sub = p.n_sub;
    a.N = ad->N;
    a.fd_nx = make_fastdiv((uint32_t)p.nx);
    a.fd_ny = make_fastdiv((uint32_t)p.ny);
    const double dt = 1.0 / p.n_sub;
    a.zeta = (T)ad->zeta;
    a.dt = (T)dt;
    a.half_dt = (T)(0.5 * dt);
    a.amp = (T)std::sqrt(2.0 * ad->zeta * p.kT / dt);
    a.neg_scale_dt = (T)dt * -(T)ad->fix.scale;
    a.fs = (T)ad->fix.scale;
    a.fis = (T)ad->fix.inv_scale;
    a.norm = (T)(1.0 / ((double)p.n_cycles * p.n_sub * std::max(1, p.n_particles)));
    a.key0 = (uint32_t)(p.seed & 0xffffffffu);
    a.key1 = (uint32_t)(p.seed >> 32);
    for (int d = 0; d < 3; ++d) a.g[d] = (T)p.body_force[d];
    a.gamma_bulk = (T)ad->co.gamma_bulk;
    a.gamma_shear = (T)ad->co.gamma_shear;
    a.gamma_ghost = (T)ad->co.gamma_ghost;
    for (int k = 0; k < Q; ++k) {
        a.amp16[k] = (T)(ad->co.noise_amp[k] * 3.4641016151377544 * 1.52587890625e-05);
        a.gam[k] = (T)(k == 4 ? ad->co.gamma_bulk : (k <= 9 ? ad->co.gamma_shear : ad->co.gamma_ghost));
    }
    a.noisy = ad->co.noisy;
    return a;
}

template <typename T>
AdRec<T> rec_at(const lbmd_adjoint *ad, int s) {
    using R4 = typename Prec<T>::real4;
    R4 *base = static_cast<R4 *>(ad->rec) + (size_t)s * ad->p.n_particles * 12;
    const int np = ad->p.n_particles;
    AdRec<T> r;
    r.R = base;
    r.V = base + np;
    r.F = base + 2 * np;
    r.U = base + 3 * np;
    r.C = base + 4 * np;
    return r;
}

template <typename T>
T *fchk_at(const lbmd_adjoint *ad, int c) {
    return static_cast<T *>(ad->fchk) + (size_t)c * 19 * ad->N;
}

template <typename T>
typename Prec<T>::real4 *pchk_at(const lbmd_adjoint *ad, int c) {
    return static_cast<typename Prec<T>::real4 *>(ad->pchk) + (size_t)c * 2 * ad->p.n_particles;
}

unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// one cycle's MD steps from the checkpoint of cycle c (node field from the
// checkpointed populations), optionally recording every MD step
template <typename T>
cudaError_t run_md(lbmd_adjoint *ad, int c, bool record) {
    using R4 = typename Prec<T>::real4;
    using N4 = typename Prec<T>::node4;
    const AdArgs<T> a = make_args<T>(ad);
    const int np = ad->p.n_particles, m = ad->p.n_sub;
    ad_moments_kernel<T><<<nb(ad->N, 256), 256, 0, ad->stream>>>(fchk_at<T>(ad, c), static_cast<N4 *>(ad->node),
                                                                  ad->N, (T)ad->fix.scale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (np == 0) return cudaSuccess;
    R4 *ck = pchk_at<T>(ad, c);
    if ((e = cudaMemcpyAsync(ad->pos, ck, np * sizeof(R4), cudaMemcpyDeviceToDevice, ad->stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(ad->vel, ck + np, np * sizeof(R4), cudaMemcpyDeviceToDevice, ad->stream)) != cudaSuccess)
        return e;
    for (int s = 0; s < m; ++s) {
        AdRec<T> r = record ? rec_at<T>(ad, s) : AdRec<T>{nullptr, nullptr, nullptr, nullptr, nullptr};
        T *drag = static_cast<T *>(ad->drag) + ((size_t)c * m + s) * np;
        ad_couple<T><<<nb(np, 128), 128, 0, ad->stream>>>(a, static_cast<R4 *>(ad->pos), static_cast<R4 *>(ad->vel),
                                                          static_cast<R4 *>(ad->old), static_cast<R4 *>(ad->fc),
                                                          static_cast<N4 *>(ad->node), drag, r,
                                                          (uint32_t)(c * m + s));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ad_transfer<T><<<nb(np, 128), 128, 0, ad->stream>>>(a, static_cast<R4 *>(ad->old), static_cast<R4 *>(ad->fc),
                                                            static_cast<N4 *>(ad->node));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t forward_t(lbmd_adjoint *ad, const double *pos0, const double *vel0, double *loss) {
    using R4 = typename Prec<T>::real4;
    using N4 = typename Prec<T>::node4;
    const AdArgs<T> a = make_args<T>(ad);
    const int np = ad->p.n_particles, m = ad->p.n_sub, K = ad->p.n_cycles;
    cudaError_t e;
    ad_init_kernel<T><<<nb(ad->N, 256), 256, 0, ad->stream>>>(fchk_at<T>(ad, 0), ad->N, (T)ad->p.rho0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (np > 0) {
        double *dp = ad->staging, *dv = ad->staging + 3 * np;
        if ((e = cudaMemcpyAsync(dp, pos0, 3 * np * sizeof(double), cudaMemcpyHostToDevice, ad->stream)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpyAsync(dv, vel0, 3 * np * sizeof(double), cudaMemcpyHostToDevice, ad->stream)) != cudaSuccess)
            return e;
        R4 *ck = pchk_at<T>(ad, 0);
        ad_particles_from_double<T><<<nb(np, 128), 128, 0, ad->stream>>>(ck, ck + np, dp, dv, np, ad->p.nx, ad->p.ny,
                                                                         ad->p.nz);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const bool full = ad->co.gamma_bulk == 0.0 && ad->co.gamma_ghost == 0.0;
    for (int c = 0; c < K; ++c) {
        if ((e = run_md<T>(ad, c, false)) != cudaSuccess) return e;
        if (np > 0) {
            R4 *nx = pchk_at<T>(ad, c + 1);
            if ((e = cudaMemcpyAsync(nx, ad->pos, np * sizeof(R4), cudaMemcpyDeviceToDevice, ad->stream)) !=
                cudaSuccess)
                return e;
            if ((e = cudaMemcpyAsync(nx + np, ad->vel, np * sizeof(R4), cudaMemcpyDeviceToDevice, ad->stream)) !=
                cudaSuccess)
                return e;
        }
        if (full)
            ad_collide_push<T, true><<<nb(ad->N, 256), 256, 0, ad->stream>>>(
                fchk_at<T>(ad, c), fchk_at<T>(ad, c + 1), static_cast<N4 *>(ad->node), a, (uint32_t)c);
        else
            ad_collide_push<T, false><<<nb(ad->N, 256), 256, 0, ad->stream>>>(
                fchk_at<T>(ad, c), fchk_at<T>(ad, c + 1), static_cast<N4 *>(ad->node), a, (uint32_t)c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // loss: the drags summed in a fixed order (MD step, then particle id)
    const int64_t nd = (int64_t)K * m * np;
    double L = 0.0;
    if (nd > 0) {
        ad_to_double_scalar<T><<<nb(nd, 256), 256, 0, ad->stream>>>(static_cast<T *>(ad->drag), ad->staging, nd);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        std::vector<double> h(nd);
        if ((e = cudaMemcpyAsync(h.data(), ad->staging, nd * sizeof(double), cudaMemcpyDeviceToHost, ad->stream)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(ad->stream)) != cudaSuccess) return e;
        for (int64_t i = 0; i < nd; ++i) L += h[i];
        L /= (double)nd;
    } else if ((e = cudaStreamSynchronize(ad->stream)) != cudaSuccess) {
        return e;
    }
    *loss = L;
    return cudaSuccess;
}

template <typename T>
cudaError_t backward_t(lbmd_adjoint *ad, double *dzeta, double *dpos) {
    using R4 = typename Prec<T>::real4;
    using N4 = typename Prec<T>::node4;
    const AdArgs<T> a = make_args<T>(ad);
    const int np = ad->p.n_particles, m = ad->p.n_sub, K = ad->p.n_cycles;
    cudaError_t e;
    const size_t fb = (size_t)19 * ad->N * sizeof(T), nbb = (size_t)ad->N * sizeof(R4);
    int cur = 0;  // fbar[cur], nbar[cur]: adjoint of the next cycle's start
    if ((e = cudaMemsetAsync(ad->fbar[cur], 0, fb, ad->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ad->nbar[cur], 0, nbb, ad->stream)) != cudaSuccess) return e;
    if (np > 0) {
        if ((e = cudaMemsetAsync(ad->Rbar, 0, np * sizeof(R4), ad->stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(ad->vbar, 0, np * sizeof(R4), ad->stream)) != cudaSuccess) return e;
    }
    for (int c = K - 1; c >= 0; --c) {
        if ((e = run_md<T>(ad, c, true)) != cudaSuccess) return e;  // node: the field after the m MD steps
        const int o = cur ^ 1;
        ad_collide_adj<T><<<nb(ad->N, 128), 128, 0, ad->stream>>>(
            fchk_at<T>(ad, c), static_cast<N4 *>(ad->node), static_cast<T *>(ad->fbar[cur]),
            static_cast<R4 *>(ad->nbar[cur]), static_cast<T *>(ad->fbar[o]), static_cast<R4 *>(ad->nbar[o]), a,
            (uint32_t)c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        for (int s = m - 1; s >= 0 && np > 0; --s) {
            AdRec<T> r = rec_at<T>(ad, s);
            T *zb = static_cast<T *>(ad->zbar) + ((size_t)c * m + s) * np;
            ad_particle_adj<T><<<nb(np, 128), 128, 0, ad->stream>>>(a, r, static_cast<R4 *>(ad->nbar[o]),
                                                                    static_cast<R4 *>(ad->Rbar),
                                                                    static_cast<R4 *>(ad->vbar),
                                                                    static_cast<R4 *>(ad->scat), zb);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            ad_scatter_adj<T><<<nb(8 * (int64_t)np, 128), 128, 0, ad->stream>>>(a, r, static_cast<R4 *>(ad->scat),
                                                                                static_cast<R4 *>(ad->nbar[o]));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        cur = o;
    }
    // gradients: positions (frac = absolute coordinate within the cell),
    // zeta summed in a fixed order
    const int64_t nz = (int64_t)K * m * np;
    std::vector<double> hz(nz);
    if (np > 0) {
        ad_to_double<T><<<nb(np, 128), 128, 0, ad->stream>>>(static_cast<R4 *>(ad->Rbar), ad->staging, np);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(dpos, ad->staging, 3 * np * sizeof(double), cudaMemcpyDeviceToHost, ad->stream)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(ad->stream)) != cudaSuccess) return e;
        ad_to_double_scalar<T><<<nb(nz, 256), 256, 0, ad->stream>>>(static_cast<T *>(ad->zbar), ad->staging, nz);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(hz.data(), ad->staging, nz * sizeof(double), cudaMemcpyDeviceToHost, ad->stream)) !=
            cudaSuccess)
            return e;
    }
    if ((e = cudaStreamSynchronize(ad->stream)) != cudaSuccess) return e;
    double z = 0.0;
    for (int64_t i = 0; i < nz; ++i) z += hz[i];
    *dzeta = z;
    return cudaSuccess;
}

bool ad_finite(double x) { return std::isfinite(x); }

}  // namespace

extern "C" {

const char *lbmd_adjoint_last_error(lbmd_adjoint *a) {
    if (a) return a->err.c_str();
    std::lock_guard<std::mutex> lock(g_ad_mutex);
    return g_ad_create_error.c_str();
}

lbmd_status lbmd_adjoint_create(const lbmd_adjoint_params *p, lbmd_adjoint **out) {
    if (!p || !out) return afail(nullptr, LBMD_ERR_ARG, "null argument");
    *out = nullptr;
    if (p->nx < 2 || p->ny < 2 || p->nz < 2 || (int64_t)p->nx * p->ny * p->nz > (1ll << 26))
        return afail(nullptr, LBMD_ERR_ARG, "lattice sides >= 2 and at most 2^26 nodes");
    if (p->n_sub < 1 || p->n_cycles < 1 || p->n_particles < 0 || p->n_particles > (1 << 24))
        return afail(nullptr, LBMD_ERR_ARG, "n_sub, n_cycles >= 1; 0 <= n_particles <= 2^24");
    if (p->precision != LBMD_FP32 && p->precision != LBMD_FP64)
        return afail(nullptr, LBMD_ERR_ARG, "the adjoint supports LBMD_FP32 and LBMD_FP64");
    if (!(p->rho0 > 0) || !(p->nu > 0) || !ad_finite(p->rho0) || !ad_finite(p->nu) || !(p->kT >= 0) ||
        !ad_finite(p->kT) || !(std::fabs(p->gamma_ghost) < 1.0))
        return afail(nullptr, LBMD_ERR_ARG, "bad fluid parameters");
    for (int d = 0; d < 3; ++d)
        if (!ad_finite(p->body_force[d])) return afail(nullptr, LBMD_ERR_ARG, "non-finite body force");
    lbmd_adjoint *a = new (std::nothrow) lbmd_adjoint();
    if (!a) return afail(nullptr, LBMD_ERR_OOM, "host allocation");
    a->p = *p;
    a->N = (int64_t)p->nx * p->ny * p->nz;
    a->rs = p->precision == LBMD_FP64 ? 8 : 4;
    lb_coefficients(p->nu, p->nu_bulk, p->gamma_ghost, p->kT, a->co);
    if (!fix_unit(p->rho0, p->precision == LBMD_FP64 ? Prec<double>::SCALE_LOG2 : Prec<float>::SCALE_LOG2, a->fix)) {
        delete a;
        return afail(nullptr, LBMD_ERR_ARG, "rho0 must lie in [2^-60, 2^60]");
    }
    if (p->stream) {
        a->stream = (cudaStream_t)p->stream;
    } else {
        if (cudaStreamCreateWithFlags(&a->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete a;
            return afail(nullptr, LBMD_ERR_CUDA, "cudaStreamCreate");
        }
        a->own_stream = true;
    }
    const size_t rs = a->rs, r4 = 4 * rs, N = (size_t)a->N;
    const size_t np = (size_t)std::max(1, p->n_particles), K = (size_t)p->n_cycles, m = (size_t)p->n_sub;
    a->staging_len = (int64_t)std::max<size_t>(8 * np, K * m * np + 8);
    struct {
        void **ptr;
        size_t bytes;
    } allocs[] = {
        {&a->fchk, (K + 1) * 19 * N * rs}, {&a->pchk, (K + 1) * 2 * np * r4}, {&a->pos, np * r4},
        {&a->vel, np * r4}, {&a->old, np * r4}, {&a->fc, np * r4}, {&a->node, N * r4},
        {&a->drag, K * m * np * rs}, {&a->rec, m * np * 12 * r4}, {&a->fbar[0], 19 * N * rs},
        {&a->fbar[1], 19 * N * rs}, {&a->nbar[0], N * r4}, {&a->nbar[1], N * r4}, {&a->Rbar, np * r4},
        {&a->vbar, np * r4}, {&a->scat, 8 * np * r4}, {&a->zbar, K * m * np * rs},
        {(void **)&a->staging, (size_t)a->staging_len * sizeof(double)},
    };
    for (auto &x : allocs) {
        cudaError_t e = cudaMalloc(x.ptr, x.bytes);
        if (e != cudaSuccess) {
            free_ad(a);
            delete a;
            return afail(nullptr, e == cudaErrorMemoryAllocation ? LBMD_ERR_OOM : LBMD_ERR_CUDA,
                         std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
    }
    *out = a;
    return LBMD_OK;
}

lbmd_status lbmd_adjoint_destroy(lbmd_adjoint *a) {
    if (!a) return LBMD_OK;
    cudaStreamSynchronize(a->stream);
    free_ad(a);
    delete a;
    return LBMD_OK;
}

lbmd_status lbmd_adjoint_forward(lbmd_adjoint *a, double zeta, const double *pos0, const double *vel0,
                                 double *loss) {
    LBMD_TRACE("lbmd_adjoint_forward");
    if (!a || !loss || !(zeta >= 0) || !ad_finite(zeta) || (a->p.n_particles > 0 && (!pos0 || !vel0)))
        return afail(a, LBMD_ERR_ARG, "bad arguments");
    for (int64_t q = 0; q < 3 * (int64_t)a->p.n_particles; ++q)
        if (!ad_finite(pos0[q]) || !ad_finite(vel0[q])) return afail(a, LBMD_ERR_ARG, "non-finite particle data");
    a->zeta = zeta;
    cudaError_t e = a->p.precision == LBMD_FP64 ? forward_t<double>(a, pos0, vel0, loss)
                                                : forward_t<float>(a, pos0, vel0, loss);
    if (e != cudaSuccess) return afail(a, LBMD_ERR_CUDA, std::string("adjoint forward: ") + cudaGetErrorString(e));
    a->have_forward = true;
    return LBMD_OK;
}

lbmd_status lbmd_adjoint_backward(lbmd_adjoint *a, double *dloss_dzeta, double *dloss_dpos0) {
    LBMD_TRACE("lbmd_adjoint_backward");
    if (!a || !dloss_dzeta || (a->p.n_particles > 0 && !dloss_dpos0)) return afail(a, LBMD_ERR_ARG, "bad arguments");
    if (!a->have_forward) return afail(a, LBMD_ERR_SEQUENCE, "backward before forward");
    cudaError_t e = a->p.precision == LBMD_FP64 ? backward_t<double>(a, dloss_dzeta, dloss_dpos0)
                                                : backward_t<float>(a, dloss_dzeta, dloss_dpos0);
    if (e != cudaSuccess) return afail(a, LBMD_ERR_CUDA, std::string("adjoint backward: ") + cudaGetErrorString(e));
    return LBMD_OK;
}

}  // extern "C"
