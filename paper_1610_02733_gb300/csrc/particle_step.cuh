// particle_step.cuh -- the argument block and the per-particle pieces of
// one MD step of Sec. 3 shared by the single-box particle kernels
// (particles.cu) and the tiled variant-B MD step (md_tile.cu): node
// velocities at the corners (Eq. (5)), the coupling force with its random
// part (Eq. (4)), and the hand-over of the transfer (Eqs. (7), (8)).
#pragma once

#include "lbmd_ctx.h"
#include "lbmd_device.cuh"
#include "particle_core.cuh"

namespace lbmd {

template <typename T>
struct PArgs {
    using P = Prec<T>;
    typename P::real4 *pos4, *vel4, *fc4, *old4, *fcons4;
    const int32_t *pid, *slot_of;
    typename P::node4 *node, *jacc;
    const int32_t *bond_count, *bond_partner;
    const double *bond_k, *bond_r0;
    const uint8_t *bond_kind;
    T lj_eps24, lj_sig2, lj_rc2;  // Lennard-Jones: 24 eps, sigma^2, r_cut^2
    float lj_filter2;             // (r_cut + rounding margin of FP32 absolute positions)^2
    // LJ Verlet lists (null when LJ is off)
    const int32_t *nb_list, *nb_count;
    int32_t *nb_invalid;
    const typename P::real4 *nb_ref4;  // positions at the list build, per id
    T nb_half_skin2;                   // (skin / 2)^2: a larger move since the build voids the lists
    int nx, ny, nz;
    FastDiv fd_nx, fd_ny;  // division by nx and ny
    int64_t np;
    T zeta, dt, half_dt, amp;
    T neg_scale_dt;  // -dt times the fixed-point scale s: -s (dt F) = F neg_scale_dt exactly
    T fis;           // 1 / s: fixed-point momentum -> real
    uint32_t key0, key1;
    const unsigned long long *lb_step;
    int n_sub, substep, noisy;
    int mig_par;  // parity of the MD step (lb_step n_sub + substep): which migrant list is filled
    int variant;
    // variant B row-gather spreading and active nodes
    const int32_t *row_start, *slot_row;
    const uint2 *occw;
    typename P::node4 *cact;          // the active nodes' records (variant A with a frozen copy: the frozen ones)
    typename P::node4 *cact_acc;      // ... the ones the transfers go to (the same unless A keeps a frozen copy)
    typename P::node4 *inactive_acc;  // where transfers to inactive nodes go (A: J_acc, B: the node field)
    int interp_compact;               // interpolate from cact (B; A with a frozen copy), else the node field
    int occ_words;
    int32_t *migrant_slot, *migrant_count;  // two lists of np_cap slots, two counters
    int gauss;         // normal variates (Box-Muller) for the random force
    int b_atomic;      // variant B spreads every particle with atomics (no row gather, no migrant lists)
    int kick_spreads;  // ... and the bond / pair kernel does it, after every particle has read the nodes
    int64_t np_cap;
};

// Variant B: the records of corners 2q, 2q+1 (nodes x0 and x0 + 1 of row
// `row`): compact record of an active node, node field entry otherwise.
template <typename T>
__device__ __forceinline__ void corner_pair(const PArgs<T> &a, uint32_t row, int x0, int x1,
                                            typename Prec<T>::node4 &n0, typename Prec<T>::node4 &n1) {
    const uint2 *wr = a.occw + (size_t)row * (uint32_t)a.occ_words;
    const uint2 w0 = wr[x0 >> 5];
    const uint2 w1 = (x1 >> 5) == (x0 >> 5) ? w0 : wr[x1 >> 5];
    const int s0 = active_slot(w0, x0), s1 = active_slot(w1, x1);
    const size_t r0 = (size_t)row * (uint32_t)a.nx;
    n0 = s0 >= 0 ? a.cact[s0] : a.node[r0 + x0];
    n1 = s1 >= 0 ? a.cact[s1] : a.node[r0 + x1];
}

// Fluid velocity at a particle with fractional offsets (fx, fy, fz) in its
// cell, Eq. (5): corners k = ox + 2 oy + 4 oz = 0..7 with weights
// delta_k = wx wy wz, u(R) = sum_k delta_k j_k / rho_k.  fetch(q, n0, n1)
// supplies the records of corners 2q, 2q+1 (lattice row q = oy + 2 oz, nodes
// x and x + 1); every caller sums in this one order with explicit fused
// multiply-adds, so the paths that fetch the records differently agree bit
// for bit whatever the compiler would contract.
template <typename T, typename Fetch>
__device__ __forceinline__ void interp_u_from(T fx, T fy, T fz, T fis, T &ux, T &uy, T &uz, Fetch &&fetch) {
    using P = Prec<T>;
    ux = T(0);
    uy = T(0);
    uz = T(0);
    const T wx[2] = {T(1) - fx, fx}, wy[2] = {T(1) - fy, fy}, wz[2] = {T(1) - fz, fz};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        typename P::node4 n[2];
        fetch(q, n[0], n[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const T w = (wx[h] * wy[q & 1] * wz[q >> 1]) / P::rho_of(n[h]);
            ux = fma(w, P::from_fix(P::jx_of(n[h]), fis), ux);
            uy = fma(w, P::from_fix(P::jy_of(n[h]), fis), uy);
            uz = fma(w, P::from_fix(P::jz_of(n[h]), fis), uz);
        }
    }
}

// The same for a particle in cell c read from global memory; variant B reads
// an active corner's compact record.
template <typename T>
__device__ __forceinline__ void interp_u(const PArgs<T> &a, const CellXYZ &c, T fx, T fy, T fz, T &ux, T &uy,
                                         T &uz) {
    using P = Prec<T>;
    uint32_t rows[4];
    corner_rows(c, a.ny, a.nz, rows);
    const int x1 = c.x + 1 == a.nx ? 0 : c.x + 1;
    interp_u_from(fx, fy, fz, a.fis, ux, uy, uz, [&](int q, typename P::node4 &n0, typename P::node4 &n1) {
        if (a.interp_compact) {  // an active corner's compact record
            corner_pair(a, rows[q], c.x, x1, n0, n1);
        } else {
            const size_t r0 = (size_t)rows[q] * (uint32_t)a.nx;
            n0 = a.node[r0 + c.x];
            n1 = a.node[r0 + x1];
        }
    });
}

// Coupling force of Eq. (4) without the conservative part: friction against
// the interpolated fluid velocity plus the random force of Philox(id, s, 1, 0)
// for the particle with id `id` in MD step s (md_step, the global MD step
// index as the counters take it).
template <typename T>
__device__ __forceinline__ void coupling_force_id(const PArgs<T> &a, uint32_t id, uint32_t md_step,
                                                  const typename Prec<T>::real4 &V, T ux, T uy, T uz, T &Fx, T &Fy,
                                                  T &Fz) {
    Fx = -a.zeta * (V.x - ux);
    Fy = -a.zeta * (V.y - uy);
    Fz = -a.zeta * (V.z - uz);
    if (a.noisy) {
        const U4 r = philox4x32_10(U4{id, md_step, 1u, 0u}, a.key0, a.key1);
        T g0, g1, g2, g3;
        if (a.gauss) {  // normal variates: Box-Muller pairs (x, y) and (z, w)
            box_muller(r.x, r.y, g0, g1);
            box_muller(r.z, r.w, g2, g3);
        } else {
            g0 = unit_uniform<T>(r.x);
            g1 = unit_uniform<T>(r.y);
            g2 = unit_uniform<T>(r.z);
        }
        Fx = fma(a.amp, g0, Fx);
        Fy = fma(a.amp, g1, Fy);
        Fz = fma(a.amp, g2, Fz);
    }
}

// The global MD step index of this launch (the particles' Philox counter).
template <typename T>
__device__ __forceinline__ uint32_t md_step_index(const PArgs<T> &a) {
    return (uint32_t)((*a.lb_step) * (unsigned long long)a.n_sub + (unsigned)a.substep);
}

// The same for the particle in slot p.
template <typename T>
__device__ __forceinline__ void coupling_force(const PArgs<T> &a, int64_t p, const typename Prec<T>::real4 &V, T ux,
                                               T uy, T uz, T &Fx, T &Fy, T &Fz) {
    coupling_force_id(a, (uint32_t)a.pid[p], md_step_index(a), V, ux, uy, uz, Fx, Fy, Fz);
}

// Newton's third law for the particle in slot p whose transfer -delta_k dt F
// belongs to the nodes around position R (cell c): variant C adds it to
// J_acc at once (forcing_update_kernel then moves it into the populations);
// variants A and B keep R for the row gather (which adds the transfers to the
// compact records, cact_acc), and a particle whose cell row
// is no longer the row bucket it was sorted into is listed as a migrant (two
// lists alternating with the parity of the MD step).
template <typename T>
__device__ __forceinline__ void hand_over(const PArgs<T> &a, int64_t p, const typename Prec<T>::real4 &R,
                                          const CellXYZ &c, T Fx, T Fy, T Fz) {
    using P = Prec<T>;
    if (a.variant == LBMD_VARIANT_C) {
        uint32_t idx[8];
        T delta[8];
        corners(c, R.x, R.y, R.z, a.nx, a.ny, a.nz, idx, delta);
        spread_to<T>(a.jacc, idx, delta, Fx * a.neg_scale_dt, Fy * a.neg_scale_dt, Fz * a.neg_scale_dt);
    } else {
        a.old4[p] = R;
        if (a.b_atomic) return;
        const int32_t srow = a.slot_row[p];
        if (srow < 0 || (uint32_t)P::cell_of(R) - (uint32_t)srow * (uint32_t)a.nx >= (uint32_t)a.nx) {
            a.migrant_slot[(int64_t)a.mig_par * a.np_cap + atomicAdd(a.migrant_count + a.mig_par, 1)] = (int32_t)p;
        }
    }
}

// Cell offset d (partner minus particle, |d| < n) to its periodic image
// nearest to zero, in [-n/2, n/2].
__device__ __forceinline__ int nearest_image(int d, int n) {
    const int h = n >> 1;
    return d > h ? d - n : (d < -h ? d + n : d);
}

// LJ Verlet lists: a particle that moved more than half the skin since the
// lists were built voids them (flag read by the pair kernel of this step).
template <typename T>
__device__ __forceinline__ void check_list_skin(const PArgs<T> &a, int64_t p, const CellXYZ &cn, T fx, T fy, T fz) {
    using P = Prec<T>;
    if (!a.nb_ref4 || *a.nb_invalid) return;
    const typename P::real4 S = a.nb_ref4[a.pid[p]];
    const CellXYZ d = cell_xyz(P::cell_of(S), a.fd_nx, a.fd_ny);
    const T dx = T(nearest_image(cn.x - d.x, a.nx)) + (fx - S.x);
    const T dy = T(nearest_image(cn.y - d.y, a.ny)) + (fy - S.y);
    const T dz = T(nearest_image(cn.z - d.z, a.nz)) + (fz - S.z);
    if (dx * dx + dy * dy + dz * dz > a.nb_half_skin2) atomicOr(a.nb_invalid, 1);
}

// Variant B: a particle's transfers spread with integer atomics (into the
// compact record of an active corner, the node field entry of an inactive
// one), from its start position and force kept in old4 / fc4: the migrants
// after the row gather or the tiled step, or every particle
// (LBMD_SPREAD_ATOMIC).
template <typename T>
__device__ __forceinline__ void spread_corner_atomic(const PArgs<T> &a, int64_t p, int k) {
    using P = Prec<T>;
    const typename P::real4 R = a.old4[p];
    const typename P::real4 F = a.fc4[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.fd_nx, a.fd_ny);
    const int ox = k & 1, oy = (k >> 1) & 1, oz = k >> 2;
    const int xn = ox ? (c.x + 1 == a.nx ? 0 : c.x + 1) : c.x;
    const int yn = oy ? (c.y + 1 == a.ny ? 0 : c.y + 1) : c.y;
    const int zn = oz ? (c.z + 1 == a.nz ? 0 : c.z + 1) : c.z;
    const T delta = (ox ? R.x : T(1) - R.x) * (oy ? R.y : T(1) - R.y) * (oz ? R.z : T(1) - R.z);
    const uint32_t row = (uint32_t)yn + (uint32_t)a.ny * (uint32_t)zn;
    const int sl = active_slot(a.occw[(size_t)row * (uint32_t)a.occ_words + (xn >> 5)], xn);
    typename P::node4 *rec = sl >= 0 ? &a.cact_acc[sl] : &a.inactive_acc[(size_t)row * (uint32_t)a.nx + xn];
    const T sx = F.x * a.neg_scale_dt, sy = F.y * a.neg_scale_dt, sz = F.z * a.neg_scale_dt;
    P::add_transfer(rec, P::to_fix_neg(delta, sx), P::to_fix_neg(delta, sy), P::to_fix_neg(delta, sz));
}

// All 8 corner transfers of the particle in slot p (position and force read
// and the cell decoded once).
template <typename T>
__device__ __forceinline__ void spread_particle_atomic(const PArgs<T> &a, int64_t p) {
    using P = Prec<T>;
    const typename P::real4 R = a.old4[p];
    const typename P::real4 F = a.fc4[p];
    const CellXYZ c = cell_xyz(P::cell_of(R), a.fd_nx, a.fd_ny);
    uint32_t idx[8], rows[4];
    T delta[8];
    corners(c, R.x, R.y, R.z, a.nx, a.ny, a.nz, idx, delta);
    corner_rows(c, a.ny, a.nz, rows);
    const int x1 = c.x + 1 == a.nx ? 0 : c.x + 1;
    const T sx = F.x * a.neg_scale_dt, sy = F.y * a.neg_scale_dt, sz = F.z * a.neg_scale_dt;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int xn = (k & 1) ? x1 : c.x;
        const int sl = active_slot(a.occw[(size_t)rows[k >> 1] * (uint32_t)a.occ_words + (xn >> 5)], xn);
        typename P::node4 *rec = sl >= 0 ? &a.cact_acc[sl] : &a.inactive_acc[idx[k]];
        P::add_transfer(rec, P::to_fix_neg(delta[k], sx), P::to_fix_neg(delta[k], sy), P::to_fix_neg(delta[k], sz));
    }
}

}  // namespace lbmd
