// particle_core.cuh -- per-particle pieces of the coupling of Sec. 3 shared
// by the single-box kernels (particles.cu) and the batched replicas
// (batch.cu): cell decoding, the 8 corners and trilinear weights of Eq. (5),
// the periodic move of a position, and the fixed-point transfer of
// Eqs. (7), (8).
#pragma once

#include "lbmd_device.cuh"

namespace lbmd {

struct CellXYZ {
    int x, y, z;
};

__device__ __forceinline__ CellXYZ cell_xyz(int64_t cell, const FastDiv &fnx, const FastDiv &fny) {
    const uint32_t c = (uint32_t)cell;
    const uint32_t row = fdiv(c, fnx);
    CellXYZ r;
    r.x = (int)(c - row * fnx.d);
    r.z = (int)fdiv(row, fny);
    r.y = (int)(row - (uint32_t)r.z * fny.d);
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

// The 4 lattice rows (y, z) of the corners, q = oy + 2 oz (corners 2q, 2q+1).
__device__ __forceinline__ void corner_rows(const CellXYZ &c, int ny, int nz, uint32_t rows[4]) {
    const int y1 = c.y + 1 == ny ? 0 : c.y + 1;
    const int z1 = c.z + 1 == nz ? 0 : c.z + 1;
    rows[0] = (uint32_t)c.y + (uint32_t)ny * (uint32_t)c.z;
    rows[1] = (uint32_t)y1 + (uint32_t)ny * (uint32_t)c.z;
    rows[2] = (uint32_t)c.y + (uint32_t)ny * (uint32_t)z1;
    rows[3] = (uint32_t)y1 + (uint32_t)ny * (uint32_t)z1;
}

// Move a fractional coordinate by dt v and carry whole cells into the index.
// The drift frac + dt v is one explicit fused multiply-add, so every kernel
// that moves particles rounds it the same way whatever the compiler would
// contract.
template <typename T>
__device__ __forceinline__ void advance(T &frac, int &c, T dt, T v, int n) {
    T x = fma(dt, v, frac);
    T s = floor(x);
    x -= s;
    if (x >= T(1)) {  // a tiny negative offset rounded up to the next node
        x = T(0);
        s += T(1);
    }
    int cn = c + (int)s;
    if (cn < 0 || cn >= n) {  // crossed the periodic boundary
        cn %= n;
        if (cn < 0) cn += n;
    }
    frac = x;
    c = cn;
}

// The transfer -delta_k Delta P of Eqs. (7), (8) in fixed point; every
// spreading path computes it this way (sx = F_x neg_scale_dt etc., equal to
// -s dt F_x for the fixed-point scale s because s is a power of two).
template <typename T>
__device__ __forceinline__ void spread_to(typename Prec<T>::node4 *field, const uint32_t idx[8], const T delta[8], T sx,
                                          T sy, T sz) {
    using P = Prec<T>;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        P::add_transfer(&field[idx[k]], P::to_fix_neg(delta[k], sx), P::to_fix_neg(delta[k], sy),
                        P::to_fix_neg(delta[k], sz));
}

// A position given in FP64 (any real number) -> cell index + fractional
// offset in the storage precision: wrapped into the box, and moved to the
// next node when the offset rounds up to 1.
template <typename T>
__device__ __forceinline__ typename Prec<T>::real4 pos_from_double(const double *x3, int nx, int ny, int nz) {
    const double L[3] = {(double)nx, (double)ny, (double)nz};
    T fr[3];
    int64_t cl[3];
    for (int d = 0; d < 3; ++d) {
        double x = x3[d];
        if (!(x >= 0.0 && x < L[d])) {  // outside the box: wrap (inside, this changes nothing)
            x -= L[d] * floor(x / L[d]);
            if (x >= L[d]) x -= L[d];
        }
        double b = floor(x);
        T f = (T)(x - b);
        if (f >= T(1)) {  // rounding to the storage precision reached the next node
            f = T(0);
            b += 1.0;
            if (b >= L[d]) b = 0.0;
        }
        fr[d] = f;
        cl[d] = (int64_t)b;
    }
    return Prec<T>::make_pos(fr[0], fr[1], fr[2], cl[0] + (int64_t)nx * (cl[1] + (int64_t)ny * cl[2]));
}

__device__ __forceinline__ void fix_add(int32_t *a, int32_t v) { atomicAdd(a, v); }
__device__ __forceinline__ void fix_add(long long *a, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(a), (unsigned long long)v);
}

}  // namespace lbmd
