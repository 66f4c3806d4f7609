// lb_core.cuh -- the MRT collision with thermal noise and forcing at one
// node (Sec. 2 collision operator, Sec. 3 forcing term), shared by the
// single-box LB kernel (lb.cu) and the batched replicas (batch.cu), so that
// both run one instruction sequence.
#pragma once

#include "lbmd_device.cuh"

namespace lbmd {

// Reciprocal norms 1/b_k, exact binary fractions.
__host__ __device__ constexpr double INV_BNORM(int k) {
    constexpr double t[Q] = {1.0, 3.0, 3.0, 3.0, 1.5, 0.75, 2.25, 9.0, 9.0, 9.0,
                             1.5, 1.5, 1.5, 4.5, 4.5, 4.5, 0.5, 0.75, 2.25};
    return t[k];
}
// 1/b_k and the norms b_k of lbmd_device.cuh (which the host's noise
// amplitudes use) are one table: checked at compile time.
constexpr bool inv_bnorm_matches() {
    for (int k = 0; k < Q; ++k)
        if (BNORM(k) * INV_BNORM(k) != 1.0) return false;
    return true;
}
static_assert(inv_bnorm_matches(), "INV_BNORM(k) must be 1 / BNORM(k)");

// The D3Q19 order pairs every moving velocity with its opposite:
// c_{2p+2} = -c_{2p+1}, p = 0..8.  Even modes (0, 4-9, 16-18) see only the
// pair sums s_p = f_{2p+1} + f_{2p+2}, odd modes (1-3, 10-15) only the
// differences d_p = f_{2p+1} - f_{2p+2}; the back-transform likewise returns
// an even part E_p and an odd part O_p with f_{2p+1} = w (E_p + O_p) and
// f_{2p+2} = w (E_p - O_p).  This halves the arithmetic of both transforms.
__host__ __device__ constexpr bool EVEN_MODE(int k) { return k == 0 || (k >= 4 && k <= 9) || k >= 16; }

// MRT collision with forcing and noise at one node; f holds f* on entry and
// f' on exit -- or, for a deviation storage form, f* - b and f' - b with b the
// stored rest values (see PopStore): the collision is linear in the moments,
// and the mass mode takes rho_m (the density, or its part sum_i (f*_i - b_i)),
// while u, the equilibria and the noise amplitudes take the density rho.  With
// sum_i w_i = 1 and sum_i w_i e_k(c_i) = 0 for k > 0 the deviations then keep
// their sum, so the mass is conserved up to the rounding of small numbers.
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
// A: any struct with the members gamma_bulk, gamma_shear, gamma_ghost,
// amp16[Q] and noisy (the single-box, batched and adjoint kernels), and for
// GAUSS (normal variates) ampg[Q]; the Philox key (key0, key1) and counters
// (node, step) come as arguments.
template <typename T, bool RELAX_FULL, typename A, bool GAUSS = false>
__device__ __forceinline__ void collide(T f[Q], T rho, T rho_m, T jx, T jy, T jz, T Fx, T Fy, T Fz, const A &a,
                                        uint32_t key0, uint32_t key1, uint32_t node, uint32_t step) {
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
    mp[0] = rho_m;
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

    if constexpr (GAUSS) {
        if (a.noisy) {
            // 15 normal variates from four Philox calls, a Box-Muller pair
            // per two words, in mode order k = 4..18
#pragma unroll
            for (uint32_t q = 0; q < 4; ++q) {
                const U4 r = philox4x32_10(U4{node, step, 0u, q}, key0, key1);
                T g[4];
                box_muller(r.x, r.y, g[0], g[1]);
                box_muller(r.z, r.w, g[2], g[3]);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int k = 4 + 4 * (int)q + t;
                    if (k < Q) mp[k] += (a.ampg[k] * sr) * g[t];
                }
            }
        }
    } else if (a.noisy) {
        // 15 variates from two Philox calls: two 16-bit halves per 32-bit
        // word, low half first, in mode order k = 4..18.  The variate
        // sqrt(12) ((h + 1/2) 2^-16 - 1/2) is (h - 32767.5) times
        // sqrt(12) 2^-16, folded into amp16[k] = amp[k] sqrt(12) 2^-16.
#pragma unroll
        for (uint32_t q = 0; q < 2; ++q) {
            const U4 r = philox4x32_10(U4{node, step, 0u, q}, key0, key1);
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

}  // namespace lbmd
