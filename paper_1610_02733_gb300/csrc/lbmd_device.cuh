// lbmd_device.cuh -- device building blocks of the GB300 LB/MD library:
// D3Q19 lattice and mode basis (Sec. 2), Philox4x32-10 counter-based noise,
// the per-precision storage policy and the fixed-point encoding of the
// momentum density.
//
// Fixed-point momentum.  The node field stores the momentum density j as a
// signed integer multiple of the unit 2^(e - 30) (FP32 build) or 2^(e - 56)
// (FP64 build), e = ceil(log2 rho0), the smallest power of two at or above
// the reference density.  Particle-to-fluid transfers (Eqs. (7), (8) of the
// paper) are added with integer atomics, which are associative: the
// accumulated value does not depend on the order in which particles are
// processed, so every run is bitwise reproducible without a fixed particle
// order or colouring.  Range: |j| < 2^(e + 1) (FP32) and |j| < 2^(e + 7)
// (FP64), i.e. a node velocity |u| = |j| / rho below 2 (FP32) / 128 (FP64)
// at rho = rho0, far above any flow an LB fluid can carry (the lattice Mach
// number must stay well below one).  The scale s = 1 / unit and its inverse
// are run-time arguments of every kernel that converts (both exact powers of
// two, so moving the scale or a sign onto a factor is exact).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbmd {

constexpr int Q = 19;

// D3Q19 velocities c_i (Sec. 2, Fig. 1a): rest, 6 nearest, 12 next-nearest.
__host__ __device__ constexpr int CX(int i) {
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int CY(int i) {
    constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int CZ(int i) {
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
}
__host__ __device__ constexpr int C2(int i) { return CX(i) * CX(i) + CY(i) * CY(i) + CZ(i) * CZ(i); }

// Lattice weights: 1/3 (rest), 1/18 (|c|^2 = 1), 1/36 (|c|^2 = 2).
__host__ __device__ constexpr double WEIGHT(int i) {
    return C2(i) == 0 ? 1.0 / 3.0 : (C2(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Orthogonal mode basis e_k(c_i): 0 mass, 1-3 momentum, 4 bulk stress,
// 5-9 shear stress, 10-18 ghost modes.  Integer-valued.
__host__ __device__ constexpr int EMODE(int k, int i) {
    const int x = CX(i), y = CY(i), z = CZ(i), c2 = C2(i);
    return k == 0    ? 1
           : k == 1  ? x
           : k == 2  ? y
           : k == 3  ? z
           : k == 4  ? c2 - 1
           : k == 5  ? 3 * x * x - c2
           : k == 6  ? y * y - z * z
           : k == 7  ? x * y
           : k == 8  ? x * z
           : k == 9  ? y * z
           : k == 10 ? (3 * c2 - 5) * x
           : k == 11 ? (3 * c2 - 5) * y
           : k == 12 ? (3 * c2 - 5) * z
           : k == 13 ? (y * y - z * z) * x
           : k == 14 ? (z * z - x * x) * y
           : k == 15 ? (x * x - y * y) * z
           : k == 16 ? 3 * c2 * c2 - 6 * c2 + 1
           : k == 17 ? (2 * c2 - 3) * (3 * x * x - c2)
                     : (2 * c2 - 3) * (y * y - z * z);
}

// Squared norms b_k = sum_i w_i e_k(c_i)^2, as exact rationals.
__host__ __device__ constexpr double BNORM(int k) {
    constexpr double t[Q] = {1.0,       1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 2.0 / 3.0, 4.0 / 3.0, 4.0 / 9.0,
                             1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 2.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 2.0 / 9.0,
                             2.0 / 9.0, 2.0 / 9.0, 2.0,       4.0 / 3.0, 4.0 / 9.0};
    return t[k];
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply-xor bijection with Weyl-sequence key updates.
// ---------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// 32 random bits -> uniform number with zero mean and unit variance,
// sqrt(12) ((x + 1/2) 2^-32 - 1/2).  The FP64 form is exact; the FP32 form
// centres first, (x - 2^31 + 1/2) 2^-32, so only one rounding remains.
__device__ __forceinline__ double unit_uniform_d(uint32_t x) {
    return 3.4641016151377544 * (((double)x + 0.5) * 2.3283064365386963e-10 - 0.5);
}
__device__ __forceinline__ float unit_uniform_f(uint32_t x) {
    const float centred = (float)(int32_t)(x ^ 0x80000000u) + 0.5f;
    return centred * (3.4641016151377544f * 2.3283064365386963e-10f);
}
// Two 32-bit Philox words -> two independent standard normal variates
// (Box & Muller, Ann. Math. Stat. 29 (1958) 610): u = (h + 1/2) 2^-24 from the
// top 24 bits h of each word (exact in FP32), r = sqrt(-2 ln u1), and the pair
// (r cos 2 pi u2, r sin 2 pi u2) from the device's log and sincospi.
__device__ __forceinline__ void box_muller(uint32_t w1, uint32_t w2, float &a, float &b) {
    const float u1 = ((float)(w1 >> 8) + 0.5f) * 5.9604644775390625e-8f;
    const float u2 = ((float)(w2 >> 8) + 0.5f) * 5.9604644775390625e-8f;
    const float r = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    a = r * cs;
    b = r * sn;
}
__device__ __forceinline__ void box_muller(uint32_t w1, uint32_t w2, double &a, double &b) {
    const double u1 = ((double)(w1 >> 8) + 0.5) * 5.9604644775390625e-8;
    const double u2 = ((double)(w2 >> 8) + 0.5) * 5.9604644775390625e-8;
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    a = r * cs;
    b = r * sn;
}

template <typename T>
__device__ __forceinline__ T unit_uniform(uint32_t x);
template <>
__device__ __forceinline__ float unit_uniform<float>(uint32_t x) {
    return unit_uniform_f(x);
}
template <>
__device__ __forceinline__ double unit_uniform<double>(uint32_t x) {
    return unit_uniform_d(x);
}

// ---------------------------------------------------------------------------
// Storage policy per precision.
// ---------------------------------------------------------------------------
struct __align__(32) D4 {
    double x, y, z, w;
};
struct __align__(32) L4 {
    long long x, y, z, w;
};

template <typename T>
struct Prec;

// FP32 node record (16 bytes, one int4): word 0 holds rho as float bits,
// word 1 j_z, words 2-3 one signed 64-bit integer S = j_y 2^32 + j_x (all in
// units of 2^(e - 30)).  The low word of S is j_x itself; the high word is j_y,
// minus one when j_x is negative.  Because S is an ordinary integer sum, a
// transfer (dx, dy, dz) is added with two atomics, one 64-bit add of
// dy 2^32 + dx and one 32-bit add of dz, and the fields stay exact as long as
// each one stays within its 32-bit range.
template <>
struct Prec<float> {
    using real = float;
    using real4 = float4;
    using fix = int32_t;
    using node4 = int4;
    static constexpr int SCALE_LOG2 = 30;  // scale at rho0 <= 1: 2^30
    // j -> fixed point with the scale s (a power of two)
    __device__ static __forceinline__ fix to_fix(float v, float s) { return __float2int_rn(v * s); }
    // to_fix(-d * dp, s) for ps = -s dp: the power-of-two scale and the sign
    // move onto dp, which is exact, so the two are bitwise equal
    __device__ static __forceinline__ fix to_fix_neg(float d, float ps) { return __float2int_rn(d * ps); }
    __device__ static __forceinline__ float from_fix(fix v, float inv_s) { return (float)v * inv_s; }
    // |v| >= 2^30, half the range of a field: the range guard's test
    __device__ static __forceinline__ bool beyond_half(fix v) {
        return (uint32_t)v + 0x40000000u >= 0x80000000u;
    }
    __device__ static __forceinline__ node4 pack(float rho, fix jx, fix jy, fix jz) {
        const long long S = (long long)jy * 4294967296LL + (long long)jx;
        return make_int4(__float_as_int(rho), jz, (int)(unsigned)(unsigned long long)S, (int)(S >> 32));
    }
    __device__ static __forceinline__ float rho_of(const node4 &n) { return __int_as_float(n.x); }
    __device__ static __forceinline__ fix jx_of(const node4 &n) { return n.z; }
    __device__ static __forceinline__ fix jy_of(const node4 &n) { return n.w + (n.z < 0 ? 1 : 0); }
    __device__ static __forceinline__ fix jz_of(const node4 &n) { return n.y; }
    __device__ static __forceinline__ void add_transfer(node4 *rec, fix dx, fix dy, fix dz) {
        const long long S = (long long)dy * 4294967296LL + (long long)dx;
        atomicAdd(reinterpret_cast<unsigned long long *>(&rec->z), (unsigned long long)S);
        atomicAdd(&rec->y, dz);
    }
    // the same update by a thread that owns the record (no concurrent writer)
    __device__ static __forceinline__ void add_transfer_reg(node4 &n, fix dx, fix dy, fix dz) {
        const long long S = (long long)(((unsigned long long)(unsigned)n.w << 32) | (unsigned)n.z) +
                            ((long long)dy * 4294967296LL + (long long)dx);
        n.y += dz;
        n.z = (int)(unsigned)(unsigned long long)S;
        n.w = (int)(S >> 32);
    }
    __device__ static __forceinline__ void add_transfer_plain(node4 *rec, fix dx, fix dy, fix dz) {
        int4 n = *rec;
        add_transfer_reg(n, dx, dy, dz);
        *rec = n;
    }
    __device__ static __forceinline__ real4 make4(float a, float b, float c, float d) {
        return make_float4(a, b, c, d);
    }
    // particle position record: frac x, y, z in [0,1) and the cell index
    __device__ static __forceinline__ int64_t cell_of(const real4 &p) { return (int64_t)(uint32_t)__float_as_int(p.w); }
    __device__ static __forceinline__ real4 make_pos(float fx, float fy, float fz, int64_t cell) {
        return make_float4(fx, fy, fz, __int_as_float((int)(uint32_t)cell));
    }
};

// FP64 node record (32 bytes): rho as double bits, then j_x, j_y, j_z as
// signed 64-bit integers in units of 2^(e - 56); a transfer is three atomics.
template <>
struct Prec<double> {
    using real = double;
    using real4 = D4;
    using fix = long long;
    using node4 = L4;
    static constexpr int SCALE_LOG2 = 56;  // scale at rho0 <= 1: 2^56
    __device__ static __forceinline__ fix to_fix(double v, double s) { return __double2ll_rn(v * s); }
    __device__ static __forceinline__ fix to_fix_neg(double d, double ps) { return __double2ll_rn(d * ps); }
    __device__ static __forceinline__ double from_fix(fix v, double inv_s) { return (double)v * inv_s; }
    // |v| >= 2^62, half the range of a field
    __device__ static __forceinline__ bool beyond_half(fix v) {
        return (unsigned long long)v + 0x4000000000000000ull >= 0x8000000000000000ull;
    }
    __device__ static __forceinline__ node4 pack(double rho, fix jx, fix jy, fix jz) {
        return L4{__double_as_longlong(rho), jx, jy, jz};
    }
    __device__ static __forceinline__ double rho_of(const node4 &n) { return __longlong_as_double(n.x); }
    __device__ static __forceinline__ fix jx_of(const node4 &n) { return n.y; }
    __device__ static __forceinline__ fix jy_of(const node4 &n) { return n.z; }
    __device__ static __forceinline__ fix jz_of(const node4 &n) { return n.w; }
    __device__ static __forceinline__ void add_transfer(node4 *rec, fix dx, fix dy, fix dz) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&rec->y), (unsigned long long)dx);
        atomicAdd(reinterpret_cast<unsigned long long *>(&rec->z), (unsigned long long)dy);
        atomicAdd(reinterpret_cast<unsigned long long *>(&rec->w), (unsigned long long)dz);
    }
    __device__ static __forceinline__ void add_transfer_reg(node4 &n, fix dx, fix dy, fix dz) {
        n.y += dx;
        n.z += dy;
        n.w += dz;
    }
    __device__ static __forceinline__ void add_transfer_plain(node4 *rec, fix dx, fix dy, fix dz) {
        L4 n = *rec;
        add_transfer_reg(n, dx, dy, dz);
        *rec = n;
    }
    __device__ static __forceinline__ real4 make4(double a, double b, double c, double d) { return D4{a, b, c, d}; }
    __device__ static __forceinline__ int64_t cell_of(const real4 &p) { return (int64_t)p.w; }
    __device__ static __forceinline__ real4 make_pos(double fx, double fy, double fz, int64_t cell) {
        return D4{fx, fy, fz, (double)cell};
    }
};

// ---------------------------------------------------------------------------
// Population storage.  FP32 / FP64 store f_i itself.  The reduced-precision
// forms store the deviation from the rest equilibrium, f_i - w_i rho0, as FP16
// or BF16 and do all arithmetic in FP32: the deviations are small (thermal
// and flow perturbations), so the 11- or 8-bit significand is spent on them
// rather than on the constant w_i rho0.  The collision's stores round the
// deviation to nearest (FP16 / BF16) or stochastically (the _SR forms below);
// every other store (initial and user-given states) rounds to nearest.
// ---------------------------------------------------------------------------
//
// The kernels do their arithmetic on what is stored: f_i itself for the
// plain forms, the deviation for the reduced ones (arith / arith_cg /
// store_arith), so that the mass moment of a deviation form is the FP32 sum of
// small deviations rather than of values near w_i rho0 -- the FP32 sum of the
// latter rounds the same way at every node of a near-uniform fluid, and the
// collision would write that rounding back into the populations every step.
// load / store convert to and from the population itself (host accessors,
// initial state).
template <typename S, typename T>
struct PopStore {  // plain storage: S == T
    __device__ static __forceinline__ T load(const S *p, T /*base*/) { return *p; }
    __device__ static __forceinline__ T load_cg(const S *p, T /*base*/) { return __ldcg(p); }
    __device__ static __forceinline__ void store(S *p, T v, T /*base*/) { *p = v; }
    __device__ static __forceinline__ T arith(const S *p) { return *p; }
    __device__ static __forceinline__ T arith_cg(const S *p) { return __ldcg(p); }
    __device__ static __forceinline__ void store_arith(S *p, T v) { *p = v; }
    static constexpr bool deviation = false;
    static constexpr bool stochastic = false;
};

// Stochastic rounding of x onto the FP16 / BF16 grid with 16 random bits r:
// with lo the grid value next to x towards zero and hi the next one away from
// zero, the result is hi when r < 2^16 (|x| - |lo|) / (|hi| - |lo|), else lo
// (Forsythe 1959; Connolly, Higham & Mary, SIAM J. Sci. Comput. 43 (2021)):
// unbiased, E[result] = x up to 2^-16 of a grid step.  For an FP32 x the
// fraction times 2^16 is exact, so the comparison is exact.
__device__ __forceinline__ __nv_bfloat16 bf16_round_stochastic(float x, uint32_t r) {
    // BF16 is the top half of FP32: the dropped 16 bits are the fraction
    const uint32_t bits = __float_as_uint(x), mag = bits & 0x7fffffffu;
    const uint32_t up = r < (mag & 0xffffu) ? 1u : 0u;
    return __ushort_as_bfloat16((unsigned short)(((bits >> 16) & 0x8000u) | ((mag >> 16) + up)));
}
__device__ __forceinline__ __half fp16_round_stochastic(float x, uint32_t r) {
    const float a = fabsf(x);
    const unsigned short lo = __half_as_ushort(__float2half_rz(a));  // towards zero, subnormals included
    const float lo_f = __half2float(__ushort_as_half(lo));
    // the grid step above lo, a power of two 2^k (k >= -24), and 2^16 / step
    // = 2^(16 - k) built from its exponent field: the product below is exact
    const float step = __half2float(__ushort_as_half((unsigned short)(lo + 1))) - lo_f;
    const float t = (a - lo_f) * __uint_as_float(0x87000000u - __float_as_uint(step));  // a - lo_f exact (Sterbenz)
    // r < t with r < 2^16 as the float 2^23 + r - 2^23 (exact, no conversion)
    const float rf = __uint_as_float(0x4B000000u | r) - 8388608.0f;
    const unsigned short up = (lo < 0x7bffu && rf < t) ? 1 : 0;
    const unsigned short sign = (unsigned short)((__float_as_uint(x) >> 16) & 0x8000u);
    return __ushort_as_half((unsigned short)(sign | (lo + up)));
}

// Storage tags of the stochastically rounded forms (same bits as __half /
// __nv_bfloat16).
struct half_sr {
    unsigned short u;
};
struct bf16_sr {
    unsigned short u;
};
template <>
struct PopStore<__half, float> {
    __device__ static __forceinline__ float load(const __half *p, float base) { return base + __half2float(*p); }
    __device__ static __forceinline__ float load_cg(const __half *p, float base) {
        return base + __half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __forceinline__ void store(__half *p, float v, float base) { *p = __float2half_rn(v - base); }
    __device__ static __forceinline__ float arith(const __half *p) { return __half2float(*p); }
    __device__ static __forceinline__ float arith_cg(const __half *p) {
        return __half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __forceinline__ void store_arith(__half *p, float d) { *p = __float2half_rn(d); }
    static constexpr bool deviation = true;
    static constexpr bool stochastic = false;
};
template <>
struct PopStore<__nv_bfloat16, float> {
    __device__ static __forceinline__ float load(const __nv_bfloat16 *p, float base) {
        return base + __bfloat162float(*p);
    }
    __device__ static __forceinline__ float load_cg(const __nv_bfloat16 *p, float base) {
        return base + __bfloat162float(__ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __forceinline__ void store(__nv_bfloat16 *p, float v, float base) {
        *p = __float2bfloat16_rn(v - base);
    }
    __device__ static __forceinline__ float arith(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    __device__ static __forceinline__ float arith_cg(const __nv_bfloat16 *p) {
        return __bfloat162float(__ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __forceinline__ void store_arith(__nv_bfloat16 *p, float d) { *p = __float2bfloat16_rn(d); }
    static constexpr bool deviation = true;
    static constexpr bool stochastic = false;
};
template <>
struct PopStore<half_sr, float> {
    __device__ static __forceinline__ float load(const half_sr *p, float base) {
        return base + __half2float(__ushort_as_half(p->u));
    }
    __device__ static __forceinline__ float load_cg(const half_sr *p, float base) {
        return base + __half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __forceinline__ void store(half_sr *p, float v, float base) {
        p->u = __half_as_ushort(__float2half_rn(v - base));
    }
    __device__ static __forceinline__ float arith(const half_sr *p) { return __half2float(__ushort_as_half(p->u)); }
    __device__ static __forceinline__ float arith_cg(const half_sr *p) {
        return __half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __forceinline__ void store_arith(half_sr *p, float d) {
        p->u = __half_as_ushort(__float2half_rn(d));
    }
    // r: 16 random bits
    __device__ static __forceinline__ void store_arith_sr(half_sr *p, float d, uint32_t r) {
        p->u = __half_as_ushort(fp16_round_stochastic(d, r));
    }
    static constexpr bool deviation = true;
    static constexpr bool stochastic = true;
};
template <>
struct PopStore<bf16_sr, float> {
    __device__ static __forceinline__ float load(const bf16_sr *p, float base) {
        return base + __bfloat162float(__ushort_as_bfloat16(p->u));
    }
    __device__ static __forceinline__ float load_cg(const bf16_sr *p, float base) {
        return base + __bfloat162float(__ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __forceinline__ void store(bf16_sr *p, float v, float base) {
        p->u = __bfloat16_as_ushort(__float2bfloat16_rn(v - base));
    }
    __device__ static __forceinline__ float arith(const bf16_sr *p) {
        return __bfloat162float(__ushort_as_bfloat16(p->u));
    }
    __device__ static __forceinline__ float arith_cg(const bf16_sr *p) {
        return __bfloat162float(__ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __forceinline__ void store_arith(bf16_sr *p, float d) {
        p->u = __bfloat16_as_ushort(__float2bfloat16_rn(d));
    }
    __device__ static __forceinline__ void store_arith_sr(bf16_sr *p, float d, uint32_t r) {
        p->u = __bfloat16_as_ushort(bf16_round_stochastic(d, r));
    }
    static constexpr bool deviation = true;
    static constexpr bool stochastic = true;
};

// Hydrodynamic moments rho = sum f_i, j = sum f_i c_i (Eqs. (1), (2)).  One
// fixed summation order, shared by every kernel that needs them, so the
// values are bitwise identical wherever they are recomputed.
template <typename T>
__device__ __forceinline__ void node_moments(const T f[Q], T &rho, T &jx, T &jy, T &jz) {
    rho = f[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) rho += f[i];
    jx = (f[1] - f[2]) + (f[7] - f[8]) + (f[9] - f[10]) + (f[11] - f[12]) + (f[13] - f[14]);
    jy = (f[3] - f[4]) + (f[7] - f[8]) + (f[10] - f[9]) + (f[15] - f[16]) + (f[17] - f[18]);
    jz = (f[5] - f[6]) + (f[11] - f[12]) + (f[14] - f[13]) + (f[15] - f[16]) + (f[18] - f[17]);
}

// The same from the values the arithmetic works on (PopStore::arith): rho_m
// is their sum (the density itself, or, for a deviation form, the density
// minus rho_base = sum_i of the stored rest values) and rho the density.
// The rest values of opposite velocities are equal, so j is the same sum.
template <bool DEV, typename T>
__device__ __forceinline__ void pop_moments(const T f[Q], T rho_base, T &rho, T &rho_m, T &jx, T &jy, T &jz) {
    node_moments(f, rho_m, jx, jy, jz);
    rho = DEV ? rho_base + rho_m : rho_m;
}

// ---------------------------------------------------------------------------
// Unsigned division by a run-time invariant d, 1 <= d < 2^31, with one
// multiply-high, a subtract, an add and two shifts (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, Fig. 4.1):
// with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0), t = mulhi(m, n),
// exact for every 32-bit n.
// ---------------------------------------------------------------------------
struct FastDiv {
    uint32_t d, m, s1, s2;
};
inline FastDiv make_fastdiv(uint32_t d) {
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    FastDiv f;
    f.d = d;
    f.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1ull);
    f.s1 = l < 1 ? l : 1u;
    f.s2 = l > 1 ? l - 1u : 0u;
    return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f) {
    const uint32_t t = __umulhi(f.m, n);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// ---------------------------------------------------------------------------
// Active nodes of variant B.  Once per LB step, after the particles are
// re-ordered, every node that is a corner of some particle's cell is marked
// active and given a slot in a compact array of node records; during the MD
// steps that compact record, not the node field entry, holds the node's
// (rho, j).  The set is described per lattice row (y, z) and 32-node word:
// uint2 {bits, base}, bit b set if node x = 32 w + b is active, base the slot
// of the word's first active node (slots run in row-major node order).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int active_words(int nx) { return (nx + 31) / 32; }

// compact slot of node x of a row whose word (x / 32) is w, or -1 if inactive
__device__ __forceinline__ int active_slot(uint2 w, int x) {
    const uint32_t b = 1u << (x & 31);
    return (w.x & b) ? (int)w.y + __popc(w.x & (b - 1u)) : -1;
}

}  // namespace lbmd
