// convert.cuh -- exact conversions between the FP64 host arrays of the C ABI
// and the FP32 device storage, on the integer pipes (bit-field arithmetic),
// and the FP32-pair sums of the particle moments.
#pragma once

#include "lbmd_device.cuh"
#include "particle_core.cuh"

namespace lbmd {

// ---------------------------------------------------------------------------
// Exact conversions between FP32 and FP64 on the integer pipes.  The FP64
// pipes of this GPU issue a small fraction of the integer rate, so the host
// accessors' per-particle conversions build the results from the IEEE 754
// binary32 / binary64 bit fields instead; every result equals the hardware
// conversion (round to nearest even where rounding occurs).  Inputs outside
// the handled ranges (subnormal results, non-finite values) take the
// hardware conversion.
// ---------------------------------------------------------------------------

// The hardware conversions for the rare inputs outside the bit-field paths,
// as volatile PTX so that the compiler keeps them inside their branches
// instead of evaluating them for every element on the FP64 pipe.
__device__ __forceinline__ double hw_f32_to_f64(float v) {
    double r;
    asm volatile("cvt.f64.f32 %0, %1;" : "=d"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float hw_f64_to_f32(double v) {
    float r;
    asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(r) : "d"(v));
    return r;
}

// FP32 -> FP64 (exact): exponent re-biased by 1023 - 127, the 23 fraction
// bits moved to the top of the 52.
__device__ __forceinline__ double exact_double(float v) {
    const uint32_t b = __float_as_uint(v);
    const uint32_t ex = (b >> 23) & 0xffu;
    if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    if (ex == 0u || ex == 0xffu) return hw_f32_to_f64(v);
    const uint32_t hi = (b & 0x80000000u) | ((ex + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

// an unsigned integer -> FP64 (exact): the leading bit becomes the implicit one
__device__ __forceinline__ double exact_double(uint32_t x) {
    if (x == 0u) return 0.0;
    const int e = 31 - __clz(x);
    const uint64_t frac = ((uint64_t)x << (52 - e)) & ((1ull << 52) - 1);
    return __longlong_as_double((long long)(((uint64_t)(e + 1023) << 52) | frac));
}

// the FP64 add for a subnormal offset (out of line: kept off the common path)
static __device__ __noinline__ double cell_plus_subnormal(uint32_t x, float f) { return (double)x + (double)f; }

// x + f rounded to nearest even as an FP64 value, for an integer x and an
// FP32 f in [0, 1): the 53-bit significand is x's bits followed by the
// leading fraction bits of f, rounded on the bits of f below them.
__device__ __forceinline__ double cell_plus_fraction(uint32_t x, float f) {
    const uint32_t fb = __float_as_uint(f);
    if (fb == 0u) return exact_double(x);
    if (x == 0u) return exact_double(f);
    const int ex = (int)(fb >> 23);
    if (ex == 0) return cell_plus_subnormal(x, f);
    const uint64_t m = (fb & 0x7fffffu) | 0x800000u;  // f = m 2^(ex - 150)
    const int b = 32 - __clz(x);                       // x + f lies in [2^(b-1), 2^b]
    const int s = 97 - ex + b;                         // m's bits below the significand's last
    uint64_t sig = (uint64_t)x << (53 - b);
    if (s <= 0) {
        sig |= m << (-s);
    } else if (s < 64) {
        sig |= m >> s;
        const uint64_t rem = m & ((1ull << s) - 1), half = 1ull << (s - 1);
        if (rem > half || (rem == half && (sig & 1ull))) sig += 1;
    }  // s >= 64: m < 2^24 is below half a unit of the last place
    int e = b - 1;
    if (sig >> 53) {  // rounded up to 2^b
        sig >>= 1;
        e += 1;
    }
    return __longlong_as_double((long long)(((uint64_t)(e + 1023) << 52) | (sig & ((1ull << 52) - 1))));
}

// F 2^-k (0 < F < 2^53) rounded to nearest even as FP32 bits; the result
// must lie in the normal range (exponent field 1..254 before rounding).
__device__ __forceinline__ uint32_t fixed_to_float_bits(uint64_t F, int k) {
    const int p = 63 - __clzll((long long)F);
    uint32_t e = (uint32_t)(p - k + 127);
    uint64_t sig;
    if (p <= 23) {
        sig = F << (23 - p);
    } else {
        const int s = p - 23;
        sig = F >> s;
        const uint64_t rem = F & ((1ull << s) - 1), half = 1ull << (s - 1);
        if (rem > half || (rem == half && (sig & 1ull))) sig += 1;
        if (sig >> 24) {
            sig >>= 1;
            e += 1;
        }
    }
    return (e << 23) | ((uint32_t)sig & 0x7fffffu);
}

// FP64 -> FP32, rounded to nearest even
__device__ __forceinline__ float round_to_float(double v) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ffu);
    if ((b << 1) == 0ull) return __uint_as_float((uint32_t)(b >> 32));  // signed zero
    if (ex < 897 || ex > 1150) return hw_f64_to_f32(v);  // subnormal or overflowing result, non-finite input
    const uint64_t mant = (b & ((1ull << 52) - 1)) | (1ull << 52);
    return __uint_as_float((uint32_t)(b >> 32 & 0x80000000u) | fixed_to_float_bits(mant, 1075 - ex));
}

// an FP64 value in the storage precision (rounded to nearest even)
__device__ __forceinline__ float to_storage(double v, float) { return round_to_float(v); }
__device__ __forceinline__ double to_storage(double v, double) { return v; }

// one coordinate by the FP64 form of pos_from_double (out of line: kept off
// the common path)
static __device__ __noinline__ void pos_coord_fp64(double x, int L, uint32_t &fbits, uint32_t &c) {
    const double Ld = (double)L;
    if (!(x >= 0.0 && x < Ld)) {
        x -= Ld * floor(x / Ld);
        if (x >= Ld) x -= Ld;
    }
    double fl = floor(x);
    float f = (float)(x - fl);
    if (f >= 1.0f) {
        f = 0.0f;
        fl += 1.0;
        if (fl >= Ld) fl = 0.0;
    }
    fbits = __float_as_uint(f);
    c = (uint32_t)(int64_t)fl;
}

// pos_from_double for FP32 storage on the integer pipes: for 0 <= x < L the integer
// part and the fraction bits are read off the binary64 fields and the
// fraction rounded to FP32 (nearest even), as the FP64 form computes them;
// other inputs (outside the box, subnormal offsets) take the FP64 form.
__device__ __forceinline__ Prec<float>::real4 pos_from_double_fp32(const double *x3, int nx, int ny, int nz) {
    const int L[3] = {nx, ny, nz};
    float fr[3];
    int64_t cl[3];
    for (int d = 0; d < 3; ++d) {
        const uint64_t b = (uint64_t)__double_as_longlong(x3[d]);
        const int ex = (int)(b >> 52);  // sign bit included: negative inputs fail the tests below
        const uint64_t mant = (b & ((1ull << 52) - 1)) | (1ull << 52);
        uint32_t c = 0, fbits = 0;
        bool ok = (b << 1) == 0ull || (ex >= 897 && ex <= 1054);  // +-0, or 2^-126 <= x < 2^32
        if (ok && (b << 1) != 0ull) {
            if (ex < 1023) {  // x < 1: the offset is x itself
                fbits = fixed_to_float_bits(mant, 1075 - ex);
            } else {
                const int k = 1075 - ex;  // fraction bits of x (<= 52)
                c = (uint32_t)(mant >> k);
                const uint64_t F = mant & ((1ull << k) - 1);
                if (F != 0ull) {
                    const int p = 63 - __clzll((long long)F);
                    if (p - k + 127 >= 1) fbits = fixed_to_float_bits(F, k);
                    else ok = false;  // offset below FP32's normal range
                }
            }
            if (fbits == 0x3f800000u) {  // the offset rounded up to 1: the next node
                fbits = 0u;
                c += 1u;
            }
            ok = ok && c < (uint32_t)L[d];
        }
        if (!ok) pos_coord_fp64(x3[d], L[d], fbits, c);  // outside the box or a subnormal offset
        fr[d] = __uint_as_float(fbits);
        cl[d] = (int64_t)c;
    }
    return Prec<float>::make_pos(fr[0], fr[1], fr[2], cl[0] + (int64_t)nx * (cl[1] + (int64_t)ny * cl[2]));
}

// ---------------------------------------------------------------------------
// Sums of FP32 values kept as unevaluated pairs hi + lo of FP32 values -- hi
// the running sum, lo the exact rounding errors of its additions (Knuth's
// two-sum) and of the products (FMA) -- about 44 significant bits on the
// FP32 pipes, for the particle sums of the FP32 forms.
// ---------------------------------------------------------------------------
struct FF {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float s = __fadd_rn(hi, x);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ void add(float x, float err) {
        add(x);
        lo = __fadd_rn(lo, err);
    }
};

// m v (three components, s[0..2]) and m v^2 (s[3]) of one particle with
// velocity (vx, vy, vz) and w = 1/m; m as the pair of the rounded reciprocal
// and its residual
__device__ __forceinline__ void add_particle_moments(FF s[4], float vx, float vy, float vz, float w) {
    const float mh = __frcp_rn(w);
    const float ml = __fmul_rn(__fmaf_rn(-mh, w, 1.0f), mh);
    const float c[3] = {vx, vy, vz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float mv = __fmul_rn(mh, c[d]);  // m v = mv + mve
        const float mve = __fmaf_rn(ml, c[d], __fmaf_rn(mh, c[d], -mv));
        s[d].add(mv, mve);
        const float q = __fmul_rn(mv, c[d]);  // m v^2 = q + qe
        s[3].add(q, __fmaf_rn(mve, c[d], __fmaf_rn(mv, c[d], -q)));
    }
}

// The block's totals of NV pairs in a fixed order (a butterfly within each
// warp, then the warps in order), as doubles in thread 0's out[]
template <int THREADS, int NV>
__device__ __forceinline__ void ff_block_sum(FF s[NV], double out[NV]) {
    __shared__ float sh[THREADS / 32][NV][2];
#pragma unroll
    for (int c = 0; c < NV; ++c)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float h = __shfl_xor_sync(0xffffffffu, s[c].hi, off);
            const float l = __shfl_xor_sync(0xffffffffu, s[c].lo, off);
            s[c].add(h, l);
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            sh[threadIdx.x >> 5][c][0] = s[c].hi;
            sh[threadIdx.x >> 5][c][1] = s[c].lo;
        }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            FF t;
            for (int w = 0; w < THREADS / 32; ++w) t.add(sh[w][c][0], sh[w][c][1]);
            out[c] = exact_double(t.hi) + exact_double(t.lo);
        }
}

template <typename T>
__device__ __forceinline__ typename Prec<T>::real4 pos_from_host(const double *x3, int nx, int ny, int nz);
template <>
__device__ __forceinline__ Prec<float>::real4 pos_from_host<float>(const double *x3, int nx, int ny, int nz) {
    return pos_from_double_fp32(x3, nx, ny, nz);
}
template <>
__device__ __forceinline__ Prec<double>::real4 pos_from_host<double>(const double *x3, int nx, int ny, int nz) {
    return pos_from_double<double>(x3, nx, ny, nz);
}

}  // namespace lbmd
