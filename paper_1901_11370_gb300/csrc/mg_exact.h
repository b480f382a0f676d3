// mg_exact.h -- exact evaluation of the constant-coefficient 5/7-point sum
//   S = sum_{j=1..M} x_j - M x_0      (x_0 the cell, x_1..x_M its neighbours)
// for FP64 inputs with integer operations only, rounded once to FP64.
//
// GB300 issues FP64 instructions at 1/64 of the FP32 rate, and the FP64
// composite residual of the defect-correction loop (r = f - A phi, Sec. 2.4)
// spends about a dozen of them per cell.  Here every value is aligned to the
// largest exponent among the M + 1 values on a grid 2^-5 of that value's
// ulp (58-bit integers), summed exactly in 64 bits, and converted back with
// round-to-nearest-even: the error is at most 0.5 ulp of S plus 2^-6 ulp of
// the largest input per term, no more than an FP64 evaluation of the same
// sum accumulates.  The caller then forms r = f - S / h^2 with one FMA.
// The residual kernel aligns a whole staged block (values and ghosts) to
// the block's largest exponent once, with mg_fix, and sums per cell in
// integers; exact_lap is the per-cell form of the same arithmetic.
//
// Plain C++ (host and device): the CPU test compiles this header with g++
// and checks it against exact rational arithmetic.
#pragma once
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define MG_HD __host__ __device__ __forceinline__
#else
#define MG_HD inline
#endif

namespace mg {

MG_HD uint64_t mg_bits(double x) {
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    return b;
}
MG_HD double mg_from_bits(uint64_t b) {
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
}
MG_HD int mg_clz64(uint64_t a) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)a);
#else
    return __builtin_clzll(a);
#endif
}

// Biased FP64 exponent field of x (0 for zero and denormals).
MG_HD int mg_expo(double x) { return (int)((mg_bits(x) >> 52) & 0x7FF); }

// x on the fixed-point grid of step 2^(emax - 1080): its 53-bit significand
// shifted left by 5 guard bits, or right (rounded to nearest) when x's
// exponent is below emax; |result| < 2^58 for every x with exponent <= emax.
MG_HD int64_t mg_fix(double x, int emax) {
    const uint64_t b = mg_bits(x);
    const int e = (int)((b >> 52) & 0x7FF);
    const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
    const int sh = emax - (e ? e : 1);  // denormals carry exponent 1 without the hidden bit
    uint64_t t = m << 5;
    if (sh >= 60) t = 0;
    else if (sh > 0) t = (t + (1ull << (sh - 1))) >> sh;
    return (b >> 63) ? -(int64_t)t : (int64_t)t;
}

// S * 2^(emax - 1080) rounded to the nearest FP64 value (ties to even);
// false when the result is outside the normal range.
MG_HD bool mg_unfix(int64_t S, int emax, double &out) {
    if (S == 0) {
        out = 0.0;
        return true;
    }
    const uint64_t a = S < 0 ? (uint64_t)(-S) : (uint64_t)S;
    int p = 63 - mg_clz64(a);
    uint64_t m;
    if (p > 52) {
        const int rb = p - 52;
        m = a >> rb;
        const uint64_t rem = a & ((1ull << rb) - 1), half = 1ull << (rb - 1);
        if (rem > half || (rem == half && (m & 1))) {
            m++;
            if (m == (1ull << 53)) {
                m >>= 1;
                p++;
            }
        }
    } else {
        m = a << (52 - p);
    }
    const int be = p + emax - 57;  // biased exponent: m 2^(p - 52) 2^(emax - 1080) = (m / 2^52) 2^(be - 1023)
    if (be <= 0 || be >= 0x7FF) return false;
    out = mg_from_bits((S < 0 ? (1ull << 63) : 0ull) | ((uint64_t)be << 52) | (m & 0xFFFFFFFFFFFFFull));
    return true;
}

// S for v[0] = x_0 and v[1..M] the neighbours, aligned to the largest
// exponent among them; false for a non-finite input or a result outside the
// normal range (the caller then uses FP64 arithmetic).
template <int M>
MG_HD bool exact_lap(const double *v, double &out) {
    int emax = 1;
#pragma unroll
    for (int j = 0; j <= M; j++) {
        const int e = mg_expo(v[j]);
        emax = e > emax ? e : emax;
    }
    if (emax == 0x7FF) return false;
    int64_t S = -(int64_t)M * mg_fix(v[0], emax);
#pragma unroll
    for (int j = 1; j <= M; j++) S += mg_fix(v[j], emax);
    return mg_unfix(S, emax, out);
}

// FP64 to FP32 rounded to nearest (ties to even) with integer operations
// (GB300 runs the conversion instruction on its FP64 pipe): normal and
// denormal results, overflow to infinity, NaN kept quiet.
MG_HD float mg_to_float(double x) {
    const uint64_t b = mg_bits(x);
    const uint32_t sign = (uint32_t)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7FF);
    const uint64_t m = b & 0xFFFFFFFFFFFFFull;
    uint32_t r;
    if (e == 0x7FF) {
        r = sign | 0x7F800000u | (m ? 0x400000u : 0u);
    } else {
        const int fe = e - 1023 + 127;  // FP32 biased exponent
        if (fe >= 0xFF) {
            r = sign | 0x7F800000u;
        } else if (fe <= 0) {
            // FP32 denormal: the significand (hidden bit included) over 2^(30 - fe)
            const int sh = 30 - fe;
            if (sh > 54 || e == 0) {
                r = sign;
            } else {
                const uint64_t mm = m | (1ull << 52);
                uint64_t q = mm >> sh;
                const uint64_t rem = mm & ((1ull << sh) - 1), half = 1ull << (sh - 1);
                if (rem > half || (rem == half && (q & 1))) q++;
                r = sign | (uint32_t)q;  // q == 2^23 carries into the smallest normal
            }
        } else {
            uint32_t q = (uint32_t)(m >> 29);
            const uint64_t rem = m & ((1ull << 29) - 1), half = 1ull << 28;
            uint32_t bits = ((uint32_t)fe << 23) | q;
            if (rem > half || (rem == half && (q & 1))) bits++;  // a carry rounds into the exponent
            r = sign | bits;
        }
    }
    float f;
    memcpy(&f, &r, sizeof f);
    return f;
}

// FP32 to FP64 (exact) with integer operations: rebias the exponent, widen
// the significand; FP32 denormals are normalised; zeros, infinities and NaN
// keep their class.
MG_HD double mg_from_float(float f) {
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    const int e = (int)((u >> 23) & 0xFF);
    uint64_t m = u & 0x7FFFFFu;
    uint64_t b;
    if (e == 0xFF) {
        b = sign | (0x7FFull << 52) | (m << 29);
    } else if (e == 0) {
        if (m == 0) {
            b = sign;
        } else {  // denormal: value m 2^-149, leading bit at position p
            const int p = 63 - mg_clz64(m);
            const uint64_t frac = (m << (52 - p)) & 0xFFFFFFFFFFFFFull;
            b = sign | ((uint64_t)(p - 149 + 1023) << 52) | frac;
        }
    } else {
        b = sign | ((uint64_t)(e - 127 + 1023) << 52) | (m << 29);
    }
    return mg_from_bits(b);
}

}  // namespace mg
