// hd_exact.cuh -- exact, order-independent sums of doubles.
//
// The global orientational order Psi_6 = (1/N) sum_j psi_j (Eq. 8) is a mean
// over up to 2^31 values.  Summed in doubles, its last bits would depend on
// the reduction tree, i.e. on the launch shape and the replica layout.  Here
// every value enters a 192-bit two's-complement integer whose least
// significant bit is worth 2^-128: a value of magnitude at least 2^-75 enters
// exactly, a smaller one is truncated toward zero (an error below 2^-128
// each), and integer addition is associative, so the total does not depend on
// the order of the additions.  The total is rounded to double once, to
// nearest with ties to even.  It therefore equals the exactly rounded sum of
// the values unless that exact sum lies within N * 2^-128 of a rounding
// boundary of the result.
//
// Range: terms of magnitude below 2^62 and totals below 2^63 in magnitude.
// A non-finite term, or one of magnitude 2^62 or more, marks the sum invalid
// and its rounded value is NaN.
//
// The functions are __host__ __device__ so that a host program can check the
// arithmetic against exact rational sums without a GPU.
#pragma once

#include <cstdint>
#include <cstring>

namespace hd {

struct Exact192 {
    unsigned long long w0, w1, w2;  // two's complement, w0 least significant, unit 2^-128
    unsigned int bad;                // a term was non-finite or out of range
};

__host__ __device__ __forceinline__ Exact192 exact_zero() { return Exact192{0ull, 0ull, 0ull, 0u}; }

__host__ __device__ __forceinline__ unsigned long long exact_bits(double v) {
#ifdef __CUDA_ARCH__
    return static_cast<unsigned long long>(__double_as_longlong(v));
#else
    unsigned long long u;
    std::memcpy(&u, &v, sizeof u);
    return u;
#endif
}

__host__ __device__ __forceinline__ double exact_from_bits(unsigned long long u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double(static_cast<long long>(u));
#else
    double v;
    std::memcpy(&v, &u, sizeof v);
    return v;
#endif
}

__host__ __device__ __forceinline__ int exact_clz64(unsigned long long a) {
#ifdef __CUDA_ARCH__
    return __clzll(static_cast<long long>(a));
#else
    return a ? __builtin_clzll(a) : 64;
#endif
}

// a += (t0, t1, t2), modulo 2^192.
__host__ __device__ __forceinline__ void exact_add3(Exact192& a, unsigned long long t0, unsigned long long t1,
                                                    unsigned long long t2) {
    const unsigned long long s0 = a.w0 + t0;
    const unsigned long long c0 = s0 < t0 ? 1ull : 0ull;
    const unsigned long long s1a = a.w1 + t1;
    const unsigned long long c1a = s1a < t1 ? 1ull : 0ull;
    const unsigned long long s1 = s1a + c0;
    const unsigned long long c1 = c1a | (s1 < c0 ? 1ull : 0ull);
    a.w0 = s0;
    a.w1 = s1;
    a.w2 = a.w2 + t2 + c1;
}

// a += b (both exact sums).
__host__ __device__ __forceinline__ void exact_merge(Exact192& a, const Exact192& b) {
    exact_add3(a, b.w0, b.w1, b.w2);
    a.bad |= b.bad;
}

// a += v.
__host__ __device__ __forceinline__ void exact_add(Exact192& a, double v) {
    const unsigned long long bits = exact_bits(v);
    const int ex = int((bits >> 52) & 0x7ffu);
    if (ex >= 1023 + 62) {  // infinity, NaN or |v| >= 2^62
        a.bad = 1u;
        return;
    }
    unsigned long long man = bits & ((1ull << 52) - 1ull);
    int e;  // |v| = man * 2^e
    if (ex == 0) {
        e = -1074;
    } else {
        man |= 1ull << 52;
        e = ex - 1075;
    }
    const int s = e + 128;  // bit of the accumulator that holds man's bit 0 (at most 137)
    unsigned long long t0 = 0ull, t1 = 0ull, t2 = 0ull;
    if (s < 0) {
        t0 = (s <= -64) ? 0ull : (man >> (-s));
    } else if (s < 64) {
        t0 = man << s;
        t1 = (s == 0) ? 0ull : (man >> (64 - s));
    } else if (s < 128) {
        const int u = s - 64;
        t1 = man << u;
        t2 = (u == 0) ? 0ull : (man >> (64 - u));
    } else {
        t2 = man << (s - 128);
    }
    if (bits >> 63) {  // subtract: add the two's complement of the magnitude
        t0 = ~t0;
        t1 = ~t1;
        t2 = ~t2;
        exact_add3(a, t0, t1, t2);
        exact_add3(a, 1ull, 0ull, 0ull);
    } else {
        exact_add3(a, t0, t1, t2);
    }
}

// The sum rounded to the nearest double (ties to even); NaN if invalid.
__host__ __device__ __forceinline__ double exact_round(const Exact192& a) {
    if (a.bad) return exact_from_bits(0x7ff8000000000000ull);
    unsigned long long w0 = a.w0, w1 = a.w1, w2 = a.w2;
    const bool neg = (w2 >> 63) != 0ull;
    if (neg) {  // magnitude = -a
        w0 = ~w0;
        w1 = ~w1;
        w2 = ~w2;
        w0 += 1ull;
        const unsigned long long c0 = (w0 == 0ull) ? 1ull : 0ull;
        w1 += c0;
        const unsigned long long c1 = (c0 && w1 == 0ull) ? 1ull : 0ull;
        w2 += c1;
    }
    // p = index of the most significant set bit (0 .. 190)
    int p;
    if (w2) p = 128 + 63 - exact_clz64(w2);
    else if (w1) p = 64 + 63 - exact_clz64(w1);
    else if (w0) p = 63 - exact_clz64(w0);
    else return 0.0;
    unsigned long long mant;
    int k;  // value = mant * 2^(k - 128)
    if (p <= 52) {
        mant = w0;
        k = 0;
    } else {
        const int sh = p - 52;  // 1 .. 138: drop sh low bits
        // mant = bits [sh, sh + 52]; round bit = bit sh - 1; sticky = bits below it
        unsigned long long lo;  // bits [sh, sh + 63]
        if (sh < 64) lo = (w0 >> sh) | (w1 << (64 - sh));
        else if (sh == 64) lo = w1;
        else if (sh < 128) lo = (w1 >> (sh - 64)) | (w2 << (128 - sh));
        else if (sh == 128) lo = w2;
        else lo = w2 >> (sh - 128);
        mant = lo & ((1ull << 53) - 1ull);
        const int rb = sh - 1;  // round bit index
        const unsigned long long word = rb < 64 ? w0 : (rb < 128 ? w1 : w2);
        const unsigned long long round = (word >> (rb & 63)) & 1ull;
        bool sticky;
        if (rb < 64) {
            sticky = (w0 & ((1ull << rb) - 1ull)) != 0ull;
        } else if (rb < 128) {
            sticky = w0 != 0ull || (w1 & ((1ull << (rb - 64)) - 1ull)) != 0ull;
        } else {
            sticky = w0 != 0ull || w1 != 0ull || (w2 & ((1ull << (rb - 128)) - 1ull)) != 0ull;
        }
        if (round && (sticky || (mant & 1ull))) mant += 1ull;  // may reach 2^53: still exact
        k = sh;
    }
    // mant <= 2^53 converts exactly; the power of two 2^(k - 128), k in 0 .. 138,
    // is a normal double, so the product is exact
    const double m = static_cast<double>(mant);
    const double scale = exact_from_bits(static_cast<unsigned long long>(1023 + k - 128) << 52);
    const double r = m * scale;
    return neg ? -r : r;
}

// The two parts of a complex sum (Re, Im).
struct ExactPair {
    Exact192 re, im;
};

#ifdef __CUDACC__
// Sum of `a` over the 32 lanes of a warp, valid in lane 0.
__device__ __forceinline__ Exact192 exact_warp_sum(Exact192 a) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Exact192 b;
        b.w0 = __shfl_down_sync(0xffffffffu, a.w0, off);
        b.w1 = __shfl_down_sync(0xffffffffu, a.w1, off);
        b.w2 = __shfl_down_sync(0xffffffffu, a.w2, off);
        b.bad = __shfl_down_sync(0xffffffffu, a.bad, off);
        exact_merge(a, b);
    }
    return a;
}

// Sum of (re, im) over the threads of a block (blockDim.x a multiple of 32,
// at most 1024), valid in thread 0.  Every thread must call it.
__device__ __forceinline__ ExactPair exact_block_sum(Exact192 re, Exact192 im) {
    __shared__ ExactPair s_warp[32];
    re = exact_warp_sum(re);
    im = exact_warp_sum(im);
    const int lane = int(threadIdx.x & 31u), warp = int(threadIdx.x >> 5);
    if (lane == 0) s_warp[warp] = ExactPair{re, im};
    __syncthreads();
    ExactPair t{exact_zero(), exact_zero()};
    if (threadIdx.x == 0) {
        for (int w = 0; w < int(blockDim.x >> 5); ++w) {
            exact_merge(t.re, s_warp[w].re);
            exact_merge(t.im, s_warp[w].im);
        }
    }
    return t;
}
#endif

}  // namespace hd
