// fft_math.cuh -- complex arithmetic and in-register DFT butterflies used by
// the stage kernels.  Dft<R, S, V>::run computes the length-R DFT
// V[s] = sum_r v[r] exp(S 2 pi i r s / R) of R values in registers, outputs in
// natural order; S = -1 is the forward exponent, S = +1 the backward one.
// Radices 8 and 16 are split into radix-2/4 steps with constant twiddles
// (the Cooley-Tukey identity of AccFFT Section 2 applied inside one
// butterfly); radices 3 and 5 use the symmetric sum/difference form.
#pragma once

#include <cuda_runtime.h>

namespace afft {

// ------------------------------------------------------- float-float ------
// FP64 transforms compute in "float-float": a value is hi + lo with two
// floats (about 48 significant bits), because GB300 executes FP32 about 58x
// faster than FP64 (measured: FFMA 73.5, DFMA 1.26 TFLOP/s).  Sums use the
// error-free TwoSum of the hi parts (Knuth), products the FMA-exact residual;
// lo is renormalised (FastTwoSum) once per radix pass.  Values are not kept
// normalised between passes: hi + lo stays exact up to the FP32 rounding of the
// lo accumulation, about 2^-48 relative.
struct dfl {
    float hi, lo;
    __host__ __device__ constexpr dfl() : hi(0.f), lo(0.f) {}
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    // compile-time split of a double constant (no FP64 instruction at run time)
    __host__ __device__ constexpr explicit dfl(double c) : hi((float)c), lo((float)(c - (double)(float)c)) {}
};
__device__ __forceinline__ dfl operator+(dfl a, dfl b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (b.hi - bb);
    return dfl(s, err + (a.lo + b.lo));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dfl(p, e);
}
__device__ __forceinline__ dfl renorm(dfl a)
{
    const float s = a.hi + a.lo;
    return dfl(s, a.lo - (s - a.hi));
}

struct dcx {
    dfl x, y;
};

template <typename V> struct RealOf;
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<dcx> { using T = dfl; };

template <typename V>
__device__ __forceinline__ V cmk(typename RealOf<V>::T x, typename RealOf<V>::T y)
{
    V v;
    v.x = x;
    v.y = y;
    return v;
}
// T(c) of a double constant for any real type (split at compile time for dfl)
template <typename V> __device__ __forceinline__ typename RealOf<V>::T rconst(double c)
{
    return typename RealOf<V>::T(c);
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cconj(V a) { return cmk<V>(a.x, -a.y); }
template <typename V>
__device__ __forceinline__ V cscale(V a, typename RealOf<V>::T s) { return cmk<V>(a.x * s, a.y * s); }
template <typename V> __device__ __forceinline__ V cmul(V a, V w)
{
    return cmk<V>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
// a * conj(w)
template <typename V> __device__ __forceinline__ V cmulc(V a, V w)
{
    return cmk<V>(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
// multiply by a twiddle from the forward table: as is (S = -1) or conjugated (S = +1)
template <int S, typename V> __device__ __forceinline__ V ctw(V a, V w)
{
    return S < 0 ? cmul(a, w) : cmulc(a, w);
}
// a * (S i): a quarter turn in the transform's direction
template <int S, typename V> __device__ __forceinline__ V crot(V a)
{
    return S < 0 ? cmk<V>(a.y, -a.x) : cmk<V>(-a.y, a.x);
}
// a * exp(S i pi/4) = a (1 + S i) / sqrt(2)
template <int S, typename V> __device__ __forceinline__ V cw8(V a)
{
    using T = typename RealOf<V>::T;
    const T h = T(0.70710678118654752440);
    return S < 0 ? cmk<V>((a.x + a.y) * h, (a.y - a.x) * h)
                 : cmk<V>((a.x - a.y) * h, (a.y + a.x) * h);
}
// a * (c + S i s) for a constant unit root
template <int S, typename V>
__device__ __forceinline__ V cwc(V a, typename RealOf<V>::T c, typename RealOf<V>::T s)
{
    return S < 0 ? cmk<V>(a.x * c + a.y * s, a.y * c - a.x * s)
                 : cmk<V>(a.x * c - a.y * s, a.y * c + a.x * s);
}

// ----------------------------------------------------------- butterflies ----
// In-register DFT_R of v[0..R-1], outputs in natural order, exponent sign S.

template <int S, typename V> __device__ __forceinline__ void dft2(V &a, V &b)
{
    const V t = csub(a, b);
    a = cadd(a, b);
    b = t;
}

template <int S, typename V> __device__ __forceinline__ void dft4(V &a0, V &a1, V &a2, V &a3)
{
    const V t0 = cadd(a0, a2), t1 = csub(a0, a2);
    const V t2 = cadd(a1, a3), t3 = crot<S>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <int R, int S, typename V> struct Dft;

template <int S, typename V> struct Dft<2, S, V> {
    static __device__ __forceinline__ void run(V *v) { dft2<S>(v[0], v[1]); }
};

template <int S, typename V> struct Dft<4, S, V> {
    static __device__ __forceinline__ void run(V *v) { dft4<S>(v[0], v[1], v[2], v[3]); }
};

// 8 = 2 x 4: DFT_4 of the even and odd samples, then w_8^s on the odd half.
template <int S, typename V> struct Dft<8, S, V> {
    static __device__ __forceinline__ void run(V *v)
    {
        dft4<S>(v[0], v[2], v[4], v[6]);
        dft4<S>(v[1], v[3], v[5], v[7]);
        const V o1 = cw8<S>(v[3]);
        const V o2 = crot<S>(v[5]);
        const V o3 = crot<S>(cw8<S>(v[7]));
        const V e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
        v[0] = cadd(e0, o0);
        v[4] = csub(e0, o0);
        v[1] = cadd(e1, o1);
        v[5] = csub(e1, o1);
        v[2] = cadd(e2, o2);
        v[6] = csub(e2, o2);
        v[3] = cadd(e3, o3);
        v[7] = csub(e3, o3);
    }
};

// 16 = 4 x 4: A_q = DFT_4 over r1 of v[q + 4 r1]; A_q[s1] *= w_16^{q s1};
// V[s1 + 4 s2] = DFT_4 over q of A_q[s1].
template <int S, typename V> struct Dft<16, S, V> {
    static __device__ __forceinline__ void run(V *v)
    {
        using T = typename RealOf<V>::T;
        const T c = T(0.92387953251128675613), s = T(0.38268343236508977173);
#pragma unroll
        for (int q = 0; q < 4; ++q) dft4<S>(v[q], v[q + 4], v[q + 8], v[q + 12]);
        // A_q[s1] sits in v[q + 4 s1]
        v[5] = cwc<S>(v[5], c, s);             // q=1,s1=1: w16^1
        v[9] = cw8<S>(v[9]);                   // q=1,s1=2: w16^2
        v[13] = cwc<S>(v[13], s, c);           // q=1,s1=3: w16^3
        v[6] = cw8<S>(v[6]);                   // q=2,s1=1: w16^2
        v[10] = crot<S>(v[10]);                // q=2,s1=2: w16^4
        v[14] = crot<S>(cw8<S>(v[14]));        // q=2,s1=3: w16^6
        v[7] = cwc<S>(v[7], s, c);             // q=3,s1=1: w16^3
        v[11] = crot<S>(cw8<S>(v[11]));        // q=3,s1=2: w16^6
        {
            const V t = cwc<S>(v[15], c, s);   // q=3,s1=3: w16^9 = -w16^1
            v[15] = cmk<V>(-t.x, -t.y);
        }
        V o[16];
#pragma unroll
        for (int s1 = 0; s1 < 4; ++s1) {
            V a0 = v[4 * s1], a1 = v[4 * s1 + 1], a2 = v[4 * s1 + 2], a3 = v[4 * s1 + 3];
            dft4<S>(a0, a1, a2, a3);
            o[s1] = a0;
            o[s1 + 4] = a1;
            o[s1 + 8] = a2;
            o[s1 + 12] = a3;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = o[i];
    }
};

template <int S, typename V> struct Dft<3, S, V> {
    static __device__ __forceinline__ void run(V *v)
    {
        using T = typename RealOf<V>::T;
        const T h = T(0.86602540378443864676);   // sin(2 pi / 3)
        const V a = cadd(v[1], v[2]);
        const V b = csub(v[1], v[2]);
        const V m = cmk<V>(v[0].x - T(0.5) * a.x, v[0].y - T(0.5) * a.y);
        const V r = crot<S>(cscale(b, h));      // S i sin(2pi/3) (v1 - v2)
        v[0] = cadd(v[0], a);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};

template <int S, typename V> struct Dft<5, S, V> {
    static __device__ __forceinline__ void run(V *v)
    {
        using T = typename RealOf<V>::T;
        const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);
        const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);
        const V a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        const V a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        const V m1 = cmk<V>(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
        const V m2 = cmk<V>(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
        const V r1 = crot<S>(cmk<V>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
        const V r2 = crot<S>(cmk<V>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
        v[0] = cadd(v[0], cadd(a1, a2));
        v[1] = cadd(m1, r1);
        v[4] = csub(m1, r1);
        v[2] = cadd(m2, r2);
        v[3] = csub(m2, r2);
    }
};


// ------------------------------------------- float-float conversions -----

// Split of a double into float-float using integer operations only (no FP64
// instruction): hi takes the top 24 significand bits, lo the remaining 29 bits
// rounded to 24 (exact to 2^-48 relative).  Flags for the tile-wide decision:
// `large` for |x| >= 2^101, inf or nan (an FFT stage grows values by up to n <=
// 2^12, which must stay below float's 2^128); `normal` for |x| >= 2^-50.
// Values below 2^-74 keep only hi (below 2^-126: zero); that is negligible when
// the tile holds some value >= 2^-50, which the caller checks.
struct DfFlags {
    bool large = false;
    bool normal = false;
};
__device__ __forceinline__ dfl dfl_from_double(double x, DfFlags &f)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned e = (unsigned)(u >> 52) & 0x7ffu;
    const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    const unsigned sgn = (unsigned)(u >> 63);
    if (e >= 1124u) {  // |x| >= 2^101, inf, nan
        f.large = true;
        return dfl(0.f, 0.f);
    }
    if (e >= 973u) f.normal = true;
    if (e < 897u) return dfl(0.f, 0.f);   // below float's normal range
    const float hi = __uint_as_float((sgn << 31) | ((e - 896u) << 23) | (unsigned)(m >> 29));
    if (e < 949u) return dfl(hi, 0.f);
    const int r = (int)(m & 0x1FFFFFFFull);
    const float lo = (float)(sgn ? -r : r) * __uint_as_float((e - 948u) << 23);
    return dfl(hi, lo);
}

// Exact float -> double by bit placement (normal floats; zero and subnormals
// give zero), then one FP64 add for hi + lo.
__device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) |
                                 ((unsigned long long)(b & 0x7fffffu) << 29);
    return e == 0 ? 0.0 : __longlong_as_double((long long)d);
}
__device__ __forceinline__ double dfl_to_double(dfl a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

// Renormalises the float-float parts of a complex value (identity otherwise).
template <typename V> __device__ __forceinline__ V cnorm(V v) { return v; }
template <> __device__ __forceinline__ dcx cnorm<dcx>(dcx v)
{
    dcx r;
    r.x = renorm(v.x);
    r.y = renorm(v.y);
    return r;
}

// Read-only cached load of one complex value.
template <typename V> __device__ __forceinline__ V ldgc(const V *p) { return __ldg(p); }
template <> __device__ __forceinline__ dcx ldgc<dcx>(const dcx *p)
{
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    dcx r;
    r.x = dfl(q.x, q.y);
    r.y = dfl(q.z, q.w);
    return r;
}

// A twiddle factor: from a table in shared memory (a CTA's staged copy) or,
// through the read-only cache, from the plan's table in global memory.
template <bool Smem, typename V> __device__ __forceinline__ V tw_ld(const V *p)
{
    if constexpr (Smem) return *p;
    else return ldgc(p);
}

// Storage <-> compute conversions (identity unless double2 <-> dcx).
template <typename CT, typename V> struct Conv {
    static __device__ __forceinline__ CT in(V v, DfFlags *) { return v; }
    static __device__ __forceinline__ V out(CT v) { return v; }
};
template <> struct Conv<dcx, double2> {
    static __device__ __forceinline__ dcx in(double2 v, DfFlags *f)
    {
        dcx r;
        r.x = dfl_from_double(v.x, *f);
        r.y = dfl_from_double(v.y, *f);
        return r;
    }
    static __device__ __forceinline__ double2 out(dcx v)
    {
        return make_double2(dfl_to_double(v.x), dfl_to_double(v.y));
    }
};

}  // namespace afft
