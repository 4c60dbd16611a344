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

template <typename V> struct RealOf;
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<double2> { using T = double; };

template <typename V>
__device__ __forceinline__ V cmk(typename RealOf<V>::T x, typename RealOf<V>::T y)
{
    V v;
    v.x = x;
    v.y = y;
    return v;
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


}  // namespace afft
