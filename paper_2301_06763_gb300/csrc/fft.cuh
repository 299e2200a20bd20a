// fft.cuh -- in-CTA Stockham FFT of one line of length P (power of two, 8..1024).
//
// The convolution theorem (Sect. 3, Eq. 11) is applied with discrete Fourier
// transforms on the doubled domain.  Each line is transformed by P/E threads,
// each holding E complex values in registers (E = 16 for P >= 16, else 8).
// The first pass is radix E on the values the thread loaded itself (no
// twiddles); the remaining passes are radix E while the remaining factor
// allows, then one radix-2/4/8 pass, exchanging through shared memory between
// passes (self-sorting Stockham order, so no bit reversal).  P = 32..256 thus
// needs one shared-memory round trip per transform.
//
// Register conventions (j = the thread's index within its line, 0 <= j < P/E):
//   input : v[r] = x[j + r * P/E],                         r = 0..E-1
//   output: v[b * R + r] = X[(j + b * P/E) + r * (P/R)],   b < E/R, r < R
// where R is the radix of the last pass.  `seam_permute` maps an output
// distribution onto the input distribution of a second transform held by the
// same thread, so a forward transform, a pointwise multiply and an inverse
// transform chain in registers.
//
// Forward: X[k] = sum_j x[j] exp(-2 pi i jk/P); inverse: the + sign, no 1/P.
// Twiddles come from a table tw[t] = exp(-2 pi i t / P) built on the host in
// double precision (std::cos / std::sin) and staged in shared memory, as is
// or in the per-pass order of fill_pass_twiddles.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"

namespace nm {

template <typename T> struct alignas(2 * sizeof(T)) cpx { T re, im; };

template <typename T> __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) {
    return {a.re + b.re, a.im + b.im};
}
template <typename T> __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) {
    return {a.re - b.re, a.im - b.im};
}
// Blackwell issues two FP32 additions as one instruction on a register pair
// (FADD2): a complex sum or difference of floats is exactly that, with the
// same rounding as the two scalar additions.  The transforms' butterflies are
// mostly such sums, and the float passes are bound by instruction issue.
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
__device__ __forceinline__ cpx<float> operator+(cpx<float> a, cpx<float> b) {
    const float2 r = __fadd2_rn(make_float2(a.re, a.im), make_float2(b.re, b.im));
    return {r.x, r.y};
}
__device__ __forceinline__ cpx<float> operator-(cpx<float> a, cpx<float> b) {
    const float2 r = __fadd2_rn(make_float2(a.re, a.im), make_float2(-b.re, -b.im));
    return {r.x, r.y};
}
// The same pairing for double-float complex values: the real and imaginary
// parts go through the identical sequence of the double-float sum, so each of
// its steps is one FADD2 on (re, im) pairs of high and of low words.
__device__ __forceinline__ cpx<df> df_cadd(float2 ah, float2 al, float2 bh, float2 bl) {
    const float2 s = __fadd2_rn(ah, bh);
    const float2 bb = __fadd2_rn(s, make_float2(-ah.x, -ah.y));
    const float2 t = __fadd2_rn(s, make_float2(-bb.x, -bb.y));
    float2 e = __fadd2_rn(__fadd2_rn(ah, make_float2(-t.x, -t.y)), __fadd2_rn(bh, make_float2(-bb.x, -bb.y)));
    e = __fadd2_rn(e, __fadd2_rn(al, bl));
    const float2 r = __fadd2_rn(s, e);
    const float2 u = __fadd2_rn(r, make_float2(-s.x, -s.y));
    const float2 lo = __fadd2_rn(e, make_float2(-u.x, -u.y));
    return {df(r.x, lo.x), df(r.y, lo.y)};
}
__device__ __forceinline__ cpx<df> operator+(cpx<df> a, cpx<df> b) {
    return df_cadd(make_float2(a.re.hi, a.im.hi), make_float2(a.re.lo, a.im.lo), make_float2(b.re.hi, b.im.hi),
                   make_float2(b.re.lo, b.im.lo));
}
__device__ __forceinline__ cpx<df> operator-(cpx<df> a, cpx<df> b) {
    return df_cadd(make_float2(a.re.hi, a.im.hi), make_float2(a.re.lo, a.im.lo), make_float2(-b.re.hi, -b.im.hi),
                   make_float2(-b.re.lo, -b.im.lo));
}
#endif

// Two float lanes operated on together: the real parts of two complex values
// of two different lines form one f2, their imaginary parts another, so a
// complex value of type cpx<f2> carries the same element of two lines and
// every step of the transform (sums, twiddle products, scaling) acts on both
// lines with one paired instruction.  With the twiddles broadcast to both
// lanes, a complex product costs 4 paired instructions (2 FMUL2, 2 FFMA2) for
// the two lines, where cpx<float> needs 4 scalar ones for each line.
struct alignas(8) f2 {
    float x, y;
    f2() = default;
    __host__ __device__ constexpr f2(float a, float b) : x(a), y(b) {}
    __host__ __device__ explicit constexpr f2(double a) : x((float)a), y((float)a) {}
    __host__ __device__ explicit constexpr f2(int a) : x((float)a), y((float)a) {}
};
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
__device__ __forceinline__ float2 as_f2(f2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ f2 of_f2(float2 a) { return {a.x, a.y}; }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return of_f2(__fadd2_rn(as_f2(a), as_f2(b))); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return of_f2(__fadd2_rn(as_f2(a), make_float2(-b.x, -b.y))); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return of_f2(__fmul2_rn(as_f2(a), as_f2(b))); }
// a * b + c, one rounding per lane
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return of_f2(__ffma2_rn(as_f2(a), as_f2(b), as_f2(c))); }
#else
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return {a.x * b.x, a.y * b.y}; }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return {fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y)}; }
#endif
__device__ __forceinline__ f2 operator-(f2 a) { return {-a.x, -a.y}; }
__device__ __forceinline__ f2& operator*=(f2& a, f2 b) { return a = a * b; }

template <typename T> __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ cpx<f2> cmul(cpx<f2> a, cpx<f2> b) {
    return {fma2(-a.im, b.im, a.re * b.re), fma2(a.re, b.im, a.im * b.re)};
}
// a * conj(b)
template <typename T> __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
    return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV> __device__ __forceinline__ cpx<T> rot4(cpx<T> a) {
    if (INV) return {-a.im, a.re};
    return {a.im, -a.re};
}
// multiply by exp(-+ i pi/4)
template <typename T, bool INV> __device__ __forceinline__ cpx<T> rot8(cpx<T> a) {
    const T h = (T)0.70710678118654752440;
    if (INV) return {(a.re - a.im) * h, (a.re + a.im) * h};
    return {(a.re + a.im) * h, (a.im - a.re) * h};
}
// multiply by exp(-+ 3 i pi/4)
template <typename T, bool INV> __device__ __forceinline__ cpx<T> rot8_3(cpx<T> a) {
    const T h = (T)0.70710678118654752440;
    if (INV) return {-(a.re + a.im) * h, (a.re - a.im) * h};
    return {(a.im - a.re) * h, -(a.re + a.im) * h};
}

template <typename T, bool INV> __device__ __forceinline__ void dft2(cpx<T>* v) {
    cpx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
}

template <typename T, bool INV> __device__ __forceinline__ void dft4(cpx<T>* v) {
    cpx<T> p0 = v[0] + v[2], q0 = v[0] - v[2];
    cpx<T> p1 = v[1] + v[3], q1 = rot4<T, INV>(v[1] - v[3]);
    v[0] = p0 + p1;
    v[2] = p0 - p1;
    v[1] = q0 + q1;
    v[3] = q0 - q1;
}

// 8-point DFT: u[n] = v[n] + v[n+4], w[n] = (v[n] - v[n+4]) W8^n, then
// X[2k] = DFT4(u)[k], X[2k+1] = DFT4(w)[k].
template <typename T, bool INV> __device__ __forceinline__ void dft8(cpx<T>* v) {
    cpx<T> u[4], w[4];
    u[0] = v[0] + v[4]; w[0] = v[0] - v[4];
    u[1] = v[1] + v[5]; w[1] = rot8<T, INV>(v[1] - v[5]);
    u[2] = v[2] + v[6]; w[2] = rot4<T, INV>(v[2] - v[6]);
    u[3] = v[3] + v[7]; w[3] = rot8_3<T, INV>(v[3] - v[7]);
    dft4<T, INV>(u);
    dft4<T, INV>(w);
    v[0] = u[0]; v[2] = u[1]; v[4] = u[2]; v[6] = u[3];
    v[1] = w[0]; v[3] = w[1]; v[5] = w[2]; v[7] = w[3];
}

// multiply by cos(a) -+ i sin(a) (forward / inverse)
template <typename T, bool INV> __device__ __forceinline__ cpx<T> rotc(cpx<T> a, T c, T s) {
    if (INV) return {a.re * c - a.im * s, a.re * s + a.im * c};
    return {a.re * c + a.im * s, a.im * c - a.re * s};
}
template <> __device__ __forceinline__ cpx<f2> rotc<f2, false>(cpx<f2> a, f2 c, f2 s) {
    return {fma2(a.im, s, a.re * c), fma2(-a.re, s, a.im * c)};
}
template <> __device__ __forceinline__ cpx<f2> rotc<f2, true>(cpx<f2> a, f2 c, f2 s) {
    return {fma2(-a.im, s, a.re * c), fma2(a.re, s, a.im * c)};
}

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
// Double-float complex products, paired as above: two double-float products
// per instruction sequence (FMUL2 / FFMA2 on pairs of high and low words).
struct df2 { float2 h, l; };
__device__ __forceinline__ df2 df2_of(df a, df b) { return {make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}; }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ df2 df2_mul(df2 x, df2 y) {
    const float2 p = __fmul2_rn(x.h, y.h);
    float2 e = __ffma2_rn(x.h, y.h, neg2(p));
    e = __ffma2_rn(x.h, y.l, e);
    e = __ffma2_rn(x.l, y.h, e);
    const float2 r = __fadd2_rn(p, e);
    return {r, __fadd2_rn(e, neg2(__fadd2_rn(r, neg2(p))))};
}
__device__ __forceinline__ cpx<df> df2_sum(df2 x, df2 y) { return df_cadd(x.h, x.l, y.h, y.l); }
__device__ __forceinline__ df2 df2_of(cpx<df> c) { return df2_of(c.re, c.im); }
__device__ __forceinline__ df2 df2_add(df2 x, df2 y) { return df2_of(df_cadd(x.h, x.l, y.h, y.l)); }

__device__ __forceinline__ cpx<df> cmul(cpx<df> a, cpx<df> b) {
    // (ar, ar) (br, bi) + (ai, ai) (-bi, br)
    return df2_sum(df2_mul(df2_of(a.re, a.re), df2_of(b.re, b.im)), df2_mul(df2_of(a.im, a.im), df2_of(-b.im, b.re)));
}
__device__ __forceinline__ cpx<df> cmulc(cpx<df> a, cpx<df> b) {
    // (ar, ar) (br, -bi) + (ai, ai) (bi, br)
    return df2_sum(df2_mul(df2_of(a.re, a.re), df2_of(b.re, -b.im)), df2_mul(df2_of(a.im, a.im), df2_of(b.im, b.re)));
}
template <> __device__ __forceinline__ cpx<df> rotc<df, false>(cpx<df> a, df c, df s) {
    return df2_sum(df2_mul(df2_of(a.re, a.im), df2_of(c, c)), df2_mul(df2_of(a.im, a.re), df2_of(s, -s)));
}
template <> __device__ __forceinline__ cpx<df> rotc<df, true>(cpx<df> a, df c, df s) {
    return df2_sum(df2_mul(df2_of(a.re, a.im), df2_of(c, c)), df2_mul(df2_of(a.im, a.re), df2_of(-s, s)));
}
template <> __device__ __forceinline__ cpx<df> rot8<df, false>(cpx<df> a) {
    const df h = df(0.70710678118654752440);
    const cpx<df> t = df2_sum(df2_of(a.re, a.im), df2_of(a.im, -a.re));
    const df2 r = df2_mul(df2_of(t), df2_of(h, h));
    return {df(r.h.x, r.l.x), df(r.h.y, r.l.y)};
}
template <> __device__ __forceinline__ cpx<df> rot8<df, true>(cpx<df> a) {
    const df h = df(0.70710678118654752440);
    const cpx<df> t = df2_sum(df2_of(a.re, a.re), df2_of(-a.im, a.im));
    const df2 r = df2_mul(df2_of(t), df2_of(h, h));
    return {df(r.h.x, r.l.x), df(r.h.y, r.l.y)};
}
template <> __device__ __forceinline__ cpx<df> rot8_3<df, false>(cpx<df> a) {
    const df h = df(0.70710678118654752440);
    const cpx<df> t = df2_sum(df2_of(-a.re, -a.re), df2_of(a.im, -a.im));
    const df2 r = df2_mul(df2_of(t), df2_of(h, h));
    return {df(r.h.x, r.l.x), df(r.h.y, r.l.y)};
}
template <> __device__ __forceinline__ cpx<df> rot8_3<df, true>(cpx<df> a) {
    const df h = df(0.70710678118654752440);
    const cpx<df> t = df2_sum(df2_of(-a.re, a.re), df2_of(-a.im, -a.im));
    const df2 r = df2_mul(df2_of(t), df2_of(h, h));
    return {df(r.h.x, r.l.x), df(r.h.y, r.l.y)};
}
#endif

// 16-point DFT as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.  DFT4 over n1 for each
// n2, multiply by W16^(n2 k1), DFT4 over n2 for each k1.
template <typename T, bool INV> __device__ __forceinline__ void dft16(cpx<T>* v) {
    const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;
    cpx<T> y[16];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        cpx<T> t[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
        dft4<T, INV>(t);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) y[n2 * 4 + k1] = t[k1];
    }
    y[5] = rotc<T, INV>(y[5], c1, s1);      // W16^1
    y[6] = rot8<T, INV>(y[6]);              // W16^2
    y[7] = rotc<T, INV>(y[7], s1, c1);      // W16^3
    y[9] = rot8<T, INV>(y[9]);              // W16^2
    y[10] = rot4<T, INV>(y[10]);            // W16^4
    y[11] = rot8_3<T, INV>(y[11]);          // W16^6
    y[13] = rotc<T, INV>(y[13], s1, c1);    // W16^3
    y[14] = rot8_3<T, INV>(y[14]);          // W16^6
    y[15] = rotc<T, INV>(y[15], -c1, -s1);  // W16^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        cpx<T> t[4] = {y[k1], y[4 + k1], y[8 + k1], y[12 + k1]};
        dft4<T, INV>(t);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
    }
}

template <typename T, bool INV, int R> __device__ __forceinline__ void dftR(cpx<T>* v) {
    if constexpr (R == 16) dft16<T, INV>(v);
    else if constexpr (R == 8) dft8<T, INV>(v);
    else if constexpr (R == 4) dft4<T, INV>(v);
    else dft2<T, INV>(v);
}

// ------------------------------------------------ first pass on padded lines
// A forward transform of a zero-padded line (Fig. 4: half of every line, more
// on the doubled and quadrupled grids) starts from registers that are zero by
// construction.  IEEE addition of a zero is not an identity (-0 + 0 = +0), so
// the compiler keeps those additions; the masked forms below drop them.  Bit r
// of the mask M says that input register r may be nonzero; every result is the
// same value the full butterfly gives, up to the sign of a zero.
template <bool LA, bool LB, typename T> __device__ __forceinline__ cpx<T> zadd(cpx<T> a, cpx<T> b) {
    if constexpr (LA && LB) return a + b;
    else if constexpr (LA) return a;
    else if constexpr (LB) return b;
    else return {T(0), T(0)};
}
template <bool LA, bool LB, typename T> __device__ __forceinline__ cpx<T> zsub(cpx<T> a, cpx<T> b) {
    if constexpr (LA && LB) return a - b;
    else if constexpr (LA) return a;
    else if constexpr (LB) return {-b.re, -b.im};
    else return {T(0), T(0)};
}

template <typename T, bool INV, unsigned M> __device__ __forceinline__ void dft4m(cpx<T>* v) {
    constexpr bool a0 = M & 1u, a1 = M & 2u, a2 = M & 4u, a3 = M & 8u;
    constexpr bool lp = a0 || a2, lq = a1 || a3;
    const cpx<T> p0 = zadd<a0, a2>(v[0], v[2]), q0 = zsub<a0, a2>(v[0], v[2]);
    const cpx<T> p1 = zadd<a1, a3>(v[1], v[3]);
    cpx<T> q1 = zsub<a1, a3>(v[1], v[3]);
    if constexpr (lq) q1 = rot4<T, INV>(q1);
    v[0] = zadd<lp, lq>(p0, p1);
    v[2] = zsub<lp, lq>(p0, p1);
    v[1] = zadd<lp, lq>(q0, q1);
    v[3] = zsub<lp, lq>(q0, q1);
}

// the 4 inputs v[n2], v[4+n2], v[8+n2], v[12+n2] of the first-stage DFT4 n2
template <unsigned M, int N2> struct Grp16 {
    static constexpr unsigned value = ((M >> N2) & 1u) | (((M >> (4 + N2)) & 1u) << 1) |
                                      (((M >> (8 + N2)) & 1u) << 2) | (((M >> (12 + N2)) & 1u) << 3);
};

template <typename T, bool INV, unsigned M, int N2>
__device__ __forceinline__ void dft16m_stage1(const cpx<T>* v, cpx<T>* y) {
    cpx<T> t[4] = {v[N2], v[4 + N2], v[8 + N2], v[12 + N2]};
    dft4m<T, INV, Grp16<M, N2>::value>(t);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) y[N2 * 4 + k1] = t[k1];
}

template <typename T, bool INV, unsigned M> __device__ __forceinline__ void dft16m(cpx<T>* v) {
    if constexpr ((M & 0xFFFFu) == 0xFFFFu) {
        dft16<T, INV>(v);
    } else {
        const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;
        constexpr bool g0 = Grp16<M, 0>::value != 0, g1 = Grp16<M, 1>::value != 0,
                       g2 = Grp16<M, 2>::value != 0, g3 = Grp16<M, 3>::value != 0;
        constexpr unsigned GL = (g0 ? 1u : 0u) | (g1 ? 2u : 0u) | (g2 ? 4u : 0u) | (g3 ? 8u : 0u);
        cpx<T> y[16];
        dft16m_stage1<T, INV, M, 0>(v, y);
        dft16m_stage1<T, INV, M, 1>(v, y);
        dft16m_stage1<T, INV, M, 2>(v, y);
        dft16m_stage1<T, INV, M, 3>(v, y);
        if constexpr (g1) {
            y[5] = rotc<T, INV>(y[5], c1, s1);
            y[6] = rot8<T, INV>(y[6]);
            y[7] = rotc<T, INV>(y[7], s1, c1);
        }
        if constexpr (g2) {
            y[9] = rot8<T, INV>(y[9]);
            y[10] = rot4<T, INV>(y[10]);
            y[11] = rot8_3<T, INV>(y[11]);
        }
        if constexpr (g3) {
            y[13] = rotc<T, INV>(y[13], s1, c1);
            y[14] = rot8_3<T, INV>(y[14]);
            y[15] = rotc<T, INV>(y[15], -c1, -s1);
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            cpx<T> t[4] = {y[k1], y[4 + k1], y[8 + k1], y[12 + k1]};
            dft4m<T, INV, GL>(t);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
        }
    }
}

template <typename T, bool INV, unsigned M> __device__ __forceinline__ void dft8m(cpx<T>* v) {
    if constexpr ((M & 0xFFu) == 0xFFu) {
        dft8<T, INV>(v);
    } else {
        constexpr bool b0 = M & 1u, b1 = M & 2u, b2 = M & 4u, b3 = M & 8u;
        constexpr bool b4 = M & 16u, b5 = M & 32u, b6 = M & 64u, b7 = M & 128u;
        constexpr unsigned UL = ((b0 || b4) ? 1u : 0u) | ((b1 || b5) ? 2u : 0u) | ((b2 || b6) ? 4u : 0u) |
                                ((b3 || b7) ? 8u : 0u);
        cpx<T> u[4], w[4];
        u[0] = zadd<b0, b4>(v[0], v[4]); w[0] = zsub<b0, b4>(v[0], v[4]);
        u[1] = zadd<b1, b5>(v[1], v[5]); w[1] = zsub<b1, b5>(v[1], v[5]);
        u[2] = zadd<b2, b6>(v[2], v[6]); w[2] = zsub<b2, b6>(v[2], v[6]);
        u[3] = zadd<b3, b7>(v[3], v[7]); w[3] = zsub<b3, b7>(v[3], v[7]);
        if constexpr (b1 || b5) w[1] = rot8<T, INV>(w[1]);
        if constexpr (b2 || b6) w[2] = rot4<T, INV>(w[2]);
        if constexpr (b3 || b7) w[3] = rot8_3<T, INV>(w[3]);
        dft4m<T, INV, UL>(u);
        dft4m<T, INV, UL>(w);
        v[0] = u[0]; v[2] = u[1]; v[4] = u[2]; v[6] = u[3];
        v[1] = w[0]; v[3] = w[1]; v[5] = w[2]; v[7] = w[3];
    }
}

// First pass of radix R = E with input mask M.
template <typename T, bool INV, int R, unsigned M> __device__ __forceinline__ void dftRm(cpx<T>* v) {
    if constexpr (R == 16) dft16m<T, INV, M>(v);
    else if constexpr (R == 8) dft8m<T, INV, M>(v);
    else dftR<T, INV, R>(v);
}

// Default values per thread for a line of length P.
template <int P> struct EOf {
    static constexpr int value = P >= 16 ? 16 : 8;
};
template <int E> struct Log2E {
    static constexpr int value = E == 16 ? 4 : 3;
};

// Radix of the pass that starts at stride NS, and of the last pass.
template <int P, int E, int NS> struct PassRadix {
    static constexpr int REM = P / NS;
    static constexpr int R = REM >= E ? E : REM;
};
template <int P, int E> struct LastRadix {
    static constexpr int calc() {
        int ns = E, R = E;
        while (ns < P) {
            R = (P / ns >= E) ? E : P / ns;
            ns *= R;
        }
        return R;
    }
    static constexpr int value = calc();
};

// Shared-memory view of the lines a CTA transforms.  Element e of the
// calling thread's line lives at base[e * ES] (+ one padding slot every E
// elements for contiguous lines, which keeps the first-pass stores of a warp
// free of bank conflicts).
template <typename T, int ES, bool PAD, int LOGE = 4> struct LineView {
    cpx<T>* base;
    __device__ __forceinline__ int off(int e) const {
        return PAD ? (e + (e >> LOGE)) * ES : e * ES;
    }
    __device__ __forceinline__ cpx<T> ld(int e) const { return base[off(e)]; }
    __device__ __forceinline__ void st(int e, cpx<T> v) const { base[off(e)] = v; }
    // the first pass's stores: elements E j + r, r < E
    template <int E> __device__ __forceinline__ void st_first(int j, const cpx<T>* v) const {
#pragma unroll
        for (int r = 0; r < E; ++r) st(E * j + r, v[r]);
    }
};

template <typename T, bool INV>
__device__ __forceinline__ cpx<T> twiddle(const cpx<T>* tw, int t) {
    cpx<T> w = tw[t];
    if (INV) w.im = -w.im;
    return w;
}

// Twiddle table of the passes after the first, pass by pass: the pass that
// starts at stride NS (radix R) multiplies value r of butterfly k by
// w^(k r P/(NS R)), w = exp(-2 pi i/P), kept at [NS - E + (r - 1) NS + k]
// (r = 1..R-1, k < NS; P - E entries in all).  The threads of one line read
// consecutive k there, which fall in distinct shared-memory banks; in the
// plain table w^t an even r puts the k of a row kernel's warp (16 threads
// of one line) on a few banks.  `w(t)` returns w^t in the table's type.
template <int P, int E, int NS = E, class C, class F>
__device__ __forceinline__ void fill_pass_twiddles(C* out, const F& w) {
    if constexpr (NS < P) {
        constexpr int R = PassRadix<P, E, NS>::R;
        for (int i = threadIdx.x; i < (R - 1) * NS; i += blockDim.x) {
            const int r = i / NS + 1, k = i % NS;
            out[NS - E + i] = w(k * r * (P / (NS * R)));
        }
        fill_pass_twiddles<P, E, NS * R>(out, w);
    }
}

// Passes after the first.  NS = product of the radices done so far.  TAIL:
// the caller writes the shared-memory line again after the transform, so the
// last pass's reads must be complete in every thread before it returns.
template <typename T, int P, int E, bool INV, int NS, bool TAIL, bool PT, class View>
__device__ __forceinline__ void fft_rest(cpx<T>* v, int j, const cpx<T>* tw, const View& sm) {
    constexpr int R = PassRadix<P, E, NS>::R;
    constexpr int NB = E / R;
    constexpr bool LAST = (NS * R == P);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int jj = j + b * (P / E);
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = sm.ld(jj + r * (P / R));
    }
    if constexpr (!LAST || TAIL) __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int jj = j + b * (P / E);
        const int k = jj & (NS - 1);
#pragma unroll
        for (int r = 1; r < R; ++r)
            v[b * R + r] = cmul(v[b * R + r], twiddle<T, INV>(tw, PT ? NS - E + (r - 1) * NS + k
                                                                      : k * r * (P / (NS * R))));
        dftR<T, INV, R>(&v[b * R]);
    }
    if constexpr (!LAST) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int jj = j + b * (P / E);
            const int k = jj & (NS - 1);
            const int base = (jj / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) sm.st(base + r * NS, v[b * R + r]);
        }
        __syncthreads();
        fft_rest<T, P, E, INV, NS * R, TAIL, PT>(v, j, tw, sm);
    }
}

// Whole-line transform.  All threads of the CTA must call it (it contains
// __syncthreads); the shared-memory line must not be in use by anyone else.
// M: bit r set when input register r may be nonzero (all set by default).
// TAIL = false when nobody writes the shared-memory line before the next
// barrier of the caller (the last transform of a kernel, or one followed by
// the caller's own barrier): the final barrier is then left out.  PT: the
// twiddles are in the per-pass order of fill_pass_twiddles (else the plain
// table tw[t] = w^t); each kernel takes the order measured faster for it.
template <typename T, int P, int E, bool INV, unsigned M = 0xFFFFu, bool TAIL = true, bool PT = false, class View>
__device__ __forceinline__ void fft_line(cpx<T>* v, int j, const cpx<T>* tw, const View& sm) {
    static_assert(P >= E, "line shorter than the values a thread holds");
    dftRm<T, INV, E, M>(v);
    if constexpr (P > E) {
        sm.template st_first<E>(j, v);
        __syncthreads();
        fft_rest<T, P, E, INV, E, TAIL, PT>(v, j, tw, sm);
    }
}

// Output index of register slot s after fft_line (see the header comment).
template <int P, int E> __device__ __forceinline__ int out_index(int j, int s) {
    constexpr int R = LastRadix<P, E>::value;
    return j + (s / R) * (P / E) + (s % R) * (P / R);
}

// Output distribution -> input distribution, same thread:
// in[b + r * (E/R)] = out[b * R + r].
template <typename T, int P, int E> __device__ __forceinline__ void seam_permute(cpx<T>* v) {
    constexpr int R = LastRadix<P, E>::value;
    constexpr int NB = E / R;
    cpx<T> t[E];
#pragma unroll
    for (int s = 0; s < E; ++s) t[s] = v[s];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) v[b + r * NB] = t[b * R + r];
}

}  // namespace nm
