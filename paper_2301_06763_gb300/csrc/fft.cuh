// fft.cuh -- in-CTA Stockham FFT of one line of length P (power of two, 8..1024).
//
// The convolution theorem (Sect. 3, Eq. 11) is applied with discrete Fourier
// transforms on the doubled domain.  Each line is transformed by P/8 threads,
// each holding 8 complex values in registers.  The first pass is radix 8 on
// the values the thread loaded itself (no twiddles); the remaining passes are
// radix 8 while the remaining factor allows, then one radix-4 or radix-2 pass,
// exchanging through shared memory between passes (self-sorting Stockham
// order, so no bit reversal).
//
// Register conventions (j = the thread's index within its line, 0 <= j < P/8):
//   input : v[r] = x[j + r * P/8],                         r = 0..7
//   output: v[b * R + r] = X[(j + b * P/8) + r * (P/R)],   b < 8/R, r < R
// where R is the radix of the last pass.  `seam_permute` maps an output
// distribution onto the input distribution of a second transform held by the
// same thread, so a forward transform, a pointwise multiply and an inverse
// transform chain in registers.
//
// Forward: X[k] = sum_j x[j] exp(-2 pi i jk/P); inverse: the + sign, no 1/P.
// Twiddles come from a table tw[t] = exp(-2 pi i t / P) built on the host in
// double precision (std::cos / std::sin) and staged in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nm {

template <typename T> struct alignas(2 * sizeof(T)) cpx { T re, im; };

template <typename T> __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) {
    return {a.re + b.re, a.im + b.im};
}
template <typename T> __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) {
    return {a.re - b.re, a.im - b.im};
}
template <typename T> __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
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

template <typename T, bool INV, int R> __device__ __forceinline__ void dftR(cpx<T>* v) {
    if (R == 8) dft8<T, INV>(v);
    else if (R == 4) dft4<T, INV>(v);
    else dft2<T, INV>(v);
}

// Radix of the pass that starts at stride NS, and of the last pass.
template <int P, int NS> struct PassRadix {
    static constexpr int REM = P / NS;
    static constexpr int R = REM >= 8 ? 8 : REM;
};
template <int P> struct LastRadix {
    static constexpr int value = (P == 8 || P == 64 || P == 512) ? 8
                               : (P == 32 || P == 256) ? 4 : 2;
};

// Shared-memory view of the lines a CTA transforms.  Element e of the
// calling thread's line lives at base[e * ES] (+ padding for contiguous lines).
template <typename T, int ES, bool PAD> struct LineView {
    cpx<T>* base;
    __device__ __forceinline__ int off(int e) const {
        return PAD ? (e + (e >> 3)) * ES : e * ES;
    }
    __device__ __forceinline__ cpx<T> ld(int e) const { return base[off(e)]; }
    __device__ __forceinline__ void st(int e, cpx<T> v) const { base[off(e)] = v; }
};

template <typename T, bool INV>
__device__ __forceinline__ cpx<T> twiddle(const cpx<T>* tw, int t) {
    cpx<T> w = tw[t];
    if (INV) w.im = -w.im;
    return w;
}

// Passes after the first.  NS = product of the radices done so far.
template <typename T, int P, bool INV, int NS, class View>
__device__ __forceinline__ void fft_rest(cpx<T>* v, int j, const cpx<T>* tw, const View& sm) {
    constexpr int R = PassRadix<P, NS>::R;
    constexpr int NB = 8 / R;
    constexpr bool LAST = (NS * R == P);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int jj = j + b * (P / 8);
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = sm.ld(jj + r * (P / R));
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int jj = j + b * (P / 8);
        const int k = jj & (NS - 1);
#pragma unroll
        for (int r = 1; r < R; ++r)
            v[b * R + r] = cmul(v[b * R + r], twiddle<T, INV>(tw, k * r * (P / (NS * R))));
        dftR<T, INV, R>(&v[b * R]);
    }
    if constexpr (!LAST) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int jj = j + b * (P / 8);
            const int k = jj & (NS - 1);
            const int base = (jj / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) sm.st(base + r * NS, v[b * R + r]);
        }
        __syncthreads();
        fft_rest<T, P, INV, NS * R>(v, j, tw, sm);
    }
}

// Whole-line transform.  All threads of the CTA must call it (it contains
// __syncthreads); the shared-memory line must not be in use by anyone else.
template <typename T, int P, bool INV, class View>
__device__ __forceinline__ void fft_line(cpx<T>* v, int j, const cpx<T>* tw, const View& sm) {
    dft8<T, INV>(v);
    if constexpr (P > 8) {
#pragma unroll
        for (int r = 0; r < 8; ++r) sm.st(8 * j + r, v[r]);
        __syncthreads();
        fft_rest<T, P, INV, 8>(v, j, tw, sm);
    }
}

// Output index of register slot s after fft_line (see the header comment).
template <int P> __device__ __forceinline__ int out_index(int j, int s) {
    constexpr int R = LastRadix<P>::value;
    return j + (s / R) * (P / 8) + (s % R) * (P / R);
}

// Output distribution -> input distribution, same thread:
// in[b + r * (8/R)] = out[b * R + r].
template <typename T, int P> __device__ __forceinline__ void seam_permute(cpx<T>* v) {
    constexpr int R = LastRadix<P>::value;
    constexpr int NB = 8 / R;
    cpx<T> t[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) t[s] = v[s];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) v[b + r * NB] = t[b * R + r];
}

}  // namespace nm
