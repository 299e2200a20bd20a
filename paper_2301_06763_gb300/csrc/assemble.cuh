// assemble.cuh -- device code of the cross-level assembly (Eq. 14 and its
// dipole variants) and of the carried Eqs. 3-6 interpolation, shared by the
// kernels of support.cu and the persistent batch kernel (persist.cu).
#pragma once
#include "../../include/nm.h"
#include "internal.h"
#include "dfloat.cuh"

namespace nm {

// ---------------------------------------------------------------- assembly
// Phi(Omega^n) = base_n + reduce(dbl_n) + sum_{k<n} interp_{k->n}(hole_k).
// Trilinear interpolation from level k straight to level n: the level-n
// centre i sits at level-k fractional index
//   u = N/2 - N/(2r) + (i + 1/2)/r - 1/2,  r = 2^(n-k),
// i.e. 2r u = (N - 1)(r - 1) + 2i, so the stencil corner and weight follow in
// integer arithmetic (shifts: N and r are powers of two) and the weights are
// exact.  The coarser levels' interpolated terms (and the reduced doubled
// grid) are summed in T; the final per-cell addition of that cross-level sum to
// the level's own potential is done in double (FP64 mode: everything in
// double).  GB300's FP64 pipe runs at 1/69 of its FP32 rate, so the FP32 path
// spends one double addition per cell.
template <typename T>
__device__ __forceinline__ void axis_stencil(int N, int lgr, int i, int& i0, T& t) {
    const int num = (N - 1) * ((1 << lgr) - 1) + 2 * i;
    i0 = num >> (lgr + 1);
    // a dyadic fraction with at most 16 bits: exact in float
    t = (T)((float)(num & ((2 << lgr) - 1)) * (1.0f / (float)(2 << lgr)));
}

// Exact float -> double in integer arithmetic (sign, exponent re-biased by
// 1023 - 127 = 896, mantissa shifted by 29; subnormals normalised, infinities
// and NaNs mapped to exponent 2047), so the FP32 path spends its FP64 pipe only
// on the final additions.
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned mag = u & 0x7fffffffu;
    if (mag - 0x00800000u < 0x7f000000u) {
        // normal numbers (exponent field 1 .. 254), the common case: the high
        // word is sign | (e + 896) << 20 | m >> 3, the low word m << 29
        return __hiloint2double((int)(((mag >> 3) + (896u << 20)) | (u & 0x80000000u)), (int)(u << 29));
    }
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    unsigned e = (u >> 23) & 0xffu;
    unsigned m = u & 0x7fffffu;
    unsigned long long ed;
    if (e == 0xffu) {
        ed = 2047ull;
    } else if (e != 0u) {
        ed = e + 896u;
    } else if (m == 0u) {
        return __longlong_as_double((long long)sign);
    } else {
        const int s = __clz(m) - 8;        // brings the leading one to bit 23
        m = (m << s) & 0x7fffffu;
        ed = (unsigned long long)(897 - s);
    }
    return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)m << 29)));
}
__device__ __forceinline__ double widen(double d) { return d; }

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    static __device__ __forceinline__ void load(const float* p, float* v) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <> struct Vec4<double> {
    static __device__ __forceinline__ void load(const double* p, double* v) {
        const double2 q0 = reinterpret_cast<const double2*>(p)[0];
        const double2 q1 = reinterpret_cast<const double2*>(p)[1];
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
};
template <> struct Vec4<df> {
    static __device__ __forceinline__ void load(const df* p, df* v) {
        const float4 q0 = reinterpret_cast<const float4*>(p)[0];
        const float4 q1 = reinterpret_cast<const float4*>(p)[1];
        v[0] = df(q0.x, q0.y); v[1] = df(q0.z, q0.w); v[2] = df(q1.x, q1.y); v[3] = df(q1.z, q1.w);
    }
};

// A level's own potential b plus the cross-level sum acc, as the double that
// phi stores: float and double widen each and add once in double; df sums in
// df first, then one conversion.
__device__ __forceinline__ double out_sum(float b, float acc) { return widen(b) + widen(acc); }
__device__ __forceinline__ double out_sum(double b, double acc) { return b + acc; }
__device__ __forceinline__ double out_sum(df b, df acc) { return df_to_double(b + acc); }

// Eqs. 3-6 on one axis: level-(n-1) position of level-n index i (i >= -1) is
// (N/2 + i)/2 - 1/4 = c + s/4: nearest coarse index c, diagonal step s.
__device__ __forceinline__ void diag_axis(int N, int i, int& c, int& s) {
    c = (N / 2 + i) >> 1;
    s = (i & 1) ? 1 : -1;
}
// The two-point rule's weights on the nearest coarse value and its diagonal
// neighbour, and one carried value (the rule plus the level's hole term).
template <typename T> __device__ __forceinline__ T diag_mix(T near, T diag) {
    return T(0.75) * near + T(0.25) * diag;
}
template <typename T> __device__ __forceinline__ T carry_value(T near, T diag, T hole) {
    return diag_mix<T>(near, diag) + hole;
}
// The two-point rule at level-n cell (z, y, x) from a level-(n-1) field
// stored from `o` on, `E` per axis.
template <typename T>
__device__ __forceinline__ T diag_value(const T* src, int o, int E, int N, int z, int y, int x) {
    int cz, sz, cy, sy, cx, sx;
    diag_axis(N, z, cz, sz);
    diag_axis(N, y, cy, sy);
    diag_axis(N, x, cx, sx);
    const T near = src[((size_t)(cz - o) * E + (cy - o)) * E + (cx - o)];
    const T diag = src[((size_t)(cz + sz - o) * E + (cy + sy - o)) * E + (cx + sx - o)];
    return diag_mix<T>(near, diag);
}

// One step of the carried interpolation on cells i = i0, i0 + stride, ...
// (below `end` when given)
template <typename T>
__device__ __forceinline__ void carry_body(const CarryArgs<T>& a, size_t i0, size_t stride,
                                           size_t end = ~(size_t)0) {
    const int N = a.N, nc = N / 2 + 2, o = N / 4 - 1;
    size_t total = (size_t)nc * nc * nc;
    if (end < total) total = end;
    for (size_t i = i0; i < total; i += stride) {
        const int x = (int)(i % nc) + o, y = (int)((i / nc) % nc) + o, z = (int)(i / ((size_t)nc * nc)) + o;
        const int ho = a.hole_origin, hE = a.hole_extent;
        const T h = a.hole[((size_t)(z - ho) * hE + (y - ho)) * hE + (x - ho)];
        a.out[i] = diag_value<T>(a.prev, a.prev_origin, a.prev_extent, N, z, y, x) + h;   // carry_value
    }
}

// The stencil weight of axis_stencil in float (a dyadic fraction with at most
// 16 bits, so exact), widened to T without the FP64 pipe.
__device__ __forceinline__ float stencil_weight(int N, int lgr, int i, int& i0) {
    const int num = (N - 1) * ((1 << lgr) - 1) + 2 * i;
    i0 = num >> (lgr + 1);
    return (float)(num & ((2 << lgr) - 1)) * (1.0f / (float)(2 << lgr));
}
template <typename T> __device__ __forceinline__ T as_t(float f);
template <> __device__ __forceinline__ float as_t<float>(float f) { return f; }
template <> __device__ __forceinline__ double as_t<double>(float f) { return widen(f); }
template <> __device__ __forceinline__ df as_t<df>(float f) { return df(f); }

// Row-wise assembly (N >= 16): a team of N/4 threads owns one fine row
// (level n, z, y), 4 cells per thread.  For each coarser level k the row's
// z and y stencils are fixed, so the team first interpolates bilinearly in
// (z, y) at every coarse x the row needs (N/2^(n-k) + 2 values) into shared
// memory, then each cell interpolates linearly along x from there: the same
// trilinear value with about a third of the loads and arithmetic.
// Rows [rb0, rb0 + rows_cta), rb0 + rows_cta * stride, ... (rb0 a multiple of
// rows_cta); `smem_rows` holds rows_cta (N/2 + 2) values of T.
template <typename T>
__device__ __forceinline__ void assemble_rows_body(const AssembleArgs<T>& a, int lgN, size_t rb0, size_t stride,
                                                   unsigned char* smem_rows) {
    const int N = 1 << lgN;
    const int team = N >> 2;                 // threads per fine row
    const int rows_cta = 256 / team;         // rows per CTA (divides N^2 for N >= 16)
    const int crw = N / 2 + 2;               // coarse values per row, at most
    const int tr = threadIdx.x / team, tl = threadIdx.x % team;
    const int x0 = 4 * tl;
    T* cr = reinterpret_cast<T*>(smem_rows) + tr * crw;
    const size_t N2 = (size_t)1 << (2 * lgN);
    const size_t rows_total = N2 * a.levels;
    for (size_t rb = rb0; rb < rows_total; rb += stride * rows_cta) {
        const int n = (int)(rb >> (2 * lgN));            // same level for the whole batch
        const size_t zy = rb + tr - ((size_t)n << (2 * lgN));
        const int z = (int)(zy >> lgN), y = (int)(zy & (N - 1));
        const size_t cell = (zy << lgN) + x0;
        T b[4];
        Vec4<T>::load(a.base[n] + cell, b);
        T acc[4] = {T(0), T(0), T(0), T(0)};
        if (a.dbl[n]) {
            const int E = 2 * N;
            const T* d = a.dbl[n];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                T s = T(0);
#pragma unroll
                for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy) {
                        const T* row = d + ((size_t)(2 * z + dz) * E + (2 * y + dy)) * E + 2 * (x0 + c);
                        s += row[0] + row[1];
                    }
                acc[c] += s * T(0.125);
            }
        }
        if (a.red[n]) {
            T r[4];
            Vec4<T>::load(a.red[n] + cell, r);
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] += r[c];
        }
        if (a.diag && n > 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                acc[c] += diag_value<T>(a.interp[n - 1], a.interp_origin[n - 1], a.interp_extent[n - 1], N, z, y,
                                        x0 + c);
        }
        for (int k = 0; k < (a.diag ? 0 : n); ++k) {
            const int lgr = n - k;
            int iz, iy, lo, hi;
            const T tz = as_t<T>(stencil_weight(N, lgr, z, iz));
            const T ty = as_t<T>(stencil_weight(N, lgr, y, iy));
            stencil_weight(N, lgr, 0, lo);
            stencil_weight(N, lgr, N - 1, hi);
            const int cnt = hi - lo + 2;
            const int o = a.interp_origin[k], E = a.interp_extent[k];
            const size_t sz = (size_t)E * E, sy = E;
            const T* src = a.interp[k] + ((size_t)(iz - o) * E + (iy - o)) * E - o;
            for (int i = tl; i < cnt; i += team) {
                const T* p = src + lo + i;
                const T c0 = p[0] + ty * (p[sy] - p[0]);
                const T c1 = p[sz] + ty * (p[sz + sy] - p[sz]);
                cr[i] = c0 + tz * (c1 - c0);
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int ix;
                const T tx = as_t<T>(stencil_weight(N, lgr, x0 + c, ix));
                const T* q = cr + (ix - lo);
                acc[c] += q[0] + tx * (q[1] - q[0]);
            }
            __syncthreads();
        }
        double2* out = reinterpret_cast<double2*>(a.phi + ((size_t)n << (3 * lgN)) + cell);
        out[0] = make_double2(out_sum(b[0], acc[0]), out_sum(b[1], acc[1]));
        out[1] = make_double2(out_sum(b[2], acc[2]), out_sum(b[3], acc[3]));
    }
}

}  // namespace nm
