// dipole3.cu -- the two extra terms of the three-level dipole scheme
// (Appendix B, Eqs. B.3-B.6) that feed the assembly of a level n < L-2:
// the potential of level n+2's mass computed on its quadrupled grid and
// reduced by 4^3 to level n's cells, or instead summed directly at level n's
// cell centres (Eq. B.6).
#include "internal.h"

namespace nm {

// One thread per output cell; its 4^3 inputs are 4 rows of 4 along x.
template <typename T>
__global__ void __launch_bounds__(256) k_reduce4(const T* __restrict__ in, T* __restrict__ out, int N) {
    const size_t N3 = (size_t)N * N * N;
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= N3) return;
    const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((size_t)N * N));
    const size_t F = 4 * (size_t)N;
    T s = T(0);
#pragma unroll
    for (int dz = 0; dz < 4; ++dz)
#pragma unroll
        for (int dy = 0; dy < 4; ++dy) {
            const T* r = in + ((4 * (size_t)z + dz) * F + (4 * (size_t)y + dy)) * F + 4 * (size_t)x;
            s += (r[0] + r[1]) + (r[2] + r[3]);
        }
    out[i] = s * T(1.0 / 64.0);
}

template <typename T>
cudaError_t run_reduce4(const T* in, T* out, int N, cudaStream_t s) {
    ProfScope ps(sizeof(T) == 4 ? "reduce4_f32" : "reduce4_f64", 1, s);
    const size_t n = (size_t)N * N * N;
    k_reduce4<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, N);
    count_launches(1);
    return cudaGetLastError();
}
template cudaError_t run_reduce4<float>(const float*, float*, int, cudaStream_t);
template cudaError_t run_reduce4<double>(const double*, double*, int, cudaStream_t);

template <typename T> __device__ __forceinline__ T rsqrt_t(T v);
template <> __device__ __forceinline__ float rsqrt_t<float>(float v) { return rsqrtf(v); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double v) { return rsqrt(v); }

// Eq. B.6 by tiles: each thread owns one target (a level-n cell), each CTA
// stages 256 source densities of level n+2 at a time in shared memory; every
// tile's partial sum is added to a double accumulator.
constexpr int kDirectTile = 256;

template <typename T> struct alignas(4 * sizeof(T)) Src4 { T x, y, z, m; };

template <typename T>
__global__ void __launch_bounds__(kDirectTile) k_direct2(const T* __restrict__ rho, const T* __restrict__ restr,
                                                          T* __restrict__ out, int N, double scale) {
    __shared__ Src4<T> src[kDirectTile];
    const size_t N3 = (size_t)N * N * N;
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const bool live = i < N3;
    const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((size_t)N * N));
    // target in level-(n+2) cell units: 4 i + 3/2 - 3N/2 (exact in float)
    const T off = T(1.5) - T(1.5) * T(N);
    const T ux = T(4 * x) + off, uy = T(4 * y) + off, uz = T(4 * z) + off;
    const int q = N / 4, h = N / 2;
    double acc = 0.0;
    for (size_t j0 = 0; j0 < N3; j0 += kDirectTile) {
        const size_t j = j0 + threadIdx.x;
        Src4<T> v{T(0), T(0), T(0), T(0)};
        if (j < N3) {
            const int sx = (int)(j % N), sy = (int)((j / N) % N), sz = (int)(j / ((size_t)N * N));
            const bool cov = restr && (unsigned)(sx - q) < (unsigned)h && (unsigned)(sy - q) < (unsigned)h &&
                             (unsigned)(sz - q) < (unsigned)h;
            v = {T(sx), T(sy), T(sz), cov ? restr[((size_t)(sz - q) * h + (sy - q)) * h + (sx - q)] : rho[j]};
        }
        __syncthreads();
        src[threadIdx.x] = v;
        __syncthreads();
        const int cnt = N3 - j0 < (size_t)kDirectTile ? (int)(N3 - j0) : kDirectTile;
        T part = T(0);
        for (int k = 0; k < cnt; ++k) {
            const Src4<T> c = src[k];
            const T dx = ux - c.x, dy = uy - c.y, dz = uz - c.z;
            part += c.m * rsqrt_t<T>(dx * dx + dy * dy + dz * dz);
        }
        acc += (double)part;
    }
    if (live) out[i] = (T)(scale * acc);
}

template <typename T>
cudaError_t run_direct2(const T* rho, const T* restr, T* out, int N, double scale, cudaStream_t s) {
    ProfScope ps(sizeof(T) == 4 ? "direct2_f32" : "direct2_f64", 1, s);
    const size_t n = (size_t)N * N * N;
    k_direct2<T><<<(unsigned)((n + kDirectTile - 1) / kDirectTile), kDirectTile, 0, s>>>(rho, restr, out, N, scale);
    count_launches(1);
    return cudaGetLastError();
}
template cudaError_t run_direct2<float>(const float*, const float*, float*, int, double, cudaStream_t);
template cudaError_t run_direct2<double>(const double*, const double*, double*, int, double, cudaStream_t);

}  // namespace nm
