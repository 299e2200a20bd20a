// conv_f32_pair.cu -- the FP32 z-seam with two columns per thread (k_zseam2),
// level grids, 16 values per thread, for both column-tile widths.
#include <mutex>

#include "internal.h"

namespace nm {

template <int P, int TX>
static cudaError_t launch_zseam2(const ConvArgs<float>& a, int np, cudaStream_t s) {
    constexpr int E = 16, NT = TX / 2 * P / E, H = P / 2 + 1;
    const size_t smem = (size_t)P * sizeof(cpx<f2>) + (size_t)(TX / 2) * P * sizeof(cpx<f2>) +
                        (size_t)H * TX * sizeof(float);
    static PerDevice<cudaError_t> prep;   // the shared-memory limit, once per device
    const cudaError_t pe = prep.get(current_device(), [&]() {
        return cudaFuncSetAttribute(k_zseam2<P, E, TX, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }, cudaErrorInvalidDevice);
    if (pe != cudaSuccess) return pe;
    // the kernel reads the spectrum as float rows over all kx
    const float* specx = unfolded_spectrum(a.spec);
    if (!specx) return cudaErrorInvalidValue;
    static ConvArgs<float> b;   // host staging of the (large) parameter block
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    b = a;
    b.spec = specx;
    k_zseam2<P, E, TX, 0><<<dim3(P / TX, P, np), NT, smem, s>>>(b);
    return cudaGetLastError();
}

template <int TX>
static cudaError_t zseam2_p(const ConvArgs<float>& a, int np, int P, cudaStream_t s) {
    switch (P) {
        case 64: return launch_zseam2<64, TX>(a, np, s);
        case 128: return launch_zseam2<128, TX>(a, np, s);
        case 256: return launch_zseam2<256, TX>(a, np, s);
        case 512: return launch_zseam2<512, TX>(a, np, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int P, int TX>
static cudaError_t launch_zseam_s(const ConvArgs<float>& a, int np, cudaStream_t s) {
    constexpr int E = 16, NT = TX * P / E, H = P / 2 + 1;
    const size_t smem = (size_t)P * sizeof(cpx<float>) + (size_t)TX * P * sizeof(cpx<float>) +
                        (size_t)H * TX * sizeof(float);
    static PerDevice<cudaError_t> prep;   // the shared-memory limit, once per device
    const cudaError_t pe = prep.get(current_device(), [&]() {
        return cudaFuncSetAttribute(k_zseam_s<P, E, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }, cudaErrorInvalidDevice);
    if (pe != cudaSuccess) return pe;
    const float* specx = unfolded_spectrum(a.spec);
    if (!specx) return cudaErrorInvalidValue;
    static ConvArgs<float> b;   // host staging of the (large) parameter block
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    b = a;
    b.spec = specx;
    k_zseam_s<P, E, TX><<<dim3(P / TX, P, np), NT, smem, s>>>(b);
    return cudaGetLastError();
}

cudaError_t run_zseam_staged_f32(const ConvArgs<float>& a, int np, int P, int TX, cudaStream_t s) {
    if (TX == 16) {
        switch (P) {
            case 64: return launch_zseam_s<64, 16>(a, np, s);
            case 128: return launch_zseam_s<128, 16>(a, np, s);
            case 256: return launch_zseam_s<256, 16>(a, np, s);
            case 512: return launch_zseam_s<512, 16>(a, np, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (TX == 32) {
        switch (P) {
            case 64: return launch_zseam_s<64, 32>(a, np, s);
            case 128: return launch_zseam_s<128, 32>(a, np, s);
            case 256: return launch_zseam_s<256, 32>(a, np, s);
            case 512: return launch_zseam_s<512, 32>(a, np, s);
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaErrorInvalidValue;
}

template <int P>
static cudaError_t launch_xfwd2(const ConvArgs<float>& a, int np, cudaStream_t s) {
    constexpr int E = 16, TPL = P / E, LINES = 256 / TPL, LP = LINES / 2, N = P / 2;
    const size_t smem = (size_t)P * sizeof(cpx<f2>) + (size_t)LP * (P + P / E) * sizeof(cpx<f2>) +
                        2 * (size_t)XfwdStage<float, P, E>::ELEMS * sizeof(float);
    static PerDevice<KernelPrep> prep;   // shared-memory limit and resident CTAs per SM, once per device
    const KernelPrep kp = prep.get(current_device(), [&]() {
        KernelPrep r;
        r.err = cudaFuncSetAttribute(k_xfwd_pipe2<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r.err == cudaSuccess)
            r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.occ, k_xfwd_pipe2<P>, 128, smem);
        return r;
    }, KernelPrep{cudaErrorInvalidDevice, 0});
    if (kp.err != cudaSuccess) return kp.err;
    const int tiles = np * (N * N / LINES);
    int grid = (kp.occ > 0 ? kp.occ : 1) * sm_count();
    if (grid > tiles) grid = tiles;
    k_xfwd_pipe2<P><<<grid, 128, smem, s>>>(a, np);
    return cudaGetLastError();
}

cudaError_t run_xfwd_paired_f32(const ConvArgs<float>& a, int np, int P, cudaStream_t s) {
    switch (P) {
        case 256: return launch_xfwd2<256>(a, np, s);
        case 512: return launch_xfwd2<512>(a, np, s);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------- pass 3, persistent (P = 256)
// The paired z-seam of k_zseam2 at P = 256 as a persistent pipeline.  Each of
// the resident CTAs (four of 128 threads per SM) walks tiles u = blockIdx.x,
// + gridDim.x, ... of a list ordered by pair, then ky, then column tile (a
// pair with one real field lists only the tiles up to kx = N), so the tiles in
// flight across the GPU at any moment are neighbours in memory.  Every thread
// fetches its own 8 live 16-byte column chunks of the next tile into a
// private slot of a staging buffer with cp.async as soon as it has moved the
// current tile's chunks from there into registers, and the next tile's
// spectrum rows follow once every thread is past the current multiply: the
// column loads of tile u + gridDim.x overlap the transforms of tile u instead
// of preceding them.  The room for the staging buffer comes from the line
// exchange, which moves the real parts and then the imaginary parts through
// one 16 KB buffer (two half-size exchanges instead of one 32 KB exchange), so
// the CTA's shared memory stays at 45 KB and four CTAs still fit an SM.
// The transforms are k_zseam2's (the same first and second 16-point passes,
// twiddles and spectrum products); the results agree with it to FP32
// rounding.
namespace zp {
constexpr int P = 256, E = 16, TX = 16, TX2 = TX / 2, NT = TX2 * (P / E), H = P / 2 + 1, LIVE = 8;
constexpr int XB = P * TX2 + TX2 * (P / E);  // f2 slots of the half exchange (padded)
constexpr int STAGE = LIVE * (P / E) * TX2;  // 16-byte column chunks of one tile
constexpr size_t SMEM = (size_t)P * sizeof(cpx<f2>) + (size_t)XB * sizeof(f2) + (size_t)STAGE * 16 +
                        (size_t)H * TX * sizeof(float);
// Slot of element e of column pair l in the half exchange: the 8 pairs of an
// element are one 64-byte run, and one 64-byte gap follows every 16
// elements, so that the stores of the first pass (elements 16 j + r) and the
// loads of the second (j + 16 r) of a warp's four lines fall in alternate
// bank halves.
__device__ __forceinline__ int xoff(int e, int l) { return e * TX2 + l + TX2 * (e >> 4); }

// One 256-point line transform over cpx<f2> with the two-step exchange.
// M: live registers of the first pass; after_first() runs once the first
// pass has consumed every input register.
template <bool INV, unsigned M, class F>
__device__ __forceinline__ void line(cpx<f2>* v, int j, int l, const cpx<f2>* sm_tw, f2* xb, const F& after_first) {
    dft16m<f2, INV, M>(v);                   // element 16 j + r in register r
    after_first();
#pragma unroll
    for (int r = 0; r < E; ++r) xb[xoff(E * j + r, l)] = v[r].re;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < E; ++r) v[r].re = xb[xoff(j + E * r, l)];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < E; ++r) xb[xoff(E * j + r, l)] = v[r].im;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < E; ++r) v[r].im = xb[xoff(j + E * r, l)];
#pragma unroll
    for (int r = 1; r < E; ++r) v[r] = cmul(v[r], twiddle<f2, INV>(sm_tw, j * r));
    dftR<f2, INV, E>(v);                     // element j + 16 s in register s
}
}  // namespace zp

__global__ void __launch_bounds__(zp::NT, 4) k_zseam2p(const __grid_constant__ ConvArgs<float> a, int npairs) {
    using namespace zp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<f2>* sm_tw = reinterpret_cast<cpx<f2>*>(smem_raw);
    f2* xb = reinterpret_cast<f2*>(sm_tw + P);
    float4* stage = reinterpret_cast<float4*>(xb + XB);
    float* sm_sp = reinterpret_cast<float*>(stage + STAGE);   // [H][TX]
    __shared__ int first[kMaxPairs + 1];                       // first tile of each pair
    if (threadIdx.x == 0) {
        int f = 0;
        for (int p = 0; p < npairs; ++p) {
            first[p] = f;
            f += P * (a.pair[p].half ? (P / 2) / TX + 1 : P / TX);
        }
        first[npairs] = f;
    }
    for (int i = threadIdx.x; i < P; i += NT) {
        const cpx<float> w = a.tw[i];
        sm_tw[i] = {f2(w.re, w.re), f2(w.im, w.im)};
    }
    __syncthreads();
    const int total = first[npairs];
    const int l = threadIdx.x % TX2, j = threadIdx.x / TX2;
    // tile u: its pair p, ky row y and first column x0
    int p = 0;
    auto locate = [&](int u, int& y, int& x0) {
        while (u >= first[p + 1]) ++p;
        const int xt = a.pair[p].half ? (P / 2) / TX + 1 : P / TX;
        const int r = u - first[p];
        y = r / xt;
        x0 = (r % xt) * TX;
    };
    auto fetch_columns = [&](int u) {
        int y, x0;
        const int p0 = p;
        locate(u, y, x0);
        const cpx<float>* col = a.pair[p].work + (size_t)y * P + x0 + 2 * l;
#pragma unroll
        for (int r = 0; r < LIVE; ++r)
            cp_async16(stage + (r * (P / E) + j) * TX2 + l, col + (size_t)(j + r * (P / E)) * P * P);
        p = p0;
    };
    auto fetch_spectrum = [&](int u) {
        int y, x0;
        const int p0 = p;
        locate(u, y, x0);
        p = p0;
        const int fy = y <= P / 2 ? y : P - y;
        const float* sp = a.spec + (size_t)fy * P + x0;
        for (int i = threadIdx.x; i < H * (TX / 4); i += NT) {
            const int fz = i / (TX / 4), c = i % (TX / 4);
            cp_async16(sm_sp + fz * TX + 4 * c, sp + (size_t)fz * H * P + 4 * c);
        }
    };
    int u = blockIdx.x;
    if (u < total) {
        fetch_columns(u);
        fetch_spectrum(u);
        cp_async_commit();
    }
    for (; u < total; u += gridDim.x) {
        int y, x0;
        locate(u, y, x0);
        const int nu = u + gridDim.x;
        cp_async_wait_all();
        __syncthreads();   // this tile's spectrum rows (every thread's copies) and the exchange buffer are free to use
        cpx<f2> v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if (r < LIVE) {
                const float4 q = stage[(r * (P / E) + j) * TX2 + l];
                v[r] = {f2(q.x, q.z), f2(q.y, q.w)};
            } else {
                v[r] = {f2(0), f2(0)};
            }
        }
        // once the first pass has consumed this thread's staged chunks, its
        // slots take the next tile's columns
        line<false, 0x00FFu>(v, j, l, sm_tw, xb, [&]() {
            if (nu < total) {
                fetch_columns(nu);
                cp_async_commit();
            }
        });
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const int kz = j + E * s;
            const int fz = kz <= P / 2 ? kz : P - kz;
            const float2 g = *reinterpret_cast<const float2*>(sm_sp + fz * TX + 2 * l);
            v[s].re *= f2(g.x, g.y);
            v[s].im *= f2(g.x, g.y);
        }
        __syncthreads();   // every thread is past the multiply and the forward exchange
        if (nu < total) {
            fetch_spectrum(nu);
            cp_async_commit();
        }
        line<true, 0xFFFFu>(v, j, l, sm_tw, xb, []() {});
        cpx<float>* col = a.pair[p].work + (size_t)y * P + x0 + 2 * l;
#pragma unroll
        for (int s = 0; s < E / 2; ++s) {   // outputs j + 16 s < P / 2
            const int e = j + E * s;
            *reinterpret_cast<float4*>(col + (size_t)e * P * P) =
                make_float4(v[s].re.x, v[s].im.x, v[s].re.y, v[s].im.y);
        }
    }
    cp_async_wait_all();
}

static cudaError_t launch_zseam2p(const ConvArgs<float>& a, int np, cudaStream_t s) {
    static PerDevice<KernelPrep> prep;   // shared-memory limit and resident CTAs per SM, once per device
    const KernelPrep kp = prep.get(current_device(), [&]() {
        KernelPrep r;
        r.err = cudaFuncSetAttribute(k_zseam2p, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zp::SMEM);
        if (r.err == cudaSuccess)
            r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.occ, k_zseam2p, zp::NT, zp::SMEM);
        return r;
    }, KernelPrep{cudaErrorInvalidDevice, 0});
    if (kp.err != cudaSuccess) return kp.err;
    const float* specx = unfolded_spectrum(a.spec);
    if (!specx) return cudaErrorInvalidValue;
    int tiles = 0;
    for (int i = 0; i < np; ++i) tiles += zp::P * (a.pair[i].half ? (zp::P / 2) / zp::TX + 1 : zp::P / zp::TX);
    int grid = (kp.occ > 0 ? kp.occ : 1) * sm_count();
    if (grid > tiles) grid = tiles;
    static ConvArgs<float> b;   // host staging of the (large) parameter block
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    b = a;
    b.spec = specx;
    k_zseam2p<<<grid, zp::NT, zp::SMEM, s>>>(b, np);
    return cudaGetLastError();
}

cudaError_t run_zseam_persist_f32(const ConvArgs<float>& a, int np, int P, cudaStream_t s) {
    if (P != zp::P) return cudaErrorInvalidValue;
    return launch_zseam2p(a, np, s);
}

cudaError_t run_zseam_paired_f32(const ConvArgs<float>& a, int np, int P, int TX, cudaStream_t s) {
    if (TX == 16) return zseam2_p<16>(a, np, P, s);
    if (TX == 32) return zseam2_p<32>(a, np, P, s);
    return cudaErrorInvalidValue;
}

}  // namespace nm
