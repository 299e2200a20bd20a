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

cudaError_t run_zseam_paired_f32(const ConvArgs<float>& a, int np, int P, int TX, cudaStream_t s) {
    if (TX == 16) return zseam2_p<16>(a, np, P, s);
    if (TX == 32) return zseam2_p<32>(a, np, P, s);
    return cudaErrorInvalidValue;
}

}  // namespace nm
