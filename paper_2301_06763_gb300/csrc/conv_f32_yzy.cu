// conv_f32_yzy.cu -- launchers of the three-pass convolution (yzy.cuh):
// kx-major x-forward, the fused y/z/y pass in clusters, kx-major x-inverse.
#include <cstdio>

#include "internal.h"
#include "yzy.cuh"

namespace nm {

bool yzy_pairs_ok(const PairDesc<float>* pairs, int npairs) {
    for (int i = 0; i < npairs; ++i) {
        const PairDesc<float>& d = pairs[i];
        if (d.src[0].mode != SRC_FULL || ((uintptr_t)d.src[0].rho & 15) ||
            (d.src[0].restr && ((uintptr_t)d.src[0].restr & 7)) || ((uintptr_t)d.work & 15))
            return false;
        if (!(d.src[1].mode == SRC_NONE || (d.src[1].mode == SRC_HOLE && d.src[1].rho == d.src[0].rho)))
            return false;
    }
    return true;
}

template <int P, int C>
static cudaError_t yzy_passes(const ConvArgs<float>& a, int np, cudaStream_t s) {
    constexpr int E = 16, TPL = P / E, LINES = 256 / TPL, N = P / 2;
    using S = YzyShape<P, C>;
    static_assert(S::SMEM <= 227 * 1024, "fused plane exceeds the shared memory of an SM");
    const size_t c = sizeof(cpx<float>);
    const size_t sm_x = (size_t)P * c + (size_t)XtShape<P>::SCR * c;
    const size_t sm_f = sm_x + 2 * (size_t)XfwdStage<float, P, E>::ELEMS * sizeof(float);
    static PerDevice<KernelPrep> prep;
    const KernelPrep kp = prep.get(current_device(), [&]() {
        KernelPrep r;
        r.err = cudaFuncSetAttribute(k_xfwd_t<float, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_f);
        if (r.err == cudaSuccess)
            r.err = cudaFuncSetAttribute(k_yzy<P, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (r.err == cudaSuccess)
            r.err = cudaFuncSetAttribute(k_xinv_t<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_x);
        if (r.err == cudaSuccess)
            r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.occ, k_xfwd_t<float, P>, 256, sm_f);
        return r;
    }, KernelPrep{cudaErrorInvalidDevice, 0});
    if (kp.err != cudaSuccess) return kp.err;
    char nm_[48];
    {
        snprintf(nm_, sizeof nm_, "xfwdT_f32_P%d", P);
        ProfScope ps(nm_, np, s);
        const int tiles = np * (N * N / LINES);
        int grid = (kp.occ > 0 ? kp.occ : 1) * sm_count();
        if (grid > tiles) grid = tiles;
        k_xfwd_t<float, P><<<grid, 256, sm_f, s>>>(a, np);
    }
    {
        snprintf(nm_, sizeof nm_, "yzy_f32_P%d", P);
        ProfScope ps(nm_, np, s);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C, P, np);
        cfg.blockDim = dim3(S::NT, 1, 1);
        cfg.dynamicSmemBytes = S::SMEM;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_yzy<P, C>, a);
        if (e != cudaSuccess) return e;
    }
    {
        snprintf(nm_, sizeof nm_, "xinvT_f32_P%d", P);
        ProfScope ps(nm_, np, s);
        k_xinv_t<P><<<dim3(N * N / LINES, np), 256, sm_x, s>>>(a);
    }
    count_launches(3);
    return cudaGetLastError();
}

template <int P, int C>
static cudaError_t yzy_chunks(const PairDesc<float>* pairs, int npairs, const float* spec, const cpx<float>* tw,
                              cudaStream_t s) {
    static ConvArgs<float> a;   // host staging of the (large) parameter block
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    a.spec = spec;
    a.tw = tw;
    for (int i0 = 0; i0 < npairs; i0 += kMaxPairs) {
        const int np = npairs - i0 < kMaxPairs ? npairs - i0 : kMaxPairs;
        for (int i = 0; i < np; ++i) a.pair[i] = pairs[i0 + i];
        cudaError_t e = yzy_passes<P, C>(a, np, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t run_conv_f32_yzy(const PairDesc<float>* pairs, int npairs, int P, int split, const float* spec,
                             const cpx<float>* tw, cudaStream_t s) {
    // the kernel reads the spectrum with fz fastest
    const float* sz = zfast_spectrum(spec);
    if (!sz || !yzy_pairs_ok(pairs, npairs)) return cudaErrorInvalidValue;
    switch (P) {
        case 64: return split == 0 ? yzy_chunks<64, 2>(pairs, npairs, sz, tw, s) : cudaErrorInvalidValue;
        case 128: return split == 0 ? yzy_chunks<128, 2>(pairs, npairs, sz, tw, s)
                                    : yzy_chunks<128, 4>(pairs, npairs, sz, tw, s);
        case 256: return split == 0 ? yzy_chunks<256, 4>(pairs, npairs, sz, tw, s)
                                    : yzy_chunks<256, 2>(pairs, npairs, sz, tw, s);
        case 512: return split == 0 ? yzy_chunks<512, 8>(pairs, npairs, sz, tw, s) : cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace nm
