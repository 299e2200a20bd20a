// conv_inst.cuh -- host dispatch of the five convolution passes for one real
// type; included once per precision (conv_f32.cu, conv_f64.cu).
#pragma once
#include <cstdio>

#include "internal.h"

namespace nm {

template <typename K>
static cudaError_t prep_kernel(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T, int P, bool DBL>
static cudaError_t conv_passes(const ConvArgs<T>& a, int np, cudaStream_t s) {
    using Gm = Geo<P, DBL>;
    constexpr int E = EOf<P>::value;
    constexpr int TPL = P / E;
    constexpr int LINES = 256 / TPL;
    constexpr int TX = Tile<T, P>::TX;
    constexpr int NT = TX * P / E;   // threads of the strided passes
    const size_t c = sizeof(cpx<T>);
    const size_t sm_x = (size_t)P * c + (size_t)LINES * (P + P / E) * c;
    const size_t sm_yz = (size_t)P * c + (size_t)TX * P * c;
    // shared-memory limits are set once per kernel (thread-safe static init)
    static const cudaError_t prepared = [&]() {
        cudaError_t e;
        if ((e = prep_kernel(k_xfwd<T, T, P, DBL>, sm_x)) != cudaSuccess) return e;
        if ((e = prep_kernel(k_ypass<T, P, TX, false, DBL>, sm_yz)) != cudaSuccess) return e;
        if ((e = prep_kernel(k_zseam<T, P, TX, DBL>, sm_yz)) != cudaSuccess) return e;
        if ((e = prep_kernel(k_ypass<T, P, TX, true, DBL>, sm_yz)) != cudaSuccess) return e;
        return prep_kernel(k_xinv<T, P, DBL>, sm_x);
    }();
    if (prepared != cudaSuccess) return prepared;
    const int rows_in = Gm::NIN * Gm::NIN;
    const int rows_out = Gm::NOUT * Gm::NOUT;
    char nm_[48];
    const char* tag = sizeof(T) == 4 ? "f32" : "f64";
    const char* geo = DBL ? "_dbl" : "";
    {
        snprintf(nm_, sizeof nm_, "xfwd%s_%s_P%d", geo, tag, P);
        ProfScope ps(nm_, np, s);
        k_xfwd<T, T, P, DBL><<<dim3((rows_in + LINES - 1) / LINES, np), 256, sm_x, s>>>(a);
    }
    {
        snprintf(nm_, sizeof nm_, "yfwd%s_%s_P%d", geo, tag, P);
        ProfScope ps(nm_, np, s);
        k_ypass<T, P, TX, false, DBL><<<dim3(P / TX, Gm::NIN, np), NT, sm_yz, s>>>(a);
    }
    {
        snprintf(nm_, sizeof nm_, "zseam%s_%s_P%d", geo, tag, P);
        ProfScope ps(nm_, np, s);
        k_zseam<T, P, TX, DBL><<<dim3(P / TX, P, np), NT, sm_yz, s>>>(a);
    }
    {
        snprintf(nm_, sizeof nm_, "yinv%s_%s_P%d", geo, tag, P);
        ProfScope ps(nm_, np, s);
        k_ypass<T, P, TX, true, DBL><<<dim3(P / TX, Gm::NOUT, np), NT, sm_yz, s>>>(a);
    }
    {
        snprintf(nm_, sizeof nm_, "xinv%s_%s_P%d", geo, tag, P);
        ProfScope ps(nm_, np, s);
        k_xinv<T, P, DBL><<<dim3((rows_out + LINES - 1) / LINES, np), 256, sm_x, s>>>(a);
    }
    count_launches(5);
    return cudaGetLastError();
}

template <typename T, bool DBL>
static cudaError_t conv_dispatch(const ConvArgs<T>& a, int np, int P, cudaStream_t s) {
    switch (P) {
        case 8: if constexpr (!DBL) return conv_passes<T, 8, DBL>(a, np, s); break;
        case 16: return conv_passes<T, 16, DBL>(a, np, s);
        case 32: return conv_passes<T, 32, DBL>(a, np, s);
        case 64: return conv_passes<T, 64, DBL>(a, np, s);
        case 128: return conv_passes<T, 128, DBL>(a, np, s);
        case 256: return conv_passes<T, 256, DBL>(a, np, s);
        case 512: return conv_passes<T, 512, DBL>(a, np, s);
        case 1024: if constexpr (DBL) return conv_passes<T, 1024, DBL>(a, np, s); break;
        default: break;
    }
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t run_conv_t(const PairDesc<T>* pairs, int npairs, int P, bool dbl,
                              const T* spec, const cpx<T>* tw, cudaStream_t s) {
    ConvArgs<T> a;
    a.spec = spec;
    a.tw = tw;
    for (int i0 = 0; i0 < npairs; i0 += kMaxPairs) {
        const int np = npairs - i0 < kMaxPairs ? npairs - i0 : kMaxPairs;
        for (int i = 0; i < np; ++i) a.pair[i] = pairs[i0 + i];
        cudaError_t e = dbl ? conv_dispatch<T, true>(a, np, P, s)
                            : conv_dispatch<T, false>(a, np, P, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace nm
