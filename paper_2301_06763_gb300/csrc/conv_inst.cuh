// conv_inst.cuh -- host dispatch of the five convolution passes for one real
// type T and one count E of values per thread; included once per (T, E) by
// the conv_*.cu translation units so the variants compile in parallel.
#pragma once
#include <cstdio>
#include <mutex>

#include "fused.cuh"
#include "internal.h"

namespace nm {

template <typename K>
static cudaError_t prep_kernel(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Persistent TMA-fed z-seam over all pairs of the launch (see tma.cuh).
template <typename T, int P, int E, int TX>
static cudaError_t zseam_tma(const ConvArgs<T>& a, int np, cudaStream_t s) {
    constexpr int NT = TX * P / E;
    const size_t c = sizeof(cpx<T>);
    const size_t smem = 2 * (size_t)P * TX * c + (size_t)P * c + 2 * sizeof(uint64_t);
    // shared-memory limit and resident CTAs per SM, once per device
    static PerDevice<KernelPrep> prep;
    const KernelPrep kp = prep.get(current_device(), [&]() {
        KernelPrep r;
        r.err = prep_kernel(k_zseam_tma<T, P, E, TX>, smem);
        if (r.err == cudaSuccess)
            r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.occ, k_zseam_tma<T, P, E, TX>, NT, smem);
        return r;
    }, KernelPrep{cudaErrorInvalidDevice, 0});
    if (kp.err != cudaSuccess) return kp.err;
    const int occ = kp.occ;
    static TmaArgs<T> ta;   // host staging of the (large) parameter block
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    ta.spec = a.spec;
    ta.tw = a.tw;
    ta.npairs = np;
    ta.fault_skip_load = fault_timeout_on() ? 1 : 0;
    ta.timeout = ta.fault_skip_load ? 200000000LL : 4000000000LL;
    ta.status = device_status_word();
    for (int i = 0; i < np; ++i) {
        cudaError_t e = encode_work_map(&ta.map[i], a.pair[i].work, P, sizeof(T) == 8, TX);
        if (e != cudaSuccess) return e;
    }
    const int total = np * P * (P / TX);
    int grid = (occ > 0 ? occ : 1) * sm_count();
    if (grid > total) grid = total;
    k_zseam_tma<T, P, E, TX><<<grid, NT, smem, s>>>(ta);
    return cudaSuccess;
}

// x and y passes fused per slab through a cluster (see fused.cuh); `fwd`
// selects the forward (x then y) or inverse (y then x) kernel.
template <typename T, int P>
static cudaError_t fused_pass(const ConvArgs<T>& a, int np, bool fwd, cudaStream_t s) {
    using F = FusedShape<T, P>;
    static PerDevice<cudaError_t> prep;
    const cudaError_t prepared = prep.get(current_device(), [&]() {
        cudaError_t e = prep_kernel(k_xyfwd<T, T, P>, F::SMEM);
        if (e == cudaSuccess) e = prep_kernel(k_yxinv<T, P>, F::SMEM_INV);
        return e;
    }, cudaErrorInvalidDevice);
    if (prepared != cudaSuccess) return prepared;
    const dim3 grid(F::N * F::C, np);
    if (fwd) k_xyfwd<T, T, P><<<grid, F::NT, F::SMEM, s>>>(a);
    else k_yxinv<T, P><<<grid, F::NT, F::SMEM_INV, s>>>(a);
    return cudaGetLastError();
}

// W = requested column-tile width of the strided passes.
template <typename T, int P, int E, int W, int GM>
static cudaError_t conv_passes(const ConvArgs<T>& a, int np, int flags, cudaStream_t s) {
    const bool tma = (flags & CONV_TMA) != 0;
    if constexpr (GM == 0 && E == 16 && !is_df<T>::value && FusedShape<T, P>::OK) {
        if (flags & CONV_FUSED) {
            constexpr int TX = Tile<P, E, W>::TX;
            const char* tag = sizeof(T) == 4 ? "f32" : "f64";
            char nm_[48];
            cudaError_t e;
            {
                snprintf(nm_, sizeof nm_, "xyfwd_%s_P%d", tag, P);
                ProfScope ps(nm_, np, s);
                if ((e = fused_pass<T, P>(a, np, true, s)) != cudaSuccess) return e;
            }
            {
                snprintf(nm_, sizeof nm_, "zseam_%s_P%d", tag, P);
                ProfScope ps(nm_, np, s);
                if (tma) {
                    if ((e = zseam_tma<T, P, E, TX>(a, np, s)) != cudaSuccess) return e;
                } else {
                    constexpr int NT = TX * P / E;
                    const size_t sm_yz = (size_t)P * sizeof(cpx<T>) + (size_t)TX * P * sizeof(cpx<T>);
                    static PerDevice<cudaError_t> prep;
                    const cudaError_t pe = prep.get(current_device(), [&]() {
                        return prep_kernel(k_zseam<T, P, E, TX, false>, sm_yz);
                    }, cudaErrorInvalidDevice);
                    if (pe != cudaSuccess) return pe;
                    k_zseam<T, P, E, TX, false><<<dim3(P / TX, P, np), NT, sm_yz, s>>>(a);
                }
            }
            {
                snprintf(nm_, sizeof nm_, "yxinv_%s_P%d", tag, P);
                ProfScope ps(nm_, np, s);
                if ((e = fused_pass<T, P>(a, np, false, s)) != cudaSuccess) return e;
            }
            count_launches(3);
            return cudaGetLastError();
        }
    }
    using Gm = Geo<P, E, GM>;
    using TIN = typename InOf<T>::type;
    constexpr int TPL = P / E;
    constexpr int LINES = 256 / TPL;
    constexpr int TX = Tile<P, E, W>::TX;
    constexpr int NT = TX * P / E;   // threads of the strided passes
    const size_t c = sizeof(cpx<T>);
    const size_t sm_x = (size_t)P * c + (size_t)LINES * (P + P / E) * c;
    const size_t sm_yz = (size_t)P * c + (size_t)TX * P * c;
    // shared-memory limits are set once per kernel and device
    static PerDevice<cudaError_t> prep;
    const cudaError_t prepared = prep.get(current_device(), [&]() {
        cudaError_t e;
        if ((e = prep_kernel(k_xfwd<T, TIN, P, E, GM>, sm_x)) != cudaSuccess) return e;
        if ((e = prep_kernel(k_ypass<T, P, E, TX, false, GM>, sm_yz)) != cudaSuccess) return e;
        if ((e = prep_kernel(k_zseam<T, P, E, TX, GM>, sm_yz)) != cudaSuccess) return e;
        if ((e = prep_kernel(k_ypass<T, P, E, TX, true, GM>, sm_yz)) != cudaSuccess) return e;
        return prep_kernel(k_xinv<T, P, E, GM>, sm_x);
    }, cudaErrorInvalidDevice);
    if (prepared != cudaSuccess) return prepared;
    const int rows_in = Gm::NIN * Gm::NIN;
    const int rows_out = Gm::NOUT * Gm::NOUT;
    char nm_[48];
    const char* tag = sizeof(T) == 4 ? "f32" : "f64";
    const char* geo = GM == 1 ? "_dbl" : GM == 2 ? "_qdp" : "";
    {
        snprintf(nm_, sizeof nm_, "xfwd%s_%s_P%d", geo, tag, P);
        ProfScope ps(nm_, np, s);
        bool pipe = false;
        if constexpr (GM == 0 && P >= 64 && E == 16) {
            // every pair a level's full field with its hole field (or alone),
            // on a 16-byte aligned density
            pipe = true;
            for (int i = 0; i < np && pipe; ++i) {
                const PairDesc<T>& d = a.pair[i];
                pipe = d.src[0].mode == SRC_FULL && ((uintptr_t)d.src[0].rho & 15) == 0 &&
                       (!d.src[0].restr || ((uintptr_t)d.src[0].restr & 7) == 0) &&
                       (d.src[1].mode == SRC_NONE || (d.src[1].mode == SRC_HOLE && d.src[1].rho == d.src[0].rho));
            }
            if (pipe && P >= 256 && sizeof(T) == 4 && !is_df<T>::value && (flags & (CONV_PAIRED | CONV_SSPEC))) {
                // FP32 with P >= 256: the x-forward takes two rows per thread
                // (measured 3-9% faster there, 7% slower at P = 128)
                if constexpr (P >= 256 && sizeof(T) == 4 && !is_df<T>::value) {
                    cudaError_t e = run_xfwd_paired_f32(a, np, P, s);
                    if (e != cudaSuccess) return e;
                }
            } else if (pipe) {
                const size_t sm_p = sm_x + 2 * (size_t)XfwdStage<TIN, P, E>::ELEMS * sizeof(TIN);
                static PerDevice<KernelPrep> prep_p;
                const KernelPrep kp = prep_p.get(current_device(), [&]() {
                    KernelPrep r;
                    r.err = prep_kernel(k_xfwd_pipe<T, TIN, P, E>, sm_p);
                    if (r.err == cudaSuccess)
                        r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.occ, k_xfwd_pipe<T, TIN, P, E>, 256,
                                                                              sm_p);
                    return r;
                }, KernelPrep{cudaErrorInvalidDevice, 0});
                if (kp.err != cudaSuccess) return kp.err;
                const int occ = kp.occ;
                const int tiles = np * (rows_in / LINES);
                int grid = (occ > 0 ? occ : 1) * sm_count();
                if (grid > tiles) grid = tiles;
                k_xfwd_pipe<T, TIN, P, E><<<grid, 256, sm_p, s>>>(a, np);
            }
        }
        if (!pipe) k_xfwd<T, TIN, P, E, GM><<<dim3((rows_in + LINES - 1) / LINES, np), 256, sm_x, s>>>(a);
    }
    {
        snprintf(nm_, sizeof nm_, "yfwd%s_%s_P%d", geo, tag, P);
        ProfScope ps(nm_, np, s);
        k_ypass<T, P, E, TX, false, GM><<<dim3(P / TX, Gm::NIN, np), NT, sm_yz, s>>>(a);
    }
    {
        snprintf(nm_, sizeof nm_, "zseam%s_%s_P%d", geo, tag, P);
        ProfScope ps(nm_, np, s);
        bool done = false;
        if constexpr (GM == 0 && E == 16 && P >= 64 && sizeof(T) == 4 && !is_df<T>::value) {
            if ((flags & CONV_ZPERSIST) && P == 256 && TX == 16) {
                cudaError_t e = run_zseam_persist_f32(a, np, P, s);
                if (e != cudaSuccess) return e;
                done = true;
            } else if (flags & CONV_PAIRED) {
                cudaError_t e = run_zseam_paired_f32(a, np, P, TX, s);
                if (e != cudaSuccess) return e;
                done = true;
            } else if ((flags & CONV_SSPEC) && !tma) {
                cudaError_t e = run_zseam_staged_f32(a, np, P, TX, s);
                if (e != cudaSuccess) return e;
                done = true;
            }
        }
        if constexpr (GM == 0 && !is_df<T>::value) {
            if (!done && tma) {
                cudaError_t e = zseam_tma<T, P, E, TX>(a, np, s);
                if (e != cudaSuccess) return e;
                done = true;
            }
        }
        if (!done) k_zseam<T, P, E, TX, GM><<<dim3(P / TX, P, np), NT, sm_yz, s>>>(a);
    }
    {
        snprintf(nm_, sizeof nm_, "yinv%s_%s_P%d", geo, tag, P);
        ProfScope ps(nm_, np, s);
        k_ypass<T, P, E, TX, true, GM><<<dim3(P / TX, Gm::NOUT, np), NT, sm_yz, s>>>(a);
    }
    {
        snprintf(nm_, sizeof nm_, "xinv%s_%s_P%d", geo, tag, P);
        ProfScope ps(nm_, np, s);
        k_xinv<T, P, E, GM><<<dim3((rows_out + LINES - 1) / LINES, np), 256, sm_x, s>>>(a);
    }
    count_launches(5);
    return cudaGetLastError();
}

// Narrow / wide column tiles: 128- and 256-byte rows for float, 128 and 256
// for double.
template <typename T> struct Widths {
    static constexpr int NARROW = sizeof(T) == 4 ? 16 : 8;
    static constexpr int WIDE = 2 * NARROW;
};

template <typename T, int P, int E, int GM>
static cudaError_t conv_width(const ConvArgs<T>& a, int np, int flags, cudaStream_t s) {
    if (flags & CONV_WIDE) return conv_passes<T, P, E, Widths<T>::WIDE, GM>(a, np, flags, s);
    return conv_passes<T, P, E, Widths<T>::NARROW, GM>(a, np, flags, s);
}

// The doubled-grid geometry is instantiated only with the default schedule
// (E = 16, narrow tiles) to bound compile time.
template <typename T, int E>
static cudaError_t conv_dispatch(const ConvArgs<T>& a, int np, int P, bool dbl, int flags,
                                 cudaStream_t s) {
    if (dbl) {
        if constexpr (E == 16 && !is_df<T>::value) {
            switch (P) {
                case 16: return conv_passes<T, 16, 16, Widths<T>::NARROW, 1>(a, np, 0, s);
                case 32: return conv_passes<T, 32, 16, Widths<T>::NARROW, 1>(a, np, 0, s);
                case 64: return conv_passes<T, 64, 16, Widths<T>::NARROW, 1>(a, np, 0, s);
                case 128: return conv_passes<T, 128, 16, Widths<T>::NARROW, 1>(a, np, 0, s);
                case 256: return conv_passes<T, 256, 16, Widths<T>::NARROW, 1>(a, np, 0, s);
                case 512: return conv_passes<T, 512, 16, Widths<T>::NARROW, 1>(a, np, 0, s);
                case 1024: return conv_passes<T, 1024, 16, Widths<T>::NARROW, 1>(a, np, 0, s);
                default: break;
            }
        }
        return cudaErrorInvalidValue;
    }
    switch (P) {
        case 8: if constexpr (E == 8) return conv_width<T, 8, 8, 0>(a, np, flags, s); break;
        case 16: return conv_width<T, 16, E, 0>(a, np, flags, s);
        case 32: return conv_width<T, 32, E, 0>(a, np, flags, s);
        case 64: return conv_width<T, 64, E, 0>(a, np, flags, s);
        case 128: return conv_width<T, 128, E, 0>(a, np, flags, s);
        case 256: return conv_width<T, 256, E, 0>(a, np, flags, s);
        case 512: return conv_width<T, 512, E, 0>(a, np, flags, s);
        default: break;
    }
    return cudaErrorInvalidValue;
}

// The quadrupled-grid geometry (E = 16, narrow tiles), P = 8N for N = 4 ..
// 128; instantiated only by the translation units that call it.
template <typename T>
static cudaError_t conv_dispatch_qdp(const ConvArgs<T>& a, int np, int P, cudaStream_t s) {
    switch (P) {
        case 32: return conv_passes<T, 32, 16, Widths<T>::NARROW, 2>(a, np, 0, s);
        case 64: return conv_passes<T, 64, 16, Widths<T>::NARROW, 2>(a, np, 0, s);
        case 128: return conv_passes<T, 128, 16, Widths<T>::NARROW, 2>(a, np, 0, s);
        case 256: return conv_passes<T, 256, 16, Widths<T>::NARROW, 2>(a, np, 0, s);
        case 512: return conv_passes<T, 512, 16, Widths<T>::NARROW, 2>(a, np, 0, s);
        case 1024: return conv_passes<T, 1024, 16, Widths<T>::NARROW, 2>(a, np, 0, s);
        default: break;
    }
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t run_conv_qdp_variant(const PairDesc<T>* pairs, int npairs, int P, const T* spec,
                                        const cpx<T>* tw, cudaStream_t s) {
    ConvArgs<T> a;
    a.spec = spec;
    a.tw = tw;
    for (int i0 = 0; i0 < npairs; i0 += kMaxPairs) {
        const int np = npairs - i0 < kMaxPairs ? npairs - i0 : kMaxPairs;
        for (int i = 0; i < np; ++i) a.pair[i] = pairs[i0 + i];
        cudaError_t e = conv_dispatch_qdp<T>(a, np, P, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T, int E>
static cudaError_t run_conv_variant(const PairDesc<T>* pairs, int npairs, int P, bool dbl,
                                    int flags, const T* spec, const cpx<T>* tw, cudaStream_t s) {
    ConvArgs<T> a;
    a.spec = spec;
    a.tw = tw;
    // real pairs (one field, second slot empty) take the half-spectrum path
    // on level grids with the separate y and z passes
    const bool halves = !dbl && !(flags & (CONV_TMA | CONV_FUSED));
    for (int i0 = 0; i0 < npairs; i0 += kMaxPairs) {
        const int np = npairs - i0 < kMaxPairs ? npairs - i0 : kMaxPairs;
        for (int i = 0; i < np; ++i) {
            a.pair[i] = pairs[i0 + i];
            a.pair[i].half = (halves && a.pair[i].src[0].mode != SRC_NONE && a.pair[i].src[1].mode == SRC_NONE) ? 1 : 0;
        }
        cudaError_t e = conv_dispatch<T, E>(a, np, P, dbl, flags, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace nm
