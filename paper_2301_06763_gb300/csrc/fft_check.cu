// fft_check.cu -- the line transform of the five passes (fft.cuh), exposed on
// its own so that a test can compare it with a reference FFT: `lines`
// contiguous lines of P complex values, transformed in place.
#include "../../include/nm.h"
#include "internal.h"

namespace nm {
nm_status record_error(nm_status st, const char* msg);

template <typename T, int P, bool INV>
__global__ void __launch_bounds__(256) k_fft_lines(cpx<T>* data, int lines) {
    constexpr int E = EOf<P>::value, TPL = P / E, LINES = 256 / TPL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* sm_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* sm_lines = sm_tw + P;
    // twiddles exp(-2 pi i t / P) in double, rounded to T, in per-pass order
    fill_pass_twiddles<P, E>(sm_tw, [](int t) {
        double s, c;
        sincospi(2.0 * (double)t / (double)P, &s, &c);
        return cpx<T>{(T)c, (T)-s};
    });
    const int line = threadIdx.x / TPL, j = threadIdx.x % TPL;
    const int l = blockIdx.x * LINES + line;
    const bool valid = l < lines;
    cpx<T>* src = data + (size_t)(valid ? l : 0) * P;
    cpx<T> v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) v[r] = valid ? src[j + r * (P / E)] : cpx<T>{T(0), T(0)};
    __syncthreads();
    fft_line<T, P, E, INV, 0xFFFFu, true, true>(v, j, sm_tw,
                                                LineView<T, 1, true, Log2E<E>::value>{sm_lines + line * (P + P / E)});
    if (valid) {
#pragma unroll
        for (int s = 0; s < E; ++s) src[out_index<P, E>(j, s)] = v[s];
    }
}

template <typename T, int P>
static cudaError_t launch_fft_lines(void* data, int lines, bool inv, cudaStream_t s) {
    constexpr int E = EOf<P>::value, TPL = P / E, LINES = 256 / TPL;
    const size_t smem = (size_t)(P + LINES * (P + P / E)) * sizeof(cpx<T>);
    const int grid = (lines + LINES - 1) / LINES;
    auto k = inv ? k_fft_lines<T, P, true> : k_fft_lines<T, P, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 256, smem, s>>>((cpx<T>*)data, lines);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t fft_lines(int P, void* data, int lines, bool inv, cudaStream_t s) {
    switch (P) {
        case 8: return launch_fft_lines<T, 8>(data, lines, inv, s);
        case 16: return launch_fft_lines<T, 16>(data, lines, inv, s);
        case 32: return launch_fft_lines<T, 32>(data, lines, inv, s);
        case 64: return launch_fft_lines<T, 64>(data, lines, inv, s);
        case 128: return launch_fft_lines<T, 128>(data, lines, inv, s);
        case 256: return launch_fft_lines<T, 256>(data, lines, inv, s);
        case 512: return launch_fft_lines<T, 512>(data, lines, inv, s);
        case 1024: return launch_fft_lines<T, 1024>(data, lines, inv, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace nm

extern "C" nm_status nm_debug_fft(int P, int precision, int inverse, int lines, void* data, void* stream) {
    if (!data || lines < 0 || (precision != NM_FP64 && precision != NM_FP32))
        return nm::record_error(NM_EINVAL, "nm_debug_fft: bad arguments");
    if (P < 8 || P > 1024 || (P & (P - 1)))
        return nm::record_error(NM_EUNSUPPORTED, "nm_debug_fft: P must be a power of two in [8, 1024]");
    if (lines == 0) return NM_OK;
    cudaError_t e = precision == NM_FP32 ? nm::fft_lines<float>(P, data, lines, inverse != 0, (cudaStream_t)stream)
                                         : nm::fft_lines<double>(P, data, lines, inverse != 0, (cudaStream_t)stream);
    if (e != cudaSuccess) return nm::record_error(NM_ECUDA, cudaGetErrorString(e));
    return NM_OK;
}
