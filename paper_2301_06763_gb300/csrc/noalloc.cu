// noalloc.cu -- nm_potential_noalloc: a nested-mesh solve that allocates nothing.
//
// Some callers cannot call cudaMalloc while they run: a hydrodynamics code that
// sizes its device pools at start-up and forbids later allocations, a process
// whose device memory is owned by another framework's allocator, or a loop for
// which cudaMalloc's implicit device-wide synchronisation would stall other
// streams.  For them this entry point runs the same original-method solve as
// nm_potential (restriction, per-level convolutions, assembly) with all of its
// scratch -- spectrum, tables, restricted densities, the convolution work
// buffer, level potentials and hole crops -- carved from one file-scope device
// array of NM_NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library holds
// that array until the process exits.
//
// The device address of the array is looked up once per device, with that
// device current, on the first call made on it (cudaGetSymbolAddress); host
// code must not use the array's name as a device pointer.  Make that first call
// before any stream capture.  All calls share the one array and it keeps the
// previous call's contents; every region of it is written before it is read
// within a call, so nothing needs clearing, but calls whose work overlaps on
// the GPU (different streams, different host threads) race on it.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/nm.h"
#include "internal.h"

namespace nm {
nm_status record_error(nm_status st, const char* msg);
}

using namespace nm;

namespace {

constexpr size_t kScratchBytes = (size_t)NM_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Layout {
    size_t oct64, oct32, gscr, ctab, tw64, tw32, restr, work, lvl, crop, carry, total;
};

Layout carve(int L, int N, bool fp32, bool diag) {
    const size_t es = fp32 ? 4 : 8, cs = 2 * es, P = 2 * (size_t)N;
    const size_t H3 = (size_t)(N + 1) * (N + 1) * (N + 1);
    const size_t N3 = (size_t)N * N * N, h3 = N3 / 8, nc = N / 2 + 2;
    Layout l{};
    size_t o = 0;
    l.oct64 = o; o += up256(H3 * 8);
    l.oct32 = o; o += up256(H3 * 4);
    l.gscr = o;  o += up256(2 * H3 * 8);
    l.ctab = o;  o += up256(P * 8);
    l.tw64 = o;  o += up256(P * 16);
    l.tw32 = o;  o += up256(P * 8);
    l.restr = o; o += up256((size_t)(L - 1) * h3 * es);
    l.work = o;  o += up256((P / 2) * P * P * cs);
    l.lvl = o;   o += up256((size_t)L * N3 * es);
    l.crop = o;  o += up256((size_t)(L - 1) * nc * nc * nc * es);
    l.carry = o; o += diag && L > 2 ? up256((size_t)(L - 2) * nc * nc * nc * es) : 0;
    l.total = o;
    return l;
}

// cos(2 pi t / P) for the spectrum and exp(-2 pi i t / P) for the transforms
__global__ void k_noalloc_tables(double* ctab, cpx<double>* tw64, cpx<float>* tw32, int P) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < P; t += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)t / (double)P, &s, &c);
        ctab[t] = c;
        tw64[t] = {c, -s};
        tw32[t] = {(float)c, (float)-s};
    }
}

template <typename T>
cudaError_t solve_static(const nm_options& o, char* base, const Layout& lay, const void* rho,
                         double* phi, cudaStream_t s) {
    const int L = o.levels, N = o.N, P = 2 * N;
    const size_t N3 = (size_t)N * N * N, h3 = N3 / 8;
    const size_t nc = N / 2 + 2, nc3 = nc * nc * nc;
    const size_t H3 = (size_t)(N + 1) * (N + 1) * (N + 1);
    double* ctab = (double*)(base + lay.ctab);
    k_noalloc_tables<<<(P + 127) / 128, 128, 0, s>>>(ctab, (cpx<double>*)(base + lay.tw64),
                                                    (cpx<float>*)(base + lay.tw32), P);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double self_term = 3.0 * std::log(2.0 + std::sqrt(3.0)) - 1.5707963267948966192313216916398;
    e = run_green_octant((double*)(base + lay.oct64), (double*)(base + lay.gscr), ctab, N, self_term, s);
    if (e != cudaSuccess) return e;
    const bool f32 = sizeof(T) == 4;
    if (f32) {
        e = run_to_float((const double*)(base + lay.oct64), (float*)(base + lay.oct32), H3, s);
        if (e != cudaSuccess) return e;
    }
    const T* spec = (const T*)(base + (f32 ? lay.oct32 : lay.oct64));
    const cpx<T>* tw = (const cpx<T>*)(base + (f32 ? lay.tw32 : lay.tw64));
    T* restr = (T*)(base + lay.restr);
    T* lvl = (T*)(base + lay.lvl);
    T* crop = (T*)(base + lay.crop);
    for (int m = L - 2; m >= 0; --m) {
        e = run_restrict<T>((const T*)rho + (size_t)(m + 1) * N3,
                            m + 1 < L - 1 ? restr + (size_t)(m + 1) * h3 : nullptr,
                            restr + (size_t)m * h3, N, s);
        if (e != cudaSuccess) return e;
    }
    for (int m = 0; m < L; ++m) {
        const double dx = o.dx0 / std::ldexp(1.0, m);
        const double scale = dx * dx * (-o.G) / ((double)P * P * P);
        const T* rho_m = (const T*)rho + (size_t)m * N3;
        PairDesc<T> d{};
        d.work = (cpx<T>*)(base + lay.work);
        d.src[0] = SrcField{rho_m, m < L - 1 ? restr + (size_t)m * h3 : nullptr, SRC_FULL, scale};
        d.dst[0] = DstField{lvl + (size_t)m * N3, DST_GRID};
        if (m < L - 1) {
            d.src[1] = SrcField{rho_m, nullptr, SRC_HOLE, scale};
            d.dst[1] = DstField{crop + (size_t)m * nc3, DST_CROP};
        } else {
            d.src[1] = SrcField{nullptr, nullptr, SRC_NONE, 0.0};
            d.dst[1] = DstField{nullptr, DST_NONE};
        }
        if (P >= 16)
            e = f32 ? run_conv_f32_e16((const PairDesc<float>*)(const void*)&d, 1, P, false, 0,
                                       (const float*)(const void*)spec, (const cpx<float>*)(const void*)tw, s)
                    : run_conv_f64_e16((const PairDesc<double>*)(const void*)&d, 1, P, false, 0,
                                       (const double*)(const void*)spec, (const cpx<double>*)(const void*)tw, s);
        else
            e = f32 ? run_conv_f32_e8((const PairDesc<float>*)(const void*)&d, 1, P, false, 0,
                                      (const float*)(const void*)spec, (const cpx<float>*)(const void*)tw, s)
                    : run_conv_f64_e8((const PairDesc<double>*)(const void*)&d, 1, P, false, 0,
                                      (const double*)(const void*)spec, (const cpx<double>*)(const void*)tw, s);
        if (e != cudaSuccess) return e;
    }
    AssembleArgs<T> a{};
    a.phi = phi;
    a.levels = L;
    a.N = N;
    for (int n = 0; n < L; ++n) {
        a.base[n] = lvl + (size_t)n * N3;
        a.dbl[n] = nullptr;
        if (n < L - 1) {
            a.interp[n] = crop + (size_t)n * nc3;
            a.interp_origin[n] = N / 4 - 1;
            a.interp_extent[n] = (int)nc;
        }
    }
    return run_assemble_interp<T>(a, o.interp, (T*)(base + lay.carry), s);
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" nm_status nm_potential_noalloc(const nm_options* opt, const void* rho, double* phi,
                                          void* stream) {
    if (!opt || !rho || !phi) return record_error(NM_EINVAL, "nm_potential_noalloc: null argument");
    const nm_options o = *opt;
    if (o.levels < 1 || o.levels > NM_MAX_LEVELS || o.N < 4 || !pow2(o.N) || !(o.dx0 > 0.0) ||
        !std::isfinite(o.dx0) || !std::isfinite(o.G) ||
        (o.precision != NM_FP64 && o.precision != NM_FP32 && o.precision != NM_FP64X) ||
        (o.interp != NM_INTERP_TRILINEAR && o.interp != NM_INTERP_DIAGONAL))
        return record_error(NM_EINVAL, "nm_potential_noalloc: invalid options");
    if (o.precision == NM_FP64X)
        return record_error(NM_EUNSUPPORTED, "nm_potential_noalloc: NM_FP64X is not built here");
    if (o.method != NM_METHOD_ORIGINAL)
        return record_error(NM_EUNSUPPORTED, "nm_potential_noalloc: only NM_METHOD_ORIGINAL is built here");
    const bool fp32 = o.precision == NM_FP32;
    const Layout lay = carve(o.levels, o.N <= 256 ? o.N : 256, fp32, o.interp == NM_INTERP_DIAGONAL);
    if (o.N > 256 || lay.total > kScratchBytes) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "nm_potential_noalloc: levels=%d N=%d %s needs %zu bytes of scratch, above the "
                 "fixed maximum of %zu bytes (NM_NOALLOC_SCRATCH_BYTES)",
                 o.levels, o.N, fp32 ? "fp32" : "fp64", lay.total, kScratchBytes);
        return record_error(NM_EINVAL, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_error(NM_ECUDA, "nm_potential_noalloc: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return record_error(NM_EUNSUPPORTED, "nm_potential_noalloc: device index");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p)
                return record_error(NM_ECUDA, "nm_potential_noalloc: cudaGetSymbolAddress failed");
            g_addr[dev] = p;
        }
        base = g_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = fp32 ? solve_static<float>(o, (char*)base, lay, rho, phi, s)
             : solve_static<double>(o, (char*)base, lay, rho, phi, s);
    if (e != cudaSuccess) return record_error(NM_ECUDA, cudaGetErrorString(e));
    return NM_OK;
}
