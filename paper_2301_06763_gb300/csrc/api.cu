// api.cu -- the C ABI of include/nm.h: plans, caches of spectra and twiddles,
// and the launch schedule of one nested-mesh solve.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/nm.h"
#include "internal.h"

namespace nm {

static std::atomic<uint64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

static thread_local std::string t_last_error;

// ------------------------------------------------------------------ profiling
struct ProfRecord {
    std::string name;
    int units;
    cudaEvent_t a, b;
};
static std::atomic<bool> g_prof_on{false};
static std::mutex g_prof_mu;
static std::vector<ProfRecord> g_prof;

ProfScope::ProfScope(const char* name, int units, cudaStream_t stream) : s(stream) {
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    ProfRecord r{name, units, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess) return;
    if (cudaEventCreate(&r.b) != cudaSuccess) { cudaEventDestroy(r.a); return; }
    cudaEventRecord(r.a, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    idx = (int)g_prof.size();
    g_prof.push_back(r);
}
ProfScope::~ProfScope() {
    if (idx < 0) return;
    cudaEvent_t b;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (idx >= (int)g_prof.size()) return;
        b = g_prof[idx].b;
    }
    cudaEventRecord(b, s);
}

static void prof_clear() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g_prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_prof.clear();
}

static nm_status fail(nm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return st;
}

// Sets the calling thread's nm_last_error message from another translation unit.
nm_status record_error(nm_status st, const char* msg) { return fail(st, "%s", msg); }

static nm_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? NM_ENOMEM : NM_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorName(e), cudaGetErrorString(e));
}

#define NM_CUDA(call, what)                               \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ------------------------------------------------------------------ caches
// Unit-cell spectrum octants are shared by every plan with the same N on the
// same device; twiddle tables by every transform of the same size.
struct Spectrum {
    int dev = -1, N = 0, refs = 0;
    bool ready = false;
    double* d64 = nullptr;
    float* d32 = nullptr;
};
struct Twiddle {
    int dev = -1, P = 0;
    cpx<double>* d64 = nullptr;
    cpx<float>* d32 = nullptr;
};

static std::mutex g_cache_mu;
static std::vector<Spectrum*> g_spectra;
static std::vector<Twiddle*> g_twiddles;

static size_t octant_count(int N) { return (size_t)(N + 1) * (N + 1) * (N + 1); }

static nm_status get_twiddle(int dev, int P, Twiddle** out) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (Twiddle* t : g_twiddles)
        if (t->dev == dev && t->P == P) { *out = t; return NM_OK; }
    std::vector<cpx<double>> h64(P);
    std::vector<cpx<float>> h32(P);
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < P; ++t) {
        const double a = two_pi * (double)t / (double)P;
        h64[t] = {std::cos(a), -std::sin(a)};
        h32[t] = {(float)h64[t].re, (float)h64[t].im};
    }
    Twiddle* tw = new Twiddle();
    tw->dev = dev;
    tw->P = P;
    cudaError_t e = cudaMalloc(&tw->d64, sizeof(cpx<double>) * P);
    if (e == cudaSuccess) e = cudaMalloc(&tw->d32, sizeof(cpx<float>) * P);
    if (e == cudaSuccess) e = cudaMemcpy(tw->d64, h64.data(), sizeof(cpx<double>) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(tw->d32, h32.data(), sizeof(cpx<float>) * P, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(tw->d64);
        cudaFree(tw->d32);
        delete tw;
        return cuda_fail(e, "twiddle table");
    }
    g_twiddles.push_back(tw);
    *out = tw;
    return NM_OK;
}

static nm_status acquire_spectrum(int dev, int N, Spectrum** out) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (Spectrum* s : g_spectra)
        if (s->dev == dev && s->N == N) { s->refs++; *out = s; return NM_OK; }
    Spectrum* s = new Spectrum();
    s->dev = dev;
    s->N = N;
    s->refs = 1;
    g_spectra.push_back(s);
    *out = s;
    return NM_OK;
}

static void release_spectrum(Spectrum* s) {
    if (!s) return;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (--s->refs > 0) return;
    cudaFree(s->d64);
    cudaFree(s->d32);
    for (size_t i = 0; i < g_spectra.size(); ++i)
        if (g_spectra[i] == s) { g_spectra.erase(g_spectra.begin() + i); break; }
    delete s;
}

// Build the octant (double) and its float copy; synchronous on `stream`, so a
// spectrum is complete before any plan on any stream uses it.
static nm_status build_spectrum(Spectrum* s, cudaStream_t stream) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (s->ready) return NM_OK;
    const int N = s->N, P = 2 * N;
    const size_t n = octant_count(N);
    std::vector<double> ctab(P);
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < P; ++t) ctab[t] = std::cos(two_pi * (double)t / (double)P);
    // Eq. 13 self term for a unit cube: 3 ln(2 + sqrt 3) - pi/2
    const double self_term = 3.0 * std::log(2.0 + std::sqrt(3.0)) - 1.5707963267948966192313216916398;
    double* d_ctab = nullptr;
    double* scratch = nullptr;
    cudaError_t e = cudaSuccess;
    if (!s->d64) e = cudaMalloc(&s->d64, n * sizeof(double));
    if (e == cudaSuccess && !s->d32) e = cudaMalloc(&s->d32, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d_ctab, P * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&scratch, 2 * n * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ctab, ctab.data(), P * sizeof(double), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = run_green_octant(s->d64, scratch, d_ctab, N, self_term, stream);
    if (e == cudaSuccess) e = run_to_float(s->d64, s->d32, n, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFree(d_ctab);
    cudaFree(scratch);
    if (e != cudaSuccess) return cuda_fail(e, "green spectrum");
    s->ready = true;
    return NM_OK;
}

}  // namespace nm

using namespace nm;

// ------------------------------------------------------------------ plan
struct nm_plan_s {
    nm_options opt;
    int dev = 0;
    int N = 0, L = 0, P = 0;
    bool fp32 = false, dipole = false;
    size_t es = 8, cs = 16;           // bytes per real / complex value
    int group = 1, group_dbl = 1;     // pairs in flight per launch
    int npairs = 0, npairs_dbl = 0;
    void* restr = nullptr;            // (L-1) * (N/2)^3 restricted densities
    void* work = nullptr;             // group * (P/2) * P^2 complex
    void* lvl = nullptr;              // L * N^3 level potentials
    void* crop = nullptr;             // (L-1) * (N/2+2)^3 hole crops (original method)
    void* dbl_work = nullptr;         // group_dbl * (2N) * (4N)^2 complex (dipole)
    void* dbl_out = nullptr;          // (L-1) * (2N)^3 (dipole)
    void* h_rho = nullptr;            // staging for nm_potential_host
    double* h_phi = nullptr;
    size_t ws_bytes = 0;
    Spectrum* spec = nullptr;
    Spectrum* spec_dbl = nullptr;
    Twiddle* tw = nullptr;
    Twiddle* tw_dbl = nullptr;
};

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

static int env_int(const char* name, int dflt) {
    const char* v = std::getenv(name);
    if (!v || !*v) return dflt;
    return std::atoi(v);
}

static void plan_free_buffers(nm_plan_t p) {
    cudaFree(p->restr);
    cudaFree(p->work);
    cudaFree(p->lvl);
    cudaFree(p->crop);
    cudaFree(p->dbl_work);
    cudaFree(p->dbl_out);
    cudaFree(p->h_rho);
    cudaFree(p->h_phi);
    p->restr = p->work = p->lvl = p->crop = p->dbl_work = p->dbl_out = p->h_rho = nullptr;
    p->h_phi = nullptr;
}

// Pairs in flight per launch: all of them while one pair's work buffer is
// small, one at a time once a buffer is large enough that keeping it resident
// in L2 between passes matters more than filling the GPU with several.
static int default_group(size_t buf_bytes, int npairs) {
    int g = env_int("NM_GROUP", 0);
    if (g <= 0) {
        const size_t budget = (size_t)64 << 20;
        g = buf_bytes >= budget ? 1 : (int)(budget / buf_bytes);
    }
    if (g > npairs) g = npairs;
    if (g < 1) g = 1;
    return g;
}

extern "C" {

nm_status nm_default_options(int levels, int N, double dx0, nm_options* opt) {
    if (!opt) return fail(NM_EINVAL, "nm_default_options: null options");
    opt->levels = levels;
    opt->N = N;
    opt->dx0 = dx0;
    opt->G = 1.0;
    opt->precision = NM_FP64;
    opt->method = NM_METHOD_ORIGINAL;
    opt->interp = NM_INTERP_TRILINEAR;
    return NM_OK;
}

nm_status nm_plan_ex(const nm_options* opt, nm_plan_t* out) {
    if (!opt || !out) return fail(NM_EINVAL, "nm_plan_ex: null argument");
    *out = nullptr;
    const nm_options o = *opt;
    if (o.levels < 1 || o.levels > NM_MAX_LEVELS)
        return fail(NM_EINVAL, "levels must be in [1, %d], got %d", NM_MAX_LEVELS, o.levels);
    if (o.N < 4 || o.N % 4 != 0)
        return fail(NM_EINVAL, "N must be a multiple of 4 (level m+1 covers [N/4, 3N/4)), got %d", o.N);
    if (!is_pow2(o.N) || o.N > 256)
        return fail(NM_EUNSUPPORTED, "N must be a power of two in [4, 256], got %d", o.N);
    if (!(o.dx0 > 0.0) || !std::isfinite(o.dx0)) return fail(NM_EINVAL, "dx0 must be finite and > 0");
    if (!std::isfinite(o.G)) return fail(NM_EINVAL, "G must be finite");
    if (o.precision != NM_FP64 && o.precision != NM_FP32) return fail(NM_EINVAL, "bad precision %d", o.precision);
    if (o.method != NM_METHOD_ORIGINAL && o.method != NM_METHOD_DIPOLE_PAIR)
        return fail(NM_EINVAL, "bad method %d", o.method);
    if (o.interp != NM_INTERP_TRILINEAR) return fail(NM_EUNSUPPORTED, "only trilinear interpolation is built");

    nm_plan_t p = new (std::nothrow) nm_plan_s();
    if (!p) return fail(NM_ENOMEM, "host allocation");
    p->opt = o;
    NM_CUDA(cudaGetDevice(&p->dev), "cudaGetDevice");
    p->N = o.N;
    p->L = o.levels;
    p->P = 2 * o.N;
    p->fp32 = o.precision == NM_FP32;
    p->dipole = o.method == NM_METHOD_DIPOLE_PAIR;
    p->es = p->fp32 ? 4 : 8;
    p->cs = 2 * p->es;
    const size_t N = o.N, L = o.levels, P = p->P;
    const size_t N3 = N * N * N, h3 = (N / 2) * (N / 2) * (N / 2);
    const size_t nc = N / 2 + 2, nc3 = nc * nc * nc;
    p->npairs = p->dipole ? (int)((L + 1) / 2) : (int)L;
    p->npairs_dbl = p->dipole ? (int)(L / 2) : 0;   // ceil((L-1)/2)
    const size_t buf = (P / 2) * P * P * p->cs;
    p->group = default_group(buf, p->npairs);
    const size_t buf_dbl = (2 * N) * (4 * N) * (4 * N) * p->cs;
    if (p->dipole) p->group_dbl = default_group(buf_dbl, p->npairs_dbl);

    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (e != cudaSuccess || bytes == 0) return;
        e = cudaMalloc(ptr, bytes);
        if (e == cudaSuccess) p->ws_bytes += bytes;
    };
    alloc(&p->restr, (L - 1) * h3 * p->es);
    alloc(&p->work, (size_t)p->group * buf);
    alloc(&p->lvl, L * N3 * p->es);
    if (!p->dipole) alloc(&p->crop, (L - 1) * nc3 * p->es);
    if (p->dipole && L > 1) {
        alloc(&p->dbl_work, (size_t)p->group_dbl * buf_dbl);
        alloc(&p->dbl_out, (L - 1) * 8 * N3 * p->es);
    }
    if (e != cudaSuccess) {
        plan_free_buffers(p);
        delete p;
        return cuda_fail(e, "plan workspace");
    }
    nm_status st = get_twiddle(p->dev, p->P, &p->tw);
    if (st == NM_OK && p->dipole && L > 1) st = get_twiddle(p->dev, 2 * p->P, &p->tw_dbl);
    if (st == NM_OK) st = acquire_spectrum(p->dev, o.N, &p->spec);
    if (st == NM_OK && p->dipole && L > 1) st = acquire_spectrum(p->dev, 2 * o.N, &p->spec_dbl);
    if (st != NM_OK) {
        release_spectrum(p->spec);
        release_spectrum(p->spec_dbl);
        plan_free_buffers(p);
        delete p;
        return st;
    }
    *out = p;
    return NM_OK;
}

nm_status nm_plan(int levels, int N, double dx0, nm_plan_t* out) {
    nm_options o;
    nm_default_options(levels, N, dx0, &o);
    return nm_plan_ex(&o, out);
}

nm_status nm_green(nm_plan_t p, void* stream) {
    if (!p) return fail(NM_EINVAL, "nm_green: null plan");
    nm_status st = build_spectrum(p->spec, (cudaStream_t)stream);
    if (st == NM_OK && p->spec_dbl) st = build_spectrum(p->spec_dbl, (cudaStream_t)stream);
    return st;
}

}  // extern "C"

// ------------------------------------------------------------------ the solve
namespace {

// Effective density fields of level m (see conv.cuh SrcField).
SrcField field(nm_plan_t p, const void* rho, int m, int mode, int P) {
    const size_t N3 = (size_t)p->N * p->N * p->N;
    const size_t h3 = N3 / 8;
    SrcField f;
    f.rho = (const char*)rho + (size_t)m * N3 * p->es;
    f.restr = (mode == SRC_FULL && m < p->L - 1) ? (const char*)p->restr + (size_t)m * h3 * p->es : nullptr;
    f.mode = mode;
    const double dx = p->opt.dx0 / std::ldexp(1.0, m);
    // density -> scaled mass: M = rho dx^3, calG = g / dx, and the inverse
    // transform's 1/P^3, so the spectrum multiply needs no per-level factor
    f.scale = dx * dx * (-p->opt.G) / ((double)P * P * P);
    return f;
}

template <typename T>
nm_status solve_t(nm_plan_t p, const void* rho, double* phi, cudaStream_t s,
                  cudaError_t (*run_conv)(const PairDesc<T>*, int, int, bool, const T*,
                                          const cpx<T>*, cudaStream_t)) {
    const int L = p->L, N = p->N, P = p->P;
    const size_t N3 = (size_t)N * N * N, h3 = N3 / 8;
    const size_t nc = N / 2 + 2, nc3 = nc * nc * nc;
    const T* spec = p->fp32 ? (const T*)(void*)p->spec->d32 : (const T*)(void*)p->spec->d64;
    const cpx<T>* tw = p->fp32 ? (const cpx<T>*)(void*)p->tw->d32 : (const cpx<T>*)(void*)p->tw->d64;
    T* lvl = (T*)p->lvl;
    cudaError_t e;
    // 1. restriction, finest -> coarsest
    for (int m = L - 2; m >= 0; --m) {
        const T* child = (const T*)rho + (size_t)(m + 1) * N3;
        const T* rchild = (m + 1 < L - 1) ? (const T*)p->restr + (size_t)(m + 1) * h3 : nullptr;
        e = run_restrict<T>(child, rchild, (T*)p->restr + (size_t)m * h3, N, s);
        if (e != cudaSuccess) return cuda_fail(e, "restriction");
    }
    // 2. level convolutions
    std::vector<PairDesc<T>> pairs;
    if (!p->dipole) {
        for (int m = 0; m < L; ++m) {
            PairDesc<T> d{};
            d.src[0] = field(p, rho, m, SRC_FULL, P);
            d.dst[0] = {lvl + (size_t)m * N3, DST_GRID};
            if (m < L - 1) {
                d.src[1] = field(p, rho, m, SRC_HOLE, P);
                d.dst[1] = {(T*)p->crop + (size_t)m * nc3, DST_CROP};
            } else {
                d.src[1] = SrcField{nullptr, nullptr, SRC_NONE, 0.0};
                d.dst[1] = {nullptr, DST_NONE};
            }
            pairs.push_back(d);
        }
    } else {
        for (int m = 0; m < L; m += 2) {
            PairDesc<T> d{};
            for (int h = 0; h < 2; ++h) {
                const int lv = m + h;
                if (lv < L) {
                    d.src[h] = field(p, rho, lv, lv < L - 1 ? SRC_HOLE : SRC_FULL, P);
                    d.dst[h] = {lvl + (size_t)lv * N3, DST_GRID};
                } else {
                    d.src[h] = SrcField{nullptr, nullptr, SRC_NONE, 0.0};
                    d.dst[h] = {nullptr, DST_NONE};
                }
            }
            pairs.push_back(d);
        }
    }
    const size_t buf = (size_t)(P / 2) * P * P;
    for (size_t g0 = 0; g0 < pairs.size(); g0 += p->group) {
        const int np = (int)std::min(pairs.size() - g0, (size_t)p->group);
        for (int i = 0; i < np; ++i) pairs[g0 + i].work = (cpx<T>*)p->work + (size_t)i * buf;
        e = run_conv(&pairs[g0], np, P, false, spec, tw, s);
        if (e != cudaSuccess) return cuda_fail(e, "level convolution");
    }
    // 3. doubled fine grids (pairwise dipole method)
    if (p->dipole && L > 1) {
        const int P2 = 2 * P;
        const T* spec2 = p->fp32 ? (const T*)(void*)p->spec_dbl->d32 : (const T*)(void*)p->spec_dbl->d64;
        const cpx<T>* tw2 = p->fp32 ? (const cpx<T>*)(void*)p->tw_dbl->d32 : (const cpx<T>*)(void*)p->tw_dbl->d64;
        std::vector<PairDesc<T>> dp;
        for (int n = 0; n < L - 1; n += 2) {
            PairDesc<T> d{};
            for (int h = 0; h < 2; ++h) {
                const int nn = n + h;
                if (nn < L - 1) {
                    d.src[h] = field(p, rho, nn + 1, SRC_FULL, P2);
                    d.dst[h] = {(T*)p->dbl_out + (size_t)nn * 8 * N3, DST_GRID};
                } else {
                    d.src[h] = SrcField{nullptr, nullptr, SRC_NONE, 0.0};
                    d.dst[h] = {nullptr, DST_NONE};
                }
            }
            dp.push_back(d);
        }
        const size_t buf2 = (size_t)(P2 / 2) * P2 * P2;
        for (size_t g0 = 0; g0 < dp.size(); g0 += p->group_dbl) {
            const int np = (int)std::min(dp.size() - g0, (size_t)p->group_dbl);
            for (int i = 0; i < np; ++i) dp[g0 + i].work = (cpx<T>*)p->dbl_work + (size_t)i * buf2;
            e = run_conv(&dp[g0], np, P2, true, spec2, tw2, s);
            if (e != cudaSuccess) return cuda_fail(e, "doubled-grid convolution");
        }
    }
    // 4. assembly
    AssembleArgs<T> a{};
    a.phi = phi;
    a.levels = L;
    a.N = N;
    for (int n = 0; n < L; ++n) {
        a.base[n] = lvl + (size_t)n * N3;
        a.dbl[n] = (p->dipole && n < L - 1) ? (const T*)p->dbl_out + (size_t)n * 8 * N3 : nullptr;
        if (n < L - 1) {
            if (p->dipole) {
                a.interp[n] = lvl + (size_t)n * N3;
                a.interp_origin[n] = 0;
                a.interp_extent[n] = N;
            } else {
                a.interp[n] = (const T*)p->crop + (size_t)n * nc3;
                a.interp_origin[n] = N / 4 - 1;
                a.interp_extent[n] = (int)nc;
            }
        }
    }
    e = run_assemble<T>(a, s);
    if (e != cudaSuccess) return cuda_fail(e, "assembly");
    return NM_OK;
}

nm_status potential_impl(nm_plan_t p, const void* rho, double* phi, cudaStream_t s) {
    if (!p->spec->ready || (p->spec_dbl && !p->spec_dbl->ready)) {
        nm_status st = nm_green(p, (void*)s);
        if (st != NM_OK) return st;
    }
    if (p->fp32) return solve_t<float>(p, rho, phi, s, run_conv_f32);
    return solve_t<double>(p, rho, phi, s, run_conv_f64);
}

}  // namespace

extern "C" {

nm_status nm_potential(nm_plan_t p, const void* rho, double* phi, void* stream) {
    if (!p || !rho || !phi) return fail(NM_EINVAL, "nm_potential: null argument");
    return potential_impl(p, rho, phi, (cudaStream_t)stream);
}

nm_status nm_potential_host(nm_plan_t p, const void* rho_host, double* phi_host, void* stream) {
    if (!p || !rho_host || !phi_host) return fail(NM_EINVAL, "nm_potential_host: null argument");
    const size_t cells = (size_t)p->L * p->N * p->N * p->N;
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->h_rho) {
        NM_CUDA(cudaMalloc(&p->h_rho, cells * p->es), "host-path staging");
        NM_CUDA(cudaMalloc((void**)&p->h_phi, cells * sizeof(double)), "host-path staging");
        p->ws_bytes += cells * (p->es + sizeof(double));
    }
    NM_CUDA(cudaMemcpyAsync(p->h_rho, rho_host, cells * p->es, cudaMemcpyHostToDevice, s), "rho upload");
    nm_status st = potential_impl(p, p->h_rho, p->h_phi, s);
    if (st != NM_OK) return st;
    NM_CUDA(cudaMemcpyAsync(phi_host, p->h_phi, cells * sizeof(double), cudaMemcpyDeviceToHost, s), "phi download");
    NM_CUDA(cudaStreamSynchronize(s), "nm_potential_host sync");
    return NM_OK;
}

nm_status nm_batch_potential(int n, const nm_plan_t* plans, const void* const* rho,
                             double* const* phi, void* stream) {
    if (n < 0 || (n > 0 && (!plans || !rho || !phi))) return fail(NM_EINVAL, "nm_batch_potential: bad arguments");
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || !rho[i] || !phi[i]) return fail(NM_EINVAL, "nm_batch_potential: null entry %d", i);
        for (int k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return fail(NM_EINVAL, "nm_batch_potential: plan %d repeated", i);
    }
    for (int i = 0; i < n; ++i) {
        nm_status st = potential_impl(plans[i], rho[i], phi[i], (cudaStream_t)stream);
        if (st != NM_OK) return st;
    }
    return NM_OK;
}

nm_status nm_workspace_bytes(nm_plan_t p, size_t* bytes) {
    if (!p || !bytes) return fail(NM_EINVAL, "nm_workspace_bytes: null argument");
    *bytes = p->ws_bytes;
    return NM_OK;
}

nm_status nm_spectrum_bytes(nm_plan_t p, size_t* bytes) {
    if (!p || !bytes) return fail(NM_EINVAL, "nm_spectrum_bytes: null argument");
    size_t b = octant_count(p->N) * (sizeof(double) + sizeof(float));
    if (p->spec_dbl) b += octant_count(2 * p->N) * (sizeof(double) + sizeof(float));
    *bytes = b;
    return NM_OK;
}

nm_status nm_get_green_octant(nm_plan_t p, double* host_out) {
    if (!p || !host_out) return fail(NM_EINVAL, "nm_get_green_octant: null argument");
    if (!p->spec->ready) {
        nm_status st = nm_green(p, nullptr);
        if (st != NM_OK) return st;
    }
    NM_CUDA(cudaMemcpy(host_out, p->spec->d64, octant_count(p->N) * sizeof(double), cudaMemcpyDeviceToHost),
            "spectrum download");
    return NM_OK;
}

nm_status nm_get_options(nm_plan_t p, nm_options* out) {
    if (!p || !out) return fail(NM_EINVAL, "nm_get_options: null argument");
    *out = p->opt;
    return NM_OK;
}

nm_status nm_destroy(nm_plan_t p) {
    if (!p) return fail(NM_EINVAL, "nm_destroy: null plan");
    cudaError_t e = cudaDeviceSynchronize();
    plan_free_buffers(p);
    release_spectrum(p->spec);
    release_spectrum(p->spec_dbl);
    delete p;
    if (e != cudaSuccess) return cuda_fail(e, "nm_destroy sync");
    return NM_OK;
}

uint64_t nm_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

nm_status nm_profile_enable(int on) {
    if (on) prof_clear();
    g_prof_on.store(on != 0);
    return NM_OK;
}

nm_status nm_profile_read(nm_kernel_stat* out, int max, int* count) {
    if (!count || (max > 0 && !out)) return fail(NM_EINVAL, "nm_profile_read: null argument");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::vector<nm_kernel_stat> agg;
    for (auto& r : g_prof) {
        cudaError_t e = cudaEventSynchronize(r.b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return cuda_fail(e, "profile events");
        nm_kernel_stat* st = nullptr;
        for (auto& a : agg)
            if (r.name == a.name) { st = &a; break; }
        if (!st) {
            agg.push_back(nm_kernel_stat{});
            st = &agg.back();
            snprintf(st->name, sizeof st->name, "%s", r.name.c_str());
        }
        st->launches += 1;
        st->units += (uint64_t)r.units;
        st->total_ms += ms;
    }
    *count = (int)agg.size();
    for (int i = 0; i < (int)agg.size() && i < max; ++i) out[i] = agg[i];
    return NM_OK;
}

const char* nm_status_string(nm_status s) {
    switch (s) {
        case NM_OK: return "NM_OK";
        case NM_EINVAL: return "NM_EINVAL";
        case NM_ENOMEM: return "NM_ENOMEM";
        case NM_ECUDA: return "NM_ECUDA";
        case NM_ETIMEOUT: return "NM_ETIMEOUT";
        case NM_EUNSUPPORTED: return "NM_EUNSUPPORTED";
    }
    return "NM_UNKNOWN";
}

const char* nm_last_error(void) { return t_last_error.c_str(); }

}  // extern "C"
