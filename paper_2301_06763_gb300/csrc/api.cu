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

#include <nvtx3/nvToolsExt.h>

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
    nvtxRangePushA(name);   // host-side range per pass launch, for timeline tools
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
    nvtxRangePop();
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
    df* ddf = nullptr;
    float* d32x = nullptr;   // float rows over all kx (paired FP32 z-seam), on demand
    float* d32z = nullptr;   // float octant with fz fastest (three-pass form), on demand
};
struct Twiddle {
    int dev = -1, P = 0;
    cpx<double>* d64 = nullptr;
    cpx<float>* d32 = nullptr;
    cpx<df>* ddf = nullptr;
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
    std::vector<cpx<df>> hdf(P);
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < P; ++t) {
        const double a = two_pi * (double)t / (double)P;
        h64[t] = {std::cos(a), -std::sin(a)};
        h32[t] = {(float)h64[t].re, (float)h64[t].im};
        hdf[t] = {df(h64[t].re), df(h64[t].im)};
    }
    Twiddle* tw = new Twiddle();
    tw->dev = dev;
    tw->P = P;
    cudaError_t e = cudaMalloc(&tw->d64, sizeof(cpx<double>) * P);
    if (e == cudaSuccess) e = cudaMalloc(&tw->d32, sizeof(cpx<float>) * P);
    if (e == cudaSuccess) e = cudaMalloc(&tw->ddf, sizeof(cpx<df>) * P);
    if (e == cudaSuccess) e = cudaMemcpy(tw->ddf, hdf.data(), sizeof(cpx<df>) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(tw->d64, h64.data(), sizeof(cpx<double>) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(tw->d32, h32.data(), sizeof(cpx<float>) * P, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(tw->d64);
        cudaFree(tw->d32);
        cudaFree(tw->ddf);
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
    cudaFree(s->ddf);
    cudaFree(s->d32x);
    cudaFree(s->d32z);
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
    if (e == cudaSuccess && !s->ddf) e = cudaMalloc(&s->ddf, n * sizeof(df));
    if (e == cudaSuccess) e = cudaMalloc(&d_ctab, P * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&scratch, 2 * n * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ctab, ctab.data(), P * sizeof(double), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = run_green_octant(s->d64, scratch, d_ctab, N, self_term, stream);
    if (e == cudaSuccess) e = run_to_float(s->d64, s->d32, n, stream);
    if (e == cudaSuccess) e = run_to_df(s->d64, s->ddf, n, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFree(d_ctab);
    cudaFree(scratch);
    if (e != cudaSuccess) return cuda_fail(e, "green spectrum");
    s->ready = true;
    return NM_OK;
}

// The float rows over all kx that the paired FP32 z-seam prefetches (built
// once per spectrum, after the octant; synchronous on `stream`).
static nm_status build_unfolded(Spectrum* s, cudaStream_t stream) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (s->d32x) return NM_OK;
    const int N = s->N;
    float* out = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)(N + 1) * (N + 1) * 2 * N * sizeof(float));
    if (e == cudaSuccess) e = run_unfold_x(s->d64, out, N, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFree(out);
        return cuda_fail(e, "unfolded spectrum");
    }
    s->d32x = out;
    return NM_OK;
}

const float* unfolded_spectrum(const float* spec) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (Spectrum* s : g_spectra)
        if (s->d32 == spec) return s->d32x;
    return nullptr;
}

// The float octant with fz fastest that the three-pass form's fused y/z/y
// pass reads (built once per spectrum, after the octant; synchronous).
static nm_status build_zfast(Spectrum* s, cudaStream_t stream) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (s->d32z) return NM_OK;
    float* out = nullptr;
    cudaError_t e = cudaMalloc(&out, octant_count(s->N) * sizeof(float));
    if (e == cudaSuccess) e = run_zfast(s->d64, out, s->N, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFree(out);
        return cuda_fail(e, "z-fast spectrum");
    }
    s->d32z = out;
    return NM_OK;
}

const float* zfast_spectrum(const float* spec) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (Spectrum* s : g_spectra)
        if (s->d32 == spec) return s->d32z;
    return nullptr;
}

// ------------------------------------------------------------------ TMA, status
static std::mutex g_dev_mu;
static int* g_status[64] = {};
static int g_sms[64] = {};
static std::atomic<int> g_fault_timeout{0};
static std::atomic<int> g_fail_alloc{0};   // > 0: the n-th next plan workspace allocation fails

int* device_status_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (!g_status[dev]) {
        int* p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) {
            cudaFree(p);
            return nullptr;
        }
        g_status[dev] = p;
    }
    return g_status[dev];
}

int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (!g_sms[dev]) {
        int n = 1;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 1;
        g_sms[dev] = n;
    }
    return g_sms[dev];
}

bool fault_timeout_on() { return g_fault_timeout.load(std::memory_order_relaxed) != 0; }

// cuTensorMapEncodeTiled, looked up once through the runtime (no libcuda link).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t encode_work_map(CUtensorMap* map, void* work, int P, bool f64, int TX) {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    });
    if (!fn) return cudaErrorNotSupported;
    const size_t es = f64 ? 8 : 4;
    const cuuint64_t dims[3] = {(cuuint64_t)2 * P, (cuuint64_t)P, (cuuint64_t)P / 2};
    const cuuint64_t strides[2] = {(cuuint64_t)2 * P * es, (cuuint64_t)2 * P * P * es};
    const cuuint32_t box[3] = {(cuuint32_t)2 * TX, 1u, (cuuint32_t)P / 2};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = fn(map, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, work, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace nm

using namespace nm;

// ------------------------------------------------------------------ plan
struct nm_plan_s {
    nm_options opt;
    int dev = 0;
    int N = 0, L = 0, P = 0;
    bool fp32 = false, dipole = false;
    bool dfx = false;                 // NM_FP64X: transforms in double-float
    bool triple = false, triple_ds = false;   // three-level dipole scheme (Appendix B), Eq. B.6 variant
    size_t es = 8, cs = 16;           // bytes per real / complex value
    nm_schedule sched{1, 16, 0, 1, 1};   // level convolutions
    int group_dbl = 1;                // doubled-grid convolutions in flight
    int npairs = 0, npairs_dbl = 0;
    int group_qdp = 1, npairs_qdp = 0;   // quadrupled-grid convolutions (three-level scheme)
    int work_slots = 0;               // work buffers allocated (>= sched.group)
    void* restr = nullptr;            // (L-1) * (N/2)^3 restricted densities
    void* work = nullptr;             // work_slots * (P/2) * P^2 complex
    void* lvl = nullptr;              // L * N^3 level potentials
    void* crop = nullptr;             // (L-1) * (N/2+2)^3 hole crops (original method)
    void* carry = nullptr;            // (L-2) * (N/2+2)^3 carried holes (diagonal interp)
    void* vbuf = nullptr;             // method C face arrays, 2 (L-1) 6 (N/2+2)^2 doubles
    void* dbl_work = nullptr;         // group_dbl * (2N) * (4N)^2 complex (dipole)
    void* dbl_out = nullptr;          // (L-1) * (2N)^3 (dipole)
    void* qdp_work = nullptr;         // group_qdp * (4N) * (8N)^2 complex (three-level scheme)
    void* qdp_out = nullptr;          // (L-2) * (4N)^3 (three-level scheme, quadrupled grids)
    void* red = nullptr;              // (L-2) * N^3 reduced quadrupled grids or Eq. B.6 sums
    void* h_rho = nullptr;            // staging for nm_potential_host
    double* h_phi = nullptr;
    void* h_rho2[2] = {nullptr, nullptr};       // double-buffered staging of nm_potential_host_many
    double* h_phi2[2] = {nullptr, nullptr};
    cudaStream_t s_in = nullptr, s_out = nullptr;   // its copy streams
    cudaEvent_t ev_in[2] = {}, ev_solved[2] = {}, ev_out[2] = {};
    size_t ws_bytes = 0;
    Spectrum* spec = nullptr;
    Spectrum* spec_dbl = nullptr;
    Spectrum* spec_qdp = nullptr;
    Twiddle* tw = nullptr;
    Twiddle* tw_dbl = nullptr;
    Twiddle* tw_qdp = nullptr;
};

namespace {

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int env_int(const char* name, int dflt) {
    const char* v = std::getenv(name);
    if (!v || !*v) return dflt;
    return std::atoi(v);
}

size_t work_buf_bytes(nm_plan_t p) { return (size_t)(p->P / 2) * p->P * p->P * p->cs; }

void plan_free_buffers(nm_plan_t p) {
    cudaFree(p->restr);
    cudaFree(p->work);
    cudaFree(p->lvl);
    cudaFree(p->crop);
    cudaFree(p->carry);
    cudaFree(p->vbuf);
    cudaFree(p->dbl_work);
    cudaFree(p->dbl_out);
    cudaFree(p->qdp_work);
    cudaFree(p->qdp_out);
    cudaFree(p->red);
    cudaFree(p->h_rho);
    cudaFree(p->h_phi);
    for (int b = 0; b < 2; ++b) {
        cudaFree(p->h_rho2[b]);
        cudaFree(p->h_phi2[b]);
        p->h_rho2[b] = nullptr;
        p->h_phi2[b] = nullptr;
        if (p->ev_in[b]) cudaEventDestroy(p->ev_in[b]);
        if (p->ev_solved[b]) cudaEventDestroy(p->ev_solved[b]);
        if (p->ev_out[b]) cudaEventDestroy(p->ev_out[b]);
        p->ev_in[b] = p->ev_solved[b] = p->ev_out[b] = nullptr;
    }
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    p->s_in = p->s_out = nullptr;
    p->restr = p->work = p->lvl = p->crop = p->carry = p->vbuf = p->dbl_work = p->dbl_out = p->h_rho = nullptr;
    p->qdp_work = p->qdp_out = p->red = nullptr;
    p->h_phi = nullptr;
}

// Pairs in flight per launch: as many as fit in 1 GiB of work buffers.  On
// GB300 one launch over all levels beats per-level launches that would keep a
// level's intermediate resident in L2 (measured for 6 x 128^3: 0.67 vs 0.78
// ms per FP32 solve), so only memory bounds the group.
int default_group(size_t buf_bytes, int npairs) {
    int g = env_int("NM_GROUP", 0);
    if (g <= 0) {
        const size_t budget = (size_t)1 << 30;
        g = buf_bytes >= budget ? 1 : (int)(budget / buf_bytes);
    }
    if (g > npairs) g = npairs;
    if (g < 1) g = 1;
    return g;
}

// (Re)size the level work buffers to hold `slots` pairs.
nm_status ensure_work_slots(nm_plan_t p, int slots) {
    if (slots <= p->work_slots && slots * 2 > p->work_slots) return NM_OK;
    NM_CUDA(cudaDeviceSynchronize(), "work buffer resize");
    const size_t buf = work_buf_bytes(p);
    if (p->work) {
        cudaFree(p->work);
        p->ws_bytes -= (size_t)p->work_slots * buf;
        p->work = nullptr;
        p->work_slots = 0;
    }
    NM_CUDA(cudaMalloc(&p->work, (size_t)slots * buf), "work buffers");
    p->work_slots = slots;
    p->ws_bytes += (size_t)slots * buf;
    return NM_OK;
}

// ---------------------------------------------------------------- schedule table
std::mutex g_tune_mu;
struct TuneEntry {
    std::string key;
    nm_schedule sched;
};
std::vector<TuneEntry> g_tune;
bool g_tune_loaded = false;

std::string tune_key(nm_plan_t p) {
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, p->dev) == cudaSuccess) name = prop.name;
    for (auto& c : name)
        if (c == '"' || c == '|') c = '_';
    char buf[256];
    snprintf(buf, sizeof buf, "%s|N%d|L%d|%s|%s", name.c_str(), p->N, p->L, p->fp32 ? "fp32" : p->dfx ? "fp64x" : "fp64",
             p->triple ? (p->triple_ds ? "dipole3_ds" : "dipole3") : p->dipole ? "dipole" : "original");
    return buf;
}

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = std::getenv("NM_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char key[300];
        nm_schedule sc;
        if (std::sscanf(line, " {\"key\": \"%299[^\"]\", \"group\": %d, \"radix\": %d, \"tile\": %d, "
                        "\"pipeline\": %d, \"fuse\": %d", key, &sc.group, &sc.radix, &sc.tile, &sc.pipeline,
                        &sc.fuse) == 6) {
            bool found = false;
            for (auto& e : g_tune)
                if (e.key == key) { e.sched = sc; found = true; }
            if (!found) g_tune.push_back({key, sc});
        }
    }
    std::fclose(f);
}

bool tune_lookup(nm_plan_t p, nm_schedule* out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    const std::string k = tune_key(p);
    for (auto& e : g_tune)
        if (e.key == k) { *out = e.sched; return true; }
    return false;
}

void tune_store(nm_plan_t p, const nm_schedule& sc) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    const std::string k = tune_key(p);
    bool found = false;
    for (auto& e : g_tune)
        if (e.key == k) { e.sched = sc; found = true; }
    if (!found) g_tune.push_back({k, sc});
    const char* path = std::getenv("NM_AUTOTUNE_CACHE");
    if (path && *path) {
        FILE* f = std::fopen(path, "a");
        if (f) {
            std::fprintf(f,
                         "{\"key\": \"%s\", \"group\": %d, \"radix\": %d, \"tile\": %d, \"pipeline\": %d, "
                         "\"fuse\": %d}\n",
                         k.c_str(), sc.group, sc.radix, sc.tile, sc.pipeline, sc.fuse);
            std::fclose(f);
        }
    }
}

bool sched_valid(nm_plan_t p, const nm_schedule& sc) {
    if (sc.group < 1 || sc.group > p->npairs) return false;
    if (sc.radix != 8 && sc.radix != 16) return false;
    if (sc.radix == 16 && p->P < 16) return false;
    if (p->dfx && sc.radix != 16) return false;
    if (sc.pipeline < 0 || sc.pipeline > 3) return false;
    // two columns per thread: FP32 level grids, 16 values per thread, P >= 64
    if (sc.pipeline == 2 && (!p->fp32 || p->dfx || sc.radix != 16 || p->P < 64 || sc.fuse)) return false;
    // the same, persistent with the next tile's columns prefetched: P = 256,
    // narrow tiles
    if (sc.pipeline == 3 && (!p->fp32 || p->dfx || sc.radix != 16 || p->P != 256 || sc.fuse || sc.tile))
        return false;
    if (sc.fuse < 0 || sc.fuse > 3) return false;
    if (sc.fuse && sc.radix != 16) return false;
    // three-pass form (fused y/z/y per kx plane): FP32 level grids of the
    // original method, 2N in 64 .. 512; tile picks the CTAs per plane (1: the
    // alternative split, built for 2N = 128 and 256); the z-seam choice does
    // not apply
    if (sc.fuse == 2) {
        if (!p->fp32 || p->dfx || p->dipole || p->P < 64 || p->P > 512 || sc.pipeline != 0) return false;
        if (sc.tile == 1 && p->P != 128 && p->P != 256) return false;
    }
    // persistent form: every step of the solve (and of every mesh batched
    // with it) as work items of one launch; FP32 original method, 2N in
    // 64 .. 512, the one-column z-seam and plain tiles
    if (sc.fuse == 3 && (!p->fp32 || p->dfx || p->dipole || p->P < 64 || p->P > 512 || sc.pipeline != 0 ||
                         sc.tile != 0))
        return false;
    return sc.tile == 0 || sc.tile == 1;
}

// ---------------------------------------------------------------- graphs of batches
struct BatchGraph {
    std::vector<const void*> key;
    cudaGraphExec_t exec = nullptr;
    bool captured = false;
    uint64_t kernels = 0;   // kernel nodes in the graph (counted again per replay)
};
std::mutex g_graph_mu;
std::vector<BatchGraph> g_graphs;   // most recent last
constexpr size_t kMaxGraphs = 32;

// Laid-out persistent batches (their device tables), keyed like the graphs;
// a captured graph may reference one, so an entry lives until a plan of it
// is destroyed or rescheduled, or until the cache is full (then every graph
// goes too).
struct PersistEntry {
    std::vector<const void*> key;
    PersistBatch* b;
};
std::mutex g_persist_mu;
std::vector<PersistEntry> g_persist;   // most recent last
constexpr size_t kMaxPersist = 256;

void persist_drop_plan(nm_plan_t p) {
    std::lock_guard<std::mutex> lk(g_persist_mu);
    for (size_t i = 0; i < g_persist.size();) {
        bool uses = false;
        for (const void* k : g_persist[i].key)
            if (k == (const void*)p) uses = true;
        if (uses) {
            persist_free(g_persist[i].b);
            g_persist.erase(g_persist.begin() + i);
        } else {
            ++i;
        }
    }
}

void graphs_drop_plan(nm_plan_t p) {
    persist_drop_plan(p);
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (size_t i = 0; i < g_graphs.size();) {
        bool uses = false;
        for (const void* k : g_graphs[i].key)
            if (k == (const void*)p) uses = true;
        if (uses) {
            if (g_graphs[i].exec) cudaGraphExecDestroy(g_graphs[i].exec);
            g_graphs.erase(g_graphs.begin() + i);
        } else {
            ++i;
        }
    }
}

}  // namespace

extern "C" {

nm_status nm_default_options(int levels, int N, double dx0, nm_options* opt) {
    if (!opt) return fail(NM_EINVAL, "nm_default_options: null options");
    opt->levels = levels;
    opt->N = N;
    opt->dx0 = dx0;
    opt->G = 1.0;
    opt->precision = NM_FP64;
    opt->method = NM_METHOD_ORIGINAL;
    opt->interp = NM_INTERP_DIAGONAL;
    return NM_OK;
}

static nm_status validate_options(const nm_options& o) {
    if (o.levels < 1 || o.levels > NM_MAX_LEVELS)
        return fail(NM_EINVAL, "levels must be in [1, %d], got %d", NM_MAX_LEVELS, o.levels);
    if (o.N < 4 || o.N % 4 != 0)
        return fail(NM_EINVAL, "N must be a multiple of 4 (level m+1 covers [N/4, 3N/4)), got %d", o.N);
    if (!is_pow2(o.N) || o.N > 256)
        return fail(NM_EUNSUPPORTED, "N must be a power of two in [4, 256], got %d", o.N);
    if (!(o.dx0 > 0.0) || !std::isfinite(o.dx0)) return fail(NM_EINVAL, "dx0 must be finite and > 0");
    if (!std::isfinite(o.G)) return fail(NM_EINVAL, "G must be finite");
    if (o.precision != NM_FP64 && o.precision != NM_FP32 && o.precision != NM_FP64X)
        return fail(NM_EINVAL, "bad precision %d", o.precision);
    if (o.precision == NM_FP64X && o.method != NM_METHOD_ORIGINAL)
        return fail(NM_EUNSUPPORTED, "NM_FP64X is built for the original method only");
    if (o.precision == NM_FP64X && o.N < 8) return fail(NM_EUNSUPPORTED, "NM_FP64X needs N >= 8");
    if (o.method != NM_METHOD_ORIGINAL && o.method != NM_METHOD_DIPOLE_PAIR && o.method != NM_METHOD_DIPOLE_TRIPLE &&
        o.method != NM_METHOD_DIPOLE_TRIPLE_DIRECT)
        return fail(NM_EINVAL, "bad method %d", o.method);
    if (o.method == NM_METHOD_DIPOLE_TRIPLE && o.N > 128)
        return fail(NM_EUNSUPPORTED, "the quadrupled grid of N = %d needs transforms of %d points (at most 1024)", o.N,
                    8 * o.N);
    if (o.interp != NM_INTERP_TRILINEAR && o.interp != NM_INTERP_DIAGONAL)
        return fail(NM_EINVAL, "bad interp %d", o.interp);
    return NM_OK;
}

// Workspace bytes of a plan with the default schedule (mirrors nm_plan_ex).
static size_t default_footprint(const nm_options& o) {
    const size_t N = o.N, L = o.levels, P = 2 * N;
    const size_t es = o.precision == NM_FP32 ? 4 : 8, cs = 2 * es;
    const bool dipole = o.method != NM_METHOD_ORIGINAL;
    const size_t N3 = N * N * N, h3 = N3 / 8, nc = N / 2 + 2;
    const int npairs = dipole ? (int)((L + 1) / 2) : (int)L;
    const size_t buf = (P / 2) * P * P * cs;
    size_t b = (L - 1) * h3 * es + (size_t)default_group(buf, npairs) * buf + L * N3 * es;
    if (!dipole) b += (L - 1) * nc * nc * nc * es;
    if (o.interp == NM_INTERP_DIAGONAL && L > 2) b += (L - 2) * nc * nc * nc * es;
    b += accel_vbuf_doubles((int)L, (int)N) * sizeof(double);
    if (dipole && L > 1) {
        const size_t buf_dbl = (2 * N) * (4 * N) * (4 * N) * cs;
        b += (size_t)default_group(buf_dbl, (int)(L / 2)) * buf_dbl + (L - 1) * 8 * N3 * es;
    }
    if ((o.method == NM_METHOD_DIPOLE_TRIPLE || o.method == NM_METHOD_DIPOLE_TRIPLE_DIRECT) && L > 2) {
        b += (L - 2) * N3 * es;
        if (o.method == NM_METHOD_DIPOLE_TRIPLE) {
            const size_t buf_qdp = (4 * N) * (8 * N) * (8 * N) * cs;
            b += (size_t)default_group(buf_qdp, (int)((L - 1) / 2)) * buf_qdp + (L - 2) * 64 * N3 * es;
        }
    }
    return b;
}

nm_status nm_footprint_bytes(const nm_options* opt, size_t* bytes) {
    if (!opt || !bytes) return fail(NM_EINVAL, "nm_footprint_bytes: null argument");
    nm_status st = validate_options(*opt);
    if (st != NM_OK) return st;
    *bytes = default_footprint(*opt);
    return NM_OK;
}

nm_status nm_plan_ex(const nm_options* opt, nm_plan_t* out) {
    if (!opt || !out) return fail(NM_EINVAL, "nm_plan_ex: null argument");
    *out = nullptr;
    const nm_options o = *opt;
    nm_status vst = validate_options(o);
    if (vst != NM_OK) return vst;

    nm_plan_t p = new (std::nothrow) nm_plan_s();
    if (!p) return fail(NM_ENOMEM, "host allocation");
    p->opt = o;
    cudaError_t ge = cudaGetDevice(&p->dev);
    if (ge != cudaSuccess) {
        delete p;
        return cuda_fail(ge, "cudaGetDevice");
    }
    p->N = o.N;
    p->L = o.levels;
    p->P = 2 * o.N;
    p->fp32 = o.precision == NM_FP32;
    p->dfx = o.precision == NM_FP64X;
    p->dipole = o.method != NM_METHOD_ORIGINAL;
    p->triple = (o.method == NM_METHOD_DIPOLE_TRIPLE || o.method == NM_METHOD_DIPOLE_TRIPLE_DIRECT) && o.levels > 2;
    p->triple_ds = o.method == NM_METHOD_DIPOLE_TRIPLE_DIRECT;
    p->es = p->fp32 ? 4 : 8;
    p->cs = 2 * p->es;
    const size_t N = o.N, L = o.levels;
    const size_t N3 = N * N * N, h3 = (N / 2) * (N / 2) * (N / 2);
    const size_t nc = N / 2 + 2, nc3 = nc * nc * nc;
    p->npairs = p->dipole ? (int)((L + 1) / 2) : (int)L;
    p->npairs_dbl = p->dipole ? (int)(L / 2) : 0;   // ceil((L-1)/2)
    p->sched.group = default_group(work_buf_bytes(p), p->npairs);
    p->sched.radix = p->P >= 16 ? 16 : 8;
    p->sched.tile = 0;
    // one column per thread, one tile per CTA; in FP32 with P >= 64 the
    // CTA's spectrum rows are staged in shared memory (measured faster than
    // the paired z-seam on the 6 x 128^3 mesh: 197 against 209 us)
    p->sched.pipeline = 0;
    p->sched.fuse = 0;
    nm_schedule tuned;
    if (tune_lookup(p, &tuned) && sched_valid(p, tuned)) p->sched = tuned;
    const size_t buf_dbl = (2 * N) * (4 * N) * (4 * N) * p->cs;
    if (p->dipole) p->group_dbl = default_group(buf_dbl, p->npairs_dbl);
    const size_t buf_qdp = (4 * N) * (8 * N) * (8 * N) * p->cs;
    p->npairs_qdp = p->triple && !p->triple_ds ? (int)((L - 1) / 2) : 0;   // ceil((L-2)/2)
    if (p->npairs_qdp) p->group_qdp = default_group(buf_qdp, p->npairs_qdp);

    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (e != cudaSuccess || bytes == 0) return;
        // test hook: the armed allocation fails as if the device were full
        if (g_fail_alloc.load() > 0 && g_fail_alloc.fetch_sub(1) == 1) {
            e = cudaErrorMemoryAllocation;
            return;
        }
        e = cudaMalloc(ptr, bytes);
        if (e == cudaSuccess) p->ws_bytes += bytes;
    };
    alloc(&p->restr, (L - 1) * h3 * p->es);
    alloc(&p->work, (size_t)p->sched.group * work_buf_bytes(p));
    if (e == cudaSuccess) p->work_slots = p->sched.group;
    alloc(&p->lvl, L * N3 * p->es);
    if (!p->dipole) alloc(&p->crop, (L - 1) * nc3 * p->es);
    if (o.interp == NM_INTERP_DIAGONAL && L > 2) alloc(&p->carry, (L - 2) * nc3 * p->es);
    alloc(&p->vbuf, accel_vbuf_doubles((int)L, (int)N) * sizeof(double));
    if (p->dipole && L > 1) {
        alloc(&p->dbl_work, (size_t)p->group_dbl * buf_dbl);
        alloc(&p->dbl_out, (L - 1) * 8 * N3 * p->es);
    }
    if (p->triple) alloc(&p->red, (L - 2) * N3 * p->es);
    if (p->npairs_qdp) {
        alloc(&p->qdp_work, (size_t)p->group_qdp * buf_qdp);
        alloc(&p->qdp_out, (L - 2) * 64 * N3 * p->es);
    }
    if (e != cudaSuccess) {
        plan_free_buffers(p);
        delete p;
        return cuda_fail(e, "plan workspace");
    }
    nm_status st = get_twiddle(p->dev, p->P, &p->tw);
    if (st == NM_OK && p->dipole && L > 1) st = get_twiddle(p->dev, 2 * p->P, &p->tw_dbl);
    if (st == NM_OK && p->npairs_qdp) st = get_twiddle(p->dev, 4 * p->P, &p->tw_qdp);
    if (st == NM_OK) st = acquire_spectrum(p->dev, o.N, &p->spec);
    if (st == NM_OK && p->dipole && L > 1) st = acquire_spectrum(p->dev, 2 * o.N, &p->spec_dbl);
    if (st == NM_OK && p->npairs_qdp) st = acquire_spectrum(p->dev, 4 * o.N, &p->spec_qdp);
    if (st != NM_OK) {
        release_spectrum(p->spec);
        release_spectrum(p->spec_dbl);
        release_spectrum(p->spec_qdp);
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
    if (st == NM_OK && p->spec_qdp) st = build_spectrum(p->spec_qdp, (cudaStream_t)stream);
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

const SrcField kNoSrc{nullptr, nullptr, SRC_NONE, 0.0};

// The level convolutions of one solve (work pointers unset).
template <typename T>
void level_pairs(nm_plan_t p, const void* rho, std::vector<PairDesc<T>>& out) {
    const int L = p->L, P = p->P;
    const size_t N3 = (size_t)p->N * p->N * p->N;
    const size_t nc = p->N / 2 + 2, nc3 = nc * nc * nc;
    T* lvl = (T*)p->lvl;
    if (!p->dipole) {
        // Eq. 14: level m's full grid (re) and hole grid (im), Fig. 5
        for (int m = 0; m < L; ++m) {
            PairDesc<T> d{};
            d.src[0] = field(p, rho, m, SRC_FULL, P);
            d.dst[0] = {lvl + (size_t)m * N3, DST_GRID};
            if (m < L - 1) {
                d.src[1] = field(p, rho, m, SRC_HOLE, P);
                d.dst[1] = {(T*)p->crop + (size_t)m * nc3, DST_CROP};
            } else {
                d.src[1] = kNoSrc;
                d.dst[1] = {nullptr, DST_NONE};
            }
            out.push_back(d);
        }
    } else {
        // Eqs. 15, B.1-B.2: hole grids of every level but the finest, and the
        // finest full grid, two real fields per complex transform
        for (int m = 0; m < L; m += 2) {
            PairDesc<T> d{};
            for (int h = 0; h < 2; ++h) {
                const int lv = m + h;
                if (lv < L) {
                    d.src[h] = field(p, rho, lv, lv < L - 1 ? SRC_HOLE : SRC_FULL, P);
                    d.dst[h] = {lvl + (size_t)lv * N3, DST_GRID};
                } else {
                    d.src[h] = kNoSrc;
                    d.dst[h] = {nullptr, DST_NONE};
                }
            }
            out.push_back(d);
        }
    }
}

// Doubled fine grids (Fig. 16): level n+1's mass on 2N cells spanning level n.
template <typename T>
void dbl_pairs(nm_plan_t p, const void* rho, std::vector<PairDesc<T>>& out) {
    const int L = p->L, P2 = 2 * p->P;
    const size_t N3 = (size_t)p->N * p->N * p->N;
    for (int n = 0; n < L - 1; n += 2) {
        PairDesc<T> d{};
        for (int h = 0; h < 2; ++h) {
            const int nn = n + h;
            if (nn < L - 1) {
                // three-level scheme: level n+1's ring only (level n+2's
                // region emptied) below level L-2, Fig. App0
                const int mode = (p->triple && nn < L - 2) ? SRC_HOLE : SRC_FULL;
                d.src[h] = field(p, rho, nn + 1, mode, P2);
                d.dst[h] = {(T*)p->dbl_out + (size_t)nn * 8 * N3, DST_GRID};
            } else {
                d.src[h] = kNoSrc;
                d.dst[h] = {nullptr, DST_NONE};
            }
        }
        out.push_back(d);
    }
}

// Quadrupled grids (Fig. App0): level n+2's mass on 4N cells spanning level n.
template <typename T>
void qdp_pairs(nm_plan_t p, const void* rho, std::vector<PairDesc<T>>& out) {
    const int L = p->L, P4 = 4 * p->P;
    const size_t N3 = (size_t)p->N * p->N * p->N;
    for (int n = 0; n < L - 2; n += 2) {
        PairDesc<T> d{};
        for (int h = 0; h < 2; ++h) {
            const int nn = n + h;
            if (nn < L - 2) {
                d.src[h] = field(p, rho, nn + 2, SRC_FULL, P4);
                d.dst[h] = {(T*)p->qdp_out + (size_t)nn * 64 * N3, DST_GRID};
            } else {
                d.src[h] = kNoSrc;
                d.dst[h] = {nullptr, DST_NONE};
            }
        }
        out.push_back(d);
    }
}

template <typename T> const T* spec_of(const Spectrum* s);
template <> const float* spec_of<float>(const Spectrum* s) { return s->d32; }
template <> const double* spec_of<double>(const Spectrum* s) { return s->d64; }
template <> const df* spec_of<df>(const Spectrum* s) { return s->ddf; }
template <typename T> const cpx<T>* tw_of(const Twiddle* t);
template <> const cpx<float>* tw_of<float>(const Twiddle* t) { return t->d32; }
template <> const cpx<double>* tw_of<double>(const Twiddle* t) { return t->d64; }
template <> const cpx<df>* tw_of<df>(const Twiddle* t) { return t->ddf; }

template <typename T>
cudaError_t run_conv(const PairDesc<T>* pairs, int n, int P, int geom, const nm_schedule& sc,
                     const T* spec, const cpx<T>* tw, cudaStream_t s) {
    const bool dbl = geom == 1;
    if constexpr (is_df<T>::value) {
        // level grids only (NM_FP64X is validated for the original method)
        if (geom != 0) return cudaErrorInvalidValue;
        return run_conv_dfx_e16(pairs, n, P, false, sc.tile ? CONV_WIDE : 0, spec, tw, s);
    } else {
        if (geom == 2) {
            if constexpr (sizeof(T) == 4) return run_conv_qdp_f32(pairs, n, P, spec, tw, s);
            else return run_conv_qdp_f64(pairs, n, P, spec, tw, s);
        }
        if constexpr (sizeof(T) == 4) {
            // three-pass form where the pairs allow it (a level's full and
            // hole fields on aligned buffers), else the five passes
            if (geom == 0 && sc.fuse == 2 && yzy_pairs_ok(pairs, n))
                return run_conv_f32_yzy(pairs, n, P, sc.tile, spec, tw, s);
        }
        const bool e16 = dbl || (sc.radix == 16 && P >= 16);
        // FP32 level grids with the one-column z-seam stage their spectrum
        // rows (the plan built the unfolded float spectrum, ensure_green)
        const bool sspec = sizeof(T) == 4 && geom == 0 && sc.pipeline == 0 && P >= 64;
        const int flags = (sc.fuse != 2 && sc.tile ? CONV_WIDE : 0) | (sc.pipeline == 1 ? CONV_TMA : 0) |
                          (sc.pipeline >= 2 ? CONV_PAIRED : 0) | (sc.pipeline == 3 ? CONV_ZPERSIST : 0) |
                          (sc.fuse == 1 ? CONV_FUSED : 0) | (sspec ? CONV_SSPEC : 0);
        if constexpr (sizeof(T) == 4) {
            return e16 ? run_conv_f32_e16(pairs, n, P, dbl, flags, spec, tw, s)
                       : run_conv_f32_e8(pairs, n, P, dbl, flags, spec, tw, s);
        } else {
            return e16 ? run_conv_f64_e16(pairs, n, P, dbl, flags, spec, tw, s)
                       : run_conv_f64_e8(pairs, n, P, dbl, flags, spec, tw, s);
        }
    }
}

template <typename T>
nm_status enqueue_restrict(nm_plan_t p, const void* rho, cudaStream_t s) {
    const int L = p->L, N = p->N;
    const size_t N3 = (size_t)N * N * N, h3 = N3 / 8;
    for (int m = L - 2; m >= 0; --m) {
        using TIN = typename InOf<T>::type;
        const TIN* child = (const TIN*)rho + (size_t)(m + 1) * N3;
        const TIN* rchild = (m + 1 < L - 1) ? (const TIN*)p->restr + (size_t)(m + 1) * h3 : nullptr;
        cudaError_t e = run_restrict<TIN>(child, rchild, (TIN*)p->restr + (size_t)m * h3, N, s);
        if (e != cudaSuccess) return cuda_fail(e, "restriction");
    }
    return NM_OK;
}

template <typename T>
AssembleArgs<T> assemble_args(nm_plan_t p, double* phi) {
    const int L = p->L, N = p->N;
    const size_t N3 = (size_t)N * N * N;
    const size_t nc = N / 2 + 2, nc3 = nc * nc * nc;
    const T* lvl = (const T*)p->lvl;
    AssembleArgs<T> a{};
    a.phi = phi;
    a.levels = L;
    a.N = N;
    // the carried Eqs. 3-6 rule reads level n-1 only (the hole crop, or the
    // carried sum once the carry chain has run); trilinear reads every k < n
    a.diag = p->opt.interp == NM_INTERP_DIAGONAL ? 1 : 0;
    for (int n = 0; n < L; ++n) {
        a.base[n] = lvl + (size_t)n * N3;
        a.dbl[n] = (p->dipole && n < L - 1) ? (const T*)p->dbl_out + (size_t)n * 8 * N3 : nullptr;
        a.red[n] = (p->triple && n < L - 2) ? (const T*)p->red + (size_t)n * N3 : nullptr;
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
    return a;
}

template <typename T>
nm_status enqueue_assemble(nm_plan_t p, double* phi, cudaStream_t s) {
    cudaError_t e = run_assemble_interp<T>(assemble_args<T>(p, phi), p->opt.interp, (T*)p->carry, s);
    if (e != cudaSuccess) return cuda_fail(e, "assembly");
    return NM_OK;
}


// One mesh of a batch (or a single solve).
struct Item {
    nm_plan_t p;
    const void* rho;
    double* phi;
};

// The restrictions of every mesh of a batch: one launch for all their levels
// (chains.cu), the per-level kernel where a mesh is too small or too deep.
template <typename T>
nm_status enqueue_restrict_batch(const std::vector<Item>& items, cudaStream_t s) {
    using TIN = typename InOf<T>::type;
    std::vector<RestrictMesh<TIN>> rm;
    for (const Item& it : items)
        if (it.p->L >= 2) rm.push_back({(const TIN*)it.rho, (TIN*)it.p->restr, it.p->N, it.p->L});
    if (rm.empty()) return NM_OK;
    cudaError_t e = run_restrict_tree<TIN>(rm.data(), (int)rm.size(), s);
    if (e != cudaSuccess) return cuda_fail(e, "restriction");
    return NM_OK;
}

// The carried interpolation of every mesh of a batch that reads the Eqs. 3-6
// rule (one launch for all their levels), then each mesh's assembly reading
// the carried sums.
template <typename T>
nm_status enqueue_assemble_batch(const std::vector<Item>& items, cudaStream_t s) {
    std::vector<CarryMesh<T>> cm;
    for (const Item& it : items) {
        nm_plan_t p = it.p;
        if (p->opt.interp != NM_INTERP_DIAGONAL || p->L < 3) continue;
        const AssembleArgs<T> a = assemble_args<T>(p, it.phi);
        const size_t N3 = (size_t)p->N * p->N * p->N, nc = p->N / 2 + 2;
        CarryMesh<T> m{};
        m.hole = a.interp[0];
        m.hole_stride = p->dipole ? N3 : nc * nc * nc;
        m.hole_origin = a.interp_origin[0];
        m.hole_extent = a.interp_extent[0];
        m.out = (T*)p->carry;
        m.N = p->N;
        m.L = p->L;
        cm.push_back(m);
    }
    if (!cm.empty()) {
        cudaError_t e = run_carry_tree<T>(cm.data(), (int)cm.size(), s);
        if (e != cudaSuccess) return cuda_fail(e, "carried interpolation");
    }
    std::vector<AssembleArgs<T>> as;
    for (const Item& it : items) {
        nm_plan_t p = it.p;
        AssembleArgs<T> a = assemble_args<T>(p, it.phi);
        if (p->opt.interp == NM_INTERP_DIAGONAL) {
            const int N = p->N;
            const size_t nc = N / 2 + 2, nc3 = nc * nc * nc;
            a.diag = 1;
            for (int n = 1; n + 1 < p->L; ++n) {
                a.interp[n] = (const T*)p->carry + (size_t)(n - 1) * nc3;
                a.interp_origin[n] = N / 4 - 1;
                a.interp_extent[n] = (int)nc;
            }
        }
        as.push_back(a);
    }
    // one mesh: the single-mesh kernel; several: one launch per kAsmMeshes
    cudaError_t e = as.size() == 1 ? run_assemble<T>(as[0], s) : run_assemble_batch<T>(as.data(), (int)as.size(), s);
    if (e != cudaSuccess) return cuda_fail(e, "assembly");
    return NM_OK;
}

// The solves of plans with the persistent schedule (fuse 3): one laid-out
// batch per set of (plan, rho, phi), built on first use (synchronously, so
// not while the caller captures a graph), then one counter reset and one
// launch per call.
std::vector<const void*> items_key(const std::vector<Item>& items) {
    std::vector<const void*> key;
    for (const Item& it : items) {
        key.push_back(it.p);
        key.push_back(it.rho);
        key.push_back(it.phi);
        const nm_schedule& sc = it.p->sched;
        key.push_back((const void*)(uintptr_t)((sc.group << 12) | (sc.radix << 4) | (sc.fuse << 3) |
                                               (sc.tile << 2) | sc.pipeline));
    }
    return key;
}

void graphs_drop_all() {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto& g : g_graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    g_graphs.clear();
}

nm_status enqueue_persistent(const std::vector<Item>& items, cudaStream_t s) {
    const std::vector<const void*> key = items_key(items);
    PersistBatch* b = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_persist_mu);
        for (size_t i = 0; i < g_persist.size(); ++i)
            if (g_persist[i].key == key) {
                PersistEntry e = g_persist[i];
                g_persist.erase(g_persist.begin() + i);
                g_persist.push_back(e);
                b = e.b;
                break;
            }
    }
    if (!b) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone)
            return fail(NM_EUNSUPPORTED, "persistent schedule: make one call with these buffers before capturing it");
        std::vector<PersistMesh> meshes;
        for (const Item& it : items) {
            nm_plan_t p = it.p;
            PersistMesh m;
            m.P = p->P;
            m.L = p->L;
            m.group = p->sched.group;
            m.rho = (const float*)it.rho;
            m.restr = (float*)p->restr;
            m.phi = it.phi;
            m.work = p->work;
            m.spec = spec_of<float>(p->spec);
            m.tw = tw_of<float>(p->tw);
            level_pairs<float>(p, it.rho, m.pairs);
            m.carry = (p->opt.interp == NM_INTERP_DIAGONAL && p->L > 2) ? (float*)p->carry : nullptr;
            m.asm_args = assemble_args<float>(p, it.phi);
            meshes.push_back(std::move(m));
        }
        b = persist_new();
        if (!b) return fail(NM_ENOMEM, "host allocation");
        if (!persist_layout(meshes, *b)) {
            persist_free(b);
            return fail(NM_EUNSUPPORTED, "persistent schedule: a mesh of this batch does not fit it (buffers must "
                                         "be 16-byte aligned)");
        }
        cudaError_t e = persist_upload(*b);
        if (e != cudaSuccess) {
            persist_free(b);
            return cuda_fail(e, "persistent batch tables");
        }
        bool drop_graphs = false;
        {
            std::lock_guard<std::mutex> lk(g_persist_mu);
            if (g_persist.size() >= kMaxPersist) {
                // a graph may still reference the oldest tables: wait for the
                // device, drop every graph, then free them
                drop_graphs = true;
                cudaDeviceSynchronize();
                persist_free(g_persist.front().b);
                g_persist.erase(g_persist.begin());
            }
            g_persist.push_back(PersistEntry{key, b});
        }
        if (drop_graphs) graphs_drop_all();
    }
    cudaError_t e = persist_launch(*b, s);
    if (e != cudaSuccess) return cuda_fail(e, "persistent batch");
    return NM_OK;
}

// Restriction, level and doubled-grid convolutions round by round, assembly.
// Every mesh uses its own workspace; in round r mesh i contributes pairs
// [r g_i, (r+1) g_i) and contributions with equal (P, radix, tile) share a
// launch per pass.  Plans with the persistent schedule go to one persistent
// launch instead.
template <typename T>
nm_status enqueue_items_rounds(const std::vector<Item>& items, cudaStream_t s);

template <typename T>
nm_status enqueue_items(const std::vector<Item>& items, cudaStream_t s) {
    if constexpr (sizeof(T) == 4 && !is_df<T>::value) {
        std::vector<Item> pers, rest;
        for (const Item& it : items) (it.p->sched.fuse == 3 ? pers : rest).push_back(it);
        if (!pers.empty()) {
            nm_status st = enqueue_persistent(pers, s);
            if (st != NM_OK) return st;
        }
        if (rest.empty()) return NM_OK;
        return enqueue_items_rounds<T>(rest, s);
    } else {
        return enqueue_items_rounds<T>(items, s);
    }
}

template <typename T>
nm_status enqueue_items_rounds(const std::vector<Item>& items, cudaStream_t s) {
    nm_status st;
    if ((st = enqueue_restrict_batch<T>(items, s)) != NM_OK) return st;
    // geometry 0: level grids; 1: doubled grids (dipole methods); 2:
    // quadrupled grids (three-level scheme)
    for (int geom = 0; geom < 3; ++geom) {
        std::vector<std::vector<PairDesc<T>>> pl(items.size());
        int rounds = 0;
        auto group_of = [&](nm_plan_t p) { return geom == 0 ? p->sched.group : geom == 1 ? p->group_dbl : p->group_qdp; };
        for (size_t i = 0; i < items.size(); ++i) {
            nm_plan_t p = items[i].p;
            if (geom == 0) level_pairs<T>(p, items[i].rho, pl[i]);
            else if (geom == 1 && p->dipole && p->L > 1) dbl_pairs<T>(p, items[i].rho, pl[i]);
            else if (geom == 2 && p->npairs_qdp) qdp_pairs<T>(p, items[i].rho, pl[i]);
            const int g = group_of(p);
            const int r = ((int)pl[i].size() + g - 1) / g;
            if (r > rounds) rounds = r;
        }
        for (int r = 0; r < rounds; ++r) {
            struct Bucket {
                int P;
                nm_schedule sc;
                const T* spec;
                const cpx<T>* tw;
                std::vector<PairDesc<T>> pairs;
            };
            std::vector<Bucket> buckets;
            for (size_t i = 0; i < items.size(); ++i) {
                nm_plan_t p = items[i].p;
                const int g = group_of(p);
                const int P = p->P << geom;
                const nm_schedule sc = geom ? nm_schedule{1, 16, 0, 0, 0} : p->sched;
                const size_t buf = (size_t)(P / 2) * P * P;
                cpx<T>* work = (cpx<T>*)(geom == 0 ? p->work : geom == 1 ? p->dbl_work : p->qdp_work);
                const Spectrum* spec = geom == 0 ? p->spec : geom == 1 ? p->spec_dbl : p->spec_qdp;
                const Twiddle* tw = geom == 0 ? p->tw : geom == 1 ? p->tw_dbl : p->tw_qdp;
                for (int q = r * g; q < (r + 1) * g && q < (int)pl[i].size(); ++q) {
                    PairDesc<T> d = pl[i][q];
                    d.work = work + (size_t)(q - r * g) * buf;
                    Bucket* b = nullptr;
                    for (auto& bb : buckets)
                        if (bb.P == P && bb.sc.radix == sc.radix && bb.sc.tile == sc.tile &&
                            bb.sc.pipeline == sc.pipeline && bb.sc.fuse == sc.fuse)
                            b = &bb;
                    if (!b) {
                        buckets.push_back({P, sc, spec_of<T>(spec), tw_of<T>(tw), {}});
                        b = &buckets.back();
                    }
                    b->pairs.push_back(d);
                }
            }
            for (auto& b : buckets) {
                cudaError_t e = run_conv<T>(b.pairs.data(), (int)b.pairs.size(), b.P, geom, b.sc, b.spec,
                                            b.tw, s);
                if (e != cudaSuccess)
                    return cuda_fail(e, geom == 0   ? "level convolution"
                                        : geom == 1 ? "doubled-grid convolution"
                                                    : "quadrupled-grid convolution");
            }
        }
    }
    // three-level scheme: level n+2's term on level n (n < L-2), reduced from
    // the quadrupled grid or summed directly (Eq. B.6)
    if constexpr (!is_df<T>::value) for (const Item& it : items) {
        nm_plan_t p = it.p;
        if (!p->triple) continue;
        const int N = p->N;
        const size_t N3 = (size_t)N * N * N, h3 = N3 / 8;
        for (int n = 0; n + 2 < p->L; ++n) {
            T* out = (T*)p->red + (size_t)n * N3;
            cudaError_t e;
            if (p->triple_ds) {
                const int m = n + 2;
                const double dx = p->opt.dx0 / std::ldexp(1.0, m);
                const T* restr = m < p->L - 1 ? (const T*)p->restr + (size_t)m * h3 : nullptr;
                e = run_direct2<T>((const T*)it.rho + (size_t)m * N3, restr, out, N, -p->opt.G * dx * dx, s);
            } else {
                e = run_reduce4<T>((const T*)p->qdp_out + (size_t)n * 64 * N3, out, N, s);
            }
            if (e != cudaSuccess) return cuda_fail(e, "three-level term");
        }
    }
    return enqueue_assemble_batch<T>(items, s);
}

nm_status ensure_green(nm_plan_t p, cudaStream_t s) {
    if (!p->spec->ready || (p->spec_dbl && !p->spec_dbl->ready) || (p->spec_qdp && !p->spec_qdp->ready)) {
        nm_status st = nm_green(p, (void*)s);
        if (st != NM_OK) return st;
    }
    // the paired z-seam and the one-column FP32 z-seam read the float spectrum
    // unfolded along kx
    const bool unfolded = p->sched.pipeline >= 2 || (p->sched.pipeline == 0 && p->fp32 && !p->dfx && p->P >= 64);
    if (unfolded && !p->spec->d32x) {
        nm_status st = build_unfolded(p->spec, s);
        if (st != NM_OK) return st;
    }
    if (p->sched.fuse == 2 && !p->spec->d32z) return build_zfast(p->spec, s);
    return NM_OK;
}

nm_status enqueue_all(const std::vector<Item>& items, cudaStream_t s) {
    std::vector<Item> f32, f64, fdf;
    for (const Item& it : items) (it.p->fp32 ? f32 : it.p->dfx ? fdf : f64).push_back(it);
    nm_status st = NM_OK;
    if (!f64.empty()) st = enqueue_items<double>(f64, s);
    if (st == NM_OK && !fdf.empty()) st = enqueue_items<df>(fdf, s);
    if (st == NM_OK && !f32.empty()) st = enqueue_items<float>(f32, s);
    return st;
}

nm_status potential_impl(nm_plan_t p, const void* rho, double* phi, cudaStream_t s) {
    nm_status st = ensure_green(p, s);
    if (st != NM_OK) return st;
    return enqueue_all({Item{p, rho, phi}}, s);
}

// One-second-scale timing of a solve with the plan's current schedule.
nm_status time_solves(nm_plan_t p, const void* rho, double* phi, int reps, cudaStream_t s, float* ms) {
    nm_status st = potential_impl(p, rho, phi, s);
    if (st != NM_OK) return st;
    cudaEvent_t a, b;
    NM_CUDA(cudaEventCreate(&a), "event");
    NM_CUDA(cudaEventCreate(&b), "event");
    cudaEventRecord(a, s);
    for (int r = 0; r < reps && st == NM_OK; ++r) st = potential_impl(p, rho, phi, s);
    cudaEventRecord(b, s);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != NM_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
    *ms /= (float)(reps > 0 ? reps : 1);
    return NM_OK;
}

// Issue a set of solves: a set seen before is replayed from its CUDA graph
// (captured on its first repeat); a new set runs eagerly.  Graphs bake in the
// pointers and schedules, which form the key.
nm_status run_items(const std::vector<Item>& items, cudaStream_t s) {
    const std::vector<const void*> key = items_key(items);
    for (const Item& it : items) {
        nm_status st = ensure_green(it.p, s);
        if (st != NM_OK) return st;
    }
    if (g_prof_on.load() || fault_timeout_on() || env_int("NM_NO_GRAPHS", 0)) return enqueue_all(items, s);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone)
        return enqueue_all(items, s);             // the caller is capturing: just record
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0;
    bool seen = false;
    {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        for (size_t i = 0; i < g_graphs.size(); ++i)
            if (g_graphs[i].key == key) {
                seen = true;
                exec = g_graphs[i].exec;
                kernels = g_graphs[i].kernels;
                BatchGraph g = g_graphs[i];
                g_graphs.erase(g_graphs.begin() + i);
                g_graphs.push_back(g);
                break;
            }
        if (!seen) {
            if (g_graphs.size() >= kMaxGraphs) {
                if (g_graphs.front().exec) cudaGraphExecDestroy(g_graphs.front().exec);
                g_graphs.erase(g_graphs.begin());
            }
            g_graphs.push_back(BatchGraph{key, nullptr, false});
        }
    }
    if (!seen) return enqueue_all(items, s);
    if (!exec) {
        cudaStream_t cs;
        NM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        nm_status st = NM_OK;
        const uint64_t before = g_launches.load();
        if (e == cudaSuccess) {
            st = enqueue_all(items, cs);
            e = cudaStreamEndCapture(cs, &graph);
        }
        // recorded, not launched: the replay below counts them
        kernels = g_launches.load() - before;
        g_launches.fetch_sub(kernels);
        if (e == cudaSuccess && st == NM_OK) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (st != NM_OK) return st;
        if (e != cudaSuccess) return cuda_fail(e, "graph capture");
        std::lock_guard<std::mutex> lk(g_graph_mu);
        for (auto& g : g_graphs)
            if (g.key == key) {
                g.exec = exec;
                g.captured = true;
                g.kernels = kernels;
            }
    }
    NM_CUDA(cudaGraphLaunch(exec, s), "graph launch");
    count_launches((int)kernels);
    return NM_OK;
}

}  // namespace

extern "C" {

nm_status nm_potential(nm_plan_t p, const void* rho, double* phi, void* stream) {
    if (!p || !rho || !phi) return fail(NM_EINVAL, "nm_potential: null argument");
    if (((uintptr_t)phi & 15) || ((uintptr_t)rho & (p->es - 1)))
        return fail(NM_EINVAL, "nm_potential: phi must be 16-byte aligned and rho element aligned");
    return run_items({Item{p, rho, phi}}, (cudaStream_t)stream);
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
    nm_status st = run_items({Item{p, p->h_rho, p->h_phi}}, s);
    if (st != NM_OK) return st;
    NM_CUDA(cudaMemcpyAsync(phi_host, p->h_phi, cells * sizeof(double), cudaMemcpyDeviceToHost, s), "phi download");
    NM_CUDA(cudaStreamSynchronize(s), "nm_potential_host sync");
    return NM_OK;
}

nm_status nm_potential_host_many(nm_plan_t p, int n, const void* const* rho_host, double* const* phi_host,
                                 void* stream) {
    if (!p || n < 0 || (n > 0 && (!rho_host || !phi_host))) return fail(NM_EINVAL, "nm_potential_host_many: bad arguments");
    for (int i = 0; i < n; ++i)
        if (!rho_host[i] || !phi_host[i]) return fail(NM_EINVAL, "nm_potential_host_many: null entry %d", i);
    if (n == 0) return NM_OK;
    const size_t cells = (size_t)p->L * p->N * p->N * p->N;
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->h_rho2[0]) {
        for (int b = 0; b < 2; ++b) {
            NM_CUDA(cudaMalloc(&p->h_rho2[b], cells * p->es), "host-path staging");
            NM_CUDA(cudaMalloc((void**)&p->h_phi2[b], cells * sizeof(double)), "host-path staging");
            NM_CUDA(cudaEventCreateWithFlags(&p->ev_in[b], cudaEventDisableTiming), "event");
            NM_CUDA(cudaEventCreateWithFlags(&p->ev_solved[b], cudaEventDisableTiming), "event");
            NM_CUDA(cudaEventCreateWithFlags(&p->ev_out[b], cudaEventDisableTiming), "event");
        }
        NM_CUDA(cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking), "copy stream");
        NM_CUDA(cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking), "copy stream");
        p->ws_bytes += 2 * cells * (p->es + sizeof(double));
    }
    nm_status st = ensure_green(p, s);
    if (st != NM_OK) return st;
    // the copy streams start after whatever the caller queued on `stream`
    NM_CUDA(cudaEventRecord(p->ev_solved[0], s), "event");
    NM_CUDA(cudaStreamWaitEvent(p->s_in, p->ev_solved[0], 0), "event wait");
    NM_CUDA(cudaStreamWaitEvent(p->s_out, p->ev_solved[0], 0), "event wait");
    for (int i = 0; i < n; ++i) {
        const int b = i & 1;
        if (i >= 2) {
            // solve i-2 has read rho buffer b; its download has read phi buffer b
            NM_CUDA(cudaStreamWaitEvent(p->s_in, p->ev_solved[b], 0), "event wait");
            NM_CUDA(cudaStreamWaitEvent(s, p->ev_out[b], 0), "event wait");
        }
        NM_CUDA(cudaMemcpyAsync(p->h_rho2[b], rho_host[i], cells * p->es, cudaMemcpyHostToDevice, p->s_in),
                "rho upload");
        NM_CUDA(cudaEventRecord(p->ev_in[b], p->s_in), "event");
        NM_CUDA(cudaStreamWaitEvent(s, p->ev_in[b], 0), "event wait");
        if ((st = run_items({Item{p, p->h_rho2[b], p->h_phi2[b]}}, s)) != NM_OK) return st;
        NM_CUDA(cudaEventRecord(p->ev_solved[b], s), "event");
        NM_CUDA(cudaStreamWaitEvent(p->s_out, p->ev_solved[b], 0), "event wait");
        NM_CUDA(cudaMemcpyAsync(phi_host[i], p->h_phi2[b], cells * sizeof(double), cudaMemcpyDeviceToHost, p->s_out),
                "phi download");
        NM_CUDA(cudaEventRecord(p->ev_out[b], p->s_out), "event");
    }
    NM_CUDA(cudaStreamSynchronize(p->s_out), "nm_potential_host_many sync");
    NM_CUDA(cudaStreamSynchronize(s), "nm_potential_host_many sync");
    return NM_OK;
}

nm_status nm_batch_potential(int n, const nm_plan_t* plans, const void* const* rho,
                             double* const* phi, void* stream) {
    if (n < 0 || (n > 0 && (!plans || !rho || !phi))) return fail(NM_EINVAL, "nm_batch_potential: bad arguments");
    int dev = 0;
    NM_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    std::vector<Item> items;
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || !rho[i] || !phi[i]) return fail(NM_EINVAL, "nm_batch_potential: null entry %d", i);
        if ((uintptr_t)phi[i] & 15) return fail(NM_EINVAL, "nm_batch_potential: phi %d not 16-byte aligned", i);
        if (plans[i]->dev != dev) return fail(NM_EINVAL, "nm_batch_potential: plan %d on another device", i);
        for (int k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return fail(NM_EINVAL, "nm_batch_potential: plan %d repeated", i);
        items.push_back({plans[i], rho[i], phi[i]});
    }
    if (n == 0) return NM_OK;
    return run_items(items, (cudaStream_t)stream);
}

nm_status nm_get_schedule(nm_plan_t p, nm_schedule* out) {
    if (!p || !out) return fail(NM_EINVAL, "nm_get_schedule: null argument");
    *out = p->sched;
    return NM_OK;
}

nm_status nm_set_schedule(nm_plan_t p, const nm_schedule* sc) {
    if (!p || !sc) return fail(NM_EINVAL, "nm_set_schedule: null argument");
    if (!sched_valid(p, *sc))
        return fail(NM_EINVAL,
                    "nm_set_schedule: group must be in [1, %d], radix 16 (P >= 16) or 8, tile 0 or 1, pipeline 0, 1, "
                    "2 (FP32, radix 16, P >= 64, not fused) or 3 (the same with P = 256, tile 0), fuse 0, 1 or 2 (2: FP32 original method, "
                    "radix 16, pipeline 0, 64 <= P <= 512, tile 1 only for P = 128 or 256) or 3 (FP32 original method, "
                    "radix 16, pipeline 0, tile 0, 64 <= P <= 512)",
                    p->npairs);
    nm_status st = ensure_work_slots(p, sc->group);
    if (st != NM_OK) return st;
    graphs_drop_plan(p);
    p->sched = *sc;
    return NM_OK;
}

nm_status nm_autotune(nm_plan_t p, const void* rho, double* phi, int reps, void* stream) {
    if (!p || !rho || !phi) return fail(NM_EINVAL, "nm_autotune: null argument");
    if ((uintptr_t)phi & 15) return fail(NM_EINVAL, "nm_autotune: phi must be 16-byte aligned");
    if (reps < 1) reps = 1;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> groups = {1, 2, p->npairs};
    std::vector<nm_schedule> cands;
    for (int g : groups)
        for (int radix : {16, 8})
            for (int tile : {0, 1})
                for (int pipe : {3, 2, 1, 0})
                    for (int fuse : {3, 2, 1, 0}) {
                        nm_schedule c{g, radix, tile, pipe, fuse};
                        if (!sched_valid(p, c)) continue;
                        bool dup = false;
                        for (auto& o : cands)
                            if (o.group == c.group && o.radix == c.radix && o.tile == c.tile &&
                                o.pipeline == c.pipeline && o.fuse == c.fuse)
                                dup = true;
                        if (!dup) cands.push_back(c);
                    }
    nm_status st = ensure_work_slots(p, p->npairs);
    if (st != NM_OK) return st;
    graphs_drop_plan(p);
    const nm_schedule keep = p->sched;
    nm_schedule best = keep;
    float best_ms = 1e30f;
    for (auto& c : cands) {
        p->sched = c;
        float ms = 0.f;
        st = time_solves(p, rho, phi, reps, s, &ms);
        if (st != NM_OK) {
            p->sched = keep;
            return st;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    p->sched = keep;
    st = nm_set_schedule(p, &best);
    if (st != NM_OK) return st;
    tune_store(p, best);
    return NM_OK;
}

nm_status nm_acceleration_ex(nm_plan_t p, const double* phi, double* g, int coarse_side, int iters,
                             void* stream) {
    if (!p || !phi || !g) return fail(NM_EINVAL, "nm_acceleration: null argument");
    if (((uintptr_t)phi | (uintptr_t)g) & 15) return fail(NM_EINVAL, "nm_acceleration: phi and g must be 16-byte aligned");
    if (coarse_side != NM_ACCEL_COARSE_MEAN && coarse_side != NM_ACCEL_COARSE_FLUX)
        return fail(NM_EINVAL, "nm_acceleration: bad coarse_side %d", coarse_side);
    if (coarse_side == NM_ACCEL_COARSE_FLUX && (iters < 1 || iters > 1000))
        return fail(NM_EINVAL, "nm_acceleration: iters must be in [1, 1000], got %d", iters);
    cudaError_t e = coarse_side == NM_ACCEL_COARSE_FLUX
                        ? run_accel_ex(phi, g, p->L, p->N, p->opt.dx0, (double*)p->vbuf, iters, (cudaStream_t)stream)
                        : run_accel(phi, g, p->L, p->N, p->opt.dx0, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "acceleration");
    return NM_OK;
}

nm_status nm_acceleration(nm_plan_t p, const double* phi, double* g, void* stream) {
    return nm_acceleration_ex(p, phi, g, NM_ACCEL_COARSE_MEAN, 0, stream);
}

nm_status nm_workspace_bytes(nm_plan_t p, size_t* bytes) {
    if (!p || !bytes) return fail(NM_EINVAL, "nm_workspace_bytes: null argument");
    *bytes = p->ws_bytes;
    return NM_OK;
}

nm_status nm_spectrum_bytes(nm_plan_t p, size_t* bytes) {
    if (!p || !bytes) return fail(NM_EINVAL, "nm_spectrum_bytes: null argument");
    // each spectrum: the octant in double, float and double-float
    const size_t per = sizeof(double) + sizeof(float) + sizeof(df);
    size_t b = octant_count(p->N) * per;
    if (p->spec_dbl) b += octant_count(2 * p->N) * per;
    if (p->spec_qdp) b += octant_count(4 * p->N) * per;
    // float rows over all kx, for the FP32 z-seams (P >= 64), and the float
    // octant with fz fastest, for the three-pass form
    if (p->fp32 && p->P >= 64) b += (size_t)(p->N + 1) * (p->N + 1) * p->P * sizeof(float);
    if (p->fp32 && p->P >= 64) b += octant_count(p->N) * sizeof(float);
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
    graphs_drop_plan(p);
    plan_free_buffers(p);
    release_spectrum(p->spec);
    release_spectrum(p->spec_dbl);
    release_spectrum(p->spec_qdp);
    delete p;
    if (e != cudaSuccess) return cuda_fail(e, "nm_destroy sync");
    return NM_OK;
}

uint64_t nm_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

nm_status nm_device_status(int clear) {
    int* w = device_status_word();
    if (!w) return fail(NM_ECUDA, "nm_device_status: no status word");
    NM_CUDA(cudaDeviceSynchronize(), "nm_device_status sync");
    int v = 0;
    NM_CUDA(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost), "nm_device_status read");
    if (clear) NM_CUDA(cudaMemset(w, 0, sizeof(int)), "nm_device_status clear");
    if (v == NM_ETIMEOUT) return fail(NM_ETIMEOUT, "a bounded device-side wait ran out");
    return NM_OK;
}

nm_status nm_debug_fail_alloc(int n) {
    if (n < 0) return fail(NM_EINVAL, "nm_debug_fail_alloc: n must be >= 0");
    g_fail_alloc.store(n);
    return NM_OK;
}

nm_status nm_debug_fault_timeout(int on) {
    g_fault_timeout.store(on ? 1 : 0);
    return NM_OK;
}

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
