// persist.cu -- every step of the solves of a batch in one persistent launch.
//
// The level convolutions of a nested mesh, and the meshes of a batch, are
// independent sub-problems (Sect. 4); within one convolution the passes follow
// one another.  Here all of them -- the restriction sweep, the five transform
// passes of every level pair, the carried interpolation and the assembly of
// every mesh -- are work items of one launch.  The host lays the items out in
// runs ("segments", one per step of one level or mesh) in an order in which
// every item's prerequisites come earlier; the CTAs of the launch take items
// in that order from a device counter (a ticket), wait until the runs they
// depend on are complete (a per-run count of finished items), do the item and
// count it as finished.  Because an item only ever waits for items with
// smaller tickets, and those were taken by CTAs that are already running, the
// launch cannot deadlock whatever the number of resident CTAs.
//
// Every wait is bounded: a CTA that has waited longer than the limit (about 2
// s of clock cycles) writes NM_ETIMEOUT to the device status word and raises
// an abort flag, and every CTA stops at its next item or wait.  The test hook
// nm_debug_fault_timeout makes finished items go uncounted, so the waits run
// out (with a short limit) without any fault.
//
// The item bodies are the device functions of the separate kernels (conv.cuh,
// assemble.cuh) with 256 threads per CTA: the row passes as they are, the
// column passes with 256 E / P columns per item.  A solve through this path
// therefore does the same arithmetic whether it runs alone or in a batch.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/nm.h"
#include "assemble.cuh"
#include "internal.h"

namespace nm {

enum PKind { PK_RESTRICT = 0, PK_XFWD, PK_YFWD, PK_ZSEAM, PK_YINV, PK_XINV, PK_CARRY, PK_ASSEMBLE };

struct PSeg {
    int kind, P;        // step, transform size 2N (N for the non-transform steps' mesh)
    int arg;            // index into the table of its kind
    int tiles;          // items in the run
    int first;          // ticket of its first item
    int wait[2], need[2];   // counters to wait for (-1: none) and the counts they must reach
    int done[2];        // counters bumped by each finished item (-1: none)
    int xt;             // column passes: x tiles per row (fewer for a real pair's half spectrum)
};
struct PPair {
    PairDesc<float> d;
    const float* spec;
    const cpx<float>* tw;
};
struct PRestrict {
    const float* child;     // level m+1 density
    const float* rchild;    // level m+1 restricted covered cells, or null
    float* out;             // level m restricted covered cells ((N/2)^3)
    int lgN;
};
struct PAsm {
    AssembleArgs<float> a;
    int lgN;
};

// Device tables of one batch (one allocation).  ctl[0] = next ticket,
// ctl[1] = abort flag; ctr = the per-run finished-item counters.
struct PTables {
    const PSeg* seg;
    const PPair* pair;
    const PRestrict* rs;
    const CarryArgs<float>* carry;
    const PAsm* as;
    int* ctl;
    int* ctr;
    int* status;
    long long timeout;
    int nseg, total, fault_skip;
};

constexpr int kPersistThreads = 256;
// shared memory of the largest item body: a row pass of P = 512 (twiddles and
// 8 padded lines) or a column pass (twiddles and a 32 KB tile)
constexpr size_t kPersistSmem = 512 * sizeof(cpx<float>) + 8 * (512 + 32) * sizeof(cpx<float>);

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: wait until counter w reaches n; false if the wait ran out or the
// launch was aborted.
__device__ __forceinline__ bool wait_count(const PTables& t, int w, int n) {
    if (w < 0) return true;
    const long long t0 = clock64();
    while (ld_acquire(t.ctr + w) < n) {
        if (ld_acquire(t.ctl + 1) != 0) return false;
        if (clock64() - t0 > t.timeout) {
            atomicExch(t.status, (int)NM_ETIMEOUT);
            atomicExch(t.ctl + 1, 1);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

// Restriction of 2 x 256 covered cells of level m (the k_restrict2 rule),
// with plain loads: the finer level's restricted values are written in this
// launch.
__device__ __forceinline__ void restrict_item(const PRestrict& r, int tile) {
    const int N = 1 << r.lgN, h = N / 2, q = N / 4, lgh = r.lgN - 1;
    const int n = (h * h * h) / 2;
    const int i = tile * kPersistThreads + threadIdx.x;
    if (i >= n) return;
    const int c = 2 * (i & (h / 2 - 1)), b = (i >> (lgh - 1)) & (h - 1), a = i >> (2 * lgh - 1);
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int z = 2 * a + dz, y = 2 * b + dy, x = 2 * c;
            const bool cov = r.rchild && (unsigned)(z - q) < (unsigned)h && (unsigned)(y - q) < (unsigned)h &&
                             (unsigned)(x - q) < (unsigned)h;
            const float* p = cov ? r.rchild + ((size_t)(z - q) * h + (y - q)) * h + (x - q)
                                 : r.child + ((size_t)z * N + y) * N + x;
            const float4 w = *reinterpret_cast<const float4*>(p);
            s0 += w.x + w.y;
            s1 += w.z + w.w;
        }
    r.out[2 * i] = s0 * 0.125f;
    r.out[2 * i + 1] = s1 * 0.125f;
}

// The assembly is light per 256-thread tile, so one of its items does kSub
// consecutive tiles.  The restriction and carry steps stay at one tile per
// item: each level of theirs waits for the previous one, and bigger items
// would lengthen that chain (measured: 0.79 -> 1.0 ms per 6 x 128^3 solve with
// 8 tiles per restriction and carry item).
constexpr int kSub = 8;

// Columns per item of the column passes: 256 threads of P / 16 per column.
template <int P> struct PCols {
    static constexpr int TX = kPersistThreads * 16 / P;
};

template <int P>
__device__ __forceinline__ void transform_item(int kind, const PPair& pp, int tile, int XT, unsigned char* smem) {
    constexpr int E = 16, TX = PCols<P>::TX;
    switch (kind) {
        case PK_XFWD: xfwd_body<float, float, P, E, 0>(pp.d, pp.tw, tile, smem); break;
        case PK_YFWD: ypass_body<float, P, E, TX, false, 0>(pp.d.work, pp.tw, tile % XT, tile / XT, smem); break;
        case PK_ZSEAM: zseam_body<float, P, E, TX, 0>(pp.d, pp.spec, pp.tw, tile % XT, tile / XT, smem); break;
        case PK_YINV: ypass_body<float, P, E, TX, true, 0>(pp.d.work, pp.tw, tile % XT, tile / XT, smem); break;
        default: xinv_body<float, P, E, 0>(pp.d, pp.tw, tile, smem); break;
    }
}

// Tickets taken per grab: one atomic per chunk of consecutive items.  A CTA
// does its chunk's items in ticket order and reports finished items per run
// (one release-add per run it leaves, and at the chunk's end) -- always before
// it waits for anything, so no count it holds back can block another CTA.
constexpr int kChunk = 4;

__global__ void __launch_bounds__(kPersistThreads, 4) k_persist(const __grid_constant__ PTables t) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_base, s_ok;
    int cur = -1;                       // run whose waits this CTA has passed
    PSeg sgc{};                         // and its description
    int pend = 0, pd0 = -1, pd1 = -1;   // thread 0: finished items not yet reported, and their counters
    auto flush = [&]() {
        if (pend && !t.fault_skip) {
            if (pd0 >= 0) red_release(t.ctr + pd0, pend);
            if (pd1 >= 0) red_release(t.ctr + pd1, pend);
        }
        pend = 0;
    };
    for (;;) {
        if (threadIdx.x == 0) {
            const int b = atomicAdd(t.ctl, kChunk);
            s_base = ld_acquire(t.ctl + 1) != 0 ? t.total : b;
        }
        __syncthreads();
        const int base = s_base;
        if (base >= t.total) break;
        const int end = base + kChunk < t.total ? base + kChunk : t.total;
        bool stop = false;
        for (int item = base; item < end; ++item) {
            // the run holding this ticket: usually the one of the previous item
            int lo = cur;
            if (lo < 0 || item < sgc.first || item >= sgc.first + sgc.tiles) {
                lo = 0;
                int hi = t.nseg - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (t.seg[mid].first <= item) lo = mid;
                    else hi = mid - 1;
                }
                if (lo != cur) sgc = t.seg[lo];
            }
            const PSeg& sg = sgc;
            if (lo != cur) {
                if (threadIdx.x == 0) {
                    flush();
                    pd0 = sg.done[0];
                    pd1 = sg.done[1];
                    s_ok = wait_count(t, sg.wait[0], sg.need[0]) && wait_count(t, sg.wait[1], sg.need[1]);
                }
                __syncthreads();
                if (!s_ok) {
                    stop = true;
                    break;
                }
                cur = lo;
            }
            const int tile = item - sg.first;
            switch (sg.kind) {
                case PK_RESTRICT: restrict_item(t.rs[sg.arg], tile); break;
                case PK_CARRY:
                    carry_body<float>(t.carry[sg.arg], (size_t)tile * kPersistThreads + threadIdx.x,
                                      kPersistThreads, (size_t)(tile + 1) * kPersistThreads);
                    break;
                case PK_ASSEMBLE: {
                    const PAsm& pa = t.as[sg.arg];
                    const int rows_cta = kPersistThreads / ((1 << pa.lgN) >> 2);
                    const size_t rows_total = ((size_t)pa.a.levels << (2 * pa.lgN));
                    for (int u = 0; u < kSub; ++u) {
                        const size_t rb = ((size_t)tile * kSub + u) * rows_cta;
                        if (rb >= rows_total) break;
                        assemble_rows_body<float>(pa.a, pa.lgN, rb, (size_t)1 << 40, smem);
                    }
                    break;
                }
                default: {
                    const PPair& pp = t.pair[sg.arg];
                    switch (sg.P) {
                        case 64: transform_item<64>(sg.kind, pp, tile, sg.xt, smem); break;
                        case 128: transform_item<128>(sg.kind, pp, tile, sg.xt, smem); break;
                        case 256: transform_item<256>(sg.kind, pp, tile, sg.xt, smem); break;
                        default: transform_item<512>(sg.kind, pp, tile, sg.xt, smem); break;
                    }
                }
            }
            __syncthreads();   // the item's results are written (and its shared memory free)
            if (threadIdx.x == 0) ++pend;
        }
        if (threadIdx.x == 0) flush();
        if (stop) break;
    }
}

// ---------------------------------------------------------------- host side
namespace {

int lg2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

size_t up16(size_t b) { return (b + 15) & ~(size_t)15; }

}  // namespace

// A batch laid out for k_persist: host copies of the tables and the device
// allocation holding them.
struct PersistBatch {
    std::vector<PSeg> seg;
    std::vector<PPair> pair;
    std::vector<PRestrict> rs;
    std::vector<CarryArgs<float>> carry;
    std::vector<PAsm> as;
    int ncounters = 0;
    int total = 0;
    void* dev = nullptr;
    size_t dev_bytes = 0;
    PTables t{};
    int grid = 0;
};

// Lays out the items of `meshes`; returns false if a mesh cannot take this
// path (checked before anything is allocated).
bool persist_layout(const std::vector<PersistMesh>& meshes, PersistBatch& b) {
    const int nm_ = (int)meshes.size();
    for (const PersistMesh& m : meshes) {
        if (m.P < 64 || m.P > 512 || m.L < 1 || m.L > NM_MAX_LEVELS || m.group < 1) return false;
        if (((uintptr_t)m.rho & 15) || ((uintptr_t)m.restr & 15) || ((uintptr_t)m.phi & 15)) return false;
        for (const PairDesc<float>& d : m.pairs)
            if (d.src[0].mode != SRC_FULL) return false;
    }
    auto add = [&](int kind, int P, int arg, int tiles, int w0, int n0, int w1, int n1, int d0, int d1) {
        PSeg s{};
        s.kind = kind;
        s.P = P;
        s.arg = arg;
        s.tiles = tiles;
        s.first = b.total;
        s.wait[0] = w0; s.need[0] = n0;
        s.wait[1] = w1; s.need[1] = n1;
        s.done[0] = d0; s.done[1] = d1;
        b.total += tiles;
        b.seg.push_back(s);
        return (int)b.seg.size() - 1;
    };
    // counters: one per run (its own index), plus one per mesh counting every
    // finished x-inverse item of that mesh (the assembly waits for all)
    std::vector<int> rs_seg(nm_ * NM_MAX_LEVELS, -1);
    std::vector<int> xi_seg(nm_ * NM_MAX_LEVELS, -1), xi_tiles(nm_, 0);
    std::vector<int> ca_seg(nm_ * NM_MAX_LEVELS, -1);
    // the per-mesh x-inverse counters come after the run counters; their
    // indices are fixed once the number of runs is known, so record the runs
    // that bump them and patch afterwards
    std::vector<std::pair<int, int>> xi_patch;   // (segment, mesh)
    std::vector<std::pair<int, int>> asm_patch;
    // 1. restriction, finest covered level first, every mesh
    for (int i = 0; i < nm_; ++i) {
        const PersistMesh& m = meshes[i];
        const int N = m.P / 2, h = N / 2;
        const size_t N3 = (size_t)N * N * N, h3 = (size_t)h * h * h;
        const int tiles = (int)((h3 / 2 + kPersistThreads - 1) / kPersistThreads);
        for (int lv = m.L - 2; lv >= 0; --lv) {
            PRestrict r;
            r.child = m.rho + (size_t)(lv + 1) * N3;
            r.rchild = lv + 1 < m.L - 1 ? m.restr + (size_t)(lv + 1) * h3 : nullptr;
            r.out = m.restr + (size_t)lv * h3;
            r.lgN = lg2(N);
            b.rs.push_back(r);
            const int w = lv + 1 < m.L - 1 ? rs_seg[i * NM_MAX_LEVELS + lv + 1] : -1;
            const int id = add(PK_RESTRICT, N, (int)b.rs.size() - 1, tiles, w, w >= 0 ? b.seg[w].tiles : 0, -1, 0,
                               -2, -1);
            b.seg[id].done[0] = id;
            rs_seg[i * NM_MAX_LEVELS + lv] = id;
        }
    }
    // 2. the transform passes, round by round (a round = the pairs that
    // occupy a mesh's work slots at once), pass by pass, every mesh
    std::vector<int> pair_base(nm_);
    for (int i = 0; i < nm_; ++i) {
        pair_base[i] = (int)b.pair.size();
        for (const PairDesc<float>& d : meshes[i].pairs) b.pair.push_back(PPair{d, meshes[i].spec, meshes[i].tw});
    }
    int rounds = 0;
    for (const PersistMesh& m : meshes) rounds = std::max(rounds, ((int)m.pairs.size() + m.group - 1) / m.group);
    std::vector<int> seg_of(b.pair.size() * 5, -1);
    for (int r = 0; r < rounds; ++r) {
        for (int pass = 0; pass < 5; ++pass) {
            for (int i = 0; i < nm_; ++i) {
                const PersistMesh& m = meshes[i];
                const int P = m.P, N = P / 2, LINES = 256 / (P / 16), TX = kPersistThreads * 16 / P;
                for (int q = r * m.group; q < (r + 1) * m.group && q < (int)m.pairs.size(); ++q) {
                    const int pi = pair_base[i] + q;
                    PPair& pp = b.pair[pi];
                    pp.d.work = (cpx<float>*)m.work + (size_t)(q - r * m.group) * (size_t)(P / 2) * P * P;
                    // a real pair: the column passes stop at the tile holding kx = N
                    pp.d.half = pp.d.src[1].mode == SRC_NONE ? 1 : 0;
                    const int XT = pp.d.half ? (P / 2) / TX + 1 : P / TX;
                    int kind = PK_XFWD + pass, tiles = 0, w0 = -1, n0 = 0, w1 = -1, n1 = 0;
                    switch (kind) {
                        case PK_XFWD:
                            tiles = N * N / LINES;
                            // the level's restricted covered cells
                            if (q < m.L - 1 && rs_seg[i * NM_MAX_LEVELS + q] >= 0) {
                                w0 = rs_seg[i * NM_MAX_LEVELS + q];
                                n0 = b.seg[w0].tiles;
                            }
                            // the work slot's previous pair is done with it
                            if (q >= m.group) {
                                w1 = seg_of[(size_t)(pi - m.group) * 5 + 4];
                                n1 = b.seg[w1].tiles;
                            }
                            break;
                        case PK_YFWD: tiles = XT * N; break;
                        case PK_ZSEAM: tiles = XT * P; break;
                        case PK_YINV: tiles = XT * N; break;
                        default: tiles = N * N / LINES; break;
                    }
                    if (pass > 0) {
                        w0 = seg_of[(size_t)pi * 5 + pass - 1];
                        n0 = b.seg[w0].tiles;
                    }
                    const int id = add(kind, P, pi, tiles, w0, n0, w1, n1, -2, -1);
                    b.seg[id].done[0] = id;
                    b.seg[id].xt = XT;
                    seg_of[(size_t)pi * 5 + pass] = id;
                    if (kind == PK_XINV) {
                        xi_seg[i * NM_MAX_LEVELS + q] = id;
                        xi_tiles[i] += tiles;
                        xi_patch.push_back({id, i});
                    }
                }
            }
        }
    }
    // 3. the carried Eqs. 3-6 interpolation, level by level, every mesh
    int max_carry = 0;
    for (const PersistMesh& m : meshes)
        if (m.carry) max_carry = std::max(max_carry, m.L - 2);
    for (int n = 1; n <= max_carry; ++n) {
        for (int i = 0; i < nm_; ++i) {
            const PersistMesh& m = meshes[i];
            if (!m.carry || n + 1 >= m.L) continue;
            const int N = m.P / 2;
            const size_t nc = N / 2 + 2, nc3 = nc * nc * nc;
            CarryArgs<float> c{};
            if (n == 1) {
                c.prev = m.asm_args.interp[0];
                c.prev_origin = m.asm_args.interp_origin[0];
                c.prev_extent = m.asm_args.interp_extent[0];
            } else {
                c.prev = m.carry + (size_t)(n - 2) * nc3;
                c.prev_origin = N / 4 - 1;
                c.prev_extent = (int)nc;
            }
            c.hole = m.asm_args.interp[n];
            c.hole_origin = m.asm_args.interp_origin[n];
            c.hole_extent = m.asm_args.interp_extent[n];
            c.out = m.carry + (size_t)(n - 1) * nc3;
            c.N = N;
            b.carry.push_back(c);
            const int wprev = n == 1 ? xi_seg[i * NM_MAX_LEVELS + 0] : ca_seg[i * NM_MAX_LEVELS + n - 1];
            const int whole = xi_seg[i * NM_MAX_LEVELS + n];
            const int tiles = (int)((nc3 + kPersistThreads - 1) / kPersistThreads);
            const int id = add(PK_CARRY, N, (int)b.carry.size() - 1, tiles, wprev, b.seg[wprev].tiles, whole,
                               b.seg[whole].tiles, -2, -1);
            b.seg[id].done[0] = id;
            ca_seg[i * NM_MAX_LEVELS + n] = id;
        }
    }
    // 4. the assembly of every mesh, after all its transforms and its carry
    for (int i = 0; i < nm_; ++i) {
        const PersistMesh& m = meshes[i];
        const int N = m.P / 2, team = N / 4, rows_cta = kPersistThreads / team;
        PAsm pa;
        pa.a = m.asm_args;
        pa.lgN = lg2(N);
        if (m.carry) {
            const size_t nc = N / 2 + 2, nc3 = nc * nc * nc;
            for (int n = 1; n + 1 < m.L; ++n) {
                pa.a.interp[n] = m.carry + (size_t)(n - 1) * nc3;
                pa.a.interp_origin[n] = N / 4 - 1;
                pa.a.interp_extent[n] = (int)nc;
            }
        }
        b.as.push_back(pa);
        const int tiles = (int)(((size_t)N * N * m.L / rows_cta + kSub - 1) / kSub);
        const int wcarry = (m.carry && m.L > 2) ? ca_seg[i * NM_MAX_LEVELS + m.L - 2] : -1;
        const int id = add(PK_ASSEMBLE, N, (int)b.as.size() - 1, tiles, -3, xi_tiles[i], wcarry,
                           wcarry >= 0 ? b.seg[wcarry].tiles : 0, -1, -1);
        asm_patch.push_back({id, i});
    }
    // per-mesh x-inverse counters
    const int nseg = (int)b.seg.size();
    for (auto& pr : xi_patch) b.seg[pr.first].done[1] = nseg + pr.second;
    for (auto& pr : asm_patch) b.seg[pr.first].wait[0] = nseg + pr.second;
    b.ncounters = nseg + nm_;
    // every wait is on an earlier run (or a mesh counter fed only by earlier runs)
    for (int s = 0; s < nseg; ++s)
        for (int k = 0; k < 2; ++k)
            if (b.seg[s].wait[k] >= nseg) {
                for (auto& pr : xi_patch)
                    if (nseg + pr.second == b.seg[s].wait[k] && pr.first >= s) return false;
            } else if (b.seg[s].wait[k] >= s) {
                return false;
            }
    return true;
}

// Uploads the tables (synchronously; outside any stream capture) and sizes
// the grid.
cudaError_t persist_upload(PersistBatch& b) {
    const size_t o_seg = 0;
    const size_t o_pair = up16(o_seg + b.seg.size() * sizeof(PSeg));
    const size_t o_rs = up16(o_pair + b.pair.size() * sizeof(PPair));
    const size_t o_carry = up16(o_rs + b.rs.size() * sizeof(PRestrict));
    const size_t o_as = up16(o_carry + b.carry.size() * sizeof(CarryArgs<float>));
    const size_t o_ctl = up16(o_as + b.as.size() * sizeof(PAsm));
    const size_t o_ctr = o_ctl + 16;
    const size_t bytes = up16(o_ctr + (size_t)b.ncounters * sizeof(int));
    std::vector<unsigned char> h(bytes, 0);
    if (!b.seg.empty()) std::memcpy(h.data() + o_seg, b.seg.data(), b.seg.size() * sizeof(PSeg));
    if (!b.pair.empty()) std::memcpy(h.data() + o_pair, b.pair.data(), b.pair.size() * sizeof(PPair));
    if (!b.rs.empty()) std::memcpy(h.data() + o_rs, b.rs.data(), b.rs.size() * sizeof(PRestrict));
    if (!b.carry.empty()) std::memcpy(h.data() + o_carry, b.carry.data(), b.carry.size() * sizeof(CarryArgs<float>));
    if (!b.as.empty()) std::memcpy(h.data() + o_as, b.as.data(), b.as.size() * sizeof(PAsm));
    cudaError_t e = cudaMalloc(&b.dev, bytes);
    if (e != cudaSuccess) return e;
    b.dev_bytes = bytes;
    e = cudaMemcpy(b.dev, h.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    unsigned char* d = (unsigned char*)b.dev;
    b.t.seg = (const PSeg*)(d + o_seg);
    b.t.pair = (const PPair*)(d + o_pair);
    b.t.rs = (const PRestrict*)(d + o_rs);
    b.t.carry = (const CarryArgs<float>*)(d + o_carry);
    b.t.as = (const PAsm*)(d + o_as);
    b.t.ctl = (int*)(d + o_ctl);
    b.t.ctr = (int*)(d + o_ctr);
    b.t.nseg = (int)b.seg.size();
    b.t.total = b.total;
    static PerDevice<KernelPrep> prep;
    const KernelPrep kp = prep.get(current_device(), []() {
        KernelPrep r;
        r.err = cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPersistSmem);
        if (r.err == cudaSuccess)
            r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.occ, k_persist, kPersistThreads, kPersistSmem);
        return r;
    }, KernelPrep{cudaErrorInvalidDevice, 0});
    if (kp.err != cudaSuccess) return kp.err;
    b.grid = std::max(1, kp.occ) * sm_count();
    const int chunks = (b.total + kChunk - 1) / kChunk;
    if (b.grid > chunks) b.grid = std::max(1, chunks);
    return cudaSuccess;
}

// Zeroes the ticket, abort flag and counters and launches the batch.
cudaError_t persist_launch(PersistBatch& b, cudaStream_t s) {
    if (b.total == 0) return cudaSuccess;
    const size_t zero_bytes = (size_t)((unsigned char*)b.t.ctr - (unsigned char*)b.t.ctl) +
                              (size_t)b.ncounters * sizeof(int);
    cudaError_t e = cudaMemsetAsync(b.t.ctl, 0, zero_bytes, s);
    if (e != cudaSuccess) return e;
    b.t.status = device_status_word();
    if (!b.t.status) return cudaErrorMemoryAllocation;
    b.t.fault_skip = fault_timeout_on() ? 1 : 0;
    // about 2 s of SM clock cycles; 0.1 s under the fault hook
    b.t.timeout = b.t.fault_skip ? 200000000LL : 4000000000LL;
    ProfScope ps("persist_f32", (int)b.pair.size(), s);
    k_persist<<<b.grid, kPersistThreads, kPersistSmem, s>>>(b.t);
    count_launches(1);
    return cudaGetLastError();
}

PersistBatch* persist_new() { return new PersistBatch(); }
void persist_free(PersistBatch* b) {
    if (!b) return;
    cudaFree(b->dev);
    delete b;
}
int persist_items(const PersistBatch* b) { return b ? b->total : 0; }

}  // namespace nm
