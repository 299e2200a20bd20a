// conv.cuh -- the per-level zero-padded convolution of Sect. 3 as five passes.
//
// Each launch transforms a set of "pairs": two real fields packed as one
// complex field re + i*im.  The kernel spectrum is real (the inverse distance
// of Eq. 10 is real and even on the doubled domain of Fig. 4), so the
// convolution of the packed field is conv(re) + i*conv(im) and both come back
// from one complex transform.
//
// Domain: FFT size P per axis.  Three geometries (GM) share the code:
//   0 level grid: an N^3 block, N = P/2, sits at [0, N) (Fig. 4: the active
//       region 1, regions 2-4 zero);
//   1 doubled fine grid (Sect. 7 / Fig. 16): the fine level's N^3 block sits
//       at [N/2, 3N/2) of a 2N-cell grid, N = P/4, period P = 4N; any period
//       >= 3N - 1 keeps the sum isolated;
//   2 quadrupled grid (Appendix B / Fig. App0): a level's N^3 block sits at
//       [3N/2, 5N/2) of a 4N-cell grid spanning the level two steps coarser,
//       N = P/8, period P = 8N (>= 5N - 1).
// In all three the output window is [0, P/2) per axis.
//
// Work buffer of one pair: [Z = P/2][P][P] complex, index (z*P + y)*P + x.
//   1 xfwd : rows (z, y) of the input block: mask, scale, pack, pad, FFT along x
//   2 yfwd : slabs z of the input block, columns x: FFT along y (input pruned)
//   3 zseam: lines (ky, kx): FFT along z, times the spectrum, inverse along z
//   4 yinv : slabs z < P/2: inverse along y, keep y < P/2
//   5 xinv : rows (z, y) < P/2: inverse along x, keep x < P/2, scatter outputs
#pragma once
#include "dfloat.cuh"
#include "fft.cuh"

namespace nm {

enum SrcMode { SRC_NONE = 0, SRC_FULL = 1, SRC_HOLE = 2 };
enum DstKind { DST_NONE = 0, DST_GRID = 1, DST_CROP = 2 };

// One real input field: a level's density block (extent NL = N), the mean of
// the finer level in its covered cells (restr, (NL/2)^3, may be null), the mode
// (full grid, or hole grid with the covered cells emptied, Fig. 5) and the
// factor turning density into the scaled mass the spectrum expects.
struct SrcField {
    const void* rho;
    const void* restr;
    int mode;
    double scale;
};
struct DstField {
    void* out;   // T*, extent P/2 grid or the hole crop
    int kind;
};
template <typename T> struct PairDesc {
    cpx<T>* work;
    SrcField src[2];
    DstField dst[2];
    // 1: the pair carries one real field (its second slot is empty, as for
    // the finest level of Eq. 14).  Its transform along x is then Hermitian,
    // X[P - kx] = conj X[kx], and so is every (z, y) row of the result: the
    // y and z passes skip the column tiles above kx = P/2 and the x-inverse
    // reads kx > P/2 as conj X[P - kx].  Set by the launcher for the
    // schedules that honour it; 0 everywhere else.
    int half;
};

constexpr int kMaxPairs = 64;
template <typename T> struct ConvArgs {
    PairDesc<T> pair[kMaxPairs];
    const T* spec;          // unit spectrum octant (P/2+1)^3, [kz][ky][kx]
    const cpx<T>* tw;       // twiddle table, P entries
};

// Stage the twiddles of a size-P line transform with E values per thread:
// the plain table (P entries), or with PT in the per-pass order (P - E).
template <int P, int E, bool PT = false, typename T>
__device__ __forceinline__ void load_twiddles(cpx<T>* sm_tw, const cpx<T>* tw) {
    if constexpr (PT) fill_pass_twiddles<P, E>(sm_tw, [&](int t) { return tw[t]; });
    else for (int i = threadIdx.x; i < P; i += blockDim.x) sm_tw[i] = tw[i];
}

// Density of a real field at block cell (z, y, x), already scaled.  All in
// the pass precision T.
template <typename T, typename TIN>
__device__ __forceinline__ T src_value(const SrcField& f, T scale, int NL, int z, int y, int x) {
    if (f.mode == SRC_NONE) return T(0);
    const int q = NL / 4, h = NL / 2;
    const bool cov = (unsigned)(z - q) < (unsigned)h && (unsigned)(y - q) < (unsigned)h &&
                     (unsigned)(x - q) < (unsigned)h;
    T v;
    if (cov) {
        if (f.mode == SRC_HOLE) return T(0);
        if (f.restr)
            v = conv_in<T, TIN>(((const TIN*)f.restr)[((size_t)(z - q) * h + (y - q)) * h + (x - q)]);
        else
            v = conv_in<T, TIN>(((const TIN*)f.rho)[((size_t)z * NL + y) * NL + x]);
    } else {
        v = conv_in<T, TIN>(((const TIN*)f.rho)[((size_t)z * NL + y) * NL + x]);
    }
    return v * scale;
}

// Both fields of a pair at block cell (z, y, x), scaled.  When the pair is a
// level's full and hole grids (Fig. 5) the density is loaded once.
template <typename T, typename TIN>
__device__ __forceinline__ cpx<T> src_pair(const SrcField& f0, const SrcField& f1, T s0, T s1, int NL,
                                           int z, int y, int x) {
    if (f0.mode == SRC_FULL && f1.mode == SRC_HOLE && f0.rho == f1.rho) {
        const int q = NL / 4, h = NL / 2;
        const bool cov = (unsigned)(z - q) < (unsigned)h && (unsigned)(y - q) < (unsigned)h &&
                         (unsigned)(x - q) < (unsigned)h;
        T v;
        if (cov && f0.restr)
            v = conv_in<T, TIN>(((const TIN*)f0.restr)[((size_t)(z - q) * h + (y - q)) * h + (x - q)]);
        else
            v = conv_in<T, TIN>(((const TIN*)f0.rho)[((size_t)z * NL + y) * NL + x]);
        return {v * s0, cov ? T(0) : v * s1};
    }
    return {src_value<T, TIN>(f0, s0, NL, z, y, x), src_value<T, TIN>(f1, s1, NL, z, y, x)};
}

template <int P, int E, int GM> struct Geo {
    static_assert(GM != 2 || E == 16, "the quadrupled grid needs 16 values per thread");
    static constexpr int NIN = GM == 0 ? P / 2 : GM == 1 ? P / 4 : P / 8;         // input block extent
    static constexpr int OFF = GM == 0 ? 0 : GM == 1 ? P / 8 : 3 * P / 16;        // its offset in the domain
    static constexpr int NOUT = P / 2;                                            // output window
    // first-pass register r holds x[j + r P/E]: nonzero only for these r
    __host__ __device__ static constexpr bool live(int r) {
        return GM == 0 ? (r < E / 2) : GM == 1 ? (r >= E / 8 && r < 3 * E / 8) : (r >= 3 * E / 16 && r < 5 * E / 16);
    }
    // the same as a register mask, for the first pass of a forward transform
    __host__ __device__ static constexpr unsigned live_mask() {
        unsigned m = 0;
        for (int r = 0; r < E; ++r)
            if (live(r)) m |= 1u << r;
        return m;
    }
    static constexpr unsigned LIVE = live_mask();
};

// ---------------------------------------------------------------- pass 1
// The body of each pass is a device function of (pair, tile, shared memory)
// that its kernel calls with its block indices, and that the persistent
// batch kernel (persist.cu) calls for the work items it takes; 256 threads
// for the row passes, TX P / E for the column passes.
template <typename T, typename TIN, int P, int E, int GM>
__device__ __forceinline__ void xfwd_body(const PairDesc<T>& d, const cpx<T>* tw, unsigned tile,
                                          unsigned char* smem_raw) {
    using G = Geo<P, E, GM>;
    constexpr int TPL = P / E;
    constexpr int LINES = 256 / TPL;
    cpx<T>* sm_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* sm_lines = sm_tw + P;
    const int line = threadIdx.x / TPL, j = threadIdx.x % TPL;
    const int row0 = tile * LINES;
    const int row = row0 + line;
    const bool valid = row < G::NIN * G::NIN;
    const int zi = row / G::NIN, yi = row % G::NIN;
    const T s0 = (T)d.src[0].scale, s1 = (T)d.src[1].scale;
    cpx<T> v[E];
    // A level's full and hole grids share one density: the CTA's rows are
    // contiguous in it, so stage them through shared memory with 16-byte
    // loads (more bytes in flight per instruction than the transform's
    // strided layout allows) and read the transform layout from there.
    const bool staged = GM == 0 && d.src[0].mode == SRC_FULL && d.src[0].rho == d.src[1].rho &&
                        (d.src[1].mode == SRC_HOLE || d.src[1].mode == SRC_NONE) &&
                        (((uintptr_t)d.src[0].rho & 15) == 0);
    if (staged) {
        constexpr int NIN = G::NIN, VEC = 16 / sizeof(TIN);
        T* stage = reinterpret_cast<T*>(sm_lines);
        const int rows = min(LINES, NIN * NIN - row0);
        const TIN* base = (const TIN*)d.src[0].rho + (size_t)row0 * NIN;
        for (int i = threadIdx.x * VEC; i < rows * NIN; i += blockDim.x * VEC) {
            TIN tmp[VEC];
            *reinterpret_cast<int4*>(tmp) = __ldg(reinterpret_cast<const int4*>(base + i));
#pragma unroll
            for (int q = 0; q < VEC; ++q) stage[i + q] = conv_in<T, TIN>(tmp[q]);
        }
        __syncthreads();
        const int q = NIN / 4, h = NIN / 2;
        const bool row_cov = (unsigned)(zi - q) < (unsigned)h && (unsigned)(yi - q) < (unsigned)h;
        const bool hole = d.src[1].mode == SRC_HOLE;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            v[r] = {T(0), T(0)};
            if (G::live(r) && valid) {
                const int xi = j + r * (P / E);
                const T val = stage[line * NIN + xi];
                const bool cov = row_cov && (unsigned)(xi - q) < (unsigned)h;
                T full = val;
                if (cov && d.src[0].restr)
                    full = conv_in<T, TIN>(((const TIN*)d.src[0].restr)[((size_t)(zi - q) * h + (yi - q)) * h + (xi - q)]);
                v[r].re = full * s0;
                v[r].im = (hole && !cov) ? val * s1 : T(0);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            v[r] = {T(0), T(0)};
            if (G::live(r) && valid) {
                const int xi = j + r * (P / E) - G::OFF;
                v[r] = src_pair<T, TIN>(d.src[0], d.src[1], s0, s1, G::NIN, zi, yi, xi);
            }
        }
    }
    load_twiddles<P, E, true>(sm_tw, tw);   // after the density loads are out
    __syncthreads();
    fft_line<T, P, E, false, G::LIVE, false, true>(v, j, sm_tw,
                                             LineView<T, 1, true, Log2E<E>::value>{sm_lines + line * (P + P / E)});
    if (valid) {
        cpx<T>* dst = d.work + ((size_t)(zi + G::OFF) * P + (yi + G::OFF)) * P;
#pragma unroll
        for (int s = 0; s < E; ++s) dst[out_index<P, E>(j, s)] = v[s];
    }
}

template <typename T, typename TIN, int P, int E, int GM>
__global__ void __launch_bounds__(256) k_xfwd(const __grid_constant__ ConvArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    xfwd_body<T, TIN, P, E, GM>(a.pair[blockIdx.y], a.tw, blockIdx.x, smem_raw);
}

// Pass 1 as a persistent pipeline (level grids whose pairs are a level's full
// and hole fields, or a full field alone; density 16-byte aligned; P >= 64).
// A tile is the LINES consecutive density rows that one round of the CTA
// transforms; each CTA walks tiles blockIdx.x, + gridDim.x, ... across all
// pairs and fetches tile k+1 into the other half of a two-tile staging buffer
// with asynchronous 16-byte copies (cp.async, completion by wait_group, which
// the hardware resolves) while it transforms tile k, so the density loads
// overlap the transforms instead of preceding them.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Staged density rows of k_xfwd_pipe: LINES rows of NIN values, each row
// padded by 64 bytes so that the two rows a warp reads (16 threads each) start
// half a bank cycle apart.
template <typename TIN, int P, int E> struct XfwdStage {
    static constexpr int LINES = 256 / (P / E), NIN = P / 2;
    static constexpr int PITCH = NIN + 64 / (int)sizeof(TIN);
    static constexpr int ELEMS = LINES * PITCH;       // one of the two buffers
};

template <typename T, typename TIN, int P, int E>
__global__ void __launch_bounds__(256) k_xfwd_pipe(const __grid_constant__ ConvArgs<T> a, int npairs) {
    using G = Geo<P, E, 0>;
    using S = XfwdStage<TIN, P, E>;
    constexpr int TPL = P / E, LINES = 256 / TPL, NIN = G::NIN;
    constexpr int TILE = LINES * NIN;                 // density values per tile
    constexpr int TILES = NIN * NIN / LINES;          // tiles per pair
    constexpr int VEC = 16 / sizeof(TIN);
    static_assert((NIN * NIN) % LINES == 0 && TILE % (256 * VEC) == 0 && NIN % VEC == 0, "tile shape");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* sm_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* sm_lines = sm_tw + P;
    TIN* stage = reinterpret_cast<TIN*>(sm_lines + LINES * (P + P / E));   // [2][LINES][PITCH]
    load_twiddles<P, E, true>(sm_tw, a.tw);
    const int line = threadIdx.x / TPL, j = threadIdx.x % TPL;
    const int total = npairs * TILES;
    auto issue = [&](int t, int b) {
        const int pr = t / TILES, row0 = (t - pr * TILES) * LINES;
        const TIN* src = (const TIN*)a.pair[pr].src[0].rho + (size_t)row0 * NIN;
        TIN* dst = stage + b * S::ELEMS;
#pragma unroll
        for (int i = threadIdx.x * VEC; i < TILE; i += 256 * VEC) {
            const int row = i / NIN;
            cp_async16(dst + row * S::PITCH + (i - row * NIN), src + i);
        }
    };
    int t = blockIdx.x;
    if (t < total) issue(t, 0);
    cp_async_commit();
    for (int k = 0; t < total; ++k, t += gridDim.x) {
        if (t + (int)gridDim.x < total) issue(t + gridDim.x, (k + 1) & 1);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const int pr = t / TILES, row0 = (t - pr * TILES) * LINES;
        const PairDesc<T>& d = a.pair[pr];
        const T s0 = (T)d.src[0].scale, s1 = (T)d.src[1].scale;
        const int row = row0 + line;
        const int zi = row / NIN, yi = row % NIN;
        const int q = NIN / 4, h = NIN / 2;
        const bool row_cov = (unsigned)(zi - q) < (unsigned)h && (unsigned)(yi - q) < (unsigned)h;
        const bool hole = d.src[1].mode == SRC_HOLE;
        const TIN* st = stage + (k & 1) * S::ELEMS + line * S::PITCH;
        cpx<T> v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            v[r] = {T(0), T(0)};
            if (G::live(r)) {
                const int xi = j + r * (P / E);
                const T val = conv_in<T, TIN>(st[xi]);
                const bool cov = row_cov && (unsigned)(xi - q) < (unsigned)h;
                T full = val;
                if (cov && d.src[0].restr)
                    full = conv_in<T, TIN>(((const TIN*)d.src[0].restr)[((size_t)(zi - q) * h + (yi - q)) * h + (xi - q)]);
                v[r].re = full * s0;
                v[r].im = (hole && !cov) ? val * s1 : T(0);
            }
        }
        fft_line<T, P, E, false, G::LIVE, false, true>(v, j, sm_tw,
                                                 LineView<T, 1, true, Log2E<E>::value>{sm_lines + line * (P + P / E)});
        cpx<T>* out = d.work + ((size_t)zi * P + yi) * P;
#pragma unroll
        for (int s = 0; s < E; ++s) out[out_index<P, E>(j, s)] = v[s];
        __syncthreads();   // this half of the stage and the line scratch are free again
    }
}

// Pass 1 as the persistent pipeline with two rows per thread (FP32 density):
// rows (z, y) and (z, y + 1), y even, go through identical arithmetic, so the
// thread carries them as one transform over cpx<f2> (lane 0 = row y, lane 1 =
// row y + 1), as the paired z-seam does for two columns; each shared-memory
// access and twiddle read then serves both rows.  128 threads = the LINES / 2 row pairs of one staged tile.  A real
// pair (d.half) writes only the columns the y and z passes read (kx < P/2 +
// 32: up to the widest column tile holding kx = P/2).
template <int P>
__global__ void __launch_bounds__(128, 4) k_xfwd_pipe2(const __grid_constant__ ConvArgs<float> a, int npairs) {
    using T = float;
    using TIN = float;
    constexpr int E = 16;
    using G = Geo<P, E, 0>;
    using S = XfwdStage<TIN, P, E>;
    constexpr int TPL = P / E, LINES = 256 / TPL, LP = LINES / 2, NIN = G::NIN;
    constexpr int TILE = LINES * NIN;
    constexpr int TILES = NIN * NIN / LINES;
    constexpr int VEC = 4;
    static_assert((NIN * NIN) % LINES == 0 && TILE % (128 * VEC) == 0 && NIN % VEC == 0 && LP * TPL == 128,
                  "tile shape");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<f2>* sm_tw = reinterpret_cast<cpx<f2>*>(smem_raw);
    cpx<f2>* sm_lines = sm_tw + P;
    TIN* stage = reinterpret_cast<TIN*>(sm_lines + LP * (P + P / E));   // [2][LINES][PITCH]
    fill_pass_twiddles<P, E>(sm_tw, [&](int t) {
        const cpx<float> w = a.tw[t];
        return cpx<f2>{f2(w.re, w.re), f2(w.im, w.im)};
    });
    const int lp = threadIdx.x / TPL, j = threadIdx.x % TPL;
    const int total = npairs * TILES;
    auto issue = [&](int t, int b) {
        const int pr = t / TILES, row0 = (t - pr * TILES) * LINES;
        const TIN* src = (const TIN*)a.pair[pr].src[0].rho + (size_t)row0 * NIN;
        TIN* dst = stage + b * S::ELEMS;
#pragma unroll
        for (int i = threadIdx.x * VEC; i < TILE; i += 128 * VEC) {
            const int row = i / NIN;
            cp_async16(dst + row * S::PITCH + (i - row * NIN), src + i);
        }
    };
    int t = blockIdx.x;
    if (t < total) issue(t, 0);
    cp_async_commit();
    for (int k = 0; t < total; ++k, t += gridDim.x) {
        if (t + (int)gridDim.x < total) issue(t + gridDim.x, (k + 1) & 1);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const int pr = t / TILES, row0 = (t - pr * TILES) * LINES;
        const PairDesc<T>& d = a.pair[pr];
        const T s0 = (T)d.src[0].scale, s1 = (T)d.src[1].scale;
        const int row = row0 + 2 * lp;                      // rows row, row + 1: same z, y even
        const int zi = row / NIN, yi = row % NIN;
        const int q = NIN / 4, h = NIN / 2;
        const bool zc = (unsigned)(zi - q) < (unsigned)h;
        const bool cov0 = zc && (unsigned)(yi - q) < (unsigned)h;
        const bool cov1 = zc && (unsigned)(yi + 1 - q) < (unsigned)h;
        const bool hole = d.src[1].mode == SRC_HOLE;
        const TIN* st = stage + (k & 1) * S::ELEMS + 2 * lp * S::PITCH;
        const TIN* rs = (const TIN*)d.src[0].restr;
        cpx<f2> v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            v[r] = {f2(0), f2(0)};
            if (G::live(r)) {
                const int xi = j + r * (P / E);
                const bool xc = (unsigned)(xi - q) < (unsigned)h;
                const T a0 = st[xi], a1 = st[S::PITCH + xi];
                T f0 = a0, f1 = a1;
                if (rs && cov0 && xc) f0 = rs[((size_t)(zi - q) * h + (yi - q)) * h + (xi - q)];
                if (rs && cov1 && xc) f1 = rs[((size_t)(zi - q) * h + (yi + 1 - q)) * h + (xi - q)];
                v[r].re = f2(f0 * s0, f1 * s0);
                v[r].im = f2((hole && !(cov0 && xc)) ? a0 * s1 : T(0), (hole && !(cov1 && xc)) ? a1 * s1 : T(0));
            }
        }
        fft_line<f2, P, E, false, G::LIVE, false, true>(v, j, sm_tw,
                                                  LineView<f2, 1, true, Log2E<E>::value>{sm_lines + lp * (P + P / E)});
        cpx<T>* out0 = d.work + ((size_t)zi * P + yi) * P;
        cpx<T>* out1 = out0 + P;
        const int kx_end = d.half ? P / 2 + 32 : P;
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const int kx = out_index<P, E>(j, s);
            if (kx < kx_end) {
                out0[kx] = {v[s].re.x, v[s].im.x};
                out1[kx] = {v[s].re.y, v[s].im.y};
            }
        }
        __syncthreads();   // this half of the stage and the line scratch are free again
    }
}

// ---------------------------------------------------------------- passes 2, 4
// tile: column tile (x); zs: slab index (z from the block's first input slab).
// The indices are unsigned, as block indices are: the compiler then knows them
// non-negative and keeps the address arithmetic of the kernel form.
template <typename T, int P, int E, int TX, bool INV, int GM>
__device__ __forceinline__ void ypass_body(cpx<T>* work, const cpx<T>* tw, unsigned tile, unsigned zs,
                                           unsigned char* smem_raw) {
    using G = Geo<P, E, GM>;
    cpx<T>* sm_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* sm_tile = sm_tw + P;
    load_twiddles<P, E>(sm_tw, tw);
    const int l = threadIdx.x % TX, j = threadIdx.x / TX;
    // blockDim.x = TX P/E: lets the compiler see which outputs of the last
    // pass the window keeps, and drop the rest
    __builtin_assume(j < P / E);
    const int z = (INV ? 0 : G::OFF) + zs;
    const int x = tile * TX + l;
    cpx<T>* slab = work + (size_t)z * P * P;
    cpx<T> v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        if (INV || G::live(r)) v[r] = slab[(size_t)(j + r * (P / E)) * P + x];
        else v[r] = {T(0), T(0)};
    }
    __syncthreads();
    fft_line<T, P, E, INV, INV ? 0xFFFFu : G::LIVE, false>(v, j, sm_tw, LineView<T, TX, false>{sm_tile + l});
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const int e = out_index<P, E>(j, s);
        if (!INV || e < G::NOUT) slab[(size_t)e * P + x] = v[s];
    }
}

// The kernel form keeps its own copy of the body: calling ypass_body from it
// compiled to a different register allocation that ran the passes 15-25 %
// slower (ptxas: 42 against 48 registers at P = 256; measured 115 against
// 97 us per y-forward at 6 x 128^3).  The arithmetic is the same.
template <typename T, int P, int E, int TX, bool INV, int GM>
__global__ void __launch_bounds__(TX * P / E) k_ypass(const __grid_constant__ ConvArgs<T> a) {
    using G = Geo<P, E, GM>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* sm_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* sm_tile = sm_tw + P;
    const PairDesc<T>& d = a.pair[blockIdx.z];
    if (d.half && blockIdx.x * TX > P / 2) return;   // the column tile is above kx = P/2 (whole CTA)
    const int l = threadIdx.x % TX, j = threadIdx.x / TX;
    __builtin_assume(j < P / E);
    const int z = (INV ? 0 : G::OFF) + blockIdx.y;
    const int x = blockIdx.x * TX + l;
    cpx<T>* slab = d.work + (size_t)z * P * P;
    cpx<T> v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        if (INV || G::live(r)) v[r] = slab[(size_t)(j + r * (P / E)) * P + x];
        else v[r] = {T(0), T(0)};
    }
    load_twiddles<P, E>(sm_tw, a.tw);   // after the column loads are out
    __syncthreads();
    fft_line<T, P, E, INV, INV ? 0xFFFFu : G::LIVE, false>(v, j, sm_tw, LineView<T, TX, false>{sm_tile + l});
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const int e = out_index<P, E>(j, s);
        if (!INV || e < G::NOUT) slab[(size_t)e * P + x] = v[s];
    }
}

// ---------------------------------------------------------------- pass 3
// Resident threads per SM the z-seam's register cap aims at: 1024 (4 CTAs of
// 256) for float and double -- the seam holds two transforms' worth of live
// values, and more warps hide its load latency -- and 512 for double-float,
// whose values take twice the registers.
template <typename T, int NT> struct ZseamMinBlocks {
    static constexpr int R = is_df<T>::value ? 512 : 1024;
    static constexpr int value = R / NT > 0 ? R / NT : 1;
};

// tile: column tile (kx); y: the ky row
template <typename T, int P, int E, int TX, int GM>
__device__ __forceinline__ void zseam_body(const PairDesc<T>& d, const T* spec, const cpx<T>* tw, unsigned tile,
                                           unsigned y,
                                           unsigned char* smem_raw) {
    using G = Geo<P, E, GM>;
    constexpr int H = P / 2 + 1;
    cpx<T>* sm_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* sm_tile = sm_tw + P;
    const int l = threadIdx.x % TX, j = threadIdx.x / TX;
    // blockDim.x = TX P/E: lets the compiler see which outputs of the last
    // pass the window keeps, and drop the rest
    __builtin_assume(j < P / E);
    const int x = tile * TX + l;
    cpx<T>* col = d.work + (size_t)y * P + x;          // element z at col[z * P * P]
    cpx<T> v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        if (G::live(r)) v[r] = col[(size_t)(j + r * (P / E)) * P * P];
        else v[r] = {T(0), T(0)};
    }
    load_twiddles<P, E, true>(sm_tw, tw);   // after the column loads are out
    __syncthreads();
    const LineView<T, TX, false> view{sm_tile + l};
    fft_line<T, P, E, false, G::LIVE, true, true>(v, j, sm_tw, view);
    const int fy = y <= P / 2 ? y : P - y;
    const int fx = x <= P / 2 ? x : P - x;
    const T* sp = spec + (size_t)fy * H + fx;
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const int kz = out_index<P, E>(j, s);
        const int fz = kz <= P / 2 ? kz : P - kz;
        const T g = ldg_t<T>(sp + (size_t)fz * H * H);
        v[s].re *= g;
        v[s].im *= g;
    }
    seam_permute<T, P, E>(v);
    fft_line<T, P, E, true, 0xFFFFu, false, true>(v, j, sm_tw, view);
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const int e = out_index<P, E>(j, s);
        if (e < G::NOUT) col[(size_t)e * P * P] = v[s];
    }
}

template <typename T, int P, int E, int TX, int GM>
__global__ void __launch_bounds__(TX * P / E, (ZseamMinBlocks<T, TX * P / E>::value))
    k_zseam(const __grid_constant__ ConvArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.pair[blockIdx.z].half && blockIdx.x * TX > P / 2) return;   // above kx = P/2 (whole CTA)
    zseam_body<T, P, E, TX, GM>(a.pair[blockIdx.z], a.spec, a.tw, blockIdx.x, blockIdx.y, smem_raw);
}

// Pass 3 in FP32 with two neighbouring columns per thread.  The lines (ky, x)
// and (ky, x + 1) go through identical arithmetic, so the thread carries them
// as one transform over cpx<f2> (lane 0 = column x, lane 1 = column x + 1):
// the twiddle and spectrum products then take half the instructions of two
// separate float transforms, and each shared-memory access moves both lines.
// TX columns per CTA, TX / 2 threads across them.  Here a.spec holds float
// rows over all kx, a.spec[(fz H + fy) P + x] = octant[fz][fy][fold(x)] (the
// launcher passes them in place of the octant): the CTA's TX columns of every
// fz row are one aligned 4 TX-byte run, copied
// to shared memory with asynchronous 16-byte copies issued before the column
// loads, so they land while the forward transform runs.
template <int NT> struct Zseam2MinBlocks {
    // 512 resident threads per SM (128 registers each): the same 1024 lines
    // in flight per SM as the one-column kernel
    static constexpr int value = 512 / NT > 0 ? 512 / NT : 1;
};

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int P, int E, int TX, int GM>
__global__ void __launch_bounds__(TX / 2 * P / E, Zseam2MinBlocks<TX / 2 * P / E>::value)
    k_zseam2(const __grid_constant__ ConvArgs<float> a) {
    using G = Geo<P, E, GM>;
    constexpr int H = P / 2 + 1, TX2 = TX / 2;
    static_assert(TX % 4 == 0, "column pairs, 16-byte spectrum runs");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<f2>* sm_tw = reinterpret_cast<cpx<f2>*>(smem_raw);
    cpx<f2>* sm_tile = sm_tw + P;
    float* sm_sp = reinterpret_cast<float*>(sm_tile + TX2 * P);      // [H][TX]
    const PairDesc<float>& d = a.pair[blockIdx.z];
    if (d.half && blockIdx.x * TX > P / 2) return;   // above kx = P/2 (whole CTA)
    const int y = blockIdx.y;
    const int fy = y <= P / 2 ? y : P - y;
    const int l = threadIdx.x % TX2, j = threadIdx.x / TX2;
    __builtin_assume(j < P / E);
    const int x = blockIdx.x * TX + 2 * l;
    cpx<float>* col = d.work + (size_t)y * P + x;      // columns x, x + 1: element z at col[z * P * P]
    // the column loads go out first: the twiddle staging below waits on its
    // own (L2) loads, and would otherwise hold them back
    cpx<f2> v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        if (G::live(r)) {
            const float4 q = *reinterpret_cast<const float4*>(col + (size_t)(j + r * (P / E)) * P * P);
            v[r] = {f2(q.x, q.z), f2(q.y, q.w)};
        } else {
            v[r] = {f2(0), f2(0)};
        }
    }
    {
        const float* sp = a.spec + (size_t)fy * P + blockIdx.x * TX;
        for (int i = threadIdx.x; i < H * (TX / 4); i += blockDim.x) {
            const int fz = i / (TX / 4), c = i % (TX / 4);
            cp_async16(sm_sp + fz * TX + 4 * c, sp + (size_t)fz * H * P + 4 * c);
        }
        cp_async_commit();
    }
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const cpx<float> w = a.tw[i];
        sm_tw[i] = {f2(w.re, w.re), f2(w.im, w.im)};
    }
    cp_async_wait_all();
    __syncthreads();
    const LineView<f2, TX2, false> view{sm_tile + l};
    fft_line<f2, P, E, false, G::LIVE>(v, j, sm_tw, view);
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const int kz = out_index<P, E>(j, s);
        const int fz = kz <= P / 2 ? kz : P - kz;
        const float2 g = *reinterpret_cast<const float2*>(sm_sp + fz * TX + 2 * l);
        v[s].re *= f2(g.x, g.y);
        v[s].im *= f2(g.x, g.y);
    }
    seam_permute<f2, P, E>(v);
    fft_line<f2, P, E, true, 0xFFFFu, false>(v, j, sm_tw, view);
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const int e = out_index<P, E>(j, s);
        if (e < G::NOUT)
            *reinterpret_cast<float4*>(col + (size_t)e * P * P) = make_float4(v[s].re.x, v[s].im.x, v[s].re.y, v[s].im.y);
    }
}

// Pass 3 in FP32, one column per thread, with the CTA's spectrum rows
// staged in shared memory: the arithmetic of zseam_body (level grids), but
// the spectrum comes from the float rows unfolded along kx (a.spec as for
// k_zseam2), so that the TX columns of every fz row are one aligned 4 TX-byte
// run; its asynchronous 16-byte copies go out right after the column loads
// and land while the forward transform runs, instead of 16 dependent L2
// loads per thread between the two transforms.
template <int P, int E, int TX>
__global__ void __launch_bounds__(TX * P / E, (ZseamMinBlocks<float, TX * P / E>::value))
    k_zseam_s(const __grid_constant__ ConvArgs<float> a) {
    using G = Geo<P, E, 0>;
    constexpr int H = P / 2 + 1;
    static_assert(TX % 4 == 0, "16-byte spectrum runs");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float>* sm_tw = reinterpret_cast<cpx<float>*>(smem_raw);
    cpx<float>* sm_tile = sm_tw + P;
    float* sm_sp = reinterpret_cast<float*>(sm_tile + TX * P);      // [H][TX]
    const PairDesc<float>& d = a.pair[blockIdx.z];
    if (d.half && blockIdx.x * TX > P / 2) return;   // above kx = P/2 (whole CTA)
    const int y = blockIdx.y;
    const int fy = y <= P / 2 ? y : P - y;
    const int l = threadIdx.x % TX, j = threadIdx.x / TX;
    __builtin_assume(j < P / E);
    const int x = blockIdx.x * TX + l;
    cpx<float>* col = d.work + (size_t)y * P + x;      // element z at col[z * P * P]
    cpx<float> v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        if (G::live(r)) v[r] = col[(size_t)(j + r * (P / E)) * P * P];
        else v[r] = {0.f, 0.f};
    }
    {
        const float* sp = a.spec + (size_t)fy * P + blockIdx.x * TX;
        for (int i = threadIdx.x; i < H * (TX / 4); i += blockDim.x) {
            const int fz = i / (TX / 4), c = i % (TX / 4);
            cp_async16(sm_sp + fz * TX + 4 * c, sp + (size_t)fz * H * P + 4 * c);
        }
        cp_async_commit();
    }
    load_twiddles<P, E, true>(sm_tw, a.tw);
    cp_async_wait_all();
    __syncthreads();
    const LineView<float, TX, false> view{sm_tile + l};
    fft_line<float, P, E, false, G::LIVE, true, true>(v, j, sm_tw, view);
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const int kz = out_index<P, E>(j, s);
        const int fz = kz <= P / 2 ? kz : P - kz;
        const float g = sm_sp[fz * TX + l];
        v[s].re *= g;
        v[s].im *= g;
    }
    seam_permute<float, P, E>(v);
    fft_line<float, P, E, true, 0xFFFFu, false, true>(v, j, sm_tw, view);
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const int e = out_index<P, E>(j, s);
        if (e < G::NOUT) col[(size_t)e * P * P] = v[s];
    }
}

// ---------------------------------------------------------------- pass 5
template <typename T, int P>
__device__ __forceinline__ void store_out(const DstField& f, int z, int y, int x, T val) {
    constexpr int E = P / 2;
    if (f.kind == DST_GRID) {
        ((T*)f.out)[((size_t)z * E + y) * E + x] = val;
    } else if (f.kind == DST_CROP) {
        const int c0 = E / 4 - 1, nc = E / 2 + 2;
        if ((unsigned)(z - c0) < (unsigned)nc && (unsigned)(y - c0) < (unsigned)nc &&
            (unsigned)(x - c0) < (unsigned)nc)
            ((T*)f.out)[((size_t)(z - c0) * nc + (y - c0)) * nc + (x - c0)] = val;
    }
}

template <typename T, int P, int E, int GM>
__device__ __forceinline__ void xinv_body(const PairDesc<T>& d, const cpx<T>* tw, unsigned tile,
                                          unsigned char* smem_raw) {
    constexpr int TPL = P / E;
    constexpr int LINES = 256 / TPL;
    constexpr int HALF = P / 2;
    cpx<T>* sm_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* sm_lines = sm_tw + P;
    const int line = threadIdx.x / TPL, j = threadIdx.x % TPL;
    const int row = tile * LINES + line;
    const bool valid = row < HALF * HALF;
    const int z = row / HALF, y = row % HALF;
    cpx<T> v[E];
    const cpx<T>* src = d.work + ((size_t)z * P + y) * P;
    // a real pair (d.half): only kx <= P/2 went through the y and z passes,
    // and kx > P/2 is read as conj X[P - kx]
    const bool half = d.half != 0;
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int kx = j + r * (P / E);
        const bool up = half && kx > P / 2;
        cpx<T> w = valid ? src[up ? P - kx : kx] : cpx<T>{T(0), T(0)};
        if (up) w.im = -w.im;
        v[r] = w;
    }
    load_twiddles<P, E, true>(sm_tw, tw);   // after the row loads are out
    __syncthreads();
    fft_line<T, P, E, true, 0xFFFFu, false, true>(v, j, sm_tw,
                                            LineView<T, 1, true, Log2E<E>::value>{sm_lines + line * (P + P / E)});
    if (valid) {
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const int e = out_index<P, E>(j, s);
            if (e < HALF) {
                store_out<T, P>(d.dst[0], z, y, e, v[s].re);
                store_out<T, P>(d.dst[1], z, y, e, v[s].im);
            }
        }
    }
}

template <typename T, int P, int E, int GM>
__global__ void __launch_bounds__(256) k_xinv(const __grid_constant__ ConvArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    xinv_body<T, P, E, GM>(a.pair[blockIdx.y], a.tw, blockIdx.x, smem_raw);
}

// Column tile width of the strided passes: at most the requested width W,
// at most 1024 threads, never wider than a row of the domain.
template <int P, int E, int W> struct Tile {
    static constexpr int A = W < P ? W : P;
    static constexpr int TX = (A * P / E > 1024) ? 1024 * E / P : A;
};

}  // namespace nm
