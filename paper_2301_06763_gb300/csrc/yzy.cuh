// yzy.cuh -- the per-level convolution of Sect. 3 in three passes (FP32, level
// grids): the x transforms as before, and the y transform, the z transform,
// the spectrum multiply (Eq. 11) and both inverse transforms fused into one
// pass per kx plane, with the plane held in shared memory.
//
// Work buffer of one pair in this form: kx-major, work[kx][z][y] (z, y < N,
// kx < P = 2N), so that everything one kx needs is one contiguous N^2 plane.
//   A k_xfwd_t : rows (z, y): mask, scale, pack, pad, FFT along x; the P
//                outputs of a row go to work[kx][z][y] through a shared-memory
//                transpose (runs of consecutive y per kx).
//   B k_yzy    : plane kx: forward y (input pruned to y < N), forward z (input
//                pruned to z < N), times the spectrum, inverse z (keep z < N),
//                inverse y (keep y < N); written back in place.
//   C k_xinv_t : rows (z, y) read from work[kx][z][y] through a shared-memory
//                transpose: inverse along x, keep x < N, scatter the outputs.
// Pass B moves 2 N^2 complex values per plane (in and out) where the y, z and
// y passes of the five-pass form move 8 N^2 + ... ; the intermediate between
// its transforms never leaves the SM.
//
// Splitting the plane over a cluster.  After the forward y transform a plane
// holds N x P complex values (all ky), 256 KB in FP32 at N = 128: more than one
// SM's shared memory.  Its ky are therefore split by residue e = ky mod C over
// a cluster of C CTAs, one residue each, with M = P / C.  From the definition
// of the zero-padded transform, w = exp(-2 pi i / P), w_M = w^C:
//   Y[C k + e] = sum_{y<N} x[y] w^{y (C k + e)} = sum_{y'<M} u_e[y'] w_M^{y' k},
//   u_e[y'] = sum_{t : y' + M t < N} x[y' + M t] w^{(y' + M t) e}
// (w^{M t C k} = 1), an M-point transform of a folded, twiddled line; and the
// inverse y transform of the processed values Y' splits the same way,
//   out[y' + M t] = sum_e w_C^{-t e} r_e[y'],   r_e[y'] = w^{-y' e} IDFT_M(Y'_e)[y']
// (w^{-M t e} = w_C^{-t e}).  Each CTA transforms its M ky columns along z in
// full (the z transform does not mix ky), and the C partial results r_e are
// summed through distributed shared memory, each CTA producing N / C rows of
// the output plane.  The sum runs over e = 0 .. C-1 in that order in every CTA.
#pragma once
#include "conv.cuh"

namespace nm {

// ---------------------------------------------------------------- shapes
// P = 2N; C = CTAs per plane (ky residues); M = P / C; E = 16 values per
// thread in every transform.
template <int P, int C> struct YzyShape {
    static constexpr int N = P / 2, M = P / C, E = 16;
    static constexpr int TY = M / E;          // threads per y line (M points)
    static constexpr int TZ = P / E;          // threads per z line (P points)
    static constexpr int NT = N * TY;         // all N y lines in one round
    static constexpr int ZL = NT / TZ;        // z lines per round (M / 2: two rounds)
    // shared-memory rows of the plane: row(z) = z + z / 16, so that the z
    // transforms' stride-16 element accesses fall on distinct banks
    static constexpr int ROWS = N + (N - 1) / 16;
    // a row holds M values with one padding slot every 16 (the y transforms'
    // first-pass stores); an odd pitch keeps a column's consecutive rows on
    // distinct banks
    static constexpr int PITCH0 = M + (M - 1) / 16;
    static constexpr int PITCH = PITCH0 % 2 ? PITCH0 : PITCH0 + 1;
    // upper halves (z >= N) of the z lines of one round, padded like the rows
    static constexpr int EXTP = N + (N - 1) / 16;
    static constexpr size_t SMEM = sizeof(cpx<float>) * ((size_t)P + M + (size_t)ROWS * PITCH + (size_t)ZL * EXTP);
    static constexpr int MINB = NT >= 1024 ? 1 : (NT >= 512 ? 2 : (NT >= 256 ? 4 : 8));
    static_assert(M >= E && P % C == 0 && N % C == 0, "residue split");
    static_assert(ZL * 2 == M, "two rounds of z lines");
};

__device__ __forceinline__ int yzy_row(int z) { return z + (z >> 4); }

// Line views for fft_line.  A y line is one padded row of the plane; a z line
// is one column k of the plane for elements e < N and one padded row of the
// round's extension area for e >= N.
struct YView {
    cpx<float>* row;
    __device__ __forceinline__ int off(int e) const { return e + (e >> 4); }
    __device__ __forceinline__ cpx<float> ld(int e) const { return row[off(e)]; }
    __device__ __forceinline__ void st(int e, cpx<float> v) const { row[off(e)] = v; }
    template <int E> __device__ __forceinline__ void st_first(int j, const cpx<float>* v) const {
#pragma unroll
        for (int r = 0; r < E; ++r) st(E * j + r, v[r]);
    }
};
template <int N, int PITCH> struct ZView {
    cpx<float>* col;   // column k of the plane: element z at col[yzy_row(z) * PITCH]
    cpx<float>* ext;   // this line's extension row
    __device__ __forceinline__ cpx<float>* at(int e) const {
        if (e < N) return col + yzy_row(e) * PITCH;
        const int u = e - N;
        return ext + u + (u >> 4);
    }
    __device__ __forceinline__ cpx<float> ld(int e) const { return *at(e); }
    __device__ __forceinline__ void st(int e, cpx<float> v) const { *at(e) = v; }
    // the first pass's stores, elements E j + r (r < E, E = 16): all in the
    // plane column or all in the extension row, so the branch is taken once
    // and each side addresses its 16 slots with constant offsets
    template <int E> __device__ __forceinline__ void st_first(int j, const cpx<float>* v) const {
        static_assert(E == 16 && N % E == 0, "first-pass block inside one half");
        if (E * j < N) {
            cpx<float>* p = col + (17 * j) * PITCH;        // yzy_row(16 j + r) = 17 j + r
#pragma unroll
            for (int r = 0; r < E; ++r) p[r * PITCH] = v[r];
        } else {
            cpx<float>* p = ext + 17 * (j - N / E);        // u = 16 (j - N/16) + r: u + u/16
#pragma unroll
            for (int r = 0; r < E; ++r) p[r] = v[r];
        }
    }
};

// ---------------------------------------------------------------- cluster
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_shared(const void* p, uint32_t rank) {
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(out)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return out;
}
__device__ __forceinline__ cpx<float> ld_cluster(uint32_t addr) {
    float a, b;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "r"(addr) : "memory");
    return {a, b};
}

// Line scratch of the kx-major x passes: the line transforms' rows, or the
// transpose of a tile's P x LINES outputs, whichever is larger.
template <int P> struct XtShape {
    static constexpr int E = 16, TPL = P / E, LINES = 256 / TPL, TP = LINES + 1;
    static constexpr int SCR = LINES * (P + P / E) > P * TP ? LINES * (P + P / E) : P * TP;
};

// ---------------------------------------------------------------- pass A
// As k_xfwd_pipe (persistent, density tiles fetched with cp.async one tile
// ahead), with the kx-major output.  Level grids whose pairs are a level's
// full and hole fields (or a full field alone) on a 16-byte aligned density.
template <typename TIN, int P>
__global__ void __launch_bounds__(256) k_xfwd_t(const __grid_constant__ ConvArgs<float> a, int npairs) {
    using T = float;
    constexpr int E = 16;
    using G = Geo<P, E, 0>;
    using S = XfwdStage<TIN, P, E>;
    constexpr int TPL = P / E, LINES = 256 / TPL, NIN = G::NIN;
    constexpr int TILE = LINES * NIN;
    constexpr int TILES = NIN * NIN / LINES;
    constexpr int VEC = 16 / sizeof(TIN);
    constexpr int TP = LINES + 1;                      // transpose pitch
    static_assert((NIN * NIN) % LINES == 0 && TILE % (256 * VEC) == 0 && NIN % VEC == 0, "tile shape");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* sm_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* sm_lines = sm_tw + P;
    TIN* stage = reinterpret_cast<TIN*>(sm_lines + XtShape<P>::SCR);
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
        __syncthreads();   // every line's last pass has read the scratch
#pragma unroll
        for (int s = 0; s < E; ++s) sm_lines[out_index<P, E>(j, s) * TP + line] = v[s];
        __syncthreads();
        // plane kx holds rows z * NIN + y contiguously: the tile's LINES rows
        // are one run per kx
        cpx<T>* out = d.work + row0;
        for (int i = threadIdx.x; i < P * LINES; i += 256) {
            const int kx = i / LINES, l = i - kx * LINES;
            out[(size_t)kx * NIN * NIN + l] = sm_lines[kx * TP + l];
        }
        __syncthreads();   // the stage half and the scratch are free again
    }
}

// ---------------------------------------------------------------- pass B
template <int P, int C>
__global__ void __launch_bounds__(YzyShape<P, C>::NT, YzyShape<P, C>::MINB)
    k_yzy(const __grid_constant__ ConvArgs<float> a) {
    using S = YzyShape<P, C>;
    constexpr int N = S::N, M = S::M, E = S::E, TY = S::TY, TZ = S::TZ, ZL = S::ZL, PITCH = S::PITCH;
    constexpr int H = N + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float>* sm_tw = reinterpret_cast<cpx<float>*>(smem_raw);   // w^t, t < P
    cpx<float>* sm_twm = sm_tw + P;                                 // w_M^t = w^{C t}, t < M
    cpx<float>* plane = sm_twm + M;                                 // [ROWS][PITCH]
    cpx<float>* ext = plane + S::ROWS * PITCH;                      // [ZL][EXTP]
    const int e = (int)cluster_rank();                              // ky residue
    const int kx = blockIdx.y;
    const PairDesc<float>& d = a.pair[blockIdx.z];
    cpx<float>* gplane = d.work + (size_t)kx * N * N;
    for (int i = threadIdx.x; i < P; i += S::NT) sm_tw[i] = a.tw[i];
    for (int i = threadIdx.x; i < M; i += S::NT) sm_twm[i] = a.tw[C * i];

    // ---- forward y: line z, M-point transform of the folded, twiddled line
    {
        const int z = threadIdx.x / TY, j = threadIdx.x % TY;
        const cpx<float>* src = gplane + (size_t)z * N;
        cpx<float> v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int y0 = j + r * TY;
            cpx<float> acc = {0.f, 0.f};
#pragma unroll
            for (int t = 0; t < N / M; ++t) {
                const int y = y0 + t * M;
                cpx<float> x = src[y];
                if (e != 0) {
                    const cpx<float> w = a.tw[(y * e) & (P - 1)];
                    x = cmul(x, w);
                }
                acc = t == 0 ? x : acc + x;
            }
            v[r] = acc;
        }
        __syncthreads();   // twiddle tables staged
        const YView view{plane + yzy_row(z) * PITCH};
        fft_line<float, M, E, false, 0xFFFFu, true>(v, j, sm_twm, view);
#pragma unroll
        for (int s = 0; s < E; ++s) view.st(out_index<M, E>(j, s), v[s]);
    }
    __syncthreads();

    // ---- z: column k (ky = C k + e), P-point transforms, spectrum, inverse
    {
        const int l = threadIdx.x / TZ, j = threadIdx.x % TZ;
        __builtin_assume(j < TZ);
        const int fx = kx <= N ? kx : P - kx;
#pragma unroll 1
        for (int rnd = 0; rnd < 2; ++rnd) {
            const int k = rnd * ZL + l;
            const int ky = C * k + e;
            const int fy = ky <= N ? ky : P - ky;
            // column k of the plane: the y transform stored element k of
            // every row at k + k / 16
            const ZView<N, PITCH> view{plane + k + (k >> 4), ext + l * S::EXTP};
            cpx<float> v[E];
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = r < E / 2 ? view.ld(j + r * TZ) : cpx<float>{0.f, 0.f};
            __syncthreads();   // the line's inputs are in registers before its slots are reused
            fft_line<float, P, E, false, Geo<P, E, 0>::LIVE, true>(v, j, sm_tw, view);
            // spectrum of this line, z fastest: [fx][fy][fz]
            const float* sp = a.spec + ((size_t)fx * H + fy) * H;
#pragma unroll
            for (int s = 0; s < E; ++s) {
                const int kz = out_index<P, E>(j, s);
                const float g = __ldg(sp + (kz <= N ? kz : P - kz));
                v[s].re *= g;
                v[s].im *= g;
            }
            seam_permute<float, P, E>(v);
            fft_line<float, P, E, true, 0xFFFFu, true>(v, j, sm_tw, view);
#pragma unroll
            for (int s = 0; s < E; ++s) {
                const int z = out_index<P, E>(j, s);
                if (z < N) view.st(z, v[s]);
            }
        }
    }
    __syncthreads();

    // ---- inverse y: line z, M-point inverse, then w^{-y' e}
    {
        const int z = threadIdx.x / TY, j = threadIdx.x % TY;
        const YView view{plane + yzy_row(z) * PITCH};
        cpx<float> v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = view.ld(j + r * TY);
        __syncthreads();
        fft_line<float, M, E, true, 0xFFFFu, true>(v, j, sm_twm, view);
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const int y = out_index<M, E>(j, s);
            cpx<float> x = v[s];
            if (e != 0) {
                const cpx<float> w = sm_tw[(y * e) & (P - 1)];
                x = cmulc(x, w);
            }
            view.st(y, x);
        }
    }
    // every CTA of the cluster holds its partial r_e
    cluster_sync_all();

    // ---- sum of the C partials: this CTA writes rows [e N/C, (e+1) N/C)
    {
        constexpr int ITEMS = (N / C) * M;
        for (int i = threadIdx.x; i < ITEMS; i += S::NT) {
            const int z = e * (N / C) + i / M, y = i % M;
            const cpx<float>* p = plane + yzy_row(z) * PITCH + y + (y >> 4);
            cpx<float> r[C];
#pragma unroll
            for (int c = 0; c < C; ++c) r[c] = c == e ? *p : ld_cluster(map_shared(p, (uint32_t)c));
            cpx<float>* dst = gplane + (size_t)z * N + y;
#pragma unroll
            for (int t = 0; t < N / M; ++t) {
                cpx<float> acc = r[0];
#pragma unroll
                for (int c = 1; c < C; ++c) {
                    // w_C^{-t c} = exp(+2 pi i t c / C), an exact table entry: w^{-(t c P / C)}
                    const int idx = ((t * c) % C) * (P / C);
                    cpx<float> x = r[c];
                    if (idx != 0) x = cmulc(x, sm_tw[idx]);
                    acc = acc + x;
                }
                dst[t * M] = acc;
            }
        }
    }
    // no CTA leaves while another may still read its plane
    cluster_sync_all();
}

// ---------------------------------------------------------------- pass C
template <int P>
__global__ void __launch_bounds__(256) k_xinv_t(const __grid_constant__ ConvArgs<float> a) {
    using T = float;
    constexpr int E = 16, TPL = P / E, LINES = 256 / TPL, HALF = P / 2, TP = LINES + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* sm_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* sm_lines = sm_tw + P;
    const PairDesc<T>& d = a.pair[blockIdx.y];
    load_twiddles<P, E, true>(sm_tw, a.tw);
    const int row0 = blockIdx.x * LINES;
    const cpx<T>* src = d.work + row0;
    // the tile's rows are one run of LINES values per kx: load them two at a
    // time (16 bytes) and transpose through shared memory
    for (int i = 2 * threadIdx.x; i < P * LINES; i += 512) {
        const int kx = i / LINES, l = i - kx * LINES;
        const float4 q = *reinterpret_cast<const float4*>(src + (size_t)kx * HALF * HALF + l);
        sm_lines[kx * TP + l] = {q.x, q.y};
        sm_lines[kx * TP + l + 1] = {q.z, q.w};
    }
    __syncthreads();
    const int line = threadIdx.x / TPL, j = threadIdx.x % TPL;
    const int row = row0 + line;
    const int z = row / HALF, y = row % HALF;
    cpx<T> v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) v[r] = sm_lines[(j + r * (P / E)) * TP + line];
    __syncthreads();
    fft_line<T, P, E, true, 0xFFFFu, false, true>(v, j, sm_tw,
                                            LineView<T, 1, true, Log2E<E>::value>{sm_lines + line * (P + P / E)});
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const int e = out_index<P, E>(j, s);
        if (e < HALF) {
            store_out<T, P>(d.dst[0], z, y, e, v[s].re);
            store_out<T, P>(d.dst[1], z, y, e, v[s].im);
        }
    }
}

}  // namespace nm
