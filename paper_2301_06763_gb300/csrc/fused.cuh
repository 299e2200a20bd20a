// fused.cuh -- the x and y passes of the level convolution (Sect. 3, Eq. 11)
// fused per z-slab through a thread-block cluster.
//
// Forward (replaces xfwd + yfwd): a cluster of C CTAs owns one slab z of one
// pair.  CTA r transforms along x the rows y in [r N/C, (r+1) N/C) of the
// masked, scaled, zero-padded density (as k_xfwd) into its own shared memory,
// laid out [y][kx].  After a cluster barrier, CTA r transforms along y the
// columns kx in [r P/C, (r+1) P/C): each column's N nonzero inputs are read
// from the shared memory of the CTAs that own them (distributed shared
// memory), and its P outputs go to the work buffer [z][ky][kx] that the
// z-seam reads.
//
// Inverse (replaces yinv + xinv): CTA r inverse-transforms along y the columns
// kx in its range from the work buffer, keeping y < N, into its shared memory
// [y][kx - r P/C]; after a cluster barrier it inverse-transforms along x the
// rows y in its range, reading all P kx values from the owning CTAs, and
// scatters the outputs x < N as k_xinv does.
//
// A closing cluster barrier keeps every CTA resident until no peer reads its
// shared memory.  The barriers are the hardware cluster barrier; all CTAs of a
// cluster run the same uniform control flow.
#pragma once
#include <cooperative_groups.h>

#include "conv.cuh"

namespace nm {

// Cluster size and tile shapes of the fused passes for (T, P).  C is the
// smallest power of two (at most the portable 8) that keeps each CTA's share
// of a slab within 32 KB; NT is chosen so both phases keep every thread busy
// (a column tile is TX = NT E / P columns wide, a row batch NT / (P/E) rows).
template <typename T, int P> struct FusedShape {
    static constexpr int N = P / 2;
    static constexpr int E = EOf<P>::value;
    static constexpr size_t CS = 2 * sizeof(T);
    static constexpr size_t SLAB = (size_t)N * P * CS;                 // one slab's x output
    static constexpr int C0 = (int)((SLAB + 32767) / 32768);
    static constexpr int C = C0 <= 1 ? 1 : C0 <= 2 ? 2 : C0 <= 4 ? 4 : 8;
    static constexpr bool OK = (SLAB / C) <= 131072 && N % C == 0 && P >= 16;
    static constexpr int RPC = N / C;                 // rows per CTA
    static constexpr int CPC = P / C;                 // kx columns per CTA
    static constexpr int TPL = P / E;                 // threads per row transform
    static constexpr int NT = (CPC * P / E) < 256 ? CPC * P / E : 256;   // threads per CTA
    static constexpr int ROWS = NT / TPL;             // rows transformed at once
    static constexpr int TX = NT * E / P;             // columns transformed at once (<= CPC)
    static constexpr int LS = P + P / E;              // padded row (x exchange)
    static constexpr int SCR = (ROWS * LS > TX * P) ? ROWS * LS : TX * P;
    static constexpr size_t SMEM = ((size_t)P + (size_t)RPC * P + SCR) * CS;   // fwd: tw + slab share + scratch
    static constexpr size_t SMEM_INV = ((size_t)P + (size_t)N * CPC + SCR) * CS;
};

template <typename T, typename TIN, int P>
__global__ void __cluster_dims__(FusedShape<T, P>::C, 1, 1) __launch_bounds__(FusedShape<T, P>::NT)
    k_xyfwd(const __grid_constant__ ConvArgs<T> a) {
    using F = FusedShape<T, P>;
    constexpr int N = F::N, E = F::E, C = F::C;
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* sm_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* slab = sm_tw + P;                    // [RPC][P]
    cpx<T>* scr = slab + F::RPC * P;
    const int rank = (int)cluster.block_rank();
    const int z = blockIdx.x / C;
    const PairDesc<T>& d = a.pair[blockIdx.y];
    load_twiddles<P, E>(sm_tw, a.tw);
    const T s0 = (T)d.src[0].scale, s1 = (T)d.src[1].scale;
    __syncthreads();
    // phase 1: rows along x
    {
        const int line = threadIdx.x / F::TPL, j = threadIdx.x % F::TPL;
        for (int y0 = 0; y0 < F::RPC; y0 += F::ROWS) {
            const int yl = y0 + line;
            const bool valid = yl < F::RPC;
            const int y = rank * F::RPC + yl;
            cpx<T> v[E];
#pragma unroll
            for (int r = 0; r < E; ++r) {
                v[r] = {T(0), T(0)};
                if (r < E / 2 && valid) {
                    const int x = j + r * (P / E);
                    v[r] = src_pair<T, TIN>(d.src[0], d.src[1], s0, s1, N, z, y, x);
                }
            }
            fft_line<T, P, E, false, (1u << (E / 2)) - 1u>(v, j, sm_tw,
                                     LineView<T, 1, true, Log2E<E>::value>{scr + line * F::LS});
            if (valid) {
#pragma unroll
                for (int s = 0; s < E; ++s) slab[yl * P + out_index<P, E>(j, s)] = v[s];
            }
        }
    }
    cluster.sync();
    // phase 2: columns along y, inputs from the owning CTAs
    {
        const int l = threadIdx.x % F::TX, j = threadIdx.x / F::TX;
        cpx<T>* dst = d.work + (size_t)z * P * P;
        for (int c0 = 0; c0 < F::CPC; c0 += F::TX) {
            const int kx = rank * F::CPC + c0 + l;
            cpx<T> v[E];
#pragma unroll
            for (int r = 0; r < E; ++r) {
                v[r] = {T(0), T(0)};
                if (r < E / 2) {
                    const int y = j + r * (P / E);
                    const cpx<T>* src = cluster.map_shared_rank(slab, y / F::RPC);
                    v[r] = src[(y % F::RPC) * P + kx];
                }
            }
            fft_line<T, P, E, false, (1u << (E / 2)) - 1u>(v, j, sm_tw, LineView<T, F::TX, false>{scr + l});
#pragma unroll
            for (int s = 0; s < E; ++s) dst[(size_t)out_index<P, E>(j, s) * P + kx] = v[s];
        }
    }
    cluster.sync();
}

template <typename T, int P>
__global__ void __cluster_dims__(FusedShape<T, P>::C, 1, 1) __launch_bounds__(FusedShape<T, P>::NT)
    k_yxinv(const __grid_constant__ ConvArgs<T> a) {
    using F = FusedShape<T, P>;
    constexpr int N = P / 2, E = F::E, C = F::C;
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T>* sm_tw = reinterpret_cast<cpx<T>*>(smem_raw);
    cpx<T>* slab = sm_tw + P;                    // [N][CPC]
    cpx<T>* scr = slab + (size_t)N * F::CPC;
    const int rank = (int)cluster.block_rank();
    const int z = blockIdx.x / C;
    const PairDesc<T>& d = a.pair[blockIdx.y];
    load_twiddles<P, E>(sm_tw, a.tw);
    __syncthreads();
    // phase 1: columns along y (inverse), keep y < N
    {
        const int l = threadIdx.x % F::TX, j = threadIdx.x / F::TX;
        const cpx<T>* src = d.work + (size_t)z * P * P;
        for (int c0 = 0; c0 < F::CPC; c0 += F::TX) {
            const int kxl = c0 + l;
            const int kx = rank * F::CPC + kxl;
            cpx<T> v[E];
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = src[(size_t)(j + r * (P / E)) * P + kx];
            fft_line<T, P, E, true>(v, j, sm_tw, LineView<T, F::TX, false>{scr + l});
#pragma unroll
            for (int s = 0; s < E; ++s) {
                const int e = out_index<P, E>(j, s);
                if (e < N) slab[e * F::CPC + kxl] = v[s];
            }
        }
    }
    cluster.sync();
    // phase 2: rows along x (inverse), inputs from the owning CTAs
    {
        const int line = threadIdx.x / F::TPL, j = threadIdx.x % F::TPL;
        for (int y0 = 0; y0 < F::RPC; y0 += F::ROWS) {
            const int yl = y0 + line;
            const bool valid = yl < F::RPC;
            const int y = rank * F::RPC + yl;
            cpx<T> v[E];
#pragma unroll
            for (int r = 0; r < E; ++r) {
                v[r] = {T(0), T(0)};
                if (valid) {
                    const int kx = j + r * (P / E);
                    const cpx<T>* src = cluster.map_shared_rank(slab, kx / F::CPC);
                    v[r] = src[y * F::CPC + kx % F::CPC];
                }
            }
            fft_line<T, P, E, true>(v, j, sm_tw,
                                    LineView<T, 1, true, Log2E<E>::value>{scr + line * F::LS});
            if (valid) {
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    const int e = out_index<P, E>(j, s);
                    if (e < N) {
                        store_out<T, P>(d.dst[0], z, y, e, v[s].re);
                        store_out<T, P>(d.dst[1], z, y, e, v[s].im);
                    }
                }
            }
        }
    }
    cluster.sync();
}

}  // namespace nm
