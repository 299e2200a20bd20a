// tma.cuh -- the z-seam pass (forward z transform, spectrum multiply, inverse
// z transform; Sect. 3, Eq. 11) as a persistent kernel fed by the Tensor
// Memory Accelerator.
//
// A tile is TX adjacent columns (kx) of one ky row, all z < N: an N x TX
// complex block at stride P^2 in the work buffer.  Each CTA walks tiles
// t = blockIdx.x, + gridDim.x, ... through two shared-memory stages: while it
// transforms tile t in stage s, the TMA engine has already loaded tile t + G
// into stage s^1, and after tile t's result has been stored back (TMA store,
// in place) stage s is refilled with tile t + 2G.  Completion of each load is
// tracked by an mbarrier; every wait is bounded in clock cycles and a CTA
// whose wait runs out stops, drains its outstanding copies (again bounded) and
// raises NM_ETIMEOUT in the library's device status word.
#pragma once
#include <cuda.h>

#include "conv.cuh"

namespace nm {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of `parity` to complete: false after `limit`
// clock cycles without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int c0, int c1,
                                             int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(map),
                 "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <typename T> struct TmaArgs {
    CUtensorMap map[kMaxPairs];   // per pair: the [P/2][P][2P] view of its work buffer
    const T* spec;                // unit spectrum octant (P/2+1)^3
    const cpx<T>* tw;             // twiddles, P entries
    int npairs;
    int fault_skip_load;          // test hook: issue no loads, so the waits run out
    long long timeout;            // clock cycles allowed per wait
    int* status;                  // device status word (NM_ETIMEOUT on timeout)
};

template <typename T, int P, int E, int TX>
__global__ void __launch_bounds__(TX * P / E) k_zseam_tma(const __grid_constant__ TmaArgs<T> a) {
    constexpr int N = P / 2, H = P / 2 + 1;
    constexpr int TILE = P * TX;          // complex values per stage
    constexpr int XT = P / TX;            // column tiles per ky row
    constexpr int TILES = P * XT;         // tiles per pair
    constexpr uint32_t TX_BYTES = (uint32_t)(N * TX * sizeof(cpx<T>));
    extern __shared__ __align__(128) unsigned char smem_tma[];
    cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_tma);
    cpx<T>* sm_tw = buf + 2 * TILE;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm_tw + P);
    const int tid = threadIdx.x, l = tid % TX, j = tid / TX;
    const int total = a.npairs * TILES;
    const int G = gridDim.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    load_twiddles<P, E>(sm_tw, a.tw);
    __syncthreads();
    // loads issued and not yet consumed, with the phase parity each completes
    // (tracked by thread 0, the only thread that issues copies)
    bool pending[2] = {false, false};
    uint32_t pend_parity[2] = {0u, 0u};
    auto issue = [&](int t, int s) {
        const int pair = t / TILES, r = t - pair * TILES;
        const int y = r / XT, x0 = (r - y * XT) * TX;
        mbar_expect_tx(&bar[s], TX_BYTES);
        tma_load_3d(buf + s * TILE, &a.map[pair], &bar[s], 2 * x0, y, 0);
        pending[s] = true;
        pend_parity[s] = (uint32_t)((((t - (int)blockIdx.x) / G) >> 1) & 1);
    };
    if (tid == 0 && !a.fault_skip_load) {
        if ((int)blockIdx.x < total) issue(blockIdx.x, 0);
        if ((int)blockIdx.x + G < total) issue(blockIdx.x + G, 1);
    }
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < total; t += G, ++it) {
        const int s = it & 1;
        cpx<T>* tile = buf + s * TILE;
        const bool got = mbar_wait(&bar[s], (uint32_t)((it >> 1) & 1), a.timeout);
        if (!__syncthreads_and(got)) {
            ok = false;
            break;
        }
        if (tid == 0) pending[s] = false;
        const int pair = t / TILES, r = t - pair * TILES;
        const int y = r / XT, x0 = (r - y * XT) * TX;
        const int x = x0 + l;
        cpx<T> v[E];
#pragma unroll
        for (int q = 0; q < E; ++q) {
            if (q < E / 2) v[q] = tile[(j + q * (P / E)) * TX + l];
            else v[q] = {T(0), T(0)};
        }
        __syncthreads();
        const LineView<T, TX, false> view{tile + l};
        fft_line<T, P, E, false, (1u << (E / 2)) - 1u>(v, j, sm_tw, view);
        const int fy = y <= P / 2 ? y : P - y;
        const int fx = x <= P / 2 ? x : P - x;
        const T* sp = a.spec + (size_t)fy * H + fx;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int kz = out_index<P, E>(j, q);
            const int fz = kz <= P / 2 ? kz : P - kz;
            const T g = __ldg(sp + (size_t)fz * H * H);
            v[q].re *= g;
            v[q].im *= g;
        }
        seam_permute<T, P, E>(v);
        fft_line<T, P, E, true>(v, j, sm_tw, view);
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int e = out_index<P, E>(j, q);
            if (e < N) tile[e * TX + l] = v[q];
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tma_store_3d(&a.map[pair], tile, 2 * x0, y, 0);
            bulk_commit();
            const int tn = t + 2 * G;
            if (tn < total && !a.fault_skip_load) {
                bulk_wait_read0();
                issue(tn, s);
            }
        }
    }
    if (tid == 0) {
        if (!ok) {
            // drain loads still in flight into this CTA's shared memory
            for (int s = 0; s < 2; ++s)
                if (pending[s]) mbar_wait(&bar[s], pend_parity[s], a.timeout);
            if (a.status) atomicExch(a.status, 4 /* NM_ETIMEOUT */);
        }
        bulk_wait0();
    }
}

}  // namespace nm
