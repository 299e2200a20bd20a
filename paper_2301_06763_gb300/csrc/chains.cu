// chains.cu -- the two level-to-level chains of a solve, each as one launch
// over every level of every mesh of a batch.
//
// Restriction (Sect. 4 and Sect. 7: the coarse grid carries the fine mass).
// restr_m, the covered cells a in [0, N/2)^3 of level m (level index
// N/4 + a), is the mean of the 8 children 2a + d on level m+1, a child
// covered by level m+2 (2a + d in [N/4, 3N/4)^3, i.e. a in [N/8, 3N/8)^3)
// taking restr_{m+1}[2a + d - N/4] instead of its own density.  Written as a
// chain, level m waits for level m+1.  Here the cells of restr_m split into a
// shell, whose children are all uncovered (raw densities of level m+1), and a
// core [N/8, 3N/8)^3, which is the plain 2x restriction R of all of
// restr_{m+1}.  Unrolled,
//   restr_m = S_m  u  R(S_{m+1})  u  R^2(S_{m+2})  u ...  u  R^(L-2-m)(restr_{L-2}),
// every piece computed from raw densities and then halved in place.  One CTA
// takes one T^3 tile of a shell S_k (or of restr_{L-2}, all of whose
// children are uncovered), restricts its (2T)^3 raw children, and halves the
// tile lg T times, writing each image R^j(tile) -- T/2^j cells a side -- to
// restr_{k-j}.  The images of distinct tiles are disjoint and together tile
// each level, so the launch leaves restr_m complete for every m >= L-2-lg T;
// coarser levels (meshes deeper than lg T + 2 levels) are finished by the
// per-level kernel afterwards.  The tile is T = min(16, N/8), which keeps
// every shell tile wholly inside or outside the core on each axis and every
// image origin even.  Each restricted value is summed in the same order as
// the per-level kernel (children pairs along x, then y, then z), so both give
// identical bits.
//
// Carried interpolation (Eqs. 3-6 applied level by level): S_0 = the hole
// potential of level 0 on its crop, S_n = D(S_{n-1}) + hole_n on the
// (N/2+2)^3 cells of level n from N/4-1 on (n = 1 .. L-2), D the two-point
// rule.  S_n at level-n index i reads S_{n-1} at (N/2+i)>>1 and one diagonal
// neighbour, so a box of S_n needs a box of S_{n-1} about half as wide plus
// a margin of one cell.  One CTA takes one tile of one S_n, computes the boxes
// of S_1 .. S_{n-1} its tile depends on in shared memory (a few hundred cells
// each), and writes the tile; the ancestors are recomputed by every CTA that
// needs them, with the per-level kernel's arithmetic, so the values are the
// same bits as the chain's.
#include "../../include/nm.h"
#include "internal.h"
#include "dfloat.cuh"
#include "assemble.cuh"

namespace nm {

static int ilog2i(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// ---------------------------------------------------------------- restriction

template <typename TIN> struct RestrictTreeArgs {
    RestrictMesh<TIN> mesh[kTreeMeshes];
    int first[kTreeMeshes + 1];   // first CTA of each mesh; first[nmesh] = grid
    int nmesh;
};

constexpr int kRestrictTile = 16;
constexpr int kRestrictThreads = 256;
// output pairs per thread and batch (a 16^3 tile: 2048 pairs, 2 batches of
// 256 x 4 for float, 4 of 256 x 2 for double, whose loads take twice the
// registers); two CTAs per SM hold the 288 tiles of a 6 x 128^3 mesh at once
template <typename TIN> struct RestrictPer { static constexpr int value = sizeof(TIN) == 4 ? 4 : 2; };

// Four consecutive densities from a 16-byte aligned address.
template <typename TIN> struct Load4;
template <> struct Load4<float> {
    static __device__ __forceinline__ void load(const float* p, float* v) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <> struct Load4<double> {
    static __device__ __forceinline__ void load(const double* p, double* v) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

// Tile edge of a mesh: min(16, N/8) (N >= 16).
__host__ __device__ inline int restrict_tile(int N) { return N / 8 < kRestrictTile ? N / 8 : kRestrictTile; }

// The s-th tile (in z, y, x order) of a G^3 tiling that lies outside the
// central [G/4, 3G/4)^3 block.
__device__ inline void shell_tile(int s, int G, int& tz, int& ty, int& tx) {
    const int g4 = G / 4, g34 = 3 * G / 4, c = G / 2;
    for (int z = 0; z < G; ++z) {
        const bool zc = z >= g4 && z < g34;
        const int cnt = zc ? G * G - c * c : G * G;
        if (s < cnt) {
            tz = z;
            if (!zc) {
                ty = s / G;
                tx = s % G;
                return;
            }
            for (int y = 0; y < G; ++y) {
                const bool yc = y >= g4 && y < g34;
                const int rc = yc ? G - c : G;
                if (s < rc) {
                    ty = y;
                    tx = yc ? (s < g4 ? s : s + c) : s;
                    return;
                }
                s -= rc;
            }
        }
        s -= cnt;
    }
    tz = ty = tx = 0;   // not reached for s below the shell count
}

// One tile of restr_k (edge T, a compile-time constant so that every index
// is shifts and masks) and its images on the coarser levels down to mmin.
template <typename TIN, int T>
__device__ __forceinline__ void restrict_tile_body(const RestrictMesh<TIN>& M, int k, int tz, int ty, int tx,
                                                   int mmin, TIN* buf0, TIN* buf1) {
    constexpr int TH = T / 2, LGT = T == 16 ? 4 : T == 8 ? 3 : T == 4 ? 2 : 1;
    constexpr int PAIRS = T * T * TH;
    constexpr int PER = RestrictPer<TIN>::value;
    const int N = M.N, h = N / 2, q = N / 4;
    const size_t N3 = (size_t)N * N * N, h3 = N3 / 8;
    // the tile of restr_k: cells [o, o + T)^3, children on level k+1 raw
    const TIN* rho = M.rho + (size_t)(k + 1) * N3;
    TIN* out = M.restr + (size_t)k * h3;
    const int oz = tz * T, oy = ty * T, ox = tx * T;
    // every thread's children loads are issued before any sum (up to PER
    // output pairs per thread), so that a CTA has its input in flight at once
#pragma unroll 1
    for (int p0 = 0; p0 < PAIRS; p0 += PER * kRestrictThreads) {
        TIN w[PER][4][4];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int p = p0 + u * kRestrictThreads + (int)threadIdx.x;
            if (p < PAIRS) {
                const int cx = 2 * (p % TH), cy = (p / TH) % T, cz = p / (TH * T);
                const TIN* src = rho + ((size_t)(2 * (oz + cz)) * N + 2 * (oy + cy)) * N + 2 * (ox + cx);
#pragma unroll
                for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy)
                        Load4<TIN>::load(src + ((size_t)dz * N + dy) * N, w[u][2 * dz + dy]);
            }
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int p = p0 + u * kRestrictThreads + (int)threadIdx.x;
            if (p < PAIRS) {
                const int cx = 2 * (p % TH), cy = (p / TH) % T, cz = p / (TH * T);
                TIN s0 = TIN(0), s1 = TIN(0);
#pragma unroll
                for (int r = 0; r < 4; ++r) {   // (dz, dy) = (0,0), (0,1), (1,0), (1,1)
                    s0 += w[u][r][0] + w[u][r][1];
                    s1 += w[u][r][2] + w[u][r][3];
                }
                s0 *= TIN(0.125);
                s1 *= TIN(0.125);
                buf0[(cz * T + cy) * T + cx] = s0;
                buf0[(cz * T + cy) * T + cx + 1] = s1;
                TIN* o = out + ((size_t)(oz + cz) * h + (oy + cy)) * h + ox + cx;
                o[0] = s0;
                o[1] = s1;
            }
        }
    }
    // images R^j(tile) on restr_{k-j}: origin (o_{j-1} + N/4) / 2
    int sz = oz, sy = oy, sx = ox;
#pragma unroll
    for (int j = 1; j <= LGT; ++j) {
        if (k - j < mmin) break;
        __syncthreads();
        const int S = T >> (j - 1), S2 = S / 2;
        const TIN* src = (j & 1) ? buf0 : buf1;
        TIN* dst = (j & 1) ? buf1 : buf0;
        sz = (sz + q) / 2;
        sy = (sy + q) / 2;
        sx = (sx + q) / 2;
        TIN* lout = M.restr + (size_t)(k - j) * h3;
        for (int c = threadIdx.x; c < S2 * S2 * S2; c += kRestrictThreads) {
            const int x = c % S2, y = (c / S2) % S2, z = c / (S2 * S2);
            TIN s0 = TIN(0);
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    const TIN* r = src + ((2 * z + dz) * S + (2 * y + dy)) * S + 2 * x;
                    s0 += r[0] + r[1];
                }
            s0 *= TIN(0.125);
            dst[(z * S2 + y) * S2 + x] = s0;
            lout[((size_t)(sz + z) * h + (sy + y)) * h + (sx + x)] = s0;
        }
    }
}

template <typename TIN>
__global__ void __launch_bounds__(kRestrictThreads, 2) k_restrict_tree(const __grid_constant__ RestrictTreeArgs<TIN> a) {
    constexpr int T_MAX = kRestrictTile;
    __shared__ TIN buf0[T_MAX * T_MAX * T_MAX];
    __shared__ TIN buf1[(T_MAX / 2) * (T_MAX / 2) * (T_MAX / 2)];
    int mi = 0;
    while (mi + 1 < a.nmesh && (int)blockIdx.x >= a.first[mi + 1]) ++mi;
    const RestrictMesh<TIN>& M = a.mesh[mi];
    const int N = M.N, L = M.L, h = N / 2;
    const int T = restrict_tile(N), lgT = __ffs(T) - 1, G = h / T;
    int mmin = L - 2 - lgT;
    if (mmin < 0) mmin = 0;
    int t = (int)blockIdx.x - a.first[mi];
    int k, tz, ty, tx;
    if (t < G * G * G) {
        k = L - 2;
        tz = t / (G * G);
        ty = (t / G) % G;
        tx = t % G;
    } else {
        t -= G * G * G;
        const int S = G * G * G - (G / 2) * (G / 2) * (G / 2);
        k = L - 3 - t / S;
        shell_tile(t % S, G, tz, ty, tx);   // k >= mmin: the launch holds no shell below
    }
    switch (T) {
        case 16: restrict_tile_body<TIN, 16>(M, k, tz, ty, tx, mmin, buf0, buf1); break;
        case 8: restrict_tile_body<TIN, 8>(M, k, tz, ty, tx, mmin, buf0, buf1); break;
        case 4: restrict_tile_body<TIN, 4>(M, k, tz, ty, tx, mmin, buf0, buf1); break;
        default: restrict_tile_body<TIN, 2>(M, k, tz, ty, tx, mmin, buf0, buf1); break;
    }
}

template <typename TIN>
cudaError_t run_restrict_tree(const RestrictMesh<TIN>* meshes, int n, cudaStream_t s) {
    // meshes the tree takes: N >= 16 (a tile of at least 2) on 16-byte
    // aligned densities; the others keep the per-level chain
    std::vector<RestrictMesh<TIN>> tree;
    for (int i = 0; i < n; ++i) {
        const RestrictMesh<TIN>& m = meshes[i];
        if (m.L < 2) continue;
        const bool ok = m.N >= 16 && ((uintptr_t)m.rho & 15) == 0 && ((uintptr_t)m.restr & 15) == 0;
        if (ok) {
            tree.push_back(m);
            continue;
        }
        const size_t N3 = (size_t)m.N * m.N * m.N, h3 = N3 / 8;
        for (int k = m.L - 2; k >= 0; --k) {
            cudaError_t e = run_restrict<TIN>(m.rho + (size_t)(k + 1) * N3,
                                              k + 1 < m.L - 1 ? m.restr + (size_t)(k + 1) * h3 : nullptr,
                                              m.restr + (size_t)k * h3, m.N, s);
            if (e != cudaSuccess) return e;
        }
    }
    for (size_t b = 0; b < tree.size(); b += kTreeMeshes) {
        const size_t e_ = b + kTreeMeshes < tree.size() ? b + kTreeMeshes : tree.size();
        RestrictTreeArgs<TIN> args{};
        int grid = 0;
        args.nmesh = (int)(e_ - b);
        for (size_t i = b; i < e_; ++i) {
            const RestrictMesh<TIN>& m = tree[i];
            const int G = (m.N / 2) / restrict_tile(m.N);
            int mmin = m.L - 2 - ilog2i(restrict_tile(m.N));
            if (mmin < 0) mmin = 0;
            args.mesh[i - b] = m;
            args.first[i - b] = grid;
            // restr_{L-2} whole, then the shells of levels L-3 .. mmin
            grid += G * G * G + (m.L - 2 - mmin) * (G * G * G - (G / 2) * (G / 2) * (G / 2));
        }
        args.first[args.nmesh] = grid;
        {
            ProfScope ps(sizeof(TIN) == 4 ? "restrict_tree_f32" : "restrict_tree_f64", args.nmesh, s);
            k_restrict_tree<TIN><<<grid, kRestrictThreads, 0, s>>>(args);
            count_launches(1);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    // levels below the tree's reach: the per-level kernel, coarsest last
    for (const RestrictMesh<TIN>& m : tree) {
        const int mmin = m.L - 2 - ilog2i(restrict_tile(m.N));
        const size_t N3 = (size_t)m.N * m.N * m.N, h3 = N3 / 8;
        for (int k = mmin - 1; k >= 0; --k) {
            cudaError_t e = run_restrict<TIN>(m.rho + (size_t)(k + 1) * N3, m.restr + (size_t)(k + 1) * h3,
                                              m.restr + (size_t)k * h3, m.N, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}
template cudaError_t run_restrict_tree<float>(const RestrictMesh<float>*, int, cudaStream_t);
template cudaError_t run_restrict_tree<double>(const RestrictMesh<double>*, int, cudaStream_t);

// ---------------------------------------------------------------- carried interpolation

template <typename T> struct CarryTreeArgs {
    CarryMesh<T> mesh[kTreeMeshes];
    int first[kTreeMeshes + 1];   // first CTA of each mesh; first[nmesh] = grid
    int nmesh;
};

constexpr int kCarryTile = 12;   // tile edge of S_n
constexpr int kCarryBox = 9;     // widest ancestor box: (kCarryTile - 1) / 2 + 3 rounded up
constexpr int kCarryThreads = 256;

// The box of level-(n-1) cells a level-n box [lo, hi] reads on one axis: the
// coarse indices (N/2 + i) >> 1 and one neighbour on either side.
__device__ __forceinline__ void parent_box(int N, int lo, int hi, int rlo, int rhi, int& plo, int& phi) {
    plo = ((N / 2 + lo) >> 1) - 1;
    phi = ((N / 2 + hi) >> 1) + 1;
    if (plo < rlo) plo = rlo;
    if (phi > rhi) phi = rhi;
}

template <typename T>
__global__ void __launch_bounds__(kCarryThreads) k_carry_tree(const __grid_constant__ CarryTreeArgs<T> a) {
    constexpr int B3 = kCarryBox * kCarryBox * kCarryBox;
    __shared__ T buf[2][B3];
    int mi = 0;
    while (mi + 1 < a.nmesh && (int)blockIdx.x >= a.first[mi + 1]) ++mi;
    const CarryMesh<T>& M = a.mesh[mi];
    const int N = M.N, nc = N / 2 + 2, o = N / 4 - 1;
    const int Gc = (nc + kCarryTile - 1) / kCarryTile, G3 = Gc * Gc * Gc;
    const int t = (int)blockIdx.x - a.first[mi];
    const int n = 1 + t / G3, r = t % G3;
    // boxes per axis: level n's tile, then its ancestors down to level 1
    int lo[16][3], hi[16][3];
    {
        const int tc[3] = {r / (Gc * Gc), (r / Gc) % Gc, r % Gc};
        for (int d = 0; d < 3; ++d) {
            lo[n][d] = o + tc[d] * kCarryTile;
            hi[n][d] = lo[n][d] + kCarryTile - 1;
            if (hi[n][d] > o + nc - 1) hi[n][d] = o + nc - 1;
        }
        for (int k = n - 1; k >= 1; --k)
            for (int d = 0; d < 3; ++d) parent_box(N, lo[k + 1][d], hi[k + 1][d], o, o + nc - 1, lo[k][d], hi[k][d]);
    }
    const size_t nc3 = (size_t)nc * nc * nc;
    const int ho = M.hole_origin, hE = M.hole_extent;
    for (int k = 1; k <= n; ++k) {
        const int ez = hi[k][0] - lo[k][0] + 1, ey = hi[k][1] - lo[k][1] + 1, ex = hi[k][2] - lo[k][2] + 1;
        const T* hole = M.hole + (size_t)k * M.hole_stride;
        const T* prev_g = M.hole;                      // S_0: level 0's hole potential
        const T* prev_s = buf[(k - 1) & 1];            // S_{k-1} on its box (k >= 2)
        T* cur = buf[k & 1];
        const int pz = k >= 2 ? lo[k - 1][0] : 0, py = k >= 2 ? lo[k - 1][1] : 0, px = k >= 2 ? lo[k - 1][2] : 0;
        const int pey = k >= 2 ? hi[k - 1][1] - lo[k - 1][1] + 1 : 0;
        const int pex = k >= 2 ? hi[k - 1][2] - lo[k - 1][2] + 1 : 0;
        // cell c = threadIdx.x + i blockDim.x of the box, its (z, y, x)
        // advanced by the fixed step instead of divided out per cell
        const int cells = ez * ey * ex;
        const int stx = kCarryThreads % ex, sty = (kCarryThreads / ex) % ey, stz = kCarryThreads / (ex * ey);
        int bx = (int)threadIdx.x % ex, by = ((int)threadIdx.x / ex) % ey, bz = (int)threadIdx.x / (ex * ey);
        const T* __restrict__ hk = hole;
        T* __restrict__ outk = M.out + (size_t)(n - 1) * nc3;
        const int lz = lo[k][0], ly = lo[k][1], lx = lo[k][2];
#pragma unroll 4
        for (int c = threadIdx.x; c < cells; c += kCarryThreads) {
            const int x = lx + bx, y = ly + by, z = lz + bz;
            int cz, sz, cy, sy, cx, sx;
            diag_axis(N, z, cz, sz);
            diag_axis(N, y, cy, sy);
            diag_axis(N, x, cx, sx);
            T near, diag;
            if (k == 1) {
                near = prev_g[((cz - ho) * hE + (cy - ho)) * hE + (cx - ho)];
                diag = prev_g[((cz + sz - ho) * hE + (cy + sy - ho)) * hE + (cx + sx - ho)];
            } else {
                near = prev_s[((cz - pz) * pey + (cy - py)) * pex + (cx - px)];
                diag = prev_s[((cz + sz - pz) * pey + (cy + sy - py)) * pex + (cx + sx - px)];
            }
            const T hv = hk[((z - ho) * hE + (y - ho)) * hE + (x - ho)];
            const T v = carry_value(near, diag, hv);
            if (k < n) cur[c] = v;
            else outk[((z - o) * nc + (y - o)) * nc + (x - o)] = v;
            bx += stx;
            int up = 0;
            if (bx >= ex) {
                bx -= ex;
                up = 1;
            }
            by += sty + up;
            up = 0;
            if (by >= ey) {
                by -= ey;
                up = 1;
            }
            bz += stz + up;
        }
        __syncthreads();
    }
}

template <typename T>
cudaError_t run_carry_tree(const CarryMesh<T>* meshes, int n, cudaStream_t s) {
    for (int b = 0; b < n; b += kTreeMeshes) {
        const int e_ = b + kTreeMeshes < n ? b + kTreeMeshes : n;
        CarryTreeArgs<T> args{};
        int grid = 0;
        for (int i = b; i < e_; ++i) {
            const CarryMesh<T>& m = meshes[i];
            if (m.L < 3) continue;   // no carried level
            const int nc = m.N / 2 + 2, Gc = (nc + kCarryTile - 1) / kCarryTile;
            args.mesh[args.nmesh] = m;
            args.first[args.nmesh] = grid;
            ++args.nmesh;
            grid += (m.L - 2) * Gc * Gc * Gc;
        }
        if (!args.nmesh) continue;
        args.first[args.nmesh] = grid;
        ProfScope ps(sizeof(T) == 4 ? "carry_tree_f32" : "carry_tree_f64", args.nmesh, s);
        k_carry_tree<T><<<grid, kCarryThreads, 0, s>>>(args);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
template cudaError_t run_carry_tree<float>(const CarryMesh<float>*, int, cudaStream_t);
template cudaError_t run_carry_tree<double>(const CarryMesh<double>*, int, cudaStream_t);
template cudaError_t run_carry_tree<df>(const CarryMesh<df>*, int, cudaStream_t);

}  // namespace nm
