// support.cu -- restriction, Green spectrum and final assembly kernels.
#include <mutex>
#include <vector>

#include "../../include/nm.h"
#include "internal.h"
#include "dfloat.cuh"
#include "assemble.cuh"

namespace nm {

static int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// ---------------------------------------------------------------- restriction
// Covered cells of level m (index [N/4, 3N/4)^3) take the mean of their 2^3
// children on level m+1 (Sect. 4 and Sect. 7: the coarse grid carries the fine
// mass).  Children that are themselves covered by level m+2 take that level's
// restricted value, so sweeping m from the finest level up gives every covered
// cell the mean of the finest data below it.
template <typename TIN>
__global__ void k_restrict(const TIN* __restrict__ rho_child, const TIN* __restrict__ restr_child,
                           TIN* __restrict__ out, int lgN) {
    const int N = 1 << lgN, h = N / 2, q = N / 4, lgh = lgN - 1;
    const int n = h * h * h;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = i & (h - 1), b = (i >> lgh) & (h - 1), a = i >> (2 * lgh);
        TIN s = TIN(0);
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const int z = 2 * a + dz, y = 2 * b + dy, x = 2 * c + dx;
                    const bool cov = restr_child && (unsigned)(z - q) < (unsigned)h &&
                                     (unsigned)(y - q) < (unsigned)h &&
                                     (unsigned)(x - q) < (unsigned)h;
                    s += cov ? restr_child[((size_t)(z - q) * h + (y - q)) * h + (x - q)]
                             : rho_child[((size_t)z * N + y) * N + x];
                }
        out[i] = s * TIN(0.125);
    }
}

// Two adjacent outputs per thread (N >= 16): their 2 x 2 x 4 children are
// contiguous runs of 4 along x, read as 16-byte vectors, and the 8 children of
// each output are either all covered by the next level or none (the covered
// range [N/4, 3N/4) starts and ends on even indices), the same for both.
template <typename TIN> struct Vec4In;
template <> struct Vec4In<float> {
    static __device__ __forceinline__ void load(const float* p, float* v) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <> struct Vec4In<double> {
    static __device__ __forceinline__ void load(const double* p, double* v) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

template <typename TIN>
__global__ void k_restrict2(const TIN* __restrict__ rho_child, const TIN* __restrict__ restr_child,
                            TIN* __restrict__ out, int lgN) {
    const int N = 1 << lgN, h = N / 2, q = N / 4, lgh = lgN - 1;
    const int n = (h * h * h) / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = 2 * (i & (h / 2 - 1)), b = (i >> (lgh - 1)) & (h - 1), a = i >> (2 * lgh - 1);
        TIN s0 = TIN(0), s1 = TIN(0);
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const int z = 2 * a + dz, y = 2 * b + dy, x = 2 * c;
                const bool cov = restr_child && (unsigned)(z - q) < (unsigned)h &&
                                 (unsigned)(y - q) < (unsigned)h && (unsigned)(x - q) < (unsigned)h;
                TIN w[4];
                if (cov)
                    Vec4In<TIN>::load(restr_child + ((size_t)(z - q) * h + (y - q)) * h + (x - q), w);
                else
                    Vec4In<TIN>::load(rho_child + ((size_t)z * N + y) * N + x, w);
                s0 += w[0] + w[1];
                s1 += w[2] + w[3];
            }
        out[2 * i] = s0 * TIN(0.125);
        out[2 * i + 1] = s1 * TIN(0.125);
    }
}

template <typename TIN>
cudaError_t run_restrict(const TIN* rho_child, const TIN* restr_child, TIN* restr_out, int N,
                         cudaStream_t s) {
    const int n = (N / 2) * (N / 2) * (N / 2);
    ProfScope ps(sizeof(TIN) == 4 ? "restrict_f32" : "restrict_f64", 1, s);
    const bool vec = N >= 16 && ((uintptr_t)rho_child & 15) == 0 && ((uintptr_t)restr_child & 15) == 0;
    if (vec) {
        k_restrict2<TIN><<<(n / 2 + 255) / 256, 256, 0, s>>>(rho_child, restr_child, restr_out, ilog2(N));
        count_launches(1);
        return cudaGetLastError();
    }
    const int blocks = (n + 255) / 256;
    k_restrict<TIN><<<blocks, 256, 0, s>>>(rho_child, restr_child, restr_out, ilog2(N));
    count_launches(1);
    return cudaGetLastError();
}
template cudaError_t run_restrict<float>(const float*, const float*, float*, int, cudaStream_t);
template cudaError_t run_restrict<double>(const double*, const double*, double*, int, cudaStream_t);

// ---------------------------------------------------------------- Green spectrum
// The unit-cell kernel of Eq. 10 (1/|d| for integer offsets d != 0, the
// Eq. 13 self term C at d = 0) on the doubled domain of Fig. 4 is real and even
// in every axis, so its 3-D transform is real and even and equals a 3-D DCT-I
// of the octant d in [0, N]^3:
//   S(k) = sum_d w(dx) w(dy) w(dz) g(d) cos(2 pi kx dx/P) cos(..y..) cos(..z..),
// w = 1 at d in {0, N}, 2 otherwise.  One axis per pass, all in double; the
// cosines come from a table of cos(2 pi t / P) built on the host.
__device__ __forceinline__ double green_unit(int a, int b, int c, double self_term) {
    if ((a | b | c) == 0) return self_term;
    return 1.0 / sqrt((double)a * a + (double)b * b + (double)c * c);
}

__global__ void k_green_fill(double* __restrict__ out, int N, double self_term) {
    const int H = N + 1;
    const size_t n = (size_t)H * H * H;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = green_unit((int)(i / ((size_t)H * H)), (int)((i / H) % H), (int)(i % H),
                            self_term);
}

// one DCT-I pass along axis 0 (x, fastest), 1 (y) or 2 (z) of an H^3 array
__global__ void k_green_axis(const double* __restrict__ in, double* __restrict__ out,
                             const double* __restrict__ ctab, int N, int axis) {
    const int H = N + 1, P = 2 * N;
    const size_t n = (size_t)H * H * H;
    const size_t stride = axis == 0 ? 1 : axis == 1 ? (size_t)H : (size_t)H * H;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)((i / stride) % H);
        const size_t base = i - (size_t)k * stride;
        double s = 0.0;
        for (int d = 0; d <= N; ++d) {
            const double w = (d == 0 || d == N) ? 1.0 : 2.0;
            s += w * in[base + (size_t)d * stride] * ctab[(k * d) % P];
        }
        out[i] = s;
    }
}

cudaError_t run_green_octant(double* out, double* scratch, const double* ctab, int N,
                             double self_term, cudaStream_t s) {
    const size_t H = N + 1;
    const size_t n = H * H * H;
    const int blocks = (int)((n + 255) / 256 < 152 * 64 ? (n + 255) / 256 : 152 * 64);
    double* t1 = scratch;
    double* t2 = scratch + n;
    ProfScope ps("green_octant", 1, s);
    k_green_fill<<<blocks, 256, 0, s>>>(out, N, self_term);
    k_green_axis<<<blocks, 256, 0, s>>>(out, t1, ctab, N, 0);
    k_green_axis<<<blocks, 256, 0, s>>>(t1, t2, ctab, N, 1);
    k_green_axis<<<blocks, 256, 0, s>>>(t2, out, ctab, N, 2);
    count_launches(4);
    return cudaGetLastError();
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

__global__ void k_to_df(const double* __restrict__ in, df* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = df_from_double(in[i]);
}

// The octant S[fz][fy][fx] (fx <= N) as float rows over the whole kx range:
// out[(fz H + fy) P + x] = S[fz][fy][x <= N ? x : P - x], so that the kx
// columns of one z-seam tile are contiguous and 16-byte aligned.
__global__ void k_unfold_x(const double* __restrict__ in, float* __restrict__ out, int N) {
    const int H = N + 1, P = 2 * N;
    const size_t n = (size_t)H * H * P;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % P);
        const size_t row = i / P;
        out[i] = (float)in[row * H + (x <= N ? x : P - x)];
    }
}

cudaError_t run_unfold_x(const double* in, float* out, int N, cudaStream_t s) {
    const size_t n = (size_t)(N + 1) * (N + 1) * 2 * N;
    const int blocks = (int)((n + 255) / 256 < 152 * 32 ? (n + 255) / 256 : 152 * 32);
    k_unfold_x<<<blocks, 256, 0, s>>>(in, out, N);
    count_launches(1);
    return cudaGetLastError();
}

// The octant ([fz][fy][fx], double) as float with fz fastest: out[(fx H + fy)
// H + fz], so that one (kx, ky) line of the fused y/z/y pass reads its
// spectrum values as one contiguous run.
__global__ void k_zfast(const double* __restrict__ in, float* __restrict__ out, int N) {
    const int H = N + 1;
    const size_t n = (size_t)H * H * H;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int fz = (int)(i % H);
        const size_t r = i / H;
        const int fy = (int)(r % H), fx = (int)(r / H);
        out[i] = (float)in[((size_t)fz * H + fy) * H + fx];
    }
}

cudaError_t run_zfast(const double* in, float* out, int N, cudaStream_t s) {
    const size_t n = (size_t)(N + 1) * (N + 1) * (N + 1);
    const int blocks = (int)((n + 255) / 256 < 152 * 32 ? (n + 255) / 256 : 152 * 32);
    k_zfast<<<blocks, 256, 0, s>>>(in, out, N);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t run_to_df(const double* in, df* out, size_t n, cudaStream_t s) {
    const int blocks = (int)((n + 255) / 256 < 152 * 32 ? (n + 255) / 256 : 152 * 32);
    k_to_df<<<blocks, 256, 0, s>>>(in, out, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t run_to_float(const double* in, float* out, size_t n, cudaStream_t s) {
    const int blocks = (int)((n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536);
    k_to_float<<<blocks, 256, 0, s>>>(in, out, n);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_carry(const __grid_constant__ CarryArgs<T> a) {
    carry_body<T>(a, blockIdx.x * (size_t)blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

template <typename T>
cudaError_t run_carry(const CarryArgs<T>& a, cudaStream_t s) {
    ProfScope ps(sizeof(T) == 4 ? "carry_f32" : "carry_f64", 1, s);
    const size_t nc = a.N / 2 + 2, total = nc * nc * nc;
    size_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_carry<T><<<(int)blocks, 256, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}
template cudaError_t run_carry<float>(const CarryArgs<float>&, cudaStream_t);
template cudaError_t run_carry<double>(const CarryArgs<double>&, cudaStream_t);
template cudaError_t run_carry<df>(const CarryArgs<df>&, cudaStream_t);

// One thread per 4 consecutive cells along x (N >= 4): the z and y stencils of
// each coarser level are shared by the 4 cells.
template <typename T>
__global__ void k_assemble(const __grid_constant__ AssembleArgs<T> a, int lgN) {
    const int N = 1 << lgN;
    const size_t N3 = (size_t)1 << (3 * lgN);
    const size_t quads = (N3 >> 2) * a.levels;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < quads;
         q += (size_t)gridDim.x * blockDim.x) {
        const size_t idx = q << 2;
        const int n = (int)(idx >> (3 * lgN));
        const size_t cell = idx & (N3 - 1);
        const int x0 = (int)(cell & (N - 1)), y = (int)((cell >> lgN) & (N - 1)),
                  z = (int)(cell >> (2 * lgN));
        T b[4];
        Vec4<T>::load(a.base[n] + cell, b);
        T acc[4] = {T(0), T(0), T(0), T(0)};   // cross-level sum
        if (a.dbl[n]) {
            const int E = 2 * N;
            const T* d = a.dbl[n];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                T s = T(0);
#pragma unroll
                for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy) {
                        const T* row = d + ((size_t)(2 * z + dz) * E + (2 * y + dy)) * E + 2 * (x0 + c);
                        s += row[0] + row[1];
                    }
                acc[c] += s * T(0.125);
            }
        }
        if (a.red[n]) {
            T r[4];
            Vec4<T>::load(a.red[n] + cell, r);
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] += r[c];
        }
        if (a.diag && n > 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                acc[c] += diag_value<T>(a.interp[n - 1], a.interp_origin[n - 1], a.interp_extent[n - 1], N, z, y,
                                        x0 + c);
        }
        for (int k = 0; k < (a.diag ? 0 : n); ++k) {
            const int lgr = n - k;
            int iz, iy;
            T tz, ty;
            axis_stencil<T>(N, lgr, z, iz, tz);
            axis_stencil<T>(N, lgr, y, iy, ty);
            const int o = a.interp_origin[k], E = a.interp_extent[k];
            const size_t sz = (size_t)E * E, sy = E;
            const T* plane = a.interp[k] + ((size_t)(iz - o) * E + (iy - o)) * E - o;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int ix;
                T tx;
                axis_stencil<T>(N, lgr, x0 + c, ix, tx);
                const T* src = plane + ix;
                const T c00 = src[0] + tx * (src[1] - src[0]);
                const T c01 = src[sy] + tx * (src[sy + 1] - src[sy]);
                const T c10 = src[sz] + tx * (src[sz + 1] - src[sz]);
                const T c11 = src[sz + sy] + tx * (src[sz + sy + 1] - src[sz + sy]);
                const T c0 = c00 + ty * (c01 - c00);
                const T c1 = c10 + ty * (c11 - c10);
                acc[c] += c0 + tz * (c1 - c0);
            }
        }
        double2* out = reinterpret_cast<double2*>(a.phi + idx);
        out[0] = make_double2(out_sum(b[0], acc[0]), out_sum(b[1], acc[1]));
        out[1] = make_double2(out_sum(b[2], acc[2]), out_sum(b[3], acc[3]));
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_assemble_rows(const __grid_constant__ AssembleArgs<T> a, int lgN) {
    extern __shared__ __align__(16) unsigned char smem_rows[];
    const int rows_cta = 256 / ((1 << lgN) >> 2);
    assemble_rows_body<T>(a, lgN, (size_t)blockIdx.x * rows_cta, gridDim.x, smem_rows);
}

template <typename T>
cudaError_t run_assemble(const AssembleArgs<T>& a, cudaStream_t s) {
    ProfScope ps(sizeof(T) == 4 ? "assemble_f32" : "assemble_f64", a.levels, s);
    const int lgN = ilog2(a.N);
    if (a.N >= 16) {
        const int team = a.N / 4, rows_cta = 256 / team;
        const size_t rows = (size_t)a.N * a.N * a.levels;
        size_t blocks = rows / rows_cta;
        if (blocks > 152 * 16) blocks = 152 * 16;
        const size_t smem = (size_t)rows_cta * (a.N / 2 + 2) * sizeof(T);
        k_assemble_rows<T><<<(int)blocks, 256, smem, s>>>(a, lgN);
    } else {
        const size_t total = (size_t)a.N * a.N * a.N * a.levels / 4;
        size_t blocks = (total + 255) / 256;
        if (blocks > 152 * 64) blocks = 152 * 64;
        k_assemble<T><<<(int)blocks, 256, 0, s>>>(a, lgN);
    }
    count_launches(1);
    return cudaGetLastError();
}
template cudaError_t run_assemble<float>(const AssembleArgs<float>&, cudaStream_t);
template cudaError_t run_assemble<double>(const AssembleArgs<double>&, cudaStream_t);
template cudaError_t run_assemble<df>(const AssembleArgs<df>&, cudaStream_t);

// Several meshes' assemblies in one launch: CTAs [first[i], first[i+1]) walk
// the rows of mesh i as k_assemble_rows does (N >= 16).
template <typename T> struct AssembleBatchArgs {
    AssembleArgs<T> mesh[kAsmMeshes];
    int first[kAsmMeshes + 1];
    int lgN[kAsmMeshes];
    int nmesh;
};

template <typename T>
__global__ void __launch_bounds__(256) k_assemble_rows_batch(const __grid_constant__ AssembleBatchArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_rows[];
    int mi = 0;
    while (mi + 1 < a.nmesh && (int)blockIdx.x >= a.first[mi + 1]) ++mi;
    const int lgN = a.lgN[mi];
    const int rows_cta = 256 / ((1 << lgN) >> 2);
    const int b = (int)blockIdx.x - a.first[mi], nb = a.first[mi + 1] - a.first[mi];
    assemble_rows_body<T>(a.mesh[mi], lgN, (size_t)b * rows_cta, nb, smem_rows);
}

template <typename T>
cudaError_t run_assemble_batch(const AssembleArgs<T>* meshes, int n, cudaStream_t s) {
    std::vector<int> rows_path;
    for (int i = 0; i < n; ++i) {
        if (meshes[i].N >= 16) {
            rows_path.push_back(i);
        } else {
            cudaError_t e = run_assemble<T>(meshes[i], s);
            if (e != cudaSuccess) return e;
        }
    }
    for (size_t b = 0; b < rows_path.size(); b += kAsmMeshes) {
        const size_t e_ = b + kAsmMeshes < rows_path.size() ? b + kAsmMeshes : rows_path.size();
        static AssembleBatchArgs<T> args;   // host staging of the (large) parameter block
        static std::mutex mu;
        std::lock_guard<std::mutex> lk(mu);
        args = AssembleBatchArgs<T>{};
        int grid = 0, levels = 0;
        size_t smem = 0;
        args.nmesh = (int)(e_ - b);
        for (size_t i = b; i < e_; ++i) {
            const AssembleArgs<T>& m = meshes[rows_path[i]];
            const int team = m.N / 4, rows_cta = 256 / team;
            const size_t rows = (size_t)m.N * m.N * m.levels;
            size_t blocks = rows / rows_cta;
            if (blocks > 152 * 16) blocks = 152 * 16;
            const size_t sm = (size_t)rows_cta * (m.N / 2 + 2) * sizeof(T);
            if (sm > smem) smem = sm;
            args.mesh[i - b] = m;
            args.lgN[i - b] = ilog2(m.N);
            args.first[i - b] = grid;
            grid += (int)blocks;
            levels += m.levels;
        }
        args.first[args.nmesh] = grid;
        ProfScope ps(sizeof(T) == 4 ? "assemble_batch_f32" : "assemble_batch_f64", levels, s);
        k_assemble_rows_batch<T><<<grid, 256, smem, s>>>(args);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
template cudaError_t run_assemble_batch<float>(const AssembleArgs<float>*, int, cudaStream_t);
template cudaError_t run_assemble_batch<double>(const AssembleArgs<double>*, int, cudaStream_t);
template cudaError_t run_assemble_batch<df>(const AssembleArgs<df>*, int, cudaStream_t);

template <typename T>
cudaError_t run_assemble_interp(AssembleArgs<T> a, int interp, T* carry, cudaStream_t s) {
    if (interp == NM_INTERP_DIAGONAL) {
        // carried Eqs. 3-6 interpolation: level n reads S_{n-1} only, with
        // S_0 = Phi^0_hole and S_n = D(S_{n-1}) + Phi^n_hole (n = 1 .. L-2)
        const int N = a.N;
        const size_t nc = N / 2 + 2, nc3 = nc * nc * nc;
        a.diag = 1;
        for (int n = 1; n + 1 < a.levels; ++n) {
            CarryArgs<T> c{};
            c.prev = a.interp[n - 1];
            c.prev_origin = a.interp_origin[n - 1];
            c.prev_extent = a.interp_extent[n - 1];
            c.hole = a.interp[n];
            c.hole_origin = a.interp_origin[n];
            c.hole_extent = a.interp_extent[n];
            c.out = carry + (size_t)(n - 1) * nc3;
            c.N = N;
            cudaError_t e = run_carry<T>(c, s);
            if (e != cudaSuccess) return e;
            a.interp[n] = c.out;
            a.interp_origin[n] = N / 4 - 1;
            a.interp_extent[n] = (int)nc;
        }
    }
    return run_assemble<T>(a, s);
}
template cudaError_t run_assemble_interp<float>(AssembleArgs<float>, int, float*, cudaStream_t);
template cudaError_t run_assemble_interp<double>(AssembleArgs<double>, int, double*, cudaStream_t);
template cudaError_t run_assemble_interp<df>(AssembleArgs<df>, int, df*, cudaStream_t);

}  // namespace nm
