// accel.cu -- gravitational acceleration g = -grad Phi of a nested potential.
//
// Central six-point stencil (Eq. 8) on every level, with the interface rules
// of Sect. 2 and Appendix A that the paper uses (its "first, simple method"):
//   fine side (method A): a missing neighbour beyond a level-n boundary
//     (n >= 1) is the ghost value of Eqs. 3-6 interpolated from level n-1:
//     the ghost centre lies a quarter coarse cell from the nearest coarse
//     centre c on each axis, Phi_B = 3/4 Phi(c) + 1/4 Phi(c + s), s the
//     diagonal step towards the ghost centre;
//   coarse side (method B): for an uncovered cell of level n, a neighbour
//     covered by level n+1 is replaced by the mean of its 2^3 children there;
//   or (method C) by a virtual value V that makes the coarse gradient across
//     the shared face equal to the mean of the fine gradients across it, the
//     fine ghosts (Eqs. 3-6) reading V in turn; iterated to a fixed count, and
//     the fine side's ghosts then read the converged V as well;
//   outer boundary of the coarsest level: second-order one-sided differences.
// All in double.  Output [level][component x, y, z][z][y][x].
#include "../../include/nm.h"
#include "internal.h"

#include <cmath>

namespace nm {

cudaError_t launch_accel(const double* phi, double* g, int levels, int N, int lg, double dx0, const double* vface,
                         cudaStream_t s);

struct AccelArgs {
    const double* phi;
    double* g;
    int levels, N, lgN;
    double inv2dx[NM_MAX_LEVELS];   // 1 / (2 dx_n) per level
    const double* vface;            // method C: converged face arrays, or null (method B)
};

// Method C face arrays.  Interface n (levels n and n+1) has 6 faces,
// f = 2 * axis + (sigma < 0), axis 0/1/2 = x/y/z, sigma = +1 for the face
// between coarse index N/4 - 1 and N/4, -1 for 3N/4 - 1 | 3N/4.  Each face is
// an (h+2)^2 array over its two tangential coordinates (u, v) = the other two
// axes in x, y, z order, index (v - N/4 + 1)(h+2) + (u - N/4 + 1), h = N/2:
// the interior holds V at the covered cells next to the face, the border the
// coarse level's own values just outside the covered block (what Eqs. 3-6
// read there).
__host__ __device__ __forceinline__ size_t vface_stride(int N) { return (size_t)(N / 2 + 2) * (N / 2 + 2); }
__device__ __forceinline__ const double* vface_at(const double* base, int N, int n, int axis, int sigma) {
    return base + ((size_t)n * 6 + 2 * axis + (sigma < 0 ? 1 : 0)) * vface_stride(N);
}
__device__ __forceinline__ int vface_index(int N, int axis, const int c[3]) {
    const int u = axis == 0 ? c[1] : c[0];
    const int v = axis == 2 ? c[1] : c[2];
    return (v - N / 4 + 1) * (N / 2 + 2) + (u - N / 4 + 1);
}

__device__ __forceinline__ size_t cidx(int lgN, int z, int y, int x) {
    return ((size_t)z << (2 * lgN)) + ((size_t)y << lgN) + (size_t)x;
}

// Eqs. 3-6: level-(n-1) coordinate of level-n index i (i may be -1 or N):
// u = (N/2 + i)/2 - 1/4 = c + s/4.
__device__ __forceinline__ void ghost_axis(int N, int i, int& c, int& s) {
    const int t = N / 2 + i;
    c = t >> 1;                        // floor (t >= N/2 - 1 >= 1)
    s = (i & 1) ? 1 : -1;
}

// Every rule above for component `ax` of g at level-n cell c3 = (x, y, z).
__device__ __noinline__ double accel_component(const AccelArgs& a, int n, const int c3[3], int ax) {
    const int N = a.N, lgN = a.lgN, L = a.levels;
    const size_t N3 = (size_t)1 << (3 * lgN);
    const int q = N / 4, h = N / 2;
    const double* p = a.phi + (size_t)n * N3;
    const bool has_fine = n < L - 1;
    const bool own_cov = has_fine && (unsigned)(c3[0] - q) < (unsigned)h && (unsigned)(c3[1] - q) < (unsigned)h &&
                         (unsigned)(c3[2] - q) < (unsigned)h;
    double v[2];
    bool ok[2];
    for (int side = 0; side < 2; ++side) {
        int nb[3] = {c3[0], c3[1], c3[2]};
        nb[ax] += side == 0 ? 1 : -1;
        const int j = nb[ax];
        ok[side] = true;
        if (j >= 0 && j < N) {
            const bool nb_cov = has_fine && (unsigned)(nb[0] - q) < (unsigned)h &&
                                (unsigned)(nb[1] - q) < (unsigned)h && (unsigned)(nb[2] - q) < (unsigned)h;
            if (nb_cov && !own_cov && a.vface) {
                // method C: the face's virtual value
                v[side] = vface_at(a.vface, N, n, ax, side == 0 ? 1 : -1)[vface_index(N, ax, c3)];
            } else if (nb_cov && !own_cov) {
                // method B: mean of the covered neighbour's children
                const double* f = a.phi + (size_t)(n + 1) * N3;
                const int fx = 2 * (nb[0] - q), fy = 2 * (nb[1] - q), fz = 2 * (nb[2] - q);
                double s = 0.0;
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        s += f[cidx(lgN, fz + dz, fy + dy, fx)] + f[cidx(lgN, fz + dz, fy + dy, fx + 1)];
                v[side] = 0.125 * s;
            } else {
                v[side] = p[cidx(lgN, nb[2], nb[1], nb[0])];
            }
        } else if (n > 0) {
            // method A: ghost value from the coarser level
            int cc[3], ss[3];
            for (int k = 0; k < 3; ++k) ghost_axis(N, nb[k], cc[k], ss[k]);
            const double* pc = a.phi + (size_t)(n - 1) * N3;
            double diag;
            if (a.vface) {
                // method C: the diagonal partner through the face's array
                const int d3[3] = {cc[0] + ss[0], cc[1] + ss[1], cc[2] + ss[2]};
                diag = vface_at(a.vface, N, n - 1, ax, side == 0 ? -1 : 1)[vface_index(N, ax, d3)];
            } else {
                diag = pc[cidx(lgN, cc[2] + ss[2], cc[1] + ss[1], cc[0] + ss[0])];
            }
            v[side] = 0.75 * pc[cidx(lgN, cc[2], cc[1], cc[0])] + 0.25 * diag;
        } else {
            ok[side] = false;
        }
    }
    if (ok[0] && ok[1]) return (v[1] - v[0]) * a.inv2dx[n];
    // outer boundary of the coarsest level: one-sided, second order
    const int sg = ok[0] ? 1 : -1;
    int n1[3] = {c3[0], c3[1], c3[2]}, n2[3] = {c3[0], c3[1], c3[2]};
    n1[ax] += sg;
    n2[ax] += 2 * sg;
    const double d = -3.0 * p[cidx(lgN, c3[2], c3[1], c3[0])] + 4.0 * p[cidx(lgN, n1[2], n1[1], n1[0])] -
                     p[cidx(lgN, n2[2], n2[1], n2[0])];
    return (sg > 0 ? -d : d) * a.inv2dx[n];
}

// Bulk pass, one thread per 4 consecutive cells along x (N >= 8): the 2 + 8
// 16-byte loads of the centre row and of the y and z neighbour rows and the 2
// halo values are all in flight together, and every cell takes the plain
// central differences (3 subtractions and 3 multiplications in double, the
// FP64 pipe's minimum for this stencil) with no branch; neighbours beyond the
// level are clamped to the cell itself.  The cells where that is wrong (the
// six boundary faces of each level and the cells next to the covered block)
// are rewritten afterwards by k_accel_fix.
__global__ void __launch_bounds__(256) k_accel_bulk(const __grid_constant__ AccelArgs a) {
    const int N = a.N, lgN = a.lgN;
    const unsigned N3 = 1u << (3 * lgN);
    const unsigned quads = (N3 >> 2) * (unsigned)a.levels;
    const unsigned qi = blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= quads) return;
    const unsigned idx = qi << 2;
    const int n = (int)(idx >> (3 * lgN));
    const unsigned cell = idx & (N3 - 1);
    const int x0 = (int)(cell & (N - 1)), y = (int)((cell >> lgN) & (N - 1)), z = (int)(cell >> (2 * lgN));
    const double* p = a.phi + idx;
    const int sy = N, sz = N << lgN;
    const int dym = y > 0 ? -sy : 0, dyp = y < N - 1 ? sy : 0;
    const int dzm = z > 0 ? -sz : 0, dzp = z < N - 1 ? sz : 0;
    const double2 c0 = reinterpret_cast<const double2*>(p)[0], c1 = reinterpret_cast<const double2*>(p)[1];
    const double xm = p[x0 > 0 ? -1 : 0], xp = p[x0 + 4 < N ? 4 : 3];
    const double2 ym0 = reinterpret_cast<const double2*>(p + dym)[0], ym1 = reinterpret_cast<const double2*>(p + dym)[1];
    const double2 yp0 = reinterpret_cast<const double2*>(p + dyp)[0], yp1 = reinterpret_cast<const double2*>(p + dyp)[1];
    const double2 zm0 = reinterpret_cast<const double2*>(p + dzm)[0], zm1 = reinterpret_cast<const double2*>(p + dzm)[1];
    const double2 zp0 = reinterpret_cast<const double2*>(p + dzp)[0], zp1 = reinterpret_cast<const double2*>(p + dzp)[1];
    const double s = a.inv2dx[n];
    double* out = a.g + (size_t)n * 3 * N3 + cell;
    double2* gx = reinterpret_cast<double2*>(out);
    double2* gy = reinterpret_cast<double2*>(out + N3);
    double2* gz = reinterpret_cast<double2*>(out + 2 * (size_t)N3);
    gx[0] = make_double2((xm - c0.y) * s, (c0.x - c1.x) * s);
    gx[1] = make_double2((c0.y - c1.y) * s, (c1.x - xp) * s);
    gy[0] = make_double2((ym0.x - yp0.x) * s, (ym0.y - yp0.y) * s);
    gy[1] = make_double2((ym1.x - yp1.x) * s, (ym1.y - yp1.y) * s);
    gz[0] = make_double2((zm0.x - zp0.x) * s, (zm0.y - zp0.y) * s);
    gz[1] = make_double2((zm1.x - zp1.x) * s, (zm1.y - zp1.y) * s);
}

// Fix-up pass after k_accel_bulk: one thread per cell of the six boundary
// faces of every level (L 6 N^2 items) and of the six layers of uncovered
// cells next to each covered block ((L-1) 6 (N/2)^2 items).  Only the
// component normal to the item's face can be wrong after the bulk pass (the
// clamped or covered neighbour lies along that axis), so each item rewrites
// that one component; an edge or corner cell is an item of each of its faces,
// one per wrong component.
__global__ void __launch_bounds__(256) k_accel_fix(const __grid_constant__ AccelArgs a) {
    const int N = a.N, lgN = a.lgN, L = a.levels, h = N / 2, q = N / 4;
    const unsigned N3 = 1u << (3 * lgN);
    const unsigned nb = (unsigned)L * 6u * (unsigned)N * N;
    const unsigned ni = (unsigned)(L - 1) * 6u * (unsigned)h * h;
    const unsigned it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= nb + ni) return;
    int n, axis, layer, u, v;
    if (it < nb) {
        const unsigned per = 6u * N * N;
        n = (int)(it / per);
        const unsigned r = it - (unsigned)n * per;
        const int f = (int)(r / ((unsigned)N * N));
        const unsigned t = r - (unsigned)f * N * N;
        axis = f >> 1;
        layer = (f & 1) ? N - 1 : 0;
        u = (int)(t % N);
        v = (int)(t / N);
    } else {
        const unsigned r0 = it - nb, per = 6u * h * h;
        n = (int)(r0 / per);
        const unsigned r = r0 - (unsigned)n * per;
        const int f = (int)(r / ((unsigned)h * h));
        const unsigned t = r - (unsigned)f * h * h;
        axis = f >> 1;
        layer = (f & 1) ? 3 * N / 4 : q - 1;
        u = (int)(t % h) + q;
        v = (int)(t / h) + q;
    }
    int c[3];
    c[axis] = layer;
    c[axis == 0 ? 1 : 0] = u;
    c[axis == 2 ? 1 : 2] = v;
    const unsigned cell = ((unsigned)c[2] << (2 * lgN)) + ((unsigned)c[1] << lgN) + (unsigned)c[0];
    a.g[(size_t)n * 3 * N3 + (size_t)axis * N3 + cell] = accel_component(a, n, c, axis);
}

// One thread per cell (N = 4).
__global__ void __launch_bounds__(256) k_accel1(const __grid_constant__ AccelArgs a) {
    const int N = a.N, lgN = a.lgN;
    const unsigned N3 = 1u << (3 * lgN);
    const unsigned total = N3 * (unsigned)a.levels;
    const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int n = (int)(idx >> (3 * lgN));
    const unsigned cell = idx & (N3 - 1);
    const int c3[3] = {(int)(cell & (N - 1)), (int)((cell >> lgN) & (N - 1)), (int)(cell >> (2 * lgN))};
    double* out = a.g + (size_t)n * 3 * N3 + cell;
    for (int ax = 0; ax < 3; ++ax) out[(size_t)ax * N3] = accel_component(a, n, c3, ax);
}

// Method C, one CTA per face of every interface.  With Phi_B = 3/4 Phi_C +
// 1/4 hat(D) (Eqs. 3-6; the four ghosts of a face cell C have as diagonal
// partners D the four cells C' + (+-1, +-1) in the face's tangential plane),
// the face condition V = Phi_C + 2 mean_f (Phi_f - Phi_B) reads
// V(C) = A(C) - 1/8 sum_D hat(D),  A(C) = -Phi_C / 2 + 2 mean_f Phi_f,
// swept `iters` times (Jacobi, two buffers) from V = Phi_n(C').
constexpr int kVirtThreads = 1024;
constexpr int kVirtPer = 16;          // face cells per thread, (N/2)^2 / 1024 at N = 256

__global__ void __launch_bounds__(kVirtThreads) k_virtual(const double* __restrict__ phi, double* w0, double* w1,
                                                          int N, int lgN, int iters) {
    const int n = blockIdx.x / 6, f = blockIdx.x % 6, axis = f >> 1, sigma = (f & 1) ? -1 : 1;
    const int q = N / 4, b = 3 * N / 4, h = N / 2, E = h + 2;
    const size_t N3 = (size_t)1 << (3 * lgN);
    const double* pc = phi + (size_t)n * N3;
    const double* pf = phi + (size_t)(n + 1) * N3;
    const int cl = sigma > 0 ? q - 1 : b, cov = cl + sigma, fl = sigma > 0 ? 0 : N - 1;
    const size_t off = (size_t)blockIdx.x * vface_stride(N);
    double* wa = w0 + off;
    double* wb = w1 + off;
    auto at = [&](const double* p, int ax_val, int u, int v) {
        int c[3];
        c[axis] = ax_val;
        c[axis == 0 ? 1 : 0] = u;
        c[axis == 2 ? 1 : 2] = v;
        return p[cidx(lgN, c[2], c[1], c[0])];
    };
    // border (constant) and initial interior of both buffers
    for (int i = threadIdx.x; i < E * E; i += blockDim.x) {
        const int u = i % E + q - 1, v = i / E + q - 1;
        const double val = at(pc, cov, u, v);
        wa[i] = val;
        wb[i] = val;
    }
    const int cells = h * h;
    const int per = (cells + kVirtThreads - 1) / kVirtThreads;
    double A[kVirtPer];
#pragma unroll
    for (int k = 0; k < kVirtPer; ++k) {
        A[k] = 0.0;
        const int t = threadIdx.x + k * kVirtThreads;
        if (k < per && t < cells) {
            const int u = t % h + q, v = t / h + q;
            const int fu = 2 * (u - q), fv = 2 * (v - q);
            const double sf = at(pf, fl, fu, fv) + at(pf, fl, fu + 1, fv) + at(pf, fl, fu, fv + 1) +
                              at(pf, fl, fu + 1, fv + 1);
            A[k] = -0.5 * at(pc, cl, u, v) + 0.5 * sf;
        }
    }
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
        const double* src = (it & 1) ? wb : wa;
        double* dst = (it & 1) ? wa : wb;
#pragma unroll
        for (int k = 0; k < kVirtPer; ++k) {
            const int t = threadIdx.x + k * kVirtThreads;
            if (k < per && t < cells) {
                const int i = (t / h + 1) * E + (t % h + 1);
                dst[i] = A[k] - 0.125 * (src[i - E - 1] + src[i - E + 1] + src[i + E - 1] + src[i + E + 1]);
            }
        }
        __syncthreads();
    }
}

cudaError_t run_accel(const double* phi, double* g, int levels, int N, double dx0, cudaStream_t s) {
    return run_accel_ex(phi, g, levels, N, dx0, nullptr, 0, s);
}

cudaError_t run_accel_ex(const double* phi, double* g, int levels, int N, double dx0, double* vbuf, int iters,
                         cudaStream_t s) {
    int lg = 0;
    while ((1 << lg) < N) ++lg;
    const double* vface = nullptr;
    if (vbuf && levels > 1) {
        double* w0 = vbuf;
        double* w1 = vbuf + (size_t)(levels - 1) * 6 * vface_stride(N);
        {
            ProfScope ps("virtual_f64", levels - 1, s);
            k_virtual<<<(levels - 1) * 6, kVirtThreads, 0, s>>>(phi, w0, w1, N, lg, iters);
            count_launches(1);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        vface = (iters & 1) ? w1 : w0;
    }
    return launch_accel(phi, g, levels, N, lg, dx0, vface, s);
}

cudaError_t launch_accel(const double* phi, double* g, int levels, int N, int lg, double dx0, const double* vface,
                         cudaStream_t s) {
    AccelArgs a{};
    a.vface = vface;
    a.phi = phi;
    a.g = g;
    a.levels = levels;
    a.N = N;
    a.lgN = lg;
    for (int n = 0; n < levels && n < NM_MAX_LEVELS; ++n) a.inv2dx[n] = std::ldexp(1.0 / (2.0 * dx0), n);
    const size_t total = (size_t)N * N * N * levels;
    if (N >= 8) {
        {
            ProfScope ps("accel_f64", levels, s);
            k_accel_bulk<<<(unsigned)((total / 4 + 255) / 256), 256, 0, s>>>(a);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const size_t items = (size_t)levels * 6 * N * N + (size_t)(levels - 1) * 6 * (N / 2) * (N / 2);
        ProfScope ps("accel_fix_f64", levels, s);
        k_accel_fix<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(a);
        count_launches(2);
    } else {
        ProfScope ps("accel_f64", levels, s);
        k_accel1<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(a);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace nm
