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
//   outer boundary of the coarsest level: second-order one-sided differences.
// All in double.  Output [level][component x, y, z][z][y][x].
#include "../../include/nm.h"
#include "internal.h"

namespace nm {

struct AccelArgs {
    const double* phi;
    double* g;
    int levels, N, lgN;
    double inv2dx0;     // 1 / (2 dx0)
};

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

__global__ void k_accel(const __grid_constant__ AccelArgs a) {
    const int N = a.N, lgN = a.lgN, L = a.levels;
    const size_t N3 = (size_t)1 << (3 * lgN);
    const size_t total = N3 * L;
    const int q = N / 4, h = N / 2;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int n = (int)(idx >> (3 * lgN));
        const size_t cell = idx & (N3 - 1);
        const int x = (int)(cell & (N - 1)), y = (int)((cell >> lgN) & (N - 1)), z = (int)(cell >> (2 * lgN));
        const double* p = a.phi + (size_t)n * N3;
        const double inv2dx = a.inv2dx0 * (double)(1 << n);
        const bool has_fine = n < L - 1;
        const bool own_cov = has_fine && (unsigned)(x - q) < (unsigned)h && (unsigned)(y - q) < (unsigned)h &&
                             (unsigned)(z - q) < (unsigned)h;
        const int c3[3] = {x, y, z};
        double gv[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            double v[2];
            bool ok[2];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                int nb[3] = {c3[0], c3[1], c3[2]};
                nb[ax] += side == 0 ? 1 : -1;
                const int j = nb[ax];
                ok[side] = true;
                if (j >= 0 && j < N) {
                    const bool nb_cov = has_fine && (unsigned)(nb[0] - q) < (unsigned)h &&
                                        (unsigned)(nb[1] - q) < (unsigned)h && (unsigned)(nb[2] - q) < (unsigned)h;
                    if (nb_cov && !own_cov) {
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
                    v[side] = 0.75 * pc[cidx(lgN, cc[2], cc[1], cc[0])] +
                              0.25 * pc[cidx(lgN, cc[2] + ss[2], cc[1] + ss[1], cc[0] + ss[0])];
                } else {
                    ok[side] = false;
                }
            }
            double d;
            if (ok[0] && ok[1]) {
                d = (v[0] - v[1]) * inv2dx;
            } else {
                // outer boundary of the coarsest level: one-sided, second order
                const int sg = ok[0] ? 1 : -1;
                int n1[3] = {c3[0], c3[1], c3[2]}, n2[3] = {c3[0], c3[1], c3[2]};
                n1[ax] += sg;
                n2[ax] += 2 * sg;
                d = (double)sg * (-3.0 * p[cidx(lgN, c3[2], c3[1], c3[0])] + 4.0 * p[cidx(lgN, n1[2], n1[1], n1[0])] -
                                  p[cidx(lgN, n2[2], n2[1], n2[0])]) * inv2dx;
            }
            gv[ax] = -d;
        }
        double* out = a.g + (size_t)n * 3 * N3 + cell;
        out[0] = gv[0];
        out[N3] = gv[1];
        out[2 * N3] = gv[2];
    }
}

cudaError_t run_accel(const double* phi, double* g, int levels, int N, double dx0, cudaStream_t s) {
    int lg = 0;
    while ((1 << lg) < N) ++lg;
    AccelArgs a{phi, g, levels, N, lg, 1.0 / (2.0 * dx0)};
    const size_t total = (size_t)N * N * N * levels;
    size_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    ProfScope ps("accel_f64", levels, s);
    k_accel<<<(int)blocks, 256, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nm
