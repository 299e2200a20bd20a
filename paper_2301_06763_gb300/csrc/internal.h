// internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "conv.cuh"
#include "per_device.h"
#include "tma.cuh"

namespace nm {

// The calling thread's current device, or -1.
inline int current_device() {
    int d = -1;
    return cudaGetDevice(&d) == cudaSuccess ? d : -1;
}
// Per-device set-up of one kernel: the error of setting its attributes, and
// its resident CTAs per SM where the launcher needs them.
struct KernelPrep {
    cudaError_t err = cudaSuccess;
    int occ = 0;
};

// Counts every kernel launched by the library (reported by nm_kernel_launches).
void count_launches(int n);

// Event bracket around one launch while profiling is on (nm_profile_enable).
struct ProfScope {
    int idx = -1;
    cudaStream_t s = nullptr;
    ProfScope(const char* name, int units, cudaStream_t stream);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;
};

// Five-pass convolution of `npairs` packed pairs of FFT size P (see conv.cuh),
// one entry point per (precision, values per thread).  `flags`: CONV_WIDE
// selects the wider column tile, CONV_TMA the persistent TMA-fed z-seam,
// CONV_FUSED the cluster-fused x/y passes (level grids only; 16 values per
// thread; sizes whose slab does not fit a cluster keep the five passes),
// CONV_PAIRED the FP32 z-seam with two columns per thread (level grids, 16
// values per thread, P >= 64; other cases keep the classic z-seam), with
// CONV_ZPERSIST its persistent prefetching form (P = 256, narrow tiles), and
// CONV_SSPEC the one-column FP32 z-seam with its spectrum rows staged in
// shared memory (level grids, 16 values per thread, P >= 64; both read the
// float spectrum unfolded along kx, which must exist).  `dbl` selects the
// doubled-fine-grid geometry (16 values, narrow tiles only).  Returns the
// first launch error.
enum { CONV_WIDE = 1, CONV_TMA = 2, CONV_FUSED = 4, CONV_PAIRED = 8, CONV_ZPERSIST = 16, CONV_SSPEC = 32 };
// k_zseam2 over np pairs of FFT size P with TX columns per CTA (16 or 32).
cudaError_t run_zseam_paired_f32(const ConvArgs<float>& a, int np, int P, int TX, cudaStream_t s);
// k_zseam_s over np pairs of FFT size P with TX columns per CTA (16 or 32).
cudaError_t run_zseam_staged_f32(const ConvArgs<float>& a, int np, int P, int TX, cudaStream_t s);
// k_zseam2p, the paired z-seam as a persistent pipeline that prefetches the
// next tile's columns (P = 256, 16 columns per tile).
cudaError_t run_zseam_persist_f32(const ConvArgs<float>& a, int np, int P, cudaStream_t s);
// k_xfwd_pipe2 (two rows per thread) over np pairs of FFT size P (256 or
// 512); needs pairs of a level's full and hole fields (or a full field alone)
// on a 16-byte aligned FP32 density.
cudaError_t run_xfwd_paired_f32(const ConvArgs<float>& a, int np, int P, cudaStream_t s);
cudaError_t run_conv_f32_e16(const PairDesc<float>* pairs, int npairs, int P, bool dbl, int flags,
                             const float* spec, const cpx<float>* tw, cudaStream_t s);
cudaError_t run_conv_f32_e8(const PairDesc<float>* pairs, int npairs, int P, bool dbl, int flags,
                            const float* spec, const cpx<float>* tw, cudaStream_t s);
cudaError_t run_conv_f64_e16(const PairDesc<double>* pairs, int npairs, int P, bool dbl, int flags,
                             const double* spec, const cpx<double>* tw, cudaStream_t s);
cudaError_t run_conv_f64_e8(const PairDesc<double>* pairs, int npairs, int P, bool dbl, int flags,
                            const double* spec, const cpx<double>* tw, cudaStream_t s);
// Double-float passes (NM_FP64X), level grids, 16 values per thread.
cudaError_t run_conv_dfx_e16(const PairDesc<df>* pairs, int npairs, int P, bool dbl, int flags, const df* spec,
                             const cpx<df>* tw, cudaStream_t s);
// Quadrupled-grid geometry (Appendix B), P = 8N, 16 values per thread.
cudaError_t run_conv_qdp_f32(const PairDesc<float>* pairs, int npairs, int P, const float* spec,
                             const cpx<float>* tw, cudaStream_t s);
cudaError_t run_conv_qdp_f64(const PairDesc<double>* pairs, int npairs, int P, const double* spec,
                             const cpx<double>* tw, cudaStream_t s);

// TMA descriptor of one work buffer ([P/2][P][P] complex, seen as
// [P/2][P][2P] reals) with a box of TX columns x 1 row x P/2 slabs.
cudaError_t encode_work_map(CUtensorMap* map, void* work, int P, bool f64, int TX);
// The library's device status word on the current device (0 = fine).
int* device_status_word();
// Test hook: while set, TMA-fed kernels issue no loads so their bounded
// waits run out (see nm_debug_fault_timeout).
bool fault_timeout_on();
int sm_count();

// Unit-cell kernel spectrum octant (N+1)^3 in double (Eqs. 10, 13, Fig. 4);
// `scratch` holds 2 (N+1)^3 doubles, `ctab` the P = 2N cosines cos(2 pi t/P).
cudaError_t run_green_octant(double* out, double* scratch, const double* ctab, int N,
                             double self_term, cudaStream_t s);
cudaError_t run_to_float(const double* in, float* out, size_t n, cudaStream_t s);
// The octant ((N+1)^3 doubles) as float rows over all 2N kx: (N+1)^2 2N floats.
cudaError_t run_unfold_x(const double* in, float* out, int N, cudaStream_t s);
// The unfolded float spectrum that belongs to the float octant `spec` (built
// by the plan before its first paired z-seam), or null.
const float* unfolded_spectrum(const float* spec);
cudaError_t run_to_df(const double* in, df* out, size_t n, cudaStream_t s);
// The octant as float with fz fastest ([fx][fy][fz], (N+1)^3 floats), read by
// the fused y/z/y pass; and the copy belonging to the float octant `spec`
// (built by the plan before its first three-pass solve), or null.
cudaError_t run_zfast(const double* in, float* out, int N, cudaStream_t s);
const float* zfast_spectrum(const float* spec);
// Three-pass convolution (yzy.cuh) of npairs level-grid pairs, FP32, P = 2N in
// 64 .. 512; `split` selects the CTAs per kx plane (0: the default for P, 1:
// the alternative where one is built).  Pairs must be a level's full and hole
// fields (or a full field alone) on a 16-byte aligned density.
cudaError_t run_conv_f32_yzy(const PairDesc<float>* pairs, int npairs, int P, int split, const float* spec,
                             const cpx<float>* tw, cudaStream_t s);
// Whether run_conv_f32_yzy takes these pairs.
bool yzy_pairs_ok(const PairDesc<float>* pairs, int npairs);

// Restriction of level m+1 onto level m's covered cells (mean of 2^3 children).
template <typename TIN>
cudaError_t run_restrict(const TIN* rho_child, const TIN* restr_child, TIN* restr_out, int N,
                         cudaStream_t s);

// Final assembly (Eq. 14 / Eqs. 15, B.1-B.2) into phi (double).
template <typename T> struct AssembleArgs {
    const T* base[16];     // per level: Phi^n (original) or Phi^n_hole (dipole), N^3
    const T* dbl[16];      // per level: (2N)^3 doubled-grid potential to reduce, or null
    const T* red[16];      // per level: an N^3 term added as it is (the reduced quadrupled
                           // grid or the direct sum of the three-level scheme), or null
    const T* interp[16];   // per level k: source of the hole potential for finer levels
    int interp_origin[16]; // level-k index of interp[k]'s first cell on each axis
    int interp_extent[16]; // its extent per axis
    double* phi;
    int levels, N;
    int diag;              // 1: Eqs. 3-6 two-point rule from interp[n-1] only
};
// One step of the carried Eqs. 3-6 interpolation: on the (N/2+2)^3 cells of
// level n from N/4-1 on, out = D(prev) + hole, prev and hole given with their
// origin and extent on their own level.
template <typename T> struct CarryArgs {
    const T* prev;
    int prev_origin, prev_extent;
    const T* hole;
    int hole_origin, hole_extent;
    T* out;
    int N;
};
template <typename T>
cudaError_t run_carry(const CarryArgs<T>& a, cudaStream_t s);
// The restriction and carried-interpolation chains of up to kTreeMeshes
// meshes per launch (chains.cu).  A mesh's restriction job: rho holds its L
// levels of N^3 densities (level m at rho + m N^3), restr receives restr_m,
// m = 0 .. L-2, at restr + m N^3/8.  Meshes with N < 16 or unaligned buffers,
// and the levels beyond a tile's depth, take the per-level kernel.
constexpr int kTreeMeshes = 32;
template <typename TIN> struct RestrictMesh {
    const TIN* rho;
    TIN* restr;
    int N, L;
};
template <typename TIN>
cudaError_t run_restrict_tree(const RestrictMesh<TIN>* meshes, int n, cudaStream_t s);
// A mesh's carried interpolation: level k's hole potential at hole + k
// hole_stride, stored from level index hole_origin on with hole_extent cells
// per axis (k = 0 .. L-2); out + (n-1) (N/2+2)^3 receives S_n, n = 1 .. L-2.
template <typename T> struct CarryMesh {
    const T* hole;
    size_t hole_stride;
    int hole_origin, hole_extent;
    T* out;
    int N, L;
};
template <typename T>
cudaError_t run_carry_tree(const CarryMesh<T>* meshes, int n, cudaStream_t s);
// run_assemble after the carry chain when interp is NM_INTERP_DIAGONAL
// (carry: (L-2) (N/2+2)^3 values of scratch).
template <typename T>
cudaError_t run_assemble_interp(AssembleArgs<T> a, int interp, T* carry, cudaStream_t s);
template <typename T>
cudaError_t run_assemble(const AssembleArgs<T>& a, cudaStream_t s);
// The assemblies of n meshes, up to kAsmMeshes per launch (meshes with
// N < 16 take run_assemble).
constexpr int kAsmMeshes = 16;
template <typename T>
cudaError_t run_assemble_batch(const AssembleArgs<T>* meshes, int n, cudaStream_t s);

// Three-level dipole scheme (dipole3.cu): out (N^3) = mean of each 4^3 block
// of in ((4N)^3); and Eq. B.6, out (N^3, level n centres) = scale * sum over
// the N^3 cells j of level n+2 of rho_j / |u_i - j| in level-(n+2) cell units
// (u_i = 4 i + 3/2 - 3N/2 per axis), rho_j from `rho` with the covered cells
// taken from `restr` ((N/2)^3, or null), scale = -G dx_{n+2}^2; float sums are
// carried in double across source tiles.
template <typename T>
cudaError_t run_reduce4(const T* in, T* out, int N, cudaStream_t s);
template <typename T>
cudaError_t run_direct2(const T* rho, const T* restr, T* out, int N, double scale, cudaStream_t s);

// Persistent batch (persist.cu): every step of the FP32 original-method
// solves of a batch as work items of one launch.  One mesh as the layout
// needs it; `pairs` are its level pairs (work pointers unset), `asm_args` its
// assembly arguments with the hole crops as interpolation sources, `carry`
// the carried-interpolation scratch (diagonal reading) or null (trilinear).
struct PersistMesh {
    int P, L, group;
    const float* rho;
    float* restr;
    double* phi;
    void* work;
    const float* spec;
    const cpx<float>* tw;
    std::vector<PairDesc<float>> pairs;
    float* carry;
    AssembleArgs<float> asm_args;
};
struct PersistBatch;
PersistBatch* persist_new();
void persist_free(PersistBatch* b);
int persist_items(const PersistBatch* b);
// Lay out the work items (host only; false if a mesh does not fit the path).
bool persist_layout(const std::vector<PersistMesh>& meshes, PersistBatch& b);
// Allocate and fill the device tables (synchronous: not while capturing).
cudaError_t persist_upload(PersistBatch& b);
// Reset the counters and launch on `s` (capturable).
cudaError_t persist_launch(PersistBatch& b, cudaStream_t s);

// g = -grad Phi of a nested potential (accel.cu).
cudaError_t run_accel(const double* phi, double* g, int levels, int N, double dx0, cudaStream_t s);
// Same with method C on the coarse side when vbuf (2 (L-1) 6 (N/2+2)^2 doubles)
// is given: `iters` sweeps of the face condition, then the stencil.
cudaError_t run_accel_ex(const double* phi, double* g, int levels, int N, double dx0, double* vbuf, int iters,
                         cudaStream_t s);
inline size_t accel_vbuf_doubles(int levels, int N) {
    return levels > 1 ? (size_t)2 * (levels - 1) * 6 * (size_t)(N / 2 + 2) * (N / 2 + 2) : 0;
}

}  // namespace nm
