// conv_dfx_e16.cu -- the convolution passes in double-float (NM_FP64X), 16
// values per thread, level grids.
#include "conv_inst.cuh"

namespace nm {
cudaError_t run_conv_dfx_e16(const PairDesc<df>* pairs, int npairs, int P, bool dbl, int flags, const df* spec,
                             const cpx<df>* tw, cudaStream_t s) {
    return run_conv_variant<df, 16>(pairs, npairs, P, dbl, flags, spec, tw, s);
}
}  // namespace nm
