// conv_f32_e8.cu -- the convolution passes in float, 8 values per thread.
#include "conv_inst.cuh"

namespace nm {
cudaError_t run_conv_f32_e8(const PairDesc<float>* pairs, int npairs, int P, bool dbl, int flags,
                          const float* spec, const cpx<float>* tw, cudaStream_t s) {
    return run_conv_variant<float, 8>(pairs, npairs, P, dbl, flags, spec, tw, s);
}
}  // namespace nm
