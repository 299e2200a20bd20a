// conv_f32_e16.cu -- the convolution passes in float, 16 values per thread.
#include "conv_inst.cuh"

namespace nm {
cudaError_t run_conv_f32_e16(const PairDesc<float>* pairs, int npairs, int P, bool dbl, int flags,
                          const float* spec, const cpx<float>* tw, cudaStream_t s) {
    return run_conv_variant<float, 16>(pairs, npairs, P, dbl, flags, spec, tw, s);
}
}  // namespace nm
