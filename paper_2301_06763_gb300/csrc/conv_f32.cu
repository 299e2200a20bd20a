// conv_f32.cu -- single-precision instantiation of the convolution passes.
#include "conv_inst.cuh"

namespace nm {
cudaError_t run_conv_f32(const PairDesc<float>* pairs, int npairs, int P, bool dbl,
                         const float* spec, const cpx<float>* tw, cudaStream_t s) {
    return run_conv_t<float>(pairs, npairs, P, dbl, spec, tw, s);
}
}  // namespace nm
