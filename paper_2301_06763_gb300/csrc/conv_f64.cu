// conv_f64.cu -- double-precision instantiation of the convolution passes.
#include "conv_inst.cuh"

namespace nm {
cudaError_t run_conv_f64(const PairDesc<double>* pairs, int npairs, int P, bool dbl,
                         const double* spec, const cpx<double>* tw, cudaStream_t s) {
    return run_conv_t<double>(pairs, npairs, P, dbl, spec, tw, s);
}
}  // namespace nm
