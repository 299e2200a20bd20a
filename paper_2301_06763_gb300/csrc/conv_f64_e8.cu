// conv_f64_e8.cu -- the convolution passes in double, 8 values per thread.
#include "conv_inst.cuh"

namespace nm {
cudaError_t run_conv_f64_e8(const PairDesc<double>* pairs, int npairs, int P, bool dbl, int flags,
                          const double* spec, const cpx<double>* tw, cudaStream_t s) {
    return run_conv_variant<double, 8>(pairs, npairs, P, dbl, flags, spec, tw, s);
}
}  // namespace nm
