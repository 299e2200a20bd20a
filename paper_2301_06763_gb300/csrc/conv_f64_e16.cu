// conv_f64_e16.cu -- the convolution passes in double, 16 values per thread.
#include "conv_inst.cuh"

namespace nm {
cudaError_t run_conv_f64_e16(const PairDesc<double>* pairs, int npairs, int P, bool dbl, int flags,
                          const double* spec, const cpx<double>* tw, cudaStream_t s) {
    return run_conv_variant<double, 16>(pairs, npairs, P, dbl, flags, spec, tw, s);
}
}  // namespace nm
