// conv_f64_qdp.cu -- the convolution passes on the quadrupled grid of the
// three-level dipole scheme (Appendix B) in double.
#include "conv_inst.cuh"

namespace nm {
cudaError_t run_conv_qdp_f64(const PairDesc<double>* pairs, int npairs, int P, const double* spec, const cpx<double>* tw,
                            cudaStream_t s) {
    return run_conv_qdp_variant<double>(pairs, npairs, P, spec, tw, s);
}
}  // namespace nm
