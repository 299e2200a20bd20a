// conv_f32_qdp.cu -- the convolution passes on the quadrupled grid of the
// three-level dipole scheme (Appendix B) in float.
#include "conv_inst.cuh"

namespace nm {
cudaError_t run_conv_qdp_f32(const PairDesc<float>* pairs, int npairs, int P, const float* spec, const cpx<float>* tw,
                            cudaStream_t s) {
    return run_conv_qdp_variant<float>(pairs, npairs, P, spec, tw, s);
}
}  // namespace nm
