// Pipelined-pair FP32-arithmetic stencil (dslash32pp.cuh) with 3 blocks per SM requested
// from the register allocator: variants 17 and 19 of dslash32.cu (lexicographic and tiled
// site order), compiled apart from the others to keep each translation unit small.
#include "dslash32pp.cuh"

namespace eig {

cudaError_t d32_launch_pp3(int prec, int gf, bool dag, int epi, const K32 &a, int cap, cudaStream_t s) {
    if (prec == 32 && gf == GF_F32_12) return d32pp_fmt<3, false, float, GF_F32_12>(dag, epi, a, cap, s);
    if (prec == 32 && gf == GF_F32_18) return d32pp_fmt<3, false, float, GF_F32_18>(dag, epi, a, cap, s);
    if (prec == 16 && gf == GF_F32_12) return d32pp_fmt<3, false, __half, GF_F32_12>(dag, epi, a, cap, s);
    return cudaErrorInvalidValue;
}

}  // namespace eig
