// Direct-load FP32 stencil variants with two RHS per thread (variants 4, 5 and 6 of
// dslash32.cu), compiled apart from the others to keep each translation unit small.
#include "dslash32.cuh"

namespace eig {

cudaError_t d32_launch_direct_rb2(int variant, int prec, int gf, bool dag, int epi, const K32 &a, int cap,
                                  cudaStream_t s) {
    if (variant == 4) return d32_direct<2, 3, 1>(prec, gf, dag, epi, a, cap, s);
    if (variant == 5) return d32_direct<2, 4, 1>(prec, gf, dag, epi, a, cap, s);
    return d32_direct<2, 3, 2>(prec, gf, dag, epi, a, cap, s);
}

}  // namespace eig
