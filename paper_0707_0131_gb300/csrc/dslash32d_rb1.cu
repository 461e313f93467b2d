// Direct-load FP32 stencil variants with one RHS per thread (variants 2, 3 and 7 of
// dslash32.cu), compiled apart from the others to keep each translation unit small.
#include "dslash32.cuh"

namespace eig {

cudaError_t d32_launch_direct_rb1(int variant, int prec, int gf, bool dag, int epi, const K32 &a, int cap,
                                  cudaStream_t s) {
    if (variant == 2) return d32_direct<1, 4, 1>(prec, gf, dag, epi, a, cap, s);
    if (variant == 3) return d32_direct<1, 5, 1>(prec, gf, dag, epi, a, cap, s);
    return d32_direct<1, 5, 2>(prec, gf, dag, epi, a, cap, s);
}

}  // namespace eig
