// Host build of the stencil's fast division for the CPU tests.
#include "../../paper_0707_0131_gb300/csrc/fastdiv.h"

extern "C" void fd_make(unsigned d, unsigned *m, unsigned *sh) {
    const eig::FastDiv f = eig::fastdiv_make(d);
    *m = f.m;
    *sh = f.sh;
}

extern "C" unsigned fd_div(unsigned n, unsigned d) { return eig::fastdiv(n, eig::fastdiv_make(d)); }

// count of n in [lo, hi) where the fast quotient differs from n / d
extern "C" long fd_check_range(unsigned d, unsigned lo, unsigned hi) {
    const eig::FastDiv f = eig::fastdiv_make(d);
    long bad = 0;
    for (unsigned long long n = lo; n < hi; n++)
        if (eig::fastdiv((unsigned)n, f) != (unsigned)(n / d)) bad++;
    return bad;
}
