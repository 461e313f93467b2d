// Double-float ("dd") Wilson stencil for the reliable updates of mixed-precision CG:
// r = b - A x with about 44 bits of precision, computed on the FP32 pipes.
//
// GB300's FP64 rate is a small fraction of its FP32 rate, so an FP64 stencil is
// ALU-bound at a few percent of HBM bandwidth.  A double-float number is an
// unevaluated sum hi + lo of two FP32 values; products use the exact FMA product
// (p = a*b, e = fma(a, b, -p)), sums the two-sum transform, and an accumulator is
// renormalised once per hop.  Complex numbers keep (re, im) in the two lanes of
// the packed FP32 instructions (fma.rn.f32x2), as in dslash32.cu.
//
// The operator is the Wilson matrix of dslash.cu.  Inputs are converted from FP64
// once per call (x), gauge links once per operator.  The final true residual of a
// solve is still computed in FP64 (dslash.cu); these kernels serve the residual
// replacements in between.
#include <cstring>

#include "kernels.cuh"
#include "prof.h"

namespace eig {

namespace {

using F2 = float2;

__device__ __forceinline__ F2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ F2 add2(F2 a, F2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ F2 sub2(F2 a, F2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ F2 mul2(F2 a, F2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ F2 neg2(F2 a) { return f2(-a.x, -a.y); }

// double-float complex: value = hi + lo, lanes (re, im)
struct DC {
    F2 hi, lo;
};

__device__ __forceinline__ DC dc(F2 hi, F2 lo) {
    DC r;
    r.hi = hi;
    r.lo = lo;
    return r;
}
// i * a, -i * a
__device__ __forceinline__ DC ix(DC a) { return dc(f2(-a.hi.y, a.hi.x), f2(-a.lo.y, a.lo.x)); }
__device__ __forceinline__ DC mix(DC a) { return dc(f2(a.hi.y, -a.hi.x), f2(a.lo.y, -a.lo.x)); }
__device__ __forceinline__ DC negd(DC a) { return dc(neg2(a.hi), neg2(a.lo)); }

// a + b (two-sum on hi, lo parts added, renormalised)
__device__ __forceinline__ DC addd(DC a, DC b) {
    const F2 s = add2(a.hi, b.hi);
    const F2 bb = sub2(s, a.hi);
    F2 e = add2(sub2(a.hi, sub2(s, bb)), sub2(b.hi, bb));
    e = add2(e, add2(a.lo, b.lo));
    const F2 h = add2(s, e);
    return dc(h, sub2(e, sub2(h, s)));
}
__device__ __forceinline__ DC subd(DC a, DC b) { return addd(a, negd(b)); }
// accumulate without renormalising: acc + b
__device__ __forceinline__ void acc_add(DC &acc, const DC &b) {
    const F2 s = add2(acc.hi, b.hi);
    const F2 bb = sub2(s, acc.hi);
    const F2 e = add2(sub2(acc.hi, sub2(s, bb)), sub2(b.hi, bb));
    acc.lo = add2(acc.lo, add2(e, b.lo));
    acc.hi = s;
}
__device__ __forceinline__ DC renorm(DC a) {
    const F2 h = add2(a.hi, a.lo);
    return dc(h, sub2(a.lo, sub2(h, a.hi)));
}
// acc += (xr broadcast) * b, xr a double-float real given as (hi, lo) scalars
__device__ __forceinline__ void acc_scale(DC &acc, float xh, float xl, const DC &b) {
    const F2 a = f2(xh, xh);
    const F2 p = mul2(a, b.hi);
    F2 e = fma2(a, b.hi, neg2(p));                 // exact error of hi * hi
    e = fma2(a, b.lo, e);                          // cross terms
    e = fma2(f2(xl, xl), b.hi, e);
    acc_add(acc, dc(p, e));
}

struct Sd {
    DC c[12];
};
struct Hd {
    DC c[6];
};
struct Ld {
    DC u[9];
};

// field layout: [12][V][k] float4 = (re_hi, im_hi, re_lo, im_lo)
__device__ __forceinline__ void load_sd(const float4 *__restrict__ p, unsigned P, unsigned o, Sd &v) {
#pragma unroll
    for (int e = 0; e < 12; e++) {
        const float4 d = p[e * P + o];
        v.c[e] = dc(f2(d.x, d.y), f2(d.z, d.w));
    }
}
__device__ __forceinline__ void load_link(const float4 *__restrict__ g, unsigned V, int mu, unsigned s, Ld &U) {
    const float4 *p = g + (unsigned)mu * 9u * V;
#pragma unroll
    for (int e = 0; e < 9; e++) {
        const float4 d = __ldg(p + e * V + s);
        U.u[e] = dc(f2(d.x, d.y), f2(d.z, d.w));
    }
}

template <int MU, int SG>
__device__ __forceinline__ void project(const Sd &p, Hd &h) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const DC a0 = p.c[c], a1 = p.c[3 + c], b0 = p.c[6 + c], b1 = p.c[9 + c];
        if (MU == 0) {
            h.c[c] = addd(a0, SG > 0 ? ix(b1) : mix(b1));
            h.c[3 + c] = addd(a1, SG > 0 ? ix(b0) : mix(b0));
        } else if (MU == 1) {
            h.c[c] = SG > 0 ? subd(a0, b1) : addd(a0, b1);
            h.c[3 + c] = SG > 0 ? addd(a1, b0) : subd(a1, b0);
        } else if (MU == 2) {
            h.c[c] = addd(a0, SG > 0 ? ix(b0) : mix(b0));
            h.c[3 + c] = addd(a1, SG > 0 ? mix(b1) : ix(b1));
        } else {
            h.c[c] = SG > 0 ? addd(a0, b0) : subd(a0, b0);
            h.c[3 + c] = SG > 0 ? addd(a1, b1) : subd(a1, b1);
        }
    }
}

template <int MU, int SG>
__device__ __forceinline__ void accumulate(Sd &acc, const Hd &h) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const DC h0 = h.c[c], h1 = h.c[3 + c];
        acc_add(acc.c[c], h0);
        acc_add(acc.c[3 + c], h1);
        if (MU == 0) {
            acc_add(acc.c[6 + c], SG > 0 ? mix(h1) : ix(h1));
            acc_add(acc.c[9 + c], SG > 0 ? mix(h0) : ix(h0));
        } else if (MU == 1) {
            acc_add(acc.c[6 + c], SG > 0 ? h1 : negd(h1));
            acc_add(acc.c[9 + c], SG > 0 ? negd(h0) : h0);
        } else if (MU == 2) {
            acc_add(acc.c[6 + c], SG > 0 ? mix(h0) : ix(h0));
            acc_add(acc.c[9 + c], SG > 0 ? ix(h1) : mix(h1));
        } else {
            acc_add(acc.c[6 + c], SG > 0 ? h0 : negd(h0));
            acc_add(acc.c[9 + c], SG > 0 ? h1 : negd(h1));
        }
    }
}

// o = U h or U^H h:  (x + i y) h = x h + y (i h)
template <bool DAGGER>
__device__ __forceinline__ void mul_link(const Ld &U, const Hd &h, Hd &o) {
    Hd ih;
#pragma unroll
    for (int e = 0; e < 6; e++) ih.c[e] = ix(h.c[e]);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        DC o0 = dc(f2(0.f, 0.f), f2(0.f, 0.f)), o1 = o0;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const DC u = DAGGER ? U.u[b * 3 + a] : U.u[a * 3 + b];
            const float yh = DAGGER ? -u.hi.y : u.hi.y, yl = DAGGER ? -u.lo.y : u.lo.y;
            acc_scale(o0, u.hi.x, u.lo.x, h.c[b]);
            acc_scale(o0, yh, yl, ih.c[b]);
            acc_scale(o1, u.hi.x, u.lo.x, h.c[3 + b]);
            acc_scale(o1, yh, yl, ih.c[3 + b]);
        }
        o.c[a] = renorm(o0);
        o.c[3 + a] = renorm(o1);
    }
}

struct KD {
    const float4 *in;
    float4 *out;      // dd output (EPI plain)
    const double2 *b; // FP64 [12][V][k] (resid)
    double2 *r;       // FP64 output (resid)
    const float4 *g;
    unsigned L0, L1, L2, L3, V, k, P;
    float dh, dl;     // 4 + m_q as double-float
    int resid, set_rho;
    CGScalars *st;
    double *h_beta, *h_rho;
    int iter;
    double *partials;
    unsigned *counter;
};

template <int MU, bool DAG>
__device__ __forceinline__ void hop(const KD &a, unsigned s, unsigned sf, unsigned sb, unsigned r, Sd &acc) {
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    Ld U;
    Sd nb;
    Hd h, uh;
    load_link(a.g, a.V, MU, s, U);
    load_sd(a.in, a.P, sf * a.k + r, nb);
    project<MU, SF>(nb, h);
    mul_link<false>(U, h, uh);
    accumulate<MU, SF>(acc, uh);
    load_link(a.g, a.V, MU, sb, U);
    load_sd(a.in, a.P, sb * a.k + r, nb);
    project<MU, SB>(nb, h);
    mul_link<true>(U, h, uh);
    accumulate<MU, SB>(acc, uh);
#pragma unroll
    for (int e = 0; e < 12; e++) acc.c[e] = renorm(acc.c[e]);
}

template <bool DAG>
__global__ void __launch_bounds__(128, 3) k_dslash_dd(const KD a) {  // 3 blocks (12 warps) per SM
    __shared__ double smem[(128 / 32) * MAX_RHS];
    const unsigned total = a.V * a.k;
    const unsigned s1 = a.L0, s2 = a.L0 * a.L1, s3 = s2 * a.L2;
    double nrm = 0.0;
    for (unsigned g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const unsigned s = g / a.k, r = g - s * a.k;
        const unsigned x = s % a.L0, y = (s / s1) % a.L1, z = (s / s2) % a.L2, t = s / s3;
        Sd acc;
#pragma unroll
        for (int e = 0; e < 12; e++) acc.c[e] = dc(f2(0.f, 0.f), f2(0.f, 0.f));
        hop<0, DAG>(a, s, x == a.L0 - 1 ? s - (a.L0 - 1) : s + 1, x == 0 ? s + (a.L0 - 1) : s - 1, r, acc);
        hop<1, DAG>(a, s, y == a.L1 - 1 ? s - (a.L1 - 1) * s1 : s + s1, y == 0 ? s + (a.L1 - 1) * s1 : s - s1, r, acc);
        hop<2, DAG>(a, s, z == a.L2 - 1 ? s - (a.L2 - 1) * s2 : s + s2, z == 0 ? s + (a.L2 - 1) * s2 : s - s2, r, acc);
        hop<3, DAG>(a, s, t == a.L3 - 1 ? s - (a.L3 - 1) * s3 : s + s3, t == 0 ? s + (a.L3 - 1) * s3 : s - s3, r, acc);
        const unsigned o = s * a.k + r;
        Sd c0;
        load_sd(a.in, a.P, o, c0);
        // out = diag * c0 - acc / 2   (halving is exact)
#pragma unroll
        for (int e = 0; e < 12; e++) {
            DC v = dc(mul2(acc.c[e].hi, f2(-0.5f, -0.5f)), mul2(acc.c[e].lo, f2(-0.5f, -0.5f)));
            acc_scale(v, a.dh, a.dl, c0.c[e]);
            v = renorm(v);
            if (!a.resid) {
                a.out[e * a.P + o] = make_float4(v.hi.x, v.hi.y, v.lo.x, v.lo.y);
            } else {  // r = b - out in FP64
                const double2 bb = a.b[e * a.P + o];
                const double re = bb.x - ((double)v.hi.x + (double)v.lo.x);
                const double im = bb.y - ((double)v.hi.y + (double)v.lo.y);
                a.r[e * a.P + o] = make_double2(re, im);
                nrm += re * re + im * im;
            }
        }
    }
    if (!a.resid) return;
    const double bs = block_reduce_rhs(nrm, (int)a.k, smem);
    const int k = (int)a.k;
    CGScalars *const sts = a.st;
    double *const h_beta = a.h_beta, *const h_rho = a.h_rho;
    const int iter = a.iter, set_rho = a.set_rho;
    grid_reduce_rhs(bs, k, a.partials, a.counter, smem, [=](int rr, double tot) {
        CGScalars &st = sts[rr];
        const long hi = (long)iter * k + rr;
        st.aux = tot;
        if (set_rho) {
            st.rho = tot;
            st.beta = tot / st.rho_prev;
            h_rho[hi] = tot;
            h_beta[hi + k] = st.beta;
        }
    });
}

// FP64 [12][V][k] double2 -> dd [12][V][k] float4, and the gauge [mu][9][V] likewise
__global__ void k_to_dd(const double2 *__restrict__ in, float4 *__restrict__ out, unsigned n) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double2 d = in[i];
        const float rh = __double2float_rn(d.x), ih = __double2float_rn(d.y);
        out[i] = make_float4(rh, ih, __double2float_rn(d.x - (double)rh), __double2float_rn(d.y - (double)ih));
    }
}

__global__ void k_from_dd(const float4 *__restrict__ in, double2 *__restrict__ out, unsigned n) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 d = in[i];
        out[i] = make_double2((double)d.x + (double)d.z, (double)d.y + (double)d.w);
    }
}

// kc FP32 fields of k = 1 (one per column, column c at cols + c * cstride float4s)
// -> double-float RHS-inner field of kc RHS (low parts zero)
__global__ void k_cols32_to_dd(const float4 *__restrict__ cols, long cstride, unsigned V, unsigned kc,
                               float4 *__restrict__ dd) {
    const unsigned n = V * 12u * kc;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned q = i % kc, rest = i / kc, s = rest % V, e = rest / V;
        const float4 f = cols[(long)q * cstride + (long)(e >> 1) * V + s];
        dd[i] = (e & 1) ? make_float4(f.z, f.w, 0.f, 0.f) : make_float4(f.x, f.y, 0.f, 0.f);
    }
}

// double-float RHS-inner field of kc RHS -> kc FP32 fields of k = 1, rounded
__global__ void k_dd_to_cols32(const float4 *__restrict__ dd, unsigned V, unsigned kc, float4 *__restrict__ cols,
                               long cstride) {
    const unsigned n = V * 6u * kc;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned q = i % kc, rest = i / kc, s = rest % V, c = rest / V;
        const float4 a = dd[((2 * c) * V + s) * kc + q], b = dd[((2 * c + 1) * V + s) * kc + q];
        cols[(long)q * cstride + (long)c * V + s] =
            make_float4(__fadd_rn(a.x, a.z), __fadd_rn(a.y, a.w), __fadd_rn(b.x, b.z), __fadd_rn(b.y, b.w));
    }
}

int grid_for(unsigned work) {
    long g = ((long)work + 127) / 128;
    const long cap = (long)device_sm_count() * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_to_dd(const void *fp64, void *dd, long n, cudaStream_t s) {
    ProfScope prof("to_dd", (double)n * 32.0, s);
    k_to_dd<<<grid_for((unsigned)n), 128, 0, s>>>(static_cast<const double2 *>(fp64), static_cast<float4 *>(dd),
                                                    (unsigned)n);
    return cudaGetLastError();
}

cudaError_t launch_from_dd(const void *dd, void *fp64, long n, cudaStream_t s) {
    ProfScope prof("from_dd", (double)n * 32.0, s);
    k_from_dd<<<grid_for((unsigned)n), 128, 0, s>>>(static_cast<const float4 *>(dd), static_cast<double2 *>(fp64),
                                                      (unsigned)n);
    return cudaGetLastError();
}

cudaError_t launch_cols32_to_dd(const void *cols, long cstride_f4, long V, int kc, void *dd, cudaStream_t s) {
    const unsigned n = (unsigned)(V * 12 * kc);
    ProfScope prof("cols_to_dd", (double)n * 24.0, s);
    k_cols32_to_dd<<<grid_for(n), 128, 0, s>>>(static_cast<const float4 *>(cols), cstride_f4, (unsigned)V,
                                                (unsigned)kc, static_cast<float4 *>(dd));
    return cudaGetLastError();
}

cudaError_t launch_dd_to_cols32(const void *dd, long V, int kc, void *cols, long cstride_f4, cudaStream_t s) {
    const unsigned n = (unsigned)(V * 6 * kc);
    ProfScope prof("dd_to_cols", (double)n * 48.0, s);
    k_dd_to_cols32<<<grid_for(n), 128, 0, s>>>(static_cast<const float4 *>(dd), (unsigned)V, (unsigned)kc,
                                                static_cast<float4 *>(cols), cstride_f4);
    return cudaGetLastError();
}

// out_dd = M in_dd (dagger: M^H)
cudaError_t launch_dslash_dd(const DslashCall &c, const void *gauge_dd, const void *in_dd, void *out_dd,
                             cudaStream_t s) {
    KD a;
    memset(&a, 0, sizeof(a));
    a.in = static_cast<const float4 *>(in_dd);
    a.out = static_cast<float4 *>(out_dd);
    a.g = static_cast<const float4 *>(gauge_dd);
    a.L0 = c.L[0];
    a.L1 = c.L[1];
    a.L2 = c.L[2];
    a.L3 = c.L[3];
    a.V = (unsigned)c.V;
    a.k = (unsigned)c.k;
    a.P = (unsigned)(c.V * c.k);
    a.dh = (float)c.diag;
    a.dl = (float)(c.diag - (double)a.dh);
    ProfScope prof("dslash_dd", (double)c.V * (4.0 * 144 + c.k * 2.0 * 192), s);
    const unsigned work = a.V * a.k;
    if (c.dagger) k_dslash_dd<true><<<grid_for(work), 128, 0, s>>>(a);
    else k_dslash_dd<false><<<grid_for(work), 128, 0, s>>>(a);
    return cudaGetLastError();
}

// r = b - M^H in_dd in FP64 output, aux = ||r||^2 (set_rho as launch_dslash_resid)
cudaError_t launch_dslash_dd_resid(const DslashCall &c, const void *gauge_dd, const void *in_dd, Field b, Field r,
                                   CGScalars *st, History h, int iter, bool set_rho, RedScratch red, cudaStream_t s) {
    KD a;
    memset(&a, 0, sizeof(a));
    a.in = static_cast<const float4 *>(in_dd);
    a.b = static_cast<const double2 *>(b.v.data);
    a.r = static_cast<double2 *>(r.v.data);
    a.g = static_cast<const float4 *>(gauge_dd);
    a.L0 = c.L[0];
    a.L1 = c.L[1];
    a.L2 = c.L[2];
    a.L3 = c.L[3];
    a.V = (unsigned)c.V;
    a.k = (unsigned)c.k;
    a.P = (unsigned)(c.V * c.k);
    a.dh = (float)c.diag;
    a.dl = (float)(c.diag - (double)a.dh);
    a.resid = 1;
    a.set_rho = set_rho;
    a.st = st;
    a.h_beta = h.beta;
    a.h_rho = h.rho;
    a.iter = iter;
    a.partials = red.partials;
    a.counter = red.counter;
    ProfScope prof("dslash_dd_resid", (double)c.V * (4.0 * 144 + c.k * 3.0 * 192), s);
    unsigned work = a.V * a.k;
    int grid = grid_for(work);
    if (grid > red.max_blocks) grid = red.max_blocks;
    if (c.dagger) k_dslash_dd<true><<<grid, 128, 0, s>>>(a);
    else k_dslash_dd<false><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace eig
