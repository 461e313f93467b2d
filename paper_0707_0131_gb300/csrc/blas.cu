// Vector kernels of the CG hot path that are not fused into the stencil:
// layout conversion at the API boundary, precision conversion for reliable
// updates, norms, and the p update of Fig. 1 step 9 fused with the eigCG window
// append of Fig. 1 step 11.13 (V(:, i) = z / sqrt(rho), z = r for P = I).
// All of them are HBM-bound streaming kernels over the chunk-major field layout.
#include <string>
#include <cstring>

#include "kernels.cuh"
#include "prof.h"

namespace eig {

template <typename S>
struct Calc {
    using C = typename SpinorStore<S>::C;
};

static double spb(Prec p) { return p == P64 ? 192.0 : (p == P32 ? 96.0 : 52.0); }

static int stream_grid(long work, int block) {
    long need = (work + block - 1) / block;
    long cap = (long)device_sm_count() * 8;
    if (need > cap) need = cap;
    return (int)(need < 1 ? 1 : need);
}

// ---------------------------------------------------------------------------------------
// natural <-> internal
// ---------------------------------------------------------------------------------------
template <typename S>
__global__ void k_pack(const double2 *__restrict__ nat, FieldView f) {
    using C = typename SpinorStore<S>::C;
    const long total = f.V * f.k;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long s = g / f.k;
        const int r = (int)(g - s * f.k);
        const double2 *src = nat + ((long)r * f.V + s) * 12;
        Spinor<C> v;
#pragma unroll
        for (int e = 0; e < 12; e++) {
            double2 d = src[e];
            v.s[e / 3][e % 3] = cmk<C>((C)d.x, (C)d.y);
        }
        SpinorStore<S>::store(f, s, r, v);
    }
}

template <typename S>
__global__ void k_unpack(FieldView f, double2 *__restrict__ nat) {
    using C = typename SpinorStore<S>::C;
    const long total = f.V * f.k;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long s = g / f.k;
        const int r = (int)(g - s * f.k);
        Spinor<C> v;
        SpinorStore<S>::load(f, s, r, v);
        double2 *dst = nat + ((long)r * f.V + s) * 12;
#pragma unroll
        for (int e = 0; e < 12; e++) dst[e] = make_double2((double)v.s[e / 3][e % 3].re, (double)v.s[e / 3][e % 3].im);
    }
}

// full-lattice FP64 field <-> half-lattice FP64 field of the sites of one parity
// (site s of parity p(x) = (x + y + z + t) mod 2 at half index s / 2; Lx even)
__global__ void k_parity_move(FieldView full, FieldView half, int parity, int L0, int L1, int L2, int to_half) {
    const long total = half.V * half.k;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long h = g / half.k;
        const int r = (int)(g - h * half.k);
        const long lh = L0 / 2, rest = h / lh;
        const int y = (int)(rest % L1), z = (int)((rest / L1) % L2), t = (int)(rest / ((long)L1 * L2));
        const long s = 2 * (h % lh) + ((parity + y + z + t) & 1) + L0 * rest;
        Spinor<double> v;
        if (to_half) {
            SpinorStore<double>::load(full, s, r, v);
            SpinorStore<double>::store(half, h, r, v);
        } else {
            SpinorStore<double>::load(half, h, r, v);
            SpinorStore<double>::store(full, s, r, v);
        }
    }
}

cudaError_t launch_parity_move(Field full, Field half, int parity, const int L[4], bool to_half, cudaStream_t s) {
    if (full.prec != P64 || half.prec != P64 || full.v.k != half.v.k || half.v.V * 2 != full.v.V || (L[0] & 1))
        return cudaErrorInvalidValue;
    ProfScope prof("parity_move", (double)half.v.V * half.v.k * 2 * 192.0, s);
    const int B = 128;
    k_parity_move<<<stream_grid(half.v.V * half.v.k, B), B, 0, s>>>(full.v, half.v, parity, L[0], L[1], L[2],
                                                                    to_half ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_pack(const double *nat, Field f, cudaStream_t s) {
    ProfScope prof("pack", (double)f.v.V * f.v.k * (192.0 + spb(f.prec)), s);
    const int B = 128;
    const int G = stream_grid(f.v.V * f.v.k, B);
    const double2 *n = reinterpret_cast<const double2 *>(nat);
    switch (f.prec) {
        case P64: k_pack<double><<<G, B, 0, s>>>(n, f.v); break;
        case P32: k_pack<float><<<G, B, 0, s>>>(n, f.v); break;
        case P16: k_pack<__half><<<G, B, 0, s>>>(n, f.v); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack(Field f, double *nat, cudaStream_t s) {
    ProfScope prof("unpack", (double)f.v.V * f.v.k * (192.0 + spb(f.prec)), s);
    const int B = 128;
    const int G = stream_grid(f.v.V * f.v.k, B);
    double2 *n = reinterpret_cast<double2 *>(nat);
    switch (f.prec) {
        case P64: k_unpack<double><<<G, B, 0, s>>>(f.v, n); break;
        case P32: k_unpack<float><<<G, B, 0, s>>>(f.v, n); break;
        case P16: k_unpack<__half><<<G, B, 0, s>>>(f.v, n); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// gauge packing: natural [V][4][3][3] complex -> per-direction planes
// ---------------------------------------------------------------------------------------
__global__ void k_pack_gauge(const double2 *__restrict__ nat, void *dst, int gformat, long V) {
    const long total = V * 4;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long s = g / 4;
        const int mu = (int)(g - s * 4);
        const double2 *u = nat + (s * 4 + mu) * 9;
        if (gformat == GF_F64_18) {
            double2 *d = static_cast<double2 *>(dst) + (long)mu * 9 * V;
            for (int e = 0; e < 9; e++) d[(long)e * V + s] = u[e];
        } else if (gformat == GF_F32_18) {
            float2 *d = static_cast<float2 *>(dst) + (long)mu * 9 * V;
            for (int e = 0; e < 9; e++) d[(long)e * V + s] = make_float2((float)u[e].x, (float)u[e].y);
        } else if (gformat == GF_F32_12) {
            float4 *d = static_cast<float4 *>(dst) + (long)mu * 3 * V;
            for (int q = 0; q < 3; q++)
                d[(long)q * V + s] = make_float4((float)u[2 * q].x, (float)u[2 * q].y, (float)u[2 * q + 1].x,
                                                 (float)u[2 * q + 1].y);
        } else {  // GF_F16_12
            uint2 *d = static_cast<uint2 *>(dst) + (long)mu * 3 * V;
            for (int q = 0; q < 3; q++) {
                __half2 h0 = __floats2half2_rn((float)u[2 * q].x, (float)u[2 * q].y);
                __half2 h1 = __floats2half2_rn((float)u[2 * q + 1].x, (float)u[2 * q + 1].y);
                d[(long)q * V + s] = make_uint2(*reinterpret_cast<uint32_t *>(&h0), *reinterpret_cast<uint32_t *>(&h1));
            }
        }
    }
}

cudaError_t launch_pack_gauge(const double *nat, void *dst, int gformat, long V, cudaStream_t s) {
    ProfScope prof("pack_gauge", (double)V * 4 * 288.0, s);
    const int B = 128;
    k_pack_gauge<<<stream_grid(V * 4, B), B, 0, s>>>(reinterpret_cast<const double2 *>(nat), dst, gformat, V);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// out = ca * a + cb * b
// ---------------------------------------------------------------------------------------
template <typename A, typename B>
struct Wider {
    using T = float;
};
template <typename B>
struct Wider<double, B> {
    using T = double;
};
template <typename A>
struct Wider<A, double> {
    using T = double;
};
template <>
struct Wider<double, double> {
    using T = double;
};

template <typename SO, typename SA, typename SB>
__global__ void k_combine(FieldView o, double ca, FieldView a, double cb, FieldView b, int has_b) {
    using C = typename Wider<typename Wider<SO, SA>::T, SB>::T;
    using CO = typename SpinorStore<SO>::C;
    using CA = typename SpinorStore<SA>::C;
    using CB = typename SpinorStore<SB>::C;
    const long total = o.V * o.k;
    const C fa = (C)ca, fb = (C)cb;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long s = g / o.k;
        const int r = (int)(g - s * o.k);
        Spinor<CA> va;
        SpinorStore<SA>::load(a, s, r, va);
        Spinor<CB> vb;
        if (has_b) SpinorStore<SB>::load(b, s, r, vb);
        Spinor<CO> vo;
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                C re = fa * (C)va.s[i][j].re, im = fa * (C)va.s[i][j].im;
                if (has_b) {
                    re += fb * (C)vb.s[i][j].re;
                    im += fb * (C)vb.s[i][j].im;
                }
                vo.s[i][j] = cmk<CO>((CO)re, (CO)im);
            }
        SpinorStore<SO>::store(o, s, r, vo);
    }
}

template <typename SO, typename SA>
static void combine_b(Field o, double ca, Field a, double cb, Field b, int G, int B, cudaStream_t s) {
    const int hb = b.v.data != nullptr;
    Prec pb = hb ? b.prec : a.prec;
    switch (pb) {
        case P64: k_combine<SO, SA, double><<<G, B, 0, s>>>(o.v, ca, a.v, cb, b.v, hb); break;
        case P32: k_combine<SO, SA, float><<<G, B, 0, s>>>(o.v, ca, a.v, cb, b.v, hb); break;
        case P16: k_combine<SO, SA, __half><<<G, B, 0, s>>>(o.v, ca, a.v, cb, b.v, hb); break;
    }
}

template <typename SO>
static void combine_a(Field o, double ca, Field a, double cb, Field b, int G, int B, cudaStream_t s) {
    switch (a.prec) {
        case P64: combine_b<SO, double>(o, ca, a, cb, b, G, B, s); break;
        case P32: combine_b<SO, float>(o, ca, a, cb, b, G, B, s); break;
        case P16: combine_b<SO, __half>(o, ca, a, cb, b, G, B, s); break;
    }
}

cudaError_t launch_combine(Field out, double ca, Field a, double cb, Field b, cudaStream_t s) {
    ProfScope prof("combine",
                   (double)out.v.V * out.v.k * (spb(out.prec) + spb(a.prec) + (b.v.data ? spb(b.prec) : 0.0)), s);
    const int B = 128;
    const int G = stream_grid(out.v.V * out.v.k, B);
    switch (out.prec) {
        case P64: combine_a<double>(out, ca, a, cb, b, G, B, s); break;
        case P32: combine_a<float>(out, ca, a, cb, b, G, B, s); break;
        case P16: combine_a<__half>(out, ca, a, cb, b, G, B, s); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// norms
// ---------------------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(256) k_norm2(FieldView f, CGScalars *st, int as_rho, double *h_rho, int iter,
                                               double *partials, unsigned *counter) {
    using C = typename SpinorStore<S>::C;
    __shared__ double smem[(256 / 32) * MAX_RHS];
    const long total = f.V * f.k;
    double n = 0.0;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long s = g / f.k;
        const int r = (int)(g - s * f.k);
        Spinor<C> v;
        SpinorStore<S>::load(f, s, r, v);
        C a = 0;
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) a += v.s[i][j].re * v.s[i][j].re + v.s[i][j].im * v.s[i][j].im;
        n += (double)a;
    }
    const double bs = block_reduce_rhs(n, f.k, smem);
    const int k = f.k;
    grid_reduce_rhs(bs, k, partials, counter, smem, [=](int r, double tot) {
        st[r].aux = tot;
        if (as_rho) {
            st[r].rho = tot;
            st[r].rho_prev = tot;
            if (h_rho) h_rho[(long)iter * k + r] = tot;
        }
    });
}

// ---------------------------------------------------------------------------------------
// Spectral preconditioner z = P^{-1} r = r + U (G (U^H r)) (Sec. 2), G = shift H^{-1} - I:
// the coefficients y = G c of one RHS, and rho = r^H z with the CG scalars of Fig. 1
// steps 3-4, 8 (preconditioned form)
// ---------------------------------------------------------------------------------------
__global__ void k_sp_coef(const double *G, const double *C, double *Y, int l) {
    for (int a = threadIdx.x; a < l; a += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int b = 0; b < l; b++) {
            const double gr = G[2 * ((long)a * l + b)], gi = G[2 * ((long)a * l + b) + 1];
            const double cr = C[2 * b], ci = C[2 * b + 1];
            re += gr * cr - gi * ci;
            im += gr * ci + gi * cr;
        }
        Y[2 * a] = re;
        Y[2 * a + 1] = im;
    }
}

cudaError_t launch_sp_coef(const double *G, const double *C, double *Y, int l, cudaStream_t s) {
    ProfScope prof("sp_coef", (double)l * l * 16.0, s);
    k_sp_coef<<<1, 256, 0, s>>>(G, C, Y, l);
    return cudaGetLastError();
}

template <typename S>
__global__ void __launch_bounds__(256) k_pcg_rho(FieldView r, FieldView z, CGScalars *st, double *h_rho,
                                                 double *h_beta, int iter, double *partials, unsigned *counter) {
    using C = typename SpinorStore<S>::C;
    __shared__ double smem[(256 / 32) * MAX_RHS];
    const long total = r.V * r.k;
    double n = 0.0;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long s = g / r.k;
        const int q = (int)(g - s * r.k);
        Spinor<C> a, b;
        SpinorStore<S>::load(r, s, q, a);
        SpinorStore<S>::load(z, s, q, b);
        C d = 0;
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) d += a.s[i][j].re * b.s[i][j].re + a.s[i][j].im * b.s[i][j].im;
        n += (double)d;
    }
    const double bs = block_reduce_rhs(n, r.k, smem);
    const int k = r.k;
    grid_reduce_rhs(bs, k, partials, counter, smem, [=](int q, double tot) {
        CGScalars &c = st[q];
        if (!c.active) return;
        if (!(tot > 0.0) || !isfinite(tot)) {  // P^{-1} not positive definite on r
            c.breakdown = 1;
            c.active = 0;
            return;
        }
        c.rho = tot;  // step 4: rho = r^H z
        h_rho[(long)iter * k + q] = tot;
        if (iter >= 1) {  // step 8: beta = rho / rho_prev (rho_prev moved by the CG epilogue)
            c.beta = tot / c.rho_prev;
            h_beta[(long)(iter + 1) * k + q] = c.beta;
        }
    });
}

cudaError_t launch_pcg_rho(Field r, Field z, CGScalars *st, History h, int iter, RedScratch red, cudaStream_t s) {
    ProfScope prof("pcg_rho", (double)r.v.V * r.v.k * 2.0 * spb(r.prec), s);
    if (z.prec != r.prec || z.v.V != r.v.V || z.v.k != r.v.k) return cudaErrorInvalidValue;
    const int B = 256;
    int G = stream_grid(r.v.V * r.v.k, B);
    if (G > red.max_blocks) G = red.max_blocks;
    switch (r.prec) {
        case P64:
            k_pcg_rho<double><<<G, B, 0, s>>>(r.v, z.v, st, h.rho, h.beta, iter, red.partials, red.counter);
            break;
        case P32:
            k_pcg_rho<float><<<G, B, 0, s>>>(r.v, z.v, st, h.rho, h.beta, iter, red.partials, red.counter);
            break;
        case P16:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_norm2(Field f, CGScalars *st, bool as_rho, History h, int iter, RedScratch red, cudaStream_t s) {
    ProfScope prof("norm2", (double)f.v.V * f.v.k * spb(f.prec), s);
    const int B = 256;
    int G = stream_grid(f.v.V * f.v.k, B);
    if (G > red.max_blocks) G = red.max_blocks;
    switch (f.prec) {
        case P64: k_norm2<double><<<G, B, 0, s>>>(f.v, st, as_rho, h.rho, iter, red.partials, red.counter); break;
        case P32: k_norm2<float><<<G, B, 0, s>>>(f.v, st, as_rho, h.rho, iter, red.partials, red.counter); break;
        case P16: k_norm2<__half><<<G, B, 0, s>>>(f.v, st, as_rho, h.rho, iter, red.partials, red.counter); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// x += alpha p (pending from the previous iteration), p = r + beta p, window append
// v = r / sqrt(rho).  x lives in the wide precision (FP64 for FP64 storage, else FP32).
// ---------------------------------------------------------------------------------------
template <typename S, typename SV>
__global__ void k_pupdate(FieldView r, FieldView p, FieldView x, int first, const CGScalars *st, FieldView v,
                          int append, unsigned long long *dev_bytes) {
    using C = typename SpinorStore<S>::C;
    using CV = typename SpinorStore<SV>::C;
    {
        bool any = false;
        for (int q = 0; q < r.k; q++) any = any || st[q].active;
        if (!any) return;
    }
    constexpr unsigned SB = SpinorStore<S>::BYTES, SBV = SpinorStore<SV>::BYTES;
    unsigned moved = 0;  // bytes this thread read and wrote
    const long total = r.V * r.k;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long s = g / r.k;
        const int q = (int)(g - s * r.k);
        const CGScalars &sc = st[q];
        // a RHS that has stopped while others in its batch go on keeps its p (and r, x)
        // untouched, so that if the final residual check resumes it, it continues exactly as
        // it would have alone
        if (!first && !sc.active && !sc.x_pending) continue;
        Spinor<C> rr, pp;
        if (first) {
            SpinorStore<S>::load(r, s, q, rr);
            pp = rr;
            moved += SB;
        } else {
            SpinorStore<S>::load(p, s, q, pp);
            moved += SB;
            if (sc.x_pending) {  // Fig. 1 step 13 of the previous iteration
                const CV al = (CV)sc.alpha;
                Spinor<CV> xx;
                SpinorStore<SV>::load(x, s, q, xx);
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++) {
                        xx.s[i][j].re += al * (CV)pp.s[i][j].re;
                        xx.s[i][j].im += al * (CV)pp.s[i][j].im;
                    }
                SpinorStore<SV>::store(x, s, q, xx);
                moved += 2 * SBV;
            }
            if (!sc.active) continue;  // x done; p stays
            SpinorStore<S>::load(r, s, q, rr);
            moved += SB;
            const C be = (C)sc.beta;
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 3; j++)
                    pp.s[i][j] = cmk<C>(rr.s[i][j].re + be * pp.s[i][j].re, rr.s[i][j].im + be * pp.s[i][j].im);
        }
        SpinorStore<S>::store(p, s, q, pp);
        moved += SB;
        if (append && sc.active) {
            const CV sc_inv = (CV)(1.0 / sqrt(sc.rho));
            Spinor<CV> vv;
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) vv.s[i][j] = cmk<CV>((CV)rr.s[i][j].re * sc_inv, (CV)rr.s[i][j].im * sc_inv);
            SpinorStore<SV>::store(v, s, q, vv);
            moved += SBV;
        }
    }
    if (dev_bytes) {
        const unsigned w = __reduce_add_sync(0xffffffffu, moved);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(dev_bytes, (unsigned long long)w);
    }
}

cudaError_t launch_pupdate(Field r, Field p, Field x, bool first, CGScalars *st, Field v_append, cudaStream_t s) {
    const int app = v_append.v.data != nullptr;
    // per batch width, like the stencils: k = 1 fields (85 MB at 24^3x64) partly stay in L2
    const std::string pname = r.v.k > 1 ? "pupdate_k" + std::to_string(r.v.k) : std::string("pupdate");
    // bytes: counted by the kernel while timing is on (RHS that have stopped move nothing),
    // else the estimate for every RHS active
    unsigned long long *devb = prof_device_bytes(pname.c_str());
    ProfScope prof(pname.c_str(),
                   devb ? 0.0
                        : (double)r.v.V * r.v.k * ((first ? 2.0 : 3.0) * spb(r.prec) + (first ? 0.0 : 2.0 * spb(x.prec))) +
                              (app ? (double)r.v.V * spb(v_append.prec) : 0.0),
                   s);
    const int B = 128;
    const int G = stream_grid(r.v.V * r.v.k, B);
    if (app && v_append.prec != x.prec) return cudaErrorInvalidValue;
    switch (r.prec) {
        case P64:
            if (x.prec != P64) return cudaErrorInvalidValue;
            k_pupdate<double, double><<<G, B, 0, s>>>(r.v, p.v, x.v, first, st, v_append.v, app, devb);
            break;
        case P32:
            if (x.prec != P32) return cudaErrorInvalidValue;
            k_pupdate<float, float><<<G, B, 0, s>>>(r.v, p.v, x.v, first, st, v_append.v, app, devb);
            break;
        case P16:
            if (x.prec != P32) return cudaErrorInvalidValue;
            k_pupdate<__half, float><<<G, B, 0, s>>>(r.v, p.v, x.v, first, st, v_append.v, app, devb);
            break;
    }
    return cudaGetLastError();
}

template <typename S, typename SV>
__global__ void k_xflush(FieldView p, FieldView x, const CGScalars *st) {
    using C = typename SpinorStore<S>::C;
    using CV = typename SpinorStore<SV>::C;
    const long total = p.V * p.k;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long s = g / p.k;
        const int q = (int)(g - s * p.k);
        if (!st[q].x_pending) continue;
        const CV al = (CV)st[q].alpha;
        Spinor<C> pp;
        Spinor<CV> xx;
        SpinorStore<S>::load(p, s, q, pp);
        SpinorStore<SV>::load(x, s, q, xx);
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                xx.s[i][j].re += al * (CV)pp.s[i][j].re;
                xx.s[i][j].im += al * (CV)pp.s[i][j].im;
            }
        SpinorStore<SV>::store(x, s, q, xx);
    }
}

__global__ void k_clear_pending(CGScalars *st, int k) {
    if (threadIdx.x < k) st[threadIdx.x].x_pending = 0;
}

cudaError_t launch_xflush(Field p, Field x, CGScalars *st, int k, cudaStream_t s) {
    ProfScope prof("xflush", (double)p.v.V * p.v.k * (spb(p.prec) + 2.0 * spb(x.prec)), s);
    const int B = 128;
    const int G = stream_grid(p.v.V * p.v.k, B);
    switch (p.prec) {
        case P64: k_xflush<double, double><<<G, B, 0, s>>>(p.v, x.v, st); break;
        case P32: k_xflush<float, float><<<G, B, 0, s>>>(p.v, x.v, st); break;
        case P16: k_xflush<__half, float><<<G, B, 0, s>>>(p.v, x.v, st); break;
    }
    k_clear_pending<<<1, 32, 0, s>>>(st, k);
    return cudaGetLastError();
}

__global__ void k_cg_init(CGScalars *st, int k, double tol2, double *h_beta) {
    const int r = threadIdx.x;
    if (r >= k) return;
    st[r].target = tol2 * st[r].aux;
    st[r].active = 1;
    st[r].breakdown = 0;
    st[r].alpha = 0.0;
    st[r].beta = 0.0;
    st[r].pAp = 0.0;
    st[r].iters = 0;
    st[r].nit = 0;
    st[r].x_pending = 0;
    if (h_beta) h_beta[k + r] = 0.0;  // beta_1 := 0
}

cudaError_t launch_cg_init(CGScalars *st, int k, double tol, History h, cudaStream_t s) {
    ProfScope prof("cg_init", 0.0, s);
    k_cg_init<<<1, 32, 0, s>>>(st, k, tol * tol, h.beta);
    return cudaGetLastError();
}

}  // namespace eig
