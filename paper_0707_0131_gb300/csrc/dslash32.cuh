// Internal header of the FP32-arithmetic Wilson stencil (dslash32*.cu).
//
// Wilson-Dirac dslash for FP32 arithmetic (FP32 or FP16 storage), the matrix-vector
// product of CG on A = M^H M (Sec. 1, Fig. 1 step 11), with the CG epilogues of
// dslash.cu.  Same operator and spin projection as dslash.cu (see there); this
// version is written for Blackwell's instruction budget:
//
//  * complex numbers are float2 and the SU(3) products use the packed FP32 FMA
//    (fma.rn.f32x2): u * h = re(u) * (h.re, h.im) + im(u) * (-h.im, h.re), two packed
//    FMAs per complex multiply-add instead of four scalar ones;
//  * each thread handles RB right-hand sides of one site, so the link loads, the
//    third-row reconstruction and the index arithmetic are shared by RB RHS;
//  * all offsets are 32-bit (the op checks that a field fits).
//
// At the Wilson stencil's arithmetic intensity (about 1320 flop per 384 algorithmic
// bytes per site in FP32) scalar FP32 code on GB300 is limited by instruction issue
// rather than by HBM; halving the FP instruction count moves it back under the
// memory roof.
#pragma once
#include <cuda_fp16.h>

#include "fastdiv.h"
#include "kernels.cuh"

namespace eig {

// arguments of one FP32-arithmetic stencil launch
struct K32 {
    const float4 *in;
    const float *in_s;
    float4 *out;
    float *out_s;
    const float4 *p;
    const float *p_s;
    float4 *r;
    float *r_s;
    float4 *x;     // FP32 x (always FP32 storage)
    float4 *tsave; // FP32, k = 1
    const void *g;
    unsigned L0, L1, L2, L3, V;  // V: output sites (V / 2 in the odd-even form)
    unsigned Vg;                 // lattice sites: stride of the link planes
    FastDiv d0, d1, d2;  // division by L0, L1, L2
    // odd-even form: output parity (or -1), centre-term input, hop coefficient
    int eo;
    unsigned lh;         // L0 / 2
    FastDiv dh;          // division by L0 / 2 (lh >= 2)
    const float4 *cen;
    const float *cen_s;
    float hcoef;
    // tiled traversal (full lattice, tile != 0): consecutive output sites run through
    // blocks of 2^tl0 x 2^tl1 x 2^tl2 x 2^tl3 lattice sites, the blocks in lexicographic
    // order (nt0 x nt1 x nt2 per t-slab), so that a CTA's sites are each other's
    // neighbours and more hop loads hit L1
    unsigned tile, tl0, tl1, tl2, tl3, nt0, nt1;
    FastDiv dt0, dt1, dt2;
    unsigned k;    // RHS per field
    unsigned P;    // V * k (chunk plane stride in vector elements)
    float diag;
    int save_t;
    CGScalars *st;
    double *h_alpha, *h_beta, *h_rho;
    int iter;
    const int *jbase;  // device iteration base added to iter (null: none)
    double *partials;
    unsigned *counter;
};

// launchers of the direct-load variants (dslash32d_rb1.cu, dslash32d_rb2.cu); variant
// numbers as in dslash32.cu, prec 32 or 16, epi one of E_PLAIN, E_NORM, E_CG
cudaError_t d32_launch_direct_rb1(int variant, int prec, int gf, bool dag, int epi, const K32 &a, int cap,
                                  cudaStream_t s);
cudaError_t d32_launch_direct_rb2(int variant, int prec, int gf, bool dag, int epi, const K32 &a, int cap,
                                  cudaStream_t s);
// launchers of the pipelined-pair variants (dslash32p2.cu, dslash32p3.cu: 2 or 3 blocks
// per SM; k >= 2, fields 32-byte aligned)
cudaError_t d32_launch_pp2(int prec, int gf, bool dag, int epi, const K32 &a, int cap, cudaStream_t s);
cudaError_t d32_launch_pp3(int prec, int gf, bool dag, int epi, const K32 &a, int cap, cudaStream_t s);
// as d32_launch_pp3, with an L1 prefetch of the hop after next (dslash32p3f.cu)
cudaError_t d32_launch_pp3f(int prec, int gf, bool dag, int epi, const K32 &a, int cap, cudaStream_t s);
// grid for a launch of `kern` (TPB threads, `smem` bytes of dynamic shared memory):
// resident blocks per SM x SMs, no more blocks than `work` threads need, at most cap
int d32_grid(const void *kern, long work, int cap, size_t smem);

namespace {

using F2 = float2;

__device__ __forceinline__ F2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ F2 add2(F2 a, F2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ F2 sub2(F2 a, F2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ F2 mul2(F2 a, F2 b) { return __fmul2_rn(a, b); }
// i * a
__device__ __forceinline__ F2 ix(F2 a) { return f2(-a.y, a.x); }
// -i * a
__device__ __forceinline__ F2 mix(F2 a) { return f2(a.y, -a.x); }

struct Sp {
    F2 c[12];  // spin * 3 + colour
};
struct Hf {
    F2 c[6];  // spin (0..1) * 3 + colour
};
struct Lk {
    F2 u[9];  // row * 3 + col
};

// ------------------------------------------------------------------------------
// storage
// ------------------------------------------------------------------------------
template <typename S>
struct Store32;

template <>
struct Store32<float> {
    static constexpr int BYTES = 96;
    // element (chunk c, site s, rhs r) at base[c * P + s * k + r], P = V * k
    __device__ static __forceinline__ void load(const float4 *__restrict__ p, const float *, unsigned P, unsigned o,
                                                Sp &v) {
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const float4 d = p[c * P + o];
            v.c[2 * c] = f2(d.x, d.y);
            v.c[2 * c + 1] = f2(d.z, d.w);
        }
    }
    __device__ static __forceinline__ void store(float4 *__restrict__ p, float *, unsigned P, unsigned o, const Sp &v) {
#pragma unroll
        for (int c = 0; c < 6; c++) p[c * P + o] = make_float4(v.c[2 * c].x, v.c[2 * c].y, v.c[2 * c + 1].x, v.c[2 * c + 1].y);
    }
};

template <>
struct Store32<__half> {
    static constexpr int BYTES = 52;
    __device__ static __forceinline__ void load(const float4 *__restrict__ pp, const float *__restrict__ scale,
                                                unsigned P, unsigned o, Sp &v) {
        const uint4 *p = reinterpret_cast<const uint4 *>(pp);
        const float sc = scale[o];
        const F2 s2 = f2(sc, sc);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const uint4 d = p[c * P + o];
            const uint32_t w[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                __half2 h = *reinterpret_cast<const __half2 *>(&w[q]);
                v.c[4 * c + q] = mul2(__half22float2(h), s2);
            }
        }
    }
    __device__ static __forceinline__ void store(float4 *__restrict__ pp, float *__restrict__ scale, unsigned P,
                                                 unsigned o, const Sp &v) {
        float mx = 0.f;
#pragma unroll
        for (int e = 0; e < 12; e++) mx = fmaxf(mx, fmaxf(fabsf(v.c[e].x), fabsf(v.c[e].y)));
        const float inv = mx > 0.f ? 1.0f / mx : 0.f;
        scale[o] = mx;
        uint4 *p = reinterpret_cast<uint4 *>(pp);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const F2 t = mul2(v.c[4 * c + q], f2(inv, inv));
                __half2 h = __float22half2_rn(t);
                w[q] = *reinterpret_cast<uint32_t *>(&h);
            }
            p[c * P + o] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
};

// row2 = conj(row0 x row1)
__device__ __forceinline__ F2 cmulf(F2 a, F2 b) { return fma2(f2(a.x, a.x), b, mul2(f2(a.y, a.y), ix(b))); }
__device__ __forceinline__ void rebuild_row2(Lk &U) {
    const F2 a = sub2(cmulf(U.u[1], U.u[5]), cmulf(U.u[2], U.u[4]));
    const F2 b = sub2(cmulf(U.u[2], U.u[3]), cmulf(U.u[0], U.u[5]));
    const F2 c = sub2(cmulf(U.u[0], U.u[4]), cmulf(U.u[1], U.u[3]));
    U.u[6] = f2(a.x, -a.y);
    U.u[7] = f2(b.x, -b.y);
    U.u[8] = f2(c.x, -c.y);
}

template <int GF>
struct Link32;

template <>
struct Link32<GF_F32_12> {
    // planes [mu][3][V] float4
    __device__ static __forceinline__ void load(const void *g, unsigned V, int mu, unsigned s, Lk &U) {
        const float4 *p = static_cast<const float4 *>(g) + (unsigned)mu * 3u * V;
        const float4 a = __ldg(p + s), b = __ldg(p + V + s), c = __ldg(p + 2 * V + s);
        U.u[0] = f2(a.x, a.y);
        U.u[1] = f2(a.z, a.w);
        U.u[2] = f2(b.x, b.y);
        U.u[3] = f2(b.z, b.w);
        U.u[4] = f2(c.x, c.y);
        U.u[5] = f2(c.z, c.w);
        rebuild_row2(U);
    }
};

template <>
struct Link32<GF_F32_18> {
    // planes [mu][9][V] float2
    __device__ static __forceinline__ void load(const void *g, unsigned V, int mu, unsigned s, Lk &U) {
        const float2 *p = static_cast<const float2 *>(g) + (unsigned)mu * 9u * V;
#pragma unroll
        for (int e = 0; e < 9; e++) U.u[e] = __ldg(p + e * V + s);
    }
};

template <>
struct Link32<GF_F16_12> {
    // planes [mu][3][V] uint2 (4 halves = 2 complex)
    __device__ static __forceinline__ void load(const void *g, unsigned V, int mu, unsigned s, Lk &U) {
        const uint2 *p = static_cast<const uint2 *>(g) + (unsigned)mu * 3u * V;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const uint2 d = __ldg(p + q * V + s);
            U.u[2 * q] = __half22float2(*reinterpret_cast<const __half2 *>(&d.x));
            U.u[2 * q + 1] = __half22float2(*reinterpret_cast<const __half2 *>(&d.y));
        }
        rebuild_row2(U);
    }
};

// ------------------------------------------------------------------------------
// spin projection (I + SG g_mu) in the chiral basis; see dslash.cu for B_mu
// ------------------------------------------------------------------------------
template <int MU, int SG>
__device__ __forceinline__ void project(const Sp &p, Hf &h) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const F2 a0 = p.c[c], a1 = p.c[3 + c], b0 = p.c[6 + c], b1 = p.c[9 + c];
        if (MU == 0) {  // B b = (i b1, i b0)
            h.c[c] = SG > 0 ? add2(a0, ix(b1)) : add2(a0, mix(b1));
            h.c[3 + c] = SG > 0 ? add2(a1, ix(b0)) : add2(a1, mix(b0));
        } else if (MU == 1) {  // B b = (-b1, b0)
            h.c[c] = SG > 0 ? sub2(a0, b1) : add2(a0, b1);
            h.c[3 + c] = SG > 0 ? add2(a1, b0) : sub2(a1, b0);
        } else if (MU == 2) {  // B b = (i b0, -i b1)
            h.c[c] = SG > 0 ? add2(a0, ix(b0)) : add2(a0, mix(b0));
            h.c[3 + c] = SG > 0 ? add2(a1, mix(b1)) : add2(a1, ix(b1));
        } else {  // B b = b
            h.c[c] = SG > 0 ? add2(a0, b0) : sub2(a0, b0);
            h.c[3 + c] = SG > 0 ? add2(a1, b1) : sub2(a1, b1);
        }
    }
}

// acc += (h, SG B^H h)
template <int MU, int SG>
__device__ __forceinline__ void accumulate(Sp &acc, const Hf &h) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const F2 h0 = h.c[c], h1 = h.c[3 + c];
        acc.c[c] = add2(acc.c[c], h0);
        acc.c[3 + c] = add2(acc.c[3 + c], h1);
        if (MU == 0) {  // B^H h = (-i h1, -i h0)
            acc.c[6 + c] = add2(acc.c[6 + c], SG > 0 ? mix(h1) : ix(h1));
            acc.c[9 + c] = add2(acc.c[9 + c], SG > 0 ? mix(h0) : ix(h0));
        } else if (MU == 1) {  // B^H h = (h1, -h0)
            acc.c[6 + c] = SG > 0 ? add2(acc.c[6 + c], h1) : sub2(acc.c[6 + c], h1);
            acc.c[9 + c] = SG > 0 ? sub2(acc.c[9 + c], h0) : add2(acc.c[9 + c], h0);
        } else if (MU == 2) {  // B^H h = (-i h0, i h1)
            acc.c[6 + c] = add2(acc.c[6 + c], SG > 0 ? mix(h0) : ix(h0));
            acc.c[9 + c] = add2(acc.c[9 + c], SG > 0 ? ix(h1) : mix(h1));
        } else {  // B^H h = h
            acc.c[6 + c] = SG > 0 ? add2(acc.c[6 + c], h0) : sub2(acc.c[6 + c], h0);
            acc.c[9 + c] = SG > 0 ? add2(acc.c[9 + c], h1) : sub2(acc.c[9 + c], h1);
        }
    }
}

// o = U h (DAGGER = false) or U^H h (true):  (x + iy) h = x h + y (i h)
template <bool DAGGER>
__device__ __forceinline__ void mul_link(const Lk &U, const Hf &h, Hf &o) {
    Hf ih;
#pragma unroll
    for (int e = 0; e < 6; e++) ih.c[e] = ix(h.c[e]);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        F2 o0 = f2(0.f, 0.f), o1 = f2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const F2 u = DAGGER ? U.u[b * 3 + a] : U.u[a * 3 + b];
            const F2 ur = f2(u.x, u.x);
            const F2 ui = DAGGER ? f2(-u.y, -u.y) : f2(u.y, u.y);
            o0 = fma2(ur, h.c[b], o0);
            o0 = fma2(ui, ih.c[b], o0);
            o1 = fma2(ur, h.c[3 + b], o1);
            o1 = fma2(ui, ih.c[3 + b], o1);
        }
        o.c[a] = o0;
        o.c[3 + a] = o1;
    }
}


// ------------------------------------------------------------------------------
// Software pipeline: the 8 hops and the centre load of a site go through a ring of
// NS stages in shared memory filled by cp.async, so that while hop h is computed
// the data of hops h+1 .. h+NS-1 is already in flight (memory-level parallelism
// without holding it in registers).  Layout [stage][slot][thread] of 16-byte slots.
// ------------------------------------------------------------------------------
constexpr int NS = 3;
constexpr int TPB = 128;

template <typename S>
struct SpSlots;
template <>
struct SpSlots<float> {
    static constexpr int N = 6;  // float4 chunks
};
template <>
struct SpSlots<__half> {
    static constexpr int N = 4;  // 3 uint4 chunks + the scale
};
template <int GF>
struct LkSlots {
    static constexpr int N = GF == GF_F32_18 ? 5 : (GF == GF_F16_12 ? 2 : 3);
};

__device__ __forceinline__ void cpa16(void *d, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(d)), "l"(g)
                 : "memory");
}
__device__ __forceinline__ void cpa8(void *d, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(d)), "l"(g)
                 : "memory");
}
__device__ __forceinline__ void cpa4(void *d, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(d)), "l"(g)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename S, int GF, int RB>
struct Pipe {
    static constexpr int NSP = SpSlots<S>::N;
    static constexpr int NLK = LkSlots<GF>::N;
    static constexpr int NSLOT = RB * NSP + NLK;
    float4 *sm;
    __device__ __forceinline__ float4 *slot(int st, int k) const { return sm + ((st * NSLOT + k) * TPB + threadIdx.x); }

    // issue the copies of one load: spinor of site ns (RB RHS), and link (mu, ls) if with_link
    __device__ __forceinline__ void issue(const K32 &a, int st, unsigned ns, unsigned r0, unsigned rstride, int mu,
                                          unsigned ls, bool with_link) const {
#pragma unroll
        for (int q = 0; q < RB; q++) {
            const unsigned o = ns * a.k + r0 + q * rstride;
            if (sizeof(S) == 4) {
#pragma unroll
                for (int c = 0; c < 6; c++) cpa16(slot(st, q * NSP + c), a.in + c * a.P + o);
            } else {
                const uint4 *p = reinterpret_cast<const uint4 *>(a.in);
#pragma unroll
                for (int c = 0; c < 3; c++) cpa16(slot(st, q * NSP + c), p + c * a.P + o);
                cpa4(slot(st, q * NSP + 3), a.in_s + o);
            }
        }
        if (with_link) {
            if (GF == GF_F32_12) {
                const float4 *g = static_cast<const float4 *>(a.g) + (unsigned)mu * 3u * a.Vg;
#pragma unroll
                for (int c = 0; c < 3; c++) cpa16(slot(st, RB * NSP + c), g + c * a.Vg + ls);
            } else if (GF == GF_F32_18) {
                const float2 *g = static_cast<const float2 *>(a.g) + (unsigned)mu * 9u * a.Vg;
#pragma unroll
                for (int e = 0; e < 9; e++)
                    cpa8(reinterpret_cast<float2 *>(slot(st, RB * NSP + e / 2)) + (e & 1), g + e * a.Vg + ls);
            } else {
                const uint2 *g = static_cast<const uint2 *>(a.g) + (unsigned)mu * 3u * a.Vg;
#pragma unroll
                for (int c = 0; c < 3; c++)
                    cpa8(reinterpret_cast<uint2 *>(slot(st, RB * NSP + c / 2)) + (c & 1), g + c * a.Vg + ls);
            }
        }
        cpa_commit();
    }

    __device__ __forceinline__ void spinor(int st, int q, Sp &v) const {
        if (sizeof(S) == 4) {
#pragma unroll
            for (int c = 0; c < 6; c++) {
                const float4 d = *slot(st, q * NSP + c);
                v.c[2 * c] = f2(d.x, d.y);
                v.c[2 * c + 1] = f2(d.z, d.w);
            }
        } else {
            const float sc = slot(st, q * NSP + 3)->x;
            const F2 s2 = f2(sc, sc);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float4 d4 = *slot(st, q * NSP + c);
                const uint4 d = *reinterpret_cast<const uint4 *>(&d4);
                const uint32_t w[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
                for (int e = 0; e < 4; e++) v.c[4 * c + e] = mul2(__half22float2(*reinterpret_cast<const __half2 *>(&w[e])), s2);
            }
        }
    }

    __device__ __forceinline__ void link(int st, Lk &U) const {
        if (GF == GF_F32_12) {
            const float4 a = *slot(st, RB * NSP), b = *slot(st, RB * NSP + 1), c = *slot(st, RB * NSP + 2);
            U.u[0] = f2(a.x, a.y);
            U.u[1] = f2(a.z, a.w);
            U.u[2] = f2(b.x, b.y);
            U.u[3] = f2(b.z, b.w);
            U.u[4] = f2(c.x, c.y);
            U.u[5] = f2(c.z, c.w);
            rebuild_row2(U);
        } else if (GF == GF_F32_18) {
#pragma unroll
            for (int e = 0; e < 9; e++) U.u[e] = reinterpret_cast<const float2 *>(slot(st, RB * NSP + e / 2))[e & 1];
        } else {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const uint2 d = reinterpret_cast<const uint2 *>(slot(st, RB * NSP + c / 2))[c & 1];
                U.u[2 * c] = __half22float2(*reinterpret_cast<const __half2 *>(&d.x));
                U.u[2 * c + 1] = __half22float2(*reinterpret_cast<const __half2 *>(&d.y));
            }
            rebuild_row2(U);
        }
    }
};

template <int MU, int SG, bool DAGGER, typename S, int GF, int RB>
__device__ __forceinline__ void hop_from(const Pipe<S, GF, RB> &pp, int st, Sp *acc) {
    Lk U;
    pp.link(st, U);
#pragma unroll
    for (int q = 0; q < RB; q++) {
        Sp nb;
        Hf h, uh;
        pp.spinor(st, q, nb);
        project<MU, SG>(nb, h);
        mul_link<DAGGER>(U, h, uh);
        accumulate<MU, SG>(acc[q], uh);
    }
}

__device__ __forceinline__ float norm2f(const Sp &v) {
    F2 n = f2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < 12; e++) n = fma2(v.c[e], v.c[e], n);
    return n.x + n.y;
}


// one hop with its loads straight to registers (MODE 1)
template <int MU, int SG, bool DAGGER, typename S, int GF, int RB>
__device__ __forceinline__ void hop_direct(const K32 &a, unsigned ns, unsigned ls, unsigned r0, unsigned rstride,
                                           Sp *acc) {
    Lk U;
    Link32<GF>::load(a.g, a.Vg, MU, ls, U);
#pragma unroll
    for (int q = 0; q < RB; q++) {
        Sp nb;
        Hf h, uh;
        Store32<S>::load(a.in, a.in_s, a.P, ns * a.k + r0 + q * rstride, nb);
        project<MU, SG>(nb, h);
        mul_link<DAGGER>(U, h, uh);
        accumulate<MU, SG>(acc[q], uh);
    }
}

__device__ __forceinline__ void pf_l1(const void *p) { asm volatile("prefetch.L1 [%0];" ::"l"(p)); }

// MODE 2: asks L1 for the data of a later hop (the spinor chunks of the thread's RB
// RHS at site ns and the link (mu, ls)) without holding registers for it
template <typename S, int GF, int RB>
__device__ __forceinline__ void prefetch_hop(const K32 &a, unsigned ns, unsigned ls, int mu, bool with_link,
                                             unsigned r0, unsigned rstride) {
#pragma unroll
    for (int q = 0; q < RB; q++) {
        const unsigned o = ns * a.k + r0 + q * rstride;
        if (sizeof(S) == 4) {
#pragma unroll
            for (int c = 0; c < 6; c++) pf_l1(a.in + c * a.P + o);
        } else {
            const uint4 *p = reinterpret_cast<const uint4 *>(a.in);
#pragma unroll
            for (int c = 0; c < 3; c++) pf_l1(p + c * a.P + o);
            pf_l1(a.in_s + o);
        }
    }
    if (!with_link) return;
    if (GF == GF_F32_12) {
        const float4 *g = static_cast<const float4 *>(a.g) + (unsigned)mu * 3u * a.Vg;
#pragma unroll
        for (int c = 0; c < 3; c++) pf_l1(g + c * a.Vg + ls);
    } else if (GF == GF_F32_18) {
        const float2 *g = static_cast<const float2 *>(a.g) + (unsigned)mu * 9u * a.Vg;
#pragma unroll
        for (int e = 0; e < 9; e++) pf_l1(g + e * a.Vg + ls);
    } else {
        const uint2 *g = static_cast<const uint2 *>(a.g) + (unsigned)mu * 3u * a.Vg;
#pragma unroll
        for (int c = 0; c < 3; c++) pf_l1(g + c * a.Vg + ls);
    }
}

enum { E_PLAIN = 0, E_NORM = 1, E_CG = 2 };

// MODE 0: loads staged through the cp.async ring (Pipe); MODE 1: loads straight to
// registers, with MINB blocks per SM requested from the register allocator; MODE 2:
// as 1, with an L1 prefetch of the next hop's data before each hop.
template <typename S, int GF, bool DAG, int EPI, int RB, int MODE, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_dslash32(const K32 a) {
    extern __shared__ __align__(16) float4 dyn_sm[];
    __shared__ double smem[(TPB / 32) * MAX_RHS];
    if (EPI != E_PLAIN) {
        bool any = false;
        for (unsigned q = 0; q < a.k; q++) any = any || a.st[q].active;
        if (!any) return;
    }
    Pipe<S, GF, RB> pp;
    pp.sm = dyn_sm;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    const unsigned KB = a.k / RB;  // thread groups per site (k and RB are powers of two)
    const unsigned kb_shift = __ffs(KB) - 1;
    const unsigned total = a.V * KB;
    const unsigned s1 = a.L0, s2 = a.L0 * a.L1, s3 = s2 * a.L2;
    float nrm[RB];
#pragma unroll
    for (int q = 0; q < RB; q++) nrm[q] = 0.f;
    for (unsigned g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        unsigned s = g >> kb_shift;  // output field index (traversal index when tiled)
        // a thread's RB RHS are KB apart, so every load instruction of a warp is contiguous
        const unsigned r0 = g & (KB - 1);
        unsigned sl, x, y, z, t;  // lattice site and its coordinates
        if (a.eo >= 0) {
            // half-lattice index: the site of parity eo in x-pair s mod lh of row s / lh
            const unsigned rest = a.lh > 1 ? fastdiv(s, a.dh) : s;
            const unsigned q2 = fastdiv(rest, a.d1);
            t = fastdiv(q2, a.d2);
            y = rest - q2 * a.L1;
            z = q2 - t * a.L2;
            x = 2 * (s - rest * a.lh) + ((a.eo + y + z + t) & 1);
            sl = x + rest * a.L0;
        } else if (a.tile) {
            const unsigned tb = a.tl0 + a.tl1 + a.tl2 + a.tl3;
            const unsigned tid = s >> tb, w = s & ((1u << tb) - 1u);
            const unsigned q1 = fastdiv(tid, a.dt0), q2 = fastdiv(q1, a.dt1), tt = fastdiv(q2, a.dt2);
            x = ((tid - q1 * a.nt0) << a.tl0) + (w & ((1u << a.tl0) - 1u));
            y = ((q1 - q2 * a.nt1) << a.tl1) + ((w >> a.tl0) & ((1u << a.tl1) - 1u));
            z = ((q2 - tt * (a.L2 >> a.tl2)) << a.tl2) + ((w >> (a.tl0 + a.tl1)) & ((1u << a.tl2) - 1u));
            t = (tt << a.tl3) + (w >> (a.tl0 + a.tl1 + a.tl2));
            sl = x + a.L0 * (y + a.L1 * (z + a.L2 * t));
            s = sl;
        } else {
            const unsigned q1 = fastdiv(s, a.d0), q2 = fastdiv(q1, a.d1);
            t = fastdiv(q2, a.d2);
            x = s - q1 * a.L0;
            y = q1 - q2 * a.L1;
            z = q2 - t * a.L2;
            sl = s;
        }
        unsigned nbr[9], lks[8];  // neighbour sites (then field indices), link sites
        nbr[0] = x == a.L0 - 1 ? sl - (a.L0 - 1) : sl + 1;
        nbr[1] = x == 0 ? sl + (a.L0 - 1) : sl - 1;
        nbr[2] = y == a.L1 - 1 ? sl - (a.L1 - 1) * s1 : sl + s1;
        nbr[3] = y == 0 ? sl + (a.L1 - 1) * s1 : sl - s1;
        nbr[4] = z == a.L2 - 1 ? sl - (a.L2 - 1) * s2 : sl + s2;
        nbr[5] = z == 0 ? sl + (a.L2 - 1) * s2 : sl - s2;
        nbr[6] = t == a.L3 - 1 ? sl - (a.L3 - 1) * s3 : sl + s3;
        nbr[7] = t == 0 ? sl + (a.L3 - 1) * s3 : sl - s3;
#pragma unroll
        for (int h = 0; h < 8; h++) lks[h] = (h & 1) ? nbr[h] : sl;
        if (a.eo >= 0) {
#pragma unroll
            for (int h = 0; h < 8; h++) nbr[h] >>= 1;  // the other parity's half-lattice field
        }
        nbr[8] = s;
        Sp acc[RB];
#pragma unroll
        for (int q = 0; q < RB; q++)
#pragma unroll
            for (int e = 0; e < 12; e++) acc[q].c[e] = f2(0.f, 0.f);
        Sp c0[RB];
        if (MODE >= 1) {
            // MODE 2: the data of hop h + 1 is requested into L1 before hop h is computed
#define EIG_PF(h)                                                                                  \
    if (MODE == 2) prefetch_hop<S, GF, RB>(a, nbr[h], h < 8 ? lks[h] : 0u, (h) >> 1, (h) < 8, r0, KB)
            EIG_PF(1);
            hop_direct<0, SF, false, S, GF, RB>(a, nbr[0], lks[0], r0, KB, acc);
            EIG_PF(2);
            hop_direct<0, SB, true, S, GF, RB>(a, nbr[1], lks[1], r0, KB, acc);
            EIG_PF(3);
            hop_direct<1, SF, false, S, GF, RB>(a, nbr[2], lks[2], r0, KB, acc);
            EIG_PF(4);
            hop_direct<1, SB, true, S, GF, RB>(a, nbr[3], lks[3], r0, KB, acc);
            EIG_PF(5);
            hop_direct<2, SF, false, S, GF, RB>(a, nbr[4], lks[4], r0, KB, acc);
            EIG_PF(6);
            hop_direct<2, SB, true, S, GF, RB>(a, nbr[5], lks[5], r0, KB, acc);
            EIG_PF(7);
            hop_direct<3, SF, false, S, GF, RB>(a, nbr[6], lks[6], r0, KB, acc);
            EIG_PF(8);
            hop_direct<3, SB, true, S, GF, RB>(a, nbr[7], lks[7], r0, KB, acc);
#undef EIG_PF
#pragma unroll
            for (int q = 0; q < RB; q++) {
                if (a.eo < 0) Store32<S>::load(a.in, a.in_s, a.P, s * a.k + r0 + q * KB, c0[q]);
                else if (a.cen) Store32<S>::load(a.cen, a.cen_s, a.P, s * a.k + r0 + q * KB, c0[q]);
                else
#pragma unroll
                    for (int e = 0; e < 12; e++) c0[q].c[e] = f2(0.f, 0.f);  // hops only
            }
        } else {
        // prologue: loads 0 .. NS-2
#pragma unroll
        for (int h = 0; h < NS - 1; h++) pp.issue(a, h % NS, nbr[h], r0, KB, h >> 1, lks[h], true);
#pragma unroll
        for (int h = 0; h < 9; h++) {
            const int nx = h + NS - 1;
            if (nx < 9) pp.issue(a, nx % NS, nbr[nx], r0, KB, nx >> 1, nx < 8 ? lks[nx] : 0u, nx < 8);
            else cpa_commit();  // keep the group count uniform
            cpa_wait<NS - 1>();
            const int st = h % NS;
            switch (h) {
                case 0: hop_from<0, SF, false>(pp, st, acc); break;
                case 1: hop_from<0, SB, true>(pp, st, acc); break;
                case 2: hop_from<1, SF, false>(pp, st, acc); break;
                case 3: hop_from<1, SB, true>(pp, st, acc); break;
                case 4: hop_from<2, SF, false>(pp, st, acc); break;
                case 5: hop_from<2, SB, true>(pp, st, acc); break;
                case 6: hop_from<3, SF, false>(pp, st, acc); break;
                case 7: hop_from<3, SB, true>(pp, st, acc); break;
                default:
#pragma unroll
                    for (int q = 0; q < RB; q++) pp.spinor(st, q, c0[q]);
            }
        }
        cpa_wait<0>();
        }
        const F2 d2 = f2(a.diag, a.diag), mh = f2(a.hcoef, a.hcoef);
#pragma unroll
        for (int q = 0; q < RB; q++) {
            const unsigned rq = r0 + q * KB;
            const unsigned o = s * a.k + rq;
            Sp out;
#pragma unroll
            for (int e = 0; e < 12; e++) out.c[e] = fma2(mh, acc[q].c[e], mul2(d2, c0[q].c[e]));
            if (EPI == E_PLAIN || EPI == E_NORM) {
                Store32<S>::store(a.out, a.out_s, a.P, o, out);
                if (EPI == E_NORM) nrm[q] += norm2f(out);
            } else {  // E_CG: r -= alpha t
                const CGScalars &st = a.st[rq];
                const float al = st.active ? (float)st.alpha : 0.f;
                const F2 mal2 = f2(-al, -al);
                Sp rr;
                Store32<S>::load(a.r, a.r_s, a.P, o, rr);
#pragma unroll
                for (int e = 0; e < 12; e++) rr.c[e] = fma2(mal2, out.c[e], rr.c[e]);
                Store32<S>::store(a.r, a.r_s, a.P, o, rr);
                nrm[q] += norm2f(rr);
                if (a.save_t) Store32<float>::store(a.tsave, nullptr, a.V, s, out);
            }
        }
    }
    if (EPI == E_PLAIN) return;
    // per-RHS block sums: thread group grp = threadIdx % KB holds RHS grp + q * KB
    double *myp = a.partials + (size_t)blockIdx.x * a.k;
#pragma unroll
    for (int q = 0; q < RB; q++) {
        const double bs = block_reduce_rhs((double)nrm[q], (int)KB, smem);
        if (threadIdx.x < KB) myp[threadIdx.x + q * KB] = bs;
    }
    const int k = (int)a.k;
    CGScalars *const sts = a.st;
    double *const h_alpha = a.h_alpha, *const h_beta = a.h_beta, *const h_rho = a.h_rho;
    const int iter = a.iter + (a.jbase ? *a.jbase : 0);
    grid_finish_rhs(k, a.partials, a.counter, smem, [=](int r, double tot) {
        CGScalars &st = sts[r];
        const long hi = (long)iter * k + r;
        if (EPI == E_NORM) {
            if (st.active) {
                st.pAp = tot;
                if (!(tot > 0.0) || !isfinite(tot)) {
                    st.breakdown = 1;
                    st.active = 0;
                    st.alpha = 0.0;
                } else {
                    st.alpha = st.rho / tot;
                }
                h_alpha[hi] = st.alpha;
                st.x_pending = st.active;
            } else {
                st.alpha = 0.0;
                st.x_pending = 0;
            }
        } else {
            if (st.active) {
                if (!isfinite(tot)) {
                    st.breakdown = 1;
                    st.active = 0;
                    return;
                }
                st.iters = iter;
                st.nit++;
                st.rho_prev = st.rho;
                st.rho = tot;
                st.beta = tot / st.rho_prev;
                h_rho[hi] = tot;
                h_beta[hi + k] = st.beta;
                if (tot <= st.target) st.active = 0;
            }
        }
    });
}


// launch of one direct-load variant (RB RHS per thread, MINB blocks per SM)
template <int RB, int MINB, int MODE, typename S, int GF, bool DAG, int EPI>
cudaError_t d32_direct_go(const K32 &a, int cap, cudaStream_t s) {
    auto kern = k_dslash32<S, GF, DAG, EPI, RB, MODE, MINB>;
    kern<<<d32_grid((const void *)kern, (long)a.V * a.k / RB, cap, 0), TPB, 0, s>>>(a);
    return cudaGetLastError();
}

template <int RB, int MINB, int MODE, typename S, int GF>
cudaError_t d32_direct_fmt(bool dag, int epi, const K32 &a, int cap, cudaStream_t s) {
    if (epi == E_PLAIN)
        return dag ? d32_direct_go<RB, MINB, MODE, S, GF, true, E_PLAIN>(a, cap, s)
                   : d32_direct_go<RB, MINB, MODE, S, GF, false, E_PLAIN>(a, cap, s);
    if (epi == E_NORM)
        return dag ? d32_direct_go<RB, MINB, MODE, S, GF, true, E_NORM>(a, cap, s)
                   : d32_direct_go<RB, MINB, MODE, S, GF, false, E_NORM>(a, cap, s);
    return dag ? d32_direct_go<RB, MINB, MODE, S, GF, true, E_CG>(a, cap, s)
               : d32_direct_go<RB, MINB, MODE, S, GF, false, E_CG>(a, cap, s);
}

template <int RB, int MINB, int MODE>
cudaError_t d32_direct(int prec, int gf, bool dag, int epi, const K32 &a, int cap, cudaStream_t s) {
    if (prec == 32 && gf == GF_F32_12) return d32_direct_fmt<RB, MINB, MODE, float, GF_F32_12>(dag, epi, a, cap, s);
    if (prec == 32 && gf == GF_F32_18) return d32_direct_fmt<RB, MINB, MODE, float, GF_F32_18>(dag, epi, a, cap, s);
    if (prec == 16 && gf == GF_F32_12) return d32_direct_fmt<RB, MINB, MODE, __half, GF_F32_12>(dag, epi, a, cap, s);
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace eig
