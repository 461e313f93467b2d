// Internal header: the pipelined-pair form of the FP32-arithmetic Wilson stencil
// (variants 16-19 of dslash32.cu), for batches of k >= 2 RHS.
//
// Same operator, spin projection and epilogues as k_dslash32 (dslash32.cuh); what
// differs is how the data reaches the registers:
//
//  * each thread takes two ADJACENT right-hand sides r0, r0 + 1 of one site.  In the
//    RHS-inner layout [chunk][site][rhs] their chunk c lies in 32 contiguous bytes, so
//    one 256-bit load (ld.global.v8.f32) brings both, and the 8 threads of a site
//    (k = 16) still cover 256 contiguous bytes per chunk;
//  * the raw data of hop h + 1 (the neighbour's spinor pair and the link) is loaded into
//    a second register set before hop h is computed, and the centre spinors (and, in the
//    CG epilogue, the residual) during the last hop, so that two hops of loads are in
//    flight per thread at all times without shared memory.
//
// At k = 16 the stencil's time per site and RHS is set by the latency of the neighbour
// loads (most hit in L2) at a dozen warps per SM, not by HBM; keeping the next hop's
// loads in flight while the current one is computed attacks exactly that.
#pragma once
#include "dslash32.cuh"

namespace eig {
namespace {

// 256-bit loads and stores (sm_100 and later).  .nc for fields that no thread writes
// during the launch; the residual r is read and written by the same thread, so it takes
// the coherent path.
__device__ __forceinline__ void ld256_nc(const void *p, float4 &a, float4 &b) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}
__device__ __forceinline__ void ld256(const void *p, float4 &a, float4 &b) {
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void st256(void *p, const float4 &a, const float4 &b) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(a.x), "f"(a.y), "f"(a.z),
                 "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}

// raw chunks of one spinor for the two RHS of a pair (a: r0, b: r0 + 1)
template <typename S>
struct PairRaw;
template <>
struct PairRaw<float> {
    static constexpr int NC = 6;  // float4 chunks of 2 complex
    float4 a[NC], b[NC];
    float2 sc;  // unused
};
template <>
struct PairRaw<__half> {
    static constexpr int NC = 3;  // chunks of 8 halves (4 complex)
    float4 a[NC], b[NC];
    float2 sc;  // one scale per RHS
};

template <typename S, bool NC_PATH>
__device__ __forceinline__ void load_pair(const float4 *base, const float *scale, unsigned P, unsigned o,
                                          PairRaw<S> &d) {
#pragma unroll
    for (int c = 0; c < PairRaw<S>::NC; c++) {
        if (NC_PATH) ld256_nc(base + c * P + o, d.a[c], d.b[c]);
        else ld256(base + c * P + o, d.a[c], d.b[c]);
    }
    if (sizeof(S) == 2) d.sc = NC_PATH ? __ldg(reinterpret_cast<const float2 *>(scale + o))
                                       : *reinterpret_cast<const float2 *>(scale + o);
}

template <typename S>
__device__ __forceinline__ void unpack_pair(const PairRaw<S> &d, int q, Sp &v) {
    if (sizeof(S) == 4) {
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const float4 x = q ? d.b[c] : d.a[c];
            v.c[2 * c] = f2(x.x, x.y);
            v.c[2 * c + 1] = f2(x.z, x.w);
        }
    } else {
        const float sc = q ? d.sc.y : d.sc.x;
        const F2 s2 = f2(sc, sc);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float4 x4 = q ? d.b[c] : d.a[c];
            const uint4 w4 = *reinterpret_cast<const uint4 *>(&x4);
            const uint32_t w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int e = 0; e < 4; e++) v.c[4 * c + e] = mul2(__half22float2(*reinterpret_cast<const __half2 *>(&w[e])), s2);
        }
    }
}

// stores the spinors of both RHS of a pair (FP16: per-RHS scale, as Store32<__half>)
template <typename S>
__device__ __forceinline__ void store_pair(float4 *base, float *scale, unsigned P, unsigned o, const Sp *v) {
    if (sizeof(S) == 4) {
#pragma unroll
        for (int c = 0; c < 6; c++)
            st256(base + c * P + o, make_float4(v[0].c[2 * c].x, v[0].c[2 * c].y, v[0].c[2 * c + 1].x, v[0].c[2 * c + 1].y),
                  make_float4(v[1].c[2 * c].x, v[1].c[2 * c].y, v[1].c[2 * c + 1].x, v[1].c[2 * c + 1].y));
    } else {
        float4 ch[2][3];
        float sc[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            float mx = 0.f;
#pragma unroll
            for (int e = 0; e < 12; e++) mx = fmaxf(mx, fmaxf(fabsf(v[q].c[e].x), fabsf(v[q].c[e].y)));
            const float inv = mx > 0.f ? 1.0f / mx : 0.f;
            sc[q] = mx;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const F2 t = mul2(v[q].c[4 * c + e], f2(inv, inv));
                    __half2 h = __float22half2_rn(t);
                    w[e] = *reinterpret_cast<uint32_t *>(&h);
                }
                const uint4 u4 = make_uint4(w[0], w[1], w[2], w[3]);
                ch[q][c] = *reinterpret_cast<const float4 *>(&u4);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; c++) st256(base + c * P + o, ch[0][c], ch[1][c]);
        *reinterpret_cast<float2 *>(scale + o) = make_float2(sc[0], sc[1]);
    }
}

template <int GF>
struct LinkRaw;
template <>
struct LinkRaw<GF_F32_12> {
    float4 v[3];
    __device__ __forceinline__ void load(const void *g, unsigned V, int mu, unsigned s) {
        const float4 *p = static_cast<const float4 *>(g) + (unsigned)mu * 3u * V;
#pragma unroll
        for (int i = 0; i < 3; i++) v[i] = __ldg(p + i * V + s);
    }
    __device__ __forceinline__ void unpack(Lk &U) const {
        U.u[0] = f2(v[0].x, v[0].y);
        U.u[1] = f2(v[0].z, v[0].w);
        U.u[2] = f2(v[1].x, v[1].y);
        U.u[3] = f2(v[1].z, v[1].w);
        U.u[4] = f2(v[2].x, v[2].y);
        U.u[5] = f2(v[2].z, v[2].w);
        rebuild_row2(U);
    }
};
template <>
struct LinkRaw<GF_F32_18> {
    float2 v[9];
    __device__ __forceinline__ void load(const void *g, unsigned V, int mu, unsigned s) {
        const float2 *p = static_cast<const float2 *>(g) + (unsigned)mu * 9u * V;
#pragma unroll
        for (int e = 0; e < 9; e++) v[e] = __ldg(p + e * V + s);
    }
    __device__ __forceinline__ void unpack(Lk &U) const {
#pragma unroll
        for (int e = 0; e < 9; e++) U.u[e] = v[e];
    }
};

template <int MU, int SG, bool DAGGER, typename S, int GF>
__device__ __forceinline__ void hop_pair(const PairRaw<S> &d, const LinkRaw<GF> &l, Sp *acc) {
    Lk U;
    l.unpack(U);
#pragma unroll
    for (int q = 0; q < 2; q++) {
        Sp nb;
        Hf h, uh;
        unpack_pair<S>(d, q, nb);
        project<MU, SG>(nb, h);
        mul_link<DAGGER>(U, h, uh);
        accumulate<MU, SG>(acc[q], uh);
    }
}

// PF: also ask L1 for the spinor pair and link of hop h + 2 while hop h is computed (no
// registers held for it), so that the register load of hop h + 1 finds them closer
template <typename S, int GF>
__device__ __forceinline__ void prefetch_pair(const K32 &a, unsigned o, int mu, unsigned ls) {
#pragma unroll
    for (int c = 0; c < PairRaw<S>::NC; c++) pf_l1(a.in + c * a.P + o);
    if (GF == GF_F32_12) {
        const float4 *g = static_cast<const float4 *>(a.g) + (unsigned)mu * 3u * a.Vg;
#pragma unroll
        for (int i = 0; i < 3; i++) pf_l1(g + i * a.Vg + ls);
    } else {
        const float2 *g = static_cast<const float2 *>(a.g) + (unsigned)mu * 9u * a.Vg;
#pragma unroll
        for (int e = 0; e < 9; e += 2) pf_l1(g + e * a.Vg + ls);
    }
}

template <typename S, int GF, bool DAG, int EPI, int MINB, bool PF = false>
__global__ void __launch_bounds__(TPB, MINB) k_dslash32pp(const K32 a) {
    __shared__ double smem[(TPB / 32) * MAX_RHS];
    if (EPI != E_PLAIN) {
        bool any = false;
        for (unsigned q = 0; q < a.k; q++) any = any || a.st[q].active;
        if (!any) return;
    }
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    const unsigned KB = a.k >> 1;  // RHS pairs per site (k a power of two >= 2)
    const unsigned kb_shift = __ffs(KB) - 1;
    const unsigned total = a.V * KB;
    const unsigned s1 = a.L0, s2 = a.L0 * a.L1, s3 = s2 * a.L2;
    float nrm[2] = {0.f, 0.f};
    for (unsigned g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        unsigned s = g >> kb_shift;  // output field index (traversal index when tiled)
        const unsigned r0 = (g & (KB - 1)) << 1;
        unsigned sl, x, y, z, t;
        if (a.eo >= 0) {
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
        unsigned nbr[8], lks[8];
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
        Sp acc[2];
#pragma unroll
        for (int q = 0; q < 2; q++)
#pragma unroll
            for (int e = 0; e < 12; e++) acc[q].c[e] = f2(0.f, 0.f);
        // two register sets: hop h is computed from one while hop h + 1 loads into the other
        PairRaw<S> sp[2];
        LinkRaw<GF> lk[2];
        PairRaw<S> rr_raw;  // CG epilogue: the residual pair, loaded during the last hop
        load_pair<S, true>(a.in, a.in_s, a.P, nbr[0] * a.k + r0, sp[0]);
        lk[0].load(a.g, a.Vg, 0, lks[0]);
        bool have_cen = true;
#pragma unroll
        for (int h = 0; h < 8; h++) {
            const int cur = h & 1, nx = cur ^ 1;
            if (PF && h + 2 < 8) prefetch_pair<S, GF>(a, nbr[h + 2] * a.k + r0, (h + 2) >> 1, lks[h + 2]);
            if (h < 7) {
                load_pair<S, true>(a.in, a.in_s, a.P, nbr[h + 1] * a.k + r0, sp[nx]);
                lk[nx].load(a.g, a.Vg, (h + 1) >> 1, lks[h + 1]);
            } else {
                // centre term: from `in` (full lattice), from `cen` (odd-even), or none
                if (a.eo < 0) load_pair<S, true>(a.in, a.in_s, a.P, s * a.k + r0, sp[nx]);
                else if (a.cen) load_pair<S, true>(a.cen, a.cen_s, a.P, s * a.k + r0, sp[nx]);
                else have_cen = false;
                if (EPI == E_CG) load_pair<S, false>(a.r, a.r_s, a.P, s * a.k + r0, rr_raw);
            }
            switch (h) {
                case 0: hop_pair<0, SF, false>(sp[cur], lk[cur], acc); break;
                case 1: hop_pair<0, SB, true>(sp[cur], lk[cur], acc); break;
                case 2: hop_pair<1, SF, false>(sp[cur], lk[cur], acc); break;
                case 3: hop_pair<1, SB, true>(sp[cur], lk[cur], acc); break;
                case 4: hop_pair<2, SF, false>(sp[cur], lk[cur], acc); break;
                case 5: hop_pair<2, SB, true>(sp[cur], lk[cur], acc); break;
                case 6: hop_pair<3, SF, false>(sp[cur], lk[cur], acc); break;
                default: hop_pair<3, SB, true>(sp[cur], lk[cur], acc); break;
            }
        }
        const F2 d2 = f2(a.diag, a.diag), mh = f2(a.hcoef, a.hcoef);
        const unsigned o = s * a.k + r0;
        Sp out[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            Sp c0;
            if (have_cen) unpack_pair<S>(sp[0], q, c0);
            else
#pragma unroll
                for (int e = 0; e < 12; e++) c0.c[e] = f2(0.f, 0.f);
#pragma unroll
            for (int e = 0; e < 12; e++) out[q].c[e] = fma2(mh, acc[q].c[e], mul2(d2, c0.c[e]));
        }
        if (EPI == E_PLAIN || EPI == E_NORM) {
            store_pair<S>(a.out, a.out_s, a.P, o, out);
            if (EPI == E_NORM) {
                nrm[0] += norm2f(out[0]);
                nrm[1] += norm2f(out[1]);
            }
        } else {  // E_CG: r -= alpha t
            Sp rr[2];
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const CGScalars &st = a.st[r0 + q];
                const float al = st.active ? (float)st.alpha : 0.f;
                const F2 mal2 = f2(-al, -al);
                unpack_pair<S>(rr_raw, q, rr[q]);
#pragma unroll
                for (int e = 0; e < 12; e++) rr[q].c[e] = fma2(mal2, out[q].c[e], rr[q].c[e]);
                nrm[q] += norm2f(rr[q]);
            }
            store_pair<S>(a.r, a.r_s, a.P, o, rr);
        }
    }
    if (EPI == E_PLAIN) return;
    // per-RHS block sums: thread group grp = threadIdx % KB holds RHS 2 grp and 2 grp + 1
    double *myp = a.partials + (size_t)blockIdx.x * a.k;
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const double bs = block_reduce_rhs((double)nrm[q], (int)KB, smem);
        if (threadIdx.x < KB) myp[2 * threadIdx.x + q] = bs;
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

template <int MINB, bool PF, typename S, int GF, bool DAG, int EPI>
cudaError_t d32pp_go(const K32 &a, int cap, cudaStream_t s) {
    auto kern = k_dslash32pp<S, GF, DAG, EPI, MINB, PF>;
    kern<<<d32_grid((const void *)kern, (long)a.V * a.k / 2, cap, 0), TPB, 0, s>>>(a);
    return cudaGetLastError();
}

template <int MINB, bool PF, typename S, int GF>
cudaError_t d32pp_fmt(bool dag, int epi, const K32 &a, int cap, cudaStream_t s) {
    if (epi == E_PLAIN)
        return dag ? d32pp_go<MINB, PF, S, GF, true, E_PLAIN>(a, cap, s)
                   : d32pp_go<MINB, PF, S, GF, false, E_PLAIN>(a, cap, s);
    if (epi == E_NORM)
        return dag ? d32pp_go<MINB, PF, S, GF, true, E_NORM>(a, cap, s)
                   : d32pp_go<MINB, PF, S, GF, false, E_NORM>(a, cap, s);
    return dag ? d32pp_go<MINB, PF, S, GF, true, E_CG>(a, cap, s) : d32pp_go<MINB, PF, S, GF, false, E_CG>(a, cap, s);
}

}  // namespace
}  // namespace eig
