// Wilson-Dirac dslash kernels: the matrix-vector product of CG on A = M^H M
// (Sec. 1; Fig. 1 step 11), with the CG vector updates and reductions fused into
// the epilogue (Fig. 1 steps 12-14).
//
//   (M psi)(x) = (4 + m_q) psi(x)
//       - 1/2 sum_mu [ (I - g_mu) U_mu(x) psi(x+mu) + (I + g_mu) U_mu(x-mu)^H psi(x-mu) ]
//   M^H = gamma5 M gamma5: the same stencil with the two projectors swapped.
//
// In the chiral basis g_mu = [[0, B_mu], [B_mu^H, 0]] with B_mu unitary, so for
// psi = (a, b) (upper and lower spin pairs) and s = +-1:
//   (I + s g_mu) psi = (h, s B_mu^H h),   h = a + s B_mu b.
// Each hop therefore projects the neighbour to a half spinor h (2 spins x 3
// colours), multiplies it by the link (two SU(3) mat-vecs instead of four) and
// rebuilds the lower spins from h.  B_1 = [[0,i],[i,0]], B_2 = [[0,-1],[1,0]],
// B_3 = diag(i,-i), B_4 = I.
//
// Threads map to (site, rhs) with rhs fastest; the RHS-inner field layout makes
// every chunk load coalesced and lets the k RHS of one site share each link load
// through L1.  Grids are persistent (a multiple of the SM count), with
// grid-stride loops.
#include <string>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "kernels.cuh"
#include "prof.h"

namespace eig {

enum Epi { EPI_PLAIN = 0, EPI_NORM = 1, EPI_CG = 2, EPI_RESID = 3 };

struct KArgs {
    FieldView in, out, p, x, r, tsave, b;
    FieldView cen;     // centre-term input (odd-even form), else in
    GaugeView g;
    int L0, L1, L2, L3;
    long V;            // output sites (V / 2 in the odd-even form)
    int k;
    double diag;
    double hcoef;      // coefficient of the hop sum (-1/2 for M)
    int eo;            // output parity (odd-even form) or -1
    int store_out, save_t, set_rho;
    CGScalars *st;
    double *h_alpha, *h_beta, *h_rho;
    int iter;
    const int *jbase;  // device iteration base added to iter (null: none)
    double *partials;
    unsigned *counter;
};

template <int MU, int SG, typename C>
__device__ __forceinline__ void project(const Spinor<C> &p, Half<C> &h) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const Cx<C> a0 = p.s[0][c], a1 = p.s[1][c], b0 = p.s[2][c], b1 = p.s[3][c];
        Cx<C> q0, q1;  // B_mu b
        if (MU == 0) {
            q0 = times_i(b1);
            q1 = times_i(b0);
        } else if (MU == 1) {
            q0 = cmk<C>(-b1.re, -b1.im);
            q1 = b0;
        } else if (MU == 2) {
            q0 = times_i(b0);
            q1 = cmk<C>(b1.im, -b1.re);
        } else {
            q0 = b0;
            q1 = b1;
        }
        if (SG > 0) {
            h.h[0][c] = a0 + q0;
            h.h[1][c] = a1 + q1;
        } else {
            h.h[0][c] = a0 - q0;
            h.h[1][c] = a1 - q1;
        }
    }
}

template <int MU, int SG, typename C>
__device__ __forceinline__ void accumulate(Spinor<C> &acc, const Half<C> &h) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const Cx<C> h0 = h.h[0][c], h1 = h.h[1][c];
        Cx<C> g0, g1;  // B_mu^H h
        if (MU == 0) {
            g0 = cmk<C>(h1.im, -h1.re);
            g1 = cmk<C>(h0.im, -h0.re);
        } else if (MU == 1) {
            g0 = h1;
            g1 = cmk<C>(-h0.re, -h0.im);
        } else if (MU == 2) {
            g0 = cmk<C>(h0.im, -h0.re);
            g1 = times_i(h1);
        } else {
            g0 = h0;
            g1 = h1;
        }
        acc.s[0][c] = acc.s[0][c] + h0;
        acc.s[1][c] = acc.s[1][c] + h1;
        if (SG > 0) {
            acc.s[2][c] = acc.s[2][c] + g0;
            acc.s[3][c] = acc.s[3][c] + g1;
        } else {
            acc.s[2][c] = acc.s[2][c] - g0;
            acc.s[3][c] = acc.s[3][c] - g1;
        }
    }
}

template <typename C>
__device__ __forceinline__ void mul_link(const Link<C> &U, const Half<C> &h, Half<C> &o) {
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            Cx<C> v = cmul(U.u[a][0], h.h[s][0]);
            v = cfma(U.u[a][1], h.h[s][1], v);
            v = cfma(U.u[a][2], h.h[s][2], v);
            o.h[s][a] = v;
        }
}

template <typename C>
__device__ __forceinline__ void mul_link_dag(const Link<C> &U, const Half<C> &h, Half<C> &o) {
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            Cx<C> v = cmul(conjg(U.u[0][a]), h.h[s][0]);
            v = cfma_conj(U.u[1][a], h.h[s][1], v);
            v = cfma_conj(U.u[2][a], h.h[s][2], v);
            o.h[s][a] = v;
        }
}

// hop of direction MU: spinors at field indices sf (x + mu) and sb (x - mu), links at
// lattice sites s (U_mu(x)) and lb (U_mu(x - mu))
template <int MU, typename S, int GF, bool DAG>
__device__ __forceinline__ void hop_dir(const KArgs &a, long s, long lb, long sf, long sb, int r,
                                        Spinor<typename SpinorStore<S>::C> &acc) {
    using C = typename SpinorStore<S>::C;
    constexpr int SF = DAG ? +1 : -1;  // forward projector  I + SF g_mu
    constexpr int SB = -SF;            // backward projector I + SB g_mu
    Spinor<C> nb;
    Half<C> h, uh;
    Link<C> U;
    SpinorStore<S>::load(a.in, sf, r, nb);
    project<MU, SF>(nb, h);
    GaugeLoad<GF>::load(a.g, MU, s, U);
    mul_link(U, h, uh);
    accumulate<MU, SF>(acc, uh);
    SpinorStore<S>::load(a.in, sb, r, nb);
    project<MU, SB>(nb, h);
    GaugeLoad<GF>::load(a.g, MU, lb, U);
    mul_link_dag(U, h, uh);
    accumulate<MU, SB>(acc, uh);
}

// out = diag * centre + hcoef * (hop sum) at output site s (a half-lattice index in the
// odd-even form: the site of parity a.eo at s, with x = 2 (s mod Lx/2) + parity bit)
template <typename S, int GF, bool DAG>
__device__ __forceinline__ void wilson_site(const KArgs &a, long s, int r, Spinor<typename SpinorStore<S>::C> &out) {
    using C = typename SpinorStore<S>::C;
    const long s1 = a.L0, s2 = (long)a.L0 * a.L1, s3 = s2 * a.L2;
    int x, y, z, t;
    long sl = s;  // lattice site
    if (a.eo >= 0) {
        const long lh = a.L0 / 2, rest = s / lh;
        y = (int)(rest % a.L1);
        z = (int)((rest / a.L1) % a.L2);
        t = (int)(rest / ((long)a.L1 * a.L2));
        x = (int)(2 * (s % lh) + ((a.eo + y + z + t) & 1));
        sl = x + a.L0 * rest;
    } else {
        x = (int)(s % a.L0);
        y = (int)((s / s1) % a.L1);
        z = (int)((s / s2) % a.L2);
        t = (int)(s / s3);
    }
    const long nf[4] = {x == a.L0 - 1 ? sl - (a.L0 - 1) : sl + 1, y == a.L1 - 1 ? sl - (a.L1 - 1) * s1 : sl + s1,
                        z == a.L2 - 1 ? sl - (a.L2 - 1) * s2 : sl + s2, t == a.L3 - 1 ? sl - (a.L3 - 1) * s3 : sl + s3};
    const long nb[4] = {x == 0 ? sl + (a.L0 - 1) : sl - 1, y == 0 ? sl + (a.L1 - 1) * s1 : sl - s1,
                        z == 0 ? sl + (a.L2 - 1) * s2 : sl - s2, t == 0 ? sl + (a.L3 - 1) * s3 : sl - s3};
    const int sh = a.eo >= 0 ? 1 : 0;  // neighbours are of the other parity: field index = site / 2
    Spinor<C> acc;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) acc.s[i][j] = cmk<C>(0, 0);
    hop_dir<0, S, GF, DAG>(a, sl, nb[0], nf[0] >> sh, nb[0] >> sh, r, acc);
    hop_dir<1, S, GF, DAG>(a, sl, nb[1], nf[1] >> sh, nb[1] >> sh, r, acc);
    hop_dir<2, S, GF, DAG>(a, sl, nb[2], nf[2] >> sh, nb[2] >> sh, r, acc);
    hop_dir<3, S, GF, DAG>(a, sl, nb[3], nf[3] >> sh, nb[3] >> sh, r, acc);
    Spinor<C> c0;
    if (a.eo < 0) SpinorStore<S>::load(a.in, s, r, c0);
    else if (a.diag != 0.0) SpinorStore<S>::load(a.cen, s, r, c0);
    else
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) c0.s[i][j] = cmk<C>(0, 0);  // hops only
    const C d = (C)a.diag;
    const C h = (C)a.hcoef;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) out.s[i][j] = cmk<C>(d * c0.s[i][j].re + h * acc.s[i][j].re,
                                                         d * c0.s[i][j].im + h * acc.s[i][j].im);
}

template <typename C>
__device__ __forceinline__ double site_norm2(const Spinor<C> &v) {
    C n = 0;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) n += v.s[i][j].re * v.s[i][j].re + v.s[i][j].im * v.s[i][j].im;
    return (double)n;
}

// x storage / window storage follow the spinor precision: FP64 for FP64, else FP32.
template <typename S>
struct Wide {
    using T = float;
};
template <>
struct Wide<double> {
    using T = double;
};

template <typename S, int GF, bool DAG, int EPI>
__global__ void __launch_bounds__(128) k_dslash(const KArgs a) {
    using C = typename SpinorStore<S>::C;
    using W = typename Wide<S>::T;
    __shared__ double smem[(128 / 32) * MAX_RHS];
    if (EPI == EPI_NORM || EPI == EPI_CG) {  // nothing to do once every RHS has stopped
        bool any = false;
        for (int q = 0; q < a.k; q++) any = any || a.st[q].active;
        if (!any) return;
    }
    const long total = a.V * a.k;
    double nrm = 0.0;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long s = g / a.k;
        const int r = (int)(g - s * a.k);
        Spinor<C> out;
        wilson_site<S, GF, DAG>(a, s, r, out);
        if (EPI == EPI_PLAIN || EPI == EPI_NORM) {
            SpinorStore<S>::store(a.out, s, r, out);
            if (EPI == EPI_NORM) nrm += site_norm2(out);
        } else if (EPI == EPI_CG) {  // r -= alpha t
            const CGScalars &st = a.st[r];
            const C al = st.active ? (C)st.alpha : (C)0;
            Spinor<C> rr;
            SpinorStore<S>::load(a.r, s, r, rr);
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    rr.s[i][j].re -= al * out.s[i][j].re;
                    rr.s[i][j].im -= al * out.s[i][j].im;
                }
            SpinorStore<S>::store(a.r, s, r, rr);
            nrm += site_norm2(rr);
            if (a.save_t) {
                Spinor<W> tw;
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++) tw.s[i][j] = cmk<W>((W)out.s[i][j].re, (W)out.s[i][j].im);
                SpinorStore<W>::store(a.tsave, s, r, tw);
            }
        } else {  // EPI_RESID: r = b - out (FP64 only)
            Spinor<C> bb;
            SpinorStore<S>::load(a.b, s, r, bb);
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) out.s[i][j] = bb.s[i][j] - out.s[i][j];
            SpinorStore<S>::store(a.r, s, r, out);
            nrm += site_norm2(out);
        }
    }
    if (EPI == EPI_PLAIN) return;
    const double bs = block_reduce_rhs(nrm, a.k, smem);
    const int k = a.k;
    CGScalars *const sts = a.st;
    double *const h_alpha = a.h_alpha, *const h_beta = a.h_beta, *const h_rho = a.h_rho;
    const int iter = a.iter + (a.jbase ? *a.jbase : 0), set_rho = a.set_rho;
    grid_reduce_rhs(bs, k, a.partials, a.counter, smem, [=](int r, double tot) {
        CGScalars &st = sts[r];
        const long hi = (long)iter * k + r;
        if (EPI == EPI_NORM) {
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
        } else if (EPI == EPI_CG) {
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
        } else {  // EPI_RESID
            st.aux = tot;
            if (set_rho) {
                st.rho = tot;
                st.beta = tot / st.rho_prev;
                h_rho[hi] = tot;
                h_beta[hi + k] = st.beta;
            }
        }
    });
}

// ------------------------------------------------------------------------------------
// launch plumbing
// ------------------------------------------------------------------------------------
static std::mutex g_occ_mu;
static std::unordered_map<const void *, int> g_occ;
static int g_sms = 0;

int device_sm_count() {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

template <typename K>
static int persistent_grid(K kern, int block, long work, int cap) {
    int sms = device_sm_count();
    int per = 0;
    {
        std::lock_guard<std::mutex> lk(g_occ_mu);
        auto it = g_occ.find((const void *)kern);
        if (it != g_occ.end()) {
            per = it->second;
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, block, 0);
            if (per < 1) per = 1;
            g_occ[(const void *)kern] = per;
        }
    }
    long need = (work + block - 1) / block;
    long grid = (long)sms * per;
    if (grid > need) grid = need;
    if (cap > 0 && grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    return (int)grid;
}

static KArgs base_args(const DslashCall &c) {
    KArgs a;
    memset(&a, 0, sizeof(a));
    a.in = c.in.v;
    a.out = c.out.v;
    a.g = c.gauge;
    a.L0 = c.L[0];
    a.L1 = c.L[1];
    a.L2 = c.L[2];
    a.L3 = c.L[3];
    a.eo = c.eo_parity;
    a.V = c.eo_parity >= 0 ? c.V / 2 : c.V;
    a.k = c.k;
    a.diag = c.diag;
    a.hcoef = c.hcoef;
    if (c.eo_parity >= 0) a.cen = c.cen.v;
    return a;
}

static double site_bytes_gauge(int gf) {
    switch (gf) {
        case GF_F64_18: return 4.0 * 144;
        case GF_F32_12: return 4.0 * 48;
        case GF_F32_18: return 4.0 * 72;
        default: return 4.0 * 24;
    }
}

// Algorithmic bytes of one launch: every link, input and output touched once.
template <int EPI>
static double dslash_bytes(const DslashCall &c, const KArgs &a) {
    const double sp = c.in.prec == P64 ? 192 : (c.in.prec == P32 ? 96 : 52);
    const double w = c.in.prec == P64 ? 192 : 96;
    double per_rhs = 2 * sp;                                                 // in + out
    if (EPI == EPI_CG) per_rhs = sp + 2 * sp + (a.save_t ? w : 0);           // u, r rw, t
    if (EPI == EPI_RESID) per_rhs = 3 * sp;                                  // u, b, r
    if (c.eo_parity >= 0 && c.diag != 0.0) per_rhs += sp;                    // centre field
    // every link once (the odd-even form touches all links for half the sites)
    return (double)c.V * site_bytes_gauge(c.gformat) + (double)a.V * c.k * per_rhs;
}

// Profile name: epilogue, storage precision and, for batched launches, the batch width
// (the single-RHS and batched stencils have different rooflines).
static std::string dslash_name(int epi, Prec p, int k) {
    static const char *names[4][3] = {{"dslash_f64", "dslash_f32", "dslash_f16"},
                                      {"dslash_norm_f64", "dslash_norm_f32", "dslash_norm_f16"},
                                      {"dslash_cg_f64", "dslash_cg_f32", "dslash_cg_f16"},
                                      {"dslash_resid_f64", "dslash_resid_f32", "dslash_resid_f16"}};
    std::string n = names[epi][p];
    if (k > 1) n += "_k" + std::to_string(k);
    return n;
}

template <int EPI>
static cudaError_t dispatch(const DslashCall &c, KArgs &a, int cap, cudaStream_t s) {
    const long work = a.V * c.k;
    const int block = 128;
    ProfScope prof(dslash_name(EPI, c.in.prec, c.k).c_str(), dslash_bytes<EPI>(c, a), s);
#define EIG_LAUNCH(S, GF)                                                                   \
    do {                                                                                    \
        if (c.dagger) {                                                                     \
            auto kern = k_dslash<S, GF, true, EPI>;                                         \
            k_dslash<S, GF, true, EPI><<<persistent_grid(kern, block, work, cap), block, 0, s>>>(a); \
        } else {                                                                            \
            auto kern = k_dslash<S, GF, false, EPI>;                                        \
            k_dslash<S, GF, false, EPI><<<persistent_grid(kern, block, work, cap), block, 0, s>>>(a); \
        }                                                                                   \
        return cudaGetLastError();                                                          \
    } while (0)
    switch (c.in.prec) {
        case P64:
            if (c.gformat == GF_F64_18) EIG_LAUNCH(double, GF_F64_18);
            break;
        case P32:
            if (EPI != EPI_RESID) {
                if (c.gformat == GF_F32_12) EIG_LAUNCH(float, GF_F32_12);
                if (c.gformat == GF_F32_18) EIG_LAUNCH(float, GF_F32_18);
            }
            break;
        case P16:
            if (EPI != EPI_RESID && c.gformat == GF_F32_12) EIG_LAUNCH(__half, GF_F32_12);
            break;
    }
#undef EIG_LAUNCH
    return cudaErrorInvalidValue;
}

cudaError_t launch_dslash(const DslashCall &c, cudaStream_t s) {
    KArgs a = base_args(c);
    if (c.in.prec != P64) {
        ProfScope prof(dslash_name(EPI_PLAIN, c.in.prec, c.k).c_str(), dslash_bytes<EPI_PLAIN>(c, a), s);
        return launch_dslash32(c, s);
    }
    return dispatch<EPI_PLAIN>(c, a, 0, s);
}

cudaError_t launch_dslash_norm(const DslashCall &c, CGScalars *st, History h, int iter, RedScratch red,
                               cudaStream_t s) {
    KArgs a = base_args(c);
    a.st = st;
    a.h_alpha = h.alpha;
    a.h_beta = h.beta;
    a.h_rho = h.rho;
    a.iter = iter;
    a.jbase = h.jbase;
    a.partials = red.partials;
    a.counter = red.counter;
    if (c.in.prec != P64) {
        ProfScope prof(dslash_name(EPI_NORM, c.in.prec, c.k).c_str(), dslash_bytes<EPI_NORM>(c, a), s);
        return launch_dslash32_norm(c, st, h, iter, red, s);
    }
    return dispatch<EPI_NORM>(c, a, red.max_blocks, s);
}

cudaError_t launch_dslash_cg(const DslashCall &c, Field r, Field t_save, CGScalars *st, History h, int iter,
                             RedScratch red, cudaStream_t s) {
    KArgs a = base_args(c);
    a.r = r.v;
    a.tsave = t_save.v;
    a.save_t = t_save.v.data != nullptr;
    a.st = st;
    a.h_alpha = h.alpha;
    a.h_beta = h.beta;
    a.h_rho = h.rho;
    a.iter = iter;
    a.jbase = h.jbase;
    a.partials = red.partials;
    a.counter = red.counter;
    if (c.in.prec != P64) {
        ProfScope prof(dslash_name(EPI_CG, c.in.prec, c.k).c_str(), dslash_bytes<EPI_CG>(c, a), s);
        return launch_dslash32_cg(c, r, t_save, st, h, iter, red, s);
    }
    return dispatch<EPI_CG>(c, a, red.max_blocks, s);
}

cudaError_t launch_dslash_resid(const DslashCall &c, Field b, Field r, CGScalars *st, History h, int iter,
                                bool set_rho, RedScratch red, cudaStream_t s) {
    KArgs a = base_args(c);
    a.b = b.v;
    a.r = r.v;
    a.st = st;
    a.h_alpha = h.alpha;
    a.h_beta = h.beta;
    a.h_rho = h.rho;
    a.iter = iter;
    a.jbase = h.jbase;
    a.set_rho = set_rho;
    a.partials = red.partials;
    a.counter = red.counter;
    return dispatch<EPI_RESID>(c, a, red.max_blocks, s);
}

}  // namespace eig
