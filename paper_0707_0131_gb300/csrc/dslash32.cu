// FP32-arithmetic Wilson stencil: the staged (cp.async) variants, the choice between
// variants and the launchers.  Kernels and design notes: dslash32.cuh.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "dslash32.cuh"
#include "prof.h"

namespace eig {

namespace {

std::mutex g_mu32;
std::unordered_map<const void *, int> g_occ32;

// Variants of the FP32 stencil:
//   0  staged loads (cp.async ring), 1 RHS per thread      1  staged, 2 RHS per thread
//   2  direct loads, 1 RHS per thread, 4 blocks/SM         3  direct, 1 RHS, 5 blocks/SM
//   4  direct loads, 2 RHS per thread, 3 blocks/SM         5  direct, 2 RHS, 4 blocks/SM
//   6  as 4, with an L1 prefetch of the next hop           7  as 3, with the L1 prefetch
//   8 + v (v = 2..7): direct variant v over the tiled site traversal (full lattice only;
//   v itself where the lattice cannot be tiled)
//  16  pipelined pair (dslash32pp.cuh): 2 adjacent RHS per thread, 256-bit loads, the
//      next hop's loads in flight while the current one is computed, 2 blocks/SM
//  17  as 16, 3 blocks/SM        18, 19: 16, 17 over the tiled site traversal
//  20  as 17, plus an L1 prefetch of the hop after next;  21: 20 over the tiled site traversal
// The fastest valid one is chosen per (volume, k, storage, link format) by
// autotune_dslash32 and cached; EIG_DSLASH_VARIANT=0..21 in the environment forces one.
constexpr int NVAR = 22;

bool is_pp(int v) { return v >= 16; }
bool is_tiled(int v) { return (v >= 8 && v < 16) || v == 18 || v == 19 || v == 21; }

int variant_rb(int v) {
    if (is_pp(v)) return 2;
    v &= 7;
    return (v == 1 || v == 4 || v == 5 || v == 6) ? 2 : 1;
}

bool variant_ok(int v, unsigned k, int gf) {
    if (v < 0 || v >= NVAR) return false;
    if (v >= 8 && v < 16 && (v & 7) < 2) return false;  // tiling only for the direct variants
    if (variant_rb(v) == 2 && (k < 2 || (k % 2) != 0)) return false;
    return true;
}

// the pipelined-pair variants load and store 32 bytes per thread: every field they touch
// must start on a 32-byte boundary (scale arrays on an 8-byte one); they do not write the
// single-RHS t_prev copy of eigCG
bool pp_aligned(const K32 &a) {
    const uintptr_t f = (uintptr_t)a.in | (uintptr_t)a.out | (uintptr_t)a.r | (uintptr_t)a.cen;
    const uintptr_t sc = (uintptr_t)a.in_s | (uintptr_t)a.out_s | (uintptr_t)a.r_s | (uintptr_t)a.cen_s;
    return (f & 31) == 0 && (sc & 7) == 0 && !a.save_t;
}

// Tiled traversal for a launch with rb RHS per thread: a tile of as many sites as a CTA
// covers (TPB / (k / rb), a power of two), its extents doubled round-robin from x while
// each divides its lattice extent and leaves at least two tiles along it.  False (and
// a.tile = 0) for the odd-even form or where no such tile exists.
bool tile_setup(K32 &a, int rb) {
    a.tile = 0;
    if (a.eo >= 0) return false;
    const unsigned kb = a.k / (unsigned)rb;
    if (kb == 0 || kb > (unsigned)TPB) return false;
    unsigned b = 0;
    while ((1u << (b + 1)) <= (unsigned)TPB / kb) b++;
    const unsigned L[4] = {a.L0, a.L1, a.L2, a.L3};
    unsigned tl[4] = {0, 0, 0, 0};
    while (b > 0) {
        bool grew = false;
        for (int d = 0; d < 4 && b > 0; d++) {
            const unsigned e = 2u << tl[d];
            if (L[d] % e == 0 && L[d] / e >= 2) {
                tl[d]++;
                b--;
                grew = true;
            }
        }
        if (!grew) return false;
    }
    a.tl0 = tl[0];
    a.tl1 = tl[1];
    a.tl2 = tl[2];
    a.tl3 = tl[3];
    a.nt0 = a.L0 >> tl[0];
    a.nt1 = a.L1 >> tl[1];
    a.dt0 = fastdiv_make(a.nt0);
    a.dt1 = fastdiv_make(a.nt1);
    a.dt2 = fastdiv_make(a.L2 >> tl[2]);
    a.tile = 1;
    return true;
}

std::mutex g_var_mu;
std::unordered_map<unsigned long long, int> g_var;

unsigned long long var_key(unsigned V, unsigned k, int prec, int gf) {
    return ((unsigned long long)V << 24) ^ ((unsigned long long)k << 8) ^ ((unsigned long long)prec << 4) ^ (unsigned)gf;
}

int forced_variant() {
    static int f = -2;
    if (f == -2) {
        const char *e = getenv("EIG_DSLASH_VARIANT");
        char *end = nullptr;
        const long v = e ? strtol(e, &end, 10) : -1;
        f = (e && end != e && *end == 0 && v >= 0 && v < NVAR) ? (int)v : -1;
    }
    return f;
}

thread_local int g_var_override = -1;  // set while autotuning

int variant_for_full(const K32 &a, int prec, int gf);

int variant_for(const K32 &a, int prec, int gf) {
    // the staged variants take the centre term from `in`: not for the odd-even form
    if (a.eo >= 0) {
        const int v = variant_for_full(a, prec, gf);
        return v <= 1 ? (variant_ok(4, a.k, gf) ? 4 : 2) : v;
    }
    return variant_for_full(a, prec, gf);
}

int variant_for_full(const K32 &a, int prec, int gf) {
    if (g_var_override >= 0 && variant_ok(g_var_override, a.k, gf)) return g_var_override;
    const int f = forced_variant();
    if (f >= 0 && variant_ok(f, a.k, gf)) return f;
    {
        std::lock_guard<std::mutex> lk(g_var_mu);
        auto it = g_var.find(var_key(a.V, a.k, prec, gf));
        if (it != g_var.end()) return it->second;
    }
    return variant_ok(1, a.k, gf) ? 1 : 0;
}

template <typename S, int GF, bool DAG, int EPI>
cudaError_t launch_staged(int rb, const K32 &a, int cap, cudaStream_t s) {
    const long work_rb1 = (long)a.V * a.k;
    if (rb == 2) {
        auto kern = k_dslash32<S, GF, DAG, EPI, 2, 0, 1>;
        const size_t sm = (size_t)NS * Pipe<S, GF, 2>::NSLOT * TPB * 16;
        kern<<<d32_grid((const void *)kern, work_rb1 / 2, cap, sm), TPB, sm, s>>>(a);
    } else {
        auto kern = k_dslash32<S, GF, DAG, EPI, 1, 0, 1>;
        const size_t sm = (size_t)NS * Pipe<S, GF, 1>::NSLOT * TPB * 16;
        kern<<<d32_grid((const void *)kern, work_rb1, cap, sm), TPB, sm, s>>>(a);
    }
    return cudaGetLastError();
}

template <typename S, int GF, bool DAG, int EPI>
cudaError_t launch_rb(const K32 &a, int cap, cudaStream_t s) {
    // the kernels split thread indices with shifts (k a power of two) and fast division
    // (extents >= 2)
    if (a.k == 0 || (a.k & (a.k - 1)) != 0 || a.L0 < 2 || a.L1 < 2 || a.L2 < 2) return cudaErrorInvalidValue;
    const int prec = sizeof(S) == 4 ? 32 : 16;
    const int v = variant_for(a, prec, GF);
    if (v <= 1) return launch_staged<S, GF, DAG, EPI>(variant_rb(v), a, cap, s);
    K32 b = a;
    if (is_tiled(v)) tile_setup(b, variant_rb(v));
    if (is_pp(v)) {
        if (!pp_aligned(b)) return d32_launch_direct_rb2(4, prec, GF, DAG, EPI, b, cap, s);
        if (v == 20 || v == 21) return d32_launch_pp3f(prec, GF, DAG, EPI, b, cap, s);
        return (v == 16 || v == 18) ? d32_launch_pp2(prec, GF, DAG, EPI, b, cap, s)
                                    : d32_launch_pp3(prec, GF, DAG, EPI, b, cap, s);
    }
    if (variant_rb(v) == 1) return d32_launch_direct_rb1(v & 7, prec, GF, DAG, EPI, b, cap, s);
    return d32_launch_direct_rb2(v & 7, prec, GF, DAG, EPI, b, cap, s);
}

template <int EPI>
cudaError_t dispatch32(const DslashCall &c, const K32 &a, int cap, cudaStream_t s) {
#define EIG32(S, GF)                                                          \
    return c.dagger ? launch_rb<S, GF, true, EPI>(a, cap, s) : launch_rb<S, GF, false, EPI>(a, cap, s)
    if (c.in.prec == P32) {
        if (c.gformat == GF_F32_12) EIG32(float, GF_F32_12);
        if (c.gformat == GF_F32_18) EIG32(float, GF_F32_18);
    } else if (c.in.prec == P16) {
        if (c.gformat == GF_F32_12) EIG32(__half, GF_F32_12);
    }
#undef EIG32
    return cudaErrorInvalidValue;
}

K32 args32(const DslashCall &c) {
    K32 a;
    memset(&a, 0, sizeof(a));
    a.in = static_cast<const float4 *>(c.in.v.data);
    a.in_s = c.in.v.scale;
    a.out = static_cast<float4 *>(c.out.v.data);
    a.out_s = c.out.v.scale;
    a.g = c.gauge.data;
    a.L0 = c.L[0];
    a.L1 = c.L[1];
    a.L2 = c.L[2];
    a.L3 = c.L[3];
    a.d0 = fastdiv_make(a.L0);
    a.d1 = fastdiv_make(a.L1);
    a.d2 = fastdiv_make(a.L2);
    a.Vg = (unsigned)c.V;
    a.eo = c.eo_parity;
    a.V = (unsigned)(c.eo_parity >= 0 ? c.V / 2 : c.V);
    a.k = (unsigned)c.k;
    a.P = a.V * a.k;
    a.diag = (float)c.diag;
    a.hcoef = (float)c.hcoef;
    a.lh = a.L0 / 2;
    if (a.lh >= 2) a.dh = fastdiv_make(a.lh);
    if (c.eo_parity >= 0) {
        a.cen = static_cast<const float4 *>(c.cen.v.data);
        a.cen_s = c.cen.v.scale;
    }
    return a;
}

}  // namespace

int d32_grid(const void *kern, long work, int cap, size_t smem) {
    int per = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu32);
        auto it = g_occ32.find(kern);
        if (it != g_occ32.end()) per = it->second;
        else {
            if (smem > 0) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, TPB, smem);
            if (per < 1) per = 1;
            g_occ32[kern] = per;
        }
    }
    long need = (work + TPB - 1) / TPB;
    long grid = (long)device_sm_count() * per;
    if (grid > need) grid = need;
    if (cap > 0 && grid > cap) grid = cap;
    return (int)(grid < 1 ? 1 : grid);
}

bool dslash32_handles(const DslashCall &c) { return c.in.prec != P64; }

std::mutex g_fmt_mu;
std::unordered_map<unsigned long long, int> g_fmt;  // (V, k, prec) -> faster link format

unsigned long long fmt_key(unsigned V, unsigned k, int prec) {
    return ((unsigned long long)V << 24) ^ ((unsigned long long)k << 8) ^ (unsigned long long)prec;
}

// EIG_DSLASH_LINKS=12 or 18 in the environment forces the FP32 link format
int forced_gformat() {
    static int f = -2;
    if (f == -2) {
        const char *e = getenv("EIG_DSLASH_LINKS");
        f = !e ? -1 : (strcmp(e, "12") == 0 ? GF_F32_12 : (strcmp(e, "18") == 0 ? GF_F32_18 : -1));
    }
    return f;
}

int dslash32_best_gformat(long V, int k, int prec) {
    if (prec == 32 && forced_gformat() >= 0) return forced_gformat();
    std::lock_guard<std::mutex> lk(g_fmt_mu);
    auto it = g_fmt.find(fmt_key((unsigned)V, (unsigned)k, prec));
    return it == g_fmt.end() ? -1 : it->second;
}

// The choice a call would be launched with: link format (-1 before the call's shape is
// tuned) and stencil variant.
int dslash32_choice(const DslashCall &c0, int *variant) {
    const int prec = c0.in.prec == P32 ? 32 : 16;
    *variant = -1;
    const int gf = dslash32_best_gformat(c0.V, c0.k, prec);
    if (gf < 0) return -1;
    DslashCall c = c0;
    c.gformat = gf;
    const K32 a = args32(c);
    *variant = variant_for(a, prec, gf);
    return gf;
}

// Times the plain stencil in every valid variant on the caller's buffers (in -> out),
// for the call's link format and the alternative one, and caches the fastest choices.
cudaError_t autotune_dslash32(const DslashCall &c0, const void *const *gauge_alts, const int *gf_alts, int n_alts,
                              cudaStream_t s) {
    const int prec = c0.in.prec == P32 ? 32 : 16;
    {
        std::lock_guard<std::mutex> lk(g_fmt_mu);
        if (g_fmt.count(fmt_key((unsigned)c0.V, (unsigned)c0.k, prec))) return cudaSuccess;
    }
    const char *le = getenv("EIG_AUTOTUNE_LOG");
    const bool log = le && le[0] == '1';
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_fmt_ms = 1e30f;
    int best_fmt = c0.gformat;
    for (int f = 0; f <= n_alts; f++) {
        DslashCall c = c0;
        if (f >= 1) {
            if (!gauge_alts[f - 1]) continue;
            c.gauge.data = const_cast<void *>(gauge_alts[f - 1]);
            c.gformat = gf_alts[f - 1];
        }
        K32 a = args32(c);
        float best = 1e30f;
        int best_v = -1;
        for (int v = 0; v < NVAR; v++) {
            if (!variant_ok(v, a.k, c.gformat)) continue;
            K32 tb = a;
            if (is_tiled(v) && !tile_setup(tb, variant_rb(v))) continue;  // same as the untiled one here
            if (is_pp(v) && !pp_aligned(a)) continue;
            if (forced_variant() >= 0 && v != forced_variant()) continue;
            g_var_override = v;
            dispatch32<E_PLAIN>(c, a, 0, s);  // warm
            cudaEventRecord(e0, s);
            for (int rep = 0; rep < 3; rep++) dispatch32<E_PLAIN>(c, a, 0, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (log)
                fprintf(stderr, "dslash32 autotune V=%u k=%u prec=%d gf=%d variant %d: %.4f ms per launch\n", a.V,
                        a.k, prec, c.gformat, v, ms / 3.0);
            if (ms < best) {
                best = ms;
                best_v = v;
            }
        }
        g_var_override = -1;
        if (best_v >= 0) {
            std::lock_guard<std::mutex> lk(g_var_mu);
            g_var[var_key(a.V, a.k, prec, c.gformat)] = best_v;
        }
        if (best < best_fmt_ms) {
            best_fmt_ms = best;
            best_fmt = c.gformat;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_fmt_mu);
        g_fmt[fmt_key((unsigned)c0.V, (unsigned)c0.k, prec)] = best_fmt;
    }
    return cudaGetLastError();
}

cudaError_t launch_dslash32(const DslashCall &c, cudaStream_t s) {
    K32 a = args32(c);
    return dispatch32<E_PLAIN>(c, a, 0, s);
}

cudaError_t launch_dslash32_norm(const DslashCall &c, CGScalars *st, History h, int iter, RedScratch red,
                                 cudaStream_t s) {
    K32 a = args32(c);
    a.st = st;
    a.h_alpha = h.alpha;
    a.h_beta = h.beta;
    a.h_rho = h.rho;
    a.iter = iter;
    a.jbase = h.jbase;
    a.partials = red.partials;
    a.counter = red.counter;
    return dispatch32<E_NORM>(c, a, red.max_blocks, s);
}

cudaError_t launch_dslash32_cg(const DslashCall &c, Field r, Field t_save, CGScalars *st, History h, int iter,
                               RedScratch red, cudaStream_t s) {
    K32 a = args32(c);
    a.r = static_cast<float4 *>(r.v.data);
    a.r_s = r.v.scale;
    a.tsave = static_cast<float4 *>(t_save.v.data);
    a.save_t = t_save.v.data != nullptr;
    a.st = st;
    a.h_alpha = h.alpha;
    a.h_beta = h.beta;
    a.h_rho = h.rho;
    a.iter = iter;
    a.jbase = h.jbase;
    a.partials = red.partials;
    a.counter = red.counter;
    return dispatch32<E_CG>(c, a, red.max_blocks, s);
}

}  // namespace eig
