// BiCGSTAB on M x = b (van der Vorst, SIAM J. Sci. Stat. Comput. 13, 631 (1992)), the
// solver Sec. 1 of the paper proposes to deflate with the eigenvectors that CG/eigCG
// compute for A = M^H M = (g5 M)^2.  One RHS; vectors in the op's storage precision
// (FP32 or FP64), x in FP64; the complex scalars rho, alpha, omega, beta live in device
// memory and are computed by the last block of each reduction, so an iteration needs
// no host round trip:
//   p = r + beta (p - omega v)        k_bicg_p
//   v = M p                           (stencil)
//   alpha = rho / (r_hat^H v)         k_bicg_alpha
//   s = r - alpha v                   k_bicg_s
//   t = M s                           (stencil)
//   omega = (t^H s) / (t^H t)         k_bicg_omega
//   x += alpha p + omega s, r = s - omega t, rho' = r_hat^H r, beta = (rho'/rho)(alpha/omega)
//                                     k_bicg_update
#include "kernels.cuh"
#include "prof.h"

namespace eig {

namespace {

constexpr int BB = 256;

// Sums NC per-thread values over the grid (fixed order: deterministic); the block
// that finishes last calls finish(tot) in thread 0.  counter must be zero on entry.
template <int NC, typename F>
__device__ __forceinline__ void grid_sum(const double (&v)[NC], double *partials, unsigned *counter, double *smem,
                                         F finish) {
    __shared__ bool am_last;
    double bs[NC];
#pragma unroll
    for (int c = 0; c < NC; c++) bs[c] = block_reduce_rhs(v[c], 1, smem);
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < NC; c++) partials[(long)blockIdx.x * NC + c] = bs[c];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double s[NC], tot[NC];
#pragma unroll
    for (int c = 0; c < NC; c++) s[c] = 0.0;
    for (long b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < NC; c++) s[c] += __ldcg(partials + b * NC + c);
#pragma unroll
    for (int c = 0; c < NC; c++) tot[c] = block_reduce_rhs(s[c], 1, smem);
    if (threadIdx.x == 0) {
        finish(tot);
        *counter = 0u;
    }
}

__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double &qr, double &qi) {
    const double d = br * br + bi * bi;
    qr = (ar * br + ai * bi) / d;
    qi = (ai * br - ar * bi) / d;
}

template <typename C>
__device__ __forceinline__ Cx<C> cx(const double *z) {
    return cmk<C>((C)z[0], (C)z[1]);
}

// p = r + beta (p - omega v)
template <typename S>
__global__ void __launch_bounds__(BB) k_bicg_p(FieldView r, FieldView p, FieldView v, const BicgScalars *sc) {
    using C = typename SpinorStore<S>::C;
    if (!sc->active) return;
    const Cx<C> be = cx<C>(sc->beta), om = cx<C>(sc->omega);
    for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < r.V; s += (long)gridDim.x * blockDim.x) {
        Spinor<C> rr, pp, vv;
        SpinorStore<S>::load(r, s, 0, rr);
        SpinorStore<S>::load(p, s, 0, pp);
        SpinorStore<S>::load(v, s, 0, vv);
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const Cx<C> d = pp.s[i][j] - cmul(om, vv.s[i][j]);
                pp.s[i][j] = cfma(be, d, rr.s[i][j]);
            }
        SpinorStore<S>::store(p, s, 0, pp);
    }
}

// alpha = rho / (r_hat^H v)
template <typename S>
__global__ void __launch_bounds__(BB) k_bicg_alpha(FieldView rh, FieldView v, BicgScalars *sc, double *partials,
                                                   unsigned *counter) {
    using C = typename SpinorStore<S>::C;
    __shared__ double smem[BB / 32];
    if (!sc->active) return;
    double acc[2] = {0.0, 0.0};
    for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < v.V; s += (long)gridDim.x * blockDim.x) {
        Spinor<C> a, b;
        SpinorStore<S>::load(rh, s, 0, a);
        SpinorStore<S>::load(v, s, 0, b);
        Cx<C> d = cmk<C>(0, 0);
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) d = cfma_conj(a.s[i][j], b.s[i][j], d);
        acc[0] += (double)d.re;
        acc[1] += (double)d.im;
    }
    grid_sum<2>(acc, partials, counter, smem, [=](const double *t) {
        if (!(t[0] * t[0] + t[1] * t[1] > 0.0) || !isfinite(t[0]) || !isfinite(t[1])) {
            sc->breakdown = 1;
            sc->active = 0;
            return;
        }
        cdiv(sc->rho[0], sc->rho[1], t[0], t[1], sc->alpha[0], sc->alpha[1]);
    });
}

// s = r - alpha v
template <typename S>
__global__ void __launch_bounds__(BB) k_bicg_s(FieldView r, FieldView v, FieldView sv, const BicgScalars *sc) {
    using C = typename SpinorStore<S>::C;
    if (!sc->active) return;
    const Cx<C> mal = cmk<C>((C)-sc->alpha[0], (C)-sc->alpha[1]);
    for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < r.V; s += (long)gridDim.x * blockDim.x) {
        Spinor<C> rr, vv;
        SpinorStore<S>::load(r, s, 0, rr);
        SpinorStore<S>::load(v, s, 0, vv);
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) rr.s[i][j] = cfma(mal, vv.s[i][j], rr.s[i][j]);
        SpinorStore<S>::store(sv, s, 0, rr);
    }
}

// omega = (t^H s) / (t^H t)
template <typename S>
__global__ void __launch_bounds__(BB) k_bicg_omega(FieldView t, FieldView sv, BicgScalars *sc, double *partials,
                                                   unsigned *counter) {
    using C = typename SpinorStore<S>::C;
    __shared__ double smem[BB / 32];
    if (!sc->active) return;
    double acc[3] = {0.0, 0.0, 0.0};
    for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < t.V; s += (long)gridDim.x * blockDim.x) {
        Spinor<C> a, b;
        SpinorStore<S>::load(t, s, 0, a);
        SpinorStore<S>::load(sv, s, 0, b);
        Cx<C> d = cmk<C>(0, 0);
        C n = 0;
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                d = cfma_conj(a.s[i][j], b.s[i][j], d);
                n += a.s[i][j].re * a.s[i][j].re + a.s[i][j].im * a.s[i][j].im;
            }
        acc[0] += (double)d.re;
        acc[1] += (double)d.im;
        acc[2] += (double)n;
    }
    grid_sum<3>(acc, partials, counter, smem, [=](const double *tt) {
        if (!(tt[2] > 0.0) || !isfinite(tt[0]) || !isfinite(tt[1]) || !isfinite(tt[2])) {
            sc->breakdown = 1;
            sc->active = 0;
            return;
        }
        sc->omega[0] = tt[0] / tt[2];
        sc->omega[1] = tt[1] / tt[2];
    });
}

// x += alpha p + omega s (FP64 x), r = s - omega t, then ||r||^2, rho' = r_hat^H r and beta
template <typename S>
__global__ void __launch_bounds__(BB) k_bicg_update(FieldView x, FieldView p, FieldView sv, FieldView t, FieldView r,
                                                    FieldView rh, BicgScalars *sc, double *partials,
                                                    unsigned *counter) {
    using C = typename SpinorStore<S>::C;
    __shared__ double smem[BB / 32];
    if (!sc->active) return;
    const Cx<double> al = cx<double>(sc->alpha), omd = cx<double>(sc->omega);
    const Cx<C> mom = cmk<C>((C)-sc->omega[0], (C)-sc->omega[1]);
    double acc[3] = {0.0, 0.0, 0.0};
    for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < r.V; s += (long)gridDim.x * blockDim.x) {
        Spinor<C> pp, ss, tt, hh;
        Spinor<double> xx;
        SpinorStore<S>::load(p, s, 0, pp);
        SpinorStore<S>::load(sv, s, 0, ss);
        SpinorStore<S>::load(t, s, 0, tt);
        SpinorStore<S>::load(rh, s, 0, hh);
        SpinorStore<double>::load(x, s, 0, xx);
        Cx<C> d = cmk<C>(0, 0);
        C n = 0;
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const Cx<double> pd = cmk<double>(pp.s[i][j].re, pp.s[i][j].im);
                const Cx<double> sd = cmk<double>(ss.s[i][j].re, ss.s[i][j].im);
                xx.s[i][j] = cfma(omd, sd, cfma(al, pd, xx.s[i][j]));
                const Cx<C> rn = cfma(mom, tt.s[i][j], ss.s[i][j]);
                tt.s[i][j] = rn;
                d = cfma_conj(hh.s[i][j], rn, d);
                n += rn.re * rn.re + rn.im * rn.im;
            }
        SpinorStore<double>::store(x, s, 0, xx);
        SpinorStore<S>::store(r, s, 0, tt);
        acc[0] += (double)n;
        acc[1] += (double)d.re;
        acc[2] += (double)d.im;
    }
    grid_sum<3>(acc, partials, counter, smem, [=](const double *v) {
        sc->rr = v[0];
        sc->iters++;
        if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2])) {
            sc->breakdown = 1;
            sc->active = 0;
            return;
        }
        if (v[0] <= sc->target) {
            sc->active = 0;
            return;
        }
        if (!(sc->omega[0] * sc->omega[0] + sc->omega[1] * sc->omega[1] > 0.0) ||
            !(sc->rho[0] * sc->rho[0] + sc->rho[1] * sc->rho[1] > 0.0)) {
            sc->breakdown = 1;
            sc->active = 0;
            return;
        }
        double q1r, q1i, q2r, q2i;
        cdiv(v[1], v[2], sc->rho[0], sc->rho[1], q1r, q1i);
        cdiv(sc->alpha[0], sc->alpha[1], sc->omega[0], sc->omega[1], q2r, q2i);
        sc->beta[0] = q1r * q2r - q1i * q2i;
        sc->beta[1] = q1r * q2i + q1i * q2r;
        sc->rho[0] = v[1];
        sc->rho[1] = v[2];
    });
}

// out = g5 in (chiral basis: g5 = diag(1, 1, -1, -1) in spin)
template <typename S>
__global__ void __launch_bounds__(BB) k_gamma5(FieldView in, FieldView out) {
    using C = typename SpinorStore<S>::C;
    const long total = in.V * in.k;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long s = g / in.k;
        const int q = (int)(g - s * in.k);
        Spinor<C> v;
        SpinorStore<S>::load(in, s, q, v);
#pragma unroll
        for (int i = 2; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) v.s[i][j] = cmk<C>(-v.s[i][j].re, -v.s[i][j].im);
        SpinorStore<S>::store(out, s, q, v);
    }
}

int grid_for(long n, int cap) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long g = (n + BB - 1) / BB;
    const long lim = (long)sms * 8;
    if (g > lim) g = lim;
    if (cap > 0 && g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

double spbytes(Prec p) { return p == P64 ? 192.0 : 96.0; }

}  // namespace

#define EIG_BICG_DISPATCH(K, ...)                                                       \
    do {                                                                                \
        if (prec == P64) K<double><<<G, BB, 0, s>>>(__VA_ARGS__);                       \
        else if (prec == P32) K<float><<<G, BB, 0, s>>>(__VA_ARGS__);                   \
        else return cudaErrorInvalidValue;                                              \
    } while (0)

cudaError_t launch_bicg_p(Field r, Field p, Field v, const BicgScalars *sc, cudaStream_t s) {
    ProfScope prof("bicg_p", r.v.V * 4.0 * spbytes(r.prec), s);
    const Prec prec = r.prec;
    const int G = grid_for(r.v.V, 0);
    EIG_BICG_DISPATCH(k_bicg_p, r.v, p.v, v.v, sc);
    return cudaGetLastError();
}

cudaError_t launch_bicg_alpha(Field rh, Field v, BicgScalars *sc, RedScratch red, cudaStream_t s) {
    ProfScope prof("bicg_dot", v.v.V * 2.0 * spbytes(v.prec), s);
    const Prec prec = v.prec;
    const int G = grid_for(v.v.V, red.max_blocks);
    EIG_BICG_DISPATCH(k_bicg_alpha, rh.v, v.v, sc, red.partials, red.counter);
    return cudaGetLastError();
}

cudaError_t launch_bicg_s(Field r, Field v, Field sv, const BicgScalars *sc, cudaStream_t s) {
    ProfScope prof("bicg_s", r.v.V * 3.0 * spbytes(r.prec), s);
    const Prec prec = r.prec;
    const int G = grid_for(r.v.V, 0);
    EIG_BICG_DISPATCH(k_bicg_s, r.v, v.v, sv.v, sc);
    return cudaGetLastError();
}

cudaError_t launch_bicg_omega(Field t, Field sv, BicgScalars *sc, RedScratch red, cudaStream_t s) {
    ProfScope prof("bicg_dot", t.v.V * 2.0 * spbytes(t.prec), s);
    const Prec prec = t.prec;
    const int G = grid_for(t.v.V, red.max_blocks);
    EIG_BICG_DISPATCH(k_bicg_omega, t.v, sv.v, sc, red.partials, red.counter);
    return cudaGetLastError();
}

cudaError_t launch_bicg_update(Field x64, Field p, Field sv, Field t, Field r, Field rh, BicgScalars *sc,
                               RedScratch red, cudaStream_t s) {
    if (x64.prec != P64) return cudaErrorInvalidValue;
    ProfScope prof("bicg_update", r.v.V * (5.0 * spbytes(r.prec) + 2.0 * 192.0), s);
    const Prec prec = r.prec;
    const int G = grid_for(r.v.V, red.max_blocks);
    EIG_BICG_DISPATCH(k_bicg_update, x64.v, p.v, sv.v, t.v, r.v, rh.v, sc, red.partials, red.counter);
    return cudaGetLastError();
}

cudaError_t launch_gamma5(Field in, Field out, cudaStream_t s) {
    if (in.prec != out.prec || in.v.V != out.v.V || in.v.k != out.v.k) return cudaErrorInvalidValue;
    ProfScope prof("gamma5", in.v.V * in.v.k * 2.0 * spbytes(in.prec), s);
    const Prec prec = in.prec;
    const int G = grid_for(in.v.V * in.v.k, 0);
    EIG_BICG_DISPATCH(k_gamma5, in.v, out.v);
    return cudaGetLastError();
}

#undef EIG_BICG_DISPATCH

}  // namespace eig
