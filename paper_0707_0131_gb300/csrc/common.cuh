// Device-side building blocks shared by the kernels: complex arithmetic, the
// storage formats of spinor fields and gauge links, and per-RHS reductions.
//
// Internal field layout ("chunk-major, RHS-inner"): a field of k right-hand
// sides over V sites is stored as [chunk][site][rhs] of a 16-byte (or 8-byte)
// vector type, so that consecutive threads (site-major, rhs-minor) touch
// consecutive addresses for every chunk and the k RHS of one site share each
// link load.  One site holds 12 complex numbers (4 spins x 3 colours) in
// spin*3+colour order:
//   FP64: 12 chunks of double2 (one complex each)
//   FP32:  6 chunks of float4  (two complex each)
//   FP16:  3 chunks of uint4   (four complex each, eight halves) plus one FP32
//          scale per (site, rhs): stored value = true value / scale, scale =
//          largest |component| of that site's 24 reals.
// Gauge links U_mu(x), per direction mu a plane over sites:
//   FP64: [mu][9][V] double2 (18 reals)
//   FP32: [mu][3][V] float4  (rows 0-1, 12 reals; row 2 = conj(row0 x row1))
//   FP32 uncompressed: [mu][9][V] float2
//   FP16: [mu][3][V] uint2   (rows 0-1 as 12 halves)
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace eig {

template <typename C>
struct Cx {
    C re, im;
};

template <typename C>
__device__ __forceinline__ Cx<C> cmk(C r, C i) {
    Cx<C> z;
    z.re = r;
    z.im = i;
    return z;
}
template <typename C>
__device__ __forceinline__ Cx<C> operator+(Cx<C> a, Cx<C> b) { return cmk<C>(a.re + b.re, a.im + b.im); }
template <typename C>
__device__ __forceinline__ Cx<C> operator-(Cx<C> a, Cx<C> b) { return cmk<C>(a.re - b.re, a.im - b.im); }
template <typename C>
__device__ __forceinline__ Cx<C> operator*(C s, Cx<C> a) { return cmk<C>(s * a.re, s * a.im); }
// i * a
template <typename C>
__device__ __forceinline__ Cx<C> times_i(Cx<C> a) { return cmk<C>(-a.im, a.re); }
template <typename C>
__device__ __forceinline__ Cx<C> conjg(Cx<C> a) { return cmk<C>(a.re, -a.im); }
// a * b
template <typename C>
__device__ __forceinline__ Cx<C> cmul(Cx<C> a, Cx<C> b) {
    return cmk<C>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// acc + a * b
template <typename C>
__device__ __forceinline__ Cx<C> cfma(Cx<C> a, Cx<C> b, Cx<C> acc) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
    return acc;
}
// acc + conj(a) * b
template <typename C>
__device__ __forceinline__ Cx<C> cfma_conj(Cx<C> a, Cx<C> b, Cx<C> acc) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
    return acc;
}

template <typename C>
struct Spinor {
    Cx<C> s[4][3];
};
template <typename C>
struct Half {  // spin-projected half spinor: 2 spins x 3 colours
    Cx<C> h[2][3];
};
template <typename C>
struct Link {
    Cx<C> u[3][3];
};

// ------------------------------------------------------------------------------------
// Field views
// ------------------------------------------------------------------------------------
struct FieldView {
    void *data;     // chunk planes
    float *scale;   // FP16 only: [V][k]
    long V;         // sites
    int k;          // RHS per field
};

template <typename S>
struct SpinorStore;

template <>
struct SpinorStore<double> {
    using C = double;
    static constexpr int NCH = 12;
    static constexpr int BYTES = 192;
    __device__ static __forceinline__ void load(const FieldView &f, long s, int r, Spinor<double> &v) {
        const double2 *p = static_cast<const double2 *>(f.data);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            double2 d = p[((long)c * f.V + s) * f.k + r];
            v.s[c / 3][c % 3] = cmk<double>(d.x, d.y);
        }
    }
    __device__ static __forceinline__ void store(const FieldView &f, long s, int r, const Spinor<double> &v) {
        double2 *p = static_cast<double2 *>(f.data);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            Cx<double> z = v.s[c / 3][c % 3];
            p[((long)c * f.V + s) * f.k + r] = make_double2(z.re, z.im);
        }
    }
};

template <>
struct SpinorStore<float> {
    using C = float;
    static constexpr int NCH = 6;
    static constexpr int BYTES = 96;
    __device__ static __forceinline__ void load(const FieldView &f, long s, int r, Spinor<float> &v) {
        const float4 *p = static_cast<const float4 *>(f.data);
#pragma unroll
        for (int c = 0; c < 6; c++) {
            float4 d = p[((long)c * f.V + s) * f.k + r];
            int e0 = 2 * c, e1 = 2 * c + 1;
            v.s[e0 / 3][e0 % 3] = cmk<float>(d.x, d.y);
            v.s[e1 / 3][e1 % 3] = cmk<float>(d.z, d.w);
        }
    }
    __device__ static __forceinline__ void store(const FieldView &f, long s, int r, const Spinor<float> &v) {
        float4 *p = static_cast<float4 *>(f.data);
#pragma unroll
        for (int c = 0; c < 6; c++) {
            int e0 = 2 * c, e1 = 2 * c + 1;
            Cx<float> a = v.s[e0 / 3][e0 % 3], b = v.s[e1 / 3][e1 % 3];
            p[((long)c * f.V + s) * f.k + r] = make_float4(a.re, a.im, b.re, b.im);
        }
    }
};

template <>
struct SpinorStore<__half> {
    using C = float;
    static constexpr int NCH = 3;
    static constexpr int BYTES = 52;
    __device__ static __forceinline__ void load(const FieldView &f, long s, int r, Spinor<float> &v) {
        const uint4 *p = static_cast<const uint4 *>(f.data);
        float sc = f.scale[s * f.k + r];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            uint4 d = p[((long)c * f.V + s) * f.k + r];
            uint32_t w[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                __half2 h = *reinterpret_cast<__half2 *>(&w[q]);
                float2 g = __half22float2(h);
                int e = 4 * c + q;
                v.s[e / 3][e % 3] = cmk<float>(g.x * sc, g.y * sc);
            }
        }
    }
    __device__ static __forceinline__ void store(const FieldView &f, long s, int r, const Spinor<float> &v) {
        float mx = 0.f;
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) mx = fmaxf(mx, fmaxf(fabsf(v.s[a][b].re), fabsf(v.s[a][b].im)));
        float inv = mx > 0.f ? 1.0f / mx : 0.f;
        f.scale[s * f.k + r] = mx;
        uint4 *p = static_cast<uint4 *>(f.data);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                int e = 4 * c + q;
                __half2 h = __floats2half2_rn(v.s[e / 3][e % 3].re * inv, v.s[e / 3][e % 3].im * inv);
                w[q] = *reinterpret_cast<uint32_t *>(&h);
            }
            p[((long)c * f.V + s) * f.k + r] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
};

// ------------------------------------------------------------------------------------
// Gauge links
// ------------------------------------------------------------------------------------
struct GaugeView {
    const void *data;
    long V;
};

enum GaugeFormat { GF_F64_18 = 0, GF_F32_12 = 1, GF_F32_18 = 2, GF_F16_12 = 3 };

template <typename C>
__device__ __forceinline__ void reconstruct_row2(Link<C> &U) {
    // row2 = conj(row0 x row1)
    U.u[2][0] = conjg(cmul(U.u[0][1], U.u[1][2]) - cmul(U.u[0][2], U.u[1][1]));
    U.u[2][1] = conjg(cmul(U.u[0][2], U.u[1][0]) - cmul(U.u[0][0], U.u[1][2]));
    U.u[2][2] = conjg(cmul(U.u[0][0], U.u[1][1]) - cmul(U.u[0][1], U.u[1][0]));
}

template <int GF>
struct GaugeLoad;

template <>
struct GaugeLoad<GF_F64_18> {
    using C = double;
    static constexpr int BYTES = 144;
    __device__ static __forceinline__ void load(const GaugeView &g, int mu, long s, Link<double> &U) {
        const double2 *p = static_cast<const double2 *>(g.data) + (long)mu * 9 * g.V;
#pragma unroll
        for (int e = 0; e < 9; e++) {
            double2 d = __ldg(p + (long)e * g.V + s);
            U.u[e / 3][e % 3] = cmk<double>(d.x, d.y);
        }
    }
};

template <>
struct GaugeLoad<GF_F32_12> {
    using C = float;
    static constexpr int BYTES = 48;
    __device__ static __forceinline__ void load(const GaugeView &g, int mu, long s, Link<float> &U) {
        const float4 *p = static_cast<const float4 *>(g.data) + (long)mu * 3 * g.V;
        float4 a = __ldg(p + s), b = __ldg(p + g.V + s), c = __ldg(p + 2 * g.V + s);
        U.u[0][0] = cmk<float>(a.x, a.y);
        U.u[0][1] = cmk<float>(a.z, a.w);
        U.u[0][2] = cmk<float>(b.x, b.y);
        U.u[1][0] = cmk<float>(b.z, b.w);
        U.u[1][1] = cmk<float>(c.x, c.y);
        U.u[1][2] = cmk<float>(c.z, c.w);
        reconstruct_row2(U);
    }
};

template <>
struct GaugeLoad<GF_F32_18> {
    using C = float;
    static constexpr int BYTES = 72;
    __device__ static __forceinline__ void load(const GaugeView &g, int mu, long s, Link<float> &U) {
        const float2 *p = static_cast<const float2 *>(g.data) + (long)mu * 9 * g.V;
#pragma unroll
        for (int e = 0; e < 9; e++) {
            float2 d = __ldg(p + (long)e * g.V + s);
            U.u[e / 3][e % 3] = cmk<float>(d.x, d.y);
        }
    }
};

template <>
struct GaugeLoad<GF_F16_12> {
    using C = float;
    static constexpr int BYTES = 24;
    __device__ static __forceinline__ void load(const GaugeView &g, int mu, long s, Link<float> &U) {
        const uint2 *p = static_cast<const uint2 *>(g.data) + (long)mu * 3 * g.V;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            uint2 d = __ldg(p + (long)q * g.V + s);
            __half2 h0 = *reinterpret_cast<__half2 *>(&d.x);
            __half2 h1 = *reinterpret_cast<__half2 *>(&d.y);
            float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
            int e0 = 2 * q, e1 = 2 * q + 1;
            U.u[e0 / 3][e0 % 3] = cmk<float>(f0.x, f0.y);
            U.u[e1 / 3][e1 % 3] = cmk<float>(f1.x, f1.y);
        }
        reconstruct_row2(U);
    }
};

// ------------------------------------------------------------------------------------
// Reductions: per-RHS sums in FP64.  Threads are laid out (site-major, rhs-minor),
// so lane l of a warp belongs to rhs l % k (k a power of two <= 32).
// ------------------------------------------------------------------------------------
constexpr int MAX_BLOCK = 256;
constexpr int MAX_RHS = 16;

// Sums v over the threads of one rhs in the block; result valid in threads 0..k-1
// (thread r holds rhs r).  smem: at least (blockDim/32)*k doubles.
__device__ __forceinline__ double block_reduce_rhs(double v, int k, double *smem) {
    for (int off = 16; off >= k; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < k) smem[warp * k + lane] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < k) {
        const int nw = blockDim.x >> 5;
        for (int w = 0; w < nw; w++) s += smem[w * k + threadIdx.x];
    }
    __syncthreads();
    return s;
}

// Last-block completion: every block writes its per-rhs partials, then the block
// that arrives last sums all partials in block order (deterministic) and runs
// `finish(rhs, total)` for each rhs.  counter must be zero on entry; it is reset.
template <typename F>
__device__ __forceinline__ void grid_reduce_rhs(double blocksum, int k, double *partials, unsigned *counter,
                                                double *smem, F finish) {
    __shared__ bool am_last;
    if (threadIdx.x < k) partials[(long)blockIdx.x * k + threadIdx.x] = blocksum;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // each thread sums a strided set of blocks for its rhs, in fixed order
    const int r = threadIdx.x % k;
    double s = 0.0;
    for (long b = threadIdx.x / k; b < gridDim.x; b += blockDim.x / k) s += __ldcg(partials + b * k + r);
    double tot = block_reduce_rhs(s, k, smem);
    if (threadIdx.x < k) finish(threadIdx.x, tot);
    if (threadIdx.x == 0) *counter = 0u;
}

// As grid_reduce_rhs, for kernels whose blocks have already written their k
// per-RHS partial sums to partials[blockIdx.x * k + r].
template <typename F>
__device__ __forceinline__ void grid_finish_rhs(int k, double *partials, unsigned *counter, double *smem, F finish) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    const int r = threadIdx.x % k;
    double s = 0.0;
    for (long b = threadIdx.x / k; b < gridDim.x; b += blockDim.x / k) s += __ldcg(partials + b * k + r);
    double tot = block_reduce_rhs(s, k, smem);
    if (threadIdx.x < k) finish(threadIdx.x, tot);
    if (threadIdx.x == 0) *counter = 0u;
}

}  // namespace eig
