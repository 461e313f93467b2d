// Allocation-free application of the Wilson operator (FP64, one RHS).
//
// Who needs it: callers that may not allocate device memory -- applications whose
// device memory belongs to another allocator or pool that forbids cudaMalloc, and
// processes that have already reserved nearly all of the device for themselves.
// eig_op_apply serves neither: an op handle owns device buffers (the gauge field in
// the library's own layout, staging for natural-layout vectors) that it allocates
// when it is created.  eig_wilson_apply_noalloc works on caller-owned device
// buffers in the natural layout of eigcg.h and allocates nothing.
//
// Scratch: A = M^H M needs the intermediate M x.  It lives in g_noalloc_scratch,
// a file-scope device array sized for NOALLOC_MAX_SITES lattice sites of one FP64
// spinor (65536 * 12 complex doubles = 12.6 MB, present on every device that
// loads this module until the process exits).  Every call shares it and it keeps
// the contents of the last call; the intermediate is written in full before it is
// read, so nothing in it has to start at zero.  Calls that overlap on the GPU
// (different streams or host threads at the same time) race on it and must be
// serialised by the caller.
//
// Set-up: the array's host-side name is not a device address.  The first call on
// each device, with that device current, looks the address up once with
// cudaGetSymbolAddress and caches it; that first call should come before any
// stream capture starts (a first call on a capturing stream is refused).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "eigcg.h"

namespace eig {

void set_last_error_message(const char *msg);

constexpr long NOALLOC_MAX_SITES = 65536;

static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_MAX_SITES * 12];

namespace {

using C = double;

// (I + SG g_mu) psi = (h, SG B_mu^H h), h = a + SG B_mu b in the chiral basis, with
// B_1 = [[0, i], [i, 0]], B_2 = [[0, -1], [1, 0]], B_3 = diag(i, -i), B_4 = I.
template <int MU, int SG>
__device__ __forceinline__ void na_project(const Spinor<C> &p, Half<C> &h) {
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
        h.h[0][c] = SG > 0 ? a0 + q0 : a0 - q0;
        h.h[1][c] = SG > 0 ? a1 + q1 : a1 - q1;
    }
}

template <int MU, int SG>
__device__ __forceinline__ void na_accumulate(Spinor<C> &acc, const Half<C> &h) {
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
        acc.s[2][c] = SG > 0 ? acc.s[2][c] + g0 : acc.s[2][c] - g0;
        acc.s[3][c] = SG > 0 ? acc.s[3][c] + g1 : acc.s[3][c] - g1;
    }
}

__device__ __forceinline__ void na_load_spinor(const double2 *f, long s, Spinor<C> &v) {
#pragma unroll
    for (int e = 0; e < 12; e++) {
        const double2 d = f[s * 12 + e];
        v.s[e / 3][e % 3] = cmk<C>(d.x, d.y);
    }
}

// acc += (I - SF g_mu) U_mu(x) psi(x+mu) + (I + SF g_mu) U_mu(x-mu)^H psi(x-mu), with the
// signs of M (SF = -1) or, through gamma5 M gamma5 = M^H, of M^H (SF = +1)
template <int MU, bool DAG>
__device__ __forceinline__ void na_hop(const double2 *g, const double2 *in, long s, long sf, long sb,
                                       Spinor<C> &acc) {
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    Spinor<C> nb;
    Half<C> h, uh;
    const double2 *U = g + (s * 4 + MU) * 9;
    na_load_spinor(in, sf, nb);
    na_project<MU, SF>(nb, h);
#pragma unroll
    for (int sp = 0; sp < 2; sp++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            Cx<C> v = cmk<C>(0, 0);
#pragma unroll
            for (int b = 0; b < 3; b++) v = cfma(cmk<C>(U[a * 3 + b].x, U[a * 3 + b].y), h.h[sp][b], v);
            uh.h[sp][a] = v;
        }
    na_accumulate<MU, SF>(acc, uh);
    const double2 *W = g + (sb * 4 + MU) * 9;
    na_load_spinor(in, sb, nb);
    na_project<MU, SB>(nb, h);
#pragma unroll
    for (int sp = 0; sp < 2; sp++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            Cx<C> v = cmk<C>(0, 0);
#pragma unroll
            for (int b = 0; b < 3; b++) v = cfma_conj(cmk<C>(W[b * 3 + a].x, W[b * 3 + a].y), h.h[sp][b], v);
            uh.h[sp][a] = v;
        }
    na_accumulate<MU, SB>(acc, uh);
}

// out = M in (DAG: M^H in) on natural layouts: spinor [V][12], gauge [V][4][9] (double2)
template <bool DAG>
__global__ void __launch_bounds__(128) k_wilson_natural(const double2 *__restrict__ g, int L0, int L1, int L2,
                                                        int L3, double diag, const double2 *__restrict__ in,
                                                        double2 *__restrict__ out) {
    const long V = (long)L0 * L1 * L2 * L3;
    const long s1 = L0, s2 = (long)L0 * L1, s3 = s2 * L2;
    for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < V; s += (long)gridDim.x * blockDim.x) {
        const int x = (int)(s % L0), y = (int)((s / s1) % L1), z = (int)((s / s2) % L2), t = (int)(s / s3);
        Spinor<C> acc;
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) acc.s[i][j] = cmk<C>(0, 0);
        na_hop<0, DAG>(g, in, s, x == L0 - 1 ? s - (L0 - 1) : s + 1, x == 0 ? s + (L0 - 1) : s - 1, acc);
        na_hop<1, DAG>(g, in, s, y == L1 - 1 ? s - (L1 - 1) * s1 : s + s1, y == 0 ? s + (L1 - 1) * s1 : s - s1, acc);
        na_hop<2, DAG>(g, in, s, z == L2 - 1 ? s - (L2 - 1) * s2 : s + s2, z == 0 ? s + (L2 - 1) * s2 : s - s2, acc);
        na_hop<3, DAG>(g, in, s, t == L3 - 1 ? s - (L3 - 1) * s3 : s + s3, t == 0 ? s + (L3 - 1) * s3 : s - s3, acc);
        Spinor<C> c0;
        na_load_spinor(in, s, c0);
#pragma unroll
        for (int e = 0; e < 12; e++) {
            const Cx<C> v = c0.s[e / 3][e % 3], a = acc.s[e / 3][e % 3];
            out[s * 12 + e] = make_double2(diag * v.re - 0.5 * a.re, diag * v.im - 0.5 * a.im);
        }
    }
}

std::mutex g_na_mu;
constexpr int NA_MAX_DEVICES = 64;
double2 *g_na_ptr[NA_MAX_DEVICES] = {nullptr};
PFN_cuMemGetAddressRange_v3020 g_range = nullptr;

eig_status na_fail(eig_status st, const char *msg) {
    set_last_error_message(msg);
    return st;
}

// true if [p, p + bytes) lies inside one device allocation of this process that the
// current device `dev` can address: device memory of `dev` itself, or managed memory
bool device_range_ok(const void *p, size_t bytes, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return false;
    if (at.type == cudaMemoryTypeDevice && at.device != dev) return false;  // another GPU's memory
    if (!g_range) return true;  // no range query available: the type check only
    CUdeviceptr base = 0;
    size_t size = 0;
    if (g_range(&base, &size, (CUdeviceptr)(uintptr_t)p) != CUDA_SUCCESS) return false;
    const uintptr_t lo = (uintptr_t)p, b = (uintptr_t)base;
    return lo >= b && lo - b + bytes <= size;
}

// true if the byte ranges [a, a + na) and [b, b + nb) share a byte
bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

}  // namespace

}  // namespace eig

extern "C" eig_status eig_wilson_apply_noalloc(const double *gauge, const int dims[4], double m_q, int which,
                                               const double *in, double *out, void *stream) {
    using namespace eig;
    if (!gauge || !dims || !in || !out) return na_fail(EIG_ERR_ARG, "eig_wilson_apply_noalloc: null argument");
    if (which < 0 || which > 2) return na_fail(EIG_ERR_ARG, "eig_wilson_apply_noalloc: which must be 0, 1 or 2");
    long V = 1;
    for (int i = 0; i < 4; i++) {
        if (dims[i] < 2) return na_fail(EIG_ERR_ARG, "eig_wilson_apply_noalloc: every extent must be >= 2");
        V *= dims[i];
        if (V > NOALLOC_MAX_SITES)
            return na_fail(EIG_ERR_BUDGET,
                           "eig_wilson_apply_noalloc: lattice exceeds the 65536-site scratch array "
                           "(use eig_op_apply)");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        return na_fail(EIG_ERR_CUDA, "eig_wilson_apply_noalloc: no usable current device");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double2 *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            // the one-time set-up makes runtime calls that do not belong inside a capture
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
                cudaGetLastError();
                return na_fail(EIG_ERR_CUDA,
                               "eig_wilson_apply_noalloc: the first call on a device sets up the scratch "
                               "address and must not run on a capturing stream; call it once before capture");
            }
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return na_fail(EIG_ERR_CUDA, "eig_wilson_apply_noalloc: cudaGetSymbolAddress of the scratch failed");
            }
            g_na_ptr[dev] = static_cast<double2 *>(p);
            if (!g_range) {
                void *fn = nullptr;
                cudaDriverEntryPointQueryResult q;
                if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 12000, cudaEnableDefault, &q) ==
                        cudaSuccess &&
                    q == cudaDriverEntryPointSuccess)
                    g_range = reinterpret_cast<PFN_cuMemGetAddressRange_v3020>(fn);
                cudaGetLastError();
            }
        }
        scratch = g_na_ptr[dev];
    }
    const size_t fbytes = (size_t)V * 12 * sizeof(double2), gbytes = (size_t)V * 36 * sizeof(double2);
    if (!device_range_ok(gauge, gbytes, dev) || !device_range_ok(in, fbytes, dev) || !device_range_ok(out, fbytes, dev))
        return na_fail(EIG_ERR_ARG,
                       "eig_wilson_apply_noalloc: gauge, in and out must be buffers of the full lattice in the "
                       "memory of the current device (or managed memory)");
    // every thread reads neighbour spinors of `in` and the links while others write `out`
    if (overlaps(in, fbytes, out, fbytes) || overlaps(gauge, gbytes, out, fbytes))
        return na_fail(EIG_ERR_ARG, "eig_wilson_apply_noalloc: out must not overlap in or gauge");
    const double2 *g = reinterpret_cast<const double2 *>(gauge);
    const double2 *x = reinterpret_cast<const double2 *>(in);
    double2 *y = reinterpret_cast<double2 *>(out);
    const int grid = (int)((V + 127) / 128);
    const double diag = 4.0 + m_q;
    if (which == 0) {
        k_wilson_natural<false><<<grid, 128, 0, s>>>(g, dims[0], dims[1], dims[2], dims[3], diag, x, y);
    } else if (which == 1) {
        k_wilson_natural<true><<<grid, 128, 0, s>>>(g, dims[0], dims[1], dims[2], dims[3], diag, x, y);
    } else {
        k_wilson_natural<false><<<grid, 128, 0, s>>>(g, dims[0], dims[1], dims[2], dims[3], diag, x, scratch);
        k_wilson_natural<true><<<grid, 128, 0, s>>>(g, dims[0], dims[1], dims[2], dims[3], diag, scratch, y);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(EIG_ERR_CUDA, cudaGetErrorString(e));
    return EIG_OK;
}
