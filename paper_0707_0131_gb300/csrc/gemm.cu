// Tall-skinny complex contractions of the eigCG window and the deflation basis:
//   * C = A^H B      (U^H r of Eq. 1, U^H V and V-bar^H W of the Sec. 4 box)
//   * Out = A Y      (U (H^{-1} c) of Eq. 1, the eigCG output V Y, Gram-Schmidt updates)
//   * V <- V (Q Z)   (Fig. 1 step 11.7, in place) fused with w^H V (step 11.8)
// Rows are complex vector entries (12 V of them per field); columns are fields.
// The row dimension is split across a persistent grid; partial sums of A^H B
// are combined in FP64 by the last block in fixed block order (deterministic).
// FP32 data is accumulated in FP32 over blocks of at most FLUSH rows and the
// blocks are summed in FP64 (the paper's FP32 vectors with FP64 dot products,
// Sec. 5.1).
#include <cstring>

#include "kernels.cuh"
#include "prof.h"

namespace eig {

constexpr int FLUSH = 512;

template <typename T>
struct C2;
template <>
struct C2<float> {
    using t = float2;
};
template <>
struct C2<double> {
    using t = double2;
};

template <typename T>
__device__ __forceinline__ long col_index(const ColSet &cs, long row, int col) {
    const int cpc = sizeof(T) == 8 ? 1 : 2;
    if (cs.col_off) return cs.col_off[col] + row;
    return ((row / cpc) * cs.ki + (col % cs.ki)) * cpc + row % cpc + (long)(col / cs.ki) * cs.col_stride;
}

template <typename T>
__device__ __forceinline__ typename C2<T>::t ld(const ColSet &cs, long row, int col) {
    return static_cast<const typename C2<T>::t *>(cs.base)[col_index<T>(cs, row, col)];
}

// ---------------------------------------------------------------------------------------
// C = A^H B.  Block: 256 threads; thread t owns outputs a = t % 64 + 64 i (i < OA),
// b = t / 64 + 4 j (j < OB).  Rows are staged through shared memory in tiles of RT.
// ---------------------------------------------------------------------------------------
constexpr int AHB_THREADS = 256;
constexpr int AHB_RT = 16;
constexpr int AHB_MAXA = 256;
constexpr int AHB_MAXB = 16;

template <typename T>
__global__ void __launch_bounds__(AHB_THREADS) k_gemm_ahb(ColSet A, ColSet B, long nrows, double *partials,
                                                          unsigned *counter, double *C) {
    using V2 = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    V2 *As = reinterpret_cast<V2 *>(sm_raw);      // [RT][nA]
    V2 *Bs = As + AHB_RT * A.ncols;               // [RT][nB]
    const int nA = A.ncols, nB = B.ncols;
    const int t = threadIdx.x;
    const int a0 = t % 64, b0 = t / 64;
    T acc_re[4][4], acc_im[4][4];
    double tot_re[4][4], tot_im[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc_re[i][j] = acc_im[i][j] = 0, tot_re[i][j] = tot_im[i][j] = 0.0;
    const long ntiles = (nrows + AHB_RT - 1) / AHB_RT;
    int since_flush = 0;
    for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long r0 = tile * AHB_RT;
        for (int L = t; L < AHB_RT * nA; L += AHB_THREADS) {
            const int rr = L % AHB_RT, c = L / AHB_RT;
            const long row = r0 + rr;
            V2 v;
            if (row < nrows) v = ld<T>(A, row, c);
            else v.x = v.y = 0;
            As[rr * nA + c] = v;
        }
        for (int L = t; L < AHB_RT * nB; L += AHB_THREADS) {
            const int rr = L % AHB_RT, c = L / AHB_RT;
            const long row = r0 + rr;
            V2 v;
            if (row < nrows) v = ld<T>(B, row, c);
            else v.x = v.y = 0;
            Bs[rr * nB + c] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < AHB_RT; rr++) {
            V2 bv[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int b = b0 + 4 * j;
                if (b < nB) bv[j] = Bs[rr * nB + b];
                else bv[j].x = bv[j].y = 0;
            }
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int a = a0 + 64 * i;
                if (a >= nA) continue;
                const V2 av = As[rr * nA + a];
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    // conj(av) * bv
                    acc_re[i][j] = fma(av.x, bv[j].x, acc_re[i][j]);
                    acc_re[i][j] = fma(av.y, bv[j].y, acc_re[i][j]);
                    acc_im[i][j] = fma(av.x, bv[j].y, acc_im[i][j]);
                    acc_im[i][j] = fma(-av.y, bv[j].x, acc_im[i][j]);
                }
            }
        }
        __syncthreads();
        since_flush += AHB_RT;
        if (since_flush >= FLUSH) {
            since_flush = 0;
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    tot_re[i][j] += (double)acc_re[i][j];
                    tot_im[i][j] += (double)acc_im[i][j];
                    acc_re[i][j] = acc_im[i][j] = 0;
                }
        }
    }
    // write this block's partial C
    double *P = partials + (long)blockIdx.x * nA * nB * 2;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int a = a0 + 64 * i, b = b0 + 4 * j;
            if (a < nA && b < nB) {
                P[(a * nB + b) * 2] = tot_re[i][j] + (double)acc_re[i][j];
                P[(a * nB + b) * 2 + 1] = tot_im[i][j] + (double)acc_im[i][j];
            }
        }
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (t == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    const int nout = nA * nB * 2;
    for (int o = t; o < nout; o += AHB_THREADS) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; b++) s += __ldcg(partials + (long)b * nout + o);
        C[o] = s;
    }
    if (t == 0) *counter = 0u;
}

cudaError_t launch_gemm_ahb(ColSet A, ColSet B, long nrows, double *C, RedScratch red, cudaStream_t s) {
    if (A.ncols < 1 || B.ncols < 1 || A.ncols > AHB_MAXA || B.ncols > AHB_MAXB || A.f64 != B.f64)
        return cudaErrorInvalidValue;
    const size_t esz = A.f64 ? 16 : 8;
    ProfScope prof("gemm_ahb", (double)nrows * (A.ncols + B.ncols) * esz, s);
    const size_t smem = (size_t)AHB_RT * (A.ncols + B.ncols) * esz;
    const long per_block = (long)A.ncols * B.ncols * 2;
    long ntiles = (nrows + AHB_RT - 1) / AHB_RT;
    long grid = (long)device_sm_count() * 2;
    if (grid > ntiles) grid = ntiles;
    const long cap = (long)red.max_blocks * MAX_RHS * 64 / per_block;
    if (grid > cap) grid = cap;
    if (grid < 1) return cudaErrorInvalidValue;
    if (A.f64) {
        cudaFuncSetAttribute(k_gemm_ahb<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_gemm_ahb<double><<<(int)grid, AHB_THREADS, smem, s>>>(A, B, nrows, red.partials, red.counter, C);
    } else {
        cudaFuncSetAttribute(k_gemm_ahb<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_gemm_ahb<float><<<(int)grid, AHB_THREADS, smem, s>>>(A, B, nrows, red.partials, red.counter, C);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Out = beta_out Out + A Y.  One thread per row; Y staged in shared memory.
// ---------------------------------------------------------------------------------------
constexpr int AY_MAXOUT = 16;

template <typename T>
__global__ void __launch_bounds__(128) k_gemm_ay(ColSet A, const double *Y, ColSet Out, double beta_out, long nrows) {
    using V2 = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    V2 *Ys = reinterpret_cast<V2 *>(sm_raw);  // [nA][nOut]
    const int nA = A.ncols, nO = Out.ncols;
    for (int L = threadIdx.x; L < nA * nO; L += blockDim.x) {
        V2 v;
        v.x = (T)Y[2 * L];
        v.y = (T)Y[2 * L + 1];
        Ys[L] = v;
    }
    __syncthreads();
    for (long row = (long)blockIdx.x * blockDim.x + threadIdx.x; row < nrows; row += (long)gridDim.x * blockDim.x) {
        T re[AY_MAXOUT], im[AY_MAXOUT];
#pragma unroll
        for (int c = 0; c < AY_MAXOUT; c++) re[c] = im[c] = 0;
        for (int a = 0; a < nA; a++) {
            const V2 v = ld<T>(A, row, a);
#pragma unroll
            for (int c = 0; c < AY_MAXOUT; c++) {
                if (c < nO) {
                    const V2 y = Ys[a * nO + c];
                    re[c] = fma(v.x, y.x, re[c]);
                    re[c] = fma(-v.y, y.y, re[c]);
                    im[c] = fma(v.x, y.y, im[c]);
                    im[c] = fma(v.y, y.x, im[c]);
                }
            }
        }
        V2 *ob = static_cast<V2 *>(Out.base);
#pragma unroll
        for (int c = 0; c < AY_MAXOUT; c++) {
            if (c < nO) {
                const long idx = col_index<T>(Out, row, c);
                V2 o;
                if (beta_out != 0.0) {
                    o = ob[idx];
                    o.x = (T)beta_out * o.x + re[c];
                    o.y = (T)beta_out * o.y + im[c];
                } else {
                    o.x = re[c];
                    o.y = im[c];
                }
                ob[idx] = o;
            }
        }
    }
}

cudaError_t launch_gemm_ay(ColSet A, const double *Y, ColSet Out, double beta_out, long nrows, cudaStream_t s) {
    if (A.ncols < 1 || Out.ncols < 1 || Out.ncols > AY_MAXOUT || A.f64 != Out.f64 || A.ncols > 512)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)A.ncols * Out.ncols * (A.f64 ? 16 : 8);
    ProfScope prof("gemm_ay", (double)nrows * (A.ncols + Out.ncols * (beta_out != 0.0 ? 2 : 1)) * (A.f64 ? 16 : 8), s);
    long grid = (nrows + 127) / 128;
    const long cap = (long)device_sm_count() * 8;
    if (grid > cap) grid = cap;
    if (A.f64) {
        cudaFuncSetAttribute(k_gemm_ay<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_gemm_ay<double><<<(int)grid, 128, smem, s>>>(A, Y, Out, beta_out, nrows);
    } else {
        cudaFuncSetAttribute(k_gemm_ay<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_gemm_ay<float><<<(int)grid, 128, smem, s>>>(A, Y, Out, beta_out, nrows);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// eigCG restart: V[:, c] = sum_a V[:, a] QZ[a, c] for c < nout, in place over the
// window slots (each thread owns whole rows, reading all m inputs before writing),
// fused with wv[c] = sum_rows conj(w_row) V_new[row, c], w = t - beta t_prev.
// ---------------------------------------------------------------------------------------
constexpr int WR_MAXOUT = 32;
constexpr int WR_THREADS = 128;

template <typename T>
__global__ void __launch_bounds__(WR_THREADS) k_window_restart(ColSet Vw, int m, const double *QZ, int nout,
                                                               const void *tv, const void *tpv,
                                                               const double *beta_dev, long nrows,
                                                               double *partials, unsigned *counter, double *wv) {
    using V2 = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    V2 *Qs = reinterpret_cast<V2 *>(sm_raw);  // [m][nout]
    __shared__ double red[(WR_THREADS / 32) * 2];
    for (int L = threadIdx.x; L < m * nout; L += blockDim.x) {
        V2 v;
        v.x = (T)QZ[2 * L];
        v.y = (T)QZ[2 * L + 1];
        Qs[L] = v;
    }
    __syncthreads();
    const T beta = (T)(*beta_dev);
    const V2 *t = static_cast<const V2 *>(tv);
    const V2 *tp = static_cast<const V2 *>(tpv);
    V2 *base = static_cast<V2 *>(Vw.base);
    T ws_re[WR_MAXOUT], ws_im[WR_MAXOUT];
#pragma unroll
    for (int c = 0; c < WR_MAXOUT; c++) ws_re[c] = ws_im[c] = 0;
    for (long row = (long)blockIdx.x * blockDim.x + threadIdx.x; row < nrows; row += (long)gridDim.x * blockDim.x) {
        T re[WR_MAXOUT], im[WR_MAXOUT];
#pragma unroll
        for (int c = 0; c < WR_MAXOUT; c++) re[c] = im[c] = 0;
        for (int a = 0; a < m; a++) {
            const V2 v = base[Vw.col_off[a] + row];
#pragma unroll
            for (int c = 0; c < WR_MAXOUT; c++) {
                if (c < nout) {
                    const V2 q = Qs[a * nout + c];
                    re[c] = fma(v.x, q.x, re[c]);
                    re[c] = fma(-v.y, q.y, re[c]);
                    im[c] = fma(v.x, q.y, im[c]);
                    im[c] = fma(v.y, q.x, im[c]);
                }
            }
        }
        const V2 tt = t[row], tq = tp[row];
        const T wr = tt.x - beta * tq.x, wi = tt.y - beta * tq.y;
#pragma unroll
        for (int c = 0; c < WR_MAXOUT; c++) {
            if (c < nout) {
                V2 o;
                o.x = re[c];
                o.y = im[c];
                base[Vw.col_off[c] + row] = o;
                // conj(w) * v
                ws_re[c] = fma(wr, re[c], ws_re[c]);
                ws_re[c] = fma(wi, im[c], ws_re[c]);
                ws_im[c] = fma(wr, im[c], ws_im[c]);
                ws_im[c] = fma(-wi, re[c], ws_im[c]);
            }
        }
    }
    // block reduction of the nout complex sums, one output at a time, in FP64
    double *P = partials + (long)blockIdx.x * nout * 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = 0; c < nout; c++) {
        double vr = (double)ws_re[c], vi = (double)ws_im[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            vr += __shfl_xor_sync(0xffffffffu, vr, off);
            vi += __shfl_xor_sync(0xffffffffu, vi, off);
        }
        if (lane == 0) {
            red[warp * 2] = vr;
            red[warp * 2 + 1] = vi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double sr = 0.0, si = 0.0;
            for (int w = 0; w < WR_THREADS / 32; w++) {
                sr += red[w * 2];
                si += red[w * 2 + 1];
            }
            P[c * 2] = sr;
            P[c * 2 + 1] = si;
        }
        __syncthreads();
    }
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    for (int o = threadIdx.x; o < nout * 2; o += blockDim.x) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; b++) s += __ldcg(partials + (long)b * nout * 2 + o);
        wv[o] = s;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

cudaError_t launch_window_restart(ColSet Vw, int m, const double *QZ, int nout, const void *t, const void *t_prev,
                                  const double *beta_dev, long nrows, double *wv, RedScratch red, cudaStream_t s) {
    if (nout < 1 || nout > WR_MAXOUT || m < nout || !Vw.col_off) return cudaErrorInvalidValue;
    const size_t smem = (size_t)m * nout * (Vw.f64 ? 16 : 8);
    ProfScope prof("window_restart", (double)nrows * (m + nout + 2) * (Vw.f64 ? 16 : 8), s);
    long grid = (nrows + WR_THREADS - 1) / WR_THREADS;
    long cap = (long)device_sm_count() * 4;
    if (grid > cap) grid = cap;
    const long pcap = (long)red.max_blocks * MAX_RHS * 64 / (nout * 2);
    if (grid > pcap) grid = pcap;
    if (Vw.f64) {
        cudaFuncSetAttribute(k_window_restart<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_window_restart<double><<<(int)grid, WR_THREADS, smem, s>>>(Vw, m, QZ, nout, t, t_prev, beta_dev, nrows,
                                                                     red.partials, red.counter, wv);
    } else {
        cudaFuncSetAttribute(k_window_restart<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_window_restart<float><<<(int)grid, WR_THREADS, smem, s>>>(Vw, m, QZ, nout, t, t_prev, beta_dev, nrows,
                                                                    red.partials, red.counter, wv);
    }
    return cudaGetLastError();
}

}  // namespace eig
