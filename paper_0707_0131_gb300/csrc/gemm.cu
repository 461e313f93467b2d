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

// ---------------------------------------------------------------------------------------
// FP32 C = A^H B, second form: A = fields addressed by base + a * stride (or slot
// offsets), B = fields or one RHS-inner field of k RHS.  32-row tiles are copied
// into double-buffered shared memory with cp.async (zero fill past the last row)
// while the previous tile is multiplied.  conj(a) b is accumulated as two packed
// FP32 sums P = sum re(a) b and Q = sum im(a) b, combined as P + (Q.im, -Q.re) at
// the end.  FP32 partial sums are folded into FP64 every AH_FL tiles.
// ---------------------------------------------------------------------------------------
constexpr int AH_RT = 32;
constexpr int AH_FL = 16;

__device__ __forceinline__ long addr32(const ColSet &cs, long row, int col) {
    if (cs.col_off) return cs.col_off[col] + row;
    if (cs.ki == 1) return (long)col * cs.col_stride + row;
    return ((row >> 1) * cs.ki + col) * 2 + (row & 1);  // RHS-inner FP32 field (2 complex per chunk)
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 8 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}

__global__ void __launch_bounds__(AHB_THREADS) k_gemm_ahb32(ColSet A, ColSet B, long nrows, double *partials,
                                                            unsigned *counter, double *C) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int nA = A.ncols, nB = B.ncols;
    const int tile_el = AH_RT * (nA + nB);
    float2 *buf0 = reinterpret_cast<float2 *>(sm_raw);  // [RT][nA] then [RT][nB]
    float2 *buf1 = buf0 + tile_el;
    double *tot = reinterpret_cast<double *>(buf1 + tile_el);  // [16 outputs][2][256 threads]
    const float2 *Ab = static_cast<const float2 *>(A.base);
    const float2 *Bb = static_cast<const float2 *>(B.base);
    const int t = threadIdx.x;
    const int a0 = t % 64, b0 = t / 64;
    float2 P[4][4], Q[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) P[i][j] = Q[i][j] = make_float2(0.f, 0.f);
    for (int q = 0; q < 32; q++) tot[q * AHB_THREADS + t] = 0.0;
    const long ntiles = (nrows + AH_RT - 1) / AH_RT;
    auto issue = [&](long tile, float2 *dst) {
        const long r0 = tile * AH_RT;
        for (int L = t; L < tile_el; L += AHB_THREADS) {
            const int isA = L < AH_RT * nA;
            const int L2 = isA ? L : L - AH_RT * nA;
            const int rr = L2 % AH_RT, c = L2 / AH_RT;
            const long row = r0 + rr;
            const bool ok = row < nrows;
            const float2 *src = isA ? Ab + (ok ? addr32(A, row, c) : 0) : Bb + (ok ? addr32(B, row, c) : 0);
            float2 *d = isA ? dst + rr * nA + c : dst + AH_RT * nA + rr * nB + c;
            cp_async8(d, src, ok);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    long tile = blockIdx.x;
    int which = 0;
    if (tile < ntiles) issue(tile, buf0);
    int since = 0;
    for (; tile < ntiles; tile += gridDim.x) {
        float2 *cur = which ? buf1 : buf0;
        if (tile + gridDim.x < ntiles) {
            issue(tile + gridDim.x, which ? buf0 : buf1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        const float2 *As = cur;
        const float2 *Bs = cur + AH_RT * nA;
#pragma unroll 4
        for (int rr = 0; rr < AH_RT; rr++) {
            float2 bv[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int b = b0 + 4 * j;
                bv[j] = b < nB ? Bs[rr * nB + b] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int a = a0 + 64 * i;
                if (a >= nA) continue;
                const float2 av = As[rr * nA + a];
                const float2 ar = make_float2(av.x, av.x), ai = make_float2(av.y, av.y);
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    P[i][j] = __ffma2_rn(ar, bv[j], P[i][j]);
                    Q[i][j] = __ffma2_rn(ai, bv[j], Q[i][j]);
                }
            }
        }
        __syncthreads();
        which ^= 1;
        if (++since == AH_FL) {
            since = 0;
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int o = (i * 4 + j) * 2;
                    tot[o * AHB_THREADS + t] += (double)P[i][j].x + (double)Q[i][j].y;
                    tot[(o + 1) * AHB_THREADS + t] += (double)P[i][j].y - (double)Q[i][j].x;
                    P[i][j] = Q[i][j] = make_float2(0.f, 0.f);
                }
        }
    }
    double *Pp = partials + (long)blockIdx.x * nA * nB * 2;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int a = a0 + 64 * i, b = b0 + 4 * j;
            const int o = (i * 4 + j) * 2;
            if (a < nA && b < nB) {
                Pp[(a * nB + b) * 2] = tot[o * AHB_THREADS + t] + (double)P[i][j].x + (double)Q[i][j].y;
                Pp[(a * nB + b) * 2 + 1] = tot[(o + 1) * AHB_THREADS + t] + (double)P[i][j].y - (double)Q[i][j].x;
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
        double sum = 0.0;
        for (unsigned b = 0; b < gridDim.x; b++) sum += __ldcg(partials + (long)b * nout + o);
        C[o] = sum;
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
        const size_t smem32 = (size_t)2 * AH_RT * (A.ncols + B.ncols) * 8 + (size_t)AHB_THREADS * 32 * 8;
        long g2 = (long)device_sm_count() * 2;
        const long nt = (nrows + AH_RT - 1) / AH_RT;
        if (g2 > nt) g2 = nt;
        if (g2 > cap) g2 = cap;
        cudaFuncSetAttribute(k_gemm_ahb32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32);
        k_gemm_ahb32<<<(int)g2, AHB_THREADS, smem32, s>>>(A, B, nrows, red.partials, red.counter, C);
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

// NO: compile-time bound on the number of outputs (8, 16 or 32) so that the
// per-thread accumulators fit in registers
template <typename T, int NO>
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
    T ws_re[NO], ws_im[NO];
#pragma unroll
    for (int c = 0; c < NO; c++) ws_re[c] = ws_im[c] = 0;
    for (long row = (long)blockIdx.x * blockDim.x + threadIdx.x; row < nrows; row += (long)gridDim.x * blockDim.x) {
        T re[NO], im[NO];
#pragma unroll
        for (int c = 0; c < NO; c++) re[c] = im[c] = 0;
        for (int a = 0; a < m; a++) {
            const V2 v = base[Vw.col_off[a] + row];
#pragma unroll
            for (int c = 0; c < NO; c++) {
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
        for (int c = 0; c < NO; c++) {
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

// FP32 restart, second form: thread per row; slot offsets and QZ in shared memory;
// out[c] = sum_a v_a q_ac accumulated as two packed sums P = sum re(v) q, R = sum
// im(v) q (out = P + i R), four column loads in flight per thread.
template <int NO>
__global__ void __launch_bounds__(WR_THREADS) k_window_restart32(ColSet Vw, int m, const double *QZ, int nout,
                                                                 const float2 *t, const float2 *tp,
                                                                 const double *beta_dev, long nrows,
                                                                 double *partials, unsigned *counter, double *wv) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    float2 *Qs = reinterpret_cast<float2 *>(sm_raw);          // [m][NO]
    long *off = reinterpret_cast<long *>(Qs + (size_t)m * NO);  // [m]
    __shared__ double red[(WR_THREADS / 32) * 2];
    for (int L = threadIdx.x; L < m * NO; L += blockDim.x) {
        const int a = L / NO, c = L % NO;
        Qs[L] = c < nout ? make_float2((float)QZ[2 * (a * nout + c)], (float)QZ[2 * (a * nout + c) + 1])
                         : make_float2(0.f, 0.f);
    }
    for (int a = threadIdx.x; a < m; a += blockDim.x) off[a] = Vw.col_off[a];
    __syncthreads();
    const float beta = (float)(*beta_dev);
    float2 *base = static_cast<float2 *>(Vw.base);
    float2 ws[NO];
#pragma unroll
    for (int c = 0; c < NO; c++) ws[c] = make_float2(0.f, 0.f);
    for (long row = (long)blockIdx.x * blockDim.x + threadIdx.x; row < nrows; row += (long)gridDim.x * blockDim.x) {
        float2 P[NO], R[NO];
#pragma unroll
        for (int c = 0; c < NO; c++) P[c] = R[c] = make_float2(0.f, 0.f);
        int a = 0;
        for (; a + 4 <= m; a += 4) {
            float2 v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) v[u] = base[off[a + u] + row];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const float2 vr = make_float2(v[u].x, v[u].x), vi = make_float2(v[u].y, v[u].y);
#pragma unroll
                for (int c = 0; c < NO; c++) {
                    const float2 q = Qs[(a + u) * NO + c];
                    P[c] = __ffma2_rn(vr, q, P[c]);
                    R[c] = __ffma2_rn(vi, q, R[c]);
                }
            }
        }
        for (; a < m; a++) {
            const float2 v = base[off[a] + row];
            const float2 vr = make_float2(v.x, v.x), vi = make_float2(v.y, v.y);
#pragma unroll
            for (int c = 0; c < NO; c++) {
                const float2 q = Qs[a * NO + c];
                P[c] = __ffma2_rn(vr, q, P[c]);
                R[c] = __ffma2_rn(vi, q, R[c]);
            }
        }
        const float2 tt = t[row], tq = tp[row];
        const float wr = tt.x - beta * tq.x, wi = tt.y - beta * tq.y;
#pragma unroll
        for (int c = 0; c < NO; c++) {
            if (c < nout) {
                const float2 o = make_float2(P[c].x - R[c].y, P[c].y + R[c].x);  // P + i R
                base[off[c] + row] = o;
                // conj(w) * o
                ws[c] = __ffma2_rn(make_float2(wr, wr), o, ws[c]);
                ws[c] = __ffma2_rn(make_float2(wi, wi), make_float2(o.y, -o.x), ws[c]);
            }
        }
    }
    double *Pp = partials + (long)blockIdx.x * nout * 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = 0; c < nout; c++) {
        double vr = 0.0, vi = 0.0;
#pragma unroll
        for (int cc = 0; cc < NO; cc++)
            if (cc == c) {
                vr = (double)ws[cc].x;
                vi = (double)ws[cc].y;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vr += __shfl_xor_sync(0xffffffffu, vr, o);
            vi += __shfl_xor_sync(0xffffffffu, vi, o);
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
            Pp[c * 2] = sr;
            Pp[c * 2 + 1] = si;
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
        double sum = 0.0;
        for (unsigned b = 0; b < gridDim.x; b++) sum += __ldcg(partials + (long)b * nout * 2 + o);
        wv[o] = sum;
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
#define EIG_WR(T, NO)                                                                                   \
    do {                                                                                                \
        cudaFuncSetAttribute(k_window_restart<T, NO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        k_window_restart<T, NO><<<(int)grid, WR_THREADS, smem, s>>>(Vw, m, QZ, nout, t, t_prev, beta_dev, nrows, \
                                                                  red.partials, red.counter, wv);        \
    } while (0)
    if (Vw.f64) {
        if (nout <= 8) EIG_WR(double, 8);
        else if (nout <= 16) EIG_WR(double, 16);
        else EIG_WR(double, 32);
    } else {
#define EIG_WR32(NO)                                                                                       \
    do {                                                                                                   \
        const size_t sm32 = (size_t)m * NO * 8 + (size_t)m * 8;                                            \
        cudaFuncSetAttribute(k_window_restart32<NO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32); \
        k_window_restart32<NO><<<(int)grid, WR_THREADS, sm32, s>>>(Vw, m, QZ, nout, static_cast<const float2 *>(t), \
                                                                 static_cast<const float2 *>(t_prev), beta_dev, nrows, \
                                                                 red.partials, red.counter, wv);            \
    } while (0)
        if (nout <= 8) EIG_WR32(8);
        else if (nout <= 16) EIG_WR32(16);
        else if (nout <= 24) EIG_WR32(24);
        else EIG_WR32(32);
#undef EIG_WR32
    }
#undef EIG_WR
    return cudaGetLastError();
}

// wv[c] = sum over rows of conj(w) V[:, c] for c < nout, w = t - beta t_prev formed on
// the fly (FP32 fields, V columns at `off` in complex units; beta read from the
// device): Fig. 1 step 11.8 after a restart whose V <- V QZ ran elsewhere.  FP32
// products per thread, FP64 block sums, the grid's sums added in a fixed order.
namespace {
template <int NO>
__global__ void __launch_bounds__(WR_THREADS) k_wdot(const float2 *__restrict__ t, const float2 *__restrict__ tp,
                                                     const double *beta_dev, const float2 *base, const long *off,
                                                     int nout, long nrows, double *partials, unsigned *counter,
                                                     double *wv) {
    __shared__ double red[(WR_THREADS / 32) * 2];
    const float beta = (float)(*beta_dev);
    float2 ws[NO];
#pragma unroll
    for (int c = 0; c < NO; c++) ws[c] = make_float2(0.f, 0.f);
    for (long row = (long)blockIdx.x * blockDim.x + threadIdx.x; row < nrows; row += (long)gridDim.x * blockDim.x) {
        const float2 tv = t[row], pv = tp[row];
        const float wr = tv.x - beta * pv.x, wi = tv.y - beta * pv.y;
#pragma unroll
        for (int c = 0; c < NO; c++)
            if (c < nout) {
                const float2 o = base[off[c] + row];
                ws[c] = __ffma2_rn(make_float2(wr, wr), o, ws[c]);                      // conj(w) * o
                ws[c] = __ffma2_rn(make_float2(wi, wi), make_float2(o.y, -o.x), ws[c]);
            }
    }
    double *Pp = partials + (long)blockIdx.x * nout * 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = 0; c < nout; c++) {
        double vr = 0.0, vi = 0.0;
#pragma unroll
        for (int cc = 0; cc < NO; cc++)
            if (cc == c) {
                vr = (double)ws[cc].x;
                vi = (double)ws[cc].y;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vr += __shfl_xor_sync(0xffffffffu, vr, o);
            vi += __shfl_xor_sync(0xffffffffu, vi, o);
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
            Pp[c * 2] = sr;
            Pp[c * 2 + 1] = si;
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
        double sum = 0.0;
        for (unsigned b = 0; b < gridDim.x; b++) sum += __ldcg(partials + (long)b * nout * 2 + o);
        wv[o] = sum;
    }
    if (threadIdx.x == 0) *counter = 0u;
}
}  // namespace

cudaError_t launch_wdot(const void *t, const void *t_prev, const double *beta_dev, const void *base, const long *off,
                        int nout, long nrows, double *wv, RedScratch red, cudaStream_t s) {
    if (nout < 1 || nout > 32) return cudaErrorInvalidValue;
    ProfScope prof("wdot", (double)nrows * (nout + 2) * 8.0, s);
    long grid = (nrows + WR_THREADS - 1) / WR_THREADS;
    long cap = (long)device_sm_count() * 4;
    if (grid > cap) grid = cap;
    const long pcap = (long)red.max_blocks * MAX_RHS * 64 / (nout * 2);
    if (grid > pcap) grid = pcap;
    auto t2 = static_cast<const float2 *>(t), p2 = static_cast<const float2 *>(t_prev);
    auto b2 = static_cast<const float2 *>(base);
#define EIG_WD(NO) \
    k_wdot<NO><<<(int)grid, WR_THREADS, 0, s>>>(t2, p2, beta_dev, b2, off, nout, nrows, red.partials, red.counter, wv)
    if (nout <= 8) EIG_WD(8);
    else if (nout <= 16) EIG_WD(16);
    else if (nout <= 24) EIG_WD(24);
    else EIG_WD(32);
#undef EIG_WD
    return cudaGetLastError();
}

}  // namespace eig
