// Tensor-core (tcgen05) C = U^H R for the deflation of a batch of RHS (Eq. 1):
// U the basis (l FP32 fields), R one RHS-inner FP32 field of k RHS.
//
// Real form.  With the complex vectors stored as interleaved (re, im) floats the
// reduction runs over K = 2N real rows:
//   Re C = sum_K U'[K, a] B1[K, c],   B1 = (re R, im R) interleaved
//   Im C = sum_K U'[K, a] B2[K, c],   B2 = (im R, -re R) interleaved
// so one GEMM D = U'^T [B1 B2] (M = l basis vectors, N = 2k, K = 2N) gives both.
// Both operands are K-major: U's columns run along K (TMA-loaded, 128-byte
// swizzle), the B tile is written by the threads from the RHS-inner field.
//
// Precision.  kind::tf32 keeps 10 mantissa bits, so each operand is split into
// hi = (x with its low 13 mantissa bits cleared) and lo = x - hi, and D =
// hi*hi + hi*lo + lo*hi (three MMAs per K step): products at about FP32 accuracy.
// The tensor pipe's own FP32 accumulation loses accuracy with the length of the
// sum (measured at 10.6M complex rows: relative error 1e-6 after 2 K tiles per
// accumulator, 3e-5 after 128), so TMEM holds two accumulators used by alternate
// groups of two K tiles; each finished group is drained into per-thread
// double-float (TwoSum) sums while the next group accumulates.  Each CTA writes
// its sums as FP64 partials; a second kernel adds the partials in a fixed order.
//
// Pipeline per CTA (128 threads): thread 0 issues the TMA loads of up to STAGES
// K tiles ahead; all threads split the A tile in place and build the B tile;
// thread 0 issues the MMAs and commits them to the stage's "empty" barrier.
// Every wait is bounded: on timeout the CTA records an error, drains its copies
// (bounded), frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "kernels.cuh"
#include "prof.h"

namespace eig {

namespace {

constexpr int KT = 32;            // K floats per tile: one 128-byte swizzle row
constexpr int TM = 128;           // M rows per tile
constexpr int STAGES = 3;
constexpr int THREADS = 128;
constexpr int MAX_CHUNK = 1 << 20;  // K tiles per CTA at most (no cap unless EIG_TC_CHUNK)
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, unsigned phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sa(b)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait: gives up after WAIT_NS nanoseconds of wall time
__device__ __noinline__ bool mbar_wait(uint64_t *b, unsigned phase) {
    if (mbar_try(b, phase)) return true;
    const uint64_t t0 = gtimer();
    for (;;) {
        for (int i = 0; i < 256; i++)
            if (mbar_try(b, phase)) return true;
        if (gtimer() - t0 > WAIT_NS) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(sa(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(sa(bar))
        : "memory");
}

// 64-bit shared memory descriptor of a K-major tile with 128-byte swizzle:
// start >> 4 in [0,14), leading offset (unused here) >> 4 in [16,30), stride offset
// (1024 B between 8-row groups) >> 4 in [32,46), descriptor version 1 in [46,48),
// layout type 2 (128-byte swizzle) in [61,64).
__device__ __forceinline__ uint64_t sdesc(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// instruction descriptor, kind::tf32: D F32 [4,6)=1, A TF32 [7,10)=2, B TF32 [10,13)=2,
// both K-major (bits 15, 16 = 0), N >> 3 in [17,23), M >> 4 in [24,29)
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sa(bar))
                 : "memory");
}

__device__ __forceinline__ float hi_tf32(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// byte offset of element (row r, float e) in a K-major 128-byte-swizzled tile
__device__ __forceinline__ uint32_t sw128(int r, int e) {
    const int chunk = e >> 2;
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((chunk ^ (r & 7)) << 4) + ((e & 3) << 2));
}

struct TcArgs {
    // B operand: complex (row n, column c) at ((n >> 1) * ki + c % ki) * 2 + (n & 1) + (c / ki) * bcol
    // in float2 units (ki = k, bcol = 0: RHS-inner field; ki = 1: one field per column)
    const float2 *R;
    int ki;
    long bcol;
    long nrows;        // complex rows N
    int l, k;          // columns of A and of B
    int ktiles;        // total K tiles
    int chunk;         // K tiles per CTA
    double *partials;  // [grid][MT * 128][N]
    int *err;
};

// s += x in double-float (hi, lo) with Knuth's TwoSum (exact error of the FP32 sum)
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// D regions: two TMEM accumulators of MT * N columns used by alternate groups of
// FLUSH K tiles; a group's result is drained into per-thread double-float sums
// while the next group accumulates in the other region.  The tensor pipe adds in
// FP32 with its own rounding, so its error grows with the accumulation length:
// draining every FLUSH tiles keeps the result at FP32-product accuracy.
constexpr int FLUSH = 2;

template <int MT, int N>
__device__ __forceinline__ void drain(uint32_t region, int warp, float *acc_hi, float *acc_lo) {
#pragma unroll
    for (int c0 = 0; c0 < MT * N; c0 += 16) {
        uint32_t v[16];
        const uint32_t addr = region + ((uint32_t)(warp * 32) << 16) + c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(addr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; j++) two_sum_add(acc_hi[c0 + j], acc_lo[c0 + j], __uint_as_float(v[j]));
    }
}

template <int MT, int N>
__global__ void __launch_bounds__(THREADS, 1) k_tc_ahb(const __grid_constant__ CUtensorMap tmap, const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    // 1024-byte aligned stage buffers: [MT] A_hi tiles, [MT] A_lo tiles, B_hi, B_lo
    unsigned char *base = sm_raw + ((1024 - (sa(sm_raw) & 1023)) & 1023);
    constexpr uint32_t a_bytes = TM * KT * 4;  // 16 KB
    constexpr uint32_t b_bytes = (uint32_t)((N + 7) / 8) * 1024;
    constexpr uint32_t stage_bytes = 2 * MT * a_bytes + 2 * b_bytes;
    constexpr uint32_t NCOLS = 2 * MT * N <= 32 ? 32 : (2 * MT * N <= 64 ? 64 : 128);
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], dfull[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int kt0 = blockIdx.x * a.chunk;
    const int nkt = min(a.chunk, a.ktiles - kt0);
    if (t == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&dfull[0], 1);
        mbar_init(&dfull[1], 1);
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sa(&tmem_base)),
                     "r"(NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;
    auto region = [&](int g) { return tmem + (uint32_t)((g & 1) * MT * N); };
    auto A_hi = [&](int s, int mt) { return base + s * stage_bytes + mt * a_bytes; };
    auto A_lo = [&](int s, int mt) { return base + s * stage_bytes + (MT + mt) * a_bytes; };
    auto B_hi = [&](int s) { return base + s * stage_bytes + 2 * MT * a_bytes; };
    auto B_lo = [&](int s) { return base + s * stage_bytes + 2 * MT * a_bytes + b_bytes; };
    auto issue = [&](int kt) {  // thread 0 only
        const int s = kt % STAGES;
        mbar_expect_tx(&full[s], MT * a_bytes);
        for (int mt = 0; mt < MT; mt++) tma_load_2d(A_hi(s, mt), &tmap, (kt0 + kt) * KT, mt * TM, &full[s]);
    };
    float acc_hi[MT * N], acc_lo[MT * N];
#pragma unroll
    for (int c = 0; c < MT * N; c++) acc_hi[c] = acc_lo[c] = 0.f;
    int issued = 0;
    if (t == 0)
        for (; issued < STAGES - 1 && issued < nkt; issued++) issue(issued);
    const uint32_t idesc = idesc_tf32(TM, N);
    int consumed = 0;
    for (int kt = 0; kt < nkt; kt++) {
        const int s = kt % STAGES;
        if (!mbar_wait(&full[s], (kt / STAGES) & 1)) {
            atomicExch(a.err, 2);
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) break;
        consumed = kt + 1;
        // split A in place: hi (low mantissa bits cleared), lo = x - hi
        for (int mt = 0; mt < MT; mt++) {
            float4 *ah = reinterpret_cast<float4 *>(A_hi(s, mt));
            float4 *al = reinterpret_cast<float4 *>(A_lo(s, mt));
            for (int i = t; i < TM * KT / 4; i += THREADS) {
                const float4 v = ah[i];
                const float4 h = make_float4(hi_tf32(v.x), hi_tf32(v.y), hi_tf32(v.z), hi_tf32(v.w));
                ah[i] = h;
                al[i] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
            }
        }
        // B tile: rows c (B1) and k + c (B2), K positions 2n' and 2n' + 1 for complex row n'
        {
            const long n0 = (long)(kt0 + kt) * (KT / 2);
            unsigned char *bh = B_hi(s), *bl = B_lo(s);
            for (int i = 2 * a.k * KT + t; i < N * KT; i += THREADS) {  // zero padding rows
                const int r = i / KT, e = i % KT;
                *reinterpret_cast<float *>(bh + sw128(r, e)) = 0.f;
                *reinterpret_cast<float *>(bl + sw128(r, e)) = 0.f;
            }
            for (int i = t; i < (KT / 2) * a.k; i += THREADS) {
                // consecutive threads take consecutive addresses: RHS first in an RHS-inner
                // field, rows first when each column is a field of its own
                const int np = a.ki == 1 ? i % (KT / 2) : i / a.k;
                const int c = a.ki == 1 ? i / (KT / 2) : i % a.k;
                const long n = n0 + np;
                float2 v = make_float2(0.f, 0.f);
                if (n < a.nrows) v = a.R[((n >> 1) * a.ki + c % a.ki) * 2 + (n & 1) + (long)(c / a.ki) * a.bcol];
                const float vals[4] = {v.x, v.y, v.y, -v.x};  // B1 (re, im), B2 (im, -re)
                for (int q = 0; q < 4; q++) {
                    const int r = q < 2 ? c : a.k + c;
                    const int e = 2 * np + (q & 1);
                    const float h = hi_tf32(vals[q]);
                    *reinterpret_cast<float *>(bh + sw128(r, e)) = h;
                    *reinterpret_cast<float *>(bl + sw128(r, e)) = vals[q] - h;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        const int g = kt / FLUSH;
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            for (int mt = 0; mt < MT; mt++) {
                const uint32_t d = region(g) + mt * N;
                for (int ks = 0; ks < KT / 8; ks++) {
                    const uint32_t off = ks * 32;  // 8 tf32 = 32 bytes along the swizzled row
                    const uint64_t ah = sdesc(sa(A_hi(s, mt)) + off), al = sdesc(sa(A_lo(s, mt)) + off);
                    const uint64_t bh = sdesc(sa(B_hi(s)) + off), bl = sdesc(sa(B_lo(s)) + off);
                    const int acc0 = (kt % FLUSH != 0 || ks > 0) ? 1 : 0;
                    mma_tf32(d, ah, bh, idesc, acc0);
                    mma_tf32(d, ah, bl, idesc, 1);
                    mma_tf32(d, al, bh, idesc, 1);
                }
            }
            mma_commit(&empty[s]);
            if (kt % FLUSH == FLUSH - 1 || kt == nkt - 1) mma_commit(&dfull[g & 1]);
            // refill: tile kt + STAGES - 1 goes to the stage of tile kt - 1, whose MMAs
            // were issued one iteration ago
            if (issued < nkt) {
                if (issued >= STAGES && !mbar_wait(&empty[issued % STAGES], ((issued / STAGES) - 1) & 1)) {
                    atomicExch(a.err, 1);
                    abort_flag = 1;
                } else {
                    issue(issued);
                    issued++;
                }
            }
        }
        __syncwarp();
        // at the first tile of group g, the previous group's region is complete: drain it
        if (kt % FLUSH == 0 && g >= 1) {
            // tcgen05.ld is warp-collective: the warp drains only if all its lanes saw the group complete
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&dfull[(g - 1) & 1], ((g - 1) >> 1) & 1));
            if (!ok) {
                atomicExch(a.err, 4);
                abort_flag = 1;
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                drain<MT, N>(region(g - 1), warp, acc_hi, acc_lo);
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        }
    }
    // after an abort, let the loads still in flight land before the CTA exits
    if (t == 0)
        for (int j = consumed; j < issued; j++) mbar_wait(&full[j % STAGES], (j / STAGES) & 1);
    // all MMAs done
    if (t == 0) mma_commit(&done);
    __syncwarp();
    if (!mbar_wait(&done, 0)) {
        atomicExch(a.err, 3);
        abort_flag = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!abort_flag) {
        // the last group has not been drained yet
        drain<MT, N>(region((nkt - 1) / FLUSH), warp, acc_hi, acc_lo);
        double *P = a.partials + (long)blockIdx.x * MT * TM * N;
#pragma unroll
        for (int mt = 0; mt < MT; mt++) {
            const int row = mt * TM + warp * 32 + lane;
#pragma unroll
            for (int c = 0; c < N; c++)
                P[(long)row * N + c] = (double)acc_hi[mt * N + c] + (double)acc_lo[mt * N + c];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOLS) : "memory");
}

// C[a][c] = sum over CTAs of D[a][c] + i D[a][k + c], FP64, fixed order
__global__ void k_tc_reduce(const double *partials, int grid, int MT, int N, int l, int k, double *C) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= l * k) return;
    const int arow = idx / k, c = idx % k;
    double re = 0.0, im = 0.0;
    const long stride = (long)MT * TM * N;
    for (int g = 0; g < grid; g++) {
        const double *P = partials + g * stride + (long)arow * N;
        re += P[c];
        im += P[k + c];
    }
    C[2 * idx] = re;
    C[2 * idx + 1] = im;
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_enc_mu;

cudaError_t get_encoder() {
    std::lock_guard<std::mutex> lk(g_enc_mu);
    if (g_encode) return cudaSuccess;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || !fn || q != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return cudaSuccess;
}

}  // namespace

// K tiles per CTA: the tiles split evenly over about one CTA per SM, at most
// MAX_CHUNK (EIG_TC_CHUNK in the environment lowers the cap)
void tc_grid(long ktiles, int *chunk, int *grid) {
    const long target = device_sm_count();
    long cap = MAX_CHUNK;
    if (const char *e = getenv("EIG_TC_CHUNK")) {
        const long v = atol(e);
        if (v >= 1 && v < cap) cap = v;
    }
    long c = (ktiles + target - 1) / target;
    if (c > cap) c = cap;  // bounds the FP32 accumulation run in TMEM
    if (c < 1) c = 1;
    *chunk = (int)c;
    *grid = (int)((ktiles + c - 1) / c);
}

size_t tc_ahb_partials_bytes(long nrows, int l, int k) {
    const int MT = (l + TM - 1) / TM;
    const int N = ((2 * k + 15) / 16) * 16;
    const long ktiles = (2 * nrows + KT - 1) / KT;
    int chunk, grid;
    tc_grid(ktiles, &chunk, &grid);
    return (size_t)grid * MT * TM * N * sizeof(double);
}

bool tc_ahb_ok(const ColSet &A, const ColSet &B) {
    if (A.f64 || B.f64 || A.col_off || B.col_off || A.ki != 1) return false;
    if (A.ncols < 1 || A.ncols > 256 || B.ncols < 1 || B.ncols > 16) return false;
    if (((uintptr_t)A.base & 15) != 0 || ((A.col_stride * 8) % 16) != 0 || ((uintptr_t)B.base & 7) != 0) return false;
    if (B.ki == 1) return true;
    return B.ki == B.ncols && B.col_stride == 0;
}

// C (nA x nB complex FP64, row-major) = A^H B, A and B FP32 column sets (tc_ahb_ok)
cudaError_t launch_tc_ahb(const ColSet &A, const ColSet &B, long nrows, double *C, double *partials, int *err,
                          cudaStream_t s) {
    if (!tc_ahb_ok(A, B)) return cudaErrorInvalidValue;
    const float *U = static_cast<const float *>(A.base);
    const long ustride_floats = 2 * A.col_stride;
    const int l = A.ncols, k = B.ncols;
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    ProfScope prof("tc_gemm_ahb", (double)nrows * (l + k) * 8.0, s);
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * nrows), (cuuint64_t)l};
    const cuuint64_t strides[1] = {(cuuint64_t)ustride_floats * 4};
    const cuuint32_t box[2] = {KT, TM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(U), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    TcArgs a;
    a.R = static_cast<const float2 *>(B.base);
    a.ki = B.ki;
    a.bcol = B.col_stride;
    a.nrows = nrows;
    a.l = l;
    a.k = k;
    const int MT = (l + TM - 1) / TM;
    const int N = ((2 * k + 15) / 16) * 16;
    a.ktiles = (int)((2 * nrows + KT - 1) / KT);
    a.partials = partials;
    a.err = err;
    int grid = 0;
    tc_grid(a.ktiles, &a.chunk, &grid);
    const size_t stage = 2 * MT * (size_t)(TM * KT * 4) + 2 * (size_t)((N + 7) / 8) * 1024;
    const size_t smem = STAGES * stage + 1024;
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, THREADS, smem, s>>>(map, a);
    };
    if (MT == 1 && N == 16) go(k_tc_ahb<1, 16>);
    else if (MT == 1) go(k_tc_ahb<1, 32>);
    else if (N == 16) go(k_tc_ahb<2, 16>);
    else go(k_tc_ahb<2, 32>);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n = l * k;
    k_tc_reduce<<<(n + 127) / 128, 128, 0, s>>>(partials, grid, MT, N, l, k, C);
    return cudaGetLastError();
}

}  // namespace eig
