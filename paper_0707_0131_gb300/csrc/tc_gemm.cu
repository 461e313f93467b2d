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
// hi = (x with its low 13 mantissa bits cleared) and lo = x - hi, and D = A_hi B +
// A_lo B with B = [B_hi B_lo] taken as one operand of width 2N (B_lo's rows follow
// B_hi's), two MMAs per K step whose halves are added when drained: products at about
// FP32 accuracy.
// The tensor pipe's own FP32 accumulation loses accuracy with the length of the
// sum (measured at 10.6M complex rows: relative error 1e-6 after 2 K tiles per
// accumulator, 3e-5 after 128), so TMEM holds two accumulators used by alternate
// groups of two K tiles; each finished group is drained into per-thread
// double-float (TwoSum) sums while the next group accumulates.  Each CTA writes
// its sums as FP64 partials; a second kernel adds the partials in a fixed order.
//
// Roles per CTA (320 threads): one lane of warp 0 keeps the TMA ring full, one lane
// of warp 1 issues the MMAs, warps 2..9 split the tiles and drain the accumulators;
// they hand stages and TMEM regions to each other through mbarriers.  Every wait is
// bounded: on timeout the CTA records an error, lets its copies land (bounded), frees
// its TMEM and returns.
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
constexpr int MAX_CHUNK = 1 << 20;  // K tiles per CTA at most (no cap unless EIG_TC_CHUNK)
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(sa(b)) : "memory");
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
// non-blocking test of the same phase (no suspension, for the fast path of a wait that
// usually finds the phase complete)
__device__ __forceinline__ bool mbar_test(uint64_t *b, unsigned phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
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
// bounded wait: gives up after limit_ns nanoseconds of wall time (WAIT_NS by default)
__device__ __noinline__ bool mbar_wait(uint64_t *b, unsigned phase, uint64_t limit_ns = WAIT_NS) {
    if (mbar_try(b, phase)) return true;
    const uint64_t t0 = gtimer();
    for (;;) {
        for (int i = 0; i < 256; i++)
            if (mbar_try(b, phase)) return true;
        if (gtimer() - t0 > limit_ns) return false;
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
// the same with A read from tensor memory (M = 128 rows in the 128 lanes, one 32-bit
// column per K element; a K step of 8 advances the address by 8 columns)
__device__ __forceinline__ void mma_tf32_ts(uint32_t dtmem, uint32_t atmem, uint64_t bdesc, uint32_t idesc, int accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtmem),
        "r"(atmem), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
// 32 consecutive TMEM columns of this thread's lane (its warp's lane quarter) from registers
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float *x) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
        "f"(x[0]), "f"(x[1]), "f"(x[2]), "f"(x[3]), "f"(x[4]), "f"(x[5]), "f"(x[6]), "f"(x[7]), "f"(x[8]), "f"(x[9]),
        "f"(x[10]), "f"(x[11]), "f"(x[12]), "f"(x[13]), "f"(x[14]), "f"(x[15]), "f"(x[16]), "f"(x[17]), "f"(x[18]),
        "f"(x[19]), "f"(x[20]), "f"(x[21]), "f"(x[22]), "f"(x[23]), "f"(x[24]), "f"(x[25]), "f"(x[26]), "f"(x[27]),
        "f"(x[28]), "f"(x[29]), "f"(x[30]), "f"(x[31])
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
    // test hook (EIG_TEST_INJECT_WAIT): CTA 0 first waits, for at most inject_ns, on an
    // mbarrier that nothing arrives on, then takes the give-up path before any copy is
    // issued, so that the error status can be exercised without a real stall
    uint64_t inject_ns;
};

// s += x in double-float (hi, lo) with Knuth's TwoSum (exact error of the FP32 sum)
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// Warp specialisation: warp 0 (one lane) keeps the TMA ring full, warp 1 (one lane)
// issues the MMAs, warps 2..9 split the A tiles in place into hi / lo, build the B
// tiles and drain the accumulators.  The roles hand stages and TMEM regions to each
// other through mbarriers only, so no role waits for work that was issued just
// before (a block-wide barrier per tile made every tile cost one MMA round trip).
//
// Accumulation: groups of FLUSH K tiles accumulate in one of NREG TMEM regions (MT * N
// columns each).  The tensor pipe adds in FP32 with its own rounding, so its error
// grows with the accumulation length; each finished group is drained into per-thread
// double-float sums, two groups behind the MMAs, and its region is then reused.
constexpr int FLUSH = 2;
constexpr int NREG = 3;
constexpr int WORKERS = 8;                    // worker warps
constexpr int TC_THREADS = 32 * (2 + WORKERS);
static_assert((KT / 2) * 16 <= 32 * WORKERS, "one B value per worker thread per tile for k <= 16");

// Worker warp w (warps 2..9) drains TMEM lanes 32 (w % 4) .. + 31 (the lane quarter a
// warp may access) and the half h = (w - 2) / 4 of the region's MT * N columns.
template <int MT, int N>
// A region holds, for M tile mt, A_mt B_hi in columns mt 2N + [0, N) and A_mt B_lo in
// mt 2N + N + [0, N); output column cc = mt N + c is the sum of the two.
__device__ __forceinline__ void drain(uint32_t region, int quarter, int half, float *acc_hi, float *acc_lo) {
    constexpr int HC = MT * N / 2;
    const uint32_t base = region + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
    for (int c0 = 0; c0 < HC; c0 += 8) {
        const int cc = half * HC + c0, mt = cc / N, c = cc % N;
        uint32_t v[8], w[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                     : "r"(base + (uint32_t)(mt * 2 * N + c))
                     : "memory");
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                     : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                     : "r"(base + (uint32_t)(mt * 2 * N + N + c))
                     : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; j++)
            two_sum_add(acc_hi[c0 + j], acc_lo[c0 + j], __uint_as_float(v[j]) + __uint_as_float(w[j]));
    }
}

template <int MT, int N, int NS>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_ahb(const __grid_constant__ CUtensorMap tmap, const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    // 1024-byte aligned stages: [MT] A tiles (TMA lands here, split in place to hi),
    // [MT] A_lo tiles, B_hi, B_lo
    unsigned char *base = sm_raw + ((1024 - (sa(sm_raw) & 1023)) & 1023);
    constexpr uint32_t a_bytes = TM * KT * 4;  // 16 KB
    constexpr uint32_t b_bytes = (uint32_t)((N + 7) / 8) * 1024;
    constexpr uint32_t stage_bytes = 2 * MT * a_bytes + 2 * b_bytes;
    constexpr uint32_t RCOLS = MT * 2 * N;  // per M tile: A B_hi, then A B_lo (drain adds them)
    constexpr uint32_t NCOLS =
        NREG * RCOLS <= 32 ? 32 : (NREG * RCOLS <= 64 ? 64 : (NREG * RCOLS <= 128 ? 128 : (NREG * RCOLS <= 256 ? 256 : 512)));
    static_assert(NREG * RCOLS <= 512, "TMEM columns");
    __shared__ __align__(8) uint64_t raw_full[NS], split_done[NS], stage_free[NS], acc_full[NREG], acc_empty[NREG],
        done, never;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ int n_issued, n_consumed;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int kt0 = blockIdx.x * a.chunk;
    const int nkt = min(a.chunk, a.ktiles - kt0);
    const int ngroups = (nkt + FLUSH - 1) / FLUSH;
    if (t == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(&raw_full[s], 1);
            mbar_init(&split_done[s], WORKERS);
            mbar_init(&stage_free[s], 1);
        }
        for (int r = 0; r < NREG; r++) {
            mbar_init(&acc_full[r], 1);
            mbar_init(&acc_empty[r], WORKERS);
        }
        mbar_init(&done, 1);
        mbar_init(&never, 1);
        abort_flag = 0;
        n_issued = 0;
        n_consumed = 0;
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
    auto region = [&](int g) { return tmem + (uint32_t)((g % NREG) * RCOLS); };
    auto A_hi = [&](int s, int mt) { return base + s * stage_bytes + mt * a_bytes; };
    auto A_lo = [&](int s, int mt) { return base + s * stage_bytes + (MT + mt) * a_bytes; };
    auto B_hi = [&](int s) { return base + s * stage_bytes + 2 * MT * a_bytes; };
    auto B_lo = [&](int s) { return base + s * stage_bytes + 2 * MT * a_bytes + b_bytes; };
    auto fail = [&](int code) {
        atomicExch(a.err, code);
        abort_flag = 1;
    };
    if (a.inject_ns && blockIdx.x == 0) {  // block-uniform
        if (t == 0 && !mbar_wait(&never, 0, a.inject_ns)) fail(7);
        __syncthreads();
    }

    if (warp == 0) {
        // ---------------- producer: TMA loads of the A tiles ----------------
        if (lane == 0) {
            int kt = 0;
            for (; kt < nkt && !abort_flag; kt++) {
                const int s = kt % NS;
                if (kt >= NS) {
                    const unsigned pf = ((kt / NS) - 1) & 1;
                    if (!mbar_test(&stage_free[s], pf) && !mbar_wait(&stage_free[s], pf)) {
                        fail(1);
                        break;
                    }
                }
                mbar_expect_tx(&raw_full[s], MT * a_bytes);
                for (int mt = 0; mt < MT; mt++) tma_load_2d(A_hi(s, mt), &tmap, (kt0 + kt) * KT, mt * TM, &raw_full[s]);
            }
            n_issued = kt;
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(TM, 2 * N);
            for (int kt = 0; kt < nkt && !abort_flag; kt++) {
                const int s = kt % NS, g = kt / FLUSH;
                const unsigned ps = (kt / NS) & 1;
                if (!mbar_test(&split_done[s], ps) && !mbar_wait(&split_done[s], ps)) {
                    fail(2);
                    break;
                }
                if (kt % FLUSH == 0 && g >= NREG) {
                    const unsigned pe = ((g / NREG) - 1) & 1;
                    if (!mbar_test(&acc_empty[g % NREG], pe) && !mbar_wait(&acc_empty[g % NREG], pe)) {
                        fail(3);
                        break;
                    }
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                // descriptors of the stage's tiles; a K step of 8 tf32 (32 bytes along the
                // swizzled row) adds 2 to the start-address field
                // B_lo's rows follow B_hi's: one MMA of width 2N takes A [B_hi B_lo]; per K step
                // A_hi [B_hi B_lo] + A_lo [B_hi B_lo] (the lo x lo term is below FP32 rounding)
                const uint64_t b0 = sdesc(sa(B_hi(s)));
#pragma unroll
                for (int mt = 0; mt < MT; mt++) {
                    const uint32_t d = region(g) + mt * 2 * N;
                    const uint64_t ah0 = sdesc(sa(A_hi(s, mt))), al0 = sdesc(sa(A_lo(s, mt)));
#pragma unroll
                    for (int ks = 0; ks < KT / 8; ks++) {
                        const uint64_t o = 2 * ks;
                        mma_tf32(d, ah0 + o, b0 + o, idesc, (kt % FLUSH != 0 || ks > 0) ? 1 : 0);
                        mma_tf32(d, al0 + o, b0 + o, idesc, 1);
                    }
                }
                mma_commit(&stage_free[s]);
                if (kt % FLUSH == FLUSH - 1 || kt == nkt - 1) mma_commit(&acc_full[g % NREG]);
            }
            mma_commit(&done);  // arrives once every MMA issued above has completed
        }
    } else {
        // ---------------- workers: split A, build B, drain ----------------
        const int wt = t - 64, quarter = warp & 3, half = (warp - 2) >> 2;
        constexpr int HC = MT * N / 2;
        float acc_hi[HC], acc_lo[HC];
#pragma unroll
        for (int c = 0; c < HC; c++) acc_hi[c] = acc_lo[c] = 0.f;
        // B values: worker thread wt < 16 k takes (row np, column c) of each tile; its value
        // for the next tile is loaded one tile ahead
        const int bnp = a.ki == 1 ? wt % (KT / 2) : wt / max(a.k, 1);
        const int bc = a.ki == 1 ? wt / (KT / 2) : wt % max(a.k, 1);
        const bool bth = wt < (KT / 2) * a.k;
        auto load_b = [&](int kt) {
            float2 v = make_float2(0.f, 0.f);
            const long n = (long)(kt0 + kt) * (KT / 2) + bnp;
            if (bth && kt < nkt && n < a.nrows)
                v = a.R[((n >> 1) * a.ki + bc % a.ki) * 2 + (n & 1) + (long)(bc / a.ki) * a.bcol];
            return v;
        };
        auto drain_group = [&](int g) {  // warp-uniform
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[g % NREG], (g / NREG) & 1));
            if (!ok) {
                fail(4);
                return false;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            drain<MT, N>(region(g), quarter, half, acc_hi, acc_lo);
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[g % NREG]);
            return true;
        };
        float2 bcur = load_b(0);
        int kt = 0;
        bool ok = true;
        for (; kt < nkt && ok && !abort_flag; kt++) {
            const int s = kt % NS, g = kt / FLUSH;
            const float2 bnext = load_b(kt + 1);
            if (!__all_sync(0xffffffffu, mbar_wait(&raw_full[s], (kt / NS) & 1))) {
                fail(5);
                break;
            }
            // split A in place: hi (low mantissa bits cleared), lo = x - hi
            for (int mt = 0; mt < MT; mt++) {
                float4 *ah = reinterpret_cast<float4 *>(A_hi(s, mt));
                float4 *al = reinterpret_cast<float4 *>(A_lo(s, mt));
                for (int i = wt; i < TM * KT / 4; i += 32 * WORKERS) {
                    const float4 v = ah[i];
                    const float4 h = make_float4(hi_tf32(v.x), hi_tf32(v.y), hi_tf32(v.z), hi_tf32(v.w));
                    ah[i] = h;
                    al[i] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
                }
            }
            // B tile: rows c (B1) and k + c (B2), K positions 2n' and 2n' + 1 for complex row n'
            unsigned char *bh = B_hi(s), *bl = B_lo(s);
            for (int i = 2 * a.k * KT + wt; i < N * KT; i += 32 * WORKERS) {  // zero padding rows
                const int r = i / KT, e = i % KT;
                *reinterpret_cast<float *>(bh + sw128(r, e)) = 0.f;
                *reinterpret_cast<float *>(bl + sw128(r, e)) = 0.f;
            }
            if (bth) {
                const float vals[4] = {bcur.x, bcur.y, bcur.y, -bcur.x};  // B1 (re, im), B2 (im, -re)
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int r = q < 2 ? bc : a.k + bc;
                    const int e = 2 * bnp + (q & 1);
                    const float h = hi_tf32(vals[q]);
                    *reinterpret_cast<float *>(bh + sw128(r, e)) = h;
                    *reinterpret_cast<float *>(bl + sw128(r, e)) = vals[q] - h;
                }
            }
            bcur = bnext;
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&split_done[s]);
            // drain the group two behind the one this tile starts
            if (kt % FLUSH == 0 && g >= 2) ok = drain_group(g - 2);
        }
        if (wt == 0) n_consumed = kt;
        if (ok && kt == nkt && !abort_flag) {
            // the last two groups
            for (int g = max(0, ngroups - 2); g < ngroups && ok; g++) ok = drain_group(g);
            if (ok) {
                double *P = a.partials + (long)blockIdx.x * MT * TM * N;
#pragma unroll
                for (int j = 0; j < HC; j++) {
                    const int col = half * HC + j;  // TMEM column within the region: mt * N + c
                    const int row = (col / N) * TM + quarter * 32 + lane;
                    P[(long)row * N + col % N] = (double)acc_hi[j] + (double)acc_lo[j];
                }
            }
        }
    }
    __syncthreads();
    if (t == 0) {
        // after an abort: let the loads still in flight land, and every MMA complete
        for (int j = n_consumed; j < n_issued; j++) mbar_wait(&raw_full[j % NS], (j / NS) & 1);
    }
    if (!mbar_wait(&done, 0)) atomicExch(a.err, 6);
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

// ------------------------------------------------------------------------------------
// Out = beta Out + A Y on the tensor cores (the U y of Eq. 1 and the basis updates of
// the growth step): D[n, (c, e)] = sum over K = (a, e') of A'[n, K] Yt[K, (c, e)], with
// M = 128 complex rows per tile, K = 2 * 16 basis columns per chunk (re, im of each)
// and N = 2k interleaved (re, im) output columns.  A job (one chunk of one tile) lands
// in shared memory as [16 columns][128 rows]: one 2D TMA copy when A's columns are
// evenly spaced, else one bulk copy per 1 KB column segment (window slots).  Worker
// threads read their row, split it into TF32 hi and lo and store both into tensor
// memory, where the MMAs read A (no shared-memory round trip for the split operand);
// Yt, split the same way, is built once per launch (k_ay_prep_b).  K <= 512, so one
// TMEM accumulator per tile stays at FP32-product accuracy without draining.
// ------------------------------------------------------------------------------------
template <int N>
struct AyStages {  // staging ring depth (copies in flight): 208 KB of shared memory with the B buffers
    static constexpr int value = N == 16 ? 12 : (N == 32 ? 11 : 9);
};
constexpr int AY_NOP = 4;         // operand buffers: A hi / lo in TMEM, B hi / lo in shared memory
constexpr int AY_TCOLS = 512;     // TMEM columns: 2 accumulators, then AY_NOP x (32 A_hi + 32 A_lo)
constexpr int AY_COLS = 16;       // basis columns per K chunk
constexpr int AY_THREADS = TC_THREADS;

struct AyArgs {
    const float2 *A;
    const long *aoff;  // column offsets (complex units) or null: column a at a * acol
    long acol;
    int nA;
    const double *Y;   // nA x k complex, row-major
    float2 *Out;       // (row n, column c) at ((n >> 1) * oki + c % oki) * 2 + (n & 1) + (c / oki) * ocol,
    int oki;           // or at ooff[c] + n when ooff is given (oki = 1)
    long ocol;
    const long *ooff;
    int k;
    float beta;
    long nrows;
    int mtiles, nch;   // M tiles, K chunks
    int *err;
    // B operand of every K chunk, split into TF32 hi and lo and laid out as the MMA reads
    // it (K-major, 128-byte swizzle): [chunk][hi, lo][N / 8 KB], built once per launch
    const unsigned char *Bpre;
    // A's columns evenly spaced (no aoff): one 2D TMA copy per job through the kernel's
    // tensor map instead of one bulk copy per column segment
    int tma;
};

// Builds AyArgs::Bpre from Y: row r = 2c + e of chunk kc's B tile holds, at K position
// 2 al + e' (basis column kc * AY_COLS + al, its re / im part e'), the real coefficient that
// turns (re, im) of U[n, col] into part e of output column c of the complex product U y
template <int N>
__global__ void k_ay_prep_b(const double *Y, int nA, int k, int nch, unsigned char *Bpre) {
    constexpr uint32_t b_bytes = (uint32_t)(N / 8) * 1024;
    const long total = (long)nch * N * KT;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int kc = (int)(idx / (N * KT)), rem = (int)(idx % (N * KT));
        const int r = rem / KT, kk = rem % KT, al = kk >> 1, ep = kk & 1, c = r >> 1, e = r & 1;
        const int col = kc * AY_COLS + al;
        float y = 0.f;
        if (c < k && col < nA) {
            const double yr = Y[2 * ((long)col * k + c)], yi = Y[2 * ((long)col * k + c) + 1];
            y = (float)(e == 0 ? (ep == 0 ? yr : -yi) : (ep == 0 ? yi : yr));
        }
        const float yh = hi_tf32(y);
        unsigned char *base = Bpre + (size_t)kc * 2 * b_bytes;
        *reinterpret_cast<float *>(base + sw128(r, kk)) = yh;
        *reinterpret_cast<float *>(base + b_bytes + sw128(r, kk)) = y - yh;
    }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(sa(dst)),
        "l"(src), "r"(bytes), "r"(sa(bar))
        : "memory");
}

// Roles: warp 0 issues the bulk copies, warp 1 the MMAs; warps 2..5 and 6..9 are two
// worker groups that take alternate jobs (a job = one K chunk of one tile): transpose and
// split the staged columns, copy in the chunk's B tile, and write the outputs of a tile
// whose last job was theirs one of their jobs later (two TMEM accumulators alternate
// between tiles).
template <int N>
__global__ void __launch_bounds__(AY_THREADS, 1) k_tc_ay(const __grid_constant__ CUtensorMap amap, const AyArgs a) {
    constexpr int AY_NSTG = AyStages<N>::value;
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char *base = sm_raw + ((1024 - (sa(sm_raw) & 1023)) & 1023);
    constexpr uint32_t stg_bytes = AY_COLS * TM * 8;            // 16 KB: [16 columns][128 rows] float2
    constexpr uint32_t b_bytes = (uint32_t)(N / 8) * 1024;
    constexpr uint32_t op_bytes = 2 * b_bytes;                   // B_hi, B_lo (A is in TMEM)
    // one accumulator holds A B_hi in its first N columns and A B_lo in the next N (B_lo's
    // rows follow B_hi's in shared memory, so one MMA of width 2N takes both)
    constexpr uint32_t ACOLS = 2 * N;                            // TMEM columns per accumulator
    constexpr uint32_t AC0 = 2 * ACOLS;                          // first A column in TMEM
    static_assert(AC0 + AY_NOP * 2 * KT <= AY_TCOLS, "TMEM columns");
    unsigned char *stg = base;
    unsigned char *ops = base + AY_NSTG * stg_bytes;
    __shared__ __align__(8) uint64_t stg_full[AY_NSTG], stg_free[AY_NSTG], op_ready[AY_NOP], op_free[AY_NOP],
        acc_full[2], acc_empty[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ int n_issued;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int my_tiles = a.mtiles > (int)blockIdx.x ? (a.mtiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int njobs = my_tiles * a.nch;
    if (t == 0) {
        // one worker group (WORKERS / 2 warps) reads, fills and drains each job or tile
        for (int i = 0; i < AY_NSTG; i++) {
            mbar_init(&stg_full[i], 1);
            mbar_init(&stg_free[i], WORKERS / 2);
        }
        for (int i = 0; i < AY_NOP; i++) {
            mbar_init(&op_ready[i], WORKERS / 2);
            mbar_init(&op_free[i], 1);
        }
        for (int i = 0; i < 2; i++) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], WORKERS / 2);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        n_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sa(&tmem_base)),
                     "r"(AY_TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;
    auto job_tile = [&](int j) { return (int)blockIdx.x + (j / a.nch) * (int)gridDim.x; };
    auto fail = [&](int code) {
        atomicExch(a.err, code);
        abort_flag = 1;
    };

    if (warp == 0) {
        // ---------------- producer: copies of the column segments ----------------
        // (one thread: slot, chunk and row position advance by counters, with no divisions
        // per job; a barrier that is already complete is taken without a call)
        if (lane == 0) {
            int j = 0, s = 0, kc = 0;
            unsigned lap = 0;  // j / AY_NSTG
            long n0 = (long)blockIdx.x * TM;
            for (; j < njobs; j++) {
                if (kc == 0 && abort_flag) break;
                if (lap > 0) {
                    const unsigned par = (lap - 1) & 1;
                    if (!mbar_test(&stg_free[s], par) && !mbar_wait(&stg_free[s], par)) {
                        fail(11);
                        break;
                    }
                    // the workers read this slot through the generic proxy; the copies write it
                    // through the async proxy
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                }
                const int c0 = kc * AY_COLS;
                if (a.tma) {
                    // box of 2 TM floats x AY_COLS columns, landing as [column][row] float2 like
                    // the bulk copies; rows and columns past the ends are filled with zeros and
                    // still counted, so the transaction is always the whole box.  x = 2 n0 is a
                    // multiple of 256 floats (1 KB).
                    mbar_expect_tx(&stg_full[s], stg_bytes);
                    tma_load_2d(stg + s * stg_bytes, &amap, (int)(2 * n0), c0, &stg_full[s]);
                } else {
                    const long rows = min((long)TM, a.nrows - n0);
                    const int nc = min(AY_COLS, a.nA - c0);
                    mbar_expect_tx(&stg_full[s], (unsigned)(nc * rows * 8));
                    for (int c = 0; c < nc; c++) {
                        const float2 *col = a.A + (a.aoff ? a.aoff[c0 + c] : (long)(c0 + c) * a.acol);
                        bulk_g2s(stg + s * stg_bytes + c * TM * 8, col + n0, (unsigned)(rows * 8), &stg_full[s]);
                    }
                }
                if (++s == AY_NSTG) {
                    s = 0;
                    lap++;
                }
                if (++kc == a.nch) {
                    kc = 0;
                    n0 += (long)gridDim.x * TM;
                }
            }
            n_issued = j;
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(TM, 2 * N);
            const uint64_t bdesc0 = sdesc(sa(ops));  // buffer o's B adds (o op_bytes) >> 4
            int o = 0, kc = 0, ti = 0;
            unsigned lap = 0;  // j / AY_NOP
            for (int j = 0; j < njobs; j++) {
                if (kc == 0 && abort_flag) break;
                const unsigned par = lap & 1;
                if (!mbar_test(&op_ready[o], par) && !mbar_wait(&op_ready[o], par)) {
                    fail(12);
                    break;
                }
                if (kc == 0 && ti >= 2) {
                    const unsigned pe = ((ti >> 1) - 1) & 1;
                    if (!mbar_test(&acc_empty[ti & 1], pe) && !mbar_wait(&acc_empty[ti & 1], pe)) {
                        fail(13);
                        break;
                    }
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t d = tmem + (uint32_t)((ti & 1) * ACOLS);
                const uint32_t ahi = tmem + AC0 + (uint32_t)(o * 2 * KT), alo = ahi + KT;
                const uint64_t b0 = bdesc0 + (uint64_t)(((uint32_t)o * op_bytes) >> 4);  // B_hi rows, then B_lo rows
                // per K step: A_hi [B_hi B_lo] + A_lo [B_hi B_lo], two MMAs of width 2N (the
                // lo x lo term is below FP32 rounding and harmless)
#pragma unroll
                for (int ks = 0; ks < KT / 8; ks++) {
                    const uint64_t bo = 2 * ks;  // 32 bytes along the swizzled row of B
                    const uint32_t ao = 8 * ks;  // 8 TMEM columns of A
                    mma_tf32_ts(d, ahi + ao, b0 + bo, idesc, (kc > 0 || ks > 0) ? 1 : 0);
                    mma_tf32_ts(d, alo + ao, b0 + bo, idesc, 1);
                }
                mma_commit(&op_free[o]);
                if (kc == a.nch - 1) mma_commit(&acc_full[ti & 1]);
                if (++o == AY_NOP) {
                    o = 0;
                    lap++;
                }
                if (++kc == a.nch) {
                    kc = 0;
                    ti++;
                }
            }
            mma_commit(&done);
        }
    } else {
        // ---------------- workers: two groups of four warps on alternate jobs ----------------
        // Each group covers the four TMEM lane quarters, so a group splits whole tiles and
        // writes whole outputs on its own; while one group waits (a barrier, its B loads, an
        // epilogue) the other splits the next job.
        const int grp = (warp - 2) >> 2, quarter = warp & 3;
        const int n = (t - 64) & (TM - 1);  // this thread's share of the B copy
        const int rt = quarter * 32 + lane;  // the tile row (TMEM lane) this thread splits
        constexpr int NB4 = (int)(2 * b_bytes / 16) / TM;  // float4 of B (hi, lo) per thread per job
        static_assert(NB4 * TM * 16 == (int)(2 * b_bytes), "B operand split evenly over a group");
        float4 bnext[NB4];
        auto load_b = [&](int j) {  // B of job j into registers, one job of this group ahead
            const float4 *src = reinterpret_cast<const float4 *>(a.Bpre + (size_t)(j % a.nch) * 2 * b_bytes);
#pragma unroll
            for (int i = 0; i < NB4; i++) bnext[i] = __ldg(src + n + TM * i);
        };
        // outputs of tile ti (rows n0 ..), from accumulator ti & 1; warp-uniform
        auto epilogue = [&](int ti) {
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[ti & 1], (ti >> 1) & 1));
            if (!ok) {
                fail(14);
                return false;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            uint32_t v[N];
            const uint32_t addr = tmem + (uint32_t)((ti & 1) * ACOLS) + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 16) {
                uint32_t w[16];  // the B_lo half of the same 16 columns
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                    "%15}, [%16];\n"
                    : "=r"(v[c0 + 0]), "=r"(v[c0 + 1]), "=r"(v[c0 + 2]), "=r"(v[c0 + 3]), "=r"(v[c0 + 4]),
                      "=r"(v[c0 + 5]), "=r"(v[c0 + 6]), "=r"(v[c0 + 7]), "=r"(v[c0 + 8]), "=r"(v[c0 + 9]),
                      "=r"(v[c0 + 10]), "=r"(v[c0 + 11]), "=r"(v[c0 + 12]), "=r"(v[c0 + 13]), "=r"(v[c0 + 14]),
                      "=r"(v[c0 + 15])
                    : "r"(addr + c0)
                    : "memory");
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                    "%15}, [%16];\n"
                    : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]),
                      "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]),
                      "=r"(w[15])
                    : "r"(addr + N + c0)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int q = 0; q < 16; q++) v[c0 + q] = __float_as_uint(__uint_as_float(v[c0 + q]) + __uint_as_float(w[q]));
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ti & 1]);
            const long row = (long)((int)blockIdx.x + ti * (int)gridDim.x) * TM + quarter * 32 + lane;
            if (row < a.nrows) {
                // columns in groups of 8: a group's addresses and (beta != 0) old values are all
                // read before its first store, so that those loads overlap instead of each
                // waiting behind the previous store
                constexpr int CG = 8;
#pragma unroll
                for (int c0 = 0; c0 < N / 2; c0 += CG) {
                    float2 *op[CG];
#pragma unroll
                    for (int q = 0; q < CG; q++) {
                        const int c = c0 + q;
                        op[q] = c >= a.k ? nullptr
                                : a.ooff ? a.Out + a.ooff[c] + row
                                         : a.Out + ((row >> 1) * a.oki + c % a.oki) * 2 + (row & 1) + (long)(c / a.oki) * a.ocol;
                    }
                    float2 r[CG];
#pragma unroll
                    for (int q = 0; q < CG; q++)
                        r[q] = make_float2(__uint_as_float(v[2 * (c0 + q)]), __uint_as_float(v[2 * (c0 + q) + 1]));
                    if (a.beta != 0.f) {
                        float2 old[CG];
#pragma unroll
                        for (int q = 0; q < CG; q++) old[q] = op[q] ? *op[q] : make_float2(0.f, 0.f);
#pragma unroll
                        for (int q = 0; q < CG; q++) {
                            r[q].x += a.beta * old[q].x;
                            r[q].y += a.beta * old[q].y;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < CG; q++)
                        if (op[q]) *op[q] = r[q];
                }
            }
            return true;
        };
        int pending = -1;  // tile whose outputs are still to be written (its last job was this group's)
        bool ok = true;
        if (grp < njobs) load_b(grp);
        for (int j = grp; j < njobs && ok && !abort_flag; j += 2) {
            const int s = j % AY_NSTG, o = j % AY_NOP, kc = j % a.nch;
            const long n0 = (long)job_tile(j) * TM;
            const long rows = min((long)TM, a.nrows - n0);
            const int nc = min(AY_COLS, a.nA - kc * AY_COLS);
            if (!__all_sync(0xffffffffu, (mbar_test(&stg_full[s], (j / AY_NSTG) & 1) || mbar_wait(&stg_full[s], (j / AY_NSTG) & 1)))) {
                fail(15);
                break;
            }
            if (j >= AY_NOP && !__all_sync(0xffffffffu, (mbar_test(&op_free[o], ((j / AY_NOP) - 1) & 1) || mbar_wait(&op_free[o], ((j / AY_NOP) - 1) & 1)))) {
                fail(16);
                break;
            }
            unsigned char *Bhi = ops + o * op_bytes;
            {
                // transpose + split: thread rt takes the 16 staged columns of row rt (K positions
                // 2c, 2c + 1 for column c) and writes hi and lo to 32 TMEM columns each of its lane
                const float2 *sg = reinterpret_cast<const float2 *>(stg + s * stg_bytes);
                float hv[KT], lv[KT];
#pragma unroll
                for (int c = 0; c < AY_COLS; c++) {
                    float2 x = make_float2(0.f, 0.f);
                    if (c < nc && rt < rows) x = sg[c * TM + rt];
                    hv[2 * c] = hi_tf32(x.x);
                    hv[2 * c + 1] = hi_tf32(x.y);
                    lv[2 * c] = x.x - hv[2 * c];
                    lv[2 * c + 1] = x.y - hv[2 * c + 1];
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&stg_free[s]);  // the staging slot has been read
                // the MMAs that read this buffer's previous contents have completed (op_free)
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + AC0 + (uint32_t)(o * 2 * KT);
                tmem_st32(ta, hv);
                tmem_st32(ta + KT, lv);
                asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
            }
            // B = Yt for this chunk (hi, then lo, contiguous as in Bpre), from the registers
            // loaded one job ahead; then the loads for this group's next job
            {
                float4 *dst = reinterpret_cast<float4 *>(Bhi);
#pragma unroll
                for (int i = 0; i < NB4; i++) dst[n + TM * i] = bnext[i];
            }
            if (j + 2 < njobs) load_b(j + 2);
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&op_ready[o]);
            // this group's previous tile, one of its jobs after that tile's last MMA was issued
            if (pending >= 0) {
                ok = epilogue(pending);
                pending = -1;
            }
            if (kc == a.nch - 1) pending = j / a.nch;
        }
        if (ok && pending >= 0 && !abort_flag) epilogue(pending);
    }
    __syncthreads();
    // after an abort: let the copies still in flight land (the last job issued on each
    // staging slot; a slot's earlier phases completed before it was refilled)
    if (t == 0)
        for (int j = max(0, n_issued - AY_NSTG); j < n_issued; j++) mbar_wait(&stg_full[j % AY_NSTG], (j / AY_NSTG) & 1);
    if (!mbar_wait(&done, 0)) atomicExch(a.err, 17);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(AY_TCOLS) : "memory");
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
    a.inject_ns = 0;
    if (const char *ev = getenv("EIG_TEST_INJECT_WAIT"))
        if (ev[0] == '1') a.inject_ns = 5000000ull;  // 5 ms
    int grid = 0;
    tc_grid(a.ktiles, &a.chunk, &grid);
    const size_t stage = 2 * MT * (size_t)(TM * KT * 4) + 2 * (size_t)((N + 7) / 8) * 1024;
    const size_t smem = (MT == 1 ? 5 : 3) * stage + 1024;  // stages of the TMA ring (k_tc_ahb's NS)
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, TC_THREADS, smem, s>>>(map, a);
    };
    if (MT == 1 && N == 16) go(k_tc_ahb<1, 16, 5>);
    else if (MT == 1) go(k_tc_ahb<1, 32, 5>);
    else if (N == 16) go(k_tc_ahb<2, 16, 3>);
    else go(k_tc_ahb<2, 32, 3>);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n = l * k;
    k_tc_reduce<<<(n + 127) / 128, 128, 0, s>>>(partials, grid, MT, N, l, k, C);
    return cudaGetLastError();
}

bool tc_ay_ok(const ColSet &A, const ColSet &Out) {
    if (A.f64 || Out.f64 || A.ki != 1) return false;
    if (A.ncols < 1 || A.ncols > 512 || Out.ncols < 1 || Out.ncols > 32) return false;
    if (((uintptr_t)A.base & 15) != 0 || ((uintptr_t)Out.base & 7) != 0) return false;
    if (!A.col_off && (A.col_stride & 1)) return false;  // 16-byte aligned column segments
    if (Out.col_off) return Out.ki == 1;
    if (Out.ki == 1) return true;
    return Out.ki == Out.ncols && Out.col_stride == 0;
}

// Out = beta Out + A Y (FP32 column sets, Y FP64 nA x nOut complex row-major, device).
// A's column offsets (col_off) must be even, as every window slot offset is.
cudaError_t launch_tc_ay(const ColSet &A, const double *Y, const ColSet &Out, double beta, long nrows, int *err,
                         void *bscratch, cudaStream_t s) {
    if (!tc_ay_ok(A, Out) || (nrows & 1) || !bscratch) return cudaErrorInvalidValue;
    ProfScope prof("tc_gemm_ay", (double)nrows * (A.ncols + Out.ncols * (beta != 0.0 ? 2 : 1)) * 8.0, s);
    AyArgs a;
    a.A = static_cast<const float2 *>(A.base);
    a.aoff = A.col_off;
    a.acol = A.col_stride;
    a.nA = A.ncols;
    a.Y = Y;
    a.Out = static_cast<float2 *>(Out.base);
    a.oki = Out.ki;
    a.ocol = Out.col_stride;
    a.ooff = Out.col_off;
    a.k = Out.ncols;
    a.beta = (float)beta;
    a.nrows = nrows;
    a.mtiles = (int)((nrows + TM - 1) / TM);
    a.nch = (A.ncols + AY_COLS - 1) / AY_COLS;
    a.err = err;
    a.Bpre = static_cast<const unsigned char *>(bscratch);
    a.tma = 0;
    CUtensorMap amap;
    memset(&amap, 0, sizeof(amap));
    if (!A.col_off && get_encoder() == cudaSuccess) {
        // A as a 2D FP32 tensor: 2 nrows floats per column (x), nA columns (y) col_stride
        // complex apart; the box is one job's staging slot (2 TM floats x AY_COLS columns)
        const cuuint64_t dims[2] = {(cuuint64_t)(2 * nrows), (cuuint64_t)A.ncols};
        const cuuint64_t strides[1] = {(cuuint64_t)A.col_stride * 8};
        const cuuint32_t box[2] = {2 * TM, AY_COLS};
        const cuuint32_t estr[2] = {1, 1};
        const CUresult r = g_encode(&amap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(A.base), dims, strides,
                                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        a.tma = r == CUDA_SUCCESS ? 1 : 0;
    }
    const int N = 2 * Out.ncols <= 16 ? 16 : (2 * Out.ncols <= 32 ? 32 : 64);
    if ((size_t)a.nch * 2 * (size_t)(N / 8) * 1024 > TC_AY_SCRATCH) return cudaErrorInvalidValue;
    {
        unsigned char *bp = static_cast<unsigned char *>(bscratch);
        const int nprep = a.nch * N * KT;
        const int pg = (nprep + 255) / 256;
        if (N == 16) k_ay_prep_b<16><<<pg, 256, 0, s>>>(Y, a.nA, a.k, a.nch, bp);
        else if (N == 32) k_ay_prep_b<32><<<pg, 256, 0, s>>>(Y, a.nA, a.k, a.nch, bp);
        else k_ay_prep_b<64><<<pg, 256, 0, s>>>(Y, a.nA, a.k, a.nch, bp);
    }
    int grid = device_sm_count();
    if (grid > a.mtiles) grid = a.mtiles;
    const int nstg = N == 16 ? 12 : (N == 32 ? 11 : 9);  // AyStages<N>
    const size_t smem = nstg * (size_t)(AY_COLS * TM * 8) + AY_NOP * 2 * (size_t)(N / 8) * 1024 + 1024;
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, AY_THREADS, smem, s>>>(amap, a);
    };
    if (N == 16) go(k_tc_ay<16>);
    else if (N == 32) go(k_tc_ay<32>);
    else go(k_tc_ay<64>);
    return cudaGetLastError();
}

}  // namespace eig
