// Host-side launchers of the CUDA kernels (definitions in dslash.cu, blas.cu, gemm.cu).
// Every launcher enqueues on `stream` and returns the launch status.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace eig {

enum Prec { P64 = 0, P32 = 1, P16 = 2 };

inline size_t field_bytes(Prec p, long V, int k) {
    switch (p) {
        case P64: return (size_t)V * k * 192;
        case P32: return (size_t)V * k * 96;
        default: return (size_t)V * k * 48;
    }
}

// Per-RHS CG scalars, FP64, resident on the device.
struct CGScalars {
    double rho;       // r^H r of the current residual
    double rho_prev;  // previous rho
    double alpha;     // alpha_j of the current iteration
    double beta;      // beta of the next p update
    double pAp;       // p^H A p = ||M p||^2
    double target;    // stop when rho <= target (tol^2 ||b||^2)
    double aux;       // last auxiliary reduction (true residual norm^2, norm of b, ...)
    int active;       // 1 while iterating
    int iters;        // last iteration in which this RHS was active
    int x_pending;    // 1: x still lacks alpha * p of the last iteration (applied by the next p update)
    int breakdown;    // 1 if pAp <= 0, NaN or Inf was met
    int nit;          // iterations this RHS took part in (a batch runs on after a RHS stops)
};

// Device scalars of one BiCGSTAB solve (complex values as re, im).
struct BicgScalars {
    double rho[2];    // r_hat^H r
    double alpha[2];  // rho / (r_hat^H v)
    double omega[2];  // (t^H s) / (t^H t)
    double beta[2];   // (rho' / rho) (alpha / omega)
    double rr;        // ||r||^2 of the recursive residual
    double target;    // stop when rr <= target
    int active;       // 1 while iterating
    int breakdown;    // 1 if a denominator vanished or a NaN/Inf appeared
    int iters;        // iterations completed
    int pad;
};

// Reduction scratch shared by the kernels of one solver stream.
struct RedScratch {
    double *partials;   // [max_blocks * MAX_RHS * 64] doubles
    unsigned *counter;  // one counter, zero between launches
    int max_blocks;
};

struct Field {
    Prec prec;
    FieldView v;
};

// History of CG scalars: alpha[j*k + r] etc. for iterations j = 0..cap-1.
// With jbase set, the iteration index a kernel is given is relative: the kernel adds
// *jbase (device), so that one captured block of iterations can be replayed.
struct History {
    double *alpha;
    double *beta;
    double *rho;
    int cap;
    const int *jbase = nullptr;
};

struct DslashCall {
    Field in, out;     // out may be unused by the CG epilogue (store_out = 0)
    GaugeView gauge;
    int gformat;       // GaugeFormat
    int L[4];
    long V;            // lattice sites (gauge planes hold V sites)
    int k;
    double diag;       // 4 + m_q
    bool dagger;
    // Odd-even form (eo_parity 0 or 1; -1: the full lattice).  Fields are half-lattice
    // fields of V / 2 sites (site s of one parity at s / 2, every extent even):
    //   out_p = diag * cen_p + hcoef * sum over the 8 hops of in_(1-p),
    // the hop sum being the bracket of the Wilson operator, so that the full operator
    // is diag = 4 + m_q, hcoef = -1/2, cen = in.
    int eo_parity = -1;
    Field cen;
    double hcoef = -0.5;
};

// ---------------------------- dslash.cu ----------------------------------------------
// out = M in (dagger: M^H in)
cudaError_t launch_dslash(const DslashCall &c, cudaStream_t s);
// CG pass 1: out = M in, pAp = ||out||^2, alpha = rho / pAp   (Fig. 1 steps 11-12)
cudaError_t launch_dslash_norm(const DslashCall &c, CGScalars *st, History h, int iter, RedScratch red,
                               cudaStream_t s);
// CG pass 2: t = M^H in; r -= alpha t; rho_new = ||r||^2; beta = rho_new / rho
// (Fig. 1 steps 11, 14 and 4/8 of the next iteration).  Step 13 (x += alpha p) is
// applied one iteration late by launch_pupdate, which reads p anyway.  If
// t_save.v.data != nullptr, t is also written there (window precision).
cudaError_t launch_dslash_cg(const DslashCall &c, Field r, Field t_save, CGScalars *st, History h, int iter,
                             RedScratch red, cudaStream_t s);
// FP64 residual: r = b - M^H in, aux = ||r||^2 (with set_rho: rho = aux, beta = rho / rho_prev,
// history beta[iter + 1] = beta, rho[iter] = rho).
cudaError_t launch_dslash_resid(const DslashCall &c, Field b, Field r, CGScalars *st, History h, int iter,
                                bool set_rho, RedScratch red, cudaStream_t s);

// dslash32.cu: FP32-arithmetic versions (FP32 / FP16 storage) of the three launches above
cudaError_t launch_dslash32(const DslashCall &c, cudaStream_t s);
cudaError_t launch_dslash32_norm(const DslashCall &c, CGScalars *st, History h, int iter, RedScratch red,
                                 cudaStream_t s);
cudaError_t launch_dslash32_cg(const DslashCall &c, Field r, Field t_save, CGScalars *st, History h, int iter,
                               RedScratch red, cudaStream_t s);
// chooses (once per volume, k and format) how many RHS each stencil thread handles
// Times every stencil variant on c's buffers (in -> out), for c's link format and for
// the same links stored in each of the n_alts other formats gf_alts (data gauge_alts);
// caches the fastest variant per format and the fastest format for (V, k, storage).
cudaError_t autotune_dslash32(const DslashCall &c, const void *const *gauge_alts, const int *gf_alts, int n_alts,
                              cudaStream_t s);
// The link format the autotuner found faster for (V, k, storage), or -1 if not tuned.
int dslash32_best_gformat(long V, int k, int prec);
// Link format (-1 before tuning) and stencil variant (0..7) the call would launch with.
int dslash32_choice(const DslashCall &c, int *variant);

// dslash_dd.cu: double-float (FP32-pair) stencil for residual replacements.  dd fields
// have the FP64 layout with float4 (re_hi, im_hi, re_lo, im_lo) per complex number.
cudaError_t launch_to_dd(const void *fp64, void *dd, long n_complex, cudaStream_t s);
// kc FP32 fields of one RHS each (column c at cols + c * cstride_f4 float4s) <->
// a double-float RHS-inner field of kc RHS
cudaError_t launch_cols32_to_dd(const void *cols, long cstride_f4, long V, int kc, void *dd, cudaStream_t s);
cudaError_t launch_dd_to_cols32(const void *dd, long V, int kc, void *cols, long cstride_f4, cudaStream_t s);
cudaError_t launch_from_dd(const void *dd, void *fp64, long n_complex, cudaStream_t s);
cudaError_t launch_dslash_dd(const DslashCall &c, const void *gauge_dd, const void *in_dd, void *out_dd,
                             cudaStream_t s);
cudaError_t launch_dslash_dd_resid(const DslashCall &c, const void *gauge_dd, const void *in_dd, Field b, Field r,
                                   CGScalars *st, History h, int iter, bool set_rho, RedScratch red, cudaStream_t s);

// ---------------------------- blas.cu -------------------------------------------------
// natural FP64 [k][V][12] complex  <->  internal field
cudaError_t launch_pack(const double *nat, Field f, cudaStream_t s);
cudaError_t launch_unpack(Field f, double *nat, cudaStream_t s);
// gauge natural [V][4][3][3] complex (device) -> internal format
cudaError_t launch_pack_gauge(const double *nat, void *dst, int gformat, long V, cudaStream_t s);
// out = ca * a + cb * b   (b may have data == nullptr; ca, cb real).  All fields same V, k.
cudaError_t launch_combine(Field out, double ca, Field a, double cb, Field b, cudaStream_t s);
// per-RHS ||f||^2 -> st[r].aux;  with as_rho: also rho = aux, rho_prev = aux, history rho[iter]
// and target = tol2 * bnorm2[r] computed elsewhere (untouched here).
cudaError_t launch_norm2(Field f, CGScalars *st, bool as_rho, History h, int iter, RedScratch red, cudaStream_t s);
// bicgstab.cu: the BiCGSTAB steps on one RHS (see there); x64 FP64, the other fields
// in one storage precision (FP64 or FP32)
cudaError_t launch_bicg_p(Field r, Field p, Field v, const BicgScalars *sc, cudaStream_t s);
cudaError_t launch_bicg_alpha(Field rh, Field v, BicgScalars *sc, RedScratch red, cudaStream_t s);
cudaError_t launch_bicg_s(Field r, Field v, Field sv, const BicgScalars *sc, cudaStream_t s);
cudaError_t launch_bicg_omega(Field t, Field sv, BicgScalars *sc, RedScratch red, cudaStream_t s);
cudaError_t launch_bicg_update(Field x64, Field p, Field sv, Field t, Field r, Field rh, BicgScalars *sc,
                               RedScratch red, cudaStream_t s);
// out = g5 in (chiral basis, g5 = diag(1, 1, -1, -1) in spin); FP64 or FP32 fields
cudaError_t launch_gamma5(Field in, Field out, cudaStream_t s);

// Spectral preconditioner (Sec. 2) pieces: Y = G C for one RHS (G l x l complex
// row-major, C and Y l complex), and rho = r^H z with Fig. 1's preconditioned scalar
// updates for the active RHS (rho, h_rho[iter], and beta, h_beta[iter + 1] for iter >= 1).
cudaError_t launch_sp_coef(const double *G, const double *C, double *Y, int l, cudaStream_t s);
cudaError_t launch_pcg_rho(Field r, Field z, CGScalars *st, History h, int iter, RedScratch red, cudaStream_t s);
// CG step 13 of the previous iteration (x += alpha p, if pending), step 9 (p = r + beta p;
// first: p = r) and eigCG step 11.13 (v = r / sqrt(rho), optional)
cudaError_t launch_pupdate(Field r, Field p, Field x, bool first, CGScalars *st, Field v_append, cudaStream_t s);
// applies a pending x += alpha p for every RHS and clears the pending flags
cudaError_t launch_xflush(Field p, Field x, CGScalars *st, int k, cudaStream_t s);
// set up per-RHS scalars: target = tol^2 * aux (aux must hold ||b||^2), active = 1, breakdown = 0
cudaError_t launch_cg_init(CGScalars *st, int k, double tol, History h, cudaStream_t s);

// ---------------------------- gemm.cu -------------------------------------------------
// A column set of complex vectors stored in fields of one precision (double or float).
// Element (row, col) sits at complex index
//   ((row / cpc) * ki + (col % ki)) * cpc + row % cpc + (col / ki) * col_stride
// where cpc = complex numbers per storage chunk (1 for FP64, 2 for FP32): ki = k for
// an RHS-inner field of k RHS, ki = 1 and col_stride = field size for separate fields.
// `cols` gives per-column base offsets (in complex units) when non-null (window slots).
struct ColSet {
    void *base;
    bool f64;
    int ki;
    long col_stride;
    int ncols;
    const long *col_off;  // device array of ncols offsets, or nullptr
};

// C (nA x nB, FP64 complex, row-major, device) = A^H B over nrows complex rows.
cudaError_t launch_gemm_ahb(ColSet A, ColSet B, long nrows, double *C, RedScratch red, cudaStream_t s);
// Out[:, c] = beta_out * Out[:, c] + sum_a A[:, a] Y[a, c]   (Y: nA x nOut FP64 complex row-major, device)
cudaError_t launch_gemm_ay(ColSet A, const double *Y, ColSet Out, double beta_out, long nrows, cudaStream_t s);
// eigCG restart (Fig. 1 step 11.7 + 11.8): in place over the window slots,
//   V[:, c] = sum_a V[:, a] QZ[a, c]  (c < nout), and  wv[c] = sum_rows conj(w) V_new[:, c],
//   w = t - beta * t_prev  (beta read from *beta_dev).  wv: FP64 complex [nout], device.
cudaError_t launch_window_restart(ColSet Vw, int m, const double *QZ, int nout, const void *t, const void *t_prev,
                                  const double *beta_dev, long nrows, double *wv, RedScratch red, cudaStream_t s);

// C (nA x nB, FP64 complex, row-major, device) = A^H B on the tensor cores (tcgen05,
// kind::tf32 with each operand split into TF32 hi + lo parts, three products per K
// step; FP32 accumulation in TMEM over two K tiles at a time, drained into
// double-float sums per thread, FP64 sum over CTAs).  A: FP32 fields, one per column (ki = 1, no offsets), column
// stride a multiple of 2 complex, 16-byte aligned, nA <= 256; B: FP32 column set of
// nB <= 16 columns, RHS-inner (ki = nB) or one field per column (ki = 1).
// tc_ahb_ok tells whether a pair qualifies.  *err (device int, zeroed by the caller)
// becomes non-zero if a bounded wait inside the kernel gave up; C is then invalid.
bool tc_ahb_ok(const ColSet &A, const ColSet &B);
size_t tc_ahb_partials_bytes(long nrows, int l, int k);
cudaError_t launch_tc_ahb(const ColSet &A, const ColSet &B, long nrows, double *C, double *partials, int *err,
                          cudaStream_t s);

// Out = beta Out + A Y on the tensor cores (kind::tf32, hi/lo split operands; K = 2 nA
// <= 1024 accumulated in one TMEM accumulator per 128-row tile).  A: FP32 fields, one
// per column (col_stride or even col_off offsets), nA <= 512; Out: FP32, nOut <= 16
// columns, RHS-inner or one field per column, not overlapping A; Y: FP64 complex
// nA x nOut row-major on the device; nrows even.  *err (device, zeroed by the caller)
// becomes non-zero if a bounded wait gave up (Out is then invalid).
bool tc_ay_ok(const ColSet &A, const ColSet &Out);
// bscratch: device scratch of at least TC_AY_SCRATCH bytes owned by the caller's handle
// (the B operand of every K chunk, built once per launch); calls that overlap on the GPU
// must use different scratch
constexpr size_t TC_AY_SCRATCH = 32 * 2 * 8192;  // up to 512 columns of A, N = 64
cudaError_t launch_tc_ay(const ColSet &A, const double *Y, const ColSet &Out, double beta, long nrows, int *err,
                         void *bscratch, cudaStream_t s);

// Copies the sites of one parity between a full-lattice FP64 field and a half-lattice
// FP64 field (to_half: full -> half), same k; Lx even.
cudaError_t launch_parity_move(Field full, Field half, int parity, const int L[4], bool to_half, cudaStream_t s);

// wv[c] = sum_rows conj(w) V[:, c] (c < nout <= 32), w = t - (*beta_dev) t_prev: FP32
// fields of nrows complex entries, V columns at base + off[c] (complex units, device)
cudaError_t launch_wdot(const void *t, const void *t_prev, const double *beta_dev, const void *base, const long *off,
                        int nout, long nrows, double *wv, RedScratch red, cudaStream_t s);

int device_sm_count();

}  // namespace eig
