/*
 * eigcg.h -- C ABI of the GB300 incremental-eigCG library (libeigcg.so).
 *
 * The library solves many right-hand sides of A x = b for the lattice-QCD normal
 * operator A = M^H M, M = m_q I - D the Wilson-Dirac matrix (Sec. 1: "the CG on
 * the A = M^H M Hermitian operator", gamma5 M = M^H gamma5), with
 *   - eigCG(nev, m): CG plus a restarted window of Lanczos vectors that yields nev
 *     Ritz pairs per solve (Sec. 3, Fig. 1);
 *   - Incremental eigCG: Ritz vectors of successive solves accumulate into a
 *     deflation basis U with H = U^H A U (Sec. 4 box);
 *   - init-CG: the Galerkin deflated initial guess of Eq. 1, restarted once near
 *     single precision (Sec. 5.3).
 *
 * Operator convention (Sec. 1 fixes only M = m_q I - D and gamma5-Hermiticity):
 *   (M psi)(x) = (4 + m_q) psi(x)
 *       - 1/2 sum_mu [ (I - g_mu) U_mu(x) psi(x+mu) + (I + g_mu) U_mu(x-mu)^H psi(x-mu) ]
 * periodic in all directions, chiral gamma basis with gamma5 = diag(1, 1, -1, -1):
 *   g1 = [[0,0,0,i],[0,0,i,0],[0,-i,0,0],[-i,0,0,0]]   g2 = [[0,0,0,-1],[0,0,1,0],[0,1,0,0],[-1,0,0,0]]
 *   g3 = [[0,0,i,0],[0,0,0,-i],[-i,0,0,0],[0,i,0,0]]   g4 = [[0,0,1,0],[0,0,0,1],[1,0,0,0],[0,1,0,0]]
 *
 * Vector arguments ("natural layout"): FP64 complex numbers, real then imaginary
 * part, ordered [rhs][site][spin 0..3][colour 0..2], site = ((t*Lz + z)*Ly + y)*Lx + x.
 * Gauge: FP64 complex [site][mu 0..3 = x,y,z,t][row][col], U_mu(x) in SU(3).
 * Vector pointers may be device pointers (any CUDA allocation of this process)
 * or host pointers (pageable or pinned); the library detects which with
 * cudaPointerGetAttributes and copies host data through its own device buffers.
 * All vector buffers stay owned by the caller.  Handles own every device
 * allocation they make and free it in their destroy call.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls return when their results are complete on the host side of
 * the call (solves synchronise the stream); an op or basis must not be used by
 * two host threads at once.
 *
 * Errors: every call returns an eig_status; 0 is success, >0 a warning, <0 an
 * error.  Nothing aborts, asserts or traps; eig_last_error() gives the message
 * of the calling thread's last failure.
 */
#ifndef EIGCG_H
#define EIGCG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EIG_OK = 0,
    EIG_NOT_CONVERGED = 1,  /* max_iter reached; x holds the last iterate          */
    EIG_ERR_ARG = -1,       /* invalid argument (null handle, bad size, bad flag)   */
    EIG_ERR_OOM = -2,       /* device allocation failed                             */
    EIG_ERR_BUDGET = -3,    /* request exceeds the handle's capacity                */
    EIG_ERR_CUDA = -4,      /* CUDA runtime error (message in eig_last_error)       */
    EIG_ERR_BREAKDOWN = -5, /* CG breakdown: p^H A p <= 0, rho <= 0, NaN or Inf     */
    EIG_ERR_TIMEOUT = -6,   /* a bounded device wait gave up                        */
    EIG_ERR_IO = -7         /* a basis file could not be opened, read or written    */
} eig_status;

/* Storage precision codes for spinor_prec. */
#define EIG_PREC_F64 64  /* FP64 storage and arithmetic                                  */
#define EIG_PREC_F32 32  /* FP32 storage and arithmetic, FP64 reductions                 */
#define EIG_PREC_F16 16  /* FP16 spinors, one FP32 scale per site; FP32 links and arithmetic */

typedef struct eig_op_s *eig_op;
typedef struct eig_basis_s *eig_basis;

typedef struct {
    int spinor_prec;        /* EIG_PREC_*; storage of Krylov vectors and links           */
    int link_compress12;    /* 1: store two rows per link, rebuild the third (FP32/F16);
                               FP32 ops also keep the other FP32 form and use, per k,
                               whichever the stencil autotuner measured faster          */
    int max_rhs;            /* largest k of one batched call (1..16); sizes buffers      */
    double reliable_delta;  /* mixed precision: FP64 residual update when ||r|| falls by
                               this factor since the last one (0 -> 0.1)                  */
    int even_odd;           /* 1: the odd-even (Schur complement) form, Sec. 5: the op's
                               matrix is A_hat = M_hat^H M_hat on the odd sites, with
                               M_hat = d - (1/d) H_oe H_eo, d = 4 + m_q, H = M - d the
                               hopping part; every extent must be even.  Solves then take
                               the full-lattice b and x of the Dirac equation M x = b (see
                               eig_eigcg_solve); the vectors of eig_op_apply,
                               eig_basis_deflate and eig_basis_vector are odd-site vectors
                               ([rhs][V/2][4][3], odd site s at s/2).  0: the full lattice. */
} eig_op_opts;

typedef struct {
    int iters;              /* CG iterations (matrix-vector products with A)             */
    int restarts;           /* eigCG window restarts, or init-CG re-deflations           */
    int reliable_updates;   /* FP64 residual replacements (mixed precision)              */
    int converged;          /* 1 if the FP64 true residual met tol                       */
    double true_rel_res;    /* ||b - A x|| / ||b|| recomputed in FP64                     */
    double ms;              /* wall time of the call on its stream                       */
    int n_ritz;             /* Ritz pairs left pending by eigCG                          */
} eig_stats;

/* Creates the operator A = M^H M for one gauge field and quark mass (Sec. 1).
 * gauge: host FP64 [V][4][3][3] complex, copied.  dims: Lx, Ly, Lz, Lt, each >= 2
 * (Lx*Ly*Lz*Lt <= 2^31 / 16).  opts may be NULL (FP64, max_rhs 1).
 * Errors: EIG_ERR_ARG, EIG_ERR_OOM, EIG_ERR_CUDA. */
eig_status eig_op_create(const double *gauge, const int dims[4], double m_q, const eig_op_opts *opts,
                         eig_op *out);
eig_status eig_op_destroy(eig_op op);
/* Releases the op's workspace (Krylov fields for max_rhs RHS, FP64 and natural-layout
 * staging, the eigCG window, the captured CG graphs) and keeps the links; bases bound to
 * the op keep their vectors and H.  The next call that needs the workspace allocates it
 * again.  For a serving loop that holds more operators' bases than it can give
 * workspaces at once (no counterpart in the paper).  Synchronises the device; other
 * threads may meanwhile use other operators (inside the library this synchronisation and
 * the frees wait for, and hold off, their CUDA-graph captures).  *freed
 * (may be NULL): bytes released.  Errors: EIG_ERR_ARG, EIG_ERR_CUDA; a later call may
 * return EIG_ERR_OOM when the workspace no longer fits. */
eig_status eig_op_trim(eig_op op, size_t *freed);

/* out = M in (which 0), M^H in (which 1) or A in (which 2) for k RHS (1..max_rhs),
 * in the op's storage precision; which 3 (FP32/FP16 ops only) applies A in the
 * double-float arithmetic of the residual replacements (about 44-bit precision).
 * in/out: natural layout, may alias.
 * This is the dslash of the CG matrix-vector product (Fig. 1 step 11). */
eig_status eig_op_apply(eig_op op, int which, const double *in, double *out, int k, void *stream);

/* The stencil launch the autotuner chose for k-RHS products of an FP32/FP16 op (the
 * matrix-vector product of Fig. 1 step 11, timed per shape on the first solve):
 * *variant 0..21 (0, 1: shared-memory staged loads of 1 or 2 RHS per thread; 2, 3, 7:
 * direct loads of 1 RHS per thread at 4 or 5 resident blocks per SM, 7 with L1
 * prefetch; 4, 5, 6: direct loads of 2 RHS per thread, 6 with L1 prefetch; 8 + v:
 * variant v over a tiled site order; 16, 17: two adjacent RHS per thread with 256-bit
 * loads and the next hop's data in flight, at 2 or 3 resident blocks per SM; 18, 19:
 * 16, 17 over the tiled order; 20, 21: 17, 19 with an L1 prefetch of the hop after next) and
 * *link_reals 12 or 18 (the resident FP32 link form used).  Both are -1 and 0 for FP64
 * ops or before the first solve with k RHS.  Odd-even ops report the half stencil.
 * Errors: EIG_ERR_ARG (null pointer, k not a power of two <= max_rhs). */
eig_status eig_op_stencil_choice(eig_op op, int k, int *variant, int *link_reals);

/* Deflation basis U (N x l, l <= max_vecs) with H = U^H A U in FP64 (Sec. 4 box),
 * stored on the device in the op's window precision (FP64 for F64 ops, else
 * FP32), plus a pending block of eigCG Ritz vectors.  Bound to one op. */
eig_status eig_basis_create(eig_op op, int max_vecs, eig_basis *out);
eig_status eig_basis_destroy(eig_basis basis);
/* Current number of basis vectors l. */
eig_status eig_basis_size(eig_basis basis, int *l);
/* Drops basis vectors beyond the first l (an earlier size); H keeps its leading block. */
eig_status eig_basis_truncate(eig_basis basis, int l);

/* eigCG(nev, m) of Fig. 1 on one RHS: CG from x (in: initial guess x~0, out:
 * solution), first deflated with the basis by Eq. 1 when basis is non-NULL and
 * non-empty (the "init-CG part" of the Sec. 4 box).  Stops when the recursive
 * ||r|| <= tol ||b||, then checks the FP64 true residual (mixed precision:
 * reliable updates continue until it meets tol).  On return the nev lowest Ritz
 * pairs of the final window are pending in the basis (if given).
 * Requires 1 <= nev, 2*nev < m <= 128.  stats may be NULL.
 * Odd-even ops: b and x (initial guess in, solution out) are full-lattice vectors of
 * M x = b; CG runs on A_hat x_o = M_hat^H b_hat, b_hat = b_o - (1/d) H_oe b_e (Sec. 5,
 * "odd-even preconditioned normal equations"), x_e = (b_e - H_eo x_o) / d is
 * reconstructed, and tol and true_rel_res refer to the odd-site normal equations. */
eig_status eig_eigcg_solve(eig_op op, eig_basis basis, const double *b, double *x, int nev, int m, double tol,
                           int max_iter, eig_stats *stats, void *stream);

/* Spectrally preconditioned eigCG (Sec. 2 "using U as a spectral preconditioner";
 * Sec. 5.2 proposes it for better interior eigenvectors near the critical mass): as
 * eig_eigcg_solve, with Fig. 1's preconditioner P^{-1} = (I - U_p U_p^H) +
 * sp_shift U_p H_p^{-1} U_p^H built from the first sp_vecs basis vectors U_p and the
 * leading block H_p of H (step 3: z = P^{-1} r, rho = r^H z; the window holds
 * z / sqrt(rho)).  For an invariant U_p, P^{-1} A keeps A's other eigenpairs and moves
 * those in span(U_p) to sp_shift, so sp_shift should lie above the eigenvalues wanted
 * next (an upper estimate of A's spectrum, e.g. (8 + m_q)^2 for the full lattice).  The
 * pending Ritz vectors are those of P^{-1} A, to be added by eig_basis_grow.  Each
 * iteration adds U_p^H r and U_p y (two passes over U_p) to the CG work.
 * Requires a non-empty basis, 1 <= sp_vecs <= its size, sp_shift > 0, an FP64 or FP32
 * op.  Errors: as eig_eigcg_solve; EIG_ERR_BREAKDOWN if H_p is not positive definite
 * or r^H z <= 0. */
eig_status eig_eigcg_solve_sp(eig_op op, eig_basis basis, const double *b, double *x, int nev, int m, double tol,
                              int max_iter, int sp_vecs, double sp_shift, eig_stats *stats, void *stream);

/* Sec. 4 box, last three lines: orthonormalises the pending Ritz vectors against U
 * (classical Gram-Schmidt twice, FP64 accumulation), W = A V-bar in FP64, extends H
 * with U^H W and V-bar^H W, appends V-bar to U.  Vectors that are numerically in
 * span(U) are dropped.  EIG_ERR_BUDGET if max_vecs would be exceeded. */
eig_status eig_basis_grow(eig_basis basis, void *stream);

/* Eq. 1 for k RHS: x0 = x~0 + U H^{-1} U^H (b - A x~0).  x_in may be NULL (x~0 = 0)
 * and may alias x0. */
eig_status eig_basis_deflate(eig_basis basis, const double *b, const double *x_in, double *x0, int k,
                             void *stream);

/* init-CG on k independent RHS (1..max_rhs) batched through one multi-RHS dslash:
 * Eq. 1 deflation (if basis non-empty), CG, one re-deflation and restart when
 * ||r||/||b|| first reaches restart_tol (Sec. 5.3; restart_tol <= tol disables it),
 * FP64 true-residual check.  x: in x~0, out solution.  stats: array of k (or NULL). */
eig_status eig_initcg_solve(eig_op op, eig_basis basis, const double *b, double *x, double tol, double restart_tol,
                            int max_iter, int k, eig_stats *stats, void *stream);

/* BiCGSTAB (van der Vorst 1992) on M x = b for one RHS, deflated with the basis as Sec. 1
 * proposes: A = M^H M = (g5 M)^2, so the eigenvectors eigCG computes for A are
 * eigenvectors of the Hermitian g5 M.  With defl_vecs > 0 and a non-empty basis, the
 * initial guess x~0 (in x) becomes x0 = x~0 + Z (Z^H g5 M Z)^{-1} Z^H g5 (b - M x~0),
 * Z = the min(defl_vecs, l) lowest Ritz vectors of A in span(U) (cached with
 * Z^H g5 M Z until the basis changes).  b, x: natural layout, full lattice.  Vectors in
 * the op's storage precision (FP64 or FP32), x in FP64; FP32 runs restart from the FP64
 * residual b - M x whenever the recursive residual has fallen by 1e5, and every solve
 * ends with the FP64 residual ||b - M x|| <= tol ||b|| (true_rel_res refers to M).
 * stats->restarts counts those restarts and breakdown restarts.  Odd-even and FP16 ops
 * are refused (EIG_ERR_ARG).  EIG_NOT_CONVERGED after max_iter iterations. */
eig_status eig_bicgstab_solve(eig_op op, eig_basis basis, const double *b, double *x, double tol, int max_iter,
                              int defl_vecs, eig_stats *stats, void *stream);

/* Rayleigh-Ritz on U (Sec. 5.2): Ritz values (eigenvalues of H, ascending) and
 * residual norms ||A u - theta u|| (FP64 operator).  evals/resnorms: host arrays of
 * at least l entries (resnorms may be NULL to skip the residuals); *n = l. */
eig_status eig_basis_ritz(eig_basis basis, double *evals, double *resnorms, int *n, void *stream);

/* Copies basis vector j (0 <= j < l) to out (natural layout, host or device). */
eig_status eig_basis_vector(eig_basis basis, int j, double *out, void *stream);
/* Ritz values of the pending block the last eigCG solve left (ascending, *n of them,
 * at most nev; evals may be NULL to query *n): the eigenvalues of Fig. 1's final
 * window that eig_basis_grow will add. */
eig_status eig_basis_pending(eig_basis basis, double *evals, int *n);
/* Copies H (l x l, FP64 complex, row-major, host) to out. */
eig_status eig_basis_h(eig_basis basis, double *out);

/* Saves the deflation basis U and H = U^H A U (Sec. 4 box) to a file, so that later
 * jobs with the same operator start from it instead of rebuilding it with Incremental
 * eigCG (the paper notes the vectors can be stored for reuse).  Layout: a 64-byte
 * header (magic "EIGBASIS", version 1, the four lattice extents, even_odd, bytes per
 * real of the stored vectors, l, complex entries per vector, m_q, a fingerprint of the
 * FP64 links), H as l x l complex FP64 row-major, then the l vectors in natural layout
 * in the basis precision (FP32 for FP32/FP16 ops, FP64 otherwise), little-endian.  The
 * pending Ritz block is not saved.  Errors: EIG_ERR_ARG, EIG_ERR_IO, EIG_ERR_CUDA. */
eig_status eig_basis_save(eig_basis basis, const char *path, void *stream);
/* Replaces the basis with one saved by eig_basis_save for an operator with the same
 * lattice, odd-even form, quark mass and links (else EIG_ERR_ARG); the vectors are
 * converted to this basis's precision.  EIG_ERR_BUDGET if the file holds more than
 * max_vecs vectors (basis unchanged); EIG_ERR_IO for an unreadable or short file
 * (basis left empty if the error comes after the header); EIG_ERR_BREAKDOWN if the
 * loaded H is not positive definite. */
eig_status eig_basis_load(eig_basis basis, const char *path, void *stream);

/* Kernel instrumentation (diagnostics; the paper reports only per-phase wall
 * times, Table 1).  Every kernel launch of the library is counted per kernel name
 * together with its algorithmic bytes (each link, input and output touched
 * once).  With eig_profile_enable(1) each launch is also bracketed by CUDA
 * events recorded on the stream it runs on.  eig_profile_read synchronises the
 * device and returns up to max entries (*n = number of kernel names seen). */
typedef struct {
    char name[40];
    long launches;
    double ms;      /* summed event time (0 unless timing was enabled) */
    double bytes;   /* summed algorithmic bytes                         */
} eig_kernel_stat;
eig_status eig_profile_enable(int on);
eig_status eig_profile_reset(void);
eig_status eig_profile_read(eig_kernel_stat *out, int max, int *n);
/* Measured arithmetic roof of this GPU (measurement aid, no counterpart in the paper):
 * fused multiply-add throughput in TFLOP/s for prec 64 (FP64) or 32 (FP32, packed
 * pairs), from independent FMA chains over a grid that fills every SM, best of two
 * timed launches on `stream` (synchronised).  The reference for kernels bound by
 * arithmetic rather than memory.  Errors: EIG_ERR_ARG, EIG_ERR_CUDA. */
eig_status eig_profile_alu_peak(int prec, double *tflops, void *stream);

/* Allocation-free M, M^H or A = M^H M (which 0, 1, 2) on one FP64 RHS.  The paper
 * has no counterpart: this entry point exists for callers that may not allocate
 * device memory (memory owned by another allocator or pool that forbids cudaMalloc,
 * a device already reserved in full), which eig_op_apply cannot serve because an op
 * handle allocates its own buffers.  It calls no allocating routine.
 * gauge ([V][4][3][3] complex), in and out ([V][4][3] complex): DEVICE pointers in
 * the natural layout above, owned by the caller, in the memory of the current device
 * (or managed memory); out must not overlap in or gauge.
 * dims: each >= 2, Lx*Ly*Lz*Lt <= 65536 sites (EIG_ERR_BUDGET beyond).
 * A keeps its intermediate M in in a static device array of 65536 sites (12.6 MB)
 * that every GPU loading the library holds until the process exits.  Every call
 * shares it: it holds the last call's data (nothing in it needs to start at zero),
 * and calls that overlap on the GPU race on it.  The first call on each device
 * (with that device current) looks up the array's address and caches it; make that
 * call before any stream capture (a first call on a capturing stream returns
 * EIG_ERR_CUDA).  Asynchronous on `stream`.
 * Errors: EIG_ERR_ARG (null pointers, host or other-device pointers, overlapping
 * buffers, bad which/dims), EIG_ERR_BUDGET, EIG_ERR_CUDA. */
eig_status eig_wilson_apply_noalloc(const double *gauge, const int dims[4], double m_q, int which, const double *in,
                                    double *out, void *stream);

/* Message of the calling thread's last error ("" if none). */
const char *eig_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* EIGCG_H */
