// Solver engine behind the C ABI of include/eigcg.h.
//
// Flow of one CG iteration j (Fig. 1, P = I), all on the caller's stream with the
// scalars alpha, beta, rho resident on the device:
//   k_pupdate          p = r + beta_j p        (+ eigCG step 11.13: V(:, i) = r / sqrt(rho))
//   k_dslash<NORM>     u = M p, pAp = ||u||^2, alpha_j = rho / pAp         (steps 11-12)
//   k_dslash<CG>       t = M^H u, x += alpha p, r -= alpha t, rho, beta_{j+1}  (steps 13-14, 4, 8)
// The host synchronises only every CHECK iterations (convergence, reliable
// updates) and at eigCG restarts, where it reads the alpha/beta history, forms the
// window projection T (Eq. 4 plus the restarted head), solves the small FP64
// eigenproblems of steps 11.3-11.6 and launches the in-place restart GEMM of step
// 11.7 with the step-11.8 row fused in.
//
// Mixed precision: Krylov vectors live in FP32 or FP16 storage; x accumulates in
// FP32 between reliable updates, which add it into an FP64 solution and replace r
// by the FP64 true residual b - A x when ||r|| has fallen by reliable_delta.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "dense.h"
#include "eigcg.h"
#include "kernels.cuh"
#include "prof.h"

namespace eig {

using cd = std::complex<double>;

struct Error {
    eig_status st;
    std::string msg;
};

static thread_local std::string g_last_error;

#define CUDA_CK(call)                                                                           \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) throw Error{EIG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

// Graph captures and device-wide synchronisation exclude each other: a
// cudaDeviceSynchronize, cudaFree or cudaFreeHost (both may synchronise the device)
// issued by one thread while another thread's stream is being captured fails and
// invalidates that capture, which happens when several operators are served from their
// own threads.  Captures hold this lock, and so does every device-wide sync and free
// (recursive: a destroy holds it over the sync and the frees of its buffers).
static std::recursive_mutex g_capture_mu;

struct DevBuf {
    void *p = nullptr;
    size_t n = 0;
    void alloc(size_t bytes) {
        release();
        if (bytes == 0) return;
        // test hook (EIG_TEST_ALLOC_LIMIT=<bytes>): a fake of a failing cudaMalloc for
        // larger requests, so that the out-of-memory path runs without exhausting a GPU
        if (const char *ev = getenv("EIG_TEST_ALLOC_LIMIT"))
            if (bytes > std::strtoull(ev, nullptr, 10))
                throw Error{EIG_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed (test limit)"};
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            throw Error{EIG_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed"};
        }
        n = bytes;
    }
    void ensure(size_t bytes) {
        if (bytes > n) alloc(bytes);
    }
    void release() {
        if (p) {
            std::lock_guard<std::recursive_mutex> cap_lock(g_capture_mu);
            cudaFree(p);
        }
        p = nullptr;
        n = 0;
    }
    ~DevBuf() { release(); }
    template <typename T>
    T *as() const {
        return static_cast<T *>(p);
    }
};

struct PinBuf {
    void *p = nullptr;
    size_t n = 0;
    void ensure(size_t bytes) {
        if (bytes <= n) return;
        if (p) {
            std::lock_guard<std::recursive_mutex> cap_lock(g_capture_mu);
            cudaFreeHost(p);
        }
        p = nullptr;
        n = 0;
        if (cudaMallocHost(&p, bytes) != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            throw Error{EIG_ERR_OOM, "cudaMallocHost failed"};
        }
        n = bytes;
    }
    ~PinBuf() {
        if (p) {
            std::lock_guard<std::recursive_mutex> cap_lock(g_capture_mu);
            cudaFreeHost(p);
        }
    }
    template <typename T>
    T *as() const {
        return static_cast<T *>(p);
    }
};

// A field buffer able to hold up to kcap RHS.
struct FieldBuf {
    Prec prec = P64;
    long V = 0;
    int kcap = 0;
    DevBuf data, scale;
    void alloc(Prec p, long v, int k) {
        prec = p;
        V = v;
        kcap = k;
        data.alloc(field_bytes(p, v, k));
        if (p == P16) scale.alloc((size_t)v * k * sizeof(float));
    }
    void release() {
        data.release();
        scale.release();
        kcap = 0;
    }
    Field view(int k) const {
        Field f;
        f.prec = prec;
        f.v.data = data.p;
        f.v.scale = scale.as<float>();
        f.v.V = V;
        f.v.k = k;
        return f;
    }
};

static Field null_field() {
    Field f;
    memset(&f, 0, sizeof(f));
    return f;
}

static Field field_at(Prec p, void *data, long V, int k) {
    Field f;
    f.prec = p;
    f.v.data = data;
    f.v.scale = nullptr;
    f.v.V = V;
    f.v.k = k;
    return f;
}

constexpr int CHECK = 16;        // iterations between host checks
constexpr int MAX_WINDOW = 128;  // largest eigCG m
constexpr int MAX_NEV = 16;
constexpr int RED_BLOCKS = 2048;

}  // namespace eig

using namespace eig;

struct eig_op_s {
    int L[4];
    long V;        // lattice sites
    long Vf;       // sites of a Krylov / basis field: V, or V / 2 for the odd-even form
    bool eo = false;
    FieldBuf tmp_e, tmp64_e;  // odd-even form: even-parity results of the first half stencil
    FieldBuf full64, be64;    // odd-even form: full-lattice b / x, and b's even part
    double m_q;
    unsigned long long gauge_hash = 0;  // fingerprint of the FP64 links (basis files)
    Prec prec;     // Krylov storage
    Prec wprec;    // window / basis / x_lo storage (P64 or P32)
    int gf_inner;
    int max_rhs;
    double delta;
    DevBuf gauge64, gauge_in, gauge_dd;  // gauge_dd: double-float copy (mixed precision)
    DevBuf gauge_alt;                    // FP32 ops: the links in the other FP32 format
    int gf_alt = -1;
    // workspace
    FieldBuf r, p, u, xlo, b64, x64, r64, u64, rsv, xsv;
    DevBuf nat_in, nat_out;
    DevBuf st;
    PinBuf st_h;
    DevBuf hist;
    int hist_cap = 0;
    PinBuf hist_h;
    DevBuf red_partials, red_counter;
    // eigCG window
    DevBuf win, tprev, tcur, col_off, qz, wv;
    int win_slots = 0;
    std::mutex mu;
    // CUDA graphs of CHECK plain CG iterations (init-CG), one per buffer set
    struct CgGraph {
        cudaGraphExec_t exec = nullptr;
        std::vector<const void *> key;
        ProfRecord rec;
    };
    std::vector<CgGraph> graphs;
    DevBuf tcerr;      // error flag of the tensor-core window restart
    PinBuf errh;
    DevBuf tcb;        // B-operand scratch of the tensor-core A Y (window restart, preconditioner)
    // spectrally preconditioned eigCG: z = P^{-1} r, G = shift H_p^{-1} - I, U_p^H r, G U_p^H r,
    // tensor-core partial sums and error flags
    FieldBuf zsp;
    DevBuf spG, spC, spY, sptc, sperr;
    PinBuf sperrh;
    // BiCGSTAB: r_hat, s, t (one RHS, Krylov precision) and the device scalars
    FieldBuf bc_rh, bc_s, bc_t;
    DevBuf bsc;
    PinBuf bsch;
    DevBuf jbase_dev;  // iteration base the replayed kernels add to their offsets
    PinBuf jbase_h;
    cudaStream_t cap_stream = nullptr;  // private stream the graphs are captured on
    bool ws = false;                    // workspace allocated (see ensure_workspace)
    ~eig_op_s() {
        for (auto &g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }

    long ncomplex() const { return Vf * 12; }
    size_t wfield_bytes() const { return field_bytes(wprec, Vf, 1); }
    RedScratch red() const {
        RedScratch r;
        r.partials = red_partials.as<double>();
        r.counter = red_counter.as<unsigned>();
        r.max_blocks = RED_BLOCKS;
        return r;
    }
    DslashCall call(Field in, Field out, bool dag, bool f64) const {
        DslashCall c;
        c.in = in;
        c.out = out;
        c.gauge.data = f64 ? gauge64.p : gauge_in.p;
        c.gauge.V = V;
        c.gformat = f64 ? GF_F64_18 : gf_inner;
        if (!f64 && prec == P32) {
            const int best = dslash32_best_gformat(V, in.v.k, 32);
            if (best == gf_alt && gauge_alt.p) {
                c.gauge.data = gauge_alt.p;
                c.gformat = gf_alt;
            }
        }
        for (int i = 0; i < 4; i++) c.L[i] = L[i];
        c.V = V;
        c.k = in.v.k;
        c.diag = 4.0 + m_q;
        c.dagger = dag;
        c.cen = Field{};
        return c;
    }
    History history(int k) const {
        History h;
        h.alpha = hist.as<double>();
        h.beta = h.alpha + (size_t)hist_cap * k;
        h.rho = h.beta + (size_t)hist_cap * k;
        h.cap = hist_cap;
        return h;
    }
    // The history layout depends on k (three arrays of cap * k doubles); the
    // allocation is tracked in doubles per array so that a later solve with more
    // RHS than an earlier one reallocates.
    size_t hist_elems = 0;
    void ensure_history(int iters, int k) {
        hist_cap = iters + 4;
        const size_t need = (size_t)hist_cap * k;
        if (need > hist_elems) {
            hist.alloc(need * 3 * sizeof(double));
            hist_elems = need;
        }
        hist_h.ensure(need * 3 * sizeof(double));
    }
};

struct eig_basis_s {
    eig_op_s *op;
    int max_vecs;
    int l = 0;
    DevBuf U;        // max_vecs window-precision fields
    DevBuf pend;     // MAX_NEV pending Ritz vectors
    DevBuf W;        // MAX_NEV scratch fields
    int npend = 0;
    std::vector<double> pend_ritz;
    std::vector<cd> H, Lc;  // H = U^H A U and its Cholesky factor (row-major l x l)
    bool chol_ok = true;
    DevBuf C, Y;            // device small matrices
    DevBuf tcpart, tcerr;   // partial sums and error flag of the tensor-core U^H R
    DevBuf tcb;             // B-operand scratch of the tensor-core A Y
    PinBuf Ch, errh;
    long gen = 0;           // bumped whenever U changes
    // BiCGSTAB deflation through g5 M: Z = lowest Ritz vectors of A in span(U) and
    // H5 = Z^H g5 M Z, valid for generation z_gen and z_n vectors
    DevBuf Z;
    std::vector<cd> H5;
    int z_n = 0;
    long z_gen = -1;
    std::mutex mu;
    long fsize() const { return op->Vf * 12; }  // complex entries per field
};

namespace eig {

static void set_error(const Error &e) { g_last_error = e.msg; }

// The workspace of an op: the Krylov fields for max_rhs RHS, FP64 staging and the
// natural-layout staging (fields of Vf sites: half-lattice fields for the odd-even form).
// Allocated when the op is created; eig_op_trim releases it together with the eigCG window
// and the CUDA graphs that point into it, and the next call that needs it allocates it again.
static void ensure_workspace(eig_op_s *op) {
    if (op->ws) return;
    const long Vf = op->Vf, V = op->V;
    const int K = op->max_rhs;
    op->r.alloc(op->prec, Vf, K);
    op->p.alloc(op->prec, Vf, K);
    op->u.alloc(op->prec, Vf, K);
    op->b64.alloc(P64, Vf, K);
    op->x64.alloc(P64, Vf, K);
    op->u64.alloc(P64, Vf, K);
    if (op->prec != P64) {
        op->xlo.alloc(P32, Vf, K);
        op->r64.alloc(P64, Vf, K);
    }
    op->rsv.alloc(op->wprec, Vf, K);
    op->xsv.alloc(op->wprec, Vf, K);
    if (op->eo) {
        op->tmp_e.alloc(op->prec, Vf, K);
        op->tmp64_e.alloc(P64, Vf, K);
        op->full64.alloc(P64, V, K);
        op->be64.alloc(P64, Vf, K);
    }
    op->nat_in.alloc((size_t)V * 12 * 16 * K);
    op->nat_out.alloc((size_t)V * 12 * 16 * K);
    op->ws = true;
}

static void release_workspace(eig_op_s *op) {
    for (auto &g : op->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    op->graphs.clear();
    for (FieldBuf *f : {&op->r, &op->p, &op->u, &op->b64, &op->x64, &op->u64, &op->xlo, &op->r64, &op->rsv, &op->xsv,
                        &op->tmp_e, &op->tmp64_e, &op->full64, &op->be64, &op->zsp, &op->bc_rh, &op->bc_s, &op->bc_t})
        f->release();
    op->nat_in.release();
    op->nat_out.release();
    op->win.release();
    op->win_slots = 0;
    op->tprev.release();
    op->tcur.release();
    op->ws = false;
}

// lets entry points defined in other files report a message through eig_last_error
void set_last_error_message(const char *msg) { g_last_error = msg ? msg : ""; }

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void sync(cudaStream_t s) { CUDA_CK(cudaStreamSynchronize(s)); }

// Sets a field to zero without reading it (fresh allocations may hold NaN patterns).
static void zero_field(Field f, cudaStream_t s) {
    CUDA_CK(cudaMemsetAsync(f.v.data, 0, field_bytes(f.prec, f.v.V, f.v.k), s));
    if (f.prec == P16 && f.v.scale) CUDA_CK(cudaMemsetAsync(f.v.scale, 0, (size_t)f.v.V * f.v.k * sizeof(float), s));
}

// ------------------------------------------------------------------------------------
// building blocks on an op
// ------------------------------------------------------------------------------------
// The call that applies M (dag: M^H) to in.  For an odd-even operator the matrix is
// M_hat = d - (1/d) H_oe H_eo on the odd sites (d = 4 + m_q, H the hopping part of M):
// this launches the first half stencil, tmp_e = H_eo in (or (H^H)_eo in), and returns
// the second, out = d in + (1/2d) (hop sum of tmp_e), which the caller launches with
// the epilogue it needs.
static DslashCall mcall(eig_op_s *op, Field in, Field out, bool dag, bool f64, cudaStream_t s) {
    DslashCall c = op->call(in, out, dag, f64);
    if (!op->eo) return c;
    Field tmp = (f64 ? op->tmp64_e : op->tmp_e).view(in.v.k);
    DslashCall c1 = c;
    c1.out = tmp;
    c1.eo_parity = 0;
    c1.diag = 0.0;
    c1.hcoef = -0.5;
    CUDA_CK(launch_dslash(c1, s));
    c.in = tmp;
    c.cen = in;
    c.eo_parity = 1;
    c.hcoef = 0.5 / c.diag;
    return c;
}

static void apply_M(eig_op_s *op, Field in, Field out, bool dag, bool f64, cudaStream_t s) {
    CUDA_CK(launch_dslash(mcall(op, in, out, dag, f64, s), s));
}

// out = A in in FP64 (uses op->u64 as scratch; in/out must not be u64)
static void apply_A64(eig_op_s *op, Field in, Field out, cudaStream_t s) {
    Field u = op->u64.view(in.v.k);
    apply_M(op, in, u, false, true, s);
    apply_M(op, u, out, true, true, s);
}

// natural (host or device) -> internal FP64 field
static void load_natural(eig_op_s *op, const double *nat, Field dst, cudaStream_t s) {
    const size_t bytes = (size_t)dst.v.V * 12 * 16 * dst.v.k;
    const double *src = nat;
    if (!is_device_ptr(nat)) {
        CUDA_CK(cudaMemcpyAsync(op->nat_in.p, nat, bytes, cudaMemcpyHostToDevice, s));
        src = op->nat_in.as<double>();
    }
    CUDA_CK(launch_pack(src, dst, s));
}

static void store_natural(eig_op_s *op, Field src, double *nat, cudaStream_t s) {
    const size_t bytes = (size_t)src.v.V * 12 * 16 * src.v.k;
    if (is_device_ptr(nat)) {
        CUDA_CK(launch_unpack(src, nat, s));
    } else {
        CUDA_CK(launch_unpack(src, op->nat_out.as<double>(), s));
        CUDA_CK(cudaMemcpyAsync(nat, op->nat_out.p, bytes, cudaMemcpyDeviceToHost, s));
    }
}

// Loads b and the initial guess x (k RHS) of a solve.  Full-lattice operators: into
// b64 / x64.  Odd-even operators: b and x are full-lattice vectors of M x = b; b64
// receives M_hat^H b_hat with b_hat = b_o - (1/d) H_oe b_e, the right-hand side of the
// odd-site normal equations, x64 the odd part of x, and op->be64 keeps b_e.
static void load_solve(eig_op_s *op, const double *b, const double *x, Field b64, Field x64, cudaStream_t s) {
    if (!op->eo) {
        load_natural(op, b, b64, s);
        load_natural(op, x, x64, s);
        return;
    }
    const int k = b64.v.k;
    Field full = op->full64.view(k), be = op->be64.view(k), u = op->u64.view(k);
    const double d = 4.0 + op->m_q;
    load_natural(op, b, full, s);
    CUDA_CK(launch_parity_move(full, be, 0, op->L, true, s));
    CUDA_CK(launch_parity_move(full, b64, 1, op->L, true, s));
    DslashCall c = op->call(be, u, false, true);  // u = H_oe b_e
    c.eo_parity = 1;
    c.diag = 0.0;
    c.hcoef = -0.5;
    CUDA_CK(launch_dslash(c, s));
    CUDA_CK(launch_combine(b64, 1.0, b64, -1.0 / d, u, s));  // b_hat
    apply_M(op, b64, u, true, true, s);                        // M_hat^H b_hat
    CUDA_CK(launch_combine(b64, 1.0, u, 0.0, null_field(), s));
    load_natural(op, x, full, s);
    CUDA_CK(launch_parity_move(full, x64, 1, op->L, true, s));
}

// Stores a solve's solution.  Odd-even operators: x_e = (b_e - H_eo x_o) / d, then the
// full-lattice x from x_e and x_o.
static void store_solve(eig_op_s *op, Field x64, double *x, cudaStream_t s) {
    if (!op->eo) {
        store_natural(op, x64, x, s);
        return;
    }
    const int k = x64.v.k;
    Field full = op->full64.view(k), be = op->be64.view(k), t = op->tmp64_e.view(k);
    const double d = 4.0 + op->m_q;
    DslashCall c = op->call(x64, t, false, true);  // t = H_eo x_o
    c.eo_parity = 0;
    c.diag = 0.0;
    c.hcoef = -0.5;
    CUDA_CK(launch_dslash(c, s));
    CUDA_CK(launch_combine(be, 1.0 / d, be, -1.0 / d, t, s));
    CUDA_CK(launch_parity_move(full, be, 0, op->L, false, s));
    CUDA_CK(launch_parity_move(full, x64, 1, op->L, false, s));
    store_natural(op, full, x, s);
}

// ------------------------------------------------------------------------------------
// eigCG window state (Fig. 1 right box), host bookkeeping of device slots
// ------------------------------------------------------------------------------------
struct Window {
    int nev, m;
    int i = 0;               // vectors in the window
    int kh = 0;              // size of the restarted Ritz head
    int j0 = 1;              // iteration whose z sits at window index kh
    std::vector<double> Mh;  // head Ritz values
    std::vector<cd> trow;    // w^H V_new of the last restart (unnormalised)
    std::vector<int> slots;  // physical slot of window index
    std::vector<int> freel;  // free slots
    int restarts = 0;
    int save_prev_at = -1;   // iteration whose t goes to t_prev
    bool tprev_is_a = true;  // which buffer currently holds t_prev
};

// Builds T (n x n) of the current window from the device history (host copy).
static void window_T(const Window &w, int n, const double *ha, const double *hb, const double *hr,
                     std::vector<cd> &T) {
    T.assign((size_t)n * n, cd(0.0));
    for (int a = 0; a < w.kh && a < n; a++) T[(size_t)a * n + a] = w.Mh[a];
    if (w.kh > 0 && w.kh < n) {
        const double sr = std::sqrt(hr[w.j0 - 1]);
        for (int a = 0; a < w.kh; a++) {
            const cd v = w.trow[a] / sr;
            T[(size_t)w.kh * n + a] = v;
            T[(size_t)a * n + w.kh] = std::conj(v);
        }
    }
    for (int q = 0; w.kh + q < n; q++) {
        const int jj = w.j0 + q;
        const int ix = w.kh + q;
        T[(size_t)ix * n + ix] = 1.0 / ha[jj] + (jj > 1 ? hb[jj] / ha[jj - 1] : 0.0);
        if (q >= 1) {
            const double off = -std::sqrt(hb[jj]) / ha[jj - 1];
            T[(size_t)ix * n + ix - 1] = off;
            T[(size_t)(ix - 1) * n + ix] = off;
        }
    }
}

// ------------------------------------------------------------------------------------
// CG driver (single or batched)
// ------------------------------------------------------------------------------------
struct Solve {
    eig_op_s *op;
    cudaStream_t s;
    int k;
    bool mixed;
    Field b64, x64, r64, u64, r, p, u, xlo;
    History h;
    RedScratch red;
    CGScalars *st;
    CGScalars *sth;
    std::vector<int> reliable;  // per RHS
    std::vector<double> rmax;   // max ||r|| since last reliable update
    int j = 0;                  // last issued iteration
    int j_checked = 0;          // history read up to here
    int j_start = 0;            // iteration index the current CG run (re)started from
    double tol;
    // spectral preconditioner from the first spl vectors of spB (Sec. 2): z = P^{-1} r
    bool sp = false;
    Field z;
    eig_basis_s *spB = nullptr;
    int spl = 0;

    void read_scalars() {
        CUDA_CK(cudaMemcpyAsync(sth, st, sizeof(CGScalars) * k, cudaMemcpyDeviceToHost, s));
        sync(s);
    }
    void write_scalars() { CUDA_CK(cudaMemcpyAsync(st, sth, sizeof(CGScalars) * k, cudaMemcpyHostToDevice, s)); }
    void read_history(int upto) {
        double *hh = op->hist_h.as<double>();
        const size_t n = (size_t)(upto + 2) * k;
        CUDA_CK(cudaMemcpyAsync(hh, h.alpha, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_CK(cudaMemcpyAsync(hh + (size_t)h.cap * k, h.beta, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_CK(cudaMemcpyAsync(hh + 2 * (size_t)h.cap * k, h.rho, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        sync(s);
    }
    const double *ha() const { return op->hist_h.as<double>(); }
    const double *hb() const { return op->hist_h.as<double>() + (size_t)h.cap * k; }
    const double *hr() const { return op->hist_h.as<double>() + 2 * (size_t)h.cap * k; }

    // r64 = b - A x64; with set_rho the CG scalars take the true residual.  final:
    // FP64 arithmetic (the reported residual); otherwise, in mixed precision, the
    // double-float stencil (residual replacements between checks).
    void true_residual(bool set_rho, bool final_check = true) {
        CUDA_CK(launch_xflush(p, xlo, st, k, s));
        if (mixed) {
            CUDA_CK(launch_combine(x64, 1.0, x64, 1.0, xlo, s));
            zero_field(xlo, s);
        }
        if (mixed && !final_check && !op->eo) {
            const long n = op->Vf * 12 * (long)k;
            CUDA_CK(launch_to_dd(x64.v.data, r64.v.data, n, s));  // r64 holds x in dd until overwritten
            CUDA_CK(launch_dslash_dd(op->call(x64, u64, false, true), op->gauge_dd.p, r64.v.data, u64.v.data, s));
            CUDA_CK(launch_dslash_dd_resid(op->call(u64, r64, true, true), op->gauge_dd.p, u64.v.data, b64, r64, st, h,
                                           j, set_rho, red, s));
        } else {
            apply_M(op, x64, u64, false, true, s);
            CUDA_CK(launch_dslash_resid(mcall(op, u64, r64, true, true, s), b64, r64, st, h, j, set_rho, red, s));
        }
        if (mixed && set_rho) CUDA_CK(launch_combine(r, 1.0, r64, 0.0, null_field(), s));
    }

    // r64 = b64 - A x64 for the deflation of the initial guess (Eq. 1): r64 = b64 when
    // every x is zero, else the double-float stencil in mixed precision (full lattice)
    // or the FP64 one.
    void initial_residual() {
        CUDA_CK(launch_norm2(x64, st, false, h, 0, red, s));
        read_scalars();
        bool zero = true;
        for (int q = 0; q < k; q++) zero = zero && sth[q].aux == 0.0;
        if (zero) {
            CUDA_CK(launch_combine(r64, 1.0, b64, 0.0, null_field(), s));
        } else if (mixed && !op->eo) {
            const long n = op->Vf * 12 * (long)k;
            CUDA_CK(launch_to_dd(x64.v.data, r64.v.data, n, s));  // r64 holds x in dd until overwritten
            CUDA_CK(launch_dslash_dd(op->call(x64, u64, false, true), op->gauge_dd.p, r64.v.data, u64.v.data, s));
            CUDA_CK(launch_dslash_dd_resid(op->call(u64, r64, true, true), op->gauge_dd.p, u64.v.data, b64, r64, st, h,
                                           0, false, red, s));
        } else {
            apply_M(op, x64, u64, false, true, s);
            apply_M(op, u64, r64, true, true, s);
            CUDA_CK(launch_combine(r64, 1.0, b64, -1.0, r64, s));
        }
    }

    // Sets up r, rho, target from b64 and the initial guess in x64.
    void start(double tol_) {
        tol = tol_;
        CUDA_CK(launch_norm2(b64, st, false, h, 0, red, s));
        CUDA_CK(launch_cg_init(st, k, tol, h, s));
        if (mixed) zero_field(xlo, s);
        true_residual(false, false);
        if (mixed) CUDA_CK(launch_combine(r, 1.0, r64, 0.0, null_field(), s));
        CUDA_CK(launch_norm2(r64, st, true, h, 0, red, s));
        read_scalars();
        for (int q = 0; q < k; q++) {
            sth[q].iters = 0;
            sth[q].nit = 0;
            if (!(sth[q].aux > sth[q].target)) sth[q].active = 0;
            if (!std::isfinite(sth[q].aux)) {
                sth[q].active = 0;
                sth[q].breakdown = 1;
            }
        }
        write_scalars();
        j = 0;
        j_checked = 0;
        j_start = 0;
        rmax.assign(k, 0.0);
        for (int q = 0; q < k; q++) rmax[q] = std::sqrt(sth[q].aux);
        reliable.assign(k, 0);
    }

    // Reliable-update test on the history since the last check (host has read it).
    bool needs_reliable() {
        // only iterations since the last check count: right after a (re)start no history of
        // this run exists yet, and a replacement there would set beta != 0 for a direction
        // that must be the residual itself
        if (!mixed || j <= j_checked) return false;
        bool trig = false;
        const double *r_ = hr();
        for (int q = 0; q < k; q++) {
            if (!sth[q].active) continue;
            for (int jj = j_checked + 1; jj <= j; jj++) {
                const double rn = std::sqrt(r_[(size_t)jj * k + q]);
                if (rn > rmax[q]) rmax[q] = rn;
            }
            const double cur = std::sqrt(r_[(size_t)j * k + q]);
            if (cur < op->delta * rmax[q]) trig = true;
        }
        return trig;
    }
    // Iterations until the next host check.  From the decay of rho over the iterations
    // since the last check, the last active RHS is predicted to converge in n more
    // iterations: the next check comes after min(n, CHECK) iterations (at least one), so
    // that near convergence no iterations are launched for RHS that have stopped.
    // Needs the history read up to j.
    int iterations_to_next_check() const {
        if (j - j_start < 2) return CHECK;
        const int j0 = std::max(j_start + 1, j - CHECK);
        const double *r_ = hr();
        double worst = 0.0;
        for (int q = 0; q < k; q++) {
            if (!sth[q].active) continue;
            const double now = r_[(size_t)j * k + q], then = r_[(size_t)j0 * k + q];
            if (!(now > 0.0) || !(then > now) || !(sth[q].target > 0.0)) return CHECK;
            const double rate = std::log(now / then) / (j - j0);  // < 0
            worst = std::max(worst, std::log(sth[q].target / now) / rate);
        }
        return (int)std::min<double>(CHECK, std::max(1.0, std::floor(worst)));
    }
    void reliable_update() {
        true_residual(true, false);
        read_scalars();
        for (int q = 0; q < k; q++) {
            rmax[q] = std::sqrt(sth[q].rho);
            reliable[q]++;
        }
    }
};

static void check_breakdown(const Solve &sv) {
    for (int q = 0; q < sv.k; q++)
        if (sv.sth[q].breakdown) throw Error{EIG_ERR_BREAKDOWN, "CG breakdown (p^H A p <= 0, NaN or Inf)"};
}

static bool tc_gemm_enabled();
static ColSet field_cols(void *base, bool f64, int k, long fsize, int ncols, bool rhs_inner);

// Plain CG iterations of init-CG run as replays of a captured graph of CHECK
// iterations unless kernel timing is on (its events would be captured too) or
// EIG_CG_GRAPH=0 is set.
static bool cg_graphs_enabled() {
    if (prof_timing()) return false;
    const char *e = getenv("EIG_CG_GRAPH");
    return !(e && e[0] == '0');
}

// The graph of CHECK iterations j0 + 1 .. j0 + CHECK for this solve's buffers (j0 is
// read by the kernels from op->jbase_dev), captured on first use.
static cudaGraphExec_t cg_graph(Solve &sv, eig_op_s *op) {
    const std::vector<const void *> key = {(const void *)(long)sv.k, sv.r.v.data, sv.p.v.data, sv.u.v.data,
                                           sv.xlo.v.data, sv.st, sv.h.alpha, sv.h.beta, sv.h.rho,
                                           (const void *)(long)op->prec};
    for (auto &g : op->graphs)
        if (g.key == key) return g.exec;
    op->jbase_dev.ensure(16);
    op->jbase_h.ensure(16);
    History hg = sv.h;
    hg.jbase = op->jbase_dev.as<int>();
    eig_op_s::CgGraph gr;
    gr.key = key;
    if (!op->cap_stream) CUDA_CK(cudaStreamCreateWithFlags(&op->cap_stream, cudaStreamNonBlocking));
    // captured on a private stream (the caller's may be the legacy stream, which
    // cannot be captured); the graph is launched on the caller's stream
    cudaStream_t s = op->cap_stream;
    cudaGraph_t graph = nullptr;
    std::lock_guard<std::recursive_mutex> cap_lock(g_capture_mu);
    CUDA_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    prof_record_begin(&gr.rec);
    cudaError_t e = cudaSuccess;
    for (int t = 1; t <= CHECK && e == cudaSuccess; t++) {
        e = launch_pupdate(sv.r, sv.p, sv.xlo, false, sv.st, null_field(), s);
        if (e == cudaSuccess)
            e = launch_dslash_norm(mcall(op, sv.p, sv.u, false, op->prec == P64, s), sv.st, hg, t, sv.red, s);
        if (e == cudaSuccess)
            e = launch_dslash_cg(mcall(op, sv.u, sv.u, true, op->prec == P64, s), sv.r, null_field(), sv.st, hg, t,
                                 sv.red, s);
    }
    prof_record_end();
    const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        throw Error{EIG_ERR_CUDA, std::string("CG graph capture failed: ") +
                                      cudaGetErrorString(e != cudaSuccess ? e : e2)};
    }
    const cudaError_t e3 = cudaGraphInstantiate(&gr.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
        cudaGetLastError();
        throw Error{EIG_ERR_CUDA, std::string("CG graph instantiation failed: ") + cudaGetErrorString(e3)};
    }
    if (op->graphs.size() >= 4) {
        cudaGraphExecDestroy(op->graphs.front().exec);
        op->graphs.erase(op->graphs.begin());
    }
    op->graphs.push_back(std::move(gr));
    return op->graphs.back().exec;
}

static ColSet basis_cols(eig_basis_s *B, int first, int n);


// z = P^{-1} r = r + U_p (G (U_p^H r)) with the spectral preconditioner of the first spl
// basis vectors, then rho = r^H z and beta_j (Fig. 1 steps 3-4 and 8 in preconditioned
// form; iter = the last finished iteration).  No host synchronisation: the contractions'
// error flags are checked when the solve ends.
static void sp_apply(Solve &sv, int iter) {
    eig_op_s *op = sv.op;
    eig_basis_s *B = sv.spB;
    cudaStream_t s = sv.s;
    const bool f64 = op->wprec == P64;
    const long nrow = op->ncomplex();
    const ColSet U = basis_cols(B, 0, sv.spl);
    const ColSet R = field_cols(sv.r.v.data, f64, 1, nrow, 1, true);
    if (tc_gemm_enabled() && tc_ahb_ok(U, R))
        CUDA_CK(launch_tc_ahb(U, R, nrow, op->spC.as<double>(), op->sptc.as<double>(), op->sperr.as<int>(), s));
    else
        CUDA_CK(launch_gemm_ahb(U, R, nrow, op->spC.as<double>(), sv.red, s));
    CUDA_CK(launch_sp_coef(op->spG.as<double>(), op->spC.as<double>(), op->spY.as<double>(), sv.spl, s));
    CUDA_CK(launch_combine(sv.z, 1.0, sv.r, 0.0, null_field(), s));
    const ColSet Z = field_cols(sv.z.v.data, f64, 1, nrow, 1, true);
    if (tc_gemm_enabled() && (nrow % 2) == 0 && tc_ay_ok(U, Z)) {
        op->tcb.ensure(TC_AY_SCRATCH);
        CUDA_CK(launch_tc_ay(U, op->spY.as<double>(), Z, 1.0, nrow, op->sperr.as<int>() + 1, op->tcb.p, s));
    } else {
        CUDA_CK(launch_gemm_ay(U, op->spY.as<double>(), Z, 1.0, nrow, s));
    }
    CUDA_CK(launch_pcg_rho(sv.r, sv.z, sv.st, sv.h, iter, sv.red, s));
}

// EIG_CG_TRACE=1: one line per host check on stderr (diagnostics)
static bool cg_trace() {
    const char *e = getenv("EIG_CG_TRACE");
    return e && e[0] == '1';
}

// Runs CG iterations until every RHS is inactive or max_iter.  With a window,
// performs the eigCG additions.  Returns false if max_iter was hit.
static bool cg_run(Solve &sv, int max_iter, Window *w, eig_op_s *op) {
    cudaStream_t s = sv.s;
    const int k = sv.k;
    int since = CHECK;  // force a check at the start
    int next_check = CHECK;
    while (true) {
        const bool restart_now = w && w->i == w->m;
        if (since >= next_check || restart_now || sv.j >= max_iter) {
            sv.read_scalars();
            bool any = false;
            for (int q = 0; q < k; q++) any = any || sv.sth[q].active;
            if (w && !any && sv.sth[0].iters < sv.j) {
                // speculative iterations after convergence appended nothing
                const int skipped = sv.j - sv.sth[0].iters;
                for (int t = 0; t < skipped; t++) {
                    w->freel.push_back(w->slots.back());
                    w->slots.pop_back();
                    w->i--;
                }
                sv.j = sv.sth[0].iters;
            }
            if (!any) break;
            if (sv.j >= max_iter) return false;
            sv.read_history(sv.j);
            const bool rel = sv.needs_reliable();
            if (rel) {
                sv.reliable_update();
                check_breakdown(sv);
            }
            sv.j_checked = sv.j;
            since = 0;
            next_check = sv.iterations_to_next_check();
            if (cg_trace()) {
                fprintf(stderr, "cg j=%d next=%d reliable=%d", sv.j, next_check, (int)rel);
                for (int q = 0; q < k; q++)
                    fprintf(stderr, " | q%d act=%d nit=%d rho=%.3e xp=%d", q, sv.sth[q].active, sv.sth[q].nit,
                            sv.sth[q].rho, sv.sth[q].x_pending);
                fprintf(stderr, "\n");
            }
        }
        if (!w && !sv.sp && since == 0 && next_check == CHECK && sv.j >= 1 && sv.j + CHECK <= max_iter &&
            cg_graphs_enabled()) {
            // CHECK plain iterations as one replayed CUDA graph
            cudaGraphExec_t g = cg_graph(sv, op);
            *op->jbase_h.as<int>() = sv.j;
            CUDA_CK(cudaMemcpyAsync(op->jbase_dev.p, op->jbase_h.p, sizeof(int), cudaMemcpyHostToDevice, s));
            CUDA_CK(cudaGraphLaunch(g, s));
            for (const auto &gr : op->graphs)
                if (gr.exec == g) prof_replay(gr.rec);
            sv.j += CHECK;
            since = CHECK;
            continue;
        }
        const int j = ++sv.j;
        since++;
        Field vapp = null_field();
        int slot = -1;
        std::vector<cd> QZ;
        std::vector<double> Mnew;
        int nout = 0;
        if (w) {
            if (restart_now) {
                // Fig. 1 steps 11.3-11.6 on the host from T_m
                std::vector<cd> T;
                window_T(*w, w->m, sv.ha(), sv.hb(), sv.hr(), T);
                QZ.resize((size_t)w->m * 2 * w->nev);
                Mnew.resize(2 * w->nev);
                nout = dense::restart_coefficients(w->m, T.data(), w->kh, w->nev,
                                                   std::max(w->m, 2 * w->nev) * 2.2e-16, QZ.data(), Mnew.data());
                if (nout < 1) throw Error{EIG_ERR_BREAKDOWN, "eigCG restart basis is empty"};
                slot = w->freel.back();  // the spare slot
            } else {
                slot = w->freel.back();
            }
            w->freel.pop_back();
            vapp = field_at(op->wprec, (char *)op->win.p + (size_t)slot * op->wfield_bytes(), op->Vf, 1);
        }
        if (sv.sp) sp_apply(sv, j - 1);  // Fig. 1 steps 3-4 and 8 with P != I
        CUDA_CK(launch_pupdate(sv.sp ? sv.z : sv.r, sv.p, sv.xlo, j == 1, sv.st, vapp, s));
        CUDA_CK(launch_dslash_norm(mcall(op, sv.p, sv.u, false, op->prec == P64, s), sv.st, sv.h, j, sv.red, s));
        Field tsave = null_field();
        if (w) {
            const bool becomes_full = !restart_now && (w->i + 1 == w->m);
            void *tp = w->tprev_is_a ? op->tprev.p : op->tcur.p;
            void *tc = w->tprev_is_a ? op->tcur.p : op->tprev.p;
            if (restart_now) tsave = field_at(op->wprec, tc, op->Vf, 1);
            else if (becomes_full) tsave = field_at(op->wprec, tp, op->Vf, 1);
        }
        CUDA_CK(launch_dslash_cg(mcall(op, sv.u, sv.u, true, op->prec == P64, s), sv.r, tsave, sv.st, sv.h, j, sv.red,
                                 s));
        if (w) {
            if (restart_now) {
                // step 11.7 (V <- V QZ in place) fused with step 11.8 (w^H V)
                const int m = w->m;
                std::vector<long> off(m);
                const long fs = (long)op->Vf * 12;
                for (int a = 0; a < m; a++) off[a] = (long)w->slots[a] * fs;
                CUDA_CK(cudaMemcpyAsync(op->col_off.p, off.data(), m * sizeof(long), cudaMemcpyHostToDevice, s));
                // tensor-core path: A is the whole window (m + 1 evenly spaced slots, one 2D TMA
                // copy per tile chunk) and QZ's rows are placed at the slots of their columns; the
                // spare slot (this iteration's vector, written above) gets zero coefficients.  All
                // m + 1 slots were written during this solve, so none holds stale non-finite data.
                const bool tcw = op->wprec != P64 && nout <= 32 && (op->ncomplex() % 2) == 0 && tc_gemm_enabled();
                const int qrows = tcw ? m + 1 : m;
                std::vector<double> qz((size_t)qrows * nout * 2, 0.0);
                for (int a = 0; a < m; a++) {
                    const size_t row = tcw ? (size_t)w->slots[a] : (size_t)a;
                    for (int c = 0; c < nout; c++) {
                        qz[(row * nout + c) * 2] = QZ[(size_t)c * m + a].real();
                        qz[(row * nout + c) * 2 + 1] = QZ[(size_t)c * m + a].imag();
                    }
                }
                op->qz.ensure(qz.size() * sizeof(double));
                CUDA_CK(cudaMemcpyAsync(op->qz.p, qz.data(), qz.size() * sizeof(double), cudaMemcpyHostToDevice, s));
                ColSet Vw;
                Vw.base = op->win.p;
                Vw.f64 = op->wprec == P64;
                Vw.ki = 1;
                Vw.col_stride = 0;
                Vw.ncols = m;
                Vw.col_off = op->col_off.as<long>();
                void *tp = w->tprev_is_a ? op->tprev.p : op->tcur.p;
                void *tc = w->tprev_is_a ? op->tcur.p : op->tprev.p;
                if (tcw) {
                    // V <- V QZ on the tensor cores, in place (each CTA reads all m + 1 slots of
                    // its rows before writing them), then w^H V_new with w = t - beta t_prev
                    // formed on the fly
                    ColSet Out = Vw;
                    Out.ncols = nout;
                    Vw.col_off = nullptr;
                    Vw.col_stride = fs;
                    Vw.ncols = m + 1;
                    op->tcerr.ensure(16);
                    op->errh.ensure(16);
                    CUDA_CK(cudaMemsetAsync(op->tcerr.p, 0, 16, s));
                    op->tcb.ensure(TC_AY_SCRATCH);
                    CUDA_CK(launch_tc_ay(Vw, op->qz.as<double>(), Out, 0.0, op->ncomplex(), op->tcerr.as<int>(),
                                         op->tcb.p, s));
                    CUDA_CK(launch_wdot(tc, tp, sv.h.beta + (size_t)j * k, op->win.p, op->col_off.as<long>(), nout,
                                        op->ncomplex(), op->wv.as<double>(), sv.red, s));
                    CUDA_CK(cudaMemcpyAsync(op->errh.p, op->tcerr.p, 4, cudaMemcpyDeviceToHost, s));
                } else {
                    CUDA_CK(launch_window_restart(Vw, m, op->qz.as<double>(), nout, tc, tp, sv.h.beta + (size_t)j * k,
                                                  op->ncomplex(), op->wv.as<double>(), sv.red, s));
                }
                // the restart reads qz/col_off asynchronously: keep host vectors alive until done
                sync(s);
                if (tcw && *op->errh.as<int>() != 0)
                    throw Error{EIG_ERR_TIMEOUT, "tensor-core window restart: a bounded wait in the kernel gave up"};
                std::vector<double> wv(2 * nout);
                CUDA_CK(cudaMemcpy(wv.data(), op->wv.p, wv.size() * sizeof(double), cudaMemcpyDeviceToHost));
                std::vector<int> newslots(w->slots.begin(), w->slots.begin() + nout);
                for (int a = nout; a < m; a++) w->freel.push_back(w->slots[a]);
                newslots.push_back(slot);
                w->slots = newslots;
                w->kh = nout;
                w->Mh.assign(Mnew.begin(), Mnew.begin() + nout);
                w->trow.resize(nout);
                for (int c = 0; c < nout; c++) w->trow[c] = cd(wv[2 * c], wv[2 * c + 1]);
                w->j0 = j;
                w->i = nout + 1;
                w->restarts++;
                if (w->i == w->m) w->tprev_is_a = !w->tprev_is_a;  // this t is the next t_prev
            } else {
                w->slots.push_back(slot);
                w->i++;
            }
        }
    }
    check_breakdown(sv);
    return true;
}

// Final FP64 residual; re-activates RHS that missed tol (up to a few times).
static bool cg_finish(Solve &sv, int max_iter, Window *w, eig_op_s *op, int &extra_rounds) {
    sv.true_residual(true);
    sv.read_scalars();
    bool again = false;
    for (int q = 0; q < sv.k; q++) {
        const double bn2 = sv.sth[q].target / (sv.tol * sv.tol);
        const bool ok = sv.sth[q].aux <= sv.tol * sv.tol * bn2 * (1.0 + 1e-12) || bn2 == 0.0;
        if (!ok && !sv.sth[q].breakdown && sv.j < max_iter && extra_rounds < 8) {
            sv.sth[q].active = 1;
            again = true;
        }
    }
    if (again) {
        extra_rounds++;
        sv.write_scalars();
        for (int q = 0; q < sv.k; q++) sv.rmax[q] = std::sqrt(sv.sth[q].aux);
    }
    (void)w;
    (void)op;
    return again;
}

// Picks the stencil variant for this k on the op's own buffers (once per op shape).
static void tune_for(eig_op_s *op, int k, cudaStream_t s) {
    if (op->prec == P64) return;
    // tuned on the primary format's call (call() picks a format only once tuned)
    DslashCall c = op->call(op->p.view(k), op->u.view(k), false, false);
    c.gauge.data = op->gauge_in.p;
    c.gformat = op->gf_inner;
    if (op->eo) {  // the half stencil of the odd-even form, on half-lattice fields
        c.eo_parity = 1;
        c.cen = op->r.view(k);
        c.hcoef = 0.5 / c.diag;
    }
    const void *alts[1] = {op->gauge_alt.p};
    const int gfs[1] = {op->gf_alt};
    CUDA_CK(autotune_dslash32(c, alts, gfs, 1, s));
}

static Solve make_solve(eig_op_s *op, int k, cudaStream_t s, int max_iter) {
    tune_for(op, k, s);
    Solve sv;
    sv.op = op;
    sv.s = s;
    sv.k = k;
    sv.mixed = op->prec != P64;
    sv.b64 = op->b64.view(k);
    sv.x64 = op->x64.view(k);
    sv.u64 = op->u64.view(k);
    sv.p = op->p.view(k);
    sv.u = op->u.view(k);
    if (sv.mixed) {
        sv.r64 = op->r64.view(k);
        sv.r = op->r.view(k);
        sv.xlo = op->xlo.view(k);
    } else {
        sv.r64 = op->r.view(k);
        sv.r = sv.r64;
        sv.xlo = sv.x64;
    }
    op->ensure_history(max_iter + 2, k);
    sv.h = op->history(k);
    sv.red = op->red();
    sv.st = op->st.as<CGScalars>();
    sv.sth = op->st_h.as<CGScalars>();
    return sv;
}

// ------------------------------------------------------------------------------------
// basis operations
// ------------------------------------------------------------------------------------
static ColSet basis_cols(eig_basis_s *B, int first, int n) {
    ColSet c;
    c.base = (char *)B->U.p + (size_t)first * B->op->wfield_bytes();
    c.f64 = B->op->wprec == P64;
    c.ki = 1;
    c.col_stride = B->fsize();
    c.ncols = n;
    c.col_off = nullptr;
    return c;
}

static ColSet field_cols(void *base, bool f64, int k, long fsize, int ncols, bool rhs_inner) {
    ColSet c;
    c.base = base;
    c.f64 = f64;
    c.ki = rhs_inner ? k : 1;
    c.col_stride = rhs_inner ? 0 : fsize;
    c.ncols = ncols;
    c.col_off = nullptr;
    return c;
}

// Gram-Schmidt in coefficient space: given the Gram matrix G (n x n row-major) of n
// vectors, returns Rinv (column c = coefficients of kept orthonormal vector c, n x r
// column-major) and the kept original indices; vectors whose remainder norm is
// <= drop are skipped.  Two projection passes per vector.
static void gram_orth(const std::vector<cd> &G, int n, double drop, std::vector<cd> &Rinv, std::vector<int> &keep) {
    Rinv.assign((size_t)n * n, cd(0.0));
    keep.clear();
    auto gdot = [&](const cd *u, const cd *v) {
        cd acc = 0.0;
        for (int a = 0; a < n; a++)
            for (int b = 0; b < n; b++) acc += std::conj(u[a]) * G[(size_t)a * n + b] * v[b];
        return acc;
    };
    std::vector<cd> v(n);
    for (int c = 0; c < n; c++) {
        std::fill(v.begin(), v.end(), cd(0.0));
        v[c] = 1.0;
        for (int pass = 0; pass < 2; pass++)
            for (int q = 0; q < (int)keep.size(); q++) {
                const cd *u = &Rinv[(size_t)q * n];
                const cd d = gdot(u, v.data());
                for (int a = 0; a < n; a++) v[a] -= d * u[a];
            }
        const double nv = std::sqrt(std::max(0.0, gdot(v.data(), v.data()).real()));
        if (!(nv > drop)) continue;
        const int q = (int)keep.size();
        for (int a = 0; a < n; a++) Rinv[(size_t)q * n + a] = v[a] / nv;
        keep.push_back(c);
    }
}

static void refactor(eig_basis_s *B) {
    const int l = B->l;
    B->Lc = B->H;
    B->chol_ok = l == 0 || dense::cholesky(l, B->Lc.data());
}

// The FP32 contractions of deflation, growth and the eigCG restart run on the tensor
// cores unless EIG_GEMM_TC=0 is set (read at every call; CUDA-core kernels then).
static bool tc_gemm_enabled() {
    const char *e = getenv("EIG_GEMM_TC");
    return !(e && e[0] == '0');
}

// C = A^H B into B->C (device) and B->Ch (host; the stream is synchronised).  FP32
// column sets go to the tensor cores when tc_gemm_enabled(); their kernel's error
// flag is read back with C and checked here.
static const cd *ahb_to_host(eig_basis_s *B, const ColSet &A, const ColSet &Bc, long nrow, cudaStream_t s) {
    eig_op_s *op = B->op;
    const size_t cb = (size_t)A.ncols * Bc.ncols * 16;
    B->C.ensure(cb);
    B->Ch.ensure(cb + 16);
    const bool tc = tc_gemm_enabled() && tc_ahb_ok(A, Bc);
    if (tc) {
        B->tcpart.ensure(tc_ahb_partials_bytes(nrow, A.ncols, Bc.ncols));
        B->tcerr.ensure(16);
        CUDA_CK(cudaMemsetAsync(B->tcerr.p, 0, 16, s));
        CUDA_CK(launch_tc_ahb(A, Bc, nrow, B->C.as<double>(), B->tcpart.as<double>(), B->tcerr.as<int>(), s));
        CUDA_CK(cudaMemcpyAsync((char *)B->Ch.p + cb, B->tcerr.p, 4, cudaMemcpyDeviceToHost, s));
    } else {
        CUDA_CK(launch_gemm_ahb(A, Bc, nrow, B->C.as<double>(), op->red(), s));
    }
    CUDA_CK(cudaMemcpyAsync(B->Ch.p, B->C.p, cb, cudaMemcpyDeviceToHost, s));
    sync(s);
    if (tc && *reinterpret_cast<const int *>((const char *)B->Ch.p + cb) != 0)
        throw Error{EIG_ERR_TIMEOUT, "tensor-core A^H B: a bounded wait in the kernel gave up"};
    return B->Ch.as<cd>();
}

// Out = beta Out + A Y; FP32 column sets go to the tensor cores when
// tc_gemm_enabled(), with the kernel's error flag read back and checked.
static void ay_run(eig_basis_s *B, const ColSet &A, const double *Y, const ColSet &Out, double beta, long nrow,
                   cudaStream_t s) {
    if (tc_gemm_enabled() && (nrow % 2) == 0 && tc_ay_ok(A, Out)) {
        B->tcerr.ensure(16);
        B->errh.ensure(16);
        CUDA_CK(cudaMemsetAsync(B->tcerr.p, 0, 16, s));
        B->tcb.ensure(TC_AY_SCRATCH);
        CUDA_CK(launch_tc_ay(A, Y, Out, beta, nrow, B->tcerr.as<int>(), B->tcb.p, s));
        CUDA_CK(cudaMemcpyAsync(B->errh.p, B->tcerr.p, 4, cudaMemcpyDeviceToHost, s));
        sync(s);
        if (*B->errh.as<int>() != 0) throw Error{EIG_ERR_TIMEOUT, "tensor-core A Y: a bounded wait in the kernel gave up"};
        return;
    }
    CUDA_CK(launch_gemm_ay(A, Y, Out, beta, nrow, s));
}

// x64 <- x64 + U H^{-1} U^H r64 for k RHS (r64 given in FP64).
static void deflate_into(eig_basis_s *B, Field r64, Field x64, cudaStream_t s) {
    eig_op_s *op = B->op;
    const int l = B->l, k = r64.v.k;
    if (l == 0) return;
    if (!B->chol_ok) throw Error{EIG_ERR_BREAKDOWN, "H = U^H A U is not positive definite"};
    Field rsv = op->rsv.view(k);
    CUDA_CK(launch_combine(rsv, 1.0, r64, 0.0, null_field(), s));
    const bool f64 = op->wprec == P64;
    ColSet R = field_cols(rsv.v.data, f64, k, B->fsize(), k, true);
    const cd *Cc = ahb_to_host(B, basis_cols(B, 0, l), R, op->ncomplex(), s);
    // solve H y = c per RHS (C is l x k row-major)
    std::vector<cd> Yc((size_t)l * k);
    for (int a = 0; a < l; a++)
        for (int q = 0; q < k; q++) Yc[(size_t)q * l + a] = Cc[(size_t)a * k + q];
    dense::chol_solve(l, B->Lc.data(), Yc.data(), k);
    std::vector<cd> Yr((size_t)l * k);
    for (int a = 0; a < l; a++)
        for (int q = 0; q < k; q++) Yr[(size_t)a * k + q] = Yc[(size_t)q * l + a];
    B->Y.ensure((size_t)l * k * 16);
    CUDA_CK(cudaMemcpyAsync(B->Y.p, Yr.data(), Yr.size() * 16, cudaMemcpyHostToDevice, s));
    Field xsv = op->xsv.view(k);
    ColSet X = field_cols(xsv.v.data, f64, k, B->fsize(), k, true);
    ay_run(B, basis_cols(B, 0, l), B->Y.as<double>(), X, 0.0, op->ncomplex(), s);
    CUDA_CK(launch_combine(x64, 1.0, x64, 1.0, xsv, s));
    sync(s);  // Yr must outlive the async copy
}

// ------------------------------------------------------------------------------------
// BiCGSTAB on M deflated through g5 M (Sec. 1: A = M^H M = (g5 M)^2, so eigenvectors of
// A are eigenvectors of the Hermitian g5 M)
// ------------------------------------------------------------------------------------
// Z = the nz lowest Ritz vectors of A in span(U) (U S, H S = S Theta) and
// H5 = Z^H g5 M Z, kept until U changes.
static void g5_setup(eig_basis_s *B, int nz, cudaStream_t s) {
    if (B->z_gen == B->gen && B->z_n == nz) return;
    eig_op_s *op = B->op;
    const int l = B->l;
    const bool f64 = op->wprec == P64;
    const long nrow = op->ncomplex();
    const size_t wfb = op->wfield_bytes();
    std::vector<double> th(nz);
    std::vector<cd> S((size_t)l * nz);
    dense::herm_eig_lowest(l, B->H.data(), nz, th.data(), S.data());
    B->Z.ensure((size_t)nz * wfb);
    const ColSet Zc = field_cols(B->Z.p, f64, 1, B->fsize(), nz, false);
    for (int c0 = 0; c0 < nz; c0 += MAX_NEV) {  // Z = U S, MAX_NEV columns per pass over U
        const int nc = std::min(MAX_NEV, nz - c0);
        std::vector<double> yr((size_t)l * nc * 2);
        for (int a = 0; a < l; a++)
            for (int c = 0; c < nc; c++) {
                yr[((size_t)a * nc + c) * 2] = S[(size_t)(c0 + c) * l + a].real();
                yr[((size_t)a * nc + c) * 2 + 1] = S[(size_t)(c0 + c) * l + a].imag();
            }
        B->Y.ensure(yr.size() * sizeof(double));
        CUDA_CK(cudaMemcpyAsync(B->Y.p, yr.data(), yr.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        const ColSet Zpart = field_cols((char *)B->Z.p + (size_t)c0 * wfb, f64, 1, B->fsize(), nc, false);
        ay_run(B, basis_cols(B, 0, l), B->Y.as<double>(), Zpart, 0.0, nrow, s);
        sync(s);  // yr must outlive the async copy
    }
    std::vector<cd> H5((size_t)nz * nz);
    for (int c0 = 0; c0 < nz; c0 += MAX_NEV) {
        const int nc = std::min(MAX_NEV, nz - c0);
        for (int j = 0; j < nc; j++) {  // W_j = g5 M z_(c0 + j)
            Field zj = field_at(op->wprec, (char *)B->Z.p + (size_t)(c0 + j) * wfb, op->Vf, 1);
            Field wj = field_at(op->wprec, (char *)B->W.p + (size_t)j * wfb, op->Vf, 1);
            apply_M(op, zj, wj, false, f64, s);
            CUDA_CK(launch_gamma5(wj, wj, s));
        }
        const cd *C = ahb_to_host(B, Zc, field_cols(B->W.p, f64, 1, B->fsize(), nc, false), nrow, s);
        for (int a = 0; a < nz; a++)
            for (int c = 0; c < nc; c++) H5[(size_t)a * nz + c0 + c] = C[(size_t)a * nc + c];
    }
    B->H5 = std::move(H5);
    B->z_n = nz;
    B->z_gen = B->gen;
}

// x64 += Z H5^{-1} Z^H g5 r64: the Galerkin condition of Eq. 1 for g5 M x = g5 b on span(Z)
static void g5_deflate(eig_basis_s *B, Field r64, Field x64, cudaStream_t s) {
    eig_op_s *op = B->op;
    const int nz = B->z_n;
    const bool f64 = op->wprec == P64;
    const long nrow = op->ncomplex();
    Field rsv = op->rsv.view(1);
    CUDA_CK(launch_combine(rsv, 1.0, r64, 0.0, null_field(), s));
    CUDA_CK(launch_gamma5(rsv, rsv, s));
    const ColSet Zc = field_cols(B->Z.p, f64, 1, B->fsize(), nz, false);
    const cd *C = ahb_to_host(B, Zc, field_cols(rsv.v.data, f64, 1, B->fsize(), 1, true), nrow, s);
    std::vector<cd> A5 = B->H5, y(C, C + nz);
    if (!dense::lu_solve(nz, A5.data(), y.data(), 1)) throw Error{EIG_ERR_BREAKDOWN, "Z^H g5 M Z is singular"};
    B->Y.ensure((size_t)nz * 16);
    CUDA_CK(cudaMemcpyAsync(B->Y.p, y.data(), (size_t)nz * 16, cudaMemcpyHostToDevice, s));
    Field xsv = op->xsv.view(1);
    ay_run(B, Zc, B->Y.as<double>(), field_cols(xsv.v.data, f64, 1, B->fsize(), 1, true), 0.0, nrow, s);
    CUDA_CK(launch_combine(x64, 1.0, x64, 1.0, xsv, s));
    sync(s);  // y must outlive the async copy
}

}  // namespace eig

// ------------------------------------------------------------------------------------
// basis files
// ------------------------------------------------------------------------------------
namespace eig {

// FNV-1a mixing (xor, multiply by the 64-bit FNV prime) applied per 64-bit word of the
// FP64 links: identifies the gauge field a saved basis belongs to.
static unsigned long long links_fingerprint(const double *g, size_t n) {
    unsigned long long h = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; i++) {
        unsigned long long w;
        memcpy(&w, g + i, sizeof w);
        h = (h ^ w) * 0x100000001b3ull;
    }
    return h;
}

// 64-byte header of a basis file; then H (l x l complex FP64, row-major) and the l
// vectors in natural layout (fsize complex entries each, real_bytes per real).
struct BasisFileHeader {
    char magic[8];
    int32_t version;
    int32_t dims[4];
    int32_t even_odd;
    int32_t real_bytes;
    int32_t l;
    int64_t fsize;
    double m_q;
    unsigned long long gauge_hash;
};
static_assert(sizeof(BasisFileHeader) == 64, "basis file header layout");
static const char BASIS_MAGIC[8] = {'E', 'I', 'G', 'B', 'A', 'S', 'I', 'S'};

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

static void io_check(bool ok, const std::string &what) {
    if (!ok) throw Error{EIG_ERR_IO, what};
}

}  // namespace eig

// ======================================================================================
// C ABI
// ======================================================================================
#define API_BEGIN try {
#define API_END                                   \
    }                                             \
    catch (const eig::Error &e) {                 \
        eig::set_error(e);                        \
        return e.st;                              \
    }                                             \
    catch (const std::exception &e) {             \
        eig::g_last_error = e.what();             \
        return EIG_ERR_CUDA;                      \
    }                                             \
    return EIG_OK;

#define ARG_CHECK(cond, msg)                                  \
    do {                                                      \
        if (!(cond)) throw eig::Error{EIG_ERR_ARG, (msg)};    \
    } while (0)

extern "C" {

const char *eig_last_error(void) { return eig::g_last_error.c_str(); }

eig_status eig_profile_enable(int on) {
    API_BEGIN
    eig::prof_enable(on != 0);
    API_END
}

eig_status eig_profile_reset(void) {
    API_BEGIN
    eig::prof_reset();
    API_END
}

eig_status eig_profile_read(eig_kernel_stat *out, int max, int *n) {
    API_BEGIN
    ARG_CHECK(n, "null argument");
    static_assert(sizeof(eig_kernel_stat) == sizeof(eig::KernelStat), "layout");
    *n = eig::prof_read(reinterpret_cast<eig::KernelStat *>(out), out ? max : 0);
    API_END
}

eig_status eig_profile_alu_peak(int prec, double *tflops, void *stream) {
    API_BEGIN
    ARG_CHECK(tflops && (prec == 64 || prec == 32), "prec must be 64 or 32, tflops non-null");
    CUDA_CK(eig::alu_peak(prec, tflops, (cudaStream_t)stream));
    API_END
}

eig_status eig_op_create(const double *gauge, const int dims[4], double m_q, const eig_op_opts *opts, eig_op *out) {
    API_BEGIN
    ARG_CHECK(gauge && dims && out, "null argument");
    *out = nullptr;
    long V = 1;
    for (int i = 0; i < 4; i++) {
        ARG_CHECK(dims[i] >= 2 && dims[i] <= 4096, "lattice extents must be in [2, 4096]");
        V *= dims[i];
    }
    ARG_CHECK(V <= (1L << 27), "lattice too large");
    ARG_CHECK(std::isfinite(m_q), "m_q must be finite");
    eig_op_opts o;
    if (opts) o = *opts;
    else {
        o.spinor_prec = EIG_PREC_F64;
        o.link_compress12 = 1;
        o.max_rhs = 1;
        o.reliable_delta = 0.1;
        o.even_odd = 0;
    }
    ARG_CHECK(o.even_odd == 0 || o.even_odd == 1, "even_odd must be 0 or 1");
    if (o.even_odd)
        for (int i = 0; i < 4; i++) ARG_CHECK(dims[i] % 2 == 0, "the odd-even form needs every lattice extent even");
    ARG_CHECK(o.spinor_prec == 64 || o.spinor_prec == 32 || o.spinor_prec == 16, "spinor_prec must be 64, 32 or 16");
    ARG_CHECK(o.max_rhs >= 1 && o.max_rhs <= MAX_RHS && (o.max_rhs & (o.max_rhs - 1)) == 0,
              "max_rhs must be a power of two in [1, 16]");
    // the FP32/FP16 stencil addresses fields and link planes with 32-bit offsets
    ARG_CHECK((unsigned long long)V * o.max_rhs * 6ull < (1ull << 32) && 36ull * V < (1ull << 32),
              "lattice volume times max_rhs too large for one op");
    std::unique_ptr<eig_op_s> op(new eig_op_s());
    for (int i = 0; i < 4; i++) op->L[i] = dims[i];
    op->V = V;
    op->eo = o.even_odd == 1;
    op->Vf = op->eo ? V / 2 : V;
    op->m_q = m_q;
    op->prec = o.spinor_prec == 64 ? P64 : (o.spinor_prec == 32 ? P32 : P16);
    op->wprec = op->prec == P64 ? P64 : P32;
    // half-precision spinors keep FP32 links (12 reals): links rounded to FP16 perturb the
    // operator the Krylov recurrences see by ~3e-4, and between residual replacements CG
    // then converges on that operator instead of A (many more iterations at cond 1e4-1e5);
    // at k RHS per launch the links are 1/k of the stencil's bytes
    op->gf_inner = op->prec == P64 ? GF_F64_18 : (op->prec == P32 ? (o.link_compress12 ? GF_F32_12 : GF_F32_18) : GF_F32_12);
    op->max_rhs = o.max_rhs;
    op->delta = (o.reliable_delta > 0.0 && o.reliable_delta < 1.0) ? o.reliable_delta : 0.1;
    const int K = o.max_rhs;
    op->gauge_hash = links_fingerprint(gauge, (size_t)V * 4 * 9 * 2);
    // gauge: host -> device staging -> packed formats
    eig::DevBuf stage;
    stage.alloc((size_t)V * 4 * 9 * 16);
    CUDA_CK(cudaMemcpy(stage.p, gauge, stage.n, cudaMemcpyHostToDevice));
    op->gauge64.alloc((size_t)V * 4 * 9 * 16);
    CUDA_CK(launch_pack_gauge(stage.as<double>(), op->gauge64.p, GF_F64_18, V, 0));
    if (op->prec != P64) {
        op->gauge_dd.alloc((size_t)V * 4 * 9 * 16);
        CUDA_CK(launch_to_dd(op->gauge64.p, op->gauge_dd.p, V * 4 * 9, 0));
        size_t gb = op->gf_inner == GF_F32_12 ? 48 : (op->gf_inner == GF_F32_18 ? 72 : 24);
        op->gauge_in.alloc((size_t)V * 4 * gb);
        CUDA_CK(launch_pack_gauge(stage.as<double>(), op->gauge_in.p, op->gf_inner, V, 0));
        if (op->prec == P32) {
            // the other FP32 link format as well: 12 reals win where the stencil is
            // memory bound (few RHS), 18 reals where it is issue bound (many RHS)
            op->gf_alt = op->gf_inner == GF_F32_12 ? GF_F32_18 : GF_F32_12;
            op->gauge_alt.alloc((size_t)V * 4 * (op->gf_alt == GF_F32_12 ? 48 : 72));
            CUDA_CK(launch_pack_gauge(stage.as<double>(), op->gauge_alt.p, op->gf_alt, V, 0));
        }
    }
    {
        std::lock_guard<std::recursive_mutex> cap_lock(g_capture_mu);
        CUDA_CK(cudaDeviceSynchronize());
    }
    ensure_workspace(op.get());
    op->st.alloc(sizeof(CGScalars) * MAX_RHS);
    op->st_h.ensure(sizeof(CGScalars) * MAX_RHS);
    op->red_partials.alloc((size_t)RED_BLOCKS * MAX_RHS * 64 * sizeof(double));
    op->red_counter.alloc(64);
    CUDA_CK(cudaMemset(op->red_counter.p, 0, 64));
    op->ensure_history(1024, K);
    *out = op.release();
    API_END
}

eig_status eig_op_destroy(eig_op op) {
    API_BEGIN
    if (op) {
        std::lock_guard<std::recursive_mutex> cap_lock(g_capture_mu);
        cudaDeviceSynchronize();
        delete op;
    }
    API_END
}

eig_status eig_op_trim(eig_op op, size_t *freed) {
    API_BEGIN
    ARG_CHECK(op, "null argument");
    std::lock_guard<std::mutex> lk(op->mu);
    std::lock_guard<std::recursive_mutex> cap_lock(g_capture_mu);  // held over the sync and the frees
    CUDA_CK(cudaDeviceSynchronize());
    size_t bytes = 0;
    for (const FieldBuf *f : {&op->r, &op->p, &op->u, &op->b64, &op->x64, &op->u64, &op->xlo, &op->r64, &op->rsv,
                              &op->xsv, &op->tmp_e, &op->tmp64_e, &op->full64, &op->be64, &op->zsp, &op->bc_rh,
                              &op->bc_s, &op->bc_t})
        bytes += f->data.n + f->scale.n;
    bytes += op->nat_in.n + op->nat_out.n + op->win.n + op->tprev.n + op->tcur.n;
    release_workspace(op);
    if (freed) *freed = bytes;
    API_END
}

eig_status eig_op_apply(eig_op op, int which, const double *in, double *out, int k, void *stream) {
    API_BEGIN
    ARG_CHECK(op && in && out, "null argument");
    ARG_CHECK(which >= 0 && which <= 3, "which must be 0 (M), 1 (M^H), 2 (A) or 3 (A in double-float)");
    ARG_CHECK(which != 3 || op->prec != P64, "which = 3 needs an FP32 or FP16 op");
    ARG_CHECK(which != 3 || !op->eo, "which = 3 is not available for odd-even operators");
    ARG_CHECK(k >= 1 && k <= op->max_rhs && (k & (k - 1)) == 0, "k must be a power of two <= max_rhs");
    std::lock_guard<std::mutex> lk(op->mu);
    ensure_workspace(op);
    cudaStream_t s = (cudaStream_t)stream;
    Field x64 = op->x64.view(k);
    load_natural(op, in, x64, s);
    if (which == 3) {  // A = M^H M in double-float arithmetic
        const long n = op->Vf * 12 * (long)k;
        Field t1 = op->u64.view(k), t2 = op->r64.view(k);
        CUDA_CK(launch_to_dd(x64.v.data, t1.v.data, n, s));
        CUDA_CK(launch_dslash_dd(op->call(x64, t2, false, true), op->gauge_dd.p, t1.v.data, t2.v.data, s));
        CUDA_CK(launch_dslash_dd(op->call(x64, t1, true, true), op->gauge_dd.p, t2.v.data, t1.v.data, s));
        CUDA_CK(launch_from_dd(t1.v.data, x64.v.data, n, s));
        store_natural(op, x64, out, s);
        sync(s);
        return EIG_OK;
    }
    Field a = op->p.view(k), b = op->u.view(k), c = op->r.view(k);
    CUDA_CK(launch_combine(a, 1.0, x64, 0.0, null_field(), s));
    const bool f64 = op->prec == P64;
    if (which == 0) apply_M(op, a, b, false, f64, s);
    else if (which == 1) apply_M(op, a, b, true, f64, s);
    else {
        apply_M(op, a, c, false, f64, s);
        apply_M(op, c, b, true, f64, s);
    }
    CUDA_CK(launch_combine(x64, 1.0, b, 0.0, null_field(), s));
    store_natural(op, x64, out, s);
    sync(s);
    API_END
}

eig_status eig_op_stencil_choice(eig_op op, int k, int *variant, int *link_reals) {
    API_BEGIN
    ARG_CHECK(op && variant && link_reals, "null argument");
    ARG_CHECK(k >= 1 && k <= op->max_rhs && (k & (k - 1)) == 0, "k must be a power of two <= max_rhs");
    *variant = -1;
    *link_reals = 0;
    if (op->prec == P64) return EIG_OK;
    // the call tune_for times: the primary link format, half stencil for odd-even ops
    DslashCall c = op->call(op->p.view(k), op->u.view(k), false, false);
    c.gauge.data = op->gauge_in.p;
    c.gformat = op->gf_inner;
    if (op->eo) {
        c.eo_parity = 1;
        c.cen = op->r.view(k);
        c.hcoef = 0.5 / c.diag;
    }
    const int gf = dslash32_choice(c, variant);
    *link_reals = gf < 0 ? 0 : (gf == GF_F32_12 || gf == GF_F16_12 ? 12 : 18);
    API_END
}

eig_status eig_basis_create(eig_op op, int max_vecs, eig_basis *out) {
    API_BEGIN
    ARG_CHECK(op && out, "null argument");
    ARG_CHECK(max_vecs >= 1 && max_vecs <= 256, "max_vecs must be in [1, 256]");
    *out = nullptr;
    std::unique_ptr<eig_basis_s> B(new eig_basis_s());
    B->op = op;
    B->max_vecs = max_vecs;
    B->U.alloc((size_t)max_vecs * op->wfield_bytes());
    B->pend.alloc((size_t)MAX_NEV * op->wfield_bytes());
    B->W.alloc((size_t)MAX_NEV * op->wfield_bytes());
    *out = B.release();
    API_END
}

eig_status eig_basis_destroy(eig_basis basis) {
    API_BEGIN
    if (basis) {
        std::lock_guard<std::recursive_mutex> cap_lock(g_capture_mu);
        cudaDeviceSynchronize();
        delete basis;
    }
    API_END
}

eig_status eig_basis_size(eig_basis basis, int *l) {
    API_BEGIN
    ARG_CHECK(basis && l, "null argument");
    *l = basis->l;
    API_END
}

eig_status eig_basis_truncate(eig_basis basis, int l) {
    API_BEGIN
    ARG_CHECK(basis, "null argument");
    ARG_CHECK(l >= 0 && l <= basis->l, "l must be in [0, current size]");
    std::lock_guard<std::mutex> lk(basis->mu);
    const int old = basis->l;
    std::vector<cd> H((size_t)l * l);
    for (int a = 0; a < l; a++)
        for (int b = 0; b < l; b++) H[(size_t)a * l + b] = basis->H[(size_t)a * old + b];
    basis->H = H;
    basis->l = l;
    basis->gen++;
    basis->npend = 0;
    refactor(basis);
    API_END
}

// eigCG (Fig. 1) on one RHS; with sp_vecs > 0 preconditioned by the spectral
// preconditioner of the basis' first sp_vecs vectors (Sec. 2): P^{-1} = (I - U_p U_p^H) +
// sp_shift U_p H_p^{-1} U_p^H, applied as r + U_p (sp_shift H_p^{-1} - I) U_p^H r.
static eig_status eigcg_impl(eig_op op, eig_basis basis, const double *b, double *x, int nev, int m, double tol,
                             int max_iter, int sp_vecs, double sp_shift, eig_stats *stats, void *stream) {
    API_BEGIN
    ARG_CHECK(op && b && x, "null argument");
    ARG_CHECK(sp_vecs == 0 || (basis && sp_vecs >= 1 && sp_vecs <= basis->l),
              "sp_vecs must be 0 or in [1, basis size]");
    ARG_CHECK(sp_vecs == 0 || (std::isfinite(sp_shift) && sp_shift > 0.0), "sp_shift must be positive");
    ARG_CHECK(sp_vecs == 0 || op->prec != P16, "spectral preconditioning needs an FP64 or FP32 op");
    ARG_CHECK(nev >= 1 && nev <= MAX_NEV, "nev must be in [1, 16]");
    ARG_CHECK(m > 2 * nev && m <= MAX_WINDOW, "need 2*nev < m <= 128");
    ARG_CHECK(tol > 0.0 && tol < 1.0, "tol must be in (0, 1)");
    ARG_CHECK(max_iter >= 1 && max_iter <= 10000000, "max_iter out of range");
    ARG_CHECK(!basis || basis->op == op, "basis belongs to another op");
    std::lock_guard<std::mutex> lk(op->mu);
    ensure_workspace(op);
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    // window storage: m + 1 slots, t_prev, t_cur
    const size_t fb = op->wfield_bytes();
    if (op->win_slots < m + 1) {
        op->win.alloc((size_t)(m + 1) * fb);
        op->win_slots = m + 1;
    }
    op->tprev.ensure(fb);
    op->tcur.ensure(fb);
    op->col_off.ensure(MAX_WINDOW * sizeof(long));
    op->qz.ensure((size_t)MAX_WINDOW * 2 * MAX_NEV * 16);
    op->wv.ensure(2 * MAX_NEV * 16);
    Solve sv = make_solve(op, 1, s, max_iter);
    load_solve(op, b, x, sv.b64, sv.x64, s);
    if (basis && basis->l > 0) {
        // init-CG part of the Sec. 4 box: x0 = x~0 + U H^{-1} U^H (b - A x~0)
        sv.initial_residual();
        deflate_into(basis, sv.r64, sv.x64, s);
    }
    sv.start(tol);
    if (sp_vecs > 0) {
        // G = shift H_p^{-1} - I from the leading sp_vecs x sp_vecs block of H
        const int lp = sp_vecs, l = basis->l;
        std::vector<cd> L((size_t)lp * lp), Inv((size_t)lp * lp, cd(0.0));
        for (int a = 0; a < lp; a++)
            for (int c = 0; c < lp; c++) L[(size_t)a * lp + c] = basis->H[(size_t)a * l + c];
        if (!dense::cholesky(lp, L.data())) throw Error{EIG_ERR_BREAKDOWN, "leading block of H is not positive definite"};
        for (int a = 0; a < lp; a++) Inv[(size_t)a * lp + a] = 1.0;
        dense::chol_solve(lp, L.data(), Inv.data(), lp);  // column q: H_p^{-1} e_q
        std::vector<double> G((size_t)lp * lp * 2);
        for (int a = 0; a < lp; a++)
            for (int c = 0; c < lp; c++) {
                const cd g = sp_shift * Inv[(size_t)c * lp + a] - (a == c ? 1.0 : 0.0);
                G[((size_t)a * lp + c) * 2] = g.real();
                G[((size_t)a * lp + c) * 2 + 1] = g.imag();
            }
        op->spG.ensure(G.size() * sizeof(double));
        CUDA_CK(cudaMemcpyAsync(op->spG.p, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        if (op->zsp.kcap < 1) op->zsp.alloc(op->prec, op->Vf, 1);
        op->spC.ensure((size_t)lp * 16);
        op->spY.ensure((size_t)lp * 16);
        op->sptc.ensure(tc_ahb_partials_bytes(op->ncomplex(), lp, 1));
        op->sperr.ensure(16);
        op->sperrh.ensure(16);
        CUDA_CK(cudaMemsetAsync(op->sperr.p, 0, 16, s));
        sync(s);  // G must outlive the async copy
        sv.sp = true;
        sv.z = op->zsp.view(1);
        sv.spB = basis;
        sv.spl = lp;
    }
    Window w;
    w.nev = nev;
    w.m = m;
    for (int q = m; q >= 0; q--) w.freel.push_back(q);  // slot 0 popped first
    int rounds = 0;
    bool ok = true;
    while (true) {
        ok = cg_run(sv, max_iter, &w, op);
        if (!ok) {
            sv.true_residual(false);  // folds x_lo (and a pending alpha p) into x
            sv.read_scalars();
            break;
        }
        if (!cg_finish(sv, max_iter, &w, op, rounds)) break;
    }
    if (sv.sp) {
        CUDA_CK(cudaMemcpyAsync(op->sperrh.p, op->sperr.p, 8, cudaMemcpyDeviceToHost, s));
        sync(s);
        if (op->sperrh.as<int>()[0] != 0 || op->sperrh.as<int>()[1] != 0)
            throw Error{EIG_ERR_TIMEOUT, "spectral preconditioner: a bounded wait in a tensor-core kernel gave up"};
    }
    // eigCG output: nev lowest Ritz pairs of the final window
    int nr = 0;
    const int J = sv.j;
    if (w.i > 0) {
        sv.read_history(J);
        std::vector<cd> T;
        window_T(w, w.i, sv.ha(), sv.hb(), sv.hr(), T);
        nr = std::min(nev, w.i);
        std::vector<double> ev(nr);
        std::vector<cd> Y((size_t)w.i * nr);
        dense::window_lowest(w.i, T.data(), w.kh, w.i, nr, ev.data(), Y.data());
        if (basis) {
            std::vector<long> off(w.i);
            const long fs = op->ncomplex();
            for (int a = 0; a < w.i; a++) off[a] = (long)w.slots[a] * fs;
            CUDA_CK(cudaMemcpyAsync(op->col_off.p, off.data(), w.i * sizeof(long), cudaMemcpyHostToDevice, s));
            // after a restart every one of the m + 1 slots was written during this solve: then A
            // is the whole window, evenly spaced (one 2D TMA copy per tile chunk on the tensor
            // cores), with Y's rows placed at the slots of their columns and zeros elsewhere
            const bool whole = w.restarts > 0;
            const int yrows = whole ? w.m + 1 : w.i;
            std::vector<double> yr((size_t)yrows * nr * 2, 0.0);
            for (int a = 0; a < w.i; a++) {
                const size_t row = whole ? (size_t)w.slots[a] : (size_t)a;
                for (int c = 0; c < nr; c++) {
                    yr[(row * nr + c) * 2] = Y[(size_t)c * w.i + a].real();
                    yr[(row * nr + c) * 2 + 1] = Y[(size_t)c * w.i + a].imag();
                }
            }
            basis->Y.ensure(yr.size() * sizeof(double));
            CUDA_CK(cudaMemcpyAsync(basis->Y.p, yr.data(), yr.size() * sizeof(double), cudaMemcpyHostToDevice, s));
            ColSet A;
            A.base = op->win.p;
            A.f64 = op->wprec == P64;
            A.ki = 1;
            A.col_stride = whole ? fs : 0;
            A.ncols = yrows;
            A.col_off = whole ? nullptr : op->col_off.as<long>();
            ColSet O = field_cols(basis->pend.p, A.f64, 1, basis->fsize(), nr, false);
            ay_run(basis, A, basis->Y.as<double>(), O, 0.0, op->ncomplex(), s);
            sync(s);
            basis->npend = nr;
            basis->pend_ritz = ev;
        }
    } else if (basis) {
        basis->npend = 0;
    }
    store_solve(op, sv.x64, x, s);
    sync(s);
    if (stats) {
        stats->iters = J;
        stats->restarts = w.restarts;
        int rel = 0;
        for (int v : sv.reliable) rel += v;
        stats->reliable_updates = rel;
        const double bn2 = sv.sth[0].target / (tol * tol);
        stats->true_rel_res = bn2 > 0 ? std::sqrt(sv.sth[0].aux / bn2) : 0.0;
        stats->converged = stats->true_rel_res <= tol * (1 + 1e-12) ? 1 : 0;
        stats->n_ritz = nr;
        stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!ok) {
        eig::g_last_error = "max_iter reached";
        return EIG_NOT_CONVERGED;
    }
    API_END
}

eig_status eig_eigcg_solve(eig_op op, eig_basis basis, const double *b, double *x, int nev, int m, double tol,
                           int max_iter, eig_stats *stats, void *stream) {
    return eigcg_impl(op, basis, b, x, nev, m, tol, max_iter, 0, 0.0, stats, stream);
}

eig_status eig_eigcg_solve_sp(eig_op op, eig_basis basis, const double *b, double *x, int nev, int m, double tol,
                              int max_iter, int sp_vecs, double sp_shift, eig_stats *stats, void *stream) {
    if (sp_vecs < 1) {
        eig::g_last_error = "sp_vecs must be >= 1 (eig_eigcg_solve solves without a preconditioner)";
        return EIG_ERR_ARG;
    }
    return eigcg_impl(op, basis, b, x, nev, m, tol, max_iter, sp_vecs, sp_shift, stats, stream);
}

eig_status eig_basis_grow(eig_basis B, void *stream) {
    API_BEGIN
    ARG_CHECK(B, "null argument");
    std::lock_guard<std::mutex> lk(B->mu);
    std::lock_guard<std::mutex> lk2(B->op->mu);
    ensure_workspace(B->op);
    eig_op_s *op = B->op;
    cudaStream_t s = (cudaStream_t)stream;
    const int np = B->npend;
    if (np == 0) return EIG_OK;
    const int l = B->l;
    const bool f64 = op->wprec == P64;
    const long nrow = op->ncomplex();
    ColSet P = field_cols(B->pend.p, f64, 1, B->fsize(), np, false);
    // classical Gram-Schmidt against U, twice
    if (l > 0) {
        for (int pass = 0; pass < 2; pass++) {
            const double *c = reinterpret_cast<const double *>(ahb_to_host(B, basis_cols(B, 0, l), P, nrow, s));
            std::vector<double> negc((size_t)l * np * 2);
            for (size_t q = 0; q < negc.size(); q++) negc[q] = -c[q];
            B->Y.ensure(negc.size() * sizeof(double));
            CUDA_CK(cudaMemcpyAsync(B->Y.p, negc.data(), negc.size() * sizeof(double), cudaMemcpyHostToDevice, s));
            ay_run(B, basis_cols(B, 0, l), B->Y.as<double>(), P, 1.0, nrow, s);
            sync(s);
        }
    }
    // orthonormalise the remainders among themselves: pivoted Cholesky of the Gram matrix
    const cd *Gp = ahb_to_host(B, P, P, nrow, s);
    std::vector<cd> G(Gp, Gp + (size_t)np * np);
    const double drop = f64 ? 1e-10 : 1e-4;
    std::vector<cd> Rinv;
    std::vector<int> keep;
    gram_orth(G, np, drop, Rinv, keep);
    const int r = (int)keep.size();
    if (r == 0) {
        B->npend = 0;
        return EIG_OK;
    }
    if (l + r > B->max_vecs) throw Error{EIG_ERR_BUDGET, "basis full (max_vecs reached)"};
    // U[:, l + c] = P Rinv[:, c]
    std::vector<double> yr((size_t)np * r * 2);
    for (int a = 0; a < np; a++)
        for (int c = 0; c < r; c++) {
            yr[((size_t)a * r + c) * 2] = Rinv[(size_t)c * np + a].real();
            yr[((size_t)a * r + c) * 2 + 1] = Rinv[(size_t)c * np + a].imag();
        }
    B->Y.ensure(yr.size() * sizeof(double));
    CUDA_CK(cudaMemcpyAsync(B->Y.p, yr.data(), yr.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    ay_run(B, P, B->Y.as<double>(), basis_cols(B, l, r), 0.0, nrow, s);
    {
        // second pass: the remainders can be nearly dependent, so orthonormalise again
        ColSet Un = basis_cols(B, l, r);
        const cd *G2p = ahb_to_host(B, Un, Un, nrow, s);
        std::vector<cd> G2(G2p, G2p + (size_t)r * r);
        std::vector<cd> R2;
        std::vector<int> keep2;
        gram_orth(G2, r, 0.0, R2, keep2);
        if ((int)keep2.size() != r) throw Error{EIG_ERR_BREAKDOWN, "basis re-orthonormalisation lost rank"};
        std::vector<double> y2((size_t)r * r * 2);
        for (int a = 0; a < r; a++)
            for (int c = 0; c < r; c++) {
                y2[((size_t)a * r + c) * 2] = R2[(size_t)c * r + a].real();
                y2[((size_t)a * r + c) * 2 + 1] = R2[(size_t)c * r + a].imag();
            }
        CUDA_CK(cudaMemcpyAsync(B->Y.p, y2.data(), y2.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        ay_run(B, Un, B->Y.as<double>(), field_cols(B->pend.p, f64, 1, B->fsize(), r, false), 0.0, nrow, s);
        CUDA_CK(cudaMemcpyAsync((char *)B->U.p + (size_t)l * op->wfield_bytes(), B->pend.p,
                                (size_t)r * op->wfield_bytes(), cudaMemcpyDeviceToDevice, s));
        sync(s);
    }
    if (op->prec != P64 && !op->eo) {
        // W = A V-bar in double-float arithmetic (about 44 bits, far below the FP32
        // rounding of the stored W), up to max_rhs columns per stencil launch
        const long cstride = (long)(op->wfield_bytes() / 16);
        for (int c0 = 0; c0 < r; c0 += op->max_rhs) {
            const int n = std::min(op->max_rhs, r - c0);
            Field xin = op->r64.view(n), mid = op->u64.view(n), wout = op->x64.view(n);
            CUDA_CK(launch_cols32_to_dd((char *)B->U.p + (size_t)(l + c0) * op->wfield_bytes(), cstride, op->Vf, n,
                                        xin.v.data, s));
            CUDA_CK(launch_dslash_dd(op->call(xin, mid, false, true), op->gauge_dd.p, xin.v.data, mid.v.data, s));
            CUDA_CK(launch_dslash_dd(op->call(mid, wout, true, true), op->gauge_dd.p, mid.v.data, wout.v.data, s));
            CUDA_CK(launch_dd_to_cols32(wout.v.data, op->Vf, n, (char *)B->W.p + (size_t)c0 * op->wfield_bytes(),
                                        cstride, s));
        }
    } else {
        // W = A V-bar with the FP64 operator
        Field x64 = op->x64.view(1), r64f = op->b64.view(1);
        for (int c = 0; c < r; c++) {
            Field uc = field_at(op->wprec, (char *)B->U.p + (size_t)(l + c) * op->wfield_bytes(), op->Vf, 1);
            Field wc = field_at(op->wprec, (char *)B->W.p + (size_t)c * op->wfield_bytes(), op->Vf, 1);
            CUDA_CK(launch_combine(x64, 1.0, uc, 0.0, null_field(), s));
            apply_A64(op, x64, r64f, s);
            CUDA_CK(launch_combine(wc, 1.0, r64f, 0.0, null_field(), s));
        }
    }
    ColSet Wc = field_cols(B->W.p, f64, 1, B->fsize(), r, false);
    const int ln = l + r;
    const cd *UW = ahb_to_host(B, basis_cols(B, 0, ln), Wc, nrow, s);  // (l + r) x r: rows 0..l-1 = U^H W, rows l.. = V-bar^H W
    std::vector<cd> Hn((size_t)ln * ln);
    for (int a = 0; a < l; a++)
        for (int bb = 0; bb < l; bb++) Hn[(size_t)a * ln + bb] = B->H[(size_t)a * l + bb];
    for (int a = 0; a < l; a++)
        for (int c = 0; c < r; c++) {
            Hn[(size_t)a * ln + l + c] = UW[(size_t)a * r + c];
            Hn[(size_t)(l + c) * ln + a] = std::conj(UW[(size_t)a * r + c]);
        }
    for (int a = 0; a < r; a++)
        for (int c = 0; c < r; c++) {
            const cd v = 0.5 * (UW[(size_t)(l + a) * r + c] + std::conj(UW[(size_t)(l + c) * r + a]));
            Hn[(size_t)(l + a) * ln + l + c] = v;
        }
    B->H = Hn;
    B->l = ln;
    B->gen++;
    B->npend = 0;
    refactor(B);
    if (!B->chol_ok) throw Error{EIG_ERR_BREAKDOWN, "H = U^H A U lost positive definiteness"};
    API_END
}

eig_status eig_basis_deflate(eig_basis B, const double *b, const double *x_in, double *x0, int k, void *stream) {
    API_BEGIN
    ARG_CHECK(B && b && x0, "null argument");
    eig_op_s *op = B->op;
    ARG_CHECK(k >= 1 && k <= op->max_rhs && (k & (k - 1)) == 0, "k must be a power of two <= max_rhs");
    std::lock_guard<std::mutex> lk(B->mu);
    std::lock_guard<std::mutex> lk2(op->mu);
    ensure_workspace(op);
    cudaStream_t s = (cudaStream_t)stream;
    Field b64 = op->b64.view(k), x64 = op->x64.view(k), r64 = (op->prec == P64 ? op->r : op->r64).view(k);
    load_natural(op, b, b64, s);
    if (x_in) {
        load_natural(op, x_in, x64, s);
        apply_A64(op, x64, r64, s);
        CUDA_CK(launch_combine(r64, 1.0, b64, -1.0, r64, s));
    } else {
        zero_field(x64, s);
        CUDA_CK(launch_combine(r64, 1.0, b64, 0.0, null_field(), s));
    }
    deflate_into(B, r64, x64, s);
    store_natural(op, x64, x0, s);
    sync(s);
    API_END
}

eig_status eig_initcg_solve(eig_op op, eig_basis basis, const double *b, double *x, double tol, double restart_tol,
                            int max_iter, int k, eig_stats *stats, void *stream) {
    API_BEGIN
    ARG_CHECK(op && b && x, "null argument");
    ARG_CHECK(k >= 1 && k <= op->max_rhs && (k & (k - 1)) == 0, "k must be a power of two <= max_rhs");
    ARG_CHECK(tol > 0.0 && tol < 1.0, "tol must be in (0, 1)");
    ARG_CHECK(max_iter >= 1 && max_iter <= 10000000, "max_iter out of range");
    ARG_CHECK(!basis || basis->op == op, "basis belongs to another op");
    std::lock_guard<std::mutex> lk(op->mu);
    ensure_workspace(op);
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    Solve sv = make_solve(op, k, s, max_iter);
    load_solve(op, b, x, sv.b64, sv.x64, s);
    const bool defl = basis && basis->l > 0;
    if (defl) {
        sv.initial_residual();
        deflate_into(basis, sv.r64, sv.x64, s);
    }
    int restarts = 0;
    bool ok = true;
    int rounds = 0;
    // per-RHS iteration counts (CGScalars::nit) count only the iterations a RHS took part
    // in: a batch runs on after one RHS has stopped (at restart_tol, at tol, or before a
    // re-activation by the final residual check)
    std::vector<int> it1(k, 0);
    if (defl && restart_tol > tol) {
        // phase 1: CG to restart_tol, then re-deflate from the current x (Sec. 5.3)
        sv.start(restart_tol);
        ok = cg_run(sv, max_iter, nullptr, op);
        const int j1 = sv.j;
        for (int q = 0; q < k; q++) it1[q] = sv.sth[q].nit;
        std::vector<int> rel1 = sv.reliable;
        if (ok) {
            sv.true_residual(false, false);  // x64 += x_lo; r64 = b - A x64
            deflate_into(basis, sv.r64, sv.x64, s);
            restarts = 1;
            sv.start(tol);
            sv.j = j1;
            sv.j_checked = j1;
            sv.j_start = j1;
            for (int q = 0; q < k; q++) sv.reliable[q] += rel1[q];
            for (int q = 0; q < k; q++) {
                sv.sth[q].iters = j1;
                sv.sth[q].nit = it1[q];  // each RHS's count goes on from its phase-1 iterations
            }
            sv.write_scalars();
        }
    } else {
        sv.start(tol);
    }
    while (ok) {
        ok = cg_run(sv, max_iter, nullptr, op);
        if (!ok) break;
        if (!cg_finish(sv, max_iter, nullptr, op, rounds)) break;
    }
    if (!ok) sv.true_residual(false), sv.read_scalars();
    store_solve(op, sv.x64, x, s);
    sync(s);
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats) {
        for (int q = 0; q < k; q++) {
            eig_stats &st = stats[q];
            st.iters = sv.sth[q].nit;
            st.restarts = restarts;
            st.reliable_updates = sv.reliable[q];
            const double bn2 = sv.sth[q].target / (tol * tol);
            st.true_rel_res = bn2 > 0 ? std::sqrt(sv.sth[q].aux / bn2) : 0.0;
            st.converged = st.true_rel_res <= tol * (1 + 1e-12) ? 1 : 0;
            st.n_ritz = 0;
            st.ms = ms;
        }
    }
    if (!ok) {
        eig::g_last_error = "max_iter reached";
        return EIG_NOT_CONVERGED;
    }
    API_END
}

eig_status eig_bicgstab_solve(eig_op op, eig_basis basis, const double *b, double *x, double tol, int max_iter,
                              int defl_vecs, eig_stats *stats, void *stream) {
    API_BEGIN
    ARG_CHECK(op && b && x, "null argument");
    ARG_CHECK(!op->eo, "BiCGSTAB runs on the full-lattice M (even_odd = 0)");
    ARG_CHECK(op->prec != P16, "BiCGSTAB needs an FP64 or FP32 op");
    ARG_CHECK(tol > 0.0 && tol < 1.0, "tol must be in (0, 1)");
    ARG_CHECK(max_iter >= 1 && max_iter <= 10000000, "max_iter out of range");
    ARG_CHECK(defl_vecs >= 0, "defl_vecs must be >= 0");
    ARG_CHECK(!basis || basis->op == op, "basis belongs to another op");
    std::lock_guard<std::mutex> lk(op->mu);
    ensure_workspace(op);
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    if (op->prec != P64) tune_for(op, 1, s);
    const bool f64 = op->prec == P64;
    Field b64 = op->b64.view(1), x64 = op->x64.view(1), rt = op->u64.view(1);
    Field r = op->r.view(1), p = op->p.view(1), v = op->u.view(1);
    if (op->bc_rh.kcap < 1) {
        op->bc_rh.alloc(op->prec, op->Vf, 1);
        op->bc_s.alloc(op->prec, op->Vf, 1);
        op->bc_t.alloc(op->prec, op->Vf, 1);
    }
    Field rh = op->bc_rh.view(1), sf = op->bc_s.view(1), tf = op->bc_t.view(1);
    op->bsc.ensure(sizeof(BicgScalars));
    op->bsch.ensure(sizeof(BicgScalars));
    BicgScalars *sc = op->bsc.as<BicgScalars>(), *sch = op->bsch.as<BicgScalars>();
    CGScalars *cst = op->st.as<CGScalars>(), *csth = op->st_h.as<CGScalars>();
    const RedScratch red = op->red();
    load_natural(op, b, b64, s);
    load_natural(op, x, x64, s);
    // ||r||^2 of a FP64 field through the CG scalars' aux slot
    auto norm2_64 = [&](Field f) {
        CUDA_CK(launch_norm2(f, cst, false, History(), 0, red, s));
        CUDA_CK(cudaMemcpyAsync(csth, cst, sizeof(CGScalars), cudaMemcpyDeviceToHost, s));
        sync(s);
        return csth->aux;
    };
    auto true_residual = [&]() {  // rt = b - M x in FP64
        apply_M(op, x64, rt, false, true, s);
        CUDA_CK(launch_combine(rt, 1.0, b64, -1.0, rt, s));
        return norm2_64(rt);
    };
    const double bn2 = norm2_64(b64);
    if (basis && basis->l > 0 && defl_vecs > 0) {
        g5_setup(basis, std::min(defl_vecs, basis->l), s);
        true_residual();
        g5_deflate(basis, rt, x64, s);
    }
    // FP32 Krylov vectors track the true residual to a few decades: restart from the
    // FP64 residual when the recursive one has fallen by 1e5
    const double rel_inner = f64 ? 0.0 : 1e-5;
    int total = 0, restarts = 0;
    double rr_true = 0.0;
    bool ok = false;
    while (true) {
        rr_true = true_residual();
        if (rr_true <= tol * tol * bn2 || bn2 == 0.0) {
            ok = true;
            break;
        }
        if (total >= max_iter || restarts > 30) break;
        CUDA_CK(launch_combine(r, 1.0, rt, 0.0, null_field(), s));
        CUDA_CK(launch_combine(rh, 1.0, r, 0.0, null_field(), s));
        zero_field(p, s);
        zero_field(v, s);
        memset(sch, 0, sizeof(BicgScalars));
        sch->rho[0] = rr_true;
        sch->alpha[0] = 1.0;
        sch->omega[0] = 1.0;
        sch->rr = rr_true;
        sch->target = std::max(tol * tol * bn2, rel_inner * rel_inner * rr_true);
        sch->active = 1;
        CUDA_CK(cudaMemcpyAsync(sc, sch, sizeof(BicgScalars), cudaMemcpyHostToDevice, s));
        while (true) {
            for (int c = 0; c < CHECK; c++) {
                CUDA_CK(launch_bicg_p(r, p, v, sc, s));
                apply_M(op, p, v, false, f64, s);
                CUDA_CK(launch_bicg_alpha(rh, v, sc, red, s));
                CUDA_CK(launch_bicg_s(r, v, sf, sc, s));
                apply_M(op, sf, tf, false, f64, s);
                CUDA_CK(launch_bicg_omega(tf, sf, sc, red, s));
                CUDA_CK(launch_bicg_update(x64, p, sf, tf, r, rh, sc, red, s));
            }
            CUDA_CK(cudaMemcpyAsync(sch, sc, sizeof(BicgScalars), cudaMemcpyDeviceToHost, s));
            sync(s);
            if (!sch->active || total + sch->iters >= max_iter) break;
        }
        total += sch->iters;
        restarts++;
    }
    store_natural(op, x64, x, s);
    sync(s);
    if (stats) {
        stats->iters = total;
        stats->restarts = std::max(0, restarts - 1);
        stats->reliable_updates = restarts;
        stats->true_rel_res = bn2 > 0 ? std::sqrt(rr_true / bn2) : 0.0;
        stats->converged = ok ? 1 : 0;
        stats->n_ritz = 0;
        stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!ok) {
        eig::g_last_error = "BiCGSTAB did not reach tol within max_iter";
        return EIG_NOT_CONVERGED;
    }
    API_END
}

eig_status eig_basis_ritz(eig_basis B, double *evals, double *resnorms, int *n, void *stream) {
    API_BEGIN
    ARG_CHECK(B && evals && n, "null argument");
    std::lock_guard<std::mutex> lk(B->mu);
    std::lock_guard<std::mutex> lk2(B->op->mu);
    ensure_workspace(B->op);
    eig_op_s *op = B->op;
    cudaStream_t s = (cudaStream_t)stream;
    const int l = B->l;
    *n = l;
    if (l == 0) return EIG_OK;
    std::vector<double> th(l);
    std::vector<cd> S((size_t)l * l);
    dense::herm_eig_lowest(l, B->H.data(), l, th.data(), S.data());
    for (int a = 0; a < l; a++) evals[a] = th[a];
    if (!resnorms) return EIG_OK;
    const bool f64 = op->wprec == P64;
    Field x64 = op->x64.view(1), r64f = op->b64.view(1);
    Field w64 = op->prec == P64 ? op->r.view(1) : op->r64.view(1);
    for (int c0 = 0; c0 < l; c0 += MAX_NEV) {
        const int nc = std::min(MAX_NEV, l - c0);
        std::vector<double> yr((size_t)l * nc * 2);
        for (int a = 0; a < l; a++)
            for (int c = 0; c < nc; c++) {
                yr[((size_t)a * nc + c) * 2] = S[(size_t)(c0 + c) * l + a].real();
                yr[((size_t)a * nc + c) * 2 + 1] = S[(size_t)(c0 + c) * l + a].imag();
            }
        B->Y.ensure(yr.size() * sizeof(double));
        CUDA_CK(cudaMemcpyAsync(B->Y.p, yr.data(), yr.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        ColSet Wc = field_cols(B->W.p, f64, 1, B->fsize(), nc, false);
        ay_run(B, basis_cols(B, 0, l), B->Y.as<double>(), Wc, 0.0, op->ncomplex(), s);
        for (int c = 0; c < nc; c++) {
            Field wc = field_at(op->wprec, (char *)B->W.p + (size_t)c * op->wfield_bytes(), op->Vf, 1);
            CUDA_CK(launch_combine(x64, 1.0, wc, 0.0, null_field(), s));
            apply_A64(op, x64, r64f, s);
            CUDA_CK(launch_combine(w64, 1.0, r64f, -th[c0 + c], x64, s));
            CUDA_CK(launch_norm2(w64, op->st.as<CGScalars>(), false, op->history(1), 0, op->red(), s));
            CGScalars h;
            CUDA_CK(cudaMemcpyAsync(&h, op->st.p, sizeof(h), cudaMemcpyDeviceToHost, s));
            sync(s);
            resnorms[c0 + c] = std::sqrt(h.aux);
        }
    }
    API_END
}

eig_status eig_basis_vector(eig_basis B, int j, double *out, void *stream) {
    API_BEGIN
    ARG_CHECK(B && out, "null argument");
    ARG_CHECK(j >= 0 && j < B->l, "j out of range");
    std::lock_guard<std::mutex> lk(B->op->mu);
    ensure_workspace(B->op);
    eig_op_s *op = B->op;
    cudaStream_t s = (cudaStream_t)stream;
    Field uc = field_at(op->wprec, (char *)B->U.p + (size_t)j * op->wfield_bytes(), op->Vf, 1);
    Field x64 = op->x64.view(1);
    CUDA_CK(launch_combine(x64, 1.0, uc, 0.0, null_field(), s));
    store_natural(op, x64, out, s);
    sync(s);
    API_END
}

eig_status eig_basis_pending(eig_basis B, double *evals, int *n) {
    API_BEGIN
    ARG_CHECK(B && n, "null argument");
    *n = B->npend;
    if (evals)
        for (int a = 0; a < B->npend; a++) evals[a] = B->pend_ritz[a];
    API_END
}

eig_status eig_basis_h(eig_basis B, double *out) {
    API_BEGIN
    ARG_CHECK(B && out, "null argument");
    memcpy(out, B->H.data(), B->H.size() * sizeof(cd));
    API_END
}

eig_status eig_basis_save(eig_basis B, const char *path, void *stream) {
    API_BEGIN
    ARG_CHECK(B && path, "null argument");
    std::lock_guard<std::mutex> lk(B->op->mu);
    ensure_workspace(B->op);
    eig_op_s *op = B->op;
    cudaStream_t s = (cudaStream_t)stream;
    BasisFileHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, BASIS_MAGIC, 8);
    h.version = 1;
    for (int i = 0; i < 4; i++) h.dims[i] = op->L[i];
    h.even_odd = op->eo ? 1 : 0;
    h.real_bytes = op->wprec == P64 ? 8 : 4;
    h.l = B->l;
    h.fsize = B->fsize();
    h.m_q = op->m_q;
    h.gauge_hash = op->gauge_hash;
    File out;
    out.f = fopen(path, "wb");
    io_check(out.f != nullptr, std::string("cannot open ") + path + " for writing");
    io_check(fwrite(&h, sizeof h, 1, out.f) == 1, "write failed");
    const size_t nh = (size_t)B->l * B->l;
    io_check(fwrite(B->H.data(), sizeof(cd), nh, out.f) == nh, "write failed");
    const size_t n = (size_t)h.fsize * 2;
    std::vector<double> v(n);
    std::vector<float> v32(h.real_bytes == 4 ? n : 0);
    Field x64 = op->x64.view(1);
    for (int j = 0; j < B->l; j++) {
        Field uc = field_at(op->wprec, (char *)B->U.p + (size_t)j * op->wfield_bytes(), op->Vf, 1);
        CUDA_CK(launch_combine(x64, 1.0, uc, 0.0, null_field(), s));
        store_natural(op, x64, v.data(), s);
        sync(s);
        if (h.real_bytes == 4) {
            for (size_t i = 0; i < n; i++) v32[i] = (float)v[i];  // exact: FP32 storage
            io_check(fwrite(v32.data(), 4, n, out.f) == n, "write failed");
        } else {
            io_check(fwrite(v.data(), 8, n, out.f) == n, "write failed");
        }
    }
    const int rc = fclose(out.f);
    out.f = nullptr;
    io_check(rc == 0, "closing the basis file failed");
    API_END
}

eig_status eig_basis_load(eig_basis B, const char *path, void *stream) {
    API_BEGIN
    ARG_CHECK(B && path, "null argument");
    std::lock_guard<std::mutex> lk(B->op->mu);
    ensure_workspace(B->op);
    eig_op_s *op = B->op;
    cudaStream_t s = (cudaStream_t)stream;
    File in;
    in.f = fopen(path, "rb");
    io_check(in.f != nullptr, std::string("cannot open ") + path);
    BasisFileHeader h;
    io_check(fread(&h, sizeof h, 1, in.f) == 1, "basis file too short");
    io_check(memcmp(h.magic, BASIS_MAGIC, 8) == 0 && h.version == 1, "not a basis file of version 1");
    for (int i = 0; i < 4; i++) ARG_CHECK(h.dims[i] == op->L[i], "basis file: lattice extents differ");
    ARG_CHECK(h.even_odd == (op->eo ? 1 : 0), "basis file: odd-even form differs");
    ARG_CHECK(h.m_q == op->m_q, "basis file: quark mass differs");
    ARG_CHECK(h.gauge_hash == op->gauge_hash, "basis file: gauge field differs");
    ARG_CHECK(h.fsize == B->fsize(), "basis file: vector length differs");
    io_check(h.real_bytes == 4 || h.real_bytes == 8, "basis file: bad precision field");
    io_check(h.l >= 0 && h.l <= 1 << 20, "basis file: bad basis size");
    if (h.l > B->max_vecs) throw Error{EIG_ERR_BUDGET, "basis file holds more vectors than max_vecs"};
    const size_t nh = (size_t)h.l * h.l;
    std::vector<cd> H(nh);
    io_check(fread(H.data(), sizeof(cd), nh, in.f) == nh, "basis file too short");
    for (const cd &z : H) io_check(std::isfinite(z.real()) && std::isfinite(z.imag()), "basis file: H not finite");
    const size_t n = (size_t)h.fsize * 2;
    std::vector<double> v(n);
    std::vector<float> v32(h.real_bytes == 4 ? n : 0);
    Field x64 = op->x64.view(1);
    // the old basis is gone from here on: an error below leaves it empty
    B->l = 0;
    B->gen++;
    B->H.clear();
    B->npend = 0;
    B->pend_ritz.clear();
    refactor(B);
    for (int j = 0; j < h.l; j++) {
        if (h.real_bytes == 4) {
            io_check(fread(v32.data(), 4, n, in.f) == n, "basis file too short");
            for (size_t i = 0; i < n; i++) v[i] = v32[i];
        } else {
            io_check(fread(v.data(), 8, n, in.f) == n, "basis file too short");
        }
        load_natural(op, v.data(), x64, s);
        Field uc = field_at(op->wprec, (char *)B->U.p + (size_t)j * op->wfield_bytes(), op->Vf, 1);
        CUDA_CK(launch_combine(uc, 1.0, x64, 0.0, null_field(), s));
        sync(s);  // v is reused for the next vector
    }
    B->l = h.l;
    B->H = std::move(H);
    refactor(B);
    if (!B->chol_ok) throw Error{EIG_ERR_BREAKDOWN, "loaded H = U^H A U is not positive definite"};
    API_END
}

}  // extern "C"
