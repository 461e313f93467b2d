/*
 * ORACLE -- test infrastructure only.  Plain FP64 CPU Wilson-Dirac operator.
 * Nothing in the product path may call this; only tests, the smoke check and
 * the CPU-baseline leg of the benchmark do.
 *
 * The paper (Sec. 1) fixes only M = m_q I - D and gamma5-Hermiticity,
 * gamma5 M = M^H gamma5, with gamma5 diagonal +-1.  The operator written out
 * here is the standard Wilson matrix (r = 1, unit lattice spacing, periodic in
 * all four directions):
 *
 *   (M psi)(x) = (4 + m_q) psi(x)
 *       - 1/2 sum_mu [ (I - g_mu) U_mu(x) psi(x+mu) + (I + g_mu) U_mu(x-mu)^H psi(x-mu) ]
 *
 * with a chiral gamma basis in which gamma5 = g1 g2 g3 g4 = diag(1, 1, -1, -1).
 * M^H is applied as gamma5 M gamma5 (the gamma5-Hermiticity of Sec. 1), and the
 * normal operator of the CG of Sec. 1 is A = M^H M.
 *
 * Every spin multiplication is an explicit 4x4 complex matrix product with the
 * gamma table below: no spin projection, no link compression, no blocking.
 *
 * Layouts: gauge [V][4][3][3] complex, spinor [V][4][3] complex, site index
 * ((t*Lz + z)*Ly + y)*Lx + x; direction mu = 0..3 <-> x, y, z, t.
 */
#include <complex.h>
#include <stddef.h>
#include <string.h>

typedef double complex cplx;

/* Chiral (DeGrand-Rossi type) Hermitian gamma matrices g[mu][row][col]. */
static const cplx GAMMA[4][4][4] = {
    /* g1 */ {{0, 0, 0, I}, {0, 0, I, 0}, {0, -I, 0, 0}, {-I, 0, 0, 0}},
    /* g2 */ {{0, 0, 0, -1}, {0, 0, 1, 0}, {0, 1, 0, 0}, {-1, 0, 0, 0}},
    /* g3 */ {{0, 0, I, 0}, {0, 0, 0, -I}, {-I, 0, 0, 0}, {0, I, 0, 0}},
    /* g4 */ {{0, 0, 1, 0}, {0, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}},
};

/* gamma5 = g1 g2 g3 g4, formed by matrix products on first use. */
static cplx GAMMA5[4][4];
static int gamma5_ready = 0;

static void matmul4(const cplx a[4][4], const cplx b[4][4], cplx c[4][4]) {
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += a[i][k] * b[k][j];
            c[i][j] = s;
        }
}

static void make_gamma5(void) {
    if (gamma5_ready) return;
    cplx t1[4][4], t2[4][4];
    matmul4(GAMMA[0], GAMMA[1], t1);
    matmul4(t1, GAMMA[2], t2);
    matmul4(t2, GAMMA[3], GAMMA5);
    gamma5_ready = 1;
}

/* Copies the gamma table out (g1..g4 then g5) as 5*16 complex numbers. */
void oracle_get_gammas(cplx *out) {
    make_gamma5();
    memcpy(out, GAMMA, sizeof(GAMMA));
    memcpy(out + 64, GAMMA5, sizeof(GAMMA5));
}

static long site_index(const int d[4], const int c[4]) {
    return ((long)(c[3] * d[2] + c[2]) * d[1] + c[1]) * d[0] + c[0];
}

/* Neighbour of site s one step in direction mu, sign +1 or -1, periodic. */
static long neighbour(const int d[4], long s, int mu, int sign) {
    int c[4];
    long r = s;
    for (int k = 0; k < 4; k++) {
        c[k] = (int)(r % d[k]);
        r /= d[k];
    }
    c[mu] = (c[mu] + sign + d[mu]) % d[mu];
    return site_index(d, c);
}

/* out = M in. */
void oracle_wilson_m(const int dims[4], double m_q, const cplx *gauge, const cplx *in, cplx *out) {
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
#pragma omp parallel for schedule(static) if (V >= 4096)
    for (long s = 0; s < V; s++) {
        cplx acc[4][3];
        for (int a = 0; a < 4; a++)
            for (int c = 0; c < 3; c++) acc[a][c] = (4.0 + m_q) * in[(s * 4 + a) * 3 + c];
        for (int mu = 0; mu < 4; mu++) {
            /* forward hop: (I - g_mu) U_mu(x) psi(x + mu) */
            long f = neighbour(dims, s, mu, +1);
            const cplx *U = gauge + (s * 4 + mu) * 9;
            cplx up[4][3];
            for (int a = 0; a < 4; a++)
                for (int c = 0; c < 3; c++) {
                    cplx v = 0;
                    for (int e = 0; e < 3; e++) v += U[c * 3 + e] * in[(f * 4 + a) * 3 + e];
                    up[a][c] = v;
                }
            for (int a = 0; a < 4; a++)
                for (int c = 0; c < 3; c++) {
                    cplx v = 0;
                    for (int b = 0; b < 4; b++) v += ((a == b ? 1.0 : 0.0) - GAMMA[mu][a][b]) * up[b][c];
                    acc[a][c] -= 0.5 * v;
                }
            /* backward hop: (I + g_mu) U_mu(x - mu)^H psi(x - mu) */
            long bk = neighbour(dims, s, mu, -1);
            const cplx *W = gauge + (bk * 4 + mu) * 9;
            cplx dn[4][3];
            for (int a = 0; a < 4; a++)
                for (int c = 0; c < 3; c++) {
                    cplx v = 0;
                    for (int e = 0; e < 3; e++) v += conj(W[e * 3 + c]) * in[(bk * 4 + a) * 3 + e];
                    dn[a][c] = v;
                }
            for (int a = 0; a < 4; a++)
                for (int c = 0; c < 3; c++) {
                    cplx v = 0;
                    for (int b = 0; b < 4; b++) v += ((a == b ? 1.0 : 0.0) + GAMMA[mu][a][b]) * dn[b][c];
                    acc[a][c] -= 0.5 * v;
                }
        }
        for (int a = 0; a < 4; a++)
            for (int c = 0; c < 3; c++) out[(s * 4 + a) * 3 + c] = acc[a][c];
    }
}

/* out = gamma5 in, site by site, with the explicit gamma5 matrix. */
static void apply_gamma5(long V, const cplx *in, cplx *out) {
    make_gamma5();
#pragma omp parallel for schedule(static) if (V >= 4096)
    for (long s = 0; s < V; s++) {
        cplx tmp[4][3];
        for (int a = 0; a < 4; a++)
            for (int c = 0; c < 3; c++) {
                cplx v = 0;
                for (int b = 0; b < 4; b++) v += GAMMA5[a][b] * in[(s * 4 + b) * 3 + c];
                tmp[a][c] = v;
            }
        for (int a = 0; a < 4; a++)
            for (int c = 0; c < 3; c++) out[(s * 4 + a) * 3 + c] = tmp[a][c];
    }
}

/* out = M^H in = gamma5 M gamma5 in.  work: V*12 complex scratch. */
void oracle_wilson_mdag(const int dims[4], double m_q, const cplx *gauge, const cplx *in, cplx *out,
                        cplx *work) {
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    apply_gamma5(V, in, work);
    oracle_wilson_m(dims, m_q, gauge, work, out);
    apply_gamma5(V, out, out);
}

/* out = A in = M^H M in.  work: V*12 complex scratch (distinct from in/out). */
void oracle_wilson_a(const int dims[4], double m_q, const cplx *gauge, const cplx *in, cplx *out,
                     cplx *work) {
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    oracle_wilson_m(dims, m_q, gauge, in, work);
    apply_gamma5(V, work, work);
    oracle_wilson_m(dims, m_q, gauge, work, out);
    apply_gamma5(V, out, out);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
