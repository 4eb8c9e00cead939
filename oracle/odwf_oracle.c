/*
 * FP64 CPU oracle for the optimal domain-wall fermion (ODWF) operator and its
 * even-odd preconditioned normal-equation solves.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  It shares no code, header or
 * table with the CUDA library, and the library never calls it.
 *
 * Everything is a plain restatement of the definitions, with naive loops:
 *
 *   4D Wilson operator at mass -m0 (the kernel H_w = gamma_5 D_w of the paper's
 *   ODWF with c = 1, d = 0, Sec. 2):
 *     (D_w psi)(x) = (4 - m0) psi(x)
 *        - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                      + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
 *   5D ODWF operator D(m_q) (Sec. 2, the operator of Eq. (1)-(2)):
 *     (D psi)_s = (rho_s D_w + 1) psi_s + (sigma_s D_w - 1) (L psi)_s
 *     L = P_+ L_+ + P_- L_-,  (L_+)_{s,s-1} = 1, (L_+)_{1,Ns} = -r,
 *                             (L_-)_{s,s+1} = 1, (L_-)_{Ns,1} = -r,
 *     r = m_q / (2 m0),  P_+- = (1 +- gamma_5)/2,  gamma_5 = g1 g2 g3 g4.
 *   Adjoint: D^dag = (D_w^dag rho + 1) + L^dag (D_w^dag sigma - 1).
 *   M = the site-local part of D (D_w -> 4 - m0);  H = D - M couples the parities.
 *   Even-odd Schur operator on even sites:
 *     S = 1 - M^{-1} H_eo M^{-1} H_oe,   S^dag = 1 - H_oe^dag M^-dag H_eo^dag M^-dag.
 *
 * Conventions: chiral basis gamma_k = [[0, -i s_k], [i s_k, 0]] (k = 1, 2, 3),
 * gamma_4 = [[0, 1], [1, 0]]; gamma_5 is computed as the product, not assumed.
 * Spinor layout psi[s][t][z][y][x][spin][colour] (complex128), gauge
 * U[mu][t][z][y][x][a][b]; mu = 0..3 <-> x, y, z, t.  Even-site fields are
 * [s][lex/2][spin][colour] over the sites with (x+y+z+t) even (all dims even).
 * Time boundary: when tbc != 0 a hop across t = Lt-1 <-> 0 carries a factor -1.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static cplx GM[5][4][4]; /* gamma_1..gamma_4 (index 0..3) and gamma_5 (index 4) */
static int g_init = 0;

static void init_gamma(void)
{
    if (g_init) return;
    const cplx Ii = _Complex_I;
    cplx sig[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -Ii}, {Ii, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(GM, 0, sizeof(GM));
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                GM[k][a][2 + b] = -Ii * sig[k][a][b];
                GM[k][2 + a][b] = Ii * sig[k][a][b];
            }
    for (int a = 0; a < 2; ++a) {
        GM[3][a][2 + a] = 1;
        GM[3][2 + a][a] = 1;
    }
    /* gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 */
    cplx t1[4][4], t2[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += GM[0][i][k] * GM[1][k][j];
            t1[i][j] = s;
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += t1[i][k] * GM[2][k][j];
            t2[i][j] = s;
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += t2[i][k] * GM[3][k][j];
            GM[4][i][j] = s;
        }
    g_init = 1;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Copy of the gamma matrices, for the tests (5 x 4 x 4 complex). */
void oracle_gammas(cplx *out)
{
    init_gamma();
    memcpy(out, GM, sizeof(GM));
}

static inline long lex(const int *L, int x, int y, int z, int t)
{
    return x + (long)L[0] * (y + (long)L[1] * (z + (long)L[2] * t));
}

/* v_out = U v (colour), or U^dag v, for each of the 4 spins */
static inline void su3_mul(const cplx *U, const cplx *v, cplx *o, int dag)
{
    for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a) {
            cplx s = 0;
            for (int b = 0; b < 3; ++b)
                s += (dag ? conj(U[3 * b + a]) : U[3 * a + b]) * v[3 * sp + b];
            o[3 * sp + a] = s;
        }
}

/* o = (1 + sgn gamma_mu) v */
static inline void spin_proj(int mu, double sgn, const cplx *v, cplx *o)
{
    for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 3; ++c) {
            cplx s = v[3 * a + c];
            for (int b = 0; b < 4; ++b) s += sgn * GM[mu][a][b] * v[3 * b + c];
            o[3 * a + c] = s;
        }
}

/*
 * 4D Wilson operator D_w (dagger = 0) or its adjoint (dagger = 1) on one 4D field.
 * The adjoint swaps the projectors: (D_w^dag psi)(x) = (4-m0) psi(x)
 *   - 1/2 sum_mu [(1 + gamma_mu) U_mu(x) psi(x+mu) + (1 - gamma_mu) U_mu(x-mu)^dag psi(x-mu)].
 */
void oracle_dw(const cplx *U, const int *L, int tbc, double m0, const cplx *in, cplx *out, int dagger)
{
    init_gamma();
    const long V = (long)L[0] * L[1] * L[2] * L[3];
    const double sf = dagger ? +1.0 : -1.0; /* forward projector 1 + sf gamma */
#pragma omp parallel for schedule(static)
    for (int t = 0; t < L[3]; ++t)
        for (int z = 0; z < L[2]; ++z)
            for (int y = 0; y < L[1]; ++y)
                for (int x = 0; x < L[0]; ++x) {
                    const int c[4] = {x, y, z, t};
                    const long i = lex(L, x, y, z, t);
                    cplx acc[12], v[12], w[12];
                    for (int k = 0; k < 12; ++k) acc[k] = (4.0 - m0) * in[12 * i + k];
                    for (int mu = 0; mu < 4; ++mu) {
                        int cf[4] = {c[0], c[1], c[2], c[3]}, cb[4] = {c[0], c[1], c[2], c[3]};
                        cf[mu] = (c[mu] + 1) % L[mu];
                        cb[mu] = (c[mu] - 1 + L[mu]) % L[mu];
                        double phf = 1.0, phb = 1.0;
                        if (tbc && mu == 3) {
                            if (c[3] == L[3] - 1) phf = -1.0;
                            if (c[3] == 0) phb = -1.0;
                        }
                        const long jf = lex(L, cf[0], cf[1], cf[2], cf[3]);
                        const long jb = lex(L, cb[0], cb[1], cb[2], cb[3]);
                        /* forward: (1 + sf gamma_mu) U_mu(x) psi(x+mu) */
                        su3_mul(U + 9 * ((long)mu * V + i), in + 12 * jf, v, 0);
                        spin_proj(mu, sf, v, w);
                        for (int k = 0; k < 12; ++k) acc[k] -= 0.5 * phf * w[k];
                        /* backward: (1 - sf gamma_mu) U_mu(x-mu)^dag psi(x-mu) */
                        su3_mul(U + 9 * ((long)mu * V + jb), in + 12 * jb, v, 1);
                        spin_proj(mu, -sf, v, w);
                        for (int k = 0; k < 12; ++k) acc[k] -= 0.5 * phb * w[k];
                    }
                    for (int k = 0; k < 12; ++k) out[12 * i + k] = acc[k];
                }
}

/* The fifth-dimension matrix L as Ns x Ns blocks of 4x4 spin matrices, built from
 * its definition: L = P_+ L_+ + P_- L_- with the -r corner entries. */
static void build_L(int Ns, double r, cplx *Lm /* [Ns][Ns][4][4] */)
{
    init_gamma();
    cplx Pp[4][4], Pm[4][4];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            const cplx id = (a == b) ? 1.0 : 0.0;
            Pp[a][b] = 0.5 * (id + GM[4][a][b]);
            Pm[a][b] = 0.5 * (id - GM[4][a][b]);
        }
    memset(Lm, 0, sizeof(cplx) * 16 * Ns * Ns);
    for (int s = 0; s < Ns; ++s) {
        /* P_+ psi_{s-1}; at s = 1 (index 0) it is -r P_+ psi_{Ns} */
        const int sm = (s == 0) ? Ns - 1 : s - 1;
        const double cm = (s == 0) ? -r : 1.0;
        /* P_- psi_{s+1}; at s = Ns it is -r P_- psi_1 */
        const int sp = (s == Ns - 1) ? 0 : s + 1;
        const double cp = (s == Ns - 1) ? -r : 1.0;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                Lm[((s * Ns + sm) * 4 + a) * 4 + b] += cm * Pp[a][b];
                Lm[((s * Ns + sp) * 4 + a) * 4 + b] += cp * Pm[a][b];
            }
    }
}

/* out_s = sum_s' L_{s,s'} in_s' (transpose = 0) or sum_s' (L_{s',s})^dag in_s' (transpose = 1);
 * fields of V sites per s-slice. */
static void apply_L(const cplx *Lm, int Ns, long V, const cplx *in, cplx *out, int transpose)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; ++i)
        for (int s = 0; s < Ns; ++s) {
            cplx acc[12] = {0};
            for (int s2 = 0; s2 < Ns; ++s2) {
                const cplx *B = transpose ? Lm + (long)(s2 * Ns + s) * 16 : Lm + (long)(s * Ns + s2) * 16;
                int nz = 0;
                for (int k = 0; k < 16; ++k) nz |= (B[k] != 0);
                if (!nz) continue;
                const cplx *v = in + 12 * ((long)s2 * V + i);
                for (int a = 0; a < 4; ++a)
                    for (int b = 0; b < 4; ++b) {
                        const cplx m = transpose ? conj(B[b * 4 + a]) : B[a * 4 + b];
                        if (m == 0) continue;
                        for (int c = 0; c < 3; ++c) acc[3 * a + c] += m * v[3 * b + c];
                    }
            }
            for (int k = 0; k < 12; ++k) out[12 * ((long)s * V + i) + k] = acc[k];
        }
}

/*
 * The 5D operator D (dagger = 0) or D^dag (dagger = 1) on a full 5D field.
 *   D   psi:  (D psi)_s   = rho_s D_w psi_s + psi_s + sigma_s D_w (L psi)_s - (L psi)_s
 *   D^dag phi: (D^dag phi)_s = rho_s D_w^dag phi_s + phi_s + (L^dag u)_s,
 *              u_s = sigma_s D_w^dag phi_s - phi_s
 */
void oracle_d5(const cplx *U, const int *L, int tbc, int Ns, double m0, double mq,
               const double *rho, const double *sigma, const cplx *in, cplx *out, int dagger)
{
    const long V = (long)L[0] * L[1] * L[2] * L[3];
    const double r = mq / (2.0 * m0);
    cplx *Lm = malloc(sizeof(cplx) * 16 * Ns * Ns);
    cplx *t1 = malloc(sizeof(cplx) * 12 * V * Ns);
    cplx *t2 = malloc(sizeof(cplx) * 12 * V * Ns);
    build_L(Ns, r, Lm);
    if (!dagger) {
        apply_L(Lm, Ns, V, in, t1, 0); /* t1 = L psi */
        for (int s = 0; s < Ns; ++s) {
            const long o = 12 * (long)s * V;
            oracle_dw(U, L, tbc, m0, in + o, t2 + o, 0);      /* D_w psi_s */
            for (long k = 0; k < 12 * V; ++k) out[o + k] = rho[s] * t2[o + k] + in[o + k];
            oracle_dw(U, L, tbc, m0, t1 + o, t2 + o, 0);      /* D_w (L psi)_s */
            for (long k = 0; k < 12 * V; ++k) out[o + k] += sigma[s] * t2[o + k] - t1[o + k];
        }
    } else {
        for (int s = 0; s < Ns; ++s) {
            const long o = 12 * (long)s * V;
            oracle_dw(U, L, tbc, m0, in + o, t2 + o, 1);      /* D_w^dag phi_s */
            for (long k = 0; k < 12 * V; ++k) {
                out[o + k] = rho[s] * t2[o + k] + in[o + k];
                t1[o + k] = sigma[s] * t2[o + k] - in[o + k]; /* u_s */
            }
        }
        apply_L(Lm, Ns, V, t1, t2, 1); /* L^dag u */
        for (long k = 0; k < 12 * V * Ns; ++k) out[k] += t2[k];
    }
    free(Lm);
    free(t1);
    free(t2);
}

/* Dense site-local matrix M = (4-m0) B + 1 - L with B = rho + sigma L, as a
 * (4 Ns) x (4 Ns) complex matrix over (s, spin); colour acts as identity. */
static void build_M(int Ns, double m0, double mq, const double *rho, const double *sigma, cplx *M)
{
    const int n = 4 * Ns;
    const double a = 4.0 - m0;
    cplx *Lm = malloc(sizeof(cplx) * 16 * Ns * Ns);
    build_L(Ns, mq / (2.0 * m0), Lm);
    memset(M, 0, sizeof(cplx) * n * n);
    for (int s = 0; s < Ns; ++s)
        for (int al = 0; al < 4; ++al) {
            M[(4 * s + al) * n + 4 * s + al] += a * rho[s] + 1.0;
            for (int s2 = 0; s2 < Ns; ++s2)
                for (int be = 0; be < 4; ++be)
                    M[(4 * s + al) * n + 4 * s2 + be] += (a * sigma[s] - 1.0) * Lm[((s * Ns + s2) * 4 + al) * 4 + be];
        }
    free(Lm);
}

/* In-place Gauss-Jordan inverse with partial pivoting; returns 0 on success. */
static int invert(int n, cplx *A)
{
    cplx *B = malloc(sizeof(cplx) * n * n);
    int rc = 0;
    memset(B, 0, sizeof(cplx) * n * n);
    for (int i = 0; i < n; ++i) B[i * n + i] = 1;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int i = c + 1; i < n; ++i)
            if (cabs(A[i * n + c]) > cabs(A[p * n + c])) p = i;
        if (cabs(A[p * n + c]) == 0) { rc = -1; break; }
        if (p != c)
            for (int j = 0; j < n; ++j) {
                cplx t = A[c * n + j]; A[c * n + j] = A[p * n + j]; A[p * n + j] = t;
                t = B[c * n + j]; B[c * n + j] = B[p * n + j]; B[p * n + j] = t;
            }
        const cplx piv = A[c * n + c];
        for (int j = 0; j < n; ++j) { A[c * n + j] /= piv; B[c * n + j] /= piv; }
        for (int i = 0; i < n; ++i) {
            if (i == c) continue;
            const cplx f = A[i * n + c];
            if (f == 0) continue;
            for (int j = 0; j < n; ++j) { A[i * n + j] -= f * A[c * n + j]; B[i * n + j] -= f * B[c * n + j]; }
        }
    }
    memcpy(A, B, sizeof(cplx) * n * n);
    free(B);
    return rc;
}

/*
 * Site-local operator on a 5D field of V sites per s-slice (any subset of sites):
 *   op 0: M,  1: M^dag,  2: M^{-1},  3: M^{-dag}.
 */
int oracle_m5(int Ns, double m0, double mq, const double *rho, const double *sigma,
              long V, const cplx *in, cplx *out, int op)
{
    const int n = 4 * Ns;
    cplx *M = malloc(sizeof(cplx) * n * n);
    build_M(Ns, m0, mq, rho, sigma, M);
    int rc = 0;
    if (op >= 2) rc = invert(n, M);
    const int herm = (op == 1 || op == 3);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; ++i) {
        cplx w[4 * 16 * 3];
        cplx *acc = (n * 3 <= (int)(sizeof(w) / sizeof(w[0]))) ? w : malloc(sizeof(cplx) * n * 3);
        for (int s = 0; s < Ns; ++s)
            for (int al = 0; al < 4; ++al)
                for (int c = 0; c < 3; ++c) {
                    cplx sum = 0;
                    for (int s2 = 0; s2 < Ns; ++s2)
                        for (int be = 0; be < 4; ++be) {
                            const int row = 4 * s + al, col = 4 * s2 + be;
                            const cplx m = herm ? conj(M[col * n + row]) : M[row * n + col];
                            sum += m * in[12 * ((long)s2 * V + i) + 3 * be + c];
                        }
                    acc[(4 * s + al) * 3 + c] = sum;
                }
        for (int s = 0; s < Ns; ++s)
            for (int k = 0; k < 12; ++k) out[12 * ((long)s * V + i) + k] = acc[4 * s * 3 + k];
        if (acc != w) free(acc);
    }
    free(M);
    return rc;
}

/*
 * The chiral shift B = diag(rho) + diag(sigma) L of the operator D = D_w B + 1 - L
 * (Sec. 2's (rho_s D_w + 1) psi_s + (sigma_s D_w - 1)(L psi)_s, regrouped), on a 5D field of
 * V sites per s-slice:  dagger = 0:  (B psi)_s = rho_s psi_s + sigma_s (L psi)_s
 *                       dagger = 1:  B^dag phi = rho phi + L^dag (sigma phi)
 */
void oracle_b5(int Ns, double m0, double mq, const double *rho, const double *sigma,
               long V, const cplx *in, cplx *out, int dagger)
{
    cplx *Lm = malloc(sizeof(cplx) * 16 * Ns * Ns);
    cplx *t = malloc(sizeof(cplx) * 12 * V * Ns);
    build_L(Ns, mq / (2.0 * m0), Lm);
    if (!dagger) {
        apply_L(Lm, Ns, V, in, t, 0);
        for (int s = 0; s < Ns; ++s)
            for (long k = 0; k < 12 * V; ++k) {
                const long o = 12 * (long)s * V + k;
                out[o] = rho[s] * in[o] + sigma[s] * t[o];
            }
    } else {
        cplx *u = malloc(sizeof(cplx) * 12 * V * Ns);
        for (int s = 0; s < Ns; ++s)
            for (long k = 0; k < 12 * V; ++k) u[12 * (long)s * V + k] = sigma[s] * in[12 * (long)s * V + k];
        apply_L(Lm, Ns, V, u, t, 1);
        for (int s = 0; s < Ns; ++s)
            for (long k = 0; k < 12 * V; ++k) {
                const long o = 12 * (long)s * V + k;
                out[o] = rho[s] * in[o] + t[o];
            }
        free(u);
    }
    free(Lm);
    free(t);
}

static int parity_of(const int *L, long i)
{
    const int x = i % L[0], y = (i / L[0]) % L[1], z = (i / ((long)L[0] * L[1])) % L[2],
              t = i / ((long)L[0] * L[1] * L[2]);
    return (x + y + z + t) & 1;
}

/* full[s][i] = half[s][i/2] on sites of parity `par`, 0 elsewhere */
static void embed(const int *L, int Ns, int par, const cplx *half, cplx *full)
{
    const long V = (long)L[0] * L[1] * L[2] * L[3];
    for (int s = 0; s < Ns; ++s)
        for (long i = 0; i < V; ++i)
            for (int k = 0; k < 12; ++k)
                full[12 * ((long)s * V + i) + k] =
                    (parity_of(L, i) == par) ? half[12 * ((long)s * (V / 2) + i / 2) + k] : 0;
}

static void extract(const int *L, int Ns, int par, const cplx *full, cplx *half)
{
    const long V = (long)L[0] * L[1] * L[2] * L[3];
    for (int s = 0; s < Ns; ++s)
        for (long i = 0; i < V; ++i)
            if (parity_of(L, i) == par)
                for (int k = 0; k < 12; ++k)
                    half[12 * ((long)s * (V / 2) + i / 2) + k] = full[12 * ((long)s * V + i) + k];
}

/* out_par = (block of D or D^dag from parity 1-par to parity par) applied to in (a 1-par field):
 * the parity-`par` part of D applied to the embedded field. */
static void hop_block(const cplx *U, const int *L, int tbc, int Ns, double m0, double mq,
                      const double *rho, const double *sigma, int par, const cplx *in_half,
                      cplx *out_half, int dagger, cplx *f1, cplx *f2)
{
    embed(L, Ns, 1 - par, in_half, f1);
    oracle_d5(U, L, tbc, Ns, m0, mq, rho, sigma, f1, f2, dagger);
    extract(L, Ns, par, f2, out_half);
}

/*
 * Even-odd Schur operator on even-site fields:
 *   dagger = 0:  out = in - M^{-1} H_eo M^{-1} H_oe in
 *   dagger = 1:  out = in - H_oe^dag M^-dag H_eo^dag M^-dag in
 */
void oracle_schur(const cplx *U, const int *L, int tbc, int Ns, double m0, double mq,
                  const double *rho, const double *sigma, const cplx *in, cplx *out, int dagger)
{
    const long V = (long)L[0] * L[1] * L[2] * L[3], Vh = V / 2;
    const long nh = 12 * Vh * Ns, nf = 12 * V * Ns;
    cplx *f1 = malloc(sizeof(cplx) * nf), *f2 = malloc(sizeof(cplx) * nf);
    cplx *a = malloc(sizeof(cplx) * nh), *b = malloc(sizeof(cplx) * nh);
    if (!dagger) {
        hop_block(U, L, tbc, Ns, m0, mq, rho, sigma, 1, in, a, 0, f1, f2); /* H_oe in */
        oracle_m5(Ns, m0, mq, rho, sigma, Vh, a, b, 2);                   /* M^-1 */
        hop_block(U, L, tbc, Ns, m0, mq, rho, sigma, 0, b, a, 0, f1, f2);  /* H_eo */
        oracle_m5(Ns, m0, mq, rho, sigma, Vh, a, b, 2);                   /* M^-1 */
        for (long k = 0; k < nh; ++k) out[k] = in[k] - b[k];
    } else {
        oracle_m5(Ns, m0, mq, rho, sigma, Vh, in, a, 3);                  /* M^-dag in */
        hop_block(U, L, tbc, Ns, m0, mq, rho, sigma, 1, a, b, 1, f1, f2);  /* H_eo^dag */
        oracle_m5(Ns, m0, mq, rho, sigma, Vh, b, a, 3);                   /* M^-dag */
        hop_block(U, L, tbc, Ns, m0, mq, rho, sigma, 0, a, b, 1, f1, f2);  /* H_oe^dag */
        for (long k = 0; k < nh; ++k) out[k] = in[k] - b[k];
    }
    free(f1); free(f2); free(a); free(b);
}

static double dot_re(const cplx *a, const cplx *b, long n)
{
    double s = 0;
    for (long k = 0; k < n; ++k) s += creal(conj(a[k]) * b[k]);
    return s;
}

/* system 0: S^dag S on even sites;  system 1: D^dag D on the full lattice */
static void normal_op(int system, const cplx *U, const int *L, int tbc, int Ns, double m0, double mq,
                      const double *rho, const double *sigma, const cplx *in, cplx *out, cplx *tmp)
{
    if (system == 0) {
        oracle_schur(U, L, tbc, Ns, m0, mq, rho, sigma, in, tmp, 0);
        oracle_schur(U, L, tbc, Ns, m0, mq, rho, sigma, tmp, out, 1);
    } else {
        oracle_d5(U, L, tbc, Ns, m0, mq, rho, sigma, in, tmp, 0);
        oracle_d5(U, L, tbc, Ns, m0, mq, rho, sigma, tmp, out, 1);
    }
}

/*
 * Conjugate gradient on the Hermitian positive-definite normal system A x = b,
 * A = S^dag S (system 0, even-site fields) or D^dag D (system 1, full fields),
 * from x = 0 (or the given x when x_is_guess), until ||b - A x|| <= tol ||b||
 * (recomputed residual) or max_iter.  Returns the iteration count, or -1 on
 * non-convergence; *res_out gets the final true relative residual.
 */
int oracle_cg(int system, const cplx *U, const int *L, int tbc, int Ns, double m0, double mq,
              const double *rho, const double *sigma, const cplx *b, cplx *x, double tol,
              int max_iter, int x_is_guess, double *res_out, double *coef_out)
{
    /* coef_out (may be NULL): 2 * max_iter doubles; iteration k writes its alpha_k and
     * beta_k to coef_out[2k], coef_out[2k+1] (the Lanczos coefficients of the Krylov
     * space, from which the extreme eigenvalues of the normal operator follow). */
    const long V = (long)L[0] * L[1] * L[2] * L[3];
    const long n = 12 * Ns * (system == 0 ? V / 2 : V);
    cplx *r = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n);
    cplx *Ap = malloc(sizeof(cplx) * n), *tmp = malloc(sizeof(cplx) * n);
    if (!x_is_guess) memset(x, 0, sizeof(cplx) * n);
    normal_op(system, U, L, tbc, Ns, m0, mq, rho, sigma, x, Ap, tmp);
    for (long k = 0; k < n; ++k) { r[k] = b[k] - Ap[k]; p[k] = r[k]; }
    const double bb = dot_re(b, b, n);
    double rr = dot_re(r, r, n);
    int it = 0, conv = 0;
    while (it < max_iter) {
        if (rr <= tol * tol * bb) { conv = 1; break; }
        normal_op(system, U, L, tbc, Ns, m0, mq, rho, sigma, p, Ap, tmp);
        const double pap = dot_re(p, Ap, n);
        const double alpha = rr / pap;
        for (long k = 0; k < n; ++k) { x[k] += alpha * p[k]; r[k] -= alpha * Ap[k]; }
        const double rr_new = dot_re(r, r, n);
        const double beta = rr_new / rr;
        for (long k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
        if (coef_out) { coef_out[2 * it] = alpha; coef_out[2 * it + 1] = beta; }
        rr = rr_new;
        ++it;
    }
    normal_op(system, U, L, tbc, Ns, m0, mq, rho, sigma, x, Ap, tmp);
    double res = 0;
    for (long k = 0; k < n; ++k) { const cplx d = b[k] - Ap[k]; res += creal(d * conj(d)); }
    res = sqrt(res / bb);
    if (res_out) *res_out = res;
    free(r); free(p); free(Ap); free(tmp);
    if (!conv && res > tol) return -1;
    return it;
}
