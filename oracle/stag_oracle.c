/*
 * stag_oracle.c -- plain, slow, FP64 CPU oracle for the even-odd preconditioned
 * staggered operator and the conjugate-gradient solve built on it.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  The CUDA product
 * path shares no code, header, table or helper with it.
 *
 * What it follows.  Sec. 3 ("CG Performance") of the paper names the method:
 * a mixed-precision conjugate-gradient inverter for HYP-smeared staggered
 * quarks on a 20^3 x 64 lattice.  The paper never writes the operator down, so
 * the oracle states the standard one-link staggered operator with these
 * conventions (each pinned by a test against a closed form or an invariant):
 *
 *   sites x = (x0,x1,x2,x3) = (x,y,z,t), lexicographic index with x fastest;
 *   parity(x) = (x0+x1+x2+x3) mod 2, even = 0;
 *   checkerboard index of a site = lex / 2 (needs L0 even);
 *   staggered phase  eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1})   (eta_0 = 1);
 *   boundary sign    b_mu(x)   = -1 if mu = t, the antiperiodic flag is set and
 *                                x_t = L_t - 1, else +1;
 *   (D psi)(x) = sum_mu [ eta_mu(x) b_mu(x) U_mu(x) psi(x+mu)
 *                       - eta_mu(x-mu) b_mu(x-mu) U_mu(x-mu)^dagger psi(x-mu) ]
 *                with periodic index wrap; both hops are ACCUMULATED (on a
 *                length-2 direction x+mu and x-mu are the same site);
 *   D_oe = odd rows, even columns of D;  D_eo = even rows, odd columns;
 *   A = M^dagger M on even sites = 4 m^2 - D_eo D_oe   (Hermitian, >= 4m^2).
 *
 * Memory layouts (all FP64, complex = (re, im) pairs):
 *   links  [4][V][3][3]  (direction, lexicographic site, row, column)
 *   full-lattice vector [V][3]; checkerboard vector [V/2][3] (cb index order).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so that
 * x86-64 and aarch64 hosts produce identical results).  A second build with
 * -fopenmp (for timing on all host cores) runs the per-site loop of
 * orc_dslash_full in parallel; every site is computed exactly as in the serial
 * build and every reduction stays serial, so its results are bit-identical.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double re, im;
} cplx;

static cplx c_add(cplx a, cplx b) { cplx r = {a.re + b.re, a.im + b.im}; return r; }
static cplx c_sub(cplx a, cplx b) { cplx r = {a.re - b.re, a.im - b.im}; return r; }
static cplx c_mul(cplx a, cplx b)
{
    cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return r;
}
static cplx c_conj(cplx a) { cplx r = {a.re, -a.im}; return r; }
static cplx c_scale(double s, cplx a) { cplx r = {s * a.re, s * a.im}; return r; }

/* ------------------------------------------------------------------ */
/* lattice geometry                                                    */
/* ------------------------------------------------------------------ */

static long volume(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static long lex_of(const int L[4], const int x[4])
{
    return x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
}

static void coords_of(const int L[4], long i, int x[4])
{
    x[0] = (int)(i % L[0]); i /= L[0];
    x[1] = (int)(i % L[1]); i /= L[1];
    x[2] = (int)(i % L[2]); i /= L[2];
    x[3] = (int)i;
}

static int parity_of(const int x[4]) { return (x[0] + x[1] + x[2] + x[3]) & 1; }

/* staggered phase eta_mu(x) = (-1)^(sum_{nu<mu} x_nu) */
static int eta(int mu, const int x[4])
{
    int s = 0;
    for (int nu = 0; nu < mu; ++nu) s += x[nu];
    return (s & 1) ? -1 : 1;
}

/* boundary sign of the link U_mu(x): antiperiodic in t */
static int bsign(int mu, const int x[4], const int L[4], int antiperiodic)
{
    return (antiperiodic && mu == 3 && x[3] == L[3] - 1) ? -1 : 1;
}

static const cplx *link_at(const cplx *U, long V, int mu, long site)
{
    return U + ((long)mu * V + site) * 9;
}

/* ------------------------------------------------------------------ */
/* the staggered operator on the full lattice                          */
/* ------------------------------------------------------------------ */

/* threads of the -fopenmp build (1 in the serial build) */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* out = D in (full lattice).  Direct transcription of the definition above. */
void orc_dslash_full(const int L[4], int antiperiodic, const double *Ud,
                     const double *ind, double *outd)
{
    const cplx *U = (const cplx *)Ud;
    const cplx *in = (const cplx *)ind;
    cplx *out = (cplx *)outd;
    long V = volume(L);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long i = 0; i < V; ++i) {
        int x[4];
        coords_of(L, i, x);
        cplx acc[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (int mu = 0; mu < 4; ++mu) {
            int xf[4] = {x[0], x[1], x[2], x[3]};
            int xb[4] = {x[0], x[1], x[2], x[3]};
            xf[mu] = (x[mu] + 1) % L[mu];
            xb[mu] = (x[mu] - 1 + L[mu]) % L[mu];
            long jf = lex_of(L, xf), jb = lex_of(L, xb);

            /* forward hop: + eta_mu(x) b_mu(x) U_mu(x) in(x+mu) */
            double sf = (double)(eta(mu, x) * bsign(mu, x, L, antiperiodic));
            const cplx *Uf = link_at(U, V, mu, i);
            for (int a = 0; a < 3; ++a) {
                cplx h = {0, 0};
                for (int b = 0; b < 3; ++b) h = c_add(h, c_mul(Uf[a * 3 + b], in[jf * 3 + b]));
                acc[a] = c_add(acc[a], c_scale(sf, h));
            }
            /* backward hop: - eta_mu(x-mu) b_mu(x-mu) U_mu(x-mu)^dagger in(x-mu) */
            double sb = (double)(eta(mu, xb) * bsign(mu, xb, L, antiperiodic));
            const cplx *Ub = link_at(U, V, mu, jb);
            for (int a = 0; a < 3; ++a) {
                cplx h = {0, 0};
                for (int b = 0; b < 3; ++b) h = c_add(h, c_mul(c_conj(Ub[b * 3 + a]), in[jb * 3 + b]));
                acc[a] = c_sub(acc[a], c_scale(sb, h));
            }
        }
        for (int a = 0; a < 3; ++a) out[i * 3 + a] = acc[a];
    }
}

/* ------------------------------------------------------------------ */
/* checkerboard (even/odd) views                                       */
/* ------------------------------------------------------------------ */

/* full[V][3] -> cb[V/2][3] for the sites of the given parity (cb = lex/2) */
void orc_gather_parity(const int L[4], int par, const double *fulld, double *cbd)
{
    const cplx *full = (const cplx *)fulld;
    cplx *cb = (cplx *)cbd;
    long V = volume(L);
    for (long i = 0; i < V; ++i) {
        int x[4];
        coords_of(L, i, x);
        if (parity_of(x) != par) continue;
        for (int a = 0; a < 3; ++a) cb[(i / 2) * 3 + a] = full[i * 3 + a];
    }
}

/* cb[V/2][3] -> full[V][3], zero on the other parity */
void orc_scatter_parity(const int L[4], int par, const double *cbd, double *fulld)
{
    const cplx *cb = (const cplx *)cbd;
    cplx *full = (cplx *)fulld;
    long V = volume(L);
    for (long i = 0; i < V; ++i) {
        int x[4];
        coords_of(L, i, x);
        for (int a = 0; a < 3; ++a) {
            cplx z = {0, 0};
            full[i * 3 + a] = (parity_of(x) == par) ? cb[(i / 2) * 3 + a] : z;
        }
    }
}

/* out_par = (D restricted to rows of parity `out_par`, columns of the other parity) in */
static void dslash_block(const int L[4], int antiperiodic, const double *U, int out_par,
                         const double *in_cb, double *out_cb)
{
    long V = volume(L);
    double *full_in = (double *)malloc(sizeof(double) * 6 * V);
    double *full_out = (double *)malloc(sizeof(double) * 6 * V);
    orc_scatter_parity(L, 1 - out_par, in_cb, full_in);
    orc_dslash_full(L, antiperiodic, U, full_in, full_out);
    orc_gather_parity(L, out_par, full_out, out_cb);
    free(full_in);
    free(full_out);
}

/* out_odd = D_oe in_even */
void orc_dslash_oe(const int L[4], int antiperiodic, const double *U, const double *in_even,
                   double *out_odd)
{
    dslash_block(L, antiperiodic, U, 1, in_even, out_odd);
}

/* out_even = D_eo in_odd */
void orc_dslash_eo(const int L[4], int antiperiodic, const double *U, const double *in_odd,
                   double *out_even)
{
    dslash_block(L, antiperiodic, U, 0, in_odd, out_even);
}

/* out_even = (4 m^2 - D_eo D_oe) in_even */
void orc_mdagm(const int L[4], int antiperiodic, const double *U, double mass,
               const double *in_even, double *out_even)
{
    long Ve = volume(L) / 2;
    double *t = (double *)malloc(sizeof(double) * 6 * Ve);
    orc_dslash_oe(L, antiperiodic, U, in_even, t);
    orc_dslash_eo(L, antiperiodic, U, t, out_even);
    double m4 = 4.0 * mass * mass;
    for (long k = 0; k < 6 * Ve; ++k) out_even[k] = m4 * in_even[k] - out_even[k];
    free(t);
}

/* ------------------------------------------------------------------ */
/* plain FP64 conjugate gradient on A = M^dagger M (even sites)        */
/* ------------------------------------------------------------------ */

/* <a,b> = sum conj(a) b, real part */
static double re_dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long k = 0; k < n; ++k) s += a[k] * b[k]; /* pairs (re,im): re*re + im*im */
    return s;
}

/* ||b - A x||_2 / ||b||_2, recomputed in FP64 (0 when b = 0 and x = 0) */
double orc_true_residual(const int L[4], int antiperiodic, const double *U, double mass,
                         const double *b, const double *x)
{
    long n = 6 * (volume(L) / 2);
    double *Ax = (double *)malloc(sizeof(double) * n);
    orc_mdagm(L, antiperiodic, U, mass, x, Ax);
    double rr = 0.0, bb = 0.0;
    for (long k = 0; k < n; ++k) {
        double d = b[k] - Ax[k];
        rr += d * d;
        bb += b[k] * b[k];
    }
    free(Ax);
    if (bb == 0.0) return sqrt(rr);
    return sqrt(rr / bb);
}

/*
 * Textbook CG: x0 = 0, r = b, p = r; loop Ap = A p, alpha = |r|^2/<p,Ap>,
 * x += alpha p, r -= alpha Ap, beta = |r_new|^2/|r_old|^2, p = r + beta p;
 * stop when |r|/|b| <= tol.  Returns 0 when the recomputed true residual is
 * <= tol, 1 when maxiter was reached first, -5 on <p,Ap> <= 0.
 */
int orc_cg(const int L[4], int antiperiodic, const double *U, double mass, const double *b,
           double *x, double tol, int maxiter, int *iters_out, double *true_res_out)
{
    long n = 6 * (volume(L) / 2);
    double *r = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *Ap = (double *)malloc(sizeof(double) * n);
    int status = 1, it = 0;
    for (long k = 0; k < n; ++k) { x[k] = 0.0; r[k] = b[k]; p[k] = b[k]; }
    double bnorm = sqrt(re_dot(n, b, b));
    double rr = bnorm * bnorm;
    if (bnorm == 0.0) {
        status = 0;
    } else {
        while (it < maxiter) {
            orc_mdagm(L, antiperiodic, U, mass, p, Ap);
            double pAp = re_dot(n, p, Ap);
            if (!(pAp > 0.0)) { status = -5; break; }
            double alpha = rr / pAp;
            for (long k = 0; k < n; ++k) { x[k] += alpha * p[k]; r[k] -= alpha * Ap[k]; }
            double rr_new = re_dot(n, r, r);
            ++it;
            if (sqrt(rr_new) / bnorm <= tol) { status = 0; break; }
            double beta = rr_new / rr;
            for (long k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
            rr = rr_new;
        }
    }
    double tr = orc_true_residual(L, antiperiodic, U, mass, b, x);
    if (status == 0 && tr > tol) status = 1;
    if (iters_out) *iters_out = it;
    if (true_res_out) *true_res_out = tr;
    free(r); free(p); free(Ap);
    return status;
}

/*
 * Several masses, one source (the multi-mass solves of the Sec. 3 workloads:
 * the shifted systems (4 m_k^2 - D_eo D_oe) x_k = b, shift 4 m_k^2): the
 * solutions are unique, so the oracle of a multi-shift solver is the plain
 * CG above run for each mass independently.  x holds nmass vectors of 6 Ve
 * doubles, one after the other; iters/true_res one entry per mass.  Returns
 * the worst orc_cg status (0 when every mass converged).
 */
int orc_cg_masses(const int L[4], int antiperiodic, const double *U, int nmass, const double *masses,
                  const double *b, double *x, double tol, int maxiter, int *iters_out, double *true_res_out)
{
    long n = 6 * (volume(L) / 2);
    int worst = 0;
    for (int k = 0; k < nmass; ++k) {
        int st = orc_cg(L, antiperiodic, U, masses[k], b, x + k * n, tol, maxiter,
                        iters_out ? iters_out + k : NULL, true_res_out ? true_res_out + k : NULL);
        if (st != 0 && (worst == 0 || st < worst)) worst = st;
    }
    return worst;
}

/*
 * The full-lattice staggered equation M x = b with M = 2m + D (the equation
 * the inverter of Sec. 3 solves; the even-site CG above is its Schur
 * complement).  With M = [[2m, D_eo], [D_oe, 2m]] on (even, odd):
 *   (4m^2 - D_eo D_oe) x_e = 2m b_e - D_eo b_o   (orc_cg),
 *   x_o = (b_o - D_oe x_e) / (2m).
 * b and x are full vectors [V][3] complex; mass > 0.  Returns orc_cg's
 * status, with its iterations and the true residual of the even system.
 */
int orc_solve_full(const int L[4], int antiperiodic, const double *U, double mass, const double *b,
                   double *x, double tol, int maxiter, int *iters_out, double *true_res_out)
{
    long n = 6 * (volume(L) / 2);
    double *be = (double *)malloc(sizeof(double) * n);
    double *bo = (double *)malloc(sizeof(double) * n);
    double *bt = (double *)malloc(sizeof(double) * n);
    double *xe = (double *)malloc(sizeof(double) * n);
    double *xo = (double *)malloc(sizeof(double) * n);
    double *t = (double *)malloc(sizeof(double) * n);
    orc_gather_parity(L, 0, b, be);
    orc_gather_parity(L, 1, b, bo);
    orc_dslash_eo(L, antiperiodic, U, bo, t);
    for (long k = 0; k < n; ++k) bt[k] = 2.0 * mass * be[k] - t[k];
    int status = orc_cg(L, antiperiodic, U, mass, bt, xe, tol, maxiter, iters_out, true_res_out);
    orc_dslash_oe(L, antiperiodic, U, xe, t);
    for (long k = 0; k < n; ++k) xo[k] = (bo[k] - t[k]) / (2.0 * mass);
    /* each scatter zeroes the other parity: combine two full vectors */
    double *xf = (double *)malloc(sizeof(double) * 2 * n);
    orc_scatter_parity(L, 0, xe, x);
    orc_scatter_parity(L, 1, xo, xf);
    for (long k = 0; k < 2 * n; ++k) x[k] += xf[k];
    free(be); free(bo); free(bt); free(xe); free(xo); free(t); free(xf);
    return status;
}

/* ------------------------------------------------------------------ */
/* reduced-precision storage (test reference for quantised inputs)      */
/* ------------------------------------------------------------------ */

/*
 * Round v to the nearest value of a binary floating-point format with
 * `mant_bits` stored fraction bits and minimum normal exponent `emin`
 * (subnormal spacing below it), ties to even.  IEEE binary16: (10, -14);
 * bfloat16: (7, -126).  Only used on |v| well inside the format's range.
 * The grid spacing at v is 2^(max(floor(log2|v|), emin) - mant_bits); v is
 * divided by a power of two (exact) and rounded with rint(), which rounds
 * half-way cases to even in the default rounding mode.
 */
double orc_round_format(double v, int mant_bits, int emin)
{
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    frexp(fabs(v), &e); /* |v| = f 2^e, f in [0.5, 1) -> floor(log2|v|) = e - 1 */
    int E = e - 1;
    if (E < emin) E = emin;
    double spacing = ldexp(1.0, E - mant_bits);
    return rint(v / spacing) * spacing;
}

/* format parameters: prec 1 = FP32 (no second rounding), 2 = FP16, 3 = BF16 */
static void format_of(int prec, int *mant, int *emin)
{
    if (prec == 2) { *mant = 10; *emin = -14; }
    else { *mant = 7; *emin = -126; }
}

/*
 * Value a vector site holds after reduced-precision storage, per site of 6 reals:
 *   prec 1 (FP32): v -> (float)v.
 *   prec 2/3 (FP16/BF16 with a per-site scale): vf = (float)v; s = max_i |vf_i|
 *   (FP32); stored code q_i = round_format(vf_i / s) with the quotient taken in
 *   FP32 (IEEE, correctly rounded); dequantised value = (float)q_i * s in FP32.
 *   A site with s = 0 stores zeros.
 */
void orc_quantize_vectors(int prec, long nsites, const double *in, double *out)
{
    for (long i = 0; i < nsites; ++i) {
        float vf[6];
        for (int k = 0; k < 6; ++k) vf[k] = (float)in[i * 6 + k];
        if (prec == 1) {
            for (int k = 0; k < 6; ++k) out[i * 6 + k] = (double)vf[k];
            continue;
        }
        int mant, emin;
        format_of(prec, &mant, &emin);
        float s = 0.0f;
        for (int k = 0; k < 6; ++k) {
            float a = fabsf(vf[k]);
            if (a > s) s = a;
        }
        for (int k = 0; k < 6; ++k) {
            if (s == 0.0f) { out[i * 6 + k] = 0.0; continue; }
            float quot = vf[k] / s;
            float q = (float)orc_round_format((double)quot, mant, emin);
            float deq = q * s;
            out[i * 6 + k] = (double)deq;
        }
    }
}

/* Value a link element holds after storage: (float)u, then (prec 2/3) rounded
 * to FP16/BF16 without scaling (|U_ij| <= 1 for SU(3)). */
void orc_round_links(int prec, long nreals, const double *in, double *out)
{
    for (long k = 0; k < nreals; ++k) {
        float f = (float)in[k];
        if (prec == 1) { out[k] = (double)f; continue; }
        int mant, emin;
        format_of(prec, &mant, &emin);
        out[k] = orc_round_format((double)f, mant, emin);
    }
}

/* ------------------------------------------------------------------ */
/* fermion force of S = phi^dagger A^{-1} phi                          */
/* ------------------------------------------------------------------ */

/*
 * Given X = A^{-1} phi on even sites, with Y = D_oe X on odd sites,
 *   dS = X^dag dD_eo Y - Y^dag dD_oe X = Psi1^dag dD Psi2,
 * Psi1 = (X on even, -Y on odd), Psi2 = (X on even, Y on odd).
 * For the link U = U_mu(x) with s = eta_mu(x) b_mu(x) the variation of D has
 * s dU at (x, x+mu) and -s dU^dagger at (x+mu, x), so dS = Re Tr(K dU) with
 *   K_mu(x) = s [ Psi2(x+mu) Psi1(x)^dag - Psi1(x+mu) Psi2(x)^dag ].
 * Output K as [4][V][3][3] complex.  (The torch-convention gradient
 * dS/dRe U + i dS/dIm U equals K^dagger.)
 */
void orc_force_K(const int L[4], int antiperiodic, const double *U, const double *X_even,
                 double *Kd)
{
    long V = volume(L), Ve = V / 2;
    cplx *K = (cplx *)Kd;
    double *Y = (double *)malloc(sizeof(double) * 6 * Ve);
    double *psi1 = (double *)malloc(sizeof(double) * 6 * V);
    double *psi2 = (double *)malloc(sizeof(double) * 6 * V);
    double *tmp = (double *)malloc(sizeof(double) * 6 * V);
    orc_dslash_oe(L, antiperiodic, U, X_even, Y);
    /* Psi2 = (X, Y); Psi1 = (X, -Y) */
    orc_scatter_parity(L, 0, X_even, psi1);
    orc_scatter_parity(L, 1, Y, tmp);
    for (long k = 0; k < 6 * V; ++k) {
        psi2[k] = psi1[k] + tmp[k];
        psi1[k] = psi1[k] - tmp[k];
    }
    const cplx *P1 = (const cplx *)psi1, *P2 = (const cplx *)psi2;
    for (int mu = 0; mu < 4; ++mu) {
        for (long i = 0; i < V; ++i) {
            int x[4], xf[4];
            coords_of(L, i, x);
            for (int d = 0; d < 4; ++d) xf[d] = x[d];
            xf[mu] = (x[mu] + 1) % L[mu];
            long j = lex_of(L, xf);
            double s = (double)(eta(mu, x) * bsign(mu, x, L, antiperiodic));
            cplx *k = K + ((long)mu * V + i) * 9;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    cplx t1 = c_mul(P2[j * 3 + a], c_conj(P1[i * 3 + b]));
                    cplx t2 = c_mul(P1[j * 3 + a], c_conj(P2[i * 3 + b]));
                    k[a * 3 + b] = c_scale(s, c_sub(t1, t2));
                }
        }
    }
    free(Y); free(psi1); free(psi2); free(tmp);
}

/*
 * Lie-algebra projection of the force for the left variation
 * U -> exp(i w T_a) U, T_a = lambda_a / 2 (Gell-Mann):
 *   f_a = dS/dw_a = Re Tr(i T_a U K),  a = 1..8, stored [4][V][8].
 */
void orc_force_lie(long nlinks, const double *Ud, const double *Kd, double *f)
{
    const cplx *U = (const cplx *)Ud, *K = (const cplx *)Kd;
    /* Gell-Mann matrices, entries (re, im), row-major */
    static const double lam[8][9][2] = {
        {{0,0},{1,0},{0,0},{1,0},{0,0},{0,0},{0,0},{0,0},{0,0}},
        {{0,0},{0,-1},{0,0},{0,1},{0,0},{0,0},{0,0},{0,0},{0,0}},
        {{1,0},{0,0},{0,0},{0,0},{-1,0},{0,0},{0,0},{0,0},{0,0}},
        {{0,0},{0,0},{1,0},{0,0},{0,0},{0,0},{1,0},{0,0},{0,0}},
        {{0,0},{0,0},{0,-1},{0,0},{0,0},{0,0},{0,1},{0,0},{0,0}},
        {{0,0},{0,0},{0,0},{0,0},{0,0},{1,0},{0,0},{1,0},{0,0}},
        {{0,0},{0,0},{0,0},{0,0},{0,0},{0,-1},{0,0},{0,1},{0,0}},
        {{0,0},{0,0},{0,0},{0,0},{0,0},{0,0},{0,0},{0,0},{0,0}},
    };
    double l8[9][2] = {{0}};
    double c8 = 1.0 / sqrt(3.0);
    l8[0][0] = c8; l8[4][0] = c8; l8[8][0] = -2.0 * c8;
    for (long n = 0; n < nlinks; ++n) {
        const cplx *u = U + n * 9, *k = K + n * 9;
        cplx UK[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                cplx s = {0, 0};
                for (int c = 0; c < 3; ++c) s = c_add(s, c_mul(u[a * 3 + c], k[c * 3 + b]));
                UK[a * 3 + b] = s;
            }
        for (int g = 0; g < 8; ++g) {
            const double (*lm)[2] = (g == 7) ? (const double (*)[2])l8 : lam[g];
            /* Tr(i T UK) = (i/2) sum_{ab} lam_ab (UK)_ba */
            cplx tr = {0, 0};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    cplx la = {lm[a * 3 + b][0], lm[a * 3 + b][1]};
                    tr = c_add(tr, c_mul(la, UK[b * 3 + a]));
                }
            /* Re( i/2 * tr ) = -Im(tr) / 2 */
            f[n * 8 + g] = -0.5 * tr.im;
        }
    }
}

/* ------------------------------------------------------------------ */
/* HYP smearing of the gauge field                                     */
/* ------------------------------------------------------------------ */
/*
 * Sec. 3 runs the CG on "HYP-smeared" staggered quarks: the one-link field U
 * of the operator above is the hypercubic-blocked field of the thin links.
 * The paper names the smearing without writing it; the oracle follows
 * Hasenfratz & Knechtli's three-level construction (Phys. Rev. D 64, 034504),
 * every level a projection back to SU(3) of the thin link plus a weighted
 * sum of staples built from the level below, all staples kept inside the
 * hypercubes that contain the link:
 *   level 1  Vb(x,mu;eta) = P[(1-a3) U_mu(x) + a3/2 sum_{+-eta} U_eta(x) U_mu(x+eta) U_eta(x+mu)^dag]
 *            (eta the one direction outside {mu, nu, rho}: the decoration
 *            {nu, rho} is written by the staple direction eta)
 *   level 2  Vt(x,mu;nu) = P[(1-a2) U_mu(x) + a2/4 sum_{+-rho, rho != mu,nu}
 *                 Vb(x,rho;s) Vb(x+rho,mu;s) Vb(x+mu,rho;s)^dag],  s = the direction outside {mu,nu,rho}
 *   level 3  V(x,mu)     = P[(1-a1) U_mu(x) + a1/6 sum_{+-nu != mu} Vt(x,nu;mu) Vt(x+nu,mu;nu) Vt(x+mu,nu;mu)^dag]
 * A staple in the negative direction -d reads the same product starting at
 * x-d with the first factor daggered and the last not:
 *   W_d(x-d)^dag W_mu(x-d) W_d(x-d+mu).
 * P = projection to SU(3): the unitary polar factor Y = X (X^dag X)^(-1/2)
 * (Newton's iteration Y <- (Y + Y^-dag)/2 from Y = X, to convergence), then
 * the determinant's phase removed with the principal cube root:
 * P(X) = Y exp(-i arg(det Y) / 3).  (Both readings are recorded with the
 * library's design notes; the parameters are Hasenfratz & Knechtli's
 * (a1, a2, a3) = (0.75, 0.6, 0.3) by default.)
 */

static void m_mul(const cplx *a, const cplx *b, cplx *c) /* c = a b */
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = {0, 0};
            for (int k = 0; k < 3; ++k) s = c_add(s, c_mul(a[i * 3 + k], b[k * 3 + j]));
            c[i * 3 + j] = s;
        }
}

static void m_dag(const cplx *a, cplx *c) /* c = a^dagger */
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c[i * 3 + j] = c_conj(a[j * 3 + i]);
}

static cplx m_det(const cplx *a)
{
    cplx t0 = c_sub(c_mul(a[4], a[8]), c_mul(a[5], a[7]));
    cplx t1 = c_sub(c_mul(a[3], a[8]), c_mul(a[5], a[6]));
    cplx t2 = c_sub(c_mul(a[3], a[7]), c_mul(a[4], a[6]));
    return c_add(c_sub(c_mul(a[0], t0), c_mul(a[1], t1)), c_mul(a[2], t2));
}

/* inverse by cofactors: inv = adj(a) / det(a) */
static void m_inv(const cplx *a, cplx *inv)
{
    cplx d = m_det(a);
    double dd = d.re * d.re + d.im * d.im;
    cplx rd = {d.re / dd, -d.im / dd};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            /* cofactor C_ji (transposed into inv_ij) */
            int r0 = (j + 1) % 3, r1 = (j + 2) % 3, c0 = (i + 1) % 3, c1 = (i + 2) % 3;
            cplx m = c_sub(c_mul(a[r0 * 3 + c0], a[r1 * 3 + c1]), c_mul(a[r0 * 3 + c1], a[r1 * 3 + c0]));
            inv[i * 3 + j] = c_mul(m, rd);
        }
}

/* P(X): unitary polar factor by Newton's iteration, determinant phase removed */
void orc_su3_project(const double *Xd, double *Wd)
{
    const cplx *X = (const cplx *)Xd;
    cplx *W = (cplx *)Wd;
    cplx Y[9], Yi[9], Yn[9];
    for (int k = 0; k < 9; ++k) Y[k] = X[k];
    for (int it = 0; it < 100; ++it) {
        m_inv(Y, Yi);
        double diff = 0.0, norm = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                cplx yid = c_conj(Yi[j * 3 + i]); /* (Y^-1)^dagger */
                cplx n = c_scale(0.5, c_add(Y[i * 3 + j], yid));
                cplx e = c_sub(n, Y[i * 3 + j]);
                diff += e.re * e.re + e.im * e.im;
                norm += n.re * n.re + n.im * n.im;
                Yn[i * 3 + j] = n;
            }
        for (int k = 0; k < 9; ++k) Y[k] = Yn[k];
        if (diff <= 1e-32 * norm) break;
    }
    cplx d = m_det(Y);
    double ph = atan2(d.im, d.re) / 3.0;
    cplx rot = {cos(ph), -sin(ph)};
    for (int k = 0; k < 9; ++k) W[k] = c_mul(Y[k], rot);
}

/* the link W(x + s d) of direction `dir` of a field [4][V][3][3], and x + s d */
static const cplx *fld(const cplx *F, long V, int dir, const int L[4], const int x[4])
{
    return F + ((long)dir * V + lex_of(L, x)) * 9;
}

static void shifted(const int L[4], const int x[4], int d, int s, int y[4])
{
    for (int k = 0; k < 4; ++k) y[k] = x[k];
    y[d] = (x[d] + s + L[d]) % L[d];
}

/*
 * acc += A(x, d) B(x+d, mu) C(x+mu, d)^dag   (positive d)
 * acc += A(x-d, d)^dag B(x-d, mu) C(x-d+mu, d) (negative d)
 * for link getters a/b/c of the same form: (field, decoration index) pairs.
 */
typedef const cplx *(*link_fn)(const void *ctx, int dir, const int y[4]);

static void add_staples_dir(const int L[4], const int x[4], int mu, int d, link_fn fa, const void *ca, link_fn fb,
                            const void *cb, link_fn fc, const void *cc, cplx *acc)
{
    int xd[4], xmu[4], xmd[4], xmdmu[4];
    cplx t[9], s[9], cd[9];
    /* positive d */
    shifted(L, x, d, 1, xd);
    shifted(L, x, mu, 1, xmu);
    m_mul(fa(ca, d, x), fb(cb, mu, xd), t);
    m_dag(fc(cc, d, xmu), cd);
    m_mul(t, cd, s);
    for (int k = 0; k < 9; ++k) acc[k] = c_add(acc[k], s[k]);
    /* negative d */
    shifted(L, x, d, -1, xmd);
    shifted(L, xmd, mu, 1, xmdmu);
    m_dag(fa(ca, d, xmd), cd);
    m_mul(cd, fb(cb, mu, xmd), t);
    m_mul(t, fc(cc, d, xmdmu), s);
    for (int k = 0; k < 9; ++k) acc[k] = c_add(acc[k], s[k]);
}

typedef struct {
    const cplx *F;
    long V;
    const int *L;
    int tag; /* decoration argument passed by the level (see the getters) */
} fctx;

/* thin links: U_dir(y) */
static const cplx *get_thin(const void *c, int dir, const int y[4])
{
    const fctx *f = (const fctx *)c;
    return fld(f->F, f->V, dir, f->L, y);
}

/* level 1 links Vb(y, dir; s), stored [4 dir][4 s][V][3][3] (s != dir), s = tag */
static const cplx *get_vb(const void *c, int dir, const int y[4])
{
    const fctx *f = (const fctx *)c;
    return f->F + (((long)dir * 4 + f->tag) * f->V + lex_of(f->L, y)) * 9;
}

/* level 2 links Vt(y, dir; nu), stored [4 dir][4 nu][V][3][3]; the
 * decoration of the link in direction `dir` is the other direction of the
 * staple: tag = the level-3 link direction mu for the side links (Vt(.,nu;mu)),
 * and the side direction nu for the middle link (Vt(.,mu;nu)) */
static const cplx *get_vt(const void *c, int dir, const int y[4])
{
    const fctx *f = (const fctx *)c;
    return f->F + (((long)dir * 4 + f->tag) * f->V + lex_of(f->L, y)) * 9;
}

/*
 * out = HYP-smeared links [4][V][3][3] of U, parameters alpha = (a1, a2, a3).
 */
void orc_hyp(const int L[4], const double *Ud, const double *alpha, double *outd)
{
    const long V = volume(L);
    const cplx *U = (const cplx *)Ud;
    cplx *out = (cplx *)outd;
    const double a1 = alpha[0], a2 = alpha[1], a3 = alpha[2];
    cplx *Vb = (cplx *)calloc((size_t)16 * V * 9, sizeof(cplx));
    cplx *Vt = (cplx *)calloc((size_t)16 * V * 9, sizeof(cplx));
    fctx thin = {U, V, L, 0};
    /* level 1: Vb(x, mu; eta) for eta != mu (eta = the staple direction) */
    for (int mu = 0; mu < 4; ++mu)
        for (int eta = 0; eta < 4; ++eta) {
            if (eta == mu) continue;
            for (long i = 0; i < V; ++i) {
                int x[4];
                coords_of(L, i, x);
                cplx acc[9] = {{0, 0}};
                add_staples_dir(L, x, mu, eta, get_thin, &thin, get_thin, &thin, get_thin, &thin, acc);
                const cplx *u = fld(U, V, mu, L, x);
                cplx X[9];
                for (int k = 0; k < 9; ++k) X[k] = c_add(c_scale(1.0 - a3, u[k]), c_scale(a3 / 2.0, acc[k]));
                orc_su3_project((const double *)X, (double *)(Vb + (((long)mu * 4 + eta) * V + i) * 9));
            }
        }
    /* level 2: Vt(x, mu; nu) for nu != mu: staples over rho not in {mu, nu},
     * built from Vb decorated by s = the direction outside {mu, nu, rho} */
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == mu) continue;
            for (long i = 0; i < V; ++i) {
                int x[4];
                coords_of(L, i, x);
                cplx acc[9] = {{0, 0}};
                for (int rho = 0; rho < 4; ++rho) {
                    if (rho == mu || rho == nu) continue;
                    int sdir = 6 - mu - nu - rho; /* 0+1+2+3 = 6 */
                    fctx vb = {Vb, V, L, sdir};
                    add_staples_dir(L, x, mu, rho, get_vb, &vb, get_vb, &vb, get_vb, &vb, acc);
                }
                const cplx *u = fld(U, V, mu, L, x);
                cplx X[9];
                for (int k = 0; k < 9; ++k) X[k] = c_add(c_scale(1.0 - a2, u[k]), c_scale(a2 / 4.0, acc[k]));
                orc_su3_project((const double *)X, (double *)(Vt + (((long)mu * 4 + nu) * V + i) * 9));
            }
        }
    /* level 3: V(x, mu): staples over nu != mu from Vt(., nu; mu) (sides) and Vt(., mu; nu) (middle) */
    for (int mu = 0; mu < 4; ++mu)
        for (long i = 0; i < V; ++i) {
            int x[4];
            coords_of(L, i, x);
            cplx acc[9] = {{0, 0}};
            for (int nu = 0; nu < 4; ++nu) {
                if (nu == mu) continue;
                fctx side = {Vt, V, L, mu}, mid = {Vt, V, L, nu};
                add_staples_dir(L, x, mu, nu, get_vt, &side, get_vt, &mid, get_vt, &side, acc);
            }
            const cplx *u = fld(U, V, mu, L, x);
            cplx X[9];
            for (int k = 0; k < 9; ++k) X[k] = c_add(c_scale(1.0 - a1, u[k]), c_scale(a1 / 6.0, acc[k]));
            orc_su3_project((const double *)X, (double *)(out + ((long)mu * V + i) * 9));
        }
    free(Vb);
    free(Vt);
}

/* ------------------------------------------------------------------ */
/* NPR: the one-colour-trace four-fermion contraction                  */
/* ------------------------------------------------------------------ */
/*
 * Sec. 4 of the paper (its DP workload, Eq. (ffop)): on every hypercube z of
 * the lattice (sites z_A = 2z + A, corners A in {0,1}^4),
 *   O(z) = sum_{A,B,C,D} [chibar1(z_A) (g_S1 x x_F1)_AB chi2(z_B)]
 *                        [chibar3(z_C) (g_S2 x x_F2)_CD chi4(z_D)]
 *                        [U_AD(z)]_{c1 c4} [U_CB(z)]_{c3 c2},
 * colour c1 of chibar1 tied to c4 of chi4 and c3 of chibar3 to c2 of chi2
 * through the links (one colour trace across the two bilinears).  The paper
 * writes the form only; the readings (recorded with the design notes):
 *   - spin-taste matrices (g_S x x_F)_AB = (1/4) Tr(g_A^dag g_S g_B g_F^dag),
 *     g_A = g_1^A1 g_2^A2 g_3^A3 g_4^A4 with Euclidean Hermitian gammas
 *     (directions x, y, z, t = bits 0..3 of A), here from explicit 4x4
 *     matrices (the chiral basis);
 *   - U_AD(z) = the average over the |A xor D|! shortest lattice paths from
 *     z_A to z_D (inside the hypercube) of the products of links along them
 *     (U_mu(y) for a step +mu, U_mu(y - mu)^dag for -mu), 1 for A = D;
 *   - chibar1, chi2, chibar3, chi4: colour-vector fields [V][3] (for NPR the
 *     columns of quark propagators); no conjugation (chibar is its own field).
 * O has [V/16] entries, hypercube index h = z0 + (L0/2)(z1 + (L1/2)(z2 + (L2/2) z3)).
 */

/* Euclidean Hermitian gamma matrices, chiral basis: g_k = [[0, -i s_k], [i s_k, 0]], g_4 = [[0, 1], [1, 0]] */
static void gamma_mat(int mu, cplx g[16])
{
    static const double sig[3][2][2][2] = {
        {{{0, 0}, {1, 0}}, {{1, 0}, {0, 0}}},
        {{{0, 0}, {0, -1}}, {{0, 1}, {0, 0}}},
        {{{1, 0}, {0, 0}}, {{0, 0}, {-1, 0}}},
    };
    for (int k = 0; k < 16; ++k) g[k].re = g[k].im = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            if (mu < 3) {
                cplx s = {sig[mu][a][b][0], sig[mu][a][b][1]};
                cplx mi = {0, -1}, pi = {0, 1};
                g[a * 4 + (2 + b)] = c_mul(mi, s);     /* upper right: -i s */
                g[(2 + a) * 4 + b] = c_mul(pi, s);     /* lower left:  +i s */
            } else if (a == b) {
                g[a * 4 + (2 + b)].re = 1.0;
                g[(2 + a) * 4 + b].re = 1.0;
            }
        }
}

static void m4_mul(const cplx *a, const cplx *b, cplx *c)
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = {0, 0};
            for (int k = 0; k < 4; ++k) s = c_add(s, c_mul(a[i * 4 + k], b[k * 4 + j]));
            c[i * 4 + j] = s;
        }
}

/* g_A for a 4-bit corner A */
static void gamma_of(int A, cplx g[16])
{
    for (int k = 0; k < 16; ++k) { g[k].re = (k % 5 == 0) ? 1.0 : 0.0; g[k].im = 0.0; }
    for (int mu = 0; mu < 4; ++mu) {
        if (!((A >> mu) & 1)) continue;
        cplx gm[16], t[16];
        gamma_mat(mu, gm);
        m4_mul(g, gm, t);
        for (int k = 0; k < 16; ++k) g[k] = t[k];
    }
}

/* out[A*16+B] = (1/4) Tr(g_A^dag g_S g_B g_F^dag) (complex) */
void orc_spin_taste(int S, int F, double *outd)
{
    cplx *out = (cplx *)outd;
    cplx gS[16], gF[16], gFd[16];
    gamma_of(S, gS);
    gamma_of(F, gF);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) gFd[i * 4 + j] = c_conj(gF[j * 4 + i]);
    for (int A = 0; A < 16; ++A) {
        cplx gA[16], gAd[16];
        gamma_of(A, gA);
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) gAd[i * 4 + j] = c_conj(gA[j * 4 + i]);
        for (int B = 0; B < 16; ++B) {
            cplx gB[16], t1[16], t2[16], t3[16];
            gamma_of(B, gB);
            m4_mul(gAd, gS, t1);
            m4_mul(t1, gB, t2);
            m4_mul(t2, gFd, t3);
            cplx tr = {0, 0};
            for (int k = 0; k < 4; ++k) tr = c_add(tr, t3[k * 5]);
            out[A * 16 + B] = c_scale(0.25, tr);
        }
    }
}

/* site of corner A of hypercube with coordinates zc */
static long corner_site(const int L[4], const int zc[4], int A)
{
    int x[4];
    for (int mu = 0; mu < 4; ++mu) x[mu] = 2 * zc[mu] + ((A >> mu) & 1);
    return lex_of(L, x);
}

/* W = average over the shortest paths from corner A to corner D of hypercube zc */
void orc_hypercube_path(const int L[4], const double *Ud, const int zc[4], int A, int D, double *Wd)
{
    const cplx *U = (const cplx *)Ud;
    cplx *W = (cplx *)Wd;
    long V = volume(L);
    int dirs[4], n = 0;
    for (int mu = 0; mu < 4; ++mu)
        if (((A ^ D) >> mu) & 1) dirs[n++] = mu;
    for (int k = 0; k < 9; ++k) { W[k].re = (k % 4 == 0) ? 1.0 : 0.0; W[k].im = 0.0; }
    if (n == 0) return;
    for (int k = 0; k < 9; ++k) W[k].re = W[k].im = 0.0;
    /* every ordering of the differing directions (permutations by Heap's enumeration over indices) */
    int perm[4] = {0, 1, 2, 3};
    int npaths = 0;
    /* enumerate all n! orderings with a plain nested loop over permutations of 0..n-1 */
    int idx[4];
    int total = 1;
    for (int k = 2; k <= n; ++k) total *= k;
    for (int p = 0; p < total; ++p) {
        /* p-th permutation in factorial numbering */
        int avail[4] = {0, 1, 2, 3}, m = n, r = p;
        for (int k = 0; k < n; ++k) {
            int f = 1;
            for (int q = 2; q <= m - 1; ++q) f *= q;
            int sel = r / f;
            r %= f;
            idx[k] = avail[sel];
            for (int q = sel; q < m - 1; ++q) avail[q] = avail[q + 1];
            --m;
        }
        cplx P[9];
        for (int k = 0; k < 9; ++k) { P[k].re = (k % 4 == 0) ? 1.0 : 0.0; P[k].im = 0.0; }
        int cur = A;
        for (int k = 0; k < n; ++k) {
            int mu = dirs[idx[k]];
            int nxt = cur ^ (1 << mu);
            cplx step[9], T[9];
            if ((cur >> mu) & 1) { /* step -mu: U_mu(z_nxt)^dag */
                m_dag(U + ((long)mu * V + corner_site(L, zc, nxt)) * 9, step);
            } else {                /* step +mu: U_mu(z_cur) */
                for (int q = 0; q < 9; ++q) step[q] = U[((long)mu * V + corner_site(L, zc, cur)) * 9 + q];
            }
            m_mul(P, step, T);
            for (int q = 0; q < 9; ++q) P[q] = T[q];
            cur = nxt;
        }
        for (int q = 0; q < 9; ++q) W[q] = c_add(W[q], P[q]);
        ++npaths;
    }
    (void)perm;
    for (int q = 0; q < 9; ++q) W[q] = c_scale(1.0 / npaths, W[q]);
}

/* O(z) for every hypercube (out [V/16] complex); returns nothing */
void orc_npr_contract(const int L[4], const double *Ud, int S1, int F1, int S2, int F2, const double *chibar1d,
                      const double *chi2d, const double *chibar3d, const double *chi4d, double *outd)
{
    const cplx *cb1 = (const cplx *)chibar1d, *c2 = (const cplx *)chi2d;
    const cplx *cb3 = (const cplx *)chibar3d, *c4 = (const cplx *)chi4d;
    cplx *out = (cplx *)outd;
    cplx st1[256], st2[256];
    orc_spin_taste(S1, F1, (double *)st1);
    orc_spin_taste(S2, F2, (double *)st2);
    int H[4] = {L[0] / 2, L[1] / 2, L[2] / 2, L[3] / 2};
    long nh = (long)H[0] * H[1] * H[2] * H[3];
    for (long h = 0; h < nh; ++h) {
        int zc[4];
        long r = h;
        zc[0] = (int)(r % H[0]); r /= H[0];
        zc[1] = (int)(r % H[1]); r /= H[1];
        zc[2] = (int)(r % H[2]);
        zc[3] = (int)(r / H[2]);
        cplx o = {0, 0};
        for (int A = 0; A < 16; ++A)
            for (int B = 0; B < 16; ++B) {
                cplx s1 = st1[A * 16 + B];
                if (s1.re == 0.0 && s1.im == 0.0) continue;
                for (int C = 0; C < 16; ++C)
                    for (int D = 0; D < 16; ++D) {
                        cplx s2 = st2[C * 16 + D];
                        if (s2.re == 0.0 && s2.im == 0.0) continue;
                        cplx Wad[9], Wcb[9];
                        orc_hypercube_path(L, Ud, zc, A, D, (double *)Wad);
                        orc_hypercube_path(L, Ud, zc, C, B, (double *)Wcb);
                        long sA = corner_site(L, zc, A), sB = corner_site(L, zc, B);
                        long sC = corner_site(L, zc, C), sD = corner_site(L, zc, D);
                        /* chibar1_c1 U_AD[c1][c4] chi4_c4 and chibar3_c3 U_CB[c3][c2] chi2_c2 */
                        cplx t1 = {0, 0}, t2 = {0, 0};
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) {
                                t1 = c_add(t1, c_mul(cb1[sA * 3 + a], c_mul(Wad[a * 3 + b], c4[sD * 3 + b])));
                                t2 = c_add(t2, c_mul(cb3[sC * 3 + a], c_mul(Wcb[a * 3 + b], c2[sB * 3 + b])));
                            }
                        o = c_add(o, c_mul(c_mul(s1, s2), c_mul(t1, t2)));
                    }
            }
        out[h] = o;
    }
}
