/*
 * Plain FP64 CPU oracle for the Wilson fermion matrix and its BiCGStab solve.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously correct statement of
 * what the GPU library computes.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it.  The GPU library never links, includes
 * or calls this file, and the two share no code, header or constant table.
 *
 * Operator (Eq. 1, Sec. 2 "Wilson Fermion Matrix"):
 *   D(x,y) = delta_{x,y} - kappa * sum_mu [ (1 - gamma_mu) U_mu(x) delta_{x+mu,y}
 *                                         + (1 + gamma_mu) U_mu(x-mu)^dag delta_{x-mu,y} ]
 *   H = the bracketed sum over mu (the hopping term), so D = 1 - kappa H,
 *   kappa = 1/(8 + 2 m0).
 *
 * Conventions (canonical layout; the GPU library follows the same convention
 * through its own code):
 *   site index   s = x + Lx*(y + Ly*(z + Lz*t))       x fastest (Sec. 4.1, layout 1)
 *   gauge field  U[s][mu][a][b]   complex (re, im)    mu = 0..3 for x, y, z, t
 *   fermion      psi[s][spin][colour] complex         4 spins x 3 colours (Sec. 2)
 *   half field   psi_p[i][spin][colour], i = s/2 over the sites s of parity
 *                p = (x+y+z+t) mod 2 (needs Lx even)
 *   gamma basis  the paper does not fix one; this oracle uses the Hermitian
 *                chiral (DeGrand-Rossi) basis written out in GAMMA below.
 *   boundaries   Sec. 2 allows periodic or antiperiodic conditions.  A hop that
 *                crosses the lattice edge in direction mu is multiplied by the
 *                phase phi_mu (forward hop) or conj(phi_mu) (backward hop);
 *                |phi_mu| = 1, so periodic is phi = 1, antiperiodic phi = -1.
 *
 * Every function works on whole fields in the canonical layout; the even-odd
 * functions embed a half field into a full-lattice field (zeros on the other
 * parity), apply the full stencil, and read back the wanted parity.  Nothing
 * is blocked, fused or reordered beyond Eq. 1 itself.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NC 3
#define NS 4
#define SITE_REALS (2 * NS * NC) /* 24 reals per fermion site */
#define LINK_REALS (2 * NC * NC) /* 18 reals per SU(3) link */

/* Hermitian chiral (DeGrand-Rossi) gamma matrices, [mu][row][col][re,im].
 * gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1). */
static const double GAMMA[4][4][4][2] = {
    /* gamma_1 (x) */
    {{{0, 0}, {0, 0}, {0, 0}, {0, 1}},
     {{0, 0}, {0, 0}, {0, 1}, {0, 0}},
     {{0, 0}, {0, -1}, {0, 0}, {0, 0}},
     {{0, -1}, {0, 0}, {0, 0}, {0, 0}}},
    /* gamma_2 (y) */
    {{{0, 0}, {0, 0}, {0, 0}, {-1, 0}},
     {{0, 0}, {0, 0}, {1, 0}, {0, 0}},
     {{0, 0}, {1, 0}, {0, 0}, {0, 0}},
     {{-1, 0}, {0, 0}, {0, 0}, {0, 0}}},
    /* gamma_3 (z) */
    {{{0, 0}, {0, 0}, {0, 1}, {0, 0}},
     {{0, 0}, {0, 0}, {0, 0}, {0, -1}},
     {{0, -1}, {0, 0}, {0, 0}, {0, 0}},
     {{0, 0}, {0, 1}, {0, 0}, {0, 0}}},
    /* gamma_4 (t) */
    {{{0, 0}, {0, 0}, {1, 0}, {0, 0}},
     {{0, 0}, {0, 0}, {0, 0}, {1, 0}},
     {{1, 0}, {0, 0}, {0, 0}, {0, 0}},
     {{0, 0}, {1, 0}, {0, 0}, {0, 0}}},
};

/* ------------------------------------------------------------------ */
/* threads                                                             */
/* ------------------------------------------------------------------ */

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_gamma(int mu, double* out /* 4x4 complex, row-major */)
{
    memcpy(out, GAMMA[mu], sizeof(GAMMA[mu]));
}

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */

static long volume(const int* L) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords(const int* L, long s, int c[4])
{
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = (int)(s % L[mu]);
        s /= L[mu];
    }
}

static long index_of(const int* L, const int c[4])
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

static int parity_of(const int* L, long s)
{
    int c[4];
    coords(L, s, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* Neighbour of s one step (+1 or -1) along mu with periodic wrap-around.
 * *crossed is set when the hop crosses the lattice edge. */
static long neighbour(const int* L, long s, int mu, int step, int* crossed)
{
    int c[4];
    coords(L, s, c);
    int v = c[mu] + step;
    *crossed = 0;
    if (v < 0) { v += L[mu]; *crossed = 1; }
    if (v >= L[mu]) { v -= L[mu]; *crossed = 1; }
    c[mu] = v;
    return index_of(L, c);
}

/* ------------------------------------------------------------------ */
/* one term of Eq. 1 at one site                                       */
/* ------------------------------------------------------------------ */

/* acc[spin][colour] += phase * (1 + sign*gamma_mu) (M v), where M is the 3x3
 * link (or its adjoint when `adjoint` is set) acting on colour and v is the
 * neighbour's 4x3 spinor. */
static void add_term(double* acc, int mu, double sign, const double* M, int adjoint,
                     const double* v, double ph_re, double ph_im)
{
    double w[NS][NC][2];
    for (int sp = 0; sp < NS; ++sp)
        for (int a = 0; a < NC; ++a) {
            double re = 0.0, im = 0.0;
            for (int b = 0; b < NC; ++b) {
                double mre, mim;
                if (adjoint) { /* (M^dag)_{ab} = conj(M_{ba}) */
                    mre = M[2 * (b * NC + a)];
                    mim = -M[2 * (b * NC + a) + 1];
                } else {
                    mre = M[2 * (a * NC + b)];
                    mim = M[2 * (a * NC + b) + 1];
                }
                double vre = v[2 * (sp * NC + b)], vim = v[2 * (sp * NC + b) + 1];
                re += mre * vre - mim * vim;
                im += mre * vim + mim * vre;
            }
            /* boundary phase */
            w[sp][a][0] = ph_re * re - ph_im * im;
            w[sp][a][1] = ph_re * im + ph_im * re;
        }
    for (int sp = 0; sp < NS; ++sp)
        for (int a = 0; a < NC; ++a) {
            double re = w[sp][a][0], im = w[sp][a][1]; /* the identity part */
            for (int tp = 0; tp < NS; ++tp) {
                double gre = sign * GAMMA[mu][sp][tp][0];
                double gim = sign * GAMMA[mu][sp][tp][1];
                re += gre * w[tp][a][0] - gim * w[tp][a][1];
                im += gre * w[tp][a][1] + gim * w[tp][a][0];
            }
            acc[2 * (sp * NC + a)] += re;
            acc[2 * (sp * NC + a) + 1] += im;
        }
}

/* (H psi)(s) following Eq. 1 term by term.  d = +1 gives H, d = -1 gives the
 * hopping term of D^dag.  Derivation of the adjoint: the forward term maps
 * psi(x+mu) to site x with (1-gamma_mu)U_mu(x); its adjoint maps psi(x) to
 * site x+mu with (1-gamma_mu)U_mu(x)^dag (gamma_mu is Hermitian).  Relabelled
 * to the receiving site y, D^dag carries (1+gamma_mu)U_mu(y) on the forward
 * neighbour and (1-gamma_mu)U_mu(y-mu)^dag on the backward one: the sign of
 * gamma_mu flips and nothing else changes. */
static void hop_site(const int* L, const double* bc, const double* U, const double* in,
                     long s, int d, double* out_site)
{
    for (int k = 0; k < SITE_REALS; ++k) out_site[k] = 0.0;
    for (int mu = 0; mu < 4; ++mu) {
        int crossed;
        /* forward: (1 - d gamma_mu) U_mu(x) psi(x + mu) */
        long f = neighbour(L, s, mu, +1, &crossed);
        double pre = crossed ? bc[2 * mu] : 1.0, pim = crossed ? bc[2 * mu + 1] : 0.0;
        add_term(out_site, mu, -(double)d, U + (s * 4 + mu) * LINK_REALS, 0,
                 in + f * SITE_REALS, pre, pim);
        /* backward: (1 + d gamma_mu) U_mu(x - mu)^dag psi(x - mu) */
        long b = neighbour(L, s, mu, -1, &crossed);
        pre = crossed ? bc[2 * mu] : 1.0;
        pim = crossed ? -bc[2 * mu + 1] : 0.0;
        add_term(out_site, mu, +(double)d, U + (b * 4 + mu) * LINK_REALS, 1,
                 in + b * SITE_REALS, pre, pim);
    }
}

/* ------------------------------------------------------------------ */
/* full-lattice operators                                              */
/* ------------------------------------------------------------------ */

/* out = H in (d = +1) or the hopping term of D^dag (d = -1), whole lattice. */
void orc_hop_full(const double* U, const double* in, double* out, const int* L,
                  const double* bc, int d)
{
    long V = volume(L);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; ++s) hop_site(L, bc, U, in, s, d, out + s * SITE_REALS);
}

/* out = D in = in - kappa H in (Eq. 1); d = -1 gives D^dag. */
void orc_D_full(const double* U, const double* in, double* out, const int* L,
                const double* bc, double kappa, int d)
{
    long V = volume(L);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; ++s) {
        double h[SITE_REALS];
        hop_site(L, bc, U, in, s, d, h);
        for (int k = 0; k < SITE_REALS; ++k)
            out[s * SITE_REALS + k] = in[s * SITE_REALS + k] - kappa * h[k];
    }
}

/* ------------------------------------------------------------------ */
/* even-odd (checkerboard) pieces                                      */
/* ------------------------------------------------------------------ */

/* The full-lattice site of parity p whose half index is i. */
static long site_of_half(const int* L, long i, int p)
{
    long s = 2 * i;
    return parity_of(L, s) == p ? s : s + 1;
}

static void embed_half(const int* L, const double* half, int p, double* full)
{
    long V = volume(L), Vh = V / 2;
    memset(full, 0, sizeof(double) * V * SITE_REALS);
    for (long i = 0; i < Vh; ++i)
        memcpy(full + site_of_half(L, i, p) * SITE_REALS, half + i * SITE_REALS,
               sizeof(double) * SITE_REALS);
}

/* out_half (parity p) = H_{p,1-p} in_half (parity 1-p): Eq. 1's hopping term
 * restricted to the two checkerboards.  The input is embedded into a full
 * field that is zero on parity p, and H is evaluated at the parity-p sites. */
void orc_hop_eo(const double* U, const double* in_half, double* out_half, const int* L,
                const double* bc, int out_parity, int d)
{
    long V = volume(L), Vh = V / 2;
    double* full = (double*)malloc(sizeof(double) * V * SITE_REALS);
    embed_half(L, in_half, 1 - out_parity, full);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < Vh; ++i)
        hop_site(L, bc, U, full, site_of_half(L, i, out_parity), d, out_half + i * SITE_REALS);
    free(full);
}

/* Same as orc_hop_eo but only at the half indices listed in `sites`; output
 * rows are written in list order (used for sampled checks at large volume). */
void orc_hop_eo_sites(const double* U, const double* in_half, const int* L, const double* bc,
                      int out_parity, int d, const long* sites, long nsites, double* out_rows)
{
    long V = volume(L);
    double* full = (double*)malloc(sizeof(double) * V * SITE_REALS);
    embed_half(L, in_half, 1 - out_parity, full);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nsites; ++k)
        hop_site(L, bc, U, full, site_of_half(L, sites[k], out_parity), d,
                 out_rows + k * SITE_REALS);
    free(full);
}

/* Schur complement on the even sites:  M_ee = 1 - kappa^2 H_eo H_oe.
 * With D = [[1, -kappa H_eo], [-kappa H_oe, 1]] in (even, odd) blocks,
 * M_ee = D_ee - D_eo D_oo^{-1} D_oe. */
void orc_Mee(const double* U, const double* in_e, double* out_e, const int* L, const double* bc,
             double kappa, int d)
{
    long Vh = volume(L) / 2;
    double* tmp = (double*)malloc(sizeof(double) * Vh * SITE_REALS);
    orc_hop_eo(U, in_e, tmp, L, bc, 1, d);   /* tmp = H_oe in_e   */
    orc_hop_eo(U, tmp, out_e, L, bc, 0, d);  /* out = H_eo tmp    */
    for (long k = 0; k < Vh * SITE_REALS; ++k) out_e[k] = in_e[k] - kappa * kappa * out_e[k];
    free(tmp);
}

/* Split a full field into its even and odd half fields. */
void orc_split(const int* L, const double* full, double* even, double* odd)
{
    long Vh = volume(L) / 2;
    for (long i = 0; i < Vh; ++i) {
        memcpy(even + i * SITE_REALS, full + site_of_half(L, i, 0) * SITE_REALS,
               sizeof(double) * SITE_REALS);
        memcpy(odd + i * SITE_REALS, full + site_of_half(L, i, 1) * SITE_REALS,
               sizeof(double) * SITE_REALS);
    }
}

/* Join even and odd half fields into a full field. */
void orc_join(const int* L, const double* even, const double* odd, double* full)
{
    long Vh = volume(L) / 2;
    for (long i = 0; i < Vh; ++i) {
        memcpy(full + site_of_half(L, i, 0) * SITE_REALS, even + i * SITE_REALS,
               sizeof(double) * SITE_REALS);
        memcpy(full + site_of_half(L, i, 1) * SITE_REALS, odd + i * SITE_REALS,
               sizeof(double) * SITE_REALS);
    }
}

/* ------------------------------------------------------------------ */
/* vector algebra on n complex numbers                                 */
/* ------------------------------------------------------------------ */

/* (a, b) = sum_i conj(a_i) b_i */
static void cdot(long n, const double* a, const double* b, double* re, double* im)
{
    double sr = 0.0, si = 0.0;
#pragma omp parallel for reduction(+ : sr, si) schedule(static)
    for (long i = 0; i < n; ++i) {
        sr += a[2 * i] * b[2 * i] + a[2 * i + 1] * b[2 * i + 1];
        si += a[2 * i] * b[2 * i + 1] - a[2 * i + 1] * b[2 * i];
    }
    *re = sr;
    *im = si;
}

static double norm2(long n, const double* a)
{
    double r, i;
    cdot(n, a, a, &r, &i);
    return r;
}

double orc_norm2(long n_complex, const double* a) { return norm2(n_complex, a); }

void orc_cdot(long n_complex, const double* a, const double* b, double* out /* re, im */)
{
    cdot(n_complex, a, b, out, out + 1);
}

/* ------------------------------------------------------------------ */
/* BiCGStab (van der Vorst 1992) on a generic linear operator          */
/* ------------------------------------------------------------------ */

typedef struct {
    const double* U;
    const int* L;
    const double* bc;
    double kappa;
    int eo; /* 0: full D, 1: M_ee */
    const double* F; /* clover term of Eq. 2, or NULL for the Wilson matrix */
} op_ctx;

void orc_clover_D_full(const double* U, const double* F, const double* in, double* out,
                       const int* L, const double* bc, double kappa, int d);
void orc_clover_Mee(const double* U, const double* F, const double* in_e, double* out_e,
                    const int* L, const double* bc, double kappa);

static void apply_op(const op_ctx* c, const double* in, double* out)
{
    if (c->F) {
        if (c->eo)
            orc_clover_Mee(c->U, c->F, in, out, c->L, c->bc, c->kappa);
        else
            orc_clover_D_full(c->U, c->F, in, out, c->L, c->bc, c->kappa, +1);
    } else if (c->eo) {
        orc_Mee(c->U, in, out, c->L, c->bc, c->kappa, +1);
    } else {
        orc_D_full(c->U, in, out, c->L, c->bc, c->kappa, +1);
    }
}

/* Solve A x = b until ||b - A x||_2 <= tol_abs (the recursively updated
 * residual).  Shadow residual rhat = r_0.  On a breakdown (rho = 0,
 * (rhat, v) = 0 or omega = 0) the iteration restarts from the current x with
 * rhat = r, at most 5 times.  Returns 0 on convergence, 1 when maxiter is
 * reached, 2 after too many breakdowns. */
static int bicgstab(const op_ctx* c, long n, const double* b, double* x, double tol_abs,
                    int maxiter, int* iters_out, int* restarts_out)
{
    size_t bytes = sizeof(double) * 2 * n;
    double* r = (double*)malloc(bytes);
    double* rh = (double*)malloc(bytes);
    double* p = (double*)malloc(bytes);
    double* v = (double*)malloc(bytes);
    double* s = (double*)malloc(bytes);
    double* t = (double*)malloc(bytes);
    int status = 1, iters = 0, restarts = 0;

    for (;;) { /* (re)start */
        apply_op(c, x, r);
        for (long k = 0; k < 2 * n; ++k) r[k] = b[k] - r[k];
        memcpy(rh, r, bytes);
        memset(p, 0, bytes);
        memset(v, 0, bytes);
        double rho_old[2] = {1, 0}, alpha[2] = {1, 0}, omega[2] = {1, 0};
        if (sqrt(norm2(n, r)) <= tol_abs) { status = 0; goto done; }
        int broke = 0;
        while (iters < maxiter) {
            double rho[2];
            cdot(n, rh, r, &rho[0], &rho[1]);
            if (rho[0] == 0.0 && rho[1] == 0.0) { broke = 1; break; }
            /* beta = (rho / rho_old) (alpha / omega) */
            double q1r, q1i, q2r, q2i, den;
            den = rho_old[0] * rho_old[0] + rho_old[1] * rho_old[1];
            q1r = (rho[0] * rho_old[0] + rho[1] * rho_old[1]) / den;
            q1i = (rho[1] * rho_old[0] - rho[0] * rho_old[1]) / den;
            den = omega[0] * omega[0] + omega[1] * omega[1];
            q2r = (alpha[0] * omega[0] + alpha[1] * omega[1]) / den;
            q2i = (alpha[1] * omega[0] - alpha[0] * omega[1]) / den;
            double beta[2] = {q1r * q2r - q1i * q2i, q1r * q2i + q1i * q2r};
            /* p = r + beta (p - omega v) */
            for (long k = 0; k < n; ++k) {
                double tr = p[2 * k] - (omega[0] * v[2 * k] - omega[1] * v[2 * k + 1]);
                double ti = p[2 * k + 1] - (omega[0] * v[2 * k + 1] + omega[1] * v[2 * k]);
                p[2 * k] = r[2 * k] + beta[0] * tr - beta[1] * ti;
                p[2 * k + 1] = r[2 * k + 1] + beta[0] * ti + beta[1] * tr;
            }
            apply_op(c, p, v);
            double rv[2];
            cdot(n, rh, v, &rv[0], &rv[1]);
            double rvabs = sqrt(rv[0] * rv[0] + rv[1] * rv[1]);
            if (rvabs < 1e-30 * sqrt(norm2(n, rh)) * sqrt(norm2(n, v))) { broke = 1; break; }
            den = rv[0] * rv[0] + rv[1] * rv[1];
            alpha[0] = (rho[0] * rv[0] + rho[1] * rv[1]) / den;
            alpha[1] = (rho[1] * rv[0] - rho[0] * rv[1]) / den;
            /* s = r - alpha v */
            for (long k = 0; k < n; ++k) {
                s[2 * k] = r[2 * k] - (alpha[0] * v[2 * k] - alpha[1] * v[2 * k + 1]);
                s[2 * k + 1] = r[2 * k + 1] - (alpha[0] * v[2 * k + 1] + alpha[1] * v[2 * k]);
            }
            ++iters;
            if (sqrt(norm2(n, s)) <= tol_abs) { /* x += alpha p, r = s */
                for (long k = 0; k < n; ++k) {
                    x[2 * k] += alpha[0] * p[2 * k] - alpha[1] * p[2 * k + 1];
                    x[2 * k + 1] += alpha[0] * p[2 * k + 1] + alpha[1] * p[2 * k];
                }
                status = 0;
                goto done;
            }
            apply_op(c, s, t);
            double ts[2];
            cdot(n, t, s, &ts[0], &ts[1]);
            double tt = norm2(n, t);
            if (tt == 0.0) { broke = 1; break; }
            omega[0] = ts[0] / tt;
            omega[1] = ts[1] / tt;
            /* x += alpha p + omega s ;  r = s - omega t */
            for (long k = 0; k < n; ++k) {
                x[2 * k] += alpha[0] * p[2 * k] - alpha[1] * p[2 * k + 1]
                          + omega[0] * s[2 * k] - omega[1] * s[2 * k + 1];
                x[2 * k + 1] += alpha[0] * p[2 * k + 1] + alpha[1] * p[2 * k]
                              + omega[0] * s[2 * k + 1] + omega[1] * s[2 * k];
                r[2 * k] = s[2 * k] - (omega[0] * t[2 * k] - omega[1] * t[2 * k + 1]);
                r[2 * k + 1] = s[2 * k + 1] - (omega[0] * t[2 * k + 1] + omega[1] * t[2 * k]);
            }
            if (sqrt(norm2(n, r)) <= tol_abs) { status = 0; goto done; }
            if (omega[0] == 0.0 && omega[1] == 0.0) { broke = 1; break; }
            rho_old[0] = rho[0];
            rho_old[1] = rho[1];
        }
        if (!broke) { status = 1; goto done; }
        if (++restarts > 5) { status = 2; goto done; }
    }
done:
    *iters_out += iters;
    *restarts_out += restarts;
    free(r); free(rh); free(p); free(v); free(s); free(t);
    return status;
}

/* ||b - D x||_2 / ||b||_2 on the full lattice (the convergence criterion). */
double orc_true_residual(const double* U, const double* b, const double* x, const int* L,
                         const double* bc, double kappa)
{
    long V = volume(L);
    double* r = (double*)malloc(sizeof(double) * V * SITE_REALS);
    orc_D_full(U, x, r, L, bc, kappa, +1);
    for (long k = 0; k < V * SITE_REALS; ++k) r[k] = b[k] - r[k];
    double rr = norm2(V * NS * NC, r), bb = norm2(V * NS * NC, b);
    free(r);
    return sqrt(rr / bb);
}

/* Solve D x = b (full lattice, canonical layout) to a true relative residual
 * ||b - D x|| / ||b|| <= tol.
 *   eo = 0: BiCGStab on D itself.
 *   eo = 1: even-odd Schur system.  b'_e = b_e + kappa H_eo b_o,
 *           M_ee x_e = b'_e, then x_o = b_o + kappa H_oe x_e.
 * x holds the initial guess on entry (zero for a cold start; for eo only its
 * even part is used).  info = {iterations, restarts, status, passes};
 * true_resid receives the final relative residual of the full system. */
int orc_solve(const double* U, const double* b, double* x, const int* L, const double* bc,
              double kappa, int eo, double tol, int maxiter, int* info, double* true_resid)
{
    long V = volume(L), Vh = V / 2;
    op_ctx c = {U, L, bc, kappa, eo, NULL};
    int iters = 0, restarts = 0, status = 1, passes = 0;
    double bnorm = sqrt(norm2(V * NS * NC, b));
    double target = tol * bnorm;
    double res = 1.0;
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * V * SITE_REALS);
        info[0] = info[1] = info[2] = info[3] = 0;
        *true_resid = 0.0;
        return 0;
    }
    if (!eo) {
        for (passes = 0; passes < 4; ++passes) {
            status = bicgstab(&c, V * NS * NC, b, x, target, maxiter - iters, &iters, &restarts);
            res = orc_true_residual(U, b, x, L, bc, kappa);
            if (res <= tol || status != 0) break;
            target *= 0.1; /* recursive residual drifted: tighten and resume */
        }
    } else {
        size_t hb = sizeof(double) * Vh * SITE_REALS;
        double* be = (double*)malloc(hb);
        double* bo = (double*)malloc(hb);
        double* xe = (double*)malloc(hb);
        double* xo = (double*)malloc(hb);
        double* tmp = (double*)malloc(hb);
        orc_split(L, b, be, bo);
        orc_split(L, x, xe, xo);
        orc_hop_eo(U, bo, tmp, L, bc, 0, +1); /* b'_e = b_e + kappa H_eo b_o */
        for (long k = 0; k < Vh * SITE_REALS; ++k) be[k] += kappa * tmp[k];
        for (passes = 0; passes < 4; ++passes) {
            status = bicgstab(&c, Vh * NS * NC, be, xe, target, maxiter - iters, &iters, &restarts);
            orc_hop_eo(U, xe, tmp, L, bc, 1, +1); /* x_o = b_o + kappa H_oe x_e */
            for (long k = 0; k < Vh * SITE_REALS; ++k) xo[k] = bo[k] + kappa * tmp[k];
            orc_join(L, xe, xo, x);
            res = orc_true_residual(U, b, x, L, bc, kappa);
            if (res <= tol || status != 0) break;
            target *= 0.1;
        }
        free(be); free(bo); free(xe); free(xo); free(tmp);
    }
    info[0] = iters;
    info[1] = restarts;
    info[2] = status;
    info[3] = passes + 1;
    *true_resid = res;
    return (res <= tol) ? 0 : (status ? status : 3);
}

/* Run exactly `niter` BiCGStab iterations on the chosen system from x = 0
 * (no convergence test).  Used to time a bounded sample of a solve whose
 * full length would take too long on the host. */
int orc_bicgstab_fixed(const double* U, const double* b_sys, double* x_sys, const int* L,
                       const double* bc, double kappa, int eo, int niter)
{
    long n = (eo ? volume(L) / 2 : volume(L)) * NS * NC;
    op_ctx c = {U, L, bc, kappa, eo, NULL};
    int iters = 0, restarts = 0;
    return bicgstab(&c, n, b_sys, x_sys, 0.0, niter, &iters, &restarts);
}

/* ------------------------------------------------------------------ */
/* clover term (Eq. 2)                                                 */
/* ------------------------------------------------------------------ */

/* Eq. 2, Sec. 2 "Clover Fermion Matrix": D_clov(x,y) = D_W(x,y) + F(x) delta_xy
 * with F(x) a 12x12 Hermitian matrix that, in a suitable basis, is block
 * diagonal with two 6x6 Hermitian blocks.  In the chiral basis used here the
 * blocks act on spins {0,1} and {2,3}: F[s][b][i][j] (complex) with
 * i, j = local_spin*3 + colour.  F is an input field, like U (the paper
 * ignores its construction).  The oracle expands it to a full 12x12 matrix
 * and multiplies it literally. */
#define CLOVER_REALS (2 * 2 * 6 * 6) /* two 6x6 complex blocks per site */

static void clover_matrix(const double* Fs, double M[12][12][2])
{
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) M[i][j][0] = M[i][j][1] = 0.0;
    for (int b = 0; b < 2; ++b)
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                M[6 * b + i][6 * b + j][0] = Fs[2 * ((b * 6 + i) * 6 + j)];
                M[6 * b + i][6 * b + j][1] = Fs[2 * ((b * 6 + i) * 6 + j) + 1];
            }
}

/* out_site += M v (12x12 complex times a 12-component site vector) */
static void add_matvec12(double M[12][12][2], const double* v, double* out_site)
{
    for (int i = 0; i < 12; ++i) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < 12; ++j) {
            re += M[i][j][0] * v[2 * j] - M[i][j][1] * v[2 * j + 1];
            im += M[i][j][0] * v[2 * j + 1] + M[i][j][1] * v[2 * j];
        }
        out_site[2 * i] += re;
        out_site[2 * i + 1] += im;
    }
}

/* out = D_clov in = D_W in + F in (Eq. 2 with D_W of Eq. 1).  F is
 * Hermitian, so the adjoint operator (d = -1) adds the same F. */
void orc_clover_D_full(const double* U, const double* F, const double* in, double* out,
                       const int* L, const double* bc, double kappa, int d)
{
    long V = volume(L);
    orc_D_full(U, in, out, L, bc, kappa, d);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; ++s) {
        double M[12][12][2];
        clover_matrix(F + s * CLOVER_REALS, M);
        add_matvec12(M, in + s * SITE_REALS, out + s * SITE_REALS);
    }
}

/* Solve the 12x12 complex system A y = v by Gaussian elimination with
 * partial pivoting (A = 1 + F(x) at one site). */
static void solve12(double A_in[12][12][2], const double* v, double* y)
{
    double A[12][13][2];
    for (int i = 0; i < 12; ++i) {
        for (int j = 0; j < 12; ++j) {
            A[i][j][0] = A_in[i][j][0];
            A[i][j][1] = A_in[i][j][1];
        }
        A[i][12][0] = v[2 * i];
        A[i][12][1] = v[2 * i + 1];
    }
    for (int c = 0; c < 12; ++c) {
        int piv = c;
        double best = A[c][c][0] * A[c][c][0] + A[c][c][1] * A[c][c][1];
        for (int r = c + 1; r < 12; ++r) {
            double m = A[r][c][0] * A[r][c][0] + A[r][c][1] * A[r][c][1];
            if (m > best) { best = m; piv = r; }
        }
        if (piv != c)
            for (int j = 0; j < 13; ++j) {
                double t0 = A[c][j][0], t1 = A[c][j][1];
                A[c][j][0] = A[piv][j][0];
                A[c][j][1] = A[piv][j][1];
                A[piv][j][0] = t0;
                A[piv][j][1] = t1;
            }
        for (int r = c + 1; r < 12; ++r) {
            /* f = A[r][c] / A[c][c] */
            double den = A[c][c][0] * A[c][c][0] + A[c][c][1] * A[c][c][1];
            double fr = (A[r][c][0] * A[c][c][0] + A[r][c][1] * A[c][c][1]) / den;
            double fi = (A[r][c][1] * A[c][c][0] - A[r][c][0] * A[c][c][1]) / den;
            for (int j = c; j < 13; ++j) {
                A[r][j][0] -= fr * A[c][j][0] - fi * A[c][j][1];
                A[r][j][1] -= fr * A[c][j][1] + fi * A[c][j][0];
            }
        }
    }
    for (int i = 11; i >= 0; --i) {
        double re = A[i][12][0], im = A[i][12][1];
        for (int j = i + 1; j < 12; ++j) {
            re -= A[i][j][0] * y[2 * j] - A[i][j][1] * y[2 * j + 1];
            im -= A[i][j][0] * y[2 * j + 1] + A[i][j][1] * y[2 * j];
        }
        double den = A[i][i][0] * A[i][i][0] + A[i][i][1] * A[i][i][1];
        y[2 * i] = (re * A[i][i][0] + im * A[i][i][1]) / den;
        y[2 * i + 1] = (im * A[i][i][0] - re * A[i][i][1]) / den;
    }
}

/* The site-diagonal part of D_clov on one parity: out = (1 + F) in
 * (inverse = 0) or out = (1 + F)^{-1} in (inverse = 1), half fields. */
void orc_clover_diag(const double* F, const double* in_half, double* out_half, const int* L,
                     int parity, int inverse)
{
    long Vh = volume(L) / 2;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < Vh; ++i) {
        long s = site_of_half(L, i, parity);
        double M[12][12][2];
        clover_matrix(F + s * CLOVER_REALS, M);
        for (int k = 0; k < 12; ++k) M[k][k][0] += 1.0;
        double* o = out_half + i * SITE_REALS;
        if (inverse) {
            solve12(M, in_half + i * SITE_REALS, o);
        } else {
            for (int k = 0; k < SITE_REALS; ++k) o[k] = 0.0;
            add_matvec12(M, in_half + i * SITE_REALS, o);
        }
    }
}

/* Schur complement of D_clov on the even sites:
 *   M_ee = A_ee - kappa^2 H_eo A_oo^{-1} H_oe,   A = 1 + F. */
void orc_clover_Mee(const double* U, const double* F, const double* in_e, double* out_e,
                    const int* L, const double* bc, double kappa)
{
    long Vh = volume(L) / 2;
    size_t hb = sizeof(double) * Vh * SITE_REALS;
    double* t1 = (double*)malloc(hb);
    double* t2 = (double*)malloc(hb);
    orc_hop_eo(U, in_e, t1, L, bc, 1, +1);   /* t1 = H_oe in       */
    orc_clover_diag(F, t1, t2, L, 1, 1);     /* t2 = A_oo^-1 t1    */
    orc_hop_eo(U, t2, t1, L, bc, 0, +1);     /* t1 = H_eo t2       */
    orc_clover_diag(F, in_e, out_e, L, 0, 0); /* out = A_ee in     */
    for (long k = 0; k < Vh * SITE_REALS; ++k) out_e[k] -= kappa * kappa * t1[k];
    free(t1);
    free(t2);
}

/* ------------------------------------------------------------------ */
/* clover solve (Eq. 2 inside the BiCGStab of Sec. 2)                  */
/* ------------------------------------------------------------------ */

/* ||b - D_clov x||_2 / ||b||_2 on the full lattice. */
double orc_clover_true_residual(const double* U, const double* F, const double* b,
                                const double* x, const int* L, const double* bc, double kappa)
{
    long V = volume(L);
    double* r = (double*)malloc(sizeof(double) * V * SITE_REALS);
    orc_clover_D_full(U, F, x, r, L, bc, kappa, +1);
    for (long k = 0; k < V * SITE_REALS; ++k) r[k] = b[k] - r[k];
    double rr = norm2(V * NS * NC, r), bb = norm2(V * NS * NC, b);
    free(r);
    return sqrt(rr / bb);
}

/* Solve D_clov x = b to a true relative residual <= tol.  With A = 1 + F:
 *   eo = 0: BiCGStab on D_clov itself;
 *   eo = 1: write D_clov in even/odd blocks [[A_ee, -k H_eo], [-k H_oe, A_oo]];
 *           eliminating x_o = A_oo^-1 (b_o + k H_oe x_e) leaves
 *           (A_ee - k^2 H_eo A_oo^-1 H_oe) x_e = b_e + k H_eo A_oo^-1 b_o.
 * Same conventions for x, info and true_resid as orc_solve. */
int orc_clover_solve(const double* U, const double* F, const double* b, double* x, const int* L,
                     const double* bc, double kappa, int eo, double tol, int maxiter, int* info,
                     double* true_resid)
{
    long V = volume(L), Vh = V / 2;
    op_ctx c = {U, L, bc, kappa, eo, F};
    int iters = 0, restarts = 0, status = 1, passes = 0;
    double bnorm = sqrt(norm2(V * NS * NC, b));
    double target = tol * bnorm;
    double res = 1.0;
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * V * SITE_REALS);
        info[0] = info[1] = info[2] = info[3] = 0;
        *true_resid = 0.0;
        return 0;
    }
    if (!eo) {
        for (passes = 0; passes < 4; ++passes) {
            status = bicgstab(&c, V * NS * NC, b, x, target, maxiter - iters, &iters, &restarts);
            res = orc_clover_true_residual(U, F, b, x, L, bc, kappa);
            if (res <= tol || status != 0) break;
            target *= 0.1;
        }
    } else {
        size_t hb = sizeof(double) * Vh * SITE_REALS;
        double* be = (double*)malloc(hb);
        double* bo = (double*)malloc(hb);
        double* xe = (double*)malloc(hb);
        double* xo = (double*)malloc(hb);
        double* t1 = (double*)malloc(hb);
        double* t2 = (double*)malloc(hb);
        orc_split(L, b, be, bo);
        orc_split(L, x, xe, xo);
        orc_clover_diag(F, bo, t1, L, 1, 1);  /* t1 = A_oo^-1 b_o       */
        orc_hop_eo(U, t1, t2, L, bc, 0, +1);  /* t2 = H_eo A_oo^-1 b_o  */
        for (long k = 0; k < Vh * SITE_REALS; ++k) be[k] += kappa * t2[k];
        for (passes = 0; passes < 4; ++passes) {
            status = bicgstab(&c, Vh * NS * NC, be, xe, target, maxiter - iters, &iters, &restarts);
            orc_hop_eo(U, xe, t1, L, bc, 1, +1); /* t1 = H_oe x_e */
            for (long k = 0; k < Vh * SITE_REALS; ++k) t1[k] = bo[k] + kappa * t1[k];
            orc_clover_diag(F, t1, xo, L, 1, 1); /* x_o = A_oo^-1 (b_o + k H_oe x_e) */
            orc_join(L, xe, xo, x);
            res = orc_clover_true_residual(U, F, b, x, L, bc, kappa);
            if (res <= tol || status != 0) break;
            target *= 0.1;
        }
        free(be); free(bo); free(xe); free(xo); free(t1); free(t2);
    }
    info[0] = iters;
    info[1] = restarts;
    info[2] = status;
    info[3] = passes + 1;
    *true_resid = res;
    return (res <= tol) ? 0 : (status ? status : 3);
}

/* orc_bicgstab_fixed for D_clov (eo = 0) or its Schur complement (eo = 1). */
int orc_clover_bicgstab_fixed(const double* U, const double* F, const double* b_sys, double* x_sys,
                              const int* L, const double* bc, double kappa, int eo, int niter)
{
    long n = (eo ? volume(L) / 2 : volume(L)) * NS * NC;
    op_ctx c = {U, L, bc, kappa, eo, F};
    int iters = 0, restarts = 0;
    return bicgstab(&c, n, b_sys, x_sys, 0.0, niter, &iters, &restarts);
}
