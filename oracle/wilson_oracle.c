/*
 * Plain FP64 CPU oracle for the Wilson-Dirac operator and its Krylov solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product (CUDA) path may link,
 * load or call this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or table with the CUDA
 * library.
 *
 * What it computes (the paper names the operator in its abstract and in
 * "Wilson inverter: Main features", and the even-odd preconditioned operator
 * 1 - kappa^2 D_eo D_oe in the caption of its Fig. 1, but prints no formula;
 * the readings below are the standard Wilson fermion with r = 1 in the
 * hopping-parameter normalisation):
 *
 *   D psi(x) = psi(x) - kappa * H psi(x)
 *   H psi(x) = sum_{mu=0..3} [ (1 - gamma_mu) U_mu(x)        psi(x + mu)
 *                            + (1 + gamma_mu) U_mu(x - mu)^+ psi(x - mu) ]
 *
 * with periodic boundaries in x, y, z and antiperiodic ones in t (every hop
 * that crosses the time boundary picks up a factor -1).  The adjoint hopping
 * term H^+ has the two projectors exchanged.  gamma_mu is the chiral
 * (DeGrand-Rossi type) basis built below from the Pauli matrices.
 *
 * The code is deliberately naive: full 4x4 spin matrices, full 3x3 links,
 * no half-spinor shortcut, no link compression, complex arithmetic from
 * <complex.h>.  Output sites are independent, so the only parallelism is an
 * OpenMP loop over output sites; all sums are taken in a fixed sequential
 * order, so results do not depend on the thread count.
 *
 * Canonical layouts (all row-major, complex double):
 *   spinor  psi[V][4][3]            site, spin, colour
 *   gauge   U[4][V][3][3]           direction, site, row, column
 *   site    i = x0 + L0*(x1 + L1*(x2 + L2*x3)),  x3 = time
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* gamma matrices                                                      */
/* ------------------------------------------------------------------ */

/* Pauli matrix sigma_k, k = 1, 2, 3. */
static void pauli(int k, cplx s[2][2])
{
    memset(s, 0, 4 * sizeof(cplx));
    if (k == 1) { s[0][1] = 1; s[1][0] = 1; }
    if (k == 2) { s[0][1] = -I; s[1][0] = I; }
    if (k == 3) { s[0][0] = 1; s[1][1] = -1; }
}

/*
 * Euclidean gamma matrices, chiral basis:
 *   gamma_mu = [[0, -i sigma_k], [i sigma_k, 0]],  mu = 0, 1, 2  <->  k = 1, 2, 3
 *   gamma_3  = [[0, 1], [1, 0]]                    (time)
 *   gamma_5  = gamma_0 gamma_1 gamma_2 gamma_3     (index 4)
 * g is written row-major, 4x4.
 */
void oracle_gamma(int mu, cplx *g)
{
    memset(g, 0, 16 * sizeof(cplx));
    if (mu >= 0 && mu <= 2) {
        cplx s[2][2];
        pauli(mu + 1, s);
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                g[a * 4 + (b + 2)] = -I * s[a][b];
                g[(a + 2) * 4 + b] = I * s[a][b];
            }
    } else if (mu == 3) {
        for (int a = 0; a < 2; a++) {
            g[a * 4 + (a + 2)] = 1;
            g[(a + 2) * 4 + a] = 1;
        }
    } else if (mu == 4) {
        cplx acc[16], tmp[16], gm[16];
        oracle_gamma(0, acc);
        for (int m = 1; m < 4; m++) {
            oracle_gamma(m, gm);
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++) {
                    cplx s = 0;
                    for (int c = 0; c < 4; c++) s += acc[a * 4 + c] * gm[c * 4 + b];
                    tmp[a * 4 + b] = s;
                }
            memcpy(acc, tmp, sizeof(acc));
        }
        memcpy(g, acc, sizeof(acc));
    }
}

/* ------------------------------------------------------------------ */
/* lattice geometry                                                    */
/* ------------------------------------------------------------------ */

static long lex_index(const int L[4], const int x[4])
{
    return x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
}

static void lex_coords(const int L[4], long i, int x[4])
{
    for (int m = 0; m < 4; m++) {
        x[m] = (int)(i % L[m]);
        i /= L[m];
    }
}

/*
 * Site x + dir*mu_hat (dir = +1 or -1) with periodic wrap.  *bc receives the
 * boundary factor of the hop: -1 when it crosses the time boundary (between
 * t = L3-1 and t = 0, either way), +1 otherwise.
 */
static long hop_site(const int L[4], const int x[4], int mu, int dir, double *bc)
{
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] += dir;
    *bc = 1.0;
    if (y[mu] >= L[mu]) { y[mu] -= L[mu]; if (mu == 3) *bc = -1.0; }
    if (y[mu] < 0)      { y[mu] += L[mu]; if (mu == 3) *bc = -1.0; }
    return lex_index(L, y);
}

/* ------------------------------------------------------------------ */
/* hopping term                                                        */
/* ------------------------------------------------------------------ */

/*
 * out_site[4][3] = H psi (x)  (dagger = 0)  or  H^+ psi (x)  (dagger = 1),
 * for one site x, straight from the definition above: for each direction,
 * transport the neighbour spinor with the link (colour), then multiply by the
 * full 4x4 matrix (1 -/+ gamma_mu) (spin), then add.
 */
static void hop_one_site(cplx out_site[4][3], const cplx *psi, const cplx *U,
                         const int L[4], long V, long i, int dagger,
                         const cplx gam[4][16])
{
    int x[4];
    lex_coords(L, i, x);
    double s = dagger ? -1.0 : 1.0;
    for (int a = 0; a < 4; a++)
        for (int c = 0; c < 3; c++) out_site[a][c] = 0;

    for (int mu = 0; mu < 4; mu++) {
        for (int dir = +1; dir >= -1; dir -= 2) {
            double bc;
            long y = hop_site(L, x, mu, dir, &bc);
            const cplx *py = psi + y * 12;
            cplx t[4][3];
            if (dir > 0) {
                /* U_mu(x) psi(x + mu) */
                const cplx *u = U + ((long)mu * V + i) * 9;
                for (int a = 0; a < 4; a++)
                    for (int c = 0; c < 3; c++) {
                        cplx acc = 0;
                        for (int d = 0; d < 3; d++) acc += u[c * 3 + d] * py[a * 3 + d];
                        t[a][c] = acc;
                    }
            } else {
                /* U_mu(x - mu)^+ psi(x - mu) */
                const cplx *u = U + ((long)mu * V + y) * 9;
                for (int a = 0; a < 4; a++)
                    for (int c = 0; c < 3; c++) {
                        cplx acc = 0;
                        for (int d = 0; d < 3; d++) acc += conj(u[d * 3 + c]) * py[a * 3 + d];
                        t[a][c] = acc;
                    }
            }
            /* spin projector: (1 - s gamma_mu) forward, (1 + s gamma_mu) backward */
            double sg = (dir > 0) ? -s : s;
            for (int a = 0; a < 4; a++)
                for (int c = 0; c < 3; c++) {
                    cplx acc = t[a][c];
                    for (int b = 0; b < 4; b++) acc += sg * gam[mu][a * 4 + b] * t[b][c];
                    out_site[a][c] += bc * acc;
                }
        }
    }
}

static void load_gammas(cplx gam[4][16])
{
    for (int mu = 0; mu < 4; mu++) oracle_gamma(mu, gam[mu]);
}

static long vol(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

/*
 * out = H psi (dagger = 0) or H^+ psi (dagger = 1) on the full lattice.
 * out_parity = 0 or 1 computes only the sites of that parity (the others are
 * set to zero); out_parity = -1 computes every site.  The input is read on
 * every site as given; to apply an even-odd block, zero the other parity of
 * the input first.
 */
void oracle_hop(cplx *out, const cplx *psi, const cplx *U, const int L[4],
                int dagger, int out_parity)
{
    long V = vol(L);
    cplx gam[4][16];
    load_gammas(gam);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; i++) {
        int x[4];
        lex_coords(L, i, x);
        int par = (x[0] + x[1] + x[2] + x[3]) & 1;
        cplx (*o)[3] = (cplx (*)[3])(out + i * 12);
        if (out_parity >= 0 && par != out_parity) {
            for (int k = 0; k < 12; k++) out[i * 12 + k] = 0;
            continue;
        }
        hop_one_site(o, psi, U, L, V, i, dagger, gam);
    }
}

/* H psi (or H^+ psi) at a list of sites only: out[n][4][3]. */
void oracle_hop_sites(cplx *out, const cplx *psi, const cplx *U, const int L[4],
                      int dagger, const long *sites, long n)
{
    long V = vol(L);
    cplx gam[4][16];
    load_gammas(gam);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; k++)
        hop_one_site((cplx (*)[3])(out + k * 12), psi, U, L, V, sites[k], dagger, gam);
}

/* out = psi - kappa * H psi   (dagger = 1: out = psi - kappa * H^+ psi = D^+ psi) */
void oracle_apply_D(cplx *out, const cplx *psi, const cplx *U, const int L[4],
                    double kappa, int dagger)
{
    long V = vol(L);
    oracle_hop(out, psi, U, L, dagger, -1);
    for (long k = 0; k < V * 12; k++) out[k] = psi[k] - kappa * out[k];
}

/* ------------------------------------------------------------------ */
/* conjugate gradient on the normal equations                          */
/* ------------------------------------------------------------------ */

static double norm2(const cplx *a, long n)
{
    double s = 0;
    for (long k = 0; k < n; k++) s += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
    return s;
}

static cplx dotc(const cplx *a, const cplx *b, long n)
{
    cplx s = 0;
    for (long k = 0; k < n; k++) s += conj(a[k]) * b[k];
    return s;
}

/*
 * Solve D x = b by the textbook conjugate gradient method (Hestenes and
 * Stiefel) applied to the normal equations D^+ D x = D^+ b.  The paper's
 * solver is a conjugate gradient on the operator and its adjoint (section
 * "Wilson inverter: Main features"); the normal-equation form is the reading
 * used here.  x holds the initial guess on entry.  Stops when the true
 * residual ||b - D x|| / ||b|| <= tol (checked every iteration with a fresh
 * application of D) or after maxiter iterations.
 * Returns 0 on convergence, 1 otherwise; *iters and *relres report the final
 * state.
 */
int oracle_cgnr(cplx *x, const cplx *b, const cplx *U, const int L[4],
                double kappa, double tol, int maxiter, int *iters, double *relres)
{
    long n = vol(L) * 12;
    cplx *r = malloc(n * sizeof(cplx));
    cplx *p = malloc(n * sizeof(cplx));
    cplx *t = malloc(n * sizeof(cplx));
    cplx *Ap = malloc(n * sizeof(cplx));
    cplx *res = malloc(n * sizeof(cplx));
    double bnorm = sqrt(norm2(b, n));
    int status = 1, k = 0;
    double rel = 0;

    /* residual of the normal equations: r = D^+ (b - D x) */
    oracle_apply_D(t, x, U, L, kappa, 0);
    for (long j = 0; j < n; j++) res[j] = b[j] - t[j];
    rel = (bnorm > 0) ? sqrt(norm2(res, n)) / bnorm : 0;
    oracle_apply_D(r, res, U, L, kappa, 1);
    memcpy(p, r, n * sizeof(cplx));
    double rr = norm2(r, n);

    for (k = 0; k < maxiter && rel > tol; k++) {
        oracle_apply_D(t, p, U, L, kappa, 0);        /* t  = D p */
        oracle_apply_D(Ap, t, U, L, kappa, 1);       /* Ap = D^+ D p */
        double pAp = creal(dotc(p, Ap, n));
        if (!(pAp > 0)) break;                       /* breakdown */
        double alpha = rr / pAp;
        for (long j = 0; j < n; j++) {
            x[j] += alpha * p[j];
            r[j] -= alpha * Ap[j];
        }
        double rr_new = norm2(r, n);
        double beta = rr_new / rr;
        rr = rr_new;
        for (long j = 0; j < n; j++) p[j] = r[j] + beta * p[j];

        oracle_apply_D(t, x, U, L, kappa, 0);
        for (long j = 0; j < n; j++) res[j] = b[j] - t[j];
        rel = sqrt(norm2(res, n)) / bnorm;
    }
    if (rel <= tol) status = 0;
    *iters = k;
    *relres = rel;
    free(r); free(p); free(t); free(Ap); free(res);
    return status;
}

/* ------------------------------------------------------------------ */
/* threads                                                             */
/* ------------------------------------------------------------------ */

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
