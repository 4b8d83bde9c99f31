/*
 * Plain FP64 CPU oracle for the asqtad even-odd CG, and for the NPR
 * four-fermion operator of Sec. 2, Eq. 1 (at the end of this file).
 * TEST INFRASTRUCTURE ONLY:
 * the tests, the smoke check and the benchmark's CPU-baseline leg call it; the
 * GPU library never does, and the two share no code.
 *
 * What it computes (the paper, "Code Optimization on Kepler GPUs and Xeon
 * Phi", Sec. 2 and Fig. 1, names the workload -- a mixed-precision CG inverter
 * for asqtad staggered quarks on a 20^3 x 64 lattice -- but prints none of the
 * operators; each definition below is the standard staggered one, written out
 * site by site with explicit coordinates):
 *
 *   staggered phases   eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y),
 *                      eta_3 = (-1)^(x+y+z)
 *   asqtad Dslash      (D psi)(x) = 1/2 sum_mu eta_mu(x) [ F_mu(x) psi(x+mu)
 *                        - F_mu(x-mu)^dag psi(x-mu) + L_mu(x) psi(x+3mu)
 *                        - L_mu(x-3mu)^dag psi(x-3mu) ]
 *                      with fat links F and long (Naik) links L that already
 *                      carry the coefficients c1 and c3;
 *   normal operator    A = M^dag M restricted to even sites = m^2 - D_eo D_oe
 *                      (M = m + D, D anti-Hermitian);
 *   CG                 Hestenes-Stiefel conjugate gradients on A x = b;
 *   multi-shift CG     Jegerlehner's shifted recurrences (hep-lat/9612014)
 *                      for (A + sigma_i) x_i = b sharing one Krylov space;
 *   int16 quantiser    the 16-bit storage format's codes, decided in FP32.
 *
 * Boundary conditions: periodic in every direction; t_sign = -1 makes a hop
 * that wraps around the t direction pick up a factor -1 (antiperiodic time).
 *
 * Arrays: links [site_lex][mu][row][col] complex (interleaved re, im);
 * colour vectors on the full lattice [site_lex][colour] complex, with
 * site_lex = x + Lx*(y + Ly*(z + Lz*t)).  Parity-half vectors are embedded in
 * full-lattice arrays (entries of the other parity are ignored on input).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------------------------------------------------------------- lattice */

void oracle_coords(const int L[4], long s, int c[4])
{
    c[0] = (int)(s % L[0]); s /= L[0];
    c[1] = (int)(s % L[1]); s /= L[1];
    c[2] = (int)(s % L[2]); s /= L[2];
    c[3] = (int)s;
}

long oracle_lex(const int L[4], const int c[4])
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

long oracle_volume(const int L[4])
{
    return (long)L[0] * L[1] * L[2] * L[3];
}

int oracle_parity(const int L[4], long s)
{
    int c[4];
    oracle_coords(L, s, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) */
int oracle_eta(const int L[4], long s, int mu)
{
    int c[4], sum = 0;
    oracle_coords(L, s, c);
    for (int nu = 0; nu < mu; nu++) sum += c[nu];
    return (sum & 1) ? -1 : 1;
}

static int floor_div(int a, int b)
{
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

/* site x + d*mu_hat (periodic); *sign gets t_sign^(number of wraps in t) */
long oracle_neighbor(const int L[4], long s, int mu, int d, int t_sign, int *sign)
{
    int c[4];
    oracle_coords(L, s, c);
    int raw = c[mu] + d;
    int wraps = floor_div(raw, L[mu]);
    c[mu] = raw - wraps * L[mu];
    int sg = 1;
    if (mu == 3 && t_sign < 0 && (wraps & 1)) sg = -1;
    if (sign) *sign = sg;
    return oracle_lex(L, c);
}

/* ----------------------------------------------------------- SU(3) algebra */

static const cplx *link_at(const double *u, long s, int mu)
{
    return (const cplx *)(u + ((s * 4 + mu) * 9) * 2);
}

static const cplx *vec_at(const double *v, long s) { return (const cplx *)(v + s * 6); }
static cplx *vec_mut(double *v, long s) { return (cplx *)(v + s * 6); }

/* y += a * W v */
static void add_mat_vec(cplx y[3], double a, const cplx *w, const cplx *v)
{
    for (int r = 0; r < 3; r++) {
        cplx t = 0;
        for (int c = 0; c < 3; c++) t += w[3 * r + c] * v[c];
        y[r] += a * t;
    }
}

/* y += a * W^dag v */
static void add_dag_mat_vec(cplx y[3], double a, const cplx *w, const cplx *v)
{
    for (int r = 0; r < 3; r++) {
        cplx t = 0;
        for (int c = 0; c < 3; c++) t += conj(w[3 * c + r]) * v[c];
        y[r] += a * t;
    }
}

/* ----------------------------------------------------------------- Dslash */

static void dslash_site(const int L[4], const double *fat, const double *lng,
                        int t_sign, const double *in, long s, cplx out[3])
{
    cplx acc[3] = {0, 0, 0};
    for (int mu = 0; mu < 4; mu++) {
        double eta = (double)oracle_eta(L, s, mu);
        int sg;
        long n;
        /* + F_mu(x) psi(x+mu) */
        n = oracle_neighbor(L, s, mu, +1, t_sign, &sg);
        add_mat_vec(acc, eta * sg, link_at(fat, s, mu), vec_at(in, n));
        /* - F_mu(x-mu)^dag psi(x-mu) */
        n = oracle_neighbor(L, s, mu, -1, t_sign, &sg);
        add_dag_mat_vec(acc, -eta * sg, link_at(fat, n, mu), vec_at(in, n));
        /* + L_mu(x) psi(x+3mu) */
        n = oracle_neighbor(L, s, mu, +3, t_sign, &sg);
        add_mat_vec(acc, eta * sg, link_at(lng, s, mu), vec_at(in, n));
        /* - L_mu(x-3mu)^dag psi(x-3mu) */
        n = oracle_neighbor(L, s, mu, -3, t_sign, &sg);
        add_dag_mat_vec(acc, -eta * sg, link_at(lng, n, mu), vec_at(in, n));
    }
    for (int c = 0; c < 3; c++) out[c] = 0.5 * acc[c];
}

/* out(x) = (D in)(x) for every x of parity out_parity (0/1), or every x (-1).
 * Entries of out at the other parity are left untouched. */
void oracle_dslash(const int L[4], const double *fat, const double *lng, int t_sign,
                   int out_parity, const double *in, double *out)
{
    long vol = oracle_volume(L);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < vol; s++) {
        if (out_parity >= 0 && oracle_parity(L, s) != out_parity) continue;
        cplx r[3];
        dslash_site(L, fat, lng, t_sign, in, s, r);
        cplx *o = vec_mut(out, s);
        for (int c = 0; c < 3; c++) o[c] = r[c];
    }
}

/* one output site of D (for sampled checks on large lattices) */
void oracle_dslash_site(const int L[4], const double *fat, const double *lng, int t_sign,
                        long s, const double *in, double *out3)
{
    cplx r[3];
    dslash_site(L, fat, lng, t_sign, in, s, r);
    memcpy(out3, r, sizeof(r));
}

/* ------------------------------------------------------- even-site vectors */

static double re_dot_even(const int L[4], const double *a, const double *b)
{
    long vol = oracle_volume(L);
    double sum = 0;
    for (long s = 0; s < vol; s++) {
        if (oracle_parity(L, s) != 0) continue;
        for (int k = 0; k < 6; k++) sum += a[s * 6 + k] * b[s * 6 + k];
    }
    return sum;
}

/* y = a*x + y on even sites */
static void axpy_even(const int L[4], double a, const double *x, double *y)
{
    long vol = oracle_volume(L);
    for (long s = 0; s < vol; s++) {
        if (oracle_parity(L, s) != 0) continue;
        for (int k = 0; k < 6; k++) y[s * 6 + k] += a * x[s * 6 + k];
    }
}

/* y = x + b*y on even sites */
static void xpby_even(const int L[4], const double *x, double b, double *y)
{
    long vol = oracle_volume(L);
    for (long s = 0; s < vol; s++) {
        if (oracle_parity(L, s) != 0) continue;
        for (int k = 0; k < 6; k++) y[s * 6 + k] = x[s * 6 + k] + b * y[s * 6 + k];
    }
}

static void copy_even(const int L[4], const double *x, double *y)
{
    long vol = oracle_volume(L);
    for (long s = 0; s < vol; s++) {
        if (oracle_parity(L, s) != 0) continue;
        for (int k = 0; k < 6; k++) y[s * 6 + k] = x[s * 6 + k];
    }
}

/* A p = m^2 p - D_eo (D_oe p) on even sites; odd entries of out are zeroed.
 * tmp: full-lattice scratch (its odd entries receive D_oe p). */
void oracle_mdagm(const int L[4], const double *fat, const double *lng, int t_sign,
                  double mass, const double *p, double *out, double *tmp)
{
    long vol = oracle_volume(L);
    oracle_dslash(L, fat, lng, t_sign, 1, p, tmp);      /* tmp_o = D_oe p_e */
    oracle_dslash(L, fat, lng, t_sign, 0, tmp, out);    /* out_e = D_eo tmp_o */
    double m2 = mass * mass;
    for (long s = 0; s < vol; s++) {
        if (oracle_parity(L, s) != 0) {
            for (int k = 0; k < 6; k++) out[s * 6 + k] = 0;
            continue;
        }
        for (int k = 0; k < 6; k++) out[s * 6 + k] = m2 * p[s * 6 + k] - out[s * 6 + k];
    }
}

/* relative true residual |b - A x| / |b| on even sites */
double oracle_true_residual(const int L[4], const double *fat, const double *lng, int t_sign,
                            double mass, const double *b, const double *x)
{
    long n = oracle_volume(L) * 6;
    double *ax = calloc(n, sizeof(double)), *tmp = calloc(n, sizeof(double));
    oracle_mdagm(L, fat, lng, t_sign, mass, x, ax, tmp);
    double rr = 0;
    long vol = oracle_volume(L);
    for (long s = 0; s < vol; s++) {
        if (oracle_parity(L, s) != 0) continue;
        for (int k = 0; k < 6; k++) {
            double d = b[s * 6 + k] - ax[s * 6 + k];
            rr += d * d;
        }
    }
    double b2 = re_dot_even(L, b, b);
    free(ax);
    free(tmp);
    return b2 > 0 ? sqrt(rr / b2) : sqrt(rr);
}

/* ------------------------------------------------------------------- CG */

/* Solve (m^2 - D_eo D_oe) x = b on even sites, x_0 = 0.
 * Stops when the recursive residual |r|/|b| <= tol and the recomputed true
 * residual |b - A x|/|b| <= tol.  If only the recursive one is below tol, r is
 * replaced by the true residual and p restarted from it.  Returns the
 * iteration count, or -1 when max_iter is reached or the recursion breaks
 * down (x and *true_res are still written). */
int oracle_cg(const int L[4], const double *fat, const double *lng, int t_sign, double mass,
              const double *b, double tol, int max_iter, double *x, double *true_res)
{
    long n = oracle_volume(L) * 6;
    double *r = calloc(n, sizeof(double)), *p = calloc(n, sizeof(double));
    double *ap = calloc(n, sizeof(double)), *tmp = calloc(n, sizeof(double));
    memset(x, 0, n * sizeof(double));
    copy_even(L, b, r);
    copy_even(L, b, p);
    double b2 = re_dot_even(L, b, b);
    double rr = b2;
    int iters = -1;
    if (b2 == 0) {
        iters = 0;
    } else {
        for (int k = 1; k <= max_iter; k++) {
            oracle_mdagm(L, fat, lng, t_sign, mass, p, ap, tmp);
            double pap = re_dot_even(L, p, ap);
            double alpha = rr / pap;
            axpy_even(L, alpha, p, x);
            axpy_even(L, -alpha, ap, r);
            double rr_new = re_dot_even(L, r, r);
            if (!isfinite(rr_new) || !(pap > 0)) break;
            if (sqrt(rr_new / b2) <= tol) {
                if (oracle_true_residual(L, fat, lng, t_sign, mass, b, x) <= tol) {
                    iters = k;
                    break;
                }
                /* the recursion drifted from the true residual: replace r by
                 * b - A x and restart the search direction from it */
                oracle_mdagm(L, fat, lng, t_sign, mass, x, ap, tmp);
                copy_even(L, b, r);
                axpy_even(L, -1.0, ap, r);
                rr = re_dot_even(L, r, r);
                copy_even(L, r, p);
                continue;
            }
            double beta = rr_new / rr;
            rr = rr_new;
            xpby_even(L, r, beta, p);
        }
    }
    if (true_res) *true_res = oracle_true_residual(L, fat, lng, t_sign, mass, b, x);
    free(r); free(p); free(ap); free(tmp);
    return iters;
}

/* Multi-shift CG: (m_i^2 - D_eo D_oe) x_i = b for i < nshift, one Krylov
 * space built on the smallest mass m_0 = min_i m_i, shifts
 * sigma_i = m_i^2 - m_0^2 >= 0.  Shifted residuals are collinear with the
 * base residual, r_i = zeta_i r, which gives (k = iteration, alpha_{-1} = 1,
 * beta_{-1} = 0, zeta_{-1} = zeta_0 = 1)
 *   zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1} /
 *                ( alpha_k beta_{k-1} (zeta_{k-1} - zeta_k)
 *                  + zeta_{k-1} alpha_{k-1} (1 + sigma alpha_k) )
 *   alpha^s_k = alpha_k zeta_{k+1} / zeta_k,  beta^s_k = beta_k (zeta_{k+1}/zeta_k)^2
 *   x^s += alpha^s_k p^s,  p^s = zeta_{k+1} r_{k+1} + beta^s_k p^s.
 * A shift stops updating once |zeta_i| |r| <= tol |b|.  x holds nshift
 * full-lattice fields.  Returns the base iteration count (-1: max_iter). */
int oracle_cg_multishift(const int L[4], const double *fat, const double *lng, int t_sign,
                         int nshift, const double *masses, const double *b, double tol,
                         int max_iter, double *x, double *true_res)
{
    long n = oracle_volume(L) * 6;
    int base = 0;
    for (int i = 1; i < nshift; i++) if (masses[i] < masses[base]) base = i;
    double m0 = masses[base];
    double *r = calloc(n, sizeof(double)), *ap = calloc(n, sizeof(double));
    double *tmp = calloc(n, sizeof(double)), *p = calloc(n * nshift, sizeof(double));
    double *sigma = calloc(nshift, sizeof(double)), *zeta = calloc(nshift, sizeof(double));
    double *zeta_prev = calloc(nshift, sizeof(double)), *zeta_next = calloc(nshift, sizeof(double));
    int *active = calloc(nshift, sizeof(int));
    memset(x, 0, n * nshift * sizeof(double));
    copy_even(L, b, r);
    for (int i = 0; i < nshift; i++) {
        copy_even(L, b, p + i * n);
        sigma[i] = masses[i] * masses[i] - m0 * m0;
        zeta[i] = zeta_prev[i] = 1.0;
        active[i] = 1;
    }
    double b2 = re_dot_even(L, b, b), rr = b2;
    double alpha_prev = 1.0, beta_prev = 0.0;
    int iters = -1;
    if (b2 == 0) iters = 0;
    for (int k = 0; iters < 0 && k < max_iter; k++) {
        double *pb = p + base * n;
        oracle_mdagm(L, fat, lng, t_sign, m0, pb, ap, tmp);
        double alpha = rr / re_dot_even(L, pb, ap);
        for (int i = 0; i < nshift; i++) {
            if (!active[i]) continue;
            double den = alpha * beta_prev * (zeta_prev[i] - zeta[i]) +
                         zeta_prev[i] * alpha_prev * (1.0 + sigma[i] * alpha);
            zeta_next[i] = zeta[i] * zeta_prev[i] * alpha_prev / den;
            axpy_even(L, alpha * zeta_next[i] / zeta[i], p + i * n, x + i * n);
        }
        axpy_even(L, -alpha, ap, r);
        double rr_new = re_dot_even(L, r, r);
        double beta = rr_new / rr;
        int any = 0;
        for (int i = 0; i < nshift; i++) {
            /* the base direction keeps driving the Krylov space while any
             * other shift is still active */
            if (!active[i] && i != base) continue;
            if (!active[i]) zeta_next[i] = 1.0;
            double ratio = zeta_next[i] / zeta[i];
            double *pi = p + i * n;
            /* p_i = zeta_next r + beta ratio^2 p_i */
            long vol = oracle_volume(L);
            for (long s = 0; s < vol; s++) {
                if (oracle_parity(L, s) != 0) continue;
                for (int q = 0; q < 6; q++)
                    pi[s * 6 + q] = zeta_next[i] * r[s * 6 + q] + beta * ratio * ratio * pi[s * 6 + q];
            }
            zeta_prev[i] = zeta[i];
            zeta[i] = zeta_next[i];
            if (active[i] && fabs(zeta[i]) * sqrt(rr_new / b2) <= tol) active[i] = 0;
            any |= active[i];
        }
        rr = rr_new;
        alpha_prev = alpha;
        beta_prev = beta;
        if (!any) iters = k + 1;
    }
    for (int i = 0; i < nshift; i++)
        if (true_res) true_res[i] = oracle_true_residual(L, fat, lng, t_sign, masses[i], b, x + i * n);
    free(r); free(ap); free(tmp); free(p); free(sigma); free(zeta); free(zeta_prev);
    free(zeta_next); free(active);
    return iters;
}

/* --------------------------------------------------------- int16 storage */

/* Spinor sites: 6 reals per site are rounded to FP32, the site norm
 * n = max_k |v_k| is taken in FP32 and each code is
 * q_k = rint(v_k * (32767 / n)) (FP32 multiply, round half to even),
 * saturated to [-32767, 32767].  A zero site gives n = 0 and zero codes. */
void oracle_quantize_spinor_i16(long nsites, const double *v, short *q, float *norm)
{
    for (long s = 0; s < nsites; s++) {
        float f[6], n = 0.0f;
        for (int k = 0; k < 6; k++) {
            f[k] = (float)v[s * 6 + k];
            float a = fabsf(f[k]);
            if (a > n) n = a;
        }
        norm[s] = n;
        if (n == 0.0f) {
            for (int k = 0; k < 6; k++) q[s * 6 + k] = 0;
            continue;
        }
        volatile float inv = 32767.0f / n;
        for (int k = 0; k < 6; k++) {
            volatile float u = f[k] * inv;
            float r = rintf(u);
            if (r > 32767.0f) r = 32767.0f;
            if (r < -32767.0f) r = -32767.0f;
            q[s * 6 + k] = (short)r;
        }
    }
}

/* Link elements with one global scale s (FP64 in, rounded to FP32):
 * q = rint(float(v) * (32767 / float(s))), saturated. */
void oracle_quantize_links_i16(long n, const double *v, double scale, short *q)
{
    float sf = (float)scale;
    volatile float inv = 32767.0f / sf;
    for (long k = 0; k < n; k++) {
        volatile float u = (float)v[k] * inv;
        float r = rintf(u);
        if (r > 32767.0f) r = 32767.0f;
        if (r < -32767.0f) r = -32767.0f;
        q[k] = (short)r;
    }
}

/* ------------------------------------------------------ fat and long links
 * The benchmark workloads' link recipe (the paper's lattices are MILC asqtad
 * ensembles, Sec. 2 and Fig. 1, which are not available here), applied to
 * thin links U:
 *   F_mu(x) = c1 [ U_mu(x) + w sum_{nu != mu} ( U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
 *                + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ) ] / (1 + 6w),
 *   L_mu(x) = c3 U_mu(x) U_mu(x+mu) U_mu(x+2mu).
 * Every neighbour is periodic; links carry no boundary sign. */

/* c = a b, a^dag b or a b^dag (3x3, row-major) */
static void mat_mul(cplx *c, const cplx *a, const cplx *b, int dag_a, int dag_b)
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx t = 0;
            for (int k = 0; k < 3; k++) {
                cplx x = dag_a ? conj(a[3 * k + i]) : a[3 * i + k];
                cplx y = dag_b ? conj(b[3 * j + k]) : b[3 * k + j];
                t += x * y;
            }
            c[3 * i + j] = t;
        }
}

void oracle_fat_long(const int L[4], const double *u, double c1, double c3, double w,
                     double *fat, double *lng)
{
    long vol = oracle_volume(L);
    #pragma omp parallel for schedule(static)
    for (long s = 0; s < vol; s++) {
        for (int mu = 0; mu < 4; mu++) {
            const cplx *umu = link_at(u, s, mu);
            long xpm = oracle_neighbor(L, s, mu, 1, 1, NULL);
            cplx staples[9] = {0}, t[9], t2[9];
            for (int nu = 0; nu < 4; nu++) {
                if (nu == mu) continue;
                /* up: U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag */
                long xpn = oracle_neighbor(L, s, nu, 1, 1, NULL);
                mat_mul(t, link_at(u, s, nu), link_at(u, xpn, mu), 0, 0);
                mat_mul(t2, t, link_at(u, xpm, nu), 0, 1);
                for (int e = 0; e < 9; e++) staples[e] += t2[e];
                /* down: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) */
                long xmn = oracle_neighbor(L, s, nu, -1, 1, NULL);
                long xmnpm = oracle_neighbor(L, xmn, mu, 1, 1, NULL);
                mat_mul(t, link_at(u, xmn, nu), link_at(u, xmn, mu), 1, 0);
                mat_mul(t2, t, link_at(u, xmnpm, nu), 0, 0);
                for (int e = 0; e < 9; e++) staples[e] += t2[e];
            }
            cplx *f = (cplx *)(fat + ((s * 4 + mu) * 9) * 2);
            for (int e = 0; e < 9; e++) f[e] = c1 * (umu[e] + w * staples[e]) / (1.0 + 6.0 * w);
            long xp2m = oracle_neighbor(L, s, mu, 2, 1, NULL);
            mat_mul(t, umu, link_at(u, xpm, mu), 0, 0);
            mat_mul(t2, t, link_at(u, xp2m, mu), 0, 0);
            cplx *l = (cplx *)(lng + ((s * 4 + mu) * 9) * 2);
            for (int e = 0; e < 9; e++) l[e] = c3 * t2[e];
        }
    }
}

/* ------------------------------------------------- asqtad fat links (MILC form)
 * The asqtad action's fat link, tree-level coefficients with the paths
 * oriented as below: one-link c1 = 5/8, 3-staple c3 = 1/16, 5-staple
 * c5 = 1/64, 7-staple c7 = 1/384, Lepage cL = -1/16 (unit links give
 * c1 + 6 c3 + 24 c5 + 48 c7 + 6 cL = 9/8); the Naik link is cN U U U with
 * cN = -1/24.  For direction mu, a staple of the mu-directed field W in
 * direction nu with sign s is
 *   s = +1:  U_nu(x) W(x+nu) U_nu(x+mu)^dag,
 *   s = -1:  U_nu(x-nu)^dag W(x-nu) U_nu(x-nu+mu),
 * and
 *   P3[nu,s]             = staple(U_mu; nu, s),
 *   P5[nu,s][rho,r]      = staple(P3[nu,s]; rho, r),          rho != mu, nu,
 *   P7[nu,s][rho,r][sg,q] = staple(P5[nu,s][rho,r]; sg, q),  sg != mu, nu, rho,
 *   Lepage[nu,s]         = staple(P3[nu,s]; nu, s),
 *   F_mu = c1 U_mu + c3 sum P3 + c5 sum P5 + c7 sum P7 + cL sum Lepage,
 * every sum over all directions and signs allowed.  Whole-lattice fields of
 * 3x3 matrices, built one staple at a time. */

static void staple_field(const int L[4], const double *u, int mu, int nu, int s,
                         const cplx *w, cplx *out)
{
    long vol = oracle_volume(L);
    #pragma omp parallel for schedule(static)
    for (long x = 0; x < vol; x++) {
        cplx t[9];
        if (s > 0) {
            long xpn = oracle_neighbor(L, x, nu, 1, 1, NULL);
            long xpm = oracle_neighbor(L, x, mu, 1, 1, NULL);
            mat_mul(t, link_at(u, x, nu), w + 9 * xpn, 0, 0);
            mat_mul(out + 9 * x, t, link_at(u, xpm, nu), 0, 1);
        } else {
            long xmn = oracle_neighbor(L, x, nu, -1, 1, NULL);
            long xmnpm = oracle_neighbor(L, xmn, mu, 1, 1, NULL);
            mat_mul(t, link_at(u, xmn, nu), w + 9 * xmn, 1, 0);
            mat_mul(out + 9 * x, t, link_at(u, xmnpm, nu), 0, 0);
        }
    }
}

static void add_field(long n, cplx *acc, double c, const cplx *a)
{
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < n; k++) acc[k] += c * a[k];
}

void oracle_asqtad_links(const int L[4], const double *u, const double coef[6], double *fat,
                         double *lng)
{
    const double c1 = coef[0], c3 = coef[1], c5 = coef[2], c7 = coef[3], cl = coef[4],
                 cn = coef[5];
    long vol = oracle_volume(L), n = 9 * vol;
    cplx *umu = malloc(sizeof(cplx) * n), *acc = malloc(sizeof(cplx) * n);
    cplx *p3 = malloc(sizeof(cplx) * n), *p5 = malloc(sizeof(cplx) * n);
    cplx *p7 = malloc(sizeof(cplx) * n), *lp = malloc(sizeof(cplx) * n);
    for (int mu = 0; mu < 4; mu++) {
        for (long x = 0; x < vol; x++)
            for (int e = 0; e < 9; e++) umu[9 * x + e] = link_at(u, x, mu)[e];
        for (long k = 0; k < n; k++) acc[k] = c1 * umu[k];
        for (int nu = 0; nu < 4; nu++) {
            if (nu == mu) continue;
            for (int s = -1; s <= 1; s += 2) {
                staple_field(L, u, mu, nu, s, umu, p3);
                add_field(n, acc, c3, p3);
                staple_field(L, u, mu, nu, s, p3, lp);
                add_field(n, acc, cl, lp);
                for (int rho = 0; rho < 4; rho++) {
                    if (rho == mu || rho == nu) continue;
                    for (int r = -1; r <= 1; r += 2) {
                        staple_field(L, u, mu, rho, r, p3, p5);
                        add_field(n, acc, c5, p5);
                        for (int sg = 0; sg < 4; sg++) {
                            if (sg == mu || sg == nu || sg == rho) continue;
                            for (int q = -1; q <= 1; q += 2) {
                                staple_field(L, u, mu, sg, q, p5, p7);
                                add_field(n, acc, c7, p7);
                            }
                        }
                    }
                }
            }
        }
        for (long x = 0; x < vol; x++) {
            cplx *f = (cplx *)(fat + ((x * 4 + mu) * 9) * 2);
            for (int e = 0; e < 9; e++) f[e] = acc[9 * x + e];
            cplx t[9];
            long xpm = oracle_neighbor(L, x, mu, 1, 1, NULL);
            long xp2m = oracle_neighbor(L, x, mu, 2, 1, NULL);
            mat_mul(t, link_at(u, x, mu), link_at(u, xpm, mu), 0, 0);
            cplx *l = (cplx *)(lng + ((x * 4 + mu) * 9) * 2);
            mat_mul(l, t, link_at(u, xp2m, mu), 0, 0);
            for (int e = 0; e < 9; e++) l[e] *= cn;
        }
    }
    free(umu); free(acc); free(p3); free(p5); free(p7); free(lp);
}

/*
 * ---- NPR one-colour four-fermion operator (Sec. 2, Eq. 1) ----
 *
 * Hypercube z (0 <= z_mu < L_mu / 2) has the 16 corner sites z_A = 2z + A,
 * A in {0,1}^4, indexed A = A_x + 2 A_y + 4 A_z + 8 A_t.
 *
 * Averaged link U_AD(z): the mean over the n! shortest paths inside the
 * hypercube from z_A to z_D (n = number of directions in which A and D
 * differ), each path the ordered product of its links; a step +mu from y
 * multiplies by U_mu(y), a step -mu by U_mu(y - mu)^dag.  U_AA = 1.
 *
 * Quark fields are propagator columns: chi^f_c(x) = G^f(x)[c][a] and
 * chibar^f_c(x) = conj(G^f(x)[c][a]), with a the source colour.  For one
 * operator with hypercube spin-taste matrices M1, M2 (16 x 16, input):
 *   O[a1][a2][a3][a4](z) = sum_{A,B,C,D} sum_{c1..c4}
 *       chibar^1_{c1}(z_A) M1[A][B] chi^2_{c2}(z_B)
 *     * chibar^3_{c3}(z_C) M2[C][D] chi^4_{c4}(z_D)
 *     * U_AD[c1][c4] * U_CB[c3][c2],
 * each chibar/chi taking the source colour a_f of its flavour f.
 *
 * Arrays: links as above; propagators [site_lex][c][a] complex; m1, m2
 * [op][A][B] complex; out [k][op][a1][a2][a3][a4] complex for the k-th
 * hypercube of zlist (hypercube index z_x + Hx (z_y + Hy (z_z + Hz z_t)),
 * H = L / 2), or of all hypercubes in order when zlist is NULL.
 */
static long corner_site(const int L[4], const int z[4], int a)
{
    int c[4];
    for (int mu = 0; mu < 4; mu++) c[mu] = 2 * z[mu] + ((a >> mu) & 1);
    return oracle_lex(L, c);
}

/* Adds the products of all shortest paths from corner x to corner d, each
 * pre-multiplied by prod (the path so far), to acc; counts them in *npaths. */
static void path_sum(const int L[4], const double *u, const int z[4], int x, int d,
                     const cplx *prod, cplx *acc, int *npaths)
{
    if (x == d) {
        for (int e = 0; e < 9; e++) acc[e] += prod[e];
        (*npaths)++;
        return;
    }
    for (int mu = 0; mu < 4; mu++) {
        if (!(((x ^ d) >> mu) & 1)) continue;
        int y = x ^ (1 << mu);
        cplx next[9];
        if (((x >> mu) & 1) == 0)     /* forward step: U_mu(z_x) */
            mat_mul(next, prod, link_at(u, corner_site(L, z, x), mu), 0, 0);
        else                          /* backward step: U_mu(z_y)^dag */
            mat_mul(next, prod, link_at(u, corner_site(L, z, y), mu), 0, 1);
        path_sum(L, u, z, y, d, next, acc, npaths);
    }
}

void oracle_npr_avg_link(const int L[4], const double *u, const int z[4], int a, int d,
                         double *out)
{
    cplx one[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    cplx acc[9] = {0};
    int npaths = 0;
    path_sum(L, u, z, a, d, one, acc, &npaths);
    cplx *o = (cplx *)out;
    for (int e = 0; e < 9; e++) o[e] = acc[e] / npaths;
}

void oracle_npr(const int L[4], const double *u, const double *g1, const double *g2,
                const double *g3, const double *g4, int nops, const double *m1,
                const double *m2, long nz, const long *zlist, double *out)
{
    const int H[4] = {L[0] / 2, L[1] / 2, L[2] / 2, L[3] / 2};
    #pragma omp parallel for schedule(dynamic)
    for (long k = 0; k < nz; k++) {
        long zi = zlist ? zlist[k] : k;
        int z[4];
        for (int mu = 0; mu < 4; mu++) {
            z[mu] = (int)(zi % H[mu]);
            zi /= H[mu];
        }
        cplx (*U)[16][9] = malloc(sizeof(cplx) * 16 * 16 * 9);
        const cplx *G[4][16];
        for (int a = 0; a < 16; a++) {
            long s = corner_site(L, z, a);
            G[0][a] = (const cplx *)(g1 + s * 18);
            G[1][a] = (const cplx *)(g2 + s * 18);
            G[2][a] = (const cplx *)(g3 + s * 18);
            G[3][a] = (const cplx *)(g4 + s * 18);
            for (int d = 0; d < 16; d++) oracle_npr_avg_link(L, u, z, a, d, (double *)U[a][d]);
        }
        for (int op = 0; op < nops; op++) {
            const cplx *M1 = (const cplx *)m1 + (long)op * 256;
            const cplx *M2 = (const cplx *)m2 + (long)op * 256;
            cplx *o = (cplx *)out + (k * nops + op) * 81;
            for (int e = 0; e < 81; e++) o[e] = 0;
            for (int A = 0; A < 16; A++)
            for (int B = 0; B < 16; B++) {
                cplx mab = M1[A * 16 + B];
                if (mab == 0) continue;
                for (int C = 0; C < 16; C++)
                for (int D = 0; D < 16; D++) {
                    cplx mcd = M2[C * 16 + D];
                    if (mcd == 0) continue;
                    for (int a1 = 0; a1 < 3; a1++)
                    for (int a2 = 0; a2 < 3; a2++)
                    for (int a3 = 0; a3 < 3; a3++)
                    for (int a4 = 0; a4 < 3; a4++) {
                        /* chibar^1(z_A) U_AD chi^4(z_D) */
                        cplx s14 = 0;
                        for (int c1 = 0; c1 < 3; c1++)
                            for (int c4 = 0; c4 < 3; c4++)
                                s14 += conj(G[0][A][3 * c1 + a1]) * U[A][D][3 * c1 + c4] *
                                       G[3][D][3 * c4 + a4];
                        /* chibar^3(z_C) U_CB chi^2(z_B) */
                        cplx s32 = 0;
                        for (int c3 = 0; c3 < 3; c3++)
                            for (int c2 = 0; c2 < 3; c2++)
                                s32 += conj(G[2][C][3 * c3 + a3]) * U[C][B][3 * c3 + c2] *
                                       G[1][B][3 * c2 + a2];
                        o[27 * a1 + 9 * a2 + 3 * a3 + a4] += mab * mcd * s14 * s32;
                    }
                }
            }
        }
        free(U);
    }
}
