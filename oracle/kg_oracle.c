/*
 * kg_oracle.c -- plain, slow, FP64 CPU oracle for the linear-scaling
 * Kubo-Greenwood method of Fan, Uppstu, Siro and Harju (arXiv 1307.0288).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code with
 * the CUDA path and is never called by it.
 *
 * Every routine follows one passage of the paper in the paper's order and
 * notation, one site and one term at a time, with no blocking, fusion or
 * reordering.  Complex vectors are arrays of (re, im) double pairs.  Dot
 * products use Neumaier-compensated summation so that the oracle's own
 * rounding error stays far below the parity tolerance.
 *
 * Readings of the paper that the code depends on (the paper is silent or
 * ambiguous there) are marked "Reading:" where they are used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_PI 3.14159265358979323846

/* Test hook: a non-zero value plants one deliberate mistake (see ora_set_mutation)
 * so the test-suite can show that its pins catch it.  Zero in normal use. */
static int g_mutation = 0;

void ora_set_mutation(int m) { g_mutation = m; }
int ora_get_mutation(void) { return g_mutation; }

/* ------------------------------------------------------------------ */
/* Lattice and Hamiltonian (Sec. 2, Eqs. 13-15)                        */
/* ------------------------------------------------------------------ */

/* Site (i, j): i in [0, nx) is the dimer-line index along x (zigzag direction),
 * j in [0, ny) the zigzag-chain index; site number n = j*nx + i.  Carbon
 * positions: x = i*sqrt(3)a/2, y = j*3a/2 + (a/2 when i+j is odd).  Sample
 * lengths L_x = sqrt(3) nx a/2, L_y = 3 ny a/2 (Sec. 2).
 *
 * kind 0: 2D sheet, periodic in x and y, transport along x.
 * kind 1: zigzag ribbon (ZGNR), periodic in x, open in y, transport along x.
 * kind 2: armchair ribbon (AGNR), periodic in y, open in x, transport along y.
 * kind 3: sheet open in x (the transport direction), periodic in y, transport along x.
 */
static void ora_position(int64_t i, int64_t j, double a, double* x, double* y) {
    *x = (double)i * sqrt(3.0) * a / 2.0;
    *y = (double)j * 1.5 * a + (((i + j) & 1) ? 0.5 * a : 0.0);
}

static double min_image(double d, double len, int periodic) {
    if (!periodic) return d;
    if (d > 0.5 * len) d -= len;
    if (d < -0.5 * len) d += len;
    return d;
}

/* Candidate bonds of site (i, j), found by distance: the three carbon sites at
 * bond length a (minimum-image distance where periodic).  Writes up to 3
 * neighbour site numbers into nb[] and returns how many there are. */
static int ora_bonded_sites(int kind, int64_t nx, int64_t ny, double a,
                            int64_t i, int64_t j, int64_t* nb) {
    const int px = (kind == 0 || kind == 1);
    const int py = (kind == 0 || kind == 2 || kind == 3);
    const double lx = sqrt(3.0) * (double)nx * a / 2.0, ly = 1.5 * (double)ny * a;
    double x0, y0;
    ora_position(i, j, a, &x0, &y0);
    int cnt = 0;
    /* Bonded atoms lie within one dimer line and one chain of (i, j). */
    for (int dj = -1; dj <= 1; dj++) {
        for (int di = -1; di <= 1; di++) {
            if (di == 0 && dj == 0) continue;
            int64_t ii = i + di, jj = j + dj;
            if (ii < 0 || ii >= nx) { if (!px) continue; ii = (ii + nx) % nx; }
            if (jj < 0 || jj >= ny) { if (!py) continue; jj = (jj + ny) % ny; }
            double x1, y1;
            ora_position(ii, jj, a, &x1, &y1);
            double dx = min_image(x1 - x0, lx, px), dy = min_image(y1 - y0, ly, py);
            double d = sqrt(dx * dx + dy * dy);
            if (fabs(d - a) < 1e-6 * a) {
                int64_t m = jj * nx + ii;
                int dup = 0;
                for (int q = 0; q < cnt; q++) dup |= (nb[q] == m);
                if (!dup && cnt < 3) nb[cnt++] = m;
            }
        }
    }
    return cnt;
}

/* Builds the scaled Hamiltonian H~ = H / E_max in CSR form.
 *   H = -gamma0 sum_<mn> |m><n| (Eq. 13) plus optional on-site energies eps_n;
 *   removed atoms (vac[n] != 0) keep an empty row and column (Sec. 2).
 * Outputs (caller-allocated): row_ptr[N+1], col[3N], val[3N] = H~_nm,
 * disp[3N] = X_n - X_m (minimum-image bond displacement along the transport
 * direction, nm), diag[N] = eps_n / E_max.  Returns the number of stored bonds.
 * Reading: under periodic boundaries X_n - X_m is the bond vector, not a
 * difference of wrapped coordinates, so [X, H] stays short-ranged. */
int64_t ora_build_hamiltonian(int kind, int64_t nx, int64_t ny, double a, double gamma0,
                              double emax, const uint8_t* vac, const double* onsite_ev,
                              int64_t* row_ptr, int64_t* col, double* val, double* disp,
                              double* diag) {
    const int px = (kind == 0 || kind == 1);
    const int py = (kind == 0 || kind == 2 || kind == 3);
    const double lx = sqrt(3.0) * (double)nx * a / 2.0, ly = 1.5 * (double)ny * a;
    const int64_t n_sites = nx * ny;
    int64_t nnz = 0;
    for (int64_t n = 0; n < n_sites; n++) {
        row_ptr[n] = nnz;
        const int64_t i = n % nx, j = n / nx;
        diag[n] = 0.0;
        if (vac && vac[n]) continue;
        if (onsite_ev) diag[n] = onsite_ev[n] / emax;
        int64_t nb[3];
        int cnt = ora_bonded_sites(kind, nx, ny, a, i, j, nb);
        double x0, y0;
        ora_position(i, j, a, &x0, &y0);
        for (int q = 0; q < cnt; q++) {
            int64_t m = nb[q];
            if (vac && vac[m]) continue;
            double x1, y1;
            ora_position(m % nx, m / nx, a, &x1, &y1);
            double dx = min_image(x1 - x0, lx, px), dy = min_image(y1 - y0, ly, py);
            double d_transport = (kind == 2) ? dy : dx;   /* X_m - X_n */
            col[nnz] = m;
            val[nnz] = -gamma0 / emax;
            disp[nnz] = -d_transport;                      /* X_n - X_m */
            nnz++;
        }
    }
    row_ptr[n_sites] = nnz;
    return nnz;
}

/* ------------------------------------------------------------------ */
/* Sparse products (Algorithm 8 and its [X, H] counterpart)            */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    const int64_t* row_ptr;
    const int64_t* col;
    const double* val;
    const double* disp;
    const double* diag;
} ora_h;

/* y = H~ x : y_n = diag_n x_n + sum_m H~_nm x_m (one row at a time, Algorithm 8). */
static void apply_h(const ora_h* h, const double* x, double* y) {
    for (int64_t n = 0; n < h->n; n++) {
        double re = h->diag[n] * x[2 * n], im = h->diag[n] * x[2 * n + 1];
        for (int64_t k = h->row_ptr[n]; k < h->row_ptr[n + 1]; k++) {
            int64_t m = h->col[k];
            re += h->val[k] * x[2 * m];
            im += h->val[k] * x[2 * m + 1];
        }
        y[2 * n] = re;
        y[2 * n + 1] = im;
    }
}

/* y = [X, H~] x : y_n = sum_m (X_n - X_m) H~_nm x_m  (Eq. 15 with H -> H~). */
static void apply_xh(const ora_h* h, const double* x, double* y) {
    for (int64_t n = 0; n < h->n; n++) {
        double re = 0.0, im = 0.0;
        for (int64_t k = h->row_ptr[n]; k < h->row_ptr[n + 1]; k++) {
            int64_t m = h->col[k];
            double c = h->disp[k] * h->val[k];
            if (g_mutation == 3) c = -c;               /* planted: transposed commutator */
            re += c * x[2 * m];
            im += c * x[2 * m + 1];
        }
        y[2 * n] = re;
        y[2 * n + 1] = im;
    }
}

void ora_apply_h(int64_t n, const int64_t* rp, const int64_t* col, const double* val,
                 const double* disp, const double* diag, const double* x, double* y) {
    ora_h h = {n, rp, col, val, disp, diag};
    apply_h(&h, x, y);
}

void ora_apply_xh(int64_t n, const int64_t* rp, const int64_t* col, const double* val,
                  const double* disp, const double* diag, const double* x, double* y) {
    ora_h h = {n, rp, col, val, disp, diag};
    apply_xh(&h, x, y);
}

/* ------------------------------------------------------------------ */
/* Compensated complex inner product <L|v> = sum_n conj(L_n) v_n       */
/* ------------------------------------------------------------------ */

static void neumaier_add(double* s, double* c, double t) {
    double u = *s + t;
    if (fabs(*s) >= fabs(t)) *c += (*s - u) + t;
    else *c += (t - u) + *s;
    *s = u;
}

static void dot(int64_t n, const double* l, const double* v, double* out_re, double* out_im) {
    double sr = 0, cr = 0, si = 0, ci = 0;
    for (int64_t k = 0; k < n; k++) {
        double lr = l[2 * k], li = l[2 * k + 1], vr = v[2 * k], vi = v[2 * k + 1];
        neumaier_add(&sr, &cr, lr * vr);
        neumaier_add(&sr, &cr, li * vi);
        if (g_mutation == 5) {                       /* planted: conjugated the wrong operand */
            neumaier_add(&si, &ci, li * vr);
            neumaier_add(&si, &ci, -lr * vi);
        } else {
            neumaier_add(&si, &ci, lr * vi);
            neumaier_add(&si, &ci, -li * vr);
        }
    }
    *out_re = sr + cr;
    *out_im = si + ci;
}

void ora_dot(int64_t n, const double* l, const double* v, double* out2) {
    dot(n, l, v, &out2[0], &out2[1]);
}

/* ------------------------------------------------------------------ */
/* Chebyshev moments C_n = <phi_L| T_n(H~) |phi_R>  (Algorithm 5, Eq. 46) */
/* ------------------------------------------------------------------ */

void ora_kpm_moments(int64_t n, const int64_t* rp, const int64_t* col, const double* val,
                     const double* disp, const double* diag, const double* phi_l,
                     const double* phi_r, int n_moments, double* c /* [M][2] */) {
    ora_h h = {n, rp, col, val, disp, diag};
    double* p0 = malloc(sizeof(double) * 2 * n);
    double* p1 = malloc(sizeof(double) * 2 * n);
    double* p2 = malloc(sizeof(double) * 2 * n);
    /* |phi_0> <- |phi_R>;  C_0 <- <phi_L|phi_0> */
    memcpy(p0, phi_r, sizeof(double) * 2 * n);
    if (n_moments > 0) dot(n, phi_l, p0, &c[0], &c[1]);
    /* |phi_1> <- H|phi_0>;  C_1 <- <phi_L|phi_1> */
    apply_h(&h, p0, p1);
    if (n_moments > 1) dot(n, phi_l, p1, &c[2], &c[3]);
    /* for n = 2 .. M-1: |phi_2> <- 2H|phi_1> - |phi_0>;  C_n <- <phi_L|phi_2> */
    for (int k = 2; k < n_moments; k++) {
        apply_h(&h, p1, p2);
        for (int64_t q = 0; q < 2 * n; q++) {
            p2[q] = 2.0 * p2[q] - (g_mutation == 1 ? 0.0 : p0[q]);   /* planted: dropped T_{n-2} */
        }
        dot(n, phi_l, p2, &c[2 * k], &c[2 * k + 1]);
        double* t = p0; p0 = p1; p1 = p2; p2 = t;
    }
    free(p0); free(p1); free(p2);
}

/* ------------------------------------------------------------------ */
/* Bessel functions J_m(x) of the first kind, m = 0..nmax              */
/* ------------------------------------------------------------------ */

/* Miller's backward recurrence: J_{m-1} = (2m/x) J_m - J_{m+1} (Abramowitz and
 * Stegun 9.1.27) run downward from a high order where the true values are
 * negligible, then normalised with J_0 + 2 sum_{k>=1} J_{2k} = 1 (A&S 9.1.46).
 * The starting order is well beyond both nmax and x, so every returned value
 * carries full relative accuracy. */
void ora_bessel_j(double x, int nmax, double* j_out) {
    for (int m = 0; m <= nmax; m++) j_out[m] = 0.0;
    if (x == 0.0) { j_out[0] = 1.0; return; }
    double ax = fabs(x);
    int top = (nmax > (int)ax ? nmax : (int)ax);
    int start = top + 40 + (int)sqrt(80.0 * (top + 1));
    if (start & 1) start++;
    double jp = 0.0, jc = 1e-300, norm = 0.0;   /* J_{start+1}, J_start (unnormalised) */
    for (int m = start; m >= 1; m--) {
        double jm = (2.0 * m / ax) * jc - jp;   /* J_{m-1} */
        jp = jc;
        jc = jm;
        int k = m - 1;
        if (k <= nmax) j_out[k] = jc;
        if (k > 0 && (k % 2) == 0) norm += 2.0 * jc;
        if (fabs(jc) > 1e250) {                 /* rescale to stay in range */
            jc *= 1e-250; jp *= 1e-250; norm *= 1e-250;
            for (int q = k; q <= nmax; q++) j_out[q] *= 1e-250;
        }
    }
    norm += jc;                                 /* + J_0 */
    for (int m = 0; m <= nmax; m++) {
        j_out[m] /= norm;
        if (x < 0 && (m & 1)) j_out[m] = -j_out[m];   /* J_m(-x) = (-1)^m J_m(x) */
    }
}

/* Number of terms N_p of the Chebyshev-Bessel series (Eqs. 36-37): the smallest
 * m greater than x with |J_m(x)| < tol, so the first omitted term is below tol.
 * (Sec. 4.2 quotes about 20 terms for x = pi at 1e-15.) */
int ora_bessel_terms(double x, double tol) {
    int nmax = (int)fabs(x) + 200;
    double* j = malloc(sizeof(double) * (nmax + 1));
    ora_bessel_j(x, nmax, j);
    int np = nmax;
    for (int m = 0; m <= nmax; m++) {
        if ((double)m > fabs(x) && fabs(j[m]) < tol) { np = m; break; }
    }
    free(j);
    return np;
}

/* ------------------------------------------------------------------ */
/* Time evolution (Sec. 3.1.3)                                         */
/* ------------------------------------------------------------------ */

/* (s i)^m for s = -1 or +1, as (re, im). */
static void ipow(int s, int m, double* re, double* im) {
    switch (m & 3) {
        case 0: *re = 1; *im = 0; break;
        case 1: *re = 0; *im = s; break;
        case 2: *re = -1; *im = 0; break;
        default: *re = 0; *im = -s; break;
    }
}

/* out += (cr + i ci) * v */
static void axpy_c(int64_t n, double cr, double ci, const double* v, double* out) {
    for (int64_t q = 0; q < n; q++) {
        double vr = v[2 * q], vi = v[2 * q + 1];
        out[2 * q] += cr * vr - ci * vi;
        out[2 * q + 1] += cr * vi + ci * vr;
    }
}

/* |out> = U(+-dt)|in> by the Chebyshev-Bessel series, Eq. (36), evaluated as in
 * Algorithm 6.  direction = +1 gives U(+dt) = exp(-i H~ tau) with factors (-i)^m;
 * direction = -1 gives U(-dt) = U(dt)^dagger with factors (+i)^m.  j[] holds
 * J_m(tau), m < np, tau = E_max dt / hbar. */
void ora_evolve(int64_t n, const int64_t* rp, const int64_t* col, const double* val,
                const double* disp, const double* diag, const double* jm, int np,
                int direction, const double* in, double* out) {
    ora_h h = {n, rp, col, val, disp, diag};
    const int s = (direction > 0) ? -1 : +1;   /* U(+dt): (-i)^m ; U(-dt): (+i)^m */
    double* p0 = malloc(sizeof(double) * 2 * n);
    double* p1 = malloc(sizeof(double) * 2 * n);
    double* p2 = malloc(sizeof(double) * 2 * n);
    double cr, ci;
    /* |phi_0> <- |in>;  |phi_1> <- H|phi_0> */
    memcpy(p0, in, sizeof(double) * 2 * n);
    apply_h(&h, p0, p1);
    /* |out> <- J_0 |phi_0> + 2 (-+i) J_1 |phi_1> */
    memset(out, 0, sizeof(double) * 2 * n);
    axpy_c(n, jm[0], 0.0, p0, out);
    if (np > 1) {
        ipow(s, 1, &cr, &ci);
        double f = (g_mutation == 2 ? 1.0 : 2.0) * jm[1];   /* planted: lost (2 - delta_m0) */
        axpy_c(n, f * cr, f * ci, p1, out);
    }
    for (int m = 2; m < np; m++) {
        /* |phi_2> <- 2H|phi_1> - |phi_0> */
        apply_h(&h, p1, p2);
        for (int64_t q = 0; q < 2 * n; q++) p2[q] = 2.0 * p2[q] - p0[q];
        /* |out> <- |out> + 2 (-+i)^m J_m |phi_2> */
        ipow(s, m, &cr, &ci);
        double f = 2.0 * jm[m];
        axpy_c(n, f * cr, f * ci, p2, out);
        double* t = p0; p0 = p1; p1 = p2; p2 = t;
    }
    free(p0); free(p1); free(p2);
}

/* |out> = [X, U(dt)]|in> by Eq. (37) with the commutator recursion Eqs. (39)
 * and (41), evaluated as in Algorithm 7. */
void ora_evolvex(int64_t n, const int64_t* rp, const int64_t* col, const double* val,
                 const double* disp, const double* diag, const double* jm, int np,
                 const double* in, double* out) {
    ora_h h = {n, rp, col, val, disp, diag};
    double* p0 = malloc(sizeof(double) * 2 * n);
    double* p1 = malloc(sizeof(double) * 2 * n);
    double* p2 = malloc(sizeof(double) * 2 * n);
    double* x0 = malloc(sizeof(double) * 2 * n);
    double* x1 = malloc(sizeof(double) * 2 * n);
    double* x2 = malloc(sizeof(double) * 2 * n);
    double* tmp = malloc(sizeof(double) * 2 * n);
    double cr, ci;
    /* |phi_0> <- |in>;  |phi_0^x> <- 0;  |phi_1> <- H|phi_0>;  |phi_1^x> <- [X,H]|in> */
    memcpy(p0, in, sizeof(double) * 2 * n);
    memset(x0, 0, sizeof(double) * 2 * n);
    apply_h(&h, p0, p1);
    apply_xh(&h, in, x1);
    /* |out> <- 2 (-i) J_1 |phi_1^x> */
    memset(out, 0, sizeof(double) * 2 * n);
    if (np > 1) {
        ipow(-1, 1, &cr, &ci);
        axpy_c(n, 2.0 * jm[1] * cr, 2.0 * jm[1] * ci, x1, out);
    }
    for (int m = 2; m < np; m++) {
        /* |phi_2> <- 2H|phi_1> - |phi_0> */
        apply_h(&h, p1, p2);
        for (int64_t q = 0; q < 2 * n; q++) p2[q] = 2.0 * p2[q] - p0[q];
        /* |phi_2^x> <- 2[X,H]|phi_1> + 2H|phi_1^x> - |phi_0^x> */
        apply_xh(&h, p1, x2);
        apply_h(&h, x1, tmp);
        for (int64_t q = 0; q < 2 * n; q++) x2[q] = 2.0 * x2[q] + 2.0 * tmp[q] - x0[q];
        /* |out> <- |out> + 2 (-i)^m J_m |phi_2^x> */
        ipow(-1, m, &cr, &ci);
        axpy_c(n, 2.0 * jm[m] * cr, 2.0 * jm[m] * ci, x2, out);
        double* t = p0; p0 = p1; p1 = p2; p2 = t;
        t = x0; x0 = x1; x1 = x2; x2 = t;
    }
    free(p0); free(p1); free(p2); free(x0); free(x1); free(x2); free(tmp);
}

/* ------------------------------------------------------------------ */
/* Velocity V = (i/hbar)[H, X] = -(i E_max/hbar) [X, H~]  (Eq. 15)     */
/* ------------------------------------------------------------------ */

/* out = V in, in nm/fs when hbar is in eV fs and E_max in eV. */
static void apply_v(const ora_h* h, double emax, double hbar, const double* in, double* out) {
    apply_xh(h, in, out);
    const double s = emax / hbar;
    for (int64_t q = 0; q < h->n; q++) {
        double re = out[2 * q], im = out[2 * q + 1];
        /* -(i s)(re + i im) = s im - i s re */
        out[2 * q] = s * im;
        out[2 * q + 1] = -s * re;
    }
}

void ora_apply_v(int64_t n, const int64_t* rp, const int64_t* col, const double* val,
                 const double* disp, const double* diag, double emax, double hbar,
                 const double* in, double* out) {
    ora_h h = {n, rp, col, val, disp, diag};
    apply_v(&h, emax, hbar, in, out);
}

/* ------------------------------------------------------------------ */
/* Correlation-time loops (Algorithms 2 and 3, Eqs. 42-44)             */
/* ------------------------------------------------------------------ */

/* VAC moments C_n^VAC(t_m) = <phi_L|T_n(H~)|phi_R>, Eq. (33), with
 * |phi_L> = V U^dagger(t_m)|phi>, |phi_R> = U^dagger(t_m) V|phi> (Sec. 3.2),
 * advanced by Eqs. (42)-(43): U^dagger(t + dt) = U^dagger(dt) U^dagger(t).
 * Reading: t_m = m dt for m = 0 .. n_times-1, so C_vv(E, 0) is included
 * (Algorithm 2 starts its loop at m = 1, but the time integral of Eq. (6)
 * starts at t = 0).  Output c[n_times][M][2]. */
void ora_vac(int64_t n, const int64_t* rp, const int64_t* col, const double* val,
             const double* disp, const double* diag, double emax, double hbar,
             const double* phi, int n_moments, int n_times, const double* jm, int np,
             double* c) {
    ora_h h = {n, rp, col, val, disp, diag};
    double* a = malloc(sizeof(double) * 2 * n);    /* U^dagger(t)|phi>   */
    double* b = malloc(sizeof(double) * 2 * n);    /* U^dagger(t) V|phi> */
    double* l = malloc(sizeof(double) * 2 * n);
    double* t = malloc(sizeof(double) * 2 * n);
    memcpy(a, phi, sizeof(double) * 2 * n);
    apply_v(&h, emax, hbar, phi, b);
    for (int m = 0; m < n_times; m++) {
        if (m > 0) {
            ora_evolve(n, rp, col, val, disp, diag, jm, np, -1, a, t);
            memcpy(a, t, sizeof(double) * 2 * n);
            ora_evolve(n, rp, col, val, disp, diag, jm, np, -1, b, t);
            memcpy(b, t, sizeof(double) * 2 * n);
        }
        apply_v(&h, emax, hbar, a, l);
        ora_kpm_moments(n, rp, col, val, disp, diag, l, b, n_moments,
                        c + (size_t)2 * n_moments * m);
    }
    free(a); free(b); free(l); free(t);
}

/* MSD moments C_n^MSD(t_m) = <phi_L|T_n(H~)|phi_L>, Eq. (34), with
 * |phi_L> = [X, U(t_m)]|phi>, advanced by Eq. (44):
 *   [X, U(t+dt)]|phi> = U(dt)[X, U(t)]|phi> + [X, U(dt)] U(t)|phi>,
 * and U(t+dt)|phi> = U(dt) U(t)|phi>.  [X, U(0)] = 0.  Output c[n_times][M][2]. */
void ora_msd(int64_t n, const int64_t* rp, const int64_t* col, const double* val,
             const double* disp, const double* diag, const double* phi, int n_moments,
             int n_times, const double* jm, int np, double* c) {
    double* psi = malloc(sizeof(double) * 2 * n);   /* U(t)|phi>      */
    double* xi = malloc(sizeof(double) * 2 * n);    /* [X, U(t)]|phi> */
    double* t1 = malloc(sizeof(double) * 2 * n);
    double* t2 = malloc(sizeof(double) * 2 * n);
    memcpy(psi, phi, sizeof(double) * 2 * n);
    memset(xi, 0, sizeof(double) * 2 * n);
    for (int m = 0; m < n_times; m++) {
        if (m > 0) {
            ora_evolve(n, rp, col, val, disp, diag, jm, np, +1, xi, t1);    /* U(dt) xi       */
            ora_evolvex(n, rp, col, val, disp, diag, jm, np, psi, t2);      /* [X,U(dt)] psi  */
            for (int64_t q = 0; q < 2 * n; q++) xi[q] = t1[q] + t2[q];
            ora_evolve(n, rp, col, val, disp, diag, jm, np, +1, psi, t1);   /* U(dt) psi      */
            memcpy(psi, t1, sizeof(double) * 2 * n);
        }
        ora_kpm_moments(n, rp, col, val, disp, diag, xi, xi, n_moments,
                        c + (size_t)2 * n_moments * m);
    }
    free(psi); free(xi); free(t1); free(t2);
}

/* ------------------------------------------------------------------ */
/* Host sums (Eqs. 29-31 and 35)                                       */
/* ------------------------------------------------------------------ */

/* Jackson damping g_n = (1 - n a) cos(pi n a) + a sin(pi n a) cot(pi a),
 * a = 1/(M + 1)  (Eq. 35). */
void ora_jackson(int n_moments, double* g) {
    const double al = 1.0 / (n_moments + (g_mutation == 4 ? 0.0 : 1.0));  /* planted: a = 1/M */
    for (int k = 0; k < n_moments; k++) {
        g[k] = (1.0 - k * al) * cos(ORA_PI * k * al) +
               al * sin(ORA_PI * k * al) / tan(ORA_PI * al);
    }
}

/* Chebyshev sum of Eqs. (29)-(31) on scaled energies e (|e| < 1), without the
 * 1/Omega factor:  out(e) = 2/(pi sqrt(1-e^2)) sum_n g_n (2 - delta_n0) T_n(e) mu_n,
 * with T_n(e) = cos(n arccos e).  mu is the real part of the moments. */
void ora_kpm_sum(int n_moments, const double* mu, const double* g, int n_e,
                 const double* e, double* out) {
    for (int q = 0; q < n_e; q++) {
        double th = acos(e[q]);
        double s = 0.0;
        for (int k = 0; k < n_moments; k++) {
            double w = (k == 0) ? 1.0 : 2.0;
            s += g[k] * w * cos(k * th) * mu[k];
        }
        out[q] = 2.0 / (ORA_PI * sqrt(1.0 - e[q] * e[q])) * s;
    }
}

/* ------------------------------------------------------------------ */
/* Fourier moments (Algorithm 4, Eqs. 25 and 45)                       */
/* ------------------------------------------------------------------ */

/* F_n = <phi_L|U(n dtau)|phi_R> for n = -N_m .. N_m (output index n + N_m), with
 * U(dtau) = exp(-i H~ tau) applied n times forward and n times backward as in
 * Algorithm 4.  For the scaled Hamiltonian the step is dtau = pi hbar, i.e. tau = pi
 * (Sec. 4.2).  j[] holds J_m(tau), m < np.  Output f[2 N_m + 1][2]. */
void ora_ftm_moments(int64_t n, const int64_t* rp, const int64_t* col, const double* val,
                     const double* disp, const double* diag, const double* phi_l,
                     const double* phi_r, int n_m, const double* jm, int np, double* f) {
    double* p = malloc(sizeof(double) * 2 * n);
    double* t = malloc(sizeof(double) * 2 * n);
    /* |phi'_R> <- |phi_R>;  F_0 <- <phi_L|phi'_R> */
    memcpy(p, phi_r, sizeof(double) * 2 * n);
    dot(n, phi_l, p, &f[2 * n_m], &f[2 * n_m + 1]);
    for (int k = 1; k <= n_m; k++) {
        /* |phi'_R> <- U(dtau)|phi'_R>;  F_k <- <phi_L|phi'_R> */
        ora_evolve(n, rp, col, val, disp, diag, jm, np, +1, p, t);
        memcpy(p, t, sizeof(double) * 2 * n);
        dot(n, phi_l, p, &f[2 * (n_m + k)], &f[2 * (n_m + k) + 1]);
    }
    memcpy(p, phi_r, sizeof(double) * 2 * n);
    for (int k = 1; k <= n_m; k++) {
        /* |phi'_R> <- U^dagger(dtau)|phi'_R>;  F_{-k} <- <phi_L|phi'_R> */
        ora_evolve(n, rp, col, val, disp, diag, jm, np, -1, p, t);
        memcpy(p, t, sizeof(double) * 2 * n);
        dot(n, phi_l, p, &f[2 * (n_m - k)], &f[2 * (n_m - k) + 1]);
    }
    free(p); free(t);
}
