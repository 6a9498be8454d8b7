/*
 * kd_oracle.c -- plain FP64 CPU oracle for the 2D Dirac FFT split-operator step.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Slow and literal on
 * purpose: every 4x4 factor is built as an explicit complex matrix from the closed
 * forms and multiplied out, the FFT is a textbook recursive radix-2 transform, and
 * the Gaussian beam is the sum over both propagation directions exactly as written
 * in the paper.  Compiled with -O2 -ffp-contract=off, no fast-math.
 *
 * Readings of the paper that this file implements (the paper is silent or garbled):
 *  - r in the beam formulas is the transverse distance |y| (2D, beam along x).
 *  - the waist is w0 = 1/(k_L epsilon) (the paper's "omega_0" is a typo).
 *  - amplitude a0 = q A0 / (m c^2); V = -q alpha.A = -m c^2 alpha.a (phi = 0).
 *  - the constant gauge A_m is a kinetic-momentum offset: pi = p + p_shift.
 *  - co-moving box: rows sit at y_min + i dy + box_vy t; the frame translation adds
 *    -box_vy p_y(canonical) to H, a phase exp(+i box_vy p_y dt / hbar) in K.
 *  - Strang step: V(t_n, dt/2), FFT, K(dt), inverse FFT / P, V(t_{n+1}, dt/2).
 *  - bispinors are normalised (u^dagger u = 1) with chi = (1, +-1)/sqrt(2).
 *  - momentum-space read-outs are discrete cell probabilities |DFT psi|^2 dx dy / P.
 *  - packet phase uses r0 relative to the grid origin (x_min, y_min), so that the
 *    inverse DFT centres the packet at r0 in absolute coordinates.
 */
#include "kd_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define OR_PI 3.14159265358979323846264338327950288

static int is_pow2(int32_t n) { return n >= 1 && (n & (n - 1)) == 0; }

/* ------------------------------------------------------------------ FFT -- */
/* Textbook decimation in time: out[k] = sum_j a[j*stride] e^{sign 2 pi i jk/n}. */
static void fft_rec(const cplx* a, int32_t n, int32_t stride, cplx* out, int32_t sign) {
    if (n == 1) {
        out[0] = a[0];
        return;
    }
    int32_t h = n / 2;
    fft_rec(a, h, 2 * stride, out, sign);
    fft_rec(a + stride, h, 2 * stride, out + h, sign);
    for (int32_t k = 0; k < h; ++k) {
        double ang = 2.0 * OR_PI * (double)k / (double)n;
        cplx w = cos(ang) + I * ((double)sign * sin(ang));
        cplx e = out[k];
        cplx o = w * out[k + h];
        out[k] = e + o;
        out[k + h] = e - o;
    }
}

int or_fft1d(double* data, int32_t n, int32_t sign) {
    if (!data || !is_pow2(n) || (sign != 1 && sign != -1)) return -1;
    cplx* in = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    if (!in || !out) { free(in); free(out); return -3; }
    memcpy(in, data, sizeof(cplx) * (size_t)n);
    fft_rec(in, n, 1, out, sign);
    memcpy(data, out, sizeof(cplx) * (size_t)n);
    free(in);
    free(out);
    return 0;
}

/* 2D transform: 1D transforms of every row, then of every column, per component.  The
 * rows (columns) are independent; a build with OpenMP (-fopenmp, the timing variant) runs
 * them on several threads, each with its own line buffers, with identical results. */
int or_fft2d(double* psi_d, int32_t nx, int32_t ny, int32_t sign) {
    if (!psi_d || !is_pow2(nx) || !is_pow2(ny) || (sign != 1 && sign != -1)) return -1;
    cplx* psi = (cplx*)psi_d;
    int32_t nmax = nx > ny ? nx : ny;
#ifdef _OPENMP
    const int nthr = omp_get_max_threads();
#else
    const int nthr = 1;
#endif
    cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)nmax * 2 * (size_t)nthr);
    if (!buf) return -3;
    for (int32_t c = 0; c < 4; ++c) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int32_t iy = 0; iy < ny; ++iy) {          /* rows: transform along x */
#ifdef _OPENMP
            cplx* line = buf + (size_t)nmax * 2 * omp_get_thread_num();
#else
            cplx* line = buf;
#endif
            cplx* res = line + nmax;
            for (int32_t ix = 0; ix < nx; ++ix) line[ix] = psi[((size_t)iy * nx + ix) * 4 + c];
            fft_rec(line, nx, 1, res, sign);
            for (int32_t ix = 0; ix < nx; ++ix) psi[((size_t)iy * nx + ix) * 4 + c] = res[ix];
        }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int32_t ix = 0; ix < nx; ++ix) {          /* columns: transform along y */
#ifdef _OPENMP
            cplx* line = buf + (size_t)nmax * 2 * omp_get_thread_num();
#else
            cplx* line = buf;
#endif
            cplx* res = line + nmax;
            for (int32_t iy = 0; iy < ny; ++iy) line[iy] = psi[((size_t)iy * nx + ix) * 4 + c];
            fft_rec(line, ny, 1, res, sign);
            for (int32_t iy = 0; iy < ny; ++iy) psi[((size_t)iy * nx + ix) * 4 + c] = res[iy];
        }
    }
    free(buf);
    return 0;
}

/* --------------------------------------------------- Dirac matrices ------ */
/* Pauli matrices sigma_x, sigma_y, sigma_z. */
static void pauli(int i, cplx s[2][2]) {
    memset(s, 0, sizeof(cplx) * 4);
    if (i == 0) { s[0][1] = 1; s[1][0] = 1; }
    if (i == 1) { s[0][1] = -I; s[1][0] = I; }
    if (i == 2) { s[0][0] = 1; s[1][1] = -1; }
}

/* Standard (Dirac) representation: alpha_i = [[0, sigma_i], [sigma_i, 0]],
 * beta = diag(1, 1, -1, -1)  (Eq. Hamiltonian operator and the text after it). */
static void alpha_mat(int i, cplx a[4][4]) {
    cplx s[2][2];
    pauli(i, s);
    memset(a, 0, sizeof(cplx) * 16);
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            a[r][c + 2] = s[r][c];
            a[r + 2][c] = s[r][c];
        }
}

static void beta_mat(cplx b[4][4]) {
    memset(b, 0, sizeof(cplx) * 16);
    b[0][0] = 1; b[1][1] = 1; b[2][2] = -1; b[3][3] = -1;
}

void or_dirac_matrices(double* ax, double* ay, double* b) {
    cplx m[4][4];
    alpha_mat(0, m);
    if (ax) memcpy(ax, m, sizeof(m));
    alpha_mat(1, m);
    if (ay) memcpy(ay, m, sizeof(m));
    beta_mat(m);
    if (b) memcpy(b, m, sizeof(m));
}

static void matvec4(cplx M[4][4], const cplx* v, cplx* out) {
    for (int r = 0; r < 4; ++r) {
        cplx acc = 0;
        for (int c = 0; c < 4; ++c) acc += M[r][c] * v[c];
        out[r] = acc;
    }
}

/* ---------------------------------------------------------------- field -- */
static double envelope(const or_field* f, double t) {
    if (f->env_T <= 0.0) return 1.0;
    if (t < 0.0 || t > f->env_T) return 0.0;
    double s = sin(OR_PI * t / f->env_T);
    return s * s;
}

/* Eqs. (Equation_of_Gaussian_beam), (Phase_of_Gaussian_beam), w(x), and the
 * standing-wave superposition (Equation_of_vector_potential), summed over d = -1, +1
 * term by term.  Returns a = qA/(m c^2). */
int or_field_a(const or_units* u, const or_field* f, double x, double y, double t,
               double* ax_out, double* ay_out) {
    if (!u || !f || !ax_out || !ay_out) return -1;
    double ax = 0.0, ay = 0.0;
    double k = f->k_L;
    double omega = u->c * k;
    double wt = omega * t + f->phase0;
    if (f->kind == 1) {
        /* plane-wave standing wave: two counter-propagating plane waves, the
         * epsilon -> 0 limit of the beams below */
        for (int d = -1; d <= 1; d += 2) ay += -sin(wt - d * k * x);
    } else if (f->kind == 2) {
        double eps = f->epsilon;
        double w0 = 1.0 / (k * eps);
        double xR = k * w0 * w0 / 2.0;
        double w = w0 * sqrt(1.0 + x * x / (xR * xR));
        double r2 = y * y;
        for (int d = -1; d <= 1; d += 2) {
            double phiG = wt - d * k * x + atan(d * x / xR) - d * x * r2 / (xR * w * w);
            double phi1 = phiG + atan(d * x / xR);
            double g = (w0 / w) * exp(-r2 / (w * w));
            ay += -g * sin(phiG);
            if (f->longitudinal) ax += -2.0 * d * g * eps * (y / w) * cos(phi1);
        }
    } else if (f->kind != 0) {
        return -1;
    }
    double s = f->a0 * envelope(f, t);
    *ax_out = s * ax;
    *ay_out = s * ay;
    return 0;
}

/* exp(-i tau V / hbar) with V = -m c^2 alpha.a:  the generator (alpha.a)^2 = |a|^2
 * gives cos(theta) I + i sin(theta) alpha.a/|a|, theta = tau m c^2 |a| / hbar. */
static void potential_factor(const or_units* u, double ax, double ay, double tau,
                             cplx M[4][4]) {
    cplx Ax[4][4], Ay[4][4];
    alpha_mat(0, Ax);
    alpha_mat(1, Ay);
    double amag = sqrt(ax * ax + ay * ay);
    double kappa = tau * u->m * u->c * u->c / u->hbar;
    double theta = kappa * amag;
    double sinc_k; /* sin(theta)/|a| */
    if (theta < 1e-8)
        sinc_k = kappa * (1.0 - theta * theta / 6.0);
    else
        sinc_k = sin(theta) / amag;
    double ct = cos(theta);
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c)
            M[r][c] = (r == c ? ct : 0.0) + I * sinc_k * (Ax[r][c] * ax + Ay[r][c] * ay);
}

void or_potential_factor(const or_units* u, double ax, double ay, double tau, double* M) {
    cplx m[4][4];
    potential_factor(u, ax, ay, tau, m);
    memcpy(M, m, sizeof(m));
}

/* exp(-i dt H0 / hbar) = cos(E dt/hbar) I - i sin(E dt/hbar) H0/E, because H0^2 = E^2. */
static void kinetic_factor(const or_units* u, double pix, double piy, double dt, cplx M[4][4]) {
    cplx Ax[4][4], Ay[4][4], B[4][4];
    alpha_mat(0, Ax);
    alpha_mat(1, Ay);
    beta_mat(B);
    double mc2 = u->m * u->c * u->c;
    double E = sqrt(mc2 * mc2 + u->c * u->c * (pix * pix + piy * piy));
    double ph = E * dt / u->hbar;
    double C = cos(ph), S = sin(ph) / E;
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            cplx H = u->c * (Ax[r][c] * pix + Ay[r][c] * piy) + B[r][c] * mc2;
            M[r][c] = (r == c ? C : 0.0) - I * S * H;
        }
}

void or_kinetic_factor(const or_units* u, double pix, double piy, double dt, double* M) {
    cplx m[4][4];
    kinetic_factor(u, pix, piy, dt, m);
    memcpy(M, m, sizeof(m));
}

/* u^s(p) of Eq. (Spinors_of_Dirac_equation) with unit-normalised chi and the overall
 * factor sqrt((E + mc^2) / (2E)), so that u^dagger u = 1. */
static void spinor_u(const or_units* u, double pix, double piy, int32_t spin, int32_t basis,
                     cplx out[4]) {
    double mc2 = u->m * u->c * u->c;
    double E = sqrt(mc2 * mc2 + u->c * u->c * (pix * pix + piy * piy));
    cplx chi[2];
    if (basis == 1) {
        chi[0] = spin > 0 ? 1.0 : 0.0;
        chi[1] = spin > 0 ? 0.0 : 1.0;
    } else {
        chi[0] = 1.0 / sqrt(2.0);
        chi[1] = (spin > 0 ? 1.0 : -1.0) / sqrt(2.0);
    }
    cplx sx[2][2], sy[2][2];
    pauli(0, sx);
    pauli(1, sy);
    double nrm = sqrt((E + mc2) / (2.0 * E));
    for (int r = 0; r < 2; ++r) {
        cplx low = 0;
        for (int c = 0; c < 2; ++c) low += u->c * (sx[r][c] * pix + sy[r][c] * piy) * chi[c];
        out[r] = nrm * chi[r];
        out[r + 2] = nrm * low / (E + mc2);
    }
}

void or_spinor_u(const or_units* u, double pix, double piy, int32_t spin, int32_t basis,
                 double* out) {
    cplx v[4];
    spinor_u(u, pix, piy, spin, basis, v);
    memcpy(out, v, sizeof(v));
}

/* ------------------------------------------------------------- grids ----- */
static int32_t signed_index(int32_t k, int32_t n) { return k < n / 2 ? k : k - n; }

static void canonical_momentum(const or_grid* g, const or_units* u, int32_t kx, int32_t ky,
                               double* px, double* py) {
    double Lx = g->x_max - g->x_min, Ly = g->y_max - g->y_min;
    *px = u->hbar * (2.0 * OR_PI / Lx) * (double)signed_index(kx, g->nx);
    *py = u->hbar * (2.0 * OR_PI / Ly) * (double)signed_index(ky, g->ny);
}

void or_momentum(const or_grid* g, const or_units* u, const or_field* f, int32_t kx,
                 int32_t ky, double* pix, double* piy) {
    double px, py;
    canonical_momentum(g, u, kx, ky, &px, &py);
    *pix = px + f->p_shift_x;
    *piy = py + f->p_shift_y;
}

static int check_grid(const or_grid* g) {
    if (!g || !is_pow2(g->nx) || !is_pow2(g->ny) || g->nx < 4 || g->ny < 4) return -1;
    if (!(g->x_max > g->x_min) || !(g->y_max > g->y_min)) return -1;
    return 0;
}

/* -------------------------------------------------------- initial state -- */
/* Eq. (Density_distribution_of_Gaussian_wave_packet) and phi(p,0) = u^s rho:
 * rho(pi) = exp(-|pi - p0|^2 / (4 sigma_p^2) - i (r0 - origin).p / hbar); the
 * continuum prefactor is dropped and the state renormalised on the grid. */
int or_init_packet(const or_units* u, const or_grid* g, const or_field* f,
                   const or_packet* pk, double* psi_d) {
    if (!u || !f || !pk || !psi_d || check_grid(g)) return -1;
    if (!(pk->sigma_p > 0.0)) return -1;
    cplx* psi = (cplx*)psi_d;
    int32_t nx = g->nx, ny = g->ny;
    double rx = pk->r0x - g->x_min, ry = pk->r0y - g->y_min;
    for (int32_t ky = 0; ky < ny; ++ky)
        for (int32_t kx = 0; kx < nx; ++kx) {
            double px, py, pix, piy;
            canonical_momentum(g, u, kx, ky, &px, &py);
            pix = px + f->p_shift_x;
            piy = py + f->p_shift_y;
            double dx = pix - pk->p0x, dy = piy - pk->p0y;
            double mag = exp(-(dx * dx + dy * dy) / (4.0 * pk->sigma_p * pk->sigma_p));
            double ph = -(rx * px + ry * py) / u->hbar;
            cplx rho = mag * (cos(ph) + I * sin(ph));
            cplx us[4];
            spinor_u(u, pix, piy, pk->spin, pk->basis, us);
            for (int c = 0; c < 4; ++c) psi[((size_t)ky * nx + kx) * 4 + c] = us[c] * rho;
        }
    int rc = or_fft2d(psi_d, nx, ny, +1);
    if (rc) return rc;
    double dxdy = (g->x_max - g->x_min) / nx * (g->y_max - g->y_min) / ny;
    double s = 0.0;
    for (size_t i = 0; i < (size_t)nx * ny * 4; ++i) s += creal(psi[i] * conj(psi[i]));
    s *= dxdy;
    if (!(s > 0.0)) return -2;
    double scale = 1.0 / sqrt(s);
    for (size_t i = 0; i < (size_t)nx * ny * 4; ++i) psi[i] *= scale;
    return 0;
}

/* ------------------------------------------------------------- the step -- */
int or_potential_step(const or_units* u, const or_grid* g, const or_field* f, double* psi_d,
                      double t, double tau) {
    if (!u || !f || !psi_d || check_grid(g)) return -1;
    cplx* psi = (cplx*)psi_d;
    int32_t nx = g->nx, ny = g->ny;
    double dx = (g->x_max - g->x_min) / nx, dy = (g->y_max - g->y_min) / ny;
    int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(|: bad)
#endif
    for (int32_t iy = 0; iy < ny; ++iy) {
        double y = g->y_min + iy * dy + f->box_vy * t;
        for (int32_t ix = 0; ix < nx; ++ix) {
            double x = g->x_min + ix * dx;
            double ax, ay;
            if (or_field_a(u, f, x, y, t, &ax, &ay)) { bad = 1; continue; }
            cplx M[4][4], out[4];
            potential_factor(u, ax, ay, tau, M);
            cplx* v = psi + ((size_t)iy * nx + ix) * 4;
            matvec4(M, v, out);
            for (int c = 0; c < 4; ++c) v[c] = out[c];
        }
    }
    return bad ? -1 : 0;
}

int or_kinetic_step(const or_units* u, const or_grid* g, const or_field* f, double* phi_d,
                    double dt) {
    if (!u || !f || !phi_d || check_grid(g)) return -1;
    cplx* phi = (cplx*)phi_d;
    int32_t nx = g->nx, ny = g->ny;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int32_t ky = 0; ky < ny; ++ky)
        for (int32_t kx = 0; kx < nx; ++kx) {
            double px, py;
            canonical_momentum(g, u, kx, ky, &px, &py);
            cplx M[4][4], out[4];
            kinetic_factor(u, px + f->p_shift_x, py + f->p_shift_y, dt, M);
            double fr = f->box_vy * py * dt / u->hbar;   /* frame translation phase */
            cplx frame = cos(fr) + I * sin(fr);
            cplx* v = phi + ((size_t)ky * nx + kx) * 4;
            matvec4(M, v, out);
            for (int c = 0; c < 4; ++c) v[c] = frame * out[c];
        }
    return 0;
}

int or_step(const or_units* u, const or_grid* g, const or_field* f, double* psi_d, double t0,
            double dt, int64_t nsteps) {
    if (!u || !f || !psi_d || check_grid(g) || nsteps < 0) return -1;
    size_t n = (size_t)g->nx * g->ny * 4;
    double invP = 1.0 / ((double)g->nx * (double)g->ny);
    cplx* psi = (cplx*)psi_d;
    for (int64_t s = 0; s < nsteps; ++s) {
        double tn = t0 + (double)s * dt;
        double tn1 = t0 + (double)(s + 1) * dt;
        int rc = or_potential_step(u, g, f, psi_d, tn, dt / 2.0);
        if (!rc) rc = or_fft2d(psi_d, g->nx, g->ny, -1);
        if (!rc) rc = or_kinetic_step(u, g, f, psi_d, dt);
        if (!rc) rc = or_fft2d(psi_d, g->nx, g->ny, +1);
        if (rc) return rc;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (size_t i = 0; i < n; ++i) psi[i] *= invP;
        rc = or_potential_step(u, g, f, psi_d, tn1, dt / 2.0);
        if (rc) return rc;
    }
    return 0;
}

/* ---------------------------------------------------------- observables -- */
int or_density_x(const or_grid* g, const double* psi_d, double* out) {
    if (check_grid(g) || !psi_d || !out) return -1;
    const cplx* psi = (const cplx*)psi_d;
    double dy = (g->y_max - g->y_min) / g->ny;
    for (int32_t ix = 0; ix < g->nx; ++ix) {
        double s = 0.0;
        for (int32_t iy = 0; iy < g->ny; ++iy)
            for (int c = 0; c < 4; ++c) {
                cplx v = psi[((size_t)iy * g->nx + ix) * 4 + c];
                s += creal(v) * creal(v) + cimag(v) * cimag(v);
            }
        out[ix] = s * dy;
    }
    return 0;
}

int or_momentum_density(const or_units* u, const or_grid* g, const or_field* f,
                        int32_t basis, const double* psi_d, double* out) {
    if (!u || !f || !psi_d || !out || check_grid(g)) return -1;
    int32_t nx = g->nx, ny = g->ny;
    size_t n = (size_t)nx * ny * 4;
    cplx* phi = (cplx*)malloc(sizeof(cplx) * n);
    if (!phi) return -3;
    memcpy(phi, psi_d, sizeof(cplx) * n);
    or_fft2d((double*)phi, nx, ny, -1);
    double dxdy = (g->x_max - g->x_min) / nx * (g->y_max - g->y_min) / ny;
    double w = dxdy / ((double)nx * (double)ny);
    for (int32_t ky = 0; ky < ny; ++ky)
        for (int32_t kx = 0; kx < nx; ++kx) {
            double pix, piy;
            or_momentum(g, u, f, kx, ky, &pix, &piy);
            const cplx* v = phi + ((size_t)ky * nx + kx) * 4;
            double p2 = 0.0;
            for (int c = 0; c < 4; ++c) p2 += creal(v[c] * conj(v[c]));
            double cs[2];
            for (int si = 0; si < 2; ++si) {
                cplx us[4];
                spinor_u(u, pix, piy, si == 0 ? 1 : -1, basis, us);
                cplx a = 0;
                for (int c = 0; c < 4; ++c) a += conj(us[c]) * v[c];
                cs[si] = creal(a * conj(a));
            }
            double* o = out + ((size_t)ky * nx + kx) * 3;
            o[0] = p2 * w;
            o[1] = cs[0] * w;
            o[2] = cs[1] * w;
        }
    free(phi);
    return 0;
}

/* Window of integer signed indices around the grid point nearest to a kinetic
 * momentum: centre round((pi - p_shift)/dp), half width floor(h/dp), clamped to the
 * grid.  Returns -1 if the centre lies outside the grid. */
static int window_axis(double pi_c, double shift, double dp, double h, int32_t n, int32_t* lo,
                       int32_t* hi, int32_t* centre) {
    double v = floor((pi_c - shift) / dp + 0.5);
    if (!(v >= -(double)(n / 2) && v <= (double)(n / 2 - 1))) return -1;
    int32_t c = (int32_t)v;
    int32_t w = (int32_t)floor(h / dp + 1e-9);
    if (w < 0) return -1;
    *centre = c;
    *lo = c - w < -(n / 2) ? -(n / 2) : c - w;
    *hi = c + w > n / 2 - 1 ? n / 2 - 1 : c + w;
    return 0;
}

int or_observe(const or_units* u, const or_grid* g, const or_field* f,
               const or_obs_spec* spec, const double* psi_d, double t, or_obs* out) {
    if (!u || !f || !spec || !psi_d || !out || check_grid(g)) return -1;
    if (!(spec->half_width >= 0.0)) return -1;
    int32_t nx = g->nx, ny = g->ny;
    double dpx = u->hbar * 2.0 * OR_PI / (g->x_max - g->x_min);
    double dpy = u->hbar * 2.0 * OR_PI / (g->y_max - g->y_min);
    int32_t ilo[3], ihi[3], ic[3], jlo[3], jhi[3], jc[3];
    double cx[3] = {spec->p_in_x, spec->p_diff_x, spec->target_x};
    double cy[3] = {spec->p_in_y, spec->p_diff_y, spec->target_y};
    for (int w = 0; w < 3; ++w) {
        if (window_axis(cx[w], f->p_shift_x, dpx, spec->half_width, nx, &ilo[w], &ihi[w], &ic[w]))
            return -2;
        if (window_axis(cy[w], f->p_shift_y, dpy, spec->half_width, ny, &jlo[w], &jhi[w], &jc[w]))
            return -2;
    }
    double* md = (double*)malloc(sizeof(double) * (size_t)nx * ny * 3);
    if (!md) return -3;
    int rc = or_momentum_density(u, g, f, spec->basis, psi_d, md);
    if (rc) { free(md); return rc; }
    memset(out, 0, sizeof(*out));
    out->t = t;
    const cplx* psi = (const cplx*)psi_d;
    double dxdy = (g->x_max - g->x_min) / nx * (g->y_max - g->y_min) / ny;
    double s = 0.0;
    for (size_t i = 0; i < (size_t)nx * ny * 4; ++i)
        s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    out->norm = s * dxdy;
    double sums[2][3] = {{0}};
    double mx[3] = {0, 0, 0};
    for (int w = 0; w < 2; ++w)
        for (int32_t j = jlo[w]; j <= jhi[w]; ++j)
            for (int32_t i = ilo[w]; i <= ihi[w]; ++i) {
                int32_t kx = (i + nx) % nx, ky = (j + ny) % ny;
                const double* o = md + ((size_t)ky * nx + kx) * 3;
                for (int q = 0; q < 3; ++q) {
                    sums[w][q] += o[q];
                    if (w == 1 && o[q] > mx[q]) mx[q] = o[q];
                }
            }
    out->pop_in = sums[0][0];
    out->cp_in = sums[0][1];
    out->cm_in = sums[0][2];
    out->pop_diff = sums[1][0];
    out->cp_diff = sums[1][1];
    out->cm_diff = sums[1][2];
    out->max_diff = mx[0];
    out->cp_max_diff = mx[1];
    out->cm_max_diff = mx[2];
    {
        int32_t kx = (ic[2] + nx) % nx, ky = (jc[2] + ny) % ny;
        const double* o = md + ((size_t)ky * nx + kx) * 3;
        out->p_target = o[0];
        out->cp_target = o[1];
        out->cm_target = o[2];
    }
    free(md);
    return 0;
}
