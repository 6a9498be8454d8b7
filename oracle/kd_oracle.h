/*
 * kd_oracle.h -- plain FP64 CPU oracle for the 2D Dirac FFT split-operator step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this library; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no source with the CUDA library.
 *
 * Paper: Ge, Ahrens & Shen, "Two-dimensional simulation of the spin-flip in the
 * Kapitza-Dirac effect" (arXiv 2307.01571).
 *   Sec. II.A  Gaussian-beam standing wave, Eqs. (Equation_of_Gaussian_beam),
 *              (Phase_of_Gaussian_beam), (Equation_of_vector_potential).
 *   Sec. II.B  Dirac Hamiltonian (Hamiltonian operator), bispinors
 *              (Spinors_of_Dirac_equation), energy (relativistic_energy_momentum_relation).
 *   Sec. II.C  Gaussian packet (Density_distribution_of_Gaussian_wave_packet),
 *              Fourier convention (fourier_transformation).
 *   Sec. II.D  FFT split-operator propagation U(t+dt, t).
 *   Sec. III   densities (probability_density), (y_integrated_probability_density),
 *              (px_momentum_space_probability_density), spin projection
 *              (Equation_of_spin_projection).
 *
 * Complex arrays are passed as interleaved doubles (re, im).  The spinor layout is
 * [ny][nx][4] complex, point-major, components in the Dirac (standard)
 * representation.  All functions return 0 on success and a negative code on a bad
 * argument; they never abort.
 */
#ifndef KD_ORACLE_H
#define KD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double m, c, hbar, q; } or_units;
typedef struct { int32_t nx, ny; double x_min, x_max, y_min, y_max; } or_grid;
typedef struct {
    int32_t kind;          /* 0 none, 1 plane standing wave, 2 Gaussian-beam standing wave */
    int32_t longitudinal;  /* 1: include the longitudinal component A_x */
    double a0;             /* q A0 / (m c^2), dimensionless amplitude */
    double k_L;            /* laser wave number; omega = c k_L */
    double epsilon;        /* beam divergence; waist w0 = 1/(k_L epsilon) */
    double env_T;          /* sin^2 envelope length; 0 = continuous wave */
    double phase0;         /* added to omega t */
    double p_shift_x, p_shift_y; /* kinetic minus canonical momentum (constant gauge) */
    double box_vy;         /* co-moving box speed along y */
} or_field;
typedef struct {
    double p0x, p0y;       /* kinetic centre momentum */
    double r0x, r0y;       /* centre position (absolute coordinates at t = 0) */
    double sigma_p;        /* momentum width parameter */
    int32_t spin;          /* +1 / -1 */
    int32_t basis;         /* 0: x-polarised chi = (1, +-1)/sqrt2; 1: z-polarised */
} or_packet;
typedef struct {
    double p_in_x, p_in_y;       /* kinetic centre of the incoming-peak window */
    double p_diff_x, p_diff_y;   /* kinetic centre of the diffracted-peak window */
    double target_x, target_y;   /* kinetic momentum for the single-cell read-out */
    double half_width;           /* window half width (infinity norm) in momentum */
    int32_t basis;               /* spin basis of the projections, as or_packet.basis */
    int32_t pad_;
} or_obs_spec;
typedef struct {
    double t;
    double norm;
    double pop_in, pop_diff;
    double cp_in, cm_in, cp_diff, cm_diff;
    double max_diff, cp_max_diff, cm_max_diff;
    double p_target, cp_target, cm_target;
} or_obs;

/* Own recursive radix-2 FFT: out[k] = sum_j in[j] exp(sign 2 pi i j k / n). */
int or_fft1d(double* data, int32_t n, int32_t sign);
/* Unnormalised 2D DFT of each of the 4 components of a [ny][nx][4] spinor. */
int or_fft2d(double* psi, int32_t nx, int32_t ny, int32_t sign);

/* Dirac matrices alpha_x, alpha_y, beta (4x4 complex, row-major). */
void or_dirac_matrices(double* alpha_x, double* alpha_y, double* beta);
/* Dimensionless field a = qA/(m c^2) at physical point (x, y) and time t. */
int or_field_a(const or_units* u, const or_field* f, double x, double y, double t,
               double* ax, double* ay);
/* exp(-i tau V / hbar), V = -q alpha.A, as a 4x4 complex matrix. */
void or_potential_factor(const or_units* u, double ax, double ay, double tau, double* M);
/* exp(-i dt H0(pi) / hbar), H0 = c alpha.pi + beta m c^2, as a 4x4 complex matrix. */
void or_kinetic_factor(const or_units* u, double pix, double piy, double dt, double* M);
/* Normalised positive-energy bispinor u^s(pi) (4 complex). */
void or_spinor_u(const or_units* u, double pix, double piy, int32_t spin, int32_t basis,
                 double* out);
/* Kinetic momentum of grid index (kx, ky) in FFT order. */
void or_momentum(const or_grid* g, const or_units* u, const or_field* f, int32_t kx,
                 int32_t ky, double* pix, double* piy);

/* phi(p, 0) = u^s rho, inverse FFT, normalise sum |psi|^2 dx dy = 1. */
int or_init_packet(const or_units* u, const or_grid* g, const or_field* f,
                   const or_packet* pk, double* psi);
/* One potential half step in place: psi <- exp(-i tau V(t)/hbar) psi. */
int or_potential_step(const or_units* u, const or_grid* g, const or_field* f, double* psi,
                      double t, double tau);
/* Kinetic step in momentum space in place: phi <- K(dt) phi (includes the frame phase). */
int or_kinetic_step(const or_units* u, const or_grid* g, const or_field* f, double* phi,
                    double dt);
/* nsteps Strang steps from time t0. */
int or_step(const or_units* u, const or_grid* g, const or_field* f, double* psi, double t0,
            double dt, int64_t nsteps);
/* Observables of a position-space state at time t. */
int or_observe(const or_units* u, const or_grid* g, const or_field* f,
               const or_obs_spec* spec, const double* psi, double t, or_obs* out);
/* Per-cell momentum-space probabilities: out[ny][nx][3] = (|phi|^2, |c+|^2, |c-|^2). */
int or_momentum_density(const or_units* u, const or_grid* g, const or_field* f,
                        int32_t basis, const double* psi, double* out);
/* y-integrated density Phi(x) over the box (nx values). */
int or_density_x(const or_grid* g, const double* psi, double* out);

#ifdef __cplusplus
}
#endif
#endif
