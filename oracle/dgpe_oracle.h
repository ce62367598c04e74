/*
 * FP64 CPU oracle for one split-step Crank-Nicolson (SSCN) step of the 3D dipolar
 * Gross-Pitaevskii equation.  TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check
 * and the benchmark's CPU-baseline leg call it; the CUDA library never links it and the
 * two share no code.
 *
 * The paper (arXiv 1610.05329, "Solution method") states the method only in words:
 * split-step Crank-Nicolson in imaginary or real time, with the dipolar term evaluated in
 * momentum space by the convolution theorem, for contact + dipolar interaction in an
 * anisotropic harmonic trap ("Nature of problem").  The equation, the kernel and the
 * discretisation below are the standard dimensionless dipolar GP model that this program
 * family solves; every reading the paper leaves open is marked [S#] and listed in the
 * design notes of the repository.
 *
 *   i dpsi/dt = [ -1/2 lap + V + g |psi|^2 + gdd Phi ] psi,
 *   V = 1/2 (nux^2 x^2 + nuy^2 y^2 + nuz^2 z^2)                            [S1]
 *   Phi = IDFT[ Ut(k) DFT(|psi|^2) ],  Ut(k) = 3 kz^2/|k|^2 - 1, Ut(0) = 0  [S2-S4, S8, S9]
 *   x_i = (i - N/2) h,  k_m = 2 pi m / (N h), m signed                     [S6, S7]
 *
 * One step (Lie splitting, "potential, then kinetic x, y, z")              [S10, S11]
 *   1. theta = dt (V + g n + gdd Phi), n = |psi|^2 of the incoming state;
 *      real time psi *= exp(-i theta), imaginary time psi *= exp(-theta).
 *   2. for d = x, y, z: Crank-Nicolson (1 - c D) psi' = (1 + c D) psi on every line, with
 *      D the 3-point second difference, Dirichlet walls psi = 0 at index 0 and N-1 [S12],
 *      c = i dt/(4 h^2) (real time) or dt/(4 h^2) (imaginary time); Thomas algorithm.
 *   3. imaginary time only: psi /= sqrt(norm), norm = hx hy hz sum |psi|^2   [S13]
 *
 * Complex arrays are C99 double complex, row-major [nx][ny][nz] (z fastest).
 */
#ifndef DGPE_ORACLE_H
#define DGPE_ORACLE_H
#include <complex.h>

#define ORC_REAL_TIME 0
#define ORC_IMAG_TIME 1

typedef struct {
  int nx, ny, nz;
  double hx, hy, hz;
  double dt;
  int mode;            /* ORC_REAL_TIME or ORC_IMAG_TIME */
  double nu[3];        /* trap frequencies nu_x, nu_y, nu_z */
  double g, gdd;       /* contact and dipolar strengths */
  double cutoff;       /* spherical cutoff radius R of the dipolar interaction; <= 0: none */
  int integration;     /* 0: rectangle rule [S13]; 1: composite Simpson on indices 0..N-2 */
  int kinetic;         /* 0: E_kin = h^3 sum 1/2 Re conj(psi)(-lap psi), 3-point Laplacian [S14];
                          1: E_kin = h^3 sum 1/2 |grad psi|^2, 5-point 4th-order gradient */
} orc_params;

typedef struct {
  double norm;         /* hx hy hz sum |psi|^2 */
  double mu;           /* chemical potential (divided by norm) */
  double energy;       /* energy functional */
  double rms[3];       /* sqrt(<d^2>), d = x, y, z */
  double e_kin, e_trap, e_contact, e_dipolar;  /* the four energy terms (sum = energy) */
} orc_obs;

int orc_num_threads(void);

/* 1D transforms, unnormalised, sign = -1 forward, +1 inverse.  In place. */
void orc_fft(double complex *x, int n, int sign);   /* recursive mixed-radix Cooley-Tukey */
void orc_dft(double complex *x, int n, int sign);   /* naive O(n^2) definition */
/* 3D transform of a [nx][ny][nz] array (unnormalised), built from orc_fft along each axis. */
void orc_fft3(double complex *x, int nx, int ny, int nz, int sign);

/* Momentum-space dipolar kernel Ut on the full [nx][ny][nz] FFT grid.  With a spherical
 * cutoff R > 0 (the interaction restricted to r < R), Ut is multiplied by
 * c(kR) = 1 + 3 cos(kR)/(kR)^2 - 3 sin(kR)/(kR)^3 = 3 int_0^{kR} j_2(x)/x dx. */
double orc_cutoff_factor(double x);
void orc_dipolar_kernel(const orc_params *p, double *ut);
/* Phi = Re IDFT[ Ut DFT(n) ] for a real density n.  Uses orc_fft3. */
void orc_dipolar_phi(const orc_params *p, const double *n, double *phi);
/* Same Phi by brute force: K = naive IDFT of Ut, then direct circular convolution.
 * O(Ntot^2); meant for grids of at most a few hundred points. */
void orc_dipolar_phi_direct(const orc_params *p, const double *n, double *phi);

/* Thomas algorithm for a general complex tridiagonal system
 *   lo[i] x[i-1] + di[i] x[i] + up[i] x[i+1] = rhs[i], i = 0..n-1  (lo[0], up[n-1] unused). */
void orc_thomas(int n, const double complex *lo, const double complex *di,
                const double complex *up, const double complex *rhs, double complex *x);

/* Sub-steps of the SSCN step, applied in place. axis: 0 = x, 1 = y, 2 = z.
 * p->dt may be negative: in real time that gives the inverse of each sub-step. */
void orc_potential_step(const orc_params *p, double complex *psi);
void orc_cn_sweep(const orc_params *p, double complex *psi, int axis);
/* Full steps: potential, CN x, CN y, CN z, then renormalisation in imaginary time. */
void orc_step(const orc_params *p, double complex *psi, int nsteps);
void orc_observables(const orc_params *p, const double complex *psi, orc_obs *o);
/* hx hy hz sum w |psi|^2 with the quadrature weights of p->integration. */
double orc_norm(const orc_params *p, const double complex *psi);

/* Discrete adjoint of one real-time step (paper's method differentiated by hand; the
 * paper itself has no adjoint).  Real-valued loss L, cotangent gbar = 2 dL/d conj(psi), so
 * that dL = Re sum conj(gbar) dpsi.  On entry gbar is the cotangent of the step's output,
 * psi_k the step's input; on exit gbar is the cotangent of psi_k and
 *   grads[0] += dL/dg,  grads[1] += dL/dgdd,  grads[2] += dL/dnu_z
 * (the step's own contribution; nu_z of p). */
void orc_adjoint_step(const orc_params *p, const double complex *psi_k, double complex *gbar, double *grads);

/* L = hx hy hz sum z^2 |psi_N|^2 after nseg * steps_per_seg real-time steps from psi0, with
 * nu_z = nu_z[s] during segment s (the other parameters from p), and its gradient by the
 * adjoint: dnu[s] = dL/dnu_z[s], dg = dL/dg, dgdd = dL/dgdd.  Keeps every state in memory
 * (meant for small grids). */
void orc_grad_z2(const orc_params *p, int nseg, int steps_per_seg, const double *nu_z,
                 const double complex *psi0, double *loss, double *dnu, double *dg, double *dgdd);

#endif
