/*
 * FP64 CPU oracle of the SSCN step of the 3D dipolar GP equation.  TEST INFRASTRUCTURE:
 * used only by the tests, the smoke check and the benchmark's CPU baseline.
 * See dgpe_oracle.h for the equation and the readings [S#] it follows.
 *
 * Written to be read against the mathematics, not to be fast: every transform is the
 * textbook recursive Cooley-Tukey, every tridiagonal solve factors its own matrix, and
 * OpenMP only splits independent lines/points between threads.
 */
#include "dgpe_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* exp(sign * 2 pi i j / n), the DFT root of unity, with j reduced mod n first. */
static double complex root(long j, int n, int sign) {
  j %= n;
  if (j < 0) j += n;
  double a = sign * TWO_PI * (double)j / (double)n;
  return cos(a) + I * sin(a);
}

static int smallest_factor(int n) {
  for (int p = 2; p * p <= n; ++p)
    if (n % p == 0) return p;
  return n;
}

/* Table of the n-th roots of unity w^j = exp(sign 2 pi i j / n), j = 0..n-1. */
static double complex *root_table(int n, int sign) {
  double complex *w = malloc(sizeof(double complex) * n);
  for (int j = 0; j < n; ++j) w[j] = root(j, n, sign);
  return w;
}

/* Decimation in time: out[k] = sum_m in[m*stride] w_n^(m k), w_n = exp(sign 2 pi i / n).
 * Split m = p*m2 + q (p = smallest prime factor of n), transform the p subsequences
 * recursively, then combine X[k + (n/p) s] = sum_q w_n^(q (k + (n/p) s)) Y_q[k].
 * tw holds the roots of the top-level size ntop; w_n^e = tw[(e mod n) * (ntop / n)]. */
static void fft_rec(const double complex *in, double complex *out, int n, long stride,
                    const double complex *tw, int ntop) {
  if (n == 1) {
    out[0] = in[0];
    return;
  }
  int p = smallest_factor(n);
  int n2 = n / p;
  long tstep = ntop / n;
  for (int q = 0; q < p; ++q) fft_rec(in + (long)q * stride, out + (long)q * n2, n2, stride * p, tw, ntop);
  double complex y[64];
  double complex *yv = (p <= 64) ? y : malloc(sizeof(double complex) * p);
  for (int k = 0; k < n2; ++k) {
    for (int q = 0; q < p; ++q) yv[q] = out[(long)q * n2 + k];
    for (int s = 0; s < p; ++s) {
      double complex acc = 0;
      for (int q = 0; q < p; ++q) acc += tw[(((long)q * (k + (long)n2 * s)) % n) * tstep] * yv[q];
      out[(long)s * n2 + k] = acc;
    }
  }
  if (yv != y) free(yv);
}

void orc_fft(double complex *x, int n, int sign) {
  double complex *tmp = malloc(sizeof(double complex) * n);
  double complex *tw = root_table(n, sign);
  fft_rec(x, tmp, n, 1, tw, n);
  memcpy(x, tmp, sizeof(double complex) * n);
  free(tw);
  free(tmp);
}

void orc_dft(double complex *x, int n, int sign) {
  double complex *out = malloc(sizeof(double complex) * n);
  for (int k = 0; k < n; ++k) {
    double complex acc = 0;
    for (int j = 0; j < n; ++j) acc += root((long)j * k, n, sign) * x[j];
    out[k] = acc;
  }
  memcpy(x, out, sizeof(double complex) * n);
  free(out);
}

/* Apply orc_fft to every line of the array along one axis. */
static void fft_axis(double complex *x, int nx, int ny, int nz, int axis, int sign) {
  int n = axis == 0 ? nx : axis == 1 ? ny : nz;
  long stride = axis == 0 ? (long)ny * nz : axis == 1 ? nz : 1;
  long nlines = (long)nx * ny * nz / n;
#pragma omp parallel
  {
    double complex *line = malloc(sizeof(double complex) * n);
#pragma omp for schedule(static)
    for (long l = 0; l < nlines; ++l) {
      long base;
      if (axis == 0) base = l;                                   /* l = j*nz + k */
      else if (axis == 1) base = (l / nz) * (long)ny * nz + l % nz; /* l = i*nz + k */
      else base = l * nz;                                        /* l = i*ny + j */
      for (int m = 0; m < n; ++m) line[m] = x[base + m * stride];
      orc_fft(line, n, sign);
      for (int m = 0; m < n; ++m) x[base + m * stride] = line[m];
    }
    free(line);
  }
}

void orc_fft3(double complex *x, int nx, int ny, int nz, int sign) {
  fft_axis(x, nx, ny, nz, 2, sign);
  fft_axis(x, nx, ny, nz, 1, sign);
  fft_axis(x, nx, ny, nz, 0, sign);
}

/* Signed wavenumber of FFT index m on a grid of n points with spacing h [S7]. */
static double wavenumber(int m, int n, double h) {
  int ms = (m <= n / 2) ? m : m - n;
  return TWO_PI * (double)ms / ((double)n * h);
}

/* c(x) = 1 + 3 cos x / x^2 - 3 sin x / x^3; below x = 0.5 its Taylor series
 * sum_{n>=2} (-1)^n 6n x^(2n-2) / (2n+1)! (the closed form cancels there). */
double orc_cutoff_factor(double x) {
  if (x >= 0.5) return 1.0 + 3.0 * cos(x) / (x * x) - 3.0 * sin(x) / (x * x * x);
  double sum = 0, fact = 120.0; /* (2n+1)! for n = 2 */
  double xp = x * x;            /* x^(2n-2) for n = 2 */
  for (int n = 2; n <= 12; ++n) {
    sum += ((n % 2) ? -1.0 : 1.0) * 6.0 * n * xp / fact;
    fact *= (2.0 * n + 2.0) * (2.0 * n + 3.0);
    xp *= x * x;
  }
  return sum;
}

/* Ut(k) = 3 kz^2 / |k|^2 - 1 (dipoles along z), Ut(0) = 0 [S2, S3, S4]; optional cutoff [S5]. */
void orc_dipolar_kernel(const orc_params *p, double *ut) {
  for (int i = 0; i < p->nx; ++i)
    for (int j = 0; j < p->ny; ++j)
      for (int k = 0; k < p->nz; ++k) {
        double kx = wavenumber(i, p->nx, p->hx);
        double ky = wavenumber(j, p->ny, p->hy);
        double kz = wavenumber(k, p->nz, p->hz);
        double k2 = kx * kx + ky * ky + kz * kz;
        double u = (k2 == 0.0) ? 0.0 : 3.0 * kz * kz / k2 - 1.0;
        if (p->cutoff > 0 && k2 > 0.0) u *= orc_cutoff_factor(sqrt(k2) * p->cutoff);
        ut[((long)i * p->ny + j) * p->nz + k] = u;
      }
}

/* Convolution theorem [S8, S9]: Phi = IDFT(Ut * DFT(n)), IDFT normalised by 1/Ntot. */
void orc_dipolar_phi(const orc_params *p, const double *n, double *phi) {
  long ntot = (long)p->nx * p->ny * p->nz;
  double complex *f = malloc(sizeof(double complex) * ntot);
  double *ut = malloc(sizeof(double) * ntot);
  for (long q = 0; q < ntot; ++q) f[q] = n[q];
  orc_fft3(f, p->nx, p->ny, p->nz, -1);
  orc_dipolar_kernel(p, ut);
  for (long q = 0; q < ntot; ++q) f[q] *= ut[q];
  orc_fft3(f, p->nx, p->ny, p->nz, +1);
  for (long q = 0; q < ntot; ++q) phi[q] = creal(f[q]) / (double)ntot;
  free(f);
  free(ut);
}

/* Brute force: the real-space kernel K(r) = (1/Ntot) sum_k Ut(k) e^{+i k.r} by the naive
 * 3D sum, then Phi(r) = sum_r' K(r - r') n(r') with periodic wrap of the index difference. */
void orc_dipolar_phi_direct(const orc_params *p, const double *n, double *phi) {
  int nx = p->nx, ny = p->ny, nz = p->nz;
  long ntot = (long)nx * ny * nz;
  double *ut = malloc(sizeof(double) * ntot);
  double *kr = malloc(sizeof(double) * ntot);
  orc_dipolar_kernel(p, ut);
  for (int a = 0; a < nx; ++a)
    for (int b = 0; b < ny; ++b)
      for (int c = 0; c < nz; ++c) {
        double complex acc = 0;
        for (int i = 0; i < nx; ++i)
          for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k)
              acc += ut[((long)i * ny + j) * nz + k] * root((long)i * a, nx, +1) *
                     root((long)j * b, ny, +1) * root((long)k * c, nz, +1);
        kr[((long)a * ny + b) * nz + c] = creal(acc) / (double)ntot;
      }
  for (int a = 0; a < nx; ++a)
    for (int b = 0; b < ny; ++b)
      for (int c = 0; c < nz; ++c) {
        double acc = 0;
        for (int i = 0; i < nx; ++i)
          for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
              int di = ((a - i) % nx + nx) % nx, dj = ((b - j) % ny + ny) % ny, dk = ((c - k) % nz + nz) % nz;
              acc += kr[((long)di * ny + dj) * nz + dk] * n[((long)i * ny + j) * nz + k];
            }
        phi[((long)a * ny + b) * nz + c] = acc;
      }
  free(ut);
  free(kr);
}

/* Thomas algorithm: forward elimination, then back substitution (no pivoting; the CN
 * matrices are strictly diagonally dominant). */
void orc_thomas(int n, const double complex *lo, const double complex *di,
                const double complex *up, const double complex *rhs, double complex *x) {
  double complex *cp = malloc(sizeof(double complex) * n);
  double complex *dp = malloc(sizeof(double complex) * n);
  cp[0] = up[0] / di[0];
  dp[0] = rhs[0] / di[0];
  for (int i = 1; i < n; ++i) {
    double complex m = di[i] - lo[i] * cp[i - 1];
    cp[i] = (i < n - 1) ? up[i] / m : 0;
    dp[i] = (rhs[i] - lo[i] * dp[i - 1]) / m;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
}

static double coord(int i, int n, double h) { return ((double)i - (double)(n / 2)) * h; }

static double trap(const orc_params *p, int i, int j, int k) {
  double x = coord(i, p->nx, p->hx), y = coord(j, p->ny, p->hy), z = coord(k, p->nz, p->hz);
  return 0.5 * (p->nu[0] * p->nu[0] * x * x + p->nu[1] * p->nu[1] * y * y + p->nu[2] * p->nu[2] * z * z);
}

/* Non-derivative part [S11]: n and Phi of the incoming state, then the exact exponential. */
void orc_potential_step(const orc_params *p, double complex *psi) {
  long ntot = (long)p->nx * p->ny * p->nz;
  double *n = malloc(sizeof(double) * ntot);
  double *phi = malloc(sizeof(double) * ntot);
  for (long q = 0; q < ntot; ++q) n[q] = creal(psi[q]) * creal(psi[q]) + cimag(psi[q]) * cimag(psi[q]);
  orc_dipolar_phi(p, n, phi);
#pragma omp parallel for collapse(2) schedule(static)
  for (int i = 0; i < p->nx; ++i)
    for (int j = 0; j < p->ny; ++j)
      for (int k = 0; k < p->nz; ++k) {
        long q = ((long)i * p->ny + j) * p->nz + k;
        double theta = p->dt * (trap(p, i, j, k) + p->g * n[q] + p->gdd * phi[q]);
        if (p->mode == ORC_REAL_TIME) psi[q] *= cexp(-I * theta);
        else psi[q] *= exp(-theta);
      }
  free(n);
  free(phi);
}

/* Crank-Nicolson along one axis [S12]: (1 - c D) psi' = (1 + c D) psi on the interior
 * points 1..N-2 of every line, D the 3-point second difference with psi = 0 on both walls
 * (old and new), c = i dt/(4 h^2) in real time and dt/(4 h^2) in imaginary time. */
void orc_cn_sweep(const orc_params *p, double complex *psi, int axis) {
  int nx = p->nx, ny = p->ny, nz = p->nz;
  int n = axis == 0 ? nx : axis == 1 ? ny : nz;
  double h = axis == 0 ? p->hx : axis == 1 ? p->hy : p->hz;
  long stride = axis == 0 ? (long)ny * nz : axis == 1 ? nz : 1;
  long nlines = (long)nx * ny * nz / n;
  double r = p->dt / (4.0 * h * h);
  double complex c = (p->mode == ORC_REAL_TIME) ? I * r : r;
  int m = n - 2; /* interior unknowns */
#pragma omp parallel
  {
    double complex *line = malloc(sizeof(double complex) * n);
    double complex *lo = malloc(sizeof(double complex) * n), *di = malloc(sizeof(double complex) * n);
    double complex *up = malloc(sizeof(double complex) * n), *rhs = malloc(sizeof(double complex) * n);
    double complex *sol = malloc(sizeof(double complex) * n);
#pragma omp for schedule(static)
    for (long l = 0; l < nlines; ++l) {
      long base;
      if (axis == 0) base = l;
      else if (axis == 1) base = (l / nz) * (long)ny * nz + l % nz;
      else base = l * nz;
      for (int t = 0; t < n; ++t) line[t] = psi[base + t * stride];
      line[0] = 0;
      line[n - 1] = 0;
      for (int t = 0; t < m; ++t) {
        int i = t + 1; /* grid index of unknown t */
        lo[t] = -c;
        di[t] = 1.0 + 2.0 * c;
        up[t] = -c;
        rhs[t] = line[i] + c * (line[i - 1] - 2.0 * line[i] + line[i + 1]);
      }
      if (m > 0) orc_thomas(m, lo, di, up, rhs, sol);
      psi[base] = 0;
      psi[base + (n - 1) * stride] = 0;
      for (int t = 0; t < m; ++t) psi[base + (t + 1) * stride] = sol[t];
    }
    free(line); free(lo); free(di); free(up); free(rhs); free(sol);
  }
}

/* Quadrature weight of grid index i on an axis of n points (times h): 1 for the rectangle
 * rule [S13]; composite Simpson (1, 4, 2, 4, ..., 4, 1)/3 on indices 0..n-2 (n - 2
 * intervals, n even) and 0 on the last point, a wall. */
static double quad_weight(const orc_params *p, int i, int n) {
  if (p->integration == 0) return 1.0;
  if (i > n - 2) return 0.0;
  if (i == 0 || i == n - 2) return 1.0 / 3.0;
  return (i % 2) ? 4.0 / 3.0 : 2.0 / 3.0;
}

static double grid_norm(const orc_params *p, const double complex *psi) {
  double s = 0;
  for (int i = 0; i < p->nx; ++i)
    for (int j = 0; j < p->ny; ++j)
      for (int k = 0; k < p->nz; ++k) {
        long q = ((long)i * p->ny + j) * p->nz + k;
        double w = quad_weight(p, i, p->nx) * quad_weight(p, j, p->ny) * quad_weight(p, k, p->nz);
        s += w * (creal(psi[q]) * creal(psi[q]) + cimag(psi[q]) * cimag(psi[q]));
      }
  return s * p->hx * p->hy * p->hz;
}

double orc_norm(const orc_params *p, const double complex *psi) { return grid_norm(p, psi); }

void orc_step(const orc_params *p, double complex *psi, int nsteps) {
  long ntot = (long)p->nx * p->ny * p->nz;
  for (int s = 0; s < nsteps; ++s) {
    orc_potential_step(p, psi);
    orc_cn_sweep(p, psi, 0);
    orc_cn_sweep(p, psi, 1);
    orc_cn_sweep(p, psi, 2);
    if (p->mode == ORC_IMAG_TIME) {
      double inv = 1.0 / sqrt(grid_norm(p, psi));
      for (long q = 0; q < ntot; ++q) psi[q] *= inv;
    }
  }
}

/* Discrete observables [S14] with the same 3-point Laplacian (zero outside the grid), or
 * with the 5-point first derivative (f(i-2) - 8 f(i-1) + 8 f(i+1) - f(i+2)) / (12 h); sums
 * weighted by the quadrature rule. */
void orc_observables(const orc_params *p, const double complex *psi, orc_obs *o) {
  int nx = p->nx, ny = p->ny, nz = p->nz;
  long ntot = (long)nx * ny * nz;
  long sx_ = (long)ny * nz, sy_ = nz;
  double dv = p->hx * p->hy * p->hz;
  double *n = malloc(sizeof(double) * ntot);
  double *phi = malloc(sizeof(double) * ntot);
  for (long q = 0; q < ntot; ++q) n[q] = creal(psi[q]) * creal(psi[q]) + cimag(psi[q]) * cimag(psi[q]);
  orc_dipolar_phi(p, n, phi);
  double sn = 0, skin = 0, strap = 0, sint = 0, sdd = 0, sx = 0, sy = 0, sz = 0;
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j)
      for (int k = 0; k < nz; ++k) {
        long q = ((long)i * ny + j) * nz + k;
        double w = quad_weight(p, i, nx) * quad_weight(p, j, ny) * quad_weight(p, k, nz);
        double complex c = psi[q];
#define AT(di, dj, dk)                                                                          \
  ((i + (di) >= 0 && i + (di) < nx && j + (dj) >= 0 && j + (dj) < ny && k + (dk) >= 0 && k + (dk) < nz) \
       ? psi[q + (di) * sx_ + (dj) * sy_ + (dk)]                                                \
       : 0)
        double ekin;
        if (p->kinetic == 0) {
          double complex lap = (AT(-1, 0, 0) - 2.0 * c + AT(1, 0, 0)) / (p->hx * p->hx) +
                               (AT(0, -1, 0) - 2.0 * c + AT(0, 1, 0)) / (p->hy * p->hy) +
                               (AT(0, 0, -1) - 2.0 * c + AT(0, 0, 1)) / (p->hz * p->hz);
          ekin = 0.5 * creal(conj(c) * (-lap));
        } else {
          double complex gx = (AT(-2, 0, 0) - 8.0 * AT(-1, 0, 0) + 8.0 * AT(1, 0, 0) - AT(2, 0, 0)) / (12.0 * p->hx);
          double complex gy = (AT(0, -2, 0) - 8.0 * AT(0, -1, 0) + 8.0 * AT(0, 1, 0) - AT(0, 2, 0)) / (12.0 * p->hy);
          double complex gz = (AT(0, 0, -2) - 8.0 * AT(0, 0, -1) + 8.0 * AT(0, 0, 1) - AT(0, 0, 2)) / (12.0 * p->hz);
          ekin = 0.5 * (creal(gx * conj(gx)) + creal(gy * conj(gy)) + creal(gz * conj(gz)));
        }
#undef AT
        double x = coord(i, nx, p->hx), y = coord(j, ny, p->hy), z = coord(k, nz, p->hz);
        sn += w * n[q];
        skin += w * ekin;
        strap += w * trap(p, i, j, k) * n[q];
        sint += w * p->g * n[q] * n[q];
        sdd += w * p->gdd * phi[q] * n[q];
        sx += w * x * x * n[q];
        sy += w * y * y * n[q];
        sz += w * z * z * n[q];
      }
  o->norm = dv * sn;
  o->e_kin = dv * skin;
  o->e_trap = dv * strap;
  o->e_contact = 0.5 * dv * sint;
  o->e_dipolar = 0.5 * dv * sdd;
  o->energy = o->e_kin + o->e_trap + o->e_contact + o->e_dipolar;
  o->mu = dv * (skin + strap + sint + sdd) / o->norm;
  o->rms[0] = sqrt(sx / sn);
  o->rms[1] = sqrt(sy / sn);
  o->rms[2] = sqrt(sz / sn);
  free(n);
  free(phi);
}

/* ---------------------------------------------------------------------------------------
 * Adjoint of one real-time step psi' = Z Y X P(psi) (oracle order: potential, x, y, z).
 *  - Each Crank-Nicolson sweep C = (1 - cD)^{-1}(1 + cD) is complex symmetric, so its adjoint
 *    is conj(C): the same sweep with c -> conj(c), i.e. dt -> -dt.
 *  - The potential step P(psi) = e^{-i theta} psi, theta = dt (V + g n + gdd Phi[n]),
 *    n = |psi|^2: with s = Im(conj(gbar1) P(psi)),
 *      gbar = e^{+i theta} gbar1 + 2 dt (g s + gdd Phi[s]) psi
 *    (Phi is a convolution with a real even kernel, hence self-adjoint), and
 *      dL/dg = dt sum s n, dL/dgdd = dt sum s Phi[n], dL/dnu_z = dt sum s nu_z z^2.
 * --------------------------------------------------------------------------------------- */
void orc_adjoint_step(const orc_params *p, const double complex *psi_k, double complex *gbar, double *grads) {
  long ntot = (long)p->nx * p->ny * p->nz;
  orc_params back = *p;
  back.dt = -p->dt;
  /* sweeps in reverse order, each adjoint = the sweep with -dt */
  orc_cn_sweep(&back, gbar, 2);
  orc_cn_sweep(&back, gbar, 1);
  orc_cn_sweep(&back, gbar, 0);
  /* potential step */
  double *n = malloc(sizeof(double) * ntot), *phin = malloc(sizeof(double) * ntot);
  double *sf = malloc(sizeof(double) * ntot), *phis = malloc(sizeof(double) * ntot);
  for (long q = 0; q < ntot; ++q) n[q] = creal(psi_k[q]) * creal(psi_k[q]) + cimag(psi_k[q]) * cimag(psi_k[q]);
  orc_dipolar_phi(p, n, phin);
  double sg = 0, sdd = 0, snu = 0;
  for (int i = 0; i < p->nx; ++i)
    for (int j = 0; j < p->ny; ++j)
      for (int k = 0; k < p->nz; ++k) {
        long q = ((long)i * p->ny + j) * p->nz + k;
        double theta = p->dt * (trap(p, i, j, k) + p->g * n[q] + p->gdd * phin[q]);
        double complex out = psi_k[q] * cexp(-I * theta);          /* P(psi) */
        double sv = cimag(conj(gbar[q]) * out);
        double z = coord(k, p->nz, p->hz);
        sf[q] = sv;
        sg += sv * n[q];
        sdd += sv * phin[q];
        snu += sv * p->nu[2] * z * z;
        gbar[q] = gbar[q] * cexp(I * theta);
      }
  orc_dipolar_phi(p, sf, phis);
  for (long q = 0; q < ntot; ++q) gbar[q] += 2.0 * p->dt * (p->g * sf[q] + p->gdd * phis[q]) * psi_k[q];
  grads[0] += p->dt * sg;
  grads[1] += p->dt * sdd;
  grads[2] += p->dt * snu;
  free(n); free(phin); free(sf); free(phis);
}

void orc_grad_z2(const orc_params *p, int nseg, int steps_per_seg, const double *nu_z,
                 const double complex *psi0, double *loss, double *dnu, double *dg, double *dgdd) {
  long ntot = (long)p->nx * p->ny * p->nz;
  int nsteps = nseg * steps_per_seg;
  double complex *states = malloc(sizeof(double complex) * ntot * (nsteps + 1));
  memcpy(states, psi0, sizeof(double complex) * ntot);
  orc_params q = *p;
  q.mode = ORC_REAL_TIME;
  for (int t = 0; t < nsteps; ++t) {
    q.nu[2] = nu_z[t / steps_per_seg];
    memcpy(states + (long)(t + 1) * ntot, states + (long)t * ntot, sizeof(double complex) * ntot);
    orc_step(&q, states + (long)(t + 1) * ntot, 1);
  }
  const double complex *last = states + (long)nsteps * ntot;
  double dv = p->hx * p->hy * p->hz, l = 0;
  double complex *gbar = malloc(sizeof(double complex) * ntot);
  for (int i = 0; i < p->nx; ++i)
    for (int j = 0; j < p->ny; ++j)
      for (int k = 0; k < p->nz; ++k) {
        long idx = ((long)i * p->ny + j) * p->nz + k;
        double z = coord(k, p->nz, p->hz);
        double nn = creal(last[idx]) * creal(last[idx]) + cimag(last[idx]) * cimag(last[idx]);
        l += dv * z * z * nn;
        gbar[idx] = 2.0 * dv * z * z * last[idx];     /* 2 dL/d conj(psi_N) */
      }
  *loss = l;
  *dg = 0;
  *dgdd = 0;
  for (int s = 0; s < nseg; ++s) dnu[s] = 0;
  for (int t = nsteps - 1; t >= 0; --t) {
    double gr[3] = {0, 0, 0};
    q.nu[2] = nu_z[t / steps_per_seg];
    orc_adjoint_step(&q, states + (long)t * ntot, gbar, gr);
    *dg += gr[0];
    *dgdd += gr[1];
    dnu[t / steps_per_seg] += gr[2];
  }
  free(gbar);
  free(states);
}
