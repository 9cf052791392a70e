/*
 * rtm_oracle.c — FP64 CPU oracle of the RTM path.  TEST INFRASTRUCTURE ONLY:
 * it is called by the tests, by the reference/CPU-baseline leg of the
 * benchmark and by the smoke check, never by the library.  It shares no code
 * with the CUDA path; both receive the same generated input arrays.
 *
 * Each function restates one step of "A workflow for seismic imaging with
 * quantified uncertainty" (arXiv 2001.06444) in the plainest form:
 *   - acoustic wave equation (§2.2, Eq. 4), discretised 2nd order in time and
 *     8th order in space (§3), the wavelet entering as the source term (§2.2);
 *   - reverse-time propagation as the exact discrete adjoint of that scheme
 *     (§3 credits an adjoint with guaranteed coercivity; the symmetric sponge
 *     placement below makes forward and adjoint the same recurrence);
 *   - source-normalised zero-lag cross-correlation imaging (§2.2, Eq. 5),
 *     per-shot normalisation, stacking over shots (§3, Fig. 2 caption) and the
 *     Laplacian filter on the brute stack (§3).
 * Readings where the paper is silent (sponge form and width, Laplacian sign and
 * border, eps, time origin) are the ones stated in the library header.
 *
 * Everything is FP64.  OpenMP (if enabled) only splits independent grid rows;
 * it never changes an arithmetic result.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int nx, nz, nb;
  double dx, dz, dt;
  int nt;
} or_grid;

/* 8th-order central second-derivative weights for offsets 0..4 (§3: "eighth
 * order in space"); the standard Fornberg values. */
static const double A8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0,
                             -1.0 / 560.0};
static const double SPONGE_ALPHA = 0.015;

typedef struct {
  int NZ, NX;
  double *c; /* (v dt)^2 on the padded grid */
  double *g; /* sponge factor g = g_x g_z   */
  double *h; /* sqrt(g)                      */
} or_model;

static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

/* 1D sponge factor at padded index I of a padded axis of length N. */
static double sponge1(int I, int N, int nb) {
  int k = I < N - 1 - I ? I : N - 1 - I; /* distance from the outer edge */
  if (k >= nb) return 1.0;
  double a = SPONGE_ALPHA * (double)(nb - k);
  return exp(-a * a);
}

static int model_setup(const or_grid *gr, const double *vel, or_model *m) {
  int NZ = gr->nz + 2 * gr->nb, NX = gr->nx + 2 * gr->nb;
  size_t n = (size_t)NZ * NX;
  m->NZ = NZ;
  m->NX = NX;
  m->c = (double *)malloc(n * sizeof(double));
  m->g = (double *)malloc(n * sizeof(double));
  m->h = (double *)malloc(n * sizeof(double));
  if (!m->c || !m->g || !m->h) return -1;
  for (int I = 0; I < NZ; ++I)
    for (int J = 0; J < NX; ++J) {
      /* velocity copied from the nearest physical cell into the sponge */
      int i = clampi(I - gr->nb, 0, gr->nz - 1);
      int j = clampi(J - gr->nb, 0, gr->nx - 1);
      double v = vel[(size_t)i * gr->nx + j];
      size_t p = (size_t)I * NX + J;
      m->c[p] = (v * gr->dt) * (v * gr->dt);
      m->g[p] = sponge1(I, NZ, gr->nb) * sponge1(J, NX, gr->nb);
      m->h[p] = sqrt(m->g[p]);
    }
  return 0;
}

static void model_free(or_model *m) {
  free(m->c);
  free(m->g);
  free(m->h);
}

/* L a on an NZ x NX grid, a taken as zero beyond the grid. */
static void laplacian8(const double *a, int NZ, int NX, double dz, double dx,
                       double *out) {
  double rz = 1.0 / (dz * dz), rx = 1.0 / (dx * dx);
#pragma omp parallel for schedule(static)
  for (int I = 0; I < NZ; ++I)
    for (int J = 0; J < NX; ++J) {
      double s = A8[0] * a[(size_t)I * NX + J] * (rz + rx);
      for (int m = 1; m <= 4; ++m) {
        double up = (I - m >= 0) ? a[(size_t)(I - m) * NX + J] : 0.0;
        double dn = (I + m < NZ) ? a[(size_t)(I + m) * NX + J] : 0.0;
        double lf = (J - m >= 0) ? a[(size_t)I * NX + (J - m)] : 0.0;
        double rt = (J + m < NX) ? a[(size_t)I * NX + (J + m)] : 0.0;
        s += A8[m] * ((up + dn) * rz + (lf + rt) * rx);
      }
      out[(size_t)I * NX + J] = s;
    }
}

/* One leapfrog update without source term:
 *   unew = h (2 h ucur + c L(h ucur)) - g^2 uold.  unew may alias uold. */
static void step(const or_model *m, const or_grid *gr, const double *ucur,
                 const double *uold, double *unew, double *hu, double *lap) {
  size_t n = (size_t)m->NZ * m->NX;
#pragma omp parallel for schedule(static)
  for (long p = 0; p < (long)n; ++p) hu[p] = m->h[p] * ucur[p];
  laplacian8(hu, m->NZ, m->NX, gr->dz, gr->dx, lap);
#pragma omp parallel for schedule(static)
  for (long p = 0; p < (long)n; ++p)
    unew[p] = m->h[p] * (2.0 * hu[p] + m->c[p] * lap[p]) - m->g[p] * m->g[p] * uold[p];
}

static size_t pidx(const or_grid *gr, int iz, int ix) {
  return (size_t)(iz + gr->nb) * (gr->nx + 2 * gr->nb) + (ix + gr->nb);
}

typedef struct {
  double *a, *b, *hu, *lap;
} or_work;

static int work_alloc(or_work *w, size_t n) {
  w->a = (double *)calloc(n, sizeof(double));
  w->b = (double *)calloc(n, sizeof(double));
  w->hu = (double *)malloc(n * sizeof(double));
  w->lap = (double *)malloc(n * sizeof(double));
  return (w->a && w->b && w->hu && w->lap) ? 0 : -1;
}
static void work_free(or_work *w) {
  free(w->a);
  free(w->b);
  free(w->hu);
  free(w->lap);
}

/* ---------------------------------------------------------------- model -- */

/* Forward modelling of one shot (Eq. 4 with the wavelet as source; the
 * `isotropicAcousticModeling` call of Listing 1).  seis[n][r] = u^{n+1}(r). */
int oracle_model(const or_grid *gr, const double *vel, int src_ix, int src_iz,
                 int nrec, const int *rec_ix, const int *rec_iz,
                 const double *wavelet, double *seis) {
  or_model m;
  if (model_setup(gr, vel, &m)) return -1;
  size_t n = (size_t)m.NZ * m.NX;
  or_work w;
  if (work_alloc(&w, n)) return -1;
  double *ucur = w.a, *uold = w.b; /* u^n, u^{n-1} */
  size_t ps = pidx(gr, src_iz, src_ix);
  for (int it = 0; it < gr->nt; ++it) {
    step(&m, gr, ucur, uold, uold, w.hu, w.lap); /* uold now holds u^{n+1} */
    uold[ps] += m.c[ps] * wavelet[it] / (gr->dx * gr->dz);
    for (int r = 0; r < nrec; ++r)
      seis[(size_t)it * nrec + r] = uold[pidx(gr, rec_iz[r], rec_ix[r])];
    double *t = ucur;
    ucur = uold;
    uold = t;
  }
  work_free(&w);
  model_free(&m);
  return 0;
}

/* Adjoint of oracle_model with respect to the wavelet: the backward
 * recurrence driven by seis, read at the source cell.
 * out[n] = w^{n+1}(source) / (dx dz), n = 0 .. nt-1. */
int oracle_adjoint_at_source(const or_grid *gr, const double *vel, int src_ix,
                             int src_iz, int nrec, const int *rec_ix,
                             const int *rec_iz, const double *seis, double *out) {
  or_model m;
  if (model_setup(gr, vel, &m)) return -1;
  size_t n = (size_t)m.NZ * m.NX;
  or_work w;
  if (work_alloc(&w, n)) return -1;
  double *wcur = w.a, *wold = w.b; /* w^{k+1}, w^{k+2} */
  size_t ps = pidx(gr, src_iz, src_ix);
  for (int k = gr->nt; k >= 1; --k) {
    step(&m, gr, wcur, wold, wold, w.hu, w.lap); /* wold now holds w^k */
    for (int r = 0; r < nrec; ++r) {
      size_t p = pidx(gr, rec_iz[r], rec_ix[r]);
      wold[p] += m.c[p] * seis[(size_t)(k - 1) * nrec + r];
    }
    out[k - 1] = wold[ps] / (gr->dx * gr->dz);
    double *t = wcur;
    wcur = wold;
    wold = t;
  }
  work_free(&w);
  model_free(&m);
  return 0;
}

/* ---------------------------------------------------- snapshot rounding -- */

/* Round y to the nearest value (ties to even) of a binary format with p
 * significant bits and smallest normal exponent emin (no overflow handling:
 * callers keep |y| within range). */
double oracle_round_format(double y, int p, int emin) {
  if (y == 0.0 || !isfinite(y)) return y;
  int e;
  frexp(y, &e); /* |y| = f 2^e, f in [0.5, 1) -> leading exponent e-1 */
  int E = e - 1 < emin ? emin : e - 1;
  double quantum = ldexp(1.0, E - p + 1);
  return nearbyint(y / quantum) * quantum;
}

/* Quantise-dequantise one snapshot of n values in place of out:
 * mode 0 exact; 1 BF16 with s = max|S|; 2 FP16 with s = max|S| / 2^15. */
void oracle_quantize_snapshot(const double *S, long n, int mode, double *out) {
  if (mode == 0) {
    memcpy(out, S, (size_t)n * sizeof(double));
    return;
  }
  double mx = 0.0;
  for (long i = 0; i < n; ++i) mx = fabs(S[i]) > mx ? fabs(S[i]) : mx;
  if (mx == 0.0) {
    memset(out, 0, (size_t)n * sizeof(double));
    return;
  }
  double s = (mode == 2) ? mx / 32768.0 : mx;
  int p = (mode == 2) ? 11 : 8;
  int emin = (mode == 2) ? -14 : -126;
  for (long i = 0; i < n; ++i) out[i] = oracle_round_format(S[i] / s, p, emin) * s;
}

/* ------------------------------------------------------------ migration -- */

/* Laplacian filter of §3 on an nz x nx image: -(D_zz + D_xx) with 3-point
 * second differences and the border value repeated outside the image. */
void oracle_image_filter(const double *img, int nz, int nx, double dz, double dx,
                         double *out) {
  for (int i = 0; i < nz; ++i)
    for (int j = 0; j < nx; ++j) {
      double c = img[(size_t)i * nx + j];
      double up = img[(size_t)clampi(i - 1, 0, nz - 1) * nx + j];
      double dn = img[(size_t)clampi(i + 1, 0, nz - 1) * nx + j];
      double lf = img[(size_t)i * nx + clampi(j - 1, 0, nx - 1)];
      double rt = img[(size_t)i * nx + clampi(j + 1, 0, nx - 1)];
      out[(size_t)i * nx + j] =
          -((up - 2.0 * c + dn) / (dz * dz) + (lf - 2.0 * c + rt) / (dx * dx));
    }
}

/* RTM of nshot shots over one model (Listing 1: forward modelling, then the
 * adjoint modelling with imaging, per shot; §3 Laplacian on the stack).
 * seis: [nshot][nt][nrec].  image: [nz][nx] (filtered if laplacian != 0).
 * num_out / den_out (nullable): per-shot raw cross-correlation and
 * illumination [nshot][nz][nx], before normalisation. */
int oracle_migrate(const or_grid *gr, const double *vel, int nshot,
                   const int *src_ix, const int *src_iz, int nrec,
                   const int *rec_ix, const int *rec_iz, const double *wavelet,
                   const double *seis, int isnap, int snap_mode, double eps,
                   int laplacian, double *image, double *num_out, double *den_out) {
  if (isnap < 1) return -2;
  or_model m;
  if (model_setup(gr, vel, &m)) return -1;
  size_t n = (size_t)m.NZ * m.NX;
  size_t npix = (size_t)gr->nz * gr->nx;
  int nsnap = gr->nt / isnap;
  double *snaps = (double *)malloc((nsnap > 0 ? nsnap : 1) * npix * sizeof(double));
  double *phys = (double *)malloc(npix * sizeof(double));
  double *num = (double *)malloc(npix * sizeof(double));
  double *den = (double *)malloc(npix * sizeof(double));
  double *stack = (double *)calloc(npix, sizeof(double));
  or_work w;
  if (!snaps || !phys || !num || !den || !stack || work_alloc(&w, n)) return -1;

  for (int s = 0; s < nshot; ++s) {
    /* forward: keep S^k = u^k for k in K (quantised if asked) */
    memset(w.a, 0, n * sizeof(double));
    memset(w.b, 0, n * sizeof(double));
    double *ucur = w.a, *uold = w.b;
    size_t ps = pidx(gr, src_iz[s], src_ix[s]);
    for (int it = 0; it < gr->nt; ++it) {
      step(&m, gr, ucur, uold, uold, w.hu, w.lap);
      uold[ps] += m.c[ps] * wavelet[it] / (gr->dx * gr->dz);
      int k = it + 1;
      if (k % isnap == 0) {
        for (int i = 0; i < gr->nz; ++i)
          for (int j = 0; j < gr->nx; ++j)
            phys[(size_t)i * gr->nx + j] = uold[pidx(gr, i, j)];
        oracle_quantize_snapshot(phys, (long)npix, snap_mode,
                                 snaps + (size_t)(k / isnap - 1) * npix);
      }
      double *t = ucur;
      ucur = uold;
      uold = t;
    }
    /* backward, imaging at k in K (Eq. 5 numerator and denominator) */
    memset(w.a, 0, n * sizeof(double));
    memset(w.b, 0, n * sizeof(double));
    memset(num, 0, npix * sizeof(double));
    memset(den, 0, npix * sizeof(double));
    double *wcur = w.a, *wold = w.b;
    const double *d = seis + (size_t)s * gr->nt * nrec;
    for (int k = gr->nt; k >= 1; --k) {
      step(&m, gr, wcur, wold, wold, w.hu, w.lap);
      for (int r = 0; r < nrec; ++r) {
        size_t p = pidx(gr, rec_iz[r], rec_ix[r]);
        wold[p] += m.c[p] * d[(size_t)(k - 1) * nrec + r];
      }
      if (k % isnap == 0) {
        const double *S = snaps + (size_t)(k / isnap - 1) * npix;
        for (int i = 0; i < gr->nz; ++i)
          for (int j = 0; j < gr->nx; ++j) {
            size_t q = (size_t)i * gr->nx + j;
            double Rv = wold[pidx(gr, i, j)];
            num[q] += S[q] * Rv;
            den[q] += S[q] * S[q];
          }
      }
      double *t = wcur;
      wcur = wold;
      wold = t;
    }
    double dmax = 0.0;
    for (size_t q = 0; q < npix; ++q) dmax = den[q] > dmax ? den[q] : dmax;
    /* a pixel with a zero denominator (never reached by the source
       wavefield, or no imaging step at all) contributes 0 */
    for (size_t q = 0; q < npix; ++q) {
      const double dd = den[q] + eps * dmax;
      stack[q] += dd > 0.0 ? num[q] / dd : 0.0;
    }
    if (num_out) memcpy(num_out + (size_t)s * npix, num, npix * sizeof(double));
    if (den_out) memcpy(den_out + (size_t)s * npix, den, npix * sizeof(double));
  }
  if (laplacian)
    oracle_image_filter(stack, gr->nz, gr->nx, gr->dz, gr->dx, image);
  else
    memcpy(image, stack, npix * sizeof(double));
  free(snaps);
  free(phys);
  free(num);
  free(den);
  free(stack);
  work_free(&w);
  model_free(&m);
  return 0;
}

/* Born (linearised) modelling whose transpose is the raw imaging numerator:
 * the background wavefield S^k of one shot scatters off the reflectivity
 * refl [nz][nx] at the imaging steps, dU^{n+1} = K dU^n - g^2 dU^{n-1}
 * + c refl S^{n+1} when n+1 is in K, and dU is recorded like oracle_model. */
int oracle_born(const or_grid *gr, const double *vel, int src_ix, int src_iz,
                int nrec, const int *rec_ix, const int *rec_iz,
                const double *wavelet, int isnap, const double *refl, double *seis) {
  or_model m;
  if (model_setup(gr, vel, &m)) return -1;
  size_t n = (size_t)m.NZ * m.NX;
  or_work w, dw;
  if (work_alloc(&w, n) || work_alloc(&dw, n)) return -1;
  double *ucur = w.a, *uold = w.b, *dcur = dw.a, *dold = dw.b;
  size_t ps = pidx(gr, src_iz, src_ix);
  for (int it = 0; it < gr->nt; ++it) {
    step(&m, gr, ucur, uold, uold, w.hu, w.lap); /* background u^{n+1} */
    uold[ps] += m.c[ps] * wavelet[it] / (gr->dx * gr->dz);
    step(&m, gr, dcur, dold, dold, dw.hu, dw.lap); /* perturbation */
    if ((it + 1) % isnap == 0)
      for (int i = 0; i < gr->nz; ++i)
        for (int j = 0; j < gr->nx; ++j) {
          size_t p = pidx(gr, i, j);
          dold[p] += m.c[p] * refl[(size_t)i * gr->nx + j] * uold[p];
        }
    for (int r = 0; r < nrec; ++r)
      seis[(size_t)it * nrec + r] = dold[pidx(gr, rec_iz[r], rec_ix[r])];
    double *t = ucur;
    ucur = uold;
    uold = t;
    t = dcur;
    dcur = dold;
    dold = t;
  }
  work_free(&w);
  work_free(&dw);
  model_free(&m);
  return 0;
}

/* ------------------------------------------------------------ utilities -- */

/* L a for a plain nz x nx field (zero outside), exposed for the stencil pins. */
void oracle_laplacian8(const double *a, int nz, int nx, double dz, double dx,
                       double *out) {
  laplacian8(a, nz, nx, dz, dx, out);
}

/* Courant number of the scheme: v dt sqrt((1/dx^2 + 1/dz^2) * 2048/315) / 2.
 * The scheme is stable for values <= 1 (§3: every RTM checks its CFL). */
double oracle_courant(double vmax, double dt, double dx, double dz) {
  double sym = 0.0; /* -(symbol of the 1D second-difference weights at pi) */
  for (int m = 0; m <= 4; ++m) sym += (m == 0 ? 1.0 : 2.0) * A8[m] * ((m % 2) ? -1.0 : 1.0);
  sym = -sym;
  return vmax * dt * sqrt((1.0 / (dx * dx) + 1.0 / (dz * dz)) * sym) / 2.0;
}

/* Number of threads the oracle's parallel loops use. */
int oracle_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Set the threads of the oracle's parallel loops (n >= 1). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* The padded-grid sponge factor g, exposed for tests: [NZ][NX]. */
int oracle_sponge(const or_grid *gr, double *g) {
  int NZ = gr->nz + 2 * gr->nb, NX = gr->nx + 2 * gr->nb;
  for (int I = 0; I < NZ; ++I)
    for (int J = 0; J < NX; ++J)
      g[(size_t)I * NX + J] = sponge1(I, NZ, gr->nb) * sponge1(J, NX, gr->nb);
  return 0;
}
