/*
 * Oracle — test infrastructure only.  Plain FP64 Ewald summation of the periodic
 * Coulomb kernel used by the paper's charge-scaled Hamiltonian (Eq. for H~,
 * "scaled_electrostatics", and the periodic sum of Eq. "nbody_periodic").
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load this library.  It shares no code with the GPU path.
 *
 * Reading of the paper (it prints no formula for the periodic kernel): the
 * periodic sum over images with tin-foil boundary conditions at infinity and a
 * uniform neutralising background (the paper asks for energies that match Ewald
 * methods, Sec. "Multipole-Accelerated Hamiltonian Interpolation").  For charges
 * q_j at x_j in a cubic box of edge L, volume V:
 *
 *   A(r) = sum_n erfc(a|r+nL|)/|r+nL| + (4 pi / V) sum_{k!=0} exp(-k^2/4a^2) cos(k.r)/k^2
 *          - pi/(a^2 V),                                   k = 2 pi m / L
 *   A(0) = xi = lim_{r->0} [A(r) - 1/r]   (self-image term; only i=j, n=0 is omitted)
 *   phi_i = sum_j q_j A(x_i - x_j)      (j = i contributes q_i xi)
 *   E     = 1/2 sum_i q_i phi_i,        grad phi_i excludes the j = i term
 *
 * All results here are in units with the Coulomb constant f = 1 (e/nm, e^2/nm);
 * the Python side multiplies by f.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288
#define OR_2_SQRTPI 1.12837916709551257389615890312154517

/* Neumaier compensated summation */
typedef struct { double s, c; } ksum_t;
static inline void kadd(ksum_t *k, double v) {
  double t = k->s + v;
  if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v; else k->c += (v - t) + k->s;
  k->s = t;
}
static inline double kval(const ksum_t *k) { return k->s + k->c; }

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Parameters: erfc(alpha rc) <= ~1e-16 and exp(-k^2/4alpha^2) <= ~1e-16 at k_max. */
void oracle_ewald_params(double L, double rc, double *alpha, int *mmax) {
  double a = 6.0 / rc;                    /* erfc(6) = 2.2e-17 */
  double kmax = 2.0 * a * sqrt(37.0);     /* exp(-37) = 8.5e-17 */
  *alpha = a;
  *mmax = (int)ceil(kmax * L / (2.0 * OR_PI));
}

/* ---- reciprocal-space vectors: half space, |m| <= mmax ---- */
typedef struct { int n; double *kx, *ky, *kz, *c; int *mx, *my, *mz; } kset_t;

static void kset_build(kset_t *ks, double L, double alpha, int mmax) {
  int side = 2 * mmax + 1;
  long cap = (long)side * side * side / 2 + 1;
  ks->kx = malloc(cap * sizeof(double)); ks->ky = malloc(cap * sizeof(double));
  ks->kz = malloc(cap * sizeof(double)); ks->c = malloc(cap * sizeof(double));
  ks->mx = malloc(cap * sizeof(int)); ks->my = malloc(cap * sizeof(int)); ks->mz = malloc(cap * sizeof(int));
  ks->n = 0;
  double V = L * L * L, tw = 2.0 * OR_PI / L;
  for (int mx = 0; mx <= mmax; ++mx)
    for (int my = -mmax; my <= mmax; ++my)
      for (int mz = -mmax; mz <= mmax; ++mz) {
        if (mx == 0 && (my < 0 || (my == 0 && mz <= 0))) continue;  /* half space, m != 0 */
        if (mx * mx + my * my + mz * mz > mmax * mmax) continue;
        double kx = tw * mx, ky = tw * my, kz = tw * mz, k2 = kx * kx + ky * ky + kz * kz;
        int i = ks->n++;
        ks->kx[i] = kx; ks->ky[i] = ky; ks->kz[i] = kz;
        ks->mx[i] = mx; ks->my[i] = my; ks->mz[i] = mz;
        /* factor 2 for the mirrored half; prefactor 4 pi / V */
        ks->c[i] = 2.0 * (4.0 * OR_PI / V) * exp(-k2 / (4.0 * alpha * alpha)) / k2;
      }
}
static void kset_free(kset_t *ks) {
  free(ks->kx); free(ks->ky); free(ks->kz); free(ks->c); free(ks->mx); free(ks->my); free(ks->mz);
}

/* per-axis phase tables e^{i 2 pi m x / L}, m = -mmax..mmax, by direct cos/sin */
static void phase_table(double x, double L, int mmax, double *re, double *im) {
  for (int m = -mmax; m <= mmax; ++m) {
    double t = 2.0 * OR_PI * m * x / L;
    re[m + mmax] = cos(t);
    im[m + mmax] = sin(t);
  }
}

/* Structure factors C_k = sum_j q_j cos(k.x_j), S_k = sum_j q_j sin(k.x_j). */
static void structure_factors(int64_t n, const double *x, const double *q, double L, int mmax,
                              const kset_t *ks, double *Ck, double *Sk) {
  int side = 2 * mmax + 1;
  int nt = oracle_num_threads();
  double *part = calloc((size_t)nt * 2 * ks->n, sizeof(double));
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double *pc = part + (size_t)tid * 2 * ks->n, *ps = pc + ks->n;
    double *tab = malloc(6 * side * sizeof(double));
    double *xr = tab, *xi = tab + side, *yr = tab + 2 * side, *yi = tab + 3 * side, *zr = tab + 4 * side,
           *zi = tab + 5 * side;
#pragma omp for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
      phase_table(x[3 * j + 0], L, mmax, xr, xi);
      phase_table(x[3 * j + 1], L, mmax, yr, yi);
      phase_table(x[3 * j + 2], L, mmax, zr, zi);
      double qj = q[j];
      for (int i = 0; i < ks->n; ++i) {
        int a = ks->mx[i] + mmax, b = ks->my[i] + mmax, c = ks->mz[i] + mmax;
        double r1 = xr[a] * yr[b] - xi[a] * yi[b], i1 = xr[a] * yi[b] + xi[a] * yr[b];
        double r2 = r1 * zr[c] - i1 * zi[c], i2 = r1 * zi[c] + i1 * zr[c];
        pc[i] += qj * r2;
        ps[i] += qj * i2;
      }
    }
    free(tab);
  }
  for (int i = 0; i < ks->n; ++i) {
    double c = 0, s = 0;
    for (int t = 0; t < nt; ++t) { c += part[(size_t)t * 2 * ks->n + i]; s += part[(size_t)t * 2 * ks->n + ks->n + i]; }
    Ck[i] = c; Sk[i] = s;
  }
  free(part);
}

/* ---- real-space cell list ---- */
typedef struct { int nc, reach; double cs; int *start, *idx; } cells_t;

static inline int wrapi(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

static void cells_build(cells_t *cl, int64_t n, const double *x, double L, double rc) {
  int nc = (int)floor(L / rc);
  if (nc < 1) nc = 1;
  if (nc > 256) nc = 256;
  cl->nc = nc; cl->cs = L / nc;
  cl->reach = (int)ceil(rc / cl->cs);
  long ncell = (long)nc * nc * nc;
  cl->start = calloc(ncell + 1, sizeof(int));
  cl->idx = malloc(n * sizeof(int));
  int *cellof = malloc(n * sizeof(int));
  for (int64_t j = 0; j < n; ++j) {
    int cx = wrapi((int)floor(x[3 * j] / cl->cs), nc), cy = wrapi((int)floor(x[3 * j + 1] / cl->cs), nc),
        cz = wrapi((int)floor(x[3 * j + 2] / cl->cs), nc);
    cellof[j] = (cz * nc + cy) * nc + cx;
    cl->start[cellof[j] + 1]++;
  }
  for (long c = 0; c < ncell; ++c) cl->start[c + 1] += cl->start[c];
  int *fill = malloc(ncell * sizeof(int));
  memcpy(fill, cl->start, ncell * sizeof(int));
  for (int64_t j = 0; j < n; ++j) cl->idx[fill[cellof[j]]++] = (int)j;
  free(fill); free(cellof);
}
static void cells_free(cells_t *cl) { free(cl->start); free(cl->idx); }

/*
 * phi and grad phi at target atoms (targets == NULL: all atoms, then *energy is set).
 * x: n x 3 positions (any real values; the kernel is periodic), q: n charges.
 * Returns 0 on success.
 */
int oracle_ewald_parts(int64_t n, const double *x, const double *q, double L, double rc, int64_t ntarget,
                       const int64_t *targets, double *phi, double *grad, double *energy, int parts);

int oracle_ewald(int64_t n, const double *x, const double *q, double L, double rc, int64_t ntarget,
                 const int64_t *targets, double *phi, double *grad, double *energy) {
  return oracle_ewald_parts(n, x, q, L, rc, ntarget, targets, phi, grad, energy, 3);
}

/* parts: bit 0 = real-space sum, bit 1 = reciprocal-space sum and self/background
 * terms (both = the full potential).  Used to time the two halves separately. */
int oracle_ewald_parts(int64_t n, const double *x, const double *q, double L, double rc, int64_t ntarget,
                       const int64_t *targets, double *phi, double *grad, double *energy, int parts) {
  double alpha; int mmax;
  oracle_ewald_params(L, rc, &alpha, &mmax);
  double V = L * L * L;
  double Qtot = 0;
  { ksum_t k = {0, 0}; for (int64_t j = 0; j < n; ++j) kadd(&k, q[j]); Qtot = kval(&k); }
  kset_t ks; kset_build(&ks, L, alpha, mmax);
  if (!(parts & 2)) ks.n = 0;
  double *Ck = malloc((ks.n + 1) * sizeof(double)), *Sk = malloc((ks.n + 1) * sizeof(double));
  if (ks.n) structure_factors(n, x, q, L, mmax, &ks, Ck, Sk);
  /* wrap a private copy of the positions into [0, L) for the cell search */
  double *xw = malloc((size_t)n * 3 * sizeof(double));
  for (int64_t j = 0; j < 3 * n; ++j) {
    double v = x[j] - floor(x[j] / L) * L;
    if (v >= L) v -= L;
    if (v < 0.0) v = 0.0;
    xw[j] = v;
  }
  cells_t cl; cells_build(&cl, n, xw, L, rc);
  int nt_all = (targets == NULL);
  int64_t nt = nt_all ? n : ntarget;
  int side = 2 * mmax + 1;
  double rc2 = rc * rc;
#pragma omp parallel
  {
    double *tab = malloc(6 * side * sizeof(double));
    double *xr = tab, *xi = tab + side, *yr = tab + 2 * side, *yi = tab + 3 * side, *zr = tab + 4 * side,
           *zi = tab + 5 * side;
#pragma omp for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
      int64_t i = nt_all ? t : targets[t];
      double xi0 = xw[3 * i], xi1 = xw[3 * i + 1], xi2 = xw[3 * i + 2];
      /* real space */
      ksum_t p = {0, 0};
      double gx = 0, gy = 0, gz = 0;
      int cx = (int)floor(xi0 / cl.cs), cy = (int)floor(xi1 / cl.cs), cz = (int)floor(xi2 / cl.cs);
      int R = (parts & 1) ? cl.reach : -1, nc = cl.nc;
      for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
          for (int dx = -R; dx <= R; ++dx) {
            int gxc = cx + dx, gyc = cy + dy, gzc = cz + dz;
            int wx = wrapi(gxc, nc), wy = wrapi(gyc, nc), wz = wrapi(gzc, nc);
            /* image shift so that the source cell sits at grid position (gxc,gyc,gzc) */
            double sx = (double)((gxc - wx) / nc) * L, sy = (double)((gyc - wy) / nc) * L,
                   sz = (double)((gzc - wz) / nc) * L;
            int c = (wz * nc + wy) * nc + wx;
            for (int s = cl.start[c]; s < cl.start[c + 1]; ++s) {
              int j = cl.idx[s];
              double d0 = xi0 - (xw[3 * j] + sx), d1 = xi1 - (xw[3 * j + 1] + sy),
                     d2 = xi2 - (xw[3 * j + 2] + sz);
              double r2 = d0 * d0 + d1 * d1 + d2 * d2;
              if (r2 >= rc2) continue;
              if (j == i && r2 == 0.0) continue;
              double r = sqrt(r2);
              double e = erfc(alpha * r) / r;
              kadd(&p, q[j] * e);
              double dr = -(e + OR_2_SQRTPI * alpha * exp(-alpha * alpha * r2)) / r; /* d/dr */
              double f = q[j] * dr / r;
              gx += f * d0; gy += f * d1; gz += f * d2;
            }
          }
      /* reciprocal space */
      phase_table(xi0, L, mmax, xr, xi);
      phase_table(xi1, L, mmax, yr, yi);
      phase_table(xi2, L, mmax, zr, zi);
      double pr = 0, rgx = 0, rgy = 0, rgz = 0;
      for (int k = 0; k < ks.n; ++k) {
        int a = ks.mx[k] + mmax, b = ks.my[k] + mmax, c = ks.mz[k] + mmax;
        double r1 = xr[a] * yr[b] - xi[a] * yi[b], i1 = xr[a] * yi[b] + xi[a] * yr[b];
        double cs = r1 * zr[c] - i1 * zi[c], sn = r1 * zi[c] + i1 * zr[c];
        double w = ks.c[k];
        pr += w * (cs * Ck[k] + sn * Sk[k]);
        double gg = w * (-sn * Ck[k] + cs * Sk[k]);
        rgx += gg * ks.kx[k]; rgy += gg * ks.ky[k]; rgz += gg * ks.kz[k];
      }
      kadd(&p, pr);
      if (parts & 2) {
        kadd(&p, -OR_2_SQRTPI * alpha * q[i]);          /* remove erf(a r)/r self limit */
        kadd(&p, -OR_PI * Qtot / (alpha * alpha * V));  /* neutralising background */
      }
      phi[t] = kval(&p);
      grad[3 * t] = gx + rgx; grad[3 * t + 1] = gy + rgy; grad[3 * t + 2] = gz + rgz;
    }
    free(tab);
  }
  if (nt_all && energy) {
    ksum_t e = {0, 0};
    for (int64_t i = 0; i < n; ++i) kadd(&e, 0.5 * q[i] * phi[i]);
    *energy = kval(&e);
  }
  cells_free(&cl); kset_free(&ks); free(Ck); free(Sk); free(xw);
  return 0;
}

/*
 * Pair kernel A(r) and grad A(r) for one displacement r (any real vector).  When
 * |r| == 0 exactly, returns the self term xi (and zero gradient).
 */
double oracle_pair_A(const double *r, double L, double rc, double *grad) {
  double alpha; int mmax;
  oracle_ewald_params(L, rc, &alpha, &mmax);
  double V = L * L * L;
  int R = (int)ceil(rc / L) + 1;
  ksum_t s = {0, 0};
  double gx = 0, gy = 0, gz = 0;
  int self = (r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0);
  for (int a = -R; a <= R; ++a)
    for (int b = -R; b <= R; ++b)
      for (int c = -R; c <= R; ++c) {
        double d0 = r[0] + a * L, d1 = r[1] + b * L, d2 = r[2] + c * L;
        double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (r2 == 0.0) continue;
        double d = sqrt(r2);
        if (d >= rc + 2.0 * L) continue;
        double e = erfc(alpha * d) / d;
        kadd(&s, e);
        double dr = -(e + OR_2_SQRTPI * alpha * exp(-alpha * alpha * r2)) / d;
        gx += dr * d0 / d; gy += dr * d1 / d; gz += dr * d2 / d;
      }
  double tw = 2.0 * OR_PI / L;
  for (int mx = 0; mx <= mmax; ++mx)
    for (int my = -mmax; my <= mmax; ++my)
      for (int mz = -mmax; mz <= mmax; ++mz) {
        if (mx == 0 && (my < 0 || (my == 0 && mz <= 0))) continue;
        if (mx * mx + my * my + mz * mz > mmax * mmax) continue;
        double kx = tw * mx, ky = tw * my, kz = tw * mz, k2 = kx * kx + ky * ky + kz * kz;
        double w = 2.0 * (4.0 * OR_PI / V) * exp(-k2 / (4.0 * alpha * alpha)) / k2;
        double ph = kx * r[0] + ky * r[1] + kz * r[2];
        kadd(&s, w * cos(ph));
        double g = -w * sin(ph);
        gx += g * kx; gy += g * ky; gz += g * kz;
      }
  kadd(&s, -OR_PI / (alpha * alpha * V));
  if (self) kadd(&s, -OR_2_SQRTPI * alpha);
  if (grad) {
    grad[0] = self ? 0.0 : gx; grad[1] = self ? 0.0 : gy; grad[2] = self ? 0.0 : gz;
  }
  return kval(&s);
}

/* Plain direct Coulomb sum over an explicit list of sources (no periodicity):
 * phi_i = sum_j q_j / |x_i - y_j| for targets x.  Used by tests as a second,
 * independent route (spherical-shell image sums). */
void oracle_direct(int64_t nt, const double *xt, int64_t ns, const double *ys, const double *qs,
                   double *phi) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nt; ++i) {
    ksum_t p = {0, 0};
    for (int64_t j = 0; j < ns; ++j) {
      double d0 = xt[3 * i] - ys[3 * j], d1 = xt[3 * i + 1] - ys[3 * j + 1], d2 = xt[3 * i + 2] - ys[3 * j + 2];
      double r2 = d0 * d0 + d1 * d1 + d2 * d2;
      if (r2 == 0.0) continue;
      kadd(&p, qs[j] / sqrt(r2));
    }
    phi[i] = kval(&p);
  }
}

/*
 * Energy only: E = 1/2 sum_{i != j or n != 0} q_i q_j erfc(a r)/r  (each pair once)
 *                + (2 pi / V) sum_{k != 0} exp(-k^2/4a^2)/k^2 |S(k)|^2
 *                - a/sqrt(pi) sum q_i^2 - pi Q^2 / (2 a^2 V)
 * (f = 1).  Same value as 1/2 sum q_i phi_i from oracle_ewald.
 */
double oracle_ewald_energy(int64_t n, const double *x, const double *q, double L, double rc) {
  double alpha; int mmax;
  oracle_ewald_params(L, rc, &alpha, &mmax);
  double V = L * L * L;
  ksum_t qs = {0, 0}, q2 = {0, 0};
  for (int64_t j = 0; j < n; ++j) { kadd(&qs, q[j]); kadd(&q2, q[j] * q[j]); }
  kset_t ks; kset_build(&ks, L, alpha, mmax);
  double *Ck = malloc(ks.n * sizeof(double)), *Sk = malloc(ks.n * sizeof(double));
  structure_factors(n, x, q, L, mmax, &ks, Ck, Sk);
  ksum_t erec = {0, 0};
  /* ks.c holds 2 * (4 pi / V) * exp()/k^2 for the half space: |S|^2 sum over the
     full space times 2 pi / V equals sum_half c/4 * |S|^2 ... written out: */
  for (int k = 0; k < ks.n; ++k) kadd(&erec, 0.5 * ks.c[k] * (Ck[k] * Ck[k] + Sk[k] * Sk[k]));
  double *xw = malloc((size_t)n * 3 * sizeof(double));
  for (int64_t j = 0; j < 3 * n; ++j) {
    double v = x[j] - floor(x[j] / L) * L;
    if (v >= L) v -= L;
    if (v < 0.0) v = 0.0;
    xw[j] = v;
  }
  cells_t cl; cells_build(&cl, n, xw, L, rc);
  double rc2 = rc * rc;
  int nt = oracle_num_threads();
  double *part = calloc((size_t)nt * 2, sizeof(double));
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    ksum_t acc = {0, 0};
#pragma omp for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
      double xi0 = xw[3 * i], xi1 = xw[3 * i + 1], xi2 = xw[3 * i + 2];
      int cx = (int)floor(xi0 / cl.cs), cy = (int)floor(xi1 / cl.cs), cz = (int)floor(xi2 / cl.cs);
      int R = cl.reach, nc = cl.nc;
      double s = 0.0;
      for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
          for (int dx = -R; dx <= R; ++dx) {
            int gxc = cx + dx, gyc = cy + dy, gzc = cz + dz;
            int wx = wrapi(gxc, nc), wy = wrapi(gyc, nc), wz = wrapi(gzc, nc);
            double sx = (double)((gxc - wx) / nc) * L, sy = (double)((gyc - wy) / nc) * L,
                   sz = (double)((gzc - wz) / nc) * L;
            int c = (wz * nc + wy) * nc + wx;
            for (int t = cl.start[c]; t < cl.start[c + 1]; ++t) {
              int j = cl.idx[t];
              double d0 = xi0 - (xw[3 * j] + sx), d1 = xi1 - (xw[3 * j + 1] + sy), d2 = xi2 - (xw[3 * j + 2] + sz);
              double r2 = d0 * d0 + d1 * d1 + d2 * d2;
              if (r2 >= rc2 || (j == i && r2 == 0.0)) continue;
              double r = sqrt(r2);
              s += q[j] * erfc(alpha * r) / r;
            }
          }
      kadd(&acc, 0.5 * q[i] * s);
    }
    part[2 * tid] = acc.s; part[2 * tid + 1] = acc.c;
  }
  ksum_t ereal = {0, 0};
  for (int t = 0; t < nt; ++t) { kadd(&ereal, part[2 * t]); kadd(&ereal, part[2 * t + 1]); }
  free(part);
  double Q = kval(&qs);
  ksum_t e = {0, 0};
  kadd(&e, kval(&ereal));
  kadd(&e, kval(&erec));
  kadd(&e, -alpha / sqrt(OR_PI) * kval(&q2));
  kadd(&e, -OR_PI * Q * Q / (2.0 * alpha * alpha * V));
  cells_free(&cl); kset_free(&ks); free(Ck); free(Sk); free(xw);
  return kval(&e);
}
