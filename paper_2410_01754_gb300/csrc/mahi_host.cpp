// Host planner: solid harmonics, FMM translation operators in a real basis, the
// periodic lattice coefficients, and the M2L offset tables.
//
// Expansion convention (scaled complex solid harmonics, Condon-Shortley phase):
//   R_00 = 1, R_mm = -(x+iy)/(2m) R_{m-1,m-1},
//   R_lm = ((2l-1) z R_{l-1,m} - r^2 R_{l-2,m}) / ((l+m)(l-m)),  R_{l,-m} = (-1)^m conj(R_lm)
//   I_00 = 1/r, I_mm = -(2m-1)(x+iy)/r^2 I_{m-1,m-1},
//   I_lm = ((2l-1) z I_{l-1,m} - ((l-1)^2 - m^2) I_{l-2,m}) / r^2
// with 1/|a-b| = sum_lm conj(R_lm(a)) I_lm(b) (|a| < |b|) and the addition theorem
// R_lm(a+b) = sum_jk R_jk(a) R_{l-j,m-k}(b).  A box of edge s at level l stores
//   multipole  M^_lm = s^-l  sum_i q_i conj(R_lm(y_i - c))        (phi = sum M_lm I_lm(x-c))
//   local      L^_lm = s^(l+1) L_lm,  phi(x) = sum L_lm conj(R_lm(x - c))
// so that every operator below is independent of the level.  Real layout: index
// l*l for m = 0, l*l + 2m - 1 (Re) and l*l + 2m (Im) for m > 0; negative m follow
// from X_{l,-m} = (-1)^m conj(X_lm), which holds for all expansions of real charges.
//
// The working (device) basis rescales every coefficient by c_lm = sqrt((l+m)!(l-m)!)
// (multipoles multiplied, locals divided) so that FP32 covers orders up to 16;
// scale_operator() converts the operators built here.
//
// FMM steps follow the paper's Fig. "fmm_scheme" (P2M, M2M, M2L, L2L, L2P); the
// periodic split follows Eq. "approx_nbody_periodic" (first image shell through
// the tree, far images through the lattice operator, tin-foil/dipole term).
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "mahi_internal.h"

namespace mahi {

using cd = std::complex<double>;

double coulomb_constant() {
  // f = N_A e^2 / (4 pi eps0) * 1e6 (J m -> kJ nm), CODATA 2018 constants.
  const double e = 1.602176634e-19, NA = 6.02214076e23, eps0 = 8.8541878128e-12;
  return NA * e * e / (4.0 * kPi * eps0) * 1e6;
}

static inline int tri(int l, int m) { return l * (l + 1) / 2 + m; }

static void regular(int P, const double r[3], std::vector<cd> &R) {
  R.assign(tri(P, P) + 1, cd(0, 0));
  const double x = r[0], y = r[1], z = r[2], r2 = x * x + y * y + z * z;
  R[0] = 1.0;
  for (int m = 0; m <= P; ++m) {
    if (m > 0) R[tri(m, m)] = -cd(x, y) / (2.0 * m) * R[tri(m - 1, m - 1)];
    if (m + 1 <= P) R[tri(m + 1, m)] = z * R[tri(m, m)];
    for (int l = m + 2; l <= P; ++l)
      R[tri(l, m)] = ((2.0 * l - 1.0) * z * R[tri(l - 1, m)] - r2 * R[tri(l - 2, m)]) / double((l + m) * (l - m));
  }
}

static void irregular(int P, const double r[3], std::vector<cd> &I) {
  I.assign(tri(P, P) + 1, cd(0, 0));
  const double x = r[0], y = r[1], z = r[2], r2 = x * x + y * y + z * z, ri2 = 1.0 / r2;
  I[0] = 1.0 / std::sqrt(r2);
  for (int m = 0; m <= P; ++m) {
    if (m > 0) I[tri(m, m)] = -(2.0 * m - 1.0) * cd(x, y) * ri2 * I[tri(m - 1, m - 1)];
    if (m + 1 <= P) I[tri(m + 1, m)] = (2.0 * m + 1.0) * z * ri2 * I[tri(m, m)];
    for (int l = m + 2; l <= P; ++l)
      I[tri(l, m)] = ((2.0 * l - 1.0) * z * I[tri(l - 1, m)] - double((l - 1) * (l - 1) - m * m) * I[tri(l - 2, m)]) * ri2;
  }
}

// value at (l, m) for any sign of m from the m >= 0 table; 0 outside |m| <= l
static inline cd at(const std::vector<cd> &T, int l, int m) {
  if (l < 0 || m > l || -m > l) return cd(0, 0);
  if (m >= 0) return T[tri(l, m)];
  cd v = std::conj(T[tri(l, -m)]);
  return (m & 1) ? -v : v;
}

// Complex coefficients of one real unit vector: at most two nonzero (l, +-m).
struct Unit {
  int l, m;
  cd cp, cm;  // coefficient at (l, m) and at (l, -m) (cm unused for m = 0)
};
static Unit unit_of(int col) {
  int l = (int)std::floor(std::sqrt((double)col) + 1e-9);
  while (l * l > col) --l;
  while ((l + 1) * (l + 1) <= col) ++l;
  int r = col - l * l;
  Unit u;
  u.l = l;
  if (r == 0) {
    u.m = 0; u.cp = 1.0; u.cm = 0.0;
  } else {
    int m = (r + 1) / 2;
    bool re = (r & 1);
    u.m = m;
    double sg = (m & 1) ? -1.0 : 1.0;
    if (re) { u.cp = 1.0; u.cm = sg; }
    else { u.cp = cd(0, 1); u.cm = cd(0, -sg); }
  }
  return u;
}

// Fill column `col` of a real operator from the complex outputs f(l, m), m >= 0.
template <class F>
static void fill_column(int p, int col, std::vector<double> &op, F f) {
  const int K = ncoef(p);
  for (int l = 0; l <= p; ++l) {
    cd v0 = f(l, 0);
    op[(size_t)(l * l) * K + col] = v0.real();
    for (int m = 1; m <= l; ++m) {
      cd v = f(l, m);
      op[(size_t)(l * l + 2 * m - 1) * K + col] = v.real();
      op[(size_t)(l * l + 2 * m) * K + col] = v.imag();
    }
  }
}

void build_m2l(int p, int ox, int oy, int oz, std::vector<double> &op) {
  const int K = ncoef(p);
  op.assign((size_t)K * K, 0.0);
  double o[3] = {(double)ox, (double)oy, (double)oz};
  std::vector<cd> I;
  irregular(2 * p, o, I);
  for (int col = 0; col < K; ++col) {
    Unit u = unit_of(col);
    // L_lm = (-1)^l sum_jk M_jk I_{j+l, k+m}(o)
    fill_column(p, col, op, [&](int l, int m) {
      cd s = u.cp * at(I, u.l + l, u.m + m);
      if (u.m) s += u.cm * at(I, u.l + l, -u.m + m);
      return (l & 1) ? -s : s;
    });
  }
}

static void child_delta(int child, double d[3]) {
  d[0] = (child & 1) ? 0.25 : -0.25;
  d[1] = (child & 2) ? 0.25 : -0.25;
  d[2] = (child & 4) ? 0.25 : -0.25;
}

void build_m2m(int p, int child, std::vector<double> &op) {
  const int K = ncoef(p);
  op.assign((size_t)K * K, 0.0);
  double dl[3];
  child_delta(child, dl);  // child centre - parent centre, in parent edges
  std::vector<cd> R;
  regular(p, dl, R);
  for (int col = 0; col < K; ++col) {
    Unit u = unit_of(col);
    // M'_lm = sum_jk M_jk 2^-j conj(R_{l-j, m-k}(delta))
    const double sc = std::ldexp(1.0, -u.l);
    fill_column(p, col, op, [&](int l, int m) {
      if (l < u.l) return cd(0, 0);
      cd s = u.cp * std::conj(at(R, l - u.l, m - u.m));
      if (u.m) s += u.cm * std::conj(at(R, l - u.l, m + u.m));
      return s * sc;
    });
  }
}

void build_l2l(int p, int child, std::vector<double> &op) {
  const int K = ncoef(p);
  op.assign((size_t)K * K, 0.0);
  double dl[3];
  child_delta(child, dl);
  std::vector<cd> R;
  regular(p, dl, R);
  for (int col = 0; col < K; ++col) {
    Unit u = unit_of(col);  // input (l, m) of the parent local
    // L'_jk = sum_lm L_lm 2^-(j+1) conj(R_{l-j, m-k}(delta))
    fill_column(p, col, op, [&](int j, int k) {
      if (u.l < j) return cd(0, 0);
      cd s = u.cp * std::conj(at(R, u.l - j, u.m - k));
      if (u.m) s += u.cm * std::conj(at(R, u.l - j, -u.m - k));
      return s * std::ldexp(1.0, -j - 1);
    });
  }
}

// ---- lattice coefficients ---------------------------------------------------
// H_K(r) = A(r) - sum_{|n|_inf <= K} 1/|r+n| - (2 pi / 3)|r|^2 for the unit box,
// harmonic for |r| < K + 1, evaluated by Ewald splitting without any singular term:
//   sum_{|n|_inf > K} erfc(a|r+n|)/|r+n| - sum_{|n|_inf <= K} erf(a|r+n|)/|r+n|
//   + 4 pi sum_{k != 0} exp(-k^2/4a^2) cos(k.r)/k^2 - pi/a^2 - (2 pi/3)|r|^2.
// (The shell sums are handled elsewhere: the first shell K = 1 by the tree, the
// shells 2..K by M2L at the root, and everything beyond by H_K.)
static double lattice_H_unit(const double r[3], int K) {
  const double a = 2.6;
  const double two_over_sqrtpi = 1.12837916709551257390;
  const double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  const int R = (int)std::ceil(rn + 2.5) + 1;
  double s = 0.0;
  for (int nx = -R; nx <= R; ++nx)
    for (int ny = -R; ny <= R; ++ny)
      for (int nz = -R; nz <= R; ++nz) {
        double dx = r[0] + nx, dy = r[1] + ny, dz = r[2] + nz;
        double d = std::sqrt(dx * dx + dy * dy + dz * dz);
        bool near = std::abs(nx) <= K && std::abs(ny) <= K && std::abs(nz) <= K;
        if (near) {
          s -= (d > 0.0) ? std::erf(a * d) / d : two_over_sqrtpi * a;
        } else if (d < 2.45) {
          s += std::erfc(a * d) / d;
        }
      }
  // shells beyond R that still hold erf terms (only when K > R) are not possible:
  // R >= |r| + 2.5 > K for the radii used here.
  const int mm = 6;
  double rec = 0.0;
  for (int mx = -mm; mx <= mm; ++mx)
    for (int my = -mm; my <= mm; ++my)
      for (int mz = -mm; mz <= mm; ++mz) {
        int m2 = mx * mx + my * my + mz * mz;
        if (m2 == 0 || m2 > mm * mm) continue;
        double k2 = 4.0 * kPi * kPi * m2;
        rec += std::exp(-k2 / (4.0 * a * a)) / k2 * std::cos(2.0 * kPi * (mx * r[0] + my * r[1] + mz * r[2]));
      }
  s += 4.0 * kPi * rec;
  s -= kPi / (a * a);
  s -= (2.0 * kPi / 3.0) * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  // erf terms of the shell beyond the loop range (|n|_inf <= K but outside R)
  for (int nx = -K; nx <= K; ++nx)
    for (int ny = -K; ny <= K; ++ny)
      for (int nz = -K; nz <= K; ++nz) {
        if (std::abs(nx) <= R && std::abs(ny) <= R && std::abs(nz) <= R) continue;
        double dx = r[0] + nx, dy = r[1] + ny, dz = r[2] + nz;
        double d = std::sqrt(dx * dx + dy * dy + dz * dz);
        s -= std::erf(a * d) / d;
      }
  return s;
}

static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
  x.resize(n); w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), pp = 0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) { double p3 = p2; p2 = p1; p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j; }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      double dz = p1 / pp;
      z -= dz;
      if (std::abs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

static std::mutex g_lat_mu;
static std::map<std::pair<int, int>, std::vector<double>> g_lat;

const std::vector<double> &lattice_coeffs(int P, int shell) {
  std::lock_guard<std::mutex> lk(g_lat_mu);
  auto key = std::make_pair(P, shell);
  auto it = g_lat.find(key);
  if (it != g_lat.end()) return it->second;
  // Project H_K on the sphere |r| = rho (0.6 of the radius where H_K stops being
  // harmonic): eta_lm = int H(rho s) R_lm(s) dOmega / (rho^l N_lm),
  // N_lm = int |R_lm(s)|^2 dOmega = 4 pi / ((2l+1) (l+m)! (l-m)!).
  const double rho = 0.6 * (shell + 1);
  const int nt = P + 64, np = 2 * nt;
  std::vector<double> gx, gw;
  gauss_legendre(nt, gx, gw);
  std::vector<cd> acc(tri(P, P) + 1, cd(0, 0)), R;
  for (int it = 0; it < nt; ++it) {
    double ct = gx[it], st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
    for (int jp = 0; jp < np; ++jp) {
      double ph = 2.0 * kPi * jp / np;
      double s[3] = {st * std::cos(ph), st * std::sin(ph), ct};
      double r[3] = {rho * s[0], rho * s[1], rho * s[2]};
      double h = lattice_H_unit(r, shell) * gw[it] * (2.0 * kPi / np);
      regular(P, s, R);
      for (size_t k = 0; k < acc.size(); ++k) acc[k] += h * R[k];
    }
  }
  std::vector<double> out((size_t)(P + 1) * (P + 1), 0.0);
  std::vector<double> lf(2 * P + 2, 0.0);
  for (int i = 1; i < (int)lf.size(); ++i) lf[i] = lf[i - 1] + std::log((double)i);
  for (int l = 0; l <= P; ++l) {
    for (int m = 0; m <= l; ++m) {
      // cubic symmetry: only even l and m = 0 mod 4 survive, all real
      if ((l & 1) || (m % 4) != 0) continue;
      if (l == 2) continue;
      double logN = std::log(4.0 * kPi / (2.0 * l + 1.0)) - lf[l + m] - lf[l - m];
      double v = acc[tri(l, m)].real() / std::exp(l * std::log(rho) + logN);
      if (m == 0) out[l * l] = v;
      else out[l * l + 2 * m - 1] = v;
    }
  }
  auto res = g_lat.emplace(key, std::move(out));
  return res.first->second;
}

void build_lattice_op(int p, std::vector<double> &op, bool with_images) {
  const int K = ncoef(p), P = 2 * p;
  // far images |n|_inf >= 4 through the lattice function H_3 ...
  const std::vector<double> &eta = lattice_coeffs(P, kLatticeShell);
  std::vector<cd> E(tri(P, P) + 1);
  for (int l = 0; l <= P; ++l) {
    E[tri(l, 0)] = eta[l * l];
    for (int m = 1; m <= l; ++m) E[tri(l, m)] = cd(eta[l * l + 2 * m - 1], eta[l * l + 2 * m]);
  }
  op.assign((size_t)K * K, 0.0);
  for (int col = 0; col < K; ++col) {
    Unit u = unit_of(col);
    // L_jk = sum_lm (-1)^l eta_{j+l, k+m} M_lm
    fill_column(p, col, op, [&](int j, int k) {
      cd s = u.cp * at(E, j + u.l, k + u.m);
      if (u.m) s += u.cm * at(E, j + u.l, k - u.m);
      return (u.l & 1) ? -s : s;
    });
  }
  // ... and the images 2 <= |n|_inf <= 3 of the root by plain M2L (offset o = n)
  if (!with_images) return;
  const OffsetTables &ot = offset_tables();
  std::vector<double> t;
  for (int o = 0; o < kNumOffsets; ++o) {
    build_m2l(p, ot.off[o][0], ot.off[o][1], ot.off[o][2], t);
    for (size_t i = 0; i < op.size(); ++i) op[i] += t[i];
  }
}

double basis_scale(int col) {
  // c_lm = sqrt((l+m)! (l-m)!) of the real coefficient index col
  int l = (int)std::floor(std::sqrt((double)col) + 1e-9);
  while (l * l > col) --l;
  while ((l + 1) * (l + 1) <= col) ++l;
  int r = col - l * l, m = (r + 1) / 2;
  return std::exp(0.5 * (std::lgamma(l + m + 1.0) + std::lgamma(l - m + 1.0)));
}

void scale_operator(int p, int kind, std::vector<double> &op) {
  const int K = ncoef(p);
  std::vector<double> c(K);
  for (int k = 0; k < K; ++k) c[k] = basis_scale(k);
  for (int r = 0; r < K; ++r)
    for (int k = 0; k < K; ++k) {
      double &v = op[(size_t)r * K + k];
      if (kind == 0) v *= c[r] / c[k];        // multipole -> multipole
      else if (kind == 1) v *= c[k] / c[r];   // local -> local
      else v /= c[r] * c[k];                  // multipole -> local
    }
}

void gradient_coeffs(int P, const double *c, double *cx, double *cy, double *cz) {
  // complex table of c (m >= 0)
  std::vector<cd> C(tri(P, P) + 1);
  for (int l = 0; l <= P; ++l) {
    C[tri(l, 0)] = c[l * l];
    for (int m = 1; m <= l; ++m) C[tri(l, m)] = cd(c[l * l + 2 * m - 1], c[l * l + 2 * m]);
  }
  auto put = [&](double *dst, int l, int m, cd v) {
    if (m == 0) dst[l * l] = v.real();
    else { dst[l * l + 2 * m - 1] = v.real(); dst[l * l + 2 * m] = v.imag(); }
  };
  // d/dz conj(R_lm) = conj(R_{l-1,m}); d/dx = 1/2 (conj R_{l-1,m+1} - conj R_{l-1,m-1});
  // d/dy = i/2 (conj R_{l-1,m-1} + conj R_{l-1,m+1})   =>  coefficient maps below
  for (int l = 0; l <= P - 1; ++l)
    for (int m = 0; m <= l; ++m) {
      cd zc = at(C, l + 1, m);
      cd xc = 0.5 * (at(C, l + 1, m - 1) - at(C, l + 1, m + 1));
      cd yc = cd(0, 0.5) * (at(C, l + 1, m + 1) + at(C, l + 1, m - 1));
      put(cz, l, m, zc); put(cx, l, m, xc); put(cy, l, m, yc);
    }
}

double lattice_eval_host(double L, int P, int shell, const double r[3]) {
  const std::vector<double> &eta = lattice_coeffs(P, shell);
  double u[3] = {r[0] / L, r[1] / L, r[2] / L};
  std::vector<cd> R;
  regular(P, u, R);
  double s = 0.0;
  for (int l = 0; l <= P; ++l) {
    s += eta[l * l] * R[tri(l, 0)].real();
    for (int m = 1; m <= l; ++m) {
      cd e(eta[l * l + 2 * m - 1], eta[l * l + 2 * m]);
      s += 2.0 * (e * std::conj(R[tri(l, m)])).real();
    }
  }
  return s / L;
}

static OffsetTables make_offsets() {
  OffsetTables t;
  for (int i = 0; i < 343; ++i) t.id[i] = -1;
  int n = 0;
  for (int ox = -3; ox <= 3; ++ox)
    for (int oy = -3; oy <= 3; ++oy)
      for (int oz = -3; oz <= 3; ++oz) {
        if (std::abs(ox) <= 1 && std::abs(oy) <= 1 && std::abs(oz) <= 1) continue;
        t.id[(ox + 3) * 49 + (oy + 3) * 7 + (oz + 3)] = n;
        t.off[n][0] = ox; t.off[n][1] = oy; t.off[n][2] = oz;
        ++n;
      }
  // interaction list of a box with child index c = (cx, cy, cz) inside its parent:
  // children 2(P+n)+b of the parent's 27 neighbours that are not its own neighbours;
  // offset o = box - source = c - 2n - b.
  for (int c = 0; c < 8; ++c) {
    int cc[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    int k = 0;
    for (int n0 = -1; n0 <= 1; ++n0)
      for (int n1 = -1; n1 <= 1; ++n1)
        for (int n2 = -1; n2 <= 1; ++n2)
          for (int b = 0; b < 8; ++b) {
            int o0 = cc[0] - 2 * n0 - (b & 1), o1 = cc[1] - 2 * n1 - ((b >> 1) & 1),
                o2 = cc[2] - 2 * n2 - ((b >> 2) & 1);
            if (std::abs(o0) <= 1 && std::abs(o1) <= 1 && std::abs(o2) <= 1) continue;
            t.list[c][k++] = t.id[(o0 + 3) * 49 + (o1 + 3) * 7 + (o2 + 3)];
          }
  }
  return t;
}

const OffsetTables &offset_tables() {
  static OffsetTables t = make_offsets();
  return t;
}

}  // namespace mahi
