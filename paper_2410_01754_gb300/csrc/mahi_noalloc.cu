// Allocation-free per-site Hamiltonian-interpolation terms.
//
// Some callers cannot allocate device memory when they need these terms: code
// that runs while a CUDA stream is being captured, a host program whose device
// memory is handed out by another runtime or a fixed pool, or an MD engine that
// computes the charge-scaled potential with its own solver and only wants the
// per-site terms on top.  mahi_site_terms_static serves them: it takes the
// potential, positions and charges from the caller, writes the caller's
// outputs, and keeps its only scratch (one energy slot per site) in a
// file-scope device array instead of a cudaMalloc'd workspace.  It runs the
// same per-site arithmetic as the k_site stage of mahi_eval.
//
// Scratch: g_site_energy, kStaticMaxSites doubles (32 KiB), plus the tables of
// the first-shell lattice function (4 x 41^2 doubles); every GPU that loads the
// library holds them until the process exits.  All calls share the scratch and
// keep the last call's contents; calls whose work overlaps on the GPU race.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>

#include "mahi_internal.h"

namespace mahi {
namespace {

constexpr int kStaticMaxSites = 4096;
constexpr int kStaticMaxSiteAtoms = 64;
constexpr int kStaticDeg = 40;                               // degree of H_1 (same as the eval path)
constexpr int kStaticCoef = (kStaticDeg + 1) * (kStaticDeg + 1);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_site_energy[kStaticMaxSites];
static __device__ __align__(256) double g_eta[4][kStaticCoef];   // H, dH/dx, dH/dy, dH/dz coefficients

std::mutex g_mu;
bool g_ready[kMaxDevices] = {};
double *g_energy_ptr[kMaxDevices] = {};
double *g_eta_ptr[kMaxDevices] = {};

using cd = std::complex<double>;
constexpr int tri(int l, int m) { return l * (l + 1) / 2 + m; }

// Fixed-size (heap-free) host evaluation of the scaled regular harmonics R_lm,
// m >= 0, at a point; out has tri(P, P) + 1 entries.
void regular_fixed(int P, const double r[3], cd *out) {
  const double x = r[0], y = r[1], z = r[2], r2 = x * x + y * y + z * z;
  out[0] = 1.0;
  for (int m = 0; m <= P; ++m) {
    if (m > 0) out[tri(m, m)] = -cd(x, y) / (2.0 * m) * out[tri(m - 1, m - 1)];
    if (m + 1 <= P) out[tri(m + 1, m)] = z * out[tri(m, m)];
    for (int l = m + 2; l <= P; ++l)
      out[tri(l, m)] = ((2.0 * l - 1.0) * z * out[tri(l - 1, m)] - r2 * out[tri(l - 2, m)]) / double((l + m) * (l - m));
  }
}

// H_1(r) for the unit box by Ewald splitting (first image shell removed, no
// singular term), as in the library's lattice coefficients.
double lattice_h1(const double r[3]) {
  const double a = 2.6, two_over_sqrtpi = 1.12837916709551257390;
  double s = 0.0;
  for (int nx = -4; nx <= 4; ++nx)
    for (int ny = -4; ny <= 4; ++ny)
      for (int nz = -4; nz <= 4; ++nz) {
        const double dx = r[0] + nx, dy = r[1] + ny, dz = r[2] + nz, d = std::sqrt(dx * dx + dy * dy + dz * dz);
        const bool near = std::abs(nx) <= 1 && std::abs(ny) <= 1 && std::abs(nz) <= 1;
        if (near) s -= (d > 0.0) ? std::erf(a * d) / d : two_over_sqrtpi * a;
        else if (d < 2.45) s += std::erfc(a * d) / d;
      }
  double rec = 0.0;
  for (int mx = -6; mx <= 6; ++mx)
    for (int my = -6; my <= 6; ++my)
      for (int mz = -6; mz <= 6; ++mz) {
        const int m2 = mx * mx + my * my + mz * mz;
        if (m2 == 0 || m2 > 36) continue;
        const double k2 = 4.0 * kPi * kPi * m2;
        rec += std::exp(-k2 / (4.0 * a * a)) / k2 * std::cos(2.0 * kPi * (mx * r[0] + my * r[1] + mz * r[2]));
      }
  return s + 4.0 * kPi * rec - kPi / (a * a) - (2.0 * kPi / 3.0) * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
}

// Coefficients of H_1 (degree kStaticDeg, real layout) and of its gradient
// (degree kStaticDeg - 1), into fixed host buffers: projection on the sphere
// |r| = 1.2 with Gauss-Legendre x trapezoid quadrature.
void h1_tables(double (*tab)[kStaticCoef]) {
  static cd acc[tri(kStaticDeg, kStaticDeg) + 1];
  static cd R[tri(kStaticDeg, kStaticDeg) + 1];
  static double gx[kStaticDeg + 64], gw[kStaticDeg + 64];
  const int P = kStaticDeg, nt = P + 64, np = 2 * nt;
  const double rho = 1.2;
  for (int i = 0; i < nt; ++i) {  // Gauss-Legendre nodes by Newton iteration
    double z = std::cos(kPi * (i + 0.75) / (nt + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= nt; ++j) { const double p3 = p2; p2 = p1; p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j; }
      pp = nt * (z * p1 - p2) / (z * z - 1.0);
      const double dz = p1 / pp;
      z -= dz;
      if (std::abs(dz) < 1e-16) break;
    }
    gx[i] = z;
    gw[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
  for (auto &v : acc) v = 0.0;
  for (int it = 0; it < nt; ++it) {
    const double ct = gx[it], st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
    for (int jp = 0; jp < np; ++jp) {
      const double ph = 2.0 * kPi * jp / np;
      const double s[3] = {st * std::cos(ph), st * std::sin(ph), ct};
      const double r[3] = {rho * s[0], rho * s[1], rho * s[2]};
      const double h = lattice_h1(r) * gw[it] * (2.0 * kPi / np);
      regular_fixed(P, s, R);
      for (int k = 0; k <= tri(P, P); ++k) acc[k] += h * R[k];
    }
  }
  std::memset(tab, 0, sizeof(double) * 4 * kStaticCoef);
  double lf[2 * kStaticDeg + 2];
  lf[0] = 0.0;
  for (int i = 1; i < 2 * kStaticDeg + 2; ++i) lf[i] = lf[i - 1] + std::log((double)i);
  for (int l = 0; l <= P; l += 2)
    for (int m = 0; m <= l; m += 4) {
      if (l == 2) continue;  // cubic symmetry: even l, m = 0 mod 4, real
      const double logN = std::log(4.0 * kPi / (2.0 * l + 1.0)) - lf[l + m] - lf[l - m];
      const double v = acc[tri(l, m)].real() / std::exp(l * std::log(rho) + logN);
      tab[0][m == 0 ? l * l : l * l + 2 * m - 1] = v;
    }
  // gradient maps: d/dz conj R_lm = conj R_{l-1,m}; d/dx = (conj R_{l-1,m+1} - conj R_{l-1,m-1})/2;
  // d/dy = i (conj R_{l-1,m-1} + conj R_{l-1,m+1})/2
  auto get = [&](int l, int m) -> cd {
    if (l < 0 || m > l || -m > l) return 0.0;
    const int am = m < 0 ? -m : m;
    cd v = am == 0 ? cd(tab[0][l * l], 0.0) : cd(tab[0][l * l + 2 * am - 1], tab[0][l * l + 2 * am]);
    if (m < 0) { v = std::conj(v); if (am & 1) v = -v; }
    return v;
  };
  for (int l = 0; l <= P - 1; ++l)
    for (int m = 0; m <= l; ++m) {
      const cd zc = get(l + 1, m), xc = 0.5 * (get(l + 1, m - 1) - get(l + 1, m + 1)),
               yc = cd(0, 0.5) * (get(l + 1, m + 1) + get(l + 1, m - 1));
      const cd g3[3] = {xc, yc, zc};
      for (int a = 0; a < 3; ++a) {
        if (m == 0) tab[1 + a][l * l] = g3[a].real();
        else { tab[1 + a][l * l + 2 * m - 1] = g3[a].real(); tab[1 + a][l * l + 2 * m] = g3[a].imag(); }
      }
    }
}

template <typename XT, typename FT>
__global__ void k_site_static(int S, double L, double fcoul, const int *__restrict__ site_ptr,
                              const int *__restrict__ site_atoms, const XT *__restrict__ x,
                              const double *__restrict__ qA, const double *__restrict__ qB,
                              const double *__restrict__ lam, const double *__restrict__ phi,
                              const double *__restrict__ eta, double *__restrict__ site_energy,
                              double *__restrict__ dEdl, FT *__restrict__ forces) {
  __shared__ double fsh[4][kStaticMaxSiteAtoms][3];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (site >= S) return;
  const int b = site_ptr[site], n = site_ptr[site + 1] - b;
  if (n < 1 || n > kStaticMaxSiteAtoms) {  // malformed site: flag it, touch nothing else
    if (lane == 0) {
      if (dEdl) dEdl[site] = nan("");
      site_energy[site] = nan("");
    }
    return;
  }
  const double *eh = eta, *ex = eta + kStaticCoef, *ey = eta + 2 * kStaticCoef, *ez = eta + 3 * kStaticCoef;
  const double V = L * L * L, c2 = 2.0 * kPi / (3.0 * V);
  const double lw = lam[site] * (1.0 - lam[site]);
  for (int k = lane; k < n * 3; k += 32) fsh[wib][k / 3][k % 3] = 0.0;
  __syncwarp();
  double ksum = 0.0, gsum = 0.0;
  for (int pi = lane; pi < n * n; pi += 32) {
    const int ia = pi / n, ja = pi % n;
    const int i = site_atoms[b + ia], j = site_atoms[b + ja];
    const double Di = qB[i] - qA[i], Dj = qB[j] - qA[j];
    double r[3];
    for (int a = 0; a < 3; ++a) {
      double v = (double)x[3 * (size_t)i + a] - (double)x[3 * (size_t)j + a];
      v -= L * rint(v / L);
      r[a] = (ia == ja) ? 0.0 : v;
    }
    // first image shell directly
    double A = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int nx = -1; nx <= 1; ++nx)
      for (int ny = -1; ny <= 1; ++ny)
        for (int nz = -1; nz <= 1; ++nz) {
          if (ia == ja && nx == 0 && ny == 0 && nz == 0) continue;
          const double d0 = r[0] + nx * L, d1 = r[1] + ny * L, d2 = r[2] + nz * L;
          const double ri = 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2), g3 = ri * ri * ri;
          A += ri;
          g0 -= g3 * d0; g1 -= g3 * d1; g2 -= g3 * d2;
        }
    // far images: H_1 and its gradient from the coefficient tables, degree
    // adapted to |r| (terms fall like (|r|/2L)^l)
    const double u[3] = {r[0] / L, r[1] / L, r[2] / L};
    const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    int P = 0;
    if (un > 0.0) P = min(kStaticDeg, max(4, (int)ceil(-39.2 / log(un / 1.9)) + 1));
    double H = 0.0, hx = 0.0, hy = 0.0, hz = 0.0;
    const double r2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double dre = 1.0, dim = 0.0;
    for (int m = 0; m <= P; ++m) {  // R_lm column by column
      if (m > 0) {
        const double f = -1.0 / (2.0 * m);
        const double tr = f * (u[0] * dre - u[1] * dim), ti = f * (u[0] * dim + u[1] * dre);
        dre = tr; dim = ti;
      }
      double pr = 0.0, pim = 0.0, cr = dre, ci = dim;
      for (int l = m; l <= P; ++l) {
        if (l > m) {
          const double inv = 1.0 / ((double)(l + m) * (l - m));
          const double nr = ((2.0 * l - 1.0) * u[2] * cr - r2 * pr) * inv, ni = ((2.0 * l - 1.0) * u[2] * ci - r2 * pim) * inv;
          pr = cr; pim = ci; cr = nr; ci = ni;
        }
        const int k = (m == 0) ? l * l : l * l + 2 * m - 1;
        const double w = (m == 0) ? 1.0 : 2.0;
        if (!(l & 1)) H += (m == 0) ? eh[k] * cr : w * (eh[k] * cr + eh[k + 1] * ci);
        else if (l < P) {
          hx += (m == 0) ? ex[k] * cr : w * (ex[k] * cr + ex[k + 1] * ci);
          hy += (m == 0) ? ey[k] * cr : w * (ey[k] * cr + ey[k + 1] * ci);
          hz += (m == 0) ? ez[k] * cr : w * (ez[k] * cr + ez[k + 1] * ci);
        }
      }
    }
    A += H / L + c2 * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    g0 += hx / (L * L) + 2.0 * c2 * r[0];
    g1 += hy / (L * L) + 2.0 * c2 * r[1];
    g2 += hz / (L * L) + 2.0 * c2 * r[2];
    ksum += Di * Dj * A;
    if (ia == ja) gsum += Di * phi[i];
    else if (forces) {
      const double wgt = lw * fcoul * Di * Dj;
      atomicAdd(&fsh[wib][ia][0], -wgt * g0);
      atomicAdd(&fsh[wib][ia][1], -wgt * g1);
      atomicAdd(&fsh[wib][ia][2], -wgt * g2);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    ksum += __shfl_xor_sync(0xffffffff, ksum, o);
    gsum += __shfl_xor_sync(0xffffffff, gsum, o);
  }
  __syncwarp();
  const double k = fcoul * ksum;
  if (lane == 0) {
    if (dEdl) dEdl[site] = gsum + (0.5 - lam[site]) * k;
    site_energy[site] = 0.5 * lw * k;
  }
  if (forces)
    for (int k3 = lane; k3 < n * 3; k3 += 32) {
      const int ia = k3 / 3, a = k3 % 3, i = site_atoms[b + ia];
      forces[3 * (size_t)i + a] = (FT)((double)forces[3 * (size_t)i + a] + fsh[wib][ia][a]);
    }
}

// fixed-order sum of the per-site energies
__global__ void k_sum_static(int S, const double *__restrict__ site_energy, double *__restrict__ out) {
  __shared__ double red[32];
  double v = 0.0;
  for (int s = threadIdx.x; s < S; s += blockDim.x) v += site_energy[s];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}

}  // namespace
}  // namespace mahi

extern "C" int mahi_site_terms_static(double box_L_nm, int32_t n_sites, const int32_t *site_ptr,
                                      const int32_t *site_atoms, const void *x, int32_t x_is_fp64, const double *qA,
                                      const double *qB, const double *lambda, const double *phi, double *dEdlambda,
                                      double *energy_correction, void *forces, void *cuda_stream) {
  using namespace mahi;
  if (!(box_L_nm > 0.0) || !std::isfinite(box_L_nm) || n_sites < 0) return MAHI_ERR_INVALID_ARG;
  if (n_sites > kStaticMaxSites) return MAHI_ERR_INVALID_ARG;  // beyond the static scratch
  if (n_sites > 0 && (!site_ptr || !site_atoms || !x || !qA || !qB || !lambda || !phi)) return MAHI_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MAHI_ERR_NO_DEVICE;
  {
    // one-time set-up for this device (the current one): resolve the device
    // addresses of the file-scope arrays and fill the lattice tables
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
      static double tab[4][kStaticCoef];
      h1_tables(tab);
      if (cudaMemcpyToSymbol(g_eta, tab, sizeof(tab)) != cudaSuccess) return MAHI_ERR_CUDA;
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_site_energy) != cudaSuccess) return MAHI_ERR_CUDA;
      g_energy_ptr[dev] = static_cast<double *>(p);
      if (cudaGetSymbolAddress(&p, g_eta) != cudaSuccess) return MAHI_ERR_CUDA;
      g_eta_ptr[dev] = static_cast<double *>(p);
      g_ready[dev] = true;
    }
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const double f = coulomb_constant();
  if (n_sites > 0) {
    const int blocks = (n_sites + 3) / 4;
    if (x_is_fp64)
      k_site_static<double, double><<<blocks, 128, 0, st>>>(n_sites, box_L_nm, f, site_ptr, site_atoms,
                                                            (const double *)x, qA, qB, lambda, phi, g_eta_ptr[dev],
                                                            g_energy_ptr[dev], dEdlambda, (double *)forces);
    else
      k_site_static<float, float><<<blocks, 128, 0, st>>>(n_sites, box_L_nm, f, site_ptr, site_atoms,
                                                          (const float *)x, qA, qB, lambda, phi, g_eta_ptr[dev],
                                                          g_energy_ptr[dev], dEdlambda, (float *)forces);
  }
  if (energy_correction) k_sum_static<<<1, 256, 0, st>>>(n_sites, g_energy_ptr[dev], energy_correction);
  return cudaGetLastError() == cudaSuccess ? MAHI_OK : MAHI_ERR_CUDA;
}
