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
// the first-shell lattice function (4 x 41^2 doubles, filled from the host
// planner's coefficients, the same ones mahi_create uploads); every GPU that
// loads the library holds them until the process exits.  All calls share the
// scratch and keep the last call's contents; calls whose work overlaps on the
// GPU race.  Every site is validated (offsets, size, atom indices) before any
// per-atom array is touched.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

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

// Coefficients of the first-shell lattice function H_1 (degree kStaticDeg, real
// layout) and of its gradient (degree kStaticDeg - 1) from the library's host
// planner: the same tables the evaluation path uploads.
void h1_tables(double (*tab)[kStaticCoef]) {
  const std::vector<double> &eta = lattice_coeffs(kStaticDeg, 1);
  std::memset(tab, 0, sizeof(double) * 4 * kStaticCoef);
  std::memcpy(tab[0], eta.data(), sizeof(double) * kStaticCoef);
  gradient_coeffs(kStaticDeg, eta.data(), tab[1], tab[2], tab[3]);
}

template <typename XT, typename FT>
__global__ void k_site_static(int S, int64_t n_atoms, double L, double fcoul, const int *__restrict__ site_ptr,
                              const int *__restrict__ site_atoms, const XT *__restrict__ x,
                              const double *__restrict__ qA, const double *__restrict__ qB,
                              const double *__restrict__ lam, const double *__restrict__ phi,
                              const double *__restrict__ eta, double *__restrict__ site_energy,
                              double *__restrict__ dEdl, FT *__restrict__ forces) {
  __shared__ double fsh[4][kStaticMaxSiteAtoms][3];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int site = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (site >= S) return;
  // validate the site before any per-atom array is read: offsets in order and
  // within site_ptr[S], 1..64 atoms, every atom index in [0, n_atoms)
  const int b = site_ptr[site], n = site_ptr[site + 1] - b, total = site_ptr[S];
  bool bad = b < 0 || n < 1 || n > kStaticMaxSiteAtoms || b + n > total;
  if (!bad) {
    bool mine = false;
    for (int a = lane; a < n; a += 32) {
      const int i = site_atoms[b + a];
      mine = mine || i < 0 || (int64_t)i >= n_atoms;
    }
    bad = __any_sync(0xffffffffu, mine);
  }
  if (bad) {  // malformed site: flag it, touch nothing else
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

extern "C" int mahi_site_terms_static(double box_L_nm, int64_t n_atoms, int32_t n_sites, const int32_t *site_ptr,
                                      const int32_t *site_atoms, const void *x, int32_t x_is_fp64, const double *qA,
                                      const double *qB, const double *lambda, const double *phi, double *dEdlambda,
                                      double *energy_correction, void *forces, void *cuda_stream) {
  using namespace mahi;
  if (!(box_L_nm > 0.0) || !std::isfinite(box_L_nm) || n_sites < 0) return MAHI_ERR_INVALID_ARG;
  if (n_sites > kStaticMaxSites) return MAHI_ERR_INVALID_ARG;  // beyond the static scratch
  if (n_sites > 0 && (n_atoms < 1 || !site_ptr || !site_atoms || !x || !qA || !qB || !lambda || !phi))
    return MAHI_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MAHI_ERR_NO_DEVICE;
  {
    // one-time set-up for this device (the current one): resolve the device
    // addresses of the file-scope arrays and fill the lattice tables
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
      static double tab[4][kStaticCoef];
      h1_tables(tab);
      cudaError_t e = cudaMemcpyToSymbol(g_eta, tab, sizeof(tab));
      if (e != cudaSuccess) return cuda_fail(e, "mahi_site_terms_static: lattice tables");
      void *p = nullptr;
      if ((e = cudaGetSymbolAddress(&p, g_site_energy)) != cudaSuccess)
        return cuda_fail(e, "mahi_site_terms_static: scratch address");
      g_energy_ptr[dev] = static_cast<double *>(p);
      if ((e = cudaGetSymbolAddress(&p, g_eta)) != cudaSuccess)
        return cuda_fail(e, "mahi_site_terms_static: table address");
      g_eta_ptr[dev] = static_cast<double *>(p);
      g_ready[dev] = true;
    }
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double f = coulomb_constant();
  double L = box_L_nm;
  int S = n_sites;
  int64_t na = n_atoms;
  double *eta = g_eta_ptr[dev], *sen = g_energy_ptr[dev];
  if (n_sites > 0) {
    // launched through cudaLaunchKernel so that the error returned is this launch's own
    void *args[] = {&S, &na, &L, &f, (void *)&site_ptr, (void *)&site_atoms, (void *)&x, (void *)&qA, (void *)&qB,
                    (void *)&lambda, (void *)&phi, &eta, &sen, &dEdlambda, &forces};
    const void *fn = x_is_fp64 ? (const void *)k_site_static<double, double> : (const void *)k_site_static<float, float>;
    const cudaError_t e = cudaLaunchKernel(fn, dim3((n_sites + 3) / 4), dim3(128), args, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "mahi_site_terms_static: site kernel");
  }
  if (energy_correction) {
    void *args[] = {&S, &sen, &energy_correction};
    const cudaError_t e = cudaLaunchKernel((const void *)k_sum_static, dim3(1), dim3(256), args, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "mahi_site_terms_static: energy sum");
  }
  return MAHI_OK;
}
