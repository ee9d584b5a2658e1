// SIMT kernels of the MAHI evaluation and the eval orchestration.
//
// Data layout (HBM):
//   part[N]            sorted by leaf (Morton order), float4/double4
//                      (x - leaf centre [nm], q~); leaves are contiguous,
//                      leaf_start[8^d + 1] gives the ranges.
//   Mexp/Lexp          all levels, level l at level_off[l], one row of `ld`
//                      coefficients per box (Morton index within the level).
//   phi_s, grad_s      far-field potential / gradient per sorted atom.
// FP64 everywhere in MAHI_FP64, FP32 particle/expansion data in the mixed modes;
// scaled charges, multipole moments of the box, energies and the per-site
// corrections are always FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <cmath>
#include <cstdio>

#include "mahi_internal.h"
#include "mahi_sync.h"

namespace mahi {

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4_16a; };  // 32 bytes, 16-byte aligned

__device__ __forceinline__ uint32_t d_spread(uint32_t v) {
  uint32_t x = v & 0x3ff;
  x = (x | (x << 16)) & 0x030000FF;
  x = (x | (x << 8)) & 0x0300F00F;
  x = (x | (x << 4)) & 0x030C30C3;
  x = (x | (x << 2)) & 0x09249249;
  return x;
}
__device__ __forceinline__ uint32_t d_compact(uint32_t x) {
  x &= 0x09249249;
  x = (x ^ (x >> 2)) & 0x030C30C3;
  x = (x ^ (x >> 4)) & 0x0300F00F;
  x = (x ^ (x >> 8)) & 0x030000FF;
  x = (x ^ (x >> 16)) & 0x000003FF;
  return x;
}
__device__ __forceinline__ uint32_t d_morton(int x, int y, int z) {
  return d_spread(x) | (d_spread(y) << 1) | (d_spread(z) << 2);
}
__device__ __forceinline__ int wrapi(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

template <typename T> __device__ __forceinline__ T rsqrt_int(int a) { return T(1) / sqrt(T(a)); }
template <typename T> __device__ __forceinline__ T sqrt_ratio(int a, int b) { return sqrt(T(a) / T(b)); }

// ---------------------------------------------------------------------------
// Recursion coefficients (filled once by the host, mahi_upload_tables):
//   device basis  Rt: a_lm = (2l-1)/sqrt((l+m)(l-m)), b_lm = sqrt((l+m-1)(l-m-1)/((l+m)(l-m))),
//                     diag_m = sqrt((2m-1)/(2m))
//   plain basis   R : ua_lm = (2l-1)/((l+m)(l-m)),  ub_lm = 1/((l+m)(l-m)),  udiag_m = 1/(2m)
// indexed by tri(l, m) = l(l+1)/2 + m.
// ---------------------------------------------------------------------------
constexpr int kTriMax = (kMaxOrder + 1) * (kMaxOrder + 2) / 2;
constexpr int kTriSite = (kSiteDegree + 1) * (kSiteDegree + 2) / 2;
__constant__ double c_a[kTriMax], c_b[kTriMax], c_diag[kMaxOrder + 1];
__constant__ float c_af[kTriMax], c_bf[kTriMax], c_diagf[kMaxOrder + 1];
__constant__ double c_ua[kTriSite], c_ub[kTriSite], c_udiag[kSiteDegree + 1];

template <typename T> __device__ __forceinline__ T tab_a(int k);
template <> __device__ __forceinline__ float tab_a<float>(int k) { return c_af[k]; }
template <> __device__ __forceinline__ double tab_a<double>(int k) { return c_a[k]; }
template <typename T> __device__ __forceinline__ T tab_b(int k);
template <> __device__ __forceinline__ float tab_b<float>(int k) { return c_bf[k]; }
template <> __device__ __forceinline__ double tab_b<double>(int k) { return c_b[k]; }
template <typename T> __device__ __forceinline__ T tab_diag(int m);
template <> __device__ __forceinline__ float tab_diag<float>(int m) { return c_diagf[m]; }
template <> __device__ __forceinline__ double tab_diag<double>(int m) { return c_diag[m]; }

// Regular harmonics of the device basis, column by column (m outer, l inner),
// O(1) state: cb(l, m, re, im) gets Rt_lm for all 0 <= m <= l <= P.
template <typename T, class CB>
__device__ __forceinline__ void rt_columns(int P, T x, T y, T z, CB cb) {
  const T r2 = x * x + y * y + z * z;
  T dre = T(1), dim = T(0);
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    if (m > 0) {
      const T f = -tab_diag<T>(m);
      const T tr = f * (x * dre - y * dim), ti = f * (x * dim + y * dre);
      dre = tr; dim = ti;
    }
    T pr = T(0), pi = T(0), cr = dre, ci = dim;
    cb(m, m, cr, ci);
#pragma unroll
    for (int l = m + 1; l <= P; ++l) {
      const int k = l * (l + 1) / 2 + m;
      const T a = tab_a<T>(k) * z, b = tab_b<T>(k) * r2;
      const T nr = a * cr - b * pr, ni = a * ci - b * pi;
      pr = cr; pi = ci; cr = nr; ci = ni;
      cb(l, m, cr, ci);
    }
  }
}

// Irregular harmonics of the device basis It_lm = I_lm / sqrt((l+m)!(l-m)!):
// It_00 = 1/r, It_mm = -diag_m (x+iy)/r^2 It_{m-1,m-1},
// It_lm = (a_lm z It_{l-1,m} - b_lm It_{l-2,m}) / r^2.
template <typename T, class CB>
__device__ __forceinline__ void it_columns(int P, T x, T y, T z, CB cb) {
  const T r2 = x * x + y * y + z * z, ir2 = T(1) / r2;
  T dre = sqrt(ir2), dim = T(0);
  for (int m = 0; m <= P; ++m) {
    if (m > 0) {
      const T f = -tab_diag<T>(m) * ir2;
      const T tr = f * (x * dre - y * dim), ti = f * (x * dim + y * dre);
      dre = tr; dim = ti;
    }
    T pr = T(0), pi = T(0), cr = dre, ci = dim;
    cb(m, m, cr, ci);
    for (int l = m + 1; l <= P; ++l) {
      const int k = l * (l + 1) / 2 + m;
      const T a = tab_a<T>(k) * z * ir2, b = tab_b<T>(k) * ir2;
      const T nr = a * cr - b * pr, ni = a * ci - b * pi;
      pr = cr; pi = ci; cr = nr; ci = ni;
      cb(l, m, cr, ci);
    }
  }
}

// Plain regular harmonics R_lm (site kernel, FP64, degree <= kSiteDegree).
template <class CB>
__device__ __forceinline__ void r_columns(int P, double x, double y, double z, CB cb) {
  const double r2 = x * x + y * y + z * z;
  double dre = 1.0, dim = 0.0;
  for (int m = 0; m <= P; ++m) {
    if (m > 0) {
      const double f = -c_udiag[m];
      const double tr = f * (x * dre - y * dim), ti = f * (x * dim + y * dre);
      dre = tr; dim = ti;
    }
    double pr = 0.0, pi = 0.0, cr = dre, ci = dim;
    cb(m, m, cr, ci);
    for (int l = m + 1; l <= P; ++l) {
      const int k = l * (l + 1) / 2 + m;
      const double a = c_ua[k] * z, b = c_ub[k] * r2;
      const double nr = a * cr - b * pr, ni = a * ci - b * pi;
      pr = cr; pi = ci; cr = nr; ci = ni;
      cb(l, m, cr, ci);
    }
  }
}

// 1/sqrt(r2) to FP64 accuracy from the FP32 hardware estimate and two FP64
// Newton-Raphson steps y <- y (3 - r2 y^2)/2 (each squares the relative error)
__device__ __forceinline__ double rsqrt_dp(double r2) {
  double y = (double)rsqrtf((float)r2);
  y = y * fma(-0.5 * r2, y * y, 1.5);
  y = y * fma(-0.5 * r2, y * y, 1.5);
  return y;
}

// real-layout index of (l, m >= 0): Re part (Im = +1 for m > 0)
__device__ __forceinline__ int ridx(int l, int m) { return m == 0 ? l * l : l * l + 2 * m - 1; }

// ---------------------------------------------------------------------------
// 1. scale charges, bin atoms into leaves.  GB300 runs FP64 at a small fraction
//    of its FP32 rate, so every per-atom FP64 operation counts: positions
//    already inside the box skip the wrap, the leaf index comes from one
//    multiplication, the leaf centres from a shared table.  Per atom this
//    writes the leaf, its slot in the leaf, q~ (FP64), the offset from the leaf
//    centre (FP64) and the working-precision particle (offset, q~), all in
//    the original atom order.
// ---------------------------------------------------------------------------
constexpr int kMaxSide = 1 << kMaxDepth;  // leaves along one edge
constexpr int kQD = 8;                    // doubles per box in box_qd: Q, Dx, Dy, Dz, T, pad
constexpr int kQDF = 8;                   // floats per box in box_qdf: Q, Dx, Dy, Dz as (hi, lo)

// wrapped coordinate in [0, L); the in-box test is exact: Lf_up is the
// smallest float >= L, so x < Lf_up <=> x < L for a float x
__device__ __forceinline__ double wrap_slow(double v, double L) {
  v -= floor(v / L) * L;
  if (v >= L) v -= L;
  if (v < 0.0) v = 0.0;
  return v;
}
__device__ __forceinline__ double wrap_coord(float x, double L, float Lf_up) {
  return (x >= 0.f && x < Lf_up) ? (double)x : wrap_slow((double)x, L);
}
__device__ __forceinline__ double wrap_coord(double x, double L, float) {
  return (x >= 0.0 && x < L) ? x : wrap_slow(x, L);
}

template <typename T, typename XT>
__global__ void k_bin(const XT *__restrict__ x, int64_t N, double L, double s, double inv_s, float Lf_up, int nb,
                      const double *__restrict__ lam, const double *__restrict__ qA, const double *__restrict__ dq,
                      const int *__restrict__ site_of, int *__restrict__ leaf_of, int *__restrict__ slot,
                      int *__restrict__ leaf_count, double *__restrict__ qt, typename V4<T>::type *__restrict__ vtmp,
                      double *__restrict__ relD) {
  __shared__ double ctab[kMaxSide];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) ctab[i] = (i + 0.5) * s;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double p[3];
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      p[a] = wrap_coord(x[3 * i + a], L, Lf_up);
      c[a] = min((int)(p[a] * inv_s), nb - 1);
      p[a] -= ctab[c[a]];
    }
    const int st = site_of[i];
    const double q = st >= 0 ? fma(lam[st], dq[i], qA[i]) : qA[i];
    qt[i] = q;
    const int leaf = (int)d_morton(c[0], c[1], c[2]);
    leaf_of[i] = leaf;
    slot[i] = atomicAdd(&leaf_count[leaf], 1);
    relD[3 * i + 0] = p[0];
    relD[3 * i + 1] = p[1];
    relD[3 * i + 2] = p[2];
    vtmp[i] = typename V4<T>::type{(T)p[0], (T)p[1], (T)p[2], (T)q};
  }
}

// deterministic reduction of per-block partials: out[k] = sum_b part[b*nk + k]
__global__ void k_reduce_partials(const double *__restrict__ part, int nblocks, int nk, double *__restrict__ out,
                                  double scale) {
  int k = blockIdx.x;
  double v = 0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += part[(size_t)b * nk + k];
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    out[k] = s * scale;
  }
}

// exclusive scan of the leaf counts (one block of 1024 threads): every thread
// owns a contiguous run of n / 1024 counts (n is a power of 8), read and
// written as int4 where the run allows it
__global__ void __launch_bounds__(1024) k_scan(const int *__restrict__ cnt, int n, int *__restrict__ start) {
  __shared__ int wsum[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int b = min(n, t * per), e = min(n, b + per);
  int loc = 0;
  const bool vec = (per % 4) == 0 && (e - b) == per;
  if (vec) {
    for (int i = b; i < e; i += 4) {
      const int4 v = *reinterpret_cast<const int4 *>(cnt + i);
      loc += v.x + v.y + v.z + v.w;
    }
  } else {
    for (int i = b; i < e; ++i) loc += cnt[i];
  }
  int inc = loc;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffff, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    int v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffff, v, o);
      if (lane >= o) v += y;
    }
    wsum[lane] = v;  // inclusive
  }
  __syncthreads();
  int run = inc - loc + (w > 0 ? wsum[w - 1] : 0);
  if (vec) {
    for (int i = b; i < e; i += 4) {
      const int4 v = *reinterpret_cast<const int4 *>(cnt + i);
      int4 o;
      o.x = run; run += v.x;
      o.y = run; run += v.y;
      o.z = run; run += v.z;
      o.w = run; run += v.w;
      *reinterpret_cast<int4 *>(start + i) = o;
    }
  } else {
    for (int i = b; i < e; ++i) { start[i] = run; run += cnt[i]; }
  }
  if (t == blockDim.x - 1) start[n] = run;
}

template <typename T>
__global__ void k_scatter(int64_t N, const int *__restrict__ leaf_of, const int *__restrict__ slot,
                          const int *__restrict__ leaf_start, const typename V4<T>::type *__restrict__ vtmp,
                          typename V4<T>::type *__restrict__ part_tmp, int *__restrict__ perm_tmp) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int pos = leaf_start[leaf_of[i]] + slot[i];
  part_tmp[pos] = vtmp[i];
  perm_tmp[pos] = (int)i;
}

// Order the atoms of every leaf by original index (deterministic layout).
template <typename T>
__global__ void k_leaf_sort(int nleaf, const int *__restrict__ leaf_start, const typename V4<T>::type *__restrict__ part_tmp,
                            const int *__restrict__ perm_tmp, typename V4<T>::type *__restrict__ part,
                            int *__restrict__ perm, int *__restrict__ inv_perm) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nleaf) return;
  int b = leaf_start[warp], e = leaf_start[warp + 1];
  for (int a = b + lane; a < e; a += 32) {
    int key = perm_tmp[a], rank = 0;
    for (int j = b; j < e; ++j) rank += (perm_tmp[j] < key);
    part[b + rank] = part_tmp[a];
    perm[b + rank] = key;
    inv_perm[key] = b + rank;
  }
}

// The FP64 charge Q, dipole D and second moment T = sum q |x - c|^2 of every
// leaf about its centre c, summed over its atoms in the sorted order.  These
// feed the l <= 1 terms of the site-atom potential and, through exact
// translation up the tree, the dipole / background term of the periodic
// kernel.  One thread per leaf: FP64 issues at a small fraction of the FP32
// rate on GB300, and a warp-wide FP64 reduction per leaf would cost far more
// instructions than the sums themselves.
// Q and D as (hi, lo) float pairs beside the FP64 row: the site-atom
// potential forms its charge/dipole terms in double-float
__device__ __forceinline__ void qd_split(const double *v, float *f) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float hi = (float)v[k];
    f[2 * k] = hi;
    f[2 * k + 1] = (float)(v[k] - (double)hi);
  }
}

__global__ void k_leaf_moments(int nleaf, const int *__restrict__ leaf_start, const int *__restrict__ perm,
                               const double *__restrict__ qt, const double *__restrict__ relD,
                               double *__restrict__ qd, float *__restrict__ qdf) {
  const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
  if (leaf >= nleaf) return;
  const int b = leaf_start[leaf], e = leaf_start[leaf + 1];
  double v[5] = {0, 0, 0, 0, 0};
#pragma unroll 4
  for (int a = b; a < e; ++a) {
    const int i = perm[a];
    const double q = qt[i], rx = relD[3 * (size_t)i], ry = relD[3 * (size_t)i + 1], rz = relD[3 * (size_t)i + 2];
    v[0] += q;
    v[1] = fma(q, rx, v[1]);
    v[2] = fma(q, ry, v[2]);
    v[3] = fma(q, rz, v[3]);
    v[4] = fma(q, rx * rx + ry * ry + rz * rz, v[4]);
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) qd[(size_t)leaf * kQD + k] = v[k];
  qd_split(v, qdf + (size_t)leaf * kQDF);
}

// ---------------------------------------------------------------------------
// 2. P2M: one warp per leaf, lanes = atoms, warp reductions per coefficient.
//    M^_lm = sum_i q_i conj(R_lm(u_i)), u = (x - c)/s
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_p2m(int nleaf, int P, int ld, T inv_s, const int *__restrict__ leaf_start,
                      const typename V4<T>::type *__restrict__ part, T *__restrict__ M) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
  if (warp >= nleaf) return;
  T *acc = reinterpret_cast<T *>(smem_raw) + (size_t)wib * ld;
  for (int k = lane; k < ld; k += 32) acc[k] = T(0);
  __syncwarp();
  const int b = leaf_start[warp], e = leaf_start[warp + 1];
  for (int base = b; base < e; base += 32) {
    const int a = base + lane;
    const bool valid = a < e;
    const typename V4<T>::type pt = valid ? part[a] : typename V4<T>::type{0, 0, 0, 0};
    const T q = valid ? pt.w : T(0);
    rt_columns<T>(P, pt.x * inv_s, pt.y * inv_s, pt.z * inv_s, [&](int l, int m, T re, T im) {
      T vr = q * re, vi = -q * im;  // conj
      for (int o = 16; o > 0; o >>= 1) {
        vr += __shfl_xor_sync(0xffffffff, vr, o);
        vi += __shfl_xor_sync(0xffffffff, vi, o);
      }
      if (lane == 0) {
        const int k = ridx(l, m);
        acc[k] += vr;
        if (m > 0) acc[k + 1] += vi;
      }
    });
  }
  __syncwarp();
  T *out = M + (size_t)warp * ld;
  for (int k = lane; k < ld; k += 32) out[k] = acc[k];
}

// P2M with the lane reduction done through shared memory: each lane writes the
// K coefficients q conj(R_lm(u)) of its atom into a row of a 32 x Ks buffer
// (Ks = K rounded up to odd, so row writes do not share banks), then lane j
// sums the columns j, j + 32, ... over the rows in row order.  Same sums in the
// same order for every run; no shuffle chains.  PP > 0 makes the order a
// compile-time constant (the harmonic recursion is then unrolled).
template <typename T, int PP>
__global__ void k_p2m_t(int nleaf, int Pr, int ld, int Ks, T inv_s, const int *__restrict__ leaf_start,
                        const typename V4<T>::type *__restrict__ part, T *__restrict__ M) {
  const int P = PP > 0 ? PP : Pr;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
  if (warp >= nleaf) return;
  T *buf = reinterpret_cast<T *>(smem_raw) + (size_t)wib * 32 * Ks;
  T *row = buf + (size_t)lane * Ks;
  constexpr int kMaxCols = (kMaxOrderMixed + 1) * (kMaxOrderMixed + 1) / 32 + 1;
  T acc[kMaxCols];
#pragma unroll
  for (int r = 0; r < kMaxCols; ++r) acc[r] = T(0);
  const int K = (P + 1) * (P + 1);
  const int b = leaf_start[warp], e = leaf_start[warp + 1];
  for (int base = b; base < e; base += 32) {
    const int a = base + lane;
    const int na = min(32, e - base);
    if (a < e) {
      const typename V4<T>::type pt = part[a];
      const T q = pt.w;
      rt_columns<T>(P, pt.x * inv_s, pt.y * inv_s, pt.z * inv_s, [&](int l, int m, T re, T im) {
        const int k = ridx(l, m);
        row[k] = q * re;
        if (m > 0) row[k + 1] = -q * im;  // conj
      });
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kMaxCols; ++r) {
      const int k = lane + 32 * r;
      if (k < K) {
        T v = acc[r];
        for (int i = 0; i < na; ++i) v += buf[(size_t)i * Ks + k];
        acc[r] = v;
      }
    }
    __syncwarp();
  }
  T *out = M + (size_t)warp * ld;
#pragma unroll
  for (int r = 0; r < kMaxCols; ++r) {
    const int k = lane + 32 * r;
    if (k < ld) out[k] = (k < K) ? acc[r] : T(0);
  }
}

// P2M for a compile-time order with a 32 x 33 staging buffer per warp
// instead of 32 x K: every lane (atom) produces its K coefficients
// q conj(R_lm(u)) in the recursion's order (m outer, l inner; re, then im for
// m > 0) and writes them into the buffer 32 at a time; after each 32 the warp
// adds up the buffer's columns (lane j: production index 32 c + j, sum over
// the 32 atoms in lane order).  Lanes without an atom carry charge 0 and add
// exact zeros.  The small buffer lets ~50 warps run per SM instead of 10.
__device__ __forceinline__ int p2m_prod_ridx(int P, int p) {
  for (int m = 0; m <= P; ++m) {
    const int per = (P - m + 1) * (m > 0 ? 2 : 1);
    if (p < per) return m > 0 ? ridx(m + p / 2, m) + (p & 1) : ridx(m + p, 0);
    p -= per;
  }
  return -1;
}

template <typename T, int PP>
__global__ void __launch_bounds__(128) k_p2m_c(int nleaf, int ld, T inv_s, const int *__restrict__ leaf_start,
                                               const typename V4<T>::type *__restrict__ part, T *__restrict__ M) {
  using V = typename V4<T>::type;
  constexpr int K = (PP + 1) * (PP + 1);
  constexpr int NC = (K + 31) / 32;
  __shared__ T buf[4][32][33];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int warp = blockIdx.x * 4 + wib;
  if (warp >= nleaf) return;  // whole warps only
  T(*bw)[33] = buf[wib];
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
  const int b = leaf_start[warp], e = leaf_start[warp + 1];
  for (int base = b; base < e; base += 32) {
    const int a = base + lane;
    const V pt = (a < e) ? part[a] : V{0, 0, 0, 0};
    const T q = pt.w;
    int pidx = 0;  // production index (a constant at every call site once unrolled)
    auto put = [&](T v) {
      bw[lane][pidx & 31] = v;
      if ((pidx & 31) == 31) {
        __syncwarp();
        T sum = T(0);
#pragma unroll 8
        for (int i = 0; i < 32; ++i) sum += bw[i][lane];
        acc[pidx >> 5] += sum;
        __syncwarp();
      }
      ++pidx;
    };
    rt_columns<T>(PP, pt.x * inv_s, pt.y * inv_s, pt.z * inv_s, [&](int l, int m, T re, T im) {
      put(q * re);
      if (m > 0) put(-q * im);  // conj
    });
    if constexpr (K % 32 != 0) {  // the last, partial group of 32
      __syncwarp();
      T sum = T(0);
#pragma unroll 8
      for (int i = 0; i < 32; ++i) sum += bw[i][lane];
      if (lane < K % 32) acc[NC - 1] += sum;
      __syncwarp();
    }
  }
  T *out = M + (size_t)warp * ld;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int p = 32 * c + lane;
    if (p < K) out[p2m_prod_ridx(PP, p)] = acc[c];
  }
  for (int k = K + lane; k < ld; k += 32) out[k] = T(0);
}

// ---------------------------------------------------------------------------
// 3. Gather-GEMM for M2M, L2L and (SIMT) M2L.  A tile of TR output rows shares
//    one operator per term; out[row] (+)= sum_terms op[term] * in[src(row, term)].
// ---------------------------------------------------------------------------
struct GemmMap {
  int kind;        // 0 = M2M, 1 = L2L, 2 = M2L
  int level;       // level of the output rows
  int nbox;        // boxes at the output level
  const int *list; // M2L: [8][189] offset ids
  const int *off;  // M2L: [316][3]
};

constexpr int TR = 32;   // rows per tile
constexpr int TK = 16;   // input coefficients per pipeline stage

__device__ __forceinline__ void cpa16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem)
               : "memory");
}

// Operators are stored transposed and zero padded: opT[term][k][n] with k, n < ld.
// Two-stage cp.async pipeline over (term, k-chunk); all source rows of the tile
// are resolved up front.
template <typename T, int NC>
__global__ void __launch_bounds__(256) k_gather_gemm(GemmMap mp, int K, int ld, const T *__restrict__ in,
                                                     T *__restrict__ out, const T *__restrict__ opsT) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nterms = (mp.kind == 0) ? 8 : (mp.kind == 1 ? 1 : kListLen);
  constexpr int LDB = 32 * NC;                         // B row stride >= ld: columns ld..LDB-1 stay zero
  T *As = reinterpret_cast<T *>(smem_raw);            // [2][TR][TK]
  T *Bs = As + 2 * TR * TK;                            // [2][TK][LDB]
  int *src = reinterpret_cast<int *>(Bs + 2 * TK * LDB);  // [nterms][TR]
  for (int i = threadIdx.x; i < 2 * TK * LDB; i += blockDim.x) Bs[i] = T(0);
  const int tid = threadIdx.x;
  const int tg = tid >> 5, cg = tid & 31;
  int c = 0, tp = blockIdx.x, nrow_par;
  if (mp.kind == 0) nrow_par = mp.nbox;
  else { nrow_par = mp.nbox / 8; c = blockIdx.x % 8; tp = blockIdx.x / 8; }
  const int row0 = tp * TR;
  const int side = 1 << mp.level;
  for (int i = tid; i < nterms * TR; i += blockDim.x) {
    const int term = i / TR, r = i % TR, P = row0 + r;
    int sidx = -1;
    if (P < nrow_par) {
      if (mp.kind == 0) sidx = 8 * P + term;
      else if (mp.kind == 1) sidx = P;
      else {
        const int box = 8 * P + c;
        const int bx = (int)d_compact(box), by = (int)d_compact(box >> 1), bz = (int)d_compact(box >> 2);
        const int oid = mp.list[c * kListLen + term];
        sidx = (int)d_morton(wrapi(bx - mp.off[oid * 3 + 0], side), wrapi(by - mp.off[oid * 3 + 1], side),
                             wrapi(bz - mp.off[oid * 3 + 2], side));
      }
    }
    src[i] = sidx;
  }
  __syncthreads();
  const int nch = ld / TK;            // ld is a multiple of 16
  const int total = nterms * nch;
  constexpr int EPV = 16 / sizeof(T);  // elements per 16-byte copy
  auto issue = [&](int it, int stg) {
    const int term = it / nch, k0 = (it % nch) * TK;
    const int oid = (mp.kind == 0) ? term : (mp.kind == 1 ? c : mp.list[c * kListLen + term]);
    const T *op = opsT + (size_t)oid * ld * ld;
    T *a = As + stg * TR * TK;
    T *b = Bs + stg * TK * LDB;
    for (int i = tid; i < TR * (TK / EPV); i += blockDim.x) {
      const int r = i / (TK / EPV), q = i % (TK / EPV);
      const int sidx = src[term * TR + r];
      T *dst = a + r * TK + q * EPV;
      if (sidx >= 0) cpa16(dst, in + (size_t)sidx * ld + k0 + q * EPV);
      else
        for (int e = 0; e < EPV; ++e) dst[e] = T(0);
    }
    const int per_row = ld / EPV;
    for (int i = tid; i < TK * per_row; i += blockDim.x) {
      const int kk = i / per_row, q = i % per_row;
      cpa16(b + kk * LDB + q * EPV, op + (size_t)(k0 + kk) * ld + q * EPV);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  T acc[4][NC];
  for (int r = 0; r < 4; ++r)
    for (int j = 0; j < NC; ++j) acc[r][j] = T(0);
  const int ncols = (K + 31) / 32;
  issue(0, 0);
  for (int it = 0; it < total; ++it) {
    if (it + 1 < total) {
      issue(it + 1, (it + 1) & 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const T *a = As + (it & 1) * TR * TK;
    const T *b = Bs + (it & 1) * TK * LDB;
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      T av[4];
      for (int r = 0; r < 4; ++r) av[r] = a[(tg * 4 + r) * TK + kk];
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const T bv = b[kk * LDB + cg + 32 * j];
        for (int r = 0; r < 4; ++r) acc[r][j] += av[r] * bv;
      }
    }
    __syncthreads();
  }
  for (int r = 0; r < 4; ++r) {
    const int P = row0 + tg * 4 + r;
    if (P >= nrow_par) continue;
    const int orow = (mp.kind == 0) ? P : 8 * P + c;
    T *o = out + (size_t)orow * ld;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int col = cg + 32 * j;
      if (j < ncols && col < K) {
        if (mp.kind == 1) o[col] += acc[r][j];
        else o[col] = acc[r][j];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// 3b. Dense GEMM for M2M and L2L (Fig. "fmm_scheme" steps 2 and 4).  Children
//     of a parent P are the consecutive rows 8P..8P+7 of the next level, so
//       M2M: M_l[P] = sum_c T_c M_{l+1}[8P+c]   is  C[nP x ld]  = A[nP x 8ld] B[8ld x ld]
//       L2L: L_l[8P+c] += T'_c L_{l-1}[P]        is  C[nP x 8ld] += A[nP x ld] B'[ld x 8ld]
//     with A and C plain row-major views of the expansion arrays and B the
//     stacked (transposed, zero-padded) operators.  64 x 64 tiles, K steps of
//     16, 256 threads with 4 x 4 outputs each, register-staged double buffer.
// ---------------------------------------------------------------------------
constexpr int GB_M = 64, GB_N = 64, GB_K = 16;

// blockIdx.z = split of the K range (nsplit = gridDim.z); with more than one
// split, split z writes its partial product to W[z] (M x N) and k_gemm_reduce
// adds the splits in order
template <typename T, bool ACC>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int Kd, const T *__restrict__ A, int lda,
                                              const T *__restrict__ B, int ldb, T *__restrict__ C, int ldc,
                                              T *__restrict__ W) {
  __shared__ __align__(16) T As[2][GB_K][GB_M + 4];  // A tile, k-major
  __shared__ __align__(16) T Bs[2][GB_K][GB_N];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
  // global -> register staging: 4 consecutive elements per thread and matrix
  const int ar = tid >> 2, ak = (tid & 3) * 4;   // A: row ar, k ak..ak+3
  const int bk = tid >> 4, bn = (tid & 15) * 4;  // B: row bk, n bn..bn+3
  T ra[4], rb[4];
  auto load = [&](int k0) {
    const int gm = m0 + ar;
#pragma unroll
    for (int e = 0; e < 4; ++e) ra[e] = (gm < M) ? A[(size_t)gm * lda + k0 + ak + e] : T(0);
    const int gn = n0 + bn;
#pragma unroll
    for (int e = 0; e < 4; ++e) rb[e] = (gn + e < N) ? B[(size_t)(k0 + bk) * ldb + gn + e] : T(0);
  };
  auto store = [&](int stg) {
#pragma unroll
    for (int e = 0; e < 4; ++e) As[stg][ak + e][ar] = ra[e];
#pragma unroll
    for (int e = 0; e < 4; ++e) Bs[stg][bk][bn + e] = rb[e];
  };
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  const int nkt = Kd / GB_K, z = blockIdx.z, nz = gridDim.z;
  const int kt0 = (int)((int64_t)z * nkt / nz), kt1 = (int)((int64_t)(z + 1) * nkt / nz);
  load(kt0 * GB_K);
  store(0);
  __syncthreads();
  for (int kt = kt0; kt < kt1; ++kt) {
    const int stg = (kt - kt0) & 1;
    if (kt + 1 < kt1) load((kt + 1) * GB_K);
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[stg][kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[stg][kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    if (kt + 1 < kt1) store(stg ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      if (nz > 1) {
        W[((size_t)z * M + gm) * N + gn] = acc[i][j];
      } else {
        T *c = C + (size_t)gm * ldc + gn;
        if (ACC) *c += acc[i][j];
        else *c = acc[i][j];
      }
    }
  }
}

// The coarse levels have few elements and up to ~80 splits, so the loads of
// eight splits are issued together (the sum itself stays in split order).
template <typename T, bool ACC>
__global__ void k_gemm_reduce(int M, int N, int nz, const T *__restrict__ W, T *__restrict__ C, int ldc) {
  const int64_t n = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    T v = W[e];
    int z = 1;
    for (; z + 8 <= nz; z += 8) {
      T w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) w[u] = W[(size_t)(z + u) * n + e];
#pragma unroll
      for (int u = 0; u < 8; ++u) v += w[u];
    }
    for (; z < nz; ++z) v += W[(size_t)z * n + e];
    T *c = C + (e / N) * ldc + (e % N);
    if (ACC) *c += v;
    else *c = v;
  }
}

// K splits that give about four blocks per SM (the coarse levels have few
// output tiles and long K loops)
static inline int gemm_splits(int M, int N, int Kd, int num_sms) {
  const int tiles = ((N + GB_N - 1) / GB_N) * ((M + GB_M - 1) / GB_M);
  const int nkt = Kd / GB_K;
  return std::max(1, std::min(nkt, (4 * num_sms + tiles - 1) / tiles));
}

template <typename T, bool ACC>
static cudaError_t launch_dense_gemm(int M, int N, int Kd, const T *A, int lda, const T *B, int ldb, T *C, int ldc,
                                     T *W, size_t w_elems, int num_sms, cudaStream_t st, int &launches) {
  if (Kd % GB_K) return cudaErrorInvalidValue;
  int nz = gemm_splits(M, N, Kd, num_sms);
  if ((size_t)nz * M * N > w_elems) nz = 1;
  dim3 grid((N + GB_N - 1) / GB_N, (M + GB_M - 1) / GB_M, nz);
  k_gemm<T, ACC><<<grid, 256, 0, st>>>(M, N, Kd, A, lda, B, ldb, C, ldc, W);
  ++launches;
  if (nz > 1) {
    const int64_t n = (int64_t)M * N;
    k_gemm_reduce<T, ACC><<<(int)std::min<int64_t>(4 * num_sms, (n + 255) / 256), 256, 0, st>>>(M, N, nz, W, C, ldc);
    ++launches;
  }
  return cudaGetLastError();
}

// workspace (elements) for the K splits of every M2M and L2L GEMM of a tree
size_t gemm_workspace_elems(int d, int ld, int num_sms) {
  size_t w = 0;
  for (int l = 0; l < d; ++l) {  // M2M into level l, L2L out of level l
    const int M = 1 << (3 * l);
    const int a = gemm_splits(M, ld, 8 * ld, num_sms), b = gemm_splits(M, 8 * ld, ld, num_sms);
    if (a > 1) w = std::max(w, (size_t)a * M * ld);
    if (b > 1) w = std::max(w, (size_t)b * M * 8 * ld);
  }
  return w;
}

// ---------------------------------------------------------------------------
// 4. Root lattice operator (FP64): L^_root = Lambda M^_root, with the monopole
//    and dipole of the root multipole taken from the FP64 moments.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_lattice(int K, int ld, double L, const double *__restrict__ lat, const double *__restrict__ lat_h3,
                          const double *__restrict__ mom, const T *__restrict__ Mroot, T *__restrict__ Lroot,
                          double *__restrict__ Lh3) {
  // one warp per output row, spread over the GPU (the FP64 rate per SM is low)
  extern __shared__ double ms[];
  for (int k = threadIdx.x; k < K; k += blockDim.x) ms[k] = (double)Mroot[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    // monopole and dipole of the root multipole from the FP64 moments:
    // M_00 = Q, M_10 = D_z, M_11 = conj(-(D_x + i D_y)/2); normalised by L^l and
    // scaled by c_10 = 1, c_11 = sqrt(2)
    ms[0] = mom[0];
    if (K > 3) {
      const double r2 = 0.70710678118654752440;
      ms[1] = mom[3] / L;
      ms[2] = -r2 * mom[1] / L;
      ms[3] = r2 * mom[2] / L;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r < K) {
    double s = 0, s3 = 0;
    for (int k = lane; k < K; k += 32) {
      s = fma(lat[(size_t)r * K + k], ms[k], s);
      s3 = fma(lat_h3[(size_t)r * K + k], ms[k], s3);
    }
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xffffffff, s, o);
      s3 += __shfl_xor_sync(0xffffffff, s3, o);
    }
    if (lane == 0) {
      Lroot[r] = (T)s;
      Lh3[r] = s3;
    }
  } else if (r < ld && lane == 0) {
    Lroot[r] = T(0);
  }
}

// ---------------------------------------------------------------------------
// 5. L2P: one warp per leaf; phi_far and grad phi_far per sorted atom (f = 1).
//    phi = (1/s) sum L^_lm conj(R_lm(u)), grad = (1/s^2) sum G^_lm conj(R_lm(u)).
// ---------------------------------------------------------------------------
// Gradient coefficients in the device basis (degree P-1) from the local c:
//   Gz_{l,m} = c_{l+1,m} sqrt((l+1+m)(l+1-m))
//   Gx_{l,m} = 1/2 (c_{l+1,m-1} sqrt((l-m+2)(l-m+1)) - c_{l+1,m+1} sqrt((l+m+2)(l+m+1)))
//   Gy_{l,m} = i/2 (c_{l+1,m+1} sqrt((l+m+2)(l+m+1)) + c_{l+1,m-1} sqrt((l-m+2)(l-m+1)))
// (from d/dz R_lm = R_{l-1,m}, d/dx R_lm = (R_{l-1,m+1} - R_{l-1,m-1})/2,
//  d/dy R_lm = -i (R_{l-1,m-1} + R_{l-1,m+1})/2 and the basis scale ratios).
template <typename T>
__device__ __forceinline__ void gradient_row_coeffs(int P, const T *c, T *cx, T *cy, T *cz, int lane = 0,
                                                    int nlanes = 1, int stride = 1) {
  auto get = [&](int l, int m, T &re, T &im) {
    if (l < 0 || m > l || -m > l) { re = T(0); im = T(0); return; }
    int am = m < 0 ? -m : m;
    if (am == 0) { re = c[stride * (l * l)]; im = T(0); }
    else { re = c[stride * (l * l + 2 * am - 1)]; im = c[stride * (l * l + 2 * am)]; }
    if (m < 0) { im = -im; if (am & 1) { re = -re; im = -im; } }
  };
  // entries (l, m), 0 <= m <= l < P, in triangular order t = l(l+1)/2 + m,
  // dealt round-robin to the calling lanes
  const int nt = P * (P + 1) / 2;
  int l = 0, t0 = 0;  // l of entry t and the first entry of row l
  for (int t = lane; t < nt; t += nlanes) {
    while (t >= t0 + l + 1) { t0 += l + 1; ++l; }
    const int m = t - t0;
    T zr, zi, ar, ai, br, bi;
    get(l + 1, m, zr, zi);
    get(l + 1, m - 1, ar, ai);
    get(l + 1, m + 1, br, bi);
    T fz = sqrt(T((l + 1 + m) * (l + 1 - m)));
    T fa = sqrt(T((l - m + 2) * (l - m + 1))), fb = sqrt(T((l + m + 2) * (l + m + 1)));
    zr *= fz; zi *= fz; ar *= fa; ai *= fa; br *= fb; bi *= fb;
    T xr = T(0.5) * (ar - br), xi = T(0.5) * (ai - bi);
    T yr = T(-0.5) * (bi + ai), yi = T(0.5) * (br + ar);
    if (m == 0) { cz[stride * (l * l)] = zr; cx[stride * (l * l)] = xr; cy[stride * (l * l)] = yr; }
    else {
      const int k = stride * (l * l + 2 * m - 1);
      cz[k] = zr; cz[k + stride] = zi; cx[k] = xr; cx[k + stride] = xi; cy[k] = yr; cy[k + stride] = yi;
    }
  }
}

// The leaf's local coefficients and the three gradient rows are kept
// interleaved per coefficient, so one vector load of shared memory serves the
// potential and the gradient of a term; PP > 0 makes the order a compile-time
// constant (the harmonic recursion is then unrolled).
template <typename T>
__device__ __forceinline__ void l2p_stage_leaf(int P, int K, const T *__restrict__ Lv, T *cf, int lane) {
  for (int k = lane; k < K; k += 32) cf[4 * k] = Lv[k];
  __syncwarp();
  gradient_row_coeffs<T>(P, cf, cf + 1, cf + 2, cf + 3, lane, 32, 4);
  __syncwarp();
}

// far-field potential f and gradient g at u = (x - leaf centre) / s from the
// staged rows cc, in the leaf's units (multiply f by 1/s and g by 1/s^2)
template <typename T, int PP>
__device__ __forceinline__ void l2p_point(int P, const typename V4<T>::type *__restrict__ cc, T ux, T uy, T uz, T &f,
                                          T &gx, T &gy, T &gz) {
  using V = typename V4<T>::type;
  const int Q = PP > 0 ? PP : P;
  f = 0; gx = 0; gy = 0; gz = 0;
  // sum over m of X_lm conj(R_lm) = X_l0 R_l0 + 2 sum_{m>0} (Xr Rr + Xi Ri)
  rt_columns<T>(Q, ux, uy, uz, [&](int l, int m, T re, T im) {
    const int k = ridx(l, m);
    const V c0 = cc[k];
    if (m == 0) {
      f += c0.x * re;
      if (l < Q) { gx += c0.y * re; gy += c0.z * re; gz += c0.w * re; }
    } else {
      const V c1 = cc[k + 1];
      f += T(2) * (c0.x * re + c1.x * im);
      if (l < Q) {
        gx += T(2) * (c0.y * re + c1.y * im);
        gy += T(2) * (c0.z * re + c1.z * im);
        gz += T(2) * (c0.w * re + c1.w * im);
      }
    }
  });
}

// One warp per leaf (six blocks of four warps per SM measured fastest, with a
// few registers spilled).
template <typename T, int PP>
__global__ void __launch_bounds__(128, 6) k_l2p(int nleaf, int Pr, int ld, T s, const int *__restrict__ leaf_start,
                      const typename V4<T>::type *__restrict__ part, const T *__restrict__ Lleaf,
                      T *__restrict__ phi, T *__restrict__ grad) {
  using V = typename V4<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = PP > 0 ? PP : Pr;
  const int K = (P + 1) * (P + 1);
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  V *cc = reinterpret_cast<V *>(smem_raw) + (size_t)wib * K;  // {c, cx, cy, cz} per coefficient
  int warp = blockIdx.x * (blockDim.x >> 5) + wib;
  if (warp >= nleaf) return;
  l2p_stage_leaf<T>(P, K, Lleaf + (size_t)warp * ld, reinterpret_cast<T *>(cc), lane);
  int b = leaf_start[warp], e = leaf_start[warp + 1];
  T inv_s = T(1) / s;
  for (int a = b + lane; a < e; a += 32) {
    V pt = part[a];
    T f, gx, gy, gz;
    l2p_point<T, PP>(P, cc, pt.x * inv_s, pt.y * inv_s, pt.z * inv_s, f, gx, gy, gz);
    phi[a] = f * inv_s;
    grad[3 * (size_t)a + 0] = gx * inv_s * inv_s;
    grad[3 * (size_t)a + 1] = gy * inv_s * inv_s;
    grad[3 * (size_t)a + 2] = gz * inv_s * inv_s;
  }
}

// ---------------------------------------------------------------------------
// 6. P2P near field + dipole/background term + outputs.  One block per target
//    leaf; threads = (target, source chunk) pairs; sources of the 27 neighbour
//    leaves (periodic images) staged in shared memory relative to the target
//    leaf centre.  Writes forces (original order), per-block energy partials,
//    and the total potential phi~ back into phi_s (sorted order).
// ---------------------------------------------------------------------------

// energy accumulator: compensated (Kahan-Babuska) in single precision, plain in FP64
template <typename T> struct SiteAccE;
template <> struct SiteAccE<float> {
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float s = h + v, bv = s - h;
    l += (h - (s - bv)) + (v - bv);
    h = s;
  }
  // sum over the warp (butterfly, same order on every run), still compensated
  __device__ __forceinline__ void warp_reduce() {
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffff, h, o), ol = __shfl_xor_sync(0xffffffff, l, o);
      l += ol;
      add(oh);
    }
  }
  __device__ __forceinline__ double value() const { return (double)h + (double)l; }
};
template <> struct SiteAccE<double> {
  double h = 0.0;
  __device__ __forceinline__ void add(double v) { h += v; }
  __device__ __forceinline__ void warp_reduce() {
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffff, h, o);
  }
  __device__ __forceinline__ double value() const { return h; }
};

__device__ __forceinline__ double rinv(double r2) { return 1.0 / sqrt(r2); }
// the hardware reciprocal square root as one instruction: subnormal inputs
// flush to zero (squared distances here are never subnormal), so no
// input-scaling fix-up is emitted around it
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// hardware reciprocal square root refined by one Newton-Raphson step
// y' = y (3 - r2 y^2) / 2, which roughly squares the relative error
__device__ __forceinline__ float rinv(float r2) {
  float y = rsqrt_ftz(r2);
  return y * fmaf(-0.5f * r2, y * y, 1.5f);
}
// near-field pair kernel: the hardware estimate alone (relative error below
// 2^-22, under the single-precision rounding of the accumulated sums)
__device__ __forceinline__ float rinv_fast(float r2) { return rsqrt_ftz(r2); }
__device__ __forceinline__ double rinv_fast(double r2) { return 1.0 / sqrt(r2); }
// staged sources per pass (16 KB in single precision): leaves of ~30 atoms
// give ~800 sources, so one pass is the rule and more blocks fit on an SM
constexpr int P2P_MAXSRC = 1024;
// FP64 1/sqrt(r2): single-precision seed and one FP64 Newton-Raphson step; the
// seed's relative error e (about 2^-23) becomes 1.5 e^2 after the step
__device__ __forceinline__ double rinv_dd(double r2) {
  const double y = (double)rsqrt_ftz((float)r2);
  return y * fma(-0.5 * r2, y * y, 1.5);
}

template <typename T, typename FT, int NT>
__global__ void __launch_bounds__(NT) k_p2p(int nb, T c2, T half_L, T s_leaf, T fc_t, const int *__restrict__ leaf_start,
                                                     const typename V4<T>::type *__restrict__ part,
                                                     const int *__restrict__ perm, const double *__restrict__ mom,
                                                     T *__restrict__ phi_s, const T *__restrict__ grad_s,
                                                     FT *__restrict__ forces, double *__restrict__ energy_part) {
  using V = typename V4<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V *src = reinterpret_cast<V *>(smem_raw);
  __shared__ int nb_start[27], nb_pre[28];
  __shared__ T red[NT][4], red2[NT][4];
  __shared__ T kc[5];
  __shared__ double ered[NT / 32];
  const int leaf = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const T s = s_leaf;  // leaf edge (the host divides once)
  const int ix = (int)d_compact(leaf), iy = (int)d_compact(leaf >> 1), iz = (int)d_compact(leaf >> 2);
  if (tid < 27) {
    int dx = tid % 3 - 1, dy = (tid / 3) % 3 - 1, dz = tid / 9 - 1;
    int n = (int)d_morton(wrapi(ix + dx, nb), wrapi(iy + dy, nb), wrapi(iz + dz, nb));
    nb_start[tid] = leaf_start[n];
    nb_pre[tid + 1] = leaf_start[n + 1] - leaf_start[n];
  }
  if (tid == 32) {
    // dipole / background term of the periodic kernel, (2 pi/3V) sum_j q_j |x_i - x_j|^2
    //   = c2 (Q |a|^2 - 2 a.D + T) with a = x_i - box centre = lc + m (lc: this
    // leaf's centre, m: the stored offset); per leaf, in the working precision
    // from the FP64 box moments (c2 = 2 pi / 3V from the host):
    //   K0 = A |lc|^2 - B.lc + C, K1 = 2 A lc - B, K2 = A,
    //   A = c2 Q, B = 2 c2 D, C = c2 T,
    // so the term is K0 + K1.m + K2 |m|^2 and its gradient K1 + 2 K2 m.  (No
    // FP64 arithmetic per leaf: on GB300 FP64 issues at a small fraction of the
    // FP32 rate, and one thread of every block would hold the others.)
    const T A = c2 * (T)mom[0], C = c2 * (T)mom[4];
    const T Bx = T(2) * c2 * (T)mom[1], By = T(2) * c2 * (T)mom[2], Bz = T(2) * c2 * (T)mom[3];
    const T lcx = ((T)ix + T(0.5)) * s - half_L, lcy = ((T)iy + T(0.5)) * s - half_L,
            lcz = ((T)iz + T(0.5)) * s - half_L;
    kc[0] = A * (lcx * lcx + lcy * lcy + lcz * lcz) - (Bx * lcx + By * lcy + Bz * lcz) + C;
    kc[1] = T(2) * A * lcx - Bx;
    kc[2] = T(2) * A * lcy - By;
    kc[3] = T(2) * A * lcz - Bz;
    kc[4] = A;
  }
  __syncthreads();
  if (tid == 0) {
    nb_pre[0] = 0;
    for (int k = 0; k < 27; ++k) nb_pre[k + 1] += nb_pre[k];
  }
  __syncthreads();
  const int tb = leaf_start[leaf], te = leaf_start[leaf + 1], nt = te - tb;
  const int nsrc_total = nb_pre[27];
  const T fc = fc_t;
  SiteAccE<T> e_acc;
  // threads = (target pair, source chunk): every thread holds two targets, so
  // each staged source serves two pairs; as many chunks as fill the block
  const int npr = (nt + 1) >> 1;
  const int nchunk = NT / max(1, min(npr, NT));
  const int tgroup = NT / nchunk;
  for (int t0 = 0; t0 < npr; t0 += tgroup) {
    const int tp = t0 + tid % tgroup, ck = tid / tgroup;
    const int ta0 = 2 * t0 + (tid % tgroup), ta1 = ta0 + min(tgroup, npr - t0);  // this round's targets
    const bool tv0 = tp < npr && ta0 < nt, tv1 = tp < npr && ta1 < nt;
    const V me0 = tv0 ? part[tb + ta0] : V{0, 0, 0, 0};
    const V me1 = tv1 ? part[tb + ta1] : V{0, 0, 0, 0};
    T f0 = 0, gx0 = 0, gy0 = 0, gz0 = 0, f1 = 0, gx1 = 0, gy1 = 0, gz1 = 0;
    for (int s0 = 0; s0 < nsrc_total; s0 += P2P_MAXSRC) {
      int ns = min(P2P_MAXSRC, nsrc_total - s0);
      __syncthreads();
      // stage the sources, shifted to this leaf's frame: warp w copies the
      // neighbour leaves w, w + 4, ...
      for (int k = warp; k < 27; k += NT / 32) {
        const int b = nb_pre[k] - s0, cnt = nb_pre[k + 1] - nb_pre[k];
        const T ox = (T)(k % 3 - 1) * s, oy = (T)((k / 3) % 3 - 1) * s, oz = (T)(k / 9 - 1) * s;
        for (int i = lane; i < cnt; i += 32) {
          const int d = b + i;
          if (d >= 0 && d < ns) {
            V v = part[nb_start[k] + i];
            v.x += ox; v.y += oy; v.z += oz;
            src[d] = v;
          }
        }
      }
      __syncthreads();
      // self: neighbour k = 13 is the leaf itself, at source index nb_pre[13] + ta
      const int self0 = (nb_pre[13] + ta0) - s0, self1 = (nb_pre[13] + ta1) - s0;
      const int per = (ns + nchunk - 1) / nchunk;
      const int jb = ck * per, je = min(ns, jb + per);
      if (tv0) {
#pragma unroll 4
        for (int j = jb; j < je; ++j) {
          const V v = src[j];
          const T rx0 = me0.x - v.x, ry0 = me0.y - v.y, rz0 = me0.z - v.z;
          const T rx1 = me1.x - v.x, ry1 = me1.y - v.y, rz1 = me1.z - v.z;
          const T r20 = rx0 * rx0 + ry0 * ry0 + rz0 * rz0, r21 = rx1 * rx1 + ry1 * ry1 + rz1 * rz1;
          const T ri0 = (j == self0) ? T(0) : rinv_fast(r20);
          const T ri1 = (j == self1 || !tv1) ? T(0) : rinv_fast(r21);
          const T qr0 = v.w * ri0, qr1 = v.w * ri1;
          f0 += qr0;
          f1 += qr1;
          const T g30 = qr0 * ri0 * ri0, g31 = qr1 * ri1 * ri1;
          gx0 -= g30 * rx0; gy0 -= g30 * ry0; gz0 -= g30 * rz0;
          gx1 -= g31 * rx1; gy1 -= g31 * ry1; gz1 -= g31 * rz1;
        }
      }
    }
    // chunk partial sums of both targets, then one thread per target finishes
    red[tid][0] = f0; red[tid][1] = gx0; red[tid][2] = gy0; red[tid][3] = gz0;
    red2[tid][0] = f1; red2[tid][1] = gx1; red2[tid][2] = gy1; red2[tid][3] = gz1;
    __syncthreads();
    const int nr = min(2 * tgroup, nt - 2 * t0);  // targets of this round
    for (int tt = tid; tt < nr; tt += NT) {
      // target ta = 2 t0 + tt: first of the pair tt (tt < w) or second of the
      // pair tt - w, w = pairs in this round
      const int w = min(tgroup, npr - t0);
      const bool second = tt >= w;
      const int p = second ? tt - w : tt;
      const int ta = 2 * t0 + tt;
      T f = 0, gx = 0, gy = 0, gz = 0;
      for (int c2i = 0; c2i < nchunk; ++c2i) {
        const int o = p + c2i * tgroup;
        const T *r = second ? red2[o] : red[o];
        f += r[0]; gx += r[1]; gy += r[2]; gz += r[3];
      }
      const V me = part[tb + ta];
      const int a = tb + ta;
      // near + far field, then the dipole / background term (in the working
      // precision from the FP64 per-leaf constants)
      T ff = f + phi_s[a];
      T g0 = gx + grad_s[3 * (size_t)a], g1 = gy + grad_s[3 * (size_t)a + 1], g2 = gz + grad_s[3 * (size_t)a + 2];
      const T mx = me.x, my = me.y, mz = me.z;
      ff += kc[0] + kc[1] * mx + kc[2] * my + kc[3] * mz + kc[4] * (mx * mx + my * my + mz * mz);
      g0 += kc[1] + T(2) * kc[4] * mx;
      g1 += kc[2] + T(2) * kc[4] * my;
      g2 += kc[3] + T(2) * kc[4] * mz;
      ff *= fc; g0 *= fc; g1 *= fc; g2 *= fc;
      const T q = me.w;
      phi_s[a] = ff;
      e_acc.add(T(0.5) * q * ff);
      int io = perm[a];
      if (forces) {
        forces[3 * (size_t)io + 0] = (FT)(-q * g0);
        forces[3 * (size_t)io + 1] = (FT)(-q * g1);
        forces[3 * (size_t)io + 2] = (FT)(-q * g2);
      }
    }
    __syncthreads();
  }
  e_acc.warp_reduce();
  if (lane == 0) ered[warp] = e_acc.value();
  __syncthreads();
  if (tid == 0) {
    double v = 0;
    for (int w = 0; w < NT / 32; ++w) v += ered[w];
    energy_part[leaf] = v;
  }
}

// ---------------------------------------------------------------------------
// 6b. Near field by Newton's third law (single precision).  Every unordered
//     pair of atoms in neighbouring leaves is evaluated once.  The block of
//     target leaf A takes the atoms of the 13 neighbours B = A + o of the
//     forward half shell (o > 0 in (z, y, x) lexicographic order; neighbour
//     k = 14 ... 26 of the 3 x 3 x 3 stencil, periodic images included) and,
//     target side only, the ordered pairs inside A.  A's sums end in phi_s /
//     grad_s; the sums of B's atoms go to slot k - 14 of those atoms
//     (slots[k - 14][N], one float4 {phi, grad} per atom), each slot written
//     by exactly one block.  k_l2p_near adds own sums, the 13 slots, the far
//     field and the dipole / background term in a fixed order, so results are
//     bitwise reproducible.
//
//     Work split: the block stages up to kN3Src sources (shifted to A's frame)
//     and up to kN3Tgt targets.  The staged list is cut into chunks of 32
//     sources (the half shell's, then A's own), dealt round-robin to the
//     warps; a warp takes every target block of TB atoms (in registers)
//     against each of its chunks, so the sum of a staged source over all
//     targets stays in one lane (accumulated in target-block order), and the
//     TB x 4 target sums are reduce-scattered over the lanes once per target
//     block and warp, then summed over the warps in warp order.  One barrier
//     per pass: no warp waits for another between target blocks.
// ---------------------------------------------------------------------------
constexpr int kN3Src = 512;  // staged sources per pass
constexpr int kN3Tgt = 64;   // targets per chunk
constexpr int kN3Slots = 13;

template <int NW>
constexpr size_t n3_smem_bytes() {
  // src, ssum [kN3Src] float4; tgt [kN3Tgt] float4; tpart [NW][4 kN3Tgt]
  // floats; tsum [kN3Tgt] float4; sidx, sk [kN3Src] ints
  return sizeof(float4) * (2 * (size_t)kN3Src + 2 * kN3Tgt) + sizeof(float) * 4 * kN3Tgt * NW +
         2 * sizeof(int) * kN3Src;
}

// V (a power of two, 4 <= V <= 32) values per lane summed over the warp; lane
// l returns the total of value l / (32 / V) (pairwise halving: at offset o a
// lane keeps the upper half of its values if bit o of its lane is set and
// sends the other half to lane l ^ o)
template <int V>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[V], int lane) {
#pragma unroll
  for (int h = V / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? v[i] : v[i + h];
      const float keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffff, send, o);
    }
  }
  float x = v[0];
#pragma unroll
  for (int o = 16 / V; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffff, x, o);
  return x;
}

template <int TB, int NT>
__global__ void __launch_bounds__(NT, (TB == 4) ? 5 : 4) k_p2p_n3(int nb, float s_leaf, int64_t N,
                                                                const int *__restrict__ leaf_start,
                                                                const float4 *__restrict__ part,
                                                                float *__restrict__ own_phi,
                                                                float *__restrict__ own_grad,
                                                                float4 *__restrict__ slots) {
  constexpr int NW = NT / 32;
  constexpr int V = 4 * TB;  // per-lane target sums: {phi, gx, gy, gz} x TB
  static_assert(V == 16 || V == 32, "TB must be 4 or 8");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4 *src = reinterpret_cast<float4 *>(smem_raw);
  float4 *ssum = src + kN3Src;         // [kN3Src] a staged source's sum over the chunk's targets
  float4 *tgt = ssum + kN3Src;         // [kN3Tgt] the chunk's targets
  float4 *tsum = tgt + kN3Tgt;         // [kN3Tgt] target sums over the passes
  float *tpart = reinterpret_cast<float *>(tsum + kN3Tgt);  // [NW][4 kN3Tgt] per-warp target sums
  int *sidx = reinterpret_cast<int *>(tpart + 4 * kN3Tgt * NW);  // sorted index of each staged source
  int *sk = sidx + kN3Src;                                       // its slot
  __shared__ int nb_start[14], nb_pre[15];                       // 13 forward neighbours, then A
  const int leaf = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float s = s_leaf;
  const int ix = (int)d_compact(leaf), iy = (int)d_compact(leaf >> 1), iz = (int)d_compact(leaf >> 2);
  if (tid < 14) {
    int n = leaf;
    if (tid < 13) {
      const int k = 14 + tid;
      n = (int)d_morton(wrapi(ix + k % 3 - 1, nb), wrapi(iy + (k / 3) % 3 - 1, nb), wrapi(iz + k / 9 - 1, nb));
    }
    nb_start[tid] = leaf_start[n];
    nb_pre[tid + 1] = leaf_start[n + 1] - leaf_start[n];
  }
  __syncthreads();
  if (tid == 0) {
    nb_pre[0] = 0;
    for (int k = 0; k < 14; ++k) nb_pre[k + 1] += nb_pre[k];
  }
  __syncthreads();
  const int a0 = nb_start[13], nt = nb_pre[14] - nb_pre[13];
  const int n_fwd = nb_pre[13], n_all = nb_pre[14];
  if (nt == 0) {
    // no targets: the forward neighbours' slots from this leaf are zero
    for (int k = warp; k < kN3Slots; k += NW)
      for (int i = lane; i < nb_pre[k + 1] - nb_pre[k]; i += 32)
        slots[(size_t)k * N + nb_start[k] + i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  for (int c0 = 0; c0 < nt; c0 += kN3Tgt) {
    const int nct = min(kN3Tgt, nt - c0);
    const int ntb = (nct + TB - 1) / TB;
    for (int s0 = 0; s0 < n_all; s0 += kN3Src) {
      const int ns = min(kN3Src, n_all - s0);
      const int ns3 = max(0, min(ns, n_fwd - s0));  // staged sources of the half shell
      __syncthreads();  // the previous pass is done with every buffer
      // the chunk's targets, padding far away and without charge; then the
      // sources: staged index d = nb_pre[k] + i - s0, one thread per source
      for (int i = tid; i < ntb * TB; i += NT)
        tgt[i] = i < nct ? part[a0 + c0 + i] : make_float4(1e3f, 1e3f, 1e3f, 0.f);
      for (int d = tid; d < ns; d += NT) {
        const int g = s0 + d;
        int k = 0;
        while (g >= nb_pre[k + 1]) ++k;
        const int kk = k < 13 ? 14 + k : 13;
        float4 v = part[nb_start[k] + g - nb_pre[k]];
        v.x += (float)(kk % 3 - 1) * s;
        v.y += (float)((kk / 3) % 3 - 1) * s;
        v.z += (float)(kk / 9 - 1) * s;
        src[d] = v;
        sidx[d] = nb_start[k] + g - nb_pre[k];
        sk[d] = k;
      }
      __syncthreads();
      const int nc3 = (ns3 + 31) >> 5, nch = nc3 + ((ns - ns3 + 31) >> 5);
      for (int tb = 0; tb < ntb; ++tb) {
        float4 t[TB];
        float acc[V];
#pragma unroll
        for (int u = 0; u < TB; ++u) t[u] = tgt[tb * TB + u];
#pragma unroll
        for (int i = 0; i < V; ++i) acc[i] = 0.f;
        for (int c = warp; c < nch; c += NW) {
          if (c < nc3) {
            // half shell: both sides of every pair
            const int j = 32 * c + lane;
            if (j < ns3) {
              const float4 v = src[j];
              float sf = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
              for (int u = 0; u < TB; ++u) {
                const float dx = t[u].x - v.x, dy = t[u].y - v.y, dz = t[u].z - v.z;
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const float ri = rsqrt_ftz(r2);
                const float ri3 = ri * ri * ri;
                const float b = v.w * ri3, e = t[u].w * ri3;
                acc[4 * u + 0] = fmaf(v.w, ri, acc[4 * u + 0]);
                acc[4 * u + 1] = fmaf(-b, dx, acc[4 * u + 1]);
                acc[4 * u + 2] = fmaf(-b, dy, acc[4 * u + 2]);
                acc[4 * u + 3] = fmaf(-b, dz, acc[4 * u + 3]);
                sf = fmaf(t[u].w, ri, sf);
                sx = fmaf(e, dx, sx);
                sy = fmaf(e, dy, sy);
                sz = fmaf(e, dz, sz);
              }
              // this lane owns source j in every target block: in-place sum
              if (tb == 0) {
                ssum[j] = make_float4(sf, sx, sy, sz);
              } else {
                float4 o = ssum[j];
                o.x += sf; o.y += sx; o.z += sy; o.w += sz;
                ssum[j] = o;
              }
            }
          } else {
            // pairs inside A: every ordered pair but the atom itself, target side
            const int j = ns3 + 32 * (c - nc3) + lane;
            if (j < ns) {
              const float4 v = src[j];
              const int ja = s0 + j - n_fwd;  // index of the source in A
#pragma unroll
              for (int u = 0; u < TB; ++u) {
                const float dx = t[u].x - v.x, dy = t[u].y - v.y, dz = t[u].z - v.z;
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const float ri = (c0 + tb * TB + u == ja) ? 0.f : rsqrt_ftz(r2);
                const float b = v.w * ri * ri * ri;
                acc[4 * u + 0] = fmaf(v.w, ri, acc[4 * u + 0]);
                acc[4 * u + 1] = fmaf(-b, dx, acc[4 * u + 1]);
                acc[4 * u + 2] = fmaf(-b, dy, acc[4 * u + 2]);
                acc[4 * u + 3] = fmaf(-b, dz, acc[4 * u + 3]);
              }
            }
          }
        }
        const float tot = warp_reduce_scatter<V>(acc, lane);
        // lane l holds value l / (32 / V): target tb TB + value / 4, component value % 4
        if ((lane & (32 / V - 1)) == 0) tpart[warp * 4 * kN3Tgt + tb * V + lane / (32 / V)] = tot;
      }
      __syncthreads();
      // the targets' sums over the warps (warp order), after earlier passes
      for (int i = tid; i < 4 * nct; i += NT) {
        float v = tpart[i];
        for (int w = 1; w < NW; ++w) v += tpart[w * 4 * kN3Tgt + i];
        float *o = reinterpret_cast<float *>(tsum) + i;
        *o = (s0 == 0) ? v : *o + v;
      }
      // slots: the first target chunk writes them, later chunks add
      for (int j = tid; j < ns3; j += NT) {
        float4 *p = slots + (size_t)sk[j] * N + sidx[j];
        float4 a = ssum[j];
        if (c0 > 0) {
          const float4 o = *p;
          a.x = o.x + a.x; a.y = o.y + a.y; a.z = o.z + a.z; a.w = o.w + a.w;
        }
        *p = a;
      }
    }
    __syncthreads();
    for (int i = tid; i < nct; i += NT) {
      const int a = a0 + c0 + i;
      const float4 v = tsum[i];
      own_phi[a] = v.x;
      own_grad[3 * (size_t)a + 0] = v.y;
      own_grad[3 * (size_t)a + 1] = v.z;
      own_grad[3 * (size_t)a + 2] = v.w;
    }
  }
}

// Far field (L2P) fused with the end of the near field: per atom, its own
// near sums (phi_s, grad_s from k_p2p_n3) + the 13 slots in order + the far
// field + the dipole / background term, times the Coulomb constant; writes the
// total potential to phi_s, the force (original order) and the leaf's energy
// partial.  One warp per leaf.
template <int PP, typename FT>
__global__ void __launch_bounds__(128, 6) k_l2p_near(int nleaf, int Pr, int ld, float s, int64_t N, float c2,
                                                     float half_L, float fc, const int *__restrict__ leaf_start,
                                                     const float4 *__restrict__ part, const float *__restrict__ Lleaf,
                                                     const int *__restrict__ perm, const double *__restrict__ mom,
                                                     const float4 *__restrict__ slots, float *__restrict__ phi_s,
                                                     const float *__restrict__ grad_s, FT *__restrict__ forces,
                                                     double *__restrict__ energy_part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = PP > 0 ? PP : Pr;
  const int K = (P + 1) * (P + 1);
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4 *cc = reinterpret_cast<float4 *>(smem_raw) + (size_t)wib * K;
  const int leaf = blockIdx.x * (blockDim.x >> 5) + wib;
  if (leaf >= nleaf) return;
  l2p_stage_leaf<float>(P, K, Lleaf + (size_t)leaf * ld, reinterpret_cast<float *>(cc), lane);
  // dipole / background term as in k_p2p: K0 + K1.m + K2 |m|^2 about the leaf centre
  const int ix = (int)d_compact(leaf), iy = (int)d_compact(leaf >> 1), iz = (int)d_compact(leaf >> 2);
  const float A = c2 * (float)mom[0], C = c2 * (float)mom[4];
  const float Bx = 2.f * c2 * (float)mom[1], By = 2.f * c2 * (float)mom[2], Bz = 2.f * c2 * (float)mom[3];
  const float lcx = ((float)ix + 0.5f) * s - half_L, lcy = ((float)iy + 0.5f) * s - half_L,
              lcz = ((float)iz + 0.5f) * s - half_L;
  const float k0 = A * (lcx * lcx + lcy * lcy + lcz * lcz) - (Bx * lcx + By * lcy + Bz * lcz) + C;
  const float k1 = 2.f * A * lcx - Bx, k2 = 2.f * A * lcy - By, k3 = 2.f * A * lcz - Bz, k4 = A;
  const int b = leaf_start[leaf], e = leaf_start[leaf + 1];
  const float inv_s = 1.f / s;
  SiteAccE<float> e_acc;
  for (int a = b + lane; a < e; a += 32) {
    const float4 me = part[a];
    float ff = phi_s[a], g0 = grad_s[3 * (size_t)a], g1 = grad_s[3 * (size_t)a + 1], g2 = grad_s[3 * (size_t)a + 2];
#pragma unroll
    for (int k = 0; k < kN3Slots; ++k) {
      const float4 v = slots[(size_t)k * N + a];
      ff += v.x; g0 += v.y; g1 += v.z; g2 += v.w;
    }
    float f, gx, gy, gz;
    l2p_point<float, PP>(P, cc, me.x * inv_s, me.y * inv_s, me.z * inv_s, f, gx, gy, gz);
    ff += f * inv_s;
    g0 += gx * inv_s * inv_s;
    g1 += gy * inv_s * inv_s;
    g2 += gz * inv_s * inv_s;
    const float mx = me.x, my = me.y, mz = me.z;
    ff += k0 + k1 * mx + k2 * my + k3 * mz + k4 * (mx * mx + my * my + mz * mz);
    g0 += k1 + 2.f * k4 * mx;
    g1 += k2 + 2.f * k4 * my;
    g2 += k3 + 2.f * k4 * mz;
    ff *= fc; g0 *= fc; g1 *= fc; g2 *= fc;
    const float q = me.w;
    phi_s[a] = ff;
    e_acc.add(0.5f * q * ff);
    if (forces) {
      const int io = perm[a];
      forces[3 * (size_t)io + 0] = (FT)(-q * g0);
      forces[3 * (size_t)io + 1] = (FT)(-q * g1);
      forces[3 * (size_t)io + 2] = (FT)(-q * g2);
    }
  }
  e_acc.warp_reduce();
  if (lane == 0) energy_part[leaf] = e_acc.value();
}

// ---------------------------------------------------------------------------
// 7. Per-site HI correction (FP64).  One warp per site.  For every pair (i, j)
//    of the site: A(r) = sum_{|n|_inf<=1} 1/|r+nL| + H(r) + (2 pi/3V)|r|^2,
//    r = minimum image of x_i - x_j, H from the lattice coefficients (degree
//    adapted to |r|); the self term A_ii (the same limit without 1/|r|) is a
//    constant of the box.  This is the paper's C_P2P + C_L + C_D for a two-form
//    site (first shell direct, lattice part, dipole/background part).  Then
//      k_s = f sum D_i D_j A_ij,  g_s = sum D_i phi~_i,
//      dE/dlam = g + (1/2 - lam) k,  E += 1/2 lam(1-lam) k,
//      F_i -= lam(1-lam) f sum_{j != i} D_i D_j grad A(r_ij),
//    and psi_i = f sum_{j in s} A_ij D_j (kept for the charge gradients).
//    Sites of up to kSiteSymMax atoms evaluate each unordered pair once and
//    gather the forces per atom in a fixed order; larger sites evaluate the
//    ordered pairs of one atom per lane.
// ---------------------------------------------------------------------------
constexpr int kMaxSiteAtoms = 64;

// A(r) and grad A(r) for r != 0 (nm), FP64
__device__ __forceinline__ void site_pair_kernel(const double r[3], double L, double c2, int Pmax,
                                                 const double *__restrict__ eta, const double *__restrict__ eta_x,
                                                 const double *__restrict__ eta_y, const double *__restrict__ eta_z,
                                                 double &A, double g[3]) {
  double a = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
  for (int nx = -1; nx <= 1; ++nx)
    for (int ny = -1; ny <= 1; ++ny)
      for (int nz = -1; nz <= 1; ++nz) {
        const double d0 = r[0] + nx * L, d1 = r[1] + ny * L, d2 = r[2] + nz * L;
        const double ri = rsqrt_dp(d0 * d0 + d1 * d1 + d2 * d2);
        a += ri;
        const double g3 = ri * ri * ri;
        g0 -= g3 * d0; g1 -= g3 * d1; g2 -= g3 * d2;
      }
  const double iL = 1.0 / L;
  const double u[3] = {r[0] * iL, r[1] * iL, r[2] * iL};
  const float un = (float)sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  // (|u| / 1.9)^P < 1e-17: the series of H converges for |u| < 1.9
  const int P = min(Pmax, max(4, (int)ceilf(-39.2f / logf(un / 1.9f)) + 1));
  double H = 0, hx = 0, hy = 0, hz = 0;
  // H lives on even degrees; its gradient coefficients on odd degrees (< P)
  r_columns(P, u[0], u[1], u[2], [&](int l, int m, double re, double im) {
    const int k = ridx(l, m);
    const double w = (m == 0) ? 1.0 : 2.0;
    if (!(l & 1)) {
      H += (m == 0) ? eta[k] * re : w * (eta[k] * re + eta[k + 1] * im);
    } else if (l < P) {
      hx += (m == 0) ? eta_x[k] * re : w * (eta_x[k] * re + eta_x[k + 1] * im);
      hy += (m == 0) ? eta_y[k] * re : w * (eta_y[k] * re + eta_y[k + 1] * im);
      hz += (m == 0) ? eta_z[k] * re : w * (eta_z[k] * re + eta_z[k + 1] * im);
    }
  });
  A = a + H * iL + c2 * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  g[0] = g0 + hx * iL * iL + 2.0 * c2 * r[0];
  g[1] = g1 + hy * iL * iL + 2.0 * c2 * r[1];
  g[2] = g2 + hz * iL * iL + 2.0 * c2 * r[2];
}

template <typename XT>
__device__ __forceinline__ void site_pair_r(const XT *__restrict__ x, int i, int j, double L, double r[3]) {
  for (int a = 0; a < 3; ++a) {
    double v = (double)x[3 * (size_t)i + a] - (double)x[3 * (size_t)j + a];
    v -= L * rint(v / L);
    r[a] = v;
  }
}

// The FP64 pair terms (grad A, A) of every unordered pair of every site of
// up to kSiteSymMax atoms, one pair per thread over all sites (the pair list
// {site, i, j, slot} is built when the site map is set): on GB300 the FP64 pipe
// is charged per warp instruction whatever the number of active lanes, so full
// warps (32 pairs) matter more than keeping a site in one block.  They depend
// only on the positions, so they are computed at the start of an evaluation
// on the side stream, where the FP64 pipe is otherwise idle, and k_site reads
// them back; pairs[site][p] with p the pair index of k_site.
template <typename XT>
__global__ void __launch_bounds__(64) k_site_pairs(int npairs, const int4 *__restrict__ plist, double L, int Pmax,
                                                   const int *__restrict__ site_ptr,
                                                   const int *__restrict__ site_atoms, const XT *__restrict__ x,
                                                   const double *__restrict__ eta, const double *__restrict__ eta_x,
                                                   const double *__restrict__ eta_y, const double *__restrict__ eta_z,
                                                   double *__restrict__ pairs) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npairs) return;
  const int4 e = plist[t];  // site, i, j (atom indices within the site), pair index
  const double V = L * L * L, c2 = 2.0 * kPi / (3.0 * V);
  const int b = site_ptr[e.x];
  double r[3], A, g[3];
  site_pair_r(x, site_atoms[b + e.y], site_atoms[b + e.z], L, r);
  site_pair_kernel(r, L, c2, Pmax, eta, eta_x, eta_y, eta_z, A, g);
  double *o = pairs + ((size_t)e.x * kSiteSymPairs + e.w) * 4;
  o[0] = g[0]; o[1] = g[1]; o[2] = g[2]; o[3] = A;
}

// pairs: the terms of k_site_pairs, or null to evaluate them here
template <typename T, typename XT, typename FT>
__global__ void k_site(int S, double L, double fcoul, int Pmax, double aii, const int *__restrict__ site_ptr,
                       const int *__restrict__ site_atoms, const XT *__restrict__ x, const double *__restrict__ dq,
                       const double *__restrict__ lam, const double *__restrict__ phi_site,
                       const double *__restrict__ eta, const double *__restrict__ eta_x,
                       const double *__restrict__ eta_y, const double *__restrict__ eta_z,
                       double *__restrict__ dEdl, double *__restrict__ site_energy, FT *__restrict__ forces,
                       double *__restrict__ psi_site, const double *__restrict__ pairs) {
  __shared__ double fsh[4][kMaxSiteAtoms][3];
  __shared__ double gbuf[4][kSiteSymPairs][4];  // grad A at r = x_lo - x_hi, then A
  const int wib = threadIdx.x >> 5;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= S) return;
  const int b = site_ptr[warp], e = site_ptr[warp + 1], n = e - b;
  const double V = L * L * L, c2 = 2.0 * kPi / (3.0 * V);
  const double lw = lam[warp] * (1.0 - lam[warp]);
  double ksum = 0.0, gsum = 0.0;
  // self terms and the charge-interpolation derivative
  for (int ia = lane; ia < n; ia += 32) {
    const double Di = dq[site_atoms[b + ia]];
    ksum += Di * Di * aii;
    gsum += Di * phi_site[b + ia];
  }
  if (n <= kSiteSymMax) {
    const int np = n * (n - 1) / 2;
    for (int p = lane; p < np; p += 32) {
      int ia = 0, rem = p;
      while (rem >= n - 1 - ia) { rem -= n - 1 - ia; ++ia; }
      const int ja = ia + 1 + rem;
      const int i = site_atoms[b + ia], j = site_atoms[b + ja];
      double A, g[3];
      if (pairs) {
        const double *o = pairs + ((size_t)warp * kSiteSymPairs + p) * 4;
        g[0] = o[0]; g[1] = o[1]; g[2] = o[2]; A = o[3];
      } else {
        double r[3];
        site_pair_r(x, i, j, L, r);
        site_pair_kernel(r, L, c2, Pmax, eta, eta_x, eta_y, eta_z, A, g);
      }
      ksum += 2.0 * dq[i] * dq[j] * A;
      gbuf[wib][p][0] = g[0]; gbuf[wib][p][1] = g[1]; gbuf[wib][p][2] = g[2]; gbuf[wib][p][3] = A;
    }
    __syncwarp();
    for (int ia = lane; ia < n; ia += 32) {
      const double Di = dq[site_atoms[b + ia]];
      double f0 = 0.0, f1 = 0.0, f2 = 0.0, ps = aii * Di;
      for (int ja = 0; ja < n; ++ja) {
        if (ja == ia) continue;
        const int lo = min(ia, ja), hi = max(ia, ja);
        const int p = lo * (2 * n - lo - 1) / 2 + (hi - lo - 1);
        const double Dj = dq[site_atoms[b + ja]];
        // gbuf holds grad A at r = x_lo - x_hi; at x_hi - x_lo it changes sign
        const double w = (ia == lo ? 1.0 : -1.0) * lw * fcoul * Di * Dj;
        f0 -= w * gbuf[wib][p][0]; f1 -= w * gbuf[wib][p][1]; f2 -= w * gbuf[wib][p][2];
        ps += gbuf[wib][p][3] * Dj;
      }
      fsh[wib][ia][0] = f0; fsh[wib][ia][1] = f1; fsh[wib][ia][2] = f2;
      if (psi_site) psi_site[b + ia] = fcoul * ps;
    }
  } else {
    for (int ia = lane; ia < n; ia += 32) {
      const int i = site_atoms[b + ia];
      const double Di = dq[i];
      double f0 = 0.0, f1 = 0.0, f2 = 0.0, ps = aii * Di;
      for (int ja = 0; ja < n; ++ja) {
        if (ja == ia) continue;
        const int j = site_atoms[b + ja];
        double r[3], A, g[3];
        site_pair_r(x, i, j, L, r);
        site_pair_kernel(r, L, c2, Pmax, eta, eta_x, eta_y, eta_z, A, g);
        ksum += Di * dq[j] * A;
        ps += A * dq[j];
        const double w = lw * fcoul * Di * dq[j];
        f0 -= w * g[0]; f1 -= w * g[1]; f2 -= w * g[2];
      }
      fsh[wib][ia][0] = f0; fsh[wib][ia][1] = f1; fsh[wib][ia][2] = f2;
      if (psi_site) psi_site[b + ia] = fcoul * ps;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    ksum += __shfl_xor_sync(0xffffffff, ksum, o);
    gsum += __shfl_xor_sync(0xffffffff, gsum, o);
  }
  __syncwarp();
  const double k = fcoul * ksum;  // phi_site already carries f
  if (lane == 0) {
    const double l0 = lam[warp];
    if (dEdl) dEdl[warp] = gsum + (0.5 - l0) * k;
    site_energy[warp] = 0.5 * lw * k;
  }
  if (forces)
    for (int k3 = lane; k3 < n * 3; k3 += 32) {
      int ia = k3 / 3, a = k3 % 3;
      int i = site_atoms[b + ia];
      forces[3 * (size_t)i + a] = (FT)((double)forces[3 * (size_t)i + a] + fsh[wib][ia][a]);
    }
}

// ---------------------------------------------------------------------------
// 7b. Sites with 2^m forms (general formulation, Eq. "iter_ham_lambda";
//     Appendix, Eqs. "lambda_list", "one_site_lambda").  Form rho of a site has
//     weight lambda~_rho = prod_l (bit l of rho ? lambda_l : 1 - lambda_l); the
//     scaled charge of a site atom is q~ = sum_rho lambda~_rho q^rho, and the
//     per-site correction that turns E(q~) into the interpolated Hamiltonian is
//       C = f/2 [sum_rho lambda~_rho G_rr - sum_rr' lambda~_r lambda~_r' G_rr'],
//       G_rr' = q^r^T A q^r' over the site's atoms (A_ii = the self term);
//     dE/dlambda_l = sum_rho d lambda~_rho/d lambda_l (q^rho . phi~ + f (G_rr/2 - (G lambda~)_r)),
//     F_i -= f sum_{j != i} W_ij grad A(r_ij),  W_ij = sum_r lambda~_r q_i^r q_j^r - q~_i q~_j.
// ---------------------------------------------------------------------------
constexpr int kMfMaxForms = 16;
constexpr int kMfMaxAtoms = 32;

__device__ __forceinline__ void mf_weights(const double *__restrict__ lam, int m, double *w) {
  for (int r = 0; r < (1 << m); ++r) {
    double v = 1.0;
    for (int l = 0; l < m; ++l) v *= ((r >> l) & 1) ? lam[l] : 1.0 - lam[l];
    w[r] = v;
  }
}

// q~ of the site atoms (overwrites what k_bin wrote for them)
template <typename T>
__global__ void k_mf_charges(int nsa, const int *__restrict__ site_atoms, const int *__restrict__ site_of,
                             const int *__restrict__ lam_off, const double *__restrict__ lam,
                             const double *__restrict__ qf, double *__restrict__ qt, typename V4<T>::type *vtmp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nsa) return;
  const int i = site_atoms[k], s = site_of[i], m = lam_off[s + 1] - lam_off[s];
  double w[kMfMaxForms];
  mf_weights(lam + lam_off[s], m, w);
  double q = 0.0;
  for (int r = 0; r < (1 << m); ++r) q += w[r] * qf[(size_t)k * kMfMaxForms + r];
  qt[i] = q;
  vtmp[i].w = (T)q;
}

template <typename XT, typename FT>
__global__ void __launch_bounds__(32) k_site_mf(int S, double L, double fcoul, int Pmax, double aii,
                                                const int *__restrict__ site_ptr, const int *__restrict__ site_atoms,
                                                const XT *__restrict__ x, const int *__restrict__ lam_off,
                                                const double *__restrict__ lam, const double *__restrict__ qf,
                                                const double *__restrict__ phi_site, const double *__restrict__ eta,
                                                const double *__restrict__ eta_x, const double *__restrict__ eta_y,
                                                const double *__restrict__ eta_z, double *__restrict__ dEdl,
                                                double *__restrict__ site_energy, FT *__restrict__ forces,
                                                double *__restrict__ psi_form) {
  __shared__ double A[kMfMaxAtoms][kMfMaxAtoms + 1];
  __shared__ double gw[kMfMaxAtoms * (kMfMaxAtoms - 1) / 2][3];  // W_ij grad A(r_ij), r = x_i - x_j, i < j
  __shared__ double qs[kMfMaxForms][kMfMaxAtoms], Tm[kMfMaxForms][kMfMaxAtoms], G[kMfMaxForms][kMfMaxForms];
  __shared__ double w[kMfMaxForms], qtl[kMfMaxAtoms];
  const int s = blockIdx.x, lane = threadIdx.x;
  if (s >= S) return;
  const int b = site_ptr[s], n = site_ptr[s + 1] - b, m = lam_off[s + 1] - lam_off[s], F = 1 << m;
  const double c2 = 2.0 * kPi / (3.0 * L * L * L);
  if (lane == 0) mf_weights(lam + lam_off[s], m, w);
  for (int e = lane; e < F * n; e += 32) {
    const int r = e / n, a = e % n;
    qs[r][a] = qf[(size_t)(b + a) * kMfMaxForms + r];
  }
  __syncwarp();
  for (int a = lane; a < n; a += 32) {
    double v = 0.0;
    for (int r = 0; r < F; ++r) v += w[r] * qs[r][a];
    qtl[a] = v;
    A[a][a] = aii;
  }
  __syncwarp();
  // pair kernel: A_ij and W_ij grad A for every unordered pair
  const int np = n * (n - 1) / 2;
  for (int p = lane; p < np; p += 32) {
    int ia = 0, rem = p;
    while (rem >= n - 1 - ia) { rem -= n - 1 - ia; ++ia; }
    const int ja = ia + 1 + rem;
    double r[3], Aij, g[3];
    site_pair_r(x, site_atoms[b + ia], site_atoms[b + ja], L, r);
    site_pair_kernel(r, L, c2, Pmax, eta, eta_x, eta_y, eta_z, Aij, g);
    A[ia][ja] = Aij;
    A[ja][ia] = Aij;
    double W = -qtl[ia] * qtl[ja];
    for (int rr = 0; rr < F; ++rr) W += w[rr] * qs[rr][ia] * qs[rr][ja];
    gw[p][0] = W * g[0]; gw[p][1] = W * g[1]; gw[p][2] = W * g[2];
  }
  __syncwarp();
  // T = A q^r per form, then G = Q T^T
  for (int e = lane; e < F * n; e += 32) {
    const int r = e / n, a = e % n;
    double v = 0.0;
    for (int j = 0; j < n; ++j) v += A[a][j] * qs[r][j];
    Tm[r][a] = v;
    // psi^r_a = f (A q^r)_a over the site (self term included), kept for the
    // charge gradients of the backward pass
    if (psi_form) psi_form[(size_t)(b + a) * kMfMaxForms + r] = fcoul * v;
  }
  __syncwarp();
  for (int e = lane; e < F * F; e += 32) {
    const int r = e / F, r2 = e % F;
    double v = 0.0;
    for (int a = 0; a < n; ++a) v += qs[r][a] * Tm[r2][a];
    G[r][r2] = v;
  }
  __syncwarp();
  if (lane == 0) {
    double c = 0.0;
    for (int r = 0; r < F; ++r) {
      double gwr = 0.0;
      for (int r2 = 0; r2 < F; ++r2) gwr += G[r][r2] * w[r2];
      c += w[r] * (G[r][r] - gwr);
    }
    site_energy[s] = 0.5 * fcoul * c;
  }
  // dE/dlambda_l, one lambda per lane
  if (dEdl)
    for (int l = lane; l < m; l += 32) {
      const double *lm = lam + lam_off[s];
      double tot = 0.0;
      for (int r = 0; r < F; ++r) {
        double dw = ((r >> l) & 1) ? 1.0 : -1.0;
        for (int k = 0; k < m; ++k)
          if (k != l) dw *= ((r >> k) & 1) ? lm[k] : 1.0 - lm[k];
        double qphi = 0.0, gwr = 0.0;
        for (int a = 0; a < n; ++a) qphi += qs[r][a] * phi_site[b + a];
        for (int r2 = 0; r2 < F; ++r2) gwr += G[r][r2] * w[r2];
        tot += dw * (qphi + fcoul * (0.5 * G[r][r] - gwr));
      }
      dEdl[lam_off[s] + l] = tot;
    }
  // forces: gather the pair terms of each atom in a fixed order
  if (forces)
    for (int ia = lane; ia < n; ia += 32) {
      double f0 = 0.0, f1 = 0.0, f2 = 0.0;
      for (int ja = 0; ja < n; ++ja) {
        if (ja == ia) continue;
        const int lo = min(ia, ja), hi = max(ia, ja);
        const int p = lo * (2 * n - lo - 1) / 2 + (hi - lo - 1);
        const double sg = ia == lo ? 1.0 : -1.0;  // grad A is odd in r
        f0 -= sg * gw[p][0]; f1 -= sg * gw[p][1]; f2 -= sg * gw[p][2];
      }
      const int i = site_atoms[b + ia];
      forces[3 * (size_t)i + 0] = (FT)((double)forces[3 * (size_t)i + 0] + fcoul * f0);
      forces[3 * (size_t)i + 1] = (FT)((double)forces[3 * (size_t)i + 1] + fcoul * f1);
      forces[3 * (size_t)i + 2] = (FT)((double)forces[3 * (size_t)i + 2] + fcoul * f2);
    }
}

// ---------------------------------------------------------------------------
// 8. FP64 charge, dipole and second moment (about the box centre) of every box
//    above the leaves by exact translation of the children's:
//    Q = sum Q_c, D = sum (D_c + Q_c o_c), T = sum (T_c + 2 o_c.D_c + Q_c |o_c|^2),
//    o_c = child centre - parent centre.  The root's values are the moments
//    of the whole box about its centre used by the dipole / background term.
// ---------------------------------------------------------------------------
__global__ void k_qd_up(int nparent, double s_child, const double *__restrict__ child, double *__restrict__ parent,
                        float *__restrict__ parent_f) {
  int P = blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= nparent) return;
  double v[5] = {0, 0, 0, 0, 0};
  for (int c = 0; c < 8; ++c) {
    const double *ch = child + (size_t)(8 * P + c) * kQD;
    const double off[3] = {((c & 1) ? 0.5 : -0.5) * s_child, ((c & 2) ? 0.5 : -0.5) * s_child,
                           ((c & 4) ? 0.5 : -0.5) * s_child};
    v[0] += ch[0];
    v[4] += ch[4] + 2.0 * (off[0] * ch[1] + off[1] * ch[2] + off[2] * ch[3]) +
            ch[0] * (off[0] * off[0] + off[1] * off[1] + off[2] * off[2]);
    for (int k = 0; k < 3; ++k) v[1 + k] += ch[1 + k] + ch[0] * off[k];
  }
  for (int k = 0; k < 5; ++k) parent[(size_t)P * kQD + k] = v[k];
  qd_split(v, parent_f + (size_t)P * kQDF);
}

// ---------------------------------------------------------------------------
// 9. Potential at the site atoms for dE/dlambda, evaluated more accurately than
//    the bulk path: FP64 near field from the original positions, then M2P from
//    every interaction-list box of every ancestor level and from the root images
//    2 <= |n|_inf <= 3 (multipole truncation only, no local expansion), the
//    far-image lattice part H_3 through its own root local expansion, and the
//    dipole/background term.  The l <= 1 multipole terms use the FP64 box charge
//    and dipole; l >= 2 use the working-precision multipoles.  One warp per site
//    atom; all sums are FP64.
//    M2P in the device basis: phi = (1/s) sum_lm M~_lm It_lm(u), u = (x - z)/s,
//    It_lm = I_lm / sqrt((l+m)!(l-m)!), recursion
//      It_00 = 1/r, It_mm = -sqrt((2m-1)/(2m)) (x+iy)/r^2 It_{m-1,m-1},
//      It_lm = (a_lm z It_{l-1,m} - b_lm It_{l-2,m}) / r^2  (a, b as for Rt).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T m2p_high(int P, const T *__restrict__ M, T ux, T uy, T uz) {
  // sum over l >= 2 of M~_lm It_lm(u): M_l0 I_l0 + 2 sum_{m>0} (Mr Ir - Mi Ii)
  T acc = T(0);
  it_columns<T>(P, ux, uy, uz, [&](int l, int m, T re, T im) {
    if (l < 2) return;
    const int k = ridx(l, m);
    acc += (m == 0) ? M[k] * re : T(2) * (M[k] * re - M[k + 1] * im);
  });
  return acc;
}

// Site-atom potential by a separation-controlled traversal of the periodic
// octree, shared by all atoms of a site.  The sources are the 343 root images
// |n|_inf <= 3 (beyond them the H_3 lattice expansion takes over).  With R the
// radius of the site's atoms about their centroid c, a box of edge s at
// distance D from c is used through its multipole (M2P at every atom) only if
// its circumradius (sqrt(3)/2) s < theta (D - R) (theta = 0.4 by default), so every multipole term
// converges at least like theta^(p+1) at every atom; otherwise it is opened,
// and unseparated leaves are summed directly.
//
// Precision.  The sites change charge, so the HI derivative needs the absolute
// potential at the site to about 1e-8 relative, which single precision per term
// does not reach over thousands of terms.  FP64 is slow on this part, so it is
// kept to dense per-site work:
//  * charge + dipole of a separated box: the double-float value at c (one per
//    box and site, added by the row's thread of atom pair 0) plus, per atom,
//    the change from c to the atom in working precision by a cancellation-free
//    difference formula, whose error is smaller by |x - c| / D;
//  * orders l >= 2: working precision (their rounding is far below the bar);
//  * direct leaves: double-float pair sums from error-free transforms (relative
//    error near 2^-44 per pair);
//  * per-thread sums in double-float, reduced in FP64 in a fixed order.
// The batches of separated boxes and leaves are dealt round-robin to G blocks
// per site; each block writes its own partial sum, so results are bitwise
// reproducible.  A compact site's lists come from k_site_lists; otherwise each
// block classifies the levels itself (the same lists in every block).
//
// Pipeline.  A block's batches form one stream over all levels; the multipole
// rows and charge/dipole rows of the next batch are copied (bulk copies on an
// mbarrier) into the second of two buffers while the current batch is
// evaluated, and, in the in-kernel traversal, a level is classified when the
// stream first reaches it (its list goes to the one of two list buffers that
// the level two above had used).  Without the overlap, each batch waited a
// full memory round trip before any arithmetic.
constexpr int kSiteThreads = 128;
constexpr int kSiteBatchMax = 64;
// dynamic shared memory of one block (lists, if any, + two batch buffers):
// with the static arrays three blocks fit on an SM
constexpr size_t kSiteSmemBudget = 64 * 1024;

__device__ __forceinline__ int pack_entry(int box, int img) { return (box << 9) | img; }

// block-wide exclusive prefix of `cnt` (per thread) in thread order; returns the
// offset of this thread and writes the total to *total.  One barrier per call:
// the warp totals alternate between the two halves of wsum (flip `parity`
// every call), so a call never overwrites totals the previous one still reads.
__device__ __forceinline__ int block_scan(int cnt, int *wsum, int parity, int *total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int *ws = wsum + 32 * parity;
  int x = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffff, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  int off = 0, tot = 0;
  for (int k = 0; k < nw; ++k) {
    if (k < w) off += ws[k];
    tot += ws[k];
  }
  *total = tot;
  return off + x - cnt;
}

// Knuth's two-sum: a + b = s + e exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bv = s - a;
  e = (a - (s - bv)) + (b - bv);
}

// double-float values h + l (|l| <= ulp(h) / 2 after normalisation), from
// the error-free transforms: Dekker's product by one FMA, Knuth's sum
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_norm(float h, float l) {
  const float s = h + l;
  return DF{s, l - (s - h)};
}
__device__ __forceinline__ DF df_from(float a) { return DF{a, 0.f}; }
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.h, -a.l}; }
__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return df_norm(s, e + (a.l + b.l));
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.h * b.h;
  return df_norm(p, fmaf(a.h, b.h, -p) + fmaf(a.h, b.l, a.l * b.h));
}
__device__ __forceinline__ DF df_sq(DF a) {
  const float p = a.h * a.h;
  return df_norm(p, fmaf(a.h, a.h, -p) + 2.f * a.h * a.l);
}
// 1 / sqrt(a) for a > 0: the hardware estimate y and one Newton-Raphson step
// whose residual 1 - a y^2 is formed in double-float; the step's relative
// error is about 1.5 e^2 for the estimate's e (2^-22): near 2^-44
__device__ __forceinline__ DF df_rsqrt(DF a) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.h));
  const float yy = y * y;
  const DF t = df_mul(a, DF{yy, fmaf(y, y, -yy)});
  const float r = (1.f - t.h) - t.l;  // 1 - t.h is exact (t.h within 2^-20 of 1)
  return df_norm(y, 0.5f * y * r);
}

// running sum in double-float (single precision) or plain FP64
template <typename T> struct SiteAcc;
template <> struct SiteAcc<float> {
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ void add(float v) {
    float s, e;
    two_sum(h, v, s, e);
    h = s;
    l += e;
  }
  __device__ __forceinline__ void add2(float vh, float vl) {
    float s, e;
    two_sum(h, vh, s, e);
    h = s;
    l += e + vl;
  }
  __device__ __forceinline__ double value() const { return (double)h + (double)l; }
};
template <> struct SiteAcc<double> {
  double h = 0.0;
  __device__ __forceinline__ void add(double v) { h += v; }
  __device__ __forceinline__ void add2(double vh, double vl) { h += vh + vl; }
  __device__ __forceinline__ double value() const { return h; }
};

// target m = h + l relative to a leaf centre (double-float; plain FP64 in h)
template <typename T> struct SiteTarget { T hx, hy, hz, lx, ly, lz; };

// m = x - g sl for a stored coordinate x and an integer leaf offset g, with
// sl = slh + sll; g slh is split exactly by an FMA
__device__ __forceinline__ void split_offset(float x, int g, float slh, float sll, float &mh, float &ml) {
  const float gf = (float)g, oh = gf * slh, oe = fmaf(gf, slh, -oh);
  two_sum(x, -oh, mh, ml);
  ml = (ml - oe) - gf * sll;
}

__device__ __forceinline__ SiteTarget<float> site_target(float x, float y, float z, int gx, int gy, int gz, float slh,
                                                         float sll) {
  SiteTarget<float> t;
  split_offset(x, gx, slh, sll, t.hx, t.lx);
  split_offset(y, gy, slh, sll, t.hy, t.ly);
  split_offset(z, gz, slh, sll, t.hz, t.lz);
  return t;
}
__device__ __forceinline__ SiteTarget<double> site_target(double x, double y, double z, int gx, int gy, int gz,
                                                          double sl) {
  return SiteTarget<double>{x - gx * sl, y - gy * sl, z - gz * sl, 0.0, 0.0, 0.0};
}

// q / |m - y| for a source y (stored coordinates relative to the leaf centre).
// Single precision: the difference and its square are kept exactly as hi + lo
// pairs; 1/sqrt comes from the hardware seed y0 and one Newton correction
// y0 (1 + res/2), whose residual res = 1 - r^2 y0^2 is formed from exact
// products; the result is vh + vl.
__device__ __forceinline__ void pair_pot(const SiteTarget<float> &m, float sx, float sy, float sz, float q,
                                         float &vh, float &vl) {
  float hx, ex, hy, ey, hz, ez;
  two_sum(m.hx, -sx, hx, ex);
  two_sum(m.hy, -sy, hy, ey);
  two_sum(m.hz, -sz, hz, ez);
  ex += m.lx; ey += m.ly; ez += m.lz;
  const float px = hx * hx, py = hy * hy, pz = hz * hz;
  const float qx = fmaf(hx, hx, -px), qy = fmaf(hy, hy, -py), qz = fmaf(hz, hz, -pz);
  float s1, t1, s2, t2;
  two_sum(px, py, s1, t1);
  two_sum(s1, pz, s2, t2);
  const float r2l = (t1 + t2) + (qx + qy + qz) + 2.0f * (hx * ex + hy * ey + hz * ez);
  const float y0 = rsqrt_ftz(s2);
  const float t = y0 * y0, te = fmaf(y0, y0, -t);
  const float u = s2 * t, ue = fmaf(s2, t, -u);
  const float res = ((1.0f - u) - ue) - fmaf(s2, te, r2l * t);
  vh = q * y0;
  vl = fmaf(q, y0, -vh) + q * (0.5f * y0 * res);
}
__device__ __forceinline__ void pair_pot(const SiteTarget<double> &m, double sx, double sy, double sz, double q,
                                         double &vh, double &vl) {
  const double dx = m.hx - sx, dy = m.hy - sy, dz = m.hz - sz;
  vh = q / sqrt(dx * dx + dy * dy + dz * dz);
  vl = 0.0;
}

__device__ __forceinline__ float site_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double site_div(double a, double b) { return a / b; }

// l >= 2 part of the M2P, sum_lm M~_lm It_lm(u) over 2 <= l <= PP, at two points
// sharing one multipole row; with the order a compile-time constant the
// recursion coefficients become immediate operands and each row load serves
// both points.
template <typename T, int PP>
__device__ __forceinline__ void m2p_high2(const T *__restrict__ M, T x0, T y0, T z0, T x1, T y1, T z1, T &v0,
                                          T &v1) {
  const T i0 = rinv(x0 * x0 + y0 * y0 + z0 * z0), i1 = rinv(x1 * x1 + y1 * y1 + z1 * z1);
  const T q0 = i0 * i0, q1 = i1 * i1, zq0 = z0 * q0, zq1 = z1 * q1;
  T dr0 = i0, di0 = T(0), dr1 = i1, di1 = T(0);
  // m = 0 terms and m > 0 terms in separate sums, the factor 2 of the latter
  // applied once at the end (exact): each m > 0 term is then two FMAs per point
  T az0 = T(0), az1 = T(0), ap0 = T(0), ap1 = T(0);
#pragma unroll
  for (int m = 0; m <= PP; ++m) {
    if (m > 0) {
      const T f = -tab_diag<T>(m);
      const T f0 = f * q0, f1 = f * q1;
      const T tr0 = f0 * (x0 * dr0 - y0 * di0), ti0 = f0 * (x0 * di0 + y0 * dr0);
      const T tr1 = f1 * (x1 * dr1 - y1 * di1), ti1 = f1 * (x1 * di1 + y1 * dr1);
      dr0 = tr0; di0 = ti0; dr1 = tr1; di1 = ti1;
    }
    T pr0 = T(0), pi0 = T(0), cr0 = dr0, ci0 = di0;
    T pr1 = T(0), pi1 = T(0), cr1 = dr1, ci1 = di1;
    if (m >= 2) {
      const int k = ridx(m, m);
      const T mr = M[k], mi = M[k + 1];
      ap0 = fma(mr, cr0, ap0); ap0 = fma(-mi, ci0, ap0);
      ap1 = fma(mr, cr1, ap1); ap1 = fma(-mi, ci1, ap1);
    }
#pragma unroll
    for (int l = m + 1; l <= PP; ++l) {
      const int k = l * (l + 1) / 2 + m;
      const T a = tab_a<T>(k), b = tab_b<T>(k);
      const T a0 = a * zq0, b0 = b * q0, a1 = a * zq1, b1 = b * q1;
      const T nr0 = a0 * cr0 - b0 * pr0, ni0 = a0 * ci0 - b0 * pi0;
      const T nr1 = a1 * cr1 - b1 * pr1, ni1 = a1 * ci1 - b1 * pi1;
      pr0 = cr0; pi0 = ci0; cr0 = nr0; ci0 = ni0;
      pr1 = cr1; pi1 = ci1; cr1 = nr1; ci1 = ni1;
      if (l >= 2) {
        const int kk = ridx(l, m);
        if (m == 0) {
          const T mr = M[kk];
          az0 = fma(mr, cr0, az0);
          az1 = fma(mr, cr1, az1);
        } else {
          const T mr = M[kk], mi = M[kk + 1];
          ap0 = fma(mr, cr0, ap0); ap0 = fma(-mi, ci0, ap0);
          ap1 = fma(mr, cr1, ap1); ap1 = fma(-mi, ci1, ap1);
        }
      }
    }
  }
  v0 = az0 + T(2) * ap0;
  v1 = az1 + T(2) * ap1;
}

// The atoms of a site (block-wide): sorted index, leaf, stored particle and
// FP64 position, the latter as the minimum images around the first atom (a
// site may straddle the box faces; the periodic decomposition holds at any
// position, and the leaf index used by the direct sums moves with the image).
template <typename V>
__device__ __forceinline__ void site_load_atoms(int n, const int *__restrict__ atoms, int d, double L,
                                                const int *__restrict__ inv_perm, const int *__restrict__ leaf_of,
                                                const V *__restrict__ part, double (*pa)[3], int (*aI)[3], V *me,
                                                int *sa_s) {
  const int nb = 1 << d;
  const double sl = L / nb;
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    const int i = atoms[a], sa = inv_perm[i];
    const int lo = leaf_of[i];  // the leaf binning put atom i in
    const V v = part[sa];
    if (me) me[a] = v;
    if (sa_s) sa_s[a] = sa;
    aI[a][0] = (int)d_compact(lo); aI[a][1] = (int)d_compact(lo >> 1); aI[a][2] = (int)d_compact(lo >> 2);
    pa[a][0] = (aI[a][0] + 0.5) * sl + (double)v.x;
    pa[a][1] = (aI[a][1] + 0.5) * sl + (double)v.y;
    pa[a][2] = (aI[a][2] + 0.5) * sl + (double)v.z;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    if (a == 0) continue;
    for (int k = 0; k < 3; ++k) {
      const double dk = rint((pa[a][k] - pa[0][k]) / L);
      pa[a][k] -= dk * L;
      aI[a][k] -= (int)dk * nb;
    }
  }
  __syncthreads();
}

// centroid c and radius R of the site's atoms (thread 0; the caller syncs)
__device__ __forceinline__ void site_centre(int n, const double (*pa)[3], double *cen) {
  double c[3] = {0, 0, 0};
  for (int a = 0; a < n; ++a)
    for (int k = 0; k < 3; ++k) c[k] += pa[a][k];
  for (int k = 0; k < 3; ++k) c[k] /= n;
  double R = 0.0;
  for (int a = 0; a < n; ++a) {
    const double dx = pa[a][0] - c[0], dy = pa[a][1] - c[1], dz = pa[a][2] - c[2];
    R = fmax(R, sqrt(dx * dx + dy * dy + dz * dz));
  }
  cen[0] = c[0]; cen[1] = c[1]; cen[2] = c[2]; cen[3] = R;
}

// One level l of the separation-controlled traversal (block-wide): the
// frontier fa[0, n0) becomes the list `sep` of separated boxes and direct
// leaves (bit 31 set) and the children of the opened boxes, the next frontier
// (back in fa; n0 becomes its size, 0 below the leaves).  A box of circumradius
// a at distance D from the centre c is separated if a < theta (D - R).  Returns
// the list length.  Capacity overflows are recorded in the status word and
// the traversal goes on with the entries that fit (all accesses stay in bounds).
__device__ int site_classify_level(int l, int d, int *fa, int *fb, int *sep, int &n0, int *wsum, int &scan_par,
                                   float cfx, float cfy, float cfz, float Rf, float Lf, float theta, int fcap,
                                   int *status) {
  const int tid = threadIdx.x;
  const float sf = ldexpf(Lf, -l), a_l = 0.86602540378443865f * sf, th = theta;
  int nsep = 0, n1 = 0;
  for (int t0 = 0; t0 < n0; t0 += blockDim.x) {
    const int t = t0 + tid;
    int kind = -1;  // 0 separated, 1 direct leaf, 2 open
    int e = 0;
    if (t < n0) {
      e = fa[t];
      const int box = e >> 9, img = e & 511;
      const int nx = img / 49 - 3, ny = (img / 7) % 7 - 3, nz = img % 7 - 3;
      const float dx = cfx - (((float)d_compact(box) + 0.5f) * sf + (float)nx * Lf),
                  dy = cfy - (((float)d_compact(box >> 1) + 0.5f) * sf + (float)ny * Lf),
                  dz = cfz - (((float)d_compact(box >> 2) + 0.5f) * sf + (float)nz * Lf);
      const float D = sqrtf(dx * dx + dy * dy + dz * dz);
      if (a_l < th * (D - Rf) * 0.9999f) kind = 0;
      else if (l == d) kind = 1;
      else kind = 2;
    }
    // one scan for both lists: separated / direct entries in the low 16
    // bits, the 8 children of an opened box in the high 16 (a chunk of at
    // most 1024 threads adds at most 8192 children)
    int tot;
    const int off = block_scan((kind == 0 || kind == 1) ? 1 : (kind == 2 ? (8 << 16) : 0), wsum, scan_par, &tot);
    scan_par ^= 1;
    const int osep = off & 0xffff, oopen = off >> 16;
    if ((kind == 0 || kind == 1) && nsep + osep < fcap) sep[nsep + osep] = (kind == 1) ? (e | (1 << 31)) : e;
    nsep += tot & 0xffff;
    if (kind == 2) {
      const int box = e >> 9, img = e & 511;
      for (int c = 0; c < 8; ++c)
        if (n1 + oopen + c < fcap) fb[n1 + oopen + c] = pack_entry(8 * box + c, img);
    }
    n1 += tot >> 16;
  }
  if (nsep > fcap || n1 > fcap) {
    if (tid == 0) *(volatile int *)(status + kStatusSiteOverflow) = 1;
    nsep = min(nsep, fcap);
    n1 = min(n1, fcap);
  }
  __syncthreads();
  for (int t = tid; t < n1; t += blockDim.x) fa[t] = fb[t];
  n0 = (l < d) ? n1 : 0;
  __syncthreads();
  return nsep;
}

// The traversal lists of every compact site (radius at most two leaf edges),
// computed once per evaluation from the geometry alone: the site's centre and
// radius and the box centres, so they are built on the side stream right after
// the sort, while the main stream runs P2M and M2M.  One block per site.
// lists[(site (d + 1) + l) fcap + i]: level l's separated boxes and direct
// leaves; counts[site (d + 2) + l]: their numbers (counts[site (d + 2)] = -1
// marks a spread site, which k_site_phi traverses atom by atom itself);
// cen_out[4 site ...]: the centre and radius.
template <typename T>
__global__ void __launch_bounds__(kSiteThreads) k_site_lists(
    int S, const int *__restrict__ site_ptr, const int *__restrict__ site_atoms, int d, double L,
    const int *__restrict__ leaf_of, const int *__restrict__ inv_perm, const typename V4<T>::type *__restrict__ part,
    float theta, int fcap, int *__restrict__ lists, int *__restrict__ counts, double *__restrict__ cen_out,
    int *__restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int *fa = reinterpret_cast<int *>(smem_raw), *fb = fa + fcap;
  __shared__ double pa[kMaxSiteAtoms][3], cen[4];
  __shared__ int aI[kMaxSiteAtoms][3], wsum[64];
  const int site = blockIdx.x, tid = threadIdx.x;
  if (site >= S) return;
  const int b0 = site_ptr[site], n = site_ptr[site + 1] - b0;
  if (n <= 0 || n > kMaxSiteAtoms) return;  // rejected when the site map is set
  site_load_atoms(n, site_atoms + b0, d, L, inv_perm, leaf_of, part, pa, aI,
                  (typename V4<T>::type *)nullptr, (int *)nullptr);
  if (tid == 0) site_centre(n, pa, cen);
  __syncthreads();
  int *cnt = counts + (size_t)site * (d + 2);
  if (tid < 4) cen_out[4 * (size_t)site + tid] = cen[tid];
  const double sl = L / (1 << d);
  if (cen[3] > 2.0 * sl) {  // spread site
    if (tid == 0) cnt[0] = -1;
    return;
  }
  for (int t = tid; t < 343 && t < fcap; t += blockDim.x) fa[t] = pack_entry(0, t);  // root images
  if (fcap < 343 && tid == 0) *(volatile int *)(status + kStatusSiteOverflow) = 1;
  __syncthreads();
  int n0 = min(343, fcap), scan_par = 0;
  const float cfx = (float)cen[0], cfy = (float)cen[1], cfz = (float)cen[2], Lf = (float)L, Rf = (float)cen[3];
  for (int l = 0; l <= d; ++l) {
    int ns = 0;
    if (n0 > 0)
      ns = site_classify_level(l, d, fa, fb, lists + ((size_t)site * (d + 1) + l) * fcap, n0, wsum, scan_par, cfx,
                               cfy, cfz, Rf, Lf, theta, fcap, status);
    if (tid == 0) cnt[l] = ns;
  }
}

// kCompact: only the compact sites, whose lists k_site_lists built (no list
// storage in shared memory, so the batches hold more rows); otherwise only the
// other sites (spread sites, or all of them when no lists were built), with
// the in-kernel traversal.  Each site is evaluated by exactly one of the two.
template <typename T, int PP, bool kCompact>
__global__ void __launch_bounds__(kSiteThreads, 3) k_site_phi(
    int S, int G, const int *__restrict__ site_ptr, const int *__restrict__ site_atoms, int d, int P, int ld,
    int lds, int nbmax, double L, const int64_t *__restrict__ level_off, const int *__restrict__ leaf_start,
    const int *__restrict__ leaf_of, const int *__restrict__ inv_perm, const typename V4<T>::type *__restrict__ part,
    const T *__restrict__ M,
    const double *__restrict__ qd, const float *__restrict__ qdf, const double *__restrict__ mom,
    const double *__restrict__ Lh3, double *__restrict__ phi_part, int *__restrict__ status, float theta, int fcap,
    uint64_t wait_ns, const int *__restrict__ pre_lists, const int *__restrict__ pre_counts,
    const double *__restrict__ pre_cen, const int *__restrict__ site_order) {
  using V = typename V4<T>::type;
  // charge/dipole rows as staged: (hi, lo) float pairs in single precision,
  // FP64 otherwise; 32 bytes either way
  constexpr bool kDF = std::is_same<T, float>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lcap = kCompact ? 0 : fcap;                 // in-kernel traversal lists
  int *fa = reinterpret_cast<int *>(smem_raw);          // frontier (current)
  int *fb = fa + lcap;                                  // frontier (next)
  int *sep0 = fb + lcap;                                // separated boxes / direct leaves, even levels
  int *sep1 = sep0 + lcap;                              // the same, odd levels
  T *Ms = reinterpret_cast<T *>(sep1 + lcap);           // [2][nbmax][lds] staged multipole rows
  double *qds = reinterpret_cast<double *>(Ms + (size_t)2 * nbmax * lds);  // [2][nbmax][32 B] Q, Dx, Dy, Dz
  // levels 0 and 1 (the root and its 8 children, which every site's first
  // batches refer to over and over through their images) stay resident: rows
  // [0] root, [1 + box] level 1
  const int nres = (d >= 1) ? 9 : 1;
  T *Mres = reinterpret_cast<T *>(qds + (size_t)2 * nbmax * 4);  // [nres][lds]
  double *qres = reinterpret_cast<double *>(Mres + (size_t)nres * lds);  // [nres][32 B]
  __shared__ double pa[kMaxSiteAtoms][3], cen[4], base_s[kSiteThreads], res_s[kSiteThreads][2];
  static_assert(kSiteThreads == 128, "the charge/dipole sums at c are reduced over 128 threads");
  __shared__ T pu[kMaxSiteAtoms][3], puu[kMaxSiteAtoms];
  __shared__ V me[kMaxSiteAtoms];
  __shared__ int sa_s[kMaxSiteAtoms], aI[kMaxSiteAtoms][3], ent_s[2][kSiteBatchMax], wsum[64];
  __shared__ int64_t lvo[kMaxDepth + 2];  // level offsets (rows)
  __shared__ uint64_t sbar[2];            // copies of batch buffer 0 / 1 complete
  __shared__ int s_abort;
  // blocks take the sites largest first (site_order), so the longest blocks
  // start early and the last wave is short; results do not depend on it
  if ((int)(blockIdx.x / G) >= S) return;
  const int site = site_order ? site_order[blockIdx.x / G] : (int)(blockIdx.x / G);
  const int g = blockIdx.x % G, tid = threadIdx.x;
  const int b0 = site_ptr[site], n = site_ptr[site + 1] - b0;
  if (n <= 0 || n > kMaxSiteAtoms) return;  // rejected when the site map is set
  // a compact site's lists may have been built by k_site_lists (pre)
  const int *pcnt = pre_counts ? pre_counts + (size_t)site * (d + 2) : nullptr;
  const bool pre = pcnt && pcnt[0] >= 0;
  if (pre != kCompact) return;  // the other instantiation takes this site
  const int nb = 1 << d;
  const double sl = L / nb;
  if (tid <= d + 1) lvo[tid] = level_off[tid];
  if (tid == 0) {
    mbar_init(&sbar[0], 1);
    mbar_init(&sbar[1], 1);
    s_abort = 0;
    fence_mbar_init();
  }
  site_load_atoms(n, site_atoms + b0, d, L, inv_perm, leaf_of, part, pa, aI, me, sa_s);
  {
    constexpr int EPV = 16 / sizeof(T);
    const int per_row = ld / EPV;
    for (int q = tid; q < nres * per_row; q += blockDim.x) {
      const int r = q / per_row, c = q - r * per_row;
      const int64_t row = (r == 0) ? level_off[0] : level_off[1] + (r - 1);
      if (P >= 2) cpa16(Mres + (size_t)r * lds + c * EPV, M + (size_t)row * ld + c * EPV);
    }
    for (int q = tid; q < 2 * nres; q += blockDim.x) {
      const int r = q >> 1;
      const int64_t row = (r == 0) ? level_off[0] : level_off[1] + (r - 1);
      if (kDF) cpa16(qres + (size_t)r * 4 + (q & 1) * 2, qdf + (size_t)row * kQDF + (q & 1) * 4);
      else cpa16(qres + (size_t)r * 4 + (q & 1) * 2, qd + (size_t)row * kQD + (q & 1) * 2);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  }
  // A compact site (radius at most two leaf edges, the usual case: the atoms
  // of one residue) shares one traversal between its atoms; a spread site (its
  // atoms scattered over the box) would have to open nearly every box near
  // any of them, so each of its atoms then takes its own traversal (a group
  // of one atom about itself).  All blocks of a site take the same decision.
  if (tid == 0) {
    if (pre) {
      for (int k = 0; k < 4; ++k) cen[k] = pre_cen[4 * (size_t)site + k];
    } else {
      site_centre(n, pa, cen);
    }
  }
  __syncthreads();
  const bool spread = !pre && cen[3] > 2.0 * sl;
  const int ngroups = spread ? n : 1;
  // phase parity of the next completion of sbar[0] / sbar[1] (the barriers
  // run on over the groups)
  uint32_t ph0 = 0, ph1 = 0;
  bool timed_out = false;  // a wait ran out: the remaining groups are skipped
  for (int grp = 0; grp < ngroups; ++grp) {
  const int ga = spread ? grp : 0, gn = spread ? 1 : n;   // atoms ga .. ga + gn - 1 of the site
  __syncthreads();
  if (spread && tid == 0) {
    cen[0] = pa[ga][0]; cen[1] = pa[ga][1]; cen[2] = pa[ga][2]; cen[3] = 0.0;
  }
  __syncthreads();
  for (int a = ga + tid; a < ga + gn; a += blockDim.x) {
    const double ux = pa[a][0] - cen[0], uy = pa[a][1] - cen[1], uz = pa[a][2] - cen[2];
    pu[a][0] = (T)ux; pu[a][1] = (T)uy; pu[a][2] = (T)uz;
    puu[a] = (T)(ux * ux + uy * uy + uz * uz);
  }
  if (!pre) {
    for (int t = tid; t < 343 && t < fcap; t += blockDim.x) fa[t] = pack_entry(0, t);  // root images
    if (fcap < 343 && tid == 0) *(volatile int *)(status + kStatusSiteOverflow) = 1;  // capacity below the root images
  }
  __syncthreads();
  // thread -> (atom pair, slot), fixed for the whole traversal; a slot takes
  // the rows slot, slot + nslot, ... of every batch
  const int npair = (gn + 1) >> 1, nslot = blockDim.x / npair;
  const int my_p = (tid < nslot * npair) ? tid % npair : -1, my_s = tid / npair;
  const int a0 = ga + (my_p < 0 ? 0 : my_p), a1 = ga + ((my_p >= 0 && my_p + npair < gn) ? my_p + npair : (my_p < 0 ? 0 : my_p));
  const int nbatch = (nslot <= nbmax) ? nslot * (nbmax / nslot) : nbmax;
  const int lane = tid & 31, warp = tid >> 5;
  SiteAcc<T> acc0, acc1;
  double base = 0.0;          // charge + dipole values at c of the rows this thread takes (FP64)
  DF base_df = df_from(0.f);  // the same in double-float
  // L and c as (hi, lo) float pairs for the double-float terms
  const DF Lsp = df_norm((float)L, (float)(L - (double)(float)L));
  const T iLt = (T)(1.0 / L);
  const float slh = (float)sl, sll = (float)(sl - (double)slh);  // leaf edge, double-float
  const DF csp[3] = {df_norm((float)cen[0], (float)(cen[0] - (double)(float)cen[0])),
                     df_norm((float)cen[1], (float)(cen[1] - (double)(float)cen[1])),
                     df_norm((float)cen[2], (float)(cen[2] - (double)(float)cen[2]))};
  int n0 = min(343, fcap), bc = 0, scan_par = 0;
  int ns0 = 0, ns1 = 0;  // entries in the lists of the last even / odd level classified
  int lcl = -1;          // deepest level classified
  const T Rf = (T)cen[3];
  // the separation test runs in single precision (its 1e-4 safety margin is far
  // above the rounding of box centres at |x| < 4L); every block of a site
  // evaluates it identically
  const float cfx = (float)cen[0], cfy = (float)cen[1], cfz = (float)cen[2], Lf = (float)L;
  // level l: the frontier fa[0, n0) becomes the list of separated boxes and
  // direct leaves (sep0 / sep1 by the parity of l) and the children of the
  // opened boxes, the next frontier
  auto classify = [&](int l) {
    int ns = 0;
    if (pre) {
      ns = pcnt[l];
    } else {
      ns = site_classify_level(l, d, fa, fb, (l & 1) ? sep1 : sep0, n0, wsum, scan_par, cfx, cfy, cfz, (float)Rf, Lf,
                               theta, fcap, status);
    }
    if (l & 1) ns1 = ns; else ns0 = ns;
    lcl = l;
  };
  // the next batch of this block at or after (level gl, entry gb): level,
  // first entry and size; classifies a level on first use; false once the
  // traversal is exhausted (uniform over the block)
  int gl = 0, gb = 0;
  auto next_batch = [&](int &bl, int &bb, int &bn) -> bool {
    for (;;) {
      if (gl > d) return false;
      if (gl > lcl) {
        if (!pre && n0 <= 0) {
          gl = d + 1;
          return false;
        }
        classify(gl);
      }
      const int nl = (gl & 1) ? ns1 : ns0;
      if (gb < nl) {
        const bool mine = (bc % G) == g;
        ++bc;
        bb = gb;
        gb += nbatch;
        if (mine) {
          bl = gl;
          bn = min(nbatch, nl - bb);
          return true;
        }
      } else {
        ++gl;
        gb = 0;
      }
    }
  };
  // copies of one batch into buffer `buf` by warp 0: its entries, and (one
  // bulk copy per row, completing on sbar[buf]) the charge/dipole rows and
  // multipole rows of its separated boxes; levels 0 and 1 are resident
  const uint32_t qrow_bytes = 32, mrow_bytes = (P >= 2) ? (uint32_t)(ld * sizeof(T)) : 0u;
  auto stage = [&](int buf, int bl, int bb, int bn) {
    if (warp != 0) return;
    const int *sp = (pre ? pre_lists + ((size_t)site * (d + 1) + bl) * fcap : ((bl & 1) ? sep1 : sep0)) + bb;
    const bool res = bl <= 1;
    const int r0 = lane, r1 = lane + 32;
    const int e0 = (r0 < bn) ? sp[r0] : -1, e1 = (r1 < bn) ? sp[r1] : -1;
    if (r0 < bn) ent_s[buf][r0] = e0;
    if (r1 < bn) ent_s[buf][r1] = e1;
    const bool c0 = !res && e0 >= 0, c1 = !res && e1 >= 0;
    const int ncp = __popc(__ballot_sync(0xffffffffu, c0)) + __popc(__ballot_sync(0xffffffffu, c1));
    if (lane == 0) mbar_arrive_expect_tx(&sbar[buf], (uint32_t)ncp * (qrow_bytes + mrow_bytes));
    __syncwarp();
    // the buffer was last read by generic loads (ordered by the block barrier)
    fence_proxy_async();
    const int64_t lo = lvo[bl];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool c = h ? c1 : c0;
      const int r = h ? r1 : r0, e = h ? e1 : e0;
      if (!c) continue;
      const int64_t row = lo + (e >> 9);
      double *qdst = qds + ((size_t)buf * nbmax + r) * 4;
      if (kDF) bulk_g2s(qdst, qdf + (size_t)row * kQDF, qrow_bytes, &sbar[buf]);
      else bulk_g2s(qdst, qd + (size_t)row * kQD, qrow_bytes, &sbar[buf]);
      if (P >= 2) bulk_g2s(Ms + ((size_t)buf * nbmax + r) * lds, M + (size_t)row * ld, mrow_bytes, &sbar[buf]);
    }
  };
  int cl = 0, cb = 0, cn = 0, cur = 0;
  bool have = next_batch(cl, cb, cn);
  if (have) stage(0, cl, cb, cn);
  while (have) {
    int nl2 = 0, nb2 = 0, nn2 = 0;
    const bool nxt = next_batch(nl2, nb2, nn2);
    if (nxt) stage(cur ^ 1, nl2, nb2, nn2);
    // the current batch's copies (bounded wait; on expiry the block records
    // the failure, drains the copies in flight and leaves the traversal)
    const uint32_t pc = cur ? ph1 : ph0;
    const bool ok = mbar_wait(&sbar[cur], pc, &s_abort, wait_ns);
    if (cur) ph1 ^= 1u; else ph0 ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) *(volatile int *)(status + kStatusSiteTimeout) = 1;
      mbar_wait_for(&sbar[cur], pc, wait_ns);
      if (nxt) mbar_wait_for(&sbar[cur ^ 1], cur ? ph0 : ph1, wait_ns);
      __syncthreads();
      timed_out = true;
      break;
    }
    const T is = iLt * (T)(1 << cl);  // 1 / s, exact scaling of 1 / L
    const int *ent = ent_s[cur];
    const T *Mb = Ms + (size_t)cur * nbmax * lds;
    // Per row: the box centre relative to c, w, and its charge/dipole values,
    // computed by every thread that takes the row (no setup phase and no
    // barrier before the rows); the FP64 / double-float value at c,
    // Q/B - (p.w)/B^3, is added by the row's thread of pair 0 only.
    auto row_values = [&](int r, int e, bool add_base, T &wx, T &wy, T &wz, T &Q, T &px, T &py, T &pz, T &B,
                          T &Bi, T &pw) {
      const int box = e >> 9, img = e & 511;
      const int nx = img / 49 - 3, ny = (img / 7) % 7 - 3, nz = img % 7 - 3;
      const double *q = (cl <= 1) ? qres + (size_t)((cl == 0) ? 0 : 1 + box) * 4
                                  : qds + ((size_t)cur * nbmax + r) * 4;
      if constexpr (kDF) {
        // double-float: w = m h - c with the odd integer m = 2 i + 1 + 2^(l+1) n
        // (exact in single precision) and h = L / 2^(l+1) = hh + hl; then
        // B^2, 1/B, p.w and Q/B - (p.w)/B^3 to about 2^-44 relative
        const float hh = ldexpf(Lsp.h, -(cl + 1)), hl = ldexpf(Lsp.l, -(cl + 1));
        const int ms = 2 << cl;
        const int mi[3] = {2 * (int)d_compact(box) + 1 + ms * nx, 2 * (int)d_compact(box >> 1) + 1 + ms * ny,
                           2 * (int)d_compact(box >> 2) + 1 + ms * nz};
        DF w[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float mf = (float)mi[k], ph = mf * hh, pe = fmaf(mf, hh, -ph);
          float sh, se;
          two_sum(ph, -csp[k].h, sh, se);
          w[k] = df_norm(sh, se + (fmaf(mf, hl, pe) - csp[k].l));
        }
        const float *qf = reinterpret_cast<const float *>(q);
        const DF Qd{qf[0], qf[1]}, pxd{qf[2], qf[3]}, pyd{qf[4], qf[5]}, pzd{qf[6], qf[7]};
        const DF B2 = df_add(df_add(df_sq(w[0]), df_sq(w[1])), df_sq(w[2]));
        const DF Bid = df_rsqrt(B2);
        const DF pwd = df_add(df_add(df_mul(pxd, w[0]), df_mul(pyd, w[1])), df_mul(pzd, w[2]));
        if (add_base) {
          const DF Bi3 = df_mul(df_sq(Bid), Bid);
          base_df = df_add(base_df, df_add(df_mul(Qd, Bid), df_neg(df_mul(pwd, Bi3))));  // at c the box centre is at -w
        }
        wx = w[0].h; wy = w[1].h; wz = w[2].h;
        px = pxd.h; py = pyd.h; pz = pzd.h;
        Q = Qd.h;
        B = B2.h * Bid.h;
        Bi = Bid.h;
        pw = pwd.h;
      } else {
        const double s = ldexp(L, -cl);
        const double dwx = (((int)d_compact(box) + 0.5) * s + nx * L) - cen[0];
        const double dwy = (((int)d_compact(box >> 1) + 0.5) * s + ny * L) - cen[1];
        const double dwz = (((int)d_compact(box >> 2) + 0.5) * s + nz * L) - cen[2];
        const double B2 = dwx * dwx + dwy * dwy + dwz * dwz, dBi = rinv_dd(B2);
        const double dQ = q[0], dpx = q[1], dpy = q[2], dpz = q[3];
        const double dpw = dpx * dwx + dpy * dwy + dpz * dwz;
        if (add_base) base += dQ * dBi - dpw * (dBi * dBi * dBi);  // at c the box centre is at -w
        wx = (T)dwx; wy = (T)dwy; wz = (T)dwz;
        px = (T)dpx; py = (T)dpy; pz = (T)dpz;
        Q = (T)dQ;
        B = (T)(B2 * dBi);
        Bi = (T)dBi;
        pw = (T)dpw;
      }
    };
    if (my_p >= 0) {
      for (int r = my_s; r < cn; r += nslot) {
        const int e = ent[r];
        if (e >= 0) {
          // charge + dipole: change from the value at c,
          //   Q (1/A - 1/B) + p.u / A^3 - (p.w) (1/A^3 - 1/B^3),
          // A = |u - w|, B = |w|, A^2 - B^2 = u.u - 2 u.w, A - B = (A^2 - B^2) / (A + B)
          T wx, wy, wz, Q, px, py, pz, B, Bi, pw;
          row_values(r, e, my_p == 0, wx, wy, wz, Q, px, py, pz, B, Bi, pw);
          const T Bi3 = Bi * Bi * Bi;
          T ux[2], uy[2], uz[2], dev[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int a = h ? a1 : a0;
            ux[h] = pu[a][0] - wx; uy[h] = pu[a][1] - wy; uz[h] = pu[a][2] - wz;
            const T A2 = ux[h] * ux[h] + uy[h] * uy[h] + uz[h] * uz[h];
            const T Ai = rinv(A2), A = A2 * Ai, Ai3 = Ai * Ai * Ai;
            const T d2 = puu[a] - T(2) * (pu[a][0] * wx + pu[a][1] * wy + pu[a][2] * wz);
            const T f1 = site_div(d2, A + B);
            const T pu_ = px * pu[a][0] + py * pu[a][1] + pz * pu[a][2];
            dev[h] = -Q * f1 * Ai * Bi + pu_ * Ai3 + pw * f1 * (A2 + A * B + B * B) * Ai3 * Bi3;
          }
          if (P >= 2) {
          const T *Mr = (cl <= 1) ? Mres + (size_t)((cl == 0) ? 0 : 1 + (e >> 9)) * lds : Mb + (size_t)r * lds;
            T v0, v1;
            if constexpr (PP > 0) {
              m2p_high2<T, PP>(Mr, ux[0] * is, uy[0] * is, uz[0] * is, ux[1] * is, uy[1] * is, uz[1] * is, v0, v1);
            } else {
              v0 = m2p_high<T>(P, Mr, ux[0] * is, uy[0] * is, uz[0] * is);
              v1 = m2p_high<T>(P, Mr, ux[1] * is, uy[1] * is, uz[1] * is);
            }
            dev[0] += v0 * is;
            dev[1] += v1 * is;
          }
          acc0.add(dev[0]);
          acc1.add(dev[1]);
        } else {
          // unseparated leaf: direct sum over its atoms
          const int box = (e & 0x7fffffff) >> 9, img = e & 511;
          const int nx = img / 49 - 3, ny = (img / 7) % 7 - 3, nz = img % 7 - 3;
          const int bx = (int)d_compact(box) + nx * nb, by = (int)d_compact(box >> 1) + ny * nb,
                    bz = (int)d_compact(box >> 2) + nz * nb;
          const int gx0 = bx - aI[a0][0], gy0 = by - aI[a0][1], gz0 = bz - aI[a0][2];
          const int gx1 = bx - aI[a1][0], gy1 = by - aI[a1][1], gz1 = bz - aI[a1][2];
          const int self0 = (gx0 == 0 && gy0 == 0 && gz0 == 0) ? sa_s[a0] : -1;
          const int self1 = (gx1 == 0 && gy1 == 0 && gz1 == 0) ? sa_s[a1] : -1;
          const V m0 = me[a0], m1 = me[a1];
          SiteTarget<T> t0, t1;
          if constexpr (kDF) {
            t0 = site_target(m0.x, m0.y, m0.z, gx0, gy0, gz0, slh, sll);
            t1 = site_target(m1.x, m1.y, m1.z, gx1, gy1, gz1, slh, sll);
          } else {
            t0 = site_target(m0.x, m0.y, m0.z, gx0, gy0, gz0, sl);
            t1 = site_target(m1.x, m1.y, m1.z, gx1, gy1, gz1, sl);
          }
          const int q2e = leaf_start[box + 1];
#pragma unroll 4
          for (int q2 = leaf_start[box]; q2 < q2e; ++q2) {
            const V src = part[q2];
            T vh, vl;
            if (q2 != self0) {
              pair_pot(t0, src.x, src.y, src.z, src.w, vh, vl);
              acc0.add2(vh, vl);
            }
            if (q2 != self1) {
              pair_pot(t1, src.x, src.y, src.z, src.w, vh, vl);
              acc1.add2(vh, vl);
            }
          }
        }
      }
    }
    // the next iteration copies into this batch's buffer
    __syncthreads();
    cur ^= 1;
    cl = nl2; cb = nb2; cn = nn2;
    have = nxt;
  }
  // the far-image lattice coefficients in working precision, over the batch
  // buffers (free now: the loop ended with a barrier and no copy in flight)
  T *Lh3s = Ms;
  if (g == 0)
    for (int k = tid; k < (P + 1) * (P + 1); k += blockDim.x) Lh3s[k] = (T)Lh3[k];
  // fixed-order reductions: the staged FP64 values, then per atom over its slots
  base_s[tid] = base + ((double)base_df.h + (double)base_df.l);
  res_s[tid][0] = acc0.value();
  res_s[tid][1] = acc1.value();
  __syncthreads();
  if (tid < 32) {
    double v = (base_s[tid] + base_s[tid + 32]) + (base_s[tid + 64] + base_s[tid + 96]);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
    if (tid == 0) cen[3] = v;  // R is no longer needed
  }
  __syncthreads();
  const double common = cen[3];
  for (int a = ga + tid; a < ga + gn; a += blockDim.x) {
    const int al = a - ga;
    const int pp = (al < npair) ? al : al - npair, hh = (al < npair) ? 0 : 1;
    double acc = common;
    for (int k = 0; k < nslot; ++k) acc += res_s[pp + k * npair][hh];
    if (g == 0) {
      // far-image lattice part: degrees 0 and 1 (the offset and the field,
      // which carry most of it) in FP64, the rest in working precision (each
      // degree is smaller by about |x| / 3.5 L, and FP64 issues at a small
      // fraction of the FP32 rate here); then the dipole / background term
      const double px = pa[a][0], py = pa[a][1], pz = pa[a][2];
      const double ax = px - 0.5 * L, ay = py - 0.5 * L, az = pz - 0.5 * L, iL = 1.0 / L;
      const double ux = ax * iL, uy = ay * iL, uz = az * iL, r11 = -tab_diag<double>(1);
      double hlow = Lh3[0];
      if (P >= 1) hlow += Lh3[1] * (tab_a<double>(1) * uz) + 2.0 * (Lh3[2] * (r11 * ux) + Lh3[3] * (r11 * uy));
      T hsum = T(0);
      rt_columns<T>(P, (T)ux, (T)uy, (T)uz, [&](int l, int m, T re, T im) {
        const int k = ridx(l, m);
        if (l >= 2) hsum += (m == 0) ? Lh3s[k] * re : T(2) * (Lh3s[k] * re + Lh3s[k + 1] * im);
      });
      const double V3 = L * L * L, c2 = 2.0 * kPi / (3.0 * V3);
      acc += (hlow + (double)hsum) * iL + c2 * (mom[0] * (ax * ax + ay * ay + az * az) -
                                                2.0 * (ax * mom[1] + ay * mom[2] + az * mom[3]) + mom[4]);
    }
    phi_part[(size_t)(b0 + a) * G + g] = acc;
  }
  if (timed_out) break;
  }  // groups
}

// phi_site = f * (sum of the parts, in part order)
__global__ void k_site_phi_sum(int nsa, int nparts, double fcoul, const double *__restrict__ phi_part,
                               double *__restrict__ phi_site) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nsa) return;
  double v = 0.0;
  for (int q = 0; q < nparts; ++q) v += phi_part[(size_t)k * nparts + q];
  phi_site[k] = fcoul * v;
}

// Total energy: kFinalBlocks blocks each sum a contiguous range of the leaf
// partials (block 0 also the site terms) in a fixed order; the block that
// finishes last adds the block sums in block order and re-arms the ticket.
// FP64 issues at a small fraction of the FP32 rate on GB300, so the sum is
// spread over many SMs instead of one.
__global__ void __launch_bounds__(256) k_final_energy(const double *__restrict__ epart, int nb,
                                                     const double *__restrict__ site_e, int S, double *blk,
                                                     unsigned int *ticket, double *__restrict__ out) {
  const int per = (nb + (int)gridDim.x - 1) / (int)gridDim.x;
  const int b0 = min(nb, (int)blockIdx.x * per), b1 = min(nb, b0 + per);
  double v2[2] = {0, 0};
  int k = 0;
  for (int i = b0 + (int)threadIdx.x; i < b1; i += blockDim.x, ++k) v2[k & 1] += epart[i];
  double v = v2[0] + v2[1];
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < S; j += blockDim.x) v += site_e[j];
  __shared__ double red[8];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    blk[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double e = 0;
    for (int b = 0; b < (int)gridDim.x; ++b) e += reinterpret_cast<volatile double *>(blk)[b];
    *out = e;
    *ticket = 0u;
  }
}

template <typename T>
__global__ void k_unpermute_phi(int64_t N, const int *__restrict__ inv_perm, const T *__restrict__ phi_s,
                                double *__restrict__ phi) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) phi[i] = (double)phi_s[inv_perm[i]];
}

// Charge and dipole coefficients of every box's multipole from the FP64 box
// moments (Q, D about the box centre).  In single precision the M2M sums of a
// box's monopole carry an absolute error of about 6e-8 of the sum of |q| over
// its atoms (1e-3 e for a level-1 box of a 200k-atom system), while the box is
// nearly neutral: through the far-field translations that shifted every
// potential by ~0.1 kJ/mol/e.  The FP64 moments rounded once to the working
// precision carry 6e-8 of |Q| instead.  Device basis, u = (x - c) / s:
//   M_00 = Q,  M_10 = D_z / s,  M_11 = -(D_x - i D_y) / (sqrt(2) s)
// (real layout: index 1 = M_10, 2 and 3 = Re and Im of M_11).
template <typename T>
__global__ void k_patch_low_multipoles(int64_t nbox, int d, double L, int ld, const int64_t *__restrict__ level_off,
                                       const double *__restrict__ qd, T *__restrict__ M) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  int l = 0;
  while (l < d && b >= level_off[l + 1]) ++l;
  const double s = L / (double)(1 << l), c = 1.0 / (1.4142135623730951 * s);
  const double *v = qd + (size_t)b * kQD;
  T *m = M + (size_t)b * ld;
  m[0] = (T)v[0];
  m[1] = (T)(v[3] / s);
  m[2] = (T)(-v[1] * c);
  m[3] = (T)(v[2] * c);
}

// ---------------------------------------------------------------------------
// orchestration
// ---------------------------------------------------------------------------
// main-stream intervals, then the two side-stream intervals (overlapping the
// main stream: the sites' FP64 pair terms during binning/P2M/M2M, the refined
// site-atom potential during L2L/L2P/P2P)
static const char *kStageNames[] = {"bin", "sort", "p2m", "m2m", "lattice", "m2l", "l2l", "near_pairs", "far_near_out", "site",
                                    "side_site_pairs", "side_site_potential"};
const char *stage_name(int i) { return (i >= 0 && i < 12) ? kStageNames[i] : "?"; }
int num_stages() { return 10; }

#define MAHI_CK(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return e_;                   \
  } while (0)

// k_site_phi with the M2P order a compile-time constant where one is built;
// `nbmax` is the argument after the row stride
template <typename T, int PP, bool C, typename... A>
static cudaError_t launch_site_phi_pp(int G, size_t smp, cudaStream_t st, int S, A... args) {
  cudaError_t e = cudaFuncSetAttribute(k_site_phi<T, PP, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
  if (e != cudaSuccess) return e;
  k_site_phi<T, PP, C><<<S * G, kSiteThreads, smp, st>>>(S, args...);
  return cudaGetLastError();
}
template <typename T, bool C, typename... A>
static cudaError_t launch_site_phi(int P, int G, size_t smp, cudaStream_t st, int S, A... args) {
  switch (P) {
    case 8: return launch_site_phi_pp<T, 8, C>(G, smp, st, S, args...);
    case 10: return launch_site_phi_pp<T, 10, C>(G, smp, st, S, args...);
    case 12: return launch_site_phi_pp<T, 12, C>(G, smp, st, S, args...);
    case 14: return launch_site_phi_pp<T, 14, C>(G, smp, st, S, args...);
    case 16: return launch_site_phi_pp<T, 16, C>(G, smp, st, S, args...);
    default: return launch_site_phi_pp<T, 0, C>(G, smp, st, S, args...);
  }
}

template <typename T, int NC>
static cudaError_t launch_gemm_nc(const GemmMap &mp, int grid, int K, int ld, const T *in, T *out, const T *ops,
                                  cudaStream_t st) {
  const int nterms = (mp.kind == 0) ? 8 : (mp.kind == 1 ? 1 : kListLen);
  size_t sm = sizeof(T) * 2 * (TR * TK + TK * (size_t)(32 * NC)) + sizeof(int) * nterms * TR;
  if (32 * NC < ld) return cudaErrorInvalidValue;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_gather_gemm<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_gather_gemm<T, NC><<<grid, 256, sm, st>>>(mp, K, ld, in, out, ops);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_gemm(const GemmMap &mp, int K, int ld, const T *in, T *out, const T *ops, cudaStream_t st) {
  int rows_par = (mp.kind == 0) ? mp.nbox : mp.nbox / 8;
  int tiles = (rows_par + TR - 1) / TR;
  int grid = (mp.kind == 0) ? tiles : tiles * 8;
  int nc = (K + 31) / 32;
  if (nc <= 1) return launch_gemm_nc<T, 1>(mp, grid, K, ld, in, out, ops, st);
  if (nc <= 2) return launch_gemm_nc<T, 2>(mp, grid, K, ld, in, out, ops, st);
  if (nc <= 3) return launch_gemm_nc<T, 3>(mp, grid, K, ld, in, out, ops, st);
  if (nc <= 4) return launch_gemm_nc<T, 4>(mp, grid, K, ld, in, out, ops, st);
  if (nc <= 6) return launch_gemm_nc<T, 6>(mp, grid, K, ld, in, out, ops, st);
  if (nc <= 8) return launch_gemm_nc<T, 8>(mp, grid, K, ld, in, out, ops, st);
  if (nc <= 11) return launch_gemm_nc<T, 11>(mp, grid, K, ld, in, out, ops, st);
  if (nc <= 14) return launch_gemm_nc<T, 14>(mp, grid, K, ld, in, out, ops, st);
  return launch_gemm_nc<T, 20>(mp, grid, K, ld, in, out, ops, st);
}

static inline void mark(mahi_ctx *h, int stage, cudaStream_t on = nullptr) {
  if (h->timing && stage < 20) {
    cudaEventRecord(h->ev[stage], on ? on : h->stream);
    h->n_ev = stage + 1;
  }
}
// side-stream interval k (0: site pair terms, 1: site-atom potential) start / end
static inline void mark_side(mahi_ctx *h, int k, int end) {
  if (h->timing) {
    cudaEventRecord(h->ev[kSideEv + 2 * k + end], h->side);
    h->side_timed |= 1 << k;
  }
}

template <typename T, typename XT, int NT>
static cudaError_t launch_p2p(mahi_ctx *h, int nleaf, int nb, const double *mom, XT *forces, cudaStream_t st) {
  using V = typename V4<T>::type;
  const size_t sm = sizeof(V) * P2P_MAXSRC;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_p2p<T, XT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_p2p<T, XT, NT><<<nleaf, NT, sm, st>>>(nb, (T)(2.0 * kPi / (3.0 * h->L * h->L * h->L)), (T)(0.5 * h->L),
                                          (T)(h->L / nb), (T)coulomb_constant(), h->leaf_start,
                                          (const V *)h->part, h->perm,
                                          mom, (T *)h->phi_s, (const T *)h->grad_s, forces, h->energy_part);
  return cudaGetLastError();
}

static cudaError_t launch_p2p_n3(mahi_ctx *h, int nleaf, int nb, cudaStream_t st) {
  constexpr int NT = 128;
  constexpr size_t sm = n3_smem_bytes<NT / 32>();
  static_assert(sm <= 227 * 1024, "near-field staging exceeds shared memory");
  const float s_leaf = (float)(h->L / nb);
  float *phi = (float *)h->phi_s, *grad = (float *)h->grad_s;
  float4 *slots = (float4 *)h->nf_slots;
  const float4 *part = (const float4 *)h->part;
  cudaError_t e;
  if (h->tune_p2p_targets == 4) {
    e = cudaFuncSetAttribute(k_p2p_n3<4, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_p2p_n3<4, NT><<<nleaf, NT, sm, st>>>(nb, s_leaf, h->N, h->leaf_start, part, phi, grad, slots);
  } else {
    e = cudaFuncSetAttribute(k_p2p_n3<8, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_p2p_n3<8, NT><<<nleaf, NT, sm, st>>>(nb, s_leaf, h->N, h->leaf_start, part, phi, grad, slots);
  }
  return cudaGetLastError();
}

template <typename XT>
static cudaError_t launch_l2p_near(mahi_ctx *h, int nleaf, int nb, const float *Lleaf, const double *mom, XT *forces,
                                   cudaStream_t st) {
  const int K = h->K, P = h->p, ld = h->ld;
  const size_t per_warp = sizeof(float4) * (size_t)K;
  const int wpb = (int)std::max<size_t>(1, std::min<size_t>(4, (40 * 1024) / per_warp));
  const dim3 gl((nleaf + wpb - 1) / wpb), bl(32 * wpb);
  const float s = (float)(h->L / nb), c2 = (float)(2.0 * kPi / (3.0 * h->L * h->L * h->L));
  const float half_L = (float)(0.5 * h->L), fc = (float)coulomb_constant();
  const float4 *part = (const float4 *)h->part, *slots = (const float4 *)h->nf_slots;
  if (P == 12)
    k_l2p_near<12, XT><<<gl, bl, per_warp * wpb, st>>>(nleaf, P, ld, s, h->N, c2, half_L, fc, h->leaf_start, part, Lleaf,
                                                       h->perm, mom, slots, (float *)h->phi_s,
                                                       (const float *)h->grad_s, forces, h->energy_part);
  else
    k_l2p_near<0, XT><<<gl, bl, per_warp * wpb, st>>>(nleaf, P, ld, s, h->N, c2, half_L, fc, h->leaf_start, part, Lleaf,
                                                      h->perm, mom, slots, (float *)h->phi_s,
                                                      (const float *)h->grad_s, forces, h->energy_part);
  return cudaGetLastError();
}

template <typename T, typename XT>
static cudaError_t eval_t(mahi_ctx *h, const XT *x, const double *lam, double *energy, XT *forces, double *dEdl) {
  using V = typename V4<T>::type;
  // The whole chain runs on the handle's stream of the greatest priority,
  // forked from the caller's stream here and joined back at the end: the side
  // stream's work (site pair terms, box moments, traversal lists, the
  // site-atom potential) then fills the SMs the chain leaves free instead of
  // delaying it.
  const cudaStream_t st_user = h->stream;
  MAHI_CK(cudaEventRecord(h->hp_ev[0], st_user));
  MAHI_CK(cudaStreamWaitEvent(h->hp, h->hp_ev[0], 0));
  const cudaStream_t st = h->hp;
  const int nb = 1 << h->d;
  const int nleaf = h->nleaf;
  const int64_t N = h->N;
  const int K = h->K, ld = h->ld, P = h->p;
  T *M = (T *)h->Mexp, *Lx = (T *)h->Lexp;
  const double *mom = h->box_qd;  // root box row: Q, D, T of the system about the box centre
  h->launches = 0;
  h->side_timed = 0;
  mark(h, 0, st);
  if (h->S > 0 && !h->multiform) {
    // the sites' FP64 pair terms need only the positions: side stream, from
    // the start (the FP64 pipe is idle during binning, P2M and M2M)
    MAHI_CK(cudaEventRecord(h->fork_ev[2], st));
    MAHI_CK(cudaStreamWaitEvent(h->side, h->fork_ev[2], 0));
    mark_side(h, 0, 0);
    if (h->n_site_pairs > 0)
      k_site_pairs<XT><<<(h->n_site_pairs + 63) / 64, 64, 0, h->side>>>(h->n_site_pairs, h->site_pair_list, h->L,
                                                                       kSiteDegree, h->site_ptr, h->site_atoms, x,
                                                                       h->eta, h->eta_x, h->eta_y, h->eta_z,
                                                                       h->site_pairs);
    mark_side(h, 0, 1);
    h->launches += 1;
  }
  MAHI_CK(cudaMemsetAsync(h->leaf_count, 0, sizeof(int) * nleaf, st));
  {
    const double s_l = h->L / nb;
    float lf = (float)h->L;
    if ((double)lf < h->L) lf = nextafterf(lf, INFINITY);  // smallest float >= L
    k_bin<T, XT><<<h->n_moment_blocks, 256, 0, st>>>(x, N, h->L, s_l, nb / h->L, lf, nb, lam, h->qA, h->dq, h->site_of,
                                                      h->leaf_of, h->slot, h->leaf_count, h->qt, (V *)h->vtmp, h->relD);
  }
  h->launches += 1;
  if (h->multiform && h->n_site_atoms > 0) {
    k_mf_charges<T><<<(h->n_site_atoms + 127) / 128, 128, 0, st>>>(h->n_site_atoms, h->site_atoms, h->site_of,
                                                                    h->mf_lam_off, lam, h->mf_q, h->qt, (V *)h->vtmp);
    h->launches += 1;
  }
  mark(h, 1, st);
  k_scan<<<1, 1024, 0, st>>>(h->leaf_count, nleaf, h->leaf_start);
  int gb = (int)((N + 255) / 256);
  k_scatter<T><<<gb, 256, 0, st>>>(N, h->leaf_of, h->slot, h->leaf_start, (const V *)h->vtmp, (V *)h->part_tmp,
                                   h->perm_tmp);
  k_leaf_sort<T><<<(nleaf * 32 + 255) / 256, 256, 0, st>>>(nleaf, h->leaf_start, (const V *)h->part_tmp, h->perm_tmp,
                                                          (V *)h->part, h->perm, h->inv_perm);
  // FP64 box moments (leaves, then up the tree) on the side stream, while the
  // main stream runs P2M and the M2M GEMMs; joined before the lattice step
  MAHI_CK(cudaEventRecord(h->fork_ev[0], st));
  MAHI_CK(cudaStreamWaitEvent(h->side, h->fork_ev[0], 0));
  k_leaf_moments<<<(nleaf + 127) / 128, 128, 0, h->side>>>(nleaf, h->leaf_start, h->perm, h->qt, h->relD,
                                                            h->box_qd + h->level_off[h->d] * kQD,
                                                            h->box_qdf + h->level_off[h->d] * kQDF);
  for (int l = h->d - 1; l >= 0; --l) {
    const int np = 1 << (3 * l);
    k_qd_up<<<(np + 127) / 128, 128, 0, h->side>>>(np, h->L / (1 << (l + 1)), h->box_qd + h->level_off[l + 1] * kQD,
                                                   h->box_qd + h->level_off[l] * kQD,
                                                   h->box_qdf + h->level_off[l] * kQDF);
  }
  MAHI_CK(cudaEventRecord(h->join_ev[0], h->side));
  h->launches += 4 + h->d;
  // the compact sites' traversal lists (geometry only), on the side stream
  // behind the box moments; the site-atom potential follows on that stream
  const bool site_pre = h->S > 0 && h->site_lists && h->site_lists_cap >= h->site_list_cap;
  if (site_pre) {
    const size_t sml = 2 * sizeof(int) * (size_t)h->site_list_cap;
    if (sml > 48 * 1024)
      MAHI_CK(cudaFuncSetAttribute(k_site_lists<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sml));
    k_site_lists<T><<<h->S, kSiteThreads, sml, h->side>>>(h->S, h->site_ptr, h->site_atoms, h->d, h->L, h->leaf_of,
                                                          h->inv_perm, (const V *)h->part, h->site_theta,
                                                          h->site_list_cap, h->site_lists, h->site_list_n,
                                                          h->site_cen, h->status_dev);
    h->launches += 1;
  }
  MAHI_CK(cudaGetLastError());
  mark(h, 2, st);
  const double s_leaf = h->L / nb;
  {
    const int Ks = K | 1;
    const size_t per_warp = 32 * (size_t)Ks * sizeof(T);
    if (sizeof(T) == 4 && P <= kMaxOrderMixed && 2 * per_warp <= 48 * 1024) {
      if (P == 12)
        k_p2m_c<T, 12><<<(nleaf + 3) / 4, 128, 0, st>>>(nleaf, ld, (T)(1.0 / s_leaf), h->leaf_start,
                                                        (const V *)h->part, M + h->level_off[h->d] * ld);
      else
        k_p2m_t<T, 0><<<(nleaf + 1) / 2, 64, 2 * per_warp, st>>>(nleaf, P, ld, Ks, (T)(1.0 / s_leaf),
                                                                 h->leaf_start, (const V *)h->part,
                                                                 M + h->level_off[h->d] * ld);
    } else {
      k_p2m<T><<<(nleaf * 32 + 127) / 128, 128, 4 * sizeof(T) * ld, st>>>(
          nleaf, P, ld, (T)(1.0 / s_leaf), h->leaf_start, (const V *)h->part, M + h->level_off[h->d] * ld);
    }
  }
  h->launches += 1;
  MAHI_CK(cudaGetLastError());
  mark(h, 3, st);
  for (int l = h->d - 1; l >= 0; --l) {
    MAHI_CK((launch_dense_gemm<T, false>(1 << (3 * l), ld, 8 * ld, M + h->level_off[l + 1] * ld, 8 * ld,
                                          (const T *)h->ops_m2m, ld, M + h->level_off[l] * ld, ld, (T *)h->gemm_ws,
                                          h->gemm_ws_elems, h->num_sms, st, h->launches)));
  }
  MAHI_CK(cudaStreamWaitEvent(st, h->join_ev[0], 0));  // box moments (mom) done
  if (sizeof(T) == 4 && P >= 1) {
    k_patch_low_multipoles<T><<<(int)((h->nbox_total + 255) / 256), 256, 0, st>>>(h->nbox_total, h->d, h->L, ld,
                                                                               h->d_level_off, h->box_qd, M);
    h->launches += 1;
  }
  mark(h, 4, st);
  k_lattice<T><<<(ld + 3) / 4, 128, sizeof(double) * K, st>>>(K, ld, h->L, h->ops_lat, h->ops_lat_h3, mom, M, Lx,
                                                    h->L_h3);
  h->launches += 1;
  MAHI_CK(cudaGetLastError());
  mark(h, 5, st);
  if (h->prec == MAHI_MIXED && h->d >= 1) {
    int rc = tc_m2l(h, st);
    if (rc != 0) return cudaErrorUnknown;
  } else {
    for (int l = 1; l <= h->d; ++l) {
      GemmMap mp{2, l, 1 << (3 * l), h->m2l_list, h->m2l_off};
      MAHI_CK(launch_gemm<T>(mp, K, ld, M + h->level_off[l] * ld, Lx + h->level_off[l] * ld, (const T *)h->ops_m2l,
                             st));
      h->launches += 1;
    }
  }
  mark(h, 6, st);
  if (h->S > 0) {
    // The site-atom potential needs only the multipoles, the box moments and
    // the lattice part, so it runs on the side stream alongside L2L, L2P and
    // P2P (it fills the SMs the coarse L2L levels leave idle); joined before
    // the per-site terms.
    MAHI_CK(cudaEventRecord(h->fork_ev[1], st));
    MAHI_CK(cudaStreamWaitEvent(h->side, h->fork_ev[1], 0));
    mark_side(h, 1, 0);
    // rows per batch: as many as two buffers of staged multipole and
    // charge/dipole rows hold beside the resident rows of levels 0 and 1 (and,
    // for the in-kernel traversal, its four lists) at three blocks per SM
    const int lds = ld + 16 / (int)sizeof(T);
    const size_t per_row = 2 * (sizeof(T) * lds + 4 * sizeof(double));
    const size_t resident = (h->d >= 1 ? 9 : 1) * (sizeof(T) * lds + 4 * sizeof(double));
    auto batch_rows = [&](size_t fixed, size_t &smp) {
      const size_t budget = std::max<size_t>(kSiteSmemBudget, fixed + 8 * per_row);
      const int nbm = (int)std::max<size_t>(8, std::min<size_t>(kSiteBatchMax, (budget - fixed) / per_row));
      smp = fixed + per_row * nbm;
      return nbm;
    };
    size_t smp = 0, smp_c = 0;
    const int nbmax = batch_rows(sizeof(int) * 4 * (size_t)h->site_list_cap + resident, smp);
    const int nbmax_c = batch_rows(resident, smp_c);
    // blocks per site: about one wave over all sites (three resident per SM),
    // unless the autotuner picked a count
    const int G = h->tune_site_blocks > 0
                      ? std::min(kSiteChunksMax, h->tune_site_blocks)
                      : std::max(1, std::min(kSiteChunksMax, (3 * h->num_sms + h->S - 1) / std::max(1, h->S)));
    if (site_pre)
      MAHI_CK((launch_site_phi<T, true>(P, G, smp_c, h->side, h->S, G, h->site_ptr, h->site_atoms, h->d, P, ld, lds,
                                         nbmax_c, h->L, h->d_level_off, h->leaf_start, h->leaf_of, h->inv_perm, (const V *)h->part,
                                         M, h->box_qd, h->box_qdf, mom, h->L_h3, h->phi_part, h->status_dev,
                                         h->site_theta, h->site_list_cap, h->wait_limit_ns, h->site_lists,
                                         h->site_list_n, h->site_cen, h->site_order)));
    // the other sites (spread ones; all of them without lists): the blocks of
    // compact sites leave at once
    MAHI_CK((launch_site_phi<T, false>(P, G, smp, h->side, h->S, G, h->site_ptr, h->site_atoms, h->d, P, ld, lds,
                                        nbmax, h->L, h->d_level_off, h->leaf_start, h->leaf_of, h->inv_perm, (const V *)h->part, M,
                                        h->box_qd, h->box_qdf, mom, h->L_h3, h->phi_part, h->status_dev,
                                        h->site_theta, h->site_list_cap, h->wait_limit_ns,
                                        site_pre ? h->site_lists : nullptr, site_pre ? h->site_list_n : nullptr,
                                        site_pre ? h->site_cen : nullptr, h->site_order)));
    h->launches += site_pre ? 1 : 0;
    k_site_phi_sum<<<(h->n_site_atoms + 127) / 128, 128, 0, h->side>>>(h->n_site_atoms, G, coulomb_constant(),
                                                                        h->phi_part, h->phi_site);
    mark_side(h, 1, 1);
    MAHI_CK(cudaEventRecord(h->join_ev[1], h->side));
  }
  for (int l = 1; l <= h->d; ++l) {
    MAHI_CK((launch_dense_gemm<T, true>(1 << (3 * (l - 1)), 8 * ld, ld, Lx + h->level_off[l - 1] * ld, ld,
                                         (const T *)h->ops_l2l, 8 * ld, Lx + h->level_off[l] * ld, 8 * ld,
                                         (T *)h->gemm_ws, h->gemm_ws_elems, h->num_sms, st, h->launches)));
  }
  mark(h, 7, st);
  const T *Lleaf = Lx + h->level_off[h->d] * ld;
  if (std::is_same<T, float>::value && h->tune_p2p_targets > 0 && h->nf_slots) {
    // near field over the half shell (both sides of every pair), then the far
    // field fused with the near-field sums and the outputs
    MAHI_CK((launch_p2p_n3(h, nleaf, nb, st)));
    mark(h, 8, st);
    MAHI_CK((launch_l2p_near<XT>(h, nleaf, nb, (const float *)Lleaf, mom, (XT *)forces, st)));
    h->launches += 2;
  } else {
    size_t per_warp = sizeof(T) * 4 * (size_t)K;
    int wpb = (int)std::max<size_t>(1, std::min<size_t>(4, (40 * 1024) / per_warp));
    const dim3 gl((nleaf + wpb - 1) / wpb), bl(32 * wpb);
    const T sl = (T)s_leaf;
    if (P == 12)
      k_l2p<T, 12><<<gl, bl, per_warp * wpb, st>>>(nleaf, P, ld, sl, h->leaf_start, (const V *)h->part, Lleaf,
                                                    (T *)h->phi_s, (T *)h->grad_s);
    else
      k_l2p<T, 0><<<gl, bl, per_warp * wpb, st>>>(nleaf, P, ld, sl, h->leaf_start, (const V *)h->part, Lleaf,
                                                   (T *)h->phi_s, (T *)h->grad_s);
    MAHI_CK(cudaGetLastError());
    mark(h, 8, st);
    // threads per target leaf: 128 unless the autotuner picked another
    switch (h->tune_p2p_threads) {
      case 64: MAHI_CK((launch_p2p<T, XT, 64>(h, nleaf, nb, mom, forces, st))); break;
      case 256: MAHI_CK((launch_p2p<T, XT, 256>(h, nleaf, nb, mom, forces, st))); break;
      default: MAHI_CK((launch_p2p<T, XT, 128>(h, nleaf, nb, mom, forces, st))); break;
    }
    h->launches += 2;
  }
  MAHI_CK(cudaGetLastError());
  mark(h, 9, st);
  if (h->S > 0) {
    MAHI_CK(cudaStreamWaitEvent(st, h->join_ev[1], 0));  // site-atom potential done
    if (h->multiform)
      k_site_mf<XT, XT><<<h->S, 32, 0, st>>>(h->S, h->L, coulomb_constant(), kSiteDegree, h->site_aii, h->site_ptr,
                                             h->site_atoms, x, h->mf_lam_off, lam, h->mf_q, h->phi_site, h->eta,
                                             h->eta_x, h->eta_y, h->eta_z, dEdl, h->site_energy, forces, h->mf_psi);
    else
      k_site<T, XT, XT><<<(h->S + 3) / 4, 128, 0, st>>>(h->S, h->L, coulomb_constant(), kSiteDegree, h->site_aii,
                                                        h->site_ptr, h->site_atoms, x, h->dq, lam, h->phi_site, h->eta,
                                                        h->eta_x, h->eta_y, h->eta_z, dEdl, h->site_energy, forces,
                                                        h->psi_site, h->site_pairs);
    h->launches += 3;
  }
  if (energy) {
    double *blk = h->energy_part + nleaf;  // kFinalBlocks block sums, then the ticket
    k_final_energy<<<kFinalBlocks, 256, 0, st>>>(h->energy_part, nleaf, h->site_energy, h->S, blk,
                                                 reinterpret_cast<unsigned int *>(blk + kFinalBlocks), energy);
    h->launches += 1;
  }
  MAHI_CK(cudaGetLastError());
  mark(h, 10, st);
  MAHI_CK(cudaEventRecord(h->hp_ev[1], st));
  MAHI_CK(cudaStreamWaitEvent(st_user, h->hp_ev[1], 0));
  return cudaSuccess;
}

int upload_tables() {
  static bool done = false;
  if (done) return 0;
  double a[kTriMax] = {0}, b[kTriMax] = {0}, dg[kMaxOrder + 1] = {0};
  float af[kTriMax] = {0}, bf[kTriMax] = {0}, dgf[kMaxOrder + 1] = {0};
  for (int l = 0; l <= kMaxOrder; ++l)
    for (int m = 0; m <= l; ++m) {
      const int k = l * (l + 1) / 2 + m;
      if (l > m) {
        a[k] = (2.0 * l - 1.0) / std::sqrt((double)(l + m) * (l - m));
        b[k] = (l - m >= 2) ? std::sqrt((double)(l + m - 1) * (l - m - 1) / ((double)(l + m) * (l - m))) : 0.0;
      }
      af[k] = (float)a[k];
      bf[k] = (float)b[k];
    }
  for (int m = 1; m <= kMaxOrder; ++m) { dg[m] = std::sqrt((2.0 * m - 1.0) / (2.0 * m)); dgf[m] = (float)dg[m]; }
  static double ua[kTriSite], ub[kTriSite], ud[kSiteDegree + 1];
  for (int l = 0; l <= kSiteDegree; ++l)
    for (int m = 0; m <= l; ++m) {
      const int k = l * (l + 1) / 2 + m;
      ua[k] = (l > m) ? (2.0 * l - 1.0) / ((double)(l + m) * (l - m)) : 0.0;
      ub[k] = (l > m) ? 1.0 / ((double)(l + m) * (l - m)) : 0.0;
    }
  ud[0] = 0.0;
  for (int m = 1; m <= kSiteDegree; ++m) ud[m] = 1.0 / (2.0 * m);
  if (cudaMemcpyToSymbol(c_a, a, sizeof(a)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_b, b, sizeof(b)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_diag, dg, sizeof(dg)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_af, af, sizeof(af)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_bf, bf, sizeof(bf)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_diagf, dgf, sizeof(dgf)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_ua, ua, sizeof(ua)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_ub, ub, sizeof(ub)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(c_udiag, ud, sizeof(ud)) != cudaSuccess) return -1;
  done = true;
  return 0;
}

// ---------------------------------------------------------------------------
// Backward of the HI energy (autograd): with g = dLoss/dE,
//   dx = -g F,  dlambda = g dE/dlambda,
//   dqA_i = g ((1 - l) phi~_i - l (1 - l) psi_i),  dqB_i = g (l phi~_i + l (1 - l) psi_i)
// for an atom of a site with lambda l; environment atoms: dqA_i = g phi~_i,
// dqB_i = 0.  phi~ is the last evaluation's potential (refined at site atoms).
// ---------------------------------------------------------------------------
template <typename T, typename FT>
__global__ void k_backward(int64_t N, int S, const double *__restrict__ gE, const FT *__restrict__ F,
                           const double *__restrict__ dEdl, const double *__restrict__ lam,
                           const int *__restrict__ inv_perm, const T *__restrict__ phi_s,
                           const int *__restrict__ site_of, const int *__restrict__ site_slot,
                           const double *__restrict__ phi_site, const double *__restrict__ psi_site,
                           FT *__restrict__ dx, double *__restrict__ dlam, double *__restrict__ dqA,
                           double *__restrict__ dqB) {
  const double g = *gE;
  const FT gf = (FT)g;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    if (dx) {
      dx[3 * i + 0] = -gf * F[3 * i + 0];
      dx[3 * i + 1] = -gf * F[3 * i + 1];
      dx[3 * i + 2] = -gf * F[3 * i + 2];
    }
    if (dqA || dqB) {
      const int sl = site_slot[i];
      double a, b;
      if (sl < 0) {
        a = g * (double)phi_s[inv_perm[i]];
        b = 0.0;
      } else {
        const double l = lam[site_of[i]], w = l * (1.0 - l), phi = phi_site[sl], psi = psi_site[sl];
        a = g * ((1.0 - l) * phi - w * psi);
        b = g * (l * phi + w * psi);
      }
      if (dqA) dqA[i] = a;
      if (dqB) dqB[i] = b;
    }
  }
  if (dlam)
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += stride) dlam[s] = g * dEdl[s];
}

int enqueue_backward(mahi_ctx *h, const double *gE, const void *forces, const double *dEdl, const double *lam,
                     int x_is_fp64, void *dx, double *dlam, double *dqA, double *dqB) {
  const int grid = (int)std::min<int64_t>(4 * (int64_t)h->num_sms, (h->N + 255) / 256);
  const bool f64 = h->prec == MAHI_FP64;
  const int nl = h->multiform ? h->n_lam : h->S;   // entries of dE/dlambda
  if (x_is_fp64) {
    if (f64)
      k_backward<double, double><<<grid, 256, 0, h->stream>>>(h->N, nl, gE, (const double *)forces, dEdl, lam,
                                                              h->inv_perm, (const double *)h->phi_s, h->site_of,
                                                              h->site_slot, h->phi_site, h->psi_site, (double *)dx,
                                                              dlam, dqA, dqB);
    else
      k_backward<float, double><<<grid, 256, 0, h->stream>>>(h->N, nl, gE, (const double *)forces, dEdl, lam,
                                                             h->inv_perm, (const float *)h->phi_s, h->site_of,
                                                             h->site_slot, h->phi_site, h->psi_site, (double *)dx,
                                                             dlam, dqA, dqB);
  } else {
    if (f64)
      k_backward<double, float><<<grid, 256, 0, h->stream>>>(h->N, nl, gE, (const float *)forces, dEdl, lam,
                                                             h->inv_perm, (const double *)h->phi_s, h->site_of,
                                                             h->site_slot, h->phi_site, h->psi_site, (float *)dx,
                                                             dlam, dqA, dqB);
    else
      k_backward<float, float><<<grid, 256, 0, h->stream>>>(h->N, nl, gE, (const float *)forces, dEdl, lam,
                                                            h->inv_perm, (const float *)h->phi_s, h->site_of,
                                                            h->site_slot, h->phi_site, h->psi_site, (float *)dx,
                                                            dlam, dqA, dqB);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Backward of the HI energy for sites with 2^m forms: with g = dLoss/dE and
// the form weights w_r of the atom's site,
//   dE/dq^r_i = w_r (phi~_i + psi^r_i - sum_r' w_r' psi^r'_i)   (site atom i),
//   dE/dq_env_i = phi~_i                                          (environment),
// from E = E(q~) + sum_s f/2 [sum_r w_r G_rr - w^T G w], q~ = sum_r w_r q^r,
// G_rr' = q^r^T A q^r' over the site, psi^r = f A q^r (Eq. "iter_ham_lambda"
// with Eq. "one_site_lambda").  One thread per atom: site atoms write their
// F_s form entries at form_off[s] + r n_s + a (the q_forms layout).
template <typename T>
__global__ void k_backward_mf_charges(int64_t N, const double *__restrict__ gE, const int *__restrict__ inv_perm,
                                      const T *__restrict__ phi_s, const int *__restrict__ site_of,
                                      const int *__restrict__ site_slot, const int *__restrict__ site_ptr,
                                      const int *__restrict__ lam_off, const int *__restrict__ form_off,
                                      const double *__restrict__ lam, const double *__restrict__ phi_site,
                                      const double *__restrict__ psi_form, double *__restrict__ dq_env,
                                      double *__restrict__ dq_forms) {
  const double g = *gE;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    const int sl = site_slot[i];
    if (sl < 0) {
      if (dq_env) dq_env[i] = g * (double)phi_s[inv_perm[i]];
      continue;
    }
    if (dq_env) dq_env[i] = 0.0;  // the q_env entries of site atoms are not used
    if (!dq_forms) continue;
    const int s = site_of[i], m = lam_off[s + 1] - lam_off[s], F = 1 << m;
    const int n = site_ptr[s + 1] - site_ptr[s], a = sl - site_ptr[s];
    double w[kMfMaxForms];
    mf_weights(lam + lam_off[s], m, w);
    double psit = 0.0;
    for (int r = 0; r < F; ++r) psit += w[r] * psi_form[(size_t)sl * kMfMaxForms + r];
    const double phi = phi_site[sl];
    for (int r = 0; r < F; ++r)
      dq_forms[form_off[s] + r * n + a] = g * w[r] * (phi + psi_form[(size_t)sl * kMfMaxForms + r] - psit);
  }
}

int enqueue_backward_forms(mahi_ctx *h, const double *gE, const void *forces, const double *dEdl, const double *lam,
                           int x_is_fp64, void *dx, double *dlam, double *dq_env, double *dq_forms) {
  const int grid = (int)std::min<int64_t>(4 * (int64_t)h->num_sms, (h->N + 255) / 256);
  // positions and lambdas as in the two-form pass (no charge outputs there)
  if (dx || dlam) {
    if (enqueue_backward(h, gE, forces, dEdl, lam, x_is_fp64, dx, dlam, nullptr, nullptr) != 0) return -1;
  }
  if (dq_env || dq_forms) {
    if (h->prec == MAHI_FP64)
      k_backward_mf_charges<double><<<grid, 256, 0, h->stream>>>(
          h->N, gE, h->inv_perm, (const double *)h->phi_s, h->site_of, h->site_slot, h->site_ptr, h->mf_lam_off,
          h->mf_form_off, lam, h->phi_site, h->mf_psi, dq_env, dq_forms);
    else
      k_backward_mf_charges<float><<<grid, 256, 0, h->stream>>>(
          h->N, gE, h->inv_perm, (const float *)h->phi_s, h->site_of, h->site_slot, h->site_ptr, h->mf_lam_off,
          h->mf_form_off, lam, h->phi_site, h->mf_psi, dq_env, dq_forms);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int enqueue_eval(mahi_ctx *h, const void *x, int x_is_fp64, const double *lambda, double *energy, void *forces,
                 double *dEdl) {
  cudaError_t e;
  if (h->prec == MAHI_FP64) {
    if (x_is_fp64) e = eval_t<double, double>(h, (const double *)x, lambda, energy, (double *)forces, dEdl);
    else e = eval_t<double, float>(h, (const float *)x, lambda, energy, (float *)forces, dEdl);
  } else {
    if (x_is_fp64) e = eval_t<float, double>(h, (const double *)x, lambda, energy, (double *)forces, dEdl);
    else e = eval_t<float, float>(h, (const float *)x, lambda, energy, (float *)forces, dEdl);
  }
  return e == cudaSuccess ? 0 : (int)e;
}

// new charges for the same site map: qA as given, D = qB - qA on site atoms,
// 0 on environment atoms (they carry qA only)
__global__ void k_update_charges(int64_t N, const double *__restrict__ qA_in, const double *__restrict__ qB_in,
                                 const int *__restrict__ site_of, double *__restrict__ qA, double *__restrict__ dq) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    const double a = qA_in[i];
    qA[i] = a;
    dq[i] = site_of[i] >= 0 ? qB_in[i] - a : 0.0;
  }
}

int enqueue_update_charges(mahi_ctx *h, const double *qA, const double *qB) {
  const int grid = (int)std::min<int64_t>(4 * (int64_t)h->num_sms, (h->N + 255) / 256);
  k_update_charges<<<grid, 256, 0, h->stream>>>(h->N, qA, qB, h->site_of, h->qA, h->dq);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

__global__ void k_patch_site_phi(int nsa, const int *__restrict__ site_atoms, const double *__restrict__ phi_site,
                                 double *__restrict__ phi) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nsa) phi[site_atoms[k]] = phi_site[k];
}

int enqueue_potential(mahi_ctx *h, double *phi) {
  int g = (int)((h->N + 255) / 256);
  if (h->prec == MAHI_FP64)
    k_unpermute_phi<double><<<g, 256, 0, h->stream>>>(h->N, h->inv_perm, (const double *)h->phi_s, phi);
  else
    k_unpermute_phi<float><<<g, 256, 0, h->stream>>>(h->N, h->inv_perm, (const float *)h->phi_s, phi);
  if (h->n_site_atoms > 0)
    k_patch_site_phi<<<(h->n_site_atoms + 255) / 256, 256, 0, h->stream>>>(h->n_site_atoms, h->site_atoms,
                                                                          h->phi_site, phi);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace mahi
