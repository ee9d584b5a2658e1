// Tensor-core M2L for sm_103a (tcgen05 + TMEM, bulk-async copies, mbarriers).
//
// For every level l >= 1 and every target box t, L~_t = sum_{o in list(c(t))}
// T~_o M~_{t-o} (Fig. "fmm_scheme", step 3; 189 offsets per box).  A CTA owns a
// tile of up to 128 targets with the same child index c (so they share the
// offset list) and accumulates
//     D[128 x Kp] = sum_o A_o[128 x Kp] B_o[Kp x Kp]^T
// in TMEM (fp32, one TMEM lane per target), where row r of A_o is the gathered
// multipole of target r's source box and B_o = T~_o (rows = output coefficient,
// K-major).  Three TF32 products per step (hi*hi + hi*lo + lo*hi) keep the
// result at FP32 accuracy: the multipoles are split into TF32 hi/lo parts once
// per evaluation, the operators once at creation.
//
// Shared-memory operand layout: no swizzle, K-major; an 8-row x 16-byte core
// matrix is 128 contiguous bytes; core matrices are ordered [k-group][row-group],
// so the descriptor strides are LBO = (#row-groups x 128 B) along K and
// SBO = 128 B along M/N.
//
// Warp roles (192 threads): warp 0 allocates TMEM, lane 0 issues the MMAs;
// warps 1-4 gather A rows with cp.async (one row per thread) whose completion
// arrives on the stage barrier asynchronously (cp.async.mbarrier.arrive), so
// the gather of stage i never waits for the MMAs of stage i-1; warp 5 lane 0
// streams B with cp.async.bulk.  Warps 0-3 drain TMEM in the epilogue.
// Every wait is bounded: on expiry the CTA records an error, stops issuing
// work, drains what is in flight and frees its TMEM.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "mahi_internal.h"

namespace mahi {

namespace tc {
constexpr int kRows = 128;       // targets per tile (MMA M)
constexpr int kKC = 16;          // input coefficients per pipeline stage
constexpr int kStages = 5;
constexpr int kThreads = 192;
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr int kMaxN = 256;       // MMA N limit: Kp <= 256, order <= 15

struct Unit {
  int level, child, p0, count;  // targets 8*(p0 + r) + child, r < count
};

struct Params {
  const float *Mhi, *Mlo;       // split multipoles, all levels (row stride ld)
  float *L;                     // locals, all levels (row stride ld)
  const unsigned char *ops;     // B images [316][nch][hi|lo]
  const int4 *units;
  const int *list;              // [8][189] offset ids
  const int *off;               // [316][3]
  const int64_t *level_off;     // [kMaxDepth + 2]
  int *error;
  int ld, nch, ngroups;         // row stride, K chunks, N row groups (Kp/8)
  int nunits;
};
}  // namespace tc

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; returns false (and raises the abort flag) on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *abort_flag) {
  for (uint32_t it = 0; it < tc::kSpinLimit; ++it) {
    if (mbar_try_wait(b, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
// arrive on the barrier once all prior cp.async copies of this thread have landed
__device__ __forceinline__ void cp_async_arrive(uint64_t *b) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(void *smem, const void *gmem, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(smem)),
      "l"(gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor (sm_100 layout): start address, leading and
// stride byte offsets (>> 4), version bits 46-47 = 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor for kind::tf32: D = f32, A = B = tf32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t tc_spread(uint32_t v) {
  uint32_t x = v & 0x3ff;
  x = (x | (x << 16)) & 0x030000FF;
  x = (x | (x << 8)) & 0x0300F00F;
  x = (x | (x << 4)) & 0x030C30C3;
  x = (x | (x << 2)) & 0x09249249;
  return x;
}
__device__ __forceinline__ uint32_t tc_compact(uint32_t x) {
  x &= 0x09249249;
  x = (x ^ (x >> 2)) & 0x030C30C3;
  x = (x ^ (x >> 4)) & 0x0300F00F;
  x = (x ^ (x >> 8)) & 0x030000FF;
  x = (x ^ (x >> 16)) & 0x000003FF;
  return x;
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(tc::kThreads, 1) k_m2l_tc(tc::Params prm) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int ng = prm.ngroups;                       // N row groups (Kp / 8)
  const uint32_t a_bytes = (kKC / 4) * (kRows / 8) * 128;   // one A operand chunk (8 KB)
  const uint32_t b_bytes = (kKC / 4) * ng * 128;            // one B operand chunk
  unsigned char *sA = smem;                                  // [stage][hi|lo][a_bytes]
  unsigned char *sB = sA + kStages * 2 * a_bytes;            // [stage][hi|lo][b_bytes]
  uint64_t *bars = reinterpret_cast<uint64_t *>(sB + kStages * 2 * b_bytes);
  uint64_t *full = bars, *bfull = bars + kStages, *empty = bars + 2 * kStages, *accb = bars + 3 * kStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 3 * kStages + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 u = prm.units[blockIdx.x];
  const int level = u.x, child = u.y, p0 = u.z, count = u.w;
  const int nit = kListLen * prm.nch;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], kRows);
      mbar_init(&bfull[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accb, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // zero the A stages once: rows beyond `count` stay zero for the whole tile
  for (uint32_t i = threadIdx.x * 16; i < kStages * 2 * a_bytes; i += kThreads * 16)
    *reinterpret_cast<float4 *>(sA + i) = make_float4(0.f, 0.f, 0.f, 0.f);
  fence_proxy_async();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp >= 1 && warp <= 4) {
    // ---------------- A producers: one target row per thread ----------------
    const int t = threadIdx.x - 32;
    const bool valid = t < count;
    const int side = 1 << level;
    int bx = 0, by = 0, bz = 0;
    if (valid) {
      const int box = 8 * (p0 + t) + child;
      bx = (int)tc_compact(box); by = (int)tc_compact(box >> 1); bz = (int)tc_compact(box >> 2);
    }
    const float *Mh = prm.Mhi + prm.level_off[level] * prm.ld;
    const float *Ml = prm.Mlo + prm.level_off[level] * prm.ld;
    const uint32_t row_off = (uint32_t)((t >> 3) * 128 + (t & 7) * 16);
    const float *src_h = Mh, *src_l = Ml;
    for (int i = 0; i < nit; ++i) {
      const int s = i % kStages, use = i / kStages;
      if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, abort_flag)) break;
      const int j = i / prm.nch, kc = i - j * prm.nch;
      if (valid && kc == 0) {
        const int oid = prm.list[child * kListLen + j];
        int gx = bx - prm.off[oid * 3 + 0], gy = by - prm.off[oid * 3 + 1], gz = bz - prm.off[oid * 3 + 2];
        gx &= side - 1; gy &= side - 1; gz &= side - 1;   // periodic wrap (side is a power of two)
        const int64_t row = (int64_t)(tc_spread(gx) | (tc_spread(gy) << 1) | (tc_spread(gz) << 2));
        src_h = Mh + row * prm.ld;
        src_l = Ml + row * prm.ld;
      }
      if (valid) {
        unsigned char *dh = sA + (s * 2 + 0) * a_bytes + row_off;
        unsigned char *dl = sA + (s * 2 + 1) * a_bytes + row_off;
#pragma unroll
        for (int g = 0; g < kKC / 4; ++g) {
          cp_async16(dh + g * (kRows / 8) * 128, src_h + kc * kKC + g * 4);
          cp_async16(dl + g * (kRows / 8) * 128, src_l + kc * kKC + g * 4);
        }
      }
      // the stage's barrier receives this thread's arrival when its copies land
      cp_async_arrive(&full[s]);
    }
    cp_async_wait_all();
  } else if (warp == 5) {
    // ---------------- B producer ----------------
    if (lane == 0) {
      const uint32_t img = 2 * b_bytes;  // hi | lo of one (offset, chunk)
      int issued = 0;
      for (int i = 0; i < nit; ++i) {
        const int s = i % kStages, use = i / kStages;
        if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, abort_flag)) break;
        const int j = i / prm.nch, kc = i - j * prm.nch;
        const int oid = prm.list[child * kListLen + j];
        const unsigned char *g = prm.ops + ((size_t)oid * prm.nch + kc) * img;
        mbar_arrive_expect_tx(&bfull[s], img);
        bulk_g2s(sB + (size_t)s * img, g, img, &bfull[s]);
        ++issued;
      }
      // the last copy into each stage is the latest phase of its barrier: wait
      // (bounded) until it has landed before the CTA can retire
      for (int i = (issued > kStages ? issued - kStages : 0); i < issued; ++i) {
        uint64_t *b = &bfull[i % kStages];
        const uint32_t par = (i / kStages) & 1;
        for (uint32_t it = 0; it < kSpinLimit && !mbar_try_wait(b, par); ++it) {
        }
      }
    }
  } else if (warp == 0 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = idesc_tf32(kRows, ng * 8);
    const uint32_t a_lbo = (kRows / 8) * 128, b_lbo = ng * 128;
    int done = 0;
    for (int i = 0; i < nit; ++i) {
      const int s = i % kStages, use = i / kStages;
      if (!mbar_wait(&full[s], use & 1, abort_flag)) break;
      if (!mbar_wait(&bfull[s], use & 1, abort_flag)) break;
      // A was written by cp.async (generic proxy): order it before the MMA reads
      fence_proxy_async();
      tc_fence_after();
      const uint32_t ah = smem_u32(sA + (s * 2 + 0) * a_bytes), al = smem_u32(sA + (s * 2 + 1) * a_bytes);
      const uint32_t bh = smem_u32(sB + (size_t)s * 2 * b_bytes), bl = bh + b_bytes;
#pragma unroll
      for (int ks = 0; ks < kKC / 8; ++ks) {
        const uint32_t ao = ks * 2 * a_lbo, bo = ks * 2 * b_lbo;
        const uint32_t acc0 = (i > 0 || ks > 0) ? 1u : 0u;
        mma_tf32(tmem, smem_desc(ah + ao, a_lbo, 128), smem_desc(bh + bo, b_lbo, 128), idesc, acc0);
        mma_tf32(tmem, smem_desc(ah + ao, a_lbo, 128), smem_desc(bl + bo, b_lbo, 128), idesc, 1u);
        mma_tf32(tmem, smem_desc(al + ao, a_lbo, 128), smem_desc(bh + bo, b_lbo, 128), idesc, 1u);
      }
      mma_commit(&empty[s]);
      ++done;
    }
    mma_commit(accb);
  }
  __syncwarp();

  // ---------------- epilogue: TMEM -> L rows ----------------
  bool ok = true;
  if (warp <= 3) {
    ok = mbar_wait(accb, 0, abort_flag);
    tc_fence_after();
    const int r = warp * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    float *Lrow = nullptr;
    if (ok && !*abort_flag && r < count) Lrow = prm.L + (prm.level_off[level] + 8 * (p0 + r) + child) * prm.ld;
    for (int c0 = 0; c0 < ng * 8; c0 += 16) {
      float v[16];
      tmem_ld16(taddr + c0, v);
      if (Lrow) {
#pragma unroll
        for (int q = 0; q < 16; q += 4)
          *reinterpret_cast<float4 *>(Lrow + c0 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicExch(prm.error, 1);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
  }
}

// Split fp32 multipoles into TF32 hi and the fp32 remainder lo = x - hi.
__global__ void k_split_tf32(const float *__restrict__ M, float *__restrict__ hi, float *__restrict__ lo, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    // round to the nearest value with 10 explicit mantissa bits (ties away from
    // zero) by integer arithmetic on the bit pattern; the remainder is exact
    const float x = M[i];
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    const float fh = __uint_as_float(u);
    hi[i] = fh;
    lo[i] = x - fh;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static inline int kpad(int p) { return nstride(p); }

size_t tc_ops_bytes(int p) {
  const int Kp = kpad(p), nch = Kp / tc::kKC, ng = Kp / 8;
  return (size_t)kNumOffsets * nch * 2 * (tc::kKC / 4) * ng * 128;
}

static inline float tf32_rna(float x) {
  // round to the nearest TF32 value (10 explicit mantissa bits), ties away
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

void tc_pack_ops(int p, const std::vector<std::vector<double>> &m2l, void *host_image) {
  const int K = ncoef(p), Kp = kpad(p), nch = Kp / tc::kKC, ng = Kp / 8;
  const size_t chunk = (size_t)(tc::kKC / 4) * ng * 128;  // bytes of hi (or lo) per chunk
  unsigned char *img = (unsigned char *)host_image;
  std::memset(img, 0, tc_ops_bytes(p));
  for (int o = 0; o < kNumOffsets; ++o)
    for (int kc = 0; kc < nch; ++kc) {
      float *hi = reinterpret_cast<float *>(img + ((size_t)o * nch + kc) * 2 * chunk);
      float *lo = reinterpret_cast<float *>(img + ((size_t)o * nch + kc) * 2 * chunk + chunk);
      for (int g = 0; g < tc::kKC / 4; ++g)
        for (int n = 0; n < Kp; ++n)
          for (int e = 0; e < 4; ++e) {
            int k = kc * tc::kKC + g * 4 + e;
            float v = (n < K && k < K) ? (float)m2l[o][(size_t)n * K + k] : 0.0f;
            float h = tf32_rna(v);
            size_t idx = ((size_t)(g * ng + n / 8) * 128 + (n % 8) * 16) / 4 + e;
            hi[idx] = h;
            lo[idx] = v - h;
          }
    }
}

int tc_build_units(mahi_ctx *h, std::vector<int> &units) {
  if (h->ld > tc::kMaxN || h->ld % tc::kKC) return -1;
  units.clear();
  for (int l = 1; l <= h->d; ++l) {
    const int per_child = 1 << (3 * (l - 1));
    for (int c = 0; c < 8; ++c)
      for (int p0 = 0; p0 < per_child; p0 += tc::kRows) {
        units.push_back(l);
        units.push_back(c);
        units.push_back(p0);
        units.push_back(std::min(tc::kRows, per_child - p0));
      }
  }
  h->tc_nunits = (int)units.size() / 4;
  return 0;
}

static size_t tc_smem_bytes(int ng) {
  const size_t a = (tc::kKC / 4) * (tc::kRows / 8) * 128, b = (size_t)(tc::kKC / 4) * ng * 128;
  return tc::kStages * 2 * (a + b) + (3 * tc::kStages + 1) * 8 + 16;
}

int tc_m2l(mahi_ctx *h) {
  // split the multipoles (all levels) into TF32 hi / lo
  const int64_t n = h->nbox_total * h->ld;
  float *Mhi = (float *)h->tc_msplit, *Mlo = Mhi + n;
  k_split_tf32<<<4 * 152, 256, 0, h->stream>>>((const float *)h->Mexp, Mhi, Mlo, n);
  tc::Params prm;
  prm.Mhi = Mhi;
  prm.Mlo = Mlo;
  prm.L = (float *)h->Lexp;
  prm.ops = (const unsigned char *)h->tc_ops;
  prm.units = (const int4 *)h->tc_units;
  prm.list = h->m2l_list;
  prm.off = h->m2l_off;
  prm.level_off = h->tc_level_off;
  prm.error = h->tc_error;
  prm.ld = h->ld;
  prm.nch = h->ld / tc::kKC;
  prm.ngroups = h->ld / 8;
  prm.nunits = h->tc_nunits;
  const size_t sm = tc_smem_bytes(prm.ngroups);
  if (sm > 227 * 1024) return -1;
  if (cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return -1;
  if (h->tc_nunits == 0) return 0;
  k_m2l_tc<<<h->tc_nunits, tc::kThreads, sm, h->stream>>>(prm);
  h->launches += 2;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace mahi
