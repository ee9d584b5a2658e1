// Tensor-core M2L for sm_103a (tcgen05 + TMEM, bulk-async copies, mbarriers).
//
// For every level l >= 1 and every target box t, L~_t = sum_{o in list(c(t))}
// T~_o M~_{t-o} (Fig. "fmm_scheme", step 3; 189 offsets per box).  A CTA owns
// tiles of up to 128 targets with the same child index c (so they share the
// offset list) and accumulates
//     D[128 x Kp] = sum_o A_o[128 x Kp] B_o[Kp x Kp]^T
// in TMEM (fp32, one TMEM lane per target), where row r of A_o is the gathered
// multipole of target r's source box and B_o = T~_o (rows = output coefficient,
// K-major).  Operands are TF32: the multipoles are rounded to TF32 hi parts
// (and lo = remainder) once per evaluation, the operators once at creation.
// Input coefficients of low degree (the first nsplit K chunks) take three
// products (hi*hi + hi*lo + lo*hi, FP32-level), the rest one (hi*hi).
//
// Shared-memory operand layout: no swizzle, K-major; an 8-row x 16-byte core
// matrix is 128 contiguous bytes; core matrices are ordered [k-group][row-group],
// so the descriptor strides are LBO = (#row-groups x 128 B) along K and
// SBO = 128 B along M/N.
//
// Warp roles (480 threads): warp 0 allocates TMEM, and its lane 0 and lane 0
// of warp 14 issue the MMAs of tile 0 and tile 1; warp 1 lane 0 streams B with
// cp.async.bulk; warps 2-9 are two groups of A producers taking the even and
// the odd pipeline items, gathering source rows with cp.async and storing
// their TF32 parts in TMEM; warps 10-13 drain TMEM in the epilogue.  Every wait
// is bounded: on expiry the CTA records an error, stops issuing work, drains
// what is in flight and frees its TMEM.

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "mahi_internal.h"
#include "mahi_sync.h"

namespace mahi {

namespace tc {
constexpr int kRows = 128;       // targets per tile (MMA M)
constexpr int kKC = 8;           // input coefficients per K chunk (one MMA K)
constexpr int kKPI = 2;          // virtual K chunks per pipeline item
constexpr int kStagesA = 4;      // A stages in tensor memory (32 columns: 2 tiles x 2 chunks x 8)
constexpr int kStagesS = 3;      // A staging slots in shared memory per producer group (cp.async)
constexpr int kStagesB = 4;      // B stages in shared memory (at most; Params::nsb is the count used)
constexpr int kDone = 8;         // done ring: one entry per item pair
constexpr int kThreads = 480;     // 15 warps: MMA (tile 0), B producer, 2 x 4 A producers, 4 epilogue, MMA (tile 1)
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s: drains of work in flight (they end in microseconds)
constexpr int kMaxN = 256;       // MMA N limit: Kp <= 256, order <= 15
constexpr int kSlotBytes = kKPI * 2 * 2 * kRows * 16;   // A staging slot: [chunk][tile][granule][row] 16 B

// A unit is up to two 128-row tiles of one child class c.  Its rows index the
// class's targets of ALL levels in one sequence (level d first, then d - 1, ...,
// 1; within a level in the class's grid order), so that the coarse levels,
// whose classes hold 1, 8, 64, ... targets, share tiles instead of occupying
// mostly empty ones: int4 {c, r0, n0, n1} = rows r0 .. r0 + n0 - 1 in tile 0
// and r0 + 128 .. r0 + 127 + n1 in tile 1.  The operators are the same for all
// levels (scale-normalised expansions), so any mix of levels can share them.
//
// Pipeline items.  Per interaction offset j the K dimension is walked as nvc =
// nch + nsplit virtual chunks: v < nch is the TF32 hi part of chunk v (with the
// hi*lo operator product too when v < nsplit), v >= nch is the lo part of
// chunk v - nch (times the operator's hi part).  An item is kKPI consecutive
// virtual chunks of one offset, so one handshake (A stage, B stage, commit)
// covers kKPI chunks; ngrp = ceil(nvc / kKPI) items per offset.

struct Params {
  const float *M;               // multipoles in the M2L source layout (see k_m2l_src_layout)
  float *L;                     // locals, all levels (row stride ld)
  const unsigned char *ops;     // B images [316][nch][hi|lo]
  const int4 *units;
  const int *list;              // [8][189] offset ids
  const int *off;               // [316][3]
  const int64_t *level_off;     // [kMaxDepth + 2]
  int *error;                   // status word slot (host-mapped), set to 1 when a wait gave up
  uint64_t wait_ns;             // limit of every bounded pipeline wait
  int selftest;                 // 1: the tile-0 issuer first waits on a barrier nothing completes
  int ld, nch, ngroups;         // row stride, K chunks, N row groups (Kp/8)
  int d;                        // tree depth (levels 1..d hold M2L targets)
  int nsplit;                   // K chunks 0..nsplit-1: three TF32 products; the rest: one
  int nvc, ngrp;                // virtual chunks and items per offset
  int nunits;
  int nfull, nrem, q;           // units done whole (round-robin), remainder units, slices per remainder unit
  int paired;                   // 1: a unit has two 128-target tiles (Kp <= 192); 0: one tile
  int nsb;                      // B stages that fit in shared memory (2..kStagesB)
  float *partial;               // [nrem * q][2][kRows][ld] partial tiles of the remainder units
};
}  // namespace tc

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
// 16-byte copy; with src_bytes = 0 the destination is zero-filled and nothing is read
__device__ __forceinline__ void cp_async16_zfill(void *smem, const void *gmem, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
               : "memory");
}
// arrive on the barrier once all prior cp.async copies of this thread have landed
__device__ __forceinline__ void cp_async_arrive(uint64_t *b) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
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
// D (tmem) += A (tmem, M lanes x 8 tf32 columns) * B (shared memory descriptor)
__device__ __forceinline__ void mma_tf32_ts(uint32_t dtmem, uint32_t atmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(dtmem),
      "r"(atmem), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t *r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
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
// the kernel: persistent, one CTA per SM (grid G).  A unit has two 128-target
// tiles of one child class (same offset list, so both tiles use every staged
// operator chunk: half the operator traffic per flop).  CTA k computes the
// whole units k, k + G, ... below nfull = G * floor(nunits / G), so all CTAs
// walk the same (offset, chunk) sequence at the same time and share the
// operator chunks in L2.  The nrem remainder units are cut along that sequence
// into q equal slices each, one slice per CTA; slices write partial tiles that
// k_m2l_tc_reduce adds up in a fixed order.
//
// The A operand (gathered multipoles) lives in tensor memory: the producer
// warps load each target's source rows from global memory, round them to TF32
// parts in registers and store them with tcgen05.st, so shared memory carries
// only the operator chunks (B).
// Warp roles: 0 = TMEM owner + tile-0 MMA issuer (one lane), 1 = B producer
// (bulk copies), 2-5 and 6-9 = A producers of the even and odd items (row t of
// both tiles = TMEM lane t; a warp may touch only its TMEM lane quarter,
// warp % 4), 10-13 = epilogue (TMEM -> L), 14 = tile-1 MMA issuer (one lane).
// TMEM columns: [0, 176) tile-0 accumulator, [192, 368) tile-1 accumulator,
// [384 + 32 s, 416 + 32 s) A stage s: tile 0 chunks 0, 1, tile 1 chunks 0, 1
// (8 columns each).
// ---------------------------------------------------------------------------
namespace tc {
constexpr uint32_t kAcc1 = 192, kAcol = 384;

// Walks the items of CTA k in order without divisions: segment (whole unit
// or remainder slice), unit, offset j and virtual chunk group g.
struct ItemIter {
  int seg, unit, i, i1, j, g;
};
__device__ __forceinline__ void iter_seg(const Params &p, int k, int nA, int nit, ItemIter &it) {
  if (it.seg < nA) {
    it.unit = k + it.seg * (int)gridDim.x;
    it.i = 0;
    it.i1 = nit;
    it.j = 0;
    it.g = 0;
  } else {
    const int sl = k % p.q;
    it.unit = p.nfull + k / p.q;
    it.i = (int)(((int64_t)sl * nit) / p.q);
    it.i1 = (int)(((int64_t)(sl + 1) * nit) / p.q);
    it.j = it.i / p.ngrp;
    it.g = it.i - it.j * p.ngrp;
  }
}
__device__ __forceinline__ void iter_begin(const Params &p, int k, int nA, int nit, ItemIter &it) {
  it.seg = 0;
  iter_seg(p, k, nA, nit, it);
}
// advance by one item; returns true when a new segment starts
__device__ __forceinline__ bool iter_next(const Params &p, int k, int nA, int nit, ItemIter &it) {
  ++it.i;
  if (++it.g == p.ngrp) {
    it.g = 0;
    ++it.j;
  }
  if (it.i < it.i1) return false;
  ++it.seg;
  iter_seg(p, k, nA, nit, it);
  return true;
}

// K chunk of virtual chunk v and whether it is the lo part
__device__ __forceinline__ int vchunk(const Params &p, int v, bool &lo) {
  lo = v >= p.nch;
  return lo ? v - p.nch : v;
}

// targets in tile h (0 or 1) of a unit
__device__ __forceinline__ int tile_count(const Params &, const int4 &u, int h) { return h == 0 ? u.z : u.w; }

// level and in-class index of merged row r of a class (levels d, d - 1, ..., 1)
__device__ __forceinline__ int row_level(int d, int r, int &tau) {
  int start = 0;
  for (int l = d; l >= 1; --l) {
    const int n = 1 << (3 * (l - 1));
    if (r < start + n) {
      tau = r - start;
      return l;
    }
    start += n;
  }
  tau = 0;
  return 0;
}

// TF32 round-to-nearest (ties away) on the bit pattern; the remainder is exact
__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  hi = u;
  lo = __float_as_uint(x - __uint_as_float(u));
}

// the source rows of one producer thread (row t of both tiles), advanced item by
// item; each row has its own level
struct ARow {
  int unit = -1, j = -1, child = 0;
  int lev[2] = {1, 1};
  int bx[2] = {0, 0}, by[2] = {0, 0}, bz[2] = {0, 0};
  bool valid[2] = {false, false};
  int rsrc[2] = {0, 0};          // float offset of the source chunk of K plane 0 (current offset j)
  int rpl[2] = {0, 0};           // floats per K plane at the row's level (8^l chunks of 8)
};

// target tau of a child class c at level l (parity class c, grid order
// z/2, y/2, x/2 within the class) -> box coordinates
__device__ __forceinline__ void class_target(int l, int c, int tau, int &x, int &y, int &z) {
  const int hb = l - 1, hm = (1 << hb) - 1;
  x = 2 * (tau & hm) + (c & 1);
  y = 2 * ((tau >> hb) & hm) + ((c >> 1) & 1);
  z = 2 * (tau >> (2 * hb)) + ((c >> 2) & 1);
}

// Copies of item (offset j, virtual chunk group g) for the 32 rows of this
// warp into staging slot `dst` ([chunk k][tile h][granule e][row] of 16 bytes;
// rows past a tile's count and virtual chunks past nvc are zero-filled).  Lane
// l copies granule (l & 1) of row 16 rh + (l >> 1) (rh = 0, 1) of each tile, so
// one warp instruction reads 16 whole 32-byte source chunks (512 contiguous
// bytes where the sources are consecutive).  Each row's source offset is
// computed by its own lane and exchanged by shuffles; the caller must
// __syncwarp() after its cp.async wait before reading rows written by other
// lanes.
__device__ __forceinline__ void arow_issue_coalesced(const Params &p, const int *s_list, const int *s_off, int t,
                                                     int lane, const ItemIter &it, ARow &a, unsigned char *dst) {
  const int unit = it.unit, j = it.j;
  if (unit != a.unit) {
    const int4 u = p.units[unit];
    a.child = u.x;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      a.valid[h] = t < tile_count(p, u, h);
      int tau = 0;
      const int l = a.valid[h] ? row_level(p.d, u.y + h * kRows + t, tau) : 1;
      a.valid[h] = a.valid[h] && l >= 1;
      a.lev[h] = a.valid[h] ? l : 1;
      class_target(a.lev[h], a.child, tau, a.bx[h], a.by[h], a.bz[h]);
      a.rpl[h] = 8 << (3 * a.lev[h]);
    }
    a.unit = unit;
    a.j = -1;
  }
  if (j != a.j) {
    const int oid = s_list[a.child * kListLen + j];
    const int ox = s_off[oid * 3 + 0], oy = s_off[oid * 3 + 1], oz = s_off[oid * 3 + 2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!a.valid[h]) continue;
      // source box, periodic wrap (the side is a power of two), in the class
      // order of the source layout
      const int l = a.lev[h], hb = l - 1, sm = (1 << l) - 1;
      const int sx = (a.bx[h] - ox) & sm, sy = (a.by[h] - oy) & sm, sz = (a.bz[h] - oz) & sm;
      const int cls = (sx & 1) | ((sy & 1) << 1) | ((sz & 1) << 2);
      const int sidx = (((cls << hb | (sz >> 1)) << hb | (sy >> 1)) << hb) | (sx >> 1);
      a.rsrc[h] = (int)(p.level_off[l] * p.ld) + sidx * kKC;
    }
    a.j = j;
  }
  const int e = lane & 1, rbase = t & ~31;
#pragma unroll
  for (int kk = 0; kk < kKPI; ++kk) {
    const int v = it.g * kKPI + kk;
    bool lo;
    const int c = vchunk(p, v, lo);
    const bool live = v < p.nvc;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      // own row as a signed 32-bit code: float offset of its source chunk, or -1
      const int mine = (live && a.valid[h]) ? a.rsrc[h] + c * a.rpl[h] : -1;
#pragma unroll
      for (int rh = 0; rh < 2; ++rh) {
        const int src = __shfl_sync(0xffffffffu, mine, 16 * rh + (lane >> 1));
        const int row = rbase + 16 * rh + (lane >> 1);
        const float *gp = p.M + (src < 0 ? 0 : src) + 4 * e;
        cp_async16_zfill(dst + (((kk * 2 + h) * 2 + e) * kRows + row) * 16, gp, src < 0 ? 0u : 16u);
      }
    }
  }
}

}  // namespace tc

// Multipoles of levels 1..d rewritten for the M2L gathers: per level, K planes
// of 8 coefficients, each plane ordered by parity class (x&1, y&1, z&1) and then
// z/2, y/2, x/2, so that the sources of consecutive targets of one class under
// one offset are consecutive 32-byte chunks.
__global__ void k_m2l_src_layout(const float *__restrict__ M, float *__restrict__ S, const int64_t *__restrict__ level_off,
                                 int ld, int d) {
  const int64_t n4 = (level_off[d + 1] - level_off[1]) * ld / 4;  // float4 granules of levels 1..d
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = e * 4 + level_off[1] * ld;  // destination float index
    int l = 1;
    while (l < d && f >= level_off[l + 1] * ld) ++l;
    const int hb = l - 1;
    const int64_t r = f - level_off[l] * ld;       // float index within the level
    const int g = (int)(r & 7);                    // 0 or 4: half of a chunk
    const int64_t ch = r >> 3;                     // chunk index
    const int64_t per_plane = (int64_t)8 << (3 * hb);
    const int kc = (int)(ch / per_plane);
    const int64_t w = ch - kc * per_plane;
    const int hm = (1 << hb) - 1;
    const int hx = (int)(w & hm), hy = (int)((w >> hb) & hm), hz = (int)((w >> (2 * hb)) & hm);
    const int cls = (int)(w >> (3 * hb));
    const int x = 2 * hx + (cls & 1), y = 2 * hy + ((cls >> 1) & 1), z = 2 * hz + ((cls >> 2) & 1);
    const int64_t box = (int64_t)(tc_spread(x) | (tc_spread(y) << 1) | (tc_spread(z) << 2));
    const float4 v = *reinterpret_cast<const float4 *>(M + (level_off[l] + box) * ld + kc * tc::kKC + g);
    *reinterpret_cast<float4 *>(S + f) = v;
  }
}

namespace tc {
__device__ __forceinline__ int64_t class_box_row(const Params &p, int l, int c, int tau) {
  int x, y, z;
  class_target(l, c, tau, x, y, z);
  return p.level_off[l] + (int64_t)(tc_spread(x) | (tc_spread(y) << 1) | (tc_spread(z) << 2));
}
}  // namespace tc

__global__ void __launch_bounds__(tc::kThreads, 1) k_m2l_tc(tc::Params prm) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int ng = prm.ngroups;                       // N row groups (Kp / 8)
  const uint32_t b_bytes = (kKC / 4) * ng * 128;    // hi (or lo) of one operator chunk
  const uint32_t b_stage = kKPI * 2 * b_bytes;      // [chunk][hi|lo] of one item
  unsigned char *sB = smem;                         // [B stage][chunk][hi|lo][b_bytes]
  const int nsb = prm.nsb;
  unsigned char *sS = sB + nsb * b_stage;           // [group][slot] A staging (kSlotBytes each)
  int *s_list = reinterpret_cast<int *>(sS + 2 * kStagesS * kSlotBytes);   // [8][189] offset ids
  int *s_off = s_list + 8 * kListLen;                                      // [316][3] offsets
  uint64_t *bars = reinterpret_cast<uint64_t *>(s_off + ((3 * kNumOffsets + 1) & ~1));
  // idle[0] is a barrier that nothing arrives on (the watchdog self-test waits on it)
  uint64_t *fullA = bars, *fullB = fullA + kStagesA, *done = fullB + kStagesB, *idle = done + kDone;
  uint64_t *accb = idle + 1, *tfree = accb + 1;
  uint64_t *mdone = tfree + 1;                      // [2] last commit of each MMA issuer
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mdone + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nit = kListLen * prm.ngrp;              // items of one unit
  const int k = blockIdx.x;
  const int nA = prm.nfull / (int)gridDim.x;        // whole units of this CTA
  int slice_len = 0;
  if (k < prm.nrem * prm.q) {
    const int j = k % prm.q;
    slice_len = (int)(((int64_t)(j + 1) * nit) / prm.q - ((int64_t)j * nit) / prm.q);
  }
  const int nloc = nA * nit + slice_len;
  const int nseg = nA + (slice_len > 0 ? 1 : 0);
  if (nloc == 0) return;                            // uniform over the block

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesA; ++s) mbar_init(&fullA[s], 4);   // the four warps of the item's producer group
    for (int s = 0; s < kStagesB; ++s) mbar_init(&fullB[s], 1);   // the B producer (plus the copies' bytes)
    for (int s = 0; s < kDone; ++s) mbar_init(&done[s], 2);       // one commit per MMA issuer and item pair
    mbar_init(idle, 1);                                           // never arrived on
    mbar_init(accb, 2);
    mbar_init(tfree, kRows);
    mbar_init(&mdone[0], 1);
    mbar_init(&mdone[1], 1);
    *abort_flag = 0;
  }
  for (int e = threadIdx.x; e < 8 * kListLen; e += blockDim.x) s_list[e] = prm.list[e];
  for (int e = threadIdx.x; e < 3 * kNumOffsets; e += blockDim.x) s_off[e] = prm.off[e];
  if (threadIdx.x == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp >= 2 && warp <= 9) {
    // ---------------- A producers: two groups of four warps take the even and
    // the odd items; row t of both tiles (TMEM lane t) per thread ----------------
    // each group copies its items kStagesS - 1 items ahead into its own staging
    // ring (cp.async groups, one per item, coalesced across the warp), then
    // every thread rounds its own rows to the TF32 part of each virtual chunk
    // and stores them in TMEM
    const int grp = (warp - 2) >> 2;
    const int quarter = warp & 3;
    const int t = quarter * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    unsigned char *ring = sS + (size_t)grp * kStagesS * kSlotBytes;
    constexpr int D = kStagesS - 1;
    const int nmine = (nloc - grp + 1) >> 1;        // items 2 jj + grp of this group
    ARow a;
    ItemIter it;                                    // issue position, D items of this group ahead
    iter_begin(prm, k, nA, nit, it);
    if (grp) iter_next(prm, k, nA, nit, it);
    ItemIter ic = it;                               // position of the item being stored
    int slot_i = 0;                                 // staging slot of the next issue
    for (int qq = 0; qq < D; ++qq) {
      if (qq < nmine) {
        arow_issue_coalesced(prm, s_list, s_off, t, lane, it, a, ring + (size_t)slot_i * kSlotBytes);
        iter_next(prm, k, nA, nit, it);
        iter_next(prm, k, nA, nit, it);
      }
      slot_i = slot_i + 1 == kStagesS ? 0 : slot_i + 1;
      cp_async_commit();
    }
    int slot_c = 0;                                 // staging slot of item jj
    for (int jj = 0; jj < nmine; ++jj) {
      const int q = 2 * jj + grp;
      if (jj + D < nmine) {
        arow_issue_coalesced(prm, s_list, s_off, t, lane, it, a, ring + (size_t)slot_i * kSlotBytes);
        iter_next(prm, k, nA, nit, it);
        iter_next(prm, k, nA, nit, it);
      }
      slot_i = slot_i + 1 == kStagesS ? 0 : slot_i + 1;
      cp_async_commit();
      cp_async_wait_group<D>();                     // this thread's copies of item q have landed
      __syncwarp();                                 // ... and those of the other lanes of the warp
      // round first: it needs only the staging slot, not the TMEM stage
      const unsigned char *src = ring + (size_t)slot_c * kSlotBytes + t * 16;
      uint32_t w[32];  // tile 0 chunk 0 | tile 0 chunk 1 | tile 1 chunk 0 | tile 1 chunk 1, 8 columns each
#pragma unroll
      for (int kk = 0; kk < kKPI; ++kk) {
        bool lo;
        vchunk(prm, ic.g * kKPI + kk, lo);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float4 x = *reinterpret_cast<const float4 *>(src + ((kk * 2 + h) * 2 + e) * kRows * 16);
            uint32_t *o = w + (h * kKPI + kk) * 8 + 4 * e;
            uint32_t hi4[4], lo4[4];
            tf32_split(x.x, hi4[0], lo4[0]);
            tf32_split(x.y, hi4[1], lo4[1]);
            tf32_split(x.z, hi4[2], lo4[2]);
            tf32_split(x.w, hi4[3], lo4[3]);
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) o[c4] = lo ? lo4[c4] : hi4[c4];
          }
      }
      __syncwarp();                                 // staging slot read by all lanes before it is refilled
      iter_next(prm, k, nA, nit, ic);
      iter_next(prm, k, nA, nit, ic);
      const int s = q % kStagesA;
      // lane 0 waits for the TMEM stage (its MMAs of item q - kStagesA done)
      // and the warp follows it; the whole warp leaves together on a timeout
      // (the TMEM store below is warp-collective)
      bool ok = true;
      // (item q - kStagesA is done when the done-ring entry of its item pair
      // has its phase complete: one commit per MMA issuer and item pair)
      if (q >= kStagesA && lane == 0) {
        const int pd = (q - kStagesA) >> 1;
        ok = mbar_wait(&done[pd % kDone], (uint32_t)((pd / kDone) & 1), abort_flag, prm.wait_ns);
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      tc_fence_after();
      tmem_st32(lane_addr + kAcol + 32u * (uint32_t)s, w);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&fullA[s]);        // one arrival per warp
      slot_c = slot_c + 1 == kStagesS ? 0 : slot_c + 1;
    }
    cp_async_wait_all();
  } else if (warp == 1) {
    // ---------------- B producer ----------------
    if (lane == 0) {
      int issued = 0, ucur = -1, child = 0, s = 0;
      ItemIter it;
      iter_begin(prm, k, nA, nit, it);
      for (int q = 0; q < nloc; ++q) {
        // stage s was last used by item q - nsb: wait until its item pair is done
        if (q >= nsb) {
          const int pd = (q - nsb) >> 1;
          if (!mbar_wait(&done[pd % kDone], (uint32_t)((pd / kDone) & 1), abort_flag, prm.wait_ns)) break;
        }
        if (it.unit != ucur) {
          child = prm.units[it.unit].x;
          ucur = it.unit;
        }
        const int oid = s_list[child * kListLen + it.j];
        // per virtual chunk: hi | lo of the operator chunk for the hi part of a
        // three-product chunk, else its hi part only
        uint32_t bytes[kKPI], total = 0;
        const unsigned char *gsrc[kKPI];
#pragma unroll
        for (int kk = 0; kk < kKPI; ++kk) {
          const int v = it.g * kKPI + kk;
          bool lo;
          const int c = vchunk(prm, v, lo);
          bytes[kk] = v >= prm.nvc ? 0u : ((!lo && c < prm.nsplit) ? 2 * b_bytes : b_bytes);
          gsrc[kk] = prm.ops + ((size_t)oid * prm.nch + c) * 2 * b_bytes;
          total += bytes[kk];
        }
        mbar_arrive_expect_tx(&fullB[s], total);
#pragma unroll
        for (int kk = 0; kk < kKPI; ++kk)
          if (bytes[kk]) bulk_g2s(sB + (size_t)s * b_stage + kk * 2 * b_bytes, gsrc[kk], bytes[kk], &fullB[s]);
        ++issued;
        iter_next(prm, k, nA, nit, it);
        if (++s == nsb) s = 0;
      }
      // the last copy into each stage is the latest phase of its barrier: wait
      // (bounded) until it has landed before the CTA can retire
      for (int i = (issued > nsb ? issued - nsb : 0); i < issued; ++i) {
        uint64_t *b = &fullB[i % nsb];
        const uint32_t par = (i / nsb) & 1;
        const uint64_t t0 = global_ns();
        for (uint32_t it2 = 0; it2 < kSpinLimit && !mbar_try_wait(b, par); ++it2)
          if ((it2 & 255) == 255 && global_ns() - t0 > kWaitNs) break;
      }
    }
  } else if ((warp == 0 || warp == 14) && lane == 0) {
    // ---------------- MMA issuers: warp 0 issues tile 0, warp 14 tile 1 ----------------
    // The issuing thread's fixed cost per item (barrier tests, fences,
    // bookkeeping) exceeds that of an MMA instruction, so an item carries
    // kKPI chunks; the two tiles are issued by two threads on different warps,
    // each committing to the done ring (count 2) once per item pair.
    const int mt = warp == 14 ? 1 : 0;
    const uint32_t idesc = idesc_tf32(kRows, ng * 8);
    const uint32_t b_lbo = ng * 128;
    const uint32_t dt = tmem + (mt ? kAcc1 : 0u);
    int ntile = 1, sa = 0, sb = 0;
    uint32_t pa = 0, pb = 0;                        // phase parities of fullA[sa], fullB[sb]
    bool first = true, seg_start = true;
    ItemIter it;
    iter_begin(prm, k, nA, nit, it);
    const uint32_t sB0 = smem_u32(sB);
    // watchdog self-test: a wait that runs out before any MMA is issued
    const bool go = !(prm.selftest && mt == 0) || mbar_wait(idle, 0, abort_flag, prm.wait_ns);
    for (int q = 0; go && q < nloc; ++q) {
      if (seg_start) {
        // new segment: the accumulators must have been drained by the epilogue
        if (it.seg >= 1 && !mbar_wait(tfree, (it.seg - 1) & 1, abort_flag, prm.wait_ns)) break;
        tc_fence_after();
        first = true;
        ntile = tile_count(prm, prm.units[it.unit], 1) > 0 ? 2 : 1;
      }
      if (!mbar_wait2(&fullA[sa], pa, &fullB[sb], pb, abort_flag, prm.wait_ns)) break;
      tc_fence_after();
      if (mt < ntile) {
#pragma unroll
        for (int kk = 0; kk < kKPI; ++kk) {
          const int v = it.g * kKPI + kk;
          if (v >= prm.nvc) break;
          bool lo;
          const int c = vchunk(prm, v, lo);
          const uint32_t bh = sB0 + (uint32_t)sb * b_stage + (uint32_t)kk * 2u * b_bytes;
          const uint64_t dbh = smem_desc(bh, b_lbo, 128);
          const uint32_t av = tmem + kAcol + 32u * (uint32_t)sa + 16u * (uint32_t)mt + 8u * (uint32_t)kk;
          mma_tf32_ts(dt, av, dbh, idesc, first ? 0u : 1u);   // hi*hi, or lo*hi for a lo part
          first = false;
          if (!lo && c < prm.nsplit) mma_tf32_ts(dt, av, smem_desc(bh + b_bytes, b_lbo, 128), idesc, 1u);  // hi*lo
        }
      }
      seg_start = iter_next(prm, k, nA, nit, it);
      // item pair done: frees the B and A stages of its two items
      if ((q & 1) || q == nloc - 1) mma_commit(&done[(q >> 1) % kDone]);
      if (seg_start || q == nloc - 1) mma_commit(accb);  // segment complete
      if (++sa == kStagesA) { sa = 0; pa ^= 1u; }
      if (++sb == nsb) { sb = 0; pb ^= 1u; }
    }
    // every MMA this thread issued has finished before TMEM can be freed
    // (also after a timeout, when the stage barriers are no longer awaited)
    mma_commit(&mdone[mt]);
    {
      const uint64_t t0 = global_ns();
      for (uint32_t it2 = 0; it2 < kSpinLimit && !mbar_try_wait(&mdone[mt], 0); ++it2)
        if ((it2 & 255) == 255 && global_ns() - t0 > kWaitNs) break;
    }
  } else if (warp >= 10 && warp <= 13) {
    // ---------------- epilogue: TMEM -> L rows, one segment at a time ----------------
    const int quarter = warp & 3;                   // TMEM lanes this warp may read
    const int r = quarter * 32 + lane;
    for (int seg = 0; seg < nseg; ++seg) {
      if (!__all_sync(0xffffffffu, mbar_wait(accb, seg & 1, abort_flag, prm.wait_ns))) break;  // warp-collective TMEM loads follow
      tc_fence_after();
      const int unit = seg < nA ? k + seg * (int)gridDim.x : prm.nfull + k / prm.q;
      const int4 u = prm.units[unit];
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int cnt = tile_count(prm, u, h);
        if (cnt == 0) continue;                     // uniform over the warp
        const uint32_t taddr = tmem + (h ? kAcc1 : 0u) + ((uint32_t)(quarter * 32) << 16);
        float *Lrow = nullptr;
        if (r < cnt) {
          if (seg < nA) {
            int tau = 0;
            const int l = row_level(prm.d, u.y + h * kRows + r, tau);
            Lrow = prm.L + class_box_row(prm, l, u.x, tau) * prm.ld;
          } else {
            Lrow = prm.partial + (((size_t)k * 2 + h) * kRows + r) * prm.ld;
          }
        }
        for (int c0 = 0; c0 < ng * 8; c0 += 16) {
          float v[16];
          tmem_ld16(taddr + c0, v);
          if (Lrow) {
#pragma unroll
            for (int e = 0; e < 16; e += 4)
              *reinterpret_cast<float4 *>(Lrow + c0 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(tfree);
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) *(volatile int *)prm.error = 1;
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// L rows of the remainder units: the q partial tiles of each, added in slice order
__global__ void k_m2l_tc_reduce(tc::Params prm) {
  const int64_t n = (int64_t)prm.nrem * 2 * tc::kRows * prm.ld;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % prm.ld);
    const int r = (int)((e / prm.ld) % tc::kRows);
    const int h = (int)((e / ((int64_t)prm.ld * tc::kRows)) % 2);
    const int ru = (int)(e / ((int64_t)prm.ld * tc::kRows * 2));
    const int4 u = prm.units[prm.nfull + ru];
    if (r >= tc::tile_count(prm, u, h)) continue;
    float v = 0.f;
    for (int sl = 0; sl < prm.q; ++sl)
      v += prm.partial[(((size_t)(ru * prm.q + sl) * 2 + h) * tc::kRows + r) * prm.ld + c];
    int tau = 0;
    const int l = tc::row_level(prm.d, u.y + h * tc::kRows + r, tau);
    prm.L[tc::class_box_row(prm, l, u.x, tau) * prm.ld + c] = v;
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

// two accumulators of Kp columns fit below the A stages only for Kp <= 192;
// the launch-shape tuning may also choose single tiles there
static inline bool tc_paired(const mahi_ctx *h) { return h->ld <= (int)tc::kAcc1 && !h->tune_m2l_single; }

int tc_build_units(mahi_ctx *h, std::vector<int> &units) {
  if (h->ld > tc::kMaxN || h->ld % tc::kKC) return -1;
  const int step = (tc_paired(h) ? 2 : 1) * tc::kRows;
  // targets of one child class over all levels 1..d, in the merged row order
  int rows = 0;
  for (int l = 1; l <= h->d; ++l) rows += 1 << (3 * (l - 1));
  units.clear();
  for (int c = 0; c < 8; ++c)
    for (int r0 = 0; r0 < rows; r0 += step) {
      units.push_back(c);
      units.push_back(r0);
      units.push_back(std::min(tc::kRows, rows - r0));
      units.push_back(step > tc::kRows ? std::max(0, std::min(tc::kRows, rows - r0 - tc::kRows)) : 0);
    }
  h->tc_nunits = (int)units.size() / 4;
  return 0;
}

// rebuild the unit table after a change of the tile choice (the device table
// was allocated for the single-tile count, the larger one)
int tc_upload_units(mahi_ctx *h) {
  std::vector<int> units;
  if (tc_build_units(h, units) != 0) return -1;
  return cudaMemcpy(h->tc_units, units.data(), units.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess
             ? 0
             : -1;
}

// dynamic shared memory of k_m2l_tc with nsb operator stages
static size_t tc_smem_bytes(int ng, int nsb) {
  const size_t b = (size_t)(tc::kKC / 4) * ng * 128;
  const size_t stage = (size_t)2 * tc::kStagesS * tc::kSlotBytes;
  const size_t tables = sizeof(int) * (8 * kListLen + ((3 * kNumOffsets + 1) & ~1));
  return nsb * tc::kKPI * 2 * b + stage + tables + (tc::kStagesA + tc::kStagesB + tc::kDone + 6) * 8 + 16;
}

int tc_m2l(mahi_ctx *h, cudaStream_t st) {
  // rewrite the multipoles of levels 1..d for coalesced gathers
  k_m2l_src_layout<<<4 * h->num_sms, 256, 0, st>>>((const float *)h->Mexp, (float *)h->tc_msrc, h->tc_level_off,
                                                         h->ld, h->d);
  h->launches += 1;
  tc::Params prm;
  prm.M = (const float *)h->tc_msrc;
  prm.L = (float *)h->Lexp;
  prm.ops = (const unsigned char *)h->tc_ops;
  prm.units = (const int4 *)h->tc_units;
  prm.list = h->m2l_list;
  prm.off = h->m2l_off;
  prm.level_off = h->tc_level_off;
  prm.error = h->status_dev + kStatusM2LTimeout;
  prm.wait_ns = h->wait_limit_ns;
  prm.selftest = h->watchdog_selftest;
  prm.ld = h->ld;
  prm.nch = h->ld / tc::kKC;
  prm.d = h->d;
  // K chunks holding the coefficients of degrees 0..split degree
  prm.nsplit = h->m2l_split_degree < 0
                   ? 0
                   : std::min(prm.nch, (ncoef(std::min(h->m2l_split_degree, h->p)) + tc::kKC - 1) / tc::kKC);
  prm.nvc = prm.nch + prm.nsplit;
  prm.ngrp = (prm.nvc + tc::kKPI - 1) / tc::kKPI;
  prm.ngroups = h->ld / 8;
  prm.nunits = h->tc_nunits;
  prm.paired = tc_paired(h) ? 1 : 0;
  // as many operator stages as fit (4 at p <= 12, 3 at p = 15), or the tuned count
  prm.nsb = tc::kStagesB;
  while (prm.nsb > 2 && tc_smem_bytes(prm.ngroups, prm.nsb) > 227 * 1024) --prm.nsb;
  if (h->tune_m2l_nsb >= 2 && h->tune_m2l_nsb < prm.nsb) prm.nsb = h->tune_m2l_nsb;
  const size_t sm = tc_smem_bytes(prm.ngroups, prm.nsb);
  if (sm > 227 * 1024) return -1;
  if (cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return -1;
  if (h->tc_nunits == 0) return 0;
  const int G = h->num_sms;
  prm.nfull = (h->tc_nunits / G) * G;
  prm.nrem = h->tc_nunits - prm.nfull;
  prm.q = prm.nrem > 0 ? G / prm.nrem : 1;
  prm.partial = (float *)h->tc_partial;
  k_m2l_tc<<<G, tc::kThreads, sm, st>>>(prm);
  if (prm.nrem > 0) {
    k_m2l_tc_reduce<<<2 * G, 256, 0, st>>>(prm);
    h->launches += 1;
  }
  h->launches += 1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace mahi
