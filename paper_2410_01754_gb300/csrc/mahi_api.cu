// C ABI of libmahi: handle management, argument checks, device workspaces and
// the host-only lattice helpers.  All compute is in mahi_kernels.cu and
// mahi_m2l_tc.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "mahi_internal.h"

using namespace mahi;

static std::mutex g_err_mu;
static char g_cuda_err[512] = "";

namespace mahi {
int cuda_fail(cudaError_t e, const char *what) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
  return MAHI_ERR_CUDA;
}

float default_site_theta(int p) {
  // theta^(p+1) = 0.4^13: the M2P truncation bound that theta = 0.4 gives at
  // p = 12, within [0.25, 0.4] (below p = 8 the bound is not held: a smaller
  // ratio would open most of the tree)
  const double t = std::pow(0.4, 13.0 / (p + 1.0));
  return (float)std::max(0.25, std::min(0.4, t));
}

int default_m2l_split_degree(int p) { return std::min(2, p); }

int default_site_list_cap(float theta) {
  if (theta >= 0.4f) return 1536;
  // children of the boxes opened at one level: 8 x the lattice points in a
  // ball of radius (sqrt(3)/2) / theta plus 1.5 box edges (site radius, margin)
  const double r = 0.86602540378443865 / theta + 1.5;
  int cap = (int)std::ceil(8.0 * 4.0 / 3.0 * kPi * r * r * r);
  cap = (cap + 255) / 256 * 256;
  return std::max(1536, std::min(kSiteListCapMax, cap));
}

// the half-shell near field's slots (13 float4 per atom), allocated when
// that scheme is first selected
int alloc_near_slots(mahi_ctx *h) {
  if (h->nf_slots) return 0;
  return cudaMalloc(&h->nf_slots, (size_t)13 * h->N * sizeof(float4)) == cudaSuccess ? 0 : -1;
}

// traversal-list buffers of the sites for the current list capacity; keeps
// buffers that are large enough (work enqueued earlier may still read them:
// the handle's streams are synchronised before any buffer is replaced)
int alloc_site_lists(mahi_ctx *h) {
  if (h->S <= 0) return 0;
  if (h->site_lists && h->site_lists_cap >= h->site_list_cap) return 0;
  if (h->site_lists) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess || cudaStreamSynchronize(h->side) != cudaSuccess) return -1;
    cudaFree(h->site_lists); cudaFree(h->site_list_n); cudaFree(h->site_cen);
    h->site_lists = nullptr; h->site_list_n = nullptr; h->site_cen = nullptr; h->site_lists_cap = 0;
  }
  const size_t nl = (size_t)h->S * (h->d + 1) * h->site_list_cap;
  if (cudaMalloc(&h->site_lists, nl * sizeof(int)) != cudaSuccess) return -1;
  if (cudaMalloc(&h->site_list_n, (size_t)h->S * (h->d + 2) * sizeof(int)) != cudaSuccess) return -1;
  if (cudaMalloc(&h->site_cen, (size_t)h->S * 4 * sizeof(double)) != cudaSuccess) return -1;
  h->site_lists_cap = h->site_list_cap;
  return 0;
}
}  // namespace mahi

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

template <typename P>
static cudaError_t dalloc(P **p, size_t bytes) {
  void *v = nullptr;
  cudaError_t e = cudaMalloc(&v, std::max<size_t>(bytes, 16));
  *p = (P *)v;
  return e;
}

static void free_all(mahi_ctx *h) {
  void *bufs[] = {h->qA, h->dq, h->site_of, h->qt, h->leaf_of, h->slot, h->leaf_count, h->leaf_start, h->perm,
                  h->perm_tmp, h->inv_perm, h->part, h->part_tmp, h->Mexp, h->Lexp, h->phi_s, h->grad_s,
                  h->ops_m2m, h->ops_l2l, h->ops_m2l, h->gemm_ws, h->ops_lat, h->eta, h->eta_x, h->eta_y, h->eta_z,
                  h->m2l_list, h->m2l_off, h->site_ptr, h->site_atoms,
                  h->energy_part, h->site_energy, h->tc_ops, h->tc_partial, h->tc_msrc, h->tc_level_off, h->tc_units, h->d_x_stage,
                  h->d_lam_stage, h->d_E_stage, h->d_dEdl_stage, h->d_F_stage, h->ops_lat_h3, h->L_h3,
                  h->box_qd, h->box_qdf, h->vtmp, h->relD, h->phi_site, h->psi_site, h->site_pairs, h->site_slot, h->mf_q, h->mf_lam_off, h->phi_part, h->d_level_off, h->mf_psi, h->mf_form_off, h->nf_slots, h->site_lists, h->site_list_n, h->site_cen, h->site_pair_list, h->site_order};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (h->status_host) cudaFreeHost(h->status_host);
  for (int i = 0; i < 32; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  for (int i = 0; i < 3; ++i)
    if (h->fork_ev[i]) cudaEventDestroy(h->fork_ev[i]);
  for (int i = 0; i < 2; ++i)
    if (h->join_ev[i]) cudaEventDestroy(h->join_ev[i]);
  if (h->side) cudaStreamDestroy(h->side);
  for (int i = 0; i < 2; ++i)
    if (h->hp_ev[i]) cudaEventDestroy(h->hp_ev[i]);
  if (h->hp) cudaStreamDestroy(h->hp);
}

// SIMT operator layout: transposed and zero padded, opT[term][k][n], k, n < ld.
template <typename T>
static cudaError_t upload_ops_t(const std::vector<std::vector<double>> &ops, int K, int ld, void **dst) {
  std::vector<T> tmp(ops.size() * (size_t)ld * ld, T(0));
  for (size_t t = 0; t < ops.size(); ++t)
    for (int n = 0; n < K; ++n)
      for (int k = 0; k < K; ++k) tmp[t * (size_t)ld * ld + (size_t)k * ld + n] = (T)ops[t][(size_t)n * K + k];
  cudaError_t e = dalloc(dst, tmp.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// L2L operators side by side for the dense GEMM: wide[k][c * ld + n] = T'_c[n][k]
template <typename T>
static cudaError_t upload_ops_wide(const std::vector<std::vector<double>> &ops, int K, int ld, void **dst) {
  const size_t W = ops.size() * (size_t)ld;
  std::vector<T> tmp((size_t)ld * W, T(0));
  for (size_t t = 0; t < ops.size(); ++t)
    for (int n = 0; n < K; ++n)
      for (int k = 0; k < K; ++k) tmp[(size_t)k * W + t * ld + n] = (T)ops[t][(size_t)n * K + k];
  cudaError_t e = dalloc(dst, tmp.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename T>
static cudaError_t upload_ops(const std::vector<std::vector<double>> &ops, void **dst) {
  size_t n = 0;
  for (auto &o : ops) n += o.size();
  std::vector<T> tmp(n);
  size_t k = 0;
  for (auto &o : ops)
    for (double v : o) tmp[k++] = (T)v;
  cudaError_t e = dalloc(dst, n * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, tmp.data(), n * sizeof(T), cudaMemcpyHostToDevice);
}

// true for device (or managed) memory, false for host memory (pinned or pageable)
static bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// host view of an array that may live on the device (copied when it does)
template <typename T>
static int host_view(const T *p, int64_t n, std::vector<T> &buf, const T **out) {
  if (!is_device_ptr(p)) {
    *out = p;
    return MAHI_OK;
  }
  buf.resize((size_t)n);
  CK(cudaMemcpy(buf.data(), p, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost));
  *out = buf.data();
  return MAHI_OK;
}

extern "C" {

double mahi_coulomb_constant(void) { return coulomb_constant(); }

const char *mahi_error_string(int code) {
  switch (code) {
    case MAHI_OK: return "ok";
    case MAHI_ERR_INVALID_ARG: return "invalid argument";
    case MAHI_ERR_BAD_SITE_MAP: return "bad site map (index out of range, empty site, site too large, or qA != qB on an environment atom)";
    case MAHI_ERR_NON_CUBIC: return "non-cubic box (unsupported)";
    case MAHI_ERR_CUDA: return "CUDA error (see mahi_last_cuda_error)";
    case MAHI_ERR_TIMEOUT: return "a bounded device wait gave up";
    case MAHI_ERR_NO_DEVICE: return "no usable sm_103 (GB300) CUDA device";
    case MAHI_ERR_STATE: return "charges not set";
    case MAHI_ERR_SITE_OVERFLOW: return "a site's traversal lists outgrew their capacity (raise MAHI_OPT_SITE_LIST_CAP)";
    default: return "unknown error";
  }
}

const char *mahi_last_cuda_error(void) { return g_cuda_err; }

const char *mahi_stage_name(int32_t i) { return stage_name(i); }

int mahi_create(double box_L_nm, int64_t n_atoms, int32_t n_sites, int32_t order_p, int32_t depth, int32_t precision,
                void *cuda_stream, mahi_t *out) {
  if (!out) return MAHI_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(box_L_nm > 0.0) || !std::isfinite(box_L_nm) || n_atoms < 1 || n_atoms > (int64_t)1 << 30 || n_sites < 0 ||
      depth < 0 || depth > kMaxDepth || order_p < 1)
    return MAHI_ERR_INVALID_ARG;
  if (precision != MAHI_FP64 && precision != MAHI_MIXED && precision != MAHI_MIXED_SIMT) return MAHI_ERR_INVALID_ARG;
  if (order_p > (precision == MAHI_FP64 ? kMaxOrder : kMaxOrderMixed)) return MAHI_ERR_INVALID_ARG;
  if (precision == MAHI_MIXED && nstride(order_p) > 256) return MAHI_ERR_INVALID_ARG;  // MMA N <= 256
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return MAHI_ERR_NO_DEVICE;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return MAHI_ERR_NO_DEVICE;
  if (prop.major * 10 + prop.minor != 103) return MAHI_ERR_NO_DEVICE;

  if (upload_tables() != 0) return cuda_fail(cudaGetLastError(), "constant tables");
  mahi_ctx *h = new (std::nothrow) mahi_ctx();
  if (!h) return MAHI_ERR_INVALID_ARG;
  h->L = box_L_nm; h->N = n_atoms; h->S = n_sites; h->p = order_p; h->d = depth; h->prec = precision;
  h->stream = (cudaStream_t)cuda_stream;
  h->device = dev;
  h->num_sms = prop.multiProcessorCount;
  h->K = ncoef(order_p);
  h->ld = nstride(order_p);
  h->nleaf = 1 << (3 * depth);
  int64_t off = 0;
  for (int l = 0; l <= depth; ++l) { h->level_off[l] = off; off += (int64_t)1 << (3 * l); }
  h->level_off[depth + 1] = off;
  h->nbox_total = off;
  const bool f64 = (precision == MAHI_FP64);
  const size_t ts = f64 ? sizeof(double) : sizeof(float);
  const size_t v4 = 4 * ts;
  const int64_t N = n_atoms;
  int rc = MAHI_OK;
  auto fail = [&](cudaError_t e, const char *w) {
    rc = cuda_fail(e, w);
    free_all(h);
    delete h;
    return rc;
  };
#define AL(ptr, bytes)                                  \
  do {                                                  \
    cudaError_t e_ = dalloc(&(ptr), (bytes));           \
    if (e_ != cudaSuccess) return fail(e_, #ptr);       \
  } while (0)
  AL(h->qA, N * 8); AL(h->dq, N * 8); AL(h->site_of, N * 4); AL(h->qt, N * 8);
  AL(h->leaf_of, N * 4); AL(h->slot, N * 4);
  AL(h->leaf_count, (size_t)h->nleaf * 4); AL(h->leaf_start, (size_t)(h->nleaf + 1) * 4);
  AL(h->perm, N * 4); AL(h->perm_tmp, N * 4); AL(h->inv_perm, N * 4);
  AL(h->part, N * v4); AL(h->part_tmp, N * v4); AL(h->vtmp, N * v4); AL(h->relD, N * 3 * 8);
  AL(h->Mexp, (size_t)h->nbox_total * h->ld * ts); AL(h->Lexp, (size_t)h->nbox_total * h->ld * ts);
  AL(h->phi_s, N * ts); AL(h->grad_s, N * 3 * ts);
  h->n_moment_blocks = (int)std::min<int64_t>(4 * 152, (N + 255) / 256);
  h->gemm_ws_elems = gemm_workspace_elems(h->d, h->ld, h->num_sms);
  if (h->gemm_ws_elems) AL(h->gemm_ws, h->gemm_ws_elems * ts);
  // leaf energy partials, then the final sum's block sums and its ticket
  AL(h->energy_part, ((size_t)h->nleaf + kFinalBlocks + 1) * 8);
  AL(h->site_energy, (size_t)std::max(1, n_sites) * 8);
  {
    cudaError_t e0 = cudaMemset(h->energy_part + h->nleaf + kFinalBlocks, 0, 8);
    if (e0 != cudaSuccess) return fail(e0, "memset");
  }
  {
    cudaError_t e = cudaMemset(h->Lexp, 0, (size_t)h->nbox_total * h->ld * ts);
    if (e != cudaSuccess) return fail(e, "memset");
    e = cudaMemset(h->Mexp, 0, (size_t)h->nbox_total * h->ld * ts);
    if (e != cudaSuccess) return fail(e, "memset");
  }

  // translation operators (host, FP64) -> device in the working precision
  const int K = h->K;
  std::vector<std::vector<double>> m2m(8), l2l(8), m2l(kNumOffsets), lat(1), lat3(1);
  for (int c = 0; c < 8; ++c) {
    build_m2m(order_p, c, m2m[c]);
    scale_operator(order_p, 0, m2m[c]);
    build_l2l(order_p, c, l2l[c]);
    scale_operator(order_p, 1, l2l[c]);
  }
  const OffsetTables &ot = offset_tables();
  for (int o = 0; o < kNumOffsets; ++o) {
    build_m2l(order_p, ot.off[o][0], ot.off[o][1], ot.off[o][2], m2l[o]);
    scale_operator(order_p, 2, m2l[o]);
  }
  build_lattice_op(order_p, lat[0]);
  scale_operator(order_p, 2, lat[0]);
  build_lattice_op(order_p, lat3[0], false);
  scale_operator(order_p, 2, lat3[0]);
  {
    cudaError_t e;
    const int ldp = h->ld;
    if (f64) {
      if ((e = upload_ops_t<double>(m2m, K, ldp, &h->ops_m2m)) != cudaSuccess) return fail(e, "ops");
      if ((e = upload_ops_wide<double>(l2l, K, ldp, &h->ops_l2l)) != cudaSuccess) return fail(e, "ops");
      if ((e = upload_ops_t<double>(m2l, K, ldp, &h->ops_m2l)) != cudaSuccess) return fail(e, "ops");
    } else {
      if ((e = upload_ops_t<float>(m2m, K, ldp, &h->ops_m2m)) != cudaSuccess) return fail(e, "ops");
      if ((e = upload_ops_wide<float>(l2l, K, ldp, &h->ops_l2l)) != cudaSuccess) return fail(e, "ops");
      if (precision != MAHI_MIXED)
        if ((e = upload_ops_t<float>(m2l, K, ldp, &h->ops_m2l)) != cudaSuccess) return fail(e, "ops");
    }
    void *tmp = nullptr;
    if ((e = upload_ops<double>(lat, &tmp)) != cudaSuccess) return fail(e, "ops");
    h->ops_lat = (double *)tmp;
    if ((e = upload_ops<double>(lat3, &tmp)) != cudaSuccess) return fail(e, "ops");
    h->ops_lat_h3 = (double *)tmp;
    AL(h->L_h3, sizeof(double) * K);
    // status word: host-mapped, so that a failure recorded by a kernel can be
    // read without a synchronisation
    {
      void *hp = nullptr, *dp = nullptr;
      if ((e = cudaHostAlloc(&hp, sizeof(int) * kStatusWords, cudaHostAllocMapped)) != cudaSuccess)
        return fail(e, "status word");
      h->status_host = (int *)hp;
      std::memset(hp, 0, sizeof(int) * kStatusWords);
      if ((e = cudaHostGetDevicePointer(&dp, hp, 0)) != cudaSuccess) return fail(e, "status word");
      h->status_dev = (int *)dp;
    }
    h->site_theta = default_site_theta(order_p);
    h->m2l_split_degree = default_m2l_split_degree(order_p);
    h->site_list_cap = default_site_list_cap(h->site_theta);
    AL(h->box_qd, sizeof(double) * 8 * h->nbox_total);
    AL(h->box_qdf, sizeof(float) * 8 * h->nbox_total);
    AL(h->d_level_off, sizeof(int64_t) * (kMaxDepth + 2));
    if ((e = cudaMemcpy(h->d_level_off, h->level_off, sizeof(int64_t) * (kMaxDepth + 2), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return fail(e, "level offsets");
    // first-shell lattice function H_1 for the per-site pair kernel, and its
    // gradient coefficients
    const int P = kSiteDegree;
    const std::vector<double> &eta = lattice_coeffs(P, 1);
    // A_ii = lim_{r->0} A(r) - 1/r: the 26 first-shell images plus H_1(0) (the
    // r^2 term vanishes); H_1(0) is the degree-0 coefficient
    h->site_aii = (6.0 + 12.0 / std::sqrt(2.0) + 8.0 / std::sqrt(3.0) + eta[0]) / box_L_nm;
    std::vector<double> ex((size_t)(P + 1) * (P + 1), 0.0), ey(ex), ez(ex);
    gradient_coeffs(P, eta.data(), ex.data(), ey.data(), ez.data());
    std::vector<std::vector<double>> v1{eta}, v2{ex}, v3{ey}, v4v{ez};
    if ((e = upload_ops<double>(v1, &tmp)) != cudaSuccess) return fail(e, "eta");
    h->eta = (double *)tmp;
    if ((e = upload_ops<double>(v2, &tmp)) != cudaSuccess) return fail(e, "eta");
    h->eta_x = (double *)tmp;
    if ((e = upload_ops<double>(v3, &tmp)) != cudaSuccess) return fail(e, "eta");
    h->eta_y = (double *)tmp;
    if ((e = upload_ops<double>(v4v, &tmp)) != cudaSuccess) return fail(e, "eta");
    h->eta_z = (double *)tmp;
    AL(h->m2l_list, sizeof(int) * 8 * kListLen);
    AL(h->m2l_off, sizeof(int) * kNumOffsets * 3);
    if ((e = cudaMemcpy(h->m2l_list, ot.list, sizeof(int) * 8 * kListLen, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(e, "list");
    if ((e = cudaMemcpy(h->m2l_off, ot.off, sizeof(int) * kNumOffsets * 3, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(e, "list");
    if (precision == MAHI_MIXED && depth >= 1) {
      std::vector<unsigned char> img(tc_ops_bytes(order_p));
      tc_pack_ops(order_p, m2l, img.data());
      AL(h->tc_ops, img.size());
      if ((e = cudaMemcpy(h->tc_ops, img.data(), img.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "tc ops");
      std::vector<int> units;
      // allocate the unit table for single tiles (the larger count), fill it for the default
      h->tune_m2l_single = true;
      int r = tc_build_units(h, units);
      h->tune_m2l_single = false;
      if (r != 0) { free_all(h); delete h; return MAHI_ERR_INVALID_ARG; }
      AL(h->tc_units, units.size() * sizeof(int));
      r = tc_build_units(h, units);
      if (r != 0) { free_all(h); delete h; return MAHI_ERR_INVALID_ARG; }
      if ((e = cudaMemcpy(h->tc_units, units.data(), units.size() * sizeof(int), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
        return fail(e, "tc units");
      AL(h->tc_partial, (size_t)h->num_sms * 2 * 128 * h->ld * sizeof(float));  // remainder-unit partial tiles
      AL(h->tc_msrc, (size_t)h->nbox_total * h->ld * sizeof(float));            // M2L source layout
      AL(h->tc_level_off, sizeof(int64_t) * (kMaxDepth + 2));
      if ((e = cudaMemcpy(h->tc_level_off, h->level_off, sizeof(int64_t) * (kMaxDepth + 2), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
        return fail(e, "tc level offsets");
    }
  }
  for (int i = 0; i < 32; ++i) {
    cudaError_t e = cudaEventCreate(&h->ev[i]);
    if (e != cudaSuccess) return fail(e, "event");
  }
  {
    cudaError_t e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&h->fork_ev[i], cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&h->join_ev[i], cudaEventDisableTiming);
    int prio_lo = 0, prio_hi = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->hp, cudaStreamNonBlocking, prio_hi);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&h->hp_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(e, "side stream");
  }
#undef AL
  (void)K;
  *out = h;
  return MAHI_OK;
}

int mahi_destroy(mahi_t h) {
  if (!h) return MAHI_OK;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
  return MAHI_OK;
}

int mahi_set_stream(mahi_t h, void *cuda_stream) {
  if (!h) return MAHI_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)cuda_stream;
  return MAHI_OK;
}

int mahi_set_charges(mahi_t h, const double *qA_in, const double *qB_in, const int32_t *site_in) {
  if (!h || !qA_in || !qB_in || !site_in) return MAHI_ERR_INVALID_ARG;
  const int64_t N = h->N;
  const int S = h->S;
  CK(cudaSetDevice(h->device));
  std::vector<double> bufA, bufB;
  std::vector<int32_t> bufS;
  const double *qA = nullptr, *qB = nullptr;
  const int32_t *site_of_atom = nullptr;
  int rc0 = host_view(qA_in, N, bufA, &qA);
  if (rc0 == MAHI_OK) rc0 = host_view(qB_in, N, bufB, &qB);
  if (rc0 == MAHI_OK) rc0 = host_view(site_in, N, bufS, &site_of_atom);
  if (rc0 != MAHI_OK) return rc0;
  std::vector<int> cnt(S, 0);
  std::vector<double> dq(N);
  for (int64_t i = 0; i < N; ++i) {
    int s = site_of_atom[i];
    if (!std::isfinite(qA[i]) || !std::isfinite(qB[i])) return MAHI_ERR_INVALID_ARG;
    if (s < -1 || s >= S) return MAHI_ERR_BAD_SITE_MAP;
    if (s == -1) {
      if (qA[i] != qB[i]) return MAHI_ERR_BAD_SITE_MAP;
      dq[i] = 0.0;
    } else {
      cnt[s]++;
      dq[i] = qB[i] - qA[i];
    }
  }
  for (int s = 0; s < S; ++s)
    if (cnt[s] == 0 || cnt[s] > 64) return MAHI_ERR_BAD_SITE_MAP;
  std::vector<int> ptr(S + 1, 0), atoms;
  for (int s = 0; s < S; ++s) ptr[s + 1] = ptr[s] + cnt[s];
  atoms.resize(ptr[S]);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (int64_t i = 0; i < N; ++i)
    if (site_of_atom[i] >= 0) atoms[fill[site_of_atom[i]]++] = (int)i;
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(h->qA, qA, N * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->dq, dq.data(), N * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->site_of, site_of_atom, N * 4, cudaMemcpyHostToDevice));
  if (h->site_ptr) { cudaFree(h->site_ptr); h->site_ptr = nullptr; }
  if (h->site_atoms) { cudaFree(h->site_atoms); h->site_atoms = nullptr; }
  if (h->phi_site) { cudaFree(h->phi_site); h->phi_site = nullptr; }
  if (h->psi_site) { cudaFree(h->psi_site); h->psi_site = nullptr; }
  if (h->site_pairs) { cudaFree(h->site_pairs); h->site_pairs = nullptr; }
  if (h->site_pair_list) { cudaFree(h->site_pair_list); h->site_pair_list = nullptr; }
  if (h->site_order) { cudaFree(h->site_order); h->site_order = nullptr; }
  if (h->phi_part) { cudaFree(h->phi_part); h->phi_part = nullptr; }
  CK(dalloc(&h->phi_site, std::max<size_t>(1, atoms.size()) * sizeof(double)));
  CK(dalloc(&h->psi_site, std::max<size_t>(1, atoms.size()) * sizeof(double)));
  CK(dalloc(&h->site_pairs, std::max<size_t>(1, (size_t)S * kSiteSymPairs * 4) * sizeof(double)));
  {
    // unordered pairs of every site of up to kSiteSymMax atoms, in k_site's pair order
    std::vector<int4> pl;
    for (int s = 0; s < S; ++s) {
      const int n = ptr[s + 1] - ptr[s];
      if (n > kSiteSymMax) continue;
      int p = 0;
      for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) pl.push_back(make_int4(s, i, j, p++));
    }
    h->n_site_pairs = (int)pl.size();
    std::vector<int> order(S);
    for (int s2 = 0; s2 < S; ++s2) order[s2] = s2;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return ptr[a + 1] - ptr[a] > ptr[b + 1] - ptr[b]; });
    CK(dalloc(&h->site_order, std::max<size_t>(1, (size_t)S) * sizeof(int)));
    if (S > 0) CK(cudaMemcpy(h->site_order, order.data(), (size_t)S * sizeof(int), cudaMemcpyHostToDevice));
    CK(dalloc(&h->site_pair_list, std::max<size_t>(1, pl.size()) * sizeof(int4)));
    if (!pl.empty()) CK(cudaMemcpy(h->site_pair_list, pl.data(), pl.size() * sizeof(int4), cudaMemcpyHostToDevice));
  }
  {
    std::vector<int> slot(N, -1);
    for (size_t k = 0; k < atoms.size(); ++k) slot[atoms[k]] = (int)k;
    if (!h->site_slot) CK(dalloc(&h->site_slot, N * sizeof(int)));
    CK(cudaMemcpy(h->site_slot, slot.data(), N * sizeof(int), cudaMemcpyHostToDevice));
  }
  CK(dalloc(&h->phi_part, std::max<size_t>(1, atoms.size()) * kSiteChunksMax * sizeof(double)));
  CK(dalloc(&h->site_ptr, (S + 1) * sizeof(int)));
  CK(dalloc(&h->site_atoms, std::max<size_t>(1, atoms.size()) * sizeof(int)));
  CK(cudaMemcpy(h->site_ptr, ptr.data(), (S + 1) * sizeof(int), cudaMemcpyHostToDevice));
  if (!atoms.empty()) CK(cudaMemcpy(h->site_atoms, atoms.data(), atoms.size() * sizeof(int), cudaMemcpyHostToDevice));
  h->n_site_atoms = (int)atoms.size();
  if (alloc_site_lists(h) != 0) return cuda_fail(cudaGetLastError(), "site lists");
  h->charges_set = true;
  h->multiform = false;  // mahi_set_forms sets it after calling this
  return MAHI_OK;
}

int mahi_set_forms(mahi_t h, const double *q_env, const int32_t *site_of_atom, const int32_t *forms_per_site,
                   const double *q_forms) {
  if (!h || !q_env || !site_of_atom || (h->S > 0 && (!forms_per_site || !q_forms))) return MAHI_ERR_INVALID_ARG;
  const int64_t N = h->N;
  const int S = h->S;
  std::vector<int> cnt(S, 0), lam_off(S + 1, 0);
  for (int sidx = 0; sidx < S; ++sidx) {
    const int F = forms_per_site[sidx];
    int m = 0;
    while ((1 << m) < F) ++m;
    if (F < 2 || F > 16 || (1 << m) != F) return MAHI_ERR_INVALID_ARG;
    lam_off[sidx + 1] = lam_off[sidx] + m;
  }
  for (int64_t i = 0; i < N; ++i) {
    const int sidx = site_of_atom[i];
    if (!std::isfinite(q_env[i])) return MAHI_ERR_INVALID_ARG;
    if (sidx < -1 || sidx >= S) return MAHI_ERR_BAD_SITE_MAP;
    if (sidx >= 0) cnt[sidx]++;
  }
  for (int sidx = 0; sidx < S; ++sidx)
    if (cnt[sidx] == 0 || cnt[sidx] > 32) return MAHI_ERR_BAD_SITE_MAP;
  // the two-form layout with dq = 0: the evaluation rescales site charges itself
  std::vector<double> qB(q_env, q_env + N);
  int rc = mahi_set_charges(h, q_env, qB.data(), site_of_atom);
  if (rc != MAHI_OK) return rc;
  // per site atom (in site_atoms order) its charges in every form, padded to 16
  std::vector<int> ptr(S + 1, 0);
  for (int sidx = 0; sidx < S; ++sidx) ptr[sidx + 1] = ptr[sidx] + cnt[sidx];
  std::vector<double> qf((size_t)std::max(1, ptr[S]) * 16, 0.0);
  size_t off = 0;
  for (int sidx = 0; sidx < S; ++sidx) {
    const int F = forms_per_site[sidx], n = cnt[sidx];
    for (int r = 0; r < F; ++r)
      for (int a = 0; a < n; ++a) {
        const double v = q_forms[off + (size_t)r * n + a];
        if (!std::isfinite(v)) return MAHI_ERR_INVALID_ARG;
        qf[(size_t)(ptr[sidx] + a) * 16 + r] = v;
      }
    off += (size_t)F * n;
  }
  if (h->mf_q) { cudaFree(h->mf_q); h->mf_q = nullptr; }
  if (h->mf_psi) { cudaFree(h->mf_psi); h->mf_psi = nullptr; }
  if (!h->mf_lam_off) CK(dalloc(&h->mf_lam_off, (S + 1) * sizeof(int)));
  if (!h->mf_form_off) CK(dalloc(&h->mf_form_off, (S + 1) * sizeof(int)));
  CK(dalloc(&h->mf_q, qf.size() * sizeof(double)));
  CK(dalloc(&h->mf_psi, qf.size() * sizeof(double)));
  CK(cudaMemcpy(h->mf_q, qf.data(), qf.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->mf_lam_off, lam_off.data(), (S + 1) * sizeof(int), cudaMemcpyHostToDevice));
  {
    std::vector<int> foff(S + 1, 0);
    for (int sidx = 0; sidx < S; ++sidx) foff[sidx + 1] = foff[sidx] + forms_per_site[sidx] * cnt[sidx];
    CK(cudaMemcpy(h->mf_form_off, foff.data(), (S + 1) * sizeof(int), cudaMemcpyHostToDevice));
    h->n_form_charges = foff[S];
  }
  h->n_lam = lam_off[S];
  h->multiform = true;
  return MAHI_OK;
}

int mahi_n_lambdas(mahi_t h) { return h ? (h->multiform ? h->n_lam : h->S) : MAHI_ERR_INVALID_ARG; }

// Reads and clears the status word (no synchronisation: only what the device
// has written so far is seen).
static int take_status(mahi_t h) {
  volatile int *st = h->status_host;
  int rc = MAHI_OK;
  if (st[kStatusM2LTimeout] || st[kStatusSiteTimeout]) rc = MAHI_ERR_TIMEOUT;
  else if (st[kStatusSiteOverflow]) rc = MAHI_ERR_SITE_OVERFLOW;
  if (rc != MAHI_OK)
    for (int i = 0; i < kStatusWords; ++i) st[i] = 0;
  return rc;
}

int mahi_get_status(mahi_t h) {
  if (!h) return MAHI_ERR_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->stream));
  return take_status(h);
}

int mahi_eval(mahi_t h, const void *x, int32_t x_is_fp64, const double *lambda, double *energy, void *forces,
              double *dEdlambda) {
  if (!h || !x || (h->S > 0 && !lambda)) return MAHI_ERR_INVALID_ARG;
  if (!h->charges_set) return MAHI_ERR_STATE;
  // a failure of an earlier evaluation that the device has reported by now
  {
    const int st = take_status(h);
    if (st != MAHI_OK) return st;
  }
  CK(cudaSetDevice(h->device));
  int r = enqueue_eval(h, x, x_is_fp64 ? 1 : 0, lambda, energy, forces, dEdlambda);
  if (r != 0) return cuda_fail((cudaError_t)r, "mahi_eval");
  return MAHI_OK;
}

int mahi_update_charges(mahi_t h, const double *qA, const double *qB) {
  if (!h || !qA || !qB) return MAHI_ERR_INVALID_ARG;
  if (!h->charges_set) return MAHI_ERR_STATE;
  if (h->multiform) return MAHI_ERR_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  if (enqueue_update_charges(h, qA, qB) != 0) return cuda_fail(cudaGetLastError(), "mahi_update_charges");
  return MAHI_OK;
}

int mahi_set_option(mahi_t h, int32_t option, double value) {
  if (!h || !std::isfinite(value)) return MAHI_ERR_INVALID_ARG;
  switch (option) {
    case MAHI_OPT_SITE_THETA:
      if (value < 0.0 || value > 0.7) return MAHI_ERR_INVALID_ARG;
      h->site_theta_set = value > 0.0;
      h->site_theta = h->site_theta_set ? (float)value : default_site_theta(h->p);
      if (!h->site_list_cap_set) h->site_list_cap = default_site_list_cap(h->site_theta);
      if (h->charges_set && alloc_site_lists(h) != 0) return cuda_fail(cudaGetLastError(), "site lists");
      return MAHI_OK;
    case MAHI_OPT_SITE_LIST_CAP:
      if (value != 0.0 && (value < 64 || value > kSiteListCapMax || value != std::floor(value)))
        return MAHI_ERR_INVALID_ARG;
      h->site_list_cap_set = value > 0.0;
      h->site_list_cap = h->site_list_cap_set ? (int)value : default_site_list_cap(h->site_theta);
      if (h->charges_set && alloc_site_lists(h) != 0) return cuda_fail(cudaGetLastError(), "site lists");
      return MAHI_OK;
    case MAHI_OPT_WAIT_LIMIT_MS:
      if (value < 0.0 || (value > 0.0 && value < 1.0) || value > 60000.0) return MAHI_ERR_INVALID_ARG;
      h->wait_limit_ns = value > 0.0 ? (uint64_t)(value * 1e6) : 2000000000ull;
      return MAHI_OK;
    case MAHI_OPT_WATCHDOG_SELFTEST:
      if (value != 0.0 && value != 1.0) return MAHI_ERR_INVALID_ARG;
      h->watchdog_selftest = (int)value;
      return MAHI_OK;
    case MAHI_OPT_M2L_SPLIT_DEGREE:
      if (value != std::floor(value) || value < -1.0 || value > h->p) return MAHI_ERR_INVALID_ARG;
      h->m2l_split_degree = (int)value;
      return MAHI_OK;
    case MAHI_OPT_M2L_SINGLE_TILE: {
      if (value != 0.0 && value != 1.0) return MAHI_ERR_INVALID_ARG;
      const bool single = value != 0.0;
      if (single == h->tune_m2l_single) return MAHI_OK;
      h->tune_m2l_single = single;
      if (h->tc_units) {
        CK(cudaSetDevice(h->device));
        CK(cudaStreamSynchronize(h->stream));   // the table may be in use by enqueued work
        if (tc_upload_units(h) != 0) return cuda_fail(cudaGetLastError(), "M2L units");
      }
      return MAHI_OK;
    }
    case MAHI_OPT_M2L_B_STAGES:
      if (value != 0.0 && value != 2.0 && value != 3.0 && value != 4.0) return MAHI_ERR_INVALID_ARG;
      h->tune_m2l_nsb = (int)value;
      return MAHI_OK;
    case MAHI_OPT_P2P_THREADS:
      if (value != 0.0 && value != 64.0 && value != 128.0 && value != 256.0) return MAHI_ERR_INVALID_ARG;
      h->tune_p2p_threads = value == 0.0 ? 128 : (int)value;
      return MAHI_OK;
    case MAHI_OPT_SITE_BLOCKS:
      if (value < 0.0 || value > kSiteChunksMax || value != std::floor(value)) return MAHI_ERR_INVALID_ARG;
      h->tune_site_blocks = (int)value;
      return MAHI_OK;
    case MAHI_OPT_P2P_TARGETS:
      if (value != 0.0 && value != -1.0 && value != 4.0 && value != 8.0) return MAHI_ERR_INVALID_ARG;
      h->tune_p2p_targets = value == 0.0 ? -1 : (int)value;
      if (h->tune_p2p_targets > 0 && h->prec != MAHI_FP64 && alloc_near_slots(h) != 0)
        return cuda_fail(cudaGetLastError(), "near-field slots");
      return MAHI_OK;
    default: return MAHI_ERR_INVALID_ARG;
  }
}

double mahi_get_option(mahi_t h, int32_t option) {
  if (!h) return -1.0;
  switch (option) {
    case MAHI_OPT_SITE_THETA: return h->site_theta;
    case MAHI_OPT_SITE_LIST_CAP: return h->site_list_cap;
    case MAHI_OPT_WAIT_LIMIT_MS: return (double)h->wait_limit_ns * 1e-6;
    case MAHI_OPT_WATCHDOG_SELFTEST: return h->watchdog_selftest;
    case MAHI_OPT_M2L_SPLIT_DEGREE: return h->m2l_split_degree;
    case MAHI_OPT_M2L_SINGLE_TILE: return h->tune_m2l_single ? 1.0 : 0.0;
    case MAHI_OPT_M2L_B_STAGES: return h->tune_m2l_nsb;
    case MAHI_OPT_P2P_THREADS: return h->tune_p2p_threads;
    case MAHI_OPT_SITE_BLOCKS: return h->tune_site_blocks;
    case MAHI_OPT_P2P_TARGETS: return h->tune_p2p_targets;
    default: return -1.0;
  }
}

int mahi_backward_forms(mahi_t h, const double *grad_energy, const void *forces, const double *dEdlambda,
                        const double *lambda, int32_t x_is_fp64, void *dx, double *dlambda, double *dEdq_env,
                        double *dEdq_forms) {
  if (!h || !grad_energy) return MAHI_ERR_INVALID_ARG;
  if (!h->charges_set) return MAHI_ERR_STATE;
  if (!h->multiform) return MAHI_ERR_INVALID_ARG;  // sites with 2^m forms only
  if (dx && !forces) return MAHI_ERR_INVALID_ARG;
  if (dlambda && h->n_lam > 0 && !dEdlambda) return MAHI_ERR_INVALID_ARG;
  if (dEdq_forms && h->S > 0 && !lambda) return MAHI_ERR_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  if (enqueue_backward_forms(h, grad_energy, forces, dEdlambda, lambda, x_is_fp64 ? 1 : 0, dx, dlambda, dEdq_env,
                             dEdq_forms) != 0)
    return cuda_fail(cudaGetLastError(), "mahi_backward_forms");
  h->launches = (dx || dlambda ? 1 : 0) + (dEdq_env || dEdq_forms ? 1 : 0);
  return MAHI_OK;
}

int mahi_backward(mahi_t h, const double *grad_energy, const void *forces, const double *dEdlambda,
                  const double *lambda, int32_t x_is_fp64, void *dx, double *dlambda, double *dEdqA, double *dEdqB) {
  if (!h || !grad_energy) return MAHI_ERR_INVALID_ARG;
  if (!h->charges_set) return MAHI_ERR_STATE;
  if (h->multiform) return MAHI_ERR_INVALID_ARG;  // two-form sites only
  if (dx && !forces) return MAHI_ERR_INVALID_ARG;
  if (dlambda && h->S > 0 && !dEdlambda) return MAHI_ERR_INVALID_ARG;
  if ((dEdqA || dEdqB) && h->S > 0 && !lambda) return MAHI_ERR_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  if (enqueue_backward(h, grad_energy, forces, dEdlambda, lambda, x_is_fp64 ? 1 : 0, dx, dlambda, dEdqA, dEdqB) != 0)
    return cuda_fail(cudaGetLastError(), "mahi_backward");
  h->launches = 1;
  return MAHI_OK;
}

int mahi_eval_host(mahi_t h, const void *x_host, int32_t x_is_fp64, const double *lambda_host, double *energy_host,
                   void *forces_host, double *dEdlambda_host) {
  if (!h || !x_host || (h->S > 0 && !lambda_host)) return MAHI_ERR_INVALID_ARG;
  if (!h->charges_set) return MAHI_ERR_STATE;
  {
    const int st0 = take_status(h);
    if (st0 != MAHI_OK) return st0;
  }
  const size_t xs = x_is_fp64 ? 8 : 4;
  const size_t xb = (size_t)h->N * 3 * xs;
  if (h->x_stage_fp64 != (x_is_fp64 ? 1 : 0)) {
    if (h->d_x_stage) cudaFree(h->d_x_stage);
    if (h->d_F_stage) cudaFree(h->d_F_stage);
    h->d_x_stage = h->d_F_stage = nullptr;
    CK(dalloc(&h->d_x_stage, xb));
    CK(dalloc(&h->d_F_stage, xb));
    h->x_stage_fp64 = x_is_fp64 ? 1 : 0;
  }
  if (!h->d_lam_stage) {
    CK(dalloc(&h->d_lam_stage, std::max(1, 4 * h->S) * 8));  // up to 4 lambdas per site (16 forms)
    CK(dalloc(&h->d_E_stage, 8));
    CK(dalloc(&h->d_dEdl_stage, std::max(1, 4 * h->S) * 8));
  }
  cudaStream_t st = h->stream;
  CK(cudaMemcpyAsync(h->d_x_stage, x_host, xb, cudaMemcpyHostToDevice, st));
  const int nl = h->multiform ? h->n_lam : h->S;
  if (nl > 0) CK(cudaMemcpyAsync(h->d_lam_stage, lambda_host, (size_t)nl * 8, cudaMemcpyHostToDevice, st));
  int r = enqueue_eval(h, h->d_x_stage, x_is_fp64 ? 1 : 0, h->d_lam_stage, h->d_E_stage, h->d_F_stage,
                       h->d_dEdl_stage);
  if (r != 0) return cuda_fail((cudaError_t)r, "mahi_eval_host");
  if (energy_host) CK(cudaMemcpyAsync(energy_host, h->d_E_stage, 8, cudaMemcpyDeviceToHost, st));
  if (forces_host) CK(cudaMemcpyAsync(forces_host, h->d_F_stage, xb, cudaMemcpyDeviceToHost, st));
  if (dEdlambda_host && h->S > 0)
    CK(cudaMemcpyAsync(dEdlambda_host, h->d_dEdl_stage, (size_t)nl * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return take_status(h);
}

int mahi_get_potential(mahi_t h, double *phi_device) {
  if (!h || !phi_device) return MAHI_ERR_INVALID_ARG;
  if (enqueue_potential(h, phi_device) != 0) return cuda_fail(cudaGetLastError(), "potential");
  return MAHI_OK;
}

int mahi_set_timing(mahi_t h, int32_t on) {
  if (!h) return MAHI_ERR_INVALID_ARG;
  h->timing = on != 0;
  return MAHI_OK;
}

int mahi_stage_times(mahi_t h, float *ms, int32_t n) {
  if (!h || !ms) return MAHI_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(h->stream));
  int ns = std::min(num_stages(), h->n_ev - 1);
  for (int i = 0; i < ns && i < n; ++i) {
    float t = 0;
    CK(cudaEventElapsedTime(&t, h->ev[i], h->ev[i + 1]));
    ms[i] = t;
  }
  // the side-stream intervals follow the main-stream stages (0 when not run)
  if (ns == num_stages()) {
    CK(cudaStreamSynchronize(h->side));
    for (int k = 0; k < 2; ++k, ++ns) {
      float t = 0;
      if (h->side_timed & (1 << k)) CK(cudaEventElapsedTime(&t, h->ev[kSideEv + 2 * k], h->ev[kSideEv + 2 * k + 1]));
      if (ns < n) ms[ns] = t;
    }
  }
  return ns;
}

int mahi_launch_count(mahi_t h) { return h ? h->launches : 0; }

int mahi_lattice_coeffs(int32_t order_p, int32_t shell, double *coeffs) {
  if (order_p < 1 || order_p > kMaxOrder || !coeffs || (shell != 1 && shell != kLatticeShell))
    return MAHI_ERR_INVALID_ARG;
  const std::vector<double> &eta = lattice_coeffs(2 * order_p, shell);
  std::memcpy(coeffs, eta.data(), eta.size() * sizeof(double));
  return MAHI_OK;
}

int mahi_lattice_eval(double box_L_nm, int32_t order_p, int32_t shell, int64_t n, const double *r, double *H) {
  if (!(box_L_nm > 0) || order_p < 1 || order_p > kMaxOrder || n < 0 || (n > 0 && (!r || !H)) ||
      (shell != 1 && shell != kLatticeShell))
    return MAHI_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i) H[i] = lattice_eval_host(box_L_nm, 2 * order_p, shell, r + 3 * i);
  return MAHI_OK;
}

}  // extern "C"
