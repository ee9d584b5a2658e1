// Batched replicas in one CUDA graph, and the launch-shape autotuner.
//
// Constant-pH runs keep many independent replicas of different sizes (their
// own box, atoms, sites and lambdas).  mahi_batch_create records one MAHI
// evaluation of every replica, back to back on one stream, into a CUDA graph;
// mahi_batch_launch replays it with a single launch call, so the host cost of
// the ~40 kernel launches per replica is paid once at capture.  Each replica
// is captured on its own branch stream, so the graph holds the replicas as
// parallel branches and the GPU runs their kernels side by side (most of a
// small replica's kernels fill a fraction of the SMs).  The graph keeps the
// pointers it was captured with: callers update positions and lambdas in
// place between launches.
//
// mahi_autotune times candidate launch shapes of the two kernels whose best
// shape depends on the system (atoms per leaf, sites) on the caller's input
// and keeps the fastest: threads per target leaf of the near field (64, 128,
// 256) and blocks per site of the site-potential traversal (the default count
// and neighbouring powers of two).  Results change only in the order of
// floating-point sums.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mahi_internal.h"

struct mahi_batch_ctx {
  std::vector<mahi_t> h;
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> branch;     // one capture stream per replica: parallel graph branches
  std::vector<cudaEvent_t> ev;          // fork event, then one join event per branch
};

namespace {
void release(mahi_batch_ctx *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->branch)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  delete b;
}
}  // namespace

namespace {
int fail_cuda(cudaError_t e) { return e == cudaSuccess ? MAHI_OK : MAHI_ERR_CUDA; }
}  // namespace

extern "C" {

int mahi_autotune(mahi_t h, const void *x, int32_t x_is_fp64, const double *lambda, int32_t reps) {
  if (!h || !x || (h->S > 0 && !lambda) || reps < 1) return MAHI_ERR_INVALID_ARG;
  if (!h->charges_set) return MAHI_ERR_STATE;
  if (cudaSetDevice(h->device) != cudaSuccess) return MAHI_ERR_CUDA;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return MAHI_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return MAHI_ERR_CUDA;
  }
  const bool timing = h->timing;
  h->timing = false;
  // near-field shapes: half shell with 8 or 4 targets per thread (single
  // precision), or all directed pairs with 64 / 128 / 256 threads per leaf
  const bool sp = h->prec != MAHI_FP64;
  const int p2p_t[5] = {8, 4, -1, -1, -1}, p2p[5] = {128, 128, 64, 128, 256};
  const int np = sp ? 5 : 3, p0 = sp ? 0 : 2;
  const int g0 = std::max(1, std::min(16, (3 * h->num_sms + h->S - 1) / std::max(1, h->S)));
  std::vector<int> gs = {0};
  if (h->S > 0) {
    if (g0 / 2 >= 1) gs.push_back(g0 / 2);
    if (g0 * 2 <= 16) gs.push_back(g0 * 2);
  }
  float best = 1e30f;
  int best_p = h->tune_p2p_threads, best_t = h->tune_p2p_targets, best_g = h->tune_site_blocks;
  int rc = MAHI_OK;
  for (int pi = p0; pi < p0 + np && rc == MAHI_OK; ++pi)
    for (size_t gi = 0; gi < gs.size() && rc == MAHI_OK; ++gi) {
      h->tune_p2p_threads = p2p[pi];
      rc = mahi_set_option(h, MAHI_OPT_P2P_TARGETS, sp ? p2p_t[pi] : -1);  // allocates the slots on first use
      if (rc != MAHI_OK) break;
      h->tune_site_blocks = gs[gi];
      // one untimed evaluation (launch attributes, caches), then reps timed
      rc = mahi_eval(h, x, x_is_fp64, lambda, nullptr, nullptr, nullptr);
      if (rc != MAHI_OK) break;
      if (cudaEventRecord(a, h->stream) != cudaSuccess) { rc = MAHI_ERR_CUDA; break; }
      for (int r = 0; r < reps && rc == MAHI_OK; ++r) rc = mahi_eval(h, x, x_is_fp64, lambda, nullptr, nullptr, nullptr);
      if (rc != MAHI_OK) break;
      float ms = 0.f;
      if (cudaEventRecord(b, h->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
          cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        rc = MAHI_ERR_CUDA;
        break;
      }
      if (ms < best) {
        best = ms;
        best_p = p2p[pi];
        best_t = sp ? p2p_t[pi] : -1;
        best_g = gs[gi];
      }
    }
  h->tune_p2p_threads = best_p;
  h->tune_p2p_targets = best_t;
  h->tune_site_blocks = best_g;
  // then the tensor-core M2L's tiling with the shapes chosen above
  if (rc == MAHI_OK && h->prec == MAHI_MIXED && h->d >= 1) {
    const bool single0 = h->tune_m2l_single;
    const int nsb0 = h->tune_m2l_nsb;
    bool best_single = single0;
    int best_nsb = nsb0;
    float best_m = 1e30f;
    const int nsbs[3] = {0, 3, 2};
    for (int si = 0; si < 2 && rc == MAHI_OK; ++si) {
      if (si == 1 && h->ld > 192) break;      // single tiles already (no pairs fit)
      rc = mahi_set_option(h, MAHI_OPT_M2L_SINGLE_TILE, si);
      for (int ni = 0; ni < 3 && rc == MAHI_OK; ++ni) {
        h->tune_m2l_nsb = nsbs[ni];
        rc = mahi_eval(h, x, x_is_fp64, lambda, nullptr, nullptr, nullptr);
        if (rc != MAHI_OK) break;
        if (cudaEventRecord(a, h->stream) != cudaSuccess) { rc = MAHI_ERR_CUDA; break; }
        for (int r = 0; r < reps && rc == MAHI_OK; ++r) rc = mahi_eval(h, x, x_is_fp64, lambda, nullptr, nullptr, nullptr);
        if (rc != MAHI_OK) break;
        float ms = 0.f;
        if (cudaEventRecord(b, h->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
            cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
          rc = MAHI_ERR_CUDA;
          break;
        }
        if (ms < best_m) {
          best_m = ms;
          best_single = si == 1;
          best_nsb = nsbs[ni];
        }
      }
    }
    const int rc2 = mahi_set_option(h, MAHI_OPT_M2L_SINGLE_TILE, best_single ? 1 : 0);
    if (rc == MAHI_OK) rc = rc2;
    h->tune_m2l_nsb = best_nsb;
  }
  h->timing = timing;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

int mahi_get_tuning(mahi_t h, int32_t *p2p_threads, int32_t *site_blocks) {
  if (!h || !p2p_threads || !site_blocks) return MAHI_ERR_INVALID_ARG;
  *p2p_threads = h->tune_p2p_threads;
  *site_blocks = h->tune_site_blocks;
  return MAHI_OK;
}

int mahi_batch_create(const mahi_t *handles, int32_t n, void *cuda_stream, const void *const *x,
                      const int32_t *x_is_fp64, const double *const *lambda, double *const *energy,
                      void *const *forces, double *const *dEdlambda, mahi_batch_t *out) {
  if (!handles || n < 1 || !x || !x_is_fp64 || !lambda || !energy || !forces || !dEdlambda || !out)
    return MAHI_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!handles[i] || !x[i]) return MAHI_ERR_INVALID_ARG;
    if (!handles[i]->charges_set) return MAHI_ERR_STATE;
    if (handles[i]->device != handles[0]->device) return MAHI_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(handles[0]->device) != cudaSuccess) return MAHI_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (st == nullptr) return MAHI_ERR_INVALID_ARG;  // the legacy stream cannot be captured
  auto *b = new mahi_batch_ctx;
  b->h.assign(handles, handles + n);
  b->stream = st;
  int rc = MAHI_OK;
  b->branch.assign(n, nullptr);
  b->ev.assign(n + 1, nullptr);
  for (int i = 0; i < n && rc == MAHI_OK; ++i)
    rc = fail_cuda(cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking));
  for (int i = 0; i <= n && rc == MAHI_OK; ++i)
    rc = fail_cuda(cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming));
  // one eager evaluation per replica first: launch attributes are set outside capture
  for (int i = 0; i < n && rc == MAHI_OK; ++i) {
    handles[i]->stream = st;
    rc = mahi_eval(handles[i], x[i], x_is_fp64[i], lambda[i], energy[i], forces[i], dEdlambda[i]);
  }
  if (rc == MAHI_OK) rc = fail_cuda(cudaStreamSynchronize(st));
  if (rc == MAHI_OK) rc = fail_cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  if (rc == MAHI_OK) {
    // the replicas are independent: each is captured on its own branch stream
    // forked from (and joined back into) the batch stream, so the graph has n
    // parallel branches and their small kernels run side by side
    rc = fail_cuda(cudaEventRecord(b->ev[0], st));
    for (int i = 0; i < n && rc == MAHI_OK; ++i) rc = fail_cuda(cudaStreamWaitEvent(b->branch[i], b->ev[0], 0));
    for (int i = 0; i < n && rc == MAHI_OK; ++i) {
      handles[i]->stream = b->branch[i];
      rc = mahi_eval(handles[i], x[i], x_is_fp64[i], lambda[i], energy[i], forces[i], dEdlambda[i]);
      handles[i]->stream = st;
      if (rc == MAHI_OK) rc = fail_cuda(cudaEventRecord(b->ev[i + 1], b->branch[i]));
      if (rc == MAHI_OK) rc = fail_cuda(cudaStreamWaitEvent(st, b->ev[i + 1], 0));
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc == MAHI_OK && e != cudaSuccess) rc = MAHI_ERR_CUDA;
    b->graph = g;
  }
  if (rc == MAHI_OK) rc = fail_cuda(cudaGraphInstantiate(&b->exec, b->graph, 0));
  if (rc != MAHI_OK) {
    for (int i = 0; i < n; ++i) handles[i]->stream = st;
    cudaGetLastError();
    release(b);
    return rc;
  }
  *out = b;
  return MAHI_OK;
}

int mahi_batch_launch(mahi_batch_t b) {
  if (!b) return MAHI_ERR_INVALID_ARG;
  return fail_cuda(cudaGraphLaunch(b->exec, b->stream));
}

int mahi_batch_destroy(mahi_batch_t b) {
  if (!b) return MAHI_OK;
  release(b);
  return MAHI_OK;
}

}  // extern "C"
