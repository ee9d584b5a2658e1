// Internal declarations shared by the host planner, the kernels and the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "../../include/mahi.h"

namespace mahi {

constexpr int kMaxOrder = 24;          // FP64 path
constexpr int kMaxOrderMixed = 16;     // FP32 exponent range of the M2L operators
constexpr int kMaxDepth = 6;
constexpr int kNumOffsets = 316;       // {-3..3}^3 minus {-1..1}^3
constexpr int kListLen = 189;          // M2L interaction list of one box
constexpr int kLatticeShell = 3;       // images |n|_inf <= 3 exactly, beyond by H_3
constexpr int kSiteDegree = 40;        // degree of H_1 in the per-site correction
constexpr int kSiteChunksMax = 16;   // blocks sharing one site in the site-potential traversal
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr int kFinalBlocks = 64;  // blocks of the final energy sum
// sites of up to kSiteSymMax atoms evaluate each unordered pair once
constexpr int kSiteSymMax = 16;
constexpr int kSiteSymPairs = kSiteSymMax * (kSiteSymMax - 1) / 2;

// Coulomb constant N_A e^2 / (4 pi eps0) in kJ mol^-1 nm e^-2 (CODATA 2018).
double coulomb_constant();

// Records a failed CUDA call for mahi_last_cuda_error and returns MAHI_ERR_CUDA.
int cuda_fail(cudaError_t e, const char *what);

// Slots of the per-handle device status word (host-mapped, set by kernels on failure).
constexpr int kStatusM2LTimeout = 0;   // a bounded wait of the tensor-core M2L gave up
constexpr int kStatusSiteOverflow = 1; // a site traversal list outgrew its capacity
constexpr int kStatusSiteTimeout = 2;  // a bounded wait of the site-atom potential gave up
constexpr int kStatusWords = 4;
// Default separation ratio of the site-atom traversal at order p (truncation
// bound theta^(p+1) of p = 12, theta = 0.4 kept at every order, within [0.25, 0.4])
float default_site_theta(int p);
// Default list capacity of the site traversal for a separation ratio theta
int default_site_list_cap(float theta);
constexpr int kSiteListCapMax = 8192;
// Default input degree up to which the tensor-core M2L uses three TF32 products
// (above it one product; -1: one product for every degree): 2, i.e. the first
// two K chunks (coefficients 0..15)
int default_m2l_split_degree(int p);
constexpr int kSideEv = 24;            // first of the four side-stream timing events of a handle

// Number of real coefficients of an order-p expansion and the padded row stride.
inline int ncoef(int p) { return (p + 1) * (p + 1); }
inline int nstride(int p) { return ((ncoef(p) + 15) / 16) * 16; }

// ---- host planner (mahi_host.cpp) -----------------------------------------
// Real translation operators at unit (level-normalised) scale, dense row-major
// [out][in] of size ncoef(p)^2.  Child index b = bx | by<<1 | bz<<2.
void build_m2m(int p, int child, std::vector<double> &op);
void build_l2l(int p, int child, std::vector<double> &op);
void build_m2l(int p, int ox, int oy, int oz, std::vector<double> &op);
// Lattice coefficients eta^ (unit box) of H_shell up to degree P, real layout (P+1)^2.
const std::vector<double> &lattice_coeffs(int P, int shell);
// Lattice operator (root local from root multipole): H_3 lattice part plus the
// root images 2 <= |n|_inf <= 3 by M2L; ncoef(p)^2, FP64, unscaled basis.
void build_lattice_op(int p, std::vector<double> &op, bool with_images = true);
// Convert an unscaled operator to the device basis: kind 0 = M2M, 1 = L2L,
// 2 = M2L / lattice.
void scale_operator(int p, int kind, std::vector<double> &op);
double basis_scale(int col);
// Derivative coefficient vectors of an order-P real expansion: given coefficients
// c of phi = sum c_lm R*_lm(u), returns d/dx, d/dy, d/dz coefficients of degree P-1.
void gradient_coeffs(int P, const double *c, double *cx, double *cy, double *cz);
// Host evaluation of H_shell(r) for box edge L from the coefficients (degree P).
double lattice_eval_host(double L, int P, int shell, const double r[3]);

// M2L offset table: id of offset (ox,oy,oz) in [-3,3]^3 (or -1), and the 189
// offsets of each child index.
struct OffsetTables {
  int id[343];
  int off[kNumOffsets][3];
  int list[8][kListLen];  // offset ids
};
const OffsetTables &offset_tables();

inline uint32_t morton_spread(uint32_t v) {
  uint32_t x = v & 0x3ff;
  x = (x | (x << 16)) & 0x030000FF;
  x = (x | (x << 8)) & 0x0300F00F;
  x = (x | (x << 4)) & 0x030C30C3;
  x = (x | (x << 2)) & 0x09249249;
  return x;
}

}  // namespace mahi

// ---- the handle ---------------------------------------------------------------
struct mahi_ctx {
  double L = 0;
  int64_t N = 0;
  int S = 0, p = 0, d = 0, prec = 0;
  int num_sms = 152;                          // streaming multiprocessors of the device
  int K = 0, ld = 0;           // coefficients per expansion, row stride
  int nleaf = 0;
  int64_t nbox_total = 0;
  int64_t level_off[mahi::kMaxDepth + 2] = {0};
  cudaStream_t stream = nullptr;
  int device = 0;
  bool charges_set = false;
  bool timing = false;
  int launches = 0;
  int n_site_atoms = 0;

  // device buffers
  void *arena = nullptr;
  size_t arena_bytes = 0;
  double *qA = nullptr, *dq = nullptr;   // N
  int *site_of = nullptr;                // N
  double *qt = nullptr;                  // N, scaled charges (FP64)
  int *leaf_of = nullptr, *slot = nullptr, *leaf_count = nullptr, *leaf_start = nullptr;
  int *perm = nullptr, *perm_tmp = nullptr, *inv_perm = nullptr;
  void *part = nullptr, *part_tmp = nullptr;  // float4 or double4, sorted by leaf
  void *vtmp = nullptr;                       // float4 or double4, original order
  double *relD = nullptr;                     // N x 3 offsets from the leaf centre (FP64)
  void *Mexp = nullptr, *Lexp = nullptr;      // expansions, all levels
  void *phi_s = nullptr, *grad_s = nullptr;   // sorted potential / gradient
  void *nf_slots = nullptr;                   // [13][N] float4: half-shell near-field sums (single precision)
  void *ops_m2m = nullptr, *ops_l2l = nullptr, *ops_m2l = nullptr;
  void *gemm_ws = nullptr;                    // K-split partials of the M2M / L2L GEMMs
  size_t gemm_ws_elems = 0;
  double *ops_lat = nullptr;                  // FP64 root operator (images 2..3 + H_3)
  double *ops_lat_h3 = nullptr;               // FP64 H_3 part alone (site-atom path)
  double *L_h3 = nullptr;                     // root local of H_3 (K doubles)
  double *box_qd = nullptr;                   // FP64 Q, D, T per box (8 doubles), all levels
  float *box_qdf = nullptr;                   // Q, D per box as (hi, lo) float pairs (8 floats), all levels
  double *phi_site = nullptr;                 // refined potential at site atoms
  double *psi_site = nullptr;                 // f sum_j A_ij D_j at site atoms (charge gradients)
  double *site_pairs = nullptr;               // [S][kSiteSymPairs][4]: grad A, A of every site pair
  int4 *site_pair_list = nullptr;             // [n_site_pairs] {site, i, j, pair index} of sites up to kSiteSymMax atoms
  int n_site_pairs = 0;
  int *site_order = nullptr;                  // [S] sites by descending atom count (site-potential blocks)
  int *site_slot = nullptr;                   // N: position in site_atoms, -1 for environment atoms
  // sites with 2^m forms (mahi_set_forms)
  bool multiform = false;
  double *mf_q = nullptr;                     // [site atom slot][16] charges per form
  int *mf_lam_off = nullptr;                  // [S + 1] offsets of each site's lambdas
  int n_lam = 0;                              // lambdas (and dE/dlambda entries) in total
  double *mf_psi = nullptr;                   // [site atom slot][16] f (A q^r) per form (backward)
  int *mf_form_off = nullptr;                 // [S + 1] offsets of each site's entries in the q_forms layout
  int n_form_charges = 0;                     // sum_s F_s n_s
  double *phi_part = nullptr;                 // its per-part partial sums
  int64_t *d_level_off = nullptr;             // device copy of level_off
  double *eta = nullptr, *eta_x = nullptr, *eta_y = nullptr, *eta_z = nullptr;  // degree 2p
  double site_aii = 0.0;                      // self term A_ii of the periodic kernel (1/nm)
  float site_theta = 0.40f;                   // separation ratio of the site-potential traversal
  bool site_theta_set = false;                // set by mahi_set_option (else the default rule)
  int site_list_cap = 1536;                   // boxes per level of one site's traversal
  int *site_lists = nullptr;                  // [S][d + 1][cap] traversal lists of compact sites (k_site_lists)
  int *site_list_n = nullptr;                 // [S][d + 2] their lengths (-1: spread site)
  double *site_cen = nullptr;                 // [S][4] site centre and radius
  int site_lists_cap = 0;                     // list capacity the buffers were sized for
  bool site_list_cap_set = false;
  uint64_t wait_limit_ns = 2000000000ull;     // bounded device waits of the tensor-core M2L
  int watchdog_selftest = 0;                  // 1: the M2L's first wait is on a barrier nothing completes
  int m2l_split_degree = 0;                   // tensor-core M2L: three TF32 products up to this input degree
  int *status_host = nullptr;                 // kStatusWords ints, host-mapped pinned memory
  int *status_dev = nullptr;                  // the same words as seen from the device
  int tune_p2p_threads = 128;                 // autotuned launch shapes (mahi_autotune)
  int tune_p2p_targets = -1;                  // near field: 4 / 8 targets per lane (half shell), -1 all directed pairs
  int tune_site_blocks = 0;                   // 0 = default count of blocks per site
  bool tune_m2l_single = false;               // tensor-core M2L: single 128-row tiles where pairs would fit
  int tune_m2l_nsb = 0;                       // tensor-core M2L operator stages (0 = as many as fit)
  int *m2l_list = nullptr;                    // [8][189] offset ids
  int *m2l_off = nullptr;                     // [316][3]
  int *site_ptr = nullptr, *site_atoms = nullptr;
  double *energy_part = nullptr;              // per-block energy partials
  double *site_energy = nullptr;              // S
  int n_moment_blocks = 0;                    // grid of k_bin
  // tensor-core M2L operand images (mixed path)
  void *tc_ops = nullptr;
  void *tc_partial = nullptr;                 // M2L partial tiles of units split across CTAs
  void *tc_msrc = nullptr;                    // multipoles in the M2L gather layout
  int64_t *tc_level_off = nullptr;            // device copy of level_off
  int *tc_units = nullptr;
  int tc_nunits = 0;
  // host staging for mahi_eval_host
  void *d_x_stage = nullptr;
  double *d_lam_stage = nullptr, *d_E_stage = nullptr, *d_dEdl_stage = nullptr;
  void *d_F_stage = nullptr;
  int x_stage_fp64 = -1;

  cudaEvent_t ev[32] = {};
  int n_ev = 0;
  int side_timed = 0;                         // bit k: side-stream interval k recorded
  // side stream for work that does not depend on the main chain (box moments
  // during P2M/M2M, the site-atom potential during L2L/L2P/P2P), forked and
  // joined with events inside every evaluation
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev[3] = {}, join_ev[2] = {};
  // stream of the greatest priority for the main chain of an evaluation,
  // forked from and joined back into the handle's stream: its blocks are
  // dispatched before the side stream's as SMs free up
  cudaStream_t hp = nullptr;
  cudaEvent_t hp_ev[2] = {};
};

namespace mahi {
// ---- kernel launchers (mahi_kernels.cu) ------------------------------------
int enqueue_eval(mahi_ctx *h, const void *x, int x_is_fp64, const double *lambda, double *energy,
                 void *forces, double *dEdl);
int enqueue_potential(mahi_ctx *h, double *phi);
int enqueue_update_charges(mahi_ctx *h, const double *qA, const double *qB);
int enqueue_backward_forms(mahi_ctx *h, const double *gE, const void *forces, const double *dEdl, const double *lam,
                           int x_is_fp64, void *dx, double *dlam, double *dq_env, double *dq_forms);
int enqueue_backward(mahi_ctx *h, const double *gE, const void *forces, const double *dEdl, const double *lam,
                     int x_is_fp64, void *dx, double *dlam, double *dqA, double *dqB);
int upload_tables();
int alloc_site_lists(mahi_ctx *h);
int alloc_near_slots(mahi_ctx *h);
size_t gemm_workspace_elems(int d, int ld, int num_sms);
const char *stage_name(int i);
int num_stages();
// tensor-core M2L (mahi_m2l_tc.cu)
size_t tc_ops_bytes(int p);
void tc_pack_ops(int p, const std::vector<std::vector<double>> &m2l, void *host_image);
int tc_build_units(mahi_ctx *h, std::vector<int> &units);
int tc_upload_units(mahi_ctx *h);
int tc_m2l(mahi_ctx *h, cudaStream_t st);
}  // namespace mahi
