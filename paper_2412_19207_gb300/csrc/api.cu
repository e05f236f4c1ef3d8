// Host runtime and C ABI of librann_dd (see include/rann_dd.h).
//
// Owns the geometry (Sec. 5 Example 1: box subdomains, windows; cell-centred
// collocation grid), the device buffers, the task lists of the batched
// kernels, and the Krylov drivers (Sec. 3, Sec. 5).  All device work runs on
// the handle's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "chol_tc.h"

// launchers from the other translation units
cudaError_t launch_matvec_H2(const ProbDev& P, const SubDev* d_sub, const int* d_cov, int Gmax,
                             const double* d_B, const double* d_x, double* d_y, int64_t N, cudaStream_t st);
cudaError_t launch_matvec_HT2(const ProbDev& P, const SubDev* d_sub, int J, const int* d_rtiles,
                              int nrtiles, const int* d_tile0, const double* d_B, const double* d_y,
                              double* d_part, double* d_z, int maxP, cudaStream_t st);
cudaError_t launch_chol_step(const CholMat* d_mats, int nmat, int maxn, int c0, int* d_fail,
                             const double* d_dmax, cudaStream_t st);
cudaError_t launch_trtri(const CholMat* d_mats, int nmat, int maxn, cudaStream_t st);
cudaError_t launch_chol_df_lookahead(const CholMat* d_mats, int nmat, int maxn, int* d_fail, const double* d_dmax,
                                     cudaStream_t st, cudaStream_t st2, cudaStream_t st3, cudaEvent_t* ev,
                                     int* nlaunch);
cudaError_t launch_split(const double* d_x, float2* d_x2, int64_t n, cudaStream_t st);
cudaError_t launch_split_pad(const SubDev* d_sub, int J, const double* d_x, float2* d_x2p, cudaStream_t st);
cudaError_t launch_rowdot_df(const SubDev* d_sub, const int* d_rtiles, int nrtiles, int tile_rows,
                             const float2* d_B2, const float2* d_x2p, float2* d_yp, cudaStream_t st);
cudaError_t launch_matvec_HT_df(const ProbDev& P, const SubDev* d_sub, int J, const int* d_rtiles, int nrtiles,
                                int tile_rows, const int* d_tile0, const int* d_cov, int Gmax, const float2* d_B2,
                                const float2* d_yp, double* d_part, double* d_z, int maxP, cudaStream_t st);
constexpr int DF_TILE_ROWS = 128;  // rows per block of the direct-load double-float matvec
cudaError_t launch_split_lower(const CholMat* d_mats, int nmat, int maxn, cudaStream_t st);
cudaError_t launch_schwarz_gather_df(int nsets, const int* d_set_ptr, const int* d_set_sub, const SubDev* d_sub,
                                     const int64_t* d_s_off, const double* d_r, float2* d_g2, int wkind,
                                     const int* d_inc_ptr, cudaStream_t st);
int schwarz_apply_rows();
int schwarz_apply_max_subs();
cudaError_t launch_schwarz_apply_multi(const CholMat* d_mats, int nsets, int maxn, const int* d_set_ptr,
                                       const int* d_set_sub, const SubDev* d_sub, const double* d_r, int64_t ldr,
                                       const int64_t* d_p_off32, double* d_part, int64_t pstride,
                                       const int64_t* d_s_off, double* d_s, int64_t lds, int* d_done, int nrhs,
                                       const int* d_inc_ptr, const int* d_inc_set, const int* d_inc_pos, int J,
                                       int ckind, double* d_z, int64_t ldz, cudaStream_t st);
cudaError_t launch_schwarz_apply_df(const CholMat* d_mats, int nsets, int maxn, const int* d_set_ptr,
                                    const int* d_set_sub, const SubDev* d_sub, const double* d_r,
                                    const int64_t* d_s_off, const int64_t* d_p_off32, double* d_part, double* d_s,
                                    int* d_done, int wkind, const int* d_inc_ptr, int ckind, double* d_z,
                                    cudaStream_t st, const float2* d_r2 = nullptr);
cudaError_t launch_x2_pairs(const CholMat* d_mats, int nsets, int maxn, cudaStream_t st);
cudaError_t launch_trmv_lower_df(const CholMat* d_mats, int nsets, int maxn, const int64_t* d_s_off,
                                 const float2* d_g2, float2* d_y2, cudaStream_t st);
cudaError_t launch_trmv_upper_df(const CholMat* d_mats, int nsets, int maxn, const int64_t* d_s_off,
                                 const int64_t* d_p_off, const float2* d_y2, double* d_part, double* d_s,
                                 cudaStream_t st);
cudaError_t launch_schwarz_gather(int nsets, const int* d_set_ptr, const int* d_set_sub, const SubDev* d_sub,
                                  const int64_t* d_s_off, const double* d_r, double* d_g, int wkind,
                                  const int* d_inc_ptr, cudaStream_t st);
cudaError_t launch_trmv_lower(const CholMat* d_mats, int nsets, int maxn, const int64_t* d_s_off,
                              const double* d_g, double* d_y, cudaStream_t st);
cudaError_t launch_trmv_upper(const CholMat* d_mats, int nsets, int maxn, const int64_t* d_s_off,
                              const int64_t* d_p_off, const double* d_y, double* d_part, double* d_s,
                              cudaStream_t st);
cudaError_t launch_schwarz_combine(const SubDev* d_sub, int J, const int* d_inc_ptr, const int* d_inc_set,
                                   const int* d_inc_pos, const int64_t* d_s_off, const double* d_s, int kind,
                                   double* d_z, cudaStream_t st);
cudaError_t launch_multidot(const double* V, int64_t ldv, int nv, const double* w, int64_t n, double* d_part,
                            double* d_out, cudaStream_t st);
cudaError_t launch_sub_combination(const double* V, int64_t ldv, int nv, const double* d_h, double* w,
                                   int64_t n, cudaStream_t st);
cudaError_t launch_add_combination(const double* V, int64_t ldv, int nv, const double* d_y, double* x,
                                   int64_t n, cudaStream_t st);
cudaError_t launch_axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t st);
cudaError_t launch_cg_update(double a, const double* p, const double* q, double* x, double* r, int64_t n,
                             cudaStream_t st);
cudaError_t launch_scale_copy(double a, const double* x, double* y, int64_t n, cudaStream_t st,
                              float2* y2 = nullptr);
cudaError_t launch_assemble_local(const double* d_pairbuf, const int64_t* d_tab, const int* d_tab_ptr,
                                  const int* d_boff, const int* d_boff_ptr, const CholMat* d_mats, int nsets,
                                  int maxn, double* d_dmax, cudaStream_t st, const int* d_which = nullptr);
int coef_grad_blocks(int64_t N);
cudaError_t launch_lmul(const ProbDev& P, const double* d_r, double* d_y, int64_t N, cudaStream_t st);
cudaError_t launch_coef_grad(const ProbDev& P, const SubDev* d_sub, const double* d_R, const double* d_b,
                             const double* d_Uw, const double* d_Ul, const double* d_r, const double* d_hl,
                             int64_t N, double* d_part, cudaStream_t st);
cudaError_t launch_add_diag(const CholMat* d_mats, const int* d_which, int nwhich, const double* d_shift,
                            int maxn, cudaStream_t st);

// ------------------------------------------------------------ errors --

static thread_local char g_err[512] = "";

void rann_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

#define CK(expr)                                                                         \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess) {                                                             \
      rann_set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, __LINE__); \
      return _e == cudaErrorMemoryAllocation ? RANN_ENOMEM : RANN_ECUDA;                 \
    }                                                                                    \
  } while (0)

#define REQUIRE(cond, status, ...)            \
  do {                                        \
    if (!(cond)) {                            \
      rann_set_error(__VA_ARGS__);            \
      return status;                          \
    }                                         \
  } while (0)

// ---------------------------------------------------- kernel families --
// Every kernel launch goes through KL(), which counts launches per family and,
// when profiling is on, brackets the launch with CUDA events on the handle's
// stream (the times are the device durations of the launches).
enum KId {
  K_POINTS, K_ASSEMBLE, K_RHS, K_GRAM, K_SYMM, K_EIG, K_PROJECT, K_PAIRGRAM, K_LOCALASM, K_ADDDIAG,
  K_CHOL, K_TRTRI, K_GATHER, K_TRMV_L, K_TRMV_U, K_COMBINE, K_MATVEC_H, K_MATVEC_HT, K_DOT, K_VEC, K_EVAL,
  K_SPLIT, K_MATVEC_H_DF, K_MATVEC_HT_DF, K_GATHER_DF, K_TRMV_L_DF, K_TRMV_U_DF, K_OZ_SPLIT, K_GRAM_OZ,
  K_PROJECT_OZ, K_EIG_VAL, K_EIG_VEC, K_EIG_ORTH, K_EIG_BACK, K_GRAMROWS, K_GRAMOP, K_PAIRGRAM_OZ, K_SCHWARZ_DF,
  K_CHOL_TC, K_COUNT
};
static const char* const KNAMES[K_COUNT] = {
  "points", "assemble", "rhs", "gram", "symmetrize", "eig_tridiag", "project", "pair_gram", "local_assemble",
  "add_diag", "cholesky", "trtri", "schwarz_gather", "trmv_lower", "trmv_upper", "schwarz_combine",
  "matvec_H", "matvec_HT", "dot", "vector", "eval", "split_df32", "matvec_H_df32", "matvec_HT_df32",
  "schwarz_gather_df32", "trmv_lower_df32", "trmv_upper_df32", "ozaki_split", "gram_ozaki", "project_ozaki", "eig_values", "eig_vectors", "eig_orth", "eig_back", "gram_rows", "gramop_df32",
  "pair_gram_ozaki", "schwarz_apply_df32", "cholesky_tc"};

// Roofline class of each family: 0 = HBM-bound (algorithmic bytes count),
// 1 = float64-ALU-bound (algorithmic flops count), 2 = bf16-tensor-core-bound
// (the flops of the digit-slice products count), 3 = double-float arithmetic
// on the float32 pipe (float64-equivalent flops count; the families marked in
// KDF below run that way in precision mode 1).
static const int KBOUND[K_COUNT] = {0, 1, 0, 1, 0, 1, 1, 1, 0, 0, 1, 1, 0, 0, 0, 0, 0, 0, 0, 0, 1,
                                     0, 0, 0, 0, 0, 0, 0, 2, 2, 1, 1, 1, 1, 0, 0, 2, 0, 2};

static bool family_is_df(int k) {
  return k == K_PAIRGRAM || k == K_CHOL || k == K_TRTRI || k == K_EIG_ORTH || k == K_EIG_BACK;
}

struct Prof {
  bool on = false;
  int64_t launches[K_COUNT] = {};
  double ms[K_COUNT] = {};
  double bytes[K_COUNT] = {};
  double flops[K_COUNT] = {};
  struct Pend { int kid; cudaEvent_t a, b; };
  std::vector<Pend> pending;
  std::vector<cudaEvent_t> pool;
};

// ------------------------------------------------------------ handle --

struct rann_dd_handle {
  cudaStream_t st = nullptr;
  cudaStream_t st_la = nullptr;   // high-priority stream of the Cholesky lookahead (created on first use)
  cudaStream_t st_inv = nullptr;  // stream of the row-block inverse inside the factorisation
  cudaEvent_t ev_la[7] = {};
  ProbDev P{};
  int J = 0, m = 0, dim = 0, Gmax = 0;
  int64_t N = 0, rows_total = 0;
  std::vector<SubDev> subs;
  std::vector<int> cov;
  std::vector<void*> allocs;
  // device geometry / weights
  SubDev* d_sub = nullptr;
  int* d_cov = nullptr;
  double* d_R = nullptr;
  double* d_b = nullptr;
  int* d_tiles = nullptr;
  int ntiles = 0;
  // assembly
  bool assembled = false;
  double* d_Psi = nullptr;
  double* d_H = nullptr;
  // pca
  bool reduced = false;
  double* d_eig = nullptr;
  double* d_V = nullptr;
  std::vector<double> eig_host;
  double* d_B = nullptr;
  int64_t dof = 0;
  int maxP = 0;
  int* d_rtiles = nullptr;
  int nrtiles = 0;
  int* d_tile0 = nullptr;
  double* d_part = nullptr;
  double* d_yscratch = nullptr;   // N
  float2* d_B2 = nullptr;         // reduced blocks as double-float pairs (inner Krylov operator)
  float2* d_x2 = nullptr;         // sum_j P_j: x as double-float pairs, each block's part 16-byte aligned
  float2* d_y2 = nullptr;         // rows_total: per-block row products B_j x_j
  int* d_dtiles = nullptr;        // (block, first row) tiles of the direct-load double-float matvec
  int ndtiles = 0;
  int* d_dtile0 = nullptr;
  double* d_dpart = nullptr;
  int nsm = 1;
  // normal matrix as block rows (inner operator of precision mode 1, built by setup_precond)
  bool gram_ready = false;
  GramRows gram{};
  std::vector<void*> gram_allocs;
  int* d_gtile = nullptr;
  int ngtile = 0;
  double gram_entries = 0;        // sum_k p_k n_k
  int gram_maxn2 = 0;
  int inner_df = 1;               // precision mode: 1 = double-float preconditioner set-up and inner iterations
  // precond
  int prec_kind = -1;
  int n_shifted = 0;
  int nsets = 0, maxn = 0;
  std::vector<int> set_ptr, set_sub;
  CholMat* d_mats = nullptr;
  int* d_set_ptr = nullptr;
  int* d_set_sub = nullptr;
  int* d_inc_ptr = nullptr;
  int* d_inc_set = nullptr;
  int* d_inc_pos = nullptr;
  int64_t* d_s_off = nullptr;
  double* d_s = nullptr;       // s_i = A_i^{-1} g_i (sum n_i)
  double* d_g = nullptr;       // gathered g_i = R_i r
  double* d_y = nullptr;       // y_i = L_i^{-1} g_i
  double* d_tpart = nullptr;   // partial sums of the transposed product
  int64_t* d_p_off = nullptr;
  double* d_Amats = nullptr;
  float2* d_A2mats = nullptr;     // double-float A_i / L_i (precision mode 1 set-up)
  int64_t* d_p_off32 = nullptr;   // per set: offset of its 32-row-block partial sums
  int max_set_size = 0;           // most subdomains in one extended set
  double* d_tpart32 = nullptr;
  int* d_adone = nullptr;          // per set: row blocks of the fused apply finished (reset by the last)
  int64_t p32_total = 0;           // doubles of the fused apply's row-block sums (one right-hand side)
  // streaming apply (sets of up to schwarz_rows_nmax() unknowns): row chunks and their column sums
  SrChunk* d_sr_chunks = nullptr;
  int* d_sr_order = nullptr;
  int* d_sr_ckptr = nullptr;
  double* d_sr_part = nullptr;
  int sr_nchunks = 0;
  int apply_cfg = 0;               // Schwarz apply configuration (0: fused 32-row blocks; >= 1: streaming)
  std::vector<int> set_n;          // n_i of the extended sets (for re-planning the streaming apply)
  int64_t s_total = 0;             // entries of the stacked set vectors s_i (sum of n_i)
  bool prec_df = false;           // the set-up kept only double-float factors
  double* d_Xmats = nullptr;
  float2* d_X2mats = nullptr;
  float2* d_g2 = nullptr;
  float2* d_ys2 = nullptr;
  double* d_pairbuf = nullptr;
  // krylov scratch
  double* d_red = nullptr;     // multidot partials
  double* d_scal = nullptr;    // small device scalars
  double* h_scal = nullptr;    // pinned host mirror
  int* d_ozerr = nullptr;      // non-zero once a tensor-core product pipeline timed out
  std::vector<size_t> alloc_bytes;   // sizes of allocs[i]
  size_t live_bytes = 0;
  int64_t alloc_cap = -1;           // injected cap on live device bytes (< 0: none)
  // phase timing: events around assemble (+ rhs), pca, setup_precond
  cudaEvent_t ph_ev[3][2] = {};
  bool ph_rec[3] = {false, false, false};
  char* h_stage = nullptr;     // pinned staging arena of the uploads
  size_t stage_cap = 0, stage_used = 0;
  Prof prof;
  // algorithmic size aggregates for the kernel accounting
  double sumNp = 0, sumNm2 = 0, sumNmp = 0, sum_n = 0, sum_n2 = 0, sum_n3 = 0, pair_flops = 0;
};

static cudaEvent_t prof_event(rann_dd_handle* h) {
  if (!h->prof.pool.empty()) { cudaEvent_t e = h->prof.pool.back(); h->prof.pool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static void prof_resolve(rann_dd_handle* h) {
  if (h->prof.pending.empty()) return;
  cudaEventSynchronize(h->prof.pending.back().b);
  for (auto& p : h->prof.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) h->prof.ms[p.kid] += ms;
    h->prof.pool.push_back(p.a);
    h->prof.pool.push_back(p.b);
  }
  h->prof.pending.clear();
}

// Launch with accounting: nkern kernels, algorithmic bytes and flops of this launch.
#define KLA(h, kid, nkern, nbytes, nflops, expr)                            \
  do {                                                                      \
    cudaEvent_t _a = nullptr, _b = nullptr;                                 \
    if ((h)->prof.on) { _a = prof_event(h); cudaEventRecord(_a, (h)->st); } \
    CK(expr);                                                               \
    (h)->prof.launches[kid] += (nkern);                                     \
    (h)->prof.bytes[kid] += (double)(nbytes);                               \
    (h)->prof.flops[kid] += (double)(nflops);                               \
    if ((h)->prof.on) {                                                     \
      _b = prof_event(h);                                                   \
      cudaEventRecord(_b, (h)->st);                                         \
      (h)->prof.pending.push_back({kid, _a, _b});                           \
      if ((h)->prof.pending.size() > 4096) prof_resolve(h);                 \
    }                                                                       \
  } while (0)
#define KL(h, kid, nkern, expr) KLA(h, kid, nkern, 0, 0, expr)
#define TRY(x) do { rann_status _s = (x); if (_s != RANN_OK) return _s; } while (0)

static cudaError_t dalloc(rann_dd_handle* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (h->alloc_cap >= 0 && h->live_bytes + bytes > (size_t)h->alloc_cap) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMallocAsync(p, bytes, h->st);
  if (e == cudaSuccess) {
    h->allocs.push_back(*p);
    h->alloc_bytes.push_back(bytes);
    h->live_bytes += bytes;
  }
  return e;
}

// Host-to-device uploads go through a pinned staging arena, so they are
// asynchronous and the host can keep enqueueing; a region is reused only after
// the stream has been synchronised (stream_sync resets the arena).
static cudaError_t stream_sync(rann_dd_handle* h) {
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e == cudaSuccess) h->stage_used = 0;
  return e;
}

template <typename T>
static cudaError_t dupload(rann_dd_handle* h, T** dst, const std::vector<T>& v) {
  cudaError_t e = dalloc(h, (void**)dst, sizeof(T) * std::max<size_t>(v.size(), 1));
  if (e != cudaSuccess || v.empty()) return e;
  const size_t bytes = sizeof(T) * v.size(), need = (bytes + 255) & ~(size_t)255;
  if (h->stage_used + need > h->stage_cap) {
    if ((e = stream_sync(h)) != cudaSuccess) return e;
    if (need > h->stage_cap) {
      if (h->h_stage) cudaFreeHost(h->h_stage);
      h->h_stage = nullptr;
      h->stage_cap = 0;
      const size_t cap = std::max<size_t>(need, (size_t)16 << 20);
      if ((e = cudaMallocHost((void**)&h->h_stage, cap)) != cudaSuccess) return e;
      h->stage_cap = cap;
    }
  }
  memcpy(h->h_stage + h->stage_used, v.data(), bytes);
  e = cudaMemcpyAsync(*dst, h->h_stage + h->stage_used, bytes, cudaMemcpyHostToDevice, h->st);
  h->stage_used += need;
  return e;
}

static void dfree(rann_dd_handle* h, void* p) {
  if (!p) return;
  auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
  if (it != h->allocs.end()) {
    cudaFreeAsync(p, h->st);
    const size_t i = (size_t)(it - h->allocs.begin());
    h->live_bytes -= h->alloc_bytes[i];
    h->alloc_bytes.erase(h->alloc_bytes.begin() + i);
    h->allocs.erase(it);
  }
}

// Phase timing (stats): events recorded on the handle's stream around
// assemble (+ rhs), pca and setup_precond, resolved when stats are filled.
static void phase_mark(rann_dd_handle* h, int ph, int which) {
  cudaEvent_t& e = h->ph_ev[ph][which];
  if (!e && cudaEventCreate(&e) != cudaSuccess) { e = nullptr; return; }
  cudaEventRecord(e, h->st);
  if (which == 0) h->ph_rec[ph] = false;
  else h->ph_rec[ph] = true;
}
static double phase_ms(rann_dd_handle* h, int ph) {
  if (!h->ph_rec[ph] || !h->ph_ev[ph][0] || !h->ph_ev[ph][1]) return 0.0;
  float ms = 0.f;
  if (cudaEventSynchronize(h->ph_ev[ph][1]) != cudaSuccess) return 0.0;
  if (cudaEventElapsedTime(&ms, h->ph_ev[ph][0], h->ph_ev[ph][1]) != cudaSuccess) return 0.0;
  return ms;
}
static void fill_phase_stats(rann_dd_handle* h, rann_dd_stats* s) {
  s->ms_assemble = phase_ms(h, 0);
  s->ms_pca = phase_ms(h, 1);
  s->ms_setup = phase_ms(h, 2);
}

// Extreme eigenvalues of the symmetric tridiagonal T (diagonal a[0..n),
// off-diagonal b[0..n-1)) by bisection on Sturm counts.
static void tridiag_extremes(const std::vector<double>& a, const std::vector<double>& b, double* lmin,
                             double* lmax) {
  const int n = (int)a.size();
  double lo = a[0], hi = a[0];
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {   // eigenvalues < x
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < n; ++i) {
      d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0.0) ++c;
    }
    return c;
  };
  for (int which = 0; which < 2; ++which) {
    double l = lo, u = hi;
    const int k = which == 0 ? 1 : n;   // the k-th smallest
    for (int it = 0; it < 200 && u - l > 1e-15 * std::max(std::fabs(l), std::fabs(u)); ++it) {
      const double mid = 0.5 * (l + u);
      if (count_below(mid) >= k) u = mid; else l = mid;
    }
    (which == 0 ? *lmin : *lmax) = 0.5 * (l + u);
  }
}

// Extreme singular values of the leading n x n upper triangle of R (row
// stride ld) by one-sided Jacobi rotations of its columns.
static void triangle_sing_extremes(const std::vector<double>& Rm, int n, int ld, double* smin, double* smax) {
  std::vector<double> G((size_t)n * n, 0.0);   // column c at G[c * n ..]
  for (int r = 0; r < n; ++r)
    for (int c = r; c < n; ++c) G[(size_t)c * n + r] = Rm[(size_t)r * ld + c];
  for (int sweep = 0; sweep < 60; ++sweep) {
    int rot = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double a = 0, bq = 0, c = 0;
        for (int r = 0; r < n; ++r) {
          const double x = G[(size_t)p * n + r], y = G[(size_t)q * n + r];
          a += x * x; bq += y * y; c += x * y;
        }
        if (std::fabs(c) <= 1e-15 * std::sqrt(a * bq)) continue;
        ++rot;
        const double zeta = (bq - a) / (2.0 * c);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int r = 0; r < n; ++r) {
          const double x = G[(size_t)p * n + r], y = G[(size_t)q * n + r];
          G[(size_t)p * n + r] = cs * x - sn * y;
          G[(size_t)q * n + r] = sn * x + cs * y;
        }
      }
    if (!rot) break;
  }
  double lo = INFINITY, hi = 0.0;
  for (int c = 0; c < n; ++c) {
    double s = 0;
    for (int r = 0; r < n; ++r) s += G[(size_t)c * n + r] * G[(size_t)c * n + r];
    s = std::sqrt(s);
    lo = std::min(lo, s);
    hi = std::max(hi, s);
  }
  *smin = lo;
  *smax = hi;
}

static uint64_t splitmix64_draw(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

extern "C" const char* rann_dd_status_string(rann_status s) {
  switch (s) {
    case RANN_OK: return "ok";
    case RANN_EINVAL: return "invalid argument";
    case RANN_ENOMEM: return "out of memory";
    case RANN_ECUDA: return "CUDA error";
    case RANN_NOT_CONVERGED: return "not converged";
    case RANN_BREAKDOWN: return "breakdown";
    case RANN_LOCAL_SINGULAR: return "local factor shifted";
    case RANN_EORDER: return "call out of order";
    case RANN_TIMEOUT: return "device wait timed out";
  }
  return "unknown";
}

extern "C" const char* rann_dd_last_error(void) { return g_err; }

// ------------------------------------------------------------ create --

extern "C" rann_status rann_dd_create(const rann_dd_desc* d, void* stream, rann_dd_handle** out) {
  REQUIRE(d && out, RANN_EINVAL, "null descriptor or output");
  *out = nullptr;
  REQUIRE(d->dim == 2 || d->dim == 3, RANN_EINVAL, "dim must be 2 or 3");
  REQUIRE(d->op >= 0 && d->op <= 2, RANN_EINVAL, "bad op");
  REQUIRE(d->neurons >= 1 && d->neurons <= RANN_MAX_M, RANN_EINVAL, "neurons must be in 1..1024");
  REQUIRE(d->f_terms >= 0 && d->f_terms <= RANN_MAX_FTERMS, RANN_EINVAL, "f_terms must be in 0..16");
  REQUIRE(d->f_terms == 0 || (d->fc && d->fa), RANN_EINVAL, "fc/fa missing");
  REQUIRE(d->rho > 0.0, RANN_EINVAL, "rho must be positive");
  REQUIRE(d->layout == RANN_LAYOUT_CELL || d->layout == RANN_LAYOUT_PAPER, RANN_EINVAL, "bad layout");
  REQUIRE(d->g_kind == RANN_G_ZERO || d->g_kind == RANN_G_SINPROD, RANN_EINVAL, "bad g_kind");
  const int ns = d->op == RANN_OP_HEAT ? d->dim - 1 : d->dim;
  if (d->op == RANN_OP_DIFFUSION) {
    REQUIRE(d->coef >= 0 && d->coef <= 2, RANN_EINVAL, "bad coef");
    REQUIRE(d->coef == RANN_COEF_CONST || ns >= 2, RANN_EINVAL, "x-y coefficients need 2 spatial dims");
    if (d->coef == RANN_COEF_MULTISCALE) REQUIRE(d->eps > 0.0, RANN_EINVAL, "eps must be positive");
    if (d->coef == RANN_COEF_PIECEWISE)
      REQUIRE(d->coef_grid >= 1 && d->coef_grid <= 8 && d->coef_vals, RANN_EINVAL, "coef_grid in 1..8 with values");
  }
  for (int i = 0; i < d->dim; ++i) {
    REQUIRE(d->sub[i] >= 1 && d->pts[i] >= 1, RANN_EINVAL, "sub/pts must be >= 1");
    REQUIRE((int64_t)d->sub[i] * d->pts[i] <= (1 << 20), RANN_EINVAL, "grid too large");
    if (d->layout == RANN_LAYOUT_PAPER) REQUIRE(d->sub[i] >= 2 && d->delta > 1.0, RANN_EINVAL, "paper layout needs l >= 2, delta > 1");
    else REQUIRE(d->overlap[i] >= 0.0, RANN_EINVAL, "overlap must be >= 0");
  }
  rann_dd_handle* h = new rann_dd_handle();
  h->st = (cudaStream_t)stream;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
      // keep freed stream-ordered allocations cached in this process's default
      // pool (by default they return to the driver at every synchronisation,
      // and the large per-call buffers are then mapped again each time)
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
    }
    if (h->nsm < 1) h->nsm = 1;
  }
  ProbDev& P = h->P;
  P.dim = d->dim; P.ns = ns; P.op = d->op; P.coef = d->coef; P.g_kind = d->g_kind; P.m = d->neurons;
  P.c0 = d->c0; P.nu = d->nu; P.coef_value = d->coef_value; P.eps = d->eps; P.rho = d->rho; P.f0 = d->f0;
  P.coef_grid = d->coef_grid;
  if (d->op == RANN_OP_DIFFUSION && d->coef == RANN_COEF_PIECEWISE)
    for (int c = 0; c < d->coef_grid * d->coef_grid; ++c) P.coef_vals[c] = d->coef_vals[c];
  P.f_terms = d->f_terms;
  for (int t = 0; t < d->f_terms; ++t) {
    P.fc[t] = d->fc[t];
    for (int i = 0; i < d->dim; ++i) P.fa[t * d->dim + i] = d->fa[t * d->dim + i];
  }
  P.layout = d->layout;
  h->dim = d->dim; h->m = d->neurons;
  h->J = 1;
  h->N = 1;
  for (int i = 0; i < d->dim; ++i) {
    P.G[i] = d->sub[i] * d->pts[i];
    P.nsub[i] = d->sub[i];
    P.sig[i] = d->layout == RANN_LAYOUT_PAPER ? 0.5 * d->delta / (double)(d->sub[i] - 1)
                                              : 0.5 * (1.0 / d->sub[i] + d->overlap[i]);
    h->J *= d->sub[i];
    h->N *= P.G[i];
    h->Gmax = std::max(h->Gmax, P.G[i]);
  }
  for (int i = d->dim; i < 3; ++i) { P.G[i] = 1; P.nsub[i] = 1; P.sig[i] = 1.0; }
  // boxes per dim: grid indices strictly inside |x_q - mu_k| < sigma
  std::vector<std::vector<int>> blo(3), bhi(3);
  for (int i = 0; i < d->dim; ++i) {
    blo[i].assign(d->sub[i], -1);
    bhi[i].assign(d->sub[i], -1);
    for (int k = 0; k < d->sub[i]; ++k) {
      double mu = host_mu(d->layout, k, d->sub[i]);
      for (int q = 0; q < P.G[i]; ++q) {
        double x = ((double)q + 0.5) / (double)P.G[i];
        if (std::fabs(x - mu) < P.sig[i]) {
          if (blo[i][k] < 0) blo[i][k] = q;
          bhi[i][k] = q + 1;
        }
      }
      if (blo[i][k] < 0) {
        delete h;
        rann_set_error("subdomain %d along dim %d holds no collocation point", k, i);
        return RANN_EINVAL;
      }
    }
  }
  h->cov.assign((size_t)3 * h->Gmax * 2, 0);
  for (int i = 0; i < 3; ++i)
    for (int q = 0; q < h->Gmax; ++q) { h->cov[(i * h->Gmax + q) * 2] = 0; h->cov[(i * h->Gmax + q) * 2 + 1] = 1; }
  for (int i = 0; i < d->dim; ++i)
    for (int q = 0; q < P.G[i]; ++q) {
      int first = -1, cnt = 0;
      for (int k = 0; k < d->sub[i]; ++k)
        if (q >= blo[i][k] && q < bhi[i][k]) { if (first < 0) first = k; ++cnt; }
      h->cov[(i * h->Gmax + q) * 2] = first;
      h->cov[(i * h->Gmax + q) * 2 + 1] = cnt;
    }
  h->subs.resize(h->J);
  int64_t row0 = 0;
  for (int j = 0; j < h->J; ++j) {
    SubDev& S = h->subs[j];
    memset(&S, 0, sizeof(S));
    int rem = j;
    S.N = 1;
    for (int i = 0; i < 3; ++i) {
      if (i < d->dim) {
        S.k[i] = rem % d->sub[i];
        rem /= d->sub[i];
        S.lo[i] = blo[i][S.k[i]];
        S.n[i] = bhi[i][S.k[i]] - blo[i][S.k[i]];
        S.mu[i] = host_mu(d->layout, S.k[i], d->sub[i]);
      } else {
        S.k[i] = 0; S.lo[i] = 0; S.n[i] = 1; S.mu[i] = 0.0;
      }
      S.N *= S.n[i];
    }
    S.row0 = row0;
    S.p = h->m;
    S.P = h->m;
    row0 += S.N;
  }
  h->rows_total = row0;
  // weights
  const int m = h->m, dim = d->dim;
  std::vector<double> R((size_t)h->J * m * dim), b((size_t)h->J * m);
  if (d->R && d->b) {
    memcpy(R.data(), d->R, sizeof(double) * R.size());
    memcpy(b.data(), d->b, sizeof(double) * b.size());
  } else {
    const uint64_t per = (uint64_t)m * dim + m;
    for (int j = 0; j < h->J; ++j)
      for (uint64_t t = 0; t < per; ++t) {
        double u = (double)(splitmix64_draw(d->seed, (uint64_t)j * per + t) >> 11) * 0x1.0p-53;
        double v = -d->w_range + 2.0 * d->w_range * u;
        if (t < (uint64_t)m * dim) R[(size_t)j * m * dim + t] = v;
        else b[(size_t)j * m + (t - (uint64_t)m * dim)] = v;
      }
  }
  std::vector<int> tiles;
  for (int j = 0; j < h->J; ++j)
    for (int r0 = 0; r0 < h->subs[j].N; r0 += 32) { tiles.push_back(j); tiles.push_back(r0); }
  h->ntiles = (int)tiles.size() / 2;
  cudaError_t e;
  if ((e = dupload(h, &h->d_sub, h->subs)) != cudaSuccess || (e = dupload(h, &h->d_cov, h->cov)) != cudaSuccess ||
      (e = dupload(h, &h->d_R, R)) != cudaSuccess || (e = dupload(h, &h->d_b, b)) != cudaSuccess ||
      (e = dupload(h, &h->d_tiles, tiles)) != cudaSuccess ||
      (e = dalloc(h, (void**)&h->d_red, sizeof(double) * 256 * 130)) != cudaSuccess ||
      (e = dalloc(h, (void**)&h->d_scal, sizeof(double) * 256)) != cudaSuccess ||
      (e = dalloc(h, (void**)&h->d_ozerr, sizeof(int))) != cudaSuccess ||
      (e = cudaMemsetAsync(h->d_ozerr, 0, sizeof(int), h->st)) != cudaSuccess ||
      (e = cudaMallocHost((void**)&h->h_scal, sizeof(double) * 256)) != cudaSuccess) {
    rann_set_error("create: %s", cudaGetErrorString(e));
    rann_dd_destroy(h);
    return e == cudaErrorMemoryAllocation ? RANN_ENOMEM : RANN_ECUDA;
  }
  *out = h;
  return RANN_OK;
}

extern "C" void rann_dd_destroy(rann_dd_handle* h) {
  if (!h) return;
  for (void* p : h->allocs) cudaFreeAsync(p, h->st);
  cudaStreamSynchronize(h->st);
  if (h->h_scal) cudaFreeHost(h->h_scal);
  if (h->h_stage) cudaFreeHost(h->h_stage);
  prof_resolve(h);
  for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
  for (cudaStream_t* sp : {&h->st_la, &h->st_inv})
    if (*sp) {
      cudaStreamSynchronize(*sp);
      cudaStreamDestroy(*sp);
    }
  for (cudaEvent_t e : h->ev_la)
    if (e) cudaEventDestroy(e);
  for (auto& pe : h->ph_ev)
    for (cudaEvent_t e : pe)
      if (e) cudaEventDestroy(e);
  delete h;
}

extern "C" rann_status rann_dd_inject_fault(rann_dd_handle* h, int kind, int64_t value) {
  REQUIRE(h, RANN_EINVAL, "null handle");
  if (kind == RANN_FAULT_WAIT_EXPIRED) {
    const int w = (int)value;
    CK(cudaMemcpyAsync(h->d_ozerr, &w, sizeof(int), cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    return RANN_OK;
  }
  if (kind == RANN_FAULT_ALLOC_CAP) {
    h->alloc_cap = value < 0 ? -1 : value;
    return RANN_OK;
  }
  rann_set_error("unknown fault kind %d", kind);
  return RANN_EINVAL;
}

extern "C" rann_status rann_dd_sizes(rann_dd_handle* h, int64_t* n_points, int64_t* n_block_rows, int* J, int* m,
                                     int64_t* dof) {
  REQUIRE(h, RANN_EINVAL, "null handle");
  if (n_points) *n_points = h->N;
  if (n_block_rows) *n_block_rows = h->rows_total;
  if (J) *J = h->J;
  if (m) *m = h->m;
  if (dof) *dof = h->reduced ? h->dof : (int64_t)h->J * h->m;
  return RANN_OK;
}

extern "C" rann_status rann_dd_points(rann_dd_handle* h, double* xyz_dev) {
  REQUIRE(h && xyz_dev, RANN_EINVAL, "null argument");
  KL(h, K_POINTS, 1, launch_points(h->P, xyz_dev, h->N, h->st));
  return RANN_OK;
}

// ---------------------------------------------------------- assemble --

extern "C" rann_status rann_dd_assemble(rann_dd_handle* h) {
  REQUIRE(h, RANN_EINVAL, "null handle");
  phase_mark(h, 0, 0);
  const size_t bytes = sizeof(double) * (size_t)h->rows_total * h->m;
  if (!h->d_Psi) {
    CK(dalloc(h, (void**)&h->d_Psi, bytes));
    CK(dalloc(h, (void**)&h->d_H, bytes));
  }
  KLA(h, K_ASSEMBLE, 1, 16.0 * h->rows_total * h->m, (double)h->rows_total * h->m * (2 * h->dim + 8), launch_assemble(h->P, h->d_sub, h->d_tiles, h->ntiles, h->d_cov, h->d_R, h->d_b, h->d_Psi, h->d_H, h->st));
  h->assembled = true;
  h->reduced = false;
  h->prec_kind = -1;
  phase_mark(h, 0, 1);
  return RANN_OK;
}

extern "C" rann_status rann_dd_rhs(rann_dd_handle* h, double* F_dev) {
  REQUIRE(h && F_dev, RANN_EINVAL, "null argument");
  KL(h, K_RHS, 1, launch_rhs(h->P, F_dev, h->N, h->st));
  if (h->ph_rec[0]) cudaEventRecord(h->ph_ev[0][1], h->st);    // the assembly phase ends with F
  return RANN_OK;
}

// --------------------------------------------------------------- pca --

static void push_tiles(std::vector<GemmTask>& out, GemmTask t, bool upper) {
  for (int tm = 0; tm < t.M; tm += 64)
    for (int tn = 0; tn < t.N; tn += 64) {
      if (upper && tn + 64 <= tm) continue;
      GemmTask x = t;
      x.tm = tm;
      x.tn = tn;
      out.push_back(x);
    }
}

extern "C" rann_status rann_dd_pca(rann_dd_handle* h, int mode, double thr, int* ranks_host) {
  REQUIRE(h, RANN_EINVAL, "null handle");
  REQUIRE(h->assembled, RANN_EORDER, "pca before assemble");
  REQUIRE(mode >= 0 && mode <= 2, RANN_EINVAL, "bad pca mode");
  REQUIRE(mode == RANN_PCA_NONE || (thr >= 0.0 && std::isfinite(thr)), RANN_EINVAL, "bad threshold");
  // a pca that fails part-way leaves the handle assembled but not reduced
  h->reduced = false;
  h->prec_kind = -1;
  phase_mark(h, 1, 0);
  const int J = h->J, m = h->m;
  const size_t mm = (size_t)m * m;
  if (!h->d_V) {
    CK(dalloc(h, (void**)&h->d_V, sizeof(double) * mm * J));
    CK(dalloc(h, (void**)&h->d_eig, sizeof(double) * (size_t)m * J));
  }
  std::vector<int> info(J, 0), dev_ranks(J, m);
  h->eig_host.assign((size_t)m * J, 0.0);
  h->sumNm2 = 0;
  for (int j = 0; j < J; ++j) h->sumNm2 += (double)h->subs[j].N * m * (m + 1);
  // Gram matrices Psi_j^T Psi_j (upper tiles) then eigen-decomposition
  {
    void* d_tasks = nullptr;
    uint16_t* d_sl = nullptr;
    int* d_e = nullptr;
    if (h->inner_df) {      // digit-slice products on the tensor cores (float64-accurate)
      const int nsl = oz_slices();
      std::vector<OzSplitTask> sp(J);
      std::vector<OzTask> gt;
      int64_t soff = 0;
      int maxKp = 0;
      for (int j = 0; j < J; ++j) {
        const int Kp = oz_kpad(h->subs[j].N);
        soff += (int64_t)nsl * oz_mpad(m) * Kp;
        maxKp = std::max(maxKp, Kp);
      }
      CK(dalloc(h, (void**)&d_sl, sizeof(uint16_t) * (size_t)soff));
      CK(dalloc(h, (void**)&d_e, sizeof(int) * (size_t)m * J));
      soff = 0;
      for (int j = 0; j < J; ++j) {
        const SubDev& S = h->subs[j];
        OzSplitTask& t = sp[j];
        t.X = h->d_Psi + S.row0 * m; t.si = 1; t.sk = m;       // row i of Psi_j^T
        t.M = m; t.K = S.N; t.Kp = oz_kpad(S.N); t.Mp = oz_mpad(m); t.e = d_e + (size_t)m * j; t.out = d_sl + soff;
        OzTask g{};
        g.ia = j; g.ib = j; g.ea = t.e; g.eb = t.e; g.C = h->d_V + mm * j;
        g.M = m; g.N = m; g.Kp = t.Kp; g.ldc = m;
        for (int tm = 0; tm < m; tm += OZ_TILE_M)      // tiles meeting the upper triangle
          for (int tn = tm; tn < m; tn += OZ_TILE_N) { g.tm = tm; g.tn = tn; gt.push_back(g); }
        soff += (int64_t)nsl * t.Mp * t.Kp;
      }
      std::vector<OzMap> maps;
      CK(oz_encode_maps(sp, maps));
      OzSplitTask* d_sp; OzTask* d_gt; OzMap* d_maps;
      CK(dupload(h, &d_sp, sp)); CK(dupload(h, &d_gt, gt)); CK(dupload(h, &d_maps, maps));
      d_tasks = d_gt;
      KLA(h, K_OZ_SPLIT, 2, (8.0 + 2.0 * nsl) * h->rows_total * m, 0,
          launch_oz_split(d_sp, J, m, maxKp, h->st));
      KLA(h, K_GRAM_OZ, 1, 2.0 * nsl * h->rows_total * m, 36.0 * h->sumNm2,
          launch_oz_gemm(d_gt, (int)gt.size(), d_maps, h->d_ozerr, h->st));
      dfree(h, d_sp); dfree(h, d_maps);
    } else {
      std::vector<GemmTask> tasks;
      for (int j = 0; j < J; ++j) {
        const SubDev& S = h->subs[j];
        GemmTask t{};
        t.A = h->d_Psi + S.row0 * m; t.B = t.A; t.C = h->d_V + mm * j;
        t.K = S.N; t.M = m; t.N = m; t.lda = m; t.ldb = m; t.ldc = m;
        push_tiles(tasks, t, true);
      }
      GemmTask* d_gt;
      CK(dupload(h, &d_gt, tasks));
      d_tasks = d_gt;
      KLA(h, K_GRAM, 1, 8.0 * h->rows_total * m, h->sumNm2, launch_gemm_tn(d_gt, (int)tasks.size(), h->st));
    }
    std::vector<double*> mats(J);
    std::vector<int> ns(J, m), lds(J, m);
    for (int j = 0; j < J; ++j) mats[j] = h->d_V + mm * j;
    double** d_mats; int* d_ns; int* d_lds;
    CK(dupload(h, &d_mats, mats)); CK(dupload(h, &d_ns, ns)); CK(dupload(h, &d_lds, lds));
    KL(h, K_SYMM, 1, launch_symmetrize(d_mats, d_ns, d_lds, J, m, h->st));
    double* d_work; int* d_info; int* d_ranks;
    CK(dalloc(h, (void**)&d_work, sizeof(double) * (size_t)syevd_work_doubles(m) * J));
    CK(dalloc(h, (void**)&d_info, sizeof(int) * J));
    CK(dalloc(h, (void**)&d_ranks, sizeof(int) * J));
    // algorithmic flops: tridiagonal reduction 4/3 m^3 per matrix; eigenvalues: the float64 Sturm
    // counts of the bisection (12 per eigenvalue, 3 flops per step; the double-float counts run on the
    // float32 pipe); the eigenvector work depends on p_j and is added below once the ranks are known
    SyevBatch sb{h->d_V, m, J, h->d_eig, d_work, d_info, d_ranks, mode, thr, h->inner_df};
    KLA(h, K_EIG, 1, 24.0 * mm * J, 4.0 / 3.0 * (double)m * mm * J, launch_syev_phase(sb, 0, h->st));
    KLA(h, K_EIG_VAL, 1, 0, h->inner_df ? 36.0 * mm * J : 0.0, launch_syev_phase(sb, 1, h->st));
    KLA(h, K_EIG_VEC, 1, 0, 0, launch_syev_phase(sb, 2, h->st));
    KLA(h, K_EIG_ORTH, 1, 0, 0, launch_syev_phase(sb, 3, h->st));
    KLA(h, K_EIG_BACK, 2, 0, 0, launch_syev_phase(sb, 4, h->st));
    CK(cudaMemcpyAsync(h->eig_host.data(), h->d_eig, sizeof(double) * m * J, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(info.data(), d_info, sizeof(int) * J, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(dev_ranks.data(), d_ranks, sizeof(int) * J, cudaMemcpyDeviceToHost, h->st));
    int ozerr = 0;
    CK(cudaMemcpyAsync(&ozerr, h->d_ozerr, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(stream_sync(h));
    if (ozerr) {
      cudaMemsetAsync(h->d_ozerr, 0, sizeof(int), h->st);
      rann_set_error("tensor-core Gram product: bounded pipeline wait %d gave up", ozerr);
      return RANN_TIMEOUT;
    }
    dfree(h, d_tasks); dfree(h, d_mats); dfree(h, d_ns); dfree(h, d_lds); dfree(h, d_work); dfree(h, d_info);
    dfree(h, d_ranks);
    if (d_sl) { dfree(h, d_sl); dfree(h, d_e); }
  }
  for (int j = 0; j < J; ++j)
    REQUIRE(info[j] == 0, RANN_ECUDA, "eigen-decomposition of subdomain %d did not converge", j);
  if (mode == RANN_PCA_NONE) {   // V = I, p = m
    std::vector<double> I(mm * J, 0.0);
    for (int j = 0; j < J; ++j)
      for (int c = 0; c < m; ++c) I[mm * j + (size_t)c * m + c] = 1.0;
    CK(cudaMemcpyAsync(h->d_V, I.data(), sizeof(double) * I.size(), cudaMemcpyHostToDevice, h->st));
    CK(stream_sync(h));
  }
  // ranks (Sec. 4): sigma_k = sqrt(max(lambda_k, 0))
  int64_t woff = 0, boff = 0;
  int poff = 0;
  h->maxP = 0;
  for (int j = 0; j < J; ++j) {
    // the eigensolver applied the rank rule (it forms only the kept eigenvectors)
    const int p = dev_ranks[j];
    REQUIRE(p >= 1 && p <= m, RANN_ECUDA, "eigensolver returned rank %d for subdomain %d", p, j);
    h->prof.flops[K_EIG_VEC] += 25.0 * (double)m * p;       // tridiagonal LU and two solves
    h->prof.flops[K_EIG_ORTH] += 4.0 * (double)m * p * p;   // two Gram-Schmidt passes
    h->prof.flops[K_EIG_BACK] += 2.0 * (double)m * m * p;   // m - 2 reflectors per vector
    SubDev& S = h->subs[j];
    S.p = p;
    S.P = p + (p & 1);
    S.woff = woff;
    S.boff = boff;
    S.poff = poff;
    woff += p;
    boff += (int64_t)S.N * S.P;
    poff += S.P;
    h->maxP = std::max(h->maxP, S.P);
    if (ranks_host) ranks_host[j] = p;
  }
  h->dof = woff;
  h->sumNp = h->sumNm2 = h->sumNmp = 0;
  for (int j = 0; j < J; ++j) {
    const SubDev& S = h->subs[j];
    h->sumNp += (double)S.N * S.p;
    h->sumNm2 += (double)S.N * m * (m + 1);
    h->sumNmp += (double)S.N * m * S.p;
  }
  if (h->d_B) dfree(h, h->d_B);
  CK(dalloc(h, (void**)&h->d_B, sizeof(double) * (size_t)boff));
  CK(cudaMemsetAsync(h->d_B, 0, sizeof(double) * (size_t)boff, h->st));
  if (h->inner_df) {        // B_j = H_j V_{p_j} from digit slices of H_j and V_{p_j}^T
    const int nsl = oz_slices(), Kp = oz_kpad(m);
    int64_t sumP = 0, srows = 0;          // slice rows: every operand padded to oz_mpad rows
    for (int j = 0; j < J; ++j) { sumP += h->subs[j].p; srows += oz_mpad(h->subs[j].N) + oz_mpad(h->subs[j].p); }
    uint16_t* d_sl; int* d_e;
    const int64_t nrows = h->rows_total + sumP;
    CK(dalloc(h, (void**)&d_sl, sizeof(uint16_t) * (size_t)(nsl * Kp) * (size_t)srows));
    CK(dalloc(h, (void**)&d_e, sizeof(int) * (size_t)nrows));
    std::vector<OzSplitTask> sp(2 * J);
    std::vector<OzTask> gt;
    int64_t vrow = h->rows_total;       // exponents of the V^T operands follow those of H
    int64_t srow = 0;
    int maxM = m;
    for (int j = 0; j < J; ++j) {
      const SubDev& S = h->subs[j];
      OzSplitTask& a = sp[2 * j];
      a.X = h->d_H + S.row0 * m; a.si = m; a.sk = 1;
      a.M = S.N; a.K = m; a.Kp = Kp; a.Mp = oz_mpad(S.N); a.e = d_e + S.row0; a.out = d_sl + (size_t)nsl * Kp * srow;
      srow += a.Mp;
      OzSplitTask& b = sp[2 * j + 1];
      b.X = h->d_V + mm * j; b.si = 1; b.sk = m;                // row c of V_{p_j}^T
      b.M = S.p; b.K = m; b.Kp = Kp; b.Mp = oz_mpad(S.p); b.e = d_e + vrow; b.out = d_sl + (size_t)nsl * Kp * srow;
      srow += b.Mp;
      vrow += S.p;
      maxM = std::max(maxM, S.N);
      OzTask g{};
      g.ia = 2 * j; g.ib = 2 * j + 1; g.ea = a.e; g.eb = b.e; g.C = h->d_B + S.boff;
      g.M = S.N; g.N = S.p; g.Kp = Kp; g.ldc = S.P;
      for (int tm = 0; tm < S.N; tm += OZ_TILE_M)
        for (int tn = 0; tn < S.p; tn += OZ_TILE_N) { g.tm = tm; g.tn = tn; gt.push_back(g); }
    }
    std::vector<OzMap> maps;
    CK(oz_encode_maps(sp, maps));
    OzSplitTask* d_sp; OzTask* d_gt; OzMap* d_maps;
    CK(dupload(h, &d_sp, sp)); CK(dupload(h, &d_gt, gt)); CK(dupload(h, &d_maps, maps));
    KLA(h, K_OZ_SPLIT, 2, (8.0 + 2.0 * nsl) * (double)m * nrows, 0, launch_oz_split(d_sp, 2 * J, maxM, Kp, h->st));
    KLA(h, K_PROJECT_OZ, 1, 2.0 * nsl * (double)m * nrows + 8.0 * h->sumNp, 36.0 * 2.0 * h->sumNmp,
        launch_oz_gemm(d_gt, (int)gt.size(), d_maps, h->d_ozerr, h->st));
    dfree(h, d_sp); dfree(h, d_gt); dfree(h, d_maps); dfree(h, d_sl); dfree(h, d_e);
  } else {
    std::vector<GemmTask> tasks;
    for (int j = 0; j < J; ++j) {
      const SubDev& S = h->subs[j];
      GemmTask t{};
      t.A = h->d_H + S.row0 * m; t.B = h->d_V + mm * j; t.C = h->d_B + S.boff;
      t.K = m; t.M = S.N; t.N = S.p; t.lda = m; t.ldb = m; t.ldc = S.P;
      push_tiles(tasks, t, false);
    }
    GemmTask* d_tasks;
    CK(dupload(h, &d_tasks, tasks));
    KLA(h, K_PROJECT, 1, 8.0 * (h->rows_total * (double)m + h->sumNp), 2.0 * h->sumNmp, launch_gemm_nn(d_tasks, (int)tasks.size(), h->st));
    dfree(h, d_tasks);
  }
  CK(cudaMemcpyAsync(h->d_sub, h->subs.data(), sizeof(SubDev) * J, cudaMemcpyHostToDevice, h->st));
  // H^T row tiles
  std::vector<int> rt, t0(J + 1, 0);
  for (int j = 0; j < J; ++j) {
    t0[j] = (int)rt.size() / 2;
    for (int r0 = 0; r0 < h->subs[j].N; r0 += 256) { rt.push_back(j); rt.push_back(r0); }
  }
  t0[J] = (int)rt.size() / 2;
  h->nrtiles = t0[J];
  std::vector<int> dft, dft0(J + 1, 0);
  for (int j = 0; j < J; ++j) {
    dft0[j] = (int)dft.size() / 2;
    for (int r0 = 0; r0 < h->subs[j].N; r0 += DF_TILE_ROWS) { dft.push_back(j); dft.push_back(r0); }
  }
  dft0[J] = (int)dft.size() / 2;
  h->ndtiles = dft0[J];
  if (h->d_rtiles) {
    dfree(h, h->d_rtiles); dfree(h, h->d_tile0); dfree(h, h->d_part); dfree(h, h->d_yscratch);
    dfree(h, h->d_B2); dfree(h, h->d_x2); dfree(h, h->d_y2);
    dfree(h, h->d_dtiles); dfree(h, h->d_dtile0); dfree(h, h->d_dpart);
  }
  CK(dalloc(h, (void**)&h->d_B2, sizeof(float2) * (size_t)std::max<int64_t>(boff, 1)));
  CK(dalloc(h, (void**)&h->d_x2, sizeof(float2) * (size_t)std::max(poff, 1)));
  CK(dalloc(h, (void**)&h->d_y2, sizeof(float2) * (size_t)std::max<int64_t>(h->rows_total, 1)));
  CK(dupload(h, &h->d_dtiles, dft));
  CK(dupload(h, &h->d_dtile0, dft0));
  CK(dalloc(h, (void**)&h->d_dpart, sizeof(double) * (size_t)std::max(h->ndtiles, 1) * h->maxP));

  KLA(h, K_SPLIT, 1, 16.0 * boff, 0, launch_split(h->d_B, h->d_B2, boff, h->st));
  CK(dupload(h, &h->d_rtiles, rt));
  CK(dupload(h, &h->d_tile0, t0));
  CK(dalloc(h, (void**)&h->d_part, sizeof(double) * (size_t)h->nrtiles * h->maxP));
  CK(dalloc(h, (void**)&h->d_yscratch, sizeof(double) * (size_t)h->N));
  h->reduced = true;
  h->prec_kind = -1;
  phase_mark(h, 1, 1);
  return RANN_OK;
}

// ------------------------------------------------------------ matvecs --

extern "C" rann_status rann_dd_matvec(rann_dd_handle* h, const double* x_dev, double* y_dev) {
  REQUIRE(h && x_dev && y_dev, RANN_EINVAL, "null argument");
  REQUIRE(h->reduced, RANN_EORDER, "matvec before pca");
  KLA(h, K_MATVEC_H, 1, 8.0 * (h->sumNp + h->N + h->dof), 2.0 * h->sumNp, launch_matvec_H2(h->P, h->d_sub, h->d_cov, h->Gmax, h->d_B, x_dev, y_dev, h->N, h->st));
  return RANN_OK;
}

extern "C" rann_status rann_dd_matvec_t(rann_dd_handle* h, const double* y_dev, double* z_dev) {
  REQUIRE(h && y_dev && z_dev, RANN_EINVAL, "null argument");
  REQUIRE(h->reduced, RANN_EORDER, "matvec before pca");
  KLA(h, K_MATVEC_HT, 2, 8.0 * (h->sumNp + h->rows_total + h->dof), 2.0 * h->sumNp, launch_matvec_HT2(h->P, h->d_sub, h->J, h->d_rtiles, h->nrtiles, h->d_tile0, h->d_B, y_dev, h->d_part,
                       z_dev, h->maxP, h->st));
  return RANN_OK;
}

extern "C" rann_status rann_dd_normal_matvec(rann_dd_handle* h, const double* x_dev, double* z_dev) {
  REQUIRE(h && x_dev && z_dev, RANN_EINVAL, "null argument");
  REQUIRE(h->reduced, RANN_EORDER, "matvec before pca");
  KLA(h, K_MATVEC_H, 1, 8.0 * (h->sumNp + h->N + h->dof), 2.0 * h->sumNp, launch_matvec_H2(h->P, h->d_sub, h->d_cov, h->Gmax, h->d_B, x_dev, h->d_yscratch, h->N, h->st));
  KLA(h, K_MATVEC_HT, 2, 8.0 * (h->sumNp + h->rows_total + h->dof), 2.0 * h->sumNp, launch_matvec_HT2(h->P, h->d_sub, h->J, h->d_rtiles, h->nrtiles, h->d_tile0, h->d_B, h->d_yscratch,
                       h->d_part, z_dev, h->maxP, h->st));
  return RANN_OK;
}

// Inner-iteration operator: z = H^T H x with double-float blocks.
// x2 / z2 (optional): double-float splits of x (read instead of x) and of z
// (written), used only on the block-row path (gram_ready).
static rann_status normal_matvec_fast(rann_dd_handle* h, const double* x, double* z, const float2* x2 = nullptr,
                                      float2* z2 = nullptr) {
  if (h->gram_ready) {
    // z_k = sum_l G_kl x_l from the block rows of H^T H
    KLA(h, K_GRAMOP, 1, 8.0 * (h->gram_entries + h->dof), 2.0 * h->gram_entries,
        launch_gram_matvec(h->gram, h->J, h->d_gtile, h->ngtile, h->gram_maxn2, x, z, h->st, x2, z2));
    return RANN_OK;
  }
  // y_j = B_j x_j row by row (per block), then z_j = B_j^T y with y summed over the blocks holding each point
  KLA(h, K_SPLIT, 1, 24.0 * h->dof, 0, launch_split_pad(h->d_sub, h->J, x, h->d_x2, h->st));
  KLA(h, K_MATVEC_H_DF, 1, 8.0 * (h->sumNp + h->rows_total + h->dof), 2.0 * h->sumNp,
      launch_rowdot_df(h->d_sub, h->d_dtiles, h->ndtiles, DF_TILE_ROWS, h->d_B2, h->d_x2, h->d_y2, h->st));
  KLA(h, K_MATVEC_HT_DF, 2, 8.0 * (h->sumNp + 2.0 * h->rows_total + h->dof), 2.0 * h->sumNp,
      launch_matvec_HT_df(h->P, h->d_sub, h->J, h->d_dtiles, h->ndtiles, DF_TILE_ROWS, h->d_dtile0, h->d_cov,
                          h->Gmax, h->d_B2, h->d_y2, h->d_dpart, z, h->maxP, h->st));
  return RANN_OK;
}

// ------------------------------------------------------------ precond --

static bool boxes_meet(const SubDev& a, const SubDev& b, int dim) {
  for (int i = 0; i < dim; ++i)
    if (std::max(a.lo[i], b.lo[i]) >= std::min(a.lo[i] + a.n[i], b.lo[i] + b.n[i])) return false;
  return true;
}

// Block rows R_k = [G_kl]_l of H^T H in double-float from the pair Gram buffer.
static rann_status build_gram_rows(rann_dd_handle* h, const std::vector<int64_t>& pair_off) {
  const int J = h->J;
  const auto& S = h->subs;
  for (int k = 0; k < J; ++k) {     // the row kernel stages at most GRAM_MAX_NBR neighbour segments
    int nq = 0;
    for (int l = 0; l < J; ++l) nq += (k <= l ? pair_off[(size_t)k * J + l] : pair_off[(size_t)l * J + k]) >= 0;
    if (nq > GRAM_MAX_NBR) return RANN_OK;
  }
  std::vector<int> p(J), n2(J), nptr(1, 0), nl, ncol, ntr, poff(J);
  std::vector<int64_t> roff(J), woff(J), noff;
  std::vector<int> gt;
  int64_t ro = 0;
  int maxp = 0, maxn2 = 0;
  h->gram_entries = 0;
  for (int k = 0; k < J; ++k) {
    int col = 0;
    for (int l = 0; l < J; ++l) {
      const int64_t off = k <= l ? pair_off[(size_t)k * J + l] : pair_off[(size_t)l * J + k];
      if (off < 0) continue;
      nl.push_back(l); ncol.push_back(col); noff.push_back(off); ntr.push_back(k > l ? 1 : 0);
      col += S[l].P;
      h->gram_entries += (double)S[k].p * S[l].p;
    }
    nptr.push_back((int)nl.size());
    p[k] = S[k].p;
    n2[k] = col;
    roff[k] = ro; woff[k] = S[k].woff; poff[k] = S[k].poff;
    ro += (int64_t)p[k] * n2[k];
    maxp = std::max(maxp, p[k]);
    maxn2 = std::max(maxn2, n2[k]);
    for (int c0 = 0; c0 < p[k]; c0 += GRAM_TILE_ROWS) { gt.push_back(k); gt.push_back(c0); }
  }
  auto up = [&](auto** dst, const auto& v) -> cudaError_t {
    cudaError_t e = dupload(h, dst, v);
    if (e == cudaSuccess) h->gram_allocs.push_back((void*)*dst);
    return e;
  };
  int *d_p, *d_n2, *d_nptr, *d_nl, *d_ncol, *d_ntr, *d_poff;
  int64_t *d_roff, *d_woff, *d_noff;
  CK(up(&d_p, p)); CK(up(&d_n2, n2)); CK(up(&d_nptr, nptr)); CK(up(&d_nl, nl)); CK(up(&d_ncol, ncol));
  CK(up(&d_ntr, ntr)); CK(up(&d_roff, roff)); CK(up(&d_poff, poff)); CK(up(&d_woff, woff)); CK(up(&d_noff, noff));
  CK(up(&h->d_gtile, gt));
  h->ngtile = (int)gt.size() / 2;
  h->gram_maxn2 = maxn2;
  float2* d_R2;
  CK(dalloc(h, (void**)&d_R2, sizeof(float2) * (size_t)std::max<int64_t>(ro, 2)));
  h->gram_allocs.push_back(d_R2);
  h->gram = GramRows{d_p, d_n2, d_roff, d_poff, d_woff, d_nptr, d_nl, d_ncol, d_noff, d_ntr, d_R2};
  KLA(h, K_GRAMROWS, 1, 16.0 * (double)ro, 0, launch_gramrows_build(h->gram, h->d_pairbuf, J, maxp, maxn2, h->st));
  h->gram_ready = true;
  return RANN_OK;
}

// ------------------------------------------------ Schwarz apply configurations --
// 0: the fused 32-row-block kernel (precision mode 1, sets of up to 27 subdomains);
// c >= 1: the streaming kernel with chunks of about 1/APPLY_CHUNKS[c] of an SM's
// share of the triangles' entries (sets of up to schwarz_rows_nmax() unknowns).
static const int APPLY_CHUNKS[RANN_APPLY_NCFG] = {0, 6, 12, 24};

static bool streaming_ok(const rann_dd_handle* h) {
  return h->prec_df && h->maxn <= schwarz_rows_nmax() && h->max_set_size <= schwarz_apply_max_subs();
}

static rann_status set_apply_config(rann_dd_handle* h, int cfg) {
  REQUIRE(cfg >= 0 && cfg < RANN_APPLY_NCFG, RANN_EINVAL, "apply configuration %d out of range", cfg);
  REQUIRE(cfg == 0 || streaming_ok(h), RANN_EINVAL,
          "streaming apply needs precision mode 1 and sets of at most %d unknowns", schwarz_rows_nmax());
  for (void* p : {(void*)h->d_sr_chunks, (void*)h->d_sr_order, (void*)h->d_sr_ckptr, (void*)h->d_sr_part}) dfree(h, p);
  h->d_sr_chunks = nullptr; h->d_sr_order = nullptr; h->d_sr_ckptr = nullptr; h->d_sr_part = nullptr;
  h->sr_nchunks = 0;
  h->apply_cfg = 0;
  if (cfg > 0) {
    int64_t tri = 0;
    for (int n : h->set_n) tri += (int64_t)n * (n + 1) / 2;
    const int64_t target = std::max<int64_t>(65536, tri / ((int64_t)h->nsm * APPLY_CHUNKS[cfg]));
    std::vector<SrChunk> chunks;
    std::vector<int> ck_ptr, order;
    int64_t ptot = 0;
    schwarz_rows_plan(h->set_n, target, chunks, ck_ptr, order, ptot);
    CK(dupload(h, &h->d_sr_chunks, chunks));
    CK(dupload(h, &h->d_sr_order, order));
    CK(dupload(h, &h->d_sr_ckptr, ck_ptr));
    CK(dalloc(h, (void**)&h->d_sr_part, sizeof(double) * (size_t)std::max<int64_t>(ptot, 1)));
    h->sr_nchunks = (int)chunks.size();
  }
  h->apply_cfg = cfg;
  return RANN_OK;
}

extern "C" rann_status rann_dd_setup_precond(rann_dd_handle* h, int kind, int overlap_level) {
  REQUIRE(h, RANN_EINVAL, "null handle");
  REQUIRE(h->reduced, RANN_EORDER, "setup_precond before pca");
  REQUIRE(kind >= RANN_PREC_NONE && kind <= RANN_PREC_RAS, RANN_EINVAL, "bad preconditioner kind");
  REQUIRE(overlap_level == 0 || overlap_level == 1, RANN_EINVAL, "overlap_level must be 0 or 1");
  // release a previous setup
  for (void* p : {(void*)h->d_mats, (void*)h->d_set_ptr, (void*)h->d_set_sub, (void*)h->d_inc_ptr,
                  (void*)h->d_inc_set, (void*)h->d_inc_pos, (void*)h->d_s_off, (void*)h->d_s,
                  (void*)h->d_Amats, (void*)h->d_Xmats, (void*)h->d_g, (void*)h->d_y, (void*)h->d_tpart,
                  (void*)h->d_p_off, (void*)h->d_X2mats, (void*)h->d_g2, (void*)h->d_ys2, (void*)h->d_A2mats,
                  (void*)h->d_p_off32, (void*)h->d_tpart32, (void*)h->d_adone, (void*)h->d_sr_chunks,
                  (void*)h->d_sr_order, (void*)h->d_sr_ckptr, (void*)h->d_sr_part})
    dfree(h, p);
  h->d_adone = nullptr;
  h->d_sr_chunks = nullptr; h->d_sr_order = nullptr; h->d_sr_ckptr = nullptr; h->d_sr_part = nullptr;
  h->sr_nchunks = 0;
  h->d_mats = nullptr; h->d_Amats = nullptr; h->d_Xmats = nullptr; h->d_X2mats = nullptr; h->d_A2mats = nullptr;
  for (void* p : h->gram_allocs) dfree(h, p);
  h->gram_allocs.clear();
  h->gram_ready = false;
  h->n_shifted = 0;
  h->prec_kind = -1;            // set once the set-up has succeeded
  if (kind == RANN_PREC_NONE) {
    h->prec_kind = kind;
    return RANN_OK;
  }
  phase_mark(h, 2, 0);
  const int J = h->J, dim = h->dim;
  const auto& S = h->subs;
  // extended sets N(i)
  h->set_ptr.assign(1, 0);
  h->set_sub.clear();
  for (int i = 0; i < J; ++i) {
    for (int k = 0; k < J; ++k)
      if (overlap_level == 0 ? k == i : boxes_meet(S[i], S[k], dim)) h->set_sub.push_back(k);
    h->set_ptr.push_back((int)h->set_sub.size());
  }
  h->nsets = J;
  h->max_set_size = 0;
  for (int i = 0; i < J; ++i) h->max_set_size = std::max(h->max_set_size, h->set_ptr[i + 1] - h->set_ptr[i]);
  // neighbour pairs (k <= l whose boxes share points) and their Gram blocks B_k^T B_l
  std::vector<int64_t> pair_off((size_t)J * J, -1);
  std::vector<GemmTask> tasks;
  std::vector<int> ridx;
  std::vector<std::pair<int64_t, int64_t>> ridx_ranges;   // (start in ridx for A rows, for B rows)
  int64_t pbuf = 0;
  std::vector<std::pair<int, int>> pairs;
  // every pair of boxes that meet (the blocks of H^T H; the local matrices A_i use those inside N(i))
  for (int k = 0; k < J; ++k)
    for (int l = k; l < J; ++l) {
      if (!boxes_meet(S[k], S[l], dim)) continue;
      pair_off[(size_t)k * J + l] = pbuf;
      pbuf += (int64_t)S[k].p * S[l].p;
      pairs.push_back({k, l});
    }
  for (auto& pr : pairs) {
    const SubDev &a = S[pr.first], &b = S[pr.second];
    int lo[3], hi[3];
    for (int i = 0; i < 3; ++i) {
      lo[i] = std::max(a.lo[i], b.lo[i]);
      hi[i] = std::min(a.lo[i] + a.n[i], b.lo[i] + b.n[i]);
    }
    int64_t startA = (int64_t)ridx.size();
    std::vector<int> rb;
    for (int q2 = lo[2]; q2 < hi[2]; ++q2)
      for (int q1 = lo[1]; q1 < hi[1]; ++q1)
        for (int q0 = lo[0]; q0 < hi[0]; ++q0) {
          ridx.push_back((q0 - a.lo[0]) + a.n[0] * ((q1 - a.lo[1]) + a.n[1] * (q2 - a.lo[2])));
          rb.push_back((q0 - b.lo[0]) + b.n[0] * ((q1 - b.lo[1]) + b.n[1] * (q2 - b.lo[2])));
        }
    int64_t startB = (int64_t)ridx.size();
    ridx.insert(ridx.end(), rb.begin(), rb.end());
    ridx_ranges.push_back({startA, startB});
  }
  h->pair_flops = 0;
  for (size_t t = 0; t < pairs.size(); ++t)
    h->pair_flops += 2.0 * (double)(ridx_ranges[t].second - ridx_ranges[t].first) * S[pairs[t].first].p *
                     S[pairs[t].second].p;
  int* d_ridx;
  CK(dupload(h, &d_ridx, ridx));
  CK(dalloc(h, (void**)&h->d_pairbuf, sizeof(double) * (size_t)std::max<int64_t>(pbuf, 1)));
  if (h->inner_df) {
    // G_kl from digit slices of the gathered operands on the tensor cores (float64-accurate);
    // a diagonal pair splits its one operand once
    const int nsl = oz_slices();
    std::vector<OzSplitTask> sp;
    std::vector<int> spa(pairs.size()), spb(pairs.size());
    int64_t soff = 0, eoff = 0;
    int maxM = 1, maxKp = 32;
    auto operand = [&](int k, int64_t start, int K) {
      OzSplitTask o{};
      o.X = h->d_B + S[k].boff; o.si = 1; o.sk = S[k].P;
      o.gather = d_ridx + start;
      o.M = S[k].p; o.K = K; o.Kp = oz_kpad(K); o.Mp = oz_mpad(o.M);
      o.e = reinterpret_cast<int*>(eoff);                    // patched below
      o.out = reinterpret_cast<uint16_t*>(soff);
      soff += (int64_t)nsl * o.Mp * o.Kp;
      eoff += o.M;
      maxM = std::max(maxM, o.M);
      maxKp = std::max(maxKp, o.Kp);
      sp.push_back(o);
      return (int)sp.size() - 1;
    };
    for (size_t t = 0; t < pairs.size(); ++t) {
      const int K = (int)(ridx_ranges[t].second - ridx_ranges[t].first);
      spa[t] = operand(pairs[t].first, ridx_ranges[t].first, K);
      spb[t] = pairs[t].first == pairs[t].second ? spa[t] : operand(pairs[t].second, ridx_ranges[t].second, K);
    }
    uint16_t* d_sl; int* d_e;
    CK(dalloc(h, (void**)&d_sl, sizeof(uint16_t) * (size_t)std::max<int64_t>(soff, 1)));
    CK(dalloc(h, (void**)&d_e, sizeof(int) * (size_t)std::max<int64_t>(eoff, 1)));
    for (auto& o : sp) {
      o.e = d_e + reinterpret_cast<int64_t>(o.e);
      o.out = d_sl + reinterpret_cast<int64_t>(o.out);
    }
    std::vector<OzTask> gt;
    for (size_t t = 0; t < pairs.size(); ++t) {
      const OzSplitTask &a = sp[spa[t]], &b = sp[spb[t]];
      OzTask g{};
      g.ia = spa[t]; g.ib = spb[t]; g.ea = a.e; g.eb = b.e;
      g.C = h->d_pairbuf + pair_off[(size_t)pairs[t].first * J + pairs[t].second];
      g.M = a.M; g.N = b.M; g.Kp = a.Kp; g.ldc = b.M;
      for (int tm = 0; tm < g.M; tm += OZ_TILE_M)
        for (int tn = 0; tn < g.N; tn += OZ_TILE_N) { g.tm = tm; g.tn = tn; gt.push_back(g); }
    }
    std::vector<OzMap> maps;
    CK(oz_encode_maps(sp, maps));
    OzSplitTask* d_sp; OzTask* d_gt; OzMap* d_maps;
    CK(dupload(h, &d_sp, sp)); CK(dupload(h, &d_gt, gt)); CK(dupload(h, &d_maps, maps));
    double split_entries = 0;
    for (auto& o : sp) split_entries += (double)o.M * o.K;
    KLA(h, K_OZ_SPLIT, 2, (8.0 + 2.0 * nsl) * split_entries, 0,
        launch_oz_split(d_sp, (int)sp.size(), maxM, maxKp, h->st));
    KLA(h, K_PAIRGRAM_OZ, 1, 2.0 * nsl * split_entries, 36.0 * h->pair_flops,
        launch_oz_gemm(d_gt, (int)gt.size(), d_maps, h->d_ozerr, h->st));
    dfree(h, d_sp); dfree(h, d_gt); dfree(h, d_maps); dfree(h, d_sl); dfree(h, d_e);
  } else {
    for (size_t t = 0; t < pairs.size(); ++t) {
      const SubDev &a = S[pairs[t].first], &b = S[pairs[t].second];
      GemmTask g{};
      g.A = h->d_B + a.boff;
      g.B = h->d_B + b.boff;
      g.C = h->d_pairbuf + pair_off[(size_t)pairs[t].first * J + pairs[t].second];
      g.ia = d_ridx + ridx_ranges[t].first;
      g.ib = d_ridx + ridx_ranges[t].second;
      g.K = (int)(ridx_ranges[t].second - ridx_ranges[t].first);
      g.M = a.p; g.N = b.p; g.lda = a.P; g.ldb = b.P; g.ldc = b.p;
      push_tiles(tasks, g, false);
    }
    GemmTask* d_tasks;
    CK(dupload(h, &d_tasks, tasks));
    KLA(h, K_PAIRGRAM, 1, 0, h->pair_flops, launch_gemm_tn(d_tasks, (int)tasks.size(), h->st));
    dfree(h, d_tasks);
  }
  if (h->inner_df) TRY(build_gram_rows(h, pair_off));
  // local matrices A_i: table of block sources
  std::vector<CholMat> mats(J);
  std::vector<int64_t> tab;      // per (i, a, b): pair offset, or -1; sign bit 1<<62 marks transpose
  std::vector<int> tab_ptr(1, 0), boffs, boff_ptr(1, 0);
  int64_t aoff = 0;
  h->maxn = 0;
  std::vector<int64_t> s_off(J + 1, 0);
  for (int i = 0; i < J; ++i) {
    int n = 0;
    for (int q = h->set_ptr[i]; q < h->set_ptr[i + 1]; ++q) { boffs.push_back(n); n += S[h->set_sub[q]].p; }
    boffs.push_back(n);
    boff_ptr.push_back((int)boffs.size());
    mats[i].n = n; mats[i].ld = (n + 3) & ~3;       // rows start 32-byte aligned in double-float
    mats[i].A = reinterpret_cast<double*>(aoff);   // patched below
    aoff += (int64_t)n * mats[i].ld;
    s_off[i + 1] = s_off[i] + n;
    h->maxn = std::max(h->maxn, n);
    for (int q = h->set_ptr[i]; q < h->set_ptr[i + 1]; ++q)
      for (int q2 = h->set_ptr[i]; q2 < h->set_ptr[i + 1]; ++q2) {
        int k = h->set_sub[q], l = h->set_sub[q2];
        int64_t off = k <= l ? pair_off[(size_t)k * J + l] : pair_off[(size_t)l * J + k];
        if (off >= 0 && k > l) off |= (int64_t)1 << 62;
        tab.push_back(off);
      }
    tab_ptr.push_back((int)tab.size());
  }
  // precision mode 1 keeps A_i, L_i and L_i^{-1} in double-float only
  h->prec_df = h->inner_df != 0;
  if (h->prec_df) {
    CK(dalloc(h, (void**)&h->d_A2mats, sizeof(float2) * (size_t)std::max<int64_t>(aoff, 1)));
  } else {
    CK(dalloc(h, (void**)&h->d_Amats, sizeof(double) * (size_t)std::max<int64_t>(aoff, 1)));
    CK(dalloc(h, (void**)&h->d_Xmats, sizeof(double) * (size_t)std::max<int64_t>(aoff, 1)));
  }
  CK(dalloc(h, (void**)&h->d_X2mats, sizeof(float2) * (size_t)std::max<int64_t>(aoff, 1)));
  // the factorisations write only the lower triangles of L_i^{-1}; the streaming apply reads the
  // entry just above the diagonal of even rows (its 16-byte copies) and relies on it being zero
  CK(cudaMemsetAsync(h->d_X2mats, 0, sizeof(float2) * (size_t)std::max<int64_t>(aoff, 1), h->st));
  h->sum_n = h->sum_n2 = h->sum_n3 = 0;
  for (int i = 0; i < J; ++i) {
    const double n = mats[i].n;
    h->sum_n += n; h->sum_n2 += n * n; h->sum_n3 += n * n * n;
  }
  for (int i = 0; i < J; ++i) {
    const int64_t o = reinterpret_cast<int64_t>(mats[i].A);
    mats[i].X2 = h->d_X2mats + o;
    if (h->prec_df) {
      mats[i].A2 = h->d_A2mats + o;
      mats[i].A = nullptr;
      mats[i].X = nullptr;
    } else {
      mats[i].A2 = nullptr;
      mats[i].A = h->d_Amats + o;
      mats[i].X = h->d_Xmats + o;
    }
  }
  int64_t* d_tab; int *d_tab_ptr, *d_boffs, *d_boff_ptr; double* d_dmax; int* d_fail;
  CK(dupload(h, &d_tab, tab)); CK(dupload(h, &d_tab_ptr, tab_ptr));
  CK(dupload(h, &d_boffs, boffs)); CK(dupload(h, &d_boff_ptr, boff_ptr));
  CK(dupload(h, &h->d_mats, mats));
  CK(dalloc(h, (void**)&d_dmax, sizeof(double) * J));
  CK(dalloc(h, (void**)&d_fail, sizeof(int) * J));
  KLA(h, K_LOCALASM, 2, 8.0 * h->sum_n2, 0, launch_assemble_local(h->d_pairbuf, d_tab, d_tab_ptr, d_boffs, d_boff_ptr, h->d_mats, J, h->maxn, d_dmax, h->st));
  // Cholesky with shift-and-retry for failed pivots: the first attempt factors
  // all J matrices; a retry reassembles only the failed ones, adds a growing
  // diagonal shift and refactors them alone (a compacted matrix list with its
  // own failure flags and diagonal maxima).  The largest diagonal entries
  // stay on the device and reach the host only when a shift is needed.
  std::vector<double> dmax;
  std::vector<int> shifted(J, 0);
  std::vector<int> active(J);
  for (int i = 0; i < J; ++i) active[i] = i;
  const CholMat* d_act = h->d_mats;
  const double* d_act_dmax = d_dmax;
  int act_maxn = h->maxn;
  std::vector<void*> retry_allocs;
  struct Frees {
    rann_dd_handle* h; std::vector<void*>* v;
    ~Frees() { for (void* p : *v) dfree(h, p); }
  } frees{h, &retry_allocs};
  std::vector<void*> tc_allocs;          // work areas of one big-panel attempt
  struct Frees2 {
    rann_dd_handle* h; std::vector<void*>* v;
    ~Frees2() { for (void* p : *v) dfree(h, p); }
  } frees2{h, &tc_allocs};
  for (int attempt = 0; attempt < 6; ++attempt) {
    const int nact = (int)active.size();
    double chol_flops = 0.0, inv_flops = 0.0;
    for (int i : active) {
      const double n = mats[i].n;
      chol_flops += n * n * n / 3.0;
      inv_flops += n * n * n / 3.0;
    }
    CK(cudaMemsetAsync(d_fail, 0, sizeof(int) * J, h->st));
    if (h->prec_df) {
      if (!h->st_la) {
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CK(cudaStreamCreateWithPriority(&h->st_la, cudaStreamNonBlocking, greatest));
        CK(cudaStreamCreateWithPriority(&h->st_inv, cudaStreamNonBlocking, least));
        for (cudaEvent_t& e : h->ev_la) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      }
      int nl = 0;
      if (act_maxn >= TC_MIN_N) {
        // big panels with the trailing updates and the inverse's products on the tensor cores
        std::vector<CholMat> am;
        for (int i : active) am.push_back(mats[i]);
        CholTcPlan plan;
        CK(chol_tc_build(am, plan, nullptr, nullptr, nullptr, nullptr));
        uint16_t *l21a, *l21b, *invb, *xib;
        int* eb;
        CK(dalloc(h, (void**)&l21a, 2 * (size_t)std::max<int64_t>(plan.l21_elems, 8)));
        CK(dalloc(h, (void**)&l21b, 2 * (size_t)std::max<int64_t>(plan.l21_elems, 8)));
        CK(dalloc(h, (void**)&invb, 2 * (size_t)std::max<int64_t>(plan.inv_elems, 8)));
        CK(dalloc(h, (void**)&xib, 2 * (size_t)std::max<int64_t>(plan.xi_elems, 8)));
        CK(dalloc(h, (void**)&eb, 4 * (size_t)std::max<int64_t>(plan.e_ints, 1)));
        for (void* p : {(void*)l21a, (void*)l21b, (void*)invb, (void*)xib, (void*)eb}) tc_allocs.push_back(p);
        uint16_t* const l21[2] = {l21a, l21b};
        CK(chol_tc_build(am, plan, l21, invb, xib, eb));
        OzSplitTask* d_split; OzGroup* d_groups; OzMap* d_maps;
        CK(dupload(h, &d_split, plan.split)); CK(dupload(h, &d_groups, plan.groups)); CK(dupload(h, &d_maps, plan.maps));
        for (void* p : {(void*)d_split, (void*)d_groups, (void*)d_maps}) tc_allocs.push_back(p);
        for (const CholMat& M : am)        // the inverse accumulates in X2 and reads its upper triangles as zeros
          CK(cudaMemsetAsync(M.X2, 0, sizeof(float2) * (size_t)M.n * M.ld, h->st));
        KLA(h, K_CHOL_TC, nl, 0, plan.flops,
            chol_tc_enqueue(plan, d_act, nact, d_fail, d_act_dmax, d_split, d_groups, d_maps, h->d_ozerr, h->st,
                            h->st_inv, &nl));
      } else {
        KLA(h, K_CHOL, nl, 0, chol_flops + inv_flops,
            launch_chol_df_lookahead(d_act, nact, act_maxn, d_fail, d_act_dmax, h->st, h->st_la, h->st_inv, h->ev_la,
                                     &nl));
      }
    } else {
      for (int c0 = 0; c0 < act_maxn; c0 += 32)
        KLA(h, K_CHOL, (act_maxn - c0 > 32) ? 3 : 1, 0, c0 == 0 ? chol_flops : 0.0,
            launch_chol_step(d_act, nact, act_maxn, c0, d_fail, d_act_dmax, h->st));
      KLA(h, K_TRTRI, 2, 0, inv_flops, launch_trtri(d_act, nact, act_maxn, h->st));
      KLA(h, K_SPLIT, 1, 6.0 * h->sum_n2, 0, launch_split_lower(d_act, nact, act_maxn, h->st));
    }
    std::vector<int> f(nact);
    int ozerr = 0;
    CK(cudaMemcpyAsync(f.data(), d_fail, sizeof(int) * nact, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&ozerr, h->d_ozerr, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(stream_sync(h));
    for (void* p : tc_allocs) dfree(h, p);
    tc_allocs.clear();
    if (ozerr) {
      cudaMemsetAsync(h->d_ozerr, 0, sizeof(int), h->st);
      rann_set_error("tensor-core product (pair Gram / local factors): bounded pipeline wait %d gave up", ozerr);
      return RANN_TIMEOUT;
    }
    std::vector<int> next;
    for (int q = 0; q < nact; ++q) if (f[q]) next.push_back(active[q]);
    if (next.empty()) break;
    if (attempt == 5) { rann_set_error("local Cholesky failed after shifts"); return RANN_ECUDA; }
    if (dmax.empty()) {
      dmax.resize(J);
      CK(cudaMemcpyAsync(dmax.data(), d_dmax, sizeof(double) * J, cudaMemcpyDeviceToHost, h->st));
      CK(stream_sync(h));
    }
    // reassemble the failed matrices and add a growing diagonal shift
    std::vector<CholMat> fm;
    std::vector<int> which, widx;
    std::vector<double> shift, fdmax;
    act_maxn = 0;
    for (int i : next) {
      shifted[i] = 1;
      widx.push_back((int)fm.size());
      fm.push_back(mats[i]);
      which.push_back(i);
      shift.push_back(dmax[i] * std::pow(10.0, -14 + 2 * attempt));
      fdmax.push_back(dmax[i]);
      act_maxn = std::max(act_maxn, mats[i].n);
    }
    int* d_which; CholMat* d_fm; int* d_widx; double* d_shift; double* d_fdmax;
    CK(dupload(h, &d_which, which)); CK(dupload(h, &d_fm, fm)); CK(dupload(h, &d_widx, widx));
    CK(dupload(h, &d_shift, shift)); CK(dupload(h, &d_fdmax, fdmax));
    for (void* p : {(void*)d_which, (void*)d_fm, (void*)d_widx, (void*)d_shift, (void*)d_fdmax}) retry_allocs.push_back(p);
    double s2 = 0.0;
    for (int i : next) s2 += (double)mats[i].n * mats[i].n;
    KLA(h, K_LOCALASM, 2, 8.0 * s2, 0, launch_assemble_local(h->d_pairbuf, d_tab, d_tab_ptr, d_boffs, d_boff_ptr,
                                                             h->d_mats, (int)next.size(), act_maxn, d_dmax, h->st,
                                                             d_which));
    KL(h, K_ADDDIAG, 1, launch_add_diag(d_fm, d_widx, (int)next.size(), d_shift, act_maxn, h->st));
    active = next;
    d_act = d_fm;
    d_act_dmax = d_fdmax;
  }
  for (int i = 0; i < J; ++i) h->n_shifted += shifted[i];
  // (X_i = L_i^{-1} for the parallel apply was formed with each factorisation attempt)
  std::vector<int64_t> p_off(J + 1, 0);
  for (int i = 0; i < J; ++i) p_off[i + 1] = p_off[i] + (int64_t)((mats[i].n + 255) / 256) * mats[i].n;
  CK(dupload(h, &h->d_p_off, p_off));
  CK(dalloc(h, (void**)&h->d_tpart, sizeof(double) * (size_t)std::max<int64_t>(p_off[J], 1)));
  {
    const int ar = schwarz_apply_rows();
    std::vector<int64_t> p32(J + 1, 0);
    for (int i = 0; i < J; ++i) p32[i + 1] = p32[i] + (int64_t)((mats[i].n + ar - 1) / ar) * mats[i].n;
    CK(dupload(h, &h->d_p_off32, p32));
    h->p32_total = p32[J];
    CK(dalloc(h, (void**)&h->d_tpart32, sizeof(double) * (size_t)std::max<int64_t>(p32[J], 1)));
    CK(dalloc(h, (void**)&h->d_adone, sizeof(int) * (size_t)J));
    CK(cudaMemsetAsync(h->d_adone, 0, sizeof(int) * (size_t)J, h->st));
  }
  h->set_n.resize(J);
  for (int i = 0; i < J; ++i) h->set_n[i] = mats[i].n;
  // default Schwarz apply: the streaming kernel for sets of 2048 unknowns and more (long rows), the
  // fused 32-row kernel below; rann_dd_tune_apply times them all
  TRY(set_apply_config(h, streaming_ok(h) && h->maxn >= 2048 ? 2 : 0));
  // incidence lists for the combine step: sets containing each subdomain, with its block offset
  std::vector<int> inc_ptr(1, 0), inc_set, inc_pos;
  for (int k = 0; k < J; ++k) {
    for (int i = 0; i < J; ++i) {
      int pos = 0;
      for (int q = h->set_ptr[i]; q < h->set_ptr[i + 1]; ++q) {
        if (h->set_sub[q] == k) { inc_set.push_back(i); inc_pos.push_back(pos); }
        pos += S[h->set_sub[q]].p;
      }
    }
    inc_ptr.push_back((int)inc_set.size());
  }
  CK(dupload(h, &h->d_set_ptr, h->set_ptr)); CK(dupload(h, &h->d_set_sub, h->set_sub));
  for (int k = 0; k < J; ++k)
    REQUIRE(inc_ptr[k + 1] - inc_ptr[k] <= 64, RANN_EINVAL, "subdomain %d lies in more than 64 extended sets", k);
  CK(dupload(h, &h->d_inc_ptr, inc_ptr)); CK(dupload(h, &h->d_inc_set, inc_set)); CK(dupload(h, &h->d_inc_pos, inc_pos));
  CK(dupload(h, &h->d_s_off, s_off));
  CK(dalloc(h, (void**)&h->d_s, sizeof(double) * (size_t)std::max<int64_t>(s_off[J], 1)));
  h->s_total = s_off[J];
  CK(dalloc(h, (void**)&h->d_g, sizeof(double) * (size_t)std::max<int64_t>(s_off[J], 1)));
  CK(dalloc(h, (void**)&h->d_y, sizeof(double) * (size_t)std::max<int64_t>(s_off[J], 1)));
  CK(dalloc(h, (void**)&h->d_g2, sizeof(float2) * (size_t)std::max<int64_t>(s_off[J], 1)));
  CK(dalloc(h, (void**)&h->d_ys2, sizeof(float2) * (size_t)std::max<int64_t>(s_off[J], 1)));
  dfree(h, d_ridx); dfree(h, d_tab); dfree(h, d_tab_ptr); dfree(h, d_boffs); dfree(h, d_boff_ptr);
  dfree(h, d_dmax); dfree(h, d_fail); dfree(h, h->d_pairbuf);
  h->d_pairbuf = nullptr;
  // the applies read L_i^{-1} with each column pair's high parts first
  if (h->prec_df) KLA(h, K_SPLIT, 1, 8.0 * (h->sum_n2 + h->sum_n), 0, launch_x2_pairs(h->d_mats, J, h->maxn, h->st));
  phase_mark(h, 2, 1);
  CK(stream_sync(h));
  h->prec_kind = kind;
  return h->n_shifted ? RANN_LOCAL_SINGULAR : RANN_OK;
}

// z = M^{-1} r, or with transpose z = M^{-T} r = sum_i R_i^T A_i^{-1} D_i R_i r
// (D_i moves to the gather, the combine sums unweighted).
static rann_status prec_apply(rann_dd_handle* h, const double* r, double* z, bool fast = false,
                              bool transpose = false, const float2* r2 = nullptr) {
  if (h->prec_kind == RANN_PREC_NONE) {
    CK(cudaMemcpyAsync(z, r, sizeof(double) * h->dof, cudaMemcpyDeviceToDevice, h->st));
    return RANN_OK;
  }
  const int wkind = transpose ? h->prec_kind : RANN_PREC_AS;
  const int ckind = transpose ? RANN_PREC_AS : h->prec_kind;
  if (fast && h->max_set_size > schwarz_apply_max_subs()) {   // the fused kernel stages a bounded set
    KLA(h, K_GATHER_DF, 1, 16.0 * h->sum_n, 0,
        launch_schwarz_gather_df(h->nsets, h->d_set_ptr, h->d_set_sub, h->d_sub, h->d_s_off, r, h->d_g2, wkind,
                                 h->d_inc_ptr, h->st));
    KLA(h, K_TRMV_L_DF, 1, 4.0 * (h->sum_n2 + h->sum_n) + 16.0 * h->sum_n, h->sum_n2 + h->sum_n,
        launch_trmv_lower_df(h->d_mats, h->nsets, h->maxn, h->d_s_off, h->d_g2, h->d_ys2, h->st));
    KLA(h, K_TRMV_U_DF, 2, 4.0 * (h->sum_n2 + h->sum_n) + 16.0 * h->sum_n, h->sum_n2 + h->sum_n,
        launch_trmv_upper_df(h->d_mats, h->nsets, h->maxn, h->d_s_off, h->d_p_off, h->d_ys2, h->d_tpart, h->d_s,
                             h->st));
  } else if (fast && h->sr_nchunks > 0) {
    // s_i = X_i^T X_i R_i r, the rows of X_i = L_i^{-1} streamed through shared memory once
    KLA(h, K_SCHWARZ_DF, 1, 4.0 * (h->sum_n2 + h->sum_n) + 8.0 * h->sum_n + 8.0 * h->dof,
        2.0 * (h->sum_n2 + h->sum_n),
        launch_schwarz_apply_rows_df(h->d_mats, h->d_sr_chunks, h->d_sr_order, h->sr_nchunks, h->d_sr_ckptr,
                                     h->d_set_ptr, h->d_set_sub, h->d_sub, r, r2, wkind, h->d_inc_ptr, h->d_sr_part,
                                     h->d_s_off, h->d_s, h->d_adone, ckind, z, h->d_ozerr, h->st));
    if (ckind == RANN_PREC_RAS) return RANN_OK;                // the restricted combine ran in the apply
  } else if (fast) {
    // s_i = X_i^T X_i R_i r with X_i = L_i^{-1} read from HBM once (fused, with the gather)
    KLA(h, K_SCHWARZ_DF, 1, 4.0 * (h->sum_n2 + h->sum_n) + 8.0 * h->sum_n + 8.0 * h->dof,
        2.0 * (h->sum_n2 + h->sum_n),
        launch_schwarz_apply_df(h->d_mats, h->nsets, h->maxn, h->d_set_ptr, h->d_set_sub, h->d_sub, r, h->d_s_off,
                                h->d_p_off32, h->d_tpart32, h->d_s, h->d_adone, wkind, h->d_inc_ptr, ckind, z,
                                h->st, r2));
    if (ckind == RANN_PREC_RAS) return RANN_OK;                // the restricted combine ran in the apply
  }
  if (fast) {
    KLA(h, K_COMBINE, 1, 8.0 * (h->sum_n + h->dof), 0, launch_schwarz_combine(h->d_sub, h->J, h->d_inc_ptr,
        h->d_inc_set, h->d_inc_pos, h->d_s_off, h->d_s, ckind, z, h->st));
    return RANN_OK;
  }
  KLA(h, K_GATHER, 1, 16.0 * h->sum_n, 0, launch_schwarz_gather(h->nsets, h->d_set_ptr, h->d_set_sub, h->d_sub,
                                                                 h->d_s_off, r, h->d_g, wkind, h->d_inc_ptr, h->st));
  KLA(h, K_TRMV_L, 1, 4.0 * (h->sum_n2 + h->sum_n) + 16.0 * h->sum_n, h->sum_n2 + h->sum_n, launch_trmv_lower(h->d_mats, h->nsets, h->maxn, h->d_s_off, h->d_g, h->d_y, h->st));
  KLA(h, K_TRMV_U, 2, 4.0 * (h->sum_n2 + h->sum_n) + 16.0 * h->sum_n, h->sum_n2 + h->sum_n, launch_trmv_upper(h->d_mats, h->nsets, h->maxn, h->d_s_off, h->d_p_off, h->d_y, h->d_tpart, h->d_s, h->st));
  KLA(h, K_COMBINE, 1, 8.0 * (h->sum_n + h->dof), 0, launch_schwarz_combine(h->d_sub, h->J, h->d_inc_ptr, h->d_inc_set, h->d_inc_pos, h->d_s_off, h->d_s,
                            ckind, z, h->st));
  return RANN_OK;
}

extern "C" rann_status rann_dd_set_apply_config(rann_dd_handle* h, int cfg) {
  REQUIRE(h, RANN_EINVAL, "null handle");
  REQUIRE(h->prec_kind >= 0, RANN_EORDER, "set_apply_config before setup_precond");
  return set_apply_config(h, cfg);
}

extern "C" rann_status rann_dd_get_apply_config(rann_dd_handle* h, int* cfg) {
  REQUIRE(h && cfg, RANN_EINVAL, "null argument");
  *cfg = h->apply_cfg;
  return RANN_OK;
}

static const float TUNE_MARGIN = 0.1f;

extern "C" rann_status rann_dd_tune_apply(rann_dd_handle* h, int reps, int* best_out, float* ms_out) {
  REQUIRE(h && best_out, RANN_EINVAL, "null argument");
  REQUIRE(h->prec_kind >= 0, RANN_EORDER, "tune_apply before setup_precond");
  REQUIRE(reps >= 1 && reps <= 100, RANN_EINVAL, "reps must be in 1..100");
  const int64_t n = std::max<int64_t>(h->dof, 1);
  double *r = nullptr, *z = nullptr;
  CK(dalloc(h, (void**)&r, sizeof(double) * (size_t)n));
  CK(dalloc(h, (void**)&z, sizeof(double) * (size_t)n));
  {
    std::vector<double> ones((size_t)n, 1.0);
    CK(cudaMemcpyAsync(r, ones.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, h->st));
    CK(stream_sync(h));
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const bool fused_ok = h->prec_df && h->max_set_size <= schwarz_apply_max_subs();
  const int cur = h->apply_cfg;
  float ms_cfg[RANN_APPLY_NCFG];
  rann_status st = RANN_OK;
  for (int cfg = 0; cfg < RANN_APPLY_NCFG && st == RANN_OK; ++cfg) {
    ms_cfg[cfg] = -1.f;
    if (ms_out) ms_out[cfg] = -1.f;
    if (cfg == 0 ? !fused_ok : !streaming_ok(h)) continue;
    if ((st = set_apply_config(h, cfg)) != RANN_OK) break;
    if ((st = prec_apply(h, r, z, h->prec_df)) != RANN_OK) break;
    // the fastest of `reps` single applies: robust to other work sharing the GPU (a batch's
    // other instances), which only ever slows a sample down
    float ms = -1.f;
    for (int k = 0; k < reps && st == RANN_OK; ++k) {
      cudaEventRecord(e0, h->st);
      st = prec_apply(h, r, z, h->prec_df);
      cudaEventRecord(e1, h->st);
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = RANN_ECUDA; break; }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (ms < 0.f || t < ms) ms = t;
    }
    if (st != RANN_OK) break;
    if (ms_out) ms_out[cfg] = ms;
    ms_cfg[cfg] = ms;
  }
  // another configuration replaces the one in effect only when it is faster by more than
  // TUNE_MARGIN: work sharing the GPU (a batch's other instances) can slow every sample of
  // one configuration, and a small gain is not worth a choice that noise may have made
  int best = cur;
  float best_ms = st == RANN_OK ? ms_cfg[cur] : -1.f;
  for (int cfg = 0; cfg < RANN_APPLY_NCFG && st == RANN_OK; ++cfg) {
    const float m = ms_cfg[cfg];
    if (m < 0.f || cfg == cur) continue;
    if (ms_cfg[cur] < 0.f ? (best_ms < 0.f || m < best_ms)
                          : (m < (1.f - TUNE_MARGIN) * ms_cfg[cur] && m < best_ms)) {
      best = cfg;
      best_ms = m;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dfree(h, r);
  dfree(h, z);
  TRY(st);
  TRY(set_apply_config(h, best));
  CK(stream_sync(h));
  *best_out = best;
  return RANN_OK;
}

cudaStream_t rann_handle_stream(const rann_dd_handle* h) { return h->st; }
int rann_handle_dim(const rann_dd_handle* h) { return h->dim; }
int rann_handle_maxn(const rann_dd_handle* h) { return h->prec_kind >= 0 ? h->maxn : 0; }
bool rann_handle_piecewise(const rann_dd_handle* h) {
  return h->P.op == RANN_OP_DIFFUSION && h->P.coef == RANN_COEF_PIECEWISE;
}

extern "C" rann_status rann_dd_set_stream(rann_dd_handle* h, void* stream) {
  REQUIRE(h, RANN_EINVAL, "null handle");
  CK(stream_sync(h));
  h->st = (cudaStream_t)stream;
  return RANN_OK;
}

extern "C" rann_status rann_dd_precond_apply(rann_dd_handle* h, const double* r_dev, double* z_dev) {
  REQUIRE(h && r_dev && z_dev, RANN_EINVAL, "null argument");
  REQUIRE(h->prec_kind >= 0, RANN_EORDER, "precond_apply before setup_precond");
  // a precision mode 1 set-up keeps only the double-float factors
  return prec_apply(h, r_dev, z_dev, h->prec_df);
}

// -------------------------------------------------------------- solves --

// After a solve: an expired bounded wait of the streaming Schwarz apply left
// its error word set (the apply then skipped its arithmetic); report it as
// RANN_TIMEOUT and clear the word, so the handle stays usable.
static rann_status solve_done(rann_dd_handle* h, rann_status st) {
  if (!h || !h->d_ozerr) return st;
  int w = 0;
  if (cudaMemcpyAsync(&w, h->d_ozerr, sizeof(int), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
      stream_sync(h) != cudaSuccess)
    return st;
  if (w) {
    cudaMemsetAsync(h->d_ozerr, 0, sizeof(int), h->st);
    rann_set_error("Schwarz apply: bounded pipeline wait %d gave up", w);
    return RANN_TIMEOUT;
  }
  return st;
}

static rann_status dot_host(rann_dd_handle* h, const double* x, const double* y, int64_t n, double* out) {
  KLA(h, K_DOT, 1, 16.0 * n, 2.0 * n, launch_multidot(x, 0, 1, y, n, h->d_red, h->d_scal, h->st));
  CK(cudaMemcpyAsync(h->h_scal, h->d_scal, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(stream_sync(h));
  *out = h->h_scal[0];
  return RANN_OK;
}


struct Workspace {
  rann_dd_handle* h;
  std::vector<double*> bufs;
  ~Workspace() { for (double* p : bufs) dfree(h, p); }
  double* get(size_t n) {
    double* p = nullptr;
    if (dalloc(h, (void**)&p, sizeof(double) * std::max<size_t>(n, 1)) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return p;
  }
};

// The Krylov iterations apply the operator and the preconditioner with
// double-float data (A_in, M_in); every residual that decides a restart or the
// exit is recomputed with the float64 operator (A_64).  The loop between two
// float64 residuals is one step of iterative refinement, so the returned W
// solves the float64 normal equations to rtol.  With inner_df = 0 both are
// float64.
static rann_status op_inner(rann_dd_handle* h, const double* x, double* z) {
  return h->inner_df ? normal_matvec_fast(h, x, z) : rann_dd_normal_matvec(h, x, z);
}
static rann_status prec_inner(rann_dd_handle* h, const double* r, double* z, const float2* r2 = nullptr) {
  return prec_apply(h, r, z, h->inner_df != 0 || h->prec_df, false, r2);
}

// CG on H^T H W = b with b = H^T F (F_dev) or b given (b_dev).
static rann_status solve_cg_impl(rann_dd_handle* h, const double* F_dev, const double* b_dev, double* W_dev,
                                 double rtol, int maxit, rann_dd_stats* stats) {
  REQUIRE(h && (F_dev || b_dev) && W_dev, RANN_EINVAL, "null argument");
  REQUIRE(h->prec_kind >= 0, RANN_EORDER, "solve before setup_precond");
  REQUIRE(h->prec_kind == RANN_PREC_AS || h->prec_kind == RANN_PREC_NONE, RANN_EINVAL,
          "CG needs a symmetric preconditioner (AS or none)");
  REQUIRE(rtol > 0 && maxit >= 0, RANN_EINVAL, "bad rtol/maxit");
  const int64_t n = h->dof;
  Workspace ws{h, {}};
  double *b = ws.get(n), *r = ws.get(n), *z = ws.get(n), *p = ws.get(n), *q = ws.get(n), *cgs = ws.get(8);
  REQUIRE(b && r && z && p && q && cgs, RANN_ENOMEM, "workspace allocation failed");
  struct Events {
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    ~Events() { for (auto x : e) if (x) cudaEventDestroy(x); }
  } evh;
  cudaEvent_t* evs = evh.e;
  for (int i = 0; i < 3; ++i) CK(cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, h->st));
  if (F_dev) TRY(rann_dd_matvec_t(h, F_dev, b));
  else CK(cudaMemcpyAsync(b, b_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemsetAsync(W_dev, 0, sizeof(double) * n, h->st));
  CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
  double bb;
  TRY(dot_host(h, b, b, n, &bb));
  const double bnorm = std::sqrt(bb);
  rann_status st = RANN_NOT_CONVERGED;
  int it = 0;
  double rel = 1.0, true_rel = 1.0, kappa = -1.0;
  if (!(bnorm > 0.0)) {
    st = std::isfinite(bb) ? RANN_OK : RANN_BREAKDOWN;
    rel = true_rel = 0.0;
  } else {
    // Iterative refinement around preconditioned CG: each cycle solves the
    // correction equation A d = r (r the float64 residual of the current W)
    // from d = 0 with the inner operator until ||r_rec|| <= rtol ||b||, adds d
    // to W (held in the recurrence's x), and recomputes the float64 residual.
    // In float64 mode the first cycle is plain PCG.
    double* d = W_dev;   // W accumulates the corrections: x_{k+1} = x_k + alpha p, per cycle from r
    double rr;
    // CG scalars on the device; the host stays at most two steps ahead and
    // stops enqueueing once the device reports done
    CgDev sd{};
    sd.pq = cgs; sd.rr = cgs + 1; sd.rz = cgs + 2; sd.rel = cgs + 4;
    sd.done = reinterpret_cast<int*>(cgs + 5);
    sd.it = sd.done + 1;
    // alpha_k, beta_k of the first cycle (its Lanczos tridiagonal estimates kappa(M^{-1} A))
    sd.lzcap = std::max(0, std::min(maxit, 4096));
    sd.lz = sd.lzcap ? ws.get(2 * (size_t)sd.lzcap) : nullptr;
    if (!sd.lz) sd.lzcap = 0;
    int* hdone = reinterpret_cast<int*>(h->h_scal + 128);
    for (int cycle = 0; cycle < 30; ++cycle) {
      if (cycle == 1) { sd.lz = nullptr; sd.lzcap = 0; }
      TRY(prec_inner(h, r, z));
      CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
      KLA(h, K_DOT, 1, 16.0 * n, 2.0 * n, launch_multidot(r, 0, 1, z, n, h->d_red, sd.rz, h->st));
      CK(cudaMemsetAsync(sd.done, 0, 2 * sizeof(int), h->st));
      *hdone = 0;
      const int kmax = maxit - it;
      int ph = 0;
      for (int i = 0; i < kmax; ++i) {
        if (i >= 2) {
          CK(cudaEventSynchronize(evs[(i - 2) % 3]));
          if (*(volatile int*)hdone) break;
        }
        TRY(op_inner(h, p, q));
        KLA(h, K_DOT, 1, 16.0 * n, 2.0 * n, launch_multidot(p, 0, 1, q, n, h->d_red, sd.pq, h->st));
        KLA(h, K_VEC, 1, 40.0 * n, 4.0 * n, launch_cg_update_dev(p, q, d, r, n, sd, ph, h->st));
        KLA(h, K_DOT, 1, 8.0 * n, 2.0 * n, launch_multidot(r, 0, 1, r, n, h->d_red, sd.rr, h->st));
        KLA(h, K_VEC, 1, 0, 0, launch_cg_check(sd, bnorm, rtol, h->st));
        TRY(prec_inner(h, r, z));
        KLA(h, K_DOT, 1, 16.0 * n, 2.0 * n, launch_multidot(r, 0, 1, z, n, h->d_red, sd.rz + (ph ^ 1), h->st));
        KLA(h, K_VEC, 1, 24.0 * n, 3.0 * n, launch_cg_direction(z, p, n, sd, ph, h->st));
        ph ^= 1;
        CK(cudaMemcpyAsync(hdone, sd.done, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        CK(cudaEventRecord(evs[i % 3], h->st));
      }
      int dv[2];
      CK(cudaMemcpyAsync(dv, sd.done, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->st));
      CK(cudaMemcpyAsync(&rel, sd.rel, sizeof(double), cudaMemcpyDeviceToHost, h->st));
      CK(stream_sync(h));
      if (cycle == 0 && sd.lz && dv[1] >= 2) {
        const int K = std::min(dv[1], sd.lzcap);
        std::vector<double> lz(2 * (size_t)K);
        CK(cudaMemcpyAsync(lz.data(), sd.lz, sizeof(double) * 2 * K, cudaMemcpyDeviceToHost, h->st));
        CK(stream_sync(h));
        std::vector<double> ta(K), tb(K - 1);
        bool ok = true;
        for (int q = 0; q < K; ++q) {
          const double al = lz[2 * q];
          ok = ok && std::isfinite(al) && al > 0.0;
          ta[q] = 1.0 / al + (q > 0 ? lz[2 * q - 1] / lz[2 * q - 2] : 0.0);
          if (q + 1 < K) tb[q] = std::sqrt(std::max(lz[2 * q + 1], 0.0)) / al;
        }
        if (ok) {
          double lmin, lmax;
          tridiag_extremes(ta, tb, &lmin, &lmax);
          kappa = lmin > 0.0 ? lmax / lmin : -1.0;
        }
      }
      it += dv[1];
      const bool inner_ok = dv[0] == 1;
      if (dv[0] == 2) { st = RANN_BREAKDOWN; break; }
      // float64 residual of the accumulated W
      TRY(rann_dd_normal_matvec(h, W_dev, q));
      CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
      KLA(h, K_VEC, 1, 24.0 * n, 3.0 * n, launch_axpby(-1.0, q, 1.0, r, n, h->st));
      TRY(dot_host(h, r, r, n, &rr));
      const double prev = true_rel;
      true_rel = std::sqrt(rr) / bnorm;
      if (!std::isfinite(true_rel)) { st = RANN_BREAKDOWN; break; }
      if (true_rel <= rtol) { st = RANN_OK; break; }
      if (!inner_ok || it >= maxit) break;
      if (true_rel >= prev) break;   // refinement no longer reduces the float64 residual
    }
  }
  CK(cudaEventRecord(e1, h->st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  if (stats) {
    stats->iters = it;
    stats->rel_res_true = true_rel;
    stats->rel_res_rec = rel;
    stats->rel_res_prec = -1.0;
    stats->ms_solve = ms;
    stats->n_shifted = h->n_shifted;
    stats->kappa_est = kappa;
    fill_phase_stats(h, stats);
  }
  if (st == RANN_NOT_CONVERGED) rann_set_error("CG reached maxit=%d at rel. residual %.3e", maxit, true_rel);
  return st;
}

static rann_status prec_inner_t(rann_dd_handle* h, const double* r, double* z) {
  return prec_apply(h, r, z, h->inner_df != 0 || h->prec_df, true);
}

// The CG variants of Sec. 5 (Table 1b) on H^T H W = H^T F: conjugate gradient
// squared (Sonneveld) and biconjugate gradients (Fletcher; the shadow
// sequence uses A^T = A and M^{-T}), preconditioned as in Barrett et al.,
// Templates (1994), shadow residual = the cycle's initial residual.  Like CG,
// each cycle solves the correction equation with the inner operator and
// preconditioner until ||r_rec|| <= rtol ||b|| and then recomputes the float64
// residual; the exit is on ||b - H^T H W|| / ||b||.
static rann_status solve_variant_impl(rann_dd_handle* h, const double* F_dev, double* W_dev, double rtol, int maxit,
                                      rann_dd_stats* stats, bool bicg) {
  REQUIRE(h && F_dev && W_dev, RANN_EINVAL, "null argument");
  REQUIRE(h->prec_kind >= 0, RANN_EORDER, "solve before setup_precond");
  REQUIRE(rtol > 0 && maxit >= 0, RANN_EINVAL, "bad rtol/maxit");
  const int64_t n = h->dof;
  Workspace ws{h, {}};
  double *b = ws.get(n), *r = ws.get(n), *rr = ws.get(n), *rt = ws.get(n), *u = ws.get(n), *pv = ws.get(n),
         *q = ws.get(n), *ph = ws.get(n), *vh = ws.get(n), *t = ws.get(n), *t2 = ws.get(n);
  REQUIRE(b && r && rr && rt && u && pv && q && ph && vh && t && t2, RANN_ENOMEM, "workspace allocation failed");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, h->st));
  TRY(rann_dd_matvec_t(h, F_dev, b));
  CK(cudaMemsetAsync(W_dev, 0, sizeof(double) * n, h->st));
  CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
  double bb;
  TRY(dot_host(h, b, b, n, &bb));
  const double bnorm = std::sqrt(bb);
  rann_status st = RANN_NOT_CONVERGED;
  int it = 0;
  double rel = 1.0, true_rel = 1.0;
  auto copy = [&](double* dst, const double* src) {
    return cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st);
  };
  auto axpby = [&](double a, const double* x, double c, double* y) -> rann_status {
    KLA(h, K_VEC, 1, 24.0 * n, 3.0 * n, launch_axpby(a, x, c, y, n, h->st));
    return RANN_OK;
  };
  if (!(bnorm > 0.0)) {
    st = std::isfinite(bb) ? RANN_OK : RANN_BREAKDOWN;
    rel = true_rel = 0.0;
  } else {
    for (int cycle = 0; cycle < 30; ++cycle) {
      CK(copy(rr, r));
      CK(copy(rt, r));
      double rho_prev = 1.0;
      bool inner_ok = false, first = true;
      while (it < maxit) {
        double rho, sigma, r2;
        if (!bicg) {
          // CGS: rho = r~.r; u = r + beta q; p = u + beta (q + beta p)
          TRY(dot_host(h, rt, rr, n, &rho));
          if (!(rho != 0.0) || !std::isfinite(rho)) { st = RANN_BREAKDOWN; break; }
          if (first) {
            CK(copy(u, rr)); CK(copy(pv, rr));
          } else {
            const double beta = rho / rho_prev;
            CK(copy(u, rr)); TRY(axpby(beta, q, 1.0, u));
            CK(copy(t, q)); TRY(axpby(beta, pv, 1.0, t));
            TRY(axpby(1.0, u, beta, t));                  // t = u + beta (q + beta p)
            CK(copy(pv, t));
          }
          TRY(prec_inner(h, pv, ph));
          TRY(op_inner(h, ph, vh));
          TRY(dot_host(h, rt, vh, n, &sigma));
          if (!(sigma != 0.0) || !std::isfinite(sigma)) { st = RANN_BREAKDOWN; break; }
          const double alpha = rho / sigma;
          CK(copy(q, u)); TRY(axpby(-alpha, vh, 1.0, q));   // q = u - alpha A M p
          CK(copy(t, u)); TRY(axpby(1.0, q, 1.0, t));       // t = u + q
          TRY(prec_inner(h, t, ph));                          // u^ = M (u + q)
          TRY(axpby(alpha, ph, 1.0, W_dev));
          TRY(op_inner(h, ph, t2));
          TRY(axpby(-alpha, t2, 1.0, rr));
        } else {
          // BiCG: z = M r, z~ = M^T r~, rho = z.r~; p = z + beta p, p~ = z~ + beta p~
          TRY(prec_inner(h, rr, ph));
          TRY(prec_inner_t(h, rt, vh));
          TRY(dot_host(h, ph, rt, n, &rho));
          if (!(rho != 0.0) || !std::isfinite(rho)) { st = RANN_BREAKDOWN; break; }
          if (first) {
            CK(copy(pv, ph)); CK(copy(u, vh));
          } else {
            const double beta = rho / rho_prev;
            TRY(axpby(1.0, ph, beta, pv));
            TRY(axpby(1.0, vh, beta, u));                    // u holds p~
          }
          TRY(op_inner(h, pv, q));
          TRY(op_inner(h, u, t));                             // A^T p~ = A p~ (H^T H is symmetric)
          TRY(dot_host(h, u, q, n, &sigma));
          if (!(sigma != 0.0) || !std::isfinite(sigma)) { st = RANN_BREAKDOWN; break; }
          const double alpha = rho / sigma;
          TRY(axpby(alpha, pv, 1.0, W_dev));
          TRY(axpby(-alpha, q, 1.0, rr));
          TRY(axpby(-alpha, t, 1.0, rt));
        }
        first = false;
        rho_prev = rho;
        ++it;
        TRY(dot_host(h, rr, rr, n, &r2));
        rel = std::sqrt(r2) / bnorm;
        if (!std::isfinite(rel)) { st = RANN_BREAKDOWN; break; }
        if (rel <= rtol) { inner_ok = true; break; }
      }
      if (st == RANN_BREAKDOWN) break;
      // float64 residual of the accumulated W
      TRY(rann_dd_normal_matvec(h, W_dev, q));
      CK(copy(r, b));
      TRY(axpby(-1.0, q, 1.0, r));
      double rr2;
      TRY(dot_host(h, r, r, n, &rr2));
      const double prev = true_rel;
      true_rel = std::sqrt(rr2) / bnorm;
      if (!std::isfinite(true_rel)) { st = RANN_BREAKDOWN; break; }
      if (true_rel <= rtol) { st = RANN_OK; break; }
      if (!inner_ok || it >= maxit) break;
      if (true_rel >= prev) break;   // refinement no longer reduces the float64 residual
    }
  }
  CK(cudaEventRecord(e1, h->st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  if (stats) {
    stats->iters = it;
    stats->rel_res_true = true_rel;
    stats->rel_res_rec = rel;
    stats->rel_res_prec = -1.0;
    stats->ms_solve = ms;
    stats->n_shifted = h->n_shifted;
    stats->kappa_est = -1.0;
    fill_phase_stats(h, stats);
  }
  if (st == RANN_NOT_CONVERGED)
    rann_set_error("%s reached maxit=%d at rel. residual %.3e", bicg ? "BiCG" : "CGS", maxit, true_rel);
  return st;
}

extern "C" rann_status rann_dd_solve_cgs(rann_dd_handle* h, const double* F_dev, double* W_dev, double rtol,
                                         int maxit, rann_dd_stats* stats) {
  return solve_done(h, solve_variant_impl(h, F_dev, W_dev, rtol, maxit, stats, false));
}

extern "C" rann_status rann_dd_solve_bicg(rann_dd_handle* h, const double* F_dev, double* W_dev, double rtol,
                                          int maxit, rann_dd_stats* stats) {
  return solve_done(h, solve_variant_impl(h, F_dev, W_dev, rtol, maxit, stats, true));
}

extern "C" rann_status rann_dd_precond_apply_t(rann_dd_handle* h, const double* r_dev, double* z_dev) {
  REQUIRE(h && r_dev && z_dev, RANN_EINVAL, "null argument");
  REQUIRE(h->prec_kind >= 0, RANN_EORDER, "precond_apply_t before setup_precond");
  return prec_apply(h, r_dev, z_dev, h->prec_df, true);
}

// Left-preconditioned GMRES on H^T H W = b with b = H^T F (F_dev) or b given (b_dev).
static rann_status solve_gmres_impl(rann_dd_handle* h, const double* F_dev, const double* b_dev, double* W_dev,
                                    double rtol, int restart, int maxit, rann_dd_stats* stats) {
  REQUIRE(h && (F_dev || b_dev) && W_dev, RANN_EINVAL, "null argument");
  REQUIRE(h->prec_kind >= 0, RANN_EORDER, "solve before setup_precond");
  REQUIRE(rtol > 0 && maxit >= 0 && restart >= 1 && restart <= GMRES_MAX_RESTART, RANN_EINVAL,
          "bad rtol/restart/maxit");
  const int64_t n = h->dof;
  const int k = restart;
  Workspace ws{h, {}};
  double *b = ws.get(n), *t = ws.get(n), *V = ws.get((size_t)(k + 1) * n), *hv = ws.get(2 * (k + 2));
  const size_t nstate = (size_t)(k + 1) * k + 2 * k + (k + 1) + 3 * (k + 2) + 4;
  double* state = ws.get(nstate);
  // double-float splits of the basis vectors and of A v_j, written by their producers
  // when the inner operator is the block-row product (its consumers then skip the split)
  const bool split2 = h->inner_df && h->gram_ready;
  double* V2d = split2 ? ws.get((size_t)(k + 1) * n) : nullptr;
  double* t2d = split2 ? ws.get(n) : nullptr;
  REQUIRE(b && t && V && hv && state && (!split2 || (V2d && t2d)), RANN_ENOMEM, "workspace allocation failed");
  float2* V2 = reinterpret_cast<float2*>(V2d);
  float2* t2 = reinterpret_cast<float2*>(t2d);
  GmresDev sd{};
  sd.H = state;
  sd.cs = sd.H + (size_t)(k + 1) * k;
  sd.sn = sd.cs + k;
  sd.g = sd.sn + k;
  sd.hv = sd.g + (k + 1);
  sd.hcol = sd.hv + 2 * (k + 2);
  sd.ww = sd.hcol + (k + 2);
  sd.inv = sd.ww + 1;
  sd.rel = sd.inv + 1;
  sd.done = reinterpret_cast<int*>(sd.rel + 1);      // two ints in the last double
  sd.jdone = sd.done + 1;
  int* hdone = reinterpret_cast<int*>(h->h_scal + 128);
  struct Events {
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    ~Events() { for (auto x : e) if (x) cudaEventDestroy(x); }
  } evh;
  cudaEvent_t* evs = evh.e;
  for (int i = 0; i < 3; ++i) CK(cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, h->st));
  if (F_dev) TRY(rann_dd_matvec_t(h, F_dev, b));
  else CK(cudaMemcpyAsync(b, b_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemsetAsync(W_dev, 0, sizeof(double) * n, h->st));
  // ||M^{-1} b||
  TRY(prec_inner(h, b, V));
  double mbb;
  TRY(dot_host(h, V, V, n, &mbb));
  const double mbnorm = std::sqrt(mbb);
  std::vector<double> Hm((size_t)(k + 1) * k), g(k + 1), y(k);
  int it = 0;
  double rel = 1.0, kappa = -1.0;
  int cycle_no = 0;
  rann_status st = RANN_NOT_CONVERGED;
  if (!(mbnorm > 0.0)) { st = std::isfinite(mbb) ? RANN_OK : RANN_BREAKDOWN; rel = 0.0; }
  bool first = true;
  while (st == RANN_NOT_CONVERGED) {
    // r = M^{-1}(b - A W) with the float64 operator (W = 0 on the first cycle)
    if (first) {
      CK(cudaMemcpyAsync(t, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
    } else {
      TRY(rann_dd_normal_matvec(h, W_dev, t));
      KLA(h, K_VEC, 1, 24.0 * n, 3.0 * n, launch_axpby(1.0, b, -1.0, t, n, h->st));
    }
    first = false;
    TRY(prec_inner(h, t, V));
    double bb;
    TRY(dot_host(h, V, V, n, &bb));
    const double beta = std::sqrt(bb);
    rel = beta / mbnorm;
    if (!std::isfinite(rel)) { st = RANN_BREAKDOWN; break; }
    if (rel <= rtol) { st = RANN_OK; break; }
    if (it >= maxit) break;
    KLA(h, K_VEC, 1, 16.0 * n, 1.0 * n, launch_scale_copy(1.0 / beta, V, V, n, h->st, V2));
    // Arnoldi steps with the Givens bookkeeping on the device; the host stays at
    // most two steps ahead and stops enqueueing once the device reports done
    CK(cudaMemsetAsync(sd.g, 0, sizeof(double) * (k + 1), h->st));
    CK(cudaMemcpyAsync(sd.g, &beta, sizeof(double), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemsetAsync(sd.done, 0, 2 * sizeof(int), h->st));
    *hdone = 0;
    const int jmax = std::min(k, maxit - it);
    for (int j = 0; j < jmax; ++j) {
      if (j >= 2) {
        CK(cudaEventSynchronize(evs[(j - 2) % 3]));
        if (*(volatile int*)hdone) break;
      }
      double* w = V + (size_t)(j + 1) * n;
      if (split2) {
        TRY(normal_matvec_fast(h, V + (size_t)j * n, t, V2 + (size_t)j * n, t2));
        TRY(prec_inner(h, t, w, t2));
      } else {
        TRY(op_inner(h, V + (size_t)j * n, t));
        TRY(prec_inner(h, t, w));
      }
      // classical Gram-Schmidt, twice
      for (int pass = 0; pass < 2; ++pass) {
        KLA(h, K_DOT, 1, 8.0 * n * (j + 2), 2.0 * n * (j + 1),
            launch_multidot(V, n, j + 1, w, n, h->d_red, sd.hv + pass * (k + 2), h->st));
        KLA(h, K_VEC, 1, 8.0 * n * (j + 3), 2.0 * n * (j + 1),
            launch_sub_combination(V, n, j + 1, sd.hv + pass * (k + 2), w, n, h->st));
      }
      KLA(h, K_DOT, 1, 8.0 * n, 2.0 * n, launch_multidot(w, 0, 1, w, n, h->d_red, sd.ww, h->st));
      KLA(h, K_VEC, 1, 0, 0, launch_gmres_givens(sd, j, k, mbnorm, rtol, h->st));
      KLA(h, K_VEC, 1, 16.0 * n, 1.0 * n,
          launch_scale_dev(w, sd.inv, n, h->st, split2 ? V2 + (size_t)(j + 1) * n : nullptr));
      CK(cudaMemcpyAsync(hdone, sd.done, sizeof(int), cudaMemcpyDeviceToHost, h->st));
      CK(cudaEventRecord(evs[j % 3], h->st));
    }
    int dj[2];
    CK(cudaMemcpyAsync(dj, sd.done, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&rel, sd.rel, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(stream_sync(h));
    const int jdone = dj[1];
    it += jdone;
    if (jdone == 0) rel = beta / mbnorm;
    if (dj[0] == 2) { st = RANN_BREAKDOWN; break; }
    if (jdone == 0) break;
    CK(cudaMemcpyAsync(Hm.data(), sd.H, sizeof(double) * (size_t)jdone * k, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(g.data(), sd.g, sizeof(double) * jdone, cudaMemcpyDeviceToHost, h->st));
    CK(stream_sync(h));
    if (cycle_no++ == 0 && jdone >= 2) {
      // the Givens-reduced Hessenberg matrix of the first cycle: its singular
      // values lie inside those of M^{-1} A
      double smin, smax;
      triangle_sing_extremes(Hm, jdone, k, &smin, &smax);
      kappa = smin > 0.0 ? smax / smin : -1.0;
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double sacc = g[i];
      for (int q = i + 1; q < jdone; ++q) sacc -= Hm[(size_t)i * k + q] * y[q];
      y[i] = Hm[(size_t)i * k + i] != 0.0 ? sacc / Hm[(size_t)i * k + i] : 0.0;
    }
    CK(cudaMemcpyAsync(hv, y.data(), sizeof(double) * jdone, cudaMemcpyHostToDevice, h->st));
    KLA(h, K_VEC, 1, 8.0 * n * (jdone + 2), 2.0 * n * jdone,
        launch_add_combination(V, n, jdone, hv, W_dev, n, h->st));
    CK(stream_sync(h));
    // the next cycle recomputes the residual in float64 and decides convergence
  }
  double precrel = rel;
  double bb2, tr;
  TRY(dot_host(h, b, b, n, &bb2));
  TRY(rann_dd_normal_matvec(h, W_dev, t));
  KLA(h, K_VEC, 1, 24.0 * n, 3.0 * n, launch_axpby(1.0, b, -1.0, t, n, h->st));
  TRY(dot_host(h, t, t, n, &tr));
  CK(cudaEventRecord(e1, h->st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  if (stats) {
    stats->iters = it;
    stats->rel_res_true = bb2 > 0 ? std::sqrt(tr / bb2) : 0.0;
    stats->rel_res_rec = precrel;
    stats->rel_res_prec = precrel;
    stats->ms_solve = ms;
    stats->n_shifted = h->n_shifted;
    stats->kappa_est = kappa;
    fill_phase_stats(h, stats);
  }
  if (st == RANN_NOT_CONVERGED) rann_set_error("GMRES reached maxit=%d at rel. residual %.3e", maxit, rel);
  return st;
}

extern "C" rann_status rann_dd_solve_cg_as(rann_dd_handle* h, const double* F_dev, double* W_dev, double rtol,
                                           int maxit, rann_dd_stats* stats) {
  REQUIRE(F_dev, RANN_EINVAL, "null F");
  return solve_done(h, solve_cg_impl(h, F_dev, nullptr, W_dev, rtol, maxit, stats));
}

// ------------------------------------------------ many right-hand sides --
// The batched path needs the double-float factors with the fused apply and the
// block-row inner operator (precision mode 1); otherwise the right-hand sides
// are handled one after another by the one-vector routines.
static bool multi_batched(rann_dd_handle* h) {
  return h->prec_df && h->inner_df && h->gram_ready && h->prec_kind != RANN_PREC_NONE &&
         h->max_set_size <= schwarz_apply_max_subs();
}

// Z_c = M^{-1} R_c for c < nr (vectors [nr][DoF]); each column equals prec_apply's.
static rann_status prec_apply_multi(rann_dd_handle* h, const double* R, double* Z, int nr, Workspace& ws) {
  const int64_t n = h->dof;
  // the streaming apply serves one column at a time (each column bit for bit the one-vector apply)
  if (!multi_batched(h) || h->sr_nchunks > 0) {
    for (int c = 0; c < nr; ++c) TRY(prec_apply(h, R + c * n, Z + c * n, h->prec_df));
    return RANN_OK;
  }
  const int64_t stot = std::max<int64_t>(h->s_total, 1);
  double* sbuf = ws.get((size_t)nr * stot);
  double* pbuf = ws.get((size_t)4 * std::max<int64_t>(h->p32_total, 1));
  REQUIRE(sbuf && pbuf, RANN_ENOMEM, "workspace allocation failed");
  KLA(h, K_SCHWARZ_DF, (nr + 3) / 4 + 1, nr * (4.0 * (h->sum_n2 + h->sum_n) / std::min(nr, 4) + 16.0 * h->sum_n),
      nr * 2.0 * (h->sum_n2 + h->sum_n),
      launch_schwarz_apply_multi(h->d_mats, h->nsets, h->maxn, h->d_set_ptr, h->d_set_sub, h->d_sub, R, n,
                                 h->d_p_off32, pbuf, std::max<int64_t>(h->p32_total, 1), h->d_s_off, sbuf, stot,
                                 h->d_adone, nr, h->d_inc_ptr, h->d_inc_set, h->d_inc_pos, h->J, h->prec_kind, Z, n,
                                 h->st));
  return RANN_OK;
}

extern "C" rann_status rann_dd_precond_apply_multi(rann_dd_handle* h, const double* R_dev, double* Z_dev, int nrhs) {
  REQUIRE(h && R_dev && Z_dev && nrhs >= 0, RANN_EINVAL, "null argument or nrhs < 0");
  REQUIRE(h->prec_kind >= 0, RANN_EORDER, "precond_apply before setup_precond");
  Workspace ws{h, {}};
  return prec_apply_multi(h, R_dev, Z_dev, nrhs, ws);
}

// Preconditioned CG (AS) for nr right-hand sides in lockstep: every launch
// serves all columns (the factor rows and the block rows of H^T H are read
// once per step for all of them), each column has its own scalars, done flag
// and iterative-refinement decisions, with the arithmetic of solve_cg_impl.
static rann_status solve_cg_multi_impl(rann_dd_handle* h, const double* F_dev, double* W_dev, int nr, double rtol,
                                       int maxit, rann_dd_stats* stats) {
  REQUIRE(h && F_dev && W_dev && nr >= 0, RANN_EINVAL, "null argument or nrhs < 0");
  REQUIRE(h->prec_kind >= 0, RANN_EORDER, "solve before setup_precond");
  REQUIRE(h->prec_kind == RANN_PREC_AS || h->prec_kind == RANN_PREC_NONE, RANN_EINVAL,
          "CG needs a symmetric preconditioner (AS or none)");
  REQUIRE(rtol > 0 && maxit >= 0, RANN_EINVAL, "bad rtol/maxit");
  const int64_t n = h->dof, N = h->N;
  if (nr == 0) return RANN_OK;
  if (!multi_batched(h)) {                         // one right-hand side after another
    rann_status worst = RANN_OK;
    for (int c = 0; c < nr; ++c) {
      const rann_status st = solve_cg_impl(h, F_dev + c * N, nullptr, W_dev + c * n, rtol, maxit,
                                           stats ? stats + c : nullptr);
      if (st != RANN_OK && worst == RANN_OK) worst = st;
    }
    return worst;
  }
  Workspace ws{h, {}};
  const size_t nv = (size_t)nr * n;
  double *b = ws.get(nv), *r = ws.get(nv), *z = ws.get(nv), *p = ws.get(nv), *q = ws.get(nv);
  double* sc = ws.get((size_t)8 * nr + 8);
  REQUIRE(b && r && z && p && q && sc, RANN_ENOMEM, "workspace allocation failed");
  CgMulti sd{};
  sd.pq = sc; sd.rr = sc + nr; sd.rz = sc + 2 * nr; sd.rel = sc + 4 * nr;
  double* d_bnorm = sc + 5 * nr;
  sd.bnorm = d_bnorm;
  sd.done = reinterpret_cast<int*>(sc + 6 * nr);    // nr ints
  sd.it = reinterpret_cast<int*>(sc + 7 * nr);      // nr ints
  sd.nr = nr;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, h->st));
  for (int c = 0; c < nr; ++c) TRY(rann_dd_matvec_t(h, F_dev + c * N, b + c * n));
  CK(cudaMemsetAsync(W_dev, 0, sizeof(double) * nv, h->st));
  CK(cudaMemcpyAsync(r, b, sizeof(double) * nv, cudaMemcpyDeviceToDevice, h->st));
  std::vector<double> bb(nr), bn(nr), rel(nr, 1.0), true_rel(nr, 1.0), hrr(nr);
  std::vector<int> it(nr, 0), active(nr, 1), hd(nr), hit(nr);
  std::vector<rann_status> st(nr, RANN_NOT_CONVERGED);
  KLA(h, K_DOT, 1, 16.0 * nv, 2.0 * nv, launch_dot_multi(b, n, b, n, n, nr, sd.rr, h->st));
  CK(cudaMemcpyAsync(bb.data(), sd.rr, sizeof(double) * nr, cudaMemcpyDeviceToHost, h->st));
  CK(stream_sync(h));
  for (int c = 0; c < nr; ++c) {
    bn[c] = std::sqrt(bb[c]);
    if (!(bn[c] > 0.0)) {
      st[c] = std::isfinite(bb[c]) ? RANN_OK : RANN_BREAKDOWN;
      rel[c] = true_rel[c] = 0.0;
      active[c] = 0;
    }
  }
  CK(cudaMemcpyAsync(d_bnorm, bn.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, h->st));
  struct Events {
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    ~Events() { for (auto x : e) if (x) cudaEventDestroy(x); }
  } evh;
  for (int i = 0; i < 3; ++i) CK(cudaEventCreateWithFlags(&evh.e[i], cudaEventDisableTiming));
  int* hdone = reinterpret_cast<int*>(h->h_scal + 128);        // pinned: nr flags (host side)
  std::vector<int> hdv(nr);
  auto any_active = [&]() { for (int c = 0; c < nr; ++c) if (active[c]) return true; return false; };
  for (int cycle = 0; cycle < 30 && any_active(); ++cycle) {
    TRY(prec_apply_multi(h, r, z, nr, ws));
    CK(cudaMemcpyAsync(p, z, sizeof(double) * nv, cudaMemcpyDeviceToDevice, h->st));
    KLA(h, K_DOT, 1, 16.0 * nv, 2.0 * nv, launch_dot_multi(r, n, z, n, n, nr, sd.rz, h->st));
    for (int c = 0; c < nr; ++c) hd[c] = active[c] ? 0 : 1;
    CK(cudaMemcpyAsync(sd.done, hd.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemsetAsync(sd.it, 0, sizeof(int) * nr, h->st));
    int kmax = 0;
    for (int c = 0; c < nr; ++c) if (active[c]) kmax = std::max(kmax, maxit - it[c]);
    int ph = 0;
    for (int i = 0; i < kmax; ++i) {
      if (i >= 2) {
        CK(cudaEventSynchronize(evh.e[(i - 2) % 3]));
        if (*(volatile int*)hdone) break;
      }
      KLA(h, K_GRAMOP, 1, 8.0 * (h->gram_entries + nv), 2.0 * h->gram_entries * nr,
          launch_gram_matvec_multi(h->gram, h->J, h->d_gtile, h->ngtile, h->gram_maxn2, p, n, q, n, nr, h->st));
      KLA(h, K_DOT, 1, 16.0 * nv, 2.0 * nv, launch_dot_multi(p, n, q, n, n, nr, sd.pq, h->st));
      KLA(h, K_VEC, 1, 40.0 * nv, 4.0 * nv, launch_cg_update_multi(p, q, W_dev, r, n, n, sd, ph, h->st));
      KLA(h, K_DOT, 1, 8.0 * nv, 2.0 * nv, launch_dot_multi(r, n, r, n, n, nr, sd.rr, h->st));
      KLA(h, K_VEC, 1, 0, 0, launch_cg_check_multi(sd, rtol, h->st));
      TRY(prec_apply_multi(h, r, z, nr, ws));
      KLA(h, K_DOT, 1, 16.0 * nv, 2.0 * nv, launch_dot_multi(r, n, z, n, n, nr, sd.rz + (ph ^ 1) * nr, h->st));
      KLA(h, K_VEC, 1, 24.0 * nv, 3.0 * nv, launch_cg_direction_multi(z, p, n, n, sd, ph, h->st));
      ph ^= 1;
      KLA(h, K_VEC, 1, 0, 0, launch_all_done(sd.done, nr, h->d_scal + 64, h->st));
      CK(cudaMemcpyAsync(hdone, h->d_scal + 64, sizeof(int), cudaMemcpyDeviceToHost, h->st));
      CK(cudaEventRecord(evh.e[i % 3], h->st));
    }
    CK(cudaMemcpyAsync(hdv.data(), sd.done, sizeof(int) * nr, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(hit.data(), sd.it, sizeof(int) * nr, cudaMemcpyDeviceToHost, h->st));
    std::vector<double> hrel(nr);
    CK(cudaMemcpyAsync(hrel.data(), sd.rel, sizeof(double) * nr, cudaMemcpyDeviceToHost, h->st));
    CK(stream_sync(h));
    std::vector<int> inner_ok(nr, 0);
    for (int c = 0; c < nr; ++c) {
      if (!active[c]) continue;
      it[c] += hit[c];
      rel[c] = hrel[c];
      inner_ok[c] = hdv[c] == 1;
      if (hdv[c] == 2) { st[c] = RANN_BREAKDOWN; active[c] = 0; }
    }
    // float64 residual of each accumulated W_c
    for (int c = 0; c < nr; ++c) {
      if (!active[c]) continue;
      TRY(rann_dd_normal_matvec(h, W_dev + c * n, q + c * n));
      CK(cudaMemcpyAsync(r + c * n, b + c * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
      KLA(h, K_VEC, 1, 24.0 * n, 3.0 * n, launch_axpby(-1.0, q + c * n, 1.0, r + c * n, n, h->st));
    }
    KLA(h, K_DOT, 1, 8.0 * nv, 2.0 * nv, launch_dot_multi(r, n, r, n, n, nr, sd.rr, h->st));
    CK(cudaMemcpyAsync(hrr.data(), sd.rr, sizeof(double) * nr, cudaMemcpyDeviceToHost, h->st));
    CK(stream_sync(h));
    for (int c = 0; c < nr; ++c) {
      if (!active[c]) continue;
      const double prev = true_rel[c];
      true_rel[c] = std::sqrt(hrr[c]) / bn[c];
      if (!std::isfinite(true_rel[c])) { st[c] = RANN_BREAKDOWN; active[c] = 0; continue; }
      if (true_rel[c] <= rtol) { st[c] = RANN_OK; active[c] = 0; continue; }
      if (!inner_ok[c] || it[c] >= maxit) { active[c] = 0; continue; }
      if (true_rel[c] >= prev) active[c] = 0;    // refinement no longer reduces the float64 residual
    }
  }
  CK(cudaEventRecord(e1, h->st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  rann_status worst = RANN_OK;
  for (int c = 0; c < nr; ++c) {
    if (stats) {
      stats[c].iters = it[c];
      stats[c].rel_res_true = true_rel[c];
      stats[c].rel_res_rec = rel[c];
      stats[c].rel_res_prec = -1.0;
      stats[c].ms_solve = ms;
      stats[c].n_shifted = h->n_shifted;
      stats[c].kappa_est = -1.0;
      fill_phase_stats(h, &stats[c]);
    }
    if (st[c] != RANN_OK && worst == RANN_OK) worst = st[c];
  }
  if (worst == RANN_NOT_CONVERGED) rann_set_error("CG (many right-hand sides) reached maxit=%d", maxit);
  return worst;
}

extern "C" rann_status rann_dd_solve_cg_as_multi(rann_dd_handle* h, const double* F_dev, double* W_dev, int nrhs,
                                                 double rtol, int maxit, rann_dd_stats* stats) {
  return solve_done(h, solve_cg_multi_impl(h, F_dev, W_dev, nrhs, rtol, maxit, stats));
}

extern "C" rann_status rann_dd_solve_gmres_ras(rann_dd_handle* h, const double* F_dev, double* W_dev, double rtol,
                                               int restart, int maxit, rann_dd_stats* stats) {
  REQUIRE(F_dev, RANN_EINVAL, "null F");
  return solve_done(h, solve_gmres_impl(h, F_dev, nullptr, W_dev, rtol, restart, maxit, stats));
}

// Left-preconditioned GMRES(k) for nr right-hand sides in lockstep: each
// Arnoldi step applies the block-row operator and the Schwarz preconditioner
// to every column's current basis vector (block rows read once per step for
// up to four columns; the factors by the streaming apply once per column, by
// the fused apply once per four columns); the Gram-Schmidt
// passes, the Givens bookkeeping (own device state and done flag per column),
// the restarts and the float64 residual decisions are per column with the
// arithmetic of solve_gmres_impl, so every column equals the one-column
// solve.  A column that converged keeps stepping while others run; its
// Givens step is then a no-op and zeroes its next basis vector.
static rann_status solve_gmres_multi_impl(rann_dd_handle* h, const double* F_dev, double* W_dev, int nr,
                                          double rtol, int restart, int maxit, rann_dd_stats* stats) {
  REQUIRE(h && F_dev && W_dev && nr >= 0, RANN_EINVAL, "null argument or nrhs < 0");
  REQUIRE(h->prec_kind >= 0, RANN_EORDER, "solve before setup_precond");
  REQUIRE(rtol > 0 && maxit >= 0 && restart >= 1 && restart <= GMRES_MAX_RESTART, RANN_EINVAL,
          "bad rtol/restart/maxit");
  const int64_t n = h->dof, N = h->N;
  if (nr == 0) return RANN_OK;
  if (!multi_batched(h)) {                         // one right-hand side after another
    rann_status worst = RANN_OK;
    for (int c = 0; c < nr; ++c) {
      const rann_status st = solve_gmres_impl(h, F_dev + c * N, nullptr, W_dev + c * n, rtol, restart, maxit,
                                              stats ? stats + c : nullptr);
      if (st != RANN_OK && worst == RANN_OK) worst = st;
    }
    return worst;
  }
  const int k = restart;
  const size_t nv = (size_t)nr * n, lv = (size_t)(k + 1) * n;      // lv: one column's basis
  const size_t nstate = (size_t)(k + 1) * k + 2 * k + (k + 1) + 3 * (k + 2) + 4;
  Workspace ws{h, {}};
  double *b = ws.get(nv), *t = ws.get(nv), *z = ws.get(nv), *V = ws.get(nr * lv);
  double *state = ws.get(nr * nstate), *hvy = ws.get((size_t)nr * (k + 2)), *sc = ws.get((size_t)2 * nr + 2);
  REQUIRE(b && t && z && V && state && hvy && sc, RANN_ENOMEM, "workspace allocation failed");
  int* d_done = reinterpret_cast<int*>(sc);                // nr flags, then nr step counts
  int* d_jdone = d_done + nr;
  std::vector<GmresDev> sd(nr);
  for (int c = 0; c < nr; ++c) {
    GmresDev& q = sd[c];
    q.H = state + c * nstate;
    q.cs = q.H + (size_t)(k + 1) * k;
    q.sn = q.cs + k;
    q.g = q.sn + k;
    q.hv = q.g + (k + 1);
    q.hcol = q.hv + 2 * (k + 2);
    q.ww = q.hcol + (k + 2);
    q.inv = q.ww + 1;
    q.rel = q.inv + 1;
    q.done = d_done + c;
    q.jdone = d_jdone + c;
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, h->st));
  for (int c = 0; c < nr; ++c) TRY(rann_dd_matvec_t(h, F_dev + c * N, b + c * n));
  CK(cudaMemsetAsync(W_dev, 0, sizeof(double) * nv, h->st));
  // ||M^{-1} b|| per column
  TRY(prec_apply_multi(h, b, z, nr, ws));
  std::vector<double> mbb(nr), mbnorm(nr), bb(nr), beta(nr), rel(nr, 1.0), Hm((size_t)(k + 1) * k), g(k + 1), y(k);
  KLA(h, K_DOT, 1, 16.0 * nv, 2.0 * nv, launch_dot_multi(z, n, z, n, n, nr, t, h->st));
  CK(cudaMemcpyAsync(mbb.data(), t, sizeof(double) * nr, cudaMemcpyDeviceToHost, h->st));
  CK(stream_sync(h));
  std::vector<int> it(nr, 0), active(nr, 1), first(nr, 1), jmaxc(nr, 0), hd(nr), hj(nr);
  std::vector<rann_status> st(nr, RANN_NOT_CONVERGED);
  for (int c = 0; c < nr; ++c) {
    mbnorm[c] = std::sqrt(mbb[c]);
    if (!(mbnorm[c] > 0.0)) {
      st[c] = std::isfinite(mbb[c]) ? RANN_OK : RANN_BREAKDOWN;
      rel[c] = 0.0;
      active[c] = 0;
    }
  }
  struct Events {
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    ~Events() { for (auto x : e) if (x) cudaEventDestroy(x); }
  } evh;
  for (int i = 0; i < 3; ++i) CK(cudaEventCreateWithFlags(&evh.e[i], cudaEventDisableTiming));
  int* hdone = reinterpret_cast<int*>(h->h_scal + 128);
  auto any_active = [&]() { for (int c = 0; c < nr; ++c) if (active[c]) return true; return false; };
  while (any_active()) {
    // r_c = M^{-1}(b_c - A W_c) with the float64 operator (W_c = 0 on a column's first cycle)
    for (int c = 0; c < nr; ++c) {
      if (!active[c]) continue;
      if (first[c]) {
        CK(cudaMemcpyAsync(t + c * n, b + c * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
      } else {
        TRY(rann_dd_normal_matvec(h, W_dev + c * n, t + c * n));
        KLA(h, K_VEC, 1, 24.0 * n, 3.0 * n, launch_axpby(1.0, b + c * n, -1.0, t + c * n, n, h->st));
      }
      first[c] = 0;
    }
    TRY(prec_apply_multi(h, t, z, nr, ws));
    KLA(h, K_DOT, 1, 16.0 * nv, 2.0 * nv, launch_dot_multi(z, n, z, n, n, nr, t, h->st));
    CK(cudaMemcpyAsync(bb.data(), t, sizeof(double) * nr, cudaMemcpyDeviceToHost, h->st));
    CK(stream_sync(h));
    int jmax = 0;
    for (int c = 0; c < nr; ++c) {
      hd[c] = 1;
      if (!active[c]) continue;
      beta[c] = std::sqrt(bb[c]);
      rel[c] = beta[c] / mbnorm[c];
      if (!std::isfinite(rel[c])) { st[c] = RANN_BREAKDOWN; active[c] = 0; continue; }
      if (rel[c] <= rtol) { st[c] = RANN_OK; active[c] = 0; continue; }
      if (it[c] >= maxit) { active[c] = 0; continue; }
      double* Vc = V + c * lv;
      KLA(h, K_VEC, 1, 16.0 * n, 1.0 * n, launch_scale_copy(1.0 / beta[c], z + c * n, Vc, n, h->st));
      CK(cudaMemsetAsync(sd[c].g, 0, sizeof(double) * (k + 1), h->st));
      CK(cudaMemcpyAsync(sd[c].g, &beta[c], sizeof(double), cudaMemcpyHostToDevice, h->st));
      hd[c] = 0;
      jmaxc[c] = std::min(k, maxit - it[c]);         // a column past its step count launches nothing
      jmax = std::max(jmax, jmaxc[c]);
    }
    if (!any_active()) break;
    CK(cudaMemcpyAsync(d_done, hd.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemsetAsync(d_jdone, 0, sizeof(int) * nr, h->st));
    *hdone = 0;
    for (int j = 0; j < jmax; ++j) {
      if (j >= 2) {
        CK(cudaEventSynchronize(evh.e[(j - 2) % 3]));
        if (*(volatile int*)hdone) break;
      }
      KLA(h, K_GRAMOP, 1, 8.0 * (h->gram_entries + nv), 2.0 * h->gram_entries * nr,
          launch_gram_matvec_multi(h->gram, h->J, h->d_gtile, h->ngtile, h->gram_maxn2, V + (size_t)j * n, lv, t,
                                   n, nr, h->st));
      TRY(prec_apply_multi(h, t, z, nr, ws));
      for (int c = 0; c < nr; ++c) {
        if (!active[c] || j >= jmaxc[c]) continue;
        double* Vc = V + c * lv;
        double* w = Vc + (size_t)(j + 1) * n;
        CK(cudaMemcpyAsync(w, z + c * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
        for (int pass = 0; pass < 2; ++pass) {
          KLA(h, K_DOT, 1, 8.0 * n * (j + 2), 2.0 * n * (j + 1),
              launch_multidot(Vc, n, j + 1, w, n, h->d_red, sd[c].hv + pass * (k + 2), h->st));
          KLA(h, K_VEC, 1, 8.0 * n * (j + 3), 2.0 * n * (j + 1),
              launch_sub_combination(Vc, n, j + 1, sd[c].hv + pass * (k + 2), w, n, h->st));
        }
        KLA(h, K_DOT, 1, 8.0 * n, 2.0 * n, launch_multidot(w, 0, 1, w, n, h->d_red, sd[c].ww, h->st));
        KLA(h, K_VEC, 1, 0, 0, launch_gmres_givens(sd[c], j, k, mbnorm[c], rtol, h->st));
        KLA(h, K_VEC, 1, 16.0 * n, 1.0 * n, launch_scale_dev(w, sd[c].inv, n, h->st));
      }
      KLA(h, K_VEC, 1, 0, 0, launch_all_done(d_done, nr, h->d_scal + 64, h->st));
      CK(cudaMemcpyAsync(hdone, h->d_scal + 64, sizeof(int), cudaMemcpyDeviceToHost, h->st));
      CK(cudaEventRecord(evh.e[j % 3], h->st));
    }
    std::vector<double> hrel(nr);
    std::vector<double> state_rel(nr);
    CK(cudaMemcpyAsync(hd.data(), d_done, sizeof(int) * nr, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(hj.data(), d_jdone, sizeof(int) * nr, cudaMemcpyDeviceToHost, h->st));
    for (int c = 0; c < nr; ++c)
      if (active[c]) CK(cudaMemcpyAsync(&state_rel[c], sd[c].rel, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(stream_sync(h));
    for (int c = 0; c < nr; ++c) {
      if (!active[c]) continue;
      const int jdone = hj[c];
      it[c] += jdone;
      rel[c] = jdone == 0 ? beta[c] / mbnorm[c] : state_rel[c];
      if (hd[c] == 2) { st[c] = RANN_BREAKDOWN; active[c] = 0; continue; }
      if (jdone == 0) { active[c] = 0; continue; }
      CK(cudaMemcpyAsync(Hm.data(), sd[c].H, sizeof(double) * (size_t)jdone * k, cudaMemcpyDeviceToHost, h->st));
      CK(cudaMemcpyAsync(g.data(), sd[c].g, sizeof(double) * jdone, cudaMemcpyDeviceToHost, h->st));
      CK(stream_sync(h));
      for (int i = jdone - 1; i >= 0; --i) {
        double sacc = g[i];
        for (int q = i + 1; q < jdone; ++q) sacc -= Hm[(size_t)i * k + q] * y[q];
        y[i] = Hm[(size_t)i * k + i] != 0.0 ? sacc / Hm[(size_t)i * k + i] : 0.0;
      }
      double* yc = hvy + (size_t)c * (k + 2);
      CK(cudaMemcpyAsync(yc, y.data(), sizeof(double) * jdone, cudaMemcpyHostToDevice, h->st));
      KLA(h, K_VEC, 1, 8.0 * n * (jdone + 2), 2.0 * n * jdone,
          launch_add_combination(V + c * lv, n, jdone, yc, W_dev + c * n, n, h->st));
      CK(stream_sync(h));
    }
  }
  // the float64 relative residual of every column
  std::vector<double> bb2(nr), tr(nr);
  KLA(h, K_DOT, 1, 16.0 * nv, 2.0 * nv, launch_dot_multi(b, n, b, n, n, nr, t, h->st));
  CK(cudaMemcpyAsync(bb2.data(), t, sizeof(double) * nr, cudaMemcpyDeviceToHost, h->st));
  CK(stream_sync(h));
  for (int c = 0; c < nr; ++c) {
    TRY(rann_dd_normal_matvec(h, W_dev + c * n, z + c * n));
    KLA(h, K_VEC, 1, 24.0 * n, 3.0 * n, launch_axpby(1.0, b + c * n, -1.0, z + c * n, n, h->st));
  }
  KLA(h, K_DOT, 1, 16.0 * nv, 2.0 * nv, launch_dot_multi(z, n, z, n, n, nr, t, h->st));
  CK(cudaMemcpyAsync(tr.data(), t, sizeof(double) * nr, cudaMemcpyDeviceToHost, h->st));
  CK(cudaEventRecord(e1, h->st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  rann_status worst = RANN_OK;
  for (int c = 0; c < nr; ++c) {
    if (stats) {
      stats[c].iters = it[c];
      stats[c].rel_res_true = bb2[c] > 0 ? std::sqrt(tr[c] / bb2[c]) : 0.0;
      stats[c].rel_res_rec = rel[c];
      stats[c].rel_res_prec = rel[c];
      stats[c].ms_solve = ms;
      stats[c].n_shifted = h->n_shifted;
      stats[c].kappa_est = -1.0;
      fill_phase_stats(h, &stats[c]);
    }
    if (st[c] != RANN_OK && worst == RANN_OK) worst = st[c];
  }
  if (worst == RANN_NOT_CONVERGED) rann_set_error("GMRES (many right-hand sides) reached maxit=%d", maxit);
  return worst;
}

extern "C" rann_status rann_dd_solve_gmres_ras_multi(rann_dd_handle* h, const double* F_dev, double* W_dev, int nrhs,
                                                     double rtol, int restart, int maxit, rann_dd_stats* stats) {
  return solve_done(h, solve_gmres_multi_impl(h, F_dev, W_dev, nrhs, rtol, restart, maxit, stats));
}

// Adjoint of the least-squares solve.  W = (H^T H)^{-1} H^T F, so for a loss
// l(W) the sensitivity to F is H lam with (H^T H) lam = dl/dW: the same
// symmetric normal matrix, solved with the stored preconditioner (CG when it
// is symmetric, GMRES(50) otherwise).
extern "C" rann_status rann_dd_solve_backward(rann_dd_handle* h, const double* gW_dev, double* lam_dev, double rtol,
                                              int maxit, rann_dd_stats* stats) {
  REQUIRE(h && gW_dev && lam_dev, RANN_EINVAL, "null argument");
  REQUIRE(h->prec_kind >= 0, RANN_EORDER, "solve_backward before setup_precond");
  if (h->prec_kind == RANN_PREC_AS || h->prec_kind == RANN_PREC_NONE)
    return solve_done(h, solve_cg_impl(h, nullptr, gW_dev, lam_dev, rtol, maxit, stats));
  return solve_done(h, solve_gmres_impl(h, nullptr, gW_dev, lam_dev, rtol, 50, maxit, stats));
}

// dl/dc0 of a loss l(W) through the least-squares solve, for -Lap u + c0 u
// (the coefficient enters H linearly: dH/dc0 = L Psi V, dF/dc0 = -G).  With
// r = F - H W and lam = (H^T H)^{-1} dl/dW (rann_dd_solve_backward),
//   dl/dc0 = r . (H_c lam) - (H lam) . G - (H lam) . (H_c W),
// where H_c x = u_hat(x) - G at the collocation points (u_hat of Eq. (netdd)
// with weights x), so every term comes from the evaluation kernel, the block
// matvec and fixed-order dot products.
extern "C" rann_status rann_dd_grad_c0(rann_dd_handle* h, const double* F_dev, const double* W_dev,
                                       const double* lam_dev, double* grad_host) {
  REQUIRE(h && F_dev && W_dev && lam_dev && grad_host, RANN_EINVAL, "null argument");
  REQUIRE(h->reduced, RANN_EORDER, "grad_c0 before pca");
  REQUIRE(h->P.op == RANN_OP_POISSON, RANN_EINVAL, "grad_c0: c0 is a coefficient of the Poisson operator only");
  const int64_t N = h->N, dof = h->dof;
  double *x, *zero, *g0, *eW, *eL, *r, *hl;
  CK(dalloc(h, (void**)&x, sizeof(double) * (size_t)N * h->dim));
  CK(dalloc(h, (void**)&zero, sizeof(double) * (size_t)std::max<int64_t>(dof, 1)));
  for (double** q : {&g0, &eW, &eL, &r, &hl}) CK(dalloc(h, (void**)q, sizeof(double) * (size_t)N));
  CK(cudaMemsetAsync(zero, 0, sizeof(double) * (size_t)std::max<int64_t>(dof, 1), h->st));
  TRY(rann_dd_points(h, x));
  TRY(rann_dd_eval(h, zero, x, N, g0));                       // G
  TRY(rann_dd_eval(h, W_dev, x, N, eW));
  TRY(rann_dd_eval(h, lam_dev, x, N, eL));
  KL(h, K_VEC, 1, launch_axpby(-1.0, g0, 1.0, eW, N, h->st));   // H_c W
  KL(h, K_VEC, 1, launch_axpby(-1.0, g0, 1.0, eL, N, h->st));   // H_c lam
  TRY(rann_dd_matvec(h, W_dev, r));
  KL(h, K_VEC, 1, launch_axpby(1.0, F_dev, -1.0, r, N, h->st));  // r = F - H W
  TRY(rann_dd_matvec(h, lam_dev, hl));                           // H lam
  double d1 = 0.0, d2 = 0.0, d3 = 0.0;
  TRY(dot_host(h, r, eL, N, &d1));
  TRY(dot_host(h, hl, g0, N, &d2));
  TRY(dot_host(h, hl, eW, N, &d3));
  *grad_host = d1 - d2 - d3;
  for (double* q : {x, zero, g0, eW, eL, r, hl}) dfree(h, q);
  return RANN_OK;
}

// U_j = V_{p_j} x_j for every subdomain (the m-vectors the evaluation kernels read).
static rann_status basis_combination(rann_dd_handle* h, const double* x, double* U) {
  const int J = h->J, m = h->m;
  std::vector<GemmTask> tasks;
  for (int j = 0; j < J; ++j) {
    const SubDev& S = h->subs[j];
    GemmTask t{};
    t.A = h->d_V + (size_t)m * m * j; t.B = x + S.woff; t.C = U + (size_t)m * j;
    t.K = S.p; t.M = m; t.N = 1; t.lda = m; t.ldb = 1; t.ldc = 1;
    push_tiles(tasks, t, false);
  }
  GemmTask* d_tasks;
  CK(dupload(h, &d_tasks, tasks));
  KL(h, K_EVAL, 1, launch_gemm_nn(d_tasks, (int)tasks.size(), h->st));
  dfree(h, d_tasks);
  return RANN_OK;
}

extern "C" rann_status rann_dd_grad_coef(rann_dd_handle* h, const double* F_dev, const double* W_dev,
                                         const double* lam_dev, double* grad_host) {
  REQUIRE(h && F_dev && W_dev && lam_dev && grad_host, RANN_EINVAL, "null argument");
  REQUIRE(h->reduced, RANN_EORDER, "grad_coef before pca");
  REQUIRE(h->P.op == RANN_OP_DIFFUSION && h->P.coef == RANN_COEF_PIECEWISE, RANN_EINVAL,
          "grad_coef: the diffusion operator with a piecewise coefficient only");
  const int64_t N = h->N;
  const int J = h->J, m = h->m, nc = h->P.coef_grid * h->P.coef_grid;
  const int nb = coef_grad_blocks(N);
  double *U, *r, *hl, *part;
  CK(dalloc(h, (void**)&U, sizeof(double) * 2 * (size_t)J * m));
  CK(dalloc(h, (void**)&r, sizeof(double) * (size_t)N));
  CK(dalloc(h, (void**)&hl, sizeof(double) * (size_t)N));
  CK(dalloc(h, (void**)&part, sizeof(double) * (size_t)nb * nc));
  TRY(basis_combination(h, W_dev, U));
  TRY(basis_combination(h, lam_dev, U + (size_t)J * m));
  TRY(rann_dd_matvec(h, W_dev, r));
  KL(h, K_VEC, 1, launch_axpby(1.0, F_dev, -1.0, r, N, h->st));   // r = F - H W
  TRY(rann_dd_matvec(h, lam_dev, hl));                             // H lam
  KLA(h, K_EVAL, 1, 8.0 * (2.0 * N + 2.0 * J * m), 0.0,
      launch_coef_grad(h->P, h->d_sub, h->d_R, h->d_b, U, U + (size_t)J * m, r, hl, N, part, h->st));
  std::vector<double> ph((size_t)nb * nc);
  CK(cudaMemcpyAsync(ph.data(), part, sizeof(double) * ph.size(), cudaMemcpyDeviceToHost, h->st));
  CK(stream_sync(h));
  for (int c = 0; c < nc; ++c) {
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += ph[(size_t)b * nc + c];
    grad_host[c] = acc;
  }
  for (double* q : {U, r, hl, part}) dfree(h, q);
  return RANN_OK;
}

extern "C" rann_status rann_dd_eval_grid_t(rann_dd_handle* h, const double* r_dev, double* gW_dev) {
  REQUIRE(h && r_dev && gW_dev, RANN_EINVAL, "null argument");
  REQUIRE(h->reduced, RANN_EORDER, "eval_grid_t before pca");
  const int64_t N = h->N;
  const int J = h->J, m = h->m;
  // t_j = Psi_j^T (L r)|_{rows_j}: the transposed block product over the unreduced
  // Psi blocks (a descriptor copy with p = P = m), then gW_j = V_{p_j}^T t_j
  std::vector<SubDev> un(h->subs);
  for (int j = 0; j < J; ++j) {
    un[j].p = m; un[j].P = m; un[j].boff = h->subs[j].row0 * m; un[j].woff = (int64_t)j * m;
  }
  SubDev* d_un;
  double *y, *t, *part;
  CK(dupload(h, &d_un, un));
  CK(dalloc(h, (void**)&y, sizeof(double) * (size_t)std::max<int64_t>(N, 1)));
  CK(dalloc(h, (void**)&t, sizeof(double) * (size_t)J * m));
  CK(dalloc(h, (void**)&part, sizeof(double) * (size_t)std::max(h->nrtiles, 1) * m));
  KL(h, K_EVAL, 1, launch_lmul(h->P, r_dev, y, N, h->st));
  KLA(h, K_EVAL, 2, 8.0 * ((double)h->rows_total * m + h->rows_total + (double)J * m), 2.0 * h->rows_total * m,
      launch_matvec_HT2(h->P, d_un, J, h->d_rtiles, h->nrtiles, h->d_tile0, h->d_Psi, y, part, t, m, h->st));
  std::vector<GemmTask> tasks;
  for (int j = 0; j < J; ++j) {
    const SubDev& S = h->subs[j];
    GemmTask g{};
    g.A = h->d_V + (size_t)m * m * j; g.B = t + (size_t)m * j; g.C = gW_dev + S.woff;
    g.K = m; g.M = S.p; g.N = 1; g.lda = m; g.ldb = 1; g.ldc = 1;
    push_tiles(tasks, g, false);
  }
  GemmTask* d_tasks;
  CK(dupload(h, &d_tasks, tasks));
  KL(h, K_EVAL, 1, launch_gemm_tn(d_tasks, (int)tasks.size(), h->st));
  CK(stream_sync(h));
  dfree(h, d_tasks); dfree(h, d_un); dfree(h, y); dfree(h, t); dfree(h, part);
  return RANN_OK;
}

extern "C" rann_status rann_dd_set_coef(rann_dd_handle* h, const double* vals_host) {
  REQUIRE(h && vals_host, RANN_EINVAL, "null argument");
  REQUIRE(h->P.op == RANN_OP_DIFFUSION && h->P.coef == RANN_COEF_PIECEWISE, RANN_EINVAL,
          "set_coef: the handle has no piecewise diffusion coefficient");
  const int nc = h->P.coef_grid * h->P.coef_grid;
  for (int c = 0; c < nc; ++c) REQUIRE(std::isfinite(vals_host[c]), RANN_EINVAL, "coefficient %d not finite", c);
  for (int c = 0; c < nc; ++c) h->P.coef_vals[c] = vals_host[c];
  // H depends on the coefficient: the handle goes back to step 3 of Algorithm 1
  h->assembled = false;
  h->reduced = false;
  h->prec_kind = -1;
  return RANN_OK;
}

extern "C" rann_status rann_dd_set_precision(rann_dd_handle* h, int mode) {
  REQUIRE(h, RANN_EINVAL, "null handle");
  REQUIRE(mode == 0 || mode == 1, RANN_EINVAL, "precision mode must be 0 (float64) or 1 (double-float)");
  h->inner_df = mode;
  return RANN_OK;
}

// ---------------------------------------------------------------- eval --

extern "C" rann_status rann_dd_eval(rann_dd_handle* h, const double* W_dev, const double* x_dev, int64_t n,
                                    double* u_dev) {
  REQUIRE(h && W_dev && (n == 0 || (x_dev && u_dev)), RANN_EINVAL, "null argument");
  REQUIRE(n >= 0, RANN_EINVAL, "negative n");
  REQUIRE(h->reduced, RANN_EORDER, "eval before pca");
  const int J = h->J, m = h->m;
  double* d_U;
  CK(dalloc(h, (void**)&d_U, sizeof(double) * (size_t)J * m));
  std::vector<GemmTask> tasks;
  for (int j = 0; j < J; ++j) {
    const SubDev& S = h->subs[j];
    GemmTask t{};
    t.A = h->d_V + (size_t)m * m * j; t.B = W_dev + S.woff; t.C = d_U + (size_t)m * j;
    t.K = S.p; t.M = m; t.N = 1; t.lda = m; t.ldb = 1; t.ldc = 1;
    push_tiles(tasks, t, false);
  }
  GemmTask* d_tasks;
  CK(dupload(h, &d_tasks, tasks));
  KL(h, K_EVAL, 1, launch_gemm_nn(d_tasks, (int)tasks.size(), h->st));
  KL(h, K_EVAL, 1, launch_eval(h->P, h->d_sub, h->d_R, h->d_b, d_U, x_dev, n, u_dev, h->st));
  CK(stream_sync(h));
  dfree(h, d_tasks);
  dfree(h, d_U);
  return RANN_OK;
}

// ---------------------------------------------------------- inspection --

extern "C" rann_status rann_dd_block_info(rann_dd_handle* h, int j, int64_t* n_rows, int* n_cols) {
  REQUIRE(h && j >= 0 && j < h->J, RANN_EINVAL, "bad subdomain index");
  if (n_rows) *n_rows = h->subs[j].N;
  if (n_cols) *n_cols = h->reduced ? h->subs[j].p : h->m;
  return RANN_OK;
}

extern "C" rann_status rann_dd_get_block(rann_dd_handle* h, int j, int which, double* out_host,
                                         int64_t* rows_host) {
  REQUIRE(h && j >= 0 && j < h->J, RANN_EINVAL, "bad subdomain index");
  REQUIRE(which >= 0 && which <= 2, RANN_EINVAL, "bad block kind");
  const SubDev& S = h->subs[j];
  if (rows_host) {
    int64_t r = 0;
    for (int a2 = 0; a2 < S.n[2]; ++a2)
      for (int a1 = 0; a1 < S.n[1]; ++a1)
        for (int a0 = 0; a0 < S.n[0]; ++a0)
          rows_host[r++] = (S.lo[0] + a0) + (int64_t)h->P.G[0] * ((S.lo[1] + a1) + (int64_t)h->P.G[1] * (S.lo[2] + a2));
  }
  if (!out_host) return RANN_OK;
  if (which < 2) {
    REQUIRE(h->assembled, RANN_EORDER, "get_block before assemble");
    const double* src = (which == 0 ? h->d_Psi : h->d_H) + S.row0 * h->m;
    CK(cudaMemcpyAsync(out_host, src, sizeof(double) * (size_t)S.N * h->m, cudaMemcpyDeviceToHost, h->st));
  } else {
    REQUIRE(h->reduced, RANN_EORDER, "get_block(B) before pca");
    CK(cudaMemcpy2DAsync(out_host, sizeof(double) * S.p, h->d_B + S.boff, sizeof(double) * S.P,
                         sizeof(double) * S.p, S.N, cudaMemcpyDeviceToHost, h->st));
  }
  CK(stream_sync(h));
  return RANN_OK;
}

extern "C" rann_status rann_dd_get_pca(rann_dd_handle* h, int j, double* eig_host, double* V_host) {
  REQUIRE(h && j >= 0 && j < h->J, RANN_EINVAL, "bad subdomain index");
  REQUIRE(h->reduced, RANN_EORDER, "get_pca before pca");
  const int m = h->m;
  if (eig_host) memcpy(eig_host, h->eig_host.data() + (size_t)m * j, sizeof(double) * m);
  if (V_host) {
    CK(cudaMemcpy2DAsync(V_host, sizeof(double) * h->subs[j].p, h->d_V + (size_t)m * m * j, sizeof(double) * m,
                         sizeof(double) * h->subs[j].p, m, cudaMemcpyDeviceToHost, h->st));
    CK(stream_sync(h));
  }
  return RANN_OK;
}

// ----------------------------------------------------------- profiling --

extern "C" rann_status rann_dd_profile_enable(rann_dd_handle* h, int on) {
  REQUIRE(h, RANN_EINVAL, "null handle");
  prof_resolve(h);
  for (int k = 0; k < K_COUNT; ++k) {
    h->prof.launches[k] = 0; h->prof.ms[k] = 0.0; h->prof.bytes[k] = 0.0; h->prof.flops[k] = 0.0;
  }
  h->prof.on = on != 0;
  return RANN_OK;
}

extern "C" rann_status rann_dd_profile_get(rann_dd_handle* h, int idx, const char** name, int64_t* launches,
                                           double* ms, double* alg_bytes, double* alg_flops, int* bound) {
  REQUIRE(h, RANN_EINVAL, "null handle");
  if (idx < 0 || idx >= K_COUNT) return RANN_EINVAL;
  prof_resolve(h);
  if (name) *name = KNAMES[idx];
  if (launches) *launches = h->prof.launches[idx];
  if (ms) *ms = h->prof.ms[idx];
  if (alg_bytes) *alg_bytes = h->prof.bytes[idx];
  if (alg_flops) *alg_flops = h->prof.flops[idx];
  if (bound) *bound = (h->inner_df && family_is_df(idx)) ? 3 : KBOUND[idx];
  return RANN_OK;
}
