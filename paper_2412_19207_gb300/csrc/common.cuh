// Internal declarations shared by the CUDA translation units of librann_dd.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "rann_dd.h"

#define RANN_MAX_DIM 3
#define RANN_MAX_FTERMS 16
#define RANN_MAX_COEF 64
#define RANN_MAX_M 1024
#define RANN_PI 3.141592653589793238462643383279502884

// Problem constants, passed by value to the kernels.
struct ProbDev {
  int dim, ns, op, coef, g_kind, m;
  double c0, nu, coef_value, eps, rho, f0;
  int coef_grid;
  double coef_vals[RANN_MAX_COEF];
  int f_terms;
  double fc[RANN_MAX_FTERMS];
  double fa[RANN_MAX_FTERMS * RANN_MAX_DIM];
  int G[RANN_MAX_DIM];       // global grid points per dim
  int nsub[RANN_MAX_DIM];    // subdomains per dim
  double sig[RANN_MAX_DIM];  // half-width per dim
  int layout;
};

// Per-subdomain block descriptor (device copy).
struct SubDev {
  int k[RANN_MAX_DIM];       // multi-index of the subdomain
  int lo[RANN_MAX_DIM];      // first global grid index of box_j per dim
  int n[RANN_MAX_DIM];       // box extent per dim
  double mu[RANN_MAX_DIM];   // centre per dim
  int N;                     // rows = prod n
  int p;                     // PCA rank
  int P;                     // padded row length of B_j (p rounded up to 2)
  int poff;                  // offset of x_j in the padded (P_j-aligned) vector copy
  int64_t row0;              // offset of block j in the unreduced row storage (rows)
  int64_t woff;              // offset of W_j
  int64_t boff;              // offset of B_j in the reduced storage (doubles)
};


// Lifts a kernel's dynamic shared-memory limit to the most this device allows
// (once per kernel, from a function-local static in the launcher).  The limit
// is a per-kernel setting shared by every host thread: setting it per launch
// to the launch's own size would race with concurrent launches of larger
// sizes from other threads (handles driven in parallel by a batch).
template <typename K>
inline cudaError_t smem_limit_max(K kernel) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes a{};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
  return e;
}

// Host-side helpers (api.cu).
void rann_set_error(const char* fmt, ...);
cudaStream_t rann_handle_stream(const rann_dd_handle* h);
int rann_handle_dim(const rann_dd_handle* h);
int rann_handle_maxn(const rann_dd_handle* h);        // largest extended set after setup_precond (else 0)
bool rann_handle_piecewise(const rann_dd_handle* h);  // RANN_COEF_PIECEWISE diffusion

static inline double host_mu(int layout, int k, int l) {
  return layout == RANN_LAYOUT_PAPER ? (double)k / (double)(l - 1) : ((double)k + 0.5) / (double)l;
}

// ---- kernel launchers (defined in the .cu files) ----
// assembly.cu
cudaError_t launch_assemble(const ProbDev& P, const SubDev* d_sub, const int* d_tiles, int ntiles,
                            const int* d_cov, const double* d_R, const double* d_b,
                            double* d_Psi, double* d_H, cudaStream_t st);
cudaError_t launch_rhs(const ProbDev& P, double* d_F, int64_t N, cudaStream_t st);
cudaError_t launch_points(const ProbDev& P, double* d_xyz, int64_t N, cudaStream_t st);
cudaError_t launch_eval(const ProbDev& P, const SubDev* d_sub, const double* d_R, const double* d_b,
                        const double* d_U, const double* d_x, int64_t n, double* d_u,
                        cudaStream_t st);

// dense.cu -- batched float64 dense kernels
struct GemmTask {            // one output tile of one batched product
  const double* A;           // TN: A is K x M (row-major, lda); NN: A is M x K
  const double* B;           // TN: B is K x N; NN: B is K x N
  double* C;                 // M x N (ldc)
  const int* ia;             // TN only: optional row gather for A (K entries)
  const int* ib;             // TN only: optional row gather for B
  int K, M, N, lda, ldb, ldc;
  int tm, tn;                // tile origin (row, col) in C
  int upper_only;            // TN symmetric: skip tiles strictly below the diagonal
  int pad_;
};
cudaError_t launch_gemm_tn(const GemmTask* d_tasks, int ntasks, cudaStream_t st);
cudaError_t launch_gemm_nn(const GemmTask* d_tasks, int ntasks, cudaStream_t st);
cudaError_t launch_gemm_tn_df(const GemmTask* d_tasks, int ntasks, cudaStream_t st);
cudaError_t launch_symmetrize(double* const* d_mats, const int* d_n, const int* d_ld, int nmat,
                              int maxn, cudaStream_t st);

// ozaki.cu -- float64-accurate products from bf16 digit slices on the tensor cores
struct OzSplitTask {         // one operand: rows i < M of x(i, k) = X[i * si + g(k) * sk], k < K
  const double* X;
  const int* gather;         // g(k) = gather[k], or k when null
  int64_t si, sk;
  int M, K, Kp, Mp;          // Kp = oz_kpad(K), Mp = oz_mpad(M) (rows M..Mp-1 of the slices are zero)
  int* e;                    // [M] row exponents (out)
  uint16_t* out;             // [oz_slices()][Kp/8][Mp][8] bf16 digit slices (out), 16-byte aligned
  int df;                    // 1: X holds double-float pairs (float2, value hi + lo) at the same indices
};
constexpr int OZ_TILE_M = 128, OZ_TILE_N = 64;   // C tile of one block (rows of A x rows of B)
struct alignas(64) OzMap { unsigned char bytes[128]; };   // a TMA tensor map of one operand's slices
struct OzTask {              // one OZ_TILE_M x OZ_TILE_N tile of C = A B^T (A: M x K slices, B: N x K slices)
  int ia, ib;                // split operands of A and B (their tensor maps: maps[2 ia], maps[2 ib + 1])
  const int* ea;
  const int* eb;
  double* C;                 // M x N (ldc)
  int M, N, Kp, ldc;
  int tm, tn;                // tile origin in C
};
// A batch of tiles of one product C (op)= A B^T for the grouped launch: the
// tiles of a group are enumerated in the kernel (row tiles of OZ_TILE_M, column
// tiles of OZ_TILE_N; with lower = 1 only the tiles that meet the lower
// triangle i >= j, and no entry above it is written).  mode: OZ_OUT_F64
// writes float64 C; OZ_OUT_DF_SUB subtracts the product from double-float C
// (float2); OZ_OUT_DF_SET writes it to double-float C.
enum { OZ_OUT_F64 = 0, OZ_OUT_DF_SUB = 1, OZ_OUT_DF_SET = 2 };
struct OzGroup {
  int ia, ib;
  const int* ea;
  const int* eb;
  void* C;
  int M, N, Kp, ldc;
  int mode, lower;
  int first;                 // index of the group's first tile in the launch
  int tiles;                 // oz_group_tiles(M, N, lower)
};
inline int oz_group_tiles(int M, int N, int lower) {
  const int RT = (M + OZ_TILE_M - 1) / OZ_TILE_M, CT = (N + OZ_TILE_N - 1) / OZ_TILE_N;
  if (!lower) return RT * CT;
  int n = 0;
  for (int r = 0; r < RT; ++r) n += CT < 2 * r + 2 ? CT : 2 * r + 2;
  return n;
}
cudaError_t launch_oz_gemm_groups(const OzGroup* d_groups, int ngroups, int ntiles, const OzMap* d_maps, int* d_err,
                                  cudaStream_t st);
int oz_slices();
int oz_kpad(int K);
inline int oz_mpad(int M) { return (M + 31) / 32 * 32; }
// Host: the two TMA tensor maps (A role, B role) of each operand's slices,
// from the device addresses in ops[].out (no device work).
cudaError_t oz_encode_maps(const std::vector<OzSplitTask>& ops, std::vector<OzMap>& maps);
cudaError_t launch_oz_split(const OzSplitTask* d_tasks, int ntasks, int maxM, int maxKp, cudaStream_t st);
// d_maps: device copy of oz_encode_maps' output (64-byte aligned); d_err: set
// non-zero if a pipeline wait timed out (the tile is then not written).
cudaError_t launch_oz_gemm(const OzTask* d_tasks, int ntiles, const OzMap* d_maps, int* d_err, cudaStream_t st);

// krylov.cu -- device-resident state of one GMRES cycle
constexpr int GMRES_MAX_RESTART = 120;
struct GmresDev {
  double* H;                 // [k + 1][k] rotated Hessenberg matrix (row-major, ld k)
  double* cs;                // [k] Givens cosines
  double* sn;                // [k] Givens sines
  double* g;                 // [k + 1] rotated right-hand side (g_0 = beta)
  double* hv;                // [2][k + 2] coefficients of the two Gram-Schmidt passes
  double* hcol;              // [k + 2] scratch column
  double* ww;                // ||w||^2 after the passes
  double* inv;               // 1 / h_{j+1,j}
  double* rel;               // residual estimate of the last step
  int* done;                 // 0 running, 1 converged or lucky breakdown, 2 non-finite
  int* jdone;                // steps that entered the Hessenberg matrix
};
cudaError_t launch_gmres_givens(const GmresDev& s, int j, int k, double mbnorm, double rtol, cudaStream_t st);
// device-resident scalars of preconditioned CG (rz ping-pongs between two slots)
struct CgDev {
  double* pq;
  double* rr;
  double* rz;                // [2]
  double* rel;
  int* done;                 // 0 running, 1 converged, 2 breakdown
  int* it;                   // updates made
  double* lz = nullptr;      // optional [2 lzcap]: alpha_k, beta_k of the Lanczos relation
  int lzcap = 0;
};
cudaError_t launch_cg_update_dev(const double* p, const double* q, double* x, double* r, int64_t n, const CgDev& s,
                                 int ph, cudaStream_t st);
cudaError_t launch_cg_check(const CgDev& s, double bnorm, double rtol, cudaStream_t st);
cudaError_t launch_cg_direction(const double* z, double* p, int64_t n, const CgDev& s, int ph, cudaStream_t st);
// many right-hand sides in lockstep: one scalar set per column c < nr
struct CgMulti {
  double* pq;                // [nr]
  double* rr;                // [nr]
  double* rz;                // [2][nr]
  double* rel;               // [nr]
  int* done;                 // [nr] 0 running, 1 converged, 2 breakdown
  int* it;                   // [nr] updates made
  const double* bnorm;       // [nr] ||b_c||
  int nr;
};
cudaError_t launch_dot_multi(const double* x, int64_t ldx, const double* y, int64_t ldy, int64_t n, int nr,
                             double* d_out, cudaStream_t st);
cudaError_t launch_cg_update_multi(const double* p, const double* q, double* x, double* r, int64_t n, int64_t ld,
                                   const CgMulti& s, int ph, cudaStream_t st);
cudaError_t launch_cg_check_multi(const CgMulti& s, double rtol, cudaStream_t st);
cudaError_t launch_cg_direction_multi(const double* z, double* p, int64_t n, int64_t ld, const CgMulti& s, int ph,
                                      cudaStream_t st);
// *(int*)d_out = 1 when done[c] != 0 for every c < nr
cudaError_t launch_all_done(const int* d_done, int nr, double* d_out, cudaStream_t st);
// y *= *a; y2 (optional): the double-float split of the result
cudaError_t launch_scale_dev(double* y, const double* a, int64_t n, cudaStream_t st, float2* y2 = nullptr);

// gramop.cu -- the normal matrix as double-float block rows R_k = [G_kl]_l
constexpr int GRAM_TILE_ROWS = 8;    // rows of R_k per block of the row-dot kernel (one warp each)
constexpr int GRAM_MAX_NBR = 27;     // most neighbours of a block row (3^3); more falls back to B^T (B x)
struct GramRows {                    // device arrays
  const int* p;                      // [J] p_k
  const int* n2;                     // [J] row length of R_k: sum of P_l over its neighbours
  const int64_t* roff;               // [J] offset of R_k in R2 (float2 units, even)
  const int* poff;                   // [J] offset of x_k in the padded double-float copy of x
  const int64_t* woff;               // [J] offset of x_k in x
  const int* nbr_ptr;                // [J + 1] neighbour lists (boxes that meet box k, increasing l)
  const int* nbr_l;                  // neighbour index l
  const int* nbr_col;                // first column of block l in R_k (block l spans P_l columns)
  const int64_t* nbr_off;            // offset of the stored Gram block of the pair in the pair buffer
  const int* nbr_tr;                 // 1: stored as G_lk (p_l x p_k), read transposed
  float2* R2;
};
cudaError_t launch_gramrows_build(const GramRows& g, const double* d_pairbuf, int J, int maxp, int maxn2,
                                  cudaStream_t st);
// z = (H^T H) x from the block rows; x2 (optional): the double-float split of x
// (staged instead of splitting x); z2 (optional): the split of z is written too
cudaError_t launch_gram_matvec(const GramRows& g, int J, const int* d_rtile, int nrtile, int maxn2,
                               const double* d_x, double* d_z, cudaStream_t st, const float2* d_x2 = nullptr,
                               float2* d_z2 = nullptr);
// the same for nr right-hand sides x_c = d_x + c ldx -> z_c = d_z + c ldz (each column
// bit-identical to launch_gram_matvec of that column)
cudaError_t launch_gram_matvec_multi(const GramRows& g, int J, const int* d_rtile, int nrtile, int maxn2,
                                     const double* d_x, int64_t ldx, double* d_z, int64_t ldz, int nr,
                                     cudaStream_t st);

// eig.cu -- batched symmetric eigen-decomposition (float64)
// Eigenpairs of `batch` m x m symmetric matrices A; ranks by the PCA rule (mode, thr);
// eigenvalues by bisection (bisect = 1) or QL (0); work holds
// batch * syevd_work_doubles(m) doubles.  Phases 0..4 (tridiagonalisation,
// eigenvalues, rank rule + inverse iteration, Gram-Schmidt, back-transformation
// + output) run in this order on one stream.
struct SyevBatch {
  double* A;
  int m, batch;
  double* w;                 // [batch][m] eigenvalues, descending
  double* work;
  int* info;
  int* ranks;
  int mode;
  double thr;
  int bisect;                // precision mode 1: bisection eigenvalues, double-float Gram-Schmidt
};
int64_t syevd_work_doubles(int m);
cudaError_t launch_syev_phase(const SyevBatch& b, int phase, cudaStream_t st);

// chol.cu -- batched uneven Cholesky and triangular solves
struct CholMat {
  double* A;                 // n x n row-major (lower triangle used): A_i, then its Cholesky factor L_i (float64 mode)
  double* X;                 // n x n row-major (lower triangle used): L_i^{-1} (float64 mode)
  float2* X2;                // L_i^{-1} as double-float pairs (same layout)
  float2* A2;                // double-float A_i, then L_i (precision mode 1; null in float64 mode)
  int n;
  int ld;
};

// apply.cu -- streaming double-float Schwarz apply (rows of X_i = L_i^{-1} read once)
struct SrChunk {             // consecutive rows [r0, r1) of set `set`, its k-th chunk, in nst stages
  int set, r0, r1, k, nst;
  int64_t poff;              // offset of the chunk's column sums (n_set doubles)
};
int schwarz_rows_nmax();
int schwarz_rows_stage();
void schwarz_rows_plan(const std::vector<int>& nvec, int64_t target, std::vector<SrChunk>& chunks,
                       std::vector<int>& ck_ptr, std::vector<int>& order, int64_t& part_total);
cudaError_t launch_schwarz_apply_rows_df(const CholMat* d_mats, const SrChunk* d_chunks, const int* d_order,
                                         int nchunks, const int* d_ck_ptr, const int* d_set_ptr,
                                         const int* d_set_sub, const SubDev* d_sub, const double* d_r,
                                         const float2* d_r2, int wkind, const int* d_inc_ptr, double* d_part,
                                         const int64_t* d_s_off, double* d_s, int* d_done, int ckind, double* d_z,
                                         int* d_err, cudaStream_t st);
