// Batched symmetric eigen-decomposition in float64 for the PCA (Sec. 4,
// Eq. (pca)): the right singular vectors and singular values of Psi_j are the
// eigenpairs of G_j = Psi_j^T Psi_j = V diag(sigma^2) V^T.  Only the p_j
// kept eigenvectors are formed.  Five kernels per batch (one phase each;
// grids span the batch and, where the phase is parallel over eigenpairs,
// parts of each matrix):
//
//   1. Householder tridiagonalisation G = Q T Q^T (Golub & Van Loan 8.3.1)
//      on the lower triangle by a cluster of blocks per matrix; reflectors
//      kept in the upper rows of G.
//   2. Eigenvalues of T.  Fast path: bisection on Sturm counts, one thread
//      per eigenvalue (Barth, Martin & Wilkinson, 1967; Kahan's LDL^T count):
//      T is scaled by a power of two to norm <= 1; 48 halvings use LDL^T
//      pivot counts in double-float arithmetic (float32 pipe), then the
//      bracket is widened, re-verified and halved 10 more times with float64
//      counts from the division-free three-term recurrence of the leading
//      principal minors (rescaled by powers of two every 8 steps), so each
//      eigenvalue ends within ~2^-52 ||T|| like a float64 QL.  Reference
//      path (precision mode 0): implicit QL with Wilkinson shifts (the tql1
//      scheme of Bowdler, Martin, Reinsch & Wilkinson, 1968), no vectors,
//      one thread's dependent chain.
//   3. Eigenvalues in descending order; the rank rule of Sec. 4 gives p_j.
//   4. Eigenvectors of T for the p_j largest eigenvalues by inverse iteration
//      (tridiagonal LU with partial pivoting, two solves; Wilkinson, The
//      Algebraic Eigenvalue Problem, Ch. 9), one thread per vector, then
//      classical Gram-Schmidt applied twice in descending order.
//   5. Back-transformation V = Q Z, one warp per vector, and the transposed
//      copy of V into G.
// Output: w[m] descending; ranks[b] = p_j; G overwritten by V (row-major
// m x m, column c = eigenvector c for c < p_j, zero beyond); info[b] != 0 if
// QL did not converge in 100 sweeps for some eigenvalue.
// Work area per matrix (doubles): Z [m][m] (rows: eigenvectors of T), the
// inverse-iteration LU [5][m][m] (entry i of vector k at [i][k]), d, e, beta
// [m] each, and 4 scalars (||T||, Gershgorin bounds).
#include <cooperative_groups.h>

#include "common.cuh"
#include "df32.cuh"

namespace {

constexpr int NT = 512;
constexpr int NW = NT / 32;

// n_active: only threads tid < n_active hold non-zero values; warps wholly beyond
// it skip their shuffle tree (their partial is zero either way, so the sum and
// its order are unchanged).  Returns scale * sum, the product formed once by
// thread 0 (1.0 * sum is the sum itself).
__device__ double block_sum(double v, double* red, int n_active = NT, double scale = 1.0) {
  if ((threadIdx.x & ~31) < n_active)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += red[w];
    red[32] = scale * s;
  }
  __syncthreads();
  return red[32];
}

// Deterministic start vector for inverse iteration, entries in [-0.5, 1.5).
__device__ __forceinline__ double start_entry(int i, int k) {
  unsigned h = (unsigned)i * 2654435761u ^ ((unsigned)k * 40503u + 0x9E3779B9u);
  h ^= h >> 15;
  h *= 2246822519u;
  h ^= h >> 13;
  return (double)(h & 2047u) / 1024.0 - 0.5;
}

constexpr float PIV_DF = 0x1p-60f;   // pivot floor of the scaled LDL^T counts
constexpr double PIV_64 = 0x1p-60;

// (ah, al) - (bh, bl) in double-float
__device__ __forceinline__ void df_diff(float ah, float al, float bh, float bl, float& rh, float& rl) {
  float s, e;
  df_two_sum(ah, -bh, s, e);
  e = __fadd_rn(e, __fsub_rn(al, bl));
  df_two_sum(s, e, rh, rl);
}

// Number of eigenvalues of the scaled T below sigma: negative pivots of
// T - sigma I = L D L^T, q_0 = d_0 - sigma, q_i = d_i - sigma - e_{i-1}^2 / q_{i-1},
// in double-float (d = dh + dl, e^2 = eh + el); a pivot below PIV_DF in
// magnitude is replaced by -PIV_DF.
__device__ int sturm_count_df(const float* __restrict__ dh, const float* __restrict__ dl,
                              const float* __restrict__ eh, const float* __restrict__ el, int m,
                              double sigma) {
  const float2 sg = df_split(sigma);
  float qh, ql;
  df_diff(dh[0], dl[0], sg.x, sg.y, qh, ql);
  if (fabsf(qh) < PIV_DF) { qh = -PIV_DF; ql = 0.f; }
  int cnt = qh < 0.f;
  for (int i = 1; i < m; ++i) {
    float ah, al;
    df_diff(dh[i], dl[i], sg.x, sg.y, ah, al);
    // t = e^2 / q: quotient, exact residual, one correction
    const float x = __fdividef(eh[i - 1], qh);
    const float ph = __fmul_rn(x, qh);
    const float pe = __fmaf_rn(x, qh, -ph);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(eh[i - 1], ph), pe), __fsub_rn(el[i - 1], __fmul_rn(x, ql)));
    const float c = __fdividef(r, qh);
    float th, tl;
    df_two_sum(x, c, th, tl);
    df_diff(ah, al, th, tl, qh, ql);
    if (fabsf(qh) < PIV_DF) { qh = -PIV_DF; ql = 0.f; }
    cnt += qh < 0.f;
  }
  return cnt;
}

// The same count in float64 from the leading principal minors
// p_{i+1} = (d_i - sigma) p_i - e_{i-1}^2 p_{i-1} (a sign change between p_i and
// p_{i+1} is a negative pivot q_i = p_{i+1} / p_i; an exact zero becomes
// q_i = -PIV_64).  Both minors are rescaled by the power of two that brings the
// larger to [1, 2) every 8 steps (|d_i - sigma| + e_{i-1}^2 <= 4, so 8 steps
// grow them by at most 2^16).
__device__ int sturm_count_f64(const double* __restrict__ ds, const double* __restrict__ e2s, int m,
                               double sigma) {
  double p0 = 1.0, p1 = ds[0] - sigma;
  if (p1 == 0.0) p1 = -PIV_64;
  int cnt = __double2hiint(p1) < 0;
  for (int i = 1; i < m; ++i) {
    double p2 = fma(ds[i] - sigma, p1, -e2s[i - 1] * p0);
    if (((__double2hiint(p2) & 0x7fffffff) | __double2loint(p2)) == 0) p2 = -PIV_64 * p1;
    cnt += (__double2hiint(p2) ^ __double2hiint(p1)) < 0;
    p0 = p1;
    p1 = p2;
    if ((i & 7) == 0) {
      const int E = max((__double2hiint(p0) >> 20) & 0x7ff, (__double2hiint(p1) >> 20) & 0x7ff);
      const double f = __hiloint2double((2046 - E) << 20, 0);   // 2^(1023 - E), E <= 2045 here
      p0 *= f;
      p1 *= f;
    }
  }
  return cnt;
}

// Per-matrix work layout.
struct SyevWork {
  double *Z, *LU, *d, *e, *beta, *meta;
  __device__ SyevWork(double* base, int m) {
    Z = base;
    LU = Z + (int64_t)m * m;
    d = LU + 5 * (int64_t)m * m;
    e = d + m;
    beta = e + m;
    meta = beta + m;            // [0] ||T||_inf-like bound, [1] [2] Gershgorin bounds
  }
};

// ---- 1. tridiagonalisation, one cluster of TC blocks per matrix ----
// Only the lower triangle of the trailing matrix A' is kept.  Per column k:
// every block forms the same reflector v from column k; the symmetric
// product A' v is accumulated from the lower rows (each row c, loaded once,
// adds v_c A'[c][0..c] to the result and contributes its dot product with v
// to entry c); rows are dealt cyclically to the TC x NW warps of the cluster,
// the per-block partial sums are exchanged through distributed shared memory
// and added in a fixed order (so every block holds the identical w); then the
// cluster applies A' -= v w^T + w v^T to the lower rows, dealt the same way.
// Each lane holds SL columns (lane + 32 t), so a row's loads are all in flight
// at once.
constexpr int TC = 2;          // blocks per matrix (cluster size; one block per SM at 512 threads)

template <int SL>
__global__ void __launch_bounds__(NT) syev_tridiag_kernel(double* __restrict__ Aall, int m,
                                                          double* __restrict__ work_all, int64_t work_stride,
                                                          int use_dp) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double sm[];
  double* v = sm;              // [m] reflector
  double* w = v + m;           // [m] symmetric product
  double* wl = w + m;          // [m] this block's partial product (read by the cluster)
  double* wdot = wl + m;       // [m] dot products of the rows this block owns
  double* part = wdot + m;     // [NW][m] per-warp partials
  // [NW][SR][33] lane partials of the row dots (SR rows per warp, padded rows);
  // summed by one thread per row instead of a 32-lane shuffle reduction
  const int SR = (m - 1 + TC * NW - 1) / (TC * NW);
  double* dpart = part + (int64_t)NW * m;
  __shared__ double red[33];
  __shared__ double sbt;       // 2 / (v^T v) of the current reflector
  __shared__ int sbt_nz;
  const int mat = blockIdx.x / TC;
  const int rank = (int)cluster.block_rank();
  double* A = Aall + (int64_t)mat * m * m;
  SyevWork W(work_all + mat * work_stride, m);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gw = rank * NW + warp;             // warp index within the cluster
  for (int k = 0; k + 2 < m; ++k) {
    const int n1 = m - k - 1;
    double loc = 0.0;
    for (int c = tid; c < n1; c += NT) {
      const double x = A[(int64_t)(k + 1 + c) * m + k];   // column k, lower part
      v[c] = x;
      loc += x * x;
    }
    const double sig2 = block_sum(loc, red, n1);
    // the reflector's scalars once per block (thread 0), shared: GB300's
    // float64 pipe would otherwise run the square root and the division for
    // every warp
    if (tid == 0) {
      const double sigma = sqrt(sig2);
      const double x0 = v[0];
      const double alpha = (x0 >= 0.0) ? -sigma : sigma;
      const double b2 = (sigma > 0.0) ? 1.0 / (sig2 + fabs(x0) * sigma) : 0.0;   // 2 / (v^T v)
      v[0] = x0 - alpha;
      sbt = b2;
      sbt_nz = b2 != 0.0;
      if (rank == 0) { W.d[k] = A[(int64_t)k * m + k]; W.e[k] = alpha; W.beta[k] = b2; }
    }
    __syncthreads();
    const double bt = sbt;
    if (sbt_nz) {
      double* Ak = A + (int64_t)(k + 1) * m + (k + 1);       // A'[c][j] = Ak[c * m + j]
      double acc[SL];
#pragma unroll
      for (int t = 0; t < SL; ++t) acc[t] = 0.0;
      for (int c = gw, si = 0; c < n1; c += TC * NW, ++si) {
        const double* R = Ak + (int64_t)c * m;
        const int tmax = c >> 5;               // last slot holding part of row c (warp-uniform)
        double x[SL];
#pragma unroll
        for (int t = 0; t < SL; ++t) {
          if (t > tmax) break;
          x[t] = (lane + 32 * t <= c) ? R[lane + 32 * t] : 0.0;
        }
        const double vc = v[c];
        double dot = 0.0;
#pragma unroll
        for (int t = 0; t < SL; ++t) {
          if (t > tmax) break;
          const int j = lane + 32 * t;
          acc[t] = fma(vc, x[t], acc[t]);
          dot = fma(x[t], (j < c) ? v[j] : 0.0, dot);
        }
        if (use_dp) {
          dpart[((int64_t)warp * SR + si) * 33 + lane] = dot;
        } else {
          for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
          if (lane == 0) wdot[c] = dot;        // row c belongs to this warp alone
        }
      }
#pragma unroll
      for (int t = 0; t < SL; ++t)
        if (lane + 32 * t < n1) part[warp * m + lane + 32 * t] = acc[t];
      __syncthreads();
      for (int j = tid; j < n1; j += NT) {
        double s = 0.0;
        for (int q = 0; q < NW; ++q) s += part[q * m + j];
        const int gj = j % (TC * NW);
        if (gj / NW == rank) {                 // dot of a row this block owns
          if (use_dp) {
            const double* dp = dpart + ((int64_t)(gj % NW) * SR + j / (TC * NW)) * 33;
            double d0 = 0.0, d1 = 0.0;
#pragma unroll
            for (int l = 0; l < 32; l += 2) { d0 += dp[l]; d1 += dp[l + 1]; }
            s += d0 + d1;
          } else {
            s += wdot[j];
          }
        }
        wl[j] = s;
      }
      cluster.sync();                          // partials visible to the cluster
      double pv = 0.0;
      for (int j = tid; j < n1; j += NT) {
        double s = 0.0;
        for (int q = 0; q < TC; ++q) s += cluster.map_shared_rank(wl, q)[j];
        s *= bt;
        w[j] = s;
        pv = fma(s, v[j], pv);
      }
      const double K = block_sum(pv, red, n1, 0.5 * bt);
      for (int j = tid; j < n1; j += NT) w[j] = fma(-K, v[j], w[j]);
      __syncthreads();
      // A' -= v w^T + w v^T on the lower rows
      for (int rr = gw; rr < n1; rr += TC * NW) {
        double* R = Ak + (int64_t)rr * m;
        const int tmax = rr >> 5;
        double x[SL];
#pragma unroll
        for (int t = 0; t < SL; ++t) {
          if (t > tmax) break;
          x[t] = (lane + 32 * t <= rr) ? R[lane + 32 * t] : 0.0;
        }
        const double vr = v[rr], wr = w[rr];
#pragma unroll
        for (int t = 0; t < SL; ++t) {
          if (t > tmax) break;
          const int j = lane + 32 * t;
          if (j <= rr) R[j] = fma(-vr, w[j], fma(-wr, v[j], x[t]));
        }
      }
    }
    if (rank == 0)
      for (int c = tid; c < n1; c += NT) A[(int64_t)k * m + k + 1 + c] = v[c];   // keep the reflector (upper part)
    cluster.sync();                            // updates visible before the next column; wl free again
  }
  if (rank == 0 && tid == 0) {
    if (m >= 2) {
      W.d[m - 2] = A[(int64_t)(m - 2) * m + m - 2];
      W.e[m - 2] = A[(int64_t)(m - 1) * m + m - 2];
      W.beta[m - 2] = 0.0;
    }
    W.d[m - 1] = A[(int64_t)(m - 1) * m + m - 1];
    W.e[m - 1] = 0.0;
    W.beta[m - 1] = 0.0;
    double t = 0.0, gl = 0.0, gu = 0.0;
    for (int i = 0; i < m; ++i) {
      const double di = W.d[i], ei = W.e[i], ep = (i > 0) ? W.e[i - 1] : 0.0;
      t = fmax(t, fabs(di) + fabs(ei));
      const double rad = fabs(ei) + fabs(ep);   // Gershgorin discs
      gl = (i == 0) ? di - rad : fmin(gl, di - rad);
      gu = (i == 0) ? di + rad : fmax(gu, di + rad);
    }
    W.meta[0] = t;
    W.meta[1] = gl;
    W.meta[2] = gu;
  }
}

template <int SL>
cudaError_t launch_tridiag(double* A, int m, int batch, double* work, int64_t ws, cudaStream_t st) {
  const int SR = (m - 1 + TC * NW - 1) / (TC * NW);
  int smem = (int)(sizeof(double) * ((size_t)(4 + NW) * m + (size_t)NW * SR * 33));
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int use_dp = 1;
  if (smem > optin - 1024) {                 // large m: shuffle-reduced row dots
    use_dp = 0;
    smem = (int)(sizeof(double) * (size_t)(4 + NW) * m);
  }
  static const cudaError_t lim = smem_limit_max(syev_tridiag_kernel<SL>);
  cudaError_t e = lim;
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(batch * TC);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = TC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, syev_tridiag_kernel<SL>, A, m, work, ws, use_dp);
}

// ---- 2. eigenvalues ----
// Bisection: one thread per eigenvalue over the whole batch, flattened
// ((matrix, k) pairs in order, BT per block), so the grid is a single wave
// with at most BT threads on any SM (the float64 counts keep the SM's
// float64 pipe busy, so an SM holding two blocks would take twice as long);
// a block stages the scaled T of every matrix its range touches.
constexpr int BT = 128;        // eigenvalues per block of the bisection
__host__ __device__ inline int bisect_mats_per_block(int m) { return (BT - 1) / m + 2; }

__global__ void __launch_bounds__(BT) syev_bisect_kernel(int m, int batch, double* __restrict__ work_all,
                                                         int64_t work_stride, double* __restrict__ wall,
                                                         int* __restrict__ info) {
  extern __shared__ double sm[];   // per matrix: ds[m], e2s[m] (double), dh, dl, eh, el [m] (float)
  const int tid = threadIdx.x;
  const int64_t total = (int64_t)batch * m;
  const int64_t g0 = (int64_t)blockIdx.x * BT;
  const int64_t g1 = (g0 + BT < total) ? g0 + BT : total;
  const int mat0 = (int)(g0 / m);
  const int nmat = (int)((g1 - 1) / m) - mat0 + 1;
  for (int lm = 0; lm < nmat; ++lm) {
    SyevWork W(work_all + (mat0 + lm) * work_stride, m);
    const double tnorm = W.meta[0];
    // scale T by 2^-sc (exact) so that its norm is at most 1
    const int sc = (tnorm > 0.0) ? ilogb(tnorm) + 1 : 0;
    double* ds = sm + (int64_t)lm * 4 * m;
    double* e2s = ds + m;
    float* dh = reinterpret_cast<float*>(e2s + m);
    float* dl = dh + m;
    float* eh = dl + m;
    float* el = eh + m;
    for (int i = tid; i < m; i += BT) {
      const double di = ldexp(W.d[i], -sc), ei = ldexp(W.e[i], -sc);
      ds[i] = di;
      e2s[i] = ei * ei;
      const float2 a = df_split(di), b = df_split(ei * ei);
      dh[i] = a.x; dl[i] = a.y; eh[i] = b.x; el[i] = b.y;
    }
  }
  __syncthreads();
  const int64_t g = g0 + tid;
  if (g >= g1) return;
  const int mat = (int)(g / m), k = (int)(g % m);   // k-th smallest eigenvalue of matrix mat
  SyevWork W(work_all + mat * work_stride, m);
  const double tnorm = W.meta[0];
  const int sc = (tnorm > 0.0) ? ilogb(tnorm) + 1 : 0;
  const double* ds = sm + (int64_t)(mat - mat0) * 4 * m;
  const double* e2s = ds + m;
  const float* dh = reinterpret_cast<const float*>(e2s + m);
  const float* dl = dh + m;
  const float* eh = dl + m;
  const float* el = eh + m;
  const double glo = ldexp(W.meta[1], -sc) - 0x1p-40, ghi = ldexp(W.meta[2], -sc) + 0x1p-40;
  double lo = glo, hi = ghi;
  for (int it = 0; it < 48; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count_df(dh, dl, eh, el, m, mid) > k) hi = mid; else lo = mid;
  }
  // float64 polish: widen, re-verify the bracket with float64 counts, halve
  double wd = 0x1p-44;
  lo -= wd;
  for (int r = 0; r < 40 && lo > glo && sturm_count_f64(ds, e2s, m, lo) > k; ++r) { wd *= 2.0; lo = fmax(lo - wd, glo); }
  wd = 0x1p-44;
  hi += wd;
  for (int r = 0; r < 40 && hi < ghi && sturm_count_f64(ds, e2s, m, hi) <= k; ++r) { wd *= 2.0; hi = fmin(hi + wd, ghi); }
  for (int it = 0; it < 10; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (sturm_count_f64(ds, e2s, m, mid) > k) hi = mid; else lo = mid;
  }
  wall[(int64_t)mat * m + m - 1 - k] = ldexp(0.5 * (lo + hi), sc);
  if (k == 0) info[mat] = 0;
}

// Reference path (precision mode 0): implicit QL without vectors (one
// thread per matrix), then a rank sort.
constexpr int VT = 128;        // threads per block of the QL rank sort
__global__ void __launch_bounds__(VT) syev_values_kernel(int m, double* __restrict__ work_all, int64_t work_stride,
                                                         double* __restrict__ wall, int* __restrict__ info) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x;
  SyevWork W(work_all + blockIdx.x * work_stride, m);
  double* ev = wall + blockIdx.x * (int64_t)m;
  const double tnorm = W.meta[0];
  double* v = sm;
  double* w = v + m;
  __shared__ int ql_fail;
  for (int i = tid; i < m; i += VT) { v[i] = W.d[i]; w[i] = W.e[i]; }
  __syncthreads();
  if (tid == 0) {
    const double t = tnorm;
    int fail = 0;
    for (int l = 0; l < m; ++l) {
      int iter = 0;
      while (true) {
        int mm = l;
        for (; mm < m - 1; ++mm) {
          double dd = fabs(v[mm]) + fabs(v[mm + 1]);
          if (fabs(w[mm]) <= 2.2e-16 * dd || fabs(w[mm]) <= 2.2e-16 * t) break;
        }
        if (mm == l) break;
        if (iter++ >= 100) { fail = 1; break; }
        double g = (v[l + 1] - v[l]) / (2.0 * w[l]);
        double r = hypot(g, 1.0);
        g = v[mm] - v[l] + w[l] / (g + copysign(r, g));
        double s = 1.0, c = 1.0, p = 0.0;
        bool early = false;
        for (int i = mm - 1; i >= l; --i) {
          double f = s * w[i], b = c * w[i];
          // plane rotation from one reciprocal square root: r = |(f, g)|,
          // s = f / r, c = g / r (|f|, |g| <= |T|, so f^2 + g^2 cannot overflow;
          // an underflow to zero is the r == 0 deflation)
          const double t2 = fma(f, f, g * g);
          if (t2 == 0.0) { w[i + 1] = 0.0; v[i + 1] -= p; w[mm] = 0.0; early = true; break; }
          const double ri = rsqrt(t2);
          r = t2 * ri;
          w[i + 1] = r;
          s = f * ri; c = g * ri;
          g = v[i + 1] - p;
          r = (v[i] - g) * s + 2.0 * c * b;
          p = s * r;
          v[i + 1] = g + p;
          g = c * r - b;
        }
        if (!early) { v[l] -= p; w[l] = g; w[mm] = 0.0; }
      }
    }
    ql_fail = fail;
  }
  __syncthreads();
  for (int t = tid; t < m; t += VT) {       // descending (rank of each eigenvalue; ties by index)
    const double x = v[t];
    int rk = 0;
    for (int j = 0; j < m; ++j) rk += (v[j] > x) || (v[j] == x && j < t);
    ev[rk] = x;
  }
  if (tid == 0) info[blockIdx.x] = ql_fail;
}

// PCA rank of Sec. 4 from the descending eigenvalues sigma_k^2 (at least 1).
__device__ int pca_rank_rule(const double* ev, int m, int mode, double thr) {
  int p = m;
  if (mode == RANN_PCA_ABS) {
    p = 0;
    for (int k = 0; k < m; ++k) if (sqrt(fmax(ev[k], 0.0)) > thr) ++p;
  } else if (mode == RANN_PCA_VARIANCE) {
    double tot = 0.0;
    for (int k = 0; k < m; ++k) tot += fmax(ev[k], 0.0);
    double cs = 0.0;
    for (int k = 0; k < m; ++k) {
      cs += fmax(ev[k], 0.0);
      if (cs >= (1.0 - thr) * tot) { p = k + 1; break; }
    }
  }
  return max(p, 1);
}

// ---- 3./4. rank rule and inverse iteration, grid (matrix, part of the vectors) ----
// One thread per kept vector; blocks of VV threads over (matrix, vector
// range), so the few hundred busy threads of a batch spread over the SMs
// (each thread's LU chain loads the SM's float64 pipe).
constexpr int VV = 64;
__global__ void __launch_bounds__(VV) syev_vectors_kernel(int m, double* __restrict__ work_all, int64_t work_stride,
                                                          const double* __restrict__ wall, int* __restrict__ ranks,
                                                          int mode, double thr) {
  extern __shared__ double sm[];
  double* d = sm;
  double* e = d + m;
  __shared__ int prank;
  const int tid = threadIdx.x;
  SyevWork W(work_all + blockIdx.x * work_stride, m);
  const double* ev = wall + blockIdx.x * (int64_t)m;
  if (tid == 0) {
    prank = pca_rank_rule(ev, m, mode, thr);
    if (blockIdx.y == 0) ranks[blockIdx.x] = prank;
  }
  for (int i = tid; i < m; i += VV) { d[i] = W.d[i]; e[i] = W.e[i]; }
  __syncthreads();
  const int p = prank;
  const int k = blockIdx.y * VV + tid;
  if (k >= p) return;
  const double tolp = 2.2e-16 * W.meta[0] + 1e-300;
  const int64_t mm = (int64_t)m * m;
  double* u0 = W.LU + k;                 // entry i at [i * m]
  double* u1 = u0 + mm;
  double* u2 = u1 + mm;
  double* ml = u2 + mm;
  double* xv = ml + mm;
  const double lam = ev[k];
  // LU of T - lam I with partial pivoting.  A row swap at step i is coded
  // in the multiplier as -(mult + 4) (|mult| <= 1 either way).  u0 keeps the
  // reciprocal of each pivot: one division per step, and the solves multiply.
  double cd = d[0] - lam, cs = (m > 1) ? e[0] : 0.0;
#pragma unroll 4
  for (int i = 0; i + 1 < m; ++i) {
    const double sub = e[i];
    const double nd = d[i + 1] - lam, ns = (i + 2 < m) ? e[i + 1] : 0.0;
    double mult, a0, a1, a2;
    const bool swap = fabs(sub) > fabs(cd);
    if (!swap) {
      if (fabs(cd) < tolp) cd = (cd < 0.0) ? -tolp : tolp;
      a0 = 1.0 / cd;
      mult = sub * a0;
      a1 = cs; a2 = 0.0;
      cd = nd - mult * cs;
      cs = ns;
    } else {
      a0 = 1.0 / sub;
      mult = cd * a0;
      a1 = nd; a2 = ns;
      cd = cs - mult * nd;
      cs = -mult * ns;
    }
    u0[(int64_t)i * m] = a0;
    u1[(int64_t)i * m] = a1;
    u2[(int64_t)i * m] = a2;
    ml[(int64_t)i * m] = swap ? -(mult + 4.0) : mult;
  }
  if (fabs(cd) < tolp) cd = (cd < 0.0) ? -tolp : tolp;
  u0[(int64_t)(m - 1) * m] = 1.0 / cd;
  for (int i = 0; i < m; ++i) xv[(int64_t)i * m] = start_entry(i, k);
  for (int it = 0; it < 2; ++it) {
#pragma unroll 4
    for (int i = 0; i + 1 < m; ++i) {      // apply the row swaps and L^{-1}
      double mc = ml[(int64_t)i * m];
      double xi = xv[(int64_t)i * m], xn = xv[(int64_t)(i + 1) * m];
      if (mc <= -3.0) {
        mc = -mc - 4.0;
        const double tmp = xi; xi = xn; xn = tmp;
      }
      xv[(int64_t)i * m] = xi;
      xv[(int64_t)(i + 1) * m] = xn - mc * xi;
    }
    double x1 = 0.0, x2 = 0.0, amax = 0.0;
#pragma unroll 4
    for (int i = m - 1; i >= 0; --i) {      // U^{-1}
      double s = xv[(int64_t)i * m];
      if (i + 1 < m) s -= u1[(int64_t)i * m] * x1;
      if (i + 2 < m) s -= u2[(int64_t)i * m] * x2;
      const double xi = s * u0[(int64_t)i * m];
      xv[(int64_t)i * m] = xi;
      x2 = x1;
      x1 = xi;
      amax = fmax(amax, fabs(xi));
    }
    const double sc = (amax > 0.0 && amax < 1e300) ? 1.0 / amax : 1.0;
    for (int i = 0; i < m; ++i) xv[(int64_t)i * m] *= sc;
  }
  double nrm = 0.0;
  for (int i = 0; i < m; ++i) { const double x = xv[(int64_t)i * m]; nrm = fma(x, x, nrm); }
  const double inv = (nrm > 0.0) ? 1.0 / sqrt(nrm) : 0.0;
  for (int i = 0; i < m; ++i) W.Z[(int64_t)k * m + i] = xv[(int64_t)i * m] * inv;
}

// ---- 4. classical Gram-Schmidt, twice, in descending order; one block per matrix ----
// z_k is staged in shared memory; the k coefficients z_j . z_k are one warp
// each (lanes over the entries, coalesced rows, fixed-order shuffle sum), and
// the subtraction z_k -= sum_j c_j z_j is one thread per entry.
__global__ void __launch_bounds__(NT) syev_orth_kernel(int m, double* __restrict__ work_all, int64_t work_stride,
                                                       const int* __restrict__ ranks) {
  __shared__ double red[33];
  extern __shared__ double sm[];
  double* coef = sm;           // [m]
  double* zs = coef + m;       // [m] current vector
  SyevWork W(work_all + blockIdx.x * work_stride, m);
  double* Z = W.Z;
  const int p = ranks[blockIdx.x], tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 1; k < p; ++k) {
    double* zk = Z + (int64_t)k * m;
    for (int i = tid; i < m; i += NT) zs[i] = zk[i];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = warp; j < k; j += NW) {
        const double* zj = Z + (int64_t)j * m;
        double s0 = 0.0, s1 = 0.0;
        int i = lane;
        for (; i + 32 < m; i += 64) { s0 = fma(zj[i], zs[i], s0); s1 = fma(zj[i + 32], zs[i + 32], s1); }
        if (i < m) s0 = fma(zj[i], zs[i], s0);
        double s = s0 + s1;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) coef[j] = s;
      }
      __syncthreads();
      for (int i = tid; i < m; i += NT) {
        double s0 = zs[i], s1 = 0.0;
        int j = 0;
        for (; j + 1 < k; j += 2) {
          s0 = fma(-coef[j], Z[(int64_t)j * m + i], s0);
          s1 = fma(-coef[j + 1], Z[(int64_t)(j + 1) * m + i], s1);
        }
        if (j < k) s0 = fma(-coef[j], Z[(int64_t)j * m + i], s0);
        zs[i] = s0 + s1;
      }
      __syncthreads();
    }
    double loc = 0.0;
    for (int i = tid; i < m; i += NT) loc = fma(zs[i], zs[i], loc);
    const double nn = block_sum(loc, red);
    const double inv = (nn > 0.0) ? 1.0 / sqrt(nn) : 0.0;
    for (int i = tid; i < m; i += NT) zk[i] = zs[i] * inv;
    __syncthreads();
  }
}

// The same Gram-Schmidt (same order, two passes) in double-float for precision
// mode 1: GB300 issues float32 at 64x its float64 rate, and one block per
// matrix was float64-bound.  Finished vectors are kept as double-float pairs
// in the inverse-iteration workspace (free by now) next to their float64
// copies in Z; coefficients, the current vector and the norm are
// double-float, the final 1/||z|| scaling float64.
__global__ void __launch_bounds__(NT) syev_orth_df_kernel(int m, double* __restrict__ work_all, int64_t work_stride,
                                                          const int* __restrict__ ranks) {
  extern __shared__ float2 smf[];
  float2* coef = smf;          // [m]
  float2* zs = coef + m;       // [m] current vector
  __shared__ float2 red2[NW];
  __shared__ double inv_s;
  SyevWork W(work_all + blockIdx.x * work_stride, m);
  double* Z = W.Z;
  float2* Z2 = reinterpret_cast<float2*>(W.LU);   // [p][m] double-float copies of the finished vectors
  const int p = ranks[blockIdx.x], tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (p > 0)
    for (int i = tid; i < m; i += NT) Z2[i] = df_split(Z[i]);
  for (int k = 1; k < p; ++k) {
    double* zk = Z + (int64_t)k * m;
    for (int i = tid; i < m; i += NT) zs[i] = df_split(zk[i]);
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = warp; j < k; j += NW) {
        const float2* zj = Z2 + (int64_t)j * m;
        float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
        int i = lane;
        for (; i + 32 < m; i += 64) {
          df_mac(h0, l0, zj[i], zs[i]);
          df_mac(h1, l1, zj[i + 32], zs[i + 32]);
        }
        if (i < m) df_mac(h0, l0, zj[i], zs[i]);
        df_add(h0, l0, h1, l1);
        df_warp_sum(h0, l0);
        if (lane == 0) coef[j] = make_float2(-h0, -l0);
      }
      __syncthreads();
      for (int i = tid; i < m; i += NT) {
        float h0 = zs[i].x, l0 = zs[i].y, h1 = 0.f, l1 = 0.f;
        int j = 0;
        for (; j + 1 < k; j += 2) {
          df_mac(h0, l0, coef[j], Z2[(int64_t)j * m + i]);
          df_mac(h1, l1, coef[j + 1], Z2[(int64_t)(j + 1) * m + i]);
        }
        if (j < k) df_mac(h0, l0, coef[j], Z2[(int64_t)j * m + i]);
        df_add(h0, l0, h1, l1);
        zs[i] = make_float2(h0, l0);
      }
      __syncthreads();
    }
    float h = 0.f, l = 0.f;
    for (int i = tid; i < m; i += NT) df_mac(h, l, zs[i], zs[i]);
    df_warp_sum(h, l);
    if (lane == 0) red2[warp] = make_float2(h, l);
    __syncthreads();
    if (tid == 0) {
      float hh = red2[0].x, ll = red2[0].y;
      for (int w = 1; w < NW; ++w) df_add(hh, ll, red2[w].x, red2[w].y);
      const double nn = df_to_double(hh, ll);
      inv_s = (nn > 0.0) ? 1.0 / sqrt(nn) : 0.0;
    }
    __syncthreads();
    const double inv = inv_s;
    for (int i = tid; i < m; i += NT) {
      const double v = df_to_double(zs[i].x, zs[i].y) * inv;
      zk[i] = v;
      Z2[(int64_t)k * m + i] = df_split(v);
    }
    __syncthreads();
  }
}

// ---- 5. back-transformation V = H_0 H_1 ... H_{m-3} Z, one warp per vector ----
constexpr int BW = 8;          // warps (vectors) per block
__global__ void __launch_bounds__(BW * 32) syev_back_kernel(const double* __restrict__ Aall, int m,
                                                            double* __restrict__ work_all, int64_t work_stride,
                                                            const int* __restrict__ ranks) {
  SyevWork W(work_all + blockIdx.x * work_stride, m);
  const double* A = Aall + blockIdx.x * (int64_t)m * m;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.y * BW + (threadIdx.x >> 5);
  if (c >= ranks[blockIdx.x]) return;
  double* z = W.Z + (int64_t)c * m;
  for (int k = m - 3; k >= 0; --k) {
    const double bt = W.beta[k];
    if (bt == 0.0) continue;
    const double* vk = A + (int64_t)k * m + k + 1;
    double s = 0.0;
    for (int i = lane; i < m - k - 1; i += 32) s = fma(vk[i], z[k + 1 + i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    s *= bt;
    for (int i = lane; i < m - k - 1; i += 32) z[k + 1 + i] = fma(-s, vk[i], z[k + 1 + i]);
    __syncwarp();
  }
}

// The same back-transformation in double-float for precision mode 1.  The
// reflectors (upper part of A, row k from column k + 1) are split once into
// the workspace (LU + m^2, row k at k m), and so are the beta_k (after them;
// a beta outside [1e-30, 1e30] is marked NaN and scaled in float64 instead);
// then one warp per vector keeps z in registers (entry lane + 32 t in slot t)
// and, for k = m - 3 .. 0, forms s = -beta_k v_k . z and z += s v_k with
// double-float products (float32 pipe; GB300's float64 unit would otherwise
// carry a conversion, product and split per reflector and vector).  Slots
// wholly above row k + 1 hold zeros of v_k and are skipped.
__global__ void __launch_bounds__(256) syev_back_split_kernel(const double* __restrict__ Aall, int m,
                                                              double* __restrict__ work_all, int64_t work_stride) {
  SyevWork W(work_all + blockIdx.y * work_stride, m);
  const double* A = Aall + blockIdx.y * (int64_t)m * m;
  float2* V2 = reinterpret_cast<float2*>(W.LU + (int64_t)m * m);
  const int64_t tot = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / m), j = (int)(e % m);
    if (k + 1 + j < m) V2[e] = df_split(A[(int64_t)k * m + k + 1 + j]);
  }
  if (blockIdx.x == 0) {
    float2* B2 = V2 + tot;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
      const double bt = W.beta[k];
      const bool ok = bt == 0.0 || (fabs(bt) >= 1e-30 && fabs(bt) <= 1e30);
      B2[k] = ok ? df_split(bt) : make_float2(__int_as_float(0x7fc00000), 0.f);
    }
  }
}

// Slot t of reflector k (entry lane + 32 t, zero outside k < i < m).
template <int SL>
__device__ __forceinline__ void back_load_reflector(const float2* __restrict__ V2, int m, int k, int lane,
                                                    float2 (&v)[SL]) {
  const float2* vk = V2 + (int64_t)k * m - (k + 1);       // vk[i] = v_k entry of z_i, i >= k + 1
#pragma unroll
  for (int t = 0; t < SL; ++t) {
    const int i = lane + 32 * t;
    v[t] = (i > k && i < m) ? vk[i] : make_float2(0.f, 0.f);
  }
}

template <int SL>
__global__ void __launch_bounds__(BW * 32) syev_back_df_kernel(int m, double* __restrict__ work_all,
                                                               int64_t work_stride, const int* __restrict__ ranks) {
  SyevWork W(work_all + blockIdx.x * work_stride, m);
  const float2* V2 = reinterpret_cast<const float2*>(W.LU + (int64_t)m * m);
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.y * BW + (threadIdx.x >> 5);
  if (c >= ranks[blockIdx.x]) return;
  double* z = W.Z + (int64_t)c * m;
  float2 zr[SL];
#pragma unroll
  for (int t = 0; t < SL; ++t) {
    const int i = lane + 32 * t;
    zr[t] = (i < m) ? df_split(z[i]) : make_float2(0.f, 0.f);
  }
  const float2* B2 = V2 + (int64_t)m * m;
  // reflector k - 1 is loaded while k is applied (the loop's only memory traffic)
  float2 vn[SL];
  float2 bn = make_float2(0.f, 0.f);
  if (m >= 3) {
    back_load_reflector<SL>(V2, m, m - 3, lane, vn);
    bn = B2[m - 3];
  }
  for (int k = m - 3; k >= 0; --k) {
    float2 vr[SL];
#pragma unroll
    for (int t = 0; t < SL; ++t) vr[t] = vn[t];
    const float2 b2 = bn;
    if (k > 0) {
      back_load_reflector<SL>(V2, m, k - 1, lane, vn);
      bn = B2[k - 1];
    }
    if (b2.x == 0.f) continue;                              // beta_k = 0
    const int t0 = (k + 1) >> 5;                            // slots t < t0 lie above the reflector
    float h = 0.f, l = 0.f;
#pragma unroll
    for (int t = 0; t < SL; ++t) {
      if (t < t0) continue;
      df_mac(h, l, vr[t], zr[t]);
    }
    df_warp_sum(h, l);
    // s = -beta_k (v_k . z) as a double-float
    float2 sb;
    if (b2.x == b2.x) {
      sb = df_mul(b2, make_float2(h, l));
      sb = make_float2(-sb.x, -sb.y);
    } else {
      sb = df_split(-W.beta[k] * df_to_double(h, l));
    }
#pragma unroll
    for (int t = 0; t < SL; ++t) {
      if (t < t0) continue;
      df_mac(zr[t].x, zr[t].y, sb, vr[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < SL; ++t) {
    const int i = lane + 32 * t;
    if (i < m) z[i] = df_to_double(zr[t].x, zr[t].y);
  }
}

// G <- V: column c of G is eigenvector c (c < p), zero beyond; 32 x 32 tiles.
__global__ void __launch_bounds__(256) syev_output_kernel(double* __restrict__ Aall, int m,
                                                          const double* __restrict__ work_all, int64_t work_stride,
                                                          const int* __restrict__ ranks) {
  __shared__ double tile[32][33];
  const double* Z = work_all + blockIdx.z * work_stride;
  double* A = Aall + blockIdx.z * (int64_t)m * m;
  const int p = ranks[blockIdx.z];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int a = e & 31, b = e >> 5;      // read Z[c0 + b][r0 + a]
    const int c = c0 + b, r = r0 + a;
    tile[b][a] = (c < p && r < m) ? Z[(int64_t)c * m + r] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int a = e & 31, b = e >> 5;      // write A[r0 + b][c0 + a]
    const int r = r0 + b, c = c0 + a;
    if (r < m && c < m) A[(int64_t)r * m + c] = tile[a][b];
  }
}

}  // namespace

int64_t syevd_work_doubles(int m) { return 6 * (int64_t)m * m + 3 * (int64_t)m + 8; }

cudaError_t launch_syev_phase(const SyevBatch& b, int phase, cudaStream_t st) {
  if (b.batch == 0) return cudaSuccess;
  const int m = b.m;
  const int64_t ws = syevd_work_doubles(m);
  cudaError_t e = cudaSuccess;
  switch (phase) {
    case 0: {
      const int sl = (m - 1 + 31) / 32;       // 32-column slots of the longest row
      if (sl <= 4) e = launch_tridiag<4>(b.A, m, b.batch, b.work, ws, st);
      else if (sl <= 8) e = launch_tridiag<8>(b.A, m, b.batch, b.work, ws, st);
      else if (sl <= 12) e = launch_tridiag<12>(b.A, m, b.batch, b.work, ws, st);
      else if (sl <= 16) e = launch_tridiag<16>(b.A, m, b.batch, b.work, ws, st);
      else if (sl <= 24) e = launch_tridiag<24>(b.A, m, b.batch, b.work, ws, st);
      else e = launch_tridiag<32>(b.A, m, b.batch, b.work, ws, st);
      if (e != cudaSuccess) return e;
      break;
    }
    case 1: {
      if (b.bisect) {
        const int64_t total = (int64_t)b.batch * m;
        const int nmat = std::min(b.batch, bisect_mats_per_block(m));
        const int smem = (int)(sizeof(double) * 4 * (size_t)m * nmat);
        static const cudaError_t lim = smem_limit_max(syev_bisect_kernel);
        if ((e = lim) != cudaSuccess) return e;
        syev_bisect_kernel<<<(unsigned)((total + BT - 1) / BT), BT, smem, st>>>(m, b.batch, b.work, ws, b.w, b.info);
      } else {
        const int smem = (int)(sizeof(double) * 2 * m);
        syev_values_kernel<<<b.batch, VT, smem, st>>>(m, b.work, ws, b.w, b.info);
      }
      break;
    }
    case 2: {
      const int smem = (int)(sizeof(double) * 2 * m);
      syev_vectors_kernel<<<dim3(b.batch, (m + VV - 1) / VV), VV, smem, st>>>(m, b.work, ws, b.w, b.ranks, b.mode,
                                                                             b.thr);
      break;
    }
    case 3: {
      const int smem = (int)(sizeof(double) * 2 * m);
      if (b.bisect)     // precision mode 1: double-float Gram-Schmidt
        syev_orth_df_kernel<<<b.batch, NT, smem, st>>>(m, b.work, ws, b.ranks);
      else
        syev_orth_kernel<<<b.batch, NT, smem, st>>>(m, b.work, ws, b.ranks);
      break;
    }
    case 4: {
      if (b.bisect) {   // precision mode 1: double-float back-transformation
        const int64_t tot = (int64_t)m * m;
        syev_back_split_kernel<<<dim3((int)std::min<int64_t>((tot + 255) / 256, 512), b.batch), 256, 0, st>>>(
            b.A, m, b.work, ws);
        const dim3 g(b.batch, (m + BW - 1) / BW);
        const int sl = (m + 31) / 32;
        if (sl <= 4) syev_back_df_kernel<4><<<g, BW * 32, 0, st>>>(m, b.work, ws, b.ranks);
        else if (sl <= 8) syev_back_df_kernel<8><<<g, BW * 32, 0, st>>>(m, b.work, ws, b.ranks);
        else if (sl <= 12) syev_back_df_kernel<12><<<g, BW * 32, 0, st>>>(m, b.work, ws, b.ranks);
        else if (sl <= 16) syev_back_df_kernel<16><<<g, BW * 32, 0, st>>>(m, b.work, ws, b.ranks);
        else if (sl <= 24) syev_back_df_kernel<24><<<g, BW * 32, 0, st>>>(m, b.work, ws, b.ranks);
        else syev_back_df_kernel<32><<<g, BW * 32, 0, st>>>(m, b.work, ws, b.ranks);
      } else {
        syev_back_kernel<<<dim3(b.batch, (m + BW - 1) / BW), BW * 32, 0, st>>>(b.A, m, b.work, ws, b.ranks);
      }
      const int nt = (m + 31) / 32;
      syev_output_kernel<<<dim3(nt, nt, b.batch), 256, 0, st>>>(b.A, m, b.work, ws, b.ranks);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
