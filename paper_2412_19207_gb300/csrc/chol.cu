// Schwarz preconditioner kernels (Sec. 3), float64.
//
// Local matrices A_i = R_i H^T H R_i^T are symmetric positive (semi)definite;
// the paper inverts them through a QR decomposition A_i = Q_i P_i.  Here the
// same matrices are factorised by Cholesky, A_i = L_i L_i^T (the factor is
// P_i^T up to row signs), batched over all subdomains with uneven sizes:
// blocked right-looking, NB = 32 columns per step (diagonal block, panel
// triangular solve, trailing symmetric rank-NB update).  A pivot that is not
// positive (relative to the largest diagonal entry) marks the matrix as
// failed; the host then refactors it with a diagonal shift.
//
// Apply: z = sum_i R_i^T D_i A_i^{-1} R_i r with A_i^{-1} = X_i^T X_i,
// X_i = L_i^{-1} computed once at set-up (block-column-parallel forward
// substitution).  Inverting the triangular factor keeps the error of a
// triangular solve (about kappa(A_i) eps relative, since kappa(L_i)^2 =
// kappa(A_i)), unlike an explicit A_i^{-1}, and turns each apply into two
// fully parallel triangular matrix-vector products instead of sequential
// substitutions.  Per-unknown sums over the sets are formed in a fixed order
// (deterministic, no atomics).
#include "common.cuh"
#include "df32.cuh"

namespace {

constexpr int NB = 32;

__global__ void potrf_diag_kernel(const CholMat* __restrict__ mats, int c0, int* __restrict__ fail,
                                  const double* __restrict__ dmax) {
  const CholMat M = mats[blockIdx.x];
  if (M.n <= c0) return;
  const int nb = min(NB, M.n - c0);
  __shared__ double a[NB][NB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int r = e / nb, c = e % nb;
    a[r][c] = M.A[(int64_t)(c0 + r) * M.ld + c0 + c];
  }
  __syncthreads();
  const double tol = 1e-15 * dmax[blockIdx.x];
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      double piv = a[j][j];
      if (!(piv > tol)) {
        fail[blockIdx.x] = 1;
        piv = fmax(fabs(piv), tol > 0.0 ? tol : 1e-300);
      }
      a[j][j] = sqrt(piv);
    }
    __syncthreads();
    for (int r = j + 1 + threadIdx.x; r < nb; r += blockDim.x) a[r][j] /= a[j][j];
    __syncthreads();
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      int r = e / nb, c = e % nb;
      if (c > j && r >= c) a[r][c] -= a[r][j] * a[c][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int r = e / nb, c = e % nb;
    if (r >= c) M.A[(int64_t)(c0 + r) * M.ld + c0 + c] = a[r][c];
  }
}

// L21 = A21 L11^{-T}: one thread per row below the diagonal block.
__global__ void trsm_panel_kernel(const CholMat* __restrict__ mats, int c0) {
  const CholMat M = mats[blockIdx.y];
  if (M.n <= c0 + NB) return;
  __shared__ double l[NB][NB + 1];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e % NB;
    l[r][c] = M.A[(int64_t)(c0 + r) * M.ld + c0 + c];
  }
  __syncthreads();
  int r = c0 + NB + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M.n) return;
  double x[NB];
  double* row = M.A + (int64_t)r * M.ld + c0;
#pragma unroll
  for (int j = 0; j < NB; ++j) x[j] = row[j];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    double s = x[j];
#pragma unroll
    for (int k = 0; k < j; ++k) s = fma(-x[k], l[j][k], s);
    x[j] = s / l[j][j];
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) row[j] = x[j];
}

// ---- double-float resident factorisation (precision mode 1) ----
// A_i, L_i and L_i^{-1} stay double-float (A2, X2): the 32 x 32 diagonal
// block is factored together with its inverse, which goes to the diagonal
// block of X2; the panel is then L21 = A21 L11^{-T} as a double-float product
// with that inverse, and the trailing update A22 -= L21 L21^T and the
// block-column inverse run on the float32 pipe with no conversions.

// Diagonal block c0 of A2: L11 back to A2 and L11^{-1} to X2, in double-float
// on the float32 pipe (the block is stored in double-float, so float64 here
// would add no accuracy, while GB300's float64 unit makes the serial
// sqrt / divide / update chain of the 32 columns its bottleneck).  Pivots are
// checked against the same tolerance as the float64 path.  Entries accumulate
// their updates unnormalised and are renormalised when read as a pivot or
// column entry.  Per column j: every thread of rows r >= j forms the pivot's
// square root itself (identical values; the diagonal goes to dg) and rows
// r > j scale their entry; then warps 1..7 update the trailing entries while
// warp 0 forms row j of L11^{-1} (lane c: x_jc by forward substitution, which
// needs only rows <= j of L11), so the inverse runs inside the column loop.
__global__ void __launch_bounds__(256) potrf_diag_df_kernel(const CholMat* __restrict__ mats, int c0,
                                                            int* __restrict__ fail, const double* __restrict__ dmax) {
  const CholMat M = mats[blockIdx.x];
  if (M.n <= c0) return;
  const int nb = min(NB, M.n - c0);
  const int tid = threadIdx.x;
  __shared__ float2 a[NB][NB + 1];
  __shared__ float2 xs[NB][NB + 1];   // xs[q][c]: row q of L11^{-1} (lane c of warp 0 owns column c)
  __shared__ float2 dg[NB];
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    a[r][c] = (r < nb && c <= r) ? M.A2[(int64_t)(c0 + r) * M.ld + c0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const double tol = 1e-15 * dmax[blockIdx.x];
  for (int j = 0; j < nb; ++j) {
    if (tid >= j && tid < nb) {
      float2 piv = df_fast(a[j][j].x, a[j][j].y);
      if (!(df_to_double(piv.x, piv.y) > tol)) {
        if (tid == j) fail[blockIdx.x] = 1;
        piv = df_split(fmax(fabs(df_to_double(piv.x, piv.y)), tol > 0.0 ? tol : 1e-300));
      }
      const float2 ljj = df_sqrt(piv);
      if (tid == j) {
        dg[j] = ljj;
      } else {
        float2 v = a[tid][j];
        df_renorm(v.x, v.y);
        a[tid][j] = df_div(v, ljj);
      }
    }
    __syncthreads();
    if (tid >= 32) {
      // a[r][c] -= l_rj l_cj for j < c <= r
      for (int e = tid - 32; e < (nb - j - 1) * NB; e += blockDim.x - 32) {
        const int r = j + 1 + e / NB, c = e % NB;
        if (c > j && r >= c) {
          const float2 lr = a[r][j], lc = a[c][j];
          float h = a[r][c].x, l = a[r][c].y;
          df_mac(h, l, make_float2(-lr.x, -lr.y), lc);
          a[r][c] = make_float2(h, l);
        }
      }
    } else if (tid <= j) {
      // x_jc = (delta_jc - sum_{c <= k < j} l_jk x_kc) / l_jj
      const int c = tid;
      float h0 = (j == c) ? 1.f : 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
      int k = c;
      for (; k + 1 < j; k += 2) {
        const float2 la = a[j][k], lb = a[j][k + 1];
        df_mac(h0, l0, make_float2(-la.x, -la.y), xs[k][c]);
        df_mac(h1, l1, make_float2(-lb.x, -lb.y), xs[k + 1][c]);
      }
      if (k < j) {
        const float2 la = a[j][k];
        df_mac(h0, l0, make_float2(-la.x, -la.y), xs[k][c]);
      }
      df_add(h0, l0, h1, l1);
      const float2 v = df_div(make_float2(h0, l0), dg[j]);
      xs[j][c] = v;
      M.X2[(int64_t)(c0 + j) * M.ld + c0 + c] = v;
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    if (r > c) M.A2[(int64_t)(c0 + r) * M.ld + c0 + c] = a[r][c];
    else if (r == c) M.A2[(int64_t)(c0 + r) * M.ld + c0 + c] = dg[r];
  }
}

// L21 = A21 L11^{-T}: row r of the panel times the stored inverse block, in
// double-float.  A block takes 32 rows (staged in shared memory); warp w forms
// columns 8w .. 8w + 7 of every row (lane = row), so the triangular bound
// on k is the same for the whole warp and no lane idles through it.
__global__ void __launch_bounds__(128) trsm_panel_df_kernel(const CholMat* __restrict__ mats, int c0) {
  const CholMat M = mats[blockIdx.y];
  if (M.n <= c0 + NB) return;
  __shared__ float2 li[NB][NB + 1];
  __shared__ float2 ar[32][NB + 1];
  const int rbase = c0 + NB + blockIdx.x * 32;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    li[r][c] = (c <= r) ? M.X2[(int64_t)(c0 + r) * M.ld + c0 + c] : make_float2(0.f, 0.f);
    ar[r][c] = (rbase + r < M.n) ? M.A2[(int64_t)(rbase + r) * M.ld + c0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int j0 = (threadIdx.x >> 5) * 8;
  float ah[8], al[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) { ah[u] = 0.f; al[u] = 0.f; }
#pragma unroll 1
  for (int k = 0; k < j0 + 8; ++k) {                 // columns j >= k only: L11^{-1} is lower triangular
    const float2 xk = ar[lane][k];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (j0 + u >= k) df_mac(ah[u], al[u], xk, li[j0 + u][k]);
  }
  const int r = rbase + lane;
  if (r < M.n) {
    float2* row = M.A2 + (int64_t)r * M.ld + c0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      df_renorm(ah[u], al[u]);
      row[j0 + u] = make_float2(ah[u], al[u]);
    }
  }
}

// A22 -= L21 L21^T on the lower triangle of A2, double-float.  The panel is
// columns [c0, c0 + NB); the updated region starts at s0 = c0 + NB + skip.
// QN = 4: the whole lower triangle from s0 in 64 x 64 tiles (one block per
// lower tile).  QN = 2: only block column [s0, s0 + NB), rows >= s0, in
// 64 x 32 tiles (one block per 64-row tile; a thread holds QN of the tile's
// 16-column groups).  Each entry is the same fixed-order sum over the panel
// whichever tile holds it, so splitting the update into the next block
// column and the rest changes no result.
template <int QN>
__global__ void __launch_bounds__(256) syrk_update_df_kernel(const CholMat* __restrict__ mats, int c0, int skip) {
  constexpr bool colpart = QN == 2;
  const CholMat M = mats[blockIdx.y];
  const int s0 = c0 + NB + skip + (colpart ? (int)blockIdx.z * NB : 0);   // z: further block columns
  if (M.n <= s0) return;
  const int T = (M.n - s0 + 63) / 64;
  const int t = blockIdx.x;
  int ti, tj;
  if (colpart) {
    if (t >= T) return;
    ti = t;
    tj = 0;
  } else {
    if (t >= T * (T + 1) / 2) return;
    ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    tj = t - ti * (ti + 1) / 2;
  }
  const int cend = colpart ? s0 + NB : M.n;       // columns written: c < cend
  const int r0 = s0 + ti * 64, q0 = s0 + tj * 64;
  __shared__ float2 sa[NB][65];
  __shared__ float2 sb[NB][65];
  for (int e = threadIdx.x; e < 64 * NB; e += 256) {
    const int rr = e / NB, k = e % NB;
    const int r = r0 + rr, q = q0 + rr;
    sa[k][rr] = (r < M.n) ? M.A2[(int64_t)r * M.ld + c0 + k] : make_float2(0.f, 0.f);
    if (rr < 16 * QN) sb[k][rr] = (q < M.n) ? M.A2[(int64_t)q * M.ld + c0 + k] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float ah[4][QN], al[4][QN];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < QN; ++q) { ah[p][q] = 0.f; al[p][q] = 0.f; }
#pragma unroll 4
  for (int k = 0; k < NB; ++k) {
    float2 a[4], b[QN];
#pragma unroll
    for (int p = 0; p < 4; ++p) a[p] = sa[k][ty + 16 * p];
#pragma unroll
    for (int q = 0; q < QN; ++q) b[q] = sb[k][tx + 16 * q];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < QN; q += 2)             // packed float32x2, two columns at a time
        df_mac_2(ah[p][q], al[p][q], ah[p][q + 1], al[p][q + 1], a[p], b[q], a[p], b[q + 1]);
    if ((k & 15) == 15)
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < QN; ++q) df_renorm(ah[p][q], al[p][q]);
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      const int r = r0 + ty + 16 * p, c = q0 + tx + 16 * q;
      if (r < M.n && c <= r && c < cend) {
        float2 v = M.A2[(int64_t)r * M.ld + c];
        df_add(v.x, v.y, -ah[p][q], -al[p][q]);
        M.A2[(int64_t)r * M.ld + c] = v;
      }
    }
}

// ---- triangular inverse X = L^{-1} ----
// Diagonal blocks: X_bb = L_bb^{-1}, one thread per column of the block.
__global__ void trtri_diag_kernel(const CholMat* __restrict__ mats) {
  const CholMat M = mats[blockIdx.y];
  const int nblk = (M.n + NB - 1) / NB;
  if ((int)blockIdx.x >= nblk) return;
  const int b0 = blockIdx.x * NB, nb = min(NB, M.n - b0);
  __shared__ double l[NB][NB + 1];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    int r = e / NB, c = e % NB;
    l[r][c] = (r < nb && c <= r) ? M.A[(int64_t)(b0 + r) * M.ld + b0 + c] : 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c >= nb) return;
  double x[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) x[r] = 0.0;
  for (int r = c; r < nb; ++r) {
    double s = (r == c) ? 1.0 : 0.0;
    for (int k = c; k < r; ++k) s = fma(-l[r][k], x[k], s);
    x[r] = s / l[r][r];
  }
  for (int r = c; r < nb; ++r) M.X[(int64_t)(b0 + r) * M.ld + b0 + c] = x[r];
}

// Row block i of X2 = L^{-1} (double-float, L from A2): for every j < i,
// X_ij = -X_ii sum_{j <= k < i} L_ik X_kj (k in increasing order, each block
// product renormalised); the diagonal blocks X_ii were written by the
// factorisation.  Row block i needs only L's rows of block i (final once
// diagonal block i is factored) and X's row blocks k < i, so it runs inside
// the factorisation's pipeline, one launch per i; grid (j, matrix).
__global__ void __launch_bounds__(256) trtri_row_df_kernel(const CholMat* __restrict__ mats, int i, int jmin) {
  const CholMat M = mats[blockIdx.y];
  const int nblk = (M.n + NB - 1) / NB;
  const int j = (int)blockIdx.x + jmin;
  if (i >= nblk || j >= i) return;
  __shared__ float2 sl[NB][NB + 1];
  __shared__ float2 sx[NB][NB + 1];
  const int t = threadIdx.x, r = t % NB, cg = (t / NB) * 4;   // row r, columns cg..cg+3
  const int cj = j * NB, ri = i * NB;
  const float2 zero = make_float2(0.f, 0.f);
  float ah[4] = {0.f, 0.f, 0.f, 0.f}, al[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k = j; k < i; ++k) {
    const int ck = k * NB;
    for (int e = t; e < NB * NB; e += 256) {
      const int a = e / NB, b = e % NB;
      sl[a][b] = (ri + a < M.n) ? M.A2[(int64_t)(ri + a) * M.ld + ck + b] : zero;   // L_ik
      // X_kj (the diagonal block X_jj is lower triangular: its upper part is never written)
      sx[a][b] = (ck + a < M.n && cj + b < M.n && (k > j || b <= a)) ? M.X2[(int64_t)(ck + a) * M.ld + cj + b]
                                                                     : zero;
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < NB; ++q) {
      const float2 lv = sl[r][q];
#pragma unroll
      for (int u = 0; u < 4; u += 2) df_mac_2(ah[u], al[u], ah[u + 1], al[u + 1], lv, sx[q][cg + u], lv, sx[q][cg + u + 1]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) df_renorm(ah[u], al[u]);
    __syncthreads();
  }
  // X_ij = -X_ii acc
  for (int e = t; e < NB * NB; e += 256) {
    const int a = e / NB, b = e % NB;
    sl[a][b] = (ri + a < M.n && b <= a) ? M.X2[(int64_t)(ri + a) * M.ld + ri + b] : zero;   // X_ii
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) sx[r][cg + u] = make_float2(ah[u], al[u]);
  __syncthreads();
  float oh[4] = {0.f, 0.f, 0.f, 0.f}, ol[4] = {0.f, 0.f, 0.f, 0.f};
  for (int q = 0; q <= r; ++q) {
    const float2 lv = sl[r][q];
#pragma unroll
    for (int u = 0; u < 4; u += 2) df_mac_2(oh[u], ol[u], oh[u + 1], ol[u + 1], lv, sx[q][cg + u], lv, sx[q][cg + u + 1]);
  }
  if (ri + r < M.n)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (cj + cg + u >= M.n) continue;
      df_renorm(oh[u], ol[u]);
      M.X2[(int64_t)(ri + r) * M.ld + cj + cg + u] = make_float2(-oh[u], -ol[u]);
    }
}

// Float64 variant of the trailing update (precision mode 0).
__global__ void __launch_bounds__(256) syrk_update_f64_kernel(const CholMat* __restrict__ mats, int c0) {
  const CholMat M = mats[blockIdx.y];
  const int s0 = c0 + NB;
  if (M.n <= s0) return;
  const int T = (M.n - s0 + 63) / 64;
  const int t = blockIdx.x;
  if (t >= T * (T + 1) / 2) return;
  int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while (ti * (ti + 1) / 2 > t) --ti;
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  const int tj = t - ti * (ti + 1) / 2;
  const int r0 = s0 + ti * 64, q0 = s0 + tj * 64;
  __shared__ double sa[NB][65];
  __shared__ double sb[NB][65];
  for (int e = threadIdx.x; e < 64 * NB; e += 256) {
    int rr = e / NB, k = e % NB;
    int r = r0 + rr, q = q0 + rr;
    sa[k][rr] = (r < M.n) ? M.A[(int64_t)r * M.ld + c0 + k] : 0.0;
    sb[k][rr] = (q < M.n) ? M.A[(int64_t)q * M.ld + c0 + k] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
#pragma unroll 8
  for (int k = 0; k < NB; ++k) {
    double a[4], b[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) { a[p] = sa[k][ty + 16 * p]; b[p] = sb[k][tx + 16 * p]; }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int r = r0 + ty + 16 * p, c = q0 + tx + 16 * q;
      if (r < M.n && c <= r) M.A[(int64_t)r * M.ld + c] -= acc[p][q];
    }
}

// Float64 variant of the block-column triangular inverse (precision mode 0).
__global__ void __launch_bounds__(256) trtri_col_f64_kernel(const CholMat* __restrict__ mats) {
  const CholMat M = mats[blockIdx.y];
  const int nblk = (M.n + NB - 1) / NB;
  const int j = blockIdx.x;
  if (j >= nblk) return;
  __shared__ double sl[NB][NB + 1];
  __shared__ double sx[NB][NB + 1];
  const int t = threadIdx.x, r = t % NB, cg = (t / NB) * 4;
  const int cj = j * NB;
  for (int i = j + 1; i < nblk; ++i) {
    const int ri = i * NB;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = j; k < i; ++k) {
      const int ck = k * NB;
      for (int e = t; e < NB * NB; e += 256) {
        int a = e / NB, b = e % NB;
        sl[a][b] = (ri + a < M.n) ? M.A[(int64_t)(ri + a) * M.ld + ck + b] : 0.0;
        sx[a][b] = (ck + a < M.n && cj + b < M.n && (k > j || b <= a)) ? M.X[(int64_t)(ck + a) * M.ld + cj + b] : 0.0;
      }
      __syncthreads();
#pragma unroll 8
      for (int q = 0; q < NB; ++q) {
        double lv = sl[r][q];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fma(lv, sx[q][cg + u], acc[u]);
      }
      __syncthreads();
    }
    for (int e = t; e < NB * NB; e += 256) {
      int a = e / NB, b = e % NB;
      sl[a][b] = (ri + a < M.n && b <= a) ? M.X[(int64_t)(ri + a) * M.ld + ri + b] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) sx[r][cg + u] = acc[u];
    __syncthreads();
    double out[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q <= r; ++q) {
      double lv = sl[r][q];
#pragma unroll
      for (int u = 0; u < 4; ++u) out[u] = fma(lv, sx[q][cg + u], out[u]);
    }
    if (ri + r < M.n)
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (cj + cg + u < M.n) M.X[(int64_t)(ri + r) * M.ld + cj + cg + u] = -out[u];
    __syncthreads();
  }
}

// ---- apply ----
// Weight of subdomain k's entries in set i when D_i moves to the input side
// (the transposed apply M^T = sum_i R_i^T A_i^{-1} D_i R_i): 0 = none.
__device__ __forceinline__ double input_weight(int wkind, int k, int i, const int* __restrict__ inc_ptr) {
  if (wkind == RANN_PREC_SAS) return 1.0 / (double)(inc_ptr[k + 1] - inc_ptr[k]);
  if (wkind == RANN_PREC_RAS) return k == i ? 1.0 : 0.0;
  return 1.0;
}

// g_i = R_i r (gather the extended-set residual).
__global__ void schwarz_gather_kernel(const int* __restrict__ set_ptr, const int* __restrict__ set_sub,
                                      const SubDev* __restrict__ subs, const int64_t* __restrict__ s_off,
                                      const double* __restrict__ r, double* __restrict__ g, int wkind,
                                      const int* __restrict__ inc_ptr) {
  const int i = blockIdx.x;
  double* gi = g + s_off[i];
  int off = 0;
  for (int q = set_ptr[i]; q < set_ptr[i + 1]; ++q) {
    const SubDev& S = subs[set_sub[q]];
    const double w = input_weight(wkind, set_sub[q], i, inc_ptr);
    for (int c = threadIdx.x; c < S.p; c += blockDim.x) gi[off + c] = w * r[S.woff + c];
    off += S.p;
  }
}

// y_i = X_i g_i, X_i lower triangular: one warp per row.
__global__ void __launch_bounds__(256) trmv_lower_kernel(const CholMat* __restrict__ mats,
                                                         const int64_t* __restrict__ s_off,
                                                         const double* __restrict__ g, double* __restrict__ y) {
  const CholMat M = mats[blockIdx.y];
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= M.n) return;
  const double* row = M.X + (int64_t)r * M.ld;
  const double* gi = g + s_off[blockIdx.y];
  double acc = 0.0;
  for (int c = lane; c <= r; c += 32) acc = fma(row[c], gi[c], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) y[s_off[blockIdx.y] + r] = acc;
}

// partial_i[rc][c] = sum over rows r of chunk rc (r >= c) of X_i[r][c] y_i[r]:
// 256-column tile ct and 256-row chunk rc >= ct, threads across columns.
constexpr int TT = 256;
__global__ void __launch_bounds__(TT) trmv_upper_partial_kernel(const CholMat* __restrict__ mats,
                                                                const int64_t* __restrict__ s_off,
                                                                const int64_t* __restrict__ p_off,
                                                                const double* __restrict__ y,
                                                                double* __restrict__ part) {
  const CholMat M = mats[blockIdx.y];
  const int T = (M.n + TT - 1) / TT;
  const int t = blockIdx.x;
  if (t >= T * (T + 1) / 2) return;
  int rc = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while (rc * (rc + 1) / 2 > t) --rc;
  while ((rc + 1) * (rc + 2) / 2 <= t) ++rc;
  const int ct = t - rc * (rc + 1) / 2;     // ct <= rc
  __shared__ double ys[TT];
  const double* yi = y + s_off[blockIdx.y];
  const int r0 = rc * TT, r1 = min(M.n, r0 + TT);
  for (int q = threadIdx.x; q < r1 - r0; q += TT) ys[q] = yi[r0 + q];
  __syncthreads();
  const int c = ct * TT + threadIdx.x;
  if (c >= M.n) return;
  double acc = 0.0;
  for (int rr = max(r0, c); rr < r1; ++rr) acc = fma(M.X[(int64_t)rr * M.ld + c], ys[rr - r0], acc);
  part[p_off[blockIdx.y] + (int64_t)rc * M.n + c] = acc;
}

// s_i[c] = sum over row chunks rc >= c / 256 of partial_i[rc][c] (fixed order).
__global__ void trmv_upper_reduce_kernel(const CholMat* __restrict__ mats, const int64_t* __restrict__ s_off,
                                         const int64_t* __restrict__ p_off, const double* __restrict__ part,
                                         double* __restrict__ s) {
  const CholMat M = mats[blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= M.n) return;
  const int T = (M.n + TT - 1) / TT;
  double acc = 0.0;
  for (int rc = c / TT; rc < T; ++rc) acc += part[p_off[blockIdx.y] + (int64_t)rc * M.n + c];
  s[s_off[blockIdx.y] + c] = acc;
}

// z[u] = sum over the sets i containing u's subdomain k (fixed order) of D_i(u) s_i[u].
__global__ void schwarz_combine_kernel(const SubDev* __restrict__ subs, int J,
                                       const int* __restrict__ inc_ptr,
                                       const int* __restrict__ inc_set,
                                       const int* __restrict__ inc_pos,
                                       const int64_t* __restrict__ s_off,
                                       const double* __restrict__ s_all, int kind,
                                       double* __restrict__ z) {
  const int k = blockIdx.x;
  const SubDev& S = subs[k];
  const int q0 = inc_ptr[k], nq = min(inc_ptr[k + 1] - q0, 64);
  __shared__ int64_t base[64];                        // s_i offsets of k's block (-1: skipped)
  if ((int)threadIdx.x < nq) {
    const int i = inc_set[q0 + threadIdx.x];
    base[threadIdx.x] = (kind == RANN_PREC_RAS && i != k) ? -1 : s_off[i] + inc_pos[q0 + threadIdx.x];
  }
  __syncthreads();
  const double scale = (kind == RANN_PREC_SAS) ? 1.0 / (double)(inc_ptr[k + 1] - q0) : 1.0;
  for (int c = threadIdx.x; c < S.p; c += blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < nq; ++q)
      if (base[q] >= 0) acc += s_all[base[q] + c];
    z[S.woff + c] = acc * scale;
  }
}

// A_i from the neighbour Gram blocks: block (a, b) of set i is G_{k_a k_b}
// (stored once for k <= l, p_k x p_l row-major; bit 62 of the table entry marks
// a transposed read) or zero when the two boxes share no point.
__global__ void assemble_local_kernel(const double* __restrict__ pairbuf, const int64_t* __restrict__ tab,
                                      const int* __restrict__ tab_ptr, const int* __restrict__ boffs,
                                      const int* __restrict__ boff_ptr, const CholMat* __restrict__ mats,
                                      const int* __restrict__ which) {
  const int i = which ? which[blockIdx.y] : (int)blockIdx.y;
  const CholMat M = mats[i];
  const int* bo = boffs + boff_ptr[i];
  const int nb = boff_ptr[i + 1] - boff_ptr[i] - 1;
  const int64_t* tb = tab + tab_ptr[i];
  const int64_t tot = (int64_t)M.n * M.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(e / M.n), c = (int)(e % M.n);
    int a = 0, b = 0;
    while (a + 1 < nb && bo[a + 1] <= r) ++a;
    while (b + 1 < nb && bo[b + 1] <= c) ++b;
    int64_t ent = tb[a * nb + b];
    double v = 0.0;
    if (ent >= 0) {
      const bool tr = (ent >> 62) & 1;
      const int64_t off = ent & ~((int64_t)1 << 62);
      const int pa = bo[a + 1] - bo[a], pb = bo[b + 1] - bo[b];
      v = tr ? pairbuf[off + (int64_t)(c - bo[b]) * pa + (r - bo[a])]
             : pairbuf[off + (int64_t)(r - bo[a]) * pb + (c - bo[b])];
    }
    if (M.A2) {
      M.A2[(int64_t)r * M.ld + c] = df_split(v);
      continue;
    }
    M.A[(int64_t)r * M.ld + c] = v;
  }
}

__global__ void dmax_kernel(const CholMat* __restrict__ mats, double* __restrict__ dmax,
                            const int* __restrict__ which) {
  const int i = which ? which[blockIdx.x] : (int)blockIdx.x;
  const CholMat M = mats[i];
  double v = 0.0;
  for (int r = threadIdx.x; r < M.n; r += blockDim.x) {
    double d;
    if (M.A2) { const float2 a = M.A2[(int64_t)r * M.ld + r]; d = df_to_double(a.x, a.y); }
    else d = M.A[(int64_t)r * M.ld + r];
    v = fmax(v, d);
  }
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = fmax(s, red[w]);
    dmax[i] = s;
  }
}

__global__ void add_diag_kernel(const CholMat* __restrict__ mats, const int* __restrict__ which,
                                const double* __restrict__ shift) {
  const CholMat M = mats[which[blockIdx.x]];
  const double s = shift[blockIdx.x];
  const float2 s2 = df_split(s);
  for (int r = threadIdx.x; r < M.n; r += blockDim.x) {
    if (M.A2) {
      float2 a = M.A2[(int64_t)r * M.ld + r];
      df_add(a.x, a.y, s2.x, s2.y);
      M.A2[(int64_t)r * M.ld + r] = a;
    } else {
      M.A[(int64_t)r * M.ld + r] += s;
    }
  }
}

// ---- double-float apply (the inner Krylov preconditioner) ----

__global__ void schwarz_gather_df_kernel(const int* __restrict__ set_ptr, const int* __restrict__ set_sub,
                                         const SubDev* __restrict__ subs, const int64_t* __restrict__ s_off,
                                         const double* __restrict__ r, float2* __restrict__ g2, int wkind,
                                         const int* __restrict__ inc_ptr) {
  const int i = blockIdx.x;
  float2* gi = g2 + s_off[i];
  int off = 0;
  for (int q = set_ptr[i]; q < set_ptr[i + 1]; ++q) {
    const SubDev& S = subs[set_sub[q]];
    const double w = input_weight(wkind, set_sub[q], i, inc_ptr);
    for (int c = threadIdx.x; c < S.p; c += blockDim.x) gi[off + c] = df_split(w * r[S.woff + c]);
    off += S.p;
  }
}

// Entry c of a row of L^{-1} in the column-pair layout (h_2k, h_2k+1, l_2k, l_2k+1).
__device__ __forceinline__ float2 x2_entry(const float* row, int c) {
  const int b = 4 * (c >> 1) + (c & 1);
  return make_float2(row[b], row[b + 2]);
}

// After the set-up (precision mode 1): every 16-byte column pair of the lower
// triangles of L^{-1}, written entry by entry as (h_0, l_0, h_1, l_1), becomes
// (h_0, h_1, l_0, l_1), the layout the applies read (the packed float32x2
// operands are then the halves of each load).  Rows are 32-byte aligned
// (ld a multiple of 4).
__global__ void __launch_bounds__(256) x2_pairs_kernel(const CholMat* __restrict__ mats) {
  const CholMat M = mats[blockIdx.y];
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= M.n) return;
  float4* row = reinterpret_cast<float4*>(M.X2 + (int64_t)r * M.ld);
  for (int c2 = threadIdx.x & 31; c2 <= (r >> 1); c2 += 32) {
    const float4 v = row[c2];
    row[c2] = make_float4(v.x, v.z, v.y, v.w);
  }
}

// y2 = X2 g2 (lower triangular) in double-float: one warp per row, four
// independent accumulator chains per lane.
__global__ void __launch_bounds__(256) trmv_lower_df_kernel(const CholMat* __restrict__ mats,
                                                            const int64_t* __restrict__ s_off,
                                                            const float2* __restrict__ g2, float2* __restrict__ y2) {
  const CholMat M = mats[blockIdx.y];
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= M.n) return;
  const float* row = reinterpret_cast<const float*>(M.X2 + (int64_t)r * M.ld);   // pairs (h, h, l, l)
  const float2* gi = g2 + s_off[blockIdx.y];
  float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
  constexpr int U = 8;                                   // independent loads in flight per lane
  for (int c0 = lane; c0 <= r; c0 += 32 * U) {
    float2 a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = (c0 + 32 * u <= r) ? x2_entry(row, c0 + 32 * u) : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (c0 + 32 * u > r) break;
      df_mac(h[u & 3], l[u & 3], a[u], gi[c0 + 32 * u]);
    }
  }
  df_add(h[0], l[0], h[1], l[1]);
  df_add(h[2], l[2], h[3], l[3]);
  df_add(h[0], l[0], h[2], l[2]);
  df_warp_sum(h[0], l[0]);
  if (lane == 0) y2[s_off[blockIdx.y] + r] = make_float2(h[0], l[0]);
}

// partial_i[rc][c] = sum over the rows of 256-row chunk rc (r >= c) of X2[r][c] y2[r]:
// 64 columns x 4 row groups per block, two chains per thread, row groups added
// in shared memory.  Block (ct, rc) with ct the 64-column tile; only chunks
// that reach the lower triangle of the tile do work.
__global__ void __launch_bounds__(256) trmv_upper_df_partial_kernel(const CholMat* __restrict__ mats,
                                                                    const int64_t* __restrict__ s_off,
                                                                    const int64_t* __restrict__ p_off,
                                                                    const float2* __restrict__ y2,
                                                                    double* __restrict__ part) {
  const CholMat M = mats[blockIdx.z];
  const int ct = blockIdx.x, rc = blockIdx.y;
  const int c0 = ct * 64, r0 = rc * TT;
  if (c0 >= M.n || r0 >= M.n || rc < c0 / TT) return;
  const int r1 = min(M.n, r0 + TT);
  __shared__ float2 ys[TT];
  __shared__ float2 red[4][64];
  const float2* yi = y2 + s_off[blockIdx.z];
  for (int q = threadIdx.x; q < r1 - r0; q += 256) ys[q] = yi[r0 + q];
  __syncthreads();
  const int cx = threadIdx.x & 63, rg = threadIdx.x >> 6;
  const int c = c0 + cx;
  float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
  if (c < M.n) {
    int rr = max(r0, c);
    rr += (rg - (rr - r0)) & 3;                       // first row of this group (rows = rg mod 4)
    constexpr int U = 8;                              // rows loaded ahead per thread
    for (; rr < r1; rr += 4 * U) {
      float2 a[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        a[u] = (rr + 4 * u < r1)
                   ? x2_entry(reinterpret_cast<const float*>(M.X2 + (int64_t)(rr + 4 * u) * M.ld), c)
                   : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < U; u += 2) {
        if (rr + 4 * u >= r1) break;
        df_mac(h0, l0, a[u], ys[rr + 4 * u - r0]);
        if (rr + 4 * u + 4 < r1) df_mac(h1, l1, a[u + 1], ys[rr + 4 * u + 4 - r0]);
      }
    }
    df_add(h0, l0, h1, l1);
  }
  red[rg][cx] = make_float2(h0, l0);
  __syncthreads();
  if (rg == 0 && c < M.n) {
    float h = red[0][cx].x, l = red[0][cx].y;
    for (int g = 1; g < 4; ++g) df_add(h, l, red[g][cx].x, red[g][cx].y);
    part[p_off[blockIdx.z] + (int64_t)rc * M.n + c] = df_to_double(h, l);
  }
}

// Fused double-float apply s_i = X_i^T (X_i g_i), g_i = R_i r, for 32-row
// blocks of X_i: the block's y rows are formed from the rows just loaded, and
// the same rows (re-read from L2) give the block's share of X_i^T y, so X_i
// crosses HBM once per apply.  part[rb][c] holds the share of row block rb;
// the last block of a set to finish adds them in a fixed order (rb ascending)
// into s_i.  The set's residual entries are split to double-float and staged
// in shared memory in one flat pass (a small table maps each column to its
// subdomain).  Rows are read as 16-byte pairs of columns (ld is a multiple of
// 4, so every row starts 32-byte aligned); the parts of the triangle away
// from the diagonal run without bounds tests.
constexpr int AR = 32;             // rows per block of the fused apply
constexpr int AMAX_SUB = 27;       // most subdomains in an extended set (3^3)
constexpr int ANT = 256;           // threads per block of the fused apply (four blocks per SM)
// (h0, l0) += a_0 x_0 and (h1, l1) += a_1 x_1 for column pairs stored high
// parts first, (h_0, h_1, l_0, l_1): the layout of L^{-1} after the set-up
// (x2_pairs_kernel) and of the staged vectors, so the packed float32x2
// operands are the two halves of each 16-byte load.
__device__ __forceinline__ void df_mac2(float& h0, float& l0, float& h1, float& l1, float4 a, float4 x) {
  float2 H = make_float2(h0, h1), L = make_float2(l0, l1);
  df_mac_f_x2(H, L, make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(x.x, x.y), make_float2(x.z, x.w));
  h0 = H.x;
  h1 = H.y;
  l0 = L.x;
  l1 = L.y;
}
// The sums of nv vectors of 32 lane partials lp[v * vstride + l], each with
// the pairing of the xor-shuffle warp sum (level o: entry l += entry l + o
// for l < o, o = 16 .. 1; df_add is symmetric, so this is bit for bit the
// value every lane of the shuffle sum ends with), left in entry 0.  The
// calling warp's lanes share the nv * o additions of each level.
__device__ __forceinline__ void df_tree_sum32(float2* lp, int vstride, int nv, int lane) {
  __syncwarp();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    for (int it = lane; it < nv * o; it += 32) {
      float2* e = lp + (it / o) * vstride + (it % o);
      float2 a = e[0];
      const float2 b = e[o];
      df_add(a.x, a.y, b.x, b.y);
      e[0] = a;
    }
    __syncwarp();
  }
}
__global__ void __launch_bounds__(ANT, 4) schwarz_apply_df_kernel(const CholMat* __restrict__ mats,
                                                               const int* __restrict__ set_ptr,
                                                               const int* __restrict__ set_sub,
                                                               const SubDev* __restrict__ subs,
                                                               const double* __restrict__ r,
                                                               const int64_t* __restrict__ p_off32,
                                                               double* __restrict__ part, int wkind,
                                                               const int* __restrict__ inc_ptr,
                                                               const int64_t* __restrict__ s_off,
                                                               double* __restrict__ s, int* __restrict__ done,
                                                               int ckind, double* __restrict__ z,
                                                               const float2* __restrict__ r2) {
  extern __shared__ float4 gs4[];                     // (g_2c, g_2c+1) as double-float pairs
  __shared__ float4 ys4[AR / 2];                      // (y_2q, y_2q+1)
  __shared__ float2 lp[AR][33];                       // lane partials of the y rows (row rr at rr / 8 of warp rr % 8)
  __shared__ int seg_c[AMAX_SUB + 1], seg_p[AMAX_SUB];
  __shared__ int64_t seg_w[AMAX_SUB];
  __shared__ double seg_d[AMAX_SUB];
  __shared__ int last, own_q;
  const int i = blockIdx.y;
  const CholMat M = mats[i];
  const int nb = (M.n + AR - 1) / AR;
  if ((int)blockIdx.x >= nb) return;
  const int rb = nb - 1 - (int)blockIdx.x;            // the long bottom row blocks start first
  const int r0 = rb * AR;
  const int r1 = min(M.n, r0 + AR);
  const int nr = r1 - r0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q0 = set_ptr[i], nq = set_ptr[i + 1] - q0;
  if (tid < nq) {                                     // the set's subdomains, one thread each
    const int k = set_sub[q0 + tid];
    seg_p[tid] = subs[k].p;
    seg_w[tid] = subs[k].woff;
    seg_d[tid] = input_weight(wkind, k, i, inc_ptr);
    if (k == i) own_q = tid;
  }
  __syncthreads();
  if (tid == 0) {
    int c = 0;
    for (int q = 0; q < nq; ++q) { seg_c[q] = c; c += seg_p[q]; }
    seg_c[nq] = c;
  }
  __syncthreads();
  const int np = (r1 + 1) >> 1;                       // column pairs below column r1 (all this block uses)
  for (int c2 = tid; c2 < np; c2 += ANT) {
    float2 v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int c = 2 * c2 + e;
      v[e] = make_float2(0.f, 0.f);
      if (c < r1) {
        int q = 0;
        while (q + 1 < nq && seg_c[q + 1] <= c) ++q;
        // unit weights (the forward apply): the producer's double-float split of r
        v[e] = r2 ? r2[seg_w[q] + (c - seg_c[q])] : df_split(seg_d[q] * r[seg_w[q] + (c - seg_c[q])]);
      }
    }
    gs4[c2] = make_float4(v[0].x, v[1].x, v[0].y, v[1].y);
  }
  if (tid < AR / 2) ys4[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  float2* ys = reinterpret_cast<float2*>(ys4);
  const int ldq = M.ld >> 1;                          // row stride in float4
  // y rows: one warp per row, lane pairs c2 = lane + 32 k; pairs with 2 c2 + 1 <= row are
  // wholly in the triangle, the pair holding the diagonal of an even row has its upper
  // element masked
  for (int rr = warp; rr < nr; rr += ANT / 32) {
    const int row = r0 + rr;
    const float4* xr = reinterpret_cast<const float4*>(M.X2 + (int64_t)row * M.ld);
    const int nfull = (row + 1) >> 1, nall = (row >> 1) + 1;
    float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
    constexpr int U = 4;
    int c2 = lane;
    for (; c2 + 32 * (U - 1) < nfull; c2 += 32 * U) {
      float4 a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) a[u] = xr[c2 + 32 * u];
#pragma unroll
      for (int u = 0; u < U; ++u) df_mac2(h[(2 * u) & 3], l[(2 * u) & 3], h[(2 * u + 1) & 3], l[(2 * u + 1) & 3], a[u],
                                          gs4[c2 + 32 * u]);
    }
    if (c2 < nall) {
      float4 a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int pc = c2 + 32 * u;
        a[u] = (pc < nall) ? xr[pc] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (2 * pc + 1 > row) { a[u].y = 0.f; a[u].w = 0.f; }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (c2 + 32 * u < nall)
          df_mac2(h[(2 * u) & 3], l[(2 * u) & 3], h[(2 * u + 1) & 3], l[(2 * u + 1) & 3], a[u], gs4[c2 + 32 * u]);
    }
    df_add(h[0], l[0], h[1], l[1]);
    df_add(h[2], l[2], h[3], l[3]);
    df_add(h[0], l[0], h[2], l[2]);
    lp[rr][lane] = make_float2(h[0], l[0]);
  }
  // each warp sums the lane partials of its rows (warp, warp + 8, ...)
  if (warp < nr) {
    const int nv = (nr - warp + ANT / 32 - 1) / (ANT / 32);
    df_tree_sum32(&lp[warp][0], (ANT / 32) * 33, nv, lane);
    if (lane < nv) ys[warp + (ANT / 32) * lane] = lp[warp + (ANT / 32) * lane][0];
  }
  __syncthreads();
  // the block's share of X^T y: thread per column pair (c, c + 1), the block's rows r >= c
  for (int c2 = tid; c2 < np; c2 += ANT) {
    const int c = 2 * c2;
    const float4* xc = reinterpret_cast<const float4*>(M.X2 + (int64_t)r0 * M.ld + c);
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f, h3 = 0.f, l3 = 0.f;
    if (nr == AR && c + 1 < r0) {                     // every row of the block is below both columns
#pragma unroll 2
      for (int q = 0; q < AR; q += 4) {
        float4 a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = xc[(q + u) * ldq];
#pragma unroll
        for (int u = 0; u < 4; u += 2) {
          const float4 y = ys4[(q + u) >> 1];
          df_mac2(h0, l0, h1, l1, a[u], make_float4(y.x, y.x, y.y, y.y));
          df_mac2(h2, l2, h3, l3, a[u + 1], make_float4(y.z, y.z, y.w, y.w));
        }
      }
    } else {                                          // diagonal block or short last block
      for (int q = 0; q < nr; q += 4) {
        float4 a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int row = r0 + q + u;
          a[u] = (q + u < nr && row >= c) ? xc[(q + u) * ldq] : make_float4(0.f, 0.f, 0.f, 0.f);
          if (row < c + 1) { a[u].y = 0.f; a[u].w = 0.f; }
        }
#pragma unroll
        for (int u = 0; u < 4; u += 2) {
          const float4 y = ys4[(q + u) >> 1];
          df_mac2(h0, l0, h1, l1, a[u], make_float4(y.x, y.x, y.y, y.y));
          df_mac2(h2, l2, h3, l3, a[u + 1], make_float4(y.z, y.z, y.w, y.w));
        }
      }
    }
    df_add(h0, l0, h2, l2);
    df_add(h1, l1, h3, l3);
    double* pr = part + p_off32[i] + (int64_t)rb * M.n;
    pr[c] = df_to_double(h0, l0);
    if (c + 1 < r1) pr[c + 1] = df_to_double(h1, l1);
  }
  // the last row block of the set to finish adds the parts
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(&done[i], 1) == nb - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (ckind == RANN_PREC_RAS) {
    // restricted combine: z_i = (s_i) restricted to subdomain i's own block, written here
    const int c0 = seg_c[own_q], pc = seg_p[own_q];
    for (int c = c0 + tid; c < c0 + pc; c += ANT) {
      double acc = 0.0;
      for (int b = c / AR; b < nb; ++b) acc += __ldcg(part + p_off32[i] + (int64_t)b * M.n + c);
      z[seg_w[own_q] + (c - c0)] = acc;
    }
  } else {
    for (int c = tid; c < M.n; c += ANT) {
      double acc = 0.0;
      for (int b = c / AR; b < nb; ++b) acc += __ldcg(part + p_off32[i] + (int64_t)b * M.n + c);
      s[s_off[i] + c] = acc;
    }
  }
  if (tid == 0) done[i] = 0;                           // ready for the next apply (stream order)
}

// schwarz_apply_df_kernel for NR right-hand sides r_c = r + c ldr (c < NR) with
// unit input weights and the plain combine (s_c = s + c lds, row-block sums in
// part + c pstride): each row of X_i is read once for all of them; per
// right-hand side the same chains in the same order, so every column is
// bit-identical to the one-vector apply.
template <int NR>
__global__ void __launch_bounds__(ANT, 2) schwarz_apply_multi_kernel(
    const CholMat* __restrict__ mats, const int* __restrict__ set_ptr, const int* __restrict__ set_sub,
    const SubDev* __restrict__ subs, const double* __restrict__ r, int64_t ldr, const int64_t* __restrict__ p_off32,
    double* __restrict__ part, int64_t pstride, const int64_t* __restrict__ s_off, double* __restrict__ s,
    int64_t lds, int* __restrict__ done) {
  extern __shared__ float4 gsm[];                      // [NR][np]
  __shared__ float4 ysm[NR][AR / 2];
  __shared__ float2 lpm[NR][AR][33];                   // lane partials of the y rows per right-hand side
  __shared__ int seg_c[AMAX_SUB + 1], seg_p[AMAX_SUB];
  __shared__ int64_t seg_w[AMAX_SUB];
  __shared__ int last;
  const int i = blockIdx.y;
  const CholMat M = mats[i];
  const int nb = (M.n + AR - 1) / AR;
  if ((int)blockIdx.x >= nb) return;
  const int rb = nb - 1 - (int)blockIdx.x;
  const int r0 = rb * AR;
  const int r1 = min(M.n, r0 + AR);
  const int nr = r1 - r0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q0 = set_ptr[i], nq = set_ptr[i + 1] - q0;
  if (tid < nq) {
    const int k = set_sub[q0 + tid];
    seg_p[tid] = subs[k].p;
    seg_w[tid] = subs[k].woff;
  }
  __syncthreads();
  if (tid == 0) {
    int c = 0;
    for (int q = 0; q < nq; ++q) { seg_c[q] = c; c += seg_p[q]; }
    seg_c[nq] = c;
  }
  __syncthreads();
  const int np = (r1 + 1) >> 1;
  const int npmax = (M.n + 1) >> 1;                    // row stride of gsm (fits the dynamic allocation)
  for (int c2 = tid; c2 < np; c2 += ANT) {
#pragma unroll
    for (int rc = 0; rc < NR; ++rc) {
      float2 v[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = 2 * c2 + e;
        v[e] = make_float2(0.f, 0.f);
        if (c < r1) {
          int q = 0;
          while (q + 1 < nq && seg_c[q + 1] <= c) ++q;
          v[e] = df_split(1.0 * r[rc * ldr + seg_w[q] + (c - seg_c[q])]);
        }
      }
      gsm[rc * npmax + c2] = make_float4(v[0].x, v[1].x, v[0].y, v[1].y);
    }
  }
  if (tid < AR / 2)
#pragma unroll
    for (int rc = 0; rc < NR; ++rc) ysm[rc][tid] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  const int ldq = M.ld >> 1;
  for (int rr = warp; rr < nr; rr += ANT / 32) {
    const int row = r0 + rr;
    const float4* xr = reinterpret_cast<const float4*>(M.X2 + (int64_t)row * M.ld);
    const int nfull = (row + 1) >> 1, nall = (row >> 1) + 1;
    float h[NR][4], l[NR][4];
#pragma unroll
    for (int rc = 0; rc < NR; ++rc)
#pragma unroll
      for (int t = 0; t < 4; ++t) { h[rc][t] = 0.f; l[rc][t] = 0.f; }
    constexpr int U = 4;
    int c2 = lane;
    for (; c2 + 32 * (U - 1) < nfull; c2 += 32 * U) {
      float4 a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) a[u] = xr[c2 + 32 * u];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int rc = 0; rc < NR; ++rc)
          df_mac2(h[rc][(2 * u) & 3], l[rc][(2 * u) & 3], h[rc][(2 * u + 1) & 3], l[rc][(2 * u + 1) & 3], a[u],
                  gsm[rc * npmax + c2 + 32 * u]);
    }
    if (c2 < nall) {
      float4 a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int pc = c2 + 32 * u;
        a[u] = (pc < nall) ? xr[pc] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (2 * pc + 1 > row) { a[u].y = 0.f; a[u].w = 0.f; }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (c2 + 32 * u < nall)
#pragma unroll
          for (int rc = 0; rc < NR; ++rc)
            df_mac2(h[rc][(2 * u) & 3], l[rc][(2 * u) & 3], h[rc][(2 * u + 1) & 3], l[rc][(2 * u + 1) & 3], a[u],
                    gsm[rc * npmax + c2 + 32 * u]);
    }
#pragma unroll
    for (int rc = 0; rc < NR; ++rc) {
      df_add(h[rc][0], l[rc][0], h[rc][1], l[rc][1]);
      df_add(h[rc][2], l[rc][2], h[rc][3], l[rc][3]);
      df_add(h[rc][0], l[rc][0], h[rc][2], l[rc][2]);
      lpm[rc][rr][lane] = make_float2(h[rc][0], l[rc][0]);
    }
  }
  if (warp < nr) {
    const int nv = (nr - warp + ANT / 32 - 1) / (ANT / 32);
#pragma unroll
    for (int rc = 0; rc < NR; ++rc) {
      df_tree_sum32(&lpm[rc][warp][0], (ANT / 32) * 33, nv, lane);
      if (lane < nv) reinterpret_cast<float2*>(ysm[rc])[warp + (ANT / 32) * lane] = lpm[rc][warp + (ANT / 32) * lane][0];
    }
  }
  __syncthreads();
  for (int c2 = tid; c2 < np; c2 += ANT) {
    const int c = 2 * c2;
    const float4* xc = reinterpret_cast<const float4*>(M.X2 + (int64_t)r0 * M.ld + c);
    float acc[NR][8];
#pragma unroll
    for (int rc = 0; rc < NR; ++rc)
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[rc][t] = 0.f;
    const bool fast = (nr == AR && c + 1 < r0);
    for (int q = 0; q < nr; q += 4) {
      float4 a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int row = r0 + q + u;
        if (fast) {
          a[u] = xc[(q + u) * ldq];
        } else {
          a[u] = (q + u < nr && row >= c) ? xc[(q + u) * ldq] : make_float4(0.f, 0.f, 0.f, 0.f);
          if (row < c + 1) { a[u].y = 0.f; a[u].w = 0.f; }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; u += 2)
#pragma unroll
        for (int rc = 0; rc < NR; ++rc) {
          const float4 y = ysm[rc][(q + u) >> 1];
          df_mac2(acc[rc][0], acc[rc][1], acc[rc][2], acc[rc][3], a[u], make_float4(y.x, y.x, y.y, y.y));
          df_mac2(acc[rc][4], acc[rc][5], acc[rc][6], acc[rc][7], a[u + 1], make_float4(y.z, y.z, y.w, y.w));
        }
    }
#pragma unroll
    for (int rc = 0; rc < NR; ++rc) {
      df_add(acc[rc][0], acc[rc][1], acc[rc][4], acc[rc][5]);
      df_add(acc[rc][2], acc[rc][3], acc[rc][6], acc[rc][7]);
      double* pr = part + rc * pstride + p_off32[i] + (int64_t)rb * M.n;
      pr[c] = df_to_double(acc[rc][0], acc[rc][1]);
      if (c + 1 < r1) pr[c + 1] = df_to_double(acc[rc][2], acc[rc][3]);
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(&done[i], 1) == nb - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int c = tid; c < M.n; c += ANT)
#pragma unroll
    for (int rc = 0; rc < NR; ++rc) {
      double a = 0.0;
      for (int b = c / AR; b < nb; ++b) a += __ldcg(part + rc * pstride + p_off32[i] + (int64_t)b * M.n + c);
      s[rc * lds + s_off[i] + c] = a;
    }
  if (tid == 0) done[i] = 0;
}

// schwarz_combine_kernel for column blockIdx.y (s_c = s_all + c lds, z_c = z + c ldz)
__global__ void schwarz_combine_multi_kernel(const SubDev* __restrict__ subs, const int* __restrict__ inc_ptr,
                                             const int* __restrict__ inc_set, const int* __restrict__ inc_pos,
                                             const int64_t* __restrict__ s_off, const double* __restrict__ s_all,
                                             int64_t lds, int kind, double* __restrict__ z, int64_t ldz) {
  const int k = blockIdx.x, col = blockIdx.y;
  const SubDev& S = subs[k];
  const int q0 = inc_ptr[k], nq = min(inc_ptr[k + 1] - q0, 64);
  __shared__ int64_t base[64];
  if ((int)threadIdx.x < nq) {
    const int i = inc_set[q0 + threadIdx.x];
    base[threadIdx.x] = (kind == RANN_PREC_RAS && i != k) ? -1 : s_off[i] + inc_pos[q0 + threadIdx.x];
  }
  __syncthreads();
  const double scale = (kind == RANN_PREC_SAS) ? 1.0 / (double)(inc_ptr[k + 1] - q0) : 1.0;
  const double* sc = s_all + col * lds;
  for (int c = threadIdx.x; c < S.p; c += blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < nq; ++q)
      if (base[q] >= 0) acc += sc[base[q] + c];
    z[col * ldz + S.woff + c] = acc * scale;
  }
}

// X2 = split(X) on the lower triangles.
__global__ void split_lower_kernel(const CholMat* __restrict__ mats) {
  const CholMat M = mats[blockIdx.y];
  const int64_t tot = (int64_t)M.n * M.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / M.n), c = (int)(e % M.n);
    if (c <= r) M.X2[(int64_t)r * M.ld + c] = df_split(M.X[(int64_t)r * M.ld + c]);
  }
}

}  // namespace

cudaError_t launch_split_lower(const CholMat* d_mats, int nmat, int maxn, cudaStream_t st) {
  if (nmat == 0) return cudaSuccess;
  int64_t tot = (int64_t)maxn * maxn;
  int gx = (int)((tot + 255) / 256);
  if (gx > 2048) gx = 2048;
  split_lower_kernel<<<dim3(gx, nmat), 256, 0, st>>>(d_mats);
  return cudaGetLastError();
}

cudaError_t launch_schwarz_gather_df(int nsets, const int* d_set_ptr, const int* d_set_sub, const SubDev* d_sub,
                                     const int64_t* d_s_off, const double* d_r, float2* d_g2, int wkind,
                                     const int* d_inc_ptr, cudaStream_t st) {
  schwarz_gather_df_kernel<<<nsets, 256, 0, st>>>(d_set_ptr, d_set_sub, d_sub, d_s_off, d_r, d_g2, wkind, d_inc_ptr);
  return cudaGetLastError();
}

cudaError_t launch_x2_pairs(const CholMat* d_mats, int nsets, int maxn, cudaStream_t st) {
  if (nsets == 0 || maxn == 0) return cudaSuccess;
  x2_pairs_kernel<<<dim3((maxn + 7) / 8, nsets), 256, 0, st>>>(d_mats);
  return cudaGetLastError();
}

cudaError_t launch_trmv_lower_df(const CholMat* d_mats, int nsets, int maxn, const int64_t* d_s_off,
                                 const float2* d_g2, float2* d_y2, cudaStream_t st) {
  trmv_lower_df_kernel<<<dim3((maxn + 7) / 8, nsets), 256, 0, st>>>(d_mats, d_s_off, d_g2, d_y2);
  return cudaGetLastError();
}

cudaError_t launch_trmv_upper_df(const CholMat* d_mats, int nsets, int maxn, const int64_t* d_s_off,
                                 const int64_t* d_p_off, const float2* d_y2, double* d_part, double* d_s,
                                 cudaStream_t st) {
  int T = (maxn + TT - 1) / TT;
  trmv_upper_df_partial_kernel<<<dim3((maxn + 63) / 64, T, nsets), 256, 0, st>>>(d_mats, d_s_off, d_p_off, d_y2,
                                                                                 d_part);
  trmv_upper_reduce_kernel<<<dim3((maxn + 255) / 256, nsets), 256, 0, st>>>(d_mats, d_s_off, d_p_off, d_part, d_s);
  return cudaGetLastError();
}

cudaError_t launch_assemble_local(const double* d_pairbuf, const int64_t* d_tab, const int* d_tab_ptr,
                                  const int* d_boff, const int* d_boff_ptr, const CholMat* d_mats, int nsets,
                                  int maxn, double* d_dmax, cudaStream_t st, const int* d_which) {
  if (nsets == 0) return cudaSuccess;
  int64_t tot = (int64_t)maxn * maxn;
  int gx = (int)((tot + 255) / 256);
  if (gx > 2048) gx = 2048;
  assemble_local_kernel<<<dim3(gx, nsets), 256, 0, st>>>(d_pairbuf, d_tab, d_tab_ptr, d_boff, d_boff_ptr, d_mats,
                                                          d_which);
  dmax_kernel<<<nsets, 256, 0, st>>>(d_mats, d_dmax, d_which);
  return cudaGetLastError();
}

cudaError_t launch_add_diag(const CholMat* d_mats, const int* d_which, int nwhich, const double* d_shift,
                            int /*maxn*/, cudaStream_t st) {
  if (nwhich == 0) return cudaSuccess;
  add_diag_kernel<<<nwhich, 256, 0, st>>>(d_mats, d_which, d_shift);
  return cudaGetLastError();
}

// One serial step of the float64 factorisation (precision mode 0).
cudaError_t launch_chol_step(const CholMat* d_mats, int nmat, int maxn, int c0, int* d_fail,
                             const double* d_dmax, cudaStream_t st) {
  const int rest = maxn - c0 - NB;
  const int T = (rest + 63) / 64;
  potrf_diag_kernel<<<nmat, 256, 0, st>>>(d_mats, c0, d_fail, d_dmax);
  if (rest > 0) {
    trsm_panel_kernel<<<dim3((rest + 127) / 128, nmat), 128, 0, st>>>(d_mats, c0);
    syrk_update_f64_kernel<<<dim3(T * (T + 1) / 2, nmat), 256, 0, st>>>(d_mats, c0);
  }
  return cudaGetLastError();
}

// The whole double-float factorisation with one block column of lookahead,
// and X = L^{-1} by row blocks inside the same pipeline.  Step s (c0 = s NB)
// splits its trailing update into block column s + 1 and the rest (columns
// >= c0 + 2 NB).  The critical path -- block column s + 1, its diagonal
// block, its panel -- runs on st2 (high priority) while the rest of step s
// runs on st; row block s + 1 of X runs on st3 once diagonal block s + 1 is
// factored.  So the latency-bound diagonal factorisations overlap the
// throughput-bound updates and inverse.  Order per entry is the serial one:
// block column s + 1 is updated by step s only after the rest of step s - 1
// (evR), the rest of step s starts only after panel s (evT), row block i of
// X after diagonal block i (evP; L's rows of block i are final by then) and
// after row block i - 1 (stream order); the regions written concurrently are
// disjoint.  ev: seven events (fork / join, two each for panels, rests and
// diagonal blocks).  *nlaunch: kernels launched.
cudaError_t launch_chol_df_lookahead(const CholMat* d_mats, int nmat, int maxn, int* d_fail, const double* d_dmax,
                                     cudaStream_t st, cudaStream_t st2, cudaStream_t st3, cudaEvent_t* ev,
                                     int* nlaunch) {
  int n = 0;
  cudaError_t e;
  auto potrf = [&](int c0) {
    potrf_diag_df_kernel<<<nmat, NB * 8, 0, st2>>>(d_mats, c0, d_fail, d_dmax);
    ++n;
  };
  auto trsm = [&](int c0) {
    trsm_panel_df_kernel<<<dim3((maxn - c0 - NB + 31) / 32, nmat), 128, 0, st2>>>(d_mats, c0);
    ++n;
  };
  auto syrk = [&](int c0, int skip, int colpart, cudaStream_t s) {
    const int T = (maxn - c0 - NB - skip + 63) / 64;
    if (colpart)
      syrk_update_df_kernel<2><<<dim3(T, nmat), 256, 0, s>>>(d_mats, c0, skip);
    else
      syrk_update_df_kernel<4><<<dim3(T * (T + 1) / 2, nmat), 256, 0, s>>>(d_mats, c0, skip);
    ++n;
  };
  const int nsteps = (maxn + NB - 1) / NB;
  if ((e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(st2, ev[0], 0)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(st3, ev[0], 0)) != cudaSuccess) return e;
  potrf(0);
  if (nsteps > 1) trsm(0);
  if ((e = cudaEventRecord(ev[1], st2)) != cudaSuccess) return e;
  for (int s = 0; s + 1 < nsteps; ++s) {
    const int c0 = s * NB;
    const bool more = maxn > c0 + 2 * NB;          // columns beyond block column s + 1
    if ((e = cudaStreamWaitEvent(st, ev[1 + (s & 1)], 0)) != cudaSuccess) return e;   // panel s
    if (more) syrk(c0, NB, 0, st);
    if ((e = cudaEventRecord(ev[3 + (s & 1)], st)) != cudaSuccess) return e;
    if (s >= 1 && (e = cudaStreamWaitEvent(st2, ev[3 + ((s - 1) & 1)], 0)) != cudaSuccess) return e;   // rest s - 1
    syrk(c0, 0, 1, st2);
    potrf(c0 + NB);
    if ((e = cudaEventRecord(ev[5 + (s & 1)], st2)) != cudaSuccess) return e;
    if (more) trsm(c0 + NB);
    if ((e = cudaEventRecord(ev[1 + ((s + 1) & 1)], st2)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st3, ev[5 + (s & 1)], 0)) != cudaSuccess) return e;   // diagonal block s + 1
    trtri_row_df_kernel<<<dim3(s + 1, nmat), 256, 0, st3>>>(d_mats, s + 1, 0);
    ++n;
  }
  if ((e = cudaEventRecord(ev[0], st2)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(st, ev[0], 0)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(ev[0], st3)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(st, ev[0], 0)) != cudaSuccess) return e;
  *nlaunch = n;
  return cudaGetLastError();
}

// Pieces of the big-panel factorisation (chol_tc.cu): the 32-column steps
// inside a panel of columns [c0, c1).
cudaError_t launch_panel_steps_df(const CholMat* d_mats, int nmat, int maxn, int c0, int c1, int* d_fail,
                                  const double* d_dmax, cudaStream_t st, int* nlaunch) {
  int n = 0;
  for (int b = c0; b < c1 && b < maxn; b += NB) {
    potrf_diag_df_kernel<<<nmat, NB * 8, 0, st>>>(d_mats, b, d_fail, d_dmax);
    ++n;
    if (maxn > b + NB) {
      trsm_panel_df_kernel<<<dim3((maxn - b - NB + 31) / 32, nmat), 128, 0, st>>>(d_mats, b);
      ++n;
    }
    const int nz = (c1 - b - NB + NB - 1) / NB;      // block columns of the panel right of b
    if (nz > 0 && maxn > b + NB) {
      const int T = (maxn - b - NB + 63) / 64;
      syrk_update_df_kernel<2><<<dim3(T, nmat, nz), 256, 0, st>>>(d_mats, b, 0);
      ++n;
    }
    const int i = b / NB, jmin = c0 / NB;
    if (i > jmin) {
      trtri_row_df_kernel<<<dim3(i - jmin, nmat), 256, 0, st>>>(d_mats, i, jmin);
      ++n;
    }
  }
  *nlaunch += n;
  return cudaGetLastError();
}

// X = L^{-1} in float64 (precision mode 0; mode 1 forms it inside the
// factorisation's pipeline).
cudaError_t launch_trtri(const CholMat* d_mats, int nmat, int maxn, cudaStream_t st) {
  if (nmat == 0) return cudaSuccess;
  int nblk = (maxn + NB - 1) / NB;
  trtri_diag_kernel<<<dim3(nblk, nmat), NB, 0, st>>>(d_mats);
  trtri_col_f64_kernel<<<dim3(nblk, nmat), 256, 0, st>>>(d_mats);
  return cudaGetLastError();
}

cudaError_t launch_schwarz_gather(int nsets, const int* d_set_ptr, const int* d_set_sub, const SubDev* d_sub,
                                  const int64_t* d_s_off, const double* d_r, double* d_g, int wkind,
                                  const int* d_inc_ptr, cudaStream_t st) {
  schwarz_gather_kernel<<<nsets, 256, 0, st>>>(d_set_ptr, d_set_sub, d_sub, d_s_off, d_r, d_g, wkind, d_inc_ptr);
  return cudaGetLastError();
}

cudaError_t launch_trmv_lower(const CholMat* d_mats, int nsets, int maxn, const int64_t* d_s_off,
                              const double* d_g, double* d_y, cudaStream_t st) {
  trmv_lower_kernel<<<dim3((maxn + 7) / 8, nsets), 256, 0, st>>>(d_mats, d_s_off, d_g, d_y);
  return cudaGetLastError();
}

cudaError_t launch_trmv_upper(const CholMat* d_mats, int nsets, int maxn, const int64_t* d_s_off,
                              const int64_t* d_p_off, const double* d_y, double* d_part, double* d_s,
                              cudaStream_t st) {
  int T = (maxn + TT - 1) / TT;
  trmv_upper_partial_kernel<<<dim3(T * (T + 1) / 2, nsets), TT, 0, st>>>(d_mats, d_s_off, d_p_off, d_y, d_part);
  trmv_upper_reduce_kernel<<<dim3((maxn + 255) / 256, nsets), 256, 0, st>>>(d_mats, d_s_off, d_p_off, d_part, d_s);
  return cudaGetLastError();
}

cudaError_t launch_schwarz_combine(const SubDev* d_sub, int J, const int* d_inc_ptr,
                                   const int* d_inc_set, const int* d_inc_pos,
                                   const int64_t* d_s_off, const double* d_s, int kind, double* d_z,
                                   cudaStream_t st) {
  if (J == 0) return cudaSuccess;
  schwarz_combine_kernel<<<J, 256, 0, st>>>(d_sub, J, d_inc_ptr, d_inc_set, d_inc_pos, d_s_off, d_s,
                                             kind, d_z);
  return cudaGetLastError();
}

template <int NR>
static cudaError_t apply_multi_launch(const CholMat* d_mats, int nsets, int maxn, const int* d_set_ptr,
                                      const int* d_set_sub, const SubDev* d_sub, const double* d_r, int64_t ldr,
                                      const int64_t* d_p_off32, double* d_part, int64_t pstride,
                                      const int64_t* d_s_off, double* d_s, int64_t lds, int* d_done, cudaStream_t st) {
  const int smem = (int)(sizeof(float4) * (size_t)((maxn + 1) / 2) * NR);
  static const cudaError_t lim = smem_limit_max(schwarz_apply_multi_kernel<NR>);
  if (lim != cudaSuccess) return lim;
  schwarz_apply_multi_kernel<NR><<<dim3((maxn + AR - 1) / AR, nsets), ANT, smem, st>>>(
      d_mats, d_set_ptr, d_set_sub, d_sub, d_r, ldr, d_p_off32, d_part, pstride, d_s_off, d_s, lds, d_done);
  return cudaGetLastError();
}

cudaError_t launch_schwarz_apply_multi(const CholMat* d_mats, int nsets, int maxn, const int* d_set_ptr,
                                       const int* d_set_sub, const SubDev* d_sub, const double* d_r, int64_t ldr,
                                       const int64_t* d_p_off32, double* d_part, int64_t pstride,
                                       const int64_t* d_s_off, double* d_s, int64_t lds, int* d_done, int nrhs,
                                       const int* d_inc_ptr, const int* d_inc_set, const int* d_inc_pos, int J,
                                       int ckind, double* d_z, int64_t ldz, cudaStream_t st) {
  if (nsets == 0 || nrhs == 0) return cudaSuccess;
  for (int c0 = 0; c0 < nrhs; c0 += 4) {              // four right-hand sides per launch
    const int k = nrhs - c0 < 4 ? nrhs - c0 : 4;
    const double* r = d_r + c0 * ldr;
    double* s = d_s + c0 * lds;
    cudaError_t e = k == 4 ? apply_multi_launch<4>(d_mats, nsets, maxn, d_set_ptr, d_set_sub, d_sub, r, ldr, d_p_off32,
                                                   d_part, pstride, d_s_off, s, lds, d_done, st)
                  : k == 3 ? apply_multi_launch<3>(d_mats, nsets, maxn, d_set_ptr, d_set_sub, d_sub, r, ldr, d_p_off32,
                                                   d_part, pstride, d_s_off, s, lds, d_done, st)
                  : k == 2 ? apply_multi_launch<2>(d_mats, nsets, maxn, d_set_ptr, d_set_sub, d_sub, r, ldr, d_p_off32,
                                                   d_part, pstride, d_s_off, s, lds, d_done, st)
                           : apply_multi_launch<1>(d_mats, nsets, maxn, d_set_ptr, d_set_sub, d_sub, r, ldr, d_p_off32,
                                                   d_part, pstride, d_s_off, s, lds, d_done, st);
    if (e != cudaSuccess) return e;
  }
  schwarz_combine_multi_kernel<<<dim3(J, nrhs), 256, 0, st>>>(d_sub, d_inc_ptr, d_inc_set, d_inc_pos, d_s_off, d_s,
                                                              lds, ckind, d_z, ldz);
  return cudaGetLastError();
}

int schwarz_apply_rows() { return AR; }
int schwarz_apply_max_subs() { return AMAX_SUB; }

cudaError_t launch_schwarz_apply_df(const CholMat* d_mats, int nsets, int maxn, const int* d_set_ptr,
                                    const int* d_set_sub, const SubDev* d_sub, const double* d_r,
                                    const int64_t* d_s_off, const int64_t* d_p_off32, double* d_part, double* d_s,
                                    int* d_done, int wkind, const int* d_inc_ptr, int ckind, double* d_z,
                                    cudaStream_t st, const float2* d_r2) {
  if (nsets == 0) return cudaSuccess;
  const int smem = (int)(sizeof(float4) * (size_t)((maxn + 1) / 2));
  static const cudaError_t lim = smem_limit_max(schwarz_apply_df_kernel);
  if (lim != cudaSuccess) return lim;
  schwarz_apply_df_kernel<<<dim3((maxn + AR - 1) / AR, nsets), ANT, smem, st>>>(
      d_mats, d_set_ptr, d_set_sub, d_sub, d_r, d_p_off32, d_part, wkind, d_inc_ptr, d_s_off, d_s, d_done, ckind, d_z,
      wkind == RANN_PREC_AS ? d_r2 : nullptr);
  return cudaGetLastError();
}
