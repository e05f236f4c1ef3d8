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
// Apply: z = sum_i R_i^T D_i A_i^{-1} R_i r: each subdomain gathers its
// extended-set residual, runs the forward and backward substitutions, and
// the per-unknown sums over the sets are formed in a fixed order
// (deterministic, no atomics).
#include "common.cuh"

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

// A22 -= L21 L21^T on the lower triangle, 64 x 64 tiles.
__global__ void __launch_bounds__(256) syrk_update_kernel(const CholMat* __restrict__ mats, int c0) {
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

// ---- apply ----
// Each extended set i: gather r_i, solve L y = r_i, L^T s = y, store s_i.
__global__ void __launch_bounds__(256) local_solve_kernel(const CholMat* __restrict__ mats,
                                                          const int* __restrict__ set_ptr,
                                                          const int* __restrict__ set_sub,
                                                          const SubDev* __restrict__ subs,
                                                          const int64_t* __restrict__ s_off,
                                                          const double* __restrict__ r,
                                                          double* __restrict__ s_all) {
  const int i = blockIdx.x;
  const CholMat M = mats[i];
  double* y = s_all + s_off[i];
  // gather
  int off = 0;
  for (int q = set_ptr[i]; q < set_ptr[i + 1]; ++q) {
    const SubDev& S = subs[set_sub[q]];
    for (int c = threadIdx.x; c < S.p; c += blockDim.x) y[off + c] = r[S.woff + c];
    off += S.p;
  }
  __syncthreads();
  const int n = M.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // forward: L y = r
  for (int b0 = 0; b0 < n; b0 += NB) {
    const int nb = min(NB, n - b0);
    if (warp == 0) {
      double yl = (lane < nb) ? y[b0 + lane] : 0.0;
      for (int j = 0; j < nb; ++j) {
        if (lane == j) yl /= M.A[(int64_t)(b0 + j) * M.ld + b0 + j];
        double yj = __shfl_sync(0xffffffffu, yl, j);
        if (lane > j && lane < nb) yl = fma(-M.A[(int64_t)(b0 + lane) * M.ld + b0 + j], yj, yl);
      }
      if (lane < nb) y[b0 + lane] = yl;
    }
    __syncthreads();
    for (int rr = b0 + nb + threadIdx.x; rr < n; rr += blockDim.x) {
      const double* Lr = M.A + (int64_t)rr * M.ld + b0;
      double s = y[rr];
      for (int k = 0; k < nb; ++k) s = fma(-Lr[k], y[b0 + k], s);
      y[rr] = s;
    }
    __syncthreads();
  }
  // backward: L^T s = y
  const int nblk = (n + NB - 1) / NB;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int b0 = bi * NB;
    const int nb = min(NB, n - b0);
    if (warp == 0) {
      double yl = (lane < nb) ? y[b0 + lane] : 0.0;
      for (int j = nb - 1; j >= 0; --j) {
        if (lane == j) yl /= M.A[(int64_t)(b0 + j) * M.ld + b0 + j];
        double yj = __shfl_sync(0xffffffffu, yl, j);
        if (lane < j) yl = fma(-M.A[(int64_t)(b0 + j) * M.ld + b0 + lane], yj, yl);
      }
      if (lane < nb) y[b0 + lane] = yl;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < b0; c += blockDim.x) {
      double s = y[c];
      for (int k = 0; k < nb; ++k) s = fma(-M.A[(int64_t)(b0 + k) * M.ld + c], y[b0 + k], s);
      y[c] = s;
    }
    __syncthreads();
  }
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
  const int q0 = inc_ptr[k], q1 = inc_ptr[k + 1];
  const double scale = (kind == RANN_PREC_SAS) ? 1.0 / (double)(q1 - q0) : 1.0;
  for (int c = threadIdx.x; c < S.p; c += blockDim.x) {
    double acc = 0.0;
    for (int q = q0; q < q1; ++q) {
      int i = inc_set[q];
      if (kind == RANN_PREC_RAS && i != k) continue;
      acc += s_all[s_off[i] + inc_pos[q] + c];
    }
    z[S.woff + c] = acc * scale;
  }
}

// A_i from the neighbour Gram blocks: block (a, b) of set i is G_{k_a k_b}
// (stored once for k <= l, p_k x p_l row-major; bit 62 of the table entry marks
// a transposed read) or zero when the two boxes share no point.
__global__ void assemble_local_kernel(const double* __restrict__ pairbuf, const int64_t* __restrict__ tab,
                                      const int* __restrict__ tab_ptr, const int* __restrict__ boffs,
                                      const int* __restrict__ boff_ptr, const CholMat* __restrict__ mats) {
  const int i = blockIdx.y;
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
    M.A[(int64_t)r * M.ld + c] = v;
  }
}

__global__ void dmax_kernel(const CholMat* __restrict__ mats, double* __restrict__ dmax) {
  const CholMat M = mats[blockIdx.x];
  double v = 0.0;
  for (int r = threadIdx.x; r < M.n; r += blockDim.x) v = fmax(v, M.A[(int64_t)r * M.ld + r]);
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = fmax(s, red[w]);
    dmax[blockIdx.x] = s;
  }
}

__global__ void add_diag_kernel(const CholMat* __restrict__ mats, const int* __restrict__ which,
                                const double* __restrict__ shift) {
  const CholMat M = mats[which[blockIdx.x]];
  const double s = shift[blockIdx.x];
  for (int r = threadIdx.x; r < M.n; r += blockDim.x) M.A[(int64_t)r * M.ld + r] += s;
}

}  // namespace

cudaError_t launch_assemble_local(const double* d_pairbuf, const int64_t* d_tab, const int* d_tab_ptr,
                                  const int* d_boff, const int* d_boff_ptr, const CholMat* d_mats, int nsets,
                                  int maxn, double* d_dmax, cudaStream_t st) {
  if (nsets == 0) return cudaSuccess;
  int64_t tot = (int64_t)maxn * maxn;
  int gx = (int)((tot + 255) / 256);
  if (gx > 2048) gx = 2048;
  assemble_local_kernel<<<dim3(gx, nsets), 256, 0, st>>>(d_pairbuf, d_tab, d_tab_ptr, d_boff, d_boff_ptr, d_mats);
  dmax_kernel<<<nsets, 256, 0, st>>>(d_mats, d_dmax);
  return cudaGetLastError();
}

cudaError_t launch_add_diag(const CholMat* d_mats, const int* d_which, int nwhich, const double* d_shift,
                            int /*maxn*/, cudaStream_t st) {
  if (nwhich == 0) return cudaSuccess;
  add_diag_kernel<<<nwhich, 256, 0, st>>>(d_mats, d_which, d_shift);
  return cudaGetLastError();
}

cudaError_t launch_chol_step(const CholMat* d_mats, int nmat, int maxn, int c0, int* d_fail,
                             const double* d_dmax, cudaStream_t st) {
  potrf_diag_kernel<<<nmat, 256, 0, st>>>(d_mats, c0, d_fail, d_dmax);
  int rest = maxn - c0 - NB;
  if (rest > 0) {
    trsm_panel_kernel<<<dim3((rest + 127) / 128, nmat), 128, 0, st>>>(d_mats, c0);
    int T = (rest + 63) / 64;
    syrk_update_kernel<<<dim3(T * (T + 1) / 2, nmat), 256, 0, st>>>(d_mats, c0);
  }
  return cudaGetLastError();
}

cudaError_t launch_local_solve(const CholMat* d_mats, int nsets, const int* d_set_ptr,
                               const int* d_set_sub, const SubDev* d_sub, const int64_t* d_s_off,
                               const double* d_r, double* d_s, cudaStream_t st) {
  if (nsets == 0) return cudaSuccess;
  local_solve_kernel<<<nsets, 256, 0, st>>>(d_mats, d_set_ptr, d_set_sub, d_sub, d_s_off, d_r, d_s);
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
