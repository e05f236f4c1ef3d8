// Batched symmetric eigen-decomposition in float64, one thread block per matrix.
//
// Sec. 4 (Eq. (pca)): the PCA of Psi_j needs its right singular vectors and
// singular values; they are the eigenpairs of the Gram matrix
// Psi_j^T Psi_j = V diag(sigma^2) V^T.  Steps (Golub & Van Loan, Ch. 8):
//   1. Householder tridiagonalisation A = Q T Q^T (reflectors kept in A);
//   2. Q accumulated backwards from the reflectors;
//   3. implicit QL iteration with Wilkinson shifts on T (the tql2 scheme of
//      Bowdler, Martin, Reinsch & Wilkinson, 1968), its plane rotations
//      applied to the eigenvector rows;
//   4. eigenpairs sorted by descending eigenvalue.
// Output: w[m] descending, and A overwritten by V (row-major, column c = the
// eigenvector of w[c]).  info[b] != 0 if QL did not converge in 60 sweeps for
// some eigenvalue.
#include "common.cuh"

namespace {

constexpr int NT = 256;

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

__global__ void __launch_bounds__(NT) syev_kernel(double* __restrict__ Aall, int m, int64_t stride,
                                                  double* __restrict__ wall,
                                                  double* __restrict__ Zall,
                                                  int* __restrict__ info) {
  extern __shared__ double sm[];
  double* v = sm;              // [m]
  double* w = v + m;           // [m]
  double* d = w + m;           // [m]
  double* e = d + m;           // [m]
  double* beta = e + m;        // [m]
  double* rc = beta + m;       // [m] rotation cos
  double* rs = rc + m;         // [m] rotation sin
  int* ri = (int*)(rs + m);    // [m] rotation index
  int* perm = ri + m;          // [m]
  __shared__ double red[33];
  __shared__ int nrot, ql_fail, done;
  __shared__ double tnorm;
  double* A = Aall + blockIdx.x * stride;
  double* Zt = Zall + blockIdx.x * stride;   // eigenvectors as rows
  const int tid = threadIdx.x;

  // ---- 1. tridiagonalisation ----
  for (int k = 0; k + 2 < m; ++k) {
    const int n1 = m - k - 1;
    double loc = 0.0;
    for (int c = tid; c < n1; c += NT) {
      double x = A[(int64_t)k * m + k + 1 + c];   // row k == column k by symmetry
      v[c] = x;
      loc += x * x;
    }
    double sig2 = block_sum(loc, red);
    double sigma = sqrt(sig2);
    double x0 = v[0];
    double alpha = (x0 >= 0.0) ? -sigma : sigma;
    double bt = 0.0;
    if (sigma > 0.0) bt = 1.0 / (sig2 + fabs(x0) * sigma);   // 2 / (v^T v)
    __syncthreads();
    if (tid == 0) { v[0] = x0 - alpha; d[k] = A[(int64_t)k * m + k]; e[k] = alpha; beta[k] = bt; }
    __syncthreads();
    if (bt != 0.0) {
      // p = bt * A' v  (A' = A[k+1:, k+1:], read by columns for coalescing)
      double pv = 0.0;
      for (int r = tid; r < n1; r += NT) {
        double s = 0.0;
        for (int c = 0; c < n1; ++c) s = fma(A[(int64_t)(k + 1 + c) * m + k + 1 + r], v[c], s);
        s *= bt;
        w[r] = s;
        pv += s * v[r];
      }
      double K = 0.5 * bt * block_sum(pv, red);
      for (int r = tid; r < n1; r += NT) w[r] = w[r] - K * v[r];
      __syncthreads();
      // A' -= v w^T + w v^T (evaluated symmetrically so that A stays exactly symmetric)
      for (int64_t e2 = tid; e2 < (int64_t)n1 * n1; e2 += NT) {
        int r = (int)(e2 / n1), c = (int)(e2 % n1);
        double s = __dadd_rn(__dmul_rn(v[r], w[c]), __dmul_rn(w[r], v[c]));
        int64_t idx = (int64_t)(k + 1 + r) * m + k + 1 + c;
        A[idx] = __dsub_rn(A[idx], s);
      }
    }
    __syncthreads();
    for (int c = tid; c < n1; c += NT) A[(int64_t)k * m + k + 1 + c] = v[c];   // keep the reflector
    __syncthreads();
  }
  if (tid == 0) {
    if (m >= 2) {
      d[m - 2] = A[(int64_t)(m - 2) * m + m - 2];
      e[m - 2] = A[(int64_t)(m - 1) * m + m - 2];
      beta[m - 2] = 0.0;
    }
    d[m - 1] = A[(int64_t)(m - 1) * m + m - 1];
    e[m - 1] = 0.0;
    beta[m - 1] = 0.0;
    ql_fail = 0;
    double t = 0.0;
    for (int i = 0; i < m; ++i) t = fmax(t, fabs(d[i]) + fabs(e[i]));
    tnorm = t;
  }
  __syncthreads();

  // ---- 2. Q = H_0 H_1 ... H_{m-3}, accumulated backwards into Zt (as Q, then transposed) ----
  for (int64_t e2 = tid; e2 < (int64_t)m * m; e2 += NT) Zt[e2] = ((e2 / m) == (e2 % m)) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = m - 3; k >= 0; --k) {
    const int n1 = m - k - 1;
    const double bt = beta[k];
    if (bt == 0.0) continue;
    for (int c = tid; c < n1; c += NT) v[c] = A[(int64_t)k * m + k + 1 + c];
    __syncthreads();
    for (int c = tid; c < n1; c += NT) {   // column k+1+c of Q
      double t = 0.0;
      for (int r = 0; r < n1; ++r) t = fma(v[r], Zt[(int64_t)(k + 1 + r) * m + k + 1 + c], t);
      t *= bt;
      for (int r = 0; r < n1; ++r) {
        int64_t idx = (int64_t)(k + 1 + r) * m + k + 1 + c;
        Zt[idx] = fma(-t, v[r], Zt[idx]);
      }
    }
    __syncthreads();
  }
  // transpose in place: Zt[c][r] = Q[r][c]
  for (int64_t e2 = tid; e2 < (int64_t)m * m; e2 += NT) {
    int r = (int)(e2 / m), c = (int)(e2 % m);
    if (r < c) {
      double a = Zt[(int64_t)r * m + c], b = Zt[(int64_t)c * m + r];
      Zt[(int64_t)r * m + c] = b;
      Zt[(int64_t)c * m + r] = a;
    }
  }
  __syncthreads();

  // ---- 3. implicit QL on (d, e); rotations of each sweep applied to rows of Zt ----
  for (int l = 0; l < m; ++l) {
    int iter = 0;
    while (true) {
      if (tid == 0) {
        int mm = l;
        for (; mm < m - 1; ++mm) {
          double dd = fabs(d[mm]) + fabs(d[mm + 1]);
          if (fabs(e[mm]) <= 2.2e-16 * dd || fabs(e[mm]) <= 2.2e-16 * tnorm) break;
        }
        nrot = 0;
        if (mm == l) {
          done = 1;
        } else if (iter >= 100) {
          done = 1;
          ql_fail = 1;
        } else {
          done = 0;
          double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
          double r = hypot(g, 1.0);
          g = d[mm] - d[l] + e[l] / (g + copysign(r, g));
          double s = 1.0, c = 1.0, p = 0.0;
          int i = mm - 1;
          bool early = false;
          for (; i >= l; --i) {
            double f = s * e[i], b = c * e[i];
            r = hypot(f, g);
            e[i + 1] = r;
            if (r == 0.0) { d[i + 1] -= p; e[mm] = 0.0; early = true; break; }
            s = f / r; c = g / r;
            g = d[i + 1] - p;
            r = (d[i] - g) * s + 2.0 * c * b;
            p = s * r;
            d[i + 1] = g + p;
            g = c * r - b;
            rc[nrot] = c; rs[nrot] = s; ri[nrot] = i; ++nrot;
          }
          if (!early) { d[l] -= p; e[l] = g; e[mm] = 0.0; }
        }
      }
      __syncthreads();
      const int dn = done, nr = nrot;
      __syncthreads();   // all threads hold done/nrot before thread 0 rewrites them
      if (dn) break;
      ++iter;
      for (int r = tid; r < m; r += NT) {
        for (int q = 0; q < nr; ++q) {
          int i = ri[q];
          double c = rc[q], s = rs[q];
          double a = Zt[(int64_t)i * m + r], b = Zt[(int64_t)(i + 1) * m + r];
          Zt[(int64_t)(i + 1) * m + r] = fma(s, a, c * b);
          Zt[(int64_t)i * m + r] = fma(c, a, -s * b);
        }
      }
      __syncthreads();
    }
  }

  // ---- 4. sort descending; V[r][c] = Zt[perm[c]][r] back into A ----
  if (tid == 0) {
    for (int c = 0; c < m; ++c) perm[c] = c;
    for (int c = 0; c < m; ++c) {
      int best = c;
      for (int q = c + 1; q < m; ++q) if (d[perm[q]] > d[perm[best]]) best = q;
      int t = perm[c]; perm[c] = perm[best]; perm[best] = t;
    }
    info[blockIdx.x] = ql_fail;
  }
  __syncthreads();
  for (int c = tid; c < m; c += NT) wall[(int64_t)blockIdx.x * m + c] = d[perm[c]];
  for (int64_t e2 = tid; e2 < (int64_t)m * m; e2 += NT) {
    int r = (int)(e2 / m), c = (int)(e2 % m);
    A[e2] = Zt[(int64_t)perm[c] * m + r];
  }
}

}  // namespace

cudaError_t launch_syevd(double* d_A, int m, int /*lda_stride*/, int batch, double* d_w,
                         double* d_work, int* d_info, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  size_t smem = sizeof(double) * 8 * (size_t)m + sizeof(int) * 2 * (size_t)m;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(syev_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  syev_kernel<<<batch, NT, smem, st>>>(d_A, m, (int64_t)m * m, d_w, d_work, d_info);
  return cudaGetLastError();
}
