// Batched float64 dense products over uneven task lists.
//
//  * gemm_tn: C = A^T B with the contraction over rows (K); A and B may be
//    read through row-index lists.  Used for the PCA Gram matrices
//    Psi_j^T Psi_j (Sec. 4) and for the neighbour Gram blocks
//    B_k^T B_l over the rows two boxes share (the blocks of A_i, Sec. 3).
//  * gemm_nn: C = A B, used for the projection B_j = H_j V_{p_j}
//    (Eq. (system_new)).
// Each task is one 64 x 64 output tile; 256 threads, 4 x 4 outputs each.
#include <algorithm>

#include "common.cuh"
#include "df32.cuh"

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256) gemm_tn_kernel(const GemmTask* __restrict__ tasks) {
  const GemmTask t = tasks[blockIdx.x];
  __shared__ double sA[TK][TM + 1];
  __shared__ double sB[TK][TN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < t.K; k0 += TK) {
    for (int e = threadIdx.x; e < TK * TM; e += 256) {
      int kk = e / TM, c = e % TM;
      int k = k0 + kk, col = t.tm + c;
      double v = 0.0;
      if (k < t.K && col < t.M) {
        int row = t.ia ? t.ia[k] : k;
        v = t.A[(int64_t)row * t.lda + col];
      }
      sA[kk][c] = v;
    }
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      int kk = e / TN, c = e % TN;
      int k = k0 + kk, col = t.tn + c;
      double v = 0.0;
      if (k < t.K && col < t.N) {
        int row = t.ib ? t.ib[k] : k;
        v = t.B[(int64_t)row * t.ldb + col];
      }
      sB[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = sA[kk][ty + 16 * q]; b[q] = sB[kk][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int r = t.tm + ty + 16 * p, c = t.tn + tx + 16 * q;
      if (r < t.M && c < t.N) t.C[(int64_t)r * t.ldc + c] = acc[p][q];
    }
}

__global__ void __launch_bounds__(256) gemm_nn_kernel(const GemmTask* __restrict__ tasks) {
  const GemmTask t = tasks[blockIdx.x];
  __shared__ double sA[TK][TM + 1];   // A^T tile: [k][row]
  __shared__ double sB[TK][TN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < t.K; k0 += TK) {
    for (int e = threadIdx.x; e < TK * TM; e += 256) {
      int r = e / TK, kk = e % TK;
      int row = t.tm + r, k = k0 + kk;
      sA[kk][r] = (row < t.M && k < t.K) ? t.A[(int64_t)row * t.lda + k] : 0.0;
    }
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      int kk = e / TN, c = e % TN;
      int k = k0 + kk, col = t.tn + c;
      sB[kk][c] = (k < t.K && col < t.N) ? t.B[(int64_t)k * t.ldb + col] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = sA[kk][ty + 16 * q]; b[q] = sB[kk][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int r = t.tm + ty + 16 * p, c = t.tn + tx + 16 * q;
      if (r < t.M && c < t.N) t.C[(int64_t)r * t.ldc + c] = acc[p][q];
    }
}

// C = A^T B in double-float with A, B given as double-float pairs (the task's
// A/B pointers address float2 arrays laid out like the float64 ones).  Used
// for the neighbour Gram blocks of the Schwarz local matrices, whose accuracy
// only affects the preconditioner.
__global__ void __launch_bounds__(256) gemm_tn_df_kernel(const GemmTask* __restrict__ tasks) {
  const GemmTask t = tasks[blockIdx.x];
  const float2* A2 = reinterpret_cast<const float2*>(t.A);
  const float2* B2 = reinterpret_cast<const float2*>(t.B);
  __shared__ float2 sA[TK][TM + 1];
  __shared__ float2 sB[TK][TN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float ah[4][4], al[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { ah[a][b] = 0.f; al[a][b] = 0.f; }
  for (int k0 = 0; k0 < t.K; k0 += TK) {
    for (int e = threadIdx.x; e < TK * TM; e += 256) {
      int kk = e / TM, c = e % TM;
      int k = k0 + kk, col = t.tm + c;
      float2 v = make_float2(0.f, 0.f);
      if (k < t.K && col < t.M) v = A2[(int64_t)(t.ia ? t.ia[k] : k) * t.lda + col];
      sA[kk][c] = v;
    }
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      int kk = e / TN, c = e % TN;
      int k = k0 + kk, col = t.tn + c;
      float2 v = make_float2(0.f, 0.f);
      if (k < t.K && col < t.N) v = B2[(int64_t)(t.ib ? t.ib[k] : k) * t.ldb + col];
      sB[kk][c] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      float2 a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = sA[kk][ty + 16 * q]; b[q] = sB[kk][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) df_mac(ah[p][q], al[p][q], a[p], b[q]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) df_renorm(ah[p][q], al[p][q]);
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int r = t.tm + ty + 16 * p, c = t.tn + tx + 16 * q;
      if (r < t.M && c < t.N) t.C[(int64_t)r * t.ldc + c] = df_to_double(ah[p][q], al[p][q]);
    }
}

// Copy the upper triangle of each square matrix into its lower triangle.
__global__ void symmetrize_kernel(double* const* __restrict__ mats, const int* __restrict__ ns,
                                  const int* __restrict__ lds) {
  double* A = mats[blockIdx.y];
  int n = ns[blockIdx.y], ld = lds[blockIdx.y];
  int64_t tot = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(e / n), c = (int)(e % n);
    if (r > c) A[(int64_t)r * ld + c] = A[(int64_t)c * ld + r];
  }
}

}  // namespace

cudaError_t launch_gemm_tn(const GemmTask* d_tasks, int ntasks, cudaStream_t st) {
  if (ntasks == 0) return cudaSuccess;
  gemm_tn_kernel<<<ntasks, 256, 0, st>>>(d_tasks);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tn_df(const GemmTask* d_tasks, int ntasks, cudaStream_t st) {
  if (ntasks == 0) return cudaSuccess;
  gemm_tn_df_kernel<<<ntasks, 256, 0, st>>>(d_tasks);
  return cudaGetLastError();
}

cudaError_t launch_gemm_nn(const GemmTask* d_tasks, int ntasks, cudaStream_t st) {
  if (ntasks == 0) return cudaSuccess;
  gemm_nn_kernel<<<ntasks, 256, 0, st>>>(d_tasks);
  return cudaGetLastError();
}

cudaError_t launch_symmetrize(double* const* d_mats, const int* d_n, const int* d_ld, int nmat,
                              int maxn, cudaStream_t st) {
  if (nmat == 0) return cudaSuccess;
  int64_t tot = (int64_t)maxn * maxn;
  int gx = (int)std::min<int64_t>((tot + 255) / 256, 1024);
  symmetrize_kernel<<<dim3(gx, nmat), 256, 0, st>>>(d_mats, d_n, d_ld);
  return cudaGetLastError();
}
