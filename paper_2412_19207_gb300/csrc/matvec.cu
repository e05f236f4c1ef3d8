// Block-sparse products with H = [B_1, ..., B_J] (Sec. 2 Eq. (system), the
// normal equations H^T H W = H^T F; block-sparse structure, Remark in Sec. 3).
//
// B_j is N_j x P_j row-major (rows = the collocation points of box_j, dim 0
// fastest; P_j = p_j rounded up to even, padding columns zero).
//  * y = H x: y_g = sum over the subdomains j whose box holds point g of
//    B_j[row_j(g), :] . x_j -- one warp per point, lanes across the row.
//  * z = H^T y: z_j = B_j^T y(rows of j) -- one block per (subdomain, row
//    chunk), threads across columns; chunk partials summed in a fixed order.
#include "common.cuh"

namespace {

constexpr int HT_ROWS = 256;    // rows per H^T chunk

__global__ void matvec_H_kernel(ProbDev P, const SubDev* __restrict__ subs, const int* __restrict__ cov,
                                int Gmax, const double* __restrict__ B, const double* __restrict__ x,
                                double* __restrict__ y, int64_t N) {
  const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= N) return;
  const int d = P.dim;
  int q[3] = {0, 0, 0}, k0[3] = {0, 0, 0}, kn[3] = {1, 1, 1};
  int64_t rem = g;
  for (int i = 0; i < d; ++i) {
    q[i] = (int)(rem % P.G[i]);
    rem /= P.G[i];
    k0[i] = cov[(i * Gmax + q[i]) * 2];
    kn[i] = cov[(i * Gmax + q[i]) * 2 + 1];
  }
  double acc = 0.0;
  for (int a2 = 0; a2 < kn[2]; ++a2)
    for (int a1 = 0; a1 < kn[1]; ++a1)
      for (int a0 = 0; a0 < kn[0]; ++a0) {
        int kk[3] = {k0[0] + a0, k0[1] + a1, k0[2] + a2};
        int j = kk[0] + P.nsub[0] * (kk[1] + P.nsub[1] * kk[2]);
        const SubDev& S = subs[j];
        int64_t r = q[0] - S.lo[0];
        if (d > 1) r += (int64_t)S.n[0] * (q[1] - S.lo[1]);
        if (d > 2) r += (int64_t)S.n[0] * S.n[1] * (q[2] - S.lo[2]);
        const double* row = B + S.boff + r * S.P;
        const double* xj = x + S.woff;
        for (int c = lane; c < S.p; c += 32) acc = fma(row[c], xj[c], acc);
      }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) y[g] = acc;
}

__global__ void matvec_HT_partial_kernel(ProbDev P, const SubDev* __restrict__ subs,
                                         const int* __restrict__ rtiles, const double* __restrict__ B,
                                         const double* __restrict__ y, double* __restrict__ part,
                                         int maxP) {
  const int j = rtiles[2 * blockIdx.x], r0 = rtiles[2 * blockIdx.x + 1];
  const SubDev& S = subs[j];
  const int nr = min(HT_ROWS, S.N - r0);
  __shared__ double yl[HT_ROWS];
  const int d = P.dim;
  for (int t = threadIdx.x; t < nr; t += blockDim.x) {
    int r = r0 + t;
    int a0 = r % S.n[0], rest = r / S.n[0];
    int64_t g = S.lo[0] + a0;
    int64_t stride = P.G[0];
    if (d > 1) { g += stride * (S.lo[1] + rest % S.n[1]); rest /= S.n[1]; stride *= P.G[1]; }
    if (d > 2) g += stride * (S.lo[2] + rest);
    yl[t] = y[g];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < S.p; c += blockDim.x) {
    const double* col = B + S.boff + (int64_t)r0 * S.P + c;
    double acc = 0.0;
    for (int t = 0; t < nr; ++t) acc = fma(col[(int64_t)t * S.P], yl[t], acc);
    part[(int64_t)blockIdx.x * maxP + c] = acc;
  }
}

__global__ void matvec_HT_final_kernel(const SubDev* __restrict__ subs, const int* __restrict__ tile0,
                                       const double* __restrict__ part, int maxP, double* __restrict__ z) {
  const int j = blockIdx.x;
  const SubDev& S = subs[j];
  const int t0 = tile0[j], t1 = tile0[j + 1];
  for (int c = threadIdx.x; c < S.p; c += blockDim.x) {
    double acc = 0.0;
    for (int t = t0; t < t1; ++t) acc += part[(int64_t)t * maxP + c];
    z[S.woff + c] = acc;
  }
}

}  // namespace

cudaError_t launch_matvec_H2(const ProbDev& P, const SubDev* d_sub, const int* d_cov, int Gmax,
                             const double* d_B, const double* d_x, double* d_y, int64_t N,
                             cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  int64_t threads = N * 32;
  matvec_H_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(P, d_sub, d_cov, Gmax, d_B, d_x, d_y, N);
  return cudaGetLastError();
}

cudaError_t launch_matvec_HT2(const ProbDev& P, const SubDev* d_sub, int J, const int* d_rtiles,
                              int nrtiles, const int* d_tile0, const double* d_B, const double* d_y,
                              double* d_part, double* d_z, int maxP, cudaStream_t st) {
  if (nrtiles == 0) return cudaSuccess;
  matvec_HT_partial_kernel<<<nrtiles, 256, 0, st>>>(P, d_sub, d_rtiles, d_B, d_y, d_part, maxP);
  matvec_HT_final_kernel<<<J, 256, 0, st>>>(d_sub, d_tile0, d_part, maxP, d_z);
  return cudaGetLastError();
}
