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
#include "df32.cuh"

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

// ---- double-float variants (the inner Krylov operator) ----

__global__ void split_kernel(const double* __restrict__ x, float2* __restrict__ x2, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    x2[t] = df_split(x[t]);
}

// Per-block row products in double-float: yp[row0_j + r] = B_j[r, :] . x_j
// (the contribution of block j to y at its r-th point).  One warp handles four
// consecutive rows at once so that each lane keeps four independent loads in
// flight; rows are contiguous, so every load is coalesced.
__global__ void __launch_bounds__(256) rowdot_df_kernel(const SubDev* __restrict__ subs,
                                                        const int* __restrict__ rtiles,
                                                        const float2* __restrict__ B2,
                                                        const float2* __restrict__ x2,
                                                        float2* __restrict__ yp) {
  const int j = rtiles[2 * blockIdx.x], r0 = rtiles[2 * blockIdx.x + 1];
  const SubDev& S = subs[j];
  const int nr = min(HT_ROWS, S.N - r0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float2* xj = x2 + S.woff;
  for (int rb = warp * 4; rb < nr; rb += 32) {      // 8 warps x 4 rows = 32 rows per sweep
    float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
    const float2* row = B2 + S.boff + (int64_t)(r0 + rb) * S.P;
    for (int c = lane; c < S.p; c += 32) {
      const float2 xv = xj[c];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (rb + u < nr) df_mac(h[u], l[u], row[(int64_t)u * S.P + c], xv);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      df_warp_sum(h[u], l[u]);
      if (lane == 0 && rb + u < nr) yp[S.row0 + r0 + rb + u] = make_float2(h[u], l[u]);
    }
  }
}

// Partial z_j over one 256-row chunk of B_j in double-float: y at each row is
// first summed from the row products of every block holding that point; then
// 64 column lanes x 4 row groups accumulate with two independent chains each,
// and the row groups are added in shared memory.  Partials stored as float64.
__global__ void __launch_bounds__(256) matvec_HT_df_partial_kernel(ProbDev P, const SubDev* __restrict__ subs,
                                                                   const int* __restrict__ rtiles,
                                                                   const int* __restrict__ cov, int Gmax,
                                                                   const float2* __restrict__ B2,
                                                                   const float2* __restrict__ yp,
                                                                   double* __restrict__ part, int maxP) {
  const int j = rtiles[2 * blockIdx.x], r0 = rtiles[2 * blockIdx.x + 1];
  const SubDev& S = subs[j];
  const int nr = min(HT_ROWS, S.N - r0);
  __shared__ float2 yl[HT_ROWS];
  __shared__ float2 red[4][64];
  const int d = P.dim;
  for (int t = threadIdx.x; t < nr; t += blockDim.x) {
    const int r = r0 + t;
    int qa[3] = {r % S.n[0], 0, 0};
    int rest = r / S.n[0];
    if (d > 1) { qa[1] = rest % S.n[1]; rest /= S.n[1]; }
    if (d > 2) qa[2] = rest;
    int q[3] = {S.lo[0] + qa[0], S.lo[1] + qa[1], S.lo[2] + qa[2]};
    int k0[3] = {0, 0, 0}, kn[3] = {1, 1, 1};
    for (int i = 0; i < d; ++i) { k0[i] = cov[(i * Gmax + q[i]) * 2]; kn[i] = cov[(i * Gmax + q[i]) * 2 + 1]; }
    float yh = 0.f, yl2 = 0.f;
    for (int a2 = 0; a2 < kn[2]; ++a2)
      for (int a1 = 0; a1 < kn[1]; ++a1)
        for (int a0 = 0; a0 < kn[0]; ++a0) {
          const int k = (k0[0] + a0) + P.nsub[0] * ((k0[1] + a1) + P.nsub[1] * (k0[2] + a2));
          const SubDev& K = subs[k];
          int64_t rk = q[0] - K.lo[0];
          if (d > 1) rk += (int64_t)K.n[0] * (q[1] - K.lo[1]);
          if (d > 2) rk += (int64_t)K.n[0] * K.n[1] * (q[2] - K.lo[2]);
          const float2 v = yp[K.row0 + rk];
          df_add(yh, yl2, v.x, v.y);
        }
    yl[t] = make_float2(yh, yl2);
  }
  __syncthreads();
  const int cx = threadIdx.x & 63, rg = threadIdx.x >> 6;
  for (int c0 = 0; c0 < S.p; c0 += 64) {
    const int c = c0 + cx;
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
    if (c < S.p) {
      const float2* col = B2 + S.boff + (int64_t)r0 * S.P + c;
      int t = rg, cnt = 0;
      for (; t + 4 < nr; t += 8) {
        df_mac(h0, l0, col[(int64_t)t * S.P], yl[t]);
        df_mac(h1, l1, col[(int64_t)(t + 4) * S.P], yl[t + 4]);
        if ((++cnt & 7) == 0) { df_renorm(h0, l0); df_renorm(h1, l1); }
      }
      if (t < nr) df_mac(h0, l0, col[(int64_t)t * S.P], yl[t]);
      df_add(h0, l0, h1, l1);
    }
    red[rg][cx] = make_float2(h0, l0);
    __syncthreads();
    if (rg == 0 && c < S.p) {
      float h = red[0][cx].x, l = red[0][cx].y;
      for (int g = 1; g < 4; ++g) df_add(h, l, red[g][cx].x, red[g][cx].y);
      part[(int64_t)blockIdx.x * maxP + c] = df_to_double(h, l);
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_split(const double* d_x, float2* d_x2, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int64_t g = (n + 255) / 256;
  split_kernel<<<(unsigned)(g > 4096 ? 4096 : g), 256, 0, st>>>(d_x, d_x2, n);
  return cudaGetLastError();
}

cudaError_t launch_rowdot_df(const SubDev* d_sub, const int* d_rtiles, int nrtiles, const float2* d_B2,
                             const float2* d_x2, float2* d_yp, cudaStream_t st) {
  if (nrtiles == 0) return cudaSuccess;
  rowdot_df_kernel<<<nrtiles, 256, 0, st>>>(d_sub, d_rtiles, d_B2, d_x2, d_yp);
  return cudaGetLastError();
}

cudaError_t launch_matvec_HT_df(const ProbDev& P, const SubDev* d_sub, int J, const int* d_rtiles, int nrtiles,
                                const int* d_tile0, const int* d_cov, int Gmax, const float2* d_B2,
                                const float2* d_yp, double* d_part, double* d_z, int maxP, cudaStream_t st) {
  if (nrtiles == 0) return cudaSuccess;
  matvec_HT_df_partial_kernel<<<nrtiles, 256, 0, st>>>(P, d_sub, d_rtiles, d_cov, Gmax, d_B2, d_yp, d_part, maxP);
  matvec_HT_final_kernel<<<J, 256, 0, st>>>(d_sub, d_tile0, d_part, maxP, d_z);
  return cudaGetLastError();
}

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
