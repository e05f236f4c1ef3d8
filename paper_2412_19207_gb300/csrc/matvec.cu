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

constexpr int HT_ROWS = 256;    // rows per H^T chunk (and the most rows of a double-float tile)

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
// (the contribution of block j to y at its r-th point).  x_j is staged in
// shared memory; a quarter warp (8 lanes) handles one row with 16-byte loads
// (two double-float entries; rows have even length P_j and start 16-byte
// aligned), four rows per warp, and sums its lanes with three shuffles.
__global__ void __launch_bounds__(256) rowdot_df_kernel(const SubDev* __restrict__ subs,
                                                        const int* __restrict__ rtiles, int tile_rows,
                                                        const float2* __restrict__ B2,
                                                        const float2* __restrict__ x2p,
                                                        float2* __restrict__ yp) {
  __shared__ float4 xs[RANN_MAX_M / 2];
  const int j = rtiles[2 * blockIdx.x], r0 = rtiles[2 * blockIdx.x + 1];
  const SubDev& S = subs[j];
  const int nr = min(tile_rows, S.N - r0);
  const int P2 = S.P >> 1;
  const float4* xj = reinterpret_cast<const float4*>(x2p + S.poff);
  for (int c = threadIdx.x; c < P2; c += blockDim.x) xs[c] = xj[c];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q = lane >> 3, sl = lane & 7;
  for (int rb = warp * 4; rb < nr; rb += 32) {      // 8 warps x 4 rows per sweep
    const int row = rb + q;
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
    if (row < nr) {
      const float4* rp = reinterpret_cast<const float4*>(B2 + S.boff + (int64_t)(r0 + row) * S.P);
#pragma unroll 4
      for (int c = sl; c < P2; c += 8) {
        const float4 b = rp[c];
        const float4 xv = xs[c];
        df_mac_pair(h0, l0, h1, l1, b, xv);
      }
      df_add(h0, l0, h1, l1);
    }
    for (int o = 4; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, h0, o);
      const float ol = __shfl_xor_sync(0xffffffffu, l0, o);
      df_add(h0, l0, oh, ol);
    }
    if (sl == 0 && row < nr) yp[S.row0 + r0 + row] = make_float2(h0, l0);
  }
}

// Partial z_j over one 256-row chunk of B_j in double-float: y at each row is
// first summed from the row products of every block holding that point; then
// each thread owns one column pair (16-byte loads) and a row group, with two
// independent chains, and the row groups are added in a fixed order in shared
// memory.  Partials stored as float64.
__global__ void __launch_bounds__(256) matvec_HT_df_partial_kernel(ProbDev P, const SubDev* __restrict__ subs,
                                                                   const int* __restrict__ rtiles, int tile_rows,
                                                                   const int* __restrict__ cov, int Gmax,
                                                                   const float2* __restrict__ B2,
                                                                   const float2* __restrict__ yp,
                                                                   double* __restrict__ part, int maxP) {
  const int j = rtiles[2 * blockIdx.x], r0 = rtiles[2 * blockIdx.x + 1];
  const SubDev& S = subs[j];
  const int nr = min(tile_rows, S.N - r0);
  __shared__ float2 yl[HT_ROWS];
  __shared__ float4 red[256];
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
  const int P2 = S.P >> 1;
  const int P2c = min(P2, 256);                  // column pairs per sweep
  const int G = 256 / P2c;                       // row groups
  const int cp = threadIdx.x % P2c, rg = threadIdx.x / P2c;
  for (int c0 = 0; c0 < P2; c0 += P2c) {
    const int c2 = c0 + cp;
    float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;   // columns 2 c2 (a) and 2 c2 + 1 (b), chain 0
    float e0 = 0.f, e1 = 0.f, f0 = 0.f, f1 = 0.f;   // chain 1
    if (rg < G && c2 < P2) {
      const float4* col = reinterpret_cast<const float4*>(B2 + S.boff + (int64_t)r0 * S.P) + c2;
      int t = rg, cnt = 0;
      for (; t + G < nr; t += 2 * G) {
        const float4 u = col[(int64_t)t * P2], w = col[(int64_t)(t + G) * P2];
        const float2 yu = yl[t], yw = yl[t + G];
        df_mac_pair(a0, a1, b0, b1, u, make_float4(yu.x, yu.y, yu.x, yu.y));
        df_mac_pair(e0, e1, f0, f1, w, make_float4(yw.x, yw.y, yw.x, yw.y));
        if ((++cnt & 7) == 0) { df_renorm(a0, a1); df_renorm(b0, b1); df_renorm(e0, e1); df_renorm(f0, f1); }
      }
      if (t < nr) {
        const float4 u = col[(int64_t)t * P2];
        df_mac_pair(a0, a1, b0, b1, u, make_float4(yl[t].x, yl[t].y, yl[t].x, yl[t].y));
      }
      df_add(a0, a1, e0, e1);
      df_add(b0, b1, f0, f1);
    }
    red[threadIdx.x] = make_float4(a0, a1, b0, b1);
    __syncthreads();
    if (rg == 0 && c2 < P2) {
      float ah = red[cp].x, al = red[cp].y, bh = red[cp].z, bl = red[cp].w;
      for (int g = 1; g < G; ++g) {
        const float4 v = red[g * P2c + cp];
        df_add(ah, al, v.x, v.y);
        df_add(bh, bl, v.z, v.w);
      }
      if (2 * c2 < S.p) part[(int64_t)blockIdx.x * maxP + 2 * c2] = df_to_double(ah, al);
      if (2 * c2 + 1 < S.p) part[(int64_t)blockIdx.x * maxP + 2 * c2 + 1] = df_to_double(bh, bl);
    }
    __syncthreads();
  }
}

// x2p[poff_j + c] = split(x[woff_j + c]) for c < p_j, zero up to P_j (each
// block's part 16-byte aligned for the row products).
__global__ void split_pad_kernel(const SubDev* __restrict__ subs, const double* __restrict__ x,
                                 float2* __restrict__ x2p) {
  const SubDev& S = subs[blockIdx.x];
  for (int c = threadIdx.x; c < S.P; c += blockDim.x)
    x2p[S.poff + c] = (c < S.p) ? df_split(x[S.woff + c]) : make_float2(0.f, 0.f);
}

}  // namespace

cudaError_t launch_split_pad(const SubDev* d_sub, int J, const double* d_x, float2* d_x2p, cudaStream_t st) {
  if (J == 0) return cudaSuccess;
  split_pad_kernel<<<J, 256, 0, st>>>(d_sub, d_x, d_x2p);
  return cudaGetLastError();
}

cudaError_t launch_split(const double* d_x, float2* d_x2, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int64_t g = (n + 255) / 256;
  split_kernel<<<(unsigned)(g > 4096 ? 4096 : g), 256, 0, st>>>(d_x, d_x2, n);
  return cudaGetLastError();
}

cudaError_t launch_rowdot_df(const SubDev* d_sub, const int* d_rtiles, int nrtiles, int tile_rows,
                             const float2* d_B2, const float2* d_x2p, float2* d_yp, cudaStream_t st) {
  if (nrtiles == 0) return cudaSuccess;
  rowdot_df_kernel<<<nrtiles, 256, 0, st>>>(d_sub, d_rtiles, tile_rows, d_B2, d_x2p, d_yp);
  return cudaGetLastError();
}

cudaError_t launch_matvec_HT_df(const ProbDev& P, const SubDev* d_sub, int J, const int* d_rtiles, int nrtiles,
                                int tile_rows, const int* d_tile0, const int* d_cov, int Gmax, const float2* d_B2,
                                const float2* d_yp, double* d_part, double* d_z, int maxP, cudaStream_t st) {
  if (nrtiles == 0) return cudaSuccess;
  matvec_HT_df_partial_kernel<<<nrtiles, 256, 0, st>>>(P, d_sub, d_rtiles, tile_rows, d_cov, Gmax, d_B2, d_yp,
                                                       d_part, maxP);
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
