// The normal matrix H^T H (Eq. (system_new), Sec. 3) as block rows for the
// inner Krylov iterations: block k of z = H^T H x is
//   z_k = sum_{l : box_l meets box_k} G_kl x_l,   G_kl = B_k^T B_l over the shared points,
// the same Gram blocks the Schwarz local matrices A_i are assembled from.
// Each block row R_k = [G_kl]_l (p_k rows; neighbour l, in increasing l,
// spans P_l = p_l rounded up to even columns, zero-padded) is stored once in
// double-float, so one application reads sum_k p_k n_k entries instead of B
// twice and its rows (~3^d p entries) stream in full 16-byte loads.
#include "common.cuh"
#include "df32.cuh"

namespace {

// R2[roff_k + c * n2_k + col] from the pair buffer (k <= l stored p_k x p_l
// row-major); neighbour l occupies P_l columns (zero beyond p_l).
__global__ void gramrows_build_kernel(const GramRows g, const double* __restrict__ pairbuf, int k0) {
  const int k = k0 + blockIdx.y;
  const int p = g.p[k], n2 = g.n2[k];
  const int64_t tot = (int64_t)p * n2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / n2), col = (int)(e % n2);
    double v = 0.0;
    for (int q = g.nbr_ptr[k]; q < g.nbr_ptr[k + 1]; ++q) {
      const int c0 = g.nbr_col[q], pl = g.p[g.nbr_l[q]];
      if (col >= c0 && col < c0 + pl + (pl & 1)) {
        const int cc = col - c0;
        const int64_t off = g.nbr_off[q];
        if (cc < pl) v = g.nbr_tr[q] ? pairbuf[off + (int64_t)cc * p + c] : pairbuf[off + (int64_t)c * pl + cc];
        break;
      }
    }
    g.R2[g.roff[k] + e] = df_split(v);
  }
}

// z[woff_k + c] = R_k[c, :] . [x_l]_l for GRAM_TILE_ROWS rows of block k: the
// neighbours' entries of x are split into double-float pairs and staged in
// shared memory in one flat pass (a small table maps each 16-byte column pair
// to its neighbour), then one warp per row with 16-byte loads and two chains
// per lane.
__global__ void __launch_bounds__(256) gram_rowdot_kernel(const GramRows g, const int* __restrict__ rtile,
                                                          const double* __restrict__ x, const float2* __restrict__ x2,
                                                          double* __restrict__ z, float2* __restrict__ z2) {
  extern __shared__ float4 xs[];
  __shared__ int seg_c4[GRAM_MAX_NBR + 1], seg_p[GRAM_MAX_NBR];
  __shared__ int64_t seg_w[GRAM_MAX_NBR];
  const int k = rtile[2 * blockIdx.x], c0 = rtile[2 * blockIdx.x + 1];
  const int p = g.p[k], n4 = g.n2[k] >> 1;
  const int q0 = g.nbr_ptr[k], nq = g.nbr_ptr[k + 1] - q0;
  if (threadIdx.x < nq) {
    const int l = g.nbr_l[q0 + threadIdx.x];
    seg_c4[threadIdx.x] = g.nbr_col[q0 + threadIdx.x] >> 1;
    seg_p[threadIdx.x] = g.p[l];
    seg_w[threadIdx.x] = g.woff[l];
  }
  if (threadIdx.x == 0) seg_c4[nq] = n4;
  __syncthreads();
  for (int i = threadIdx.x; i < n4; i += blockDim.x) {
    int q = 0;
    while (q + 1 < nq && seg_c4[q + 1] <= i) ++q;
    const int e = 2 * (i - seg_c4[q]);
    float2 a, b;
    if (x2) {                                      // the producer's double-float split of x
      const float2* xl = x2 + seg_w[q];
      a = xl[e];
      b = (e + 1 < seg_p[q]) ? xl[e + 1] : make_float2(0.f, 0.f);
    } else {
      const double* xl = x + seg_w[q];
      a = df_split(xl[e]);
      b = (e + 1 < seg_p[q]) ? df_split(xl[e + 1]) : make_float2(0.f, 0.f);
    }
    xs[i] = make_float4(a.x, a.y, b.x, b.y);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = c0 + warp;
  if (c >= min(c0 + GRAM_TILE_ROWS, p)) return;
  const float4* row = reinterpret_cast<const float4*>(g.R2 + g.roff[k] + (int64_t)c * g.n2[k]);
  float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
  constexpr int U = 8;                         // independent 16-byte loads in flight per lane
  for (int i0 = lane; i0 < n4; i0 += 32 * U) {
    float4 a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = (i0 + 32 * u < n4) ? row[i0 + 32 * u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (i0 + 32 * u >= n4) break;
      const float4 xv = xs[i0 + 32 * u];
      df_mac_pair(h0, l0, h1, l1, a[u], xv);
    }
  }
  df_add(h0, l0, h1, l1);
  df_warp_sum(h0, l0);
  if (lane == 0) {
    const double v = df_to_double(h0, l0);
    z[g.woff[k] + c] = v;
    if (z2) z2[g.woff[k] + c] = df_split(v);
  }
}

// gram_rowdot_kernel for NR right-hand sides x_c = x + c ldx (c < NR): each row
// of R_k is read once for all of them; per right-hand side the same chains in
// the same order as the one-vector kernel, so every column is bit-identical
// to a one-vector product.
template <int NR>
__global__ void __launch_bounds__(256) gram_rowdot_multi_kernel(const GramRows g, const int* __restrict__ rtile,
                                                                const double* __restrict__ x, int64_t ldx,
                                                                double* __restrict__ z, int64_t ldz) {
  extern __shared__ float4 xsm[];                 // [NR][n4]
  __shared__ int seg_c4[GRAM_MAX_NBR + 1], seg_p[GRAM_MAX_NBR];
  __shared__ int64_t seg_w[GRAM_MAX_NBR];
  const int k = rtile[2 * blockIdx.x], c0 = rtile[2 * blockIdx.x + 1];
  const int p = g.p[k], n4 = g.n2[k] >> 1;
  const int q0 = g.nbr_ptr[k], nq = g.nbr_ptr[k + 1] - q0;
  if (threadIdx.x < nq) {
    const int l = g.nbr_l[q0 + threadIdx.x];
    seg_c4[threadIdx.x] = g.nbr_col[q0 + threadIdx.x] >> 1;
    seg_p[threadIdx.x] = g.p[l];
    seg_w[threadIdx.x] = g.woff[l];
  }
  if (threadIdx.x == 0) seg_c4[nq] = n4;
  __syncthreads();
  for (int i = threadIdx.x; i < n4; i += blockDim.x) {
    int q = 0;
    while (q + 1 < nq && seg_c4[q + 1] <= i) ++q;
    const int e = 2 * (i - seg_c4[q]);
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      const double* xl = x + c * ldx + seg_w[q];
      const float2 a = df_split(xl[e]);
      const float2 b = (e + 1 < seg_p[q]) ? df_split(xl[e + 1]) : make_float2(0.f, 0.f);
      xsm[c * n4 + i] = make_float4(a.x, a.y, b.x, b.y);
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rr = c0 + warp;
  if (rr >= min(c0 + GRAM_TILE_ROWS, p)) return;
  const float4* row = reinterpret_cast<const float4*>(g.R2 + g.roff[k] + (int64_t)rr * g.n2[k]);
  float h0[NR], l0[NR], h1[NR], l1[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) { h0[c] = 0.f; l0[c] = 0.f; h1[c] = 0.f; l1[c] = 0.f; }
  constexpr int U = 8;
  for (int i0 = lane; i0 < n4; i0 += 32 * U) {
    float4 a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = (i0 + 32 * u < n4) ? row[i0 + 32 * u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (i0 + 32 * u >= n4) break;
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        const float4 xv = xsm[c * n4 + i0 + 32 * u];
        df_mac_pair(h0[c], l0[c], h1[c], l1[c], a[u], xv);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NR; ++c) {
    df_add(h0[c], l0[c], h1[c], l1[c]);
    df_warp_sum(h0[c], l0[c]);
    if (lane == 0) z[c * ldz + g.woff[k] + rr] = df_to_double(h0[c], l0[c]);
  }
}

}  // namespace

cudaError_t launch_gramrows_build(const GramRows& g, const double* d_pairbuf, int J, int maxp, int maxn2,
                                  cudaStream_t st) {
  if (J == 0) return cudaSuccess;
  const int64_t per = (int64_t)maxp * maxn2;
  const int gx = (int)std::min<int64_t>((per + 255) / 256, 1024);
  for (int k0 = 0; k0 < J; k0 += 65535) {
    gramrows_build_kernel<<<dim3(gx, std::min(J - k0, 65535)), 256, 0, st>>>(g, d_pairbuf, k0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_gram_matvec(const GramRows& g, int J, const int* d_rtile, int nrtile, int maxn2,
                               const double* d_x, double* d_z, cudaStream_t st, const float2* d_x2, float2* d_z2) {
  if (J == 0) return cudaSuccess;
  const int smem = (int)(sizeof(float2) * (size_t)maxn2);
  static const cudaError_t lim = smem_limit_max(gram_rowdot_kernel);
  if (lim != cudaSuccess) return lim;
  gram_rowdot_kernel<<<nrtile, 32 * GRAM_TILE_ROWS, smem, st>>>(g, d_rtile, d_x, d_x2, d_z, d_z2);
  return cudaGetLastError();
}

template <int NR>
static cudaError_t gram_multi_launch(const GramRows& g, const int* d_rtile, int nrtile, int maxn2, const double* d_x,
                                     int64_t ldx, double* d_z, int64_t ldz, cudaStream_t st) {
  const int smem = (int)(sizeof(float2) * (size_t)maxn2 * NR);
  static const cudaError_t lim = smem_limit_max(gram_rowdot_multi_kernel<NR>);
  if (lim != cudaSuccess) return lim;
  gram_rowdot_multi_kernel<NR><<<nrtile, 32 * GRAM_TILE_ROWS, smem, st>>>(g, d_rtile, d_x, ldx, d_z, ldz);
  return cudaGetLastError();
}

cudaError_t launch_gram_matvec_multi(const GramRows& g, int J, const int* d_rtile, int nrtile, int maxn2,
                                     const double* d_x, int64_t ldx, double* d_z, int64_t ldz, int nr,
                                     cudaStream_t st) {
  if (J == 0) return cudaSuccess;
  for (int c0 = 0; c0 < nr; c0 += 4) {            // four right-hand sides per launch
    const int k = std::min(4, nr - c0);
    const double* x = d_x + c0 * ldx;
    double* z = d_z + c0 * ldz;
    cudaError_t e = k == 4 ? gram_multi_launch<4>(g, d_rtile, nrtile, maxn2, x, ldx, z, ldz, st)
                  : k == 3 ? gram_multi_launch<3>(g, d_rtile, nrtile, maxn2, x, ldx, z, ldz, st)
                  : k == 2 ? gram_multi_launch<2>(g, d_rtile, nrtile, maxn2, x, ldx, z, ldz, st)
                           : gram_multi_launch<1>(g, d_rtile, nrtile, maxn2, x, ldx, z, ldz, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
