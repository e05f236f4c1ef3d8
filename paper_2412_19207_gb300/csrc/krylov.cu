// Vector kernels for the Krylov solvers (PCG and GMRES on the normal
// equations, Sec. 3/5), float64.  Reductions are deterministic: each dot
// product is one block reduction with a fixed summation order.
#include "common.cuh"
#include "df32.cuh"

namespace {

constexpr int RT = 256;     // threads per reduction block

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v) {
  __shared__ double red[RT / 32];
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < RT / 32) ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
  }
  return s;   // valid in thread 0
}

// out[i] = V[i] . w, block i (vectors of Krylov length; fixed summation order)
__global__ void __launch_bounds__(RT) multidot_rows(const double* __restrict__ V, int64_t ldv,
                                                    const double* __restrict__ w, int64_t n,
                                                    double* __restrict__ out) {
  const double* v = V + blockIdx.x * ldv;
  double s0 = 0.0, s1 = 0.0;
  int64_t t = threadIdx.x;
  for (; t + RT < n; t += 2 * RT) { s0 = fma(v[t], w[t], s0); s1 = fma(v[t + RT], w[t + RT], s1); }
  if (t < n) s0 = fma(v[t], w[t], s0);
  const double s = block_sum(s0 + s1);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// w -= sum_i h[i] V[i]
__global__ void sub_combination(const double* __restrict__ V, int64_t ldv, int nv,
                                const double* __restrict__ h, double* __restrict__ w, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double s = w[t];
    for (int i = 0; i < nv; ++i) s = fma(-h[i], V[i * ldv + t], s);
    w[t] = s;
  }
}

// y = a * x + b * y
__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    y[t] = fma(a, x[t], b * y[t]);
}

// x += a p ; r -= a q
__global__ void cg_update_kernel(double a, const double* __restrict__ p, const double* __restrict__ q,
                                 double* __restrict__ x, double* __restrict__ r, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    x[t] = fma(a, p[t], x[t]);
    r[t] = fma(-a, q[t], r[t]);
  }
}

// y = a x (and its double-float split into y2 when given)
__global__ void scale_copy_kernel(double a, const double* __restrict__ x, double* __restrict__ y,
                                  float2* __restrict__ y2, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double v = a * x[t];
    y[t] = v;
    if (y2) y2[t] = df_split(v);
  }
}

// x += V^T y for GMRES: x[t] += sum_i y[i] V[i][t]
__global__ void add_combination(const double* __restrict__ V, int64_t ldv, int nv,
                                const double* __restrict__ y, double* __restrict__ x, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double s = x[t];
    for (int i = 0; i < nv; ++i) s = fma(y[i], V[i * ldv + t], s);
    x[t] = s;
  }
}

// One Arnoldi step's bookkeeping on the device (Saad & Schultz's GMRES with
// Givens rotations): column j of the Hessenberg matrix from the two
// Gram-Schmidt passes and ||w||, the earlier rotations applied, a new rotation
// zeroing h_{j+1,j}, the residual estimate |g_{j+1}| / ||M^{-1} b||, and the
// scale 1 / h_{j+1,j} that normalises the next basis vector.  The cycle stops
// (done = 1) at the tolerance or a lucky breakdown, done = 2 on a non-finite
// estimate; a step after done changes nothing.  The column and the rotations
// are staged in shared memory; one thread runs the rotation chain.
__global__ void __launch_bounds__(128) gmres_givens_kernel(GmresDev s, int j, int k, double mbnorm, double rtol) {
  __shared__ double hj[GMRES_MAX_RESTART + 2], cs[GMRES_MAX_RESTART], sn[GMRES_MAX_RESTART];
  __shared__ int skip;
  const int t = threadIdx.x;
  if (t == 0) skip = *s.done;
  // the column from the two passes and the earlier rotations, loaded in parallel
  for (int i = t; i <= j; i += blockDim.x) hj[i] = s.hv[i] + s.hv[(k + 2) + i];
  for (int i = t; i < j; i += blockDim.x) { cs[i] = s.cs[i]; sn[i] = s.sn[i]; }
  __syncthreads();
  if (skip) { if (t == 0) *s.inv = 0.0; return; }
  if (t == 0) {
    const double nrm = sqrt(*s.ww);
    hj[j + 1] = nrm;
    *s.inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int i = 0; i < j; ++i) {
      const double a = cs[i] * hj[i] + sn[i] * hj[i + 1];
      hj[i + 1] = -sn[i] * hj[i] + cs[i] * hj[i + 1];
      hj[i] = a;
    }
    const double den = hypot(hj[j], hj[j + 1]);
    double c = 1.0, sj = 0.0;
    if (den != 0.0) { c = hj[j] / den; sj = hj[j + 1] / den; }
    s.cs[j] = c;
    s.sn[j] = sj;
    hj[j] = c * hj[j] + sj * hj[j + 1];
    hj[j + 1] = 0.0;
    const double gj = s.g[j];
    s.g[j + 1] = -sj * gj;
    s.g[j] = c * gj;
    const double rel = fabs(s.g[j + 1]) / mbnorm;
    *s.rel = rel;
    *s.jdone = j + 1;
    if (!isfinite(rel)) *s.done = 2;
    else if (rel <= rtol || hj[j] == 0.0) *s.done = 1;
  }
  __syncthreads();
  for (int i = t; i <= j; i += blockDim.x) s.H[(int64_t)i * k + j] = hj[i];
}

// y *= *a (a device scalar), and the double-float split of the result into y2 when given
__global__ void scale_dev_kernel(double* __restrict__ y, const double* __restrict__ a, float2* __restrict__ y2,
                                 int64_t n) {
  const double f = *a;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double v = y[t] * f;
    y[t] = v;
    if (y2) y2[t] = df_split(v);
  }
}

// Preconditioned CG steps with the scalars on the device (Hestenes & Stiefel):
// x += alpha p, r -= alpha q with alpha = (r.z) / (p.q); a step after done
// (converged, breakdown) changes nothing.  done = 2 when p.q is not positive
// and finite.
__global__ void cg_update_dev_kernel(const double* __restrict__ p, const double* __restrict__ q,
                                     double* __restrict__ x, double* __restrict__ r, int64_t n, CgDev s, int ph) {
  if (*s.done) return;
  const double pq = *s.pq, rz = s.rz[ph];
  if (!(pq > 0.0) || !isfinite(pq)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *s.done = 2;
    return;
  }
  const double alpha = rz / pq;
  if (s.lz && blockIdx.x == 0 && threadIdx.x == 0) {
    const int kk = *s.it;
    if (kk < s.lzcap) s.lz[2 * kk] = alpha;
  }
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    x[t] = fma(alpha, p[t], x[t]);
    r[t] = fma(-alpha, q[t], r[t]);
  }
}

// After an update: count it and test ||r|| / ||b|| (one thread).
__global__ void cg_check_kernel(CgDev s, double bnorm, double rtol) {
  if (*s.done) return;
  const double rel = sqrt(*s.rr) / bnorm;
  *s.rel = rel;
  *s.it += 1;
  if (!isfinite(rel)) *s.done = 2;
  else if (rel <= rtol) *s.done = 1;
}

// p = z + (rz_new / rz_old) p
__global__ void cg_direction_kernel(const double* __restrict__ z, double* __restrict__ p, int64_t n, CgDev s, int ph) {
  if (*s.done) return;
  const double beta = s.rz[ph ^ 1] / s.rz[ph];
  if (s.lz && blockIdx.x == 0 && threadIdx.x == 0) {
    const int kk = *s.it - 1;                        // the update this direction follows
    if (kk >= 0 && kk < s.lzcap) s.lz[2 * kk + 1] = beta;
  }
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    p[t] = fma(beta, p[t], z[t]);
}

// ---- many right-hand sides in lockstep (vectors [nr][ld], one scalar set per column) ----
// out[c] = x_c . y_c: the same block reduction as multidot_rows, one block per column
__global__ void __launch_bounds__(RT) dot_multi_kernel(const double* __restrict__ x, int64_t ldx,
                                                       const double* __restrict__ y, int64_t ldy, int64_t n,
                                                       double* __restrict__ out) {
  const double* v = x + blockIdx.x * ldx;
  const double* w = y + blockIdx.x * ldy;
  double s0 = 0.0, s1 = 0.0;
  int64_t t = threadIdx.x;
  for (; t + RT < n; t += 2 * RT) { s0 = fma(v[t], w[t], s0); s1 = fma(v[t + RT], w[t + RT], s1); }
  if (t < n) s0 = fma(v[t], w[t], s0);
  const double s = block_sum(s0 + s1);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// cg_update_dev_kernel for column blockIdx.y
__global__ void cg_update_multi_kernel(const double* __restrict__ p, const double* __restrict__ q,
                                       double* __restrict__ x, double* __restrict__ r, int64_t n, int64_t ld,
                                       CgMulti s, int ph) {
  const int c = blockIdx.y;
  if (s.done[c]) return;
  const double pq = s.pq[c], rz = s.rz[ph * s.nr + c];
  if (!(pq > 0.0) || !isfinite(pq)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) s.done[c] = 2;
    return;
  }
  const double alpha = rz / pq;
  const int64_t o = c * ld;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    x[o + t] = fma(alpha, p[o + t], x[o + t]);
    r[o + t] = fma(-alpha, q[o + t], r[o + t]);
  }
}

// cg_check_kernel for every column (thread per column)
__global__ void cg_check_multi_kernel(CgMulti s, double rtol) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= s.nr || s.done[c]) return;
  const double rel = sqrt(s.rr[c]) / s.bnorm[c];
  s.rel[c] = rel;
  s.it[c] += 1;
  if (!isfinite(rel)) s.done[c] = 2;
  else if (rel <= rtol) s.done[c] = 1;
}

// cg_direction_kernel for column blockIdx.y
__global__ void cg_direction_multi_kernel(const double* __restrict__ z, double* __restrict__ p, int64_t n, int64_t ld,
                                          CgMulti s, int ph) {
  const int c = blockIdx.y;
  if (s.done[c]) return;
  const double beta = s.rz[(ph ^ 1) * s.nr + c] / s.rz[ph * s.nr + c];
  const int64_t o = c * ld;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    p[o + t] = fma(beta, p[o + t], z[o + t]);
}

// *out = 1 when every column is done (one warp)
__global__ void all_done_kernel(const int* __restrict__ done, int nr, int* __restrict__ out) {
  int all = 1;
  for (int c = threadIdx.x; c < nr; c += 32) all &= (done[c] != 0);
  all = __all_sync(0xffffffffu, all);
  if (threadIdx.x == 0) *out = all;
}

inline unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (unsigned)(g > 1216 ? 1216 : (g < 1 ? 1 : g));
}

}  // namespace

cudaError_t launch_multidot(const double* V, int64_t ldv, int nv, const double* w, int64_t n,
                            double* d_part, double* d_out, cudaStream_t st) {
  // one block per vector: out[i] = V[i] . w, one deterministic block reduction each
  multidot_rows<<<nv, RT, 0, st>>>(V, ldv, w, n, d_out);
  return cudaGetLastError();
}

cudaError_t launch_dot(const double* x, const double* y, int64_t n, double* d_part, double* d_out,
                       cudaStream_t st) {
  return launch_multidot(x, 0, 1, y, n, d_part, d_out, st);
}

cudaError_t launch_sub_combination(const double* V, int64_t ldv, int nv, const double* d_h, double* w,
                                   int64_t n, cudaStream_t st) {
  sub_combination<<<grid_for(n), 256, 0, st>>>(V, ldv, nv, d_h, w, n);
  return cudaGetLastError();
}

cudaError_t launch_add_combination(const double* V, int64_t ldv, int nv, const double* d_y, double* x,
                                   int64_t n, cudaStream_t st) {
  add_combination<<<grid_for(n), 256, 0, st>>>(V, ldv, nv, d_y, x, n);
  return cudaGetLastError();
}

cudaError_t launch_dot_multi(const double* x, int64_t ldx, const double* y, int64_t ldy, int64_t n, int nr,
                             double* d_out, cudaStream_t st) {
  if (nr <= 0) return cudaSuccess;
  dot_multi_kernel<<<nr, RT, 0, st>>>(x, ldx, y, ldy, n, d_out);
  return cudaGetLastError();
}

cudaError_t launch_cg_update_multi(const double* p, const double* q, double* x, double* r, int64_t n, int64_t ld,
                                   const CgMulti& s, int ph, cudaStream_t st) {
  cg_update_multi_kernel<<<dim3(grid_for(n), s.nr), 256, 0, st>>>(p, q, x, r, n, ld, s, ph);
  return cudaGetLastError();
}

cudaError_t launch_cg_check_multi(const CgMulti& s, double rtol, cudaStream_t st) {
  cg_check_multi_kernel<<<(s.nr + 127) / 128, 128, 0, st>>>(s, rtol);
  return cudaGetLastError();
}

cudaError_t launch_cg_direction_multi(const double* z, double* p, int64_t n, int64_t ld, const CgMulti& s, int ph,
                                      cudaStream_t st) {
  cg_direction_multi_kernel<<<dim3(grid_for(n), s.nr), 256, 0, st>>>(z, p, n, ld, s, ph);
  return cudaGetLastError();
}

cudaError_t launch_all_done(const int* d_done, int nr, double* d_out, cudaStream_t st) {
  all_done_kernel<<<1, 32, 0, st>>>(d_done, nr, reinterpret_cast<int*>(d_out));
  return cudaGetLastError();
}

cudaError_t launch_axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t st) {
  axpby_kernel<<<grid_for(n), 256, 0, st>>>(a, x, b, y, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_update(double a, const double* p, const double* q, double* x, double* r, int64_t n,
                             cudaStream_t st) {
  cg_update_kernel<<<grid_for(n), 256, 0, st>>>(a, p, q, x, r, n);
  return cudaGetLastError();
}

cudaError_t launch_scale_copy(double a, const double* x, double* y, int64_t n, cudaStream_t st, float2* y2) {
  scale_copy_kernel<<<grid_for(n), 256, 0, st>>>(a, x, y, y2, n);
  return cudaGetLastError();
}

cudaError_t launch_gmres_givens(const GmresDev& s, int j, int k, double mbnorm, double rtol, cudaStream_t st) {
  gmres_givens_kernel<<<1, 128, 0, st>>>(s, j, k, mbnorm, rtol);
  return cudaGetLastError();
}

cudaError_t launch_scale_dev(double* y, const double* a, int64_t n, cudaStream_t st, float2* y2) {
  scale_dev_kernel<<<grid_for(n), 256, 0, st>>>(y, a, y2, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_update_dev(const double* p, const double* q, double* x, double* r, int64_t n, const CgDev& s,
                                 int ph, cudaStream_t st) {
  cg_update_dev_kernel<<<grid_for(n), 256, 0, st>>>(p, q, x, r, n, s, ph);
  return cudaGetLastError();
}

cudaError_t launch_cg_check(const CgDev& s, double bnorm, double rtol, cudaStream_t st) {
  cg_check_kernel<<<1, 1, 0, st>>>(s, bnorm, rtol);
  return cudaGetLastError();
}

cudaError_t launch_cg_direction(const double* z, double* p, int64_t n, const CgDev& s, int ph, cudaStream_t st) {
  cg_direction_kernel<<<grid_for(n), 256, 0, st>>>(z, p, n, s, ph);
  return cudaGetLastError();
}
