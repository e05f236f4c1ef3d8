// Batched symmetric eigen-decomposition in float64 for the PCA (Sec. 4,
// Eq. (pca)): the right singular vectors and singular values of Psi_j are the
// eigenpairs of G_j = Psi_j^T Psi_j = V diag(sigma^2) V^T.  One thread block
// per matrix; only the p_j kept eigenvectors are formed.
//
//   1. Householder tridiagonalisation G = Q T Q^T (Golub & Van Loan 8.3.1),
//      reflectors kept in the rows of G; the symmetric rank-2 update is done
//      once per lower element and mirrored, so the matrix stays exactly
//      symmetric.
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
//   5. Back-transformation V = Q Z, one warp per vector.
// Output: w[m] descending; ranks[b] = p_j; G overwritten by V (row-major
// m x m, column c = eigenvector c for c < p_j, zero beyond); info[b] != 0 if
// QL did not converge in 100 sweeps for some eigenvalue.
#include "common.cuh"
#include "df32.cuh"

namespace {

constexpr int NT = 512;
constexpr int NW = NT / 32;

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += red[w];
    red[32] = s;
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

__global__ void __launch_bounds__(NT) syev_kernel(double* __restrict__ Aall, int m, int64_t stride,
                                                  double* __restrict__ wall, double* __restrict__ work_all,
                                                  int64_t work_stride, int* __restrict__ info,
                                                  int* __restrict__ ranks, int mode, double thr, int bisect) {
  extern __shared__ double sm[];
  double* v = sm;              // [m] reflector / QL diagonal copy
  double* w = v + m;           // [m] symmetric product / QL off-diagonal copy
  double* d = w + m;           // [m] tridiagonal diagonal (later: Gram-Schmidt coefficients)
  double* e = d + m;           // [m] tridiagonal off-diagonal
  double* beta = e + m;        // [m] reflector scalars
  double* ev = beta + m;       // [m] eigenvalues, descending
  double* ds = ev + m;         // [m] bisection: scaled diagonal
  double* e2s = ds + m;        // [m] bisection: scaled squared off-diagonal
  float* dh = reinterpret_cast<float*>(e2s + m);   // [m] x 4: double-float copies of ds, e2s
  float* dl = dh + m;
  float* eh = dl + m;
  float* el = eh + m;
  __shared__ double gbounds[3];
  __shared__ double red[33];
  __shared__ double tnorm;
  __shared__ int ql_fail, prank;
  double* A = Aall + blockIdx.x * stride;
  double* Z = work_all + blockIdx.x * work_stride;   // rows: eigenvectors
  double* LU = Z + (int64_t)m * m;                   // 5 m NT doubles, [i][thread]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // ---- 1. tridiagonalisation ----
  for (int k = 0; k + 2 < m; ++k) {
    const int n1 = m - k - 1;
    double loc = 0.0;
    for (int c = tid; c < n1; c += NT) {
      double x = A[(int64_t)k * m + k + 1 + c];   // row k == column k by symmetry
      v[c] = x;
      loc += x * x;
    }
    const double sig2 = block_sum(loc, red);
    const double sigma = sqrt(sig2);
    const double x0 = v[0];
    const double alpha = (x0 >= 0.0) ? -sigma : sigma;
    const double bt = (sigma > 0.0) ? 1.0 / (sig2 + fabs(x0) * sigma) : 0.0;   // 2 / (v^T v)
    __syncthreads();
    if (tid == 0) { v[0] = x0 - alpha; d[k] = A[(int64_t)k * m + k]; e[k] = alpha; beta[k] = bt; }
    __syncthreads();
    if (bt != 0.0) {
      double pv = 0.0;
      for (int r = tid; r < n1; r += NT) {   // p = bt A' v, A' read by columns (coalesced over r)
        double s = 0.0;
        const double* col = A + (int64_t)(k + 1) * m + k + 1 + r;
        for (int c = 0; c < n1; ++c) s = fma(col[(int64_t)c * m], v[c], s);
        s *= bt;
        w[r] = s;
        pv = fma(s, v[r], pv);
      }
      const double K = 0.5 * bt * block_sum(pv, red);
      for (int r = tid; r < n1; r += NT) w[r] = fma(-K, v[r], w[r]);
      __syncthreads();
      // A' -= v w^T + w v^T: each lower element once, mirrored to the upper one
      for (int rr = warp; rr < n1; rr += NW) {
        double* row = A + (int64_t)(k + 1 + rr) * m + k + 1;
        const double vr = v[rr], wr = w[rr];
        for (int cc = lane; cc <= rr; cc += 32) {
          double s = fma(-vr, w[cc], fma(-wr, v[cc], row[cc]));
          row[cc] = s;
          if (cc != rr) A[(int64_t)(k + 1 + cc) * m + k + 1 + rr] = s;
        }
      }
    }
    __syncthreads();
    for (int c = tid; c < n1; c += NT) A[(int64_t)k * m + k + 1 + c] = v[c];   // keep the reflector
    __syncthreads();
  }

  // ---- 2. eigenvalues of T ----
  if (tid == 0) {
    if (m >= 2) {
      d[m - 2] = A[(int64_t)(m - 2) * m + m - 2];
      e[m - 2] = A[(int64_t)(m - 1) * m + m - 2];
      beta[m - 2] = 0.0;
    }
    d[m - 1] = A[(int64_t)(m - 1) * m + m - 1];
    e[m - 1] = 0.0;
    beta[m - 1] = 0.0;
    double t = 0.0, gl = 0.0, gu = 0.0;
    for (int i = 0; i < m; ++i) {
      t = fmax(t, fabs(d[i]) + fabs(e[i]));
      v[i] = d[i];
      w[i] = e[i];
      const double rad = fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0);   // Gershgorin discs
      gl = (i == 0) ? d[i] - rad : fmin(gl, d[i] - rad);
      gu = (i == 0) ? d[i] + rad : fmax(gu, d[i] + rad);
    }
    tnorm = t;
    gbounds[0] = gl;
    gbounds[1] = gu;
    ql_fail = 0;
  }
  __syncthreads();
  if (bisect) {
    // scale T by 2^-sc (exact) so that its norm is at most 1
    const int sc = (tnorm > 0.0) ? ilogb(tnorm) + 1 : 0;
    for (int i = tid; i < m; i += NT) {
      const double di = ldexp(d[i], -sc), ei = ldexp(e[i], -sc);
      ds[i] = di;
      e2s[i] = ei * ei;
      const float2 a = df_split(di), b = df_split(ei * ei);
      dh[i] = a.x; dl[i] = a.y; eh[i] = b.x; el[i] = b.y;
    }
    __syncthreads();
    const double glo = ldexp(gbounds[0], -sc) - 0x1p-40, ghi = ldexp(gbounds[1], -sc) + 0x1p-40;
    for (int k = tid; k < m; k += NT) {          // k-th smallest eigenvalue
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
      ev[m - 1 - k] = ldexp(0.5 * (lo + hi), sc);
    }
  } else if (tid == 0) {
    // implicit QL without vectors (one thread)
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

  // ---- 3. QL path: sort descending (rank of each eigenvalue; ties by index) ----
  if (!bisect) {
    for (int t = tid; t < m; t += NT) {
      const double x = v[t];
      int rk = 0;
      for (int j = 0; j < m; ++j) rk += (v[j] > x) || (v[j] == x && j < t);
      ev[rk] = x;
    }
    __syncthreads();
  }
  // ---- rank rule (Sec. 4) ----
  if (tid == 0) {
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
    prank = max(p, 1);
  }
  __syncthreads();
  const int p = prank;

  // ---- 4. eigenvectors of T by inverse iteration ----
  const double tolp = 2.2e-16 * tnorm + 1e-300;
  double* u0 = LU;
  double* u1 = LU + (int64_t)m * NT;
  double* u2 = LU + 2 * (int64_t)m * NT;
  double* ml = LU + 3 * (int64_t)m * NT;
  double* xv = LU + 4 * (int64_t)m * NT;
  for (int k0 = 0; k0 < p; k0 += NT) {
    const int k = k0 + tid;
    if (k < p) {
      const double lam = ev[k];
      // LU of T - lam I with partial pivoting.  A row swap at step i is coded
      // in the multiplier as -(mult + 4) (|mult| <= 1 either way).
      double cd = d[0] - lam, cs = (m > 1) ? e[0] : 0.0;
      for (int i = 0; i + 1 < m; ++i) {
        const double sub = e[i];
        const double nd = d[i + 1] - lam, ns = (i + 2 < m) ? e[i + 1] : 0.0;
        double mult, a0, a1, a2;
        const bool swap = fabs(sub) > fabs(cd);
        if (!swap) {
          if (fabs(cd) < tolp) cd = (cd < 0.0) ? -tolp : tolp;
          mult = sub / cd;
          a0 = cd; a1 = cs; a2 = 0.0;
          cd = nd - mult * cs;
          cs = ns;
        } else {
          mult = cd / sub;
          a0 = sub; a1 = nd; a2 = ns;
          cd = cs - mult * nd;
          cs = -mult * ns;
        }
        u0[(int64_t)i * NT + tid] = a0;
        u1[(int64_t)i * NT + tid] = a1;
        u2[(int64_t)i * NT + tid] = a2;
        ml[(int64_t)i * NT + tid] = swap ? -(mult + 4.0) : mult;
      }
      if (fabs(cd) < tolp) cd = (cd < 0.0) ? -tolp : tolp;
      u0[(int64_t)(m - 1) * NT + tid] = cd;
      for (int i = 0; i < m; ++i) xv[(int64_t)i * NT + tid] = start_entry(i, k);
      for (int it = 0; it < 2; ++it) {
        for (int i = 0; i + 1 < m; ++i) {      // apply the row swaps and L^{-1}
          double mc = ml[(int64_t)i * NT + tid];
          double xi = xv[(int64_t)i * NT + tid], xn = xv[(int64_t)(i + 1) * NT + tid];
          if (mc <= -3.0) {
            mc = -mc - 4.0;
            const double tmp = xi; xi = xn; xn = tmp;
          }
          xv[(int64_t)i * NT + tid] = xi;
          xv[(int64_t)(i + 1) * NT + tid] = xn - mc * xi;
        }
        double x1 = 0.0, x2 = 0.0, amax = 0.0;
        for (int i = m - 1; i >= 0; --i) {      // U^{-1}
          double s = xv[(int64_t)i * NT + tid];
          if (i + 1 < m) s -= u1[(int64_t)i * NT + tid] * x1;
          if (i + 2 < m) s -= u2[(int64_t)i * NT + tid] * x2;
          const double xi = s / u0[(int64_t)i * NT + tid];
          xv[(int64_t)i * NT + tid] = xi;
          x2 = x1;
          x1 = xi;
          amax = fmax(amax, fabs(xi));
        }
        const double sc = (amax > 0.0 && amax < 1e300) ? 1.0 / amax : 1.0;
        for (int i = 0; i < m; ++i) xv[(int64_t)i * NT + tid] *= sc;
      }
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) { const double x = xv[(int64_t)i * NT + tid]; nrm = fma(x, x, nrm); }
      const double inv = (nrm > 0.0) ? 1.0 / sqrt(nrm) : 0.0;
      for (int i = 0; i < m; ++i) Z[(int64_t)k * m + i] = xv[(int64_t)i * NT + tid] * inv;
    }
  }
  __syncthreads();
  // ---- classical Gram-Schmidt, twice, in descending order ----
  for (int k = 1; k < p; ++k) {
    double* zk = Z + (int64_t)k * m;
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = tid; j < k; j += NT) {
        const double* zj = Z + (int64_t)j * m;
        double s = 0.0;
        for (int i = 0; i < m; ++i) s = fma(zj[i], zk[i], s);
        d[j] = s;
      }
      __syncthreads();
      for (int i = tid; i < m; i += NT) {
        double s = zk[i];
        for (int j = 0; j < k; ++j) s = fma(-d[j], Z[(int64_t)j * m + i], s);
        zk[i] = s;
      }
      __syncthreads();
    }
    double loc = 0.0;
    for (int i = tid; i < m; i += NT) loc = fma(zk[i], zk[i], loc);
    const double nn = block_sum(loc, red);
    const double inv = (nn > 0.0) ? 1.0 / sqrt(nn) : 0.0;
    for (int i = tid; i < m; i += NT) zk[i] *= inv;
    __syncthreads();
  }
  // ---- 5. back-transformation V = H_0 H_1 ... H_{m-3} Z, one warp per vector ----
  for (int c = warp; c < p; c += NW) {
    double* z = Z + (int64_t)c * m;
    for (int k = m - 3; k >= 0; --k) {
      const double bt = beta[k];
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
  __syncthreads();
  // ---- output ----
  for (int c = tid; c < m; c += NT) wall[(int64_t)blockIdx.x * m + c] = ev[c];
  for (int64_t e2 = tid; e2 < (int64_t)m * m; e2 += NT) {
    const int r = (int)(e2 / m), c = (int)(e2 % m);
    A[e2] = (c < p) ? Z[(int64_t)c * m + r] : 0.0;
  }
  if (tid == 0) {
    info[blockIdx.x] = ql_fail;
    ranks[blockIdx.x] = p;
  }
}

}  // namespace

int64_t syevd_work_doubles(int m) { return (int64_t)m * m + 5 * (int64_t)m * NT; }

cudaError_t launch_syevd(double* d_A, int m, int batch, double* d_w, double* d_work, int* d_info, int* d_ranks,
                         int mode, double thr, int bisect, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  const size_t smem = sizeof(double) * 10 * (size_t)m;
  cudaError_t e = cudaFuncSetAttribute(syev_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  syev_kernel<<<batch, NT, smem, st>>>(d_A, m, (int64_t)m * m, d_w, d_work, syevd_work_doubles(m), d_info,
                                       d_ranks, mode, thr, bisect);
  return cudaGetLastError();
}
