// Collocation assembly, right-hand side and evaluation kernels (float64).
//
// Sec. 2 Eq. (netdd)/(system): (H_j)_{ik} = A[L omega_j phi_j^k](x_i) and
// Sec. 4: (Psi_j)_{ik} = omega_j phi_j^k(x_i), with phi_j^k = tanh(s_k . (x - mu_j) + b_k),
// s_k = R_k / sigma (inputs normalised to [-1,1]^d per subdomain, Sec. 5).
//
// The subdomain grid is a tensor product and the windows of Sec. 5 are
// products of 1D factors, so sum_k omega_hat_k = prod_i (sum_{k_i} w_{k_i}(x_i))
// and omega_j = prod_i nu_i with the 1D normalised window nu_i = w_{j_i}/S_i.
// With g = L omega_j = prod_i e_i (e_i = l_i nu_i, l_i the 1D factor of L) the
// operator applied to g * phi is, for A v = -alpha Lap_S v + beta . grad v + c0 v,
//   A[g phi] = phi P0 + phi' (sum_i P_i s_i + Q phi |s_S|^2),
//   P0 = -alpha Lap_S g + beta . grad g + c0 g,  P_i = -2 alpha [i in S] d_i g + g beta_i,
//   Q = 2 alpha g,  phi' = 1 - phi^2,
// using grad phi = phi' s and Lap_S phi = -2 phi phi' |s_S|^2.  The per-point
// terms are computed once per row tile; each (row, neuron) entry then costs d
// FMAs, one tanh and a handful of FMAs.
#include "common.cuh"

namespace {

constexpr int TR = 32;          // rows per assembly tile
constexpr int NT = 256;         // threads per assembly block

struct D3 { double v, d1, d2; };

// 1D window factor w(x) = [1 + cos(pi u)]^2, u = (x - mu)/sig, zero for |u| >= 1.
__device__ __forceinline__ D3 wfun(double x, double mu, double sig) {
  double u = (x - mu) / sig;
  if (!(fabs(u) < 1.0)) return {0.0, 0.0, 0.0};
  double s, c;
  sincospi(u, &s, &c);
  double h = 1.0 + c;
  double k = RANN_PI / sig;
  double hp = -k * s;
  double hpp = -k * k * c;
  return {h * h, 2.0 * h * hp, 2.0 * (hp * hp + h * hpp)};
}

// Covering subdomain range along a dim for an arbitrary coordinate x.
__device__ __forceinline__ void cover_range(const ProbDev& P, int i, double x, int* k0, int* k1) {
  int l = P.nsub[i];
  double s = P.sig[i];
  int lo, hi;
  if (P.layout == RANN_LAYOUT_PAPER) {
    double dm = 1.0 / (double)(l - 1);
    lo = (int)floor((x - s) / dm) - 1;
    hi = (int)ceil((x + s) / dm) + 1;
  } else {
    lo = (int)floor((x - s) * l - 0.5) - 1;
    hi = (int)ceil((x + s) * l - 0.5) + 1;
  }
  *k0 = max(lo, 0);
  *k1 = min(hi, l - 1);
}

__device__ __forceinline__ double mu_of(const ProbDev& P, int i, int k) {
  int l = P.nsub[i];
  return P.layout == RANN_LAYOUT_PAPER ? (double)k / (double)(l - 1) : ((double)k + 0.5) / (double)l;
}

// 1D normalised window nu = w_own / S and its derivatives, where S sums the
// windows of all subdomains along this dim that cover x.
__device__ __forceinline__ D3 nu_fun(const ProbDev& P, int i, double x, int kown) {
  int k0, k1;
  cover_range(P, i, x, &k0, &k1);
  double S = 0, S1 = 0, S2 = 0;
  D3 w = {0, 0, 0};
  for (int k = k0; k <= k1; ++k) {
    D3 t = wfun(x, mu_of(P, i, k), P.sig[i]);
    S += t.v; S1 += t.d1; S2 += t.d2;
    if (k == kown) w = t;
  }
  if (!(S > 0.0)) return {0.0, 0.0, 0.0};
  double nu = w.v / S;
  double nu1 = (w.d1 - nu * S1) / S;
  double nu2 = (w.d2 - 2.0 * nu1 * S1 - nu * S2) / S;
  return {nu, nu1, nu2};
}

// 1D factor of the constraint L along dim i.
__device__ __forceinline__ D3 lfun(const ProbDev& P, int i, double x) {
  double r = 1.0 / P.rho;
  if (P.op == RANN_OP_HEAT && i == P.dim - 1) {
    double t = tanh(x * r);
    double t1 = (1.0 - t * t) * r;
    return {t, t1, -2.0 * t * t1 * r};
  }
  double a = tanh(x * r), b = tanh((1.0 - x) * r);
  double a1 = (1.0 - a * a) * r, b1 = -(1.0 - b * b) * r;
  double a2 = -2.0 * a * a1 * r, b2 = 2.0 * b * b1 * r;
  return {a * b, a1 * b + a * b1, a2 * b + 2.0 * a1 * b1 + a * b2};
}

// Smooth cell indicator S(x; c) of the piecewise coefficient and its derivative.
__device__ __forceinline__ void sbox(double x, int c, int g, double* v, double* d) {
  double w = 1.0 / (8.0 * g);
  double tl = 1.0, dl = 0.0, tr = -1.0, dr = 0.0;
  if (c > 0) { tl = tanh((x - (double)c / g) / w); dl = (1.0 - tl * tl) / w; }
  if (c < g - 1) { tr = tanh((x - (double)(c + 1) / g) / w); dr = (1.0 - tr * tr) / w; }
  *v = 0.5 * (tl - tr);
  *d = 0.5 * (dl - dr);
}

// Diffusion coefficient a and its spatial gradient.
__device__ __forceinline__ void coef_fun(const ProbDev& P, const double* x, double* a, double* ga) {
  ga[0] = ga[1] = ga[2] = 0.0;
  if (P.coef == RANN_COEF_CONST) { *a = P.coef_value; return; }
  if (P.coef == RANN_COEF_MULTISCALE) {
    double k = 2.0 / P.eps;   // sin(2 pi x / eps) = sinpi(k x)
    double sx, cx, sy, cy;
    sincospi(k * x[0], &sx, &cx);
    sincospi(k * x[1], &sy, &cy);
    *a = 2.0 + sx * sy;
    ga[0] = RANN_PI * k * cx * sy;
    ga[1] = RANN_PI * k * sx * cy;
    return;
  }
  // the cell factors stay in registers: loops over the largest grid (8),
  // fully unrolled, with the cells beyond g skipped
  const int g = P.coef_grid;
  double vx[8], dx[8], vy[8], dy[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    vx[c] = dx[c] = vy[c] = dy[c] = 0.0;
    if (c < g) { sbox(x[0], c, g, &vx[c], &dx[c]); sbox(x[1], c, g, &vy[c], &dy[c]); }
  }
  double s = 0, sx = 0, sy = 0;
#pragma unroll
  for (int cy = 0; cy < 8; ++cy) {
    if (cy >= g) break;
    double rv = 0, rd = 0;                    // sum_cx v vx, sum_cx v dx along row cy
#pragma unroll
    for (int cx = 0; cx < 8; ++cx) {
      if (cx >= g) break;
      const double v = P.coef_vals[cy * g + cx];
      rv += v * vx[cx];
      rd += v * dx[cx];
    }
    s += rv * vy[cy];
    sx += rd * vy[cy];
    sy += rv * dy[cy];
  }
  *a = s; ga[0] = sx; ga[1] = sy;
}

// Operator coefficients: A v = -alpha Lap_S v + beta . grad v + c0 v.
__device__ __forceinline__ void op_coefs(const ProbDev& P, const double* x, double* alpha,
                                         double* beta, double* c0) {
  beta[0] = beta[1] = beta[2] = 0.0;
  *c0 = 0.0;
  if (P.op == RANN_OP_POISSON) { *alpha = 1.0; *c0 = P.c0; }
  else if (P.op == RANN_OP_DIFFUSION) {
    double a, ga[3];
    coef_fun(P, x, &a, ga);
    *alpha = a;
    for (int i = 0; i < P.ns; ++i) beta[i] = -ga[i];
  } else {
    *alpha = P.nu;
    beta[P.dim - 1] = 1.0;
  }
}

// Per-point terms of block j at point x: omega_j, P0, P_i, Q.
__device__ void point_terms(const ProbDev& P, const int* kj, const double* x, double* out) {
  int d = P.dim;
  D3 e[RANN_MAX_DIM];
  double om = 1.0;
  for (int i = 0; i < d; ++i) {
    D3 nu = nu_fun(P, i, x[i], kj[i]);
    D3 l = lfun(P, i, x[i]);
    om *= nu.v;
    e[i] = {l.v * nu.v, l.d1 * nu.v + l.v * nu.d1, l.d2 * nu.v + 2.0 * l.d1 * nu.d1 + l.v * nu.d2};
  }
  double g = 1.0, dg[RANN_MAX_DIM], d2g[RANN_MAX_DIM];
  for (int i = 0; i < d; ++i) g *= e[i].v;
  for (int i = 0; i < d; ++i) {
    double rest = 1.0;
    for (int l = 0; l < d; ++l) if (l != i) rest *= e[l].v;
    dg[i] = e[i].d1 * rest;
    d2g[i] = e[i].d2 * rest;
  }
  double alpha, beta[3], c0;
  op_coefs(P, x, &alpha, beta, &c0);
  double lapS = 0.0, bdg = 0.0;
  for (int i = 0; i < P.ns; ++i) lapS += d2g[i];
  for (int i = 0; i < d; ++i) bdg += beta[i] * dg[i];
  out[0] = om;
  out[1] = -alpha * lapS + bdg + c0 * g;
  for (int i = 0; i < d; ++i) out[2 + i] = (i < P.ns ? -2.0 * alpha * dg[i] : 0.0) + g * beta[i];
  out[2 + d] = 2.0 * alpha * g;
}

__global__ void __launch_bounds__(NT) assemble_kernel(ProbDev P, const SubDev* __restrict__ subs,
                                                      const int* __restrict__ tiles,
                                                      const double* __restrict__ R,
                                                      const double* __restrict__ bias,
                                                      double* __restrict__ Psi,
                                                      double* __restrict__ H) {
  extern __shared__ double sm[];
  const int d = P.dim, m = P.m;
  const int j = tiles[2 * blockIdx.x], r0 = tiles[2 * blockIdx.x + 1];
  const SubDev& S = subs[j];
  const int nrow = min(TR, S.N - r0);
  const int PT = 3 + d;                      // omega, P0, P_0..P_{d-1}, Q
  double* spt = sm;                          // [TR][PT]
  double* sxh = spt + TR * PT;               // [TR][d]  x - mu
  double* sneu = sxh + TR * d;               // [m][d + 2]: s_i, |s_S|^2, b
  for (int t = threadIdx.x; t < nrow; t += blockDim.x) {
    int r = r0 + t;
    int a0 = r % S.n[0];
    int rest = r / S.n[0];
    int qa[3] = {a0, 0, 0};
    if (d > 1) { qa[1] = rest % S.n[1]; rest /= S.n[1]; }
    if (d > 2) qa[2] = rest;
    double x[3];
    for (int i = 0; i < d; ++i) x[i] = ((double)(S.lo[i] + qa[i]) + 0.5) / (double)P.G[i];
    point_terms(P, S.k, x, spt + t * PT);
    for (int i = 0; i < d; ++i) sxh[t * d + i] = x[i] - S.mu[i];
  }
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    double n2 = 0.0;
    for (int i = 0; i < d; ++i) {
      double s = R[((int64_t)j * m + k) * d + i] / P.sig[i];
      sneu[k * (d + 2) + i] = s;
      if (i < P.ns) n2 += s * s;
    }
    sneu[k * (d + 2) + d] = n2;
    sneu[k * (d + 2) + d + 1] = bias[(int64_t)j * m + k];
  }
  __syncthreads();
  const int64_t base = (S.row0 + r0) * (int64_t)m;
  const int total = nrow * m;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int r = idx / m, k = idx - r * m;
    const double* pt = spt + r * PT;
    const double* sn = sneu + k * (d + 2);
    const double* xh = sxh + r * d;
    double z = sn[d + 1];
    double ps = 0.0;
    for (int i = 0; i < d; ++i) { z = fma(sn[i], xh[i], z); ps = fma(pt[2 + i], sn[i], ps); }
    double ph = tanh(z);
    double php = 1.0 - ph * ph;
    double h = fma(ph, pt[1], php * fma(pt[2 + d] * ph, sn[d], ps));
    Psi[base + idx] = pt[0] * ph;
    H[base + idx] = h;
  }
}

__global__ void rhs_kernel(ProbDev P, double* __restrict__ F, int64_t N) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= N) return;
  const int d = P.dim;
  double x[3];
  int64_t rem = g;
  for (int i = 0; i < d; ++i) { x[i] = ((double)(rem % P.G[i]) + 0.5) / (double)P.G[i]; rem /= P.G[i]; }
  double f = P.f0;
  for (int t = 0; t < P.f_terms; ++t) {
    double term = P.fc[t];
    for (int i = 0; i < P.ns; ++i) term *= sinpi(P.fa[t * d + i] * x[i]);
    f += term;
  }
  double AG = 0.0;
  if (P.g_kind == RANN_G_SINPROD) {
    // A G for G = prod_i sin(pi x_i): Lap_S G = -ns pi^2 G, d_i G = pi cos(pi x_i) prod_{l != i} sin(pi x_l)
    double alpha, beta[3], c0;
    op_coefs(P, x, &alpha, beta, &c0);
    double s[3] = {1.0, 1.0, 1.0}, c[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (i < P.ns) sincospi(x[i], &s[i], &c[i]);
    const double G = s[0] * s[1] * s[2];
    const double lap = -(double)P.ns * RANN_PI * RANN_PI * G;
    const double bg = RANN_PI * (beta[0] * c[0] * s[1] * s[2] + beta[1] * s[0] * c[1] * s[2] +
                                 beta[2] * s[0] * s[1] * c[2]);
    AG = -alpha * lap + bg + c0 * G;
  }
  F[g] = f - AG;
}

__global__ void points_kernel(ProbDev P, double* __restrict__ xyz, int64_t N) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= N) return;
  int64_t rem = g;
  for (int i = 0; i < P.dim; ++i) {
    xyz[g * P.dim + i] = ((double)(rem % P.G[i]) + 0.5) / (double)P.G[i];
    rem /= P.G[i];
  }
}

// u_hat(x) = L(x) sum_j omega_j(x) sum_k phi_jk(x) U_jk + G(x), U_j = V_{p_j} W_j.
__global__ void eval_kernel(ProbDev P, const SubDev* __restrict__ subs, const double* __restrict__ R,
                            const double* __restrict__ bias, const double* __restrict__ U,
                            const double* __restrict__ X, int64_t n, double* __restrict__ out) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int d = P.dim, m = P.m;
  double x[3] = {0, 0, 0};
  for (int i = 0; i < d; ++i) x[i] = X[t * d + i];
  double L = 1.0, G = (P.g_kind == RANN_G_SINPROD) ? 1.0 : 0.0;
  for (int i = 0; i < d; ++i) L *= lfun(P, i, x[i]).v;
  if (P.g_kind == RANN_G_SINPROD)
    for (int i = 0; i < P.ns; ++i) G *= sinpi(x[i]);
  int k0[3] = {0, 0, 0}, k1[3] = {0, 0, 0};
  for (int i = 0; i < d; ++i) cover_range(P, i, x[i], &k0[i], &k1[i]);
  double total = 0.0;
  for (int c2 = k0[2]; c2 <= (d > 2 ? k1[2] : 0); ++c2)
    for (int c1 = k0[1]; c1 <= k1[1]; ++c1)
      for (int c0 = k0[0]; c0 <= k1[0]; ++c0) {
        int kk[3] = {c0, c1, c2};
        double om = 1.0;
        for (int i = 0; i < d && om != 0.0; ++i) om *= nu_fun(P, i, x[i], kk[i]).v;
        if (om == 0.0) continue;
        int j = c0 + P.nsub[0] * (c1 + P.nsub[1] * c2);
        const SubDev& S = subs[j];
        double acc = 0.0;
        for (int k = 0; k < m; ++k) {
          double z = bias[(int64_t)j * m + k];
          for (int i = 0; i < d; ++i) z = fma(R[((int64_t)j * m + k) * d + i] / P.sig[i], x[i] - S.mu[i], z);
          acc = fma(tanh(z), U[(int64_t)j * m + k], acc);
        }
        total = fma(om, acc, total);
      }
  out[t] = L * total + G;
}

// Coefficient gradient of a loss through the least-squares solve for the
// piecewise diffusion coefficient a = sum_c a_c s_c (Sec. 2, normal
// equations, differentiated).  A v = -div(a grad v) is linear in a, so
// (dH/da_c) x at a point is A_c[v_x] = -s_c Lap v_x - grad s_c . grad v_x,
// with v_x = L sum_j omega_j (Phi_j . U_j), U_j = V_{p_j} x_j, and
// dF/da_c = -A_c[G].  With r = F - H W and h = H lam the gradient is
//   dl/da_c = sum_i s_c(x_i) Q_i + grad s_c(x_i) . Gv_i,
//   Q_i = -r_i Lap v_lam + h_i Lap u_hat,  Gv_i = -r_i grad v_lam + h_i grad u_hat
// (u_hat = v_W + G).  One thread per collocation point forms v, grad v and
// Lap v for both coefficient sets (sharing the tanh of every neuron), then
// the block sums of the g^2 cell terms go to part[block][c] (fixed order).
constexpr int CG_T = 128;
__global__ void __launch_bounds__(CG_T) coef_grad_kernel(ProbDev P, const SubDev* __restrict__ subs,
                                                         const double* __restrict__ R,
                                                         const double* __restrict__ bias,
                                                         const double* __restrict__ Uw,
                                                         const double* __restrict__ Ul,
                                                         const double* __restrict__ res,
                                                         const double* __restrict__ hl, int64_t N,
                                                         double* __restrict__ part) {
  __shared__ double wsum[CG_T / 32][64];
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int d = P.dim, m = P.m, ns = P.ns, gq = P.coef_grid, nc = gq * gq;
  double Q = 0.0, Gv[3] = {0.0, 0.0, 0.0};
  double xs[3] = {0.5, 0.5, 0.5};
  if (t < N) {
    int64_t rem = t;
    for (int i = 0; i < d; ++i) { xs[i] = ((double)(rem % P.G[i]) + 0.5) / (double)P.G[i]; rem /= P.G[i]; }
    // v, grad v, Lap_S v for the two coefficient sets
    double va[4] = {0, 0, 0, 0}, la = 0.0;       // W: grad (up to 3), Lap
    double vb[4] = {0, 0, 0, 0}, lb = 0.0;       // lam
    D3 lf[3];
    for (int i = 0; i < d; ++i) lf[i] = lfun(P, i, xs[i]);
    int k0[3] = {0, 0, 0}, k1[3] = {0, 0, 0};
    for (int i = 0; i < d; ++i) cover_range(P, i, xs[i], &k0[i], &k1[i]);
    for (int c2 = k0[2]; c2 <= (d > 2 ? k1[2] : 0); ++c2)
      for (int c1 = k0[1]; c1 <= k1[1]; ++c1)
        for (int c0 = k0[0]; c0 <= k1[0]; ++c0) {
          const int kk[3] = {c0, c1, c2};
          D3 e[3];
          bool zero = false;
          for (int i = 0; i < d; ++i) {
            const D3 nu = nu_fun(P, i, xs[i], kk[i]);
            if (nu.v == 0.0 && nu.d1 == 0.0 && nu.d2 == 0.0) { zero = true; break; }
            e[i] = {lf[i].v * nu.v, lf[i].d1 * nu.v + lf[i].v * nu.d1,
                    lf[i].d2 * nu.v + 2.0 * lf[i].d1 * nu.d1 + lf[i].v * nu.d2};
          }
          if (zero) continue;
          // g = L omega_j and its derivatives
          double gv = 1.0, dg[3], lapg = 0.0;
          for (int i = 0; i < d; ++i) gv *= e[i].v;
          for (int i = 0; i < d; ++i) {
            double rest = 1.0;
            for (int l = 0; l < d; ++l) if (l != i) rest *= e[l].v;
            dg[i] = e[i].d1 * rest;
            if (i < ns) lapg += e[i].d2 * rest;
          }
          const int j = c0 + P.nsub[0] * (c1 + P.nsub[1] * c2);
          const SubDev& S = subs[j];
          // Phi . U, grad, Lap_S for both sets
          double pa = 0, pb = 0, ga[3] = {0, 0, 0}, gb[3] = {0, 0, 0}, qa = 0, qb = 0;
          for (int k = 0; k < m; ++k) {
            double z = bias[(int64_t)j * m + k];
            double sk[3], n2 = 0.0;
            for (int i = 0; i < d; ++i) {
              sk[i] = R[((int64_t)j * m + k) * d + i] / P.sig[i];
              z = fma(sk[i], xs[i] - S.mu[i], z);
              if (i < ns) n2 += sk[i] * sk[i];
            }
            const double ph = tanh(z), php = 1.0 - ph * ph, lap = -2.0 * ph * php * n2;
            const double uw = Uw[(int64_t)j * m + k], ul = Ul[(int64_t)j * m + k];
            pa = fma(uw, ph, pa);
            pb = fma(ul, ph, pb);
            for (int i = 0; i < d; ++i) { ga[i] = fma(uw * php, sk[i], ga[i]); gb[i] = fma(ul * php, sk[i], gb[i]); }
            qa = fma(uw, lap, qa);
            qb = fma(ul, lap, qb);
          }
          double cross_a = 0.0, cross_b = 0.0;
          for (int i = 0; i < ns; ++i) { cross_a += dg[i] * ga[i]; cross_b += dg[i] * gb[i]; }
          for (int i = 0; i < d; ++i) {
            va[i] += dg[i] * pa + gv * ga[i];
            vb[i] += dg[i] * pb + gv * gb[i];
          }
          la += lapg * pa + 2.0 * cross_a + gv * qa;
          lb += lapg * pb + 2.0 * cross_b + gv * qb;
        }
    // u_hat = v_W + G
    if (P.g_kind == RANN_G_SINPROD) {
      double s[3] = {1.0, 1.0, 1.0}, c[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (i < ns) sincospi(xs[i], &s[i], &c[i]);
      va[0] += RANN_PI * c[0] * s[1] * s[2];
      va[1] += RANN_PI * s[0] * c[1] * s[2];
      va[2] += RANN_PI * s[0] * s[1] * c[2];
      la += -(double)ns * RANN_PI * RANN_PI * (s[0] * s[1] * s[2]);
    }
    const double ri = res[t], hi = hl[t];
    Q = -ri * lb + hi * la;
    for (int i = 0; i < ns; ++i) Gv[i] = -ri * vb[i] + hi * va[i];
  }
  // cell terms s_c Q + grad s_c . Gv, summed over the block (warp shuffles, then warps in order)
  double sx[8], dx[8], sy[8], dy[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    sx[c] = dx[c] = sy[c] = dy[c] = 0.0;
    if (c < gq) { sbox(xs[0], c, gq, &sx[c], &dx[c]); sbox(xs[1], c, gq, &sy[c], &dy[c]); }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int cy = 0; cy < 8; ++cy) {
    if (cy >= gq) break;
#pragma unroll
    for (int cx = 0; cx < 8; ++cx) {
      if (cx >= gq) break;
      double v = (t < N) ? (sx[cx] * sy[cy] * Q + dx[cx] * sy[cy] * Gv[0] + sx[cx] * dy[cy] * Gv[1]) : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) wsum[warp][cy * gq + cx] = v;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    double acc = 0.0;
    for (int w = 0; w < CG_T / 32; ++w) acc += wsum[w][c];
    part[(int64_t)blockIdx.x * nc + c] = acc;
  }
}

// y_i = L(x_i) r_i at the collocation points (the diagonal factor of the
// evaluation matrix, u_hat = L sum_j omega_j Phi_j V_{p_j} W_j + G).
__global__ void lmul_kernel(ProbDev P, const double* __restrict__ r, double* __restrict__ y, int64_t N) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= N) return;
  int64_t rem = g;
  double L = 1.0;
  for (int i = 0; i < P.dim; ++i) {
    const double x = ((double)(rem % P.G[i]) + 0.5) / (double)P.G[i];
    rem /= P.G[i];
    L *= lfun(P, i, x).v;
  }
  y[g] = L * r[g];
}

}  // namespace

cudaError_t launch_assemble(const ProbDev& P, const SubDev* d_sub, const int* d_tiles, int ntiles,
                            const int* /*d_cov*/, const double* d_R, const double* d_b,
                            double* d_Psi, double* d_H, cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  size_t smem = sizeof(double) * ((size_t)TR * (3 + P.dim) + (size_t)TR * P.dim + (size_t)P.m * (P.dim + 2));
  if (smem > 48 * 1024) {
    static const cudaError_t lim = smem_limit_max(assemble_kernel);
    if (lim != cudaSuccess) return lim;
  }
  assemble_kernel<<<ntiles, NT, smem, st>>>(P, d_sub, d_tiles, d_R, d_b, d_Psi, d_H);
  return cudaGetLastError();
}

cudaError_t launch_rhs(const ProbDev& P, double* d_F, int64_t N, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  rhs_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(P, d_F, N);
  return cudaGetLastError();
}

cudaError_t launch_points(const ProbDev& P, double* d_xyz, int64_t N, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  points_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(P, d_xyz, N);
  return cudaGetLastError();
}

cudaError_t launch_eval(const ProbDev& P, const SubDev* d_sub, const double* d_R, const double* d_b,
                        const double* d_U, const double* d_x, int64_t n, double* d_u,
                        cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  eval_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(P, d_sub, d_R, d_b, d_U, d_x, n, d_u);
  return cudaGetLastError();
}

int coef_grad_blocks(int64_t N) { return (int)((N + CG_T - 1) / CG_T); }

cudaError_t launch_coef_grad(const ProbDev& P, const SubDev* d_sub, const double* d_R, const double* d_b,
                             const double* d_Uw, const double* d_Ul, const double* d_r, const double* d_hl,
                             int64_t N, double* d_part, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  coef_grad_kernel<<<coef_grad_blocks(N), CG_T, 0, st>>>(P, d_sub, d_R, d_b, d_Uw, d_Ul, d_r, d_hl, N, d_part);
  return cudaGetLastError();
}

cudaError_t launch_lmul(const ProbDev& P, const double* d_r, double* d_y, int64_t N, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  lmul_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(P, d_r, d_y, N);
  return cudaGetLastError();
}
