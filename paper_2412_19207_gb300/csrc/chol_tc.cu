// Double-float local Cholesky factors and their inverses with the big
// products on the tensor cores (Sec. 3: the local matrices A_i of the
// Schwarz preconditioners; A_i = L_i L_i^T, applied through X_i = L_i^{-1}).
//
// Blocked right-looking factorisation over panels of TC_NB = 256 columns.
// Per panel [c0, c1) of every matrix (one launch serves all matrices):
//   1. the panel itself in 32-column steps on the float32 pipe (double-float:
//      diagonal block with its inverse, panel solve, rank-32 updates of the
//      panel's own columns, and the panel's diagonal block of X by row blocks);
//   2. the trailing update A22 -= L21 L21^T of columns >= c1 (lower
//      triangle) as a digit-slice product on the tensor cores, subtracted
//      straight from the double-float A2;
//   3. the panel's rows of X = L^{-1}: L X = I gives, for the row block
//      I = [c0, c1), X_{I,<c0} = X_II R_I with R_I = -sum_{K<I} L_IK X_K,<c0,
//      and R accumulates in X2 itself: once X_{I,<c1} is final, the rows
//      below receive R_{I'} -= L_{I'I} X_{I,<c1} (one more tensor-core
//      product that reads the same slices of L21 as step 2).
// Steps 1-2 run on the handle's stream and step 3 on a second stream (the
// inverse of panel P overlaps the trailing update of panel P); events keep
// every read after its producer: the inverse of panel P needs panel P and
// the slices of L21(P); the slices of L21(P + 2) reuse the buffer of L21(P)
// only after the inverse of panel P has read it.
// X2 starts at zero (the inverse accumulates R in place and the products read
// X_II and X_{I,<c1} as full blocks, whose upper triangles are zero).
// The products are float64-accurate (digit slices of the float64 value
// hi + lo of every double-float entry, exact chunk sums); the factor keeps
// the double-float representation.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "chol_tc.h"

// chol.cu
cudaError_t launch_panel_steps_df(const CholMat* d_mats, int nmat, int maxn, int c0, int c1, int* d_fail,
                                  const double* d_dmax, cudaStream_t st, int* nlaunch);

// Enumerates every step's operands and products.  With null buffers it only
// sizes them (the largest per-step slice regions and the exponent count);
// with buffers it also fills the split tasks and groups and encodes the
// tensor maps.
cudaError_t chol_tc_build(const std::vector<CholMat>& mats, CholTcPlan& P, uint16_t* const l21_buf[2],
                          uint16_t* inv_buf, uint16_t* xi_buf, int* e_buf) {
  const bool bind = l21_buf && l21_buf[0] && l21_buf[1] && inv_buf && xi_buf && e_buf;
  const int nsl = oz_slices();
  P.split.clear();
  P.groups.clear();
  P.maps.clear();
  P.steps.clear();
  P.maxn = 0;
  P.flops = 0.0;
  P.l21_elems = P.inv_elems = P.xi_elems = 0;
  for (const CholMat& M : mats) P.maxn = std::max(P.maxn, M.n);
  int64_t e_off = 0;
  auto operand = [&](const void* X, int64_t si, int64_t sk, int M, int K, uint16_t* base, int64_t& off) {
    OzSplitTask t{};
    t.X = reinterpret_cast<const double*>(X);
    t.si = si;
    t.sk = sk;
    t.M = M;
    t.K = K;
    t.Kp = oz_kpad(K);
    t.Mp = oz_mpad(M);
    t.e = bind ? e_buf + e_off : nullptr;
    t.out = bind ? base + off : nullptr;
    t.df = 1;
    e_off += M;
    off += (int64_t)nsl * t.Kp * t.Mp;
    P.split.push_back(t);
    return (int)P.split.size() - 1;
  };
  auto group = [&](int ia, int ib, void* C, int M, int N, int ldc, int mode, int lower, int& first) {
    OzGroup g{};
    g.ia = ia;
    g.ib = ib;
    g.ea = P.split[ia].e;
    g.eb = P.split[ib].e;
    g.C = C;
    g.M = M;
    g.N = N;
    g.Kp = P.split[ia].Kp;
    g.ldc = ldc;
    g.mode = mode;
    g.lower = lower;
    g.first = first;
    g.tiles = oz_group_tiles(M, N, lower);
    first += g.tiles;
    P.groups.push_back(g);
  };
  const size_t nm = mats.size();
  for (int c0 = 0; c0 < P.maxn; c0 += TC_NB) {
    const int c1 = c0 + TC_NB;
    CholTcPlan::Step S{};
    S.c0 = c0;
    S.c1 = c1;
    uint16_t* lb = bind ? l21_buf[P.steps.size() & 1] : nullptr;
    int64_t lo = 0, io = 0, xo = 0;
    // operands: L21 (handle's stream), X_II and R_I, then X_{I,<c1} (second stream)
    std::vector<int> a_l21(nm, -1), a_xii(nm, -1), a_ri(nm, -1), a_xi(nm, -1);
    S.sp_l21 = (int)P.split.size();
    for (size_t i = 0; i < nm; ++i) {
      const CholMat& M = mats[i];
      if (M.n <= c1) continue;
      a_l21[i] = operand(M.A2 + (int64_t)c1 * M.ld + c0, M.ld, 1, M.n - c1, TC_NB, lb, lo);
      S.maxM_l21 = std::max(S.maxM_l21, M.n - c1);
    }
    S.n_l21 = (int)P.split.size() - S.sp_l21;
    S.sp_inv = (int)P.split.size();
    for (size_t i = 0; i < nm; ++i) {
      const CholMat& M = mats[i];
      if (M.n <= c0 || c0 == 0) continue;
      const int Ki = std::min(c1, M.n) - c0;
      a_xii[i] = operand(M.X2 + (int64_t)c0 * M.ld + c0, M.ld, 1, Ki, Ki, inv_buf, io);
      a_ri[i] = operand(M.X2 + (int64_t)c0 * M.ld, 1, M.ld, c0, Ki, inv_buf, io);
      S.maxM_inv = std::max(S.maxM_inv, std::max(c0, Ki));
      S.maxKp_inv = std::max(S.maxKp_inv, oz_kpad(Ki));
    }
    S.n_inv = (int)P.split.size() - S.sp_inv;
    S.sp_xi = (int)P.split.size();
    for (size_t i = 0; i < nm; ++i) {
      const CholMat& M = mats[i];
      if (M.n <= c1) continue;                       // X_{I,<c1} feeds only the rows below the panel
      a_xi[i] = operand(M.X2 + (int64_t)c0 * M.ld, 1, M.ld, c1, TC_NB, xi_buf, xo);
      S.maxM_xi = std::max(S.maxM_xi, c1);
    }
    S.n_xi = (int)P.split.size() - S.sp_xi;
    P.l21_elems = std::max(P.l21_elems, lo);
    P.inv_elems = std::max(P.inv_elems, io);
    P.xi_elems = std::max(P.xi_elems, xo);
    // products (flops: 36 slice products of 2 M N K each; the lower group counts its half)
    int first = 0;
    S.g_trail = (int)P.groups.size();
    for (size_t i = 0; i < nm; ++i)
      if (a_l21[i] >= 0) {
        const CholMat& M = mats[i];
        group(a_l21[i], a_l21[i], M.A2 + (int64_t)c1 * M.ld + c1, M.n - c1, M.n - c1, M.ld, OZ_OUT_DF_SUB, 1, first);
        P.flops += 36.0 * (double)(M.n - c1) * (M.n - c1 + 1) * TC_NB;
      }
    S.ng_trail = (int)P.groups.size() - S.g_trail;
    S.tiles_trail = first;
    first = 0;
    S.g_ii = (int)P.groups.size();
    for (size_t i = 0; i < nm; ++i)
      if (a_xii[i] >= 0) {
        const CholMat& M = mats[i];
        const int Ki = std::min(c1, M.n) - c0;
        group(a_xii[i], a_ri[i], M.X2 + (int64_t)c0 * M.ld, Ki, c0, M.ld, OZ_OUT_DF_SET, 0, first);
        P.flops += 36.0 * 2.0 * Ki * c0 * Ki;
      }
    S.ng_ii = (int)P.groups.size() - S.g_ii;
    S.tiles_ii = first;
    first = 0;
    S.g_iii = (int)P.groups.size();
    for (size_t i = 0; i < nm; ++i)
      if (a_xi[i] >= 0) {
        const CholMat& M = mats[i];
        group(a_l21[i], a_xi[i], M.X2 + (int64_t)c1 * M.ld, M.n - c1, c1, M.ld, OZ_OUT_DF_SUB, 0, first);
        P.flops += 36.0 * 2.0 * (M.n - c1) * c1 * TC_NB;
      }
    S.ng_iii = (int)P.groups.size() - S.g_iii;
    S.tiles_iii = first;
    P.steps.push_back(S);
  }
  P.e_ints = e_off;
  return bind ? oz_encode_maps(P.split, P.maps) : cudaSuccess;
}

cudaError_t chol_tc_enqueue(const CholTcPlan& P, const CholMat* d_mats, int nmat, int* d_fail, const double* d_dmax,
                            const OzSplitTask* d_split, const OzGroup* d_groups, const OzMap* d_maps, int* d_err,
                            cudaStream_t st, cudaStream_t st2, int* nlaunch) {
  const int nst = (int)P.steps.size();
  std::vector<cudaEvent_t> ev_pan(nst), ev_l21(nst), ev_inv(nst);
  cudaError_t e = cudaSuccess;
  auto mk = [&](std::vector<cudaEvent_t>& v) {
    for (auto& x : v)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
  };
  mk(ev_pan);
  mk(ev_l21);
  mk(ev_inv);
  cudaEvent_t ev0 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st2, ev0, 0);
  int n = 0;
  for (int s = 0; s < nst && e == cudaSuccess; ++s) {
    const CholTcPlan::Step& S = P.steps[s];
    // 1. the panel (handle's stream)
    if ((e = launch_panel_steps_df(d_mats, nmat, P.maxn, S.c0, S.c1, d_fail, d_dmax, st, &n)) != cudaSuccess) break;
    if ((e = cudaEventRecord(ev_pan[s], st)) != cudaSuccess) break;
    // 2. slices of L21 (the buffer of step s - 2 is free once its inverse product has run) and the
    //    trailing update
    if (s >= 2 && (e = cudaStreamWaitEvent(st, ev_inv[s - 2], 0)) != cudaSuccess) break;
    if (S.n_l21) {
      if ((e = launch_oz_split(d_split + S.sp_l21, S.n_l21, S.maxM_l21, oz_kpad(TC_NB), st)) != cudaSuccess) break;
      n += 2;
    }
    if ((e = cudaEventRecord(ev_l21[s], st)) != cudaSuccess) break;
    if (S.ng_trail) {
      if ((e = launch_oz_gemm_groups(d_groups + S.g_trail, S.ng_trail, S.tiles_trail, d_maps, d_err, st)) !=
          cudaSuccess)
        break;
      ++n;
    }
    // 3. the panel's rows of X (second stream)
    if ((e = cudaStreamWaitEvent(st2, ev_pan[s], 0)) != cudaSuccess) break;
    if (S.n_inv) {
      if ((e = launch_oz_split(d_split + S.sp_inv, S.n_inv, S.maxM_inv, S.maxKp_inv, st2)) != cudaSuccess) break;
      if ((e = launch_oz_gemm_groups(d_groups + S.g_ii, S.ng_ii, S.tiles_ii, d_maps, d_err, st2)) != cudaSuccess)
        break;
      n += 3;
    }
    if (S.n_xi) {
      if ((e = launch_oz_split(d_split + S.sp_xi, S.n_xi, S.maxM_xi, oz_kpad(TC_NB), st2)) != cudaSuccess) break;
      if ((e = cudaStreamWaitEvent(st2, ev_l21[s], 0)) != cudaSuccess) break;
      if ((e = launch_oz_gemm_groups(d_groups + S.g_iii, S.ng_iii, S.tiles_iii, d_maps, d_err, st2)) != cudaSuccess)
        break;
      n += 3;
    }
    if ((e = cudaEventRecord(ev_inv[s], st2)) != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev0, st2);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev0, 0);
  for (auto* v : {&ev_pan, &ev_l21, &ev_inv})
    for (cudaEvent_t x : *v)
      if (x) cudaEventDestroy(x);
  if (ev0) cudaEventDestroy(ev0);
  *nlaunch += n;
  return e == cudaSuccess ? cudaGetLastError() : e;
}
