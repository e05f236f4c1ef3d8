// Streaming double-float Schwarz apply: s_i = X_i^T (X_i g_i) with
// X_i = L_i^{-1} (lower triangle, double-float) and g_i = R_i r, for the local
// inverses of Sec. 3 (A_i^{-1} = L_i^{-T} L_i^{-1}), with every entry of X_i
// read from HBM exactly once.
//
// The product splits by rows: X^T X g = sum_r x_r (x_r . g), x_r the r-th
// row.  A block takes a chunk of consecutive rows of one set.  A producer
// warp streams the rows into a ring of shared-memory stages (1D bulk copies,
// a "full" mbarrier per stage, and an "empty" mbarrier the consumer warps
// arrive on when they are done with it).  The sixteen consumer warps use
// every staged row twice: (1) its dot product with g (kept in shared memory):
// the stage's column pairs, rows concatenated, are split evenly over the
// warps, and each warp sums every row piece it holds over its lanes; the
// pieces of a row are then added in warp order (these reductions add the
// high parts error-free and renormalise once at the end); (2) its share
// x_r y_r of the column sums: teams of threads own the columns cyclically (a
// team is as small as the longest row allows, so short rows keep every
// thread busy) and take the stage's rows in turn, with the sums in registers
// and each entry loaded one pair ahead of its arithmetic.  At the end the
// teams' sums are added in team order and written as the chunk's part; the
// last chunk of a set to finish adds the parts in chunk order into s_i (or,
// for the restricted combine, into z).  Every sum has a fixed order, so the
// result does not depend on scheduling.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "df32.cuh"
#include "mbar.cuh"

namespace {

constexpr int SR_C = 512;                       // consumer threads
constexpr int SR_W = SR_C / 32;
constexpr int SR_G = 2;                         // consumer groups, taking the stages in turn
constexpr int SR_GC = SR_C / SR_G;              // threads of a group
constexpr int SR_GW = SR_W / SR_G;              // warps of a group
constexpr int SR_T = SR_C + 32;                 // and one producer warp
constexpr int SR_PPT = 12;                      // column pairs per thread in the column-sum pass
static_assert(SR_PPT == 12, "the column-sum pass spells out its twelve cases");
constexpr int SR_NMAX = 2 * SR_GC * SR_PPT;     // longest row (6144 columns)
constexpr int SR_STAGE = 7168;                  // double-float entries per stage (56 KB)
constexpr int SR_NST = 3;                       // stages in the ring
constexpr int SR_MAXROWS = 32;                  // rows per stage
constexpr int SR_MAXSUB = 27;                   // subdomains per extended set (3^3)
constexpr int SR_ERR_WAIT = 0x5A00;             // error word: a stage wait gave up
constexpr int SR_SMEM = (SR_NMAX + SR_NST * SR_STAGE) * 8;   // g_i, then the stages

struct SrPlan {
  int r0, nr;                                   // first row and row count of the stage
  int off[SR_MAXROWS];                          // row offsets in the stage (double-float entries, even)
  int pfx[SR_MAXROWS + 1];                      // prefix sums of the rows' column pairs
};

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// barrier over `n` consumer threads (named barrier `id`)
__device__ __forceinline__ void consumers_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
// the same barrier, returning whether v holds in every participating thread
__device__ __forceinline__ bool consumers_all(int id, int n, bool v) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 q, %1, 0;\n bar.red.and.pred p, %2, %3, q;\n selp.s32 %0, 1, 0, p;\n}\n"
      : "=r"(r) : "r"((int)v), "r"(id), "r"(n) : "memory");
  return r != 0;
}

__device__ __forceinline__ double sr_weight(int wkind, int k, int i, const int* __restrict__ inc_ptr) {
  if (wkind == RANN_PREC_SAS) return 1.0 / (double)(inc_ptr[k + 1] - inc_ptr[k]);
  if (wkind == RANN_PREC_RAS) return k == i ? 1.0 : 0.0;
  return 1.0;
}

// double-float entries of row r that one copy moves: r + 1 rounded up to even
// (16-byte multiple); never past the row's leading dimension (a multiple of 4)
__host__ __device__ __forceinline__ int sr_len(int r) { return (r + 2) & ~1; }

__global__ void __launch_bounds__(SR_T, 1) schwarz_apply_rows_df_kernel(
    const CholMat* __restrict__ mats, const SrChunk* __restrict__ chunks, const int* __restrict__ order,
    const int* __restrict__ ck_ptr, const int* __restrict__ set_ptr, const int* __restrict__ set_sub,
    const SubDev* __restrict__ subs, const double* __restrict__ r, const float2* __restrict__ r2, int wkind,
    const int* __restrict__ inc_ptr, double* __restrict__ part, const int64_t* __restrict__ s_off,
    double* __restrict__ s, int* __restrict__ done, int ckind, double* __restrict__ z, int* __restrict__ err) {
  extern __shared__ __align__(128) float4 sr_buf[];   // g_i (SR_NMAX entries), then SR_NST stages
  __shared__ __align__(8) uint64_t full[SR_NST], empty[SR_NST];
  __shared__ SrPlan plan[SR_NST];
  __shared__ float2 wp[SR_G][SR_MAXROWS][SR_GW];      // per group and row: the warps' sums of their pieces
  __shared__ float2 ysm[SR_G][SR_MAXROWS];            // y_r of the group's current stage
  __shared__ int seg_c[SR_MAXSUB + 1], seg_p[SR_MAXSUB];
  __shared__ int64_t seg_w[SR_MAXSUB];
  __shared__ double seg_d[SR_MAXSUB];
  __shared__ int own_q, last, issued;
  __shared__ volatile int abort_flag;

  const SrChunk C = chunks[order[blockIdx.x]];
  const int i = C.set;
  const CholMat M = mats[i];
  const int n = M.n, NS = C.nst;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q0 = set_ptr[i], nq = set_ptr[i + 1] - q0;
  float4* const gsm = sr_buf;                         // g_i by column pairs, high parts then low parts
  float4* const stages = sr_buf + SR_NMAX / 2;
  if (tid < nq) {
    const int k = set_sub[q0 + tid];
    seg_p[tid] = subs[k].p;
    seg_w[tid] = subs[k].woff;
    seg_d[tid] = sr_weight(wkind, k, i, inc_ptr);
    if (k == i) own_q = tid;
  }
  if (tid == 0) {
    abort_flag = 0;
    issued = 0;
    for (int st = 0; st < SR_NST; ++st) {
      mbar_init(smem_u32(&full[st]), 1);
      mbar_init(smem_u32(&empty[st]), SR_GW);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    int c = 0;
    for (int q = 0; q < nq; ++q) { seg_c[q] = c; c += seg_p[q]; }
    seg_c[nq] = c;
  }
  __syncthreads();

  // consumer group grp takes stages grp, grp + SR_G, ...; in the column-sum pass its
  // teams of GS threads own the column pairs c2 = lt + GS k (k < SR_PPT)
  const int grp = warp / SR_GW, gw = warp - grp * SR_GW, gtid = tid - grp * SR_GC;
  int tw = 1;                                         // warps per team: the fewest that divide the
  while (tw < SR_GW && (SR_GW % tw != 0 || 64 * tw * SR_PPT < n)) ++tw;   // group and cover n columns
  const int GS = 32 * tw, nt = SR_GC / GS, tau = gtid / GS, lt = gtid - tau * GS;
  const int gs_log = 5 + (tw >= 2) + (tw >= 4) + (tw >= 8);   // GS = 2^gs_log (tw divides SR_GW = 8)
  const int team = grp * nt + tau, nteams = SR_G * nt;
  float2 ah[SR_PPT], al[SR_PPT];                      // column sums of the pairs (2 c2, 2 c2 + 1)
#pragma unroll
  for (int k = 0; k < SR_PPT; ++k) ah[k] = al[k] = make_float2(0.f, 0.f);

  if (warp == SR_W) {
    // ---- producer warp: stage the chunk's rows, SR_NST stages ahead of the consumers
    int cursor = C.r0;
    for (int st = 0; st < NS; ++st) {
      const int slot = st % SR_NST;
      int ok = 1;
      if (lane == 0) {
        if (st >= SR_NST)
          ok = mbar_wait(smem_u32(&empty[slot]), (uint32_t)(st / SR_NST - 1) & 1u, &abort_flag, err, SR_ERR_WAIT + 2);
        if (ok && abort_flag) ok = 0;
        if (ok) {
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // consumers' reads before the refill
          SrPlan& P = plan[slot];
          P.r0 = cursor;
          int used = 0, nr = 0, pairs = 0;
          while (cursor < C.r1 && nr < SR_MAXROWS && used + sr_len(cursor) <= SR_STAGE) {
            P.off[nr] = used;
            P.pfx[nr] = pairs;
            used += sr_len(cursor);
            pairs += (cursor >> 1) + 1;
            ++nr;
            ++cursor;
          }
          P.nr = nr;
          P.pfx[nr] = pairs;
          mbar_expect_tx(smem_u32(&full[slot]), (uint32_t)used * 8u);
          issued = st + 1;
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      __syncwarp();
      const SrPlan& P = plan[slot];
      const uint32_t base = smem_u32(stages) + (uint32_t)slot * (uint32_t)SR_STAGE * 8u;
      for (int j = lane; j < P.nr; j += 32) {
        const int row = P.r0 + j;
        bulk_g2s(base + (uint32_t)P.off[j] * 8u, M.X2 + (int64_t)row * M.ld, (uint32_t)sr_len(row) * 8u,
                 smem_u32(&full[slot]));
      }
    }
  } else {
    // ---- consumer warps
    // g_i in shared memory, columns below C.r1 (all the chunk's rows reach)
    float* const gf = reinterpret_cast<float*>(gsm);  // pair c2: (h_2c2, h_2c2+1, l_2c2, l_2c2+1)
    for (int c = tid; c < ((C.r1 + 1) & ~1); c += SR_C) {
      float2 v = make_float2(0.f, 0.f);
      if (c < C.r1) {
        int lo = 0, hi = nq - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (seg_c[mid] <= c) lo = mid;
          else hi = mid - 1;
        }
        v = r2 ? r2[seg_w[lo] + (c - seg_c[lo])] : df_split(seg_d[lo] * r[seg_w[lo] + (c - seg_c[lo])]);
      }
      gf[4 * (c >> 1) + (c & 1)] = v.x;
      gf[4 * (c >> 1) + (c & 1) + 2] = v.y;
    }
    consumers_sync(1, SR_C);                          // g_i staged for both groups
    const int bar_a = 2 + 2 * grp, bar_b = 3 + 2 * grp;
    for (int st = grp; st < NS; st += SR_G) {
      const int slot = st % SR_NST;
      const bool got = mbar_wait(smem_u32(&full[slot]), (uint32_t)(st / SR_NST) & 1u, &abort_flag, err,
                                 SR_ERR_WAIT + 1);
      if (!consumers_all(bar_a, SR_GC, got)) break;
      const SrPlan& P = plan[slot];
      const float4* stage = stages + (size_t)slot * (SR_STAGE / 2);
      const int R = P.nr, TP = P.pfx[R];
      // (1) dot products over the warps' shares of the stage's column pairs
      {
        const int a = (int)(((int64_t)gw * TP) / SR_GW), b = (int)(((int64_t)(gw + 1) * TP) / SR_GW);
        for (int j = 0; j < R; ++j) {
          const int p0 = P.pfx[j], p1 = P.pfx[j + 1];
          const int lo = max(a, p0) - p0, hi = min(b, p1) - p0;
          float h = 0.f, l = 0.f;
          if (lo < hi) {
            const float4* xr = stage + (P.off[j] >> 1);
            // accumulators (even column, odd column) of two pairs per lane, packed
            float2 H0 = make_float2(0.f, 0.f), L0 = H0, H1 = H0, L1 = H0;
            int c2 = lo + lane;
            for (; c2 + 32 < hi; c2 += 64) {          // two pairs per lane in flight (the entry above
              const float4 x0 = xr[c2], y0 = gsm[c2]; // the diagonal in a row's last pair is zero)
              const float4 x1 = xr[c2 + 32];
              const float4 y1 = gsm[c2 + 32];
              df_mac_f_x2(H0, L0, make_float2(x0.x, x0.y), make_float2(x0.z, x0.w), make_float2(y0.x, y0.y),
                          make_float2(y0.z, y0.w));
              df_mac_f_x2(H1, L1, make_float2(x1.x, x1.y), make_float2(x1.z, x1.w), make_float2(y1.x, y1.y),
                          make_float2(y1.z, y1.w));
            }
            if (c2 < hi) {
              const float4 x0 = xr[c2];
              const float4 y0 = gsm[c2];
              df_mac_f_x2(H0, L0, make_float2(x0.x, x0.y), make_float2(x0.z, x0.w), make_float2(y0.x, y0.y),
                          make_float2(y0.z, y0.w));
            }
            df_reduce_add_x2(H0, L0, H1, L1);
            h = H0.x; l = L0.x;
            df_reduce_add(h, l, H0.y, L0.y);
            df_warp_sum_lazy(h, l);
          }
          if (lane == 0) wp[grp][j][gw] = make_float2(h, l);
        }
      }
      consumers_sync(bar_b, SR_GC);
      // y_r = the row's pieces added in warp order: warp w of the group takes rows w, w + SR_GW
      for (int j = gw; j < R; j += SR_GW) {
        float2 v = lane < SR_GW ? wp[grp][j][lane] : make_float2(0.f, 0.f);
#pragma unroll
        for (int o = SR_GW / 2; o > 0; o >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, v.x, o);
          const float ol = __shfl_xor_sync(0xffffffffu, v.y, o);
          df_reduce_add(v.x, v.y, oh, ol);
        }
        df_renorm(v.x, v.y);
        if (lane == 0) ysm[grp][j] = v;
      }
      consumers_sync(bar_b, SR_GC);
      // (2) column sums: team tau takes rows tau, tau + nt, ...; a row reaches kact of the thread's
      // SR_PPT column pairs, entered at the last of them (the bodies fall through down to k = 0)
      for (int j = tau; j < R; j += nt) {
        const int nall = ((P.r0 + j) >> 1) + 1;
        const float4* xr = stage + (P.off[j] >> 1) + lt;
        const float2 y = ysm[grp][j];
        const float2 yh = make_float2(y.x, y.x), yl = make_float2(y.y, y.y), nyh = make_float2(-y.x, -y.x);
        const int kact = nall > lt ? min(SR_PPT, ((nall - lt - 1) >> gs_log) + 1) : 0;
        // the next pair's entry is loaded before this pair's arithmetic (two buffers, by parity)
        float4 xb0 = make_float4(0.f, 0.f, 0.f, 0.f), xb1 = xb0;
        if (kact > 0) {
          if ((kact - 1) & 1) xb1 = xr[GS * (kact - 1)];
          else xb0 = xr[GS * (kact - 1)];
        }
#define SR_BUF(k) (((k) & 1) ? xb1 : xb0)
#define SR_COLSUM(k)                                                                                    \
  case (k) + 1: {                                                                                       \
    if ((k) > 0) SR_BUF((k) + 1) = xr[GS * ((k) > 0 ? (k) - 1 : 0)];                                    \
    const float4 x = SR_BUF(k);                                                                         \
    df_mac_f_x2n(ah[k], al[k], make_float2(x.x, x.y), make_float2(x.z, x.w), yh, yl, nyh);              \
  }
        switch (kact) {
          SR_COLSUM(11) SR_COLSUM(10) SR_COLSUM(9) SR_COLSUM(8) SR_COLSUM(7) SR_COLSUM(6)
          SR_COLSUM(5) SR_COLSUM(4) SR_COLSUM(3) SR_COLSUM(2) SR_COLSUM(1) SR_COLSUM(0)
          default: break;
        }
#undef SR_COLSUM
#undef SR_BUF
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[slot]));
    }
  }
  __syncthreads();
  if (abort_flag && tid == SR_C) {
    // let the copies in flight land before the block's shared memory is reused or released: only
    // a slot's latest stage can have copies in flight (a slot is refilled after its stage's release)
    for (int st = max(0, issued - SR_NST); st < issued; ++st)
      mbar_drain(smem_u32(&full[st % SR_NST]), (uint32_t)(st / SR_NST) & 1u);
  }
  __syncthreads();
  // the chunk's column sums (columns < C.r1): the teams' sums (group 0's, then group 1's)
  // added in team order
  double* pr = part + C.poff;
  if (!abort_flag && tid < SR_C) {
    {
      const int np = (C.r1 + 1) >> 1;
#pragma unroll
      for (int k = 0; k < SR_PPT; ++k) {
        const int c2 = lt + GS * k;
        if (c2 < np) stages[(size_t)team * np + c2] = make_float4(ah[k].x, al[k].x, ah[k].y, al[k].y);
      }
      consumers_sync(1, SR_C);
      for (int c2 = tid; c2 < np; c2 += SR_C) {
        float4 v = stages[c2];
        for (int t2 = 1; t2 < nteams; ++t2) {
          const float4 u = stages[(size_t)t2 * np + c2];
          df_add(v.x, v.y, u.x, u.y);
          df_add(v.z, v.w, u.z, u.w);
        }
        const int c = 2 * c2;
        pr[c] = df_to_double(v.x, v.y);
        if (c + 1 < C.r1) pr[c + 1] = df_to_double(v.z, v.w);
      }
    }
  }
  // the last chunk of the set to finish adds the parts (chunk order)
  __threadfence();
  __syncthreads();
  const int k0 = ck_ptr[i], k1 = ck_ptr[i + 1];
  if (tid == 0) last = (atomicAdd(&done[i], 1) == k1 - k0 - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (!abort_flag) {
    const bool ras = ckind == RANN_PREC_RAS;
    const int c0 = ras ? seg_c[own_q] : 0, c1 = ras ? c0 + seg_p[own_q] : n;
    for (int c = c0 + tid; c < c1; c += SR_T) {
      int k = k0;
      while (chunks[k].r1 <= c) ++k;                 // the first chunk with a row >= c
      double acc = 0.0;
      for (; k + 8 <= k1; k += 8) {                  // eight loads in flight, added in chunk order
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(part + chunks[k + u].poff + c);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
      }
      for (; k < k1; ++k) acc += __ldcg(part + chunks[k].poff + c);
      if (ras) z[seg_w[own_q] + (c - c0)] = acc;
      else s[s_off[i] + c] = acc;
    }
  }
  if (tid == 0) done[i] = 0;                          // ready for the next apply (stream order)
}

}  // namespace

int schwarz_rows_nmax() { return SR_NMAX; }
int schwarz_rows_stage() { return SR_STAGE; }

// Rows of each set cut into chunks of about `target` entries of the triangle
// (a chunk never spans two sets); parts are laid out chunk after chunk, n_i
// doubles each.  Launch order: the larger chunks first.
void schwarz_rows_plan(const std::vector<int>& nvec, int64_t target, std::vector<SrChunk>& chunks,
                       std::vector<int>& ck_ptr, std::vector<int>& order, int64_t& part_total) {
  chunks.clear();
  ck_ptr.assign(1, 0);
  part_total = 0;
  for (int i = 0; i < (int)nvec.size(); ++i) {
    const int n = nvec[i];
    int row = 0, k = 0;
    while (row < n) {
      SrChunk c{};
      c.set = i;
      c.r0 = row;
      int64_t el = 0;
      while (row < n && (el == 0 || el + row + 1 <= target)) { el += row + 1; ++row; }
      c.r1 = row;
      c.k = k++;
      c.nst = 0;                                   // stages: the rows packed as the producer packs them
      for (int r2 = c.r0; r2 < c.r1; ++c.nst) {
        int used = 0, nr = 0;
        while (r2 < c.r1 && nr < SR_MAXROWS && used + sr_len(r2) <= SR_STAGE) { used += sr_len(r2); ++nr; ++r2; }
      }
      c.poff = part_total;
      part_total += n;
      chunks.push_back(c);
    }
    ck_ptr.push_back((int)chunks.size());
  }
  order.resize(chunks.size());
  for (size_t c = 0; c < chunks.size(); ++c) order[c] = (int)c;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int64_t ea = (int64_t)(chunks[a].r1 - chunks[a].r0) * (chunks[a].r0 + chunks[a].r1 + 1);
    const int64_t eb = (int64_t)(chunks[b].r1 - chunks[b].r0) * (chunks[b].r0 + chunks[b].r1 + 1);
    return ea > eb;
  });
}

cudaError_t launch_schwarz_apply_rows_df(const CholMat* d_mats, const SrChunk* d_chunks, const int* d_order,
                                         int nchunks, const int* d_ck_ptr, const int* d_set_ptr,
                                         const int* d_set_sub, const SubDev* d_sub, const double* d_r,
                                         const float2* d_r2, int wkind, const int* d_inc_ptr, double* d_part,
                                         const int64_t* d_s_off, double* d_s, int* d_done, int ckind, double* d_z,
                                         int* d_err, cudaStream_t st) {
  if (nchunks == 0) return cudaSuccess;
  const int smem = SR_SMEM;
  static const cudaError_t lim = smem_limit_max(schwarz_apply_rows_df_kernel);
  if (lim != cudaSuccess) return lim;
  schwarz_apply_rows_df_kernel<<<nchunks, SR_T, smem, st>>>(d_mats, d_chunks, d_order, d_ck_ptr, d_set_ptr, d_set_sub,
                                                             d_sub, d_r, d_r2, wkind, d_inc_ptr, d_part, d_s_off, d_s,
                                                             d_done, ckind, d_z, d_err);
  return cudaGetLastError();
}
