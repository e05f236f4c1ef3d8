// Float64-accurate products on the bf16 tensor cores (Ozaki splitting).
//
// GB300 executes float64 at 1/70 of its float32 rate while its bf16 tensor
// cores run ~1500x faster than float64, so the dense float64 contractions --
// the Gram matrices Psi_j^T Psi_j of the PCA (Sec. 4), the reduced blocks
// H_j V_{p_j} (Eq. (system_new)) and the neighbour Gram blocks B_k^T B_l of
// the Schwarz matrices (Sec. 3; operands gathered to the shared rows) -- are
// formed from exact integer digit slices:
//   * each row i of an operand is scaled by 2^{-e_i} (e_i = ceil(log2 max_k |x_ik|)),
//     rounded to the 56-bit fixed-point integer X = round(x 2^{56 - e_i}) and
//     written in balanced base 128, x = 2^{e_i} sum_{q=1}^{8} d_q 2^{-7q} + O(2^{e_i - 57}),
//     d_1 in [-128, 128], d_q in [-64, 63] for q > 1 -- all exact in bf16
//     (integer arithmetic on the float64 bit pattern; finite inputs);
//   * C_ij = 2^{e_i + e_j} sum_{s} 2^{-7s} sum_{q + r = s} (D^A_q D^B_r^T)_ij.
//     The 36 slice products of the weight groups s = 2..9 are kept (the rest
//     lie below 2^-63 relative); the products of one group accumulate on the
//     tensor cores in float32, exact because every partial sum over a
//     256-long k chunk is an integer below 2^24 (group s = g + 2 is bounded
//     by 256 * 4096 (g + 3) for g >= 1 and by 2^22 for g = 0); at the end of
//     a chunk the eight group sums are joined exactly in integers,
//     hi = sum_{s<=5} c_s 128^{5-s} and lo = sum_{s>=6} c_s 128^{9-s}, which
//     accumulate over the chunks without rounding (exact for K < 2^17); the
//     tile ends with the single rounding of hi 2^-35 + lo 2^-63 to float64.
// The error is a few units of 2^-53 K max_k|a_ik| max_k|b_jk|, the float64
// bound.  The scheme is that of Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59 (2012).
//
// Blackwell mapping of one 128 x 64 tile of C: the eight group accumulators
// (8 x 64 float32 columns) fill the 512 columns of tensor memory; a 4-stage
// ring of k steps of 16 is filled by 4-D TMA boxes (all eight slices of the
// tile's 128 A rows and 64 B rows; each box row is a 32-row group, 512
// contiguous bytes, landing in the no-swizzle K-major core-matrix layout); one
// thread issues the 36 tcgen05.mma of a k step; eight warps drain the
// accumulators to the integer chunk sums through tcgen05.ld.
#include "common.cuh"
#include "df32.cuh"
#include "mbar.cuh"
#include <cuda.h>
#include <cudaTypedefs.h>

namespace {

constexpr int OZ_Q = 8;             // digit slices per operand
constexpr int OZ_NG = 8;            // weight groups s = 2..9 (g = s - 2 = q + r, zero-based)
constexpr int OZ_TK = 16;           // k of one stage (one tcgen05.mma step)
constexpr int OZ_CHUNK_STEPS = 16;  // 256 k per exact float32 accumulation
constexpr int OZ_STAGES = 3;
constexpr int OZ_A_BYTES = OZ_Q * OZ_TILE_M * OZ_TK * 2;   // 32 KB
constexpr int OZ_B_BYTES = OZ_Q * OZ_TILE_N * OZ_TK * 2;   // 16 KB
constexpr int OZ_STAGE_BYTES = OZ_A_BYTES + OZ_B_BYTES;
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE_BYTES + OZ_TILE_M * (OZ_TILE_N + 1) * 8 + 1024;   // ring, output staging, alignment slack
constexpr int OZ_DRAIN_WARPS = 8;   // warps 2..9: lane quarter w % 4, column half (w - 2) / 4
constexpr int OZ_THREADS = 32 * (2 + OZ_DRAIN_WARPS);
static_assert(OZ_NG * OZ_TILE_N == 512, "the group accumulators fill tensor memory");

__device__ __forceinline__ uint32_t bf16_of_small_int(int d) {
  // |d| <= 128: exactly representable in bf16 (8 significant bits), whose
  // pattern is the upper half of the float32 one.  The float32 value comes
  // without a conversion instruction: 1.5 2^23 + d has d in its low mantissa
  // bits (|d| < 2^22), and subtracting 1.5 2^23 leaves d exactly.
  return __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16;
}

// The float64 bit pattern of operand entry idx (a double-float pair is read
// as the float64 value hi + lo).
__device__ __forceinline__ long long oz_bits(const OzSplitTask& t, int64_t idx) {
  if (t.df) {
    const float2 v = reinterpret_cast<const float2*>(t.X)[idx];
    return __double_as_longlong((double)v.x + (double)v.y);
  }
  return reinterpret_cast<const long long*>(t.X)[idx];
}

// e_i of 32 rows of one operand per block (deterministic integer max of |x|'s bits).
__global__ void __launch_bounds__(256) oz_scale_kernel(const OzSplitTask* __restrict__ tasks) {
  const OzSplitTask t = tasks[blockIdx.y];
  const int i0 = blockIdx.x * 32;
  if (i0 >= t.M) return;
  __shared__ long long red[8][33];
  const int a = threadIdx.x & 31, b = threadIdx.x >> 5;
  const long long ABS = 0x7FFFFFFFFFFFFFFFll;
  if (t.sk == 1 && !t.gather) {   // rows contiguous in k: warp b owns rows i0 + b + 8c, lanes stride k
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + b + 8 * c;
      long long mx = 0;
      if (i < t.M)
        for (int k = a; k < t.K; k += 32) mx = max(mx, oz_bits(t, (int64_t)i * t.si + k) & ABS);
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (a == 0) red[0][b + 8 * c] = mx;
    }
  } else {              // rows contiguous in i: lane a owns row i0 + a, warps stride k
    const int i = i0 + a;
    long long mx = 0;
    if (i < t.M)
      for (int k = b; k < t.K; k += 8) {
        const int64_t kk = t.gather ? t.gather[k] : k;
        mx = max(mx, oz_bits(t, (int64_t)i * t.si + kk * t.sk) & ABS);
      }
    red[b][a] = mx;
    __syncthreads();
    if (b == 0) {
      for (int w = 1; w < 8; ++w) mx = max(mx, red[w][a]);
      red[0][a] = mx;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32 && i0 + (int)threadIdx.x < t.M) {
    const long long m = red[0][threadIdx.x];
    const int E = (int)(m >> 52);
    int e = 0;                                       // all-zero row
    if (m != 0) e = (E == 0) ? -1022 : ((m & 0xFFFFFFFFFFFFFll) == 0 ? E - 1023 : E - 1022);
    t.e[i0 + threadIdx.x] = e;                       // max |x_i.| <= 2^e
  }
}

// Digit slices of a 32-row x 64-k tile.  Slice q of row i, column k sits at
// out[q Mp Kp + ((k / 8) Mp + i) 8 + k % 8]: 8 k of a row contiguous, then the
// rows (32-row groups are 512 contiguous bytes), then the groups of 8 k, then
// the slices; zero for k >= K and for the padding rows M <= i < Mp.
__global__ void __launch_bounds__(256) oz_split_kernel(const OzSplitTask* __restrict__ tasks) {
  const OzSplitTask t = tasks[blockIdx.z];
  const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
  if (i0 >= t.Mp || k0 >= t.Kp) return;
  __shared__ long long tile[32][65];
  if (t.sk == 1 && !t.gather) {                      // rows contiguous in k
    for (int e = threadIdx.x; e < 2048; e += 256) {
      const int kk = e & 63, ii = e >> 6, i = i0 + ii, k = k0 + kk;
      tile[ii][kk] = (i < t.M && k < t.K) ? oz_bits(t, (int64_t)i * t.si + k) : 0;
    }
  } else {                                           // columns contiguous in i (or gathered k)
    for (int e = threadIdx.x; e < 2048; e += 256) {
      const int ii = e & 31, kk = e >> 5, i = i0 + ii, k = k0 + kk;
      tile[ii][kk] = (i < t.M && k < t.K) ? oz_bits(t, (int64_t)i * t.si + (int64_t)(t.gather ? t.gather[k] : k) * t.sk)
                                          : 0;
    }
  }
  __syncthreads();
  // thread: row i0 + (tid % 32), 8 k starting at k0 + 8 (tid / 32); a warp writes 512
  // contiguous bytes of every slice
  const int ii = threadIdx.x & 31, kc = threadIdx.x >> 5, i = i0 + ii;
  if (k0 + 8 * kc >= t.Kp) return;
  const int ei = (i < t.M) ? t.e[i] : 0;
  uint32_t w[OZ_Q][4];
#pragma unroll
  for (int k8 = 0; k8 < 8; ++k8) {
    // X = round(|x| 2^{56 - e_i}) with the sign of x, from the float64 fields
    const long long bits = tile[ii][8 * kc + k8];
    const int E = (int)((bits >> 52) & 0x7ff);
    long long v = 0;
    if (E != 0) {                                    // zero and subnormals give 0
      const long long mant = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
      const int sh = E - 1075 + 56 - ei;             // <= 4 since |x| <= 2^{e_i}
      if (sh >= 0) v = mant << sh;
      else if (sh > -60) v = (mant + (1ll << (-sh - 1))) >> (-sh);
      if (bits < 0) v = -v;
    }
    // balanced base-128 digits: adding 64 (1 + 128 + ... + 128^6) makes the seven
    // low digits d + 64 in [0, 127] plain base-128 digits of u, and the leading
    // digit u >> 49 (|lead| <= 128)
    const long long u = v + 0x1020408102040ll;
    uint32_t d16[OZ_Q];
    d16[0] = bf16_of_small_int((int)(u >> 49));
#pragma unroll
    for (int q = 1; q < OZ_Q; ++q) d16[q] = bf16_of_small_int((int)((u >> (7 * (OZ_Q - 1 - q))) & 127) - 64);
#pragma unroll
    for (int q = 0; q < OZ_Q; ++q) {
      if (k8 & 1) w[q][k8 >> 1] |= d16[q] << 16;
      else w[q][k8 >> 1] = d16[q];
    }
  }
  const int64_t slice = (int64_t)t.Mp * t.Kp;
  uint16_t* o = t.out + ((int64_t)((k0 >> 3) + kc) * t.Mp + i) * 8;
#pragma unroll
  for (int q = 0; q < OZ_Q; ++q)
    *reinterpret_cast<uint4*>(o + q * slice) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

// ---- Blackwell primitives (inline PTX; barriers in mbar.cuh) ----
// 4-D TMA box (32-row groups of 8 k, groups, 2 groups of 8 k, 8 slices) into shared memory;
// completes on bar.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(dst), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor, no swizzle, K-major: start, leading (k
// direction) and stride (8-row direction) byte offsets, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// D (+)= A B^T; COL selects the A collector buffer: 0 none, 1 fill (keep A for the
// next MMAs), 2 use (A as kept), 3 last use (A as kept, then released).
template <int COL>
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
  if constexpr (COL == 0)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem), "l"(adesc), "l"(bdesc),
        "r"(idesc), "r"(acc));
  else if constexpr (COL == 1)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  else if constexpr (COL == 2)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

// 32 lanes x 8 consecutive float32 columns of tensor memory (this warp's lane quarter).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// c_a 128 + c_b from two group sums (exact integers in float32; |result| < 2^31)
__device__ __forceinline__ int join2(uint32_t a, uint32_t b) {
  return __float2int_rn(__uint_as_float(a)) * 128 + __float2int_rn(__uint_as_float(b));
}

// One 128 x 64 tile of C = A B^T from the digit slices.
//   warp 0, one lane: TMA producer over the k steps (stage ring with full /
//           empty barriers);
//   warp 1: allocates the 512 tensor-memory columns; one lane issues the MMAs
//           (group g = q + r at columns 64 g; the first k step of a chunk
//           overwrites);
//   warps 2..9: drain each chunk's group sums into the exact integers hi / lo
//           (lo carried into hi above 2^28, so lo stays 32-bit) and write the tile.
struct OzTile {               // one tile: operands, their row exponents, sizes, origin in C
  int ia, ib;
  const int* ea;
  const int* eb;
  int M, N, Kp, tm, tn;
};
// The tile entry (hi 2^-35 + lo 2^-63) 2^ex from the exact integer sums, in float64: one rounding.
__device__ __forceinline__ double oz_f64_of(long long hi, int lo, int ex) {
  const double v = fma((double)hi, 0x1p-35, (double)lo * 0x1p-63);
  // times 2^ex: a power-of-two factor built from its exponent field when it is normal
  return (ex >= -1022 && ex <= 1023) ? v * __longlong_as_double((long long)(ex + 1023) << 52) : ldexp(v, ex);
}
// The same entry as a double-float without float64 arithmetic (GB300's float64 pipe runs at
// 1/64 of float32): hi = c2 2^48 + c1 2^24 + c0 with c1, c0 in [0, 2^24) converts to floats
// exactly; the pieces (and lo, rounded to 24 bits: far below the product's error) are added
// with error-free float32 steps, then scaled by 2^(ex - 35).  About 2^-47 relative, the
// double-float format's own accuracy.
__device__ __forceinline__ float2 oz_df_of(long long hi, int lo, int ex) {
  const float a = __int2float_rn((int)(hi >> 48)) * 0x1p48f;
  const float b = __int2float_rn((int)((hi >> 24) & 0xFFFFFF)) * 0x1p24f;
  const float c = __int2float_rn((int)(hi & 0xFFFFFF));
  const float d = __int2float_rn(lo) * 0x1p-28f;
  float s, e;
  df_two_sum(a, b, s, e);
  df_add(s, e, c, 0.f);
  df_add(s, e, d, 0.f);
  const int k = ex - 35;
  if (k >= -126 && k <= 127) {
    const float f = __int_as_float((k + 127) << 23);
    return make_float2(s * f, e * f);
  }
  return make_float2(ldexpf(s, k), ldexpf(e, k));
}
// Output of the grouped launch: float64 C, or double-float C minus (plus) the product.
struct OzEpi {
  static constexpr bool kDf = true;         // can write double-float outputs
  void* C;
  int ldc, mode, lower;
  __device__ __forceinline__ void operator()(int i, int j, long long hi, int lo, int ex) const {
    if (mode == OZ_OUT_F64) {
      reinterpret_cast<double*>(C)[(int64_t)i * ldc + j] = oz_f64_of(hi, lo, ex);
      return;
    }
    put_df(i, j, oz_df_of(hi, lo, ex));
  }
  __device__ __forceinline__ bool df() const { return mode != OZ_OUT_F64; }
  __device__ __forceinline__ void put_df(int i, int j, float2 s) const {
    if (lower && j > i) return;
    float2* p = reinterpret_cast<float2*>(C) + (int64_t)i * ldc + j;
    if (mode == OZ_OUT_DF_SET) {
      *p = s;
    } else {
      float2 c = *p;
      df_add(c.x, c.y, -s.x, -s.y);
      *p = c;
    }
  }
};
struct OzEpiF64 {
  static constexpr bool kDf = false;
  double* C;
  int ldc;
  __device__ __forceinline__ void operator()(int i, int j, long long hi, int lo, int ex) const {
    C[(int64_t)i * ldc + j] = oz_f64_of(hi, lo, ex);
  }
  __device__ __forceinline__ bool df() const { return false; }
};
constexpr int OZ_EP_LD = OZ_TILE_N + 1;   // row stride of the staged double-float tile (2-way banks)
constexpr int OZ_EP_BATCH = 8;            // rows of C each drain warp reads before it updates them

// Double-float output of a tile through shared memory: every drain thread stages its 32 entries
// (the operand ring is free, all MMAs have completed); then each drain warp takes rows rr = w,
// w + 8, ... and, OZ_EP_BATCH rows at a time, first loads the rows' 64-entry segments of C
// (coalesced; up to 16 loads in flight per lane), then updates and stores them.
__device__ __forceinline__ void oz_epilogue_df(const OzTile& t, const OzEpi& epi, float2* tile, int dw, int lane) {
  const bool sub = epi.mode == OZ_OUT_DF_SUB;
  for (int r0 = dw; r0 < OZ_TILE_M; r0 += OZ_DRAIN_WARPS * OZ_EP_BATCH) {
    float2 cv[OZ_EP_BATCH][2];
#pragma unroll
    for (int b = 0; b < OZ_EP_BATCH; ++b)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rr = r0 + b * OZ_DRAIN_WARPS, i = t.tm + rr, j = t.tn + lane + 32 * h;
        cv[b][h] = make_float2(0.f, 0.f);
        if (sub && rr < OZ_TILE_M && i < t.M && j < t.N && !(epi.lower && j > i))
          cv[b][h] = reinterpret_cast<const float2*>(epi.C)[(int64_t)i * epi.ldc + j];
      }
#pragma unroll
    for (int b = 0; b < OZ_EP_BATCH; ++b)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rr = r0 + b * OZ_DRAIN_WARPS, i = t.tm + rr, j = t.tn + lane + 32 * h;
        if (rr < OZ_TILE_M && i < t.M && j < t.N && !(epi.lower && j > i)) {
          const float2 v = tile[rr * OZ_EP_LD + lane + 32 * h];
          float2 c = cv[b][h];
          if (sub) df_add(c.x, c.y, -v.x, -v.y);
          else c = v;
          reinterpret_cast<float2*>(epi.C)[(int64_t)i * epi.ldc + j] = c;
        }
      }
  }
}

// Persistent tile loop: block b takes tiles b, b + gridDim.x, ... (fetch(i, t, epi) fills
// tile i's operands and output).  The roles of one tile (above) run over the whole
// sequence with running stage and chunk counters, so the producer streams the next tile's
// operands and the MMA thread starts its products as soon as the drain warps have read the
// accumulators, while the drain warps still finish the previous tile's output.  The output
// staging area of the double-float epilogue follows the operand ring.
template <class Fetch>
__device__ __forceinline__ void oz_tiles_run(const Fetch& fetch, int ntiles, const OzMap* __restrict__ maps,
                                             int* __restrict__ err) {
  using Epi = typename Fetch::Epi;
  extern __shared__ uint8_t oz_dyn[];
  __shared__ __align__(8) uint64_t bar_full[OZ_STAGES], bar_empty[OZ_STAGES], bar_accf, bar_acce, bar_fin;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, issued, consumed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = (smem_u32(oz_dyn) + 1023u) & ~1023u;
  volatile int* abort = &abort_flag;
  if (tid == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_accf), 1);
    mbar_init(smem_u32(&bar_acce), OZ_DRAIN_WARPS);
    mbar_init(smem_u32(&bar_fin), 1);
    abort_flag = 0;
    issued = 0;
    consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      int g = 0;                                  // stages issued so far (all tiles)
      for (int b = (int)blockIdx.x; ok && b < ntiles; b += (int)gridDim.x) {
        OzTile t;
        Epi epi;
        fetch(b, t, epi);
        const void* ma = &maps[2 * t.ia];        // A role: 128-row boxes
        const void* mb = &maps[2 * t.ib + 1];    // B role: 64-row boxes
        const int nks = t.Kp / OZ_TK;
        for (int ks = 0; ks < nks; ++ks, ++g) {
          const int s = g % OZ_STAGES;
          if (g >= OZ_STAGES && !(ok = mbar_wait(smem_u32(&bar_empty[s]), ((g / OZ_STAGES) - 1) & 1, abort, err, 1)))
            break;
          const uint32_t full = smem_u32(&bar_full[s]);
          const uint32_t sa = sbase + s * OZ_STAGE_BYTES;
          mbar_expect_tx(full, OZ_STAGE_BYTES);
          tma_load_4d(sa, ma, 0, t.tm / 32, 2 * ks, 0, full);
          tma_load_4d(sa + OZ_A_BYTES, mb, 0, t.tn / 32, 2 * ks, 0, full);
          issued = g + 1;
        }
      }
      // every stage's release (an MMA commit) has landed before the block's shared memory is given up
      for (int q = max(g - OZ_STAGES, 0); ok && q < g; ++q)
        ok = mbar_wait(smem_u32(&bar_empty[q % OZ_STAGES]), (q / OZ_STAGES) & 1, abort, err, 5);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // kind::f16 instruction descriptor: f32 accumulator, bf16 A and B, both K-major, N = 64, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_TILE_N >> 3) << 17) |
                             ((uint32_t)(OZ_TILE_M >> 4) << 24);
      // stage layout: slice q, k group c, row i, k % 8 at ((q * 2 + c) * rows + i) * 16 + 2 (k % 8) bytes
      const uint64_t a0 = smem_desc(sbase, OZ_TILE_M * 16, 128);
      const uint64_t b0 = smem_desc(sbase + OZ_A_BYTES, OZ_TILE_N * 16, 128);
      bool ok = true;
      int g = 0, cg = 0;                          // stages and accumulation chunks consumed so far
      for (int b = (int)blockIdx.x; ok && b < ntiles; b += (int)gridDim.x) {
        OzTile t;
        Epi epi;
        fetch(b, t, epi);
        const int nks = t.Kp / OZ_TK;
        for (int ks = 0; ks < nks; ++ks, ++g) {
          const int s = g % OZ_STAGES, kc = ks % OZ_CHUNK_STEPS;
          if (kc == 0 && cg > 0) {                // the drain has read the previous chunk's accumulators
            if (!(ok = mbar_wait(smem_u32(&bar_acce), (cg - 1) & 1, abort, err, 2))) break;
            tc_fence_after();
          }
          if (!(ok = mbar_wait(smem_u32(&bar_full[s]), (g / OZ_STAGES) & 1, abort, err, 3))) break;
          tc_fence_after();
          const uint64_t soff = (uint64_t)((s * OZ_STAGE_BYTES) >> 4);
          // A slice q meets B slices r = 0..7-q back to back: it is read from shared
          // memory once and kept in the collector buffer for the following MMAs
#pragma unroll
          for (int q = 0; q < OZ_Q; ++q) {
            const uint64_t ad = a0 + soff + (uint64_t)(q * (OZ_TILE_M * 2));
            const int acc = (kc != 0 || q != 0) ? 1 : 0;
#pragma unroll
            for (int r = 0; r < OZ_Q - q; ++r) {
              const uint32_t d = tbase + (uint32_t)((q + r) * OZ_TILE_N);
              const uint64_t bd = b0 + soff + (uint64_t)(r * (OZ_TILE_N * 2));
              if (q == OZ_Q - 1) tc_mma<0>(d, ad, bd, idesc, acc);
              else if (r == 0) tc_mma<1>(d, ad, bd, idesc, acc);
              else if (r == OZ_Q - 1 - q) tc_mma<3>(d, ad, bd, idesc, acc);
              else tc_mma<2>(d, ad, bd, idesc, acc);
            }
          }
          tc_commit(smem_u32(&bar_empty[s]));    // the stage is free once these MMAs have read it
          if (kc == OZ_CHUNK_STEPS - 1 || ks == nks - 1) {
            tc_commit(smem_u32(&bar_accf));
            ++cg;
          }
          consumed = g + 1;
        }
      }
    }
  } else {
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const uint32_t trow = tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 32);
    float2* const stage_out = reinterpret_cast<float2*>(oz_dyn + (sbase - smem_u32(oz_dyn)) + OZ_STAGES * OZ_STAGE_BYTES);
    int cg = 0;                                   // accumulation chunks drained so far
    for (int b = (int)blockIdx.x; b < ntiles; b += (int)gridDim.x) {
      OzTile t;
      Epi epi;
      fetch(b, t, epi);
      const int nch = (t.Kp / OZ_TK + OZ_CHUNK_STEPS - 1) / OZ_CHUNK_STEPS;
      long long hi[32];
      int lo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) { hi[j] = 0; lo[j] = 0; }
      bool ok = true;
      for (int c = 0; c < nch; ++c, ++cg) {
        // every lane waits; the warp continues together (tcgen05.ld is warp-collective)
        if (!(ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&bar_accf), cg & 1, abort, err, 4)))) break;
        tc_fence_after();
#pragma unroll
        for (int sub = 0; sub < 4; ++sub) {
          uint32_t v[4][8];
          int p0[8], p1[8];
#pragma unroll
          for (int g = 0; g < 4; ++g) tmem_ld8(trow + g * OZ_TILE_N + sub * 8, v[g]);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 8; ++j) { p0[j] = join2(v[0][j], v[1][j]); p1[j] = join2(v[2][j], v[3][j]); }
#pragma unroll
          for (int g = 0; g < 4; ++g) tmem_ld8(trow + (g + 4) * OZ_TILE_N + sub * 8, v[g]);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int p2 = join2(v[0][j], v[1][j]), p3 = join2(v[2][j], v[3][j]);
            const long long hc = ((long long)p0[j] << 14) + p1[j];       // sum_{s<=5} c_s 128^{5-s}
            const long long lt = ((long long)p2 << 14) + p3 + lo[sub * 8 + j];
            const long long carry = lt >> 28;                            // floor(lt / 2^28)
            lo[sub * 8 + j] = (int)(lt - (carry << 28));
            hi[sub * 8 + j] += hc + carry;
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_acce));
      }
      // one decision for all drain warps (the staged epilogue synchronises them)
      int go = (ok && !*abort) ? 1 : 0;
      asm volatile(
          "{\n .reg .pred p, q;\n setp.ne.s32 q, %0, 0;\n bar.red.and.pred p, 2, %1, q;\n selp.s32 %0, 1, 0, p;\n}\n"
          : "+r"(go) : "n"(OZ_DRAIN_WARPS * 32) : "memory");
      if (!go) break;
      const int i = t.tm + quarter * 32 + lane;
      bool staged = false;
      if constexpr (Epi::kDf) {
        if (epi.df()) {
          staged = true;
          const int rl = quarter * 32 + lane, ea = (i < t.M) ? t.ea[i] : 0;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int jj = t.tn + half * 32 + j;
            stage_out[rl * OZ_EP_LD + half * 32 + j] =
                (i < t.M && jj < t.N) ? oz_df_of(hi[j], lo[j], ea + t.eb[jj]) : make_float2(0.f, 0.f);
          }
          asm volatile("bar.sync 1, %0;\n" ::"n"(OZ_DRAIN_WARPS * 32) : "memory");
          oz_epilogue_df(t, epi, stage_out, warp - 2, lane);
          asm volatile("bar.sync 1, %0;\n" ::"n"(OZ_DRAIN_WARPS * 32) : "memory");   // staging free again
        }
      }
      if (!staged && i < t.M) {
        const int ea = t.ea[i];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int jj = t.tn + half * 32 + j;
          if (jj < t.N) epi(i, jj, hi[j], lo[j], ea + t.eb[jj]);
        }
      }
    }
  }
  __syncthreads();
  if (*abort) {
    // let the copies and MMAs in flight finish before the memory is released (bounded)
    if (tid == 0)
      for (int q = consumed; q < issued; ++q) mbar_drain(smem_u32(&bar_full[q % OZ_STAGES]), (q / OZ_STAGES) & 1);
    if (tid == 32) {                           // the MMA-issuing thread: its commit covers all its MMAs
      tc_commit(smem_u32(&bar_fin));
      mbar_drain(smem_u32(&bar_fin), 0);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  __syncwarp();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tbase));
}

struct OzFetchTasks {                             // one task per tile (float64 output)
  using Epi = OzEpiF64;
  const OzTask* tasks;
  __device__ __forceinline__ void operator()(int b, OzTile& t, OzEpiF64& epi) const {
    const OzTask& q = tasks[b];
    t = OzTile{q.ia, q.ib, q.ea, q.eb, q.M, q.N, q.Kp, q.tm, q.tn};
    epi = OzEpiF64{q.C, q.ldc};
  }
};

// Grouped launch: tile b belongs to the group with the largest first <= b; within
// the group row tiles come in order, and in a lower group row tile r has
// min(CT, 2 r + 2) column tiles (those meeting j <= i).
struct OzFetchGroups {
  using Epi = OzEpi;
  const OzGroup* groups;
  int ngroups;
  __device__ __forceinline__ void operator()(int b, OzTile& t, OzEpi& epi) const {
    int lo = 0, hi = ngroups - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (groups[mid].first <= b) lo = mid; else hi = mid - 1;
    }
    const OzGroup& G = groups[lo];
    int id = b - G.first;
    const int RT = (G.M + OZ_TILE_M - 1) / OZ_TILE_M, CT = (G.N + OZ_TILE_N - 1) / OZ_TILE_N;
    int r = 0;
    for (; r < RT; ++r) {
      const int cnt = G.lower ? min(CT, 2 * r + 2) : CT;
      if (id < cnt) break;
      id -= cnt;
    }
    t = OzTile{G.ia, G.ib, G.ea, G.eb, G.M, G.N, G.Kp, r * OZ_TILE_M, id * OZ_TILE_N};
    epi = OzEpi{G.C, G.ldc, G.mode, G.lower};
  }
};

__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_tc_kernel(const OzTask* __restrict__ tasks, int ntiles, const OzMap* __restrict__ maps,
                      int* __restrict__ err) {
  oz_tiles_run(OzFetchTasks{tasks}, ntiles, maps, err);
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_grp_kernel(const OzGroup* __restrict__ groups, int ngroups, int ntiles, const OzMap* __restrict__ maps,
                       int* __restrict__ err) {
  oz_tiles_run(OzFetchGroups{groups, ngroups}, ntiles, maps, err);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

int oz_slices() { return OZ_Q; }

// blocks of the persistent tile kernels: one per SM (each holds the SM's whole tensor memory)
static int oz_resident_blocks() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    n = sms > 0 ? sms : 1;
  }
  return n;
}
int oz_kpad(int K) { return (K + 31) / 32 * 32; }

cudaError_t oz_encode_maps(const std::vector<OzSplitTask>& ops, std::vector<OzMap>& maps) {
  static_assert(sizeof(OzMap) == sizeof(CUtensorMap), "tensor map size");
  maps.assign(2 * ops.size(), OzMap{});
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  for (size_t o = 0; o < ops.size(); ++o) {
    const OzSplitTask& t = ops[o];
    if (t.M < 0 || t.Kp < 0 || t.Kp % 32 != 0 || t.Mp != oz_mpad(t.M) || (reinterpret_cast<uintptr_t>(t.out) & 15))
      return cudaErrorInvalidValue;
    // dims innermost first: (row % 32, k % 8) as 256 contiguous elements, row / 32, k / 8,
    // slice; byte strides of dims 1..3.  An empty operand (no rows or no k) gets a
    // one-element extent: no tile reads it (K = 0 runs no k step).
    const cuuint64_t G32 = (cuuint64_t)std::max(t.Mp / 32, 1), G8 = (cuuint64_t)std::max(t.Kp / 8, 1);
    const cuuint64_t dims[4] = {256, G32, G8, (cuuint64_t)OZ_Q};
    const cuuint64_t strides[3] = {512, G32 * 512, G32 * G8 * 512};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int role = 0; role < 2; ++role) {
      const cuuint32_t box[4] = {256, (cuuint32_t)((role == 0 ? OZ_TILE_M : OZ_TILE_N) / 32), 2, (cuuint32_t)OZ_Q};
      CUresult r = enc(reinterpret_cast<CUtensorMap*>(&maps[2 * o + role]), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                       const_cast<uint16_t*>(t.out), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_oz_split(const OzSplitTask* d_tasks, int ntasks, int maxM, int maxKp, cudaStream_t st) {
  if (ntasks == 0) return cudaSuccess;
  oz_scale_kernel<<<dim3((maxM + 31) / 32, ntasks), 256, 0, st>>>(d_tasks);
  oz_split_kernel<<<dim3((maxKp + 63) / 64, (maxM + 31) / 32, ntasks), 256, 0, st>>>(d_tasks);
  return cudaGetLastError();
}

cudaError_t launch_oz_gemm(const OzTask* d_tasks, int ntiles, const OzMap* d_maps, int* d_err, cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  if (reinterpret_cast<uintptr_t>(d_maps) & 63) return cudaErrorInvalidValue;   // tensor maps: 64-byte aligned
  static const cudaError_t lim = smem_limit_max(oz_gemm_tc_kernel);
  if (lim != cudaSuccess) return lim;
  oz_gemm_tc_kernel<<<std::min(ntiles, oz_resident_blocks()), OZ_THREADS, OZ_SMEM, st>>>(d_tasks, ntiles, d_maps, d_err);
  return cudaGetLastError();
}

cudaError_t launch_oz_gemm_groups(const OzGroup* d_groups, int ngroups, int ntiles, const OzMap* d_maps, int* d_err,
                                  cudaStream_t st) {
  if (ntiles == 0 || ngroups == 0) return cudaSuccess;
  if (reinterpret_cast<uintptr_t>(d_maps) & 63) return cudaErrorInvalidValue;   // tensor maps: 64-byte aligned
  static const cudaError_t lim = smem_limit_max(oz_gemm_grp_kernel);
  if (lim != cudaSuccess) return lim;
  oz_gemm_grp_kernel<<<std::min(ntiles, oz_resident_blocks()), OZ_THREADS, OZ_SMEM, st>>>(d_groups, ngroups, ntiles,
                                                                                          d_maps, d_err);
  return cudaGetLastError();
}
