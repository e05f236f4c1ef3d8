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
//     256-long k chunk is an integer below 2^24 (group 9 peaks at
//     256 * 40960 < 2^24); at the end of a chunk the eight group sums are
//     joined exactly in two 46-bit integers, hi = sum_{s<=5} c_s 128^{5-s} and
//     lo = sum_{s>=6} c_s 128^{9-s}, which enter the float64 accumulator as
//     hi 2^-35 + lo 2^-63 (two roundings per chunk).
// The error is a few units of 2^-53 K max_k|a_ik| max_k|b_jk|, the float64
// bound.  The scheme is that of Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59 (2012).
#include "common.cuh"

namespace {

constexpr int OZ_Q = 8;            // digit slices per operand
constexpr int OZ_SMAX = 9;         // largest weight group q + r kept
constexpr int OZ_NG = OZ_SMAX - 1; // weight groups s = 2..9
constexpr int OZ_CHUNK = 256;      // k span of one exact float32 accumulation
constexpr int OZ_TM = 64, OZ_TN = 64, OZ_TK = 32;
constexpr int OZ_THREADS = 512;    // 16 warps, each a 16 x 16 sub-tile
constexpr int OZ_LDW = OZ_TK / 2 + 4;   // shared row length in 32-bit words (2 bf16 each; padded)
constexpr int OZ_ROWS = 2 * OZ_Q * OZ_TM;           // staged rows: A_1..A_8 then B_1..B_8
constexpr int OZ_STAGE_WORDS = OZ_ROWS * OZ_LDW;    // one k step (80 KB)
static_assert(OZ_CHUNK % OZ_TK == 0, "chunk must be a multiple of the k step");
static_assert(OZ_TM == OZ_TN, "A and B tiles share the staging layout");

__device__ __forceinline__ uint16_t bf16_of_small_int(int d) {
  // |d| <= 128: exactly representable in bf16 (8 significant bits); the bf16
  // pattern is the upper half of the float32 pattern.
  return (uint16_t)(__float_as_uint((float)d) >> 16);
}

// e_i of 32 rows of one operand per block (deterministic integer max of |x|'s bits).
__global__ void __launch_bounds__(256) oz_scale_kernel(const OzSplitTask* __restrict__ tasks) {
  const OzSplitTask t = tasks[blockIdx.y];
  const int i0 = blockIdx.x * 32;
  if (i0 >= t.M) return;
  __shared__ long long red[8][33];
  const int a = threadIdx.x & 31, b = threadIdx.x >> 5;
  const long long* X = reinterpret_cast<const long long*>(t.X);
  const long long ABS = 0x7FFFFFFFFFFFFFFFll;
  if (t.sk == 1 && !t.gather) {   // rows contiguous in k: warp b owns rows i0 + b + 8c, lanes stride k
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + b + 8 * c;
      long long mx = 0;
      if (i < t.M)
        for (int k = a; k < t.K; k += 32) mx = max(mx, X[(int64_t)i * t.si + k] & ABS);
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (a == 0) red[0][b + 8 * c] = mx;
    }
  } else {              // rows contiguous in i: lane a owns row i0 + a, warps stride k
    const int i = i0 + a;
    long long mx = 0;
    if (i < t.M)
      for (int k = b; k < t.K; k += 8) {
        const int64_t kk = t.gather ? t.gather[k] : k;
        mx = max(mx, X[(int64_t)i * t.si + kk * t.sk] & ABS);
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

// Digit slices of a 32 x 32 tile: slice q of row i at out[q * M * Kp + i * Kp + k],
// zero for k >= K (padding up to Kp).
__global__ void __launch_bounds__(256) oz_split_kernel(const OzSplitTask* __restrict__ tasks) {
  const OzSplitTask t = tasks[blockIdx.z];
  const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  if (i0 >= t.M || k0 >= t.Kp) return;
  __shared__ long long tile[32][33];
  const long long* X = reinterpret_cast<const long long*>(t.X);
  const bool kfast = (t.sk == 1 && !t.gather);
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int a = e & 31, b = e >> 5;
    const int ii = kfast ? b : a, kk = kfast ? a : b;
    const int i = i0 + ii, k = k0 + kk;
    long long v = 0;
    if (i < t.M && k < t.K) v = X[(int64_t)i * t.si + (int64_t)(t.gather ? t.gather[k] : k) * t.sk];
    tile[ii][kk] = v;
  }
  __syncthreads();
  const int64_t slice = (int64_t)t.M * t.Kp;
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int kk = e & 31, ii = e >> 5;
    const int i = i0 + ii, k = k0 + kk;
    if (i >= t.M) continue;
    // X = round(|x| 2^{56 - e_i}) with the sign of x, from the float64 fields
    const long long bits = tile[ii][kk];
    const int E = (int)((bits >> 52) & 0x7ff);
    long long v = 0;
    if (E != 0) {                                    // zero and subnormals give 0
      const long long mant = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
      const int sh = E - 1075 + 56 - t.e[i];         // <= 4 since |x| <= 2^{e_i}
      if (sh >= 0) v = mant << sh;
      else if (sh > -60) v = (mant + (1ll << (-sh - 1))) >> (-sh);
      if (bits < 0) v = -v;
    }
    uint16_t* o = t.out + (int64_t)i * t.Kp + k;
#pragma unroll
    for (int q = OZ_Q - 1; q >= 1; --q) {            // balanced base-128 digits, least significant first
      const long long d = ((v + 64) & 127) - 64;
      v = (v - d) >> 7;                              // exact: v - d is a multiple of 128
      o[q * slice] = bf16_of_small_int((int)d);
    }
    o[0] = bf16_of_small_int((int)v);                // leading digit, |v| <= 128
  }
}

__device__ __forceinline__ void mma_bf16_16816(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* gptr, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gptr), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Stage the 16 digit-slice tiles (A_1..A_8 rows tm.., B_1..B_8 rows tn..) of
// the k step starting at k0: 16 x 64 rows x 64 bytes, 16-byte copies; rows
// past M (N) are zero-filled.
__device__ __forceinline__ void oz_stage(const OzTask& t, uint32_t sbase, int k0) {
  const int kw = t.Kp >> 1;
  const uint32_t* gA = reinterpret_cast<const uint32_t*>(t.A);
  const uint32_t* gB = reinterpret_cast<const uint32_t*>(t.B);
  for (int c = threadIdx.x; c < OZ_ROWS * 4; c += OZ_THREADS) {
    const int srow = c >> 2, part = c & 3;
    const int sl = srow / OZ_TM, row = srow % OZ_TM;
    const bool isA = sl < OZ_Q;
    const int q = isA ? sl : sl - OZ_Q;
    const int gi = (isA ? t.tm : t.tn) + row, lim = isA ? t.M : t.N;
    const uint32_t* base = isA ? gA : gB;
    const int64_t slice = (int64_t)lim * kw;
    const bool ok = gi < lim;
    const uint32_t* src = base + (ok ? q * slice + (int64_t)gi * kw + (k0 >> 1) + part * 4 : 0);
    cp_async16(sbase + (uint32_t)((srow * OZ_LDW + part * 4) * 4), src, ok ? 16 : 0);
  }
}

// One 64 x 64 tile of C = A B^T from the digit slices: 16 warps of 16 x 16
// (1 x 2 mma tiles of 16 x 8), eight float32 accumulator sets (one per
// weight group), k steps double-buffered through cp.async.
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(const OzTask* __restrict__ tasks) {
  extern __shared__ __align__(16) uint32_t oz_smem[];
  const OzTask t = tasks[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 2) * 16, wn = (warp & 3) * 16;
  const int g = lane >> 2, tq = lane & 3;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(oz_smem);
  float acc[OZ_NG][2][4];
  double acc64[2][4];
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc64[b][c] = 0.0;
#pragma unroll
      for (int s = 0; s < OZ_NG; ++s) acc[s][b][c] = 0.f;
    }
  const int nks = t.Kp / OZ_TK;
  oz_stage(t, sbase, 0);
  cp_async_commit();
  for (int ks = 0; ks < nks; ++ks) {
    if (ks + 1 < nks) {
      oz_stage(t, sbase + (uint32_t)(((ks + 1) & 1) * OZ_STAGE_WORDS * 4), (ks + 1) * OZ_TK);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const uint32_t* S = oz_smem + (ks & 1) * OZ_STAGE_WORDS;
#pragma unroll
    for (int kk = 0; kk < OZ_TK / 2; kk += 8) {      // two k16 mma steps (8 words each)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        uint32_t bf[OZ_Q][2];
        const int cn = wn + nt * 8 + g;
#pragma unroll
        for (int r = 0; r < OZ_Q; ++r) {
          const uint32_t* Br = S + ((OZ_Q + r) * OZ_TM + cn) * OZ_LDW + kk + tq;
          bf[r][0] = Br[0];
          bf[r][1] = Br[4];
        }
#pragma unroll
        for (int q = 0; q < OZ_Q; ++q) {
          uint32_t af[4];
          const uint32_t* Aq = S + (q * OZ_TM + wm + g) * OZ_LDW + kk + tq;
          af[0] = Aq[0];
          af[1] = Aq[8 * OZ_LDW];
          af[2] = Aq[4];
          af[3] = Aq[8 * OZ_LDW + 4];
#pragma unroll
          for (int r = 0; r < OZ_Q; ++r)
            if (q + r + 2 <= OZ_SMAX) mma_bf16_16816(acc[q + r][nt], af, bf[r][0], bf[r][1]);
        }
      }
    }
    const int kend = (ks + 1) * OZ_TK;
    if (kend % OZ_CHUNK == 0 || ks + 1 == nks) {
      // the group sums are exact integers below 2^24: join them exactly in two
      // 46-bit integers and add to the float64 accumulator
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          long long hi = 0, lo = 0;
#pragma unroll
          for (int s = 0; s < 4; ++s) hi = hi * 128 + __float2int_rn(acc[s][b][c]);
#pragma unroll
          for (int s = 4; s < OZ_NG; ++s) lo = lo * 128 + __float2int_rn(acc[s][b][c]);
          acc64[b][c] = fma((double)hi, 0x1p-35, acc64[b][c]);
          acc64[b][c] = fma((double)lo, 0x1p-63, acc64[b][c]);
#pragma unroll
          for (int s = 0; s < OZ_NG; ++s) acc[s][b][c] = 0.f;
        }
    }
    __syncthreads();                                 // stage (ks & 1) is refilled next iteration
  }
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = t.tm + wm + g + (c >= 2 ? 8 : 0);
      const int j = t.tn + wn + nt * 8 + 2 * tq + (c & 1);
      if (i < t.M && j < t.N) t.C[(int64_t)i * t.ldc + j] = ldexp(acc64[nt][c], t.ea[i] + t.eb[j]);
    }
}

}  // namespace

int oz_slices() { return OZ_Q; }
int oz_kpad(int K) { return (K + OZ_TK - 1) / OZ_TK * OZ_TK; }

cudaError_t launch_oz_split(const OzSplitTask* d_tasks, int ntasks, int maxM, int maxKp, cudaStream_t st) {
  if (ntasks == 0) return cudaSuccess;
  oz_scale_kernel<<<dim3((maxM + 31) / 32, ntasks), 256, 0, st>>>(d_tasks);
  oz_split_kernel<<<dim3((maxKp + 31) / 32, (maxM + 31) / 32, ntasks), 256, 0, st>>>(d_tasks);
  return cudaGetLastError();
}

cudaError_t launch_oz_gemm(const OzTask* d_tasks, int ntiles, cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  const int smem = (int)(2 * OZ_STAGE_WORDS * sizeof(uint32_t));
  cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  oz_gemm_kernel<<<ntiles, OZ_THREADS, smem, st>>>(d_tasks);
  return cudaGetLastError();
}
