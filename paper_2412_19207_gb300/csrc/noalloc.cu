// rann_dd_matvec_t_noalloc: the transposed block product z_j = B_j^T y(rows_j)
// for callers that cannot allocate device memory.
//
// Who cannot allocate: a host program that hands all device memory to one
// allocator of its own (a framework's caching pool, or a fixed arena reserved
// at start-up) gets failures from cudaMalloc once that arena holds the device,
// and a latency-critical loop cannot afford the device-wide synchronisation a
// cudaMalloc/cudaFree may imply.  This entry point therefore allocates
// nothing: the per-row-tile partial sums live in a file-scope device array of
// fixed size, and the block descriptors in a second one, filled by an
// asynchronous copy to that array's device address.  The caller passes every
// input and output.
//
// Limits and sharing: at most NA_MAX_BLOCKS blocks, and (number of 256-row
// tiles) x (largest n_cols) <= NA_MAX_SCRATCH doubles (8 MiB).  Every GPU
// that loads the library holds both arrays until the process exits.  All
// calls share them and they keep the last call's contents; every partial sum
// a call reads is written earlier by the same call, so nothing needs
// clearing.  Calls that overlap on the GPU (different streams, or concurrent
// host threads) race on the arrays.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int NA_MAX_BLOCKS = 4096;
constexpr int64_t NA_MAX_SCRATCH = (int64_t)1 << 20;   // doubles
constexpr int NA_ROWS = 256;
constexpr int NA_MAX_DEVICES = 64;

struct NaBlock {
  int64_t boff;     // offset of B_j in B_dev (doubles)
  int64_t row_off;  // offset of block j's row indices in rows_dev
  int64_t zoff;     // offset of z_j in z_dev
  int n_rows, n_cols, ld, tile0;
};

static __device__ __align__(256) double g_na_scratch[NA_MAX_SCRATCH];
static __device__ __align__(256) NaBlock g_na_blocks[NA_MAX_BLOCKS];

__global__ void na_partial_kernel(const NaBlock* __restrict__ blocks, int J, const double* __restrict__ B,
                                  const int64_t* __restrict__ rows, const double* __restrict__ y,
                                  double* __restrict__ scratch, int maxcols) {
  // block of this tile: last j with tile0 <= blockIdx.x
  int lo = 0, hi = J - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (blocks[mid].tile0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const NaBlock b = blocks[lo];
  const int r0 = ((int)blockIdx.x - b.tile0) * NA_ROWS;
  const int nr = min(NA_ROWS, b.n_rows - r0);
  __shared__ double yl[NA_ROWS];
  for (int t = threadIdx.x; t < nr; t += blockDim.x) yl[t] = y[rows[b.row_off + r0 + t]];
  __syncthreads();
  for (int c = threadIdx.x; c < b.n_cols; c += blockDim.x) {
    const double* col = B + b.boff + (int64_t)r0 * b.ld + c;
    double acc = 0.0;
    for (int t = 0; t < nr; ++t) acc = fma(col[(int64_t)t * b.ld], yl[t], acc);
    scratch[(int64_t)blockIdx.x * maxcols + c] = acc;
  }
}

__global__ void na_final_kernel(const NaBlock* __restrict__ blocks, const double* __restrict__ scratch,
                                int maxcols, double* __restrict__ z) {
  const NaBlock b = blocks[blockIdx.x];
  const int ntiles = (b.n_rows + NA_ROWS - 1) / NA_ROWS;
  for (int c = threadIdx.x; c < b.n_cols; c += blockDim.x) {
    double acc = 0.0;
    for (int t = 0; t < ntiles; ++t) acc += scratch[(int64_t)(b.tile0 + t) * maxcols + c];
    z[b.zoff + c] = acc;
  }
}

std::mutex g_na_mutex;
double* g_na_scratch_ptr[NA_MAX_DEVICES] = {};
NaBlock* g_na_blocks_ptr[NA_MAX_DEVICES] = {};
NaBlock g_na_host[NA_MAX_BLOCKS];   // host staging for the descriptor copy (under g_na_mutex)

}  // namespace

extern "C" rann_status rann_dd_matvec_t_noalloc(int J, const int64_t* boff, const int* n_rows, const int* n_cols,
                                                const int* ld, const int64_t* row_off, const int64_t* zoff,
                                                const double* B_dev, const int64_t* rows_dev, const double* y_dev,
                                                double* z_dev, void* stream) {
  if (J < 1 || J > NA_MAX_BLOCKS) {
    rann_set_error("matvec_t_noalloc: J = %d outside 1..%d", J, NA_MAX_BLOCKS);
    return RANN_EINVAL;
  }
  if (!boff || !n_rows || !n_cols || !ld || !row_off || !zoff || !B_dev || !rows_dev || !y_dev || !z_dev) {
    rann_set_error("matvec_t_noalloc: null argument");
    return RANN_EINVAL;
  }
  int64_t tiles = 0;
  int maxcols = 1;
  for (int j = 0; j < J; ++j) {
    if (n_rows[j] < 0 || n_cols[j] < 0 || ld[j] < n_cols[j] || boff[j] < 0 || row_off[j] < 0 || zoff[j] < 0) {
      rann_set_error("matvec_t_noalloc: bad descriptor for block %d", j);
      return RANN_EINVAL;
    }
    tiles += ((int64_t)n_rows[j] + NA_ROWS - 1) / NA_ROWS;   // 64-bit: no wrap for n_rows near INT_MAX
    maxcols = std::max(maxcols, n_cols[j]);
  }
  if (tiles * maxcols > NA_MAX_SCRATCH) {   // also bounds every tile index below by 2^20
    rann_set_error("matvec_t_noalloc: %lld row tiles x %d columns exceed the %lld-double scratch array",
                   (long long)tiles, maxcols, (long long)NA_MAX_SCRATCH);
    return RANN_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    rann_set_error("matvec_t_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    return RANN_ECUDA;
  }
  double* scratch;
  NaBlock* blocks;
  cudaStream_t st = (cudaStream_t)stream;
  {
    // once per device, with that device current: the device addresses of the
    // two arrays (in host code their names are host-side stand-ins)
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_scratch_ptr[dev]) {
      void* ps = nullptr;
      void* pb = nullptr;
      e = cudaGetSymbolAddress(&ps, g_na_scratch);
      if (e == cudaSuccess) e = cudaGetSymbolAddress(&pb, g_na_blocks);
      if (e != cudaSuccess) {
        rann_set_error("matvec_t_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return RANN_ECUDA;
      }
      g_na_scratch_ptr[dev] = (double*)ps;
      g_na_blocks_ptr[dev] = (NaBlock*)pb;
    }
    scratch = g_na_scratch_ptr[dev];
    blocks = g_na_blocks_ptr[dev];
    int t0 = 0;
    for (int j = 0; j < J; ++j) {
      g_na_host[j] = {boff[j], row_off[j], zoff[j], n_rows[j], n_cols[j], ld[j], t0};
      t0 += (n_rows[j] + NA_ROWS - 1) / NA_ROWS;
    }
    // from pageable memory: returns once the table is staged, so the host array may be reused
    e = cudaMemcpyAsync(blocks, g_na_host, sizeof(NaBlock) * J, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess && tiles > 0) {
    na_partial_kernel<<<(unsigned)tiles, 256, 0, st>>>(blocks, J, B_dev, rows_dev, y_dev, scratch, maxcols);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    na_final_kernel<<<J, 256, 0, st>>>(blocks, scratch, maxcols, z_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    rann_set_error("matvec_t_noalloc: %s", cudaGetErrorString(e));
    return RANN_ECUDA;
  }
  return RANN_OK;
}
