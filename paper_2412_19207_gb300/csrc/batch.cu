// Batches of problem instances (the many independent problems of the weak-
// scaling runs, Sec. 5, Table 2): a pool of host worker threads, each with
// its own CUDA stream, takes instances largest first and runs each through
// the whole path -- assembly, F, PCA, Schwarz set-up, the preconditioned
// solve and optionally the gradient of the grid misfit -- with the handle
// moved onto the worker's stream, so the kernels of different instances, of
// any grid size, overlap on the device while each worker drives its
// instance's host-side control.  The Schwarz apply configuration is tuned
// once per size class and reused by the class's other instances.
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "common.cuh"

namespace {

constexpr int MF_BLOCKS = 64;

// r = 2 (u - u_obs) and per-block sums of (u - u_obs)^2 (fixed order)
__global__ void __launch_bounds__(256) misfit_kernel(const double* __restrict__ u, const double* __restrict__ uo,
                                                     int64_t n, double* __restrict__ r, double* __restrict__ part) {
  __shared__ double sm[256];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const double d = u[i] - uo[i];
    r[i] = 2.0 * d;
    acc = fma(d, d, acc);
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

struct Tuning {                       // size class -> apply configuration, shared by the workers
  std::mutex mu;
  std::condition_variable cv;
  std::map<std::pair<int, int>, int> done;
  std::set<std::pair<int, int>> busy;
};

// device scratch of one instance, on the worker's stream
struct Scratch {
  cudaStream_t st;
  std::vector<void*> ptrs;
  double* get(size_t n) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, sizeof(double) * std::max<size_t>(n, 1), st) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<double*>(p);
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
  }
};

#define STEP(x)                         \
  do {                                  \
    const rann_status _s = (x);         \
    if (_s != RANN_OK) return _s;       \
  } while (0)

rann_status run_one(rann_dd_handle* h, cudaStream_t st, const rann_dd_pipeline& c, double* F, double* W,
                    const double* uo, double* gF, double* gc, rann_dd_pipeline_out& out, Tuning& tu) {
  int64_t np = 0, dof = 0;
  int J = 0, m = 0;
  STEP(rann_dd_sizes(h, &np, nullptr, &J, &m, nullptr));
  STEP(rann_dd_assemble(h));
  STEP(rann_dd_rhs(h, F));
  std::vector<int> ranks((size_t)J);
  STEP(rann_dd_pca(h, c.pca_mode, c.pca_thr, ranks.data()));
  const rann_status ss = rann_dd_setup_precond(h, c.prec_kind, 1);
  if (ss != RANN_OK && ss != RANN_LOCAL_SINGULAR) return ss;
  STEP(rann_dd_sizes(h, nullptr, nullptr, nullptr, nullptr, &dof));
  out.dof = dof;
  if (c.autotune) {
    const std::pair<int, int> key{J, (rann_handle_maxn(h) + 63) / 64};
    std::unique_lock<std::mutex> lk(tu.mu);
    tu.cv.wait(lk, [&] { return tu.done.count(key) || !tu.busy.count(key); });
    auto it = tu.done.find(key);
    if (it != tu.done.end()) {
      const int cfg = it->second;
      lk.unlock();
      STEP(rann_dd_set_apply_config(h, cfg));
    } else {
      tu.busy.insert(key);
      lk.unlock();
      int best = 0;
      const rann_status ts = rann_dd_tune_apply(h, 5, &best, nullptr);
      if (ts != RANN_OK) rann_dd_get_apply_config(h, &best);
      lk.lock();
      tu.done[key] = best;
      tu.busy.erase(key);
      lk.unlock();
      tu.cv.notify_all();
      STEP(ts);
    }
  }
  rann_dd_get_apply_config(h, &out.apply_config);
  rann_status fs = c.solver == 0 ? rann_dd_solve_cg_as(h, F, W, c.rtol, c.maxit, &out.forward)
                                 : rann_dd_solve_gmres_ras(h, F, W, c.rtol, c.restart, c.maxit, &out.forward);
  if (fs != RANN_OK && fs != RANN_NOT_CONVERGED) return fs;
  if (!c.backward) return fs;
  // misfit gradient: dl/dW = 2 E^T (u_hat - u_obs), lam = (H^T H)^{-1} dl/dW, dl/dF = H lam
  Scratch sc{st, {}};
  double* xyz = sc.get((size_t)np * rann_handle_dim(h));
  double* u = sc.get((size_t)np);
  double* r = sc.get((size_t)np);
  double* part = sc.get(MF_BLOCKS);
  double* gW = sc.get((size_t)dof);
  double* lam = sc.get((size_t)dof);
  if (!xyz || !u || !r || !part || !gW || !lam) {
    rann_set_error("batch: scratch allocation failed");
    return RANN_ENOMEM;
  }
  STEP(rann_dd_points(h, xyz));
  STEP(rann_dd_eval(h, W, xyz, np, u));
  misfit_kernel<<<MF_BLOCKS, 256, 0, st>>>(u, uo, np, r, part);
  if (cudaGetLastError() != cudaSuccess) {
    rann_set_error("batch: misfit kernel launch failed");
    return RANN_ECUDA;
  }
  double hp[MF_BLOCKS];
  if (cudaMemcpyAsync(hp, part, sizeof(hp), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    rann_set_error("batch: misfit read-back failed");
    return RANN_ECUDA;
  }
  double loss = 0.0;
  for (int b = 0; b < MF_BLOCKS; ++b) loss += hp[b];
  out.loss = loss;
  STEP(rann_dd_eval_grid_t(h, r, gW));
  const rann_status bs = rann_dd_solve_backward(h, gW, lam, c.rtol, c.maxit, &out.adjoint);
  if (bs != RANN_OK && bs != RANN_NOT_CONVERGED) return bs;
  if (gF) STEP(rann_dd_matvec(h, lam, gF));
  if (gc && rann_handle_piecewise(h)) STEP(rann_dd_grad_coef(h, F, W, lam, gc));
  return fs != RANN_OK ? fs : bs;
}

}  // namespace

struct rann_dd_batch {
  int dev = 0;
  std::vector<cudaStream_t> streams;
};

extern "C" rann_status rann_dd_batch_create(int nworkers, rann_dd_batch** out) {
  if (!out || nworkers < 1 || nworkers > 64) {
    rann_set_error("rann_dd_batch_create: nworkers must be in 1..64");
    return RANN_EINVAL;
  }
  *out = nullptr;
  rann_dd_batch* b = new rann_dd_batch();
  cudaGetDevice(&b->dev);
  for (int w = 0; w < nworkers; ++w) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t t : b->streams) cudaStreamDestroy(t);
      delete b;
      rann_set_error("rann_dd_batch_create: stream creation failed");
      return RANN_ECUDA;
    }
    b->streams.push_back(s);
  }
  *out = b;
  return RANN_OK;
}

extern "C" void rann_dd_batch_destroy(rann_dd_batch* b) {
  if (!b) return;
  for (cudaStream_t s : b->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  delete b;
}

extern "C" rann_status rann_dd_batch_run(rann_dd_batch* b, int n, rann_dd_handle* const* hs,
                                         const rann_dd_pipeline* cfg, double* const* F_dev, double* const* W_dev,
                                         const double* const* u_obs_dev, double* const* grad_F_dev,
                                         double* const* grad_coef_host, rann_dd_pipeline_out* out) {
  if (!b || n < 0 || (n > 0 && (!hs || !cfg || !F_dev || !W_dev || !out))) {
    rann_set_error("rann_dd_batch_run: null argument");
    return RANN_EINVAL;
  }
  if (n == 0) return RANN_OK;
  if (cfg->backward && !u_obs_dev) {
    rann_set_error("rann_dd_batch_run: backward needs u_obs");
    return RANN_EINVAL;
  }
  for (int k = 0; k < n; ++k) {
    if (!hs[k] || !F_dev[k] || !W_dev[k] || (cfg->backward && !u_obs_dev[k])) {
      rann_set_error("rann_dd_batch_run: instance %d has a null handle or buffer", k);
      return RANN_EINVAL;
    }
    for (int l = 0; l < k; ++l)
      if (hs[l] == hs[k]) {
        rann_set_error("rann_dd_batch_run: instance %d repeats the handle of instance %d", k, l);
        return RANN_EINVAL;
      }
  }
  // largest first (points x neurons)
  std::vector<int> order(n);
  std::vector<int64_t> size(n, 0);
  for (int k = 0; k < n; ++k) {
    int64_t np = 0;
    int m = 0;
    rann_dd_sizes(hs[k], &np, nullptr, nullptr, &m, nullptr);
    size[k] = np * m;
    order[k] = k;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return size[a] > size[c]; });
  std::vector<rann_status> st(n, RANN_OK);
  std::vector<std::string> msg(n);
  std::atomic<int> next{0};
  Tuning tu;
  const int nw = std::min<int>((int)b->streams.size(), n);
  auto worker = [&](int w) {
    cudaSetDevice(b->dev);
    const cudaStream_t s = b->streams[w];
    for (int i; (i = next.fetch_add(1)) < n;) {
      const int k = order[i];
      rann_dd_handle* h = hs[k];
      out[k] = rann_dd_pipeline_out{};
      const cudaStream_t keep = rann_handle_stream(h);
      rann_status r = rann_dd_set_stream(h, s);
      if (r == RANN_OK)
        r = run_one(h, s, *cfg, F_dev[k], W_dev[k], cfg->backward ? u_obs_dev[k] : nullptr,
                    grad_F_dev ? grad_F_dev[k] : nullptr, grad_coef_host ? grad_coef_host[k] : nullptr, out[k], tu);
      if (r != RANN_OK && r != RANN_NOT_CONVERGED) msg[k] = rann_dd_last_error();
      const rann_status back = rann_dd_set_stream(h, keep);
      if (r == RANN_OK || r == RANN_NOT_CONVERGED) {
        if (back != RANN_OK) { r = back; msg[k] = rann_dd_last_error(); }
      }
      out[k].status = r;
      st[k] = r;
    }
  };
  std::vector<std::thread> pool;
  for (int w = 0; w < nw; ++w) pool.emplace_back(worker, w);
  for (std::thread& t : pool) t.join();
  for (int k = 0; k < n; ++k)
    if (st[k] != RANN_OK && st[k] != RANN_NOT_CONVERGED) {
      rann_set_error("instance %d: %s", k, msg[k].c_str());
      return st[k];
    }
  return RANN_OK;
}
