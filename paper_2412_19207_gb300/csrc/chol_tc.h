// Host plan of the big-panel double-float Cholesky with tensor-core updates
// (chol_tc.cu).
#pragma once
#include <vector>

#include "common.cuh"

constexpr int TC_NB = 256;          // panel width: one exact 256-long chunk of the digit-slice products
constexpr int TC_MIN_N = 512;       // local matrices from this size on take the big-panel path

struct CholTcPlan {
  struct Step {
    int c0, c1;
    int sp_l21, n_l21, maxM_l21;    // split tasks of L21 (handle's stream)
    int sp_inv, n_inv, maxM_inv, maxKp_inv;   // X_II and R_I
    int sp_xi, n_xi, maxM_xi;       // X_{I,<c1}
    int g_trail, ng_trail, tiles_trail;       // A22 -= L21 L21^T
    int g_ii, ng_ii, tiles_ii;                // X_{I,<c0} = X_II R_I
    int g_iii, ng_iii, tiles_iii;             // R_{I'} -= L21 X_{I,<c1}
  };
  std::vector<Step> steps;
  std::vector<OzSplitTask> split;
  std::vector<OzGroup> groups;
  std::vector<OzMap> maps;
  int maxn = 0;
  int64_t l21_elems = 0, inv_elems = 0, xi_elems = 0;   // bf16 elements of one slice region
  int64_t e_ints = 0;
  double flops = 0.0;               // flops of the digit-slice products
};

cudaError_t chol_tc_build(const std::vector<CholMat>& mats, CholTcPlan& P, uint16_t* const l21_buf[2],
                          uint16_t* inv_buf, uint16_t* xi_buf, int* e_buf);
cudaError_t chol_tc_enqueue(const CholTcPlan& P, const CholMat* d_mats, int nmat, int* d_fail, const double* d_dmax,
                            const OzSplitTask* d_split, const OzGroup* d_groups, const OzMap* d_maps, int* d_err,
                            cudaStream_t st, cudaStream_t st2, int* nlaunch);
