// Device-side control of the shrink (Sec. 5.1.1 rank policy and the Lanczos convergence test) for
// the per-iteration graph: after every Lanczos cycle one thread applies the test the host would
// apply to the Ritz values and residual estimates, records the outcome, and sets the condition of
// the graph's `while` node (repeat the thick-restarted cycle while neither converged nor grown nor
// out of budget).  On convergence it also writes the rank r_k = #{theta_i > tau} and the scale
// theta_i - tau of the Ritz-vector kernels and the fused update, which read them from device
// memory, so the whole SVT iteration runs without the host.
#include "common.cuh"
#include "internal.h"

namespace svt {

__global__ void k_cycle_decide(const LoopParams* __restrict__ prm, LoopState* __restrict__ st,
                               const double* __restrict__ theta, const double* __restrict__ res, int K,
                               double* __restrict__ scale, cudaGraphConditionalHandle cond, int set_cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int cyc = st->cycles;
  const double tol = prm->tol;
  // stagnation: a cluster the working precision cannot separate further keeps its residuals above
  // tol; after 10 cycles of one pass the tolerance is relaxed 30x, after 25 cycles 300x
  const double tol_c = cyc >= 25 ? 300.0 * tol : (cyc >= 10 ? 30.0 * tol : tol);
  const double tau = prm->tau;
  const int s_eff = min(prm->s, K);
  int status;
  int conv = 0;
  if (!isfinite(theta[0]) || !isfinite(res[0])) {
    status = kLoopNumeric;
  } else {
    // Ritz values are lower bounds of the singular values: theta_s > tau proves sigma_s > tau
    const bool grow = !prm->strict && theta[s_eff - 1] > tau && prm->s < prm->kmin;
    bool all_conv = !grow;
    for (int i = 0; i < s_eff && all_conv; ++i) {
      const bool above = prm->strict || theta[i] > tau;
      const bool ok = res[i] <= tol_c * theta[0] ||
                      (!above && res[i] <= 1e-3 * theta[0] && theta[i] + res[i] <= tau);
      if (!ok) all_conv = false;
      else ++conv;
      if (!above) break;
    }
    if (all_conv) status = kLoopConverged;
    else if (grow) status = kLoopGrow;
    else if (cyc + 1 >= prm->max_cycles) status = kLoopBudget;
    else status = kLoopContinue;
  }
  int r = 0;
  if (status == kLoopConverged) {
    while (r < s_eff && theta[r] > tau) ++r;
    for (int i = 0; i < r; ++i) scale[i] = theta[i] - tau;
  }
  st->status = status;
  st->cycles = cyc + 1;
  st->conv = conv;
  st->s_eff = s_eff;
  st->r = r;
  st->relaxed = (status == kLoopConverged && cyc >= 10) ? 1 : 0;
  st->res_fail = (isfinite(theta[0]) && theta[0] > 0.0) ? res[min(conv, s_eff - 1)] / theta[0] : 0.0;
  if (set_cond) cudaGraphSetConditional(cond, status == kLoopContinue ? 1u : 0u);
}

int launch_cycle_decide(const LoopParams* prm, LoopState* st, const double* theta, const double* res, int K,
                        double* scale, cudaGraphConditionalHandle cond, int set_cond, cudaStream_t s) {
  k_cycle_decide<<<1, 32, 0, s>>>(prm, st, theta, res, K, scale, cond, set_cond);
  return 1;
}

}  // namespace svt
