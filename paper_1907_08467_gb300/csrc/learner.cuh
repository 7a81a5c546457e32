// Learner-side targets over a rollout kept on the device (paper Appendix,
// "A2C": the bootstrapped N-step return of the policy and value costs;
// "V-trace": the off-policy target with truncated importance weights, in
// the recursive form the paper implements, and the actor's advantage).
//
// Layout: the rollout's per-step rewards, dones and behaviour probabilities
// live in a ring of `depth` slots of n envs each (time-major, as the rollout
// loop writes them); step t of the T steps is slot (start + t) mod depth.
// Values V(s_t) ([T + 1][n], row T the bootstrap value) and target
// probabilities pi ([T][n]) come from the learner; outputs are [T][n].
//
// One thread per env walks its T steps from the last back to the first, so
// every load and store of a step is one coalesced row of the time-major
// arrays.  fp32 throughout, each operation rounded once (no contraction into
// fused multiply-adds), in this order per step t (g = gamma, or 0 after a
// done):
//   N-step:   R_t = r_t + g R_{t+1},  R_T = V(s_T)
//   V-trace:  ratio = pi_t / mu_t,  rho = min(rho_bar, ratio),  c = min(c_bar, ratio)
//             delta = rho ((r_t + g V_{t+1}) - V_t)
//             v_t   = (V_t + delta) + (g c)(v_{t+1} - V_{t+1}),  v_T = V(s_T)
//             A_t   = rho ((r_t + g v_{t+1}) - V_t)
#pragma once
#include <cstdint>

namespace atari {

__global__ void __launch_bounds__(256) k_nstep_returns(const float *rew, const uint8_t *done, int depth, int start,
                                                      const float *values, int T, int n, float gamma, float *ret) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float R = values[(size_t)T * n + i];
  for (int t = T - 1; t >= 0; --t) {
    const size_t s = (size_t)((start + t) % depth) * n + i;
    const float g = done[s] ? 0.0f : gamma;
    R = __fadd_rn(rew[s], __fmul_rn(g, R));
    ret[(size_t)t * n + i] = R;
  }
}

__global__ void __launch_bounds__(256) k_vtrace(const float *rew, const uint8_t *done, const float *mu, int depth,
                                               int start, const float *values, const float *pi, int T, int n,
                                               float gamma, float rho_bar, float c_bar, float *vs, float *adv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v_next = values[(size_t)T * n + i];  // v_T = V(s_T)
  float V_next = v_next;
  for (int t = T - 1; t >= 0; --t) {
    const size_t s = (size_t)((start + t) % depth) * n + i;
    const size_t o = (size_t)t * n + i;
    const float r = rew[s];
    const float g = done[s] ? 0.0f : gamma;
    const float ratio = __fdiv_rn(pi[o], mu[s]);
    // a NaN ratio (0 / 0) takes the truncation level, as min(level, NaN) does below
    const float rho = ratio < rho_bar ? ratio : rho_bar;
    const float c = ratio < c_bar ? ratio : c_bar;
    const float V = values[o];
    const float delta = __fmul_rn(rho, __fsub_rn(__fadd_rn(r, __fmul_rn(g, V_next)), V));
    const float v = __fadd_rn(__fadd_rn(V, delta), __fmul_rn(__fmul_rn(g, c), __fsub_rn(v_next, V_next)));
    adv[o] = __fmul_rn(rho, __fsub_rn(__fadd_rn(r, __fmul_rn(g, v_next)), V));
    vs[o] = v;
    v_next = v;
    V_next = V;
  }
}

}  // namespace atari
