// Inference-path loop: a linear softmax policy over the 84x84x4 stack and a
// device rollout ring (paper Section 4: inference-only throughput, with the
// emulator and the network both on the GPU and no host copies).
//
// Policy: logits[j] = sum_k stack[k] * W[k][j], stack flattened as plane *
// 7056 + row * 84 + column, W bf16 [28224][18], fp32 accumulation in a fixed
// order so every run (and the oracle) gets the same bits: 441 chunks of 64
// sequential fused multiply-adds, chunk partials reduced by the pairwise
// tree s[i] += s[i + h], h = 256 .. 1, over 512 zero-padded slots.  Softmax
// weights exp(l_j - max l) by Cody-Waite reduction (ln 2 split into 355/512
// and a remainder) and a degree-7 Taylor polynomial; the action is the
// smallest j whose running sum of weights exceeds u * total, with u the
// 24-bit fraction of the env's Philox word (env key, step, 4 << 8, episode),
// or the last action of nonzero weight when rounding leaves none.
#pragma once
#include <cstdint>

#include "device_machine.cuh"

namespace atari {

constexpr int POLICY_K = 28224, POLICY_A = 18, POLICY_CHUNKS = 441;
constexpr uint32_t PURPOSE_POLICY = 4;

__device__ __forceinline__ float exp_cw(float x) {
  if (x < -87.0f) return 0.0f;
  const float kf = rintf(__fmul_rn(x, 1.44269504088896341f));
  float r = __fmaf_rn(-kf, 0.693359375f, x);
  r = __fmaf_rn(-kf, -2.12194440e-4f, r);
  float p = 1.0f / 5040.0f;
  p = __fmaf_rn(p, r, 1.0f / 720.0f);
  p = __fmaf_rn(p, r, 1.0f / 120.0f);
  p = __fmaf_rn(p, r, 1.0f / 24.0f);
  p = __fmaf_rn(p, r, 1.0f / 6.0f);
  p = __fmaf_rn(p, r, 0.5f);
  p = __fmaf_rn(p, r, 1.0f);
  p = __fmaf_rn(p, r, 1.0f);
  const int k = (int)kf;
  if (k < -126) return 0.0f;
  return __fmul_rn(p, __int_as_float((k + 127) << 23));
}

constexpr int POLICY_TPB = 64;     // envs (threads) per block
constexpr int POLICY_DEPTH = 9;    // partial-sum stack entries: the tree over 512 slots has 9 levels

// One thread per env.  The tree's leaves (the 512 chunk slots, 441 chunks
// and zero padding) are visited in bit-reversed slot order k -> c = rev9(k).
// In that order the two slots the tree adds at every level (i and i + h)
// are neighbours, so the tree is the one a binary counter builds from left
// to right.  Each chunk partial is pushed on a stack and added to the entries
// below it as the carry of k ripples (leaf k merges trailing_ones(k) times):
// the same additions of the same operands as the halving tree, hence the same
// bits.  The block stages chunk c of W, widened to fp32 (exact), in shared
// memory once for all its envs; every env's 84x84x4 stack is read once.
// mu_out (may be null) receives the behaviour probability of the sampled
// action, its weight over the total (fp32 division), for a V-trace buffer.
__global__ void __launch_bounds__(POLICY_TPB) k_policy(const uint8_t *obs, const uint16_t *W, const uint8_t *state,
                                                      uint8_t *actions, float *logits_out, float *mu_out, int n,
                                                      uint64_t seed) {
  __shared__ float wsm[64 * POLICY_A];
  __shared__ float stk[POLICY_DEPTH * POLICY_A][POLICY_TPB];
  const int t = threadIdx.x;
  const int i = blockIdx.x * POLICY_TPB + t;
  const bool live = i < n;
  const uint8_t *xs = obs + (size_t)(live ? i : 0) * POLICY_K;  // idle threads read env 0 and discard it
  int sp = 0;
#pragma unroll 1
  for (uint32_t k = 0; k < 512; ++k) {
    const uint32_t c = __brev(k) >> 23;
    float acc[POLICY_A];
#pragma unroll
    for (int j = 0; j < POLICY_A; ++j) acc[j] = 0.0f;
    if (c < (uint32_t)POLICY_CHUNKS) {  // the same for every thread of the block
      __syncthreads();                  // the previous chunk's readers are done
      const uint16_t *wc = W + (size_t)c * 64 * POLICY_A;
      for (int q = t; q < 64 * POLICY_A; q += POLICY_TPB) wsm[q] = __uint_as_float((uint32_t)wc[q] << 16);
      __syncthreads();
      const uint4 *x4 = reinterpret_cast<const uint4 *>(xs + (size_t)c * 64);
#pragma unroll 1
      for (int q4 = 0; q4 < 4; ++q4) {
        const uint4 xv4 = x4[q4];
        const uint32_t xw[4] = {xv4.x, xv4.y, xv4.z, xv4.w};
#pragma unroll
        for (int b = 0; b < 16; ++b) {
          const float xv = (float)((xw[b >> 2] >> (8 * (b & 3))) & 0xFF);
          const float *wr = wsm + (q4 * 16 + b) * POLICY_A;
#pragma unroll
          for (int j = 0; j < POLICY_A; ++j) acc[j] = __fmaf_rn(xv, wr[j], acc[j]);
        }
      }
    }
#pragma unroll 1
    for (uint32_t m = __ffs(~k) - 1; m > 0; --m) {
      --sp;
#pragma unroll
      for (int j = 0; j < POLICY_A; ++j) acc[j] = __fadd_rn(stk[sp * POLICY_A + j][t], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < POLICY_A; ++j) stk[sp * POLICY_A + j][t] = acc[j];
    ++sp;
  }
  if (live) {
    float l[POLICY_A];
    float m = stk[0][t];
#pragma unroll
    for (int j = 0; j < POLICY_A; ++j) {
      l[j] = stk[j][t];
      m = l[j] > m ? l[j] : m;
    }
    float e[POLICY_A], tot = 0.0f;
#pragma unroll
    for (int j = 0; j < POLICY_A; ++j) {
      e[j] = exp_cw(__fsub_rn(l[j], m));
      tot = __fadd_rn(tot, e[j]);
    }
    const uint8_t *st = state + (size_t)i * 256;
    const uint32_t *ew = reinterpret_cast<const uint32_t *>(st + S::EPISODE);
    const uint32_t x = philox_x0(seed, ew[2], ew[1], PURPOSE_POLICY << 8, ew[0]);
    const float thr = __fmul_rn(__fmul_rn(__uint2float_rn(x >> 8), 5.9604644775390625e-08f), tot);
    float c = 0.0f;
    int act = -1, last = 0;
#pragma unroll
    for (int j = 0; j < POLICY_A; ++j) {
      c = __fadd_rn(c, e[j]);
      if (e[j] > 0.0f) last = j;
      if (act < 0 && c > thr) act = j;
    }
    const int a = act < 0 ? last : act;
    actions[i] = (uint8_t)a;
    if (mu_out) {
      float ea = e[0];
#pragma unroll
      for (int j = 1; j < POLICY_A; ++j) ea = j == a ? e[j] : ea;
      mu_out[i] = __fdiv_rn(ea, tot);
    }
    if (logits_out) {
#pragma unroll
      for (int j = 0; j < POLICY_A; ++j) logits_out[(size_t)i * POLICY_A + j] = l[j];
    }
  }
}

// Append the newest stack plane, the reward and (ring_dones not null) the
// done flag of every env to ring slot `slot`.
__global__ void k_ring_append(const uint8_t *obs, const int32_t *rewards, const uint8_t *dones, uint8_t *ring_planes,
                              float *ring_rewards, uint8_t *ring_dones, int n, int slot) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const uint4 *src = reinterpret_cast<const uint4 *>(obs + (size_t)i * 4 * 7056 + 3 * 7056);
  uint4 *dst = reinterpret_cast<uint4 *>(ring_planes + ((size_t)slot * n + i) * 7056);
  for (int q = threadIdx.x; q < 7056 / 16; q += blockDim.x) dst[q] = src[q];
  if (threadIdx.x == 0) {
    ring_rewards[(size_t)slot * n + i] = (float)rewards[i];
    if (ring_dones) ring_dones[(size_t)slot * n + i] = dones[i];
  }
}

}  // namespace atari
