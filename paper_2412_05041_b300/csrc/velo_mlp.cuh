// Ghost-rejection network: candidate features and warp-level bfloat16
// tensor-core inference (12 -> 32 -> 32 -> 1, ReLU, ReLU, logit).
//
// The paper's first stage keeps tracks by a simplified fit's quality
// (Sec. "HLT1 details and results"); the learned form scores each candidate
// with this small network instead of the 3-hit rule, the loose chi2/ndf cut
// staying in place.  Arithmetic (the CPU oracle emulates the same steps):
//   x_k  = bf16((f_k - mean_k) * inv_std_k)                  (round to nearest even)
//   h1_j = bf16(relu(sum_k bf16(W1[j][k]) x_k + b1_j))        float32 accumulation
//   h2_j = relu(sum_k bf16(W2[j][k]) h1_k + b2_j)             float32
//   logit = sum_j W3[j] h2_j + b3                             float32
// The two hidden layers run as mma.sync.m16n8k16 bf16 -> f32 on one warp's 32
// candidates (two 16-row tiles, one after the other through the same staging
// tiles; layer 1 = 8 MMAs, layer 2 = 16 MMAs).  The
// contraction is 32 x 12 x 32 per warp: a few hundred FLOPs per candidate, so
// latency, not tensor throughput, bounds it and the warp-synchronous MMA is
// the right size of tool; the accumulation order inside an MMA is the
// hardware's, so GPU and oracle logits agree to float32 rounding, not bits.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "velo.h"

namespace velo {

constexpr int kFeat = VELO_N_FEATURES;  // 12
constexpr int kHid = VELO_MLP_HIDDEN;   // 32
constexpr int kKPad = 16;               // features padded to one MMA k-step

// Network constants in shared memory (loaded once per CTA).
struct MlpWeights {
  __nv_bfloat16 w1[kHid * kKPad];  // [hidden][k], k >= 12 zero
  __nv_bfloat16 w2[kHid * kHid];   // [hidden][k]
  float b1[kHid], b2[kHid], w3[kHid];
  float mean[kFeat], istd[kFeat];
  float b3;
};

// Per-warp staging tiles (one 16-candidate m-tile at a time).
struct MlpTiles {
  __nv_bfloat16 x[16 * kKPad];  // 16 candidates x 16 inputs
  __nv_bfloat16 h[16 * kHid];   // 16 candidates x 32 first-layer outputs
};

// blob (float32): mean[12], inv_std[12], W1[32][12], b1[32], W2[32][32], b2[32], W3[32], b3
__device__ __forceinline__ void mlp_load(const float* blob, MlpWeights& W, int tid, int nthreads) {
  const float* mean = blob;
  const float* istd = blob + kFeat;
  const float* W1 = blob + 2 * kFeat;
  const float* b1 = W1 + kHid * kFeat;
  const float* W2 = b1 + kHid;
  const float* b2 = W2 + kHid * kHid;
  const float* W3 = b2 + kHid;
  for (int i = tid; i < kHid * kKPad; i += nthreads) {
    const int j = i / kKPad, k = i % kKPad;
    W.w1[i] = __float2bfloat16_rn(k < kFeat ? W1[j * kFeat + k] : 0.0f);
  }
  for (int i = tid; i < kHid * kHid; i += nthreads) W.w2[i] = __float2bfloat16_rn(W2[i]);
  for (int i = tid; i < kHid; i += nthreads) {
    W.b1[i] = b1[i];
    W.b2[i] = b2[i];
    W.w3[i] = W3[i];
  }
  for (int i = tid; i < kFeat; i += nthreads) {
    W.mean[i] = mean[i];
    W.istd[i] = istd[i];
  }
  if (tid == 0) W.b3 = W3[kHid];
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Logit of this lane's candidate (features f[12]); every lane of the warp
// must call it (lanes without a candidate pass zeros and ignore the result).
__device__ __forceinline__ float mlp_logit_warp(const float* f, const MlpWeights& W, MlpTiles& T) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  float part[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};  // [m-tile][row g / row g+8]
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {  // candidates 16 mt .. 16 mt + 15 (lanes of that half)
    if ((lane >> 4) == mt) {
#pragma unroll
      for (int k = 0; k < kKPad; ++k)
        T.x[(lane & 15) * kKPad + k] =
            __float2bfloat16_rn(k < kFeat ? __fmul_rn(__fsub_rn(f[k], W.mean[k]), W.istd[k]) : 0.0f);
    }
    __syncwarp();
    // layer 1: rows = candidates, cols = hidden units (four n-tiles), one k-step
    {
      const __nv_bfloat16* xr0 = T.x + g * kKPad;
      const __nv_bfloat16* xr8 = T.x + (g + 8) * kKPad;
      const uint32_t a0 = pack_bf16(xr0[2 * t4], xr0[2 * t4 + 1]);
      const uint32_t a1 = pack_bf16(xr8[2 * t4], xr8[2 * t4 + 1]);
      const uint32_t a2 = pack_bf16(xr0[2 * t4 + 8], xr0[2 * t4 + 9]);
      const uint32_t a3 = pack_bf16(xr8[2 * t4 + 8], xr8[2 * t4 + 9]);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const __nv_bfloat16* wr = W.w1 + (nt * 8 + g) * kKPad;  // B[k][n] = W1[n][k]
        const uint32_t b0 = pack_bf16(wr[2 * t4], wr[2 * t4 + 1]);
        const uint32_t b1 = pack_bf16(wr[2 * t4 + 8], wr[2 * t4 + 9]);
        float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        mma_bf16(c, a0, a1, a2, a3, b0, b1);
        const int col = nt * 8 + 2 * t4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = g + (q >= 2 ? 8 : 0), cc = col + (q & 1);
          const float a = __fadd_rn(c[q], W.b1[cc]);
          T.h[row * kHid + cc] = __float2bfloat16_rn(a > 0.0f ? a : 0.0f);
        }
      }
    }
    __syncwarp();
    // layer 2 (two k-steps) and layer 3 on the accumulators
    const __nv_bfloat16* hr0 = T.h + g * kHid;
    const __nv_bfloat16* hr8 = T.h + (g + 8) * kHid;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const int k0 = ks * 16 + 2 * t4;
        const uint32_t a0 = pack_bf16(hr0[k0], hr0[k0 + 1]);
        const uint32_t a1 = pack_bf16(hr8[k0], hr8[k0 + 1]);
        const uint32_t a2 = pack_bf16(hr0[k0 + 8], hr0[k0 + 9]);
        const uint32_t a3 = pack_bf16(hr8[k0 + 8], hr8[k0 + 9]);
        const __nv_bfloat16* wr = W.w2 + (nt * 8 + g) * kHid;  // B[k][n] = W2[n][k]
        const uint32_t b0 = pack_bf16(wr[k0], wr[k0 + 1]);
        const uint32_t b1 = pack_bf16(wr[k0 + 8], wr[k0 + 9]);
        mma_bf16(c, a0, a1, a2, a3, b0, b1);
      }
      const int col = nt * 8 + 2 * t4;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int cc = col + (q & 1);
        float h2 = __fadd_rn(c[q], W.b2[cc]);
        h2 = h2 > 0.0f ? h2 : 0.0f;
        part[mt][q >> 1] = __fadd_rn(part[mt][q >> 1], __fmul_rn(W.w3[cc], h2));
      }
    }
    __syncwarp();  // the tiles are rewritten for the next m-tile
  }
  // sum the four lanes of a group (each holds 8 of the 32 hidden units of its rows)
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      part[mt][r] = __fadd_rn(part[mt][r], __shfl_xor_sync(0xFFFFFFFFu, part[mt][r], 1));
      part[mt][r] = __fadd_rn(part[mt][r], __shfl_xor_sync(0xFFFFFFFFu, part[mt][r], 2));
    }
  // this lane's candidate is row (lane % 16) of m-tile lane / 16: held by group (lane % 8)
  // (every lane sends both halves: a shuffle returns the value the source lane passes)
  const int src = 4 * (lane & 7), hi = (lane & 15) >= 8;
  float sel[2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const float lo_half = __shfl_sync(0xFFFFFFFFu, part[mt][0], src);
    const float hi_half = __shfl_sync(0xFFFFFFFFu, part[mt][1], src);
    sel[mt] = hi ? hi_half : lo_half;
  }
  __syncwarp();
  return __fadd_rn(lane < 16 ? sel[0] : sel[1], W.b3);
}

// The 12 candidate features (binary32, the oracle's order): hits ascending in z.
__device__ __forceinline__ void candidate_features(uint32_t n, const float* x, const float* y, const float* z,
                                                   const uint32_t* mod, const float* st, float chi2ndf, float* f) {
  f[0] = (float)n;
  f[1] = chi2ndf;
  f[2] = st[2];
  f[3] = st[3];
  f[4] = z[0];
  f[5] = z[n - 1];
  f[6] = (float)((int)(mod[n - 1] - mod[0] + 1) - (int)n);
  float sx = 0.0f, sxx = 0.0f, sy = 0.0f, syy = 0.0f, mx = 0.0f;
  for (uint32_t i = 0; i < n; ++i) {
    const float dz = __fsub_rn(z[i], z[0]);
    const float rx = __fsub_rn(__fsub_rn(x[i], st[0]), __fmul_rn(st[2], dz));
    const float ry = __fsub_rn(__fsub_rn(y[i], st[1]), __fmul_rn(st[3], dz));
    sx = __fadd_rn(sx, rx);
    sxx = __fadd_rn(sxx, __fmul_rn(rx, rx));
    sy = __fadd_rn(sy, ry);
    syy = __fadd_rn(syy, __fmul_rn(ry, ry));
    mx = fmaxf(mx, fmaxf(fabsf(rx), fabsf(ry)));
  }
  const float fn = (float)n;
  f[7] = __fdiv_rn(sx, fn);
  f[8] = __fsqrt_rn(__fdiv_rn(sxx, fn));
  f[9] = __fdiv_rn(sy, fn);
  f[10] = __fsqrt_rn(__fdiv_rn(syy, fn));
  f[11] = mx;
}

}  // namespace velo
