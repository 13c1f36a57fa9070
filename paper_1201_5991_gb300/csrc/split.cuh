// The scaled two-part FP16 split of the panel row tiles that feeds the tensor-core trailing
// update (see update_tc.cu): for row tile i and NT tile columns of a panel (NT = 4: a 256-wide
// sub-panel, NT = 8: a 512-wide super-panel), every row r is scaled by 2^e_r so that its largest
// entry lies in [2^14, 2^15), and each scaled entry a is split into hi = fp16(a) and
// lo = fp16((a - hi) 2^11), written in the shared-memory operand image of the update (K-major,
// 128-byte swizzle).
#pragma once

#include <cuda_fp16.h>

#include "internal.h"

namespace bddc {

constexpr int kPanelTiles = 8;                  // tile columns of a super-panel (the split buffer's row pitch)
constexpr uint32_t kTilePart = 64 * 128;        // one FP16 part of one 64 x 64 tile (8 KB)
constexpr uint32_t kSplitTile = 2 * kTilePart;  // hi and lo of one tile (16 KB)

__device__ __forceinline__ int64_t split_tile_index(int i, int j, int Bc) {
  return i < Bc ? ((int64_t)i * (i + 1) / 2 + j) : ((int64_t)Bc * (Bc + 1) / 2 + (int64_t)(i - Bc) * Bc + j);
}

__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  return (uint32_t)(r * 128 + (((k >> 3) ^ (r & 7)) << 4) + (k & 7) * 2);
}

__device__ __forceinline__ void store4h(uint8_t* part, uint32_t off, const __half* h) {
  __half2 lo = __halves2half2(h[0], h[1]), hi = __halves2half2(h[2], h[3]);
  uint2 v;
  v.x = *(uint32_t*)&lo;
  v.y = *(uint32_t*)&hi;
  *(uint2*)(part + off) = v;
}

// Split the panel tiles L(i, kb0 .. kb0 + NT - 1) of subdomain s; 64 NT threads, thread (r, c4)
// takes row r of tile column kb0 + c4 (the NT threads of a row, adjacent lanes, share its scale).
template <int NT>
__device__ __forceinline__ void split_row_tile(const LevelDev& L, int s, const SubMeta& m, int i, int kb0,
                                               uint8_t* __restrict__ split, uint8_t* __restrict__ split_signed,
                                               float* __restrict__ rscale, const int64_t* __restrict__ prow_off) {
  static_assert(NT == 4 || NT == 8, "panel width");
  const int r = threadIdx.x / NT, c4 = threadIdx.x % NT;
  const float4* t =
      (const float4*)((const float*)L.tiles + m.tile_off + split_tile_index(i, kb0 + c4, m.Bc) * NB2 + r * NB);
  float4 v[16];
  float mx = 0.f;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    v[u] = __ldcg(t + u);
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v[u].x), fabsf(v[u].y)), fmaxf(fabsf(v[u].z), fabsf(v[u].w))));
  }
#pragma unroll
  for (int o = 1; o < NT; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int ex = 0;
  if (mx > 0.f) {
    int k;
    frexpf(mx, &k);   // mx = f 2^k, f in [0.5, 1)
    ex = 15 - k;      // mx 2^ex in [2^14, 2^15)
  }
  const int64_t row = prow_off[s] + i;
  if (c4 == 0) rscale[row * NB + r] = ldexpf(1.f, -ex);   // exact power of two
  uint8_t* dst = split + (row * kPanelTiles + c4) * (int64_t)kSplitTile;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const float a[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
    __half h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float sa = ldexpf(a[e], ex);
      h[e] = __float2half_rn(sa);
      l[e] = __float2half_rn((sa - __half2float(h[e])) * 2048.f);
    }
    const uint32_t off = sw128_off(r, 4 * u);
    store4h(dst, off, h);
    store4h(dst + kTilePart, off, l);
    if (split_signed) {   // indefinite levels: the B operand is L(j, q) S_q (pivot signs of column q)
      const float* sq = (const float*)L.sgn + m.vec_off + (int64_t)(kb0 + c4) * NB + 4 * u;
      uint8_t* dsg = split_signed + (row * kPanelTiles + c4) * (int64_t)kSplitTile;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (sq[e] < 0.f) {
          h[e] = __hneg(h[e]);
          l[e] = __hneg(l[e]);
        }
      store4h(dsg, off, h);
      store4h(dsg + kTilePart, off, l);
    }
  }
}

}  // namespace bddc
