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

// Split one 64-row block of NT tile columns into the split row `row`; 64 NT threads (2 NT warps).
// Warp w takes tile column c = w / 2 (source tile src, row-major 64 x 64, or null for zeros) and
// the rows 32 (w % 2) .. + 31; lane l the four entries 4 (l % 16) .. + 3 of the rows 2k + l / 16,
// so that 16 lanes read a 256-byte row of a tile at once and write its 128-byte FP16 image at
// once.  Pass 1 loads the warp's 32 rows (16 float4 per lane) and records each row's maximum
// within the tile; after one barrier, pass 2 takes the row's maximum over the NT tiles and writes
// the scaled parts.  rowmul: per-row factors (+-1) applied to the entries, or null.  sq: the pivot signs
// of the warp's 64 columns for the signed copy (split_signed), or null (zero tile).
template <int NT>
__device__ __forceinline__ void split_rows(const float* src, const float* __restrict__ rowmul,
                                           int64_t row, uint8_t* __restrict__ split,
                                           uint8_t* __restrict__ split_signed, float* __restrict__ rscale,
                                           const float* sq) {
  static_assert(NT == 4 || NT == 8, "panel width");
  __shared__ float pmax[NT][NB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = warp >> 1, r0 = 32 * (warp & 1), u = lane & 15, half = lane >> 4;
  const float4* t = src ? (const float4*)src + u : nullptr;
  float4 v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int r = r0 + 2 * k + half;
    v[k] = t ? __ldcg(t + r * (NB / 4)) : make_float4(0.f, 0.f, 0.f, 0.f);
    float mx = fmaxf(fmaxf(fabsf(v[k].x), fabsf(v[k].y)), fmaxf(fabsf(v[k].z), fabsf(v[k].w)));
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (u == 0) pmax[c][r] = mx;
  }
  __syncthreads();
  uint8_t* dst = split + (row * kPanelTiles + c) * (int64_t)kSplitTile;
  uint8_t* dsg = split_signed ? split_signed + (row * kPanelTiles + c) * (int64_t)kSplitTile : nullptr;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int r = r0 + 2 * k + half;
    float mx = 0.f;
#pragma unroll
    for (int q = 0; q < NT; ++q) mx = fmaxf(mx, pmax[q][r]);
    int ex = 0;
    if (mx > 0.f) {
      int e;
      frexpf(mx, &e);   // mx = f 2^e, f in [0.5, 1)
      ex = 15 - e;      // mx 2^ex in [2^14, 2^15)
    }
    if (c == 0 && u == 0) rscale[row * NB + r] = ldexpf(1.f, -ex);   // exact power of two
    const float rm = rowmul ? rowmul[r] : 1.f;
    const float a[4] = {rm * v[k].x, rm * v[k].y, rm * v[k].z, rm * v[k].w};
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
    if (dsg) {   // indefinite levels: the B operand is L(j, q) S_q (pivot signs of column q)
      if (sq) {
        const float* sqc = sq + 4 * u;
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (sqc[e] < 0.f) {
            h[e] = __hneg(h[e]);
            l[e] = __hneg(l[e]);
          }
      }
      store4h(dsg, off, h);
      store4h(dsg + kTilePart, off, l);
    }
  }
}

// Split the panel tiles L(i, kb0 .. kb0 + NT - 1) of subdomain s into the split row prow_off[s] + i
// (tile columns kb0 + c >= Bc, which exist only in a subdomain's last panel, as zeros).
template <int NT>
__device__ __forceinline__ void split_row_tile(const LevelDev& L, int s, const SubMeta& m, int i, int kb0,
                                               uint8_t* __restrict__ split, uint8_t* __restrict__ split_signed,
                                               float* __restrict__ rscale, const int64_t* __restrict__ prow_off) {
  const int c = threadIdx.x >> 6;
  const float* src =
      kb0 + c < m.Bc ? (const float*)L.tiles + m.tile_off + split_tile_index(i, kb0 + c, m.Bc) * NB2 : nullptr;
  const float* sq = src ? (const float*)L.sgn + m.vec_off + (int64_t)(kb0 + c) * NB : nullptr;   // column signs
  split_rows<NT>(src, nullptr, prow_off[s] + i, split, split_signed, rscale, sq);
}

}  // namespace bddc
