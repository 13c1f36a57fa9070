// Inner Schur operator from the stored factor (mixed precision only).
//
// The trailing block of the partial factorisation of A_i = K_i + C_i^T R C_i is the factor of
// the augmented local Schur complement: L_GG S L_GG^T = S_i + C_i^T R C_i, S_i = K_GG -
// K_GI K_II^{-1} K_IG (Sec. 2).  So S~_i x = L_GG S (L_GG^T x) - C_i^T R C_i x reproduces S_i up to
// the FP32 rounding of the factorisation, with two triangular matrix-vector PRODUCTS over the
// interface block rows: unlike the triangular solves they carry no dependency chain, so every
// (subdomain, block row) is an independent CTA and the pass streams the interface triangle at
// full bandwidth.  It serves as the cheap operator of the inner iteration of the mixed solver;
// the outer iteration applies the FP64 operator.  Several right-hand sides share each pass over
// the triangle (up to eight per launch).
#include "internal.h"

namespace bddc {

namespace {

__device__ __forceinline__ int64_t tile_index_t(int i, int j, int Bc) {
  return i < Bc ? ((int64_t)i * (i + 1) / 2 + j) : ((int64_t)Bc * (Bc + 1) / 2 + (int64_t)(i - Bc) * Bc + j);
}

// y1_j = sum_{i >= j} L(i,j)^T x_i over the interface block rows; block (o, s, group) makes
// output block j = nIb + o for NR right-hand sides (column r at x + r * n_vec).  Warp w takes the
// tile rows w, w+8, ..., lane l the columns 2l, 2l+1, so every row is one coalesced 256-byte
// read, applied to all NR columns; the eight warps' column sums are added at the end in a fixed
// order (no barrier inside the tile loop).
template <int NR>
__global__ void __launch_bounds__(256) k_trmv_t(LevelDev L, const float* __restrict__ x, float* __restrict__ y1) {
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  const int o = blockIdx.x;
  if (o >= m.nGb) return;
  const int j = m.nIb + o;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ float part[8][NR][64];
  const int64_t c0 = (int64_t)blockIdx.z * NR * L.n_vec;   // first column of this group
  const float* tiles = (const float*)L.tiles + m.tile_off;
  const float* xv = x + c0 + m.vec_off;
  const int nGrow = m.nIb * NB + m.nG;   // padded rows beyond the interface hold no data
  float ax[NR], ay[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) ax[q] = ay[q] = 0.f;
#pragma unroll 2
  for (int i = j; i < m.Bc; ++i) {
    const float* t = tiles + tile_index_t(i, j, m.Bc) * NB2 + 2 * lane;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int row = warp + 8 * r;
      const int grow = i * NB + row;
      const float2 a = __ldg((const float2*)(t + row * NB));
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        const float xr = grow < nGrow ? __ldg(xv + q * L.n_vec + grow) : 0.f;
        ax[q] += a.x * xr;
        ay[q] += a.y * xr;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    part[warp][q][2 * lane] = ax[q];
    part[warp][q][2 * lane + 1] = ay[q];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NR * 64; e += 256) {
    const int q = e / 64, c = e % 64;
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) v += part[w][q][c];
    y1[c0 + q * L.n_vec + m.vec_off + (int64_t)j * NB + c] = v;
  }
}

// y_i = sum_{nIb <= j <= i} L(i,j) S_j y1_j; block (o', s, group) makes output block i = nIb + o
// with o = nGb - 1 - o' (the longest block rows are scheduled first, so that the short ones fill
// the tail of the launch).  Warp w takes rows w, w+8, ..., lane l the columns 2l, 2l+1.
template <int NR>
__global__ void __launch_bounds__(256) k_trmv_n(LevelDev L, const float* __restrict__ y1, float* __restrict__ y) {
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  if ((int)blockIdx.x >= m.nGb) return;
  const int o = m.nGb - 1 - (int)blockIdx.x;
  const int i = m.nIb + o;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c0 = (int64_t)blockIdx.z * NR * L.n_vec;
  const float* tiles = (const float*)L.tiles + m.tile_off;
  const float* yv = y1 + c0 + m.vec_off;
  const float* sg = (const float*)L.sgn + m.vec_off;
  float acc[8][NR];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[r][q] = 0.f;
#pragma unroll 2
  for (int j = m.nIb; j <= i; ++j) {
    float2 sj = make_float2(1.f, 1.f);
    if (L.indefinite) sj = *(const float2*)(sg + (int64_t)j * NB + 2 * lane);
    const float* t = tiles + tile_index_t(i, j, m.Bc) * NB2 + 2 * lane;
    float2 a[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = __ldg((const float2*)(t + (warp + 8 * r) * NB));
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      float2 b = *(const float2*)(yv + q * L.n_vec + (int64_t)j * NB + 2 * lane);
      b.x *= sj.x;
      b.y *= sj.y;
#pragma unroll
      for (int r = 0; r < 8; ++r) acc[r][q] += a[r].x * b.x + a[r].y * b.y;
    }
  }
#pragma unroll
  for (int q = 0; q < NR; ++q)
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      float v = acc[r][q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) y[c0 + q * L.n_vec + m.vec_off + (int64_t)i * NB + warp + 8 * r] = v;
    }
}

// y -= C^T R C x over the padded local interface vectors (FP64); one warp per constraint row.
// Distinct rows touch disjoint positions (each local DOF lies in one glob and has one
// component), so the update needs no atomics.
__global__ void k_sub_ctrc(LevelDev L, const int32_t* __restrict__ crow_sub, int64_t total_rows,
                           const double* __restrict__ x, double* __restrict__ y) {
  const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= total_rows) return;
  x += (int64_t)blockIdx.y * L.n_vec;   // column blockIdx.y of a block of right-hand sides
  y += (int64_t)blockIdx.y * L.n_vec;
  const int s = crow_sub[g];
  const SubMeta m = L.meta[s];
  const double rq = L.rho[s] * L.c_rho[g];
  if (rq == 0.0) return;
  const int64_t a = L.c_ptr[g], b = L.c_ptr[g + 1];
  double t = 0.0;
  for (int64_t e = a + lane; e < b; e += 32) t += L.c_val[e] * x[m.vec_off + L.c_pos[e]];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  for (int64_t e = a + lane; e < b; e += 32) y[m.vec_off + L.c_pos[e]] -= rq * t * L.c_val[e];
}

}  // namespace

template <int NR>
void launch_trmv_nr(const LevelDev& L, const dim3& grid, const float* x, float* y1, float* y, cudaStream_t st) {
  note_launch();
  k_trmv_t<NR><<<grid, 256, 0, st>>>(L, x, y1);
  note_launch();
  k_trmv_n<NR><<<grid, 256, 0, st>>>(L, y1, y);
}

void launch_trmv_schur(const LevelDev& L, int max_nGb, const float* x, float* y1, float* y, cudaStream_t st, int nr) {
  if (max_nGb <= 0 || L.n_sub <= 0 || nr <= 0) return;
  // columns in groups of 8, 4, 2, 1: each group reads the interface triangle once per product
  for (int r0 = 0; r0 < nr;) {
    const int left = nr - r0;
    const int g = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    const int ng = left / g;
    const dim3 grid((unsigned)max_nGb, (unsigned)L.n_sub, (unsigned)ng);
    const int64_t off = (int64_t)r0 * L.n_vec;
    if (g == 8)
      launch_trmv_nr<8>(L, grid, x + off, y1 + off, y + off, st);
    else if (g == 4)
      launch_trmv_nr<4>(L, grid, x + off, y1 + off, y + off, st);
    else if (g == 2)
      launch_trmv_nr<2>(L, grid, x + off, y1 + off, y + off, st);
    else
      launch_trmv_nr<1>(L, grid, x + off, y1 + off, y + off, st);
    r0 += ng * g;
  }
}

void launch_sub_ctrc(const LevelDev& L, const int32_t* crow_sub, int64_t total_rows, const double* x, double* y,
                     cudaStream_t st, int nr) {
  if (total_rows <= 0) return;
  note_launch();
  k_sub_ctrc<<<dim3((unsigned)((total_rows + 7) / 8), nr), 256, 0, st>>>(L, crow_sub, total_rows, x, y);
}

}  // namespace bddc
