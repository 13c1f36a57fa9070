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

// ---- explicit augmented Schur complement (snapshot of the trailing interface block) ----------

// tile (i, j), 0 <= j <= i < nGb, of a subdomain's explicit Schur complement
__device__ __forceinline__ int64_t schur_tile(const SubMeta& m, int i, int j) {
  return m.schur_off + ((int64_t)i * (i + 1) / 2 + j) * NB2;
}

// block (t, s): copy interface tile t (row-major numbering of the lower triangle) of subdomain s
// if its interior columns are all eliminated and no interface column yet (nIb == b)
__global__ void __launch_bounds__(256) k_schur_snapshot(LevelDev L, int b) {
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  if (m.nIb != b) return;
  const int64_t t = blockIdx.x;
  if (t >= (int64_t)m.nGb * (m.nGb + 1) / 2) return;
  int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((int64_t)(i + 1) * (i + 2) / 2 <= t) ++i;
  while ((int64_t)i * (i + 1) / 2 > t) --i;
  const int j = (int)(t - (int64_t)i * (i + 1) / 2);
  const float4* src = (const float4*)((const float*)L.tiles + m.tile_off + tile_index_t(m.nIb + i, m.nIb + j, m.Bc) * NB2);
  float4* dst = (float4*)(L.schur + schur_tile(m, i, j));
  for (int e = threadIdx.x; e < NB2 / 4; e += blockDim.x) dst[e] = __ldcg(src + e);
}

// One pass over the stored lower tiles of M for y = M x.  Block (o, s, group) takes block row
// i = nGb - 1 - o (longest rows first).  The row's tiles (contiguous) stream through a ring of
// kSymvStages shared-memory stages, one 16 KB cp.async.bulk per tile (completion on an mbarrier
// per stage; every stage but the one being read has its copy in flight).  Warp w takes the tile
// rows w, w + 8, ..., w + 56, lane l the columns 2 l, 2 l + 1 (every row one 256-byte read).
//   row part      y_i += M_ij x_j: per (row, right-hand side) over the lane's columns, added over
//                 the lanes once at the end of the block row;
//   column part   M_ij^T x_i (j < i): per lane over the warp's rows, then over the eight warps
//                 through shared memory (double-buffered, one barrier per tile) and written to
//                 part (64 floats per tile and right-hand side), added later in order;
// the diagonal tile holds M_ii in its lower triangle only (the factorisation updates the full
// tile but its upper part never held the matrix): its row part uses the lower triangle, its
// column part the strict lower triangle, both into y_i.  Waits are bounded: a copy that never
// lands sets status[2] (the result is then garbage and the host reports the timeout).
constexpr int kSymvStages = 4;
constexpr long long kSymvSpins = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tile_g2s(float* dst, const float* src, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"((uint32_t)(NB2 * 4))
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"((uint32_t)(NB2 * 4)), "r"(smem_u32(bar))
               : "memory");
}

template <int NR>
__global__ void __launch_bounds__(256) k_schur_symv_rows(LevelDev L, const float* __restrict__ x,
                                                         const int64_t* __restrict__ part_off, int64_t part_stride,
                                                         float* __restrict__ part, float* __restrict__ y) {
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  if ((int)blockIdx.x >= m.nGb) return;
  const int i = m.nGb - 1 - (int)blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t c0q = (int64_t)blockIdx.z * NR * L.n_vec;   // first column of this group
  const float* xv = x + c0q + m.vec_off + (int64_t)m.nIb * NB;
  extern __shared__ __align__(128) float ring[];             // kSymvStages x NB2
  __shared__ __align__(8) uint64_t full[kSymvStages];
  __shared__ __align__(16) float cred[2][8][NR][NB];
  __shared__ float dcol[NR][NB];
  const float* Mrow = L.schur + schur_tile(m, i, 0);
  const int ntile = i + 1;
  if (tid == 0) {
    for (int k = 0; k < kSymvStages; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[k])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t issued = 0;
  if (tid == 0) {
    const int pre = ntile < kSymvStages ? ntile : kSymvStages;
    for (int k = 0; k < pre; ++k) tile_g2s(ring + k * NB2, Mrow + (int64_t)k * NB2, &full[k]);
    issued = (uint32_t)pre;
  }
  float xi[NR][8];   // x_i at this thread's rows
#pragma unroll
  for (int q = 0; q < NR; ++q)
#pragma unroll
    for (int r = 0; r < 8; ++r) xi[q][r] = xv[q * L.n_vec + (int64_t)i * NB + warp + 8 * r];
  float acc[8][NR];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[r][q] = 0.f;
  float* prow = part + (int64_t)blockIdx.z * NR * part_stride + part_off[s] + (int64_t)i * (i - 1) / 2 * NB;
  bool lost = false;
  for (int j = 0; j < ntile; ++j) {
    float2 xj[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) xj[q] = __ldg((const float2*)(xv + q * L.n_vec + (int64_t)j * NB + 2 * lane));
    const int slot = j % kSymvStages;
    {
      long long spins = 0;
      while (!mbar_try_wait(&full[slot], (uint32_t)(j / kSymvStages) & 1u))
        if (++spins > kSymvSpins) {
          if (!lost) atomicExch(L.status + 2, 5);
          lost = true;
          break;
        }
    }
    const float* T = ring + slot * NB2 + 2 * lane;
    float2 a[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = *(const float2*)(T + (warp + 8 * r) * NB);
    float2 cs[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) cs[q] = make_float2(0.f, 0.f);
    if (j < i) {
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          acc[r][q] += a[r].x * xj[q].x + a[r].y * xj[q].y;
          cs[q].x += a[r].x * xi[q][r];
          cs[q].y += a[r].y * xi[q][r];
        }
    } else {   // diagonal tile: lower triangle for the row part, strict lower for the column part
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int row = warp + 8 * r, c = 2 * lane;
        const float ax = c <= row ? a[r].x : 0.f, ay = c + 1 <= row ? a[r].y : 0.f;
        const float bx = c < row ? a[r].x : 0.f, by = c + 1 < row ? a[r].y : 0.f;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          acc[r][q] += ax * xj[q].x + ay * xj[q].y;
          cs[q].x += bx * xi[q][r];
          cs[q].y += by * xi[q][r];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) *(float2*)&cred[j & 1][warp][q][2 * lane] = cs[q];
    __syncthreads();   // the stage is read by every thread; cred[j & 1] is complete
    if (tid == 0 && j + kSymvStages < ntile) {
      tile_g2s(ring + slot * NB2, Mrow + (int64_t)(j + kSymvStages) * NB2, &full[slot]);
      ++issued;
    }
    // column sums of tile j over the warps (cred[j & 1] is next written at tile j + 2, after
    // the barrier of tile j + 1, which these threads reach only after this reduction)
    if (tid < NR * NB) {
      const int q = tid / NB, c = tid % NB;
      float v = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) v += cred[j & 1][w][q][c];
      if (j < i)
        prow[q * part_stride + (int64_t)j * NB + c] = v;
      else
        dcol[q][c] = v;
    }
  }
  // row sums over the lanes, fixed order (xor butterfly)
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[r][q] += __shfl_xor_sync(0xffffffffu, acc[r][q], o);
  __syncthreads();   // dcol is complete
  if (lane == 0) {
    float* yv = y + c0q + m.vec_off + (int64_t)m.nIb * NB + (int64_t)i * NB;
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int q = 0; q < NR; ++q) yv[q * L.n_vec + warp + 8 * r] = acc[r][q] + dcol[q][warp + 8 * r];
  }
  // after a lost wait, copies may still be landing in this CTA's shared memory: wait (bounded)
  // for the last phase issued on every stage before the CTA exits
  if (tid == 0 && lost)
    for (uint32_t c = issued > (uint32_t)kSymvStages ? issued - kSymvStages : 0u; c < issued; ++c) {
      long long spins = 0;
      while (!mbar_try_wait(&full[c % kSymvStages], (c / kSymvStages) & 1u) && ++spins < kSymvSpins) {
      }
    }
}

// y_j += sum_{i > j} part(i, j); block (j, s, group).  Every column's rows i are split into 4
// interleaved segments (i = j + 1 + g, j + 5 + g, ...), whose partial sums are added in segment
// order: a fixed order, the same for any number of columns per launch.
template <int NR>
__global__ void __launch_bounds__(256) k_schur_symv_cols(LevelDev L, const int64_t* __restrict__ part_off,
                                                         int64_t part_stride, const float* __restrict__ part,
                                                         float* __restrict__ y) {
  constexpr int G = 4;   // row segments
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  const int j = blockIdx.x;
  if (j >= m.nGb - 1) return;
  __shared__ float ps[G][NR * NB];
  const int64_t c0q = (int64_t)blockIdx.z * NR;
  for (int w = threadIdx.x; w < G * NR * NB; w += blockDim.x) {
    const int e = w % (NR * NB), g = w / (NR * NB);
    const int q = e / NB, c = e % NB;
    const float* p = part + (c0q + q) * part_stride + part_off[s];
    float v = 0.f;
    for (int i = j + 1 + g; i < m.nGb; i += G) v += p[((int64_t)i * (i - 1) / 2 + j) * NB + c];
    ps[g][e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NR * NB; e += blockDim.x) {
    const int q = e / NB, c = e % NB;
    float t = ps[0][e];
#pragma unroll
    for (int h = 1; h < G; ++h) t += ps[h][e];
    float* yv = y + (c0q + q) * L.n_vec + m.vec_off + (int64_t)m.nIb * NB + (int64_t)j * NB + c;
    *yv = *yv + t;
  }
}

}  // namespace

void launch_schur_snapshot(const LevelDev& L, int b, int max_nGb, cudaStream_t st) {
  if (max_nGb <= 0 || L.n_sub <= 0 || !L.schur) return;
  note_launch();
  k_schur_snapshot<<<dim3((unsigned)((int64_t)max_nGb * (max_nGb + 1) / 2), (unsigned)L.n_sub), 256, 0, st>>>(L, b);
}

template <int NR>
void launch_symv_nr(const LevelDev& L, const dim3& grid, const int64_t* part_off, int64_t part_stride, const float* x,
                    float* part, float* y, cudaStream_t st) {
  const size_t dyn = sizeof(float) * kSymvStages * NB2;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_schur_symv_rows<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    attr = true;
  }
  note_launch();
  k_schur_symv_rows<NR><<<grid, 256, dyn, st>>>(L, x, part_off, part_stride, part, y);
  note_launch();
  k_schur_symv_cols<NR><<<grid, 256, 0, st>>>(L, part_off, part_stride, part, y);
}

void launch_schur_symv(const LevelDev& L, int max_nGb, const int64_t* part_off, int64_t part_stride, const float* x,
                       float* part, float* y, cudaStream_t st, int nr) {
  if (max_nGb <= 0 || L.n_sub <= 0 || nr <= 0) return;
  // columns in groups of 4, 2, 1 (the row kernel keeps 4 NR row sums and 4 NR column sums per lane)
  for (int r0 = 0; r0 < nr;) {
    const int left = nr - r0;
    const int g = left >= 4 ? 4 : left >= 2 ? 2 : 1;
    const int ng = left / g;
    const dim3 grid((unsigned)max_nGb, (unsigned)L.n_sub, (unsigned)ng);
    const int64_t off = (int64_t)r0 * L.n_vec;
    float* pp = part + (int64_t)r0 * part_stride;
    if (g == 4)
      launch_symv_nr<4>(L, grid, part_off, part_stride, x + off, pp, y + off, st);
    else if (g == 2)
      launch_symv_nr<2>(L, grid, part_off, part_stride, x + off, pp, y + off, st);
    else
      launch_symv_nr<1>(L, grid, part_off, part_stride, x + off, pp, y + off, st);
    r0 += ng * g;
  }
}

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
