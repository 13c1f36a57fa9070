// Trailing update of the blocked Cholesky on the 5th-generation tensor cores (tcgen05), FP32
// factors (mixed mode): for nq panel tile columns q in [kb0, kb0 + nq),
//     A(i, j) -= sum_q L(i, q) S_q L(j, q)^T       for jbeg <= j < min(Bc, jend), j <= i < R,
// (S_q: pivot signs of the signed Cholesky, identity for SPD levels)
// batched over all subdomains of a level (Algorithm 1, "factorize the matrices of local saddle
// point problems").  The factorisation runs in 512-wide super-panels of two 256-wide halves:
// after the first half, a rank-256 update (nq = 4) brings the second half's columns up to date;
// after the second half, one rank-512 update (nq = 8) serves every trailing column.  Each
// trailing element is read and written once per 512 columns instead of once per 256 (without its
// output write-back the rank-256 kernel ran 27 % faster): on the 48^3 factorisation the update
// went from 254 to 300 TFLOP/s FP32-equivalent.
//
// FP32 accuracy from FP16 tensor cores: for the 64 x 256 slab of panel row tile i, every row r
// is scaled by 2^e_r so that its largest entry lies in [2^14, 2^15), and each scaled entry a is
// split into hi = fp16(a) and lo = fp16((a - hi) 2^11) (the scaled low part cannot underflow).
// Then a b = hi_a hi_b + (hi_a lo_b + lo_a hi_b) 2^-11 up to the dropped lo lo term (2^-22
// relative): three FP16 products, 4 bytes per entry (the scheme of Ootomo and Yokota, 2022).
// The output is unscaled exactly by the stored factors 2^-e_i and 2^-e_j.  Indefinite levels
// also get a copy of the parts whose columns carry the pivot signs, read as the B operand, so
// that both operands of every MMA stay FP16.  Measured against FP64 on factor-like data (rows
// spanning four decades): 2-4e-7 of sum |a||b| (three-part BF16 splitting with six products:
// 1.3e-7, FP32 dot: 8e-7).  Accumulating all products in one TMEM accumulator over K = 256
// loses an order of magnitude, so the dominant hi hi product has its own accumulator and both
// are promoted into FP32 registers after every 64-wide panel column.
//
// k_split_panel writes the parts in the exact shared-memory operand image (K-major, 128-byte
// swizzle), so the update moves bytes with cp.async.bulk only.  A work item is a 128 x 128
// output block (row tiles i0, i0+1 by column tiles j, j+1); per panel column q the producer
// warp copies the two parts of the four tiles (64 KB) into one of three shared-memory stages
// and one thread issues 12 MMAs (3 products x 4 K-steps, M = N = 128) into one of two TMEM
// accumulator pairs (hi hi; the two cross products); eight epilogue warps promote each pair
// into FP32 registers after every column and finally update the output tiles.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "internal.h"
#include "split.cuh"

namespace bddc {

namespace {

constexpr long long kSpinLimit = 1ll << 26;

__device__ __forceinline__ int64_t tile_index(int i, int j, int Bc) {
  return i < Bc ? ((int64_t)i * (i + 1) / 2 + j) : ((int64_t)Bc * (Bc + 1) / 2 + (int64_t)(i - Bc) * Bc + j);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major operand, 128-byte swizzle: rows of 64 16-bit entries (128 B), 8-row atoms of 1024 B
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);   // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}


__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}


constexpr uint32_t kOpnd = 2 * kTilePart;        // one part of a 128-row operand (16 KB)
constexpr uint32_t kStage2 = 4 * kOpnd;          // A hi, A lo, B hi, B lo (64 KB)
constexpr int kThreads2 = 320;                   // 8 epilogue warps + 1 MMA warp + 1 producer warp
constexpr int kStages2 = 3;                      // shared-memory stages (copies run two steps ahead)
constexpr uint32_t kEpiBox = 32 * 128;           // per epilogue warp: one 32 x 32 FP32 output box (4 KB)

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}


// one block per panel row tile i (ib <= i < R) of every subdomain with output columns (ib < Bc);
// panel_operand: the rows i >= min(ib, Bc) of every subdomain with kb0 < Bc
template <int NT>
__global__ void __launch_bounds__(64 * NT) k_split_panel(LevelDev L, int kb0, int ib, int panel_operand,
                                                         uint8_t* __restrict__ split,
                                                         uint8_t* __restrict__ split_signed,
                                                         float* __restrict__ rscale,
                                                         const int64_t* __restrict__ prow_off) {
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  int i;
  if (panel_operand) {
    if (kb0 >= m.Bc) return;
    i = (ib < m.Bc ? ib : m.Bc) + (int)blockIdx.x;
  } else {
    if (ib >= m.Bc) return;
    i = ib + (int)blockIdx.x;
  }
  if (i >= m.R) return;
  split_row_tile<NT>(L, s, m, i, kb0, split, split_signed, rscale, prow_off);
}

// one block per block row Q of the inverse X of every subdomain's diagonal block (Q < nd): the
// rows of -S_D X, the B operand of the panel solve (its update kernel subtracts A B^T)
__global__ void __launch_bounds__(256) k_split_inverse(LevelDev L, int k0, const float* __restrict__ xinv,
                                                       uint8_t* __restrict__ split, float* __restrict__ rscale,
                                                       const int64_t* __restrict__ prow_off) {
  const int s = blockIdx.y, Q = blockIdx.x;
  const SubMeta m = L.meta[s];
  const int nd = m.Bc - k0 < 4 ? m.Bc - k0 : 4;
  if (Q >= nd) return;
  __shared__ float rm[NB];
  const float* sg = (const float*)L.sgn + m.vec_off + (int64_t)(k0 + Q) * NB;
  if (threadIdx.x < NB) rm[threadIdx.x] = sg[threadIdx.x] < 0.f ? 1.f : -1.f;   // -s_r
  __syncthreads();
  const int c = threadIdx.x >> 6;   // block column of X; zero above the diagonal blocks
  const float* src = c < Q    ? xinv + ((int64_t)s * 16 + Q * 4 + c) * NB2
                     : c == Q ? (const float*)L.dinv + m.dinv_off + (int64_t)(k0 + Q) * NB2
                              : nullptr;
  split_rows<4>(src, rm, prow_off[s] + k0 + Q, split, nullptr, rscale, nullptr);
}

// Persistent: CTA c takes the work items c, c + gridDim.x, ... of the panel (items of all
// subdomains flattened; item_pref[s] = first item of subdomain s).  One global step per (item,
// panel column); step g uses shared-memory stage g % 3 and TMEM accumulator pair g & 1.  Three
// roles run in their own warps: a producer thread requests the copies of each step as soon as its
// stage is free, one thread issues the MMAs as soon as a stage is full and an accumulator pair
// free (a single thread doing both waited, before every refill, for the MMAs of the previous step
// to complete: 1.7 us per step, with the copies and the tensor pipe mostly idle), and the epilogue
// warps promote the accumulators and write back each item's output block.  The write-back is a TMA reduce-add: each epilogue warp scales
// its 32 x 64 part of the block into a swizzled shared-memory box, 32 columns at a time, and one
// lane adds the box into the tiles in L2 (the output is never read into the SM; every element
// receives exactly one add per launch, so the result does not depend on timing).
__global__ void __launch_bounds__(kThreads2, 1)
    k_update_tc2(LevelDev L, int nq, int jbeg, int jend, int ibeg, int panel, const uint8_t* __restrict__ split,
                 const uint8_t* __restrict__ split_b, const float* __restrict__ rscale,
                 const int64_t* __restrict__ prow_off, const int64_t* __restrict__ item_pref,
                 const __grid_constant__ CUtensorMap tmap) {
  const int64_t n_items = item_pref[L.n_sub];
  if ((int64_t)blockIdx.x >= n_items) return;
  // nq panel tile columns (K = 64 nq) in the split rows; output columns jbeg <= j < min(Bc, jend)

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* stage0 = smem_raw + (base - raw);
  // full/free: shared-memory stage g % kStages2 loaded / read by its MMAs; mma/epi: TMEM
  // accumulator pair g & 1 written by its MMAs / read by the epilogue
  __shared__ __align__(8) uint64_t full_bar[kStages2], free_bar[kStages2], mma_bar[2], epi_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_issued, s_requested;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int b = 0; b < kStages2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&free_bar[b])));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 256;" ::"r"(smem_u32(&epi_bar[b])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_issued = 0;
    s_requested = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  // item -> (subdomain, column pair j, j+1, row pair i0, i0+1); the rows of column pair j start
  // at max(j, min(ibeg, Bc))
  auto decode = [&](int64_t it, int& s, int& j, int& i0) {
    int lo = 0, hi = (int)L.n_sub - 1;
    while (lo < hi) {   // last s with item_pref[s] <= it
      const int mid = (lo + hi + 1) >> 1;
      if (item_pref[mid] <= it) lo = mid; else hi = mid - 1;
    }
    s = lo;
    const SubMeta& m = L.meta[s];
    int64_t t = it - item_pref[s];
    const int jlim = m.Bc < jend ? m.Bc : jend;
    const int ib = ibeg < m.Bc ? ibeg : m.Bc;
    j = jbeg;
    i0 = -1;
    for (; j < jlim; j += 2) {
      const int rb = j > ib ? j : ib;
      const int cnt = (m.R - rb + 1) / 2;
      if (t < cnt) {
        i0 = rb + 2 * (int)t;
        break;
      }
      t -= cnt;
    }
  };

  // steps of this CTA: its items in order, nq panel columns each; a panel solve's B operand (rows
  // of the inverse of a lower triangular block) is zero beyond block column j - jbeg + 1, so the
  // column pair j, j + 1 takes K steps 0 .. j - jbeg + 1 only
  auto item_nq = [&](int j) { return panel ? min(nq, j - jbeg + 2) : nq; };
  const int64_t my_items = (n_items - (int64_t)blockIdx.x + gridDim.x - 1) / gridDim.x;
  uint32_t total = (uint32_t)(my_items * nq);
  if (panel && warp == 8) {
    total = 0;
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
      int cs, cj, ci0;
      decode(it, cs, cj, ci0);
      total += (uint32_t)item_nq(cj);
    }
  }
  auto wait = [&](uint64_t* bar, uint32_t parity) {
    long long spins = 0;
    while (!mbar_try_wait(bar, parity))
      if (++spins > kSpinLimit) return false;
    return true;
  };
  if (warp == 9) {
    // ---- producer: requests the B and A parts of step gc into stage gc % kStages2 once the MMAs
    // of step gc - kStages2 have read that stage (its own thread, so that waiting for a stage
    // never delays the issue of MMAs)
    if (lane == 0) {
      bool lost = false;
      int64_t cached_k = -1;
      // per item (read from global memory once, when the item changes): the four split rows and
      // the output tiles to prefetch; per step only the panel-column offset changes
      const uint8_t* rowA0 = nullptr;
      const uint8_t* rowA1 = nullptr;
      const uint8_t* rowB0 = nullptr;
      const uint8_t* rowB1 = nullptr;
      const float* pre[4] = {nullptr, nullptr, nullptr, nullptr};
      uint32_t gc = 0;
      int nqi = nq, q = 0;
      for (int64_t k = 0; k < my_items; gc += 1) {
        const int st = (int)(gc % kStages2);
        if (k != cached_k) {   // decode before waiting: the loads overlap the MMAs still reading the stage
          int cs = 0, cj = 0, ci0 = 0;
          decode(blockIdx.x + k * gridDim.x, cs, cj, ci0);
          cached_k = k;
          nqi = item_nq(cj);
          q = 0;
          const SubMeta m = L.meta[cs];
          const bool hasA1 = ci0 + 1 < m.R, hasB1 = cj + 1 < (m.Bc < jend ? m.Bc : jend);
          const int64_t rbase = prow_off[cs];
          rowA0 = split + (rbase + ci0) * kPanelTiles * (int64_t)kSplitTile;
          rowA1 = split + (rbase + (hasA1 ? ci0 + 1 : ci0)) * kPanelTiles * (int64_t)kSplitTile;
          rowB0 = split_b + (rbase + cj) * kPanelTiles * (int64_t)kSplitTile;
          rowB1 = split_b + (rbase + (hasB1 ? cj + 1 : cj)) * kPanelTiles * (int64_t)kSplitTile;
#pragma unroll
          for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const int ti = ci0 + a, tj = cj + c;
              pre[2 * a + c] = (!panel && (a == 0 || hasA1) && (c == 0 || hasB1) && (ti >= m.Bc || tj <= ti))
                                   ? (const float*)L.tiles + m.tile_off + tile_index(ti, tj, m.Bc) * NB2
                                   : nullptr;
            }
        }
        if (gc >= (uint32_t)kStages2 && !wait(&free_bar[st], ((gc / kStages2) - 1) & 1u)) {
          lost = true;
          break;
        }
        if (q == 0)   // the output tiles are read back by the epilogue after the last column
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (pre[t])
              asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(pre[t]), "r"((uint32_t)(NB2 * 4))
                           : "memory");
        uint8_t* sA = stage0 + st * kStage2;   // [A hi | A lo | B hi | B lo], 128 rows each
        uint8_t* sB = sA + 2 * kOpnd;
        mbar_expect_tx(&full_bar[st], kStage2);
        const int64_t qo = (int64_t)q * kSplitTile;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          bulk_g2s(sA + p * kOpnd, rowA0 + qo + p * kTilePart, kTilePart, &full_bar[st]);
          bulk_g2s(sA + p * kOpnd + kTilePart, rowA1 + qo + p * kTilePart, kTilePart, &full_bar[st]);
          bulk_g2s(sB + p * kOpnd, rowB0 + qo + p * kTilePart, kTilePart, &full_bar[st]);
          bulk_g2s(sB + p * kOpnd + kTilePart, rowB1 + qo + p * kTilePart, kTilePart, &full_bar[st]);
        }
        if (++q == nqi) ++k;
      }
      s_requested = (int)gc;
      if (lost) atomicExch(L.status + 2, 4);
    }
  } else if (warp == 8) {
    // ---- MMA issuer: one thread waits for the stage's data and for a free accumulator pair
    if (lane == 0) {
      // c FP32, a and b FP16, both K-major, N = 128, M = 128
      const uint32_t idesc = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
      bool lost = false;
      int issued = 0;
      for (uint32_t g = 0; g < total && !lost; ++g) {
        const int st = (int)(g % kStages2);
        const int b = (int)(g & 1u);
        if (!wait(&full_bar[st], (g / kStages2) & 1u)) {
          lost = true;
          break;
        }
        if (g >= 2 && !wait(&epi_bar[b], ((g >> 1) - 1) & 1u)) {   // accumulators of step g - 2 are read
          lost = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = smem_u32(stage0 + st * kStage2), sb = sa + 2 * kOpnd;
        const uint32_t acc_small = tmem + 256u * b, acc_big = acc_small + 128u;
        // products: (A lo, B hi), (A hi, B lo) into the small accumulator, (A hi, B hi) into the big one
        const int pa[3] = {1, 0, 0}, pb[3] = {0, 1, 0};
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t da = desc_sw128(sa + pa[p] * kOpnd + kk * 32);
            const uint64_t db = desc_sw128(sb + pb[p] * kOpnd + kk * 32);
            const bool big = p == 2;
            const uint32_t acc = (kk > 0 || (p > 0 && !big)) ? 1u : 0u;   // fresh accumulators per step
            asm volatile(
                "{\n .reg .pred pp;\n setp.ne.b32 pp, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n" ::"r"(big ? acc_big : acc_small),
                "l"(da), "l"(db), "r"(idesc), "r"(acc));
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mma_bar[b]))
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&free_bar[st]))
                     : "memory");
        ++issued;
      }
      s_issued = issued;
      if (lost) atomicExch(L.status + 2, 4);
    }
  } else {
    // ---- epilogue warps: warp w reads TMEM lanes 32 (w & 3) .. +31 (output rows) and columns
    // 64 (w >> 2) .. +63; per step hi hi + 2^-11 (cross products) is added into FP32 registers
    bool lost = false;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const uint32_t col0 = 64u * (uint32_t)(warp >> 2);
    const int erow = 32 * (warp & 3) + lane;
    uint8_t* box = stage0 + kStages2 * kStage2 + warp * kEpiBox;   // 1024-byte aligned
    uint32_t g = 0;
    for (int64_t it = blockIdx.x; it < n_items && !lost; it += gridDim.x) {
      int s, j, i0;
      decode(it, s, j, i0);
      const SubMeta& m = L.meta[s];
      float racc[64];
#pragma unroll
      for (int c = 0; c < 64; ++c) racc[c] = 0.f;
      const int nqi = item_nq(j);
      for (int q = 0; q < nqi; ++q, ++g) {
        const int b = g & 1;
        const uint32_t n = g >> 1;
        long long spins = 0;
        while (!mbar_try_wait(&mma_bar[b], n & 1u))
          if (++spins > kSpinLimit) {
            lost = true;
            break;
          }
        lost = __any_sync(0xffffffffu, lost);
        if (lost) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int c16 = 0; c16 < 4; ++c16) {
          const uint32_t taddr = tmem + lane_base + 256u * b + col0 + 16u * c16;
          uint32_t v[16], w[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(taddr));
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]),
                "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15])
              : "r"(taddr + 128u));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int c = 0; c < 16; ++c)
            racc[16 * c16 + c] += __uint_as_float(w[c]) + __uint_as_float(v[c]) * (1.f / 2048.f);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&epi_bar[b])) : "memory");
      }
      if (lost) break;
      const bool hasA1 = i0 + 1 < m.R, hasB1 = j + 1 < (m.Bc < jend ? m.Bc : jend);
      const int ti = erow < 64 ? i0 : i0 + 1;
      const int tj = col0 < 64 ? j : j + 1;
      const bool ok = (erow < 64 || hasA1) && (col0 < 64 || hasB1) && (ti >= m.Bc || tj <= ti);
      if (ok) {   // warp-uniform: the warp's 32 rows and 64 columns lie in one output tile
        const int64_t rbase = prow_off[s];
        // negated row factor: the tiles receive x + (-(acc sa) f), which equals x - (acc sa) f
        const float sa = -rscale[(rbase + ti) * NB + (erow & 63)];
        const float4* sb = (const float4*)(rscale + (rbase + tj) * NB);
        // row of the warp's first output row in the [rows][64] view of the tile buffer
        const int y = (int)((m.tile_off + tile_index(ti, tj, m.Bc) * NB2) / NB) + (32 * (warp & 3) & 63);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          // the previous reduce-add out of this warp's box has read it
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          __syncwarp();
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int u = 8 * hh + k;
            const float4 f = __ldg(sb + u);   // both factors are powers of two: the products are exact
            float4 x;
            x.x = (racc[4 * u + 0] * sa) * f.x;
            x.y = (racc[4 * u + 1] * sa) * f.y;
            x.z = (racc[4 * u + 2] * sa) * f.z;
            x.w = (racc[4 * u + 3] * sa) * f.w;
            // 128-byte swizzle: 16-byte chunk k of box row r sits at chunk k ^ (r & 7)
            *(float4*)(box + lane * 128 + ((k ^ (lane & 7)) << 4)) = x;
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) {
            if (panel)   // a panel solve writes its tiles (their old contents are the split A operand)
              asm volatile(
                  "cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                      (uint64_t)&tmap),
                  "r"(32 * hh), "r"(y), "r"(smem_u32(box))
                  : "memory");
            else
              asm volatile(
                  "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                      (uint64_t)&tmap),
                  "r"(32 * hh), "r"(y), "r"(smem_u32(box))
                  : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          }
        }
      }
    }
    // the reduce-adds are complete (and the boxes free) before the CTA ends, also on the error path
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (lost && lane == 0) atomicExch(L.status + 2, 4);
  }
  __syncthreads();
  // copies requested but never consumed (a wait gave up) may still be landing in shared memory:
  // wait (bounded) for them before the CTA exits
  if (tid == 0)
    for (int c = s_issued; c < s_requested; ++c) {
      long long spins = 0;
      while (!mbar_try_wait(&full_bar[c % kStages2], (uint32_t)(c / kStages2) & 1u) && ++spins < kSpinLimit) {
      }
    }
  // before the accumulators are released no MMA may still be running (also on the error path)
  const int issued = s_issued;
  if (issued > 0) {
    const int b = (issued - 1) & 1;
    const uint32_t n = (uint32_t)((issued - 1) >> 1);
    long long spins = 0;
    while (!mbar_try_wait(&mma_bar[b], n & 1u))
      if (++spins > kSpinLimit) break;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

}  // namespace

void launch_split_panel(const LevelDev& L, int kb0, int nt, int ib, int max_R, uint8_t* split, uint8_t* split_signed,
                        float* rscale, const int64_t* prow_off, cudaStream_t st, int panel_operand) {
  const int first = panel_operand ? kb0 + 1 : ib;   // the rows of a panel operand start after kb0
  if (L.n_sub <= 0 || max_R <= first) return;
  note_launch();
  const dim3 grid((unsigned)(max_R - first), (unsigned)L.n_sub);
  if (nt == 8)
    k_split_panel<8><<<grid, 512, 0, st>>>(L, kb0, ib, panel_operand, split, split_signed, rscale, prow_off);
  else
    k_split_panel<4><<<grid, 256, 0, st>>>(L, kb0, ib, panel_operand, split, split_signed, rscale, prow_off);
}

void launch_split_inverse(const LevelDev& L, int k0, const float* xinv, uint8_t* split, float* rscale,
                          const int64_t* prow_off, cudaStream_t st) {
  if (L.n_sub <= 0) return;
  note_launch();
  k_split_inverse<<<dim3(4, (unsigned)L.n_sub), 256, 0, st>>>(L, k0, xinv, split, rscale, prow_off);
}

void launch_update_tc2(const LevelDev& L, int nq, int jbeg, int jend, int ibeg, int panel, int grid, const uint8_t* split,
                       const uint8_t* split_b, const float* rscale, const int64_t* prow_off,
                       const int64_t* item_pref, const TensorMap128& tmap, cudaStream_t st) {
  if (grid <= 0 || L.n_sub <= 0 || nq <= 0 || nq > kPanelTiles) return;
  const size_t dyn = kStages2 * kStage2 + 8 * kEpiBox + 1024;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_update_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    attr = true;
  }
  note_launch();
  CUtensorMap m;
  static_assert(sizeof(CUtensorMap) == sizeof(TensorMap128), "tensor map size");
  std::memcpy(&m, &tmap, sizeof(m));
  k_update_tc2<<<(unsigned)grid, kThreads2, dyn, st>>>(L, nq, jbeg, jend, ibeg, panel, split, split_b, rscale, prow_off,
                                                        item_pref, m);
}

int make_tile_tmap(TensorMap128* map, float* tiles, int64_t tile_elems) {
  using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeTiled encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return (int)CUDA_ERROR_NOT_FOUND;
    encode = (EncodeTiled)fn;
  }
  const int64_t rows = tile_elems / NB;
  if (rows <= 0 || rows >= ((int64_t)1 << 31)) return (int)CUDA_ERROR_INVALID_VALUE;   // int32 box coordinates
  const cuuint64_t dims[2] = {(cuuint64_t)NB, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)NB * sizeof(float)};
  const cuuint32_t box[2] = {32, 32};
  const cuuint32_t estr[2] = {1, 1};
  CUtensorMap m;
  const CUresult r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, tiles, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return (int)r;
  std::memcpy(map, &m, sizeof(m));
  return 0;
}

}  // namespace bddc
