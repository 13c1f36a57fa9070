// Trailing update of the blocked Cholesky on the 5th-generation tensor cores (tcgen05), FP32
// factors (mixed mode): for one super-panel of up to W = 4 tile columns q in [kb0, kb1),
//     A(i, j) -= sum_q L(i, q) S_q L(j, q)^T       for kb1 <= j < Bc, j <= i < R,
// (S_q: pivot signs of the signed Cholesky, identity for SPD levels)
// batched over all subdomains of a level.  This is the rank-256 update that follows the
// factorisation of a 256-wide panel (Algorithm 1, "factorize the matrices of local saddle
// point problems").
//
// FP32 accuracy from BF16 tensor cores: every FP32 operand is split into three BF16 parts
// a = a0 + a1 + a2 (each the BF16 rounding of what remains), and six products
// a0b0 + a0b1 + a1b0 + a0b2 + a1b1 + a2b0 are accumulated in FP32 in tensor memory
// (the bf16x3 scheme of Henry, Tang and Heinecke, ARITH 2019).  Accuracy of the tensor-core
// accumulation, measured on GB300 against FP64 for K = 256: one accumulator for all six
// products 2.0e-6, the dominant a0b0 in its own accumulator 1.9e-7, and in addition promoting
// both partial sums to FP32 registers after every 64-wide K chunk 7.7e-8 (FP32 FMA: 1.5e-7).
// The kernel uses the last scheme: per chunk, fresh accumulators (small products in TMEM
// columns [0, 64), a0b0 in [64, 128)) are read back and added in FP32.
//
// One CTA (256 threads) per output pair of tiles (i0, j), (i0+1, j): M = 128 rows, N = 64
// columns.  Per tile column q the CTA loads the three FP32 tiles, splits them into BF16
// parts stored K-major with the 128-byte swizzle, and one thread issues 24 MMAs
// (6 products x 4 K-steps of 16) into two 128 x 64 FP32 accumulators in TMEM; tcgen05.commit
// signals an mbarrier when the shared-memory operands may be reused.  The epilogue reads the
// accumulator with tcgen05.ld and subtracts it from the tiles in global memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace bddc {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kPartA = 128 * 128;   // bytes of one BF16 part of A (128 rows x 64)
constexpr uint32_t kPartB = 64 * 128;    // bytes of one BF16 part of B (64 rows x 64)
constexpr uint32_t kStage = 3 * kPartA + 3 * kPartB;
constexpr long long kSpinLimit = 1ll << 26;

__device__ __forceinline__ int64_t tile_index(int i, int j, int Bc) {
  return i < Bc ? ((int64_t)i * (i + 1) / 2 + j) : ((int64_t)Bc * (Bc + 1) / 2 + (int64_t)(i - Bc) * Bc + j);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major operand, 128-byte swizzle: rows of 64 BF16 (128 B), 8-row atoms of 1024 B
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);   // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  return (uint32_t)(r * 128 + (((k >> 3) ^ (r & 7)) << 4) + (k & 7) * 2);
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

__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  x -= __bfloat162float(a);
  b = __float2bfloat16_rn(x);
  x -= __bfloat162float(b);
  c = __float2bfloat16_rn(x);
}

__device__ __forceinline__ void store4(uint8_t* part, uint32_t off, __nv_bfloat16 a, __nv_bfloat16 b,
                                       __nv_bfloat16 c, __nv_bfloat16 d) {
  __nv_bfloat162 lo, hi;
  lo.x = a;
  lo.y = b;
  hi.x = c;
  hi.y = d;
  uint2 v;
  v.x = *(uint32_t*)&lo;
  v.y = *(uint32_t*)&hi;
  *(uint2*)(part + off) = v;
}

__global__ void __launch_bounds__(kThreads, 2)
    k_update_tc(LevelDev L, int kb0, int kb1) {
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  // work item -> (column j, row pair i0)
  int t = blockIdx.x, j = kb1, i0 = -1;
  for (; j < m.Bc; ++j) {
    const int cnt = (m.R - j + 1) / 2;
    if (t < cnt) {
      i0 = j + 2 * t;
      break;
    }
    t -= cnt;
  }
  if (i0 < 0 || kb0 >= m.Bc) return;
  const int qend = kb1 < m.Bc ? kb1 : m.Bc;
  const bool has1 = i0 + 1 < m.R;

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;   // swizzle atoms need 1024-byte alignment
  uint8_t* sA = smem_raw + (base - raw);
  uint8_t* sB = sA + 3 * kPartA;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const float* tiles = (const float*)L.tiles + m.tile_off;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
  bool lost = false;

  // registers: 12 float4 per thread = tiles (i0,q), (i0+1,q), (j,q)
  float4 rg[12];
  auto load_chunk = [&](int q) {
    const float4* a0 = (const float4*)(tiles + tile_index(i0, q, m.Bc) * NB2);
    const float4* a1 = has1 ? (const float4*)(tiles + tile_index(i0 + 1, q, m.Bc) * NB2) : nullptr;
    const float4* b = (const float4*)(tiles + tile_index(j, q, m.Bc) * NB2);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      rg[u] = __ldcg(a0 + tid + 256 * u);
      rg[4 + u] = has1 ? __ldcg(a1 + tid + 256 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
      rg[8 + u] = __ldcg(b + tid + 256 * u);
    }
  };
  // FP32 running sums of this thread's output row (TMEM lane) and 32 columns
  const int erow = 32 * (warp & 3) + lane;
  const int ec0 = 32 * (warp >> 2);
  float racc[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) racc[c] = 0.f;
  // wait for the MMAs of the last chunk, then add both TMEM partial sums into racc
  uint32_t phase = 0;
  auto promote = [&]() {
    long long spins = 0;
    while (!mbar_try_wait(&bar, phase & 1u)) {
      if (++spins > kSpinLimit) {
        lost = true;
        break;
      }
    }
    ++phase;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)ec0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t v[16], w[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr + 16u * h));
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]),
            "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15])
          : "r"(taddr + 64u + 16u * h));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int c = 0; c < 16; ++c) racc[16 * h + c] += __uint_as_float(w[c]) + __uint_as_float(v[c]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  };
  load_chunk(kb0);
  for (int q = kb0; q < qend; ++q) {
    if (q > kb0) promote();   // also frees the shared-memory stage and the accumulators
    const float* sq = (const float*)L.sgn + m.vec_off + (int64_t)q * NB;   // pivot signs of column q
#pragma unroll
    for (int u = 0; u < 12; ++u) {
      const int f = tid + 256 * (u & 3);        // float4 index inside the tile
      const int r = (f * 4) / NB, k = (f * 4) % NB;
      if (u >= 8 && L.indefinite) {             // B = L(j,q) S_q
        rg[u].x *= sq[k];
        rg[u].y *= sq[k + 1];
        rg[u].z *= sq[k + 2];
        rg[u].w *= sq[k + 3];
      }
      __nv_bfloat16 p0[4], p1[4], p2[4];
      split3(rg[u].x, p0[0], p1[0], p2[0]);
      split3(rg[u].y, p0[1], p1[1], p2[1]);
      split3(rg[u].z, p0[2], p1[2], p2[2]);
      split3(rg[u].w, p0[3], p1[3], p2[3]);
      if (u < 8) {
        const uint32_t off = sw128_off(r + (u >= 4 ? 64 : 0), k);
        store4(sA, off, p0[0], p0[1], p0[2], p0[3]);
        store4(sA + kPartA, off, p1[0], p1[1], p1[2], p1[3]);
        store4(sA + 2 * kPartA, off, p2[0], p2[1], p2[2], p2[3]);
      } else {
        const uint32_t off = sw128_off(r, k);
        store4(sB, off, p0[0], p0[1], p0[2], p0[3]);
        store4(sB + kPartB, off, p1[0], p1[1], p1[2], p1[3]);
        store4(sB + 2 * kPartB, off, p2[0], p2[1], p2[2], p2[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // small products into columns [0, 64), the dominant a0 b0 into columns [64, 128)
      const int pa[6] = {2, 1, 0, 1, 0, 0}, pb[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
      for (int p = 0; p < 6; ++p)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t da = desc_sw128(base + pa[p] * kPartA + kk * 32);
          const uint64_t db = desc_sw128(base + 3 * kPartA + pb[p] * kPartB + kk * 32);
          const bool big = p == 5;
          const uint32_t acc = (kk > 0 || (p > 0 && !big)) ? 1u : 0u;   // fresh accumulators per chunk
          asm volatile(
              "{\n .reg .pred pp;\n setp.ne.b32 pp, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n" ::"r"(tmem + (big ? 64u : 0u)),
              "l"(da), "l"(db), "r"(idesc), "r"(acc));
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar))
                   : "memory");
    }
    if (q + 1 < qend) load_chunk(q + 1);   // overlaps with the MMAs just issued
  }
  promote();
  if (lost && lane == 0) atomicExch(L.status + 2, 3);
  // epilogue: subtract the update from the output tiles
  {
    const int ti = erow < 64 ? i0 : i0 + 1;
    if (erow < 64 || has1) {
      float* c = (float*)L.tiles + m.tile_off + tile_index(ti, j, m.Bc) * NB2 + (erow & 63) * NB + ec0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float4 x = *(float4*)(c + 4 * u);
        x.x -= racc[4 * u + 0];
        x.y -= racc[4 * u + 1];
        x.z -= racc[4 * u + 2];
        x.w -= racc[4 * u + 3];
        *(float4*)(c + 4 * u) = x;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

}  // namespace

void launch_update_tc(const LevelDev& L, int kb0, int kb1, int max_items, cudaStream_t st) {
  if (max_items <= 0 || L.n_sub <= 0) return;
  const size_t dyn = kStage + 1024;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    attr = true;
  }
  note_launch();
  k_update_tc<<<dim3((unsigned)max_items, (unsigned)L.n_sub), kThreads, dyn, st>>>(L, kb0, kb1);
}

}  // namespace bddc
