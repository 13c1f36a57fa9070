// Streaming triangular sweeps with the tiled factors, batched over all subdomains of a level:
// forward y = S L^{-1} b and backward L^T x = y over the interior block rows (the discrete
// Dirichlet problems of the Schur operator, Sec. 2) or over the interface block rows (the
// constrained Neumann problem of Eq. sub_cor, restricted to the interface).  S holds the pivot
// signs of the signed Cholesky (identity for SPD levels), so the pair solves L S L^T x = b.
//
// Design (GB300): the sweep is bound by reading the factor from HBM once.  A persistent grid
// of 2 CTAs per SM takes block-row tasks (subdomain s, block row i) from a global counter in
// dependency order (all subdomains' first rows, then their second rows, ...).  A task
// streams its row of NB x NB tiles (forward) or its column of tiles (backward) into a ring of
// shared-memory stages with cp.async.bulk, completion tracked by mbarriers, while the solution
// blocks it depends on are published by other CTAs in a publication buffer that is filled with
// all-ones words before the launch: a block is ready when none of its words is all-ones any
// more (every word is written once, atomically, and no arithmetic result has that NaN bit
// pattern: NaN results are canonical, and a computed all-ones word is published as the
// canonical NaN).  The consumer polls the data itself, one L2 round trip instead of a flag
// acquire followed by the data load, and the producer needs no fence.  A task only waits for
// tasks handed out before it, so the scheme cannot deadlock whatever the residency.  Every wait
// is bounded; a timeout sets status[2] and the kernel finishes without waiting further (the host
// reports BDDC_ERR_TIMEOUT).  A wait for a published block that gives up stages the block as it
// is and goes on, so every tile copy is still consumed and no access leaves the task's own rows;
// a tile wait that gives up drains the ring before exit.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace bddc {

namespace {

constexpr int kThreads = 256;
constexpr int kYSlots = 16;          // solution blocks staged in shared memory at a time
constexpr long long kSpinLimit = 1ll << 24;
constexpr long long kProbeSpins = 32;   // publication wait limit of the timeout probe

__device__ __forceinline__ int64_t tile_index(int i, int j, int Bc) {
  return i < Bc ? ((int64_t)i * (i + 1) / 2 + j) : ((int64_t)Bc * (Bc + 1) / 2 + (int64_t)(i - Bc) * Bc + j);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
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

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// publication words: relaxed (coherent at L2) loads and stores; all-ones = not yet written
__device__ __forceinline__ bool pub_ld2(const float* p, float2& v) {
  uint32_t a, b;
  asm volatile("ld.relaxed.gpu.global.v2.b32 {%0, %1}, [%2];" : "=r"(a), "=r"(b) : "l"(p) : "memory");
  v = make_float2(__uint_as_float(a), __uint_as_float(b));
  return a != 0xFFFFFFFFu && b != 0xFFFFFFFFu;
}
__device__ __forceinline__ bool pub_ld2(const double* p, double2& v) {
  unsigned long long a, b;
  asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
  v = make_double2(__longlong_as_double((long long)a), __longlong_as_double((long long)b));
  return a != ~0ull && b != ~0ull;
}
__device__ __forceinline__ void pub_st(float* p, float x) {
  uint32_t a = __float_as_uint(x);
  if (a == 0xFFFFFFFFu) a = 0x7FFFFFFFu;
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(a) : "memory");
}
__device__ __forceinline__ void pub_st(double* p, double x) {
  unsigned long long a = (unsigned long long)__double_as_longlong(x);
  if (a == ~0ull) a = 0x7FFFFFFFFFFFFFFFull;
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(a) : "memory");
}

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

// One task: (subdomain, block row).  Forward consumes tiles (i, B0..i-1) then D_i^{-1};
// backward consumes tiles (B1-1..i+1, i) then D_i^{-1}.  NR right-hand sides are solved together
// (column r at vec + r * vstride): every factor tile is streamed from HBM once per task and
// applied to all of them from shared memory.
template <typename T, int S, bool BWD, int NR>
__global__ void __launch_bounds__(kThreads, 2)
    k_sweep(LevelDev L, T* __restrict__ vec, int64_t vstride, const int2* __restrict__ tasks, int ntasks, int part,
            int* __restrict__ ctrl, T* pub) {
  using V2 = typename Vec2<T>::type;
  constexpr int YS = NR == 1 ? kYSlots : (NR == 2 ? 8 : 4);   // solution blocks staged at a time
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* stage = (T*)smem_raw;                       // S tiles of NB*NB
  __shared__ __align__(8) uint64_t full[S];
  __shared__ __align__(16) T ybuf[YS][NR][NB];
  __shared__ T red[kThreads / 32][NR][NB];
  __shared__ __align__(16) T rhs[NR][NB];
  __shared__ T s_sg[NB];                         // pivot signs of the task's block row (indefinite)
  __shared__ int s_task;
  __shared__ int s_rdy[kYSlots];                 // poll result per candidate block
  int* counter = ctrl;
  int* status = L.status;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int k = 0; k < S; ++k) mbar_init(&full[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t cons = 0;     // tiles consumed by this CTA (ring position and phase)
  uint32_t issued = 0;   // tiles issued (thread 0)
  bool lost = false;     // a tile wait gave up: drain before exit
  for (;;) {
    if (tid == 0) s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_task;
    if (t >= ntasks) break;
    const int sub = tasks[t].x, i = tasks[t].y;
    const SubMeta m = L.meta[sub];
    if (!BWD && L.indefinite && tid < NB) s_sg[tid] = ((const T*)L.sgn)[m.vec_off + (int64_t)i * NB + tid];
    // interior part: the block rows that hold interior DOFs (padding identity block rows, whose
    // rows and columns of L are unit vectors and whose right-hand sides are zero, are skipped)
    const int B0 = part == 0 ? 0 : m.nIb, B1 = part == 0 ? (m.nI + NB - 1) / NB : m.Bc;
    const int nL = BWD ? (B1 - 1 - i) : (i - B0);   // factor tiles before D_i^{-1}
    const int ntile = nL + 1;
    const T* tiles = (const T*)L.tiles + m.tile_off;
    const T* dinv = (const T*)L.dinv + m.dinv_off + (int64_t)i * NB2;
    T* v = vec + m.vec_off;
    T* pv = pub + m.vec_off;   // this subdomain's published blocks (same layout as v)
    auto tile_src = [&](int k) -> const T* {
      if (k == nL) return dinv;
      const int j = BWD ? (B1 - 1 - k) : (B0 + k);
      return BWD ? tiles + tile_index(j, i, m.Bc) * NB2 : tiles + tile_index(i, j, m.Bc) * NB2;
    };
    // the task's own right-hand side block depends on no other task: read it into rhs now, off
    // the chain of dependent rows (the diagonal step subtracts the updates in place)
    for (int e = tid; e < NR * NB; e += kThreads) rhs[e / NB][e % NB] = __ldcg(v + (e / NB) * vstride + i * NB + e % NB);
    __syncthreads();
    // prologue: fill the ring
    if (tid == 0) {
      const int pre = ntile < S ? ntile : S;
      for (int k = 0; k < pre; ++k) {
        const uint32_t slot = (cons + k) % S;
        mbar_expect_tx(&full[slot], (uint32_t)(NB2 * sizeof(T)));
        bulk_g2s(stage + slot * NB2, tile_src(k), (uint32_t)(NB2 * sizeof(T)), &full[slot]);
      }
      issued += pre;
    }
    T acc[8][NR];        // forward: rows warp + 8 r, this lane's two columns, every right-hand side
    T accc[NR][2];       // backward: this lane's two columns, summed over the warp's rows
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[r][q] = (T)0;
#pragma unroll
    for (int q = 0; q < NR; ++q) accc[q][0] = accc[q][1] = (T)0;
    int staged_end = 0;   // tiles [staged_begin, staged_end) have their solution block in ybuf
    for (int k = 0; k < ntile; ++k) {
      if (k < nL && k >= staged_end) {
        // wait until the next solution blocks are published, then stage up to YS of them: warp w
        // polls blocks k + w and k + w + 8 (all their words at once), writes the ready ones into
        // ybuf, and the consecutive ready blocks from k are staged
        const int want = nL - k < YS ? nL - k : YS;
        int cnt = 0;
        long long spins = 0;
        for (;;) {
          __syncthreads();   // every thread has read s_rdy of the previous poll
          for (int b = warp; b < want; b += kThreads / 32) {
            const int j = BWD ? (B1 - 1 - (k + b)) : (B0 + k + b);
            V2 y[NR];
            bool ok = true;
#pragma unroll
            for (int q = 0; q < NR; ++q) ok &= pub_ld2(pv + q * vstride + j * NB + 2 * lane, y[q]);
            // the timeout probe waits for a word that nothing sets (status[3]) instead
            if (L.wait_probe) ok = ld_acquire(status + 3) != 0;
            ok = __all_sync(0xffffffffu, ok);
            if (ok) {
              V2 sg = {(T)1, (T)1};
              if (!BWD && L.indefinite)   // solved rows hold S_j y_j: the update needs y_j
                sg = *(const V2*)((const T*)L.sgn + m.vec_off + (int64_t)j * NB + 2 * lane);
#pragma unroll
              for (int q = 0; q < NR; ++q) {
                y[q].x *= sg.x;
                y[q].y *= sg.y;
                *(V2*)&ybuf[(k + b) % YS][q][2 * lane] = y[q];
              }
            }
            if (lane == 0) s_rdy[b] = ok ? 1 : 0;
          }
          __syncthreads();
          cnt = 0;
          while (cnt < want && s_rdy[cnt]) ++cnt;
          if (cnt > 0) break;
          if (++spins > (L.wait_probe ? kProbeSpins : kSpinLimit)) {
            if (tid == 0) atomicExch(status + 2, 1);
            cnt = 1;   // stage the block as it is and go on (error path)
            break;
          }
          __nanosleep(64);
        }
        staged_end = k + cnt;
      }
      // wait for the tile
      const uint32_t slot = cons % S, parity = (cons / S) & 1u;
      {
        long long spins = 0;
        while (!mbar_try_wait(&full[slot], parity)) {
          if (++spins > kSpinLimit) {
            if (tid == 0) atomicExch(status + 2, 2);
            lost = true;
            break;
          }
        }
      }
      const T* tl = stage + slot * NB2;
      if (k < nL) {
        const int ys = k % YS;
        if (!BWD) {
          V2 a[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) a[r] = *(const V2*)(tl + (warp + 8 * r) * NB + 2 * lane);
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            const V2 yv = *(const V2*)(&ybuf[ys][q][2 * lane]);
#pragma unroll
            for (int r = 0; r < 8; ++r) acc[r][q] += a[r].x * yv.x + a[r].y * yv.y;
          }
        } else {
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int row = warp + 8 * r;
            const V2 a = *(const V2*)(tl + row * NB + 2 * lane);
#pragma unroll
            for (int q = 0; q < NR; ++q) {
              const T x = ybuf[ys][q][row];
              accc[q][0] += a.x * x;
              accc[q][1] += a.y * x;
            }
          }
        }
      } else {
        // diagonal block: right-hand side, then D_i^{-1} (forward) or D_i^{-T} (backward)
        if (!BWD) {
#pragma unroll
          for (int q = 0; q < NR; ++q)
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              T a = acc[r][q];
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
              if (lane == 0) rhs[q][warp + 8 * r] -= a;
            }
          __syncthreads();
          const bool signed_rows = L.indefinite != 0;   // forward output is S L^{-1} b
          V2 a[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) a[r] = *(const V2*)(tl + (warp + 8 * r) * NB + 2 * lane);
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            const V2 rv = *(const V2*)(&rhs[q][2 * lane]);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              T yv = a[r].x * rv.x + a[r].y * rv.y;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) yv += __shfl_xor_sync(0xffffffffu, yv, o);
              if (lane == 0) {
                const T out = signed_rows ? yv * s_sg[warp + 8 * r] : yv;
                v[q * vstride + i * NB + warp + 8 * r] = out;
                pub_st(pv + q * vstride + i * NB + warp + 8 * r, out);
              }
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            red[warp][q][2 * lane] = accc[q][0];
            red[warp][q][2 * lane + 1] = accc[q][1];
          }
          __syncthreads();
          for (int e = tid; e < NR * NB; e += kThreads) {
            const int q = e / NB, c = e % NB;
            T a = (T)0;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) a += red[w][q][c];
            rhs[q][c] -= a;
          }
          __syncthreads();
          T p[NR][2];
#pragma unroll
          for (int q = 0; q < NR; ++q) p[q][0] = p[q][1] = (T)0;
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int row = warp + 8 * r;
            const V2 a = *(const V2*)(tl + row * NB + 2 * lane);
#pragma unroll
            for (int q = 0; q < NR; ++q) {
              p[q][0] += a.x * rhs[q][row];
              p[q][1] += a.y * rhs[q][row];
            }
          }
          __syncthreads();
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            red[warp][q][2 * lane] = p[q][0];
            red[warp][q][2 * lane + 1] = p[q][1];
          }
          __syncthreads();
          for (int e = tid; e < NR * NB; e += kThreads) {
            const int q = e / NB, c = e % NB;
            T a = (T)0;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) a += red[w][q][c];
            v[q * vstride + i * NB + c] = a;
            pub_st(pv + q * vstride + i * NB + c, a);
          }
        }
      }
      __syncthreads();   // every thread is done with this stage
      ++cons;
      if (tid == 0 && k + S < ntile) {
        const uint32_t ns = (cons + S - 1) % S;   // the slot just released
        mbar_expect_tx(&full[ns], (uint32_t)(NB2 * sizeof(T)));
        bulk_g2s(stage + ns * NB2, tile_src(k + S), (uint32_t)(NB2 * sizeof(T)), &full[ns]);
        ++issued;
      }
    }
  }
  // After a lost tile wait, copies may still be in flight into this CTA's shared memory:
  // wait (bounded) for the last phase issued on every slot before the CTA exits.
  if (tid == 0 && lost) {
    for (uint32_t c = (issued > (uint32_t)S ? issued - S : 0u); c < issued; ++c) {
      long long spins = 0;
      while (!mbar_try_wait(&full[c % S], (c / S) & 1u) && ++spins < kSpinLimit) {
      }
    }
  }
}

}  // namespace

// Task lists, control words and the publication buffer live in the level (see capi.cpp); this
// entry launches one sweep.  ctrl[0] (the task counter) must be zero and pub all-ones over the
// columns of the launch (memsets in the stream).
template <typename T, int S, int NR>
void launch_sweep_s(const LevelDev& L, T* vec, const int2* tasks, int ntasks, int part, int backward, int* ctrl,
                    T* pub, int grid, cudaStream_t st) {
  const size_t dyn = (size_t)S * NB2 * sizeof(T);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_sweep<T, S, false, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    cudaFuncSetAttribute(k_sweep<T, S, true, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    attr = true;
  }
  cudaMemsetAsync(ctrl, 0, sizeof(int), st);
  cudaMemsetAsync(pub, 0xFF, sizeof(T) * (size_t)L.n_vec * NR, st);
  note_launch();
  if (backward)
    k_sweep<T, S, true, NR><<<grid, kThreads, dyn, st>>>(L, vec, L.n_vec, tasks, ntasks, part, ctrl, pub);
  else
    k_sweep<T, S, false, NR><<<grid, kThreads, dyn, st>>>(L, vec, L.n_vec, tasks, ntasks, part, ctrl, pub);
}

template <typename T, int S>
void launch_sweep_nr(const LevelDev& L, T* vec, const int2* tasks, int ntasks, int part, int backward, int* ctrl,
                     T* pub, int grid, int nr, cudaStream_t st) {
  // right-hand sides in groups of up to 8 (FP32) / 4 (FP64), each group one launch over the factor
  constexpr int kMaxNR = sizeof(T) == 4 ? 8 : 4;
  for (int r0 = 0; r0 < nr;) {
    const int left = nr - r0;
    const int g = left >= kMaxNR ? kMaxNR : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    T* v = vec + (int64_t)r0 * L.n_vec;
    if (g == 8)
      launch_sweep_s<T, S, (sizeof(T) == 4 ? 8 : 4)>(L, v, tasks, ntasks, part, backward, ctrl, pub, grid, st);
    else if (g == 4)
      launch_sweep_s<T, S, 4>(L, v, tasks, ntasks, part, backward, ctrl, pub, grid, st);
    else if (g == 2)
      launch_sweep_s<T, S, 2>(L, v, tasks, ntasks, part, backward, ctrl, pub, grid, st);
    else
      launch_sweep_s<T, S, 1>(L, v, tasks, ntasks, part, backward, ctrl, pub, grid, st);
    r0 += g;
  }
}

// deep: the longer tile ring (FP32: 6 stages, FP64: 3); shallow: FP32 4, FP64 2.  nr columns of
// length n_vec at vec; pub holds min(nr, 8) such columns of T.
template <typename T>
void launch_sweep(const LevelDev& L, T* vec, const int2* tasks, int ntasks, int part, int backward, int* ctrl,
                  void* pub, int grid_max, int deep, cudaStream_t st, int nr) {
  if (ntasks <= 0 || nr <= 0) return;
  T* pb = (T*)pub;
  const int grid = ntasks < grid_max ? ntasks : grid_max;
  if (sizeof(T) == 4) {
    if (deep)
      launch_sweep_nr<T, 6>(L, vec, tasks, ntasks, part, backward, ctrl, pb, grid, nr, st);
    else
      launch_sweep_nr<T, 4>(L, vec, tasks, ntasks, part, backward, ctrl, pb, grid, nr, st);
  } else {
    if (deep)
      launch_sweep_nr<T, 3>(L, vec, tasks, ntasks, part, backward, ctrl, pb, grid, nr, st);
    else
      launch_sweep_nr<T, 2>(L, vec, tasks, ntasks, part, backward, ctrl, pb, grid, nr, st);
  }
}

template void launch_sweep<float>(const LevelDev&, float*, const int2*, int, int, int, int*, void*, int, int,
                                  cudaStream_t, int);
template void launch_sweep<double>(const LevelDev&, double*, const int2*, int, int, int, int*, void*, int, int,
                                   cudaStream_t, int);

}  // namespace bddc
