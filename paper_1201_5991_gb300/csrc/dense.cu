// Dense per-subdomain kernels, batched over all subdomains of a level.
//
//  * Partial Cholesky of the augmented matrix [A_i; C_i], A_i = K_i + rho C_i^T C_i
//    (right-looking, NB x NB tiles): gives L_i (A_i = L_i L_i^T) and Y_i = C_i L_i^{-T}.
//    With the local order (interior, interface) the leading block of L_i factors K_II
//    ("prepare interior correction", Algorithm 1) and the trailing block factors the
//    constrained Neumann problem of Eq. psi_def / Eq. sub_cor restricted to the interface.
//  * G_i = Y_i Y_i^T = C_i A_i^{-1} C_i^T (FP64), its Cholesky factor and inverse;
//    Psi_i = A_i^{-1} C_i^T G_i^{-1} (so C_i Psi_i = I and K_i Psi_i = -C_i^T Lambda_i with
//    Lambda_i = R - G_i^{-1}), K_Ci = Psi_i^T K_i Psi_i = -Lambda_i = G_i^{-1} - R, where
//    R = diag(rho c_rho) (rho on the rows that augment A_i, 0 on Stokes pressure rows).
#include "internal.h"

namespace bddc {

namespace {

__device__ __forceinline__ int64_t tile_index(int i, int j, int Bc) {
  return i < Bc ? ((int64_t)i * (i + 1) / 2 + j) : ((int64_t)Bc * (Bc + 1) / 2 + (int64_t)(i - Bc) * Bc + j);
}

template <typename T>
__device__ __forceinline__ T* tile_ptr(const SubMeta& m, void* base, int i, int j) {
  return (T*)base + m.tile_off + tile_index(i, j, m.Bc) * NB2;
}

__device__ __forceinline__ void flag_breakdown(int* status, int sub) {
  atomicExch(status + 0, 1);
  atomicMin(status + 1, sub);
}

constexpr int LDS = NB + 4;   // k-major shared tile stride (multiple of 4 for vector loads)

template <typename T>
__device__ __forceinline__ void load_kmajor(T* s, const T* __restrict__ g) {
  // s[m * LDS + r] = g[r * NB + m]
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int r = t / NB, m = t % NB;
    s[m * LDS + r] = g[t];
  }
}

// 16-byte aligned vectors of four entries (global or shared memory)
template <typename T>
__device__ __forceinline__ void load4(T (&v)[4], const T* p);
template <>
__device__ __forceinline__ void load4<float>(float (&v)[4], const float* p) {
  const float4 a = *(const float4*)p;
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
template <>
__device__ __forceinline__ void load4<double>(double (&v)[4], const double* p) {
  const double2 a = *(const double2*)p, b = *(const double2*)(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}
template <typename T>
__device__ __forceinline__ void store4(T* p, const T (&v)[4]);
template <>
__device__ __forceinline__ void store4<float>(float* p, const float (&v)[4]) {
  *(float4*)p = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store4<double>(double* p, const double (&v)[4]) {
  *(double2*)p = make_double2(v[0], v[1]);
  *(double2*)(p + 2) = make_double2(v[2], v[3]);
}

// acc[i][j] += sum_m A[4ty+i][m] * B[4tx+j][m] with both operands k-major in shared memory
template <typename T>
__device__ __forceinline__ void gemm_nt_4x4(const T* As, const T* Bs, T acc[4][4], int tx, int ty) {
#pragma unroll 8
  for (int m = 0; m < NB; ++m) {
    T a[4], b[4];
    load4(a, As + m * LDS + 4 * ty);   // LDS and the tile offsets keep these 16-byte aligned
    load4(b, Bs + m * LDS + 4 * tx);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
  }
}

// ---- step k, part 1: factor the diagonal tile and invert it -------------------------------
// One CTA of 256 threads; smem_raw holds 2 NB (NB + 1) entries of T.  Called by k_potrf_diag and,
// for the next block column of a panel, by the in-panel update kernel right after it has updated
// that diagonal tile (so that the factorisation of a panel's later diagonal tiles overlaps the
// rest of the previous step's update instead of taking a launch of its own).
template <typename T>
__device__ void factor_diag_tile(const LevelDev& L, const SubMeta& m, int s, int k, unsigned char* smem_raw) {
  T(*A)[NB + 1] = (T(*)[NB + 1])smem_raw;                 // the tile, then its factor L
  T(*X)[NB + 1] = (T(*)[NB + 1])(smem_raw + sizeof(T) * NB * (NB + 1));   // L^{-1}
  __shared__ int bad;
  T* g = tile_ptr<T>(m, L.tiles, k, k);
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int r = t / NB, c = t % NB;
    A[r][c] = c <= r ? g[t] : (T)0;
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  __shared__ T sg[NB];
  __shared__ T dd[NB];   // pivots as used by the elimination (1 where a pivot failed)
  // Right-looking elimination on the unscaled columns: at column j every entry below the pivot
  // is updated as a_ic -= (a_ij / d_j) a_cj (d_j = a_jj after the updates of the columns before
  // j), which equals l_ij s_j l_cj with l_ij = a_ij / (s_j sqrt|d_j|), s_j = sign d_j; the columns
  // are scaled to L afterwards.  Blocked by panels of 16 columns, with three barriers per panel:
  //   (a1) warp 0 eliminates inside the 16 x 16 diagonal block (warp-synchronous steps);
  //   (a2) one thread per row below it applies the panel's 16 eliminations to its 16 panel
  //        entries and keeps the multipliers a_ij / d_j (in X, unused until the inverse);
  //   (b)  the trailing block takes a_rc -= sum_j (a_rj / d_j) a_cj over the panel columns.
  // Every entry receives the same updates in the same order (j ascending) as column by column.
  {
    constexpr int PW = 16;
    T(*F)[PW + 1] = (T(*)[PW + 1])(&X[0][0]);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int p0 = 0; p0 < NB; p0 += PW) {
      if (warp == 0) {
        const int i = p0 + (lane & 15), half = lane >> 4;
        for (int jj = 0; jj < PW; ++jj) {
          const int j = p0 + jj;
          T d = A[j][j];
          // a failed pivot (flagged below from the same value) continues as 1, as in the scaling
          if (L.indefinite ? !(fabs(d) > (T)1e-30) : !(d > (T)0)) d = (T)1;
          if (lane == 0) dd[j] = d;
          if (i > j) {
            const T f = A[i][j] / d;
            for (int c = j + 1 + half; c <= i; c += 2) A[i][c] -= f * A[c][j];
          }
          __syncwarp();
        }
      }
      __syncthreads();
      const int nb = NB - p0 - PW;   // rows below the diagonal block
      if (tid < nb) {
        const int i = p0 + PW + tid;
        T a[PW];
#pragma unroll
        for (int jj = 0; jj < PW; ++jj) a[jj] = A[i][p0 + jj];
#pragma unroll
        for (int jj = 0; jj < PW; ++jj) {
          const T f = a[jj] / dd[p0 + jj];
          F[tid][jj] = f;
#pragma unroll
          for (int c = jj + 1; c < PW; ++c) a[c] -= f * A[p0 + c][p0 + jj];
        }
#pragma unroll
        for (int jj = 0; jj < PW; ++jj) A[i][p0 + jj] = a[jj];
      }
      __syncthreads();
      for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int r = e / nb, c = e % nb;
        if (c > r) continue;
        T acc = A[p0 + PW + r][p0 + PW + c];
#pragma unroll
        for (int jj = 0; jj < PW; ++jj) acc -= F[r][jj] * A[p0 + PW + c][p0 + jj];
        A[p0 + PW + r][p0 + PW + c] = acc;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x < NB) {
    const int j = threadIdx.x;
    T d = A[j][j];
    T sj = (T)1;
    bool b = false;
    if (L.indefinite) {
      if (!(fabs(d) > (T)1e-30)) {
        b = true;
        d = (T)1;
      }
      if (d < (T)0) {
        sj = (T)-1;
        d = -d;
      }
    } else if (!(d > (T)0)) {
      b = true;
      d = (T)1;
    }
    if (b) bad = 1;
    sg[j] = sj;
    X[0][j] = sqrt(d);   // pivots, kept in the first row of X until the inverse is formed
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int r = t / NB, c = t % NB;
    if (r > c) A[r][c] /= X[0][c] * sg[c];
  }
  __syncthreads();
  if (threadIdx.x < NB) A[threadIdx.x][threadIdx.x] = X[0][threadIdx.x];
  __syncthreads();
  if (threadIdx.x < NB) ((T*)L.sgn)[m.vec_off + (int64_t)k * NB + threadIdx.x] = sg[threadIdx.x];
  if (threadIdx.x == 0 && bad) flag_breakdown(L.status, s);
  // X = L^{-1} by 16 x 16 blocks: the four diagonal blocks X_PP = L_PP^{-1} by forward
  // substitution (one warp each, one lane per column), then the blocks below the diagonal by
  // their distance d = Q - P: X_QP = -X_QQ (sum_{P <= K < Q} L_QK X_KP), the inner sum into a
  // scratch block first (3 - d + 1 blocks per distance, one entry per thread and block).
  {
    constexpr int PW = 16;
    __shared__ T Tq[3][PW][PW + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp < 4 && lane < PW) {
      const int p0 = PW * warp, c = p0 + lane;
      for (int r = p0; r < c; ++r) X[r][c] = (T)0;
      X[c][c] = (T)1 / A[c][c];
      for (int i = c + 1; i < p0 + PW; ++i) {
        T part = (T)0;
        for (int q = c; q < i; ++q) part += A[i][q] * X[q][c];
        X[i][c] = -part / A[i][i];
      }
    }
    __syncthreads();
    for (int dist = 1; dist < 4; ++dist) {
      const int nblk = 4 - dist;
      for (int e = tid; e < nblk * PW * PW; e += blockDim.x) {   // T = sum_K L_QK X_KP
        const int bq = e / (PW * PW), r = (e / PW) % PW, c = e % PW;
        const int P = bq, Q = bq + dist;
        T acc = (T)0;
        for (int K = P; K < Q; ++K)
          for (int q = 0; q < PW; ++q) acc += A[PW * Q + r][PW * K + q] * X[PW * K + q][PW * P + c];
        Tq[bq][r][c] = acc;
      }
      __syncthreads();
      for (int e = tid; e < nblk * PW * PW; e += blockDim.x) {   // X_QP = -X_QQ T
        const int bq = e / (PW * PW), r = (e / PW) % PW, c = e % PW;
        const int P = bq, Q = bq + dist;
        T acc = (T)0;
        for (int q = 0; q <= r; ++q) acc += X[PW * Q + r][PW * Q + q] * Tq[bq][q][c];
        X[PW * Q + r][PW * P + c] = -acc;
      }
      __syncthreads();
    }
  }
  T* dv = (T*)L.dinv + m.dinv_off + (int64_t)k * NB2;
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int r = t / NB, c = t % NB;
    dv[t] = c <= r ? X[r][c] : (T)0;
    g[t] = A[r][c];
  }
}

template <typename T>
__global__ void k_potrf_diag(LevelDev L, int k) {
  const int s = blockIdx.x;
  const SubMeta m = L.meta[s];
  if (k >= m.Bc) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  factor_diag_tile<T>(L, m, s, k, smem_raw);
}

// ---- step k, part 2: panel L(i,k) = A(i,k) L_kk^{-T} for i = k+1 .. R-1 --------------------
// rlim > 0: only the rows of the diagonal block, i < min(rlim, Bc) (the rows below it are solved
// on the tensor cores with the block's inverse)
template <typename T>
__global__ void k_trsm_panel(LevelDev L, int k, int rlim) {
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  const int i = k + 1 + blockIdx.x;
  const int ilim = rlim > 0 ? (rlim < m.Bc ? rlim : m.Bc) : m.R;
  if (k >= m.Bc || i >= ilim) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = (T*)smem_raw;
  T* Xs = As + NB * LDS;
  T* g = tile_ptr<T>(m, L.tiles, i, k);
  load_kmajor(As, g);
  load_kmajor(Xs, (const T*)L.dinv + m.dinv_off + (int64_t)k * NB2);
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4] = {};
  gemm_nt_4x4(As, Xs, acc, tx, ty);
  __syncthreads();
  const T* sk = (const T*)L.sgn + m.vec_off + (int64_t)k * NB;   // L(i,k) = A(i,k) L_kk^{-T} S_k
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    T v[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) v[b] = acc[a][b] * sk[4 * tx + b];
    store4(g + (4 * ty + a) * NB + 4 * tx, v);
  }
}

// ---- inverse of a sub-panel's 256 x 256 diagonal block (FP32, the tensor-core panel solve) ----
// X = L_D^{-1} for the block D = [k0, k0 + nd) (nd = min(4, Bc - k0)): X_QQ = L_QQ^{-1} (the stored
// inverse of the diagonal tile) and X_QP = -X_QQ sum_{P <= K < Q} L_QK X_KP for P < Q.  Block row
// Q needs the tiles L_QK (K < Q) and the rows of X above it, so it is formed during step k0 + Q of
// the block's factorisation, by blocks of that step's in-block update launch (next to the one that
// factors tile Q + 1).  One CTA of 256 threads takes 16 columns c0 .. c0 + 15 of X_QP (thread:
// row r, columns cg .. cg + 3), the sums in ascending K and t; X_QP is stored as a row-major tile
// at xinv + (s * 16 + 4 Q + P) * 4096 (the diagonal tiles X_QQ are read from the inverses).
__device__ void xinv_row_part(const LevelDev& L, const SubMeta& m, int s, int k0, int Q, int P, int c0,
                              float* __restrict__ xinv, unsigned char* smem_raw) {
  float(*Ls)[NB + 1] = (float(*)[NB + 1])smem_raw;                               // L_QK, then L_QQ^{-1}
  float(*Xk)[16] = (float(*)[16])(smem_raw + sizeof(float) * NB * (NB + 1));     // X_KP(:, c0 ..)
  float(*Ts)[16] = (float(*)[16])(smem_raw + sizeof(float) * NB * (NB + 1 + 16));
  const int tid = threadIdx.x, r = tid >> 2, cg = 4 * (tid & 3);
  const float* dinv = (const float*)L.dinv + m.dinv_off;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int K = P; K < Q; ++K) {   // T = sum_K L_QK X_KP
    const float* lq = tile_ptr<float>(m, L.tiles, k0 + Q, k0 + K);
    const float* xk = K == P ? dinv + (int64_t)(k0 + P) * NB2 : xinv + ((int64_t)s * 16 + 4 * K + P) * NB2;
    for (int e = tid; e < NB2; e += blockDim.x) Ls[e >> 6][e & 63] = lq[e];
    for (int e = tid; e < NB * 16; e += blockDim.x) Xk[e >> 4][e & 15] = xk[(e >> 4) * NB + c0 + (e & 15)];
    __syncthreads();
#pragma unroll 8
    for (int t = 0; t < NB; ++t) {
      const float a = Ls[r][t];
      const float4 x = *(const float4*)&Xk[t][cg];
      acc[0] += a * x.x;
      acc[1] += a * x.y;
      acc[2] += a * x.z;
      acc[3] += a * x.w;
    }
    __syncthreads();
  }
  *(float4*)&Ts[r][cg] = make_float4(acc[0], acc[1], acc[2], acc[3]);
  const float* dQ = dinv + (int64_t)(k0 + Q) * NB2;   // X_QP = -L_QQ^{-1} T (lower triangular)
  for (int e = tid; e < NB2; e += blockDim.x) Ls[e >> 6][e & 63] = dQ[e];
  __syncthreads();
  float y[4] = {0.f, 0.f, 0.f, 0.f};
  for (int t = 0; t <= r; ++t) {
    const float a = Ls[r][t];
    const float4 x = *(const float4*)&Ts[t][cg];
    y[0] += a * x.x;
    y[1] += a * x.y;
    y[2] += a * x.z;
    y[3] += a * x.w;
  }
  float* dst = xinv + ((int64_t)s * 16 + 4 * Q + P) * NB2 + r * NB + c0 + cg;
  *(float4*)dst = make_float4(-y[0], -y[1], -y[2], -y[3]);
}

// ---- step k, part 3: trailing update A(i,j) -= L(i,k) L(j,k)^T, k < j <= i, j < min(Bc, jmax) --
// fuse_next: the block that updates the next diagonal tile (k+1, k+1) (always block 0 of its
// subdomain) factors and inverts it right away, and step k+1 launches no k_potrf_diag.
// rlim > 0: only rows i < min(rlim, Bc) (the diagonal block of a sub-panel).  xinv (FP32 panel
// solves): the blocks n_upd .. n_upd + 4 xq - 1 of the grid form block row xq = k - k0 of the
// inverse of the diagonal block [k0, k0 + 4) (block column P = e / 4, columns 16 (e % 4) ..).
template <typename T>
__global__ void k_syrk_update(LevelDev L, int k, int jmax, int fuse_next, int rlim, int n_upd, float* xinv,
                              int k0) {
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  if ((int)blockIdx.x >= n_upd) {
    if constexpr (sizeof(T) == 4) {
      const int e = (int)blockIdx.x - n_upd, Q = k - k0;
      extern __shared__ __align__(16) unsigned char smem_raw[];
      if (xinv && Q < m.Bc - k0) xinv_row_part(L, m, s, k0, Q, e >> 2, 16 * (e & 3), xinv, smem_raw);
    }
    return;
  }
  if (k >= m.Bc) return;
  const int jend = jmax < m.Bc ? jmax : m.Bc;
  const int ilim = rlim > 0 ? (rlim < m.Bc ? rlim : m.Bc) : m.R;
  int t = blockIdx.x, j = k + 1, i = -1;
  for (; j < jend; ++j) {
    const int cnt = ilim - j;
    if (t < cnt) {
      i = j + t;
      break;
    }
    t -= cnt;
  }
  if (i < 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = (T*)smem_raw;
  T* Bs = As + NB * LDS;
  load_kmajor(As, tile_ptr<T>(m, L.tiles, i, k));
  load_kmajor(Bs, tile_ptr<T>(m, L.tiles, j, k));
  __syncthreads();
  if (L.indefinite) {   // A(i,j) -= L(i,k) S_k L(j,k)^T: fold S_k into the k-major B operand
    const T* sk = (const T*)L.sgn + m.vec_off + (int64_t)k * NB;
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) Bs[(t / NB) * LDS + (t % NB)] *= sk[t / NB];
    __syncthreads();
  }
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4] = {};
  gemm_nt_4x4(As, Bs, acc, tx, ty);
  T* c = tile_ptr<T>(m, L.tiles, i, j);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    T v[4];
    load4(v, c + (4 * ty + a) * NB + 4 * tx);
#pragma unroll
    for (int b = 0; b < 4; ++b) v[b] -= acc[a][b];
    store4(c + (4 * ty + a) * NB + 4 * tx, v);
  }
  if (fuse_next && i == k + 1 && j == k + 1) {   // block-uniform
    __syncthreads();   // the updated tile is in global memory, visible to the whole block
    factor_diag_tile<T>(L, m, s, k + 1, smem_raw);
  }
}

// ---- G = Y_G Y_G^T in FP64, Cholesky, inverse; K_C = G^{-1} - rho I ----------------------
// one warp per entry (a, b), a >= b, of one subdomain's G; lanes stride over the interface
// columns (contiguous inside a tile row), FP64 products, fixed-order warp reduction
template <typename T>
__global__ void k_gram(LevelDev L) {
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  const int nc = m.nc;
  const int pair = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (pair >= nc * nc) return;
  const int a = pair / nc, b = pair % nc;
  if (b > a) return;
  const T* ya = tile_ptr<T>(m, L.tiles, m.Bc + a / NB, m.nIb) + (a % NB) * NB;
  const T* yb = tile_ptr<T>(m, L.tiles, m.Bc + b / NB, m.nIb) + (b % NB) * NB;
  const T* sG = (const T*)L.sgn + m.vec_off + (int64_t)m.nIb * NB;   // G = Y S Y^T
  double acc = 0.0;
  for (int c = lane; c < m.nGb * NB; c += 32) {
    const int64_t o = (int64_t)(c / NB) * NB2 + (c % NB);
    acc += (double)ya[o] * (double)sG[c] * (double)yb[o];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    double* G = L.Ginv + m.g_off;
    G[a * nc + b] = acc;
    G[b * nc + a] = acc;
  }
}

// G^{-1} by Gauss-Jordan elimination with partial pivoting (indefinite levels), FP64, one block
// per subdomain; W (the K_C buffer) holds the eliminated copy of G.
__device__ void gauss_jordan_inverse(double* G, double* W, int n, int* bad) {
  __shared__ int piv_row;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    W[t] = G[t];
    G[t] = (t / n == t % n) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      int best = j;
      double bv = fabs(W[j * n + j]);
      for (int i = j + 1; i < n; ++i)
        if (fabs(W[i * n + j]) > bv) {
          bv = fabs(W[i * n + j]);
          best = i;
        }
      if (!(bv > 0.0)) *bad = 1;
      piv_row = best;
    }
    __syncthreads();
    const int pr = piv_row;
    if (pr != j)
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double a = W[j * n + c], b = W[pr * n + c];
        W[j * n + c] = b;
        W[pr * n + c] = a;
        a = G[j * n + c];
        b = G[pr * n + c];
        G[j * n + c] = b;
        G[pr * n + c] = a;
      }
    __syncthreads();
    const double inv = W[j * n + j] != 0.0 ? 1.0 / W[j * n + j] : 0.0;
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      W[j * n + c] *= inv;
      G[j * n + c] *= inv;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
      const int i = t / n, c = t % n;
      if (i == j) continue;
      const double f = W[i * n + j];
      if (c != j) W[i * n + c] -= f * W[j * n + c];
      G[i * n + c] -= f * G[j * n + c];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (i != j) W[i * n + j] = 0.0;
    __syncthreads();
  }
}

__global__ void k_small_chol_inv(LevelDev L) {
  const int s = blockIdx.x;
  const SubMeta m = L.meta[s];
  const int n = m.nc;
  if (n == 0) return;
  if (L.indefinite) {
    __shared__ int badi;
    if (threadIdx.x == 0) badi = 0;
    __syncthreads();
    double* G = L.Ginv + m.g_off;
    double* W = L.KC + m.g_off;
    gauss_jordan_inverse(G, W, n, &badi);
    __syncthreads();
    if (threadIdx.x == 0 && badi) flag_breakdown(L.status, s);
    const double rho = L.rho[s];
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
      const int a = t / n, b = t % n;
      W[t] = G[t] - (a == b ? rho * L.c_rho[m.c_off + a] : 0.0);   // K_C = G^{-1} - R
    }
    return;
  }
  double* G = L.Ginv + m.g_off;   // in: G (full), out: G^{-1}
  double* W = L.KC + m.g_off;     // scratch for L^{-1}, then K_C
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double d = G[j * n + j];
      if (!(d > 0.0)) {
        bad = 1;
        d = 1.0;
      }
      G[j * n + j] = sqrt(d);
    }
    __syncthreads();
    const double piv = G[j * n + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) G[i * n + j] /= piv;
    __syncthreads();
    const int w = n - 1 - j;
    for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
      const int i = j + 1 + t / w, c = j + 1 + t % w;
      if (c <= i) G[i * n + c] -= G[i * n + j] * G[c * n + j];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) flag_breakdown(L.status, s);
  // W = L^{-1} (lower), one column per thread
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    for (int r = 0; r < c; ++r) W[r * n + c] = 0.0;
    W[c * n + c] = 1.0 / G[c * n + c];
    for (int i = c + 1; i < n; ++i) {
      double acc = 0.0;
      for (int q = c; q < i; ++q) acc += G[i * n + q] * W[q * n + c];
      W[i * n + c] = -acc / G[i * n + i];
    }
  }
  __syncthreads();
  // G^{-1} = W^T W
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int a = t / n, b = t % n;
    double acc = 0.0;
    for (int q = (a > b ? a : b); q < n; ++q) acc += W[q * n + a] * W[q * n + b];
    G[t] = acc;   // safe: G's lower part (the factor) is no longer read
  }
  __syncthreads();
  const double rho = L.rho[s];
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int a = t / n, b = t % n;
    W[t] = G[t] - (a == b ? rho * L.c_rho[m.c_off + a] : 0.0);   // K_C = G^{-1} - R
  }
}

// Z = Y_G^T G^{-1}, written into the Psi buffer (rows: interface padded positions)
template <typename T>
__global__ void k_psi_rhs(LevelDev L) {
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  const int nc = m.nc;
  if (nc == 0) return;
  const int rows = m.nGb * NB;
  const int64_t total = (int64_t)rows * nc;
  const double* Gi = L.Ginv + m.g_off;
  T* Z = (T*)L.psi + m.psi_off;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / nc), q = (int)(t % nc);
    const int jb = m.nIb + c / NB, cc = c % NB;
    double acc = 0.0;
    for (int p = 0; p < nc; ++p) {
      const T y = tile_ptr<T>(m, L.tiles, m.Bc + p / NB, jb)[(p % NB) * NB + cc];
      acc += (double)y * Gi[p * nc + q];
    }
    Z[t] = (T)acc;   // Z = Y^T G^{-1}
  }
}

// Psi_G = L_GG^{-T} Z, right-looking over the interface block rows from the bottom: at step t,
// block row i = Bc - 1 - t of every subdomain is final once X_i = D_i^T Z_i (D_i the stored inverse
// of the diagonal tile), and every block row j < i above it receives Z_j -= L(i, j)^T X_i.  The
// updates of a step are independent (one CTA per (j, subdomain, 16 columns)), so a step is one
// wide launch instead of a per-CTA chain of dependent tiles.
template <typename T>
__global__ void __launch_bounds__(256) k_psi_final(LevelDev L, int t) {
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  const int i = m.Bc - 1 - t, c0 = 16 * blockIdx.x, nc = m.nc;
  if (i < m.nIb || c0 >= nc) return;
  __shared__ T Ds[NB][NB + 1];
  __shared__ __align__(16) T Zs[NB][16];
  const T* dv = (const T*)L.dinv + m.dinv_off + (int64_t)i * NB2;
  T* Zi = (T*)L.psi + m.psi_off + (int64_t)(i - m.nIb) * NB * nc;
  for (int e = threadIdx.x; e < NB2; e += blockDim.x) Ds[e / NB][e % NB] = dv[e];
  for (int e = threadIdx.x; e < NB * 16; e += blockDim.x) {
    const int r = e / 16, q = e % 16;
    Zs[r][q] = c0 + q < nc ? Zi[(int64_t)r * nc + c0 + q] : (T)0;
  }
  __syncthreads();
  const int r = threadIdx.x >> 2, q4 = 4 * (threadIdx.x & 3);
  T x[4] = {};
#pragma unroll 8
  for (int mm = 0; mm < NB; ++mm) {   // X_i = D_i^T Z_i
    const T d = Ds[mm][r];
#pragma unroll
    for (int b = 0; b < 4; ++b) x[b] += d * Zs[mm][q4 + b];
  }
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if (c0 + q4 + b < nc) Zi[(int64_t)r * nc + c0 + q4 + b] = x[b];
}

template <typename T>
__global__ void __launch_bounds__(256) k_psi_update(LevelDev L, int t) {
  const int s = blockIdx.y;
  const SubMeta m = L.meta[s];
  const int i = m.Bc - 1 - t, j = m.nIb + (int)blockIdx.x, c0 = 16 * blockIdx.z, nc = m.nc;
  if (j >= i || c0 >= nc) return;
  __shared__ T Ls[NB][NB + 1];
  __shared__ __align__(16) T Xs[NB][16];
  const T* lt = (const T*)L.tiles + m.tile_off + tile_index(i, j, m.Bc) * NB2;
  const T* Xi = (const T*)L.psi + m.psi_off + (int64_t)(i - m.nIb) * NB * nc;
  T* Zj = (T*)L.psi + m.psi_off + (int64_t)(j - m.nIb) * NB * nc;
  for (int e = threadIdx.x; e < NB2; e += blockDim.x) Ls[e / NB][e % NB] = lt[e];
  for (int e = threadIdx.x; e < NB * 16; e += blockDim.x) {
    const int r = e / 16, q = e % 16;
    Xs[r][q] = c0 + q < nc ? Xi[(int64_t)r * nc + c0 + q] : (T)0;
  }
  __syncthreads();
  const int c = threadIdx.x >> 2, q4 = 4 * (threadIdx.x & 3);
  T acc[4] = {};
#pragma unroll 8
  for (int r = 0; r < NB; ++r) {   // (L(i, j)^T X_i)[c] = sum_r L(i, j)[r][c] X_i[r]
    const T l = Ls[r][c];
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[b] += l * Xs[r][q4 + b];
  }
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if (c0 + q4 + b < nc) Zj[(int64_t)c * nc + c0 + q4 + b] -= acc[b];
}

// v_G -= Y_G^T G^{-1} Y_G v_G  (the constraint part of Eq. sub_cor): t = Y_G v and the final
// update stream the constraint block rows of the factor (k_rows_matvec / k_cols_matvec below);
// mu = G^{-1} t takes one warp per row of G^{-1}.
__global__ void k_cc_mu(LevelDev L, const int32_t* __restrict__ crow_sub, int64_t total_rows,
                        const double* __restrict__ t, double* __restrict__ mu) {
  const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= total_rows) return;
  t += (int64_t)blockIdx.y * total_rows;
  mu += (int64_t)blockIdx.y * total_rows;
  const int s = crow_sub[g];
  const SubMeta m = L.meta[s];
  const int p = (int)(g - m.c_off);
  const double* Gi = L.Ginv + m.g_off + (int64_t)p * m.nc;
  double acc = 0.0;
  for (int q = lane; q < m.nc; q += 32) acc += Gi[q] * t[m.c_off + q];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) mu[g] = acc;
}

// ---- products with Y_G and Psi_G^T, both held as ncb x nGb tiles of NB x NB per subdomain ----
// MODE 0: M = Y_G, the constraint block rows of the factor (the forward sweep left S L^{-1} r in
// the vector, so its entries are multiplied by the pivot signs S first); MODE 1: M = Psi_G^T
// (psiT).  Row p of M belongs to coarse DOF p of the subdomain, column c to interface position c.
template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};

template <typename T, int MODE>
__device__ __forceinline__ const T* m_tile(const LevelDev& L, const SubMeta& m, int rb, int j) {
  if (MODE == 0) return tile_ptr<T>(m, L.tiles, m.Bc + rb, m.nIb + j);
  return (const T*)L.psiT + m.psiT_off + ((int64_t)rb * m.nGb + j) * NB2;
}

// Row products over four tile columns: block (z, rb, s) adds the columns 4z .. 4z+3 of the
// coarse rows rb NB .. rb NB + 63 of subdomain s for NR right-hand sides (column q at
// vec + q n_vec) and writes part[(q sum_nc + c_off + p) zmax + z] (zero where the subdomain has
// no such tile columns).  Warp w takes the rows w, w+8, .., lane l the columns 2l, 2l+1 of every
// tile, so each tile row is one coalesced 256-byte read; rows past nc are not read.
template <typename T, int NR, int MODE>
__global__ void __launch_bounds__(256) k_rows_matvec(LevelDev L, const T* __restrict__ vec, double* __restrict__ part,
                                                     int zmax, int64_t sum_nc) {
  using V2 = typename Pair<T>::type;
  const int z = blockIdx.x, rb = blockIdx.y, s = blockIdx.z;
  const SubMeta m = L.meta[s];
  if (rb >= m.ncb) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = 4 * z, j1 = min(m.nGb, j0 + 4);
  __shared__ __align__(16) T xs[NR][4][NB];
  const T* v = vec + m.vec_off + (int64_t)m.nIb * NB;
  const T* sg = (const T*)L.sgn + m.vec_off + (int64_t)m.nIb * NB;
  for (int e = threadIdx.x; e < NR * 4 * NB; e += blockDim.x) {
    const int q = e / (4 * NB), jj = (e / NB) % 4, c = e % NB;
    const int j = j0 + jj;
    T x = (T)0;
    if (j < j1) {
      x = v[(int64_t)q * L.n_vec + (int64_t)j * NB + c];
      if (MODE == 0 && L.indefinite) x *= sg[(int64_t)j * NB + c];
    }
    xs[q][jj][c] = x;
  }
  __syncthreads();
  const int rows = min(NB, m.nc - rb * NB);
  T acc[8][NR];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[r][q] = (T)0;
  for (int j = j0; j < j1; ++j) {
    const T* t = m_tile<T, MODE>(L, m, rb, j) + 2 * lane;
    V2 xv[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) xv[q] = *(const V2*)&xs[q][j - j0][2 * lane];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int row = warp + 8 * r;
      if (row < rows) {
        const V2 a = __ldg((const V2*)(t + row * NB));
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[r][q] += a.x * xv[q].x + a.y * xv[q].y;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int row = warp + 8 * r;
    if (row >= rows) continue;   // warp-uniform
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      T a = acc[r][q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) part[((int64_t)q * sum_nc + m.c_off + rb * NB + row) * zmax + z] = (double)a;
    }
  }
}

// out[q sum_nc + g] = sum_{z < zmax} part[(q sum_nc + g) zmax + z], in order
__global__ void k_sum_parts(const double* __restrict__ part, int zmax, int64_t total, double* __restrict__ out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int64_t o = (int64_t)blockIdx.y * total + g;
  double t = 0.0;
  for (int z = 0; z < zmax; ++z) t += part[o * zmax + z];
  out[o] = t;
}

// Column products: block (j, s) makes v[nIb NB + j NB + c] += sign sum_p M[p][j NB + c] zsub_p
// for the 64 positions of interface tile column j and NR right-hand sides (zsub column q at
// zsub + q sum_nc, per-subdomain coarse vectors); the eight warps' partial sums are added in a
// fixed order.
template <typename T, int NR, int MODE>
__global__ void __launch_bounds__(256) k_cols_matvec(LevelDev L, T* __restrict__ vec, const double* __restrict__ zsub,
                                                     int64_t sum_nc, T sign) {
  using V2 = typename Pair<T>::type;
  const int j = blockIdx.x, s = blockIdx.y;
  const SubMeta m = L.meta[s];
  if (j >= m.nGb || m.nc == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ T zs[NR][NB];
  __shared__ T red[8][NR][NB];
  T acc[NR][2];
#pragma unroll
  for (int q = 0; q < NR; ++q) acc[q][0] = acc[q][1] = (T)0;
  for (int rb = 0; rb < m.ncb; ++rb) {
    const int rows = min(NB, m.nc - rb * NB);
    __syncthreads();
    for (int e = threadIdx.x; e < NR * NB; e += blockDim.x) {
      const int q = e / NB, p = e % NB;
      zs[q][p] = p < rows ? (T)zsub[(int64_t)q * sum_nc + m.c_off + rb * NB + p] : (T)0;
    }
    __syncthreads();
    const T* t = m_tile<T, MODE>(L, m, rb, j) + 2 * lane;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int row = warp + 8 * r;
      if (row < rows) {
        const V2 a = __ldg((const V2*)(t + row * NB));
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const T zq = zs[q][row];
          acc[q][0] += a.x * zq;
          acc[q][1] += a.y * zq;
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    red[warp][q][2 * lane] = acc[q][0];
    red[warp][q][2 * lane + 1] = acc[q][1];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NR * NB; e += blockDim.x) {
    const int q = e / NB, c = e % NB;
    T a = (T)0;
#pragma unroll
    for (int w = 0; w < 8; ++w) a += red[w][q][c];
    T* v = vec + (int64_t)q * L.n_vec + m.vec_off + (int64_t)m.nIb * NB + (int64_t)j * NB + c;
    *v = *v + sign * a;
  }
}

// psiT tile (rb, j)[p][c] = Psi_G[(j NB + c) nc + rb NB + p], zero outside nG x nc (set-up)
template <typename T>
__global__ void k_psi_transpose(LevelDev L) {
  const int j = blockIdx.x, rb = blockIdx.y, s = blockIdx.z;
  const SubMeta m = L.meta[s];
  if (j >= m.nGb || rb >= m.ncb) return;
  const T* P = (const T*)L.psi + m.psi_off;
  T* out = (T*)L.psiT + m.psiT_off + ((int64_t)rb * m.nGb + j) * NB2;
  __shared__ T ts[NB][NB + 1];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int c = e / NB, p = e % NB;
    const int gc = j * NB + c, gp = rb * NB + p;
    ts[c][p] = (gc < m.nG && gp < m.nc) ? P[(int64_t)gc * m.nc + gp] : (T)0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) out[e] = ts[e % NB][e / NB];
}

// ---- explicit inverse of the coarsest factor (FP32 copy, mixed form) ------------------------
// W = A_C^{-1} = L^{-T} S L^{-1} of the single-subdomain coarsest level, whose block rows are all
// "interior" (identity padding past the last DOF).  CTA c substitutes the identity columns
// c CW .. c CW + CW - 1 through the tiled factor: forward y_i = D_i (e_i - sum_{j<i} L_ij y_j),
// t = S y, backward x_i = D_i^T (t_i - sum_{j>i} L_ji^T x_j), with D_i the stored inverses of the
// diagonal tiles (the same steps as the sweeps, in the same precision).  Column q of the result is
// kept at W + (c CW + q) n_pad, so W is stored column after column; A_C is symmetric, so row q of
// the stored matrix is row q of A_C^{-1} up to rounding.  Each product of a tile with a 64 x CW
// block runs from shared memory, the tile k-major, every thread a block of CW/16 rows x 4 columns.
template <int CW>
__global__ void __launch_bounds__(256) k_coarse_inverse(LevelDev L, float* __restrict__ W) {
  constexpr int RR = CW / 16;                 // rows per thread
  constexpr int CG = CW / 4;                  // column groups of four
  const SubMeta m = L.meta[0];
  const int nb = m.Bc;
  const int64_t npad = (int64_t)nb * NB;
  const int c0 = blockIdx.x * CW;
  if (c0 >= npad) return;
  __shared__ __align__(16) float As[NB][NB + 4];   // tile, k-major: As[k][r]
  __shared__ __align__(16) float Bs[NB][CW + 4];   // 64 x CW block: Bs[k][c]
  const int tid = threadIdx.x;
  const int cg = tid % CG, rg = tid / CG;          // columns 4 cg .. +3, rows RR rg .. +RR-1
  float* Wc = W + (int64_t)c0 * npad;              // this CTA's columns, each of npad entries
  const float* tiles = (const float*)L.tiles + m.tile_off;
  const float* dinv = (const float*)L.dinv + m.dinv_off;
  const float* sgn = (const float*)L.sgn + m.vec_off;
  auto load_tile = [&](const float* t, bool transpose) {   // As[k][r] = t[r][k] (or t[k][r])
    for (int e = tid; e < NB2; e += 256) {
      const int a = e / NB, b = e % NB;
      if (transpose) As[b][a] = t[e]; else As[a][b] = t[e];
    }
  };
  auto load_block = [&](int blk) {                  // Bs[k][c] = W column c, rows of block blk
    for (int e = tid; e < NB * CW; e += 256) {
      const int c = e / NB, k = e % NB;
      Bs[k][c] = Wc[(int64_t)c * npad + (int64_t)blk * NB + k];
    }
  };
  auto mma = [&](float (&acc)[RR][4]) {
#pragma unroll 8
    for (int k = 0; k < NB; ++k) {
      float a[RR], b[4];
#pragma unroll
      for (int r = 0; r < RR; ++r) a[r] = As[k][RR * rg + r];
      const float4 bv = *(const float4*)&Bs[k][4 * cg];
      b[0] = bv.x; b[1] = bv.y; b[2] = bv.z; b[3] = bv.w;
#pragma unroll
      for (int r = 0; r < RR; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] += a[r] * b[q];
    }
  };
  auto store_block = [&](int blk, const float (&v)[RR][4]) {
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) Wc[(int64_t)(4 * cg + q) * npad + (int64_t)blk * NB + RR * rg + r] = v[r][q];
  };
  // forward: y_i = D_i (e_i - sum_{j<i} L_ij y_j)
  for (int i = 0; i < nb; ++i) {
    float acc[RR][4] = {};
    for (int j = 0; j < i; ++j) {
      __syncthreads();
      load_tile(tiles + ((int64_t)i * (i + 1) / 2 + j) * NB2, true);
      load_block(j);
      __syncthreads();
      mma(acc);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t row = (int64_t)i * NB + RR * rg + r;
        Bs[RR * rg + r][4 * cg + q] = (row == c0 + 4 * cg + q ? 1.f : 0.f) - acc[r][q];
      }
    load_tile(dinv + (int64_t)i * NB2, true);
    __syncthreads();
    float y[RR][4] = {};
    mma(y);
    store_block(i, y);
  }
  __syncthreads();
  // t = S y (pivot signs of the signed factor; all +1 on SPD levels)
  for (int e = tid; e < NB * CW; e += 256) {
    const int c = e / NB;
    for (int64_t row = e % NB; row < npad; row += NB) Wc[(int64_t)c * npad + row] *= sgn[row];
  }
  // backward: x_i = D_i^T (t_i - sum_{j>i} L_ji^T x_j)
  for (int i = nb - 1; i >= 0; --i) {
    float acc[RR][4] = {};
    for (int j = i + 1; j < nb; ++j) {
      __syncthreads();
      load_tile(tiles + ((int64_t)j * (j + 1) / 2 + i) * NB2, false);
      load_block(j);
      __syncthreads();
      mma(acc);
    }
    __syncthreads();
    load_block(i);
    __syncthreads();
    float rhs[RR][4];
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) rhs[r][q] = Bs[RR * rg + r][4 * cg + q] - acc[r][q];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) Bs[RR * rg + r][4 * cg + q] = rhs[r][q];
    load_tile(dinv + (int64_t)i * NB2, false);
    __syncthreads();
    float x[RR][4] = {};
    mma(x);
    store_block(i, x);
  }
}

// y = W x for nr columns (x, y: columns of n_vec, padded local positions 0 .. npad-1); one warp
// per output row, lanes along the row (coalesced), FP32 sums in a fixed order.
template <int NR>
__global__ void k_coarse_apply(const float* __restrict__ W, int64_t npad, const float* __restrict__ x,
                               float* __restrict__ y, int64_t n_vec) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= npad) return;
  const int64_t c0 = (int64_t)blockIdx.y * NR;
  const float* w = W + row * npad;
  float acc[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) acc[q] = 0.f;
  for (int64_t c = 4 * lane; c < npad; c += 128) {
    const float4 a = *(const float4*)(w + c);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const float4 b = *(const float4*)(x + (c0 + q) * n_vec + c);
      acc[q] += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
    }
  }
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    float v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) y[(c0 + q) * n_vec + row] = v;
  }
}

}  // namespace

void launch_coarse_inverse(const LevelDev& L, int64_t npad, float* W, cudaStream_t st) {
  if (npad <= 0) return;
  note_launch();
  if (npad <= 2048)
    k_coarse_inverse<16><<<(unsigned)((npad + 15) / 16), 256, 0, st>>>(L, W);
  else
    k_coarse_inverse<64><<<(unsigned)((npad + 63) / 64), 256, 0, st>>>(L, W);
}

void launch_coarse_apply(const float* W, int64_t npad, const float* x, float* y, int64_t n_vec, int nr,
                         cudaStream_t st) {
  if (npad <= 0 || nr <= 0) return;
  const unsigned gx = (unsigned)((npad + 7) / 8);
  for (int r0 = 0; r0 < nr;) {
    const int left = nr - r0;
    const int g = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    const int ng = left / g;
    const float* xs = x + (int64_t)r0 * n_vec;
    float* ys = y + (int64_t)r0 * n_vec;
    note_launch();
    if (g == 8)
      k_coarse_apply<8><<<dim3(gx, ng), 256, 0, st>>>(W, npad, xs, ys, n_vec);
    else if (g == 4)
      k_coarse_apply<4><<<dim3(gx, ng), 256, 0, st>>>(W, npad, xs, ys, n_vec);
    else if (g == 2)
      k_coarse_apply<2><<<dim3(gx, ng), 256, 0, st>>>(W, npad, xs, ys, n_vec);
    else
      k_coarse_apply<1><<<dim3(gx, ng), 256, 0, st>>>(W, npad, xs, ys, n_vec);
    r0 += ng * g;
  }
}

template <typename T>
void launch_potrf_step(const LevelDev& L, int k, int max_R, int max_tiles, int jmax, cudaStream_t st, int skip_diag,
                       int fuse_next, int rlim, float* xinv, int k0) {
  const unsigned ns = (unsigned)L.n_sub;
  const size_t sm = 2 * NB * LDS * sizeof(T);
  const size_t sm_diag = 2 * NB * (NB + 1) * sizeof(T);
  static bool attr = false;   // opt in to more than 48 KB of dynamic shared memory once
  if (!attr) {
    cudaFuncSetAttribute(k_potrf_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_diag);
    cudaFuncSetAttribute(k_trsm_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_syrk_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  static_assert(2 * NB * LDS >= 2 * NB * (NB + 1), "the update's shared memory holds the diagonal factorisation");
  if (!skip_diag) { note_launch(); k_potrf_diag<T><<<ns, 256, sm_diag, st>>>(L, k); }
  const int panel = (rlim > 0 && rlim < max_R ? rlim : max_R) - k - 1;
  if (panel > 0) { note_launch(); k_trsm_panel<T><<<dim3((unsigned)panel, ns), 256, sm, st>>>(L, k, rlim); }
  static_assert(sizeof(float) * NB * (NB + 1 + 32) <= 2 * NB * LDS * sizeof(float), "block inverse shared memory");
  const int xq = xinv && sizeof(T) == 4 ? k - k0 : 0;   // block row of the diagonal block's inverse
  if (max_tiles > 0 || xq > 0) {
    note_launch();
    k_syrk_update<T><<<dim3((unsigned)(max_tiles + 4 * xq), ns), 256, sm, st>>>(L, k, jmax, fuse_next, rlim, max_tiles,
                                                                               xinv, k0);
  }
}

template <typename T>
void launch_gram_chol_t(const LevelDev& L, int max_nc, cudaStream_t st) {
  const unsigned ns = (unsigned)L.n_sub;
  const unsigned gx = (unsigned)(((int64_t)max_nc * max_nc + 7) / 8);
  { note_launch(); k_gram<T><<<dim3(gx, ns), 256, 0, st>>>(L); }
  { note_launch(); k_small_chol_inv<<<ns, 256, 0, st>>>(L); }
}

void launch_gram_chol(const LevelDev& L, int precision_fp32, int max_nc, cudaStream_t st) {
  if (precision_fp32)
    launch_gram_chol_t<float>(L, max_nc, st);
  else
    launch_gram_chol_t<double>(L, max_nc, st);
}

template <typename T>
void launch_psi(const LevelDev& L, int max_nGb, int max_nc, cudaStream_t st) {
  const unsigned ns = (unsigned)L.n_sub;
  if (max_nc <= 0 || max_nGb <= 0) return;
  { note_launch(); k_psi_rhs<T><<<dim3(16, ns), 256, 0, st>>>(L); }
  const unsigned chunks = (unsigned)((max_nc + 15) / 16);
  for (int t = 0; t < max_nGb; ++t) {   // block row Bc - 1 - t of every subdomain, bottom up
    { note_launch(); k_psi_final<T><<<dim3(chunks, ns), 256, 0, st>>>(L, t); }
    if (max_nGb - 1 - t > 0)
      { note_launch(); k_psi_update<T><<<dim3((unsigned)(max_nGb - 1 - t), ns, chunks), 256, 0, st>>>(L, t); }
  }
}

// The solve-phase launches below take nr right-hand sides: local vectors of n_vec, per-subdomain
// coarse vectors of sum nc entries per column.
template <typename T, int MODE>
void rows_matvec(const LevelDev& L, const T* vec, double* part, int64_t sum_nc, int max_nGb, int max_ncb,
                 cudaStream_t st, int nr) {
  const int zmax = rows_zmax(max_nGb);
  const dim3 grid((unsigned)zmax, (unsigned)max_ncb, (unsigned)L.n_sub);
  constexpr int kMaxNR = sizeof(T) == 4 ? 8 : 4;
  for (int r0 = 0; r0 < nr;) {
    const int left = nr - r0;
    const int g = left >= kMaxNR ? kMaxNR : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    const T* v = vec + (int64_t)r0 * L.n_vec;
    double* pt = part + (int64_t)r0 * sum_nc * zmax;
    note_launch();
    if (g == 8)
      k_rows_matvec<T, (sizeof(T) == 4 ? 8 : 4), MODE><<<grid, 256, 0, st>>>(L, v, pt, zmax, sum_nc);
    else if (g == 4)
      k_rows_matvec<T, 4, MODE><<<grid, 256, 0, st>>>(L, v, pt, zmax, sum_nc);
    else if (g == 2)
      k_rows_matvec<T, 2, MODE><<<grid, 256, 0, st>>>(L, v, pt, zmax, sum_nc);
    else
      k_rows_matvec<T, 1, MODE><<<grid, 256, 0, st>>>(L, v, pt, zmax, sum_nc);
    r0 += g;
  }
}

template <typename T, int MODE>
void cols_matvec(const LevelDev& L, T* vec, const double* zsub, int64_t sum_nc, int max_nGb, T sign, cudaStream_t st,
                 int nr) {
  const dim3 grid((unsigned)max_nGb, (unsigned)L.n_sub);
  constexpr int kMaxNR = sizeof(T) == 4 ? 8 : 4;
  for (int r0 = 0; r0 < nr;) {
    const int left = nr - r0;
    const int g = left >= kMaxNR ? kMaxNR : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    T* v = vec + (int64_t)r0 * L.n_vec;
    const double* zz = zsub + (int64_t)r0 * sum_nc;
    note_launch();
    if (g == 8)
      k_cols_matvec<T, (sizeof(T) == 4 ? 8 : 4), MODE><<<grid, 256, 0, st>>>(L, v, zz, sum_nc, sign);
    else if (g == 4)
      k_cols_matvec<T, 4, MODE><<<grid, 256, 0, st>>>(L, v, zz, sum_nc, sign);
    else if (g == 2)
      k_cols_matvec<T, 2, MODE><<<grid, 256, 0, st>>>(L, v, zz, sum_nc, sign);
    else
      k_cols_matvec<T, 1, MODE><<<grid, 256, 0, st>>>(L, v, zz, sum_nc, sign);
    r0 += g;
  }
}

template <typename T>
void launch_constraint_corr(const LevelDev& L, T* vec, const int32_t* crow_sub, int64_t total_rows, double* t,
                            double* mu, double* part, int max_nGb, int max_ncb, cudaStream_t st, int nr) {
  if (total_rows <= 0 || max_nGb <= 0) return;
  rows_matvec<T, 0>(L, vec, part, total_rows, max_nGb, max_ncb, st, nr);
  const int zmax = rows_zmax(max_nGb);
  note_launch();
  k_sum_parts<<<dim3((unsigned)((total_rows + 255) / 256), (unsigned)nr), 256, 0, st>>>(part, zmax, total_rows, t);
  const unsigned g = (unsigned)((total_rows + 7) / 8);
  { note_launch(); k_cc_mu<<<dim3(g, nr), 256, 0, st>>>(L, crow_sub, total_rows, t, mu); }
  cols_matvec<T, 0>(L, vec, mu, total_rows, max_nGb, (T)-1, st, nr);
}

template <typename T>
void launch_psi_t_apply(const LevelDev& L, const T* vec, double* part, int64_t sum_nc, double* rc_sub, int max_nGb,
                        int max_ncb, cudaStream_t st, int nr) {
  if (sum_nc <= 0 || max_nGb <= 0) return;
  rows_matvec<T, 1>(L, vec, part, sum_nc, max_nGb, max_ncb, st, nr);
  const int zmax = rows_zmax(max_nGb);
  note_launch();
  k_sum_parts<<<dim3((unsigned)((sum_nc + 255) / 256), (unsigned)nr), 256, 0, st>>>(part, zmax, sum_nc, rc_sub);
}

template <typename T>
void launch_psi_apply_add(const LevelDev& L, const double* zc_sub, int64_t sum_nc, T* vec, int max_nGb, int max_ncb,
                          cudaStream_t st, int nr) {
  if (sum_nc <= 0 || max_nGb <= 0) return;
  (void)max_ncb;
  cols_matvec<T, 1>(L, vec, zc_sub, sum_nc, max_nGb, (T)1, st, nr);
}

template <typename T>
void launch_psi_transpose(const LevelDev& L, int max_nGb, int max_ncb, cudaStream_t st) {
  if (max_nGb <= 0 || max_ncb <= 0) return;
  note_launch();
  k_psi_transpose<T><<<dim3((unsigned)max_nGb, (unsigned)max_ncb, (unsigned)L.n_sub), 256, 0, st>>>(L);
}

#define INST(T)                                                                                 \
  template void launch_potrf_step<T>(const LevelDev&, int, int, int, int, cudaStream_t, int, int, int, float*, int); \
  template void launch_psi<T>(const LevelDev&, int, int, cudaStream_t);                          \
  template void launch_constraint_corr<T>(const LevelDev&, T*, const int32_t*, int64_t, double*, double*, double*, \
                                         int, int, cudaStream_t, int);                                     \
  template void launch_psi_t_apply<T>(const LevelDev&, const T*, double*, int64_t, double*, int, int, cudaStream_t, \
                                      int);                                                              \
  template void launch_psi_apply_add<T>(const LevelDev&, const double*, int64_t, T*, int, int, cudaStream_t, int); \
  template void launch_psi_transpose<T>(const LevelDev&, int, int, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace bddc
