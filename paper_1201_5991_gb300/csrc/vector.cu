// Vector kernels of the solve phase: interface gather/scatter with weights (r_i = E_i^T r,
// z = sum E_i z_i, Sec. 2), FP64 sparse products with K_i, coarse gather/scatter with R_Ci,
// deterministic FP64 reductions and the device-side PCG recurrences, and the element
// contraction of the adjoint gradient.
//
// All sums run in a fixed order (ascending subdomain for the interface / coarse sums, a
// fixed grid and tree for the dot products), so results are bit-reproducible.
#include "internal.h"

namespace bddc {

namespace {

// Several right-hand sides: blockIdx.y selects the column; every vector of a block stores its
// columns one after another with its own length as the stride (local vectors n_vec, interface
// vectors n_iface, level vectors n_dof, coarse vectors n_coarse, per-subdomain coarse vectors sum nc).
template <typename T>
__global__ void k_gather_iface(LevelDev L, const double* __restrict__ x, int weighted, T* __restrict__ loc) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.n_vec) return;
  x += (int64_t)blockIdx.y * L.n_iface;
  loc += (int64_t)blockIdx.y * L.n_vec;
  const int32_t g = L.loc2iface[p];
  double v = 0.0;
  if (g >= 0) v = weighted ? L.w[p] * x[g] : x[g];
  loc[p] = (T)v;
}

template <typename T>
__global__ void k_scatter_iface(LevelDev L, const T* __restrict__ loc, int weighted, double* __restrict__ y) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.n_iface) return;
  loc += (int64_t)blockIdx.y * L.n_vec;
  y += (int64_t)blockIdx.y * L.n_iface;
  double s = 0.0;
  for (int64_t o = L.iface_ptr[g]; o < L.iface_ptr[g + 1]; ++o) {
    const int64_t p = L.iface_occ[o];
    s += weighted ? L.w[p] * (double)loc[p] : (double)loc[p];
  }
  y[g] = s;
}

// part: 0 interior positions only, 1 interface only, 2 all
template <typename T>
__global__ void k_gather_glob(LevelDev L, const double* __restrict__ x, int part, T* __restrict__ loc) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.n_vec) return;
  x += (int64_t)blockIdx.y * L.n_dof;
  loc += (int64_t)blockIdx.y * L.n_vec;
  const int32_t g = L.loc2glob[p];
  const bool is_if = L.loc2iface[p] >= 0;
  double v = 0.0;
  if (g >= 0 && (part == 2 || (part == 0 && !is_if) || (part == 1 && is_if))) v = x[g];
  loc[p] = (T)v;
}

template <typename T>
__global__ void k_scatter_interior(LevelDev L, const T* __restrict__ loc, double* __restrict__ y) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.n_vec) return;
  const int32_t g = L.loc2glob[p];
  if (g >= 0 && L.loc2iface[p] < 0) y[(int64_t)blockIdx.y * L.n_dof + g] = (double)loc[(int64_t)blockIdx.y * L.n_vec + p];
}

// y[row] = beta*y[row] + alpha * (K_i x)[row] for the rows of a list (interior rows, interface
// rows or all rows of every subdomain); 16 lanes per row, two rows per warp.
__global__ void k_spmv(LevelDev L, const int64_t* __restrict__ rows, int64_t nrows, const double* __restrict__ x,
                       double* __restrict__ y, double alpha, double beta, const int32_t* __restrict__ row_sub) {
  const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 4) + (threadIdx.x >> 4);
  const int l = threadIdx.x & 15;
  const bool valid = g < nrows;
  const int64_t row = rows[valid ? g : 0];
  const int s = row_sub[row];
  x += (int64_t)blockIdx.y * L.n_vec;
  y += (int64_t)blockIdx.y * L.n_vec;
  const double* xs = x + L.meta[s].vec_off;
  double acc = 0.0, acc2 = 0.0;
  if (valid) {
    // two entries per lane and iteration: both loads are issued before either product (the
    // rows hold up to 81 entries, so a single chain of dependent loads left the kernel
    // latency-bound); the two partial sums are added at the end, in a fixed order
    const int64_t q1 = L.row_ptr[row + 1];
    int64_t q = L.row_ptr[row] + l;
    for (; q + 16 < q1; q += 32) {
      const double v0 = L.val[q], v1 = L.val[q + 16];
      const int c0 = L.col[q], c1 = L.col[q + 16];
      acc += v0 * xs[c0];
      acc2 += v1 * xs[c1];
    }
    if (q < q1) acc += L.val[q] * xs[L.col[q]];
  }
  acc += acc2;
  for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (valid && l == 0) y[row] = (beta == 0.0 ? 0.0 : beta * y[row]) + alpha * acc;
}

template <typename Tin, typename Tout>
__global__ void k_convert(const Tin* __restrict__ in, Tout* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (Tout)in[i];
}

template <typename T>
__global__ void k_add_to_double(double* __restrict__ y, const T* __restrict__ x, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += (double)x[i];
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, double a, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

__global__ void k_coarse_gather(LevelDev L, const double* __restrict__ rc_sub, int64_t sum_nc, double* __restrict__ rC) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.n_coarse) return;
  rc_sub += (int64_t)blockIdx.y * sum_nc;
  double s = 0.0;
  for (int64_t o = L.cinv_ptr[g]; o < L.cinv_ptr[g + 1]; ++o) s += rc_sub[L.cinv_occ[o]];
  rC[(int64_t)blockIdx.y * L.n_coarse + g] = s;
}

__global__ void k_coarse_scatter(const int32_t* __restrict__ sub_coarse, int64_t total, const double* __restrict__ zC,
                                 int64_t n_coarse, double* __restrict__ zc_sub) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < total) zc_sub[(int64_t)blockIdx.y * total + t] = zC[(int64_t)blockIdx.y * n_coarse + sub_coarse[t]];
}

// deterministic dot: fixed grid, per-block tree, then a single block over the partials
__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                              double* __restrict__ partial) {
  __shared__ double red[256];
  a += (int64_t)blockIdx.y * n;
  b += (int64_t)blockIdx.y * n;
  partial += (int64_t)blockIdx.y * gridDim.x;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_dot_final(const double* __restrict__ partial, int nblk, double* __restrict__ out, int ostride) {
  __shared__ double red[256];
  partial += (int64_t)blockIdx.x * nblk;
  out += (int64_t)blockIdx.x * ostride;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += 256) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// scal layout (see capi.cpp): 0 rz, 1 pq, 2 alpha, 3 beta, 4 rz_new, 5 rr, 6 gg, 7 z.r_old, 8 frozen
__global__ void k_pcg_scalars(double* scal, int stage, int flexible, int nr) {
  if ((int)threadIdx.x >= nr) return;
  scal += 16 * threadIdx.x;   // column threadIdx.x of a block of right-hand sides
  if (scal[8] != 0.0) {   // converged column: freeze the iterate
    scal[2] = 0.0;
    scal[3] = 0.0;
    return;
  }
  if (stage == 0) {
    const double pq = scal[1];
    scal[2] = pq != 0.0 ? scal[0] / pq : 0.0;
  } else {
    const double rz_old = scal[0];
    const double num = flexible ? (scal[4] - scal[7]) : scal[4];
    scal[3] = rz_old != 0.0 ? num / rz_old : 0.0;
    scal[0] = scal[4];
  }
}

__global__ void k_pcg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                         const double* __restrict__ q, const double* __restrict__ scal, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t o = (int64_t)blockIdx.y * n;
  const double a = scal[16 * blockIdx.y + 2];
  x[o + i] += a * p[o + i];
  r[o + i] -= a * q[o + i];
}

__global__ void k_pcg_p(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ scal,
                        int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t o = (int64_t)blockIdx.y * n;
  p[o + i] = z[o + i] + scal[16 * blockIdx.y + 3] * p[o + i];
}

// grad[e] = -(1/coef_e) * sum_k lam_k,e^T K_e u_k,e ; one warp per element
__global__ void k_grad_contract(int64_t n_elems, int ne, const double* __restrict__ ke,
                                const int32_t* __restrict__ slot_elem, const double* __restrict__ coef,
                                const int32_t* __restrict__ conn, int ndof, const double* __restrict__ lam,
                                const double* __restrict__ u, int nrhs, int64_t n_full, double* __restrict__ grad) {
  const int64_t slot = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (slot >= n_elems) return;
  const int64_t e = slot_elem[slot];
  const double* K = ke + slot * (int64_t)ne * ne;
  const int32_t* cn = conn + e * (int64_t)(ne / ndof);
  auto dof = [&](int a) { return (int64_t)cn[a / ndof] * ndof + a % ndof; };
  double acc = 0.0;
  for (int k = 0; k < nrhs; ++k) {
    const double* lk = lam + (int64_t)k * n_full;
    const double* uk = u + (int64_t)k * n_full;
    for (int a = lane; a < ne; a += 32) {
      double t = 0.0;
      for (int b = 0; b < ne; ++b) t += K[a * ne + b] * uk[dof(b)];
      acc += lk[dof(a)] * t;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) grad[e] = -acc / coef[e];
}

__global__ void k_expand_free(const double* __restrict__ xf, const int64_t* __restrict__ free_of_full,
                              int64_t n_full, int nrhs, int64_t n_free, double* __restrict__ xfull) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_full * nrhs) return;
  const int64_t k = i / n_full, j = i % n_full;
  const int64_t f = free_of_full[j];
  xfull[i] = f >= 0 ? xf[k * n_free + f] : 0.0;
}

// dst[dst_off[k] + t] = src[src_off[k] + t], t < len[k]; one block per segment
__global__ void k_copy_segments(const double* __restrict__ src, const int64_t* __restrict__ src_off,
                                double* __restrict__ dst, const int64_t* __restrict__ dst_off,
                                const int64_t* __restrict__ len, int64_t n) {
  const int64_t k = blockIdx.x;
  if (k >= n) return;
  for (int64_t t = threadIdx.x; t < len[k]; t += blockDim.x) dst[dst_off[k] + t] = src[src_off[k] + t];
}

// g[k] = f[idx[k]] - t[k] (column blockIdx.y; f has columns of length fstride)
__global__ void k_iface_rhs(double* __restrict__ g, const double* __restrict__ f, int64_t fstride,
                            const int64_t* __restrict__ idx, const double* __restrict__ t, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t o = (int64_t)blockIdx.y * n;
  if (k < n) g[o + k] = f[(int64_t)blockIdx.y * fstride + idx[k]] - t[o + k];
}

// u[idx[k]] = v[k] (column blockIdx.y; u has columns of length ustride)
__global__ void k_put_indexed(double* __restrict__ u, int64_t ustride, const int64_t* __restrict__ idx,
                              const double* __restrict__ v, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) u[(int64_t)blockIdx.y * ustride + idx[k]] = v[(int64_t)blockIdx.y * n + k];
}

// BiCGstab (right preconditioned) device scalars; layout: 0 rho, 1 alpha, 2 omega, 3 rho_new,
// 4 rh.v, 5 t.s, 6 t.t, 7 beta.  A zero denominator (breakdown) yields 0, which the host sees as
// a stalled residual.
__global__ void k_bicg_scalars(double* S, int stage) {
  if (threadIdx.x != 0) return;
  if (stage == 3) {          // start: rho = alpha = omega = 1
    S[0] = S[1] = S[2] = 1.0;
  } else if (stage == 0) {   // beta = (rho_new / rho) (alpha / omega)
    S[7] = (S[0] != 0.0 && S[2] != 0.0) ? (S[3] / S[0]) * (S[1] / S[2]) : 0.0;
    S[0] = S[3];
  } else if (stage == 1) {   // alpha = rho / (rh . v)
    S[1] = S[4] != 0.0 ? S[0] / S[4] : 0.0;
  } else {                   // omega = (t . s) / (t . t)
    S[2] = S[6] != 0.0 ? S[5] / S[6] : 0.0;
  }
}

// p = r + beta (p - omega v)
__global__ void k_bicg_p(double* __restrict__ p, const double* __restrict__ r, const double* __restrict__ v,
                         const double* __restrict__ S, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = r[i] + S[7] * (p[i] - S[2] * v[i]);
}

// s = r - alpha v
__global__ void k_bicg_s(double* __restrict__ sv, const double* __restrict__ r, const double* __restrict__ v,
                         const double* __restrict__ S, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) sv[i] = r[i] - S[1] * v[i];
}

// x += alpha ph + omega sh ; r = s - omega t
__global__ void k_bicg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ ph,
                          const double* __restrict__ sh, const double* __restrict__ sv, const double* __restrict__ t,
                          const double* __restrict__ S, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] += S[1] * ph[i] + S[2] * sh[i];
  r[i] = sv[i] - S[2] * t[i];
}

// ---- flexible GMRES building blocks (fixed-order, reproducible) ----
// partial[i * nblk + b] = sum over the grid-stride slice b of V_i . w, for i < nv (grid nblk x nv)
__global__ void k_multidot_partial(const double* __restrict__ V, int64_t ldv, const double* __restrict__ w, int64_t n,
                                   double* __restrict__ partial) {
  __shared__ double red[256];
  const double* v = V + (int64_t)blockIdx.y * ldv;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += v[i] * w[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// out[i] = sum_b partial[i * nblk + b]; one block per i
__global__ void k_multidot_final(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
  __shared__ double red[256];
  const double* p = partial + (int64_t)blockIdx.x * nblk;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += 256) s += p[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// w += alpha sum_{i < nv} c_i V_i, i ascending
__global__ void k_combine(double* __restrict__ w, const double* __restrict__ V, int64_t ldv, int nv,
                          const double* __restrict__ c, double alpha, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double acc = 0.0;
  for (int i = 0; i < nv; ++i) acc += c[i] * V[(int64_t)i * ldv + k];
  w[k] += alpha * acc;
}

// dst = src / sqrt(*nrm2) (dst = 0 when the norm vanishes: lucky breakdown)
__global__ void k_scale_by_norm(double* __restrict__ dst, const double* __restrict__ src,
                                const double* __restrict__ nrm2, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double s = *nrm2 > 0.0 ? 1.0 / sqrt(*nrm2) : 0.0;
  dst[k] = src[k] * s;
}

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <typename T>
void launch_gather_iface(const LevelDev& L, const double* x, int weighted, T* loc, cudaStream_t st, int nr) {
  if (L.n_vec > 0) { note_launch(); k_gather_iface<T><<<dim3(nblocks(L.n_vec, 256), nr), 256, 0, st>>>(L, x, weighted, loc); }
}
template <typename T>
void launch_scatter_iface(const LevelDev& L, const T* loc, int weighted, double* y, cudaStream_t st, int nr) {
  if (L.n_iface > 0) { note_launch(); k_scatter_iface<T><<<dim3(nblocks(L.n_iface, 256), nr), 256, 0, st>>>(L, loc, weighted, y); }
}
template <typename T>
void launch_gather_glob(const LevelDev& L, const double* x, int part, T* loc, cudaStream_t st, int nr) {
  if (L.n_vec > 0) { note_launch(); k_gather_glob<T><<<dim3(nblocks(L.n_vec, 256), nr), 256, 0, st>>>(L, x, part, loc); }
}
template <typename T>
void launch_scatter_interior(const LevelDev& L, const T* loc, double* y, cudaStream_t st, int nr) {
  if (L.n_vec > 0) { note_launch(); k_scatter_interior<T><<<dim3(nblocks(L.n_vec, 256), nr), 256, 0, st>>>(L, loc, y); }
}
void launch_spmv_rows(const LevelDev& L, const int64_t* rows, int64_t nrows, const double* x, double* y, double alpha,
                      double beta, const int32_t* row_sub, cudaStream_t st, int nr) {
  if (nrows > 0) { note_launch(); k_spmv<<<dim3(nblocks(nrows, 16), nr), 256, 0, st>>>(L, rows, nrows, x, y, alpha, beta, row_sub); }
}
template <typename Tin, typename Tout>
void launch_convert(const Tin* in, Tout* out, int64_t n, cudaStream_t st) {
  if (n > 0) { note_launch(); k_convert<Tin, Tout><<<nblocks(n, 256), 256, 0, st>>>(in, out, n); }
}
template <typename T>
void launch_add_to_double(double* y, const T* x, int64_t n, cudaStream_t st) {
  if (n > 0) { note_launch(); k_add_to_double<T><<<nblocks(n, 256), 256, 0, st>>>(y, x, n); }
}
void launch_axpy_loc(double* y, const double* x, double a, int64_t n, cudaStream_t st) {
  if (n > 0) { note_launch(); k_axpy<<<nblocks(n, 256), 256, 0, st>>>(y, x, a, n); }
}
void launch_coarse_gather(const LevelDev& L, const double* rc_sub, int64_t sum_nc, double* rC, cudaStream_t st, int nr) {
  if (L.n_coarse > 0) { note_launch(); k_coarse_gather<<<dim3(nblocks(L.n_coarse, 256), nr), 256, 0, st>>>(L, rc_sub, sum_nc, rC); }
}
void launch_coarse_scatter_n(const int32_t* sub_coarse, int64_t total, const double* zC, int64_t n_coarse,
                             double* zc_sub, cudaStream_t st, int nr) {
  if (total > 0) { note_launch(); k_coarse_scatter<<<dim3(nblocks(total, 256), nr), 256, 0, st>>>(sub_coarse, total, zC, n_coarse, zc_sub); }
}
void launch_dot(const double* a, const double* b, int64_t n, double* partial, int nblk, double* out, cudaStream_t st,
                int nr, int ostride) {
  { note_launch(); k_dot_partial<<<dim3(nblk, nr), 256, 0, st>>>(a, b, n, partial); }
  { note_launch(); k_dot_final<<<nr, 256, 0, st>>>(partial, nblk, out, ostride); }
}
void launch_pcg_update_x_r(double* x, double* r, const double* p, const double* q, const double* scal, int64_t n,
                           cudaStream_t st, int nr) {
  if (n > 0) { note_launch(); k_pcg_xr<<<dim3(nblocks(n, 256), nr), 256, 0, st>>>(x, r, p, q, scal, n); }
}
void launch_pcg_update_p(double* p, const double* z, const double* scal, int64_t n, cudaStream_t st, int nr) {
  if (n > 0) { note_launch(); k_pcg_p<<<dim3(nblocks(n, 256), nr), 256, 0, st>>>(p, z, scal, n); }
}
void launch_pcg_scalars(double* scal, int stage, int flexible, cudaStream_t st, int nr) {
  { note_launch(); k_pcg_scalars<<<1, 32, 0, st>>>(scal, stage, flexible, nr); }
}
void launch_grad_contract_slots(int64_t n_elems, int ne, const double* ke, const int32_t* slot_elem, const double* coef,
                                const int32_t* conn, int ndof, const double* lam, const double* u, int nrhs,
                                int64_t n_full, double* grad, cudaStream_t st) {
  if (n_elems > 0)
    { note_launch(); k_grad_contract<<<nblocks(n_elems, 8), 256, 0, st>>>(n_elems, ne, ke, slot_elem, coef, conn, ndof, lam, u,
                                                          nrhs, n_full, grad); }
}
void launch_expand_free(const double* xf, const int64_t* free_of_full, int64_t n_full, int nrhs, int64_t n_free,
                        double* xfull, cudaStream_t st) {
  if (n_full > 0)
    { note_launch(); k_expand_free<<<nblocks(n_full * nrhs, 256), 256, 0, st>>>(xf, free_of_full, n_full, nrhs, n_free, xfull); }
}

void launch_copy_segments(const double* src, const int64_t* src_off, double* dst, const int64_t* dst_off,
                          const int64_t* len, int64_t n, cudaStream_t st) {
  if (n > 0) { note_launch(); k_copy_segments<<<(unsigned)n, 256, 0, st>>>(src, src_off, dst, dst_off, len, n); }
}
void launch_iface_rhs(double* g, const double* f, int64_t fstride, const int64_t* idx, const double* t, int64_t n,
                      cudaStream_t st, int nr) {
  if (n > 0) { note_launch(); k_iface_rhs<<<dim3(nblocks(n, 256), nr), 256, 0, st>>>(g, f, fstride, idx, t, n); }
}
void launch_put_indexed(double* u, int64_t ustride, const int64_t* idx, const double* v, int64_t n, cudaStream_t st,
                        int nr) {
  if (n > 0) { note_launch(); k_put_indexed<<<dim3(nblocks(n, 256), nr), 256, 0, st>>>(u, ustride, idx, v, n); }
}

void launch_multidot(const double* V, int64_t ldv, int nv, const double* w, int64_t n, double* partial, int nblk,
                     double* out, cudaStream_t st) {
  if (nv <= 0) return;
  note_launch();
  k_multidot_partial<<<dim3(nblk, nv), 256, 0, st>>>(V, ldv, w, n, partial);
  note_launch();
  k_multidot_final<<<nv, 256, 0, st>>>(partial, nblk, out);
}
void launch_combine(double* w, const double* V, int64_t ldv, int nv, const double* c, double alpha, int64_t n,
                    cudaStream_t st) {
  if (n > 0 && nv > 0) { note_launch(); k_combine<<<nblocks(n, 256), 256, 0, st>>>(w, V, ldv, nv, c, alpha, n); }
}
void launch_scale_by_norm(double* dst, const double* src, const double* nrm2, int64_t n, cudaStream_t st) {
  if (n > 0) { note_launch(); k_scale_by_norm<<<nblocks(n, 256), 256, 0, st>>>(dst, src, nrm2, n); }
}

void launch_bicg_scalars(double* S, int stage, cudaStream_t st) {
  note_launch();
  k_bicg_scalars<<<1, 32, 0, st>>>(S, stage);
}
void launch_bicg_p(double* p, const double* r, const double* v, const double* S, int64_t n, cudaStream_t st) {
  if (n > 0) { note_launch(); k_bicg_p<<<nblocks(n, 256), 256, 0, st>>>(p, r, v, S, n); }
}
void launch_bicg_s(double* sv, const double* r, const double* v, const double* S, int64_t n, cudaStream_t st) {
  if (n > 0) { note_launch(); k_bicg_s<<<nblocks(n, 256), 256, 0, st>>>(sv, r, v, S, n); }
}
void launch_bicg_xr(double* x, double* r, const double* ph, const double* sh, const double* sv, const double* t,
                    const double* S, int64_t n, cudaStream_t st) {
  if (n > 0) { note_launch(); k_bicg_xr<<<nblocks(n, 256), 256, 0, st>>>(x, r, ph, sh, sv, t, S, n); }
}

#define INST(T)                                                                             \
  template void launch_gather_iface<T>(const LevelDev&, const double*, int, T*, cudaStream_t, int); \
  template void launch_scatter_iface<T>(const LevelDev&, const T*, int, double*, cudaStream_t, int); \
  template void launch_gather_glob<T>(const LevelDev&, const double*, int, T*, cudaStream_t, int);  \
  template void launch_scatter_interior<T>(const LevelDev&, const T*, double*, cudaStream_t, int);  \
  template void launch_add_to_double<T>(double*, const T*, int64_t, cudaStream_t);
INST(float)
INST(double)
#undef INST
template void launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace bddc
