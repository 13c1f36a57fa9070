// Assembly kernels: element matrices, sub-assembly of K_i (Sec. 2: "obtained by the
// sub-assembling of element matrices"), the augmented matrix K_i + rho C_i^T C_i with the
// constraint rows appended, and the interface weights.
//
// Every reduction here runs in a fixed order (one warp per matrix row, contributions in
// ascending element order), so two runs give bit-identical factors.
#include "internal.h"

namespace bddc {

namespace {

__device__ __forceinline__ int64_t tile_index(int i, int j, int Bc) {
  return i < Bc ? ((int64_t)i * (i + 1) / 2 + j) : ((int64_t)Bc * (Bc + 1) / 2 + (int64_t)(i - Bc) * Bc + j);
}

// One warp per element.  Q1 element (SIMPLEX = false): lexicographic local nodes, 2-point Gauss
// rule per direction; the Gauss point g has reference coordinates xi_d = (2 bit_d(g) - 1)/sqrt(3).
// Linear simplex (SIMPLEX = true; triangles, tetrahedra): the affine map from the reference
// simplex, N_0 = 1 - sum_d xi_d and N_a = xi_{a-1}, has constant gradients, so one point with
// weight 1/DIM! (the reference volume) integrates the constant integrand exactly; |det J| makes
// the element independent of its vertex orientation.
template <int DIM, bool SIMPLEX>
__global__ void k_elem_q1p1(int physics, int64_t n_elems, const double* __restrict__ coords,
                          const int32_t* __restrict__ conn, const double* __restrict__ coef, double nu,
                          const int32_t* __restrict__ slot_elem, double* __restrict__ ke) {
  constexpr int NN = SIMPLEX ? DIM + 1 : 1 << DIM;   // nodes
  constexpr int NG = SIMPLEX ? 1 : NN;               // quadrature points
  constexpr int WARPS = 4;
  __shared__ double sG[WARPS][NG][NN][DIM];   // [gp][node][d] physical gradients
  __shared__ double sW[WARPS][NG];            // detJ * weight
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slot = (int64_t)blockIdx.x * WARPS + w;
  if (slot >= n_elems) return;
  const int64_t e = slot_elem ? slot_elem[slot] : slot;
  const double gq = 0.57735026918962576451;   // 1/sqrt(3)
  if (lane < NG) {
    double G[NN][DIM];
    if (SIMPLEX) {
      for (int a = 0; a < NN; ++a)
        for (int d = 0; d < DIM; ++d) G[a][d] = a == 0 ? -1.0 : (a - 1 == d ? 1.0 : 0.0);
    } else {
      double xi[DIM];
      for (int d = 0; d < DIM; ++d) xi[d] = ((lane >> d) & 1) ? gq : -gq;
      for (int a = 0; a < NN; ++a)
        for (int d = 0; d < DIM; ++d) {
          double v = (((a >> d) & 1) ? 1.0 : -1.0) * 0.5;
          for (int d2 = 0; d2 < DIM; ++d2)
            if (d2 != d) v *= (1.0 + (((a >> d2) & 1) ? 1.0 : -1.0) * xi[d2]) * 0.5;
          G[a][d] = v;
        }
    }
    double J[DIM][DIM];
    for (int d = 0; d < DIM; ++d)
      for (int d2 = 0; d2 < DIM; ++d2) {
        double s = 0.0;
        for (int a = 0; a < NN; ++a) s += coords[(int64_t)conn[e * NN + a] * DIM + d] * G[a][d2];
        J[d][d2] = s;
      }
    double inv[DIM][DIM], det;
    if (DIM == 2) {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      inv[0][0] = J[1][1] / det;
      inv[0][1] = -J[0][1] / det;
      inv[1][0] = -J[1][0] / det;
      inv[1][1] = J[0][0] / det;
    } else {
      double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
      inv[0][0] = c00 / det;
      inv[1][0] = c01 / det;
      inv[2][0] = c02 / det;
      inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
      inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
      inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
      inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
      inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
      inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    }
    for (int a = 0; a < NN; ++a)
      for (int d = 0; d < DIM; ++d) {
        double s = 0.0;
        for (int d2 = 0; d2 < DIM; ++d2) s += G[a][d2] * inv[d2][d];
        sG[w][lane][a][d] = s;
      }
    sW[w][lane] = SIMPLEX ? fabs(det) / (DIM == 2 ? 2.0 : 6.0) : det;
  }
  __syncwarp();
  const double E = coef[e];
  if (physics == 0) {
    for (int idx = lane; idx < NN * NN; idx += 32) {
      int a = idx / NN, b = idx % NN;
      double s = 0.0;
      for (int g = 0; g < NG; ++g) {
        double d = 0.0;
        for (int k = 0; k < DIM; ++k) d += sG[w][g][a][k] * sG[w][g][b][k];
        s += sW[w][g] * d;
      }
      ke[slot * NN * NN + idx] = E * s;
    }
  } else {
    const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = E / (2.0 * (1.0 + nu));
    constexpr int ND = NN * DIM;
    // lane p takes the node pair (a, b), a <= b, and makes the DIM x DIM block
    //   K_ab[i][j] = sum_g w_g (lam ga_i gb_j + mu ga_j gb_i + mu (ga . gb) delta_ij)
    //             = lam P_ij + mu P_ji + mu tr(P) delta_ij,   P = sum_g w_g ga gb^T
    // (ga, gb: physical gradients of the shape functions of nodes a, b at Gauss point g) and its
    // mirror K_ba = K_ab^T: DIM^2 products per Gauss point and pair (FP64 is the scarce unit)
    double* kout = ke + slot * ND * ND;
    for (int p = lane; p < NN * (NN + 1) / 2; p += 32) {
      int a = 0, r = p;
      while (r >= NN - a) {
        r -= NN - a;
        ++a;
      }
      const int b = a + r;
      double P[DIM][DIM];
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = 0; j < DIM; ++j) P[i][j] = 0.0;
#pragma unroll 2
      for (int g = 0; g < NG; ++g) {
        const double wg = sW[w][g];
        double ga[DIM], gb[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          ga[k] = wg * sG[w][g][a][k];
          gb[k] = sG[w][g][b][k];
        }
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
          for (int j = 0; j < DIM; ++j) P[i][j] += ga[i] * gb[j];
      }
      double tr = 0.0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) tr += P[k][k];
      double blk[DIM][DIM];
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = 0; j < DIM; ++j) blk[i][j] = lam * P[i][j] + mu * P[j][i] + (i == j ? mu * tr : 0.0);
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
          kout[(a * DIM + i) * ND + b * DIM + j] = blk[i][j];
          if (a != b) kout[(b * DIM + j) * ND + a * DIM + i] = blk[i][j];
        }
    }
  }
}

// Taylor-Hood Q2-Q1 hex (Stokes, Sec. 4), one block per element, DOF slot 4a + c (node a of 27,
// component c: u, v, w, p).  A[(a,i),(b,j)] = coef delta_ij int grad phi_a . grad phi_b,
// B[(p,3),(b,j)] = -coef int psi_p d phi_b / dx_j (psi_p: Q1 function of vertex p) and its
// transpose; 3x3x3 Gauss rule, isoparametric Q2 geometry; pressure slots of non-vertex nodes
// stay zero.  Thread t accumulates entries t, t+256, ... of the 27x27 Laplacian and the 8x81 B.
__global__ void __launch_bounds__(256) k_elem_q2q1(int64_t n_elems, const double* __restrict__ coords,
                                                   const int32_t* __restrict__ conn, const double* __restrict__ coef,
                                                   const int32_t* __restrict__ slot_elem, double* __restrict__ ke) {
  constexpr int NE = 108, NLAP = 27 * 27, NB_ = 8 * 81, NACC = (NLAP + NB_ + 255) / 256;
  const int64_t slot = blockIdx.x;
  if (slot >= n_elems) return;
  const int64_t e = slot_elem ? slot_elem[slot] : slot;
  __shared__ double X[27][3], Gr[27][3], Gx[27][3], psi[8], Ji[3][3], wd;
  const int tid = threadIdx.x;
  if (tid < 81) X[tid / 3][tid % 3] = coords[(int64_t)conn[e * 27 + tid / 3] * 3 + tid % 3];
  double acc[NACC];
#pragma unroll
  for (int u = 0; u < NACC; ++u) acc[u] = 0.0;
  const double gq[3] = {-0.77459666924148337704, 0.0, 0.77459666924148337704};   // +-sqrt(3/5), 0
  const double gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  __syncthreads();
  for (int g = 0; g < 27; ++g) {
    const double xi[3] = {gq[g % 3], gq[(g / 3) % 3], gq[g / 9]};
    if (tid < 27) {
      const int ix[3] = {tid % 3, (tid / 3) % 3, tid / 9};
      double f[3], d[3];
      for (int k = 0; k < 3; ++k) {
        const double x = xi[k];
        f[k] = ix[k] == 0 ? 0.5 * x * (x - 1.0) : (ix[k] == 1 ? 1.0 - x * x : 0.5 * x * (x + 1.0));
        d[k] = ix[k] == 0 ? x - 0.5 : (ix[k] == 1 ? -2.0 * x : x + 0.5);
      }
      Gr[tid][0] = d[0] * f[1] * f[2];
      Gr[tid][1] = f[0] * d[1] * f[2];
      Gr[tid][2] = f[0] * f[1] * d[2];
    }
    if (tid >= 32 && tid < 40) {
      const int p = tid - 32;
      double v = 1.0;
      for (int k = 0; k < 3; ++k) v *= 0.5 * (1.0 + (((p >> k) & 1) ? 1.0 : -1.0) * xi[k]);
      psi[p] = v;
    }
    __syncthreads();
    if (tid == 0) {
      double J[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double sacc = 0.0;
          for (int n = 0; n < 27; ++n) sacc += X[n][a] * Gr[n][b];
          J[a][b] = sacc;
        }
      const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
      Ji[0][0] = c00 / det;
      Ji[1][0] = c01 / det;
      Ji[2][0] = c02 / det;
      Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
      Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
      Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
      Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
      Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
      Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
      wd = gw[g % 3] * gw[(g / 3) % 3] * gw[g / 9] * det;
    }
    __syncthreads();
    if (tid < 81) {
      const int a = tid / 3, k = tid % 3;
      Gx[a][k] = Gr[a][0] * Ji[0][k] + Gr[a][1] * Ji[1][k] + Gr[a][2] * Ji[2][k];
    }
    __syncthreads();
    const double w = wd;
#pragma unroll
    for (int u = 0; u < NACC; ++u) {
      const int t = tid + 256 * u;
      if (t < NLAP) {
        const int a = t / 27, b = t % 27;
        acc[u] += w * (Gx[a][0] * Gx[b][0] + Gx[a][1] * Gx[b][1] + Gx[a][2] * Gx[b][2]);
      } else if (t < NLAP + NB_) {
        const int q = t - NLAP, p = q / 81, r = q % 81;
        acc[u] -= w * psi[p] * Gx[r / 3][r % 3];
      }
    }
    __syncthreads();
  }
  double* K = ke + slot * (int64_t)NE * NE;
  for (int t = tid; t < NE * NE; t += 256) K[t] = 0.0;
  __syncthreads();
  const double cf = coef[e];
#pragma unroll
  for (int u = 0; u < NACC; ++u) {
    const int t = tid + 256 * u;
    if (t < NLAP) {
      const int a = t / 27, b = t % 27;
      for (int i = 0; i < 3; ++i) K[(4 * a + i) * NE + 4 * b + i] = cf * acc[u];
    } else if (t < NLAP + NB_) {
      const int q = t - NLAP, p = q / 81, r = q % 81, b = r / 3, j = r % 3;
      const int a = 2 * (p & 1) + 6 * ((p >> 1) & 1) + 18 * ((p >> 2) & 1);   // vertex node of pressure p
      K[(4 * a + 3) * NE + 4 * b + j] = cf * acc[u];
      K[(4 * b + j) * NE + 4 * a + 3] = cf * acc[u];
    }
  }
}

// Dirichlet lifting: lift[g] = - sum over the element rows (slot, a) holding free DOF g of
// sum_b K_e[a][b] u_d[b] (u_d: prescribed values of the element's slots, 0 on free slots).
// One warp per free DOF, element rows in a fixed order.
__global__ void k_lift(int64_t n_free, int ne, const int64_t* __restrict__ lptr, const int32_t* __restrict__ lslot,
                       const int32_t* __restrict__ la, const double* __restrict__ ke, const double* __restrict__ ud,
                       double* __restrict__ lift) {
  const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= n_free) return;
  double acc = 0.0;
  for (int64_t c = lptr[g]; c < lptr[g + 1]; ++c) {
    const int64_t k = lslot[c];
    const double* row = ke + k * (int64_t)ne * ne + (int64_t)la[c] * ne;
    const double* u = ud + k * (int64_t)ne;
    for (int b = lane; b < ne; b += 32) acc += row[b] * u[b];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) lift[g] = -acc;
}

// One warp per padded local row: CSR values of K_i from the element matrices containing the
// row's DOF, in ascending element order.
__global__ void k_csr_values(LevelDev L, const int32_t* __restrict__ row_sub) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= L.n_vec) return;
  const int64_t p0 = L.row_ptr[row], p1 = L.row_ptr[row + 1];
  for (int64_t q = p0 + lane; q < p1; q += 32) L.val[q] = 0.0;
  __syncwarp();
  const int32_t* cols = L.col + p0;
  const int len = (int)(p1 - p0);
  for (int64_t c = L.rc_ptr[row]; c < L.rc_ptr[row + 1]; ++c) {
    const int k = L.rc_elem[c], a = L.rc_a[c];
    const int64_t eo = L.ed_off[k];
    const int ne = (int)(L.ed_off[k + 1] - eo);
    const double* kr = L.ke + L.ke_off[k] + (int64_t)a * ne;
    for (int b = lane; b < ne; b += 32) {
      const int col = L.eldof[eo + b];
      if (col < 0) continue;
      int lo = 0, hi = len - 1;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (cols[mid] < col) lo = mid + 1; else hi = mid;
      }
      L.val[p0 + lo] += kr[b];
    }
    __syncwarp();
  }
  if (lane == 0 && len > 0) {
    const int s = row_sub[row];
    const int r = (int)(row - L.meta[s].vec_off);
    double d = 0.0;
    for (int q = 0; q < len; ++q)
      if (cols[q] == r) d = L.val[p0 + q];
    L.diag[row] = d;
  }
}

// One warp per padded row: write the lower part of the row into the tiles; identity on
// padding rows.  Tiles are zeroed beforehand.
template <typename T>
__global__ void k_densify(LevelDev L, const int32_t* __restrict__ row_sub) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= L.n_vec) return;
  const int s = row_sub[row];
  const SubMeta m = L.meta[s];
  const int r = (int)(row - m.vec_off);
  T* tiles = (T*)L.tiles;
  const int i = r / NB, rr = r % NB;
  const bool pad = (r >= m.nI && r < m.nIb * NB) || (r >= m.nIb * NB + m.nG);
  if (pad) {
    if (lane == 0) tiles[m.tile_off + tile_index(i, i, m.Bc) * NB2 + rr * NB + rr] = (T)1;
    return;
  }
  for (int64_t q = L.row_ptr[row] + lane; q < L.row_ptr[row + 1]; q += 32) {
    const int c = L.col[q];
    if (c > r) continue;
    tiles[m.tile_off + tile_index(i, c / NB, m.Bc) * NB2 + rr * NB + (c % NB)] = (T)L.val[q];
  }
}

// One block per subdomain: rho = mean diag K_i, A += C^T R C with R = diag(rho c_rho) (rows one
// after another; c_rho = 0 leaves a row unaugmented),
// then the constraint rows into block rows Bc .. Bc+ncb-1.
template <typename T>
__global__ void k_add_constraints(LevelDev L) {
  const int s = blockIdx.x;
  const SubMeta m = L.meta[s];
  __shared__ double red[256];
  double acc = 0.0;
  for (int r = threadIdx.x; r < m.nI; r += blockDim.x) acc += L.diag[m.vec_off + r];
  for (int r = threadIdx.x; r < m.nG; r += blockDim.x) acc += L.diag[m.vec_off + m.nIb * NB + r];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  const double rho = m.n > 0 ? red[0] / (double)m.n : 1.0;
  if (threadIdx.x == 0) L.rho[s] = rho;
  T* tiles = (T*)L.tiles;
  for (int q = 0; q < m.nc; ++q) {
    const int64_t e0 = L.c_ptr[m.c_off + q], e1 = L.c_ptr[m.c_off + q + 1];
    const int cnt = (int)(e1 - e0);
    const double rq = rho * L.c_rho[m.c_off + q];   // 0 for rows that are not augmented (Stokes pressures)
    for (int t = threadIdx.x; t < cnt * cnt && rq != 0.0; t += blockDim.x) {
      const int x = t / cnt, y = t % cnt;
      const int pa = L.c_pos[e0 + x], pb = L.c_pos[e0 + y];
      if (pb > pa) continue;
      T* p = tiles + m.tile_off + tile_index(pa / NB, pb / NB, m.Bc) * NB2 + (pa % NB) * NB + (pb % NB);
      *p = (T)((double)*p + rq * L.c_val[e0 + x] * L.c_val[e0 + y]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int pa = L.c_pos[e0 + t];
      tiles[m.tile_off + tile_index(m.Bc + q / NB, pa / NB, m.Bc) * NB2 + (q % NB) * NB + (pa % NB)] =
          (T)L.c_val[e0 + t];
    }
    __syncthreads();
  }
}

// Interface weights: stiffness D_i(j) = K_i(jj) / sum_k K_k(jj), or multiplicity 1/count (also
// used where the diagonal sum is zero, as for Stokes pressures).
__global__ void k_weights(LevelDev L, int multiplicity) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.n_iface) return;
  const int64_t o0 = L.iface_ptr[g], o1 = L.iface_ptr[g + 1];
  if (multiplicity) {
    const double w = 1.0 / (double)(o1 - o0);
    for (int64_t o = o0; o < o1; ++o) L.w[L.iface_occ[o]] = w;
    return;
  }
  double s = 0.0;
  for (int64_t o = o0; o < o1; ++o) s += L.diag[L.iface_occ[o]];
  if (!(s > 0.0)) {   // zero diagonal (Stokes pressures): multiplicity weights
    const double w = 1.0 / (double)(o1 - o0);
    for (int64_t o = o0; o < o1; ++o) L.w[L.iface_occ[o]] = w;
    return;
  }
  for (int64_t o = o0; o < o1; ++o) L.w[L.iface_occ[o]] = L.diag[L.iface_occ[o]] / s;
}

}  // namespace

void launch_elem_q1p1(int physics, int dim, int simplex, int64_t n_elems, const double* coords, const int32_t* conn,
                    const double* coef, double nu, const int32_t* slot_elem, double* ke, cudaStream_t st) {
  if (n_elems <= 0) return;
  const int blocks = (int)((n_elems + 3) / 4);
  note_launch();
  if (dim == 2 && simplex)
    k_elem_q1p1<2, true><<<blocks, 128, 0, st>>>(physics, n_elems, coords, conn, coef, nu, slot_elem, ke);
  else if (dim == 2)
    k_elem_q1p1<2, false><<<blocks, 128, 0, st>>>(physics, n_elems, coords, conn, coef, nu, slot_elem, ke);
  else if (simplex)
    k_elem_q1p1<3, true><<<blocks, 128, 0, st>>>(physics, n_elems, coords, conn, coef, nu, slot_elem, ke);
  else
    k_elem_q1p1<3, false><<<blocks, 128, 0, st>>>(physics, n_elems, coords, conn, coef, nu, slot_elem, ke);
}

void launch_elem_q2q1(int64_t n_elems, const double* coords, const int32_t* conn, const double* coef,
                      const int32_t* slot_elem, double* ke, cudaStream_t st) {
  if (n_elems <= 0) return;
  note_launch();
  k_elem_q2q1<<<(unsigned)n_elems, 256, 0, st>>>(n_elems, coords, conn, coef, slot_elem, ke);
}

// ke[k] = ke_elem[slot_elem[k]]: element matrices computed in element order, gathered into slots
__global__ void k_gather_elems(int64_t n_elems, int64_t ne2, const int32_t* __restrict__ slot_elem,
                               const double* __restrict__ ke_elem, double* __restrict__ ke) {
  const int64_t k = blockIdx.x;
  if (k >= n_elems) return;
  const double* src = ke_elem + (int64_t)slot_elem[k] * ne2;
  double* dst = ke + k * ne2;
  for (int64_t t = threadIdx.x; t < ne2; t += blockDim.x) dst[t] = __ldcs(src + t);
}

void launch_gather_elems(int64_t n_elems, int ne, const int32_t* slot_elem, const double* ke_elem, double* ke,
                         cudaStream_t st) {
  if (n_elems <= 0) return;
  note_launch();
  k_gather_elems<<<(unsigned)n_elems, 128, 0, st>>>(n_elems, (int64_t)ne * ne, slot_elem, ke_elem, ke);
}

void launch_lift(int64_t n_free, int ne, const int64_t* lptr, const int32_t* lslot, const int32_t* la,
                 const double* ke, const double* ud, double* lift, cudaStream_t st) {
  if (n_free <= 0) return;
  note_launch();
  k_lift<<<(unsigned)((n_free + 7) / 8), 256, 0, st>>>(n_free, ne, lptr, lslot, la, ke, ud, lift);
}

// CSR pattern of K_i on the device: one warp per padded local row marks, in a per-warp bitmap
// over the subdomain's padded positions, the positions of every element containing the row;
// the set bits, read in ascending order, are the row's columns.  Pass 1 (cnt != null) counts,
// pass 2 (col != null) writes at row_ptr.
__global__ void k_csr_pattern(LevelDev L, int64_t n_rows, const int32_t* __restrict__ row_sub, int words,
                              int32_t* __restrict__ cnt, const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col) {
  extern __shared__ uint32_t bm_all[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (row >= n_rows) return;
  uint32_t* bm = bm_all + (size_t)warp * words;
  const SubMeta m = L.meta[row_sub[row]];
  const int nw = (m.Bc * NB + 31) >> 5;
  for (int w = lane; w < nw; w += 32) bm[w] = 0u;
  __syncwarp();
  for (int64_t c = L.rc_ptr[row]; c < L.rc_ptr[row + 1]; ++c) {
    const int64_t k = L.rc_elem[c];
    for (int64_t t = L.ed_off[k] + lane; t < L.ed_off[k + 1]; t += 32) {
      const int32_t p = L.eldof[t];
      if (p >= 0) atomicOr(&bm[p >> 5], 1u << (p & 31));
    }
  }
  __syncwarp();
  if (cnt) {
    int tot = 0;
    for (int w = lane; w < nw; w += 32) tot += __popc(bm[w]);
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) cnt[row] = tot;
    return;
  }
  int64_t out = row_ptr[row];
  for (int w0 = 0; w0 < nw; w0 += 32) {
    const int w = w0 + lane;
    uint32_t bits = w < nw ? bm[w] : 0u;
    const int pc = __popc(bits);
    int pre = pc;   // inclusive prefix over the lanes
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += v;
    }
    int64_t dst = out + (pre - pc);
    while (bits) {
      const int b = __ffs(bits) - 1;
      col[dst++] = (int32_t)(w * 32 + b);
      bits &= bits - 1;
    }
    out += __shfl_sync(0xffffffffu, pre, 31);
  }
}

void launch_csr_pattern(const LevelDev& L, int64_t n_rows, const int32_t* row_sub, int max_len, int32_t* cnt,
                        const int64_t* row_ptr, int32_t* col, cudaStream_t st) {
  if (n_rows <= 0) return;
  const int words = (max_len + 31) / 32;
  const size_t sm = (size_t)8 * words * sizeof(uint32_t);
  static size_t attr = 0;
  if (sm > 48 * 1024 && sm > attr) {
    cudaFuncSetAttribute(k_csr_pattern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = sm;
  }
  note_launch();
  k_csr_pattern<<<(unsigned)((n_rows + 7) / 8), 256, sm, st>>>(L, n_rows, row_sub, words, cnt, row_ptr, col);
}

void launch_csr_values(const LevelDev& L, int64_t n_rows_total, const int32_t* row_sub, cudaStream_t st) {
  (void)n_rows_total;
  if (L.n_vec <= 0) return;
  { note_launch(); k_csr_values<<<(unsigned)((L.n_vec + 7) / 8), 256, 0, st>>>(L, row_sub); }
}

template <typename T>
void launch_densify_rows(const LevelDev& L, const int32_t* row_sub, cudaStream_t st) {
  if (L.n_vec <= 0) return;
  { note_launch(); k_densify<T><<<(unsigned)((L.n_vec + 7) / 8), 256, 0, st>>>(L, row_sub); }
}

template <typename T>
void launch_add_constraints(const LevelDev& L, cudaStream_t st) {
  if (L.n_sub <= 0) return;
  { note_launch(); k_add_constraints<T><<<(unsigned)L.n_sub, 256, 0, st>>>(L); }
}

void launch_weights(const LevelDev& L, int multiplicity, const double*, cudaStream_t st) {
  if (L.n_iface <= 0) return;
  { note_launch(); k_weights<<<(unsigned)((L.n_iface + 255) / 256), 256, 0, st>>>(L, multiplicity); }
}

template void launch_densify_rows<float>(const LevelDev&, const int32_t*, cudaStream_t);
template void launch_densify_rows<double>(const LevelDev&, const int32_t*, cudaStream_t);
template void launch_add_constraints<float>(const LevelDev&, cudaStream_t);
template void launch_add_constraints<double>(const LevelDev&, cudaStream_t);

}  // namespace bddc
