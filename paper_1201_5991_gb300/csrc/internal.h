// Internal declarations shared by the host orchestration (capi.cpp) and the kernels.
//
// Device layout of one BDDC level (all subdomains of a level are batched in every launch):
//   * A subdomain's local DOFs live in a padded local vector of Bc*NB entries:
//       [interior (nI) | pad to nIb*NB | interface (nG) | pad to Bc*NB],  Bc = nIb + nGb.
//     The identity padding decouples, so the leading nIb block rows of the factor are the
//     Cholesky factor of K_II and the trailing nGb block rows hold the factor of the
//     Schur complement plus rho C^T C.
//   * The augmented matrix [K_i + rho C_i^T C_i ; C_i] is stored as NB x NB tiles, row-major
//     inside a tile, tiles ordered block row after block row; block row i holds tiles
//     j = 0 .. min(i, Bc-1).  Block rows Bc .. Bc+ncb-1 hold the constraint rows; after the
//     partial Cholesky they hold Y = C L^{-T} (nonzero only in interface columns).
//   * The inverses of the Bc diagonal factor tiles are kept next to the factor.
//   * Symmetric indefinite levels (Stokes) use a signed Cholesky A = L S L^T with S = diag(+-1)
//     and no pivoting (velocities precede pressures in both blocks); SPD levels have S = I.
//     Then the constraint block rows hold Y S (Y = C L^{-T}), G = C A^{-1} C^T = (Y S) S (Y S)^T,
//     Psi = L^{-T} (Y S)^T G^{-1}, and the forward sweep leaves S L^{-1} r.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace bddc {

constexpr int NB = 64;            // tile edge
constexpr int64_t NB2 = NB * NB;

struct SubMeta {
  int32_t n, nI, nG, nc;          // local sizes
  int32_t nIb, nGb, ncb, Bc;      // block counts; Bc = nIb + nGb
  int32_t R;                      // block rows = Bc + ncb
  int32_t pad0;
  int64_t tile_off;               // element offset of the tiles in the level's tile buffer
  int64_t dinv_off;               // element offset of the Bc diagonal inverses
  int64_t vec_off;                // offset of the padded local vector
  int64_t row_off;                // offset into the level's CSR row pointer (Bc*NB + 1 entries)
  int64_t c_off;                  // offset of the per-subdomain coarse vector (nc)
  int64_t g_off;                  // offset of nc x nc matrices (G^{-1}, K_C)
  int64_t psi_off;                // offset of Psi_G (nGb*NB rows x nc, row-major)
  int64_t psiT_off;               // offset of Psi_G^T as ncb x nGb tiles (set-up copy for the solve phase)
  int64_t schur_off;              // offset of the explicit augmented Schur complement (nGb (nGb+1)/2 tiles)
};

// Raw device pointers of one level, passed by value to kernels.
struct LevelDev {
  int64_t n_sub;
  int64_t n_dof;                  // level DOFs (level 1: free DOFs; level l: coarse DOFs of l-1)
  int64_t n_iface;
  int64_t n_coarse;
  int64_t n_vec;                  // total padded local length
  const SubMeta* meta;
  // CSR of K_i per subdomain over padded positions (FP64)
  const int64_t* row_ptr;         // [sum (Bc*NB+1)], absolute offsets into col/val
  const int32_t* col;             // padded local column
  double* val;
  // element -> padded local positions, element matrices
  const int64_t* ke_off;          // [n_elems + 1] offsets into ke (ne_k^2 each)
  const int64_t* ed_off;          // [n_elems + 1] offsets into eldof
  const int32_t* eldof;           // padded local position, -1 prescribed
  double* ke;                     // element matrices (row-major)
  const int64_t* rc_ptr;          // row contributions: absolute offsets, per padded row
  const int32_t* rc_elem;         // element slot
  const int32_t* rc_a;            // row inside the element matrix
  // constraint rows: per subdomain row list (CSR over padded positions)
  const int64_t* c_ptr;           // [total rows + 1]
  const int32_t* c_pos;           // padded local position
  const double* c_val;
  // maps
  const int32_t* loc2iface;       // [n_vec] interface index or -1
  const int32_t* loc2glob;        // [n_vec] level DOF id or -1
  const int64_t* iface_ptr;       // [n_iface + 1] occurrences of an interface DOF
  const int64_t* iface_occ;       //   flat padded positions, ascending subdomain
  const int64_t* glob_occ_ptr;    // [n_dof + 1] occurrences of every level DOF
  const int64_t* glob_occ;
  const int32_t* sub_coarse;      // [sum nc] global coarse ids (R_Ci)
  const int64_t* cinv_ptr;        // [n_coarse + 1] occurrences of a coarse DOF
  const int64_t* cinv_occ;        //   flat indices into per-subdomain coarse vectors
  double* w;                      // [n_vec] interface weights (0 elsewhere)
  double* diag;                   // [n_vec] diagonal of K_i
  double* rho;                    // [n_sub]
  double* Ginv;                   // [sum nc*nc]
  double* KC;                     // [sum nc*nc] local coarse matrices K_Ci
  void* tiles;                    // factor tiles (float or double)
  void* dinv;                     // diagonal inverses
  void* psi;                      // Psi_G
  void* psiT;                     // Psi_G^T in tiles: tile (rb, j) of a subdomain at psiT_off + (rb nGb + j) NB2
  float* schur;                   // explicit augmented Schur complement of the interface (mixed inner operator), or null
  void* sgn;                      // [n_vec] pivot signs of the signed Cholesky (T; +1 for SPD levels)
  const double* c_rho;            // [sum nc] 1 where a constraint row is augmented by rho, else 0
  int indefinite;                 // 1: negative pivots allowed (Stokes), 0: SPD
  int wait_probe;                 // test only: sweeps poll status[3] (never set) instead of the published solution blocks
  int* status;                    // [4]: breakdown flag, lowest breakdown subdomain, timeout code, a word
                                  // nothing writes (the publication wait of the timeout probe)
};

// Counts every kernel launch of the library (defined in capi.cpp).
void note_launch();

// Read-only view of a set-up handle for the entry point in noalloc.cu (defined in capi.cpp).
struct GradView {
  int64_t n_elems, n_full, n_free;
  int ne;
  const double* ke;               // level-1 element matrices in slot order
  const int32_t* slot_elem;
  const double* coef;
  const int32_t* conn;            // element -> nodes; full DOF of element slot a: conn[a / ndof] ndof + a % ndof
  int ndof;                       // DOFs per node
  const int64_t* free_of_full;    // full DOF -> free id or -1
  const double* dir_full;         // [n_full] prescribed values (0 on free DOFs), or null when all zero
  int coef_linear;                // 1: K_e is linear in coef_e (Poisson, elasticity), 0: Stokes
  cudaStream_t stream;
};

// ---------------------------------------------------------------- assembly (assemble.cu)
// Q1 boxes (simplex = 0, 2**dim nodes) or linear simplices (simplex = 1, dim + 1 nodes); element
// slot k takes element slot_elem[k] (slot_elem null: element k) and its matrix goes to ke + k ne^2
void launch_elem_q1p1(int physics, int dim, int simplex, int64_t n_elems, const double* coords, const int32_t* conn,
                      const double* coef, double nu, const int32_t* slot_elem, double* ke, cudaStream_t st);
void launch_elem_q2q1(int64_t n_elems, const double* coords, const int32_t* conn, const double* coef,
                      const int32_t* slot_elem, double* ke, cudaStream_t st);
// ke + k ne^2 = ke_elem + slot_elem[k] ne^2 for every slot k (ne^2 doubles each)
void launch_gather_elems(int64_t n_elems, int ne, const int32_t* slot_elem, const double* ke_elem, double* ke,
                         cudaStream_t st);
void launch_lift(int64_t n_free, int ne, const int64_t* lptr, const int32_t* lslot, const int32_t* la,
                 const double* ke, const double* ud, double* lift, cudaStream_t st);
// CSR pattern of K_i (pass 1: cnt[row] = row length; pass 2: col at row_ptr)
void launch_csr_pattern(const LevelDev& L, int64_t n_rows, const int32_t* row_sub, int max_len, int32_t* cnt,
                        const int64_t* row_ptr, int32_t* col, cudaStream_t st);
void launch_csr_values(const LevelDev& L, int64_t n_rows_total, const int32_t* row_sub, cudaStream_t st);
template <typename T>
void launch_densify_rows(const LevelDev& L, const int32_t* row_sub, cudaStream_t st);
template <typename T>
void launch_add_constraints(const LevelDev& L, cudaStream_t st);
void launch_weights(const LevelDev& L, int multiplicity, const double* unused, cudaStream_t st);

// ---------------------------------------------------------------- dense factor (dense.cu)
// one block column k: diagonal tile + inverse, panel, trailing update of columns (k, jmax).
// skip_diag: the diagonal tile k was factored by the previous step's update (fuse_next there);
// fuse_next: the update's block for tile (k+1, k+1) factors it (only when max_tiles > 0 and
// k + 1 < jmax, i.e. that tile receives its last update in this step).
// rlim > 0: the rows of the diagonal block only (i < min(rlim, Bc) in the panel and the update).
// xinv (FP32, rlim = k0 + 4): the step also forms block row k - k0 of X = L_D^{-1}, the inverse of
// the diagonal block D = [k0, k0 + nd) (nd = min(4, Bc - k0)), X_QP = -X_QQ sum_{P <= K < Q} L_QK X_KP
// for P < Q, as row-major 64 x 64 tiles at xinv + (s * 16 + 4 Q + P) * 4096 (X_QQ = L_QQ^{-1} stays
// in the stored inverses); a step with no in-block update tiles then launches for X alone.
template <typename T>
void launch_potrf_step(const LevelDev& L, int k, int max_R, int max_tiles, int jmax, cudaStream_t st,
                       int skip_diag = 0, int fuse_next = 0, int rlim = 0, float* xinv = nullptr, int k0 = 0);
// update_tc.cu, FP32 levels with tensor cores: rank-(64 nt) update of the output columns
// ib <= j < jend from the nt panel tile columns kb0 .. kb0+nt-1 (nt = 4 or 8).  k_split_panel
// writes the two scaled FP16 parts of the panel tiles L(i, kb0 + q), i >= ib, at
// split + ((prow_off[s] + i) * 8 + q) * 16 KB (indefinite levels: also a copy with the pivot
// signs on the columns at split_signed) and the row unscaling factors 2^-e_r at
// rscale[(prow_off[s] + i) * 64 + r]; the update (nq = nt, jbeg = ib) makes 128 x 128 output
// blocks from them (persistent grid; item_pref[s] = first work item of subdomain s,
// item_pref[n_sub] = number of items; split_b = split_signed on indefinite levels, else split)
// panel_operand = 1: the rows i >= min(ib, Bc) of every subdomain with kb0 < Bc (the rows below
// a sub-panel's diagonal block, before their panel solve), columns >= Bc as zeros.
void launch_split_panel(const LevelDev& L, int kb0, int nt, int ib, int max_R, uint8_t* split, uint8_t* split_signed,
                        float* rscale, const int64_t* prow_off, cudaStream_t st, int panel_operand = 0);
// The B operand of a sub-panel's panel solve L(i, D) = A(i, D) X^T S_D: the rows of -S_D X (block
// row Q of xinv and L_QQ^{-1}, pivot signs of the block's columns) split like the panel rows into
// the split rows prow_off[s] + k0 + Q, tile columns 0 .. 3, with their unscaling factors in rscale.
void launch_split_inverse(const LevelDev& L, int k0, const float* xinv, uint8_t* split, float* rscale,
                          const int64_t* prow_off, cudaStream_t st);
// The update adds its output into the tiles with TMA reduce-adds through this tensor map: the
// FP32 tile buffer viewed as [tile_elems / 64 rows][64 columns], 32 x 32 boxes, 128-byte
// swizzle.  make_tile_tmap returns 0 or the driver's error code.
struct TensorMap128 {
  alignas(64) uint64_t opaque[16];   // a CUtensorMap
};
int make_tile_tmap(TensorMap128* map, float* tiles, int64_t tile_elems);
// ibeg: the output rows start at max(j, min(ibeg, Bc)) (0 for a trailing update; k0 + 4 for the
// panel solve of the sub-panel [k0, k0 + 4), whose output columns are jbeg = k0 .. jend = k0 + 4).
// panel = 1 (a panel solve): the output is stored instead of subtracted (the product is -A B^T
// with B the split rows of -S_D X; the tiles' old contents are the A operand, already split), and
// the column pair j, j + 1 takes the K steps 0 .. j - jbeg + 1 (X is block lower triangular).
void launch_update_tc2(const LevelDev& L, int nq, int jbeg, int jend, int ibeg, int panel, int grid, const uint8_t* split,
                       const uint8_t* split_b, const float* rscale, const int64_t* prow_off,
                       const int64_t* item_pref, const TensorMap128& tmap, cudaStream_t st);
void launch_gram_chol(const LevelDev& L, int precision_fp32, int max_nc, cudaStream_t st);
template <typename T>
void launch_psi(const LevelDev& L, int max_nGb, int max_nc, cudaStream_t st);
// Explicit inverse W = A^{-1} of a single-subdomain level held in an FP32 factor (the coarsest
// level's FP32 copy), npad x npad stored column after column; and y = W x for nr columns of n_vec
// (padded local positions).
void launch_coarse_inverse(const LevelDev& L, int64_t npad, float* W, cudaStream_t st);
void launch_coarse_apply(const float* W, int64_t npad, const float* x, float* y, int64_t n_vec, int nr,
                         cudaStream_t st);
// sweep.cu: forward (backward = 0) or backward triangular sweep over part 0 (interior
// block rows) or part 1 (interface block rows) of every subdomain; ctrl is the task counter and
// pub a publication buffer of n_vec x min(nr, 8) words of T (both reset by the launch).
// Solve-phase launches take nr right-hand sides (default 1); a block of them stores its columns one
// after another, each vector kind with its own length as the stride (local vectors n_vec,
// interface vectors n_iface, level vectors n_dof, coarse vectors n_coarse, per-subdomain coarse
// vectors sum nc).  The factor-streaming kernels read each factor tile once per group of columns.
template <typename T>
void launch_sweep(const LevelDev& L, T* vec, const int2* tasks, int ntasks, int part, int backward, int* ctrl,
                  void* pub, int grid_max, int deep, cudaStream_t st, int nr = 1);
// crow_sub: subdomain of every constraint row (flat over the level); t, mu: scratch [nr][total_rows]
template <typename T>
void launch_constraint_corr(const LevelDev& L, T* vec, const int32_t* crow_sub, int64_t total_rows, double* t,
                            double* mu, double* part, int max_nGb, int max_ncb, cudaStream_t st, int nr = 1);
// The products with Y_G (constraint block rows of the factor) and with Psi_G^T (psiT) stream
// those tiles once per group of up to 8 right-hand sides: row products t = M v over chunks of 4
// tile columns (partial sums part[(c_off + p) * zmax + z], zmax = ceil(max_nGb / 4), summed in a
// fixed order), column products v += M^T z one CTA per interface tile column.
template <typename T>
void launch_psi_t_apply(const LevelDev& L, const T* vec, double* part, int64_t sum_nc, double* rc_sub,
                        int max_nGb, int max_ncb, cudaStream_t st, int nr = 1);
template <typename T>
void launch_psi_apply_add(const LevelDev& L, const double* zc_sub, int64_t sum_nc, T* vec, int max_nGb,
                          int max_ncb, cudaStream_t st, int nr = 1);
// psiT from Psi_G (set-up, after launch_psi)
template <typename T>
void launch_psi_transpose(const LevelDev& L, int max_nGb, int max_ncb, cudaStream_t st);
inline int rows_zmax(int max_nGb) { return (max_nGb + 3) / 4; }

// ---------------------------------------------------------------- vectors (vector.cu)
template <typename T>
void launch_gather_iface(const LevelDev& L, const double* x, int weighted, T* loc, cudaStream_t st, int nr = 1);
template <typename T>
void launch_scatter_iface(const LevelDev& L, const T* loc, int weighted, double* y, cudaStream_t st, int nr = 1);
template <typename T>
void launch_gather_glob(const LevelDev& L, const double* x, int part, T* loc, cudaStream_t st, int nr = 1);
template <typename T>
void launch_scatter_interior(const LevelDev& L, const T* loc, double* y, cudaStream_t st, int nr = 1);
// rows: flat padded row indices (interior rows, interface rows or both, of every subdomain)
void launch_spmv_rows(const LevelDev& L, const int64_t* rows, int64_t nrows, const double* x, double* y, double alpha,
                      double beta, const int32_t* row_sub, cudaStream_t st, int nr = 1);
template <typename Tin, typename Tout>
void launch_convert(const Tin* in, Tout* out, int64_t n, cudaStream_t st);
void launch_axpy_loc(double* y, const double* x, double a, int64_t n, cudaStream_t st);
template <typename T>
void launch_add_to_double(double* y, const T* x, int64_t n, cudaStream_t st);
void launch_coarse_gather(const LevelDev& L, const double* rc_sub, int64_t sum_nc, double* rC, cudaStream_t st,
                          int nr = 1);
void launch_coarse_scatter_n(const int32_t* sub_coarse, int64_t total, const double* zC, int64_t n_coarse,
                             double* zc_sub, cudaStream_t st, int nr = 1);
// nr dot products of the columns of a and b (length n each): out[k * ostride], partial [nr][nblk]
void launch_dot(const double* a, const double* b, int64_t n, double* partial, int nblk, double* out,
                cudaStream_t st, int nr = 1, int ostride = 16);
// PCG of a block of right-hand sides: column k keeps its scalars at scal[16 k ..]
void launch_pcg_update_x_r(double* x, double* r, const double* p, const double* q, const double* scal,
                           int64_t n, cudaStream_t st, int nr = 1);
void launch_pcg_update_p(double* p, const double* z, const double* scal, int64_t n, cudaStream_t st, int nr = 1);
void launch_pcg_scalars(double* scal, int stage, int flexible, cudaStream_t st, int nr = 1);
// conn: element -> nodes (ne / ndof per element); the full DOF of element slot a is
// conn[a / ndof] * ndof + a % ndof
void launch_grad_contract_slots(int64_t n_elems, int ne, const double* ke, const int32_t* slot_elem,
                                const double* coef, const int32_t* conn, int ndof, const double* lam,
                                const double* u, int nrhs, int64_t n_full, double* grad, cudaStream_t st);
void launch_expand_free(const double* xf, const int64_t* free_of_full, int64_t n_full, int nrhs,
                        int64_t n_free, double* xfull, cudaStream_t st);
void launch_copy_segments(const double* src, const int64_t* src_off, double* dst, const int64_t* dst_off,
                          const int64_t* len, int64_t n, cudaStream_t st);
// g = f[idx] - t per column (f columns of length fstride); u[idx] = v per column (u columns of ustride)
void launch_iface_rhs(double* g, const double* f, int64_t fstride, const int64_t* idx, const double* t, int64_t n,
                      cudaStream_t st, int nr = 1);
void launch_put_indexed(double* u, int64_t ustride, const int64_t* idx, const double* v, int64_t n, cudaStream_t st,
                        int nr = 1);
// inner Schur operator from the stored factor (trmv.cu): y = L_GG S L_GG^T x over the
// interface block rows of an FP32 level (y1 scratch), and y -= C^T R C x (FP64, local vectors)
// Explicit form of the same operator: at the point of the factorisation where every interior
// column has been eliminated and no interface column yet (block column b = nIb of the subdomain),
// the trailing interface block of the tiles is S_i + C_i^T R C_i; launch_schur_snapshot copies it,
// for the subdomains with nIb == b, as the lower triangle of tiles (i, j), 0 <= j <= i < nGb, at
// schur + schur_off.  launch_schur_symv then applies it once per tile: y_i = sum_j M_ij x_j over
// the stored lower tiles and, for j < i, the column part M_ij^T x_i into part (64 floats per tile
// and right-hand side), added in a fixed order by a second kernel.  part holds
// sum_s nGb (nGb - 1) / 2 x 64 floats per right-hand side (tri_off: its per-subdomain offsets).
void launch_schur_snapshot(const LevelDev& L, int b, int max_nGb, cudaStream_t st);
void launch_schur_symv(const LevelDev& L, int max_nGb, const int64_t* part_off, int64_t part_stride, const float* x,
                       float* part, float* y, cudaStream_t st, int nr = 1);
void launch_trmv_schur(const LevelDev& L, int max_nGb, const float* x, float* y1, float* y, cudaStream_t st,
                       int nr = 1);
void launch_sub_ctrc(const LevelDev& L, const int32_t* crow_sub, int64_t total_rows, const double* x, double* y,
                     cudaStream_t st, int nr = 1);
// flexible GMRES (vector.cu): out[i] = V_i . w (i < nv, partial holds nv * nblk doubles);
// w += alpha sum_i c_i V_i; dst = src / sqrt(*nrm2)
void launch_multidot(const double* V, int64_t ldv, int nv, const double* w, int64_t n, double* partial, int nblk,
                     double* out, cudaStream_t st);
void launch_combine(double* w, const double* V, int64_t ldv, int nv, const double* c, double alpha, int64_t n,
                    cudaStream_t st);
void launch_scale_by_norm(double* dst, const double* src, const double* nrm2, int64_t n, cudaStream_t st);
// BiCGstab (vector.cu)
void launch_bicg_scalars(double* S, int stage, cudaStream_t st);
void launch_bicg_p(double* p, const double* r, const double* v, const double* S, int64_t n, cudaStream_t st);
void launch_bicg_s(double* sv, const double* r, const double* v, const double* S, int64_t n, cudaStream_t st);
void launch_bicg_xr(double* x, double* r, const double* ph, const double* sh, const double* sv, const double* t,
                    const double* S, int64_t n, cudaStream_t st);

}  // namespace bddc
