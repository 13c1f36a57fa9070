// C ABI of the GB300 multilevel BDDC library: host orchestration of Algorithm 1 (set-up)
// and Algorithm 2 (application) with PCG on the reduced interface problem (Sec. 2).
// Every numerical step runs in the kernels of assemble.cu, dense.cu and vector.cu; this
// file prepares index arrays, allocates device memory and enqueues launches.
#include <cuda_runtime.h>
#if defined(__GLIBC__) || defined(__linux__)
#include <malloc.h>
#endif

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/bddc.h"
#include "analysis.h"
#include "internal.h"

namespace bddc {

std::atomic<int64_t> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

thread_local std::string g_err;

struct Fail {
  int code;
};

[[noreturn]] void fail(int code, const std::string& msg) {
  g_err = msg;
  throw Fail{code};
}

void ck(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  if (e == cudaErrorMemoryAllocation) fail(BDDC_ERR_OOM, std::string(what) + ": out of device memory");
  fail(BDDC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ------------------------------------------------------------------ device memory helpers
// The library's device memory comes from one private stream-ordered pool per device whose
// release threshold keeps freed blocks cached: a handle set up after another one was freed (a
// new mesh, new coefficients through a fresh set-up) reuses them instead of paying for
// cudaMalloc of several GB again.  The device's default pool is left untouched.
cudaMemPool_t library_pool() {
  static std::mutex mu;
  static std::unordered_map<int, cudaMemPool_t> pools;
  int dev = 0;
  ck(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> g(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  ck(cudaMemPoolCreate(&pool, &props), "cudaMemPoolCreate");
  uint64_t keep = ~0ull;
  ck(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep), "cudaMemPoolSetAttribute");
  pools[dev] = pool;
  return pool;
}

// Host arrays that are written in full before use: default-initialised elements (no zero fill
// of tens of MB on the set-up's critical path).
template <typename T>
struct NoInitAlloc : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <typename U>
  NoInitAlloc(const NoInitAlloc<U>&) {}
  template <typename U>
  void construct(U* p) {
    ::new ((void*)p) U;
  }
  template <typename U, typename... A>
  void construct(U* p, A&&... a) {
    ::new ((void*)p) U(std::forward<A>(a)...);
  }
};
template <typename T>
using raw_vector = std::vector<T, NoInitAlloc<T>>;

struct DevArena {
  std::vector<void*> ptrs;
  int64_t bytes = 0;
  double upload_ms = 0.0;       // host time spent in upload (pageable copies stage synchronously)
  int64_t upload_bytes = 0;
  cudaStream_t st = nullptr;   // allocations and frees are ordered on the handle's stream
  template <typename T>
  T* alloc(int64_t n) {
    if (n <= 0) n = 1;
    void* p = nullptr;
    ck(cudaMallocFromPoolAsync(&p, sizeof(T) * (size_t)n, library_pool(), st), "cudaMallocFromPoolAsync");
    ptrs.push_back(p);
    bytes += (int64_t)sizeof(T) * n;
    return (T*)p;
  }
  template <typename T>
  T* upload(const raw_vector<T>& v, cudaStream_t st) {
    return upload_n(v.data(), (int64_t)v.size(), st);
  }
  template <typename T>
  T* upload_n(const T* v, int64_t n, cudaStream_t st) {
    const double t0 = now_ms();
    T* p = alloc<T>(n);
    if (n > 0) ck(cudaMemcpyAsync(p, v, sizeof(T) * n, cudaMemcpyHostToDevice, st), "upload");
    upload_ms += now_ms() - t0;
    upload_bytes += (int64_t)(sizeof(T) * n);
    return p;
  }
  template <typename T>
  T* upload(const std::vector<T>& v, cudaStream_t st) {
    const double t0 = now_ms();
    T* p = alloc<T>((int64_t)v.size());
    if (!v.empty()) ck(cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st), "upload");
    upload_ms += now_ms() - t0;
    upload_bytes += (int64_t)(sizeof(T) * v.size());
    return p;
  }
  void free_one(void* p) {   // return one allocation to the pool early (stream-ordered)
    for (size_t k = 0; k < ptrs.size(); ++k)
      if (ptrs[k] == p) {
        cudaFreeAsync(p, st);
        ptrs.erase(ptrs.begin() + (int64_t)k);
        return;
      }
  }
  void release() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
    if (!ptrs.empty()) cudaStreamSynchronize(st);
    ptrs.clear();
    bytes = 0;
  }
};

// ------------------------------------------------------------------ one level
struct Level {
  LevelMesh mesh;
  LevelMaps maps;
  bool coarsest = false;
  bool fp32 = false;           // precision of tiles / preconditioner vectors
  // host-side metadata
  std::vector<SubMeta> meta;
  int64_t n_vec = 0, tile_elems = 0, dinv_elems = 0, psi_elems = 0, g_elems = 0, sum_nc = 0;
  int max_R = 0, max_Bc = 0, max_nc = 0, max_nG = 0, max_nGb = 0, max_ncb = 0;
  int64_t psiT_elems = 0;
  // explicit augmented Schur complement of the interface (mixed inner operator, level 1 only)
  bool explicit_schur = false;
  int64_t schur_elems = 0;
  int64_t symv_stride = 0;            // floats of the symmetric product's column parts per right-hand side
  int64_t* symv_part_off = nullptr;   // [n_sub] their offsets
  float* symv_part = nullptr;         // [blk][symv_stride]
  std::vector<char> snap_start, snap_mid;   // per super-panel p: some nIb == 8p / == 8p + 4
  std::vector<int> max_tiles;  // per factor step k
  std::vector<double> step_flops;  // tile flops of factor step k (all subdomains)
  std::vector<int> narrow_tiles;   // per step k: in-panel update tiles (256-wide sub-panels)
  std::vector<double> panel_flops; // per step k: flops of the CUDA-core steps (tensor-core path)
  std::vector<int> block_tiles;    // per step k: update tiles inside the sub-panel's diagonal block
  std::vector<double> block_flops; // per step k: flops of the diagonal block's CUDA-core steps
  bool tc_panels = false;          // panel solves below the diagonal blocks on the tensor cores
  float* xinv = nullptr;           // [n_sub][4 x 4 tiles] inverse of the current diagonal block
  // per 512-wide super-panel p and launch u of the tensor cores (0: rank-256 update of the second
  // half's columns, 1: rank-512 update of the trailing columns, 2: rank-256 update of all trailing
  // columns, 3 / 4: panel solve of the first / second half): 128 x 128 work items and
  // FP32-equivalent flops (panel solves: those of the triangular solve they replace)
  std::vector<int64_t> tc_items;    // [kTcLaunches p + u], all subdomains
  std::vector<double> tc_flops;     // [kTcLaunches p + u]
  int64_t* item_pref = nullptr;     // [kTcLaunches p + u][n_sub + 1] first work item of every subdomain
  uint8_t* split = nullptr;        // scaled FP16 parts of the current super-panel (pre-split update)
  uint8_t* split_signed = nullptr; // indefinite levels: the same with the pivot signs on the columns
  float* rscale = nullptr;         // their row unscaling factors (powers of two)
  int64_t* prow_off = nullptr;     // [n_sub] first split row of every subdomain
  TensorMap128 tile_tmap{};        // the FP32 tiles as [rows][64] for the update's TMA reduce-adds
  double trsv_bytes[2] = {0, 0};   // algorithmic bytes of one sweep over part 0 / part 1
  double trmv_bytes = 0;           // algorithmic bytes of one factor-based inner Schur product
  // sweep task lists [part][direction] in dependency order and their control words
  int2* tasks[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};       // [part][dir], subdomain order
  int2* tasks_big[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [part][dir], longest chains first
  int2* tasks_by_sub[2] = {nullptr, nullptr};     // interior tasks [dir] grouped per subdomain
  std::vector<int> task_sub_off[2];               // their per-subdomain offsets
  int ntasks[2][2] = {{0, 0}, {0, 0}};
  // coarsest level of the mixed form: FP32 copy of the FP64 factor for the preconditioner's solves
  bool solve32 = false;
  LevelDev d32{};
  float* v32 = nullptr;            // [blk][n_vec] FP32 input of the coarse solve
  float* v32b = nullptr;           // [blk][n_vec] FP32 output of the explicit inverse
  float* winv = nullptr;           // explicit inverse of the FP32 copy (n_vec x n_vec), or null
  // sweep launch configuration per part (autotuned): CTAs per SM, deep tile ring, task order
  int sweep_ctas[2] = {2, 2};
  int sweep_deep[2] = {1, 1};
  int sweep_order[2] = {0, 0};
  int* ctrl = nullptr;         // task counter of the sweeps
  void* pub = nullptr;         // sweep publication buffer: n_vec x min(blk, 8) words of the factor's type
  int64_t* rows[3] = {nullptr, nullptr, nullptr};   // interior rows, interface rows, all rows
  int64_t nrows[3] = {0, 0, 0};
  int32_t* crow_sub = nullptr;                      // subdomain of every constraint row
  double* cc_t = nullptr;                           // [sum_nc] scratch of the constraint correction
  double* cc_mu = nullptr;
  int ne_uniform = 0;          // level 1: entries per element row
  // device
  LevelDev d{};
  int32_t* row_sub = nullptr;
  int32_t* slot_elem = nullptr;
  int64_t* seg_src = nullptr;  // levels > 1: K_C offsets of the previous level per element slot
  int64_t* seg_len = nullptr;
  int64_t* iface_dofs = nullptr;
  // work vectors
  void* locA = nullptr;        // T[n_vec]
  void* locB = nullptr;        // T[n_vec]
  double* dl0 = nullptr;       // double[n_vec]
  double* dl1 = nullptr;
  double* dl2 = nullptr;
  double* dl3 = nullptr;
  double* rc_sub = nullptr;    // [sum_nc]
  double* psi_part = nullptr;  // [sum_nc * rows_zmax(max_nGb)] partial sums of Psi^T r and Y r
  double* zc_sub = nullptr;
  double* rC = nullptr;        // [n_coarse]
  double* zC = nullptr;
  double* gi0 = nullptr;       // [n_iface]
  double* gi1 = nullptr;
  double* gi2 = nullptr;
  double* gv0 = nullptr;       // [n_dof] (levels > 1)
  int blk = 1;                 // right-hand sides the work vectors hold
};

int64_t pad_pos(const SubMeta& m, int64_t r) { return r < m.nI ? r : (int64_t)m.nIb * NB + (r - m.nI); }

constexpr int kMaxBlock = 8;   // right-hand sides solved together (one pass over the factors)
constexpr int64_t kMaxCoarseInverse = 16384;   // padded coarse sizes with an explicit FP32 inverse (1 GiB)

// Work vectors of the solve phase of one level for blocks of up to blk right-hand sides (every
// column of a block has the vector kind's own length, see internal.h).
void alloc_level_work(Level& L, DevArena& A, int blk) {
  const int64_t nv = L.n_vec * blk;
  if (L.fp32) {
    L.locA = A.alloc<float>(nv);
    L.locB = A.alloc<float>(nv);
  } else {
    L.locA = A.alloc<double>(nv);
    L.locB = A.alloc<double>(nv);
  }
  L.pub = A.alloc<double>(L.n_vec * std::min(blk, 8));
  if (L.explicit_schur) L.symv_part = A.alloc<float>(std::max<int64_t>(L.symv_stride, 1) * blk);
  L.dl0 = A.alloc<double>(nv);
  L.dl1 = A.alloc<double>(nv);
  L.dl2 = A.alloc<double>(nv);
  L.dl3 = A.alloc<double>(nv);
  L.cc_t = A.alloc<double>(L.sum_nc * blk);
  L.cc_mu = A.alloc<double>(L.sum_nc * blk);
  L.rc_sub = A.alloc<double>(L.sum_nc * blk);
  L.psi_part = A.alloc<double>(L.sum_nc * rows_zmax(L.max_nGb) * blk);
  L.zc_sub = A.alloc<double>(L.sum_nc * blk);
  L.rC = A.alloc<double>(L.maps.n_coarse * blk);
  L.zC = A.alloc<double>(L.maps.n_coarse * blk);
  L.gi0 = A.alloc<double>(L.maps.n_iface * blk);
  L.gi1 = A.alloc<double>(L.maps.n_iface * blk);
  L.gi2 = A.alloc<double>(L.maps.n_iface * blk);
  L.gv0 = A.alloc<double>(L.mesh.n_dof * blk);
  if (L.solve32) {
    L.v32 = A.alloc<float>(nv);
    L.v32b = A.alloc<float>(nv);
  }
  L.blk = blk;
}

constexpr int kSub = 4;     // tile columns of a CUDA-core sub-panel (256)
constexpr int kPanel = 8;   // tile columns of a tensor-core super-panel (512, two sub-panels)
constexpr int kTcLaunches = 5;   // tensor-core launch kinds per super-panel (three updates, two panel solves)

}  // namespace
}  // namespace bddc

using namespace bddc;

struct bddc_handle_s {
  bddc_opts opts{};
  unsigned constraints = 0;
  cudaStream_t st = nullptr;
  bool analysis_only = false;
  // level-1 mesh data (host copies)
  int dim = 3, npe = 8, ndof = 1, physics = 0;
  int64_t n_nodes = 0, n_elems = 0, n_full = 0, n_free = 0;
  double nu = 0.0;
  std::vector<double> coords, coef;
  std::vector<int32_t> conn;
  std::vector<int64_t> free_of_full;   // full DOF -> free id or -1
  std::vector<std::vector<int32_t>> parts;
  std::vector<int64_t> n_parts;
  int n_levels = 2;
  std::vector<Level> lv;               // BDDC levels 1..L-1, then the coarsest
  DevArena arena;
  // device copies of level-1 mesh data
  double* d_coords = nullptr;
  int32_t* d_conn = nullptr;
  double* d_coef = nullptr;
  // set-up only: level-1 element matrices in element order, computed while the host analyses
  // the mesh (ke_early until numeric_setup gathers them into element slots)
  double* ke_elem = nullptr;
  bool ke_early = false;
  int64_t* d_free_of_full = nullptr;
  int* d_status = nullptr;
  // non-zero prescribed values: lift = -K_fd u_d, added to every right-hand side
  bool has_lift = false;
  std::vector<double> dir_full;        // [n_full] prescribed values, 0 on free DOFs
  double* d_dir_full = nullptr;
  double* d_lift = nullptr;            // [n_free]
  double* d_lift_ud = nullptr;         // [n_elems * ne] prescribed values of each element slot
  int64_t* d_lift_ptr = nullptr;       // free DOF -> its (slot, row) occurrences in lifting elements
  int32_t* d_lift_slot = nullptr;
  int32_t* d_lift_a = nullptr;
  // PCG
  double* scal = nullptr;              // [16]
  double* partial = nullptr;           // [kDotBlocks]
  double* h_scal = nullptr;            // pinned [16]
  double *vx = nullptr, *vr = nullptr, *vz = nullptr, *vp = nullptr, *vq = nullptr, *vrold = nullptr, *vg = nullptr;
  double *vs = nullptr, *vsh = nullptr, *vt = nullptr;   // BiCGstab s, M^{-1} s, S M^{-1} s
  // flexible GMRES(kRestart): Krylov basis V, preconditioned basis Z, Arnoldi column scratch
  double *gm_V = nullptr, *gm_Z = nullptr, *gm_w = nullptr, *gm_h = nullptr, *gm_partial = nullptr;
  double* h_gm = nullptr;              // pinned: Arnoldi column (two passes + norm) and y
  double* fcol = nullptr;              // [n_free] work
  double* ucol = nullptr;
  double *full_a = nullptr, *full_b = nullptr;
  int refine_steps = 0;                // interior-solve steps of the FP64 Schur operator
  bool use_outer = false;              // mixed PCG: FP64 outer refinement around an inner PCG
  int inner_steps = 0;                 // inner operator: 0 = from the stored factor, k = k interior-solve steps
  int cur_steps = 0;                   // steps used by the next interior solves
  int grid_max = 304;                  // persistent sweep grid: 2 CTAs per SM
  int blk = 1;                         // right-hand sides the Krylov work vectors hold
  cudaStream_t cap_st = nullptr;       // private stream for graph capture
  cudaGraphExec_t iter_graph = nullptr;  // one captured Krylov iteration
  int iter_graph_key = -1;               // graph_key() of the captured iteration
  int64_t graph_kernels = 0;           // kernel nodes in iter_graph
  bddc_stats stats{};
  bool factored = false;
  // optional per-class CUDA-event timing
  struct ProfRec {
    cudaEvent_t a, b;
    int cls;
    double bytes, flops;
  };
  std::vector<ProfRec> prof_pending;
  std::vector<ProfRec> graph_prof;     // event pairs recorded by every replay of iter_graph
  std::vector<cudaEvent_t> event_pool;
  ~bddc_handle_s() {
    if (iter_graph) cudaGraphExecDestroy(iter_graph);
    if (cap_st) cudaStreamDestroy(cap_st);
    for (auto& r : prof_pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto& r : graph_prof) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : event_pool) cudaEventDestroy(e);
    if (h_gm) cudaFreeHost(h_gm);
  }
};

namespace bddc {
namespace {

constexpr int kDotBlocks = 304;   // 2 x SM count of a GB300; fixed for reproducible sums

constexpr int kRestart = 50;   // flexible GMRES restart length

int krylov_kind(const bddc_handle_s* h) {
  if (h->opts.krylov != 0) return h->opts.krylov;
  if (h->physics != BDDC_STOKES) return BDDC_KRYLOV_PCG;
  return h->opts.precision == BDDC_PREC_MIXED ? BDDC_KRYLOV_FGMRES : BDDC_KRYLOV_BICGSTAB;
}


// Event record that also works inside stream capture (there it becomes an event-record node of
// the graph instead of a capture-internal dependency).
void record_event(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ck(cudaStreamIsCapturing(st, &cs), "cudaStreamIsCapturing");
  if (cs == cudaStreamCaptureStatusActive)
    ck(cudaEventRecordWithFlags(e, st, cudaEventRecordExternal), "cudaEventRecordWithFlags");
  else
    ck(cudaEventRecord(e, st), "cudaEventRecord");
}

cudaEvent_t take_event(bddc_handle_s* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  ck(cudaEventCreate(&e), "cudaEventCreate");
  return e;
}

// Records CUDA events around one launch (or one group of launches) of a kernel class on the
// handle's stream when profiling is on.
struct ProfScope {
  bddc_handle_s* h;
  int cls;
  double bytes, flops;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfScope(bddc_handle_s* h_, int cls_, double bytes_, double flops_, cudaStream_t st_)
      : h(h_), cls(cls_), bytes(bytes_), flops(flops_), st(st_) {
    if (h->opts.profile) {
      a = take_event(h);
      record_event(a, st);
    }
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = nullptr;
    try {
      b = take_event(h);
    } catch (...) {
      return;
    }
    try {
      record_event(b, st);
    } catch (...) {
      return;
    }
    h->prof_pending.push_back({a, b, cls, bytes, flops});
  }
};

// After a replay of iter_graph has completed: add the durations of its captured event pairs.
void accumulate_graph_profile(bddc_handle_s* h) {
  for (auto& r : h->graph_prof) {
    float ms = 0.f;
    ck(cudaEventElapsedTime(&ms, r.a, r.b), "cudaEventElapsedTime");
    h->stats.prof_ms[r.cls] += ms;
    h->stats.prof_launches[r.cls] += 1;
    h->stats.prof_bytes[r.cls] += r.bytes;
    h->stats.prof_flops[r.cls] += r.flops;
  }
}

void flush_profile(bddc_handle_s* h) {
  if (h->prof_pending.empty()) return;
  ck(cudaStreamSynchronize(h->st), "sync");
  for (auto& r : h->prof_pending) {
    float ms = 0.f;
    ck(cudaEventElapsedTime(&ms, r.a, r.b), "cudaEventElapsedTime");
    h->stats.prof_ms[r.cls] += ms;
    h->stats.prof_launches[r.cls] += 1;
    h->stats.prof_bytes[r.cls] += r.bytes;
    h->stats.prof_flops[r.cls] += r.flops;
    h->event_pool.push_back(r.a);
    h->event_pool.push_back(r.b);
  }
  h->prof_pending.clear();
}

constexpr int64_t kMaxSubdomains = 65535;   // CUDA's limit on gridDim.y

// fn(i, w) / fn(i) for i in [0, n) on the host worker pool (analysis.h)
void parallel_for_worker(int64_t n, const std::function<void(int64_t, int)>& fn) { host_parallel(n, fn); }

void parallel_for(int64_t n, const std::function<void(int64_t)>& fn) {
  host_parallel(n, [&](int64_t i, int) { fn(i); });
}

// ------------------------------------------------------------------ level preparation
void build_level1_mesh(bddc_handle_s* h, LevelMesh* out) {
  LevelMesh& m = *out;
  m.dim = h->dim;
  m.ncomp = h->ndof;
  m.n_nodes = h->n_nodes;
  m.n_elems = h->n_elems;
  m.n_sub = h->n_parts[0];
  m.coords = h->coords;
  m.nd_ptr.resize(h->n_nodes + 1);
  m.nd_comp.resize(h->n_full);
  for (int64_t p = 0; p <= h->n_nodes; ++p) m.nd_ptr[p] = p * h->ndof;
  for (int64_t p = 0; p < h->n_nodes; ++p)
    for (int c = 0; c < h->ndof; ++c) m.nd_comp[p * h->ndof + c] = c;
  m.nd_id = h->free_of_full;
  m.en_ptr.resize(h->n_elems + 1);
  m.en.resize(h->n_elems * h->npe);
  for (int64_t e = 0; e <= h->n_elems; ++e) m.en_ptr[e] = e * h->npe;
  const int64_t chunk = 4096;
  parallel_for((h->n_elems + chunk - 1) / chunk, [&](int64_t b) {
    const int64_t e1 = std::min(h->n_elems, (b + 1) * chunk) * h->npe;
    for (int64_t q = b * chunk * h->npe; q < e1; ++q) m.en[q] = h->conn[q];
  });
  m.part = h->parts[0];
  m.n_dof = h->n_free;
  if (h->physics == BDDC_STOKES) {          // constant velocities float; pressures ordered last
    m.rigid_mask = 7u;
    m.rigid_points = 1;
    m.last_comp = 3;
  } else if (h->physics == BDDC_ELASTICITY) {
    m.rigid_mask = (1u << h->ndof) - 1u;
    m.rigid_points = h->dim == 3 ? 3 : 2;
  } else {
    m.rigid_mask = 1u;
    m.rigid_points = 1;
  }
}

// Single-subdomain "level" holding the coarsest problem: all DOFs interior.
void build_coarsest_mesh(const Level& prev, LevelMesh* out) {
  std::vector<int32_t> part(prev.maps.n_sub(), 0);
  next_level_mesh(prev.mesh, prev.maps, part.data(), 1, out);
}


// Host arrays of one level, built from its mesh and maps, then uploaded.
void prepare_level(bddc_handle_s* h, Level& L, DevArena& A, cudaStream_t st) {
  const LevelMaps& mp = L.maps;
  const LevelMesh& ms = L.mesh;
  const int64_t ns = mp.n_sub();
  double tph = now_ms();
  auto ph = [&](const char* what) {   // opts.verbose >= 3: host times of the preparation's parts
    const double t = now_ms();
    if (h->opts.verbose >= 3) fprintf(stderr, "bddc prepare:   %-24s %8.2f ms\n", what, t - tph);
    tph = t;
  };
  L.meta.resize(ns);
  int64_t tile = 0, dinv = 0, vec = 0, coff = 0, goff = 0, psi = 0, psiT = 0, schur = 0, symv = 0;
  L.max_R = L.max_Bc = L.max_nc = L.max_nG = L.max_nGb = L.max_ncb = 0;
  // the explicit inner operator snapshots the trailing interface block when the interior is
  // eliminated; the batched factorisation reaches that point for every subdomain at a sub-panel
  // boundary only if the interior block count is a multiple of kSub (identity tiles pad it)
  L.explicit_schur = false;
  if (&L == &h->lv[0] && L.fp32 && h->opts.tensor_cores && h->physics != BDDC_STOKES &&
      krylov_kind(h) == BDDC_KRYLOV_PCG && h->opts.inner_operator != 1) {
    double base = 0.0, padded = 0.0;
    for (int64_t s = 0; s < ns; ++s) {
      const double b = (double)ceil_div(mp.sub_nI[s], NB), bp = (double)(ceil_div(ceil_div(mp.sub_nI[s], NB), kSub) * kSub);
      base += b * (b + 1) / 2;
      padded += bp * (bp + 1) / 2;
    }
    L.explicit_schur = h->opts.inner_operator == 2 || padded <= 1.08 * base;
  }
  for (int64_t s = 0; s < ns; ++s) {
    SubMeta& m = L.meta[s];
    m.n = (int32_t)(mp.sub_dof_ptr[s + 1] - mp.sub_dof_ptr[s]);
    m.nI = (int32_t)mp.sub_nI[s];
    m.nG = m.n - m.nI;
    m.nc = (int32_t)(mp.sub_coarse_ptr[s + 1] - mp.sub_coarse_ptr[s]);
    m.nIb = (int32_t)ceil_div(m.nI, NB);
    if (L.explicit_schur) m.nIb = (int32_t)(ceil_div(m.nIb, kSub) * kSub);
    m.nGb = (int32_t)ceil_div(m.nG, NB);
    m.ncb = (int32_t)ceil_div(m.nc, NB);
    m.Bc = m.nIb + m.nGb;
    m.R = m.Bc + m.ncb;
    m.pad0 = 0;
    m.tile_off = tile;
    tile += ((int64_t)m.Bc * (m.Bc + 1) / 2 + (int64_t)m.ncb * m.Bc) * NB2;
    m.dinv_off = dinv;
    dinv += (int64_t)m.Bc * NB2;
    m.vec_off = vec;
    vec += (int64_t)m.Bc * NB;
    m.row_off = 0;
    m.c_off = coff;
    coff += m.nc;
    m.g_off = goff;
    goff += (int64_t)m.nc * m.nc;
    m.psi_off = psi;
    psi += (int64_t)m.nGb * NB * m.nc;
    m.psiT_off = psiT;
    psiT += (int64_t)m.ncb * m.nGb * NB2;
    m.schur_off = schur;
    if (L.explicit_schur) schur += (int64_t)m.nGb * (m.nGb + 1) / 2 * NB2;
    symv += (int64_t)m.nGb * (m.nGb - 1) / 2 * NB;
    L.max_R = std::max(L.max_R, (int)m.R);
    L.max_Bc = std::max(L.max_Bc, (int)m.Bc);
    L.max_nc = std::max(L.max_nc, (int)m.nc);
    L.max_nG = std::max(L.max_nG, (int)m.nG);
    L.max_nGb = std::max(L.max_nGb, (int)m.nGb);
    L.max_ncb = std::max(L.max_ncb, (int)m.ncb);
  }
  L.n_vec = vec;
  L.tile_elems = tile;
  L.dinv_elems = dinv;
  L.psi_elems = psi;
  L.psiT_elems = psiT;
  L.schur_elems = schur;
  L.symv_stride = L.explicit_schur ? symv : 0;
  L.g_elems = goff;
  L.sum_nc = coff;
  L.max_tiles.assign(L.max_Bc, 0);
  L.step_flops.assign(L.max_Bc, 0.0);
  L.narrow_tiles.assign(L.max_Bc, 0);
  L.panel_flops.assign(L.max_Bc, 0.0);
  L.block_tiles.assign(L.max_Bc, 0);
  L.block_flops.assign(L.max_Bc, 0.0);
  const int n_super = (L.max_Bc + kPanel - 1) / kPanel + 1;
  L.tc_items.assign(kTcLaunches * (size_t)n_super, 0);
  L.tc_flops.assign(kTcLaunches * (size_t)n_super, 0.0);
  L.snap_start.assign(n_super, 0);
  L.snap_mid.assign(n_super, 0);
  const double nb3 = (double)NB * NB * NB;
  const double wsz = L.fp32 ? 4.0 : 8.0;
  L.trsv_bytes[0] = L.trsv_bytes[1] = 0.0;
  L.trmv_bytes = 0.0;
  for (int64_t s = 0; s < ns; ++s) {
    const SubMeta& m = L.meta[s];
    for (int k = 0; k < m.Bc; ++k) {
      int64_t cnt = 0;
      for (int j = k + 1; j < m.Bc; ++j) cnt += m.R - j;
      L.max_tiles[k] = std::max(L.max_tiles[k], (int)cnt);
      L.step_flops[k] += nb3 / 3.0 + nb3 * (double)(m.R - k - 1) + 2.0 * nb3 * (double)cnt;
    }
    for (int k = 0; k < m.Bc; ++k) {
      const int kb1 = (k / kSub + 1) * kSub;
      int64_t cnt = 0;
      for (int j = k + 1; j < std::min(kb1, (int)m.Bc); ++j) cnt += m.R - j;
      L.narrow_tiles[k] = std::max(L.narrow_tiles[k], (int)cnt);
      L.panel_flops[k] += nb3 / 3.0 + nb3 * (double)(m.R - k - 1) + 2.0 * nb3 * (double)cnt;
      const int ilim = std::min(kb1, (int)m.Bc);   // the diagonal block's rows
      int64_t bcnt = 0;
      for (int j = k + 1; j < ilim; ++j) bcnt += ilim - j;
      L.block_tiles[k] = std::max(L.block_tiles[k], (int)bcnt);
      L.block_flops[k] += nb3 / 3.0 + nb3 * (double)(ilim - k - 1) + 2.0 * nb3 * (double)bcnt;
    }
    for (int kb0 = 0; kb0 < m.Bc; kb0 += kPanel) {
      int64_t tiles[2] = {0, 0};
      for (int j = kb0 + kSub; j < std::min(kb0 + kPanel, (int)m.Bc); ++j) tiles[0] += m.R - j;
      for (int j = kb0 + kPanel; j < m.Bc; ++j) tiles[1] += m.R - j;
      const int p = kb0 / kPanel;
      L.tc_flops[kTcLaunches * p] += 2.0 * nb3 * kSub * (double)tiles[0];
      L.tc_flops[kTcLaunches * p + 1] += 2.0 * nb3 * kPanel * (double)tiles[1];
      L.tc_flops[kTcLaunches * p + 2] += 2.0 * nb3 * kSub * (double)(tiles[0] + tiles[1]);
      for (int half = 0; half < 2; ++half) {   // panel solves: rows below the block by its columns
        const int k0 = kb0 + half * kSub;
        const int nd = std::min(kSub, (int)m.Bc - k0);
        if (nd <= 0) continue;
        const double rows = (double)NB * (m.R - std::min(k0 + kSub, (int)m.Bc));
        L.tc_flops[kTcLaunches * p + 3 + half] += rows * (double)(NB * nd) * (NB * nd);
      }
    }
    if (L.explicit_schur) {   // where this subdomain's interior ends: a super-panel start or middle
      if (m.nIb % kPanel == 0) L.snap_start[m.nIb / kPanel] = 1;
      else L.snap_mid[m.nIb / kPanel] = 1;
    }
    // a sweep reads the stored triangle once and the vector in and out
    L.trsv_bytes[0] += wsz * (0.5 * (double)m.nI * (m.nI + 1) + 2.0 * m.nI);
    L.trsv_bytes[1] += wsz * (0.5 * (double)m.nG * (m.nG + 1) + 2.0 * m.nG);
    L.trmv_bytes += wsz * ((double)m.nG * (m.nG + 1) + 4.0 * m.nG);   // the triangle twice, vectors
  }

  ph("layout");
  // element slots (subdomain order) and their padded local DOF positions; an element's matrix
  // DOFs are the DOFs of its nodes in node order
  const int64_t nel = ms.n_elems;
  raw_vector<int32_t> slot_elem(nel);
  raw_vector<int64_t> ke_off(nel + 1), ed_off(nel + 1);
  // per subdomain (in parallel): the slots' element ids and DOF counts as offsets within the
  // subdomain; then the subdomains' totals are scanned and added
  std::vector<int64_t> sub_ed(ns + 1, 0), sub_ke(ns + 1, 0);
  parallel_for(ns, [&](int64_t s) {
    int64_t ed = 0, ke = 0;
    for (int64_t k = mp.sub_elem_ptr[s]; k < mp.sub_elem_ptr[s + 1]; ++k) {
      const int64_t e = mp.sub_elems[k];
      slot_elem[k] = (int32_t)e;
      int64_t nek = 0;
      for (int64_t q = ms.en_ptr[e]; q < ms.en_ptr[e + 1]; ++q) nek += ms.nd_ptr[ms.en[q] + 1] - ms.nd_ptr[ms.en[q]];
      ed_off[k + 1] = ed += nek;
      ke_off[k + 1] = ke += nek * nek;
    }
    sub_ed[s + 1] = ed;
    sub_ke[s + 1] = ke;
  });
  for (int64_t s = 0; s < ns; ++s) {
    sub_ed[s + 1] += sub_ed[s];
    sub_ke[s + 1] += sub_ke[s];
  }
  ke_off[0] = ed_off[0] = 0;
  parallel_for(ns, [&](int64_t s) {
    for (int64_t k = mp.sub_elem_ptr[s]; k < mp.sub_elem_ptr[s + 1]; ++k) {
      ed_off[k + 1] += sub_ed[s];
      ke_off[k + 1] += sub_ke[s];
    }
  });
  raw_vector<int32_t> eldof(ed_off[nel]);
  std::vector<int32_t> loc2iface(L.n_vec, -1), loc2glob(L.n_vec, -1), row_sub(L.n_vec);
  // row contributions (ascending element slot) per padded row: every row of subdomain s only
  // receives contributions from the slots of s, so counts and lists are built per subdomain
  std::vector<int64_t> rc_ptr(L.n_vec + 1, 0);
  std::vector<std::vector<int32_t>> pos_of(kHostWorkers);   // per worker: level DOF -> padded position
  std::atomic<bool> missing{false};
  parallel_for_worker(ns, [&](int64_t s, int w) {
    const SubMeta& m = L.meta[s];
    std::vector<int32_t>& pos = pos_of[w];
    if ((int64_t)pos.size() < ms.n_dof) pos.assign(ms.n_dof, -1);
    for (int64_t q = mp.sub_dof_ptr[s]; q < mp.sub_dof_ptr[s + 1]; ++q) {
      const int64_t pp = pad_pos(m, q - mp.sub_dof_ptr[s]);
      pos[mp.sub_dofs[q]] = (int32_t)pp;
      loc2glob[m.vec_off + pp] = (int32_t)mp.sub_dofs[q];
      loc2iface[m.vec_off + pp] = (int32_t)mp.sub_iface[q];
    }
    for (int64_t p = 0; p < (int64_t)m.Bc * NB; ++p) row_sub[m.vec_off + p] = (int32_t)s;
    for (int64_t k = mp.sub_elem_ptr[s]; k < mp.sub_elem_ptr[s + 1]; ++k) {
      const int64_t e = slot_elem[k];
      int64_t t = ed_off[k];
      for (int64_t a = ms.en_ptr[e]; a < ms.en_ptr[e + 1]; ++a)
        for (int64_t q = ms.nd_ptr[ms.en[a]]; q < ms.nd_ptr[ms.en[a] + 1]; ++q, ++t) {
          const int64_t d = ms.nd_id[q];
          int32_t pp = -1;
          if (d >= 0) {
            pp = d < ms.n_dof ? pos[d] : -1;
            if (pp < 0) {   // every DOF of a subdomain's element belongs to the subdomain
              missing = true;
              continue;
            }
            rc_ptr[m.vec_off + pp + 1]++;
          }
          eldof[t] = pp;
        }
    }
    for (int64_t q = mp.sub_dof_ptr[s]; q < mp.sub_dof_ptr[s + 1]; ++q) pos[mp.sub_dofs[q]] = -1;
  });
  if (missing) fail(BDDC_ERR_INVALID, "an element DOF is missing from its subdomain's local numbering");
  {   // scan of the row counts: within every subdomain's rows in parallel, then across subdomains
    std::vector<int64_t> tot(ns + 1, 0);
    parallel_for(ns, [&](int64_t s) {
      const SubMeta& m = L.meta[s];
      int64_t* r = rc_ptr.data() + m.vec_off + 1;
      for (int64_t p = 1; p < (int64_t)m.Bc * NB; ++p) r[p] += r[p - 1];
      tot[s + 1] = m.Bc > 0 ? r[(int64_t)m.Bc * NB - 1] : 0;
    });
    for (int64_t s = 0; s < ns; ++s) tot[s + 1] += tot[s];
    parallel_for(ns, [&](int64_t s) {
      const SubMeta& m = L.meta[s];
      int64_t* r = rc_ptr.data() + m.vec_off + 1;
      for (int64_t p = 0; p < (int64_t)m.Bc * NB; ++p) r[p] += tot[s];
    });
  }
  raw_vector<int32_t> rc_elem(rc_ptr[L.n_vec]), rc_a(rc_ptr[L.n_vec]);
  parallel_for(ns, [&](int64_t s) {
    const SubMeta& m = L.meta[s];
    std::vector<int64_t> fill(rc_ptr.begin() + m.vec_off, rc_ptr.begin() + m.vec_off + (int64_t)m.Bc * NB);
    for (int64_t k = mp.sub_elem_ptr[s]; k < mp.sub_elem_ptr[s + 1]; ++k)
      for (int64_t t = ed_off[k]; t < ed_off[k + 1]; ++t)
        if (eldof[t] >= 0) {
          const int64_t r = eldof[t];
          rc_elem[fill[r]] = (int32_t)k;
          rc_a[fill[r]] = (int32_t)(t - ed_off[k]);
          fill[r]++;
        }
  });
  ph("element dofs, row lists");
  // constraint rows over padded positions
  std::vector<int64_t> c_ptr(mp.c_ptr.size());
  std::vector<int32_t> c_pos(mp.c_col.size());
  for (size_t i = 0; i < mp.c_ptr.size(); ++i) c_ptr[i] = mp.c_ptr[i];
  parallel_for(ns, [&](int64_t s) {
    const SubMeta& m = L.meta[s];
    int64_t r0 = mp.sub_coarse_ptr[s], r1 = mp.sub_coarse_ptr[s + 1];
    for (int64_t t = mp.c_ptr[r0]; t < mp.c_ptr[r1]; ++t) c_pos[t] = (int32_t)pad_pos(m, mp.c_col[t]);
  });
  // interface and coarse occurrence lists (ascending subdomain)
  std::vector<int64_t> iface_ptr(mp.n_iface + 1, 0), cinv_ptr(mp.n_coarse + 1, 0);
  for (int64_t p = 0; p < L.n_vec; ++p)
    if (loc2iface[p] >= 0) iface_ptr[loc2iface[p] + 1]++;
  for (int64_t g = 0; g < mp.n_iface; ++g) iface_ptr[g + 1] += iface_ptr[g];
  std::vector<int64_t> iface_occ(iface_ptr[mp.n_iface]);
  {
    std::vector<int64_t> fill(iface_ptr.begin(), iface_ptr.end() - 1);
    for (int64_t p = 0; p < L.n_vec; ++p)
      if (loc2iface[p] >= 0) iface_occ[fill[loc2iface[p]]++] = p;
  }
  std::vector<int32_t> sub_coarse(mp.sub_coarse.size());
  for (size_t t = 0; t < mp.sub_coarse.size(); ++t) {
    sub_coarse[t] = (int32_t)mp.sub_coarse[t];
    cinv_ptr[mp.sub_coarse[t] + 1]++;
  }
  for (int64_t g = 0; g < mp.n_coarse; ++g) cinv_ptr[g + 1] += cinv_ptr[g];
  std::vector<int64_t> cinv_occ(cinv_ptr[mp.n_coarse]);
  {
    std::vector<int64_t> fill(cinv_ptr.begin(), cinv_ptr.end() - 1);
    for (size_t t = 0; t < mp.sub_coarse.size(); ++t) cinv_occ[fill[mp.sub_coarse[t]]++] = (int64_t)t;
  }

  ph("constraint, occurrence");
  // ---- upload
  LevelDev& d = L.d;
  d.n_sub = ns;
  d.n_dof = ms.n_dof;
  d.n_iface = mp.n_iface;
  d.n_coarse = mp.n_coarse;
  d.n_vec = L.n_vec;
  d.meta = A.upload(L.meta, st);
  d.ke_off = A.upload(ke_off, st);
  d.ed_off = A.upload(ed_off, st);
  d.eldof = A.upload(eldof, st);
  d.ke = A.alloc<double>(ke_off[nel]);
  d.rc_ptr = A.upload(rc_ptr, st);
  d.rc_elem = A.upload(rc_elem, st);
  d.rc_a = A.upload(rc_a, st);
  ph("uploads 1");
  {
    // CSR pattern of every K_i over padded positions, built on the device: per row the union of
    // the local positions of the elements containing it (ascending)
    int max_len = 0;
    for (const SubMeta& m : L.meta) max_len = std::max(max_len, m.Bc * NB);
    if ((size_t)8 * ((max_len + 31) / 32) * 4 > 227 * 1024)
      fail(BDDC_ERR_INVALID, "a subdomain has more than 58,000 local DOFs (dense local factors are not built for that)");
    L.row_sub = A.upload(row_sub, st);
    int32_t* cnt = A.alloc<int32_t>(L.n_vec);
    launch_csr_pattern(d, L.n_vec, L.row_sub, max_len, cnt, nullptr, nullptr, st);
    std::vector<int32_t> hc(L.n_vec);
    if (L.n_vec > 0) ck(cudaMemcpyAsync(hc.data(), cnt, sizeof(int32_t) * L.n_vec, cudaMemcpyDeviceToHost, st), "d2h");
    ck(cudaStreamSynchronize(st), "sync");
    std::vector<int64_t> row_ptr(L.n_vec + 1, 0);
    for (int64_t r = 0; r < L.n_vec; ++r) row_ptr[r + 1] = row_ptr[r] + hc[r];
    d.row_ptr = A.upload(row_ptr, st);
    d.col = A.alloc<int32_t>(row_ptr[L.n_vec]);
    d.val = A.alloc<double>(row_ptr[L.n_vec]);
    launch_csr_pattern(d, L.n_vec, L.row_sub, max_len, nullptr, d.row_ptr, (int32_t*)d.col, st);
  }
  ph("csr pattern (device)");
  d.c_ptr = A.upload(c_ptr, st);
  d.c_pos = A.upload(c_pos, st);
  d.c_val = A.upload(mp.c_val, st);
  d.loc2iface = A.upload(loc2iface, st);
  d.loc2glob = A.upload(loc2glob, st);
  d.iface_ptr = A.upload(iface_ptr, st);
  d.iface_occ = A.upload(iface_occ, st);
  d.glob_occ_ptr = nullptr;
  d.glob_occ = nullptr;
  d.sub_coarse = A.upload(sub_coarse, st);
  d.cinv_ptr = A.upload(cinv_ptr, st);
  d.cinv_occ = A.upload(cinv_occ, st);
  {
    // constraint rows that augment A_i (Sec. 2 saddle point, Eq. psi_def): the rows of the
    // components carrying the floating modes; Stokes pressure averages stay in the saddle point
    std::vector<double> c_rho(L.sum_nc, 0.0);
    for (int64_t t = 0; t < L.sum_nc; ++t)
      c_rho[t] = ((ms.rigid_mask >> mp.coarse_comp[mp.sub_coarse[t]]) & 1u) ? 1.0 : 0.0;
    d.c_rho = A.upload(c_rho, st);
  }
  d.indefinite = h->physics == BDDC_STOKES ? 1 : 0;
  d.wait_probe = h->opts.wait_probe ? 1 : 0;
  d.sgn = L.fp32 ? (void*)A.alloc<float>(L.n_vec) : (void*)A.alloc<double>(L.n_vec);
  d.w = A.alloc<double>(L.n_vec);
  d.diag = A.alloc<double>(L.n_vec);
  d.rho = A.alloc<double>(ns);
  d.Ginv = A.alloc<double>(L.g_elems);
  d.KC = A.alloc<double>(L.g_elems);
  const size_t ts = L.fp32 ? sizeof(float) : sizeof(double);
  if (L.fp32 && h->opts.tensor_cores) {
    // pre-split panel buffer: kPanel tiles of 16 KB (FP16 hi and lo parts) for every block row
    std::vector<int64_t> po(ns);
    int64_t rows = 0;
    for (int64_t s = 0; s < ns; ++s) {
      po[s] = rows;
      rows += L.meta[s].R;
    }
    L.prow_off = A.upload(po, st);
    L.split = A.alloc<uint8_t>(rows * kPanel * 2 * NB2 * 2);
    if (h->physics == BDDC_STOKES) L.split_signed = A.alloc<uint8_t>(rows * kPanel * 2 * NB2 * 2);
    L.rscale = A.alloc<float>(rows * NB);
    L.tc_panels = h->opts.tensor_cores != 2;
    if (L.tc_panels) L.xinv = A.alloc<float>(ns * 16 * NB2);
    // work items (128 x 128 output blocks) of the updates of every super-panel, flattened over the
    // subdomains; update 0 covers the columns [kb0 + kSub, kb0 + kPanel), update 1 the columns
    // >= kb0 + kPanel, update 2 (a super-panel where some interior ends in the middle, explicit
    // inner operator) the columns >= kb0 + kSub
    const int nu = (int)L.tc_items.size();
    std::vector<int64_t> pref((size_t)nu * (ns + 1), 0);
    for (int u = 0; u < nu; ++u) {
      const int kb0 = (u / kTcLaunches) * kPanel, v = u % kTcLaunches;
      int jbeg = kb0 + (v == 1 ? kPanel : kSub), jend = v == 0 ? kb0 + kPanel : (1 << 30), ibeg = 0;
      if (v >= 3) {   // panel solve of half v - 3: columns [k0, k0 + kSub), rows from k0 + kSub
        jbeg = kb0 + (v - 3) * kSub;
        jend = ibeg = jbeg + kSub;
      }
      int64_t acc = 0;
      for (int64_t s = 0; s < ns; ++s) {
        pref[(size_t)u * (ns + 1) + s] = acc;
        const SubMeta& m = L.meta[s];
        const int ib = std::min(ibeg, (int)m.Bc);
        for (int j = jbeg; j < std::min((int)m.Bc, jend); j += 2) acc += (m.R - std::max(j, ib) + 1) / 2;
      }
      pref[(size_t)u * (ns + 1) + ns] = acc;
      L.tc_items[u] = acc;
    }
    L.item_pref = A.upload(pref, st);
  }
  if (L.fp32) {
    d.tiles = A.alloc<float>(L.tile_elems);
    if (L.split) {
      const int r = make_tile_tmap(&L.tile_tmap, (float*)d.tiles, L.tile_elems);
      if (r) fail(BDDC_ERR_CUDA, "cuTensorMapEncodeTiled for the factor tiles failed (error " + std::to_string(r) + ")");
    }
    d.dinv = A.alloc<float>(L.dinv_elems);
    d.psi = A.alloc<float>(L.psi_elems);
    d.psiT = A.alloc<float>(L.psiT_elems);
    d.schur = L.explicit_schur ? A.alloc<float>(L.schur_elems) : nullptr;
    if (L.explicit_schur) {
      std::vector<int64_t> po(ns);
      int64_t o = 0;
      for (int64_t s2 = 0; s2 < ns; ++s2) {
        po[s2] = o;
        o += (int64_t)L.meta[s2].nGb * (L.meta[s2].nGb - 1) / 2 * NB;
      }
      L.symv_part_off = A.upload(po, st);
    }
  } else {
    d.tiles = A.alloc<double>(L.tile_elems);
    d.dinv = A.alloc<double>(L.dinv_elems);
    d.psi = A.alloc<double>(L.psi_elems);
    d.psiT = A.alloc<double>(L.psiT_elems);
    d.schur = nullptr;
  }
  (void)ts;
  d.status = h->d_status;
  ph("uploads 2, tc items");
  // sweep tasks: block rows of all subdomains, interleaved by depth so that every task's
  // dependencies come earlier in the list
  // (bucketing variant: within every depth the subdomains with the longest chains come first, so
  // uneven subdomains start their critical paths earliest)
  for (int part = 0; part < 2; ++part) {
    std::vector<int64_t> by_len(ns);
    for (int64_t s = 0; s < ns; ++s) by_len[s] = s;
    std::stable_sort(by_len.begin(), by_len.end(), [&](int64_t a, int64_t b) {
      const int la = part == 0 ? (int)ceil_div(L.meta[a].nI, NB) : L.meta[a].nGb;
      const int lb = part == 0 ? (int)ceil_div(L.meta[b].nI, NB) : L.meta[b].nGb;
      return la > lb;
    });
    for (int order = 0; order < 2; ++order)
      for (int dir = 0; dir < 2; ++dir) {
        std::vector<int2> tl;
        int depth = 0;
        for (bool more = true; more; ++depth) {
          more = false;
          for (int64_t k = 0; k < ns; ++k) {
            const int64_t s = order == 0 ? k : by_len[k];
            const SubMeta& m = L.meta[s];
            // interior: the block rows holding interior DOFs (identity tiles that pad the
            // interior block count carry no data: their rows and columns of L are unit vectors)
            const int B0 = part == 0 ? 0 : m.nIb, B1 = part == 0 ? (int)ceil_div(m.nI, NB) : m.Bc;
            if (B0 + depth < B1) {
              more = true;
              tl.push_back(make_int2((int)s, dir == 0 ? B0 + depth : B1 - 1 - depth));
            }
          }
        }
        L.ntasks[part][dir] = (int)tl.size();
        (order == 0 ? L.tasks : L.tasks_big)[part][dir] = A.upload(tl, st);
        if (order == 0 && part == 0) {   // the same tasks grouped per subdomain (batching ablation)
          std::vector<int2> bys(tl.size());
          std::vector<int> off(ns + 1, 0);
          for (const int2& t : tl) off[t.x + 1]++;
          for (int64_t q = 0; q < ns; ++q) off[q + 1] += off[q];
          std::vector<int> fill(off.begin(), off.end() - 1);
          for (const int2& t : tl) bys[fill[t.x]++] = t;
          L.tasks_by_sub[dir] = A.upload(bys, st);
          L.task_sub_off[dir] = off;
        }
      }
  }
  ph("sweep tasks");
  L.ctrl = A.alloc<int>(1);   // task counter of the sweeps
  {
    std::vector<int64_t> rl[3];
    std::vector<int32_t> cs;
    std::vector<int64_t> o0(ns + 1, 0), o1(ns + 1, 0), oc(ns + 1, 0);
    for (int64_t s = 0; s < ns; ++s) {
      o0[s + 1] = o0[s] + L.meta[s].nI;
      o1[s + 1] = o1[s] + L.meta[s].nG;
      oc[s + 1] = oc[s] + L.meta[s].nc;
    }
    rl[0].resize(o0[ns]);
    rl[1].resize(o1[ns]);
    rl[2].resize(o0[ns] + o1[ns]);
    cs.resize(oc[ns]);
    parallel_for(ns, [&](int64_t s) {
      const SubMeta& m = L.meta[s];
      for (int r = 0; r < m.nI; ++r) rl[0][o0[s] + r] = rl[2][o0[s] + r] = m.vec_off + r;
      for (int r = 0; r < m.nG; ++r)
        rl[1][o1[s] + r] = rl[2][o0[ns] + o1[s] + r] = m.vec_off + (int64_t)m.nIb * NB + r;
      for (int q = 0; q < m.nc; ++q) cs[oc[s] + q] = (int32_t)s;
    });
    for (int k = 0; k < 3; ++k) {
      L.nrows[k] = (int64_t)rl[k].size();
      L.rows[k] = A.upload(rl[k], st);
    }
    L.crow_sub = A.upload(cs, st);
  }
  ph("row lists");
  L.slot_elem = A.upload(slot_elem, st);
  L.iface_dofs = A.upload(mp.iface_dofs, st);
  alloc_level_work(L, A, 1);
  ph("work buffers");
}

// Element matrices of levels > 1 come from the previous level's K_Ci: segment copies.
void prepare_level_segments(Level& L, const Level& prev, DevArena& A, cudaStream_t st) {
  const int64_t nel = L.mesh.n_elems;
  std::vector<int64_t> src(nel), len(nel);
  std::vector<int32_t> slot_elem(nel);
  for (int64_t s = 0; s < L.maps.n_sub(); ++s)
    for (int64_t k = L.maps.sub_elem_ptr[s]; k < L.maps.sub_elem_ptr[s + 1]; ++k) slot_elem[k] = (int32_t)L.maps.sub_elems[k];
  for (int64_t k = 0; k < nel; ++k) {
    const SubMeta& pm = prev.meta[slot_elem[k]];
    src[k] = pm.g_off;
    len[k] = (int64_t)pm.nc * pm.nc;
  }
  L.seg_src = A.upload(src, st);
  L.seg_len = A.upload(len, st);
}

// ------------------------------------------------------------------ numeric set-up
template <typename T>
void factor_level(bddc_handle_s* h, Level& L, cudaStream_t st) {
  LevelDev& d = L.d;
  launch_csr_values(d, L.n_vec, L.row_sub, st);
  if (!L.coarsest) launch_weights(d, h->opts.weights == BDDC_WEIGHTS_MULTIPLICITY, nullptr, st);
  ck(cudaMemsetAsync(d.tiles, 0, sizeof(T) * (size_t)std::max<int64_t>(L.tile_elems, 1), st), "memset tiles");
  launch_densify_rows<T>(d, L.row_sub, st);
  launch_add_constraints<T>(d, st);
  if (sizeof(T) == 4 && h->opts.tensor_cores) {
    // 512-wide super-panels of two 256-wide sub-panels.  Per sub-panel: its 256 x 256 diagonal
    // block factored on CUDA cores and inverted (X = L_D^{-1}); the rows below it solved on the
    // tensor cores as L(i, D) = A(i, D) X^T S_D (tensor_cores = 2: on CUDA cores, tile by tile).
    // After the first sub-panel a rank-256 tcgen05 update brings the second sub-panel's columns
    // up to date; after the second, one rank-512 update serves every trailing column.
    for (int kb0 = 0; kb0 < L.max_Bc; kb0 += kPanel) {
      const int p = kb0 / kPanel;
      // explicit inner operator: the trailing interface block of every subdomain whose interior
      // ends here is its augmented Schur complement (all interior updates applied, no interface
      // column factored yet)
      if (L.explicit_schur && L.snap_start[p]) launch_schur_snapshot(d, kb0, L.max_nGb, st);
      // a super-panel in which some interior ends after its first half takes two rank-256
      // updates of all trailing columns instead of the rank-256 / rank-512 pair, so that the
      // Schur complement exists between them
      const bool split_mid = L.explicit_schur && L.snap_mid[p];
      for (int half = 0; half < 2; ++half) {
        const int k0 = kb0 + half * kSub, k1 = k0 + kSub;
        const int u = kTcLaunches * p + (half ? 1 : (split_mid ? 2 : 0));
        const int nq = split_mid ? kSub : (half ? kPanel : kSub);   // K tiles of the update
        const int kq = split_mid ? k0 : kb0;                        // its first K column
        const int jend = (half || split_mid) ? (1 << 30) : kb0 + kPanel;
        if (k0 < L.max_Bc && L.tc_panels) {
          {
            double fl = 0.0;
            for (int k = k0; k < std::min(k1, L.max_Bc); ++k) fl += L.block_flops[k];
            ProfScope ps(h, BDDC_PROF_FACTOR, 0.0, fl, st);
            bool fused = false;
            for (int k = k0; k < std::min(k1, L.max_Bc); ++k) {
              const bool fuse = k + 1 < k1 && L.block_tiles[k] > 0;
              launch_potrf_step<T>(d, k, L.max_R, L.block_tiles[k], k1, st, fused, fuse, k1, L.xinv, k0);
              fused = fuse;
            }
            launch_split_inverse(d, k0, L.xinv, L.split, L.rscale, L.prow_off, st);
            launch_split_panel(d, k0, kSub, k1, L.max_R, L.split, nullptr, L.rscale, L.prow_off, st, 1);
          }
          const int up = kTcLaunches * p + 3 + half;
          if (L.tc_items[up] > 0) {
            ProfScope ps(h, BDDC_PROF_TC_PANEL, 0.0, L.tc_flops[up], st);
            launch_update_tc2(d, kSub, k0, k1, k1, 1, (int)std::min<int64_t>(L.tc_items[up], h->grid_max / 2),
                              L.split, L.split, L.rscale, L.prow_off, L.item_pref + (size_t)up * (d.n_sub + 1),
                              L.tile_tmap, st);
          }
          if (L.split && L.tc_items[u] > 0) {
            ProfScope ps(h, BDDC_PROF_FACTOR, 0.0, 0.0, st);
            launch_split_panel(d, kq, nq, k1, L.max_R, L.split, L.split_signed, L.rscale, L.prow_off, st);
          }
        } else {
          double fl = 0.0;
          for (int k = k0; k < std::min(k1, L.max_Bc); ++k) fl += L.panel_flops[k];
          ProfScope ps(h, BDDC_PROF_FACTOR, 0.0, fl, st);
          bool fused = false;   // the previous step's update factored this step's diagonal tile
          for (int k = k0; k < std::min(k1, L.max_Bc); ++k) {
            const bool fuse = k + 1 < k1 && L.narrow_tiles[k] > 0;
            launch_potrf_step<T>(d, k, L.max_R, L.narrow_tiles[k], k1, st, fused, fuse);
            fused = fuse;
          }
          if (L.split && L.tc_items[u] > 0)
            launch_split_panel(d, kq, nq, k1, L.max_R, L.split, L.split_signed, L.rscale, L.prow_off, st);
        }
        const int64_t items = L.tc_items[u];
        if (L.split && items > 0) {   // no launch where no subdomain has columns left
          const double fl = (split_mid && half) ? 0.5 * L.tc_flops[u] : L.tc_flops[u];
          ProfScope ps(h, BDDC_PROF_TC_UPDATE, 0.0, fl, st);
          launch_update_tc2(d, nq, k1, jend, 0, 0, (int)std::min<int64_t>(items, h->grid_max / 2), L.split,
                            L.split_signed ? L.split_signed : L.split, L.rscale, L.prow_off,
                            L.item_pref + (size_t)u * (d.n_sub + 1), L.tile_tmap, st);
        }
        if (split_mid && half == 0) launch_schur_snapshot(d, k1, L.max_nGb, st);
      }
    }
  } else {
    bool fused = false;
    for (int k = 0; k < L.max_Bc; ++k) {
      ProfScope ps(h, BDDC_PROF_FACTOR, 0.0, L.step_flops[k], st);
      const bool fuse = L.max_tiles[k] > 0;
      launch_potrf_step<T>(d, k, L.max_R, L.max_tiles[k], 1 << 30, st, fused, fuse);
      fused = fuse;
    }
  }
  if (L.max_nc > 0) {
    launch_gram_chol(d, L.fp32 ? 1 : 0, L.max_nc, st);
    launch_psi<T>(d, L.max_nGb, L.max_nc, st);
    launch_psi_transpose<T>(d, L.max_nGb, L.max_ncb, st);   // the solve phase streams Psi_G^T by tiles
  }
  ck(cudaGetLastError(), "factor launch");
}

void check_status(bddc_handle_s* h, int level) {
  int st[4];
  ck(cudaMemcpyAsync(st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost, h->st), "status");
  ck(cudaStreamSynchronize(h->st), "sync");
  if (st[2]) fail(BDDC_ERR_TIMEOUT, "a bounded device-side wait gave up (code " + std::to_string(st[2]) + ")");
  if (st[0]) {
    h->stats.breakdown_level = level;
    h->stats.breakdown_sub = st[1];
    fail(BDDC_ERR_BREAKDOWN, "non-positive pivot on level " + std::to_string(level) + " subdomain " +
                                 std::to_string(st[1]));
  }
}

// A bounded wait that gave up explains whatever else went wrong in the same call (NaN, no
// convergence): report it first.
void throw_if_timeout(bddc_handle_s* h) {
  int st[4];
  if (cudaMemcpyAsync(st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost, h->st) != cudaSuccess) return;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return;
  if (st[2]) fail(BDDC_ERR_TIMEOUT, "a bounded device-side wait gave up (code " + std::to_string(st[2]) + ")");
}

void reset_status(bddc_handle_s* h) {
  int init[4] = {0, 0x7fffffff, 0, 0};
  ck(cudaMemcpyAsync(h->d_status, init, sizeof(init), cudaMemcpyHostToDevice, h->st), "status init");
}

// ------------------------------------------------------------------ solve-phase building blocks
// Every building block acts on nb right-hand sides at once (nb <= the level's block capacity);
// a block stores its columns one after another (see internal.h).

// launches of a sweep or factor product over nb columns (groups of 8/4/2/1, or 4/2/1 in FP64)
int column_groups(int nb, int max_nr) {
  int n = 0;
  for (int r = 0; r < nb; ++n) {
    const int left = nb - r;
    r += left >= max_nr ? max_nr : left >= 4 ? 4 : left >= 2 ? 2 : 1;
  }
  return n;
}

template <typename T>
void trsv_one(bddc_handle_s* h, Level& L, T* v, int part, int backward, cudaStream_t st, int nb = 1) {
  const bool copy32 = sizeof(T) == 4 && L.solve32;   // FP32 copy of an FP64 factor
  const double groups = column_groups(nb, sizeof(T) == 4 ? 8 : 4);
  ProfScope ps(h, L.coarsest ? BDDC_PROF_COARSE : part == 0 ? BDDC_PROF_TRSV : BDDC_PROF_TRSV_IFACE,
               groups * (copy32 ? 0.5 * L.trsv_bytes[part] : L.trsv_bytes[part]), 0.0, st);
  launch_sweep<T>(copy32 ? L.d32 : L.d, v, (L.sweep_order[part] ? L.tasks_big : L.tasks)[part][backward], L.ntasks[part][backward],
                  part, backward, L.ctrl, L.pub, h->grid_max / 2 * L.sweep_ctas[part], L.sweep_deep[part], st, nb);
}

template <typename T>
void trsv_pair(bddc_handle_s* h, Level& L, T* v, int part, cudaStream_t st, int nb = 1) {
  trsv_one<T>(h, L, v, part, 0, st, nb);
  trsv_one<T>(h, L, v, part, 1, st, nb);
}

// w = K_II^{-1} v on level 1 (interior positions), FP64 accuracy.
// FP64 factors: two sweeps.  FP32 factors: iterative refinement with the FP64 K_II.
void interior_solve_l1(bddc_handle_s* h, Level& L, const double* v, double* w, cudaStream_t st, int nb = 1) {
  const int64_t n = L.n_vec * nb;
  if (!L.fp32) {
    ck(cudaMemcpyAsync(w, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy");
    trsv_pair<double>(h, L, w, 0, st, nb);
    return;
  }
  float* t = (float*)L.locB;
  double* r = L.dl3;
  ck(cudaMemsetAsync(w, 0, sizeof(double) * n, st), "memset");
  const int steps = std::max(1, h->cur_steps);
  for (int it = 0; it < steps; ++it) {
    launch_convert<double, float>(it == 0 ? v : r, t, n, st);
    trsv_pair<float>(h, L, t, 0, st, nb);
    launch_add_to_double<float>(w, t, n, st);
    if (it + 1 < steps) {
      ck(cudaMemcpyAsync(r, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy");
      launch_spmv_rows(L.d, L.rows[0], L.nrows[0], w, r, -1.0, 1.0, L.row_sub, st, nb);
    }
  }
}

// y = S x on the level-1 interface (Sec. 2, discrete Dirichlet problems).  With cur_steps = 0
// on an FP32 level: the inner operator S~ = sum R_i^T (L_GG S L_GG^T - C_i^T R C_i) R_i from the
// stored factor (no interior solves).
void schur_apply(bddc_handle_s* h, const double* x, double* y, cudaStream_t st, int nb = 1) {
  Level& L = h->lv[0];
  const int64_t n = L.n_vec * nb;
  if (L.fp32 && h->cur_steps == 0) {
    launch_gather_iface<double>(L.d, x, 0, L.dl0, st, nb);
    launch_convert<double, float>(L.dl0, (float*)L.locA, n, st);
    const float* yf = (const float*)L.locA;
    if (L.explicit_schur) {   // one pass over the lower triangle of S_i + C_i^T R C_i
      ProfScope ps(h, BDDC_PROF_TRMV, column_groups(nb, 4) * 0.5 * L.trmv_bytes, 0.0, st);
      launch_schur_symv(L.d, L.max_nGb, L.symv_part_off, L.symv_stride, (const float*)L.locA, L.symv_part,
                        (float*)L.locB, st, nb);
      yf = (const float*)L.locB;
    } else {
      ProfScope ps(h, BDDC_PROF_TRMV, column_groups(nb, 8) * L.trmv_bytes, 0.0, st);
      launch_trmv_schur(L.d, L.max_nGb, (const float*)L.locA, (float*)L.locB, (float*)L.locA, st, nb);
    }
    launch_convert<float, double>(yf, L.dl1, n, st);
    launch_sub_ctrc(L.d, L.crow_sub, L.sum_nc, L.dl0, L.dl1, st, nb);
    launch_scatter_iface<double>(L.d, L.dl1, 0, y, st, nb);
    return;
  }
  launch_gather_iface<double>(L.d, x, 0, L.dl0, st, nb);                 // x_i = R_i x
  ck(cudaMemsetAsync(L.dl1, 0, sizeof(double) * n, st), "memset");
  launch_spmv_rows(L.d, L.rows[0], L.nrows[0], L.dl0, L.dl1, 1.0, 0.0, L.row_sub, st, nb);  // v = K_IG x_i
  interior_solve_l1(h, L, L.dl1, L.dl2, st, nb);                        // w = K_II^{-1} v
  launch_axpy_loc(L.dl0, L.dl2, -1.0, n, st);                           // t = [-w ; x_i]
  launch_spmv_rows(L.d, L.rows[1], L.nrows[1], L.dl0, L.dl1, 1.0, 0.0, L.row_sub, st, nb);  // y_i = K_GG x_i - K_GI w
  launch_scatter_iface<double>(L.d, L.dl1, 0, y, st, nb);                // y = sum R_i^T y_i
}

// g = f_G - sum R_i^T K_GI K_II^{-1} f_I   (f: nb columns of n_free)
void condensed_rhs(bddc_handle_s* h, const double* f, double* g, cudaStream_t st, int nb = 1) {
  Level& L = h->lv[0];
  launch_gather_glob<double>(L.d, f, 0, L.dl1, st, nb);
  interior_solve_l1(h, L, L.dl1, L.dl2, st, nb);
  launch_spmv_rows(L.d, L.rows[1], L.nrows[1], L.dl2, L.dl0, 1.0, 0.0, L.row_sub, st, nb);
  launch_scatter_iface<double>(L.d, L.dl0, 0, L.gi0, st, nb);
  launch_iface_rhs(g, f, L.d.n_dof, L.iface_dofs, L.gi0, L.d.n_iface, st, nb);
}

// u_I = K_II^{-1} (f_I - K_IG u_G), u_G = u_hat
void recover(bddc_handle_s* h, const double* f, const double* uG, double* u, cudaStream_t st, int nb = 1) {
  Level& L = h->lv[0];
  launch_gather_iface<double>(L.d, uG, 0, L.dl0, st, nb);
  launch_gather_glob<double>(L.d, f, 0, L.dl1, st, nb);
  launch_spmv_rows(L.d, L.rows[0], L.nrows[0], L.dl0, L.dl1, -1.0, 1.0, L.row_sub, st, nb);
  interior_solve_l1(h, L, L.dl1, L.dl2, st, nb);
  ck(cudaMemsetAsync(u, 0, sizeof(double) * h->n_free * nb, st), "memset");
  launch_scatter_interior<double>(L.d, L.dl2, u, st, nb);
  launch_put_indexed(u, h->n_free, L.iface_dofs, uG, L.d.n_iface, st, nb);
}

void coarsest_solve(bddc_handle_s* h, const double* rC, double* zC, cudaStream_t st, int nb = 1) {
  Level& C = h->lv.back();
  if (C.solve32) {   // mixed form: the preconditioner's coarse solve with the FP32 copy of the factor
    launch_gather_glob<float>(C.d32, rC, 2, C.v32, st, nb);
    if (C.winv) {     // explicit inverse of that copy: one product
      ProfScope ps(h, BDDC_PROF_COARSE, 4.0 * (double)C.n_vec * C.n_vec * column_groups(nb, 8), 0.0, st);
      launch_coarse_apply(C.winv, C.n_vec, C.v32, C.v32b, C.n_vec, nb, st);
      launch_scatter_interior<float>(C.d32, C.v32b, zC, st, nb);
      return;
    }
    trsv_pair<float>(h, C, C.v32, 0, st, nb);
    launch_scatter_interior<float>(C.d32, C.v32, zC, st, nb);
    return;
  }
  double* v = (double*)C.locA;
  launch_gather_glob<double>(C.d, rC, 2, v, st, nb);
  trsv_pair<double>(h, C, v, 0, st, nb);
  launch_scatter_interior<double>(C.d, v, zC, st, nb);
}

void full_step(bddc_handle_s* h, int l, const double* r, double* z, cudaStream_t st, int nb);

// One interface step of Algorithm 2 on BDDC level l: distribute, subdomain corrections,
// coarse residual, coarse correction (coarsest solve or the next level), combine.
template <typename T>
void interface_step_t(bddc_handle_s* h, int l, const double* rhat, double* zhat, cudaStream_t st, int nb) {
  Level& L = h->lv[l];
  T* v = (T*)L.locA;
  launch_gather_iface<T>(L.d, rhat, 1, v, st, nb);          // r_i = E_i^T r_hat
  launch_psi_t_apply<T>(L.d, v, L.psi_part, L.sum_nc, L.rc_sub, L.max_nGb, L.max_ncb, st, nb);   // Psi_i^T r_i
  launch_coarse_gather(L.d, L.rc_sub, L.sum_nc, L.rC, st, nb);   // r_C = sum R_Ci^T Psi_i^T r_i
  trsv_one<T>(h, L, v, 1, 0, st, nb);                       // Eq. sub_cor via the trailing factor
  launch_constraint_corr<T>(L.d, v, L.crow_sub, L.sum_nc, L.cc_t, L.cc_mu, L.psi_part, L.max_nGb, L.max_ncb, st,
                            nb);
  trsv_one<T>(h, L, v, 1, 1, st, nb);
  const bool last = l + 2 == (int)h->lv.size();
  if (last)
    coarsest_solve(h, L.rC, L.zC, st, nb);
  else
    full_step(h, l + 1, L.rC, L.zC, st, nb);
  launch_coarse_scatter_n(L.d.sub_coarse, L.sum_nc, L.zC, L.d.n_coarse, L.zc_sub, st, nb);
  launch_psi_apply_add<T>(L.d, L.zc_sub, L.sum_nc, v, L.max_nGb, L.max_ncb, st, nb);   // Psi_i R_Ci z_C + z_i
  launch_scatter_iface<T>(L.d, v, 1, zhat, st, nb);            // z_hat = sum E_i (...)
}

void interface_step(bddc_handle_s* h, int l, const double* rhat, double* zhat, cudaStream_t st, int nb) {
  if (h->lv[l].fp32)
    interface_step_t<float>(h, l, rhat, zhat, st, nb);
  else
    interface_step_t<double>(h, l, rhat, zhat, st, nb);
}

// Levels l > 1: interior pre-correction, interface step, interior post-correction
template <typename T>
void full_step_t(bddc_handle_s* h, int l, const double* r, double* z, cudaStream_t st, int nb) {
  Level& L = h->lv[l];
  const int64_t n = L.n_vec * nb;
  T* v = (T*)L.locB;
  launch_gather_glob<T>(L.d, r, 0, v, st, nb);                     // r_I
  trsv_pair<T>(h, L, v, 0, st, nb);                                // u1 = A_II^{-1} r_I
  launch_convert<T, double>(v, L.dl0, n, st);
  launch_spmv_rows(L.d, L.rows[1], L.nrows[1], L.dl0, L.dl1, 1.0, 0.0, L.row_sub, st, nb);   // (A_GI u1)_i
  launch_scatter_iface<double>(L.d, L.dl1, 0, L.gi0, st, nb);
  launch_iface_rhs(L.gi1, r, L.d.n_dof, L.iface_dofs, L.gi0, L.d.n_iface, st, nb);   // r'_G = r_G - A_GI u1
  interface_step(h, l, L.gi1, L.gi2, st, nb);                       // z_G
  launch_gather_iface<double>(L.d, L.gi2, 0, L.dl0, st, nb);
  launch_gather_glob<double>(L.d, r, 0, L.dl1, st, nb);
  launch_spmv_rows(L.d, L.rows[0], L.nrows[0], L.dl0, L.dl1, -1.0, 1.0, L.row_sub, st, nb);  // r_I - A_IG z_G
  launch_convert<double, T>(L.dl1, v, n, st);
  trsv_pair<T>(h, L, v, 0, st, nb);                                 // z_I
  ck(cudaMemsetAsync(z, 0, sizeof(double) * L.d.n_dof * nb, st), "memset");
  launch_scatter_interior<T>(L.d, v, z, st, nb);
  launch_put_indexed(z, L.d.n_dof, L.iface_dofs, L.gi2, L.d.n_iface, st, nb);
}

void full_step(bddc_handle_s* h, int l, const double* r, double* z, cudaStream_t st, int nb) {
  if (h->lv[l].fp32)
    full_step_t<float>(h, l, r, z, st, nb);
  else
    full_step_t<double>(h, l, r, z, st, nb);
}

void precond(bddc_handle_s* h, const double* r, double* z, cudaStream_t st, int nb = 1) {
  interface_step(h, 0, r, z, st, nb);
}

double dot_host(bddc_handle_s* h, const double* a, const double* b, int64_t n) {
  launch_dot(a, b, n, h->partial, kDotBlocks, h->scal + 15, h->st);
  ck(cudaMemcpyAsync(h->h_scal + 15, h->scal + 15, sizeof(double), cudaMemcpyDeviceToHost, h->st), "d2h");
  ck(cudaStreamSynchronize(h->st), "sync");
  return h->h_scal[15];
}

// Choose the number of FP64 refinement steps of the interior solves (FP32 factors): run the
// refinement on a probe right-hand side until the FP64 residual stops decreasing.
void choose_refinement(bddc_handle_s* h) {
  Level& L = h->lv[0];
  if (!L.fp32) {
    h->refine_steps = h->cur_steps = 0;
    return;
  }
  if (h->opts.refine_steps > 0) {
    h->refine_steps = h->cur_steps = h->opts.refine_steps;
    return;
  }
  cudaStream_t st = h->st;
  const int64_t n = L.n_vec;
  std::vector<double> ones(L.d.n_iface, 1.0);
  ck(cudaMemcpyAsync(L.gi1, ones.data(), sizeof(double) * ones.size(), cudaMemcpyHostToDevice, st), "h2d");
  launch_gather_iface<double>(L.d, L.gi1, 0, L.dl0, st);
  double* v = h->full_a;   // n_vec-sized scratch allocated for this purpose
  double* w = h->full_b;
  ck(cudaMemsetAsync(v, 0, sizeof(double) * n, st), "memset");
  launch_spmv_rows(L.d, L.rows[0], L.nrows[0], L.dl0, v, 1.0, 0.0, L.row_sub, st);
  const double nv = std::sqrt(dot_host(h, v, v, n));
  // the refinement of interior_solve_l1 run step by step: after step s, w and the residual
  // r = v - K_II w are exactly those of an interior solve with s steps (the same operations in
  // the same order), so one pass measures every step count
  int best = 1;
  double prev = 1e300;
  float* t = (float*)L.locB;
  double* r = L.dl3;
  ck(cudaMemsetAsync(w, 0, sizeof(double) * n, st), "memset");
  for (int steps = 1; steps <= 8; ++steps) {
    h->refine_steps = h->cur_steps = steps;
    launch_convert<double, float>(steps == 1 ? v : r, t, n, st);
    trsv_pair<float>(h, L, t, 0, st);
    launch_add_to_double<float>(w, t, n, st);
    ck(cudaMemcpyAsync(r, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy");
    launch_spmv_rows(L.d, L.rows[0], L.nrows[0], w, r, -1.0, 1.0, L.row_sub, st);
    const double rel = nv > 0 ? std::sqrt(dot_host(h, r, r, n)) / nv : 0.0;
    if (rel > 0.5 * prev) break;          // stagnated at round-off: the previous count suffices
    best = steps;
    if (rel < 4e-16) break;
    prev = rel;
  }
  h->refine_steps = h->cur_steps = best;
}

// ------------------------------------------------------------------ autotuner
// Launch variants of the streaming sweeps, timed with CUDA events on the level's own factors:
// CTAs per SM of the persistent grid (1, 2), tile-ring depth (shallow, deep), task order (subdomain
// order, longest chains first).  The sweeps compute the same result bit for bit in every variant
// (each block row adds its tile contributions in a fixed order), so the choice only moves time.
// Results are cached per level shape (precision, subdomain count, block-row histogram).
std::mutex g_tune_mu;
std::map<std::string, std::array<int, 6>> g_tune_cache;

std::string level_shape_key(const Level& L) {
  std::string k = (L.fp32 || L.solve32 ? "f" : "d") + std::to_string(L.meta.size()) + ":";
  for (const SubMeta& m : L.meta) k += std::to_string(m.nIb) + "," + std::to_string(m.nGb) + ";";
  return k;
}

template <typename T>
void tune_sweeps(bddc_handle_s* h, Level& L, cudaStream_t st) {
  const std::string key = level_shape_key(L);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      for (int p = 0; p < 2; ++p) {
        L.sweep_ctas[p] = it->second[3 * p];
        L.sweep_deep[p] = it->second[3 * p + 1];
        L.sweep_order[p] = it->second[3 * p + 2];
      }
      return;
    }
  }
  const double t0 = now_ms();
  const int saved_profile = h->opts.profile;
  h->opts.profile = 0;
  T* v = (sizeof(T) == 4 && L.solve32) ? (T*)L.v32 : (T*)L.locA;
  ck(cudaMemsetAsync(v, 0, sizeof(T) * (size_t)L.n_vec, st), "memset");
  cudaEvent_t a, b;
  ck(cudaEventCreate(&a), "cudaEventCreate");
  ck(cudaEventCreate(&b), "cudaEventCreate");
  for (int p = 0; p < 2; ++p) {
    if (L.ntasks[p][0] == 0) continue;
    float best = 1e30f;
    int bc = 2, bd = 1, bo = 0;
    for (int order = 0; order < 2; ++order)
      for (int deep = 1; deep >= 0; --deep)
        for (int ctas = 2; ctas >= 1; --ctas) {
          L.sweep_ctas[p] = ctas;
          L.sweep_deep[p] = deep;
          L.sweep_order[p] = order;
          trsv_pair<T>(h, L, v, p, st);   // warm-up
          ck(cudaEventRecord(a, st), "cudaEventRecord");
          for (int r = 0; r < 2; ++r) trsv_pair<T>(h, L, v, p, st);
          ck(cudaEventRecord(b, st), "cudaEventRecord");
          ck(cudaEventSynchronize(b), "cudaEventSynchronize");
          float ms = 0.f;
          ck(cudaEventElapsedTime(&ms, a, b), "cudaEventElapsedTime");
          if (ms < 0.97f * best) {   // a variant must win clearly to replace an earlier one
            best = ms;
            bc = ctas;
            bd = deep;
            bo = order;
          }
        }
    L.sweep_ctas[p] = bc;
    L.sweep_deep[p] = bd;
    L.sweep_order[p] = bo;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->opts.profile = saved_profile;
  h->stats.tune_ms += now_ms() - t0;
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune_cache[key] = {L.sweep_ctas[0], L.sweep_deep[0], L.sweep_order[0], L.sweep_ctas[1], L.sweep_deep[1],
                       L.sweep_order[1]};
}

void numeric_setup(bddc_handle_s* h) {
  cudaStream_t st = h->st;
  const double t0 = now_ms();
  reset_status(h);
  h->stats.tune_ms = 0.0;
  ck(cudaMemcpyAsync(h->d_coef, h->coef.data(), sizeof(double) * h->n_elems, cudaMemcpyHostToDevice, st), "coef");
  for (size_t l = 0; l < h->lv.size(); ++l) {
    Level& L = h->lv[l];
    if (l == 0) {
      if (h->ke_early) {   // computed in element order at the start of the set-up
        launch_gather_elems(h->n_elems, h->npe * h->ndof, L.slot_elem, h->ke_elem, L.d.ke, st);
        h->arena.free_one(h->ke_elem);
        h->ke_elem = nullptr;
        h->ke_early = false;
      } else if (h->physics == BDDC_STOKES)
        launch_elem_q2q1(h->n_elems, h->d_coords, h->d_conn, h->d_coef, L.slot_elem, L.d.ke, st);
      else
        launch_elem_q1p1(h->physics, h->dim, h->npe == h->dim + 1, h->n_elems, h->d_coords, h->d_conn, h->d_coef,
                         h->nu, L.slot_elem, L.d.ke, st);
      if (h->has_lift)
        launch_lift(h->n_free, h->npe * h->ndof, h->d_lift_ptr, h->d_lift_slot, h->d_lift_a, L.d.ke, h->d_lift_ud,
                    h->d_lift, st);
    } else {
      const Level& P = h->lv[l - 1];
      launch_copy_segments(P.d.KC, L.seg_src, L.d.ke, L.d.ke_off, L.seg_len, L.mesh.n_elems, st);
    }
    if (L.fp32)
      factor_level<float>(h, L, st);
    else
      factor_level<double>(h, L, st);
    check_status(h, (int)l + 1);
    if (L.coarsest && h->opts.precision == BDDC_PREC_MIXED) {
      // the coarsest factorisation stays FP64; its solves inside the FP32 preconditioner use an FP32
      // copy (FP64 arithmetic on GB300 runs at 1/64 of FP32 and made these short sweeps compute-bound)
      if (!L.solve32) {
        L.d32 = L.d;
        L.d32.tiles = h->arena.alloc<float>(L.tile_elems);
        L.d32.dinv = h->arena.alloc<float>(L.dinv_elems);
        L.d32.sgn = h->arena.alloc<float>(L.n_vec);
        L.v32 = h->arena.alloc<float>(L.n_vec * L.blk);
        L.v32b = h->arena.alloc<float>(L.n_vec * L.blk);
        if (L.n_vec <= kMaxCoarseInverse) L.winv = h->arena.alloc<float>(L.n_vec * L.n_vec);
        L.solve32 = true;
      }
      launch_convert<double, float>((const double*)L.d.tiles, (float*)L.d32.tiles, L.tile_elems, st);
      launch_convert<double, float>((const double*)L.d.dinv, (float*)L.d32.dinv, L.dinv_elems, st);
      launch_convert<double, float>((const double*)L.d.sgn, (float*)L.d32.sgn, L.n_vec, st);
      // the preconditioner's coarse solves then are one product with the explicit inverse (a
      // sweep pair over the coarse factor is a chain of dependent block rows: latency-bound)
      if (L.winv) launch_coarse_inverse(L.d32, L.n_vec, L.winv, st);
    }
    if (h->opts.autotune && !L.winv) {   // the explicit inverse replaces the coarsest sweeps
      if (L.fp32 || L.solve32)
        tune_sweeps<float>(h, L, st);
      else
        tune_sweeps<double>(h, L, st);
      check_status(h, (int)l + 1);
    }
    for (int p = 0; p < 2; ++p) {
      h->stats.sweep_ctas[2 * l + p] = L.sweep_ctas[p];
      h->stats.sweep_deep[2 * l + p] = L.sweep_deep[p];
      h->stats.sweep_order[2 * l + p] = L.sweep_order[p];
    }
  }
  choose_refinement(h);
  check_status(h, 0);   // the refinement probe's sweeps
  h->stats.factor_ms = now_ms() - t0;
  flush_profile(h);
  h->stats.refine_steps = h->refine_steps;
  h->cur_steps = h->refine_steps;
  h->use_outer = false;
  h->inner_steps = 0;
  if (h->lv[0].fp32 && krylov_kind(h) == BDDC_KRYLOV_PCG && h->opts.inner_steps >= 0 &&
      h->opts.inner_steps < h->refine_steps) {
    h->use_outer = true;
    h->inner_steps = h->opts.inner_steps;
  }
  h->stats.inner_steps = h->use_outer ? h->inner_steps : -1;
  h->stats.inner_operator = h->use_outer ? (h->lv[0].explicit_schur ? 2 : 1) : 0;
  h->factored = true;
}

// Repeated set-ups allocate and free tens of MB of host index arrays; with glibc's defaults the
// freed heap top is returned to the kernel and the next set-up faults it in again.  Padding and
// retaining the heap top keeps those pages (opts.retain_host_memory, once per process).
void retain_host_heap() {
#ifdef __GLIBC__
  static std::once_flag once;
  std::call_once(once, []() {
    mallopt(M_TOP_PAD, 256 << 20);
    mallopt(M_TRIM_THRESHOLD, 1 << 30);
  });
#endif
}

void analysis(bddc_handle_s* h, const bddc_mesh* mesh, const bddc_partition* part,
              const std::function<void()>& after_input = {}) {
  if (h->opts.retain_host_memory) retain_host_heap();
  const double t0 = now_ms();
  if (!mesh || !part) fail(BDDC_ERR_INVALID, "null mesh or partition");
  if (h->opts.krylov < BDDC_KRYLOV_AUTO || h->opts.krylov > BDDC_KRYLOV_FGMRES) fail(BDDC_ERR_INVALID, "unknown Krylov method");
  if (mesh->dim != 2 && mesh->dim != 3) fail(BDDC_ERR_INVALID, "dim must be 2 or 3");
  if (mesh->physics != BDDC_POISSON && mesh->physics != BDDC_ELASTICITY && mesh->physics != BDDC_STOKES)
    fail(BDDC_ERR_INVALID, "unknown physics");
  if (mesh->physics == BDDC_STOKES) {
    if (mesh->dim != 3 || mesh->nodes_per_elem != 27 || mesh->dofs_per_node != 4)
      fail(BDDC_ERR_INVALID, "Stokes needs Q2-Q1 hexahedra: dim 3, 27 nodes per element, 4 DOFs per node");
  } else if (mesh->nodes_per_elem != (1 << mesh->dim) && mesh->nodes_per_elem != mesh->dim + 1) {
    fail(BDDC_ERR_INVALID, "Poisson and elasticity take Q1 boxes (2**dim nodes) or linear simplices (dim + 1 nodes)");
  }
  if (mesh->physics == BDDC_ELASTICITY && (mesh->dim != 3 || mesh->dofs_per_node != 3))
    fail(BDDC_ERR_INVALID, "elasticity needs dim 3 and 3 DOFs per node");
  if (mesh->physics == BDDC_POISSON && mesh->dofs_per_node != 1) fail(BDDC_ERR_INVALID, "Poisson needs 1 DOF per node");
  if (part->n_levels < 2 || part->n_levels > BDDC_MAX_LEVELS) fail(BDDC_ERR_INVALID, "n_levels out of range");
  if (mesh->n_nodes <= 0 || mesh->n_elems <= 0 || !mesh->coords || !mesh->conn || !mesh->coef || !mesh->dirichlet)
    fail(BDDC_ERR_INVALID, "empty mesh or null array");
  h->dim = mesh->dim;
  h->npe = mesh->nodes_per_elem;
  h->ndof = mesh->dofs_per_node;
  h->physics = mesh->physics;
  h->n_nodes = mesh->n_nodes;
  h->n_elems = mesh->n_elems;
  h->nu = mesh->nu;
  h->n_full = h->n_nodes * h->ndof;
  h->coords.assign(mesh->coords, mesh->coords + h->n_nodes * h->dim);
  h->conn.assign(mesh->conn, mesh->conn + h->n_elems * h->npe);
  h->coef.assign(mesh->coef, mesh->coef + h->n_elems);
  {   // element checks in chunks on the host pool; the first failing element is reported
    constexpr int64_t kChunk = 8192;
    std::atomic<int64_t> bad_coef{INT64_MAX}, bad_conn{INT64_MAX};
    host_parallel((h->n_elems + kChunk - 1) / kChunk, [&](int64_t b, int) {
      const int64_t e0 = b * kChunk, e1 = std::min(h->n_elems, e0 + kChunk);
      for (int64_t e = e0; e < e1; ++e) {
        if (!(h->coef[e] > 0.0)) {
          int64_t cur = bad_coef.load();
          while (e < cur && !bad_coef.compare_exchange_weak(cur, e)) {
          }
        }
        for (int a = 0; a < h->npe; ++a) {
          const int32_t p = h->conn[e * h->npe + a];
          if (p < 0 || p >= h->n_nodes) {
            int64_t cur = bad_conn.load();
            while (e < cur && !bad_conn.compare_exchange_weak(cur, e)) {
            }
          }
        }
      }
    });
    if (bad_coef.load() != INT64_MAX)
      fail(BDDC_ERR_INVALID, "coefficient must be positive (element " + std::to_string(bad_coef.load()) + ")");
    if (bad_conn.load() != INT64_MAX) fail(BDDC_ERR_INVALID, "connectivity references a missing node");
  }
  if (h->npe == h->dim + 1)   // linear simplices: a flat element has no inverse Jacobian
    for (int64_t e = 0; e < h->n_elems; ++e) {
      double J[3][3] = {{0}}, h2 = 0.0;
      const double* x0 = &h->coords[(int64_t)h->conn[e * h->npe] * h->dim];
      for (int a = 1; a <= h->dim; ++a) {
        const double* xa = &h->coords[(int64_t)h->conn[e * h->npe + a] * h->dim];
        for (int d = 0; d < h->dim; ++d) {
          J[a - 1][d] = xa[d] - x0[d];
          h2 = std::max(h2, std::fabs(J[a - 1][d]));
        }
      }
      const double det = h->dim == 2 ? J[0][0] * J[1][1] - J[0][1] * J[1][0]
                                     : J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      if (!(std::fabs(det) > 1e-12 * std::pow(h2, h->dim)))
        fail(BDDC_ERR_INVALID, "degenerate simplex (element " + std::to_string(e) + ")");
    }
  h->free_of_full.assign(h->n_full, -1);
  h->n_free = 0;
  for (int64_t q = 0; q < h->n_full; ++q)
    if (!mesh->dirichlet[q]) h->free_of_full[q] = h->n_free++;
  h->dir_full.clear();   // kept only when a prescribed value is non-zero
  h->has_lift = false;
  if (mesh->dir_values)
    for (int64_t q = 0; q < h->n_full; ++q)
      if (mesh->dirichlet[q] && mesh->dir_values[q] != 0.0) {
        if (!std::isfinite(mesh->dir_values[q])) fail(BDDC_ERR_INVALID, "non-finite prescribed value");
        if (!h->has_lift) h->dir_full.assign(h->n_full, 0.0);
        h->dir_full[q] = mesh->dir_values[q];
        h->has_lift = true;
      }
  h->n_levels = part->n_levels;
  h->parts.clear();
  h->n_parts.clear();
  for (int l = 0; l + 1 < h->n_levels; ++l) {
    if (!part->part[l] || part->n_parts[l] <= 0) fail(BDDC_ERR_INVALID, "missing partition of level " + std::to_string(l + 1));
    if (part->n_parts[l] > kMaxSubdomains)   // batched launches put the subdomains on grid.y
      fail(BDDC_ERR_INVALID, "level " + std::to_string(l + 1) + " has more than 65,535 subdomains");
    const int64_t n_items = l == 0 ? h->n_elems : h->n_parts[l - 1];
    h->parts.emplace_back(part->part[l], part->part[l] + n_items);
    h->n_parts.push_back(part->n_parts[l]);
  }
  h->lv.clear();
  h->lv.resize(h->n_levels);   // L-1 BDDC levels + coarsest
  std::string err;
  double tp = t0;
  auto phase = [&](const char* what, int level) {   // opts.verbose >= 2: host phase times on stderr
    const double t = now_ms();
    if (h->opts.verbose >= 2) fprintf(stderr, "bddc analysis: %-16s level %d %8.2f ms\n", what, level, t - tp);
    tp = t;
  };
  phase("input", 0);
  if (after_input) {   // device work that needs only the validated inputs (overlaps the analysis)
    after_input();
    phase("early device", 0);
  }
  for (int l = 0; l + 1 < h->n_levels; ++l) {
    Level& L = h->lv[l];
    if (l == 0)
      build_level1_mesh(h, &L.mesh);
    else
      next_level_mesh(h->lv[l - 1].mesh, h->lv[l - 1].maps, h->parts[l].data(), h->n_parts[l], &L.mesh);
    phase("mesh", l + 1);
    const bool allc = (h->opts.all_corners >> l) & 1u;
    if (!analyze_level(L.mesh, h->constraints, allc, &L.maps, &err)) fail(BDDC_ERR_INVALID, "level " + std::to_string(l + 1) + ": " + err);
    phase("analyze", l + 1);
    L.fp32 = h->opts.precision == BDDC_PREC_MIXED;
    h->stats.n_sub[l] = L.maps.n_sub();
    h->stats.n_dof[l] = L.mesh.n_dof;
    h->stats.n_iface[l] = L.maps.n_iface;
    h->stats.n_coarse[l] = L.maps.n_coarse;
    h->stats.n_promoted[l] = L.maps.n_promoted;
  }
  Level& C = h->lv.back();
  C.coarsest = true;
  C.fp32 = false;
  build_coarsest_mesh(h->lv[h->n_levels - 2], &C.mesh);
  phase("mesh", h->n_levels);
  if (!analyze_level(C.mesh, 0u, false, &C.maps, &err)) fail(BDDC_ERR_INVALID, "coarsest level: " + err);
  phase("analyze", h->n_levels);
  h->stats.n_levels = h->n_levels;
  h->stats.analysis_ms = now_ms() - t0;
}

// The level-1 element matrices depend only on the validated inputs: upload the mesh and compute
// them in element order on the handle's stream right away, so that the GPU works while the host
// analyses the mesh and prepares the levels; numeric_setup gathers them into element slots.
void early_device(bddc_handle_s* h) {
  cudaStream_t st = h->st;
  DevArena& A = h->arena;
  h->d_coords = A.upload(h->coords, st);
  h->d_conn = A.upload(h->conn, st);
  h->d_coef = A.alloc<double>(h->n_elems);
  ck(cudaMemcpyAsync(h->d_coef, h->coef.data(), sizeof(double) * h->n_elems, cudaMemcpyHostToDevice, st), "coef");
  const int64_t ne = (int64_t)h->npe * h->ndof;
  h->ke_elem = A.alloc<double>(h->n_elems * ne * ne);
  if (h->physics == BDDC_STOKES)
    launch_elem_q2q1(h->n_elems, h->d_coords, h->d_conn, h->d_coef, nullptr, h->ke_elem, st);
  else
    launch_elem_q1p1(h->physics, h->dim, h->npe == h->dim + 1, h->n_elems, h->d_coords, h->d_conn, h->d_coef, h->nu,
                     nullptr, h->ke_elem, st);
  h->ke_early = true;
}

void device_setup(bddc_handle_s* h) {
  const double t0 = now_ms();
  cudaStream_t st = h->st;
  DevArena& A = h->arena;
  {
    int dev = 0, sms = 0;
    ck(cudaGetDevice(&dev), "cudaGetDevice");
    ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    h->grid_max = 2 * std::max(1, sms);
  }
  h->d_status = A.alloc<int>(4);
  if (!h->d_coords) {
    h->d_coords = A.upload(h->coords, st);
    h->d_conn = A.upload(h->conn, st);
    h->d_coef = A.alloc<double>(h->n_elems);
  }
  h->d_free_of_full = A.upload(h->free_of_full, st);
  for (size_t l = 0; l < h->lv.size(); ++l) {
    const double tl = now_ms(), u0 = A.upload_ms;
    const int64_t b0 = A.upload_bytes;
    prepare_level(h, h->lv[l], A, st);
    if (l > 0) prepare_level_segments(h->lv[l], h->lv[l - 1], A, st);
    if (h->opts.verbose >= 2)
      fprintf(stderr, "bddc prepare: level %d %8.2f ms (uploads %.2f ms, %.1f MB)\n", (int)l + 1, now_ms() - tl,
              A.upload_ms - u0, (double)(A.upload_bytes - b0) / 1e6);
  }
  if (h->has_lift) {
    // occurrences (slot, element row) of every free DOF in elements that touch a non-zero
    // prescribed value, in slot order; u_d of every slot
    const Level& L = h->lv[0];
    const int ne = h->npe * h->ndof;
    const int64_t nel = h->n_elems;
    std::vector<int32_t> slot_elem(nel);
    for (int64_t s = 0; s < L.maps.n_sub(); ++s)
      for (int64_t k = L.maps.sub_elem_ptr[s]; k < L.maps.sub_elem_ptr[s + 1]; ++k)
        slot_elem[k] = (int32_t)L.maps.sub_elems[k];
    std::vector<double> ud((size_t)nel * ne, 0.0);
    std::vector<int64_t> ptr(h->n_free + 1, 0);
    std::vector<char> lifting(nel, 0);
    auto full_dof = [&](int64_t e, int a) {
      return (int64_t)h->conn[e * h->npe + a / h->ndof] * h->ndof + a % h->ndof;
    };
    for (int64_t k = 0; k < nel; ++k) {
      const int64_t e = slot_elem[k];
      for (int a = 0; a < ne; ++a) {
        const double v = h->dir_full[full_dof(e, a)];
        ud[(size_t)k * ne + a] = v;
        if (v != 0.0) lifting[k] = 1;
      }
      if (lifting[k])
        for (int a = 0; a < ne; ++a) {
          const int64_t g = h->free_of_full[full_dof(e, a)];
          if (g >= 0) ptr[g + 1]++;
        }
    }
    for (int64_t g = 0; g < h->n_free; ++g) ptr[g + 1] += ptr[g];
    std::vector<int32_t> lslot(ptr[h->n_free]), la(ptr[h->n_free]);
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t k = 0; k < nel; ++k) {
      if (!lifting[k]) continue;
      const int64_t e = slot_elem[k];
      for (int a = 0; a < ne; ++a) {
        const int64_t g = h->free_of_full[full_dof(e, a)];
        if (g < 0) continue;
        lslot[fill[g]] = (int32_t)k;
        la[fill[g]] = a;
        fill[g]++;
      }
    }
    h->d_dir_full = A.upload(h->dir_full, st);
    h->d_lift_ud = A.upload(ud, st);
    h->d_lift_ptr = A.upload(ptr, st);
    h->d_lift_slot = A.upload(lslot, st);
    h->d_lift_a = A.upload(la, st);
    h->d_lift = A.alloc<double>(h->n_free);
  }
  h->scal = A.alloc<double>(16);
  h->partial = A.alloc<double>(kDotBlocks);
  ck(cudaMallocHost(&h->h_scal, sizeof(double) * 16), "cudaMallocHost");
  const int64_t ni = std::max<int64_t>(h->lv[0].d.n_iface, 1);
  h->vx = A.alloc<double>(ni);
  h->vr = A.alloc<double>(ni);
  h->vz = A.alloc<double>(ni);
  h->vp = A.alloc<double>(ni);
  h->vq = A.alloc<double>(ni);
  h->vrold = A.alloc<double>(ni);
  h->vg = A.alloc<double>(ni);
  h->vs = A.alloc<double>(ni);
  h->vsh = A.alloc<double>(ni);
  h->vt = A.alloc<double>(ni);
  if (krylov_kind(h) == BDDC_KRYLOV_FGMRES) {
    h->gm_V = A.alloc<double>(ni * (kRestart + 1));
    h->gm_Z = A.alloc<double>(ni * kRestart);
    h->gm_w = A.alloc<double>(ni);
    h->gm_h = A.alloc<double>(3 * (kRestart + 1) + 2);
    h->gm_partial = A.alloc<double>((int64_t)kDotBlocks * (kRestart + 1));
    ck(cudaMallocHost(&h->h_gm, sizeof(double) * (3 * (kRestart + 1) + 2)), "cudaMallocHost");
  }
  h->fcol = A.alloc<double>(h->n_free);
  h->ucol = A.alloc<double>(h->n_free);
  const int64_t nbig = std::max<int64_t>(h->n_full, h->lv[0].n_vec);
  h->full_a = A.alloc<double>(nbig);
  h->full_b = A.alloc<double>(nbig);
  const double ts = now_ms();
  ck(cudaStreamSynchronize(st), "sync");
  if (h->opts.verbose >= 2) fprintf(stderr, "bddc prepare: final sync %8.2f ms\n", now_ms() - ts);
  h->stats.prepare_ms = now_ms() - t0;
}

// ------------------------------------------------------------------ PCG (Sec. 4)
struct PcgResult {
  int iterations = 0;
  int outer = 0;              // FP64 outer refinement steps (pcg_refined)
  bool converged = false;
  double rel = 0.0;
  double gnorm = 0.0;
  std::vector<double> alpha, beta;
};

// One full PCG iteration (Sec. 4) on the level-1 interface for a block of nb right-hand sides,
// all on the device: q = S p, alpha = r.z / p.q, x += alpha p, r -= alpha q, ||r||^2,
// z = M^{-1} r (Algorithm 2), beta (Fletcher-Reeves or flexible), p = z + beta p.  Column k keeps
// its scalars at scal[16 k ..]; a column whose flag scal[16 k + 8] is set stays frozen.
void pcg_body(bddc_handle_s* h, double* x, int flexible, cudaStream_t st, int nb) {
  const int64_t n = h->lv[0].d.n_iface;
  double* S = h->scal;
  schur_apply(h, h->vp, h->vq, st, nb);
  launch_dot(h->vp, h->vq, n, h->partial, kDotBlocks, S + 1, st, nb);
  launch_pcg_scalars(S, 0, flexible, st, nb);
  if (flexible) ck(cudaMemcpyAsync(h->vrold, h->vr, sizeof(double) * n * nb, cudaMemcpyDeviceToDevice, st), "copy");
  launch_pcg_update_x_r(x, h->vr, h->vp, h->vq, S, n, st, nb);
  launch_dot(h->vr, h->vr, n, h->partial, kDotBlocks, S + 5, st, nb);
  precond(h, h->vr, h->vz, st, nb);
  launch_dot(h->vr, h->vz, n, h->partial, kDotBlocks, S + 4, st, nb);
  if (flexible) launch_dot(h->vz, h->vrold, n, h->partial, kDotBlocks, S + 7, st, nb);
  launch_pcg_scalars(S, 1, flexible, st, nb);
  launch_pcg_update_p(h->vp, h->vz, S, n, st, nb);
}

// One right-preconditioned BiCGstab iteration (van der Vorst; the Krylov method of the Stokes
// experiments of Sec. 4), all on the device.  Vectors: x, r = vr, rh = vrold (fixed shadow
// residual), p = vp, ph = M^{-1} p = vz, v = S ph = vq, s = vs, sh = M^{-1} s = vsh, t = S sh = vt.
// Scalars: 0 rho, 1 alpha, 2 omega, 3 rho_new, 4 rh.v, 5 t.s, 6 t.t, 7 beta, 8 r.r.
void bicg_body(bddc_handle_s* h, double* x, cudaStream_t st) {
  const int64_t n = h->lv[0].d.n_iface;
  double* S = h->scal;
  launch_dot(h->vrold, h->vr, n, h->partial, kDotBlocks, S + 3, st);
  launch_bicg_scalars(S, 0, st);
  launch_bicg_p(h->vp, h->vr, h->vq, S, n, st);
  precond(h, h->vp, h->vz, st);
  schur_apply(h, h->vz, h->vq, st);
  launch_dot(h->vrold, h->vq, n, h->partial, kDotBlocks, S + 4, st);
  launch_bicg_scalars(S, 1, st);
  launch_bicg_s(h->vs, h->vr, h->vq, S, n, st);
  precond(h, h->vs, h->vsh, st);
  schur_apply(h, h->vsh, h->vt, st);
  launch_dot(h->vt, h->vs, n, h->partial, kDotBlocks, S + 5, st);
  launch_dot(h->vt, h->vt, n, h->partial, kDotBlocks, S + 6, st);
  launch_bicg_scalars(S, 2, st);
  launch_bicg_xr(x, h->vr, h->vz, h->vsh, h->vs, h->vt, S, n, st);
  launch_dot(h->vr, h->vr, n, h->partial, kDotBlocks, S + 8, st);
}

// kind 0/1: PCG with Fletcher-Reeves / flexible beta (nb columns); 2: BiCGstab (one column)
void iteration_body(bddc_handle_s* h, double* x, int kind, cudaStream_t st, int nb) {
  if (kind == 2)
    bicg_body(h, x, st);
  else
    pcg_body(h, x, kind, st, nb);
}

// Capture one Krylov iteration into a CUDA graph (once per handle and key; the buffers never
// move while a graph is cached).  A captured iteration depends on the method (0/1: PCG with
// Fletcher-Reeves / flexible beta, 2: BiCGstab), on the interior-solve steps of the Schur operator
// and on the number of right-hand sides of the block.
int graph_key(const bddc_handle_s* h, int kind, int nb) { return kind | (h->cur_steps << 3) | (nb << 8); }

void capture_iteration(bddc_handle_s* h, int kind, int nb) {
  if (!h->cap_st) ck(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking), "cudaStreamCreate");
  cudaGraph_t g = nullptr;
  flush_profile(h);   // events recorded so far belong to eager launches
  const int64_t launches0 = g_launches.load();
  ck(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  try {
    iteration_body(h, h->vx, kind, h->cap_st, nb);
  } catch (...) {
    cudaStreamEndCapture(h->cap_st, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  ck(cudaStreamEndCapture(h->cap_st, &g), "cudaStreamEndCapture");
  // captured kernels did not run: count them once per replay instead
  h->graph_kernels = g_launches.load() - launches0;
  g_launches.fetch_sub(h->graph_kernels);
  h->graph_prof.insert(h->graph_prof.end(), h->prof_pending.begin(), h->prof_pending.end());
  h->prof_pending.clear();
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  ck(e, "cudaGraphInstantiate");
  h->iter_graph = ex;
  h->iter_graph_key = graph_key(h, kind, nb);
}

void drop_graph(bddc_handle_s* h) {
  if (!h->iter_graph) return;
  cudaGraphExecDestroy(h->iter_graph);
  h->iter_graph = nullptr;
  h->iter_graph_key = -1;
  for (auto& r : h->graph_prof) {
    h->event_pool.push_back(r.a);
    h->event_pool.push_back(r.b);
  }
  h->graph_prof.clear();
}

void drop_graph_if_kind_differs(bddc_handle_s* h, int kind, int nb) {
  if (h->iter_graph && h->iter_graph_key != graph_key(h, kind, nb)) drop_graph(h);
}

// Work vectors for blocks of up to kMaxBlock right-hand sides: allocated at the first solve with
// more than one right-hand side (a set-up allocates for one); the cached iteration graph, which
// refers to the old buffers, is dropped.
void ensure_block(bddc_handle_s* h, int nb) {
  if (h->blk >= nb) return;
  const int blk = kMaxBlock;
  ck(cudaStreamSynchronize(h->st), "sync");
  drop_graph(h);
  DevArena& A = h->arena;
  for (Level& L : h->lv) alloc_level_work(L, A, blk);
  const int64_t ni = std::max<int64_t>(h->lv[0].d.n_iface, 1) * blk;
  h->vx = A.alloc<double>(ni);
  h->vr = A.alloc<double>(ni);
  h->vz = A.alloc<double>(ni);
  h->vp = A.alloc<double>(ni);
  h->vq = A.alloc<double>(ni);
  h->vrold = A.alloc<double>(ni);
  h->vg = A.alloc<double>(ni);
  h->vs = A.alloc<double>(ni);
  h->vsh = A.alloc<double>(ni);
  h->vt = A.alloc<double>(ni);
  h->scal = A.alloc<double>(16 * blk);
  h->partial = A.alloc<double>((int64_t)kDotBlocks * blk);
  if (h->h_scal) cudaFreeHost(h->h_scal);
  h->h_scal = nullptr;
  ck(cudaMallocHost(&h->h_scal, sizeof(double) * 16 * blk), "cudaMallocHost");
  h->fcol = A.alloc<double>(h->n_free * blk);
  h->ucol = A.alloc<double>(h->n_free * blk);
  h->blk = blk;
}

// r = g - S x, z = M^{-1} r, p = z, rz = r.z  (start, or restart after a failed true-residual
// check) for every column of the block
void pcg_start(bddc_handle_s* h, const double* g, double* x, bool x_zero, cudaStream_t st, int nb) {
  const int64_t n = h->lv[0].d.n_iface;
  double* S = h->scal;
  ck(cudaMemcpyAsync(h->vr, g, sizeof(double) * n * nb, cudaMemcpyDeviceToDevice, st), "copy");
  if (!x_zero) {
    schur_apply(h, x, h->vq, st, nb);
    launch_axpy_loc(h->vr, h->vq, -1.0, n * nb, st);
  }
  precond(h, h->vr, h->vz, st, nb);
  ck(cudaMemcpyAsync(h->vp, h->vz, sizeof(double) * n * nb, cudaMemcpyDeviceToDevice, st), "copy");
  launch_dot(h->vr, h->vz, n, h->partial, kDotBlocks, S + 0, st, nb);
}

// Freeze column k of the running block PCG (its alpha and beta become 0 from the next kernel on).
void freeze_column(bddc_handle_s* h, int k) {
  h->h_scal[16 * k + 8] = 1.0;
  ck(cudaMemcpyAsync(h->scal + 16 * k + 8, h->h_scal + 16 * k + 8, sizeof(double), cudaMemcpyHostToDevice, h->st),
     "h2d");
}

// PCG on the level-1 interface (Sec. 4) for nb right-hand sides g (columns of n_iface) in
// lockstep: every iteration applies S and the preconditioner to the whole block, so each factor
// tile is read once for all columns.  Column k stops at ||r_k|| / ||g_k|| <= tol[k] once its true
// residual confirms it (after one failed confirmation every column restarts from its iterate with
// the true residual; after a second the column stops as not converged); stopped columns stay
// frozen while the others continue.  x: nb columns.
std::vector<PcgResult> pcg(bddc_handle_s* h, const double* g, double* x, const std::vector<double>& tol, int maxit,
                           int nb) {
  cudaStream_t st = h->st;
  const int64_t n = h->lv[0].d.n_iface;
  std::vector<PcgResult> res(nb);
  const int flexible = h->opts.flexible < 0 ? (h->opts.precision == BDDC_PREC_MIXED) : h->opts.flexible;
  ck(cudaMemsetAsync(x, 0, sizeof(double) * n * nb, st), "memset");
  if (n == 0) {
    for (auto& r : res) r.converged = true;
    return res;
  }
  double* S = h->scal;
  ck(cudaMemsetAsync(S, 0, sizeof(double) * 16 * nb, st), "memset");
  launch_dot(g, g, n, h->partial, kDotBlocks, S + 6, st, nb);
  ck(cudaMemcpyAsync(h->h_scal, S, sizeof(double) * 16 * nb, cudaMemcpyDeviceToHost, st), "d2h");
  ck(cudaStreamSynchronize(st), "sync");
  std::vector<double> gg(nb);
  std::vector<char> frozen(nb, 0), checked(nb, 0);
  int active = nb;
  for (int k = 0; k < nb; ++k) {
    gg[k] = h->h_scal[16 * k + 6];
    if (!std::isfinite(gg[k])) fail(BDDC_ERR_NAN, "NaN in the condensed right-hand side");
    res[k].gnorm = std::sqrt(gg[k]);
    if (gg[k] == 0.0) {
      res[k].converged = true;
      frozen[k] = 1;
      --active;
      freeze_column(h, k);
    }
  }
  if (active == 0) return res;
  pcg_start(h, g, x, true, st, nb);
  const bool graphs = h->opts.use_graph && x == h->vx;
  drop_graph_if_kind_differs(h, flexible, nb);
  for (int it = 1; it <= maxit; ++it) {
    bool replayed = false;
    if (graphs && h->iter_graph) {
      ck(cudaGraphLaunch(h->iter_graph, st), "cudaGraphLaunch");
      g_launches.fetch_add(h->graph_kernels);
      replayed = true;
    } else {
      pcg_body(h, x, flexible, st, nb);   // the first iteration runs eagerly, then it is captured
      if (graphs) capture_iteration(h, flexible, nb);
    }
    ck(cudaMemcpyAsync(h->h_scal, S, sizeof(double) * 16 * nb, cudaMemcpyDeviceToHost, st), "d2h");
    ck(cudaStreamSynchronize(st), "sync");
    if (replayed && !h->graph_prof.empty()) accumulate_graph_profile(h);
    std::vector<int> check;
    for (int k = 0; k < nb; ++k) {
      if (frozen[k]) continue;
      const double* sk = h->h_scal + 16 * k;
      res[k].iterations = it;
      res[k].alpha.push_back(sk[2]);
      res[k].beta.push_back(sk[3]);
      const double rel = std::sqrt(sk[5] / gg[k]);
      if (!std::isfinite(rel)) fail(BDDC_ERR_NAN, "NaN in the Krylov recurrence");
      res[k].rel = rel;
      if (rel <= tol[k]) check.push_back(k);
    }
    if (check.empty()) continue;
    schur_apply(h, x, h->vq, st, nb);                                 // true residuals g - S x
    ck(cudaMemcpyAsync(h->vrold, g, sizeof(double) * n * nb, cudaMemcpyDeviceToDevice, st), "copy");
    launch_axpy_loc(h->vrold, h->vq, -1.0, n * nb, st);
    launch_dot(h->vrold, h->vrold, n, h->partial, kDotBlocks, S + 9, st, nb);
    ck(cudaMemcpyAsync(h->h_scal, S, sizeof(double) * 16 * nb, cudaMemcpyDeviceToHost, st), "d2h");
    ck(cudaStreamSynchronize(st), "sync");
    bool restart = false;
    for (int k : check) {
      const double rel_true = std::sqrt(h->h_scal[16 * k + 9] / gg[k]);
      if (rel_true <= tol[k] || checked[k]) {
        res[k].rel = rel_true;
        res[k].converged = rel_true <= tol[k];
        frozen[k] = 1;
        --active;
      } else {
        checked[k] = 1;
        restart = true;
      }
    }
    for (int k = 0; k < nb; ++k)   // the readback overwrote the host copies of the flags
      if (frozen[k]) freeze_column(h, k);
    if (active == 0) return res;
    if (restart) pcg_start(h, g, x, false, st, nb);   // restart from the iterates with the true residuals
  }
  return res;
}

// Right-preconditioned BiCGstab on the level-1 interface; stops on ||r|| / ||g|| <= tol once
// the true residual g - S x confirms it (the recurrence continues otherwise).
PcgResult bicgstab(bddc_handle_s* h, const double* g, double* x, double tol, int maxit) {
  cudaStream_t st = h->st;
  const int64_t n = h->lv[0].d.n_iface;
  PcgResult res;
  ck(cudaMemsetAsync(x, 0, sizeof(double) * n, st), "memset");
  if (n == 0) {
    res.converged = true;
    return res;
  }
  double* S = h->scal;
  ck(cudaMemsetAsync(S, 0, sizeof(double) * 16, st), "memset");
  launch_dot(g, g, n, h->partial, kDotBlocks, S + 10, st);
  ck(cudaMemcpyAsync(h->vr, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy");
  ck(cudaMemcpyAsync(h->vrold, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy");
  ck(cudaMemsetAsync(h->vp, 0, sizeof(double) * n, st), "memset");
  ck(cudaMemsetAsync(h->vq, 0, sizeof(double) * n, st), "memset");
  launch_bicg_scalars(S, 3, st);
  ck(cudaMemcpyAsync(h->h_scal, S, sizeof(double) * 16, cudaMemcpyDeviceToHost, st), "d2h");
  ck(cudaStreamSynchronize(st), "sync");
  const double gg = h->h_scal[10];
  if (!std::isfinite(gg)) fail(BDDC_ERR_NAN, "NaN in the condensed right-hand side");
  res.gnorm = std::sqrt(gg);
  if (gg == 0.0) {
    res.converged = true;
    return res;
  }
  const bool graphs = h->opts.use_graph && x == h->vx;
  drop_graph_if_kind_differs(h, 2, 1);
  for (int it = 1; it <= maxit; ++it) {
    bool replayed = false;
    if (graphs && h->iter_graph) {
      ck(cudaGraphLaunch(h->iter_graph, st), "cudaGraphLaunch");
      g_launches.fetch_add(h->graph_kernels);
      replayed = true;
    } else {
      bicg_body(h, x, st);
      if (graphs) capture_iteration(h, 2, 1);
    }
    ck(cudaMemcpyAsync(h->h_scal, S, sizeof(double) * 16, cudaMemcpyDeviceToHost, st), "d2h");
    ck(cudaStreamSynchronize(st), "sync");
    if (replayed && !h->graph_prof.empty()) accumulate_graph_profile(h);
    res.iterations = it;
    const double rel = std::sqrt(h->h_scal[8] / gg);
    if (!std::isfinite(rel)) fail(BDDC_ERR_NAN, "NaN in the Krylov recurrence");
    res.rel = rel;
    if (rel <= tol) {
      schur_apply(h, x, h->vq, st);
      ck(cudaMemcpyAsync(h->vs, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy");
      launch_axpy_loc(h->vs, h->vq, -1.0, n, st);
      launch_dot(h->vs, h->vs, n, h->partial, kDotBlocks, S + 9, st);
      ck(cudaMemcpyAsync(h->h_scal + 9, S + 9, sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
      ck(cudaStreamSynchronize(st), "sync");
      const double rel_true = std::sqrt(h->h_scal[9] / gg);
      res.rel = rel_true;
      if (rel_true <= tol) {
        res.converged = true;
        return res;
      }
    }
  }
  return res;
}

void lanczos(const PcgResult& r, double* lmin, double* lmax) {
  const int k = (int)r.alpha.size();
  *lmin = *lmax = 1.0;
  if (k == 0) return;
  // tridiagonal eigenvalues by bisection (Sturm sequence)
  std::vector<double> a(k), b(k, 0.0);
  for (int j = 0; j < k; ++j) {
    a[j] = 1.0 / r.alpha[j] + (j > 0 && j - 1 < (int)r.beta.size() ? r.beta[j - 1] / r.alpha[j - 1] : 0.0);
    if (j + 1 < k && j < (int)r.beta.size()) b[j] = std::sqrt(std::max(r.beta[j], 0.0)) / r.alpha[j];
  }
  double lo = 1e300, hi = -1e300;
  for (int j = 0; j < k; ++j) {
    double rad = (j > 0 ? std::fabs(b[j - 1]) : 0.0) + std::fabs(b[j]);
    lo = std::min(lo, a[j] - rad);
    hi = std::max(hi, a[j] + rad);
  }
  auto count_below = [&](double x) {
    int cnt = 0;
    double d = 1.0;
    for (int j = 0; j < k; ++j) {
      d = a[j] - x - (j > 0 ? b[j - 1] * b[j - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) ++cnt;
    }
    return cnt;
  };
  auto kth = [&](int idx) {
    double l = lo, u = hi;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (l + u);
      if (count_below(mid) > idx) u = mid; else l = mid;
    }
    return 0.5 * (l + u);
  };
  *lmin = kth(0);
  *lmax = kth(k - 1);
}

// Flexible GMRES(kRestart) with right preconditioning (Saad): the Krylov basis V is built from
// S z_j with z_j = M^{-1} v_j kept in Z, so the update x += Z y stays exact for a preconditioner
// that is not a fixed linear operator (FP32 factors of an indefinite saddle point: their rounding
// error, ~kappa * 2^-24, breaks BiCGstab's short recurrences).  Classical Gram-Schmidt applied
// twice; Givens rotations and the small triangular solve on the host.
PcgResult fgmres(bddc_handle_s* h, const double* g, double* x, double tol, int maxit) {
  cudaStream_t st = h->st;
  const int64_t n = h->lv[0].d.n_iface;
  const int m = kRestart;
  PcgResult res;
  ck(cudaMemsetAsync(x, 0, sizeof(double) * n, st), "memset");
  if (n == 0) {
    res.converged = true;
    return res;
  }
  double* S = h->scal;
  double* hd0 = h->gm_h;              // [m + 1] first Gram-Schmidt pass
  double* hd1 = h->gm_h + (m + 1);    // [m + 1] second pass
  double* hnrm = h->gm_h + 2 * (m + 1);
  double* yd = h->gm_h + 2 * (m + 1) + 2;   // [m]
  double* hh = h->h_gm;               // pinned mirror of gm_h
  launch_dot(g, g, n, h->partial, kDotBlocks, S + 0, st);
  ck(cudaMemcpyAsync(h->h_scal, S, sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
  ck(cudaStreamSynchronize(st), "sync");
  const double gg = h->h_scal[0];
  if (!std::isfinite(gg)) fail(BDDC_ERR_NAN, "NaN in the condensed right-hand side");
  res.gnorm = std::sqrt(gg);
  if (gg == 0.0) {
    res.converged = true;
    return res;
  }
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  int it = 0;
  bool first = true;
  while (it < maxit) {
    // r = g - S x (x = 0 on the first cycle), v_0 = r / ||r||
    ck(cudaMemcpyAsync(h->gm_w, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy");
    if (!first) {
      schur_apply(h, x, h->vq, st);
      launch_axpy_loc(h->gm_w, h->vq, -1.0, n, st);
    }
    launch_dot(h->gm_w, h->gm_w, n, h->partial, kDotBlocks, hnrm, st);
    launch_scale_by_norm(h->gm_V, h->gm_w, hnrm, n, st);
    ck(cudaMemcpyAsync(hh + 2 * (m + 1), hnrm, sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
    ck(cudaStreamSynchronize(st), "sync");
    const double beta = std::sqrt(hh[2 * (m + 1)]);
    if (!std::isfinite(beta)) fail(BDDC_ERR_NAN, "NaN in the Krylov recurrence");
    res.rel = beta / res.gnorm;
    if (res.rel <= tol) {   // the true residual of the current iterate meets the tolerance
      res.converged = true;
      return res;
    }
    first = false;
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;   // Arnoldi steps of this cycle
    while (k < m && it < maxit) {
      const int j = k;
      double* Vj = h->gm_V + (int64_t)j * n;
      double* Zj = h->gm_Z + (int64_t)j * n;
      precond(h, Vj, Zj, st);
      schur_apply(h, Zj, h->gm_w, st);
      launch_multidot(h->gm_V, n, j + 1, h->gm_w, n, h->gm_partial, kDotBlocks, hd0, st);
      launch_combine(h->gm_w, h->gm_V, n, j + 1, hd0, -1.0, n, st);
      launch_multidot(h->gm_V, n, j + 1, h->gm_w, n, h->gm_partial, kDotBlocks, hd1, st);
      launch_combine(h->gm_w, h->gm_V, n, j + 1, hd1, -1.0, n, st);
      launch_dot(h->gm_w, h->gm_w, n, h->partial, kDotBlocks, hnrm, st);
      launch_scale_by_norm(h->gm_V + (int64_t)(j + 1) * n, h->gm_w, hnrm, n, st);
      ck(cudaMemcpyAsync(hh, h->gm_h, sizeof(double) * (2 * (m + 1) + 1), cudaMemcpyDeviceToHost, st), "d2h");
      ck(cudaStreamSynchronize(st), "sync");
      double* col = &H[(size_t)j * (m + 1)];   // column j of the Hessenberg matrix
      for (int i = 0; i <= j; ++i) col[i] = hh[i] + hh[(m + 1) + i];
      col[j + 1] = std::sqrt(std::max(hh[2 * (m + 1)], 0.0));
      for (int i = 0; i < j; ++i) {   // earlier rotations
        const double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
      }
      const double a = col[j], b = col[j + 1];
      const double rr = std::hypot(a, b);
      cs[j] = rr > 0.0 ? a / rr : 1.0;
      sn[j] = rr > 0.0 ? b / rr : 0.0;
      col[j] = rr;
      col[j + 1] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++k;
      ++it;
      res.iterations = it;
      res.rel = std::fabs(gv[j + 1]) / res.gnorm;
      if (!std::isfinite(res.rel)) fail(BDDC_ERR_NAN, "NaN in the Krylov recurrence");
      if (res.rel <= tol || rr == 0.0) break;
    }
    // y = R^{-1} g (upper triangular after the rotations), x += Z y
    for (int i = k - 1; i >= 0; --i) {
      double sacc = gv[i];
      for (int l = i + 1; l < k; ++l) sacc -= H[(size_t)l * (m + 1) + i] * y[l];
      const double d = H[(size_t)i * (m + 1) + i];
      y[i] = d != 0.0 ? sacc / d : 0.0;
    }
    std::copy(y.begin(), y.begin() + k, hh + 2 * (m + 1) + 2);
    ck(cudaMemcpyAsync(yd, hh + 2 * (m + 1) + 2, sizeof(double) * k, cudaMemcpyHostToDevice, st), "h2d");
    launch_combine(x, h->gm_Z, n, k, yd, 1.0, n, st);
    ck(cudaStreamSynchronize(st), "sync");
    // the next cycle starts from the true residual and stops there if it meets the tolerance
  }
  // iteration cap: report the true residual
  schur_apply(h, x, h->vq, st);
  ck(cudaMemcpyAsync(h->gm_w, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy");
  launch_axpy_loc(h->gm_w, h->vq, -1.0, n, st);
  launch_dot(h->gm_w, h->gm_w, n, h->partial, kDotBlocks, S + 9, st);
  ck(cudaMemcpyAsync(h->h_scal + 9, S + 9, sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
  ck(cudaStreamSynchronize(st), "sync");
  res.rel = std::sqrt(h->h_scal[9] / gg);
  res.converged = res.rel <= tol;
  return res;
}

// Mixed-precision iterative refinement around PCG (the outer iteration that restores FP64
// accuracy), for a block of nb right-hand sides: x += S~^{-1} r with r = g - S x, where S is the
// FP64 Schur operator (interior solves refined to FP64 accuracy) and S~ the same operator with
// h->inner_steps interior-solve steps (0: products with the stored interface factor, no interior
// solve; k >= 1: k interior-solve steps).  Each inner PCG reduces a column's residual by eta (never
// below what the outer tolerance needs), starting from opts.inner_tol and adapted per column to its
// observed outer reduction within the solve (so repeated solves are bitwise identical); an outer
// step that fails to halve some column's residual switches the inner operator to the FP64 one.
// Columns that meet the tolerance get a zero outer residual, so the inner PCG leaves them alone.
// The solution is left in h->vs; h->vt holds the outer residual.
std::vector<PcgResult> pcg_refined(bddc_handle_s* h, const double* g, double tol, int maxit, int nb) {
  constexpr int kMaxOuter = 40;
  cudaStream_t st = h->st;
  const int64_t n = h->lv[0].d.n_iface;
  double* xo = h->vs;
  double* ro = h->vt;
  std::vector<PcgResult> res(nb);
  ck(cudaMemsetAsync(xo, 0, sizeof(double) * std::max<int64_t>(n, 1) * nb, st), "memset");
  if (n == 0) {
    for (auto& r : res) r.converged = true;
    return res;
  }
  auto norms = [&](const double* v) {   // ||v_k|| of every column
    launch_dot(v, v, n, h->partial, kDotBlocks, h->scal, st, nb, 16);
    ck(cudaMemcpyAsync(h->h_scal, h->scal, sizeof(double) * 16 * nb, cudaMemcpyDeviceToHost, st), "d2h");
    ck(cudaStreamSynchronize(st), "sync");
    std::vector<double> out(nb);
    for (int k = 0; k < nb; ++k) out[k] = std::sqrt(h->h_scal[16 * k]);
    return out;
  };
  ck(cudaMemcpyAsync(ro, g, sizeof(double) * n * nb, cudaMemcpyDeviceToDevice, st), "copy");
  const std::vector<double> gnorm = norms(g);
  std::vector<char> done(nb, 0);
  int left = nb;
  for (int k = 0; k < nb; ++k) {
    if (!std::isfinite(gnorm[k])) fail(BDDC_ERR_NAN, "NaN in the condensed right-hand side");
    res[k].gnorm = gnorm[k];
    if (gnorm[k] == 0.0) {
      res[k].converged = true;
      done[k] = 1;
      --left;
    }
  }
  std::vector<double> rnorm = gnorm, eta(nb, h->opts.inner_tol > 0.0 ? std::min(h->opts.inner_tol, 0.5) : 1e-2),
                      tin(nb, 1.0);
  int inner = h->inner_steps;
  int its = 0;
  for (int outer = 0; outer < kMaxOuter && its < maxit && left > 0; ++outer) {
    for (int k = 0; k < nb; ++k) {
      if (done[k]) {
        ck(cudaMemsetAsync(ro + (int64_t)k * n, 0, sizeof(double) * n, st), "memset");
        tin[k] = 1.0;
      } else {
        tin[k] = std::max(eta[k], 0.5 * tol * gnorm[k] / rnorm[k]);
      }
    }
    h->cur_steps = inner;
    std::vector<PcgResult> in = pcg(h, ro, h->vx, tin, maxit - its, nb);
    h->cur_steps = h->refine_steps;
    int most = 0;
    for (int k = 0; k < nb; ++k) {
      if (done[k]) continue;
      res[k].iterations += in[k].iterations;
      res[k].outer = outer + 1;
      most = std::max(most, in[k].iterations);
      if (outer == 0) {
        res[k].alpha = in[k].alpha;
        res[k].beta = in[k].beta;
      }
    }
    its += most;
    launch_axpy_loc(xo, h->vx, 1.0, n * nb, st);
    schur_apply(h, xo, h->vq, st, nb);                        // r = g - S x with the FP64 operator
    ck(cudaMemcpyAsync(ro, g, sizeof(double) * n * nb, cudaMemcpyDeviceToDevice, st), "copy");
    launch_axpy_loc(ro, h->vq, -1.0, n * nb, st);
    const std::vector<double> rn = norms(ro);
    bool stagnated = false;
    for (int k = 0; k < nb; ++k) {
      if (done[k]) continue;
      if (!std::isfinite(rn[k])) fail(BDDC_ERR_NAN, "NaN in the outer refinement");
      res[k].rel = rn[k] / gnorm[k];
      if (res[k].rel <= tol) {
        res[k].converged = true;
        done[k] = 1;
        --left;
        continue;
      }
      // the outer reduction shows how accurate the inner operator is: ask the next inner solve for
      // about that much (solving further is lost at the restart), unless the inner solve itself
      // was the limit
      const double ratio = rn[k] / rnorm[k];
      if (ratio > 0.5)
        stagnated = true;                                   // stagnation: inner operator = FP64 one
      else if (ratio > 2.0 * tin[k])
        eta[k] = std::min(0.1, std::max(1e-4, ratio));
      else
        eta[k] = std::max(1e-4, 0.5 * eta[k]);
      rnorm[k] = rn[k];
    }
    if (stagnated) inner = h->refine_steps;
  }
  return res;
}

int solve_impl(bddc_handle_s* h, const double* rhs, double* x, int nrhs, double tol, bddc_stats* stats,
               bool with_lift) {
  if (!h->factored) fail(BDDC_ERR_INVALID, "handle has no numeric set-up");
  if (nrhs < 1) fail(BDDC_ERR_INVALID, "nrhs must be >= 1");
  if (!(tol > 0.0)) fail(BDDC_ERR_INVALID, "tol must be positive");
  cudaStream_t st = h->st;
  const double t0 = now_ms();
  ck(cudaMemsetAsync(h->d_status + 2, 0, sizeof(int), st), "status reset");   // timeout code of this call
  h->cur_steps = h->refine_steps;
  int maxits = 0, max_outer = 0;
  bool all_conv = true;
  double worst = 0.0;
  PcgResult first;
  const int kind = krylov_kind(h);
  // PCG solves the right-hand sides in blocks of up to kMaxBlock (one pass over the factors per
  // block and iteration); BiCGstab and flexible GMRES one at a time
  const bool blocked = kind == BDDC_KRYLOV_PCG;
  if (blocked && nrhs > 1) ensure_block(h, std::min(nrhs, kMaxBlock));
  const int bmax = blocked ? h->blk : 1;
  for (int k0 = 0; k0 < nrhs;) {
    const int nb = std::min(bmax, nrhs - k0);
    const double* f = rhs + (int64_t)k0 * h->n_free;
    double* u = x + (int64_t)k0 * h->n_free;
    if (with_lift && h->has_lift) {   // f - K_fd u_d
      ck(cudaMemcpyAsync(h->fcol, f, sizeof(double) * h->n_free * nb, cudaMemcpyDeviceToDevice, st), "copy");
      for (int k = 0; k < nb; ++k) launch_axpy_loc(h->fcol + (int64_t)k * h->n_free, h->d_lift, 1.0, h->n_free, st);
      f = h->fcol;
    }
    const bool refined = blocked && h->use_outer;
    std::vector<PcgResult> r;
    try {
      condensed_rhs(h, f, h->vg, st, nb);
      if (kind == BDDC_KRYLOV_BICGSTAB)
        r.push_back(bicgstab(h, h->vg, h->vx, tol, h->opts.maxit));
      else if (kind == BDDC_KRYLOV_FGMRES)
        r.push_back(fgmres(h, h->vg, h->vx, tol, h->opts.maxit));
      else if (refined)
        r = pcg_refined(h, h->vg, tol, h->opts.maxit, nb);
      else
        r = pcg(h, h->vg, h->vx, std::vector<double>(nb, tol), h->opts.maxit, nb);
    } catch (const Fail& e) {
      if (e.code != BDDC_ERR_TIMEOUT) throw_if_timeout(h);
      throw;
    }
    recover(h, f, refined ? h->vs : h->vx, u, st, nb);
    for (int k = 0; k < nb; ++k) {
      maxits = std::max(maxits, r[k].iterations);
      max_outer = std::max(max_outer, r[k].outer);
      all_conv = all_conv && r[k].converged;
      worst = std::max(worst, r[k].rel);
    }
    if (k0 == 0) first = r[0];
    k0 += nb;
  }
  check_status(h, 0);
  h->stats.iterations = maxits;
  h->stats.outer_iterations = max_outer;
  h->stats.converged = all_conv ? 1 : 0;
  h->stats.rel_residual = worst;
  h->stats.rhs_norm = first.gnorm;
  lanczos(first, &h->stats.lambda_min, &h->stats.lambda_max);
  h->stats.solve_ms = now_ms() - t0;
  h->stats.factor_bytes = h->arena.bytes;
  flush_profile(h);
  if (stats) *stats = h->stats;
  if (!all_conv) {
    g_err = "Krylov iteration cap reached";
    return BDDC_ERR_NOT_CONVERGED;
  }
  return BDDC_OK;
}

template <typename F>
int guarded(F&& fn) {
  try {
    g_err.clear();
    return fn();
  } catch (const Fail& f) {
    return f.code;
  } catch (const std::exception& e) {
    g_err = e.what();
    return BDDC_ERR_INVALID;
  }
}

}  // namespace

// ---- accessors used by noalloc.cu (read-only views of a set-up handle) --------------------
void set_last_error(const char* msg) { g_err = msg ? msg : ""; }

bool grad_view(bddc_handle_s* h, GradView* v) {
  if (!h || !h->factored || h->lv.empty()) return false;
  const Level& L = h->lv[0];
  v->n_elems = h->n_elems;
  v->n_full = h->n_full;
  v->n_free = h->n_free;
  v->ne = h->npe * h->ndof;
  v->ke = L.d.ke;
  v->slot_elem = L.slot_elem;
  v->coef = h->d_coef;
  v->conn = h->d_conn;
  v->ndof = h->ndof;
  v->free_of_full = h->d_free_of_full;
  v->dir_full = h->has_lift ? h->d_dir_full : nullptr;
  v->coef_linear = h->physics != BDDC_STOKES;
  v->stream = h->st;
  return true;
}

int adjoint_solve_into(bddc_handle_s* h, const double* dJdu, double* lam, int nrhs, double tol) {
  return guarded([&]() { return solve_impl(h, dJdu, lam, nrhs, tol, nullptr, false); });
}

}  // namespace bddc

// ====================================================================== C ABI
extern "C" {

void bddc_default_opts(bddc_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = BDDC_PREC_MIXED;
  o->weights = BDDC_WEIGHTS_STIFFNESS;
  o->all_corners = 0;
  o->maxit = 500;
  o->refine_steps = 0;
  o->flexible = -1;
  o->use_graph = 1;
  o->verbose = 0;
  o->profile = 0;
  o->tensor_cores = 1;
  o->autotune = 1;
  o->inner_operator = 0;
  o->retain_host_memory = 1;
}

int bddc_analyze(const bddc_mesh* mesh, const bddc_partition* part, unsigned constraints, const bddc_opts* opts,
                 bddc_handle* out) {
  return guarded([&]() {
    if (!out) fail(BDDC_ERR_INVALID, "null output handle");
    *out = nullptr;
    auto* h = new bddc_handle_s();
    if (opts) h->opts = *opts; else bddc_default_opts(&h->opts);
    h->constraints = constraints;
    h->analysis_only = true;
    try {
      analysis(h, mesh, part);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
    return BDDC_OK;
  });
}

int bddc_setup(const bddc_mesh* mesh, const bddc_partition* part, unsigned constraints, const bddc_opts* opts,
               void* stream, bddc_handle* out) {
  return guarded([&]() {
    if (!out) fail(BDDC_ERR_INVALID, "null output handle");
    *out = nullptr;
    auto* h = new bddc_handle_s();
    if (opts) h->opts = *opts; else bddc_default_opts(&h->opts);
    if (h->opts.maxit <= 0) h->opts.maxit = 500;
    h->constraints = constraints;
    h->st = (cudaStream_t)stream;
    h->arena.st = h->st;
    try {
      analysis(h, mesh, part, [h]() { early_device(h); });
      device_setup(h);
      numeric_setup(h);
    } catch (...) {
      h->arena.release();
      if (h->h_scal) cudaFreeHost(h->h_scal);
      delete h;
      throw;
    }
    *out = h;
    return BDDC_OK;
  });
}

int bddc_update_coef(bddc_handle h, const double* coef) {
  return guarded([&]() {
    if (!h || h->analysis_only || !coef) fail(BDDC_ERR_INVALID, "bad handle or coefficients");
    for (int64_t e = 0; e < h->n_elems; ++e)
      if (!(coef[e] > 0.0)) fail(BDDC_ERR_INVALID, "coefficient must be positive");
    h->coef.assign(coef, coef + h->n_elems);
    h->factored = false;
    numeric_setup(h);
    return BDDC_OK;
  });
}

int bddc_solve(bddc_handle h, const double* rhs, double* x, int nrhs, double tol, bddc_stats* stats) {
  return guarded([&]() {
    if (!h || h->analysis_only || !rhs || !x) fail(BDDC_ERR_INVALID, "bad handle or vectors");
    return solve_impl(h, rhs, x, nrhs, tol, stats, true);
  });
}

int bddc_solve_host(bddc_handle h, const double* rhs_host, double* x_host, int nrhs, double tol, bddc_stats* stats) {
  return guarded([&]() {
    if (!h || h->analysis_only || !rhs_host || !x_host) fail(BDDC_ERR_INVALID, "bad handle or vectors");
    const size_t bytes = sizeof(double) * (size_t)h->n_free * (size_t)nrhs;
    double *dr = nullptr, *dx = nullptr;
    ck(cudaMallocAsync(&dr, bytes, h->st), "cudaMallocAsync");
    ck(cudaMallocAsync(&dx, bytes, h->st), "cudaMallocAsync");
    int rc;
    try {
      ck(cudaMemcpyAsync(dr, rhs_host, bytes, cudaMemcpyHostToDevice, h->st), "h2d");
      rc = solve_impl(h, dr, dx, nrhs, tol, stats, true);
      ck(cudaMemcpyAsync(x_host, dx, bytes, cudaMemcpyDeviceToHost, h->st), "d2h");
      ck(cudaStreamSynchronize(h->st), "sync");
    } catch (...) {
      cudaFreeAsync(dr, h->st);
      cudaFreeAsync(dx, h->st);
      throw;
    }
    cudaFreeAsync(dr, h->st);
    cudaFreeAsync(dx, h->st);
    return rc;
  });
}

int bddc_apply_precond(bddc_handle h, const double* r, double* z, int nrhs) {
  return guarded([&]() {
    if (!h || !h->factored || !r || !z || nrhs < 1) fail(BDDC_ERR_INVALID, "bad arguments");
    const int64_t n = h->lv[0].d.n_iface;
    if (nrhs > 1) ensure_block(h, std::min(nrhs, kMaxBlock));
    for (int k0 = 0; k0 < nrhs; k0 += h->blk)
      precond(h, r + k0 * n, z + k0 * n, h->st, std::min(h->blk, nrhs - k0));
    ck(cudaStreamSynchronize(h->st), "sync");
    return BDDC_OK;
  });
}

int bddc_apply_schur(bddc_handle h, const double* x, double* y, int nrhs) {
  return guarded([&]() {
    if (!h || !h->factored || !x || !y || nrhs < 1) fail(BDDC_ERR_INVALID, "bad arguments");
    const int64_t n = h->lv[0].d.n_iface;
    if (nrhs > 1) ensure_block(h, std::min(nrhs, kMaxBlock));
    for (int k0 = 0; k0 < nrhs; k0 += h->blk)
      schur_apply(h, x + k0 * n, y + k0 * n, h->st, std::min(h->blk, nrhs - k0));
    ck(cudaStreamSynchronize(h->st), "sync");
    return BDDC_OK;
  });
}

int bddc_apply_inner_schur(bddc_handle h, const double* x, double* y, int nrhs) {
  return guarded([&]() {
    if (!h || !h->factored || !x || !y || nrhs < 1) fail(BDDC_ERR_INVALID, "bad arguments");
    if (!h->lv[0].fp32 || krylov_kind(h) != BDDC_KRYLOV_PCG)
      fail(BDDC_ERR_INVALID, "the inner operator exists for mixed-precision PCG handles only");
    const int64_t n = h->lv[0].d.n_iface;
    if (nrhs > 1) ensure_block(h, std::min(nrhs, kMaxBlock));
    const int saved = h->cur_steps;
    h->cur_steps = 0;   // schur_apply's inner form
    for (int k0 = 0; k0 < nrhs; k0 += h->blk)
      schur_apply(h, x + k0 * n, y + k0 * n, h->st, std::min(h->blk, nrhs - k0));
    h->cur_steps = saved;
    ck(cudaStreamSynchronize(h->st), "sync");
    return BDDC_OK;
  });
}

int bddc_grad(bddc_handle h, const double* dJdu, const double* u, int nrhs, double tol, double* grad_coef,
              double* grad_rhs) {
  return guarded([&]() {
    if (!h || !h->factored || !dJdu || !u || nrhs < 1) fail(BDDC_ERR_INVALID, "bad arguments");
    if (grad_coef && h->physics == BDDC_STOKES)
      fail(BDDC_ERR_INVALID, "the coefficient gradient needs element matrices linear in the coefficient "
                             "(Poisson, elasticity); the viscosity scales only the viscous block");
    cudaStream_t st = h->st;
    const size_t bytes = sizeof(double) * (size_t)h->n_free * nrhs;
    double* lam = grad_rhs;
    double* own = nullptr;
    if (!lam) {
      ck(cudaMallocAsync(&own, bytes, st), "cudaMallocAsync");
      lam = own;
    }
    int rc;
    try {
      rc = solve_impl(h, dJdu, lam, nrhs, tol, nullptr, false);   // K lambda = dJ/du (K symmetric)
      if (grad_coef && (rc == BDDC_OK || rc == BDDC_ERR_NOT_CONVERGED)) {
        double *lf = nullptr, *uf = nullptr;
        const size_t fb = sizeof(double) * (size_t)h->n_full * nrhs;
        ck(cudaMallocAsync(&lf, fb, st), "cudaMallocAsync");
        ck(cudaMallocAsync(&uf, fb, st), "cudaMallocAsync");
        launch_expand_free(lam, h->d_free_of_full, h->n_full, nrhs, h->n_free, lf, st);
        launch_expand_free(u, h->d_free_of_full, h->n_full, nrhs, h->n_free, uf, st);
        if (h->has_lift)   // prescribed values enter K_e u_e
          for (int k = 0; k < nrhs; ++k) launch_axpy_loc(uf + (int64_t)k * h->n_full, h->d_dir_full, 1.0, h->n_full, st);
        const Level& L = h->lv[0];
        launch_grad_contract_slots(h->n_elems, h->npe * h->ndof, L.d.ke, L.slot_elem, h->d_coef, h->d_conn, h->ndof,
                                   lf, uf, nrhs, h->n_full, grad_coef, st);
        cudaFreeAsync(lf, st);
        cudaFreeAsync(uf, st);
      }
      ck(cudaStreamSynchronize(st), "sync");
    } catch (...) {
      if (own) cudaFreeAsync(own, st);
      throw;
    }
    if (own) cudaFreeAsync(own, st);
    return rc;
  });
}

int bddc_get_maps(bddc_handle h, int level, bddc_level_maps* out) {
  return guarded([&]() {
    if (!h || !out || level < 1 || level >= (int)h->lv.size()) fail(BDDC_ERR_INVALID, "bad level");
    const Level& L = h->lv[level - 1];
    const LevelMaps& m = L.maps;
    out->n_dof = L.mesh.n_dof;
    out->n_sub = m.n_sub();
    out->n_iface = m.n_iface;
    out->n_coarse = m.n_coarse;
    out->n_globs = m.n_globs();
    out->n_promoted = m.n_promoted;
    out->iface_dofs = m.iface_dofs.data();
    out->sub_dof_ptr = m.sub_dof_ptr.data();
    out->sub_dofs = m.sub_dofs.data();
    out->sub_nI = m.sub_nI.data();
    out->sub_iface = m.sub_iface.data();
    out->sub_wmult = m.sub_wmult.data();
    out->sub_coarse_ptr = m.sub_coarse_ptr.data();
    out->sub_coarse = m.sub_coarse.data();
    out->c_ptr = m.c_ptr.data();
    out->c_col = m.c_col.data();
    out->c_val = m.c_val.data();
    out->glob_ptr = m.glob_ptr.data();
    out->glob_nodes = m.glob_nodes.data();
    out->glob_kind = m.glob_kind.data();
    out->glob_promoted = m.glob_promoted.data();
    out->coarse_glob = m.coarse_glob.data();
    out->coarse_comp = m.coarse_comp.data();
    return BDDC_OK;
  });
}

int bddc_get_coarse(bddc_handle h, int level, double* kc, int64_t n) {
  return guarded([&]() {
    if (!h || !h->factored || !kc || level < 1 || level >= (int)h->lv.size())
      fail(BDDC_ERR_INVALID, "bddc_get_coarse: needs a set-up handle, a BDDC level and a buffer");
    const Level& L = h->lv[level - 1];
    if (n < L.g_elems)
      fail(BDDC_ERR_INVALID, "bddc_get_coarse: buffer of " + std::to_string(n) + " entries, needs " +
                                 std::to_string(L.g_elems));
    if (L.g_elems > 0)
      ck(cudaMemcpyAsync(kc, L.d.KC, sizeof(double) * (size_t)L.g_elems, cudaMemcpyDeviceToHost, h->st), "d2h");
    ck(cudaStreamSynchronize(h->st), "sync");
    return BDDC_OK;
  });
}

int bddc_tc_update_check(int64_t n, int rank, float* a, double* ms) {
  return guarded([&]() {
    if (rank != 256 && rank != 512) fail(BDDC_ERR_INVALID, "bddc_tc_update_check: rank must be 256 or 512");
    const int nt = rank / NB;
    if (!a || n < (int64_t)(nt + 1) * NB || n % NB != 0 || n > 64 * 1024)
      fail(BDDC_ERR_INVALID, "bddc_tc_update_check: n must be a multiple of 64 in [rank + 64, 65536]");
    const int nb = (int)(n / NB);
    cudaStream_t st = nullptr;
    DevArena A;
    A.st = st;
    try {
      // one subdomain whose nb x nb block matrix is all "interior": tile (i, j), j <= i, holds a's block
      SubMeta m{};
      m.n = m.nI = (int32_t)n;
      m.nIb = m.Bc = m.R = nb;
      const int64_t tile_elems = (int64_t)nb * (nb + 1) / 2 * NB2;
      std::vector<float> tiles((size_t)tile_elems);
      for (int i = 0; i < nb; ++i)
        for (int j = 0; j <= i; ++j) {
          float* t = tiles.data() + ((int64_t)i * (i + 1) / 2 + j) * NB2;
          for (int r = 0; r < NB; ++r)
            std::memcpy(t + r * NB, a + ((int64_t)i * NB + r) * n + (int64_t)j * NB, sizeof(float) * NB);
        }
      LevelDev d{};
      d.n_sub = 1;
      d.n_vec = n;
      std::vector<SubMeta> meta{m};
      d.meta = A.upload(meta, st);
      d.tiles = A.upload(tiles, st);
      d.sgn = A.upload(std::vector<float>((size_t)n, 1.f), st);
      d.status = A.upload(std::vector<int>{0, 0x7fffffff, 0, 0}, st);
      const int64_t* prow_off = A.upload(std::vector<int64_t>{0}, st);
      uint8_t* split = A.alloc<uint8_t>((int64_t)nb * kPanel * 2 * NB2 * 2);
      float* rscale = A.alloc<float>((int64_t)nb * NB);
      int64_t items = 0;
      for (int j = nt; j < nb; j += 2) items += (nb - j + 1) / 2;
      const int64_t* item_pref = A.upload(std::vector<int64_t>{0, items}, st);
      TensorMap128 tmap{};
      const int r = make_tile_tmap(&tmap, (float*)d.tiles, tile_elems);
      if (r) fail(BDDC_ERR_CUDA, "cuTensorMapEncodeTiled failed (error " + std::to_string(r) + ")");
      int dev = 0, sms = 0;
      ck(cudaGetDevice(&dev), "cudaGetDevice");
      ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
      cudaEvent_t e0, e1;
      ck(cudaEventCreate(&e0), "cudaEventCreate");
      ck(cudaEventCreate(&e1), "cudaEventCreate");
      launch_split_panel(d, 0, nt, nt, nb, split, nullptr, rscale, prow_off, st);
      ck(cudaEventRecord(e0, st), "cudaEventRecord");
      launch_update_tc2(d, nt, nt, nb, 0, 0, (int)std::min<int64_t>(items, std::max(1, sms)), split, split, rscale,
                        prow_off, item_pref, tmap, st);
      ck(cudaEventRecord(e1, st), "cudaEventRecord");
      ck(cudaGetLastError(), "tensor-core update launch");
      ck(cudaEventSynchronize(e1), "cudaEventSynchronize");
      float t = 0.f;
      ck(cudaEventElapsedTime(&t, e0, e1), "cudaEventElapsedTime");
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (ms) *ms = t;
      int status[4];
      ck(cudaMemcpy(status, d.status, sizeof(status), cudaMemcpyDeviceToHost), "d2h");
      if (status[2]) fail(BDDC_ERR_TIMEOUT, "a bounded wait of the tensor-core update gave up");
      ck(cudaMemcpy(tiles.data(), d.tiles, sizeof(float) * (size_t)tile_elems, cudaMemcpyDeviceToHost), "d2h");
      for (int i = nt; i < nb; ++i)
        for (int j = nt; j <= i; ++j) {
          const float* t2 = tiles.data() + ((int64_t)i * (i + 1) / 2 + j) * NB2;
          for (int r2 = 0; r2 < NB; ++r2)
            std::memcpy(a + ((int64_t)i * NB + r2) * n + (int64_t)j * NB, t2 + r2 * NB, sizeof(float) * NB);
        }
    } catch (...) {
      A.release();
      throw;
    }
    A.release();
    return BDDC_OK;
  });
}

int bddc_get_stats(bddc_handle h, bddc_stats* out) {
  return guarded([&]() {
    if (!h || !out) fail(BDDC_ERR_INVALID, "bad arguments");
    flush_profile(h);
    *out = h->stats;
    return BDDC_OK;
  });
}

int bddc_batching_ablation(bddc_handle h, double* ms) {
  return guarded([&]() {
    if (!h || !ms || !h->factored || h->lv.empty() || !h->lv[0].fp32 || h->physics == BDDC_STOKES)
      fail(BDDC_ERR_INVALID, "the ablation needs a set-up mixed-precision SPD handle");
    Level& L = h->lv[0];
    cudaStream_t st = h->st;
    const int saved_profile = h->opts.profile;
    h->opts.profile = 0;
    cudaEvent_t a, b;
    ck(cudaEventCreate(&a), "cudaEventCreate");
    ck(cudaEventCreate(&b), "cudaEventCreate");
    auto elapsed = [&]() {
      ck(cudaEventSynchronize(b), "cudaEventSynchronize");
      float t = 0.f;
      ck(cudaEventElapsedTime(&t, a, b), "cudaEventElapsedTime");
      return (double)t;
    };
    float* v = (float*)L.locA;
    ck(cudaMemsetAsync(v, 0, sizeof(float) * (size_t)L.n_vec, st), "memset");
    // (1) interior sweep pair: one launch per direction vs one per subdomain and direction
    const int grid = h->grid_max / 2 * L.sweep_ctas[0];
    trsv_pair<float>(h, L, v, 0, st);
    ck(cudaEventRecord(a, st), "cudaEventRecord");
    trsv_pair<float>(h, L, v, 0, st);
    ck(cudaEventRecord(b, st), "cudaEventRecord");
    ms[0] = elapsed();
    ck(cudaEventRecord(a, st), "cudaEventRecord");
    for (int dir = 0; dir < 2; ++dir)
      for (int64_t s = 0; s < (int64_t)L.meta.size(); ++s) {
        const int o0 = L.task_sub_off[dir][s], o1 = L.task_sub_off[dir][s + 1];
        launch_sweep<float>(L.d, v, L.tasks_by_sub[dir] + o0, o1 - o0, 0, dir, L.ctrl, L.pub, grid,
                            L.sweep_deep[0], st);
      }
    ck(cudaEventRecord(b, st), "cudaEventRecord");
    ms[1] = elapsed();
    // (2) CUDA-core tiled factorisation of level 1 (every step: diagonal tile, panel, trailing
    // update): batched over all subdomains vs launched per subdomain; both start from the
    // assembled tiles
    auto assemble_tiles = [&]() {
      ck(cudaMemsetAsync(L.d.tiles, 0, sizeof(float) * (size_t)std::max<int64_t>(L.tile_elems, 1), st), "memset");
      launch_densify_rows<float>(L.d, L.row_sub, st);
      launch_add_constraints<float>(L.d, st);
    };
    assemble_tiles();
    ck(cudaEventRecord(a, st), "cudaEventRecord");
    for (int k = 0; k < L.max_Bc; ++k) launch_potrf_step<float>(L.d, k, L.max_R, L.max_tiles[k], 1 << 30, st);
    ck(cudaEventRecord(b, st), "cudaEventRecord");
    ms[2] = elapsed();
    assemble_tiles();
    ck(cudaEventRecord(a, st), "cudaEventRecord");
    for (int64_t s = 0; s < (int64_t)L.meta.size(); ++s) {
      LevelDev one = L.d;
      one.meta = L.d.meta + s;
      one.n_sub = 1;
      const SubMeta& m = L.meta[s];
      for (int k = 0; k < m.Bc; ++k) {
        int64_t cnt = 0;
        for (int j = k + 1; j < m.Bc; ++j) cnt += m.R - j;
        launch_potrf_step<float>(one, k, m.R, (int)cnt, 1 << 30, st);
      }
    }
    ck(cudaEventRecord(b, st), "cudaEventRecord");
    ms[3] = elapsed();
    // restore the level-1 factors of the handle's own path (deterministic: bit-identical)
    reset_status(h);
    factor_level<float>(h, L, st);
    check_status(h, 1);
    h->opts.profile = saved_profile;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ck(cudaStreamSynchronize(st), "sync");
    return BDDC_OK;
  });
}

int bddc_reset_profile(bddc_handle h) {
  return guarded([&]() {
    if (!h) fail(BDDC_ERR_INVALID, "null handle");
    flush_profile(h);
    for (int c = 0; c < BDDC_PROF_CLASSES; ++c) {
      h->stats.prof_ms[c] = 0.0;
      h->stats.prof_launches[c] = 0;
      h->stats.prof_bytes[c] = 0.0;
      h->stats.prof_flops[c] = 0.0;
    }
    return BDDC_OK;
  });
}

int64_t bddc_kernel_launches(void) { return g_launches.load(); }

int bddc_sizes(bddc_handle h, int64_t* n_free, int64_t* n_iface) {
  return guarded([&]() {
    if (!h) fail(BDDC_ERR_INVALID, "null handle");
    if (n_free) *n_free = h->n_free;
    if (n_iface) *n_iface = h->lv.empty() ? 0 : h->lv[0].maps.n_iface;
    return BDDC_OK;
  });
}

void bddc_free(bddc_handle h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  h->arena.release();
  if (h->h_scal) cudaFreeHost(h->h_scal);
  delete h;
}

const char* bddc_last_error(void) { return g_err.c_str(); }

}  // extern "C"
