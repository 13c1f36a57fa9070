// bddc_grad_noalloc: the adjoint gradient of bddc_grad without any device allocation.
//
// bddc_grad allocates, on every call, the full-DOF copies of the adjoint and of the solution
// that its element contraction kernel reads.  Some callers cannot let a library allocate:
// applications that hand (almost) all device memory to their own pool, where a cudaMalloc from
// the library fails or fragments that pool, and latency-critical loops, where cudaMalloc /
// cudaFree would stall (cudaFree synchronises the device).  For them this variant keeps that
// scratch in one fixed file-scope device array, kNoAllocScratchBytes (16 MiB) large, that every
// GPU which loads the library holds until the process exits.  Right-hand sides are contracted
// one at a time, so the limit is 2 * n_full * 8 bytes <= 16 MiB, i.e. n_full <= 1,048,576
// (n_full = nodes * DOFs per node, prescribed DOFs included); larger meshes are rejected with
// BDDC_ERR_INVALID.  The adjoint solve itself uses only the buffers the handle allocated at
// set-up, once the handle is warm: its first solve (and the first after a change of Krylov
// method) captures the CUDA graph of one iteration and creates that graph's stream and events.
// The call synchronises the handle's stream, so it cannot run inside a stream capture.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/bddc.h"
#include "internal.h"

namespace bddc {
void set_last_error(const char* msg);
bool grad_view(bddc_handle_s* h, GradView* v);
int adjoint_solve_into(bddc_handle_s* h, const double* dJdu, double* lam, int nrhs, double tol);
}  // namespace bddc

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
constexpr int64_t kScratchDoubles = (int64_t)(kNoAllocScratchBytes / sizeof(double));

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mtx;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once per device.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mtx);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// out_l / out_u: full-DOF copies (zero on prescribed DOFs) of one right-hand side
__global__ void k_expand_pair(const double* __restrict__ lam, const double* __restrict__ u,
                              const int64_t* __restrict__ free_of_full, const double* __restrict__ dir_full,
                              int64_t n_full, double* __restrict__ out_l, double* __restrict__ out_u) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_full) return;
  const int64_t f = free_of_full[j];
  out_l[j] = f >= 0 ? lam[f] : 0.0;
  out_u[j] = f >= 0 ? u[f] : (dir_full ? dir_full[j] : 0.0);   // prescribed values enter K_e u_e
}

// grad[e] += -(1/coef_e) lam_e^T K_e u_e for one right-hand side; one warp per element
__global__ void k_grad_contract_accum(int64_t n_elems, int ne, const double* __restrict__ ke,
                                      const int32_t* __restrict__ slot_elem, const double* __restrict__ coef,
                                      const int32_t* __restrict__ conn, int ndof, const double* __restrict__ lamf,
                                      const double* __restrict__ uf, double* __restrict__ grad) {
  const int64_t slot = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (slot >= n_elems) return;
  const int64_t e = slot_elem[slot];
  const double* K = ke + slot * (int64_t)ne * ne;
  const int32_t* cn = conn + e * (int64_t)(ne / ndof);
  auto dof = [&](int a) { return (int64_t)cn[a / ndof] * ndof + a % ndof; };
  double acc = 0.0;
  for (int a = lane; a < ne; a += 32) {
    double t = 0.0;
    for (int b = 0; b < ne; ++b) t += K[a * ne + b] * uf[dof(b)];
    acc += lamf[dof(a)] * t;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) grad[e] += -acc / coef[e];
}

}  // namespace

extern "C" int bddc_grad_noalloc(bddc_handle h, const double* dJdu, const double* u, int nrhs, double tol,
                                 double* grad_coef, double* grad_rhs) {
  using namespace bddc;
  GradView v{};
  if (!h || !dJdu || !u || !grad_rhs || nrhs < 1 || !grad_view(h, &v)) {
    set_last_error("bddc_grad_noalloc: needs a set-up handle, dJdu, u, nrhs >= 1 and a grad_rhs buffer");
    return BDDC_ERR_INVALID;
  }
  if (grad_coef && !v.coef_linear) {
    set_last_error("bddc_grad_noalloc: the coefficient gradient needs element matrices linear in the coefficient "
                   "(Poisson, elasticity)");
    return BDDC_ERR_INVALID;
  }
  if (2 * v.n_full > kScratchDoubles) {
    const std::string msg = "bddc_grad_noalloc: mesh too large for the fixed 16 MiB scratch (needs 2 x " +
                            std::to_string(v.n_full) + " doubles, at most n_full = " +
                            std::to_string(kScratchDoubles / 2) + "); use bddc_grad";
    set_last_error(msg.c_str());
    return BDDC_ERR_INVALID;
  }
  void* scratch = nullptr;
  cudaError_t ce = scratch_address(&scratch);
  if (ce != cudaSuccess) {
    const std::string msg = std::string("bddc_grad_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(ce);
    set_last_error(msg.c_str());
    return BDDC_ERR_CUDA;
  }
  // adjoint solve K lambda = dJ/du into the caller's grad_rhs (no allocation)
  const int rc = adjoint_solve_into(h, dJdu, grad_rhs, nrhs, tol);
  if (rc != BDDC_OK && rc != BDDC_ERR_NOT_CONVERGED) return rc;
  if (grad_coef) {
    double* lf = (double*)scratch;
    double* uf = lf + v.n_full;
    cudaStream_t st = v.stream;
    ce = cudaMemsetAsync(grad_coef, 0, sizeof(double) * (size_t)v.n_elems, st);
    for (int k = 0; k < nrhs && ce == cudaSuccess; ++k) {
      note_launch();
      k_expand_pair<<<(unsigned)((v.n_full + 255) / 256), 256, 0, st>>>(
          grad_rhs + (int64_t)k * v.n_free, u + (int64_t)k * v.n_free, v.free_of_full, v.dir_full, v.n_full, lf, uf);
      note_launch();
      k_grad_contract_accum<<<(unsigned)((v.n_elems + 7) / 8), 256, 0, st>>>(v.n_elems, v.ne, v.ke, v.slot_elem,
                                                                              v.coef, v.conn, v.ndof, lf, uf, grad_coef);
      ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
      const std::string msg = std::string("bddc_grad_noalloc: ") + cudaGetErrorString(ce);
      set_last_error(msg.c_str());
      return BDDC_ERR_CUDA;
    }
  }
  return rc;
}
