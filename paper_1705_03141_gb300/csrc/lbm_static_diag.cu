// Allocation-free variant of the diagnostics reduction (lbm_diag_fields_static).
//
// Some callers cannot allocate device memory at all: code that runs inside a
// host framework owning every device allocation through its own pool, real-time
// loops where any cudaMalloc (and the implicit synchronisation it brings) is
// forbidden, or callers that only hold device pointers handed to them.  For
// them this entry point reduces caller-owned rho_r / rho_b fields to the same
// four diagnostics as lbm_diag without allocating anything: its only scratch,
// the per-block partial sums, lives in the file-scope array below, which every
// GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"

namespace {

// Scratch of the allocation-free reduction: one row of lbmk::DIAG_VALS doubles
// per thread block of the partial pass plus one row for the final values.
// 65536 blocks of 256 nodes each: boxes of up to 16,777,216 nodes (3.7 MB).
constexpr int kStaticBlocks = 65536;
constexpr long long kStaticMaxNodes = (long long)kStaticBlocks * lbmk::DIAG_THREADS;
static __device__ __align__(256) double g_diag_scratch[(kStaticBlocks + 1) * lbmk::DIAG_VALS];

// Final pass: combines the partials in a fixed order (one warp per value) and
// writes mass_r, mass_b, z_leading_edge and dp_laplace to out[0..3].
__global__ void k_diag_final_static(int nblocks, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double v[lbmk::DIAG_VALS];
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k < lbmk::DIAG_VALS) {
    double a = k == 6 ? -1.0 : 0.0;
    for (int b = lane; b < nblocks; b += 32) {
      const double p = partial[(long long)b * lbmk::DIAG_VALS + k];
      a = k == 6 ? fmax(a, p) : a + p;
    }
    a = k == 6 ? lbmk::warp_max(a) : lbmk::warp_sum(a);
    if (lane == 0) v[k] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = v[0];
    out[1] = v[1];
    out[2] = v[6];
    out[3] = (v[3] > 0 && v[5] > 0) ? v[2] / v[3] - v[4] / v[5] : 0.0;
  }
}

// Device address of g_diag_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

lbm_status scratch_for_current_device(double** out, const char** why) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    *why = "no usable current CUDA device";
    return LBM_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_diag_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      *why = "cudaGetSymbolAddress of the static scratch failed";
      return LBM_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return LBM_OK;
}

// device memory of the current device, or managed memory (reachable from every device)
bool on_device(const void* ptr, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// host memory the runtime knows (pinned, registered) or plain pageable memory
bool on_host(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

}  // namespace

extern "C" lbm_status lbm_diag_fields_static(const double* rhoR, const double* rhoB, int nx, int ny, int nz,
                                              double rho_r0, double rho_b0, double* out, void* cuda_stream,
                                              const char** err) {
  const char* dummy = nullptr;
  const char** why = err ? err : &dummy;
  *why = "";
  if (!rhoR || !rhoB || !out) {
    *why = "rhoR, rhoB and out must not be NULL";
    return LBM_EINVAL;
  }
  if (nx < 1 || ny < 1 || nz < 1) {
    *why = "box dimensions must be >= 1";
    return LBM_EINVAL;
  }
  const long long N = (long long)nx * ny * nz;
  if (N > kStaticMaxNodes) {
    *why = "box too large for the static scratch: at most 16777216 nodes (65536 blocks of 256)";
    return LBM_EINVAL;
  }
  if (!(rho_r0 > 0) || !(rho_b0 > 0)) {
    *why = "rho_r0 and rho_b0 must be > 0";
    return LBM_EINVAL;
  }
  const double alpha_b = 8.0 / 27.0;
  const double alpha_r = 1.0 - (1.0 - alpha_b) / (rho_r0 / rho_b0);  // gamma = (1-alpha_b)/(1-alpha_r)
  if (!(alpha_r >= 0.0 && alpha_r < 1.0)) {  // the range lbm_create accepts
    *why = "density ratio rho_r0/rho_b0 must be >= 19/27 (alpha_r in [0,1))";
    return LBM_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    *why = "no usable current CUDA device";
    return LBM_ECUDA;
  }
  if (!on_device(rhoR, dev) || !on_device(rhoB, dev)) {
    *why = "rhoR and rhoB must be device memory of the current device";
    return LBM_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const bool out_dev = !on_host(out);
  if (out_dev && !on_device(out, dev)) {
    *why = "out must be host memory or device memory of the current device";
    return LBM_EINVAL;
  }
  if (!out_dev) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
      cudaGetLastError();
      *why = "cudaStreamIsCapturing failed on cuda_stream";
      return LBM_ECUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) {
      *why = "out must be device memory while cuda_stream is being captured (a host result needs a synchronisation)";
      return LBM_EINVAL;
    }
  }
  double* scratch = nullptr;
  lbm_status st = scratch_for_current_device(&scratch, why);
  if (st != LBM_OK) return st;

  lbmk::Geom G;
  G.nx = nx;
  G.nxs = nx;  // the diagnostics read plain fields only
  G.ny = ny;
  G.nz = nz;
  G.Ns = 0;
  for (int f = 0; f < 6; ++f) G.bc[f] = 0;
  G.inflow = 0;
  G.xc = G.yc = G.r2 = 0.0;
  const int nblocks = (int)((N + lbmk::DIAG_THREADS - 1) / lbmk::DIAG_THREADS);
  double* partial = scratch;
  double* result = scratch + (long long)kStaticBlocks * lbmk::DIAG_VALS;

  lbmk::k_diag_partial<<<nblocks, lbmk::DIAG_THREADS, 0, s>>>(G, alpha_r, alpha_b, rhoR, rhoB, partial);
  k_diag_final_static<<<1, 32 * lbmk::DIAG_VALS, 0, s>>>(nblocks, partial, out_dev ? out : result);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !out_dev) {
    e = cudaMemcpyAsync(out, result, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return LBM_ECUDA;
  }
  return LBM_OK;
}
