// Host-side table of kernel launchers for one storage type (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmk {
struct Geom;
struct Phys;

struct KernelSet {
  size_t pop_elem_bytes;  // bytes per stored value
  int pop_planes;         // stored planes per direction (2 plain, 1 packed)
  size_t pop_node_bytes;  // bytes of the population region per storage node (records included)
  size_t dens_bytes;      // bytes per node of the pass-1 field
  size_t real_bytes;      // bytes of the compute type (outflow plane history)
  // pass 1; with fix non-null it writes the fixed-point accumulators of the fused density pass
  // instead of dens (priming the fused pass from a stored state)
  // shape: block shape of the one-node kernels (0: 32x4x2, 1: 32x2x4, 2: 32x8x1; variants 1 and 3)
  cudaError_t (*density)(void* pop, const Geom& G, const Phys& P, int layout, void* dens, int* flag, void* fix,
                         int shape, cudaStream_t s);
  // pass 2.  variant: 1 = one node per thread, 2 = two nodes per thread (FP32 arithmetic, nx even),
  // 3 = one node per thread with the fused density pass (reads cur, accumulates into nxt, which
  // must be zero), 4 = software-pipelined one node per thread (packed storage), 5 = the interior
  // tiles by the TMA-pipelined kernel and the boundary tiles by variant 1 (packed storage; boxes
  // with periodic or no-slip x faces, odd nx or no interior tile run variant 1).  counter: the
  // two-entry step index of k_collide_stream.
  cudaError_t (*collide)(void* pop, const Geom& G, const Phys& P, int odd, const void* dens, long long* counter,
                         int variant, const void* cur, void* nxt, int* flag, int shape, cudaStream_t s);
  // convective outflow; with fix non-null it also rewrites the top plane's accumulators
  cudaError_t (*outflow)(void* pop, const Geom& G, const Phys& P, int layout, void* top, void* fix, cudaStream_t s);
  cudaError_t (*init)(void* pop, const Geom& G, const Phys& P, const double* rr, const double* rb, const double* u,
                      cudaStream_t s);
  cudaError_t (*get_pop)(void* pop, const Geom& G, const Phys& P, int layout, int pdir, double* out_r, double* out_b,
                         cudaStream_t s);
  cudaError_t (*set_pop)(void* pop, const Geom& G, const Phys& P, int layout, int pdir, const double* in_r,
                         const double* in_b, cudaStream_t s);
  cudaError_t (*top_from_state)(void* pop, const Geom& G, const Phys& P, int layout, void* top, cudaStream_t s);
  cudaError_t (*macro)(void* pop, const Geom& G, const Phys& P, int layout, double* rr, double* rb, double* u,
                       cudaStream_t s);
  bool has_paired;        // a two-nodes-per-thread pass 2 exists for this storage
  bool has_fused;         // a fused-density pass 2 exists for this storage (FP32 arithmetic)
  bool has_pipelined;     // a software-pipelined pass 2 exists for this storage (packed)
  // compact storage (per-node colour records): the state after lbm_init_fields / a population
  // upload has no records, so its first step takes the densities from dens instead of pass 1,
  // and the I/O kernels below replace init / macro / set_pop
  bool compact;
  cudaError_t (*init_c)(void* pop, const Geom& G, const Phys& P, const double* rr, const double* rb,
                        const double* u, void* dens, cudaStream_t s);
  cudaError_t (*macro_c)(void* pop, const Geom& G, const Phys& P, int layout, const void* dens, double* rr,
                         double* rb, double* u, cudaStream_t s);
  cudaError_t (*set_pop_c)(void* pop, const Geom& G, const Phys& P, int layout, int pdir, const double* in_r,
                           const double* in_b, double* acc_r, double* acc_b, cudaStream_t s);
  cudaError_t (*dens_from_acc)(const Geom& G, const double* acc_r, const double* acc_b, void* dens, cudaStream_t s);
  // pass 1 preceded, on the plane z = nz-1, by the convective outflow of the step before (top: the
  // outflow history), so that runs of steps launch the outflow kernel once at their end; null for
  // compact storage
  cudaError_t (*density_fold)(void* pop, const Geom& G, const Phys& P, int layout, void* dens, int* flag, void* top,
                              int shape, cudaStream_t s);
};

const KernelSet* kernels_f64();
const KernelSet* kernels_f32();
const KernelSet* kernels_f16();
const KernelSet* kernels_bf16();
const KernelSet* kernels_c16();
const KernelSet* kernels_cbf16();
}  // namespace lbmk
