// Compact 16-bit storage (half or bfloat16 totals + one colour record per node), FP32 arithmetic.
#include "lbm_compact.cuh"
#include "lbm_launch.cuh"
#include "../../include/lbm.h"

namespace lbmk {

// tensor maps of the pipelined compact pass 1: the totals as (word, plane, block, y, z + 1) and
// the records as (4 x, y, z + 1) floats, over the whole storage including the ghost planes
template <bool B>
static bool density_maps(const CompactStore<B>& st, const Geom& G, DcMaps& M) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const cuuint64_t XC = (cuuint64_t)G.nxs / 32, ny = (cuuint64_t)G.ny, nzg = (cuuint64_t)G.nz + 2;
  const cuuint64_t td[5] = {32, (cuuint64_t)CPLANES, XC, ny, nzg};
  const cuuint64_t ts[4] = {64, 64 * (cuuint64_t)CPLANES, 64 * (cuuint64_t)CPLANES * XC,
                            64 * (cuuint64_t)CPLANES * XC * ny};
  const cuuint32_t brest[5] = {32, 1, 1, BY, BZ};
  // the same totals as 8-byte words (224 per 32-node block of 28 planes): long rows for the boxes
  const cuuint64_t wd[4] = {8 * (cuuint64_t)CPLANES, XC, ny, nzg};
  const cuuint64_t ws[3] = {64 * (cuuint64_t)CPLANES, 64 * (cuuint64_t)CPLANES * XC, 64 * (cuuint64_t)CPLANES * XC * ny};
  const cuuint32_t bgrp[4] = {72, 1, BY + 2, BZ}, beven[4] = {8 * (cuuint32_t)CPLANES, 1, BY, BZ};
  const cuuint64_t rd[3] = {4 * (cuuint64_t)G.nxs, ny, nzg};
  const cuuint64_t rs[2] = {16 * (cuuint64_t)G.nxs, 16 * (cuuint64_t)G.nxs * ny};
  const cuuint32_t brec[3] = {4 * TX, TY, TZ};
  return encode(enc, &M.rest, CU_TENSOR_MAP_DATA_TYPE_UINT16, 5, st.A, td, ts, brest) &&
         encode(enc, &M.grp, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, st.A, wd, ws, bgrp) &&
         encode(enc, &M.even, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, st.A, wd, ws, beven) &&
         encode(enc, &M.rec, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, st.rec, rd, rs, brec);
}

static int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return n;
}

template <bool B>
struct LaunchCompact {
  using Store = CompactStore<B>;
  static Store make(void* p, const Geom& G) {
    // population blocks first (56 bytes per storage node), then the records (16 bytes per node)
    return Store{static_cast<uint16_t*>(p), reinterpret_cast<float4*>(static_cast<char*>(p) + (size_t)56 * G.Ns),
                 G.Ns};
  }
  static KConst<float> kc(const Phys& P) { return make_kconst<float>(P); }
  // pass 1: shape 3 the TMA pipeline (k_density_ct; x faces that reflect and at least 3 tiles along
  // y and z, checked at creation), otherwise one block per 32x4x2 tile
  static cudaError_t density(void* pop, const Geom& G, const Phys& P, int layout, void* dens, int* flag, void*,
                             int shape, cudaStream_t s) {
    const Store st = make(pop, G);
    if (shape != 3) {
      k_density_c<B><<<grid3(G), dim3(BX, BY, BZ), 0, s>>>(st, G, kc(P), layout, static_cast<float2*>(dens), flag);
      return cudaGetLastError();
    }
    DcMaps M;
    if (!density_maps(st, G, M)) return cudaErrorNotSupported;
    using K0 = decltype(&k_density_ct<B, 0, DC_NG, DC_S, DC_MINB>);
    const K0 kern[2] = {&k_density_ct<B, 0, DC_NG, DC_S, DC_MINB>, &k_density_ct<B, 1, DC_NG, DC_S, DC_MINB>};
    static const bool attr =
        cudaFuncSetAttribute(kern[0], cudaFuncAttributeMaxDynamicSharedMemorySize, DC_SMEM) == cudaSuccess &&
        cudaFuncSetAttribute(kern[1], cudaFuncAttributeMaxDynamicSharedMemorySize, DC_SMEM) == cudaSuccess;
    if (!attr) return cudaErrorInvalidValue;
    const int ntx = (G.nx + BX - 1) / BX, nty = (G.ny + BY - 1) / BY, ntz = (G.nz + BZ - 1) / BZ;
    const int ntiles = ntx * nty * ntz;
    static const int nsm = sm_count();
    const int per = DC_MINB * DC_NG;  // tiles a wave of blocks computes at once
    const int grid = nsm > 0 && ntiles > per * nsm ? DC_MINB * nsm : (ntiles + DC_NG - 1) / DC_NG;
    kern[layout ? 1 : 0]<<<grid, DC_THREADS, DC_SMEM, s>>>(st, G, kc(P), M, static_cast<float2*>(dens), flag, ntx,
                                                          nty, ntiles);
    return cudaGetLastError();
  }
  static cudaError_t collide(void* pop, const Geom& G, const Phys& P, int odd, const void* dens, long long* counter,
                             int, const void*, void*, int*, int, cudaStream_t s) {
    k_collide_stream_c<B><<<grid3(G), dim3(BX, BY, BZ), 0, s>>>(make(pop, G), G, kc(P), odd,
                                                                 static_cast<const float2*>(dens), counter);
    return cudaGetLastError();
  }
  static cudaError_t outflow(void* pop, const Geom& G, const Phys& P, int layout, void*, void*, cudaStream_t s) {
    const int64_t warps = (int64_t)G.nx * G.ny;
    k_outflow_c<B><<<blocks1(warps * 32, 256), 256, 0, s>>>(make(pop, G), G, kc(P), layout);
    return cudaGetLastError();
  }
  static cudaError_t get_pop(void* pop, const Geom& G, const Phys& P, int layout, int pdir, double* out_r,
                             double* out_b, cudaStream_t s) {
    const int64_t N = (int64_t)G.nx * G.ny * G.nz;
    k_get_pop_c<B><<<blocks1(N, 256), 256, 0, s>>>(make(pop, G), G, kc(P), layout, pdir, out_r, out_b);
    return cudaGetLastError();
  }
  static cudaError_t init_c(void* pop, const Geom& G, const Phys& P, const double* rr, const double* rb,
                            const double* u, void* dens, cudaStream_t s) {
    const int64_t N = (int64_t)G.nx * G.ny * G.nz;
    k_init_c<B><<<blocks1(N, 256), 256, 0, s>>>(make(pop, G), G, kc(P), rr, rb, u, static_cast<float2*>(dens));
    return cudaGetLastError();
  }
  static cudaError_t macro_c(void* pop, const Geom& G, const Phys& P, int layout, const void* dens, double* rr,
                             double* rb, double* u, cudaStream_t s) {
    const int64_t N = (int64_t)G.nx * G.ny * G.nz;
    k_macro_c<B><<<blocks1(N, 256), 256, 0, s>>>(make(pop, G), G, kc(P), layout, static_cast<const float2*>(dens), rr,
                                                 rb, u);
    return cudaGetLastError();
  }
  static cudaError_t set_pop_c(void* pop, const Geom& G, const Phys& P, int layout, int pdir, const double* in_r,
                               const double* in_b, double* acc_r, double* acc_b, cudaStream_t s) {
    const int64_t N = (int64_t)G.nx * G.ny * G.nz;
    k_set_pop_c<B><<<blocks1(N, 256), 256, 0, s>>>(make(pop, G), G, kc(P), layout, pdir, in_r, in_b, acc_r, acc_b);
    return cudaGetLastError();
  }
  static cudaError_t dens_from_acc(const Geom& G, const double* acc_r, const double* acc_b, void* dens,
                                   cudaStream_t s) {
    const int64_t N = (int64_t)G.nx * G.ny * G.nz;
    k_dens_from_acc<<<blocks1(N, 256), 256, 0, s>>>(G, acc_r, acc_b, static_cast<float2*>(dens));
    return cudaGetLastError();
  }
  static const KernelSet* table() {
    static const KernelSet ks = {2, 1, 56 + 16, sizeof(float2), sizeof(float), &density, &collide, &outflow,
                                 nullptr, &get_pop, nullptr, nullptr, nullptr, false, false, false, true,
                                 &init_c, &macro_c, &set_pop_c, &dens_from_acc};
    return &ks;
  }
};

const KernelSet* kernels_c16() { return LaunchCompact<false>::table(); }
const KernelSet* kernels_cbf16() { return LaunchCompact<true>::table(); }

// Self-test of the pipeline's primitives: one tiled TMA copy of a 16 x 16 box of a 32 x 32 FP32
// tensor (origin (8, 4)) completes on barrier a with its exact byte count, and barrier b, armed
// for 16 bytes that no copy delivers, makes the bounded wait run out.  No copy is in flight when
// the block leaves (the box has landed before the wait on b starts).
static __global__ void k_tma_selftest(const __grid_constant__ CUtensorMap map, const float* __restrict__ src,
                                      long long cycles, int* __restrict__ result) {
  __shared__ __align__(128) float box[16 * 16];
  __shared__ uint64_t a, b;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&a, 1);
    mbar_init(&b, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(&a, sizeof(box));
    tma_load_2d(box, &map, &a, 8, 4);
    mbar_arrive_expect_tx(&b, 16);
  }
  __syncthreads();
  const bool landed = mbar_wait(&a, 0, kWaitCycles);
  int ok = landed ? 1 : 0;
  if (landed)
    for (int i = tid; i < 16 * 16; i += blockDim.x) ok &= box[i] == src[(4 + i / 16) * 32 + 8 + i % 16] ? 1 : 0;
  if (!ok) atomicAnd(result, 0);
  if (landed && !mbar_wait(&b, 0, cycles)) atomicOr(result + 1, 1);
}

}  // namespace lbmk

extern "C" lbm_status lbm_selftest_tma(void* cuda_stream, long long wait_cycles, int* copy_ok, int* timed_out) {
  using namespace lbmk;
  if (!copy_ok || !timed_out || wait_cycles < 1 || wait_cycles > kWaitCycles) return LBM_EINVAL;
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) return LBM_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  float* src = nullptr;
  int* res = nullptr;
  if (cudaMalloc(&src, 32 * 32 * sizeof(float)) != cudaSuccess) return LBM_ENOMEM;
  if (cudaMalloc(&res, 2 * sizeof(int)) != cudaSuccess) {
    cudaFree(src);
    return LBM_ENOMEM;
  }
  float host[32 * 32];
  for (int i = 0; i < 32 * 32; ++i) host[i] = 0.25f * (float)i - 17.0f;
  const int init[2] = {1, 0};
  int out[2] = {0, 0};
  lbm_status st = LBM_OK;
  CUtensorMap map;
  const cuuint64_t dims[2] = {32, 32}, strides[1] = {32 * sizeof(float)};
  const cuuint32_t box[2] = {16, 16};
  if (cudaMemcpyAsync(src, host, sizeof(host), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(res, init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess)
    st = LBM_ECUDA;
  else if (!encode(enc, &map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, src, dims, strides, box))
    st = LBM_ECUDA;
  if (st == LBM_OK) {
    k_tma_selftest<<<1, 128, 0, s>>>(map, src, wait_cycles, res);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(out, res, sizeof(out), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = LBM_ECUDA;
  }
  cudaFree(src);
  cudaFree(res);
  *copy_ok = out[0];
  *timed_out = out[1];
  return st;
}
