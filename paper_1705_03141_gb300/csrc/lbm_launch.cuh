// Template launchers behind lbmk::KernelSet (internal).
#pragma once
#include <stdlib.h>
#include <string.h>

#include "lbm_dispatch.h"
#include "lbm_kernels.cuh"
#include "lbm_pipe.cuh"
#include "lbm_tma_host.h"

namespace lbmk {

template <class B = BlkDefault>
inline dim3 grid3(const Geom& G) {
  return dim3((unsigned)((G.nx + B::BX - 1) / B::BX), (unsigned)((G.ny + B::BY - 1) / B::BY),
              (unsigned)((G.nz + B::BZ - 1) / B::BZ));
}
inline unsigned blocks1(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <class Store>
struct StoreTraits;
// minb: resident 256-thread blocks per SM the one-node kernels are compiled for (4: 64 registers,
// 32 warps; measured faster than 3 once the red populations are summed as they load);
// minb2: the two-node kernel; minb_pf: the pipelined kernel (68 KB of shared memory per block)
template <>
struct StoreTraits<PlainStore<double>> {
  static constexpr bool paired = false;
  static constexpr int minb = 1, minb2 = 1, minb_pf = 1;
  static PlainStore<double> make(void* p, const Geom& G) { return {static_cast<double*>(p), G.Ns}; }
};
template <>
struct StoreTraits<PlainStore<float>> {
  static constexpr bool paired = true;
  static constexpr int minb = 4, minb2 = 2, minb_pf = 3;
  static PlainStore<float> make(void* p, const Geom& G) { return {static_cast<float*>(p), G.Ns}; }
};
template <bool B>
struct StoreTraits<PackedStore<B>> {
  static constexpr bool paired = true;
  static constexpr int minb = 4, minb2 = 2, minb_pf = 3;
  static PackedStore<B> make(void* p, const Geom& G) { return {static_cast<uint32_t*>(p), G.Ns}; }
};

template <class Store>
struct Launch {
  using Tr = StoreTraits<Store>;
  using DT = typename DensOf<Store>::type;
  using R = typename DensOf<Store>::real;
  static KConst<R> kc(const Phys& P) { return make_kconst<R>(P); }

  static constexpr bool fused = !std::is_same<R, double>::value;
  static constexpr bool pipelined = Store::PLANES == 27;  // packed storage

  template <class B>
  static cudaError_t density_b(void* pop, const Geom& G, const Phys& P, int layout, void* dens, int* flag, void* fix,
                               void* top, cudaStream_t s) {
    if constexpr (fused) {
      if (fix) {
        k_density<Store, true, B><<<grid3<B>(G), dim3(B::BX, B::BY, B::BZ), 0, s>>>(
            Tr::make(pop, G), G, kc(P), layout, static_cast<DT*>(dens), flag, static_cast<unsigned long long*>(fix),
            nullptr);
        return cudaGetLastError();
      }
    }
    k_density<Store, false, B><<<grid3<B>(G), dim3(B::BX, B::BY, B::BZ), 0, s>>>(
        Tr::make(pop, G), G, kc(P), layout, static_cast<DT*>(dens), flag, nullptr, static_cast<R*>(top));
    return cudaGetLastError();
  }
  static cudaError_t density_top(void* pop, const Geom& G, const Phys& P, int layout, void* dens, int* flag,
                                 void* fix, void* top, int shape, cudaStream_t s) {
    if constexpr (!std::is_same<R, double>::value) {  // FP64 keeps the default shape
      if (shape == 1) return density_b<Blk<2, 4>>(pop, G, P, layout, dens, flag, fix, top, s);
      if (shape == 2) return density_b<Blk<8, 1>>(pop, G, P, layout, dens, flag, fix, top, s);
    }
    return density_b<BlkDefault>(pop, G, P, layout, dens, flag, fix, top, s);
  }
  static cudaError_t density(void* pop, const Geom& G, const Phys& P, int layout, void* dens, int* flag, void* fix,
                             int shape, cudaStream_t s) {
    return density_top(pop, G, P, layout, dens, flag, fix, nullptr, shape, s);
  }
  // pass 1 of a step that first completes the step before with its convective outflow
  static cudaError_t density_fold(void* pop, const Geom& G, const Phys& P, int layout, void* dens, int* flag,
                                  void* top, int shape, cudaStream_t s) {
    return density_top(pop, G, P, layout, dens, flag, nullptr, top, shape, s);
  }
  // Tensor map of the pass-1 field for the TMA tile of k_collide_stream: 8-byte cells (rho, phi)
  // over (x, y, z + 1), planes z = -1 .. nz (dens points at plane 0, one plane above the start of
  // its buffer), box 36 x TY x TZ.  False where a TMA copy cannot be used: no driver entry point,
  // odd nx (row strides must be multiples of 16 bytes) or a misaligned buffer; also where the
  // environment variable LBM_NO_TMA is set when the launch is made (or captured into a graph):
  // the tiles are then loaded as for boxes that cross a periodic face, with the same values.
  template <class B>
  static bool dens_map(const Geom& G, const void* dens, CUtensorMap* m) {
    if (!std::is_same<DT, float2>::value || (G.nx & 1) || getenv("LBM_NO_TMA") != nullptr) return false;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    char* base = const_cast<char*>(static_cast<const char*>(dens)) - (size_t)G.nx * G.ny * sizeof(DT);
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)G.nx, (cuuint64_t)G.ny, (cuuint64_t)G.nz + 2};
    const cuuint64_t strides[2] = {(cuuint64_t)G.nx * sizeof(DT), (cuuint64_t)G.nx * G.ny * sizeof(DT)};
    const cuuint32_t box[3] = {(cuuint32_t)B::TXT, (cuuint32_t)B::TY, (cuuint32_t)B::TZ};
    return encode(enc, m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, base, dims, strides, box);
  }
  template <class B>
  static cudaError_t collide_b(void* pop, const Geom& G, const Phys& P, int odd, const void* dens, long long* counter,
                               bool fused_pass, const FusedIO& io, cudaStream_t s) {
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    if constexpr (fused) {
      if (fused_pass) {
        k_collide_stream<Store, Tr::minb, true, B><<<grid3<B>(G), dim3(B::BX, B::BY, B::BZ), 0, s>>>(
            Tr::make(pop, G), G, kc(P), odd, static_cast<const DT*>(dens), counter, io, map, 0, TileSplit{}, 0);
        return cudaGetLastError();
      }
    }
    const int tma = dens_map<B>(G, dens, &map) ? 1 : 0;
    k_collide_stream<Store, Tr::minb, false, B><<<grid3<B>(G), dim3(B::BX, B::BY, B::BZ), 0, s>>>(
        Tr::make(pop, G), G, kc(P), odd, static_cast<const DT*>(dens), counter, io, map, tma, TileSplit{}, 0);
    return cudaGetLastError();
  }
  // Variant 5 (packed storage): the boundary tiles by the one-node kernel, then the interior tiles
  // by the TMA-pipelined kernel (lbm_pipe.cuh).  cudaErrorNotSupported where it does not apply:
  // an x face that is periodic or bounces back (the mirror of the staged rows assumes a
  // reflecting face), odd nx, no interior tile, or a tensor map that cannot be encoded.
  static bool tp_applies(const Geom& G) { return pipelined_tiles(G); }
  static TileSplit tile_split(const Geom& G) { return default_tile_split(G); }
  static cudaError_t collide_tp(void* pop, const Geom& G, const Phys& P, int odd, const void* dens,
                                long long* counter, const FusedIO& io, cudaStream_t s) {
    if constexpr (pipelined) {
      if (!tp_applies(G)) return cudaErrorNotSupported;
      TpMaps M;
      memset(&M, 0, sizeof(M));
      if (!dens_map<BlkDefault>(G, dens, &M.dens)) return cudaErrorNotSupported;
      const EncodeTiledFn enc = encode_tiled();
      const cuuint64_t XC = (cuuint64_t)G.nxs / 32;
      const cuuint64_t dims[5] = {32, 27, XC, (cuuint64_t)G.ny, (cuuint64_t)G.nz + 2};
      const cuuint64_t strides[4] = {128, 27 * 128, 27 * 128 * XC, 27 * 128 * XC * (cuuint64_t)G.ny};
      const cuuint32_t beven[5] = {32, 27, 1, BY, BZ}, bgrp[5] = {32, 3, 1, BY, BZ};
      if (!encode(enc, &M.even, CU_TENSOR_MAP_DATA_TYPE_UINT32, 5, pop, dims, strides, beven) ||
          !encode(enc, &M.grp, CU_TENSOR_MAP_DATA_TYPE_UINT32, 5, pop, dims, strides, bgrp))
        return cudaErrorNotSupported;
      const TileSplit ts = tile_split(G);
      // boundary tiles first (block 0 is the tile at the origin: it advances the step counter)
      k_collide_stream<Store, Tr::minb, false, BlkDefault><<<ts.boundary(), dim3(BX, BY, BZ), 0, s>>>(
          Tr::make(pop, G), G, kc(P), odd, static_cast<const DT*>(dens), counter, io, M.dens, 1, ts, 1);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      using KT = decltype(&k_collide_stream_tp<Store::IS_BF16, 0>);
      const KT kern[2] = {&k_collide_stream_tp<Store::IS_BF16, 0>, &k_collide_stream_tp<Store::IS_BF16, 1>};
      static const bool attr =
          cudaFuncSetAttribute(kern[0], cudaFuncAttributeMaxDynamicSharedMemorySize, TP_SMEM) == cudaSuccess &&
          cudaFuncSetAttribute(kern[1], cudaFuncAttributeMaxDynamicSharedMemorySize, TP_SMEM) == cudaSuccess;
      if (!attr) return cudaErrorInvalidValue;
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const int n = ts.interior(), blocks = n < TP_MINB * sms ? n : TP_MINB * sms;
      kern[odd ? 1 : 0]<<<blocks, TP_THREADS, TP_SMEM, s>>>(Tr::make(pop, G), G, kc(P), M, ts, io.flag);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  static cudaError_t collide(void* pop, const Geom& G, const Phys& P, int odd, const void* dens, long long* counter,
                             int variant, const void* cur, void* nxt, int* flag, int shape, cudaStream_t s) {
    if constexpr (Tr::paired) {
      if (variant == 2) {
        k_collide_stream2<Store, Tr::minb2><<<grid3(G), dim3(PX, PY, PZ), 0, s>>>(
            Tr::make(pop, G), G, make_kconst<F2>(P), odd, static_cast<const float2*>(dens), counter);
        return cudaGetLastError();
      }
    }
    if constexpr (pipelined) {
      if (variant == 4) {
        static bool attr = false;  // first launch per process: allow the 68 KB of dynamic shared memory
        if (!attr) {
          cudaError_t e = cudaFuncSetAttribute(k_collide_stream_pf<Store, Tr::minb_pf>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, PF_SMEM);
          if (e != cudaSuccess) return e;
          attr = true;
        }
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const dim3 g3 = grid3(G);
        const int ntiles = (int)(g3.x * g3.y * g3.z);
        const int blocks = ntiles < sms * Tr::minb_pf ? ntiles : sms * Tr::minb_pf;
        k_collide_stream_pf<Store, Tr::minb_pf><<<blocks, dim3(BX, BY, BZ), PF_SMEM, s>>>(
            Tr::make(pop, G), G, kc(P), odd, static_cast<const float2*>(dens), counter, (int)g3.x, (int)g3.y, ntiles);
        return cudaGetLastError();
      }
    }
    FusedIO io{static_cast<const unsigned long long*>(cur), static_cast<unsigned long long*>(nxt), flag};
    if constexpr (pipelined) {
      if (variant == 5) {
        const cudaError_t e = collide_tp(pop, G, P, odd, dens, counter, io, s);
        if (e != cudaErrorNotSupported) return e;  // else the box has no pipelined tiles: variant 1
      }
    }
    const bool fp = variant == 3;
    if constexpr (!std::is_same<R, double>::value) {
      if (shape == 1) return collide_b<Blk<2, 4>>(pop, G, P, odd, dens, counter, fp, io, s);
      if (shape == 2) return collide_b<Blk<8, 1>>(pop, G, P, odd, dens, counter, fp, io, s);
    }
    return collide_b<BlkDefault>(pop, G, P, odd, dens, counter, fp, io, s);
  }
  static cudaError_t outflow(void* pop, const Geom& G, const Phys& P, int layout, void* top, void* fix,
                             cudaStream_t s) {
    const int64_t warps = (int64_t)G.nx * G.ny;  // one warp per column of the top plane
    k_outflow<Store><<<blocks1(warps * 32, 256), 256, 0, s>>>(Tr::make(pop, G), G, kc(P), layout,
                                                              static_cast<R*>(top),
                                                              static_cast<unsigned long long*>(fix));
    return cudaGetLastError();
  }
  static cudaError_t init(void* pop, const Geom& G, const Phys& P, const double* rr, const double* rb, const double* u,
                          cudaStream_t s) {
    const int64_t N = (int64_t)G.nx * G.ny * G.nz;
    k_init<Store><<<blocks1(N, 256), 256, 0, s>>>(Tr::make(pop, G), G, kc(P), rr, rb, u);
    return cudaGetLastError();
  }
  static cudaError_t get_pop(void* pop, const Geom& G, const Phys& P, int layout, int pdir, double* out_r,
                             double* out_b, cudaStream_t s) {
    const int64_t N = (int64_t)G.nx * G.ny * G.nz;
    k_get_pop<Store><<<blocks1(N, 256), 256, 0, s>>>(Tr::make(pop, G), G, kc(P), layout, pdir, out_r, out_b);
    return cudaGetLastError();
  }
  static cudaError_t set_pop(void* pop, const Geom& G, const Phys& P, int layout, int pdir, const double* in_r,
                             const double* in_b, cudaStream_t s) {
    const int64_t N = (int64_t)G.nx * G.ny * G.nz;
    k_set_pop<Store><<<blocks1(N, 256), 256, 0, s>>>(Tr::make(pop, G), G, kc(P), layout, pdir, in_r, in_b);
    return cudaGetLastError();
  }
  static cudaError_t top_from_state(void* pop, const Geom& G, const Phys& P, int layout, void* top, cudaStream_t s) {
    const int64_t Pn = (int64_t)G.nx * G.ny;
    k_top_from_state<Store><<<blocks1(Pn, 128), 128, 0, s>>>(Tr::make(pop, G), G, kc(P), layout, static_cast<R*>(top));
    return cudaGetLastError();
  }
  static cudaError_t macro(void* pop, const Geom& G, const Phys& P, int layout, double* rr, double* rb, double* u,
                           cudaStream_t s) {
    const int64_t N = (int64_t)G.nx * G.ny * G.nz;
    k_macro<Store><<<blocks1(N, 256), 256, 0, s>>>(Tr::make(pop, G), G, kc(P), layout, rr, rb, u);
    return cudaGetLastError();
  }
  static const KernelSet* table() {
    static const KernelSet ks = {
        sizeof(typename std::conditional<std::is_same<Store, PlainStore<double>>::value, double,
                                         typename std::conditional<std::is_same<Store, PlainStore<float>>::value, float,
                                                                   uint32_t>::type>::type),
        (std::is_same<Store, PlainStore<double>>::value || std::is_same<Store, PlainStore<float>>::value) ? 2 : 1,
        (size_t)Store::PLANES * sizeof(typename std::conditional<
                                    std::is_same<Store, PlainStore<double>>::value, double,
                                    typename std::conditional<std::is_same<Store, PlainStore<float>>::value,
                                                              float, uint32_t>::type>::type),
        sizeof(DT),
        sizeof(R),
        &density, &collide, &outflow, &init, &get_pop, &set_pop, &top_from_state, &macro, Tr::paired, fused,
        pipelined, false, nullptr, nullptr, nullptr, nullptr, &density_fold};
    return &ks;
  }
};

}  // namespace lbmk
