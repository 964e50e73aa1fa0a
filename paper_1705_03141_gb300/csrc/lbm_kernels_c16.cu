// Compact 16-bit storage (half or bfloat16 totals + one colour record per node), FP32 arithmetic.
#include "lbm_compact.cuh"
#include "lbm_launch.cuh"

namespace lbmk {

template <bool B>
struct LaunchCompact {
  using Store = CompactStore<B>;
  static Store make(void* p, const Geom& G) {
    // population blocks first (56 bytes per storage node), then the records (16 bytes per node)
    return Store{static_cast<uint16_t*>(p), reinterpret_cast<float4*>(static_cast<char*>(p) + (size_t)56 * G.Ns),
                 G.Ns};
  }
  static KConst<float> kc(const Phys& P) { return make_kconst<float>(P); }
  static cudaError_t density(void* pop, const Geom& G, const Phys& P, int layout, void* dens, int* flag, void*, int,
                             cudaStream_t s) {
    k_density_c<B><<<grid3(G), dim3(BX, BY, BZ), 0, s>>>(make(pop, G), G, kc(P), layout, static_cast<float2*>(dens),
                                                          flag);
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

}  // namespace lbmk
