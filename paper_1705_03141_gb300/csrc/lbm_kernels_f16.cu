// Packed 16-bit storage (half or bfloat16 deviation + 16-bit red fraction), FP32 arithmetic.
#include <type_traits>
#include "lbm_launch.cuh"
namespace lbmk {
const KernelSet* kernels_f16() { return Launch<PackedStore<false>>::table(); }
const KernelSet* kernels_bf16() { return Launch<PackedStore<true>>::table(); }
}
