// FP32 storage and arithmetic.
#include <type_traits>
#include "lbm_launch.cuh"
namespace lbmk {
const KernelSet* kernels_f32() { return Launch<PlainStore<float>>::table(); }
}
