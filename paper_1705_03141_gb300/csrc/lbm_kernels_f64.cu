// FP64 storage and arithmetic: the mode that matches the FP64 CPU oracle.
#include <type_traits>
#include "lbm_launch.cuh"
namespace lbmk {
const KernelSet* kernels_f64() { return Launch<PlainStore<double>>::table(); }
}
