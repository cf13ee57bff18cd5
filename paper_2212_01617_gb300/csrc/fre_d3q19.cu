// Kernel instantiations for the D3Q19 lattice (all storage formats).
#include "fre_batch_kernels.cuh"
#include "fre_ws.cuh"

namespace fre {

const KernelSet *kernels_d3q19(int precision) {
    switch (precision) {
        case FRE_FP64: return kernel_set_ws<19, FRE_FP64>();
        case FRE_FP32: return kernel_set_ws<19, FRE_FP32>();
        case FRE_FP16DEV: return kernel_set_ws<19, FRE_FP16DEV>();
        case FRE_BF16DEV: return kernel_set_ws<19, FRE_BF16DEV>();
        default: return nullptr;
    }
}

const BatchKernels *batch_kernels_d3q19(int precision) {
    switch (precision) {
        case FRE_FP64: return BatchLaunchers<19, FRE_FP64>::set();
        case FRE_FP32: return BatchLaunchers<19, FRE_FP32>::set();
        case FRE_FP16DEV: return BatchLaunchers<19, FRE_FP16DEV>::set();
        case FRE_BF16DEV: return BatchLaunchers<19, FRE_BF16DEV>::set();
        default: return nullptr;
    }
}

}  // namespace fre
