// Kernel instantiations for the D2Q9 lattice (all storage formats).
#include "fre_kernels.cuh"

namespace fre {

const KernelSet *kernels_d2q9(int precision) {
    switch (precision) {
        case FRE_FP64: return Launchers<9, FRE_FP64>::set();
        case FRE_FP32: return Launchers<9, FRE_FP32>::set();
        case FRE_FP16DEV: return Launchers<9, FRE_FP16DEV>::set();
        case FRE_BF16DEV: return Launchers<9, FRE_BF16DEV>::set();
        default: return nullptr;
    }
}

}  // namespace fre
