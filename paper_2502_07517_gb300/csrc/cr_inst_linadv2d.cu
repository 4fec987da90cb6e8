// Kernel instantiations for linadv2d: FP64 for N in [1, 2, 3, 4].
#include "cr_launch.cuh"

namespace crk {

const KernelSet* kernels_linadv2d(int N, int mixed) {
  if (!mixed) {
    switch (N) {
      case 1: return Impl<2, 1, EqLinAdv, double, false>::set();
      case 2: return Impl<2, 2, EqLinAdv, double, false>::set();
      case 3: return Impl<2, 3, EqLinAdv, double, false>::set();
      case 4: return Impl<2, 4, EqLinAdv, double, false>::set();
    }
    return nullptr;
  }
  return nullptr;
}

}  // namespace crk
