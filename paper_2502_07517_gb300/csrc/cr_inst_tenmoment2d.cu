// Kernel instantiations for tenmoment2d: FP64 for N in [1, 2, 3, 4], FP32_BULK for N in [3].
#include "cr_launch.cuh"

namespace crk {

const KernelSet* kernels_tenmoment2d(int N, int mixed) {
  if (!mixed) {
    switch (N) {
      case 1: return Impl<2, 1, EqTenMoment, double, false>::set();
      case 2: return Impl<2, 2, EqTenMoment, double, false>::set();
      case 3: return Impl<2, 3, EqTenMoment, double, false>::set();
      case 4: return Impl<2, 4, EqTenMoment, double, false>::set();
    }
    return nullptr;
  }
  switch (N) {
    case 3: return Impl<2, 3, EqTenMoment, float, true>::set();
  }
  return nullptr;
}

}  // namespace crk
