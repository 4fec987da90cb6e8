// Kernel instantiations for tenmoment1d: FP64 for N in [1, 2, 3, 4], FP32_BULK for N in [3].
#include "cr_launch.cuh"

namespace crk {

const KernelSet* kernels_tenmoment1d(int N, int mixed) {
  if (!mixed) {
    switch (N) {
      case 1: return Impl<1, 1, EqTenMoment, double, false>::set();
      case 2: return Impl<1, 2, EqTenMoment, double, false>::set();
      case 3: return Impl<1, 3, EqTenMoment, double, false>::set();
      case 4: return Impl<1, 4, EqTenMoment, double, false>::set();
    }
    return nullptr;
  }
  switch (N) {
    case 3: return Impl<1, 3, EqTenMoment, float, true>::set();
  }
  return nullptr;
}

}  // namespace crk
