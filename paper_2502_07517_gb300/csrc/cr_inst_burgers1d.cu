// Kernel instantiations for burgers1d: FP64 for N in [1, 2, 3, 4].
#include "cr_launch.cuh"

namespace crk {

const KernelSet* kernels_burgers1d(int N, int mixed) {
  if (!mixed) {
    switch (N) {
      case 1: return Impl<1, 1, EqBurgers, double, false>::set();
      case 2: return Impl<1, 2, EqBurgers, double, false>::set();
      case 3: return Impl<1, 3, EqBurgers, double, false>::set();
      case 4: return Impl<1, 4, EqBurgers, double, false>::set();
    }
    return nullptr;
  }
  return nullptr;
}

}  // namespace crk
