// Kernel instantiations for euler1d with gravity (Sec. 5.5): FP64 for N in [1, 2, 3, 4], FP32_BULK for N in [3, 4].
#include "cr_launch.cuh"

namespace crk {

const KernelSet* kernels_euler1d_grav(int N, int mixed) {
  if (!mixed) {
    switch (N) {
      case 1: return Impl<1, 1, EqEulerG<1>, double, false>::set();
      case 2: return Impl<1, 2, EqEulerG<1>, double, false>::set();
      case 3: return Impl<1, 3, EqEulerG<1>, double, false>::set();
      case 4: return Impl<1, 4, EqEulerG<1>, double, false>::set();
    }
    return nullptr;
  }
  switch (N) {
    case 3: return Impl<1, 3, EqEulerG<1>, float, true>::set();
    case 4: return Impl<1, 4, EqEulerG<1>, float, true>::set();
  }
  return nullptr;
}

}  // namespace crk
