// Kernel instantiations for varadv1d: FP64 for N in [1, 2, 3, 4].
#include "cr_launch.cuh"

namespace crk {

const KernelSet* kernels_varadv1d(int N, int mixed) {
  if (!mixed) {
    switch (N) {
      case 1: return Impl<1, 1, EqVarAdv, double, false>::set();
      case 2: return Impl<1, 2, EqVarAdv, double, false>::set();
      case 3: return Impl<1, 3, EqVarAdv, double, false>::set();
      case 4: return Impl<1, 4, EqVarAdv, double, false>::set();
    }
    return nullptr;
  }
  return nullptr;
}

}  // namespace crk
