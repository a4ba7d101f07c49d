// Kernel instantiations for windows 3 (one unit per group so the
// library compiles in parallel).
#include "fnr_kernels.cuh"

namespace fnr {

const void *get_kernel_k3(int esize, int k, int algo) {
  switch (k) {
    case 3:
      return esize == 1 ? kernel_for<uint8_t, 3>(algo) : kernel_for<uint16_t, 3>(algo);
    default:
      return nullptr;
  }
}

}  // namespace fnr
