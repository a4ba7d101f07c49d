// Kernel instantiations for windows 5, 7 (one unit per group so the
// library compiles in parallel).
#include "fnr_kernels.cuh"

namespace fnr {

const void *get_kernel_k5_7(int esize, int k, int algo) {
  switch (k) {
    case 5:
      return esize == 1 ? kernel_for<uint8_t, 5>(algo) : kernel_for<uint16_t, 5>(algo);
    case 7:
      return esize == 1 ? kernel_for<uint8_t, 7>(algo) : kernel_for<uint16_t, 7>(algo);
    default:
      return nullptr;
  }
}

}  // namespace fnr
