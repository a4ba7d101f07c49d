// Kernel instantiations for windows 9, 11 (one unit per group so the
// library compiles in parallel).
#include "fnr_kernels.cuh"

namespace fnr {

const void *get_kernel_k9_11(int esize, int k, int algo) {
  switch (k) {
    case 9:
      return esize == 1 ? kernel_for<uint8_t, 9>(algo) : kernel_for<uint16_t, 9>(algo);
    case 11:
      return esize == 1 ? kernel_for<uint8_t, 11>(algo) : kernel_for<uint16_t, 11>(algo);
    default:
      return nullptr;
  }
}

}  // namespace fnr
