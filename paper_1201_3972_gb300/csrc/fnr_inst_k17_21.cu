// Kernel instantiations for windows 17, 19, 21 (one unit per group so the
// library compiles in parallel).
#include "fnr_kernels.cuh"

namespace fnr {

const void *get_kernel_k17_21(int esize, int k, int algo) {
  switch (k) {
    case 17:
      return esize == 1 ? kernel_for<uint8_t, 17>(algo) : kernel_for<uint16_t, 17>(algo);
    case 19:
      return esize == 1 ? kernel_for<uint8_t, 19>(algo) : kernel_for<uint16_t, 19>(algo);
    case 21:
      return esize == 1 ? kernel_for<uint8_t, 21>(algo) : kernel_for<uint16_t, 21>(algo);
    default:
      return nullptr;
  }
}

}  // namespace fnr
