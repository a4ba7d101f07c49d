// Kernel instantiations for windows 13, 15 (one unit per group so the
// library compiles in parallel).
#include "fnr_kernels.cuh"

namespace fnr {

const void *get_kernel_k13_15(int esize, int k, int algo) {
  switch (k) {
    case 13:
      return esize == 1 ? kernel_for<uint8_t, 13>(algo) : kernel_for<uint16_t, 13>(algo);
    case 15:
      return esize == 1 ? kernel_for<uint8_t, 15>(algo) : kernel_for<uint16_t, 15>(algo);
    default:
      return nullptr;
  }
}

}  // namespace fnr
