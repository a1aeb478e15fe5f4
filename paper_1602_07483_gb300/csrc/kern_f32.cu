// kern_f32.cu -- step and auxiliary kernels with float storage.
#include "lbpf_table_impl.cuh"

namespace lbpf {
const KernelTable& table_f32() {
  static const KernelTable t = build_table<float>();
  return t;
}
}  // namespace lbpf
