// kern_f32.cu -- step and auxiliary kernels with float storage.
#include "lbpf_table_impl.cuh"

namespace lbpf {
const KernelTable& table_f32() {
  static const KernelTable t = [] {
    KernelTable k = build_table<float>();
    add_fixed_kernels_f32(k);
    add_step_kernels_f32(k);
    return k;
  }();
  return t;
}
}  // namespace lbpf
