// kern_f16.cu -- step and auxiliary kernels with __half storage.
#include "lbpf_table_impl.cuh"

namespace lbpf {
const KernelTable& table_f16() {
  static const KernelTable t = [] {
    KernelTable k = build_table<__half>();
    add_fixed_kernels_f16(k);
    add_step_kernels_f16(k);
    return k;
  }();
  return t;
}
}  // namespace lbpf
