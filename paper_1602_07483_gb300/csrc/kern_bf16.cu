// kern_bf16.cu -- step and auxiliary kernels with __nv_bfloat16 storage.
#include "lbpf_table_impl.cuh"

namespace lbpf {
const KernelTable& table_bf16() {
  static const KernelTable t = [] {
    KernelTable k = build_table<__nv_bfloat16>();
    add_fixed_kernels_bf16(k);
    add_step_kernels_bf16(k);
    return k;
  }();
  return t;
}
}  // namespace lbpf
