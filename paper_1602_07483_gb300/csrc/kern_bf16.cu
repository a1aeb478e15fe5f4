// kern_bf16.cu -- step and auxiliary kernels with __nv_bfloat16 storage.
#include "lbpf_table_impl.cuh"

namespace lbpf {
const KernelTable& table_bf16() {
  static const KernelTable t = build_table<__nv_bfloat16>();
  return t;
}
}  // namespace lbpf
