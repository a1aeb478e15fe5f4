// kern_f16.cu -- step and auxiliary kernels with __half storage.
#include "lbpf_table_impl.cuh"

namespace lbpf {
const KernelTable& table_f16() {
  static const KernelTable t = build_table<__half>();
  return t;
}
}  // namespace lbpf
