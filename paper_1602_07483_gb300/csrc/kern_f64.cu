// kern_f64.cu -- step and auxiliary kernels with double storage.
#include "lbpf_table_impl.cuh"

namespace lbpf {
const KernelTable& table_f64() {
  static const KernelTable t = build_table<double>();
  return t;
}
}  // namespace lbpf
