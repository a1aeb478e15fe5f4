// kern_f64.cu -- step and auxiliary kernels with double storage.
#include "lbpf_table_impl.cuh"

namespace lbpf {
const KernelTable& table_f64() {
  static const KernelTable t = [] {
    KernelTable k = build_table<double>();
    add_fixed_kernels_f64(k);
    return k;
  }();
  return t;
}
}  // namespace lbpf
