// kern_step_f16.cu -- one-launch step kernels with __half storage (a translation unit of
// their own so that they compile in parallel with the two-kernel set).
#include "lbpf_table_impl.cuh"

namespace lbpf {
void add_step_kernels_f16(KernelTable& t) { fill_step_kernels<__half>(t); }
}  // namespace lbpf
