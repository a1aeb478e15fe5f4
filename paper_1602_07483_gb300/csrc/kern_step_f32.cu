// kern_step_f32.cu -- one-launch step kernels with float storage (a translation unit of
// their own so that they compile in parallel with the two-kernel set).
#include "lbpf_table_impl.cuh"

namespace lbpf {
void add_step_kernels_f32(KernelTable& t) { fill_step_kernels<float>(t); }
}  // namespace lbpf
