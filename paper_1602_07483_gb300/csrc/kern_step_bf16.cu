// kern_step_bf16.cu -- one-launch step kernels with __nv_bfloat16 storage (a translation unit of
// their own so that they compile in parallel with the two-kernel set).
#include "lbpf_table_impl.cuh"

namespace lbpf {
void add_step_kernels_bf16(KernelTable& t) { fill_step_kernels<__nv_bfloat16>(t); }
}  // namespace lbpf
