// kern_bf16_b8.cu -- the 3D step kernels with __nv_bfloat16 storage compiled for blocks of
// MAX_BLOCK_ROWS rows (a translation unit of its own so that it compiles in parallel).
#include "lbpf_table_impl.cuh"

namespace lbpf {
void add_fixed_kernels_bf16(KernelTable& t) { fill_step_kernels_fixed<__nv_bfloat16>(t); }
}  // namespace lbpf
