// kern_f32_b8.cu -- the 3D step kernels with float storage compiled for blocks of
// MAX_BLOCK_ROWS rows (a translation unit of its own so that it compiles in parallel).
#include "lbpf_table_impl.cuh"

namespace lbpf {
void add_fixed_kernels_f32(KernelTable& t) { fill_step_kernels_fixed<float>(t); }
}  // namespace lbpf
