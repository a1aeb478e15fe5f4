// kern_f64_b8.cu -- the 3D step kernels with double storage compiled for blocks of
// MAX_BLOCK_ROWS rows (a translation unit of its own so that it compiles in parallel).
#include "lbpf_table_impl.cuh"

namespace lbpf {
void add_fixed_kernels_f64(KernelTable& t) { fill_step_kernels_fixed<double>(t); }
}  // namespace lbpf
