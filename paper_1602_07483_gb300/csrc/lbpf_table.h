// lbpf_table.h -- per-storage table of kernel launchers (host side).
#pragma once

#include <cuda_runtime.h>

#include "lbpf_dev.cuh"

namespace lbpf {

struct LatRT;

using StepLaunch = cudaError_t (*)(dim3 grid, dim3 block, size_t smem, cudaStream_t st, const SimDev* sims,
                                   const WorkItem* items, int s6);
using OneLaunchFn = cudaError_t (*)(dim3 grid, dim3 block, size_t smem, cudaStream_t st, const SimDev* sims,
                                    const WorkItem* items, const StepSched& sc, int s6);

struct KernelTable {
  int sbytes;            // bytes per stored population
  int tbytes;            // bytes of the compute type
  bool shifted;          // FP16/BF16 codec
  // indexed by lattice_slot(q): 7, 15, 19, 5, 9; theta additionally 0 (frozen) in the last slot.
  // Only pairings of one dimension are instantiated (the others are null).  Last index: the
  // block-height variant (block_variant): 1 for blocks of the height compiled in (8 rows in
  // 3D, one row in 2D), 0 for any height (the 2D entries are the one-row kernel in both).
  StepLaunch phi[5][2];
  StepLaunch uth[5][6][2];
  const void* phi_fn[5][2];
  const void* uth_fn[5][6][2];
  // one-launch step kernels (k_step) by phi, U and theta slots; null where not instantiated
  // (FP64, and lattice triples other than D3Q19 x D3Q19 x {frozen, D3Q7, D3Q19} and
  // D2Q9 x D2Q5 x D2Q5)
  OneLaunchFn step[5][5][6];
  const void* step_fn[5][5][6];
  cudaError_t (*init_scalar)(cudaStream_t, int nx, int ny, int nz, const double* cen, const double* rad, int nseed,
                             double c, void* out);
  cudaError_t (*init_pop)(cudaStream_t, const SimDev& sd, const LatRT& Lp, const LatRT& Lu, const LatRT& Lt,
                          const void* phi0, double U0, double theta0);
  // `prev`: the previous level of the field's moment (phi^{n-1} for g, theta^{n-1} for f), the
  // FP16/BF16 codec shift of those fields
  cudaError_t (*pack)(cudaStream_t, const SimDev& sd, int field, int par, const LatRT& L, int i, const double* gi,
                      const double* gj, const void* prev);
  cudaError_t (*unpack)(cudaStream_t, const SimDev& sd, int field, int par, const LatRT& L, int i, double* gi,
                        double* gj, const void* prev);
  cudaError_t (*to_double)(cudaStream_t, double* out, const void* in, long long n);
  cudaError_t (*from_double)(cudaStream_t, void* out, const double* in, long long n);
  cudaError_t (*sums)(cudaStream_t, const void* phi, const void* U, const void* th, double theta0, double k,
                      long long n, double* part, int nblk);
  cudaError_t (*tip)(cudaStream_t, const void* phi, int nx, int ny, int nz, int axis, int cx, int cy, int cz,
                     double* out);
};

// kernels compiled in translation units of their own (parallel compilation): the
// 8-row 3D step kernels of each storage type, and the one-launch step kernels
void add_fixed_kernels_f64(KernelTable& t);
void add_fixed_kernels_f32(KernelTable& t);
void add_fixed_kernels_f16(KernelTable& t);
void add_fixed_kernels_bf16(KernelTable& t);
void add_step_kernels_f32(KernelTable& t);
void add_step_kernels_f16(KernelTable& t);
void add_step_kernels_bf16(KernelTable& t);

const KernelTable& table_f64();
const KernelTable& table_f32();
const KernelTable& table_f16();
const KernelTable& table_bf16();

// slot of a lattice in the kernel tables: D3Q7, D3Q15, D3Q19, D2Q5, D2Q9, then q_theta = 0; -1 otherwise
inline int lattice_slot(int q) {
  switch (q) {
    case 7: return 0;
    case 15: return 1;
    case 19: return 2;
    case 5: return 3;
    case 9: return 4;
    case 0: return 5;
    default: return -1;
  }
}
inline bool lattice_is_2d(int q) { return q == 5 || q == 9; }

// kernel variant for blocks of `by` rows: the compiled-in height (MAX_BLOCK_ROWS in 3D, one
// row in 2D) or the general kernel
inline int block_variant(int q_phi, int by) { return by == (lattice_is_2d(q_phi) ? 1 : MAX_BLOCK_ROWS) ? 1 : 0; }

// populations with e_y != 0 (they cross block rows in the moment gather)
inline int ny_count(int q) {
  switch (q) {
    case 7: return 2;
    case 15: case 19: return 10;
    default: return 0;  // the 2D lattices have no kernel-y links
  }
}

// shared-memory bytes of the step kernels for a block of 32 x by threads: four ring planes of (by+2) x 34 scalars (eight with the
// FP16/BF16 codec: phi^{n-1} in k_phi, theta^{n-1} in k_uth when theta evolves) and a double-buffered plane of the e_y != 0
// populations
inline size_t phi_smem_bytes(const KernelTable& t, int qp, int by) {
  const size_t rs = 34u * (size_t)(by + 2);
  return ((t.shifted ? 8 : 4) * rs + 2 * (size_t)ny_count(qp) * 32u * by) * t.tbytes;
}
inline size_t uth_smem_bytes(const KernelTable& t, int qu, int qt, int by) {
  const size_t rs = 34u * (size_t)(by + 2);
  return ((t.shifted && qt ? 8 : 4) * rs + 2 * (size_t)(ny_count(qu) + ny_count(qt)) * 32u * by) * t.tbytes;
}
inline size_t step_smem_bytes(const KernelTable& t, int qp, int qu, int qt, int by) {
  const size_t a = phi_smem_bytes(t, qp, by), b = uth_smem_bytes(t, qu, qt, by);
  return a > b ? a : b;
}

}  // namespace lbpf
