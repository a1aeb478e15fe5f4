// lbpf_table_impl.cuh -- builds the KernelTable of one storage type.  Included by
// one translation unit per storage type so the template instantiations compile
// in parallel.
#pragma once

#include "lbpf_aux.cuh"
#include "lbpf_table.h"

namespace lbpf {

constexpr int AUX_THREADS = 256;

inline int aux_blocks(long long n) {
  long long b = (n + AUX_THREADS - 1) / AUX_THREADS;
  if (b > 152LL * 32) b = 152LL * 32;
  return (int)(b < 1 ? 1 : b);
}

template <int QP, typename S, int BYC>
cudaError_t launch_phi(dim3 g, dim3 b, size_t smem, cudaStream_t st, const SimDev* sims, const WorkItem* items,
                       int s6) {
  k_phi<QP, S, BYC><<<g, b, smem, st>>>(sims, items, s6);
  return cudaGetLastError();
}

template <int QU, int QT, typename S, int BYC>
cudaError_t launch_uth(dim3 g, dim3 b, size_t smem, cudaStream_t st, const SimDev* sims, const WorkItem* items,
                       int s6) {
  k_uth<QU, QT, S, BYC><<<g, b, smem, st>>>(sims, items, s6);
  return cudaGetLastError();
}

template <int QP, int QU, int QT, typename S>
cudaError_t launch_step_one(dim3 g, dim3 b, size_t smem, cudaStream_t st, const SimDev* sims, const WorkItem* items,
                            const StepSched& sc, int s6) {
  k_step<QP, QU, QT, S><<<g, b, smem, st>>>(sims, items, sc, s6);
  return cudaGetLastError();
}

// The lattice triples with a one-launch step kernel: the paper's 3D benchmarks (D3Q19 for
// phi and U with theta frozen, on D3Q7 or on D3Q19) and its 2D set (D2Q9, D2Q5, D2Q5).
template <typename S>
void fill_step_kernels(KernelTable& t) {
#define LBPF_STEP(qa, qb, qc)                                                                     \
  t.step[lattice_slot(qa)][lattice_slot(qb)][lattice_slot(qc)] = launch_step_one<qa, qb, qc, S>; \
  t.step_fn[lattice_slot(qa)][lattice_slot(qb)][lattice_slot(qc)] = (const void*)k_step<qa, qb, qc, S>;
  LBPF_STEP(19, 19, 0) LBPF_STEP(19, 19, 7) LBPF_STEP(19, 19, 19) LBPF_STEP(9, 5, 5)
#undef LBPF_STEP
}

template <typename S>
struct AuxImpl {
  using T = typename Codec<S>::T;
  static cudaError_t init_scalar(cudaStream_t st, int nx, int ny, int nz, const double* cen, const double* rad,
                                 int nseed, double c, void* out) {
    const long long n = (long long)nx * ny * nz;
    k_init_scalar<T><<<aux_blocks(n), AUX_THREADS, 0, st>>>(nx, ny, nz, cen, rad, nseed, c, (T*)out);
    return cudaGetLastError();
  }
  static cudaError_t init_pop(cudaStream_t st, const SimDev& sd, const LatRT& Lp, const LatRT& Lu, const LatRT& Lt,
                              const void* phi0, double U0, double theta0) {
    k_init_pop<S><<<aux_blocks(sd.nsite), AUX_THREADS, 0, st>>>(sd, Lp, Lu, Lt, (const T*)phi0, U0, theta0);
    return cudaGetLastError();
  }
  static cudaError_t pack(cudaStream_t st, const SimDev& sd, int field, int par, const LatRT& L, int i,
                          const double* gi, const double* gj, const void* prev) {
    k_pack<S><<<aux_blocks(sd.nsite), AUX_THREADS, 0, st>>>(sd, field, par, L, i, gi, gj, (const T*)prev);
    return cudaGetLastError();
  }
  static cudaError_t unpack(cudaStream_t st, const SimDev& sd, int field, int par, const LatRT& L, int i, double* gi,
                            double* gj, const void* prev) {
    k_unpack<S><<<aux_blocks(sd.nsite), AUX_THREADS, 0, st>>>(sd, field, par, L, i, gi, gj, (const T*)prev);
    return cudaGetLastError();
  }
  static cudaError_t to_double(cudaStream_t st, double* out, const void* in, long long n) {
    k_to_double<T><<<aux_blocks(n), AUX_THREADS, 0, st>>>(out, (const T*)in, n);
    return cudaGetLastError();
  }
  static cudaError_t from_double(cudaStream_t st, void* out, const double* in, long long n) {
    k_from_double<T><<<aux_blocks(n), AUX_THREADS, 0, st>>>((T*)out, in, n);
    return cudaGetLastError();
  }
  static cudaError_t sums(cudaStream_t st, const void* phi, const void* U, const void* th, double theta0, double k,
                          long long n, double* part, int nblk) {
    k_sums<T><<<nblk, 256, 0, st>>>((const T*)phi, (const T*)U, (const T*)th, theta0, k, n, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sums_final<<<1, 32, 0, st>>>(part, nblk, part + 4 * nblk, k, n, th == nullptr, theta0);
    return cudaGetLastError();
  }
  static cudaError_t tip(cudaStream_t st, const void* phi, int nx, int ny, int nz, int axis, int cx, int cy, int cz,
                         double* out) {
    k_tip<T><<<1, dim3(32, 17), 0, st>>>((const T*)phi, nx, ny, nz, axis, cx, cy, cz, out);
    return cudaGetLastError();
  }
};

// The two-kernel step's kernels for blocks of any height (3D) and the one-row kernels (2D).
template <typename S>
void fill_step_kernels_general(KernelTable& t) {
#define LBPF_PHI3(q)                                          \
  t.phi[lattice_slot(q)][0] = launch_phi<q, S, 0>;             \
  t.phi_fn[lattice_slot(q)][0] = (const void*)k_phi<q, S, 0>;
#define LBPF_PHI2(q)                                                                       \
  t.phi[lattice_slot(q)][0] = t.phi[lattice_slot(q)][1] = launch_phi<q, S, 1>;              \
  t.phi_fn[lattice_slot(q)][0] = t.phi_fn[lattice_slot(q)][1] = (const void*)k_phi<q, S, 1>;
  LBPF_PHI3(7) LBPF_PHI3(15) LBPF_PHI3(19) LBPF_PHI2(5) LBPF_PHI2(9)
#undef LBPF_PHI3
#undef LBPF_PHI2
#define LBPF_UTH3(qa, qb)                                                            \
  t.uth[lattice_slot(qa)][lattice_slot(qb)][0] = launch_uth<qa, qb, S, 0>;            \
  t.uth_fn[lattice_slot(qa)][lattice_slot(qb)][0] = (const void*)k_uth<qa, qb, S, 0>;
#define LBPF_UTH2(qa, qb)                                                                              \
  t.uth[lattice_slot(qa)][lattice_slot(qb)][0] = t.uth[lattice_slot(qa)][lattice_slot(qb)][1] =         \
      launch_uth<qa, qb, S, 1>;                                                                        \
  t.uth_fn[lattice_slot(qa)][lattice_slot(qb)][0] = t.uth_fn[lattice_slot(qa)][lattice_slot(qb)][1] =   \
      (const void*)k_uth<qa, qb, S, 1>;
  LBPF_UTH3(7, 0) LBPF_UTH3(7, 7) LBPF_UTH3(7, 15) LBPF_UTH3(7, 19)
  LBPF_UTH3(15, 0) LBPF_UTH3(15, 7) LBPF_UTH3(15, 15) LBPF_UTH3(15, 19)
  LBPF_UTH3(19, 0) LBPF_UTH3(19, 7) LBPF_UTH3(19, 15) LBPF_UTH3(19, 19)
  LBPF_UTH2(5, 0) LBPF_UTH2(5, 5) LBPF_UTH2(5, 9)
  LBPF_UTH2(9, 0) LBPF_UTH2(9, 5) LBPF_UTH2(9, 9)
#undef LBPF_UTH3
#undef LBPF_UTH2
}

// The 3D two-kernel step's kernels compiled for blocks of MAX_BLOCK_ROWS rows.
template <typename S>
void fill_step_kernels_fixed(KernelTable& t) {
#define LBPF_PHI3(q)                                                         \
  t.phi[lattice_slot(q)][1] = launch_phi<q, S, MAX_BLOCK_ROWS>;               \
  t.phi_fn[lattice_slot(q)][1] = (const void*)k_phi<q, S, MAX_BLOCK_ROWS>;
  LBPF_PHI3(7) LBPF_PHI3(15) LBPF_PHI3(19)
#undef LBPF_PHI3
#define LBPF_UTH3(qa, qb)                                                                           \
  t.uth[lattice_slot(qa)][lattice_slot(qb)][1] = launch_uth<qa, qb, S, MAX_BLOCK_ROWS>;              \
  t.uth_fn[lattice_slot(qa)][lattice_slot(qb)][1] = (const void*)k_uth<qa, qb, S, MAX_BLOCK_ROWS>;
  LBPF_UTH3(7, 0) LBPF_UTH3(7, 7) LBPF_UTH3(7, 15) LBPF_UTH3(7, 19)
  LBPF_UTH3(15, 0) LBPF_UTH3(15, 7) LBPF_UTH3(15, 15) LBPF_UTH3(15, 19)
  LBPF_UTH3(19, 0) LBPF_UTH3(19, 7) LBPF_UTH3(19, 15) LBPF_UTH3(19, 19)
#undef LBPF_UTH3
}

template <typename S>
KernelTable build_table() {
  KernelTable t{};
  t.sbytes = (int)sizeof(S);
  t.tbytes = (int)sizeof(typename Codec<S>::T);
  t.shifted = Codec<S>::shifted;
  fill_step_kernels_general<S>(t);
  t.init_scalar = AuxImpl<S>::init_scalar;
  t.init_pop = AuxImpl<S>::init_pop;
  t.pack = AuxImpl<S>::pack;
  t.unpack = AuxImpl<S>::unpack;
  t.to_double = AuxImpl<S>::to_double;
  t.from_double = AuxImpl<S>::from_double;
  t.sums = AuxImpl<S>::sums;
  t.tip = AuxImpl<S>::tip;
  return t;
}

}  // namespace lbpf
