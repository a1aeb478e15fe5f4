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

template <int QP, typename S>
cudaError_t launch_phi(dim3 g, dim3 b, size_t smem, cudaStream_t st, const SimDev* sims, const WorkItem* items,
                       int s6) {
  k_phi<QP, S><<<g, b, smem, st>>>(sims, items, s6);
  return cudaGetLastError();
}

template <int QU, int QT, typename S>
cudaError_t launch_uth(dim3 g, dim3 b, size_t smem, cudaStream_t st, const SimDev* sims, const WorkItem* items,
                       int s6) {
  k_uth<QU, QT, S><<<g, b, smem, st>>>(sims, items, s6);
  return cudaGetLastError();
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

template <typename S>
KernelTable build_table() {
  KernelTable t{};
  t.sbytes = (int)sizeof(S);
  t.tbytes = (int)sizeof(typename Codec<S>::T);
  t.shifted = Codec<S>::shifted;
#define LBPF_PHI(q)                                   \
  t.phi[lattice_slot(q)] = launch_phi<q, S>;          \
  t.phi_fn[lattice_slot(q)] = (const void*)k_phi<q, S>;
  LBPF_PHI(7) LBPF_PHI(15) LBPF_PHI(19) LBPF_PHI(5) LBPF_PHI(9)
#undef LBPF_PHI
#define LBPF_UTH(qa, qb)                                                \
  t.uth[lattice_slot(qa)][lattice_slot(qb)] = launch_uth<qa, qb, S>;    \
  t.uth_fn[lattice_slot(qa)][lattice_slot(qb)] = (const void*)k_uth<qa, qb, S>;
  LBPF_UTH(7, 0) LBPF_UTH(7, 7) LBPF_UTH(7, 15) LBPF_UTH(7, 19)
  LBPF_UTH(15, 0) LBPF_UTH(15, 7) LBPF_UTH(15, 15) LBPF_UTH(15, 19)
  LBPF_UTH(19, 0) LBPF_UTH(19, 7) LBPF_UTH(19, 15) LBPF_UTH(19, 19)
  LBPF_UTH(5, 0) LBPF_UTH(5, 5) LBPF_UTH(5, 9)
  LBPF_UTH(9, 0) LBPF_UTH(9, 5) LBPF_UTH(9, 9)
#undef LBPF_UTH
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
