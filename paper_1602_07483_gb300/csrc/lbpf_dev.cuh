// lbpf_dev.cuh -- device code of the lattice-Boltzmann phase-field step for sm_103a.
//
// One time step (Sec. 3.4, "Algorithm implementation") on D3Q7/D3Q15/D3Q19, or on
// D2Q5/D2Q9 over an nz = 1 grid, is two kernels:
//   k_phi : phi collision (Eq. collision stage, non-local term) + streaming with
//           bounce-back, using phi^n, U^n, theta^n; writes the post-collision
//           populations and phi^{n+1}.
//   k_uth : U collision (Eq. LBE_Eq_Transport with the equilibrium of
//           Eq. Feq_Transport) and theta collision (Eq. LBE_Eq_Temp) with
//           phi^{n+1}, dphi/dt = (phi^{n+1} - phi^n)/dt; writes the post-collision
//           populations, U^{n+1} and theta^{n+1}.
//
// Storage ("pull" layout): buffer A holds, at node x, the post-collision value
// g*_i(x) of the previous step.  The population entering the collision at x is
// g_i(x,t) = A_i(x - e_i), or A_{i'}(x) when x - e_i is outside the domain
// (halfway bounce-back).  The non-local term g_i(x + e_i, t) of the phase-field
// collision is then A_i(x) itself for every non-boundary node.
//
// Each thread block owns a 30 x (BY-2) column of the xy plane and marches in z
// over a chunk of planes; a block is 32 x BY threads, one node per thread and
// plane.  For every plane the block recomputes the
// collisions on a one-node halo (32 x BY nodes) and gathers the streamed
// populations of its interior nodes into the zeroth moment of the next step:
// populations with e_y = 0 come from the thread itself or its x-neighbour lane
// by warp shuffle, the others through a double-buffered shared-memory plane, so
// each plane needs a single barrier.  The moment fields cost one scalar write
// per node and the distributions are read once and written once.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lbpf_plan.h"

namespace lbpf {

// ---------------------------------------------------------------- lattices
// Table 1 (e_i) and Table 2 (w_i, A_i, B_i, e^2) of Sec. 3.4.
template <int Q>
struct Lat;

template <>
struct Lat<7> {
  static constexpr double e2 = 0.25;
  static constexpr bool has_y = true;  // links along the kernel's y axis (false: a 2D lattice in the xz plane)
  static constexpr int diag0 = 1;      // first index of the diagonal weight class (none: an axis index)
  __host__ __device__ static constexpr int cls(int i) { return i == 0 ? 0 : 1; }  // 0 rest, 1 axis, 2 diagonal
  __host__ __device__ static constexpr int ex(int i) { return i == 1 ? 1 : (i == 3 ? -1 : 0); }
  __host__ __device__ static constexpr int ey(int i) { return i == 2 ? 1 : (i == 4 ? -1 : 0); }
  __host__ __device__ static constexpr int ez(int i) { return i == 5 ? 1 : (i == 6 ? -1 : 0); }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : (i == 1 ? 3 : (i == 2 ? 4 : (i == 3 ? 1 : (i == 4 ? 2 : (i == 5 ? 6 : 5)))));
  }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 0.25 : 0.125; }
  __host__ __device__ static constexpr double B(int i) { return i == 0 ? -0.75 : 0.125; }
};

// The accessors are switch expressions so that, with the population loops
// unrolled, every lookup folds to an immediate.
template <>
struct Lat<15> {
  static constexpr double e2 = 1.0 / 3.0;
  static constexpr bool has_y = true;
  static constexpr int diag0 = 7;
  __host__ __device__ static constexpr int cls(int i) { return i == 0 ? 0 : (i <= 6 ? 1 : 2); }
  // e_0..e_6 as D3Q7, then the cube diagonals
  __host__ __device__ static constexpr int ex(int i) {
    switch (i) {
      case 1: case 7: case 10: case 11: case 14: return 1;
      case 3: case 8: case 9: case 12: case 13: return -1;
      default: return 0;
    }
  }
  __host__ __device__ static constexpr int ey(int i) {
    switch (i) {
      case 2: case 7: case 8: case 11: case 12: return 1;
      case 4: case 9: case 10: case 13: case 14: return -1;
      default: return 0;
    }
  }
  __host__ __device__ static constexpr int ez(int i) {
    switch (i) {
      case 5: case 7: case 8: case 9: case 10: return 1;
      case 6: case 11: case 12: case 13: case 14: return -1;
      default: return 0;
    }
  }
  __host__ __device__ static constexpr int opp(int i) {
    switch (i) {
      case 1: return 3; case 2: return 4; case 3: return 1; case 4: return 2; case 5: return 6; case 6: return 5;
      case 7: return 13; case 8: return 14; case 9: return 11; case 10: return 12;
      case 11: return 9; case 12: return 10; case 13: return 7; case 14: return 8;
      default: return 0;
    }
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 2.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0);
  }
  __host__ __device__ static constexpr double B(int i) {
    return i == 0 ? -7.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0);
  }
};

template <>
struct Lat<19> {
  static constexpr double e2 = 1.0 / 3.0;
  static constexpr bool has_y = true;
  static constexpr int diag0 = 7;
  __host__ __device__ static constexpr int cls(int i) { return i == 0 ? 0 : (i <= 6 ? 1 : 2); }
  // e_0..e_6 as D3Q7, then the twelve edge diagonals
  __host__ __device__ static constexpr int ex(int i) {
    switch (i) {
      case 1: case 7: case 9: case 11: case 13: return 1;
      case 3: case 8: case 10: case 12: case 14: return -1;
      default: return 0;
    }
  }
  __host__ __device__ static constexpr int ey(int i) {
    switch (i) {
      case 2: case 7: case 8: case 15: case 17: return 1;
      case 4: case 9: case 10: case 16: case 18: return -1;
      default: return 0;
    }
  }
  __host__ __device__ static constexpr int ez(int i) {
    switch (i) {
      case 5: case 11: case 12: case 15: case 16: return 1;
      case 6: case 13: case 14: case 17: case 18: return -1;
      default: return 0;
    }
  }
  __host__ __device__ static constexpr int opp(int i) {
    switch (i) {
      case 1: return 3; case 2: return 4; case 3: return 1; case 4: return 2; case 5: return 6; case 6: return 5;
      case 7: return 10; case 8: return 9; case 9: return 8; case 10: return 7;
      case 11: return 14; case 12: return 13; case 13: return 12; case 14: return 11;
      case 15: return 18; case 16: return 17; case 17: return 16; case 18: return 15;
      default: return 0;
    }
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr double B(int i) {
    return i == 0 ? -2.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};
// Table 3 (e_i) and Table 4 (w_i, A_i, B_i, e^2) of Sec. 3.4: the 2D lattices.  A 2D
// grid (nx, ny) runs as a kernel grid (nx, 1, ny): the paper's y axis becomes the
// kernel's marching axis z, so ey() below is always 0 and ez() holds the paper's e_y.
// Population order and memory layout are unchanged (one kernel plane row per paper row).
template <>
struct Lat<5> {
  static constexpr double e2 = 1.0 / 3.0;
  static constexpr bool has_y = false;
  static constexpr int diag0 = 1;
  __host__ __device__ static constexpr int cls(int i) { return i == 0 ? 0 : 1; }
  __host__ __device__ static constexpr int ex(int i) { return i == 1 ? 1 : (i == 3 ? -1 : 0); }
  __host__ __device__ static constexpr int ey(int) { return 0; }
  __host__ __device__ static constexpr int ez(int i) { return i == 2 ? 1 : (i == 4 ? -1 : 0); }
  __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i <= 2 ? i + 2 : i - 2); }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
  __host__ __device__ static constexpr double B(int i) { return i == 0 ? -2.0 / 3.0 : 1.0 / 6.0; }
};

template <>
struct Lat<9> {
  static constexpr double e2 = 1.0 / 3.0;
  static constexpr bool has_y = false;
  static constexpr int diag0 = 5;
  __host__ __device__ static constexpr int cls(int i) { return i == 0 ? 0 : (i <= 4 ? 1 : 2); }
  // paper's e_0..e_4 as D2Q5, then (1,1), (-1,1), (-1,-1), (1,-1); second component in ez()
  __host__ __device__ static constexpr int ex(int i) {
    switch (i) {
      case 1: case 5: case 8: return 1;
      case 3: case 6: case 7: return -1;
      default: return 0;
    }
  }
  __host__ __device__ static constexpr int ey(int) { return 0; }
  __host__ __device__ static constexpr int ez(int i) {
    switch (i) {
      case 2: case 5: case 6: return 1;
      case 4: case 7: case 8: return -1;
      default: return 0;
    }
  }
  __host__ __device__ static constexpr int opp(int i) {
    switch (i) {
      case 1: return 3; case 2: return 4; case 3: return 1; case 4: return 2;
      case 5: return 7; case 6: return 8; case 7: return 5; case 8: return 6;
      default: return 0;
    }
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr double B(int i) {
    return i == 0 ? -5.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};
// A_i = 1 for the rest population and 0 otherwise on all five lattices.

// Populations with e_y != 0 cross block rows during the moment gather and go
// through shared memory; yslot(i) numbers them 0..NY-1 (-1 for e_y = 0).
template <int Q>
struct YSlots {
  __host__ __device__ static constexpr int count() {
    int c = 0;
    for (int i = 0; i < Q; ++i) c += Lat<Q>::ey(i) != 0;
    return c;
  }
  __host__ __device__ static constexpr int slot(int i) {
    if (Lat<Q>::ey(i) == 0) return -1;
    int c = 0;
    for (int j = 0; j < i; ++j) c += Lat<Q>::ey(j) != 0;
    return c;
  }
};
template <int Q>
struct NYOf {
  static constexpr int value = YSlots<Q>::count();
};
template <>
struct NYOf<0> {
  static constexpr int value = 0;
};

// ---------------------------------------------------------------- storage codec
// FP64/FP32: stored as is.  FP16/BF16: stored = (f - shift) * scale, decoded to
// FP32; `shift` removes the bulk value so the stored number is the small part.
template <typename S>
struct Codec;
// raw(s) / pack(v): the stored number itself as T and back (round to nearest), for
// arithmetic done directly in the scaled units (f - shift) * scale.
// dec64 / enc64: the same codec evaluated in FP64 for state import and export: with a
// power-of-two scale, s / scale + shift is exact in FP64, so export then import returns
// every stored number unchanged.
template <>
struct Codec<double> {
  using T = double;
  static constexpr bool shifted = false;
  __device__ static __forceinline__ T dec(double s, T, T) { return s; }
  __device__ static __forceinline__ double enc(T v, T, T) { return v; }
  __device__ static __forceinline__ T raw(double s) { return s; }
  __device__ static __forceinline__ double pack(T v) { return v; }
  __device__ static __forceinline__ double dec64(double s, double, double) { return s; }
  __device__ static __forceinline__ double enc64(double v, double, double) { return v; }
};
template <>
struct Codec<float> {
  using T = float;
  static constexpr bool shifted = false;
  __device__ static __forceinline__ T dec(float s, T, T) { return s; }
  __device__ static __forceinline__ float enc(T v, T, T) { return v; }
  __device__ static __forceinline__ T raw(float s) { return s; }
  __device__ static __forceinline__ float pack(T v) { return v; }
  __device__ static __forceinline__ double dec64(float s, double, double) { return (double)s; }
  __device__ static __forceinline__ float enc64(double v, double, double) { return (float)v; }
};
template <>
struct Codec<__half> {
  using T = float;
  static constexpr bool shifted = true;
  __device__ static __forceinline__ T dec(__half s, T shift, T inv_scale) {
    return fmaf(__half2float(s), inv_scale, shift);
  }
  __device__ static __forceinline__ __half enc(T v, T shift, T scale) { return __float2half_rn((v - shift) * scale); }
  __device__ static __forceinline__ T raw(__half s) { return __half2float(s); }
  __device__ static __forceinline__ __half pack(T v) { return __float2half_rn(v); }
  __device__ static __forceinline__ double dec64(__half s, double shift, double inv_scale) {
    return (double)__half2float(s) * inv_scale + shift;
  }
  __device__ static __forceinline__ __half enc64(double v, double shift, double scale) {
    return __double2half((v - shift) * scale);
  }
};
template <>
struct Codec<__nv_bfloat16> {
  using T = float;
  static constexpr bool shifted = true;
  __device__ static __forceinline__ T dec(__nv_bfloat16 s, T shift, T inv_scale) {
    return fmaf(__bfloat162float(s), inv_scale, shift);
  }
  __device__ static __forceinline__ __nv_bfloat16 enc(T v, T shift, T scale) {
    return __float2bfloat16_rn((v - shift) * scale);
  }
  __device__ static __forceinline__ T raw(__nv_bfloat16 s) { return __bfloat162float(s); }
  __device__ static __forceinline__ __nv_bfloat16 pack(T v) { return __float2bfloat16_rn(v); }
  __device__ static __forceinline__ double dec64(__nv_bfloat16 s, double shift, double inv_scale) {
    return (double)__bfloat162float(s) * inv_scale + shift;
  }
  __device__ static __forceinline__ __nv_bfloat16 enc64(double v, double shift, double scale) {
    return __double2bfloat16((v - shift) * scale);
  }
};

// ---------------------------------------------------------------- descriptors
// Per-simulation constants and buffers, resident in device memory.
struct SimDev {
  int nx, ny, nz, q_theta;
  long long nsite;
  void* pop[2][3];  // [buffer][g, h, f] in the storage type, [Q][z][y][x]
  void* phi[3];     // phi levels (compute type); level s%3 is phi^n at step s
  void* U[2];       // U^n at buffer s%2
  void* th[3];      // theta levels (unused when q_theta == 0); level s%3 is theta^n at step s
  double inv2dx;    // 1 / (2 dx)
  double c_eta;     // e^-2 (W0^2/tau0) dt/dx^2: eta_phi = c_eta a_s^2 + 1/2 (Eq. LBE_RelaxationTime)
  double c_N;       // e^-2 (dt/dx) W0^2/tau0: the N term of g^(0) (Eq. Feq_Phase)
  double dt_tau0;   // dt / tau0
  double lamM, lam; // lambda Mc_inf, lambda (Eq. LBE_SourceTerm)
  double eps1, eps2, grad2_min;
  int aniso, antitrapping;
  double k;
  double inv_etaU;  // 1 / eta_U (Eq. RelaxationTime_Concentration)
  double c_J;       // e^-2 dt/dx of the U lattice (Eq. Feq_Transport)
  double D_dx2;     // D / dx^2
  double D;
  double at_amp;    // W0 / (2 sqrt2), Eq. (AntiTrapping_Current)
  double dt, inv_dt;
  double inv_etaT;  // 1 / eta_theta (Eq. ThermalDiffusivity)
  double theta0;
  double shift_h, shift_f;       // FP16/BF16 codec: h shifted by w_i U0; f initially by w_i theta0
  double scale[3], inv_scale[3]; // FP16/BF16 codec scales of g, h, f
};

#ifndef LBPF_MAX_BLOCK_ROWS
#define LBPF_MAX_BLOCK_ROWS 8
#endif
constexpr int MAX_BLOCK_ROWS = LBPF_MAX_BLOCK_ROWS;  // blocks of at most 32 x 8 threads

// Resident blocks per SM the step kernels are compiled for (register budget:
// 65536 / (256 x blocks) registers per thread).  Measured on 512^3: k_phi runs
// best at three blocks (80 registers); k_uth at two (at 80 registers it spills).
#ifndef LBPF_PHI_MIN_BLOCKS
#define LBPF_PHI_MIN_BLOCKS 3
#endif
#ifndef LBPF_UTH_MIN_BLOCKS
#define LBPF_UTH_MIN_BLOCKS 2
#endif
// The 2D lattices run one-warp blocks; their launch bounds (counted in 256-thread
// blocks) set the register budget that decides how many warps an SM holds.  Measured
// on 8192^2 FP32: 64 registers (four 256-thread blocks) for both kernels, 21.2 -> 26.4
// GLUPS.  FP64 has budgets of its own (at 64 registers it spills).
#ifndef LBPF_PHI2D_MIN_BLOCKS
#define LBPF_PHI2D_MIN_BLOCKS 4
#endif
#ifndef LBPF_UTH2D_MIN_BLOCKS
#define LBPF_UTH2D_MIN_BLOCKS 4
#endif
// FP64 storage and arithmetic (values take two registers)
#ifndef LBPF_PHI64_MIN_BLOCKS
#define LBPF_PHI64_MIN_BLOCKS 3
#endif
#ifndef LBPF_UTH64_MIN_BLOCKS
#define LBPF_UTH64_MIN_BLOCKS 2
#endif

// ---------------------------------------------------------------- anisotropy
// a_s(n) and N = |grad phi|^2 a_s d a_s / d(grad phi) (Eq. TermesAnisotropes),
// written with n = grad phi / |grad phi| so that FP32 stays in range for small
// gradients.  kind 0: Eq. (Anisotropic-Function_As), derivatives of
// Eq. (Derivees_As); kind 1: Eq. (As_K41-K61) with its analytic derivatives.
template <typename T>
__device__ __forceinline__ T aniso_N(int kind, T e1, T e2, T gx, T gy, T gz, T G2, T& Nx, T& Ny, T& Nz) {
  const T iG = (sizeof(T) == 8) ? T(1) / sqrt(G2) : (T)rsqrtf((float)G2);
  const T nx = gx * iG, ny = gy * iG, nz = gz * iG;
  const T x2 = nx * nx, y2 = ny * ny, z2 = nz * nz;
  const T s4 = x2 * x2 + y2 * y2 + z2 * z2;
  T as, dx, dy, dz;  // dx = G * d a_s / d(d_x phi)
  if (kind == 0) {
    as = T(1) - T(3) * e1 + T(4) * e1 * s4;
    const T c = T(16) * e1;
    dx = c * nx * (x2 - s4);
    dy = c * ny * (y2 - s4);
    dz = c * nz * (z2 - s4);
  } else {
    const T p3 = x2 * y2 * z2;
    as = T(1) + e1 * (s4 - T(0.6)) + e2 * (T(3) * s4 + T(66) * p3 - T(17.0 / 7.0));
    const T cs = T(4) * (e1 + T(3) * e2);
    const T cp = T(132) * e2;
    dx = cs * nx * (x2 - s4) + cp * nx * y2 * z2 * (T(1) - T(3) * x2);
    dy = cs * ny * (y2 - s4) + cp * ny * x2 * z2 * (T(1) - T(3) * y2);
    dz = cs * nz * (z2 - s4) + cp * nz * x2 * y2 * (T(1) - T(3) * z2);
  }
  const T G = G2 * iG;
  const T f = G * as;  // |grad phi|^2 a_s / |grad phi|
  Nx = f * dx;
  Ny = f * dy;
  Nz = f * dz;
  return as;
}

// Read-only (non-coherent) load: the distributions read by a step kernel are
// never written by the same launch.
template <typename S>
__device__ __forceinline__ S ldro(const S* p) { return __ldg(p); }

__device__ __forceinline__ int slot4(int z) { return (z + 4) & 3; }  // z >= -1

// Products and sums that are never fused into an FMA: the collision loops are
// instantiated per row kind, and these keep the rounding identical in every
// instantiation (a node recomputed as a halo equals its owner's value bit for bit).
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }

// 1/x: IEEE division in FP64, the hardware approximate reciprocal in FP32
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }

// Scalar-field ring: four planes of (BY + 2) x 34 values around the block
// region (mirror ghosts by clamping).  Each thread owns up to RPT elements of a
// plane; their in-plane offsets are computed once, and the plane two ahead of
// the collision plane is fetched into registers one iteration early.
constexpr int RPT = 2;  // 34 x (BY + 2) <= RPT x 32 x BY for BY >= 3

struct RingMap {
  int off[RPT];  // in-plane offset (y * nx + x), or -1 when the slot is unused
  __device__ __forceinline__ void init(int x0, int y0, int nx, int ny, int RW, int RS, int tid, int nthr) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int idx = tid + r * nthr;
      off[r] = -1;
      if (idx < RS) {
        const int ly = idx / RW;
        const int lx = idx - ly * RW;
        const int gx = min(max(x0 - 2 + lx, 0), nx - 1);
        const int gy = min(max(y0 - 2 + ly, 0), ny - 1);
        off[r] = gy * nx + gx;
      }
    }
  }
};

template <typename T>
struct RingRegs {
  T v[RPT];
  // CG: through L2 (ld.global.cg) instead of the read-only path, for data written earlier
  // in the same launch
  template <bool CG = false>
  __device__ __forceinline__ void fetch(const RingMap& m, const T* __restrict__ src, int z, int nz, long long plane) {
    const T* p = src + (long long)min(max(z, 0), nz - 1) * plane;
#pragma unroll
    for (int r = 0; r < RPT; ++r)
      if (m.off[r] >= 0) v[r] = CG ? __ldcg(p + m.off[r]) : ldro(p + m.off[r]);
  }
  __device__ __forceinline__ void store(const RingMap& m, T* __restrict__ dst, int tid, int nthr) const {
#pragma unroll
    for (int r = 0; r < RPT; ++r)
      if (m.off[r] >= 0) dst[tid + r * nthr] = v[r];
  }
};

// ---------------------------------------------------------------- phase field
// One tile of the phase-field phase: the block's 30 x (BY-2) columns over planes [z0, z1).
// BYC: the block height BY when fixed at compile time (its index arithmetic then folds into
// constants), 0 to take it from blockDim.y.
template <int QP, typename S, int BYC>
__device__ __forceinline__ void phi_tile(const SimDev* __restrict__ sims, const WorkItem it, int s6) {
  using C = Codec<S>;
  using T = typename C::T;
  using L = Lat<QP>;
  using YS = YSlots<QP>;
  constexpr int NY = NYOf<QP>::value;
  const SimDev& sd = sims[it.sim];
  const int nx = sd.nx, ny = sd.ny, nz = sd.nz;
  const int BY = BYC > 0 ? BYC : (int)blockDim.y;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx, nthr = 32 * BY;
  const int x = it.x0 - 1 + tx;
  const int par = s6 & 1;
  // element offsets fit in 32 bits (Q * nsite < 2^32 is checked at create)
  const unsigned NS = (unsigned)sd.nsite;
  const unsigned plane = (unsigned)ny * (unsigned)nx;
  const S* __restrict__ gin = (const S*)sd.pop[par][0];
  S* __restrict__ gout = (S*)sd.pop[par ^ 1][0];
  const T* __restrict__ phin = (const T*)sd.phi[s6 % 3];
  const T* __restrict__ phim = (const T*)sd.phi[(s6 + 2) % 3];
  T* __restrict__ phinew = (T*)sd.phi[(s6 + 1) % 3];
  const T* __restrict__ Un = (const T*)sd.U[par];
  const T* __restrict__ thn = (const T*)sd.th[s6 % 3];
  const bool has_th = sd.q_theta != 0;

  constexpr bool HY = L::has_y;  // false: 2D lattice, one-row blocks without y halo
  const int RW = 34, RS = HY ? RW * (BY + 2) : RW, PS = BY * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);  // phi^n     [4][BY+2][34]
  T* ringm = ring + 4 * RS;                  // phi^{n-1} [4][BY+2][34] (codec shift only)
  T* sG = ring + (C::shifted ? 8 : 4) * RS;  // [2][NY][BY][32]

  const T inv2dx = (T)sd.inv2dx, c_eta = (T)sd.c_eta, c_N = (T)sd.c_N, dt_tau0 = (T)sd.dt_tau0;
  const T lamM = (T)sd.lamM, lam = (T)sd.lam, e1 = (T)sd.eps1, e2 = (T)sd.eps2, g2min = (T)sd.grad2_min;
  const T theta0 = (T)sd.theta0, scale = (T)sd.scale[0], iscale = (T)sd.inv_scale[0];
  const int kind = sd.aniso;

  const int zlo = max(it.z0 - 1, 0), zhi = min(it.z1, nz - 1);
  RingMap rm;
  rm.init(it.x0, it.y0, nx, ny, RW, RS, tid, nthr);
  {
    RingRegs<T> a;
    for (int z = zlo - 1; z <= zlo + 1; ++z) {
      a.fetch(rm, phin, z, nz, plane);
      a.store(rm, ring + slot4(z) * RS, tid, nthr);
      if (C::shifted) {
        a.fetch(rm, phim, z, nz, plane);
        a.store(rm, ringm + slot4(z) * RS, tid, nthr);
      }
    }
  }
  RingRegs<T> pf, pfm;
  if (zlo + 2 <= zhi + 1) {
    pf.fetch(rm, phin, zlo + 2, nz, plane);
    if (C::shifted) pfm.fetch(rm, phim, zlo + 2, nz, plane);
  }
  T a0A = 0, a1A = 0, a2A = 0;  // moments of planes zc-1, zc, zc+1
  int buf = 0;
  __syncthreads();

  for (int zc = zlo; zc <= zhi; ++zc) {
    T* sGb = sG + buf * NY * PS;
    const T* R0 = ring + slot4(zc) * RS;
    const T* Rp = ring + slot4(zc + 1) * RS;
    const T* Rm = ring + slot4(zc - 1) * RS;
    auto collide_row = [&](auto row_kind, T& acc0, T& acc1, T& acc2) {
      constexpr int KIND = decltype(row_kind)::value;  // 0 interior row, 1 top halo, 2 bottom halo
      auto row_needs = [](int ey) { return KIND == 0 || (KIND == 1 && ey == 1) || (KIND == 2 && ey == -1); };
      const int ly = ty;
      const int y = HY ? it.y0 - 1 + ly : it.y0 + ly;  // row 0 is a halo row except in one-row blocks
      const bool in_xy = x >= 0 && x < nx && y >= 0 && y < ny;
      const bool icol = in_xy && tx >= 1 && tx <= TILE_X && (!HY || (ly >= 1 && ly <= BY - 2));
      const int rc = HY ? (ly + 1) * RW + (tx + 1) : tx + 1;
      const unsigned site = ((unsigned)zc * (unsigned)ny + (unsigned)y) * (unsigned)nx + (unsigned)x;
      // wall node (standard collision): on a wall the lattice has links through
      // wall node (standard collision) on a face the lattice has links through; for the 3D
      // lattices the predicate keeps the order of the 3D-only kernels (the compiler's
      // schedule of the step kernels is sensitive to it)
      const bool bnd = L::has_y ? (x == 0 || y == 0 || zc == 0 || x == nx - 1 || y == ny - 1 || zc == nz - 1)
                                : (x == 0 || zc == 0 || x == nx - 1 || zc == nz - 1);
      T gs[QP];
#pragma unroll
      for (int i = 0; i < QP; ++i) gs[i] = T(0);
      if (in_xy) {
        const T Usite = ldro(Un + site);
        const T thsite = has_th ? ldro(thn + site) : theta0;
        // pulled populations g_i(x,t) and non-local values g_i(x+e_i,t), all loads first
        T gpull[QP], gnl[QP];
        if (!bnd) {
#pragma unroll
          for (int i = 0; i < QP; ++i) {
            const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
            if (!row_needs(ey)) continue;
            const unsigned own = (unsigned)i * NS + site;
            const unsigned off = (unsigned)(ez * (int)plane + ey * nx + ex);
            gpull[i] = C::raw(ldro(gin + (own - off)));
            if (C::shifted)  // stored units with the source's shift: Gp + S w phi_ref(src)
              gpull[i] = fma(rmul(scale, (T)L::w(i)), (ringm + slot4(zc - ez) * RS)[rc - ey * RW - ex], gpull[i]);
            gnl[i] = C::raw(ldro(gin + own));
          }
        } else {
          // wall node: bounce-back for links from outside, standard collision (no non-local term)
#pragma unroll
          for (int i = 0; i < QP; ++i) {
            const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
            if (!row_needs(ey)) continue;
            const int sx = x - ex, sy = y - ey, sz = zc - ez;
            const bool inside = sx >= 0 && sx < nx && sy >= 0 && sy < ny && sz >= 0 && sz < nz;
            const unsigned src = inside ? site - (unsigned)(ez * (int)plane + ey * nx + ex) : site;
            const int ii = inside ? i : L::opp(i);
            gpull[i] = C::raw(ldro(gin + ((unsigned)ii * NS + src)));
            if (C::shifted)
              gpull[i] = fma(rmul(scale, (T)L::w(i)), (ringm + slot4(inside ? sz : zc) * RS)[inside ? rc - ey * RW - ex : rc],
                             gpull[i]);
            gnl[i] = T(0);
          }
        }
        const T ph = R0[rc];
        // centred gradient with mirror ghosts (clamped ring)
        const T gx = (R0[rc + 1] - R0[rc - 1]) * inv2dx;
        const T gy = HY ? (R0[rc + RW] - R0[rc - RW]) * inv2dx : T(0);
        const T gz = (Rp[rc] - Rm[rc]) * inv2dx;
        const T G2 = gx * gx + gy * gy + gz * gz;
        T as = 1, Nx = 0, Ny = 0, Nz = 0;
        if (G2 >= g2min) as = aniso_N<T>(kind, e1, e2, gx, gy, gz, G2, Nx, Ny, Nz);
        const T as2 = as * as;
        const T inv_eta = rcp(c_eta * as2 + T(0.5));
        const T omp2 = T(1) - ph * ph;
        const T Qdt = (ph - (lamM * Usite + lam * thsite) * omp2) * omp2 * dt_tau0;
        const T a2 = bnd ? T(1) : as2;
        const T inv_a2 = bnd ? T(1) : rcp(a2);
        const T oma2 = T(1) - a2;
        const bool store = icol && zc >= it.z0 && zc < it.z1;
        // g* = [g (1 - 1/eta) - (1 - a^2) g_nl + g0/eta + w Q dt/tau0] / a^2 with
        // g0 = w (phi - e.N c_N): per weight class (rest, axis, diagonal) the terms
        // without e_i are one constant, and the e.N part is a signed sum of scaled N
        const T omw = T(1) - inv_eta;
        const T kph = radd(rmul(inv_eta, ph), Qdt);
        const T ncN = rmul(inv_eta, c_N);
        T Kc[3], nxc[3], nyc[3], nzc[3], Sc[3];
        // FP16/BF16: the populations stay in the stored units G = (g - w phi_ref) S, phi_ref
        // the phi of the step before at the node that stored them (phi^{n-1}); with
        // Gp' = Gp + S w phi_ref(src) (pulled) and G* = (g* - w phi^n) S the collision becomes
        //   G* = [omw Gp' - oma2 Gn + S (eq - w (oma2 phi_ref(x) + a^2 phi^n))] / a^2
        // and the value gathered for phi^{n+1} is G* + S w phi^n
        const T phr_x = C::shifted ? (ringm + slot4(zc) * RS)[rc] : T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T wc = (T)L::w(c == 0 ? 0 : (c == 1 ? 1 : L::diag0));
          Kc[c] = rmul(wc, kph);
          const T nc = rmul(-wc, ncN);
          nxc[c] = rmul(nc, Nx);
          nyc[c] = rmul(nc, Ny);
          nzc[c] = rmul(nc, Nz);
          if (C::shifted) {
            Kc[c] = rmul(scale, radd(Kc[c], -rmul(wc, radd(rmul(oma2, phr_x), rmul(a2, ph)))));
            nxc[c] = rmul(scale, nxc[c]);
            nyc[c] = rmul(scale, nyc[c]);
            nzc[c] = rmul(scale, nzc[c]);
            Sc[c] = rmul(scale, rmul(wc, ph));
          }
        }
#pragma unroll
        for (int i = 0; i < QP; ++i) {
          const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
          if (!row_needs(ey)) continue;
          const int c = L::cls(i);
          T eq = Kc[c];
          if (ex) eq = radd(eq, ex > 0 ? nxc[c] : -nxc[c]);
          if (ey) eq = radd(eq, ey > 0 ? nyc[c] : -nyc[c]);
          if (ez) eq = radd(eq, ez > 0 ? nzc[c] : -nzc[c]);
          const T g = rmul(fma(-oma2, gnl[i], fma(gpull[i], omw, eq)), inv_a2);
          const auto enc = C::pack(g);
          if (store) gout[(unsigned)i * NS + site] = enc;
          gs[i] = C::shifted ? radd(C::raw(enc), Sc[c]) : g;
          if (ey != 0) sGb[YS::slot(i) * PS + ly * 32 + tx] = gs[i];
        }
      }
      if (KIND == 0) {
        // populations with e_y = 0: from this lane or the x-neighbour lane (all lanes shuffle)
        T sv[QP];
  #pragma unroll
        for (int i = 0; i < QP; ++i) {
          const int ex = L::ex(i), ey = L::ey(i);
          sv[i] = gs[i];
          if (ey == 0 && ex > 0) sv[i] = __shfl_up_sync(0xffffffffu, gs[i], 1);
          if (ey == 0 && ex < 0) sv[i] = __shfl_down_sync(0xffffffffu, gs[i], 1);
        }
        if (icol) {
          if (!bnd) {
  #pragma unroll
            for (int i = 0; i < QP; ++i) {
              const int ey = L::ey(i), ez = L::ez(i);
              if (ey != 0) continue;
              if (ez < 0) acc0 += sv[i];
              else if (ez > 0) acc2 += sv[i];
              else acc1 += sv[i];
            }
          } else {
  #pragma unroll
            for (int i = 0; i < QP; ++i) {
              const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
              if (!row_needs(ey)) continue;
              if (ey != 0) continue;
              const int sx = x - ex, sz = zc - ez;
              const bool sin = sx >= 0 && sx < nx;
              if (sin) {
                if (ez < 0) acc0 += sv[i];
                else if (ez > 0) acc2 += sv[i];
                else acc1 += sv[i];
              }
              if (!sin || sz < 0 || sz >= nz) acc1 += gs[L::opp(i)];
            }
          }
        }
      }
    };
    // rows 0 and BY-1 are halo rows: they only feed the e_y = +1 / -1 populations to the block
    if (!HY) collide_row(std::integral_constant<int, 0>{}, a0A, a1A, a2A);
    else if (ty == 0) collide_row(std::integral_constant<int, 1>{}, a0A, a1A, a2A);
    else if (ty == BY - 1) collide_row(std::integral_constant<int, 2>{}, a0A, a1A, a2A);
    else collide_row(std::integral_constant<int, 0>{}, a0A, a1A, a2A);
    // ring plane zc+2 (its slot last held plane zc-2), then prefetch zc+3
    if (zc + 2 <= zhi + 1) {
      pf.store(rm, ring + slot4(zc + 2) * RS, tid, nthr);
      if (C::shifted) pfm.store(rm, ringm + slot4(zc + 2) * RS, tid, nthr);
    }
    if (zc + 3 <= zhi + 1) {
      pf.fetch(rm, phin, zc + 3, nz, plane);
      if (C::shifted) pfm.fetch(rm, phim, zc + 3, nz, plane);
    }
    __syncthreads();
    // populations with e_y != 0: from the neighbouring rows through shared memory
    auto gather_row = [&](const int r, T& acc0, T& acc1, T& acc2) {
      const int ly = ty;
      const int y = HY ? it.y0 - 1 + ly : it.y0 + ly;  // row 0 is a halo row except in one-row blocks
      const bool icol = x >= 0 && x < nx && y >= 0 && y < ny && tx >= 1 && tx <= TILE_X && (!HY || (ly >= 1 && ly <= BY - 2));
      if (icol) {
        const bool inner = L::has_y ? (x >= 1 && y >= 1 && zc >= 1 && x <= nx - 2 && y <= ny - 2 && zc <= nz - 2)
                                    : (x >= 1 && zc >= 1 && x <= nx - 2 && zc <= nz - 2);
        if (inner) {
#pragma unroll
          for (int i = 0; i < QP; ++i) {
            const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
            if (ey == 0) continue;
            const T v = sGb[YS::slot(i) * PS + (ly - ey) * 32 + tx - ex];
            if (ez < 0) acc0 += v;
            else if (ez > 0) acc2 += v;
            else acc1 += v;
          }
        } else {
#pragma unroll
          for (int i = 0; i < QP; ++i) {
            const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
            if (ey == 0) continue;
            const int sx = x - ex, sy = y - ey, sz = zc - ez;
            const bool sin = sx >= 0 && sx < nx && sy >= 0 && sy < ny;
            if (sin) {
              const T v = sGb[YS::slot(i) * PS + (ly - ey) * 32 + tx - ex];
              if (ez < 0) acc0 += v;
              else if (ez > 0) acc2 += v;
              else acc1 += v;
            }
            if (!sin || sz < 0 || sz >= nz) acc1 += sGb[YS::slot(L::opp(i)) * PS + ly * 32 + tx];
          }
        }
        const int zw = zc - 1;
        // FP16/BF16: the gathered values are in stored units (scale is a power of two)
        auto mP = [&](T a) { return C::shifted ? rmul(a, iscale) : a; };
        if (zw >= it.z0 && zw < it.z1 && zw >= 0) phinew[((unsigned)zw * ny + y) * (unsigned)nx + x] = mP(acc0);
        if (zc == nz - 1 && zc >= it.z0 && zc < it.z1) phinew[((unsigned)zc * ny + y) * (unsigned)nx + x] = mP(acc1);
      }
      acc0 = acc1;
      acc1 = acc2;
      acc2 = 0;
    };
    gather_row(0, a0A, a1A, a2A);
    buf ^= 1;
  }
}

template <int QP, typename S, int BYC>
__global__ void __launch_bounds__(32 * MAX_BLOCK_ROWS, sizeof(S) == 8 ? LBPF_PHI64_MIN_BLOCKS
                                                       : (Lat<QP>::has_y ? LBPF_PHI_MIN_BLOCKS : LBPF_PHI2D_MIN_BLOCKS)) k_phi(const SimDev* __restrict__ sims, const WorkItem* __restrict__ items,
                                                int s6) {
  phi_tile<QP, S, BYC>(sims, items[blockIdx.x], s6);
}

// ---------------------------------------------------------------- U and theta
// One tile of the U/theta phase.  COH: phi^{n+1} is read through L2 (ld.global.cg), for
// launches in which other blocks of the same launch write it.  BYC as for phi_tile.
template <int QU, int QT, typename S, bool COH, int BYC>
__device__ __forceinline__ void uth_tile(const SimDev* __restrict__ sims, const WorkItem it, int s6) {
  using C = Codec<S>;
  using T = typename C::T;
  using LU = Lat<QU>;
  using LT = Lat<(QT > 0 ? QT : 7)>;
  using YU = YSlots<QU>;
  using YT = YSlots<(QT > 0 ? QT : 7)>;
  constexpr int NYU = NYOf<QU>::value;
  constexpr int NYT = NYOf<QT>::value;
  constexpr int QTA = QT > 0 ? QT : 1;
  const SimDev& sd = sims[it.sim];
  const int nx = sd.nx, ny = sd.ny, nz = sd.nz;
  const int BY = BYC > 0 ? BYC : (int)blockDim.y;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx, nthr = 32 * BY;
  const int x = it.x0 - 1 + tx;
  const int par = s6 & 1;
  const unsigned NS = (unsigned)sd.nsite;
  const unsigned plane = (unsigned)ny * (unsigned)nx;
  const S* __restrict__ hin = (const S*)sd.pop[par][1];
  S* __restrict__ hout = (S*)sd.pop[par ^ 1][1];
  const S* __restrict__ fin = (const S*)sd.pop[par][2];
  S* __restrict__ fout = (S*)sd.pop[par ^ 1][2];
  const T* __restrict__ phin = (const T*)sd.phi[s6 % 3];
  const T* __restrict__ phi1 = (const T*)sd.phi[(s6 + 1) % 3];
  const T* __restrict__ Un = (const T*)sd.U[par];
  T* __restrict__ Unew = (T*)sd.U[par ^ 1];
  const T* __restrict__ thn = (const T*)sd.th[s6 % 3];
  T* __restrict__ thnew = (T*)sd.th[(s6 + 1) % 3];
  const T* __restrict__ thm = (const T*)sd.th[(s6 + 2) % 3];  // theta^{n-1}: the FP16/BF16 shift of f

  constexpr bool HY = LU::has_y;  // false: 2D lattices, one-row blocks without y halo
  const int RW = 34, RS = HY ? RW * (BY + 2) : RW, PS = BY * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);  // phi^{n+1} [4][BY+2][34]
  // FP16/BF16 with theta evolving: theta^{n-1} [4][BY+2][34], the shift of each stored f
  constexpr bool TSH = C::shifted && QT > 0;
  T* ringt = ring + 4 * RS;
  T* sH = ring + (TSH ? 8 : 4) * RS;         // [2][NYU + NYT][BY][32]
  constexpr int NYA = NYU + NYT;

  const T inv2dx = (T)sd.inv2dx, k = (T)sd.k, inv_etaU = (T)sd.inv_etaU, c_J = (T)sd.c_J;
  const T D_dx2 = (T)sd.D_dx2, D = (T)sd.D, at_amp = (T)sd.at_amp, inv_dt = (T)sd.inv_dt, dt = (T)sd.dt;
  const T g2min = (T)sd.grad2_min, inv_etaT = (T)sd.inv_etaT;
  const T sh_h = (T)sd.shift_h, sc_h = (T)sd.scale[1], isc_h = (T)sd.inv_scale[1];
  const T sc_f = (T)sd.scale[2], isc_f = (T)sd.inv_scale[2];
  const bool at_on = sd.antitrapping != 0;
  const T opk = T(1) + k, omk = T(1) - k;

  const int zlo = max(it.z0 - 1, 0), zhi = min(it.z1, nz - 1);
  RingMap rm;
  rm.init(it.x0, it.y0, nx, ny, RW, RS, tid, nthr);
  {
    RingRegs<T> a;
    for (int z = zlo - 1; z <= zlo + 1; ++z) {
      a.template fetch<COH>(rm, phi1, z, nz, plane);
      a.store(rm, ring + slot4(z) * RS, tid, nthr);
      if (TSH) {
        a.fetch(rm, thm, z, nz, plane);
        a.store(rm, ringt + slot4(z) * RS, tid, nthr);
      }
    }
  }
  RingRegs<T> pf, pft;
  if (zlo + 2 <= zhi + 1) {
    pf.template fetch<COH>(rm, phi1, zlo + 2, nz, plane);
    if (TSH) pft.fetch(rm, thm, zlo + 2, nz, plane);
  }
  T u0A = 0, u1A = 0, u2A = 0, t0A = 0, t1A = 0, t2A = 0;
  int buf = 0;
  __syncthreads();

  for (int zc = zlo; zc <= zhi; ++zc) {
    T* sHb = sH + buf * NYA * PS;
    T* sFb = sHb + NYU * PS;
    const T* R0 = ring + slot4(zc) * RS;
    const T* Rp = ring + slot4(zc + 1) * RS;
    const T* Rm = ring + slot4(zc - 1) * RS;
    auto collide_row = [&](auto row_kind, T& u0, T& u1, T& u2, T& t0, T& t1, T& t2) {
      constexpr int KIND = decltype(row_kind)::value;  // 0 interior row, 1 top halo, 2 bottom halo
      auto row_needs = [](int ey) { return KIND == 0 || (KIND == 1 && ey == 1) || (KIND == 2 && ey == -1); };
      const int ly = ty;
      const int y = HY ? it.y0 - 1 + ly : it.y0 + ly;  // row 0 is a halo row except in one-row blocks
      const bool in_xy = x >= 0 && x < nx && y >= 0 && y < ny;
      const bool icol = in_xy && tx >= 1 && tx <= TILE_X && (!HY || (ly >= 1 && ly <= BY - 2));
      const int rc = HY ? (ly + 1) * RW + (tx + 1) : tx + 1;
      const unsigned site = ((unsigned)zc * (unsigned)ny + (unsigned)y) * (unsigned)nx + (unsigned)x;
      const bool inner = LU::has_y ? (x >= 1 && y >= 1 && zc >= 1 && x <= nx - 2 && y <= ny - 2 && zc <= nz - 2)
                                   : (x >= 1 && zc >= 1 && x <= nx - 2 && zc <= nz - 2);
      T hs[QU], fs[QTA];
#pragma unroll
      for (int i = 0; i < QU; ++i) hs[i] = T(0);
#pragma unroll
      for (int i = 0; i < QTA; ++i) fs[i] = T(0);
      if (in_xy) {
        const T U = ldro(Un + site);
        const T phn = ldro(phin + site);
        const T th = QT > 0 ? ldro(thn + site) : T(0);
        // pulled populations, all loads first; interior nodes need no wall checks
        if (inner) {
#pragma unroll
          for (int i = 0; i < QU; ++i) {
            const int ex = LU::ex(i), ey = LU::ey(i), ez = LU::ez(i);
            if (!row_needs(ey)) continue;
            hs[i] = C::raw(ldro(hin + ((unsigned)i * NS + site - (unsigned)(ez * (int)plane + ey * nx + ex))));
          }
#pragma unroll
          for (int i = 0; i < QT; ++i) {
            const int ex = LT::ex(i), ey = LT::ey(i), ez = LT::ez(i);
            if (!row_needs(ey)) continue;
            fs[i] = C::raw(ldro(fin + ((unsigned)i * NS + site - (unsigned)(ez * (int)plane + ey * nx + ex))));
            if (TSH)  // stored units with the source's shift: F + S w theta^{n-1}(src)
              fs[i] = fma(rmul(sc_f, (T)LT::w(i)), (ringt + slot4(zc - ez) * RS)[rc - ey * RW - ex], fs[i]);
          }
        } else {
#pragma unroll
          for (int i = 0; i < QU; ++i) {
            const int ex = LU::ex(i), ey = LU::ey(i), ez = LU::ez(i);
            if (!row_needs(ey)) continue;
            const int sx = x - ex, sy = y - ey, sz = zc - ez;
            const bool inside = sx >= 0 && sx < nx && sy >= 0 && sy < ny && sz >= 0 && sz < nz;
            const unsigned src = inside ? site - (unsigned)(ez * (int)plane + ey * nx + ex) : site;
            const int ii = inside ? i : LU::opp(i);
            hs[i] = C::raw(ldro(hin + ((unsigned)ii * NS + src)));
          }
#pragma unroll
          for (int i = 0; i < QT; ++i) {
            const int ex = LT::ex(i), ey = LT::ey(i), ez = LT::ez(i);
            if (!row_needs(ey)) continue;
            const int sx = x - ex, sy = y - ey, sz = zc - ez;
            const bool inside = sx >= 0 && sx < nx && sy >= 0 && sy < ny && sz >= 0 && sz < nz;
            const unsigned src = inside ? site - (unsigned)(ez * (int)plane + ey * nx + ex) : site;
            const int ii = inside ? i : LT::opp(i);
            fs[i] = C::raw(ldro(fin + ((unsigned)ii * NS + src)));
            if (TSH)
              fs[i] = fma(rmul(sc_f, (T)LT::w(i)), (ringt + slot4(inside ? sz : zc) * RS)[inside ? rc - ey * RW - ex : rc],
                          fs[i]);
          }
        }
        // phi^{n+1} at the node and its six neighbours (mirror ghosts)
        const T pc = R0[rc];
        const T pxp = R0[rc + 1], pxm = R0[rc - 1], pyp = HY ? R0[rc + RW] : pc, pym = HY ? R0[rc - RW] : pc, pzp = Rp[rc], pzm = Rm[rc];
        // q(phi) = (1 - phi)/2, zeta(phi) = ((1+k) - (1-k) phi)/2
        auto qf = [&](T p) { return T(0.5) * (T(1) - p); };
        // 1/zeta at the node and its six neighbours with one division (batch inversion):
        // 2 zeta = (1+k) - (1-k) phi
        const T d0 = opk - omk * pc, d1 = opk - omk * pxp, d2 = opk - omk * pxm, d3 = opk - omk * pyp,
                d4 = opk - omk * pym, d5 = opk - omk * pzp, d6 = opk - omk * pzm;
        const T p1 = d0 * d1, p2 = p1 * d2, p3 = p2 * d3, p4 = p3 * d4, p5 = p4 * d5, p6 = p5 * d6;
        T rr = T(2) * rcp(p6);  // 2 / (d0 ... d6)
        const T iz_zm = rr * p5;
        rr *= d6;
        const T iz_zp = rr * p4;
        rr *= d5;
        const T iz_ym = rr * p3;
        rr *= d4;
        const T iz_yp = rr * p2;
        rr *= d3;
        const T iz_xm = rr * p1;
        rr *= d2;
        const T iz_xp = rr * d0;
        const T izc = rr * d1;
        const T qc = qf(pc), qzc = qc * izc;
        const T gpx = (pxp - pxm) * inv2dx, gpy = (pyp - pym) * inv2dx, gpz = (pzp - pzm) * inv2dx;
        const T Fx = (iz_xp - iz_xm) * inv2dx, Fy = (iz_yp - iz_ym) * inv2dx, Fz = (iz_zp - iz_zm) * inv2dx;
        const T gqzx = (qf(pxp) * iz_xp - qf(pxm) * iz_xm) * inv2dx;
        const T gqzy = (qf(pyp) * iz_yp - qf(pym) * iz_ym) * inv2dx;
        const T gqzz = (qf(pzp) * iz_zp - qf(pzm) * iz_zm) * inv2dx;
        // div(D q grad(1/zeta)) in compact face form, face q = mean of nodal q
        const T divDqF =
            D_dx2 * (T(0.5) * (qc + qf(pxp)) * (iz_xp - izc) - T(0.5) * (qc + qf(pxm)) * (izc - iz_xm) +
                     T(0.5) * (qc + qf(pyp)) * (iz_yp - izc) - T(0.5) * (qc + qf(pym)) * (izc - iz_ym) +
                     T(0.5) * (qc + qf(pzp)) * (iz_zp - izc) - T(0.5) * (qc + qf(pzm)) * (izc - iz_zm));
        const T dphi = pc - phn;  // phi^{n+1} - phi^n
        const T dphidt = dphi * inv_dt;
        const T fU = T(1) + omk * U;
        T jx = 0, jy = 0, jz = 0;
        const T G2 = gpx * gpx + gpy * gpy + gpz * gpz;
        if (at_on && G2 >= g2min) {
          const T iG = (sizeof(T) == 8) ? T(1) / sqrt(G2) : rsqrtf((float)G2);
          const T amp = -at_amp * fU * dphidt * iG;
          jx = amp * gpx;
          jy = amp * gpy;
          jz = amp * gpz;
        }
        const T DqU = D * U;
        const T Jx = DqU * (gqzx + qc * Fx) + jx * izc;
        const T Jy = DqU * (gqzy + qc * Fy) + jy * izc;
        const T Jz = DqU * (gqzz + qc * Fz) + jz * izc;
        const T Ssrc = U * divDqF + (jx * Fx + jy * Fy + jz * Fz);
        const T src_dt = (Ssrc + fU * T(0.5) * dphidt * izc) * dt;
        const T qzU = qzc * U;
        const bool store = icol && zc >= it.z0 && zc < it.z1;
        // h* = h (1 - 1/eta_U) + h0/eta_U + w (S + Q_U/zeta) dt with
        // h0 = A U + B (q/zeta U + e.J c_J): per weight class one constant plus e.(scaled J)
        const T omU = T(1) - inv_etaU;
        T KU[3], jxc[3], jyc[3], jzc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int ic = c == 0 ? 0 : (c == 1 ? 1 : LU::diag0);
          const T wc = (T)LU::w(ic), Bc = (T)LU::B(ic);
          KU[c] = radd(rmul(inv_etaU, radd(c == 0 ? U : T(0), rmul(Bc, qzU))), rmul(wc, src_dt));
          const T jc = rmul(rmul(inv_etaU, Bc), c_J);
          jxc[c] = rmul(jc, Jx);
          jyc[c] = rmul(jc, Jy);
          jzc[c] = rmul(jc, Jz);
          if (C::shifted) {
            // FP16/BF16: the populations stay in the stored units H = (h - w U0) S, so
            // H* = H (1 - 1/eta_U) + S (h0/eta_U + w src dt - w U0 / eta_U)
            KU[c] = rmul(sc_h, radd(KU[c], -rmul(rmul(wc, sh_h), inv_etaU)));
            jxc[c] = rmul(sc_h, jxc[c]);
            jyc[c] = rmul(sc_h, jyc[c]);
            jzc[c] = rmul(sc_h, jzc[c]);
          }
        }
#pragma unroll
        for (int i = 0; i < QU; ++i) {
          const int ex = LU::ex(i), ey = LU::ey(i), ez = LU::ez(i);
          if (!row_needs(ey)) continue;
          const int c = LU::cls(i);
          T eq = KU[c];
          if (ex) eq = radd(eq, ex > 0 ? jxc[c] : -jxc[c]);
          if (ey) eq = radd(eq, ey > 0 ? jyc[c] : -jyc[c]);
          if (ez) eq = radd(eq, ez > 0 ? jzc[c] : -jzc[c]);
          const T h = fma(hs[i], omU, eq);
          const auto enc = C::pack(h);
          if (store) hout[(unsigned)i * NS + site] = enc;
          hs[i] = C::raw(enc);
          if (ey != 0) sHb[YU::slot(i) * PS + ly * 32 + tx] = hs[i];
        }
        if (QT > 0) {
          // f* = f (1 - 1/eta_T) + w (theta/eta_T + Q_theta dt) with Q_theta dt = dphi / 2
          const T omT = T(1) - inv_etaT;
          T kT = radd(rmul(inv_etaT, th), rmul(T(0.5), dphi));
          // FP16/BF16: f is stored as F = (f - w theta_ref) S with theta_ref the theta of the
          // storing node one step earlier; with F' = F + S w theta^{n-1}(src) (pulled) and
          // F* = (f* - w theta^n) S the update is F* = F' (1 - 1/eta_T) + w S (dphi/2 - theta^n (1 - 1/eta_T)),
          // and the value gathered for theta^{n+1} is F* + S w theta^n
          if (C::shifted) kT = rmul(sc_f, radd(rmul(T(0.5), dphi), -rmul(th, omT)));
#pragma unroll
          for (int i = 0; i < QT; ++i) {
            const int ey = LT::ey(i);
            if (!row_needs(ey)) continue;
            const T wi = (T)LT::w(i);
            const T f = fma(fs[i], omT, rmul(wi, kT));
            const auto enc = C::pack(f);
            if (store) fout[(unsigned)i * NS + site] = enc;
            fs[i] = C::shifted ? radd(C::raw(enc), rmul(rmul(sc_f, wi), th)) : C::raw(enc);
            if (ey != 0) sFb[YT::slot(i) * PS + ly * 32 + tx] = fs[i];
          }
        }
      }
      if (KIND == 0) {
        // populations with e_y = 0: from this lane or the x-neighbour lane (all lanes shuffle)
        T hv[QU], fv[QTA];
  #pragma unroll
        for (int i = 0; i < QU; ++i) {
          const int ex = LU::ex(i), ey = LU::ey(i);
          hv[i] = hs[i];
          if (ey == 0 && ex > 0) hv[i] = __shfl_up_sync(0xffffffffu, hs[i], 1);
          if (ey == 0 && ex < 0) hv[i] = __shfl_down_sync(0xffffffffu, hs[i], 1);
        }
  #pragma unroll
        for (int i = 0; i < QT; ++i) {
          const int ex = LT::ex(i), ey = LT::ey(i);
          fv[i] = fs[i];
          if (ey == 0 && ex > 0) fv[i] = __shfl_up_sync(0xffffffffu, fs[i], 1);
          if (ey == 0 && ex < 0) fv[i] = __shfl_down_sync(0xffffffffu, fs[i], 1);
        }
        if (icol) {
          if (inner) {
  #pragma unroll
            for (int i = 0; i < QU; ++i) {
              const int ey = LU::ey(i), ez = LU::ez(i);
              if (ey != 0) continue;
              if (ez < 0) u0 += hv[i];
              else if (ez > 0) u2 += hv[i];
              else u1 += hv[i];
            }
  #pragma unroll
            for (int i = 0; i < QT; ++i) {
              const int ey = LT::ey(i), ez = LT::ez(i);
              if (ey != 0) continue;
              if (ez < 0) t0 += fv[i];
              else if (ez > 0) t2 += fv[i];
              else t1 += fv[i];
            }
          } else {
  #pragma unroll
            for (int i = 0; i < QU; ++i) {
              const int ex = LU::ex(i), ey = LU::ey(i), ez = LU::ez(i);
              if (!row_needs(ey)) continue;
              if (ey != 0) continue;
              const int sx = x - ex, sz = zc - ez;
              const bool sin = sx >= 0 && sx < nx;
              if (sin) {
                if (ez < 0) u0 += hv[i];
                else if (ez > 0) u2 += hv[i];
                else u1 += hv[i];
              }
              if (!sin || sz < 0 || sz >= nz) u1 += hs[LU::opp(i)];
            }
  #pragma unroll
            for (int i = 0; i < QT; ++i) {
              const int ex = LT::ex(i), ey = LT::ey(i), ez = LT::ez(i);
              if (!row_needs(ey)) continue;
              if (ey != 0) continue;
              const int sx = x - ex, sz = zc - ez;
              const bool sin = sx >= 0 && sx < nx;
              if (sin) {
                if (ez < 0) t0 += fv[i];
                else if (ez > 0) t2 += fv[i];
                else t1 += fv[i];
              }
              if (!sin || sz < 0 || sz >= nz) t1 += fs[LT::opp(i)];
            }
          }
        }
      }
    };
    // rows 0 and BY-1 are halo rows: they only feed the e_y = +1 / -1 populations to the block
    if (!HY) collide_row(std::integral_constant<int, 0>{}, u0A, u1A, u2A, t0A, t1A, t2A);
    else if (ty == 0) collide_row(std::integral_constant<int, 1>{}, u0A, u1A, u2A, t0A, t1A, t2A);
    else if (ty == BY - 1) collide_row(std::integral_constant<int, 2>{}, u0A, u1A, u2A, t0A, t1A, t2A);
    else collide_row(std::integral_constant<int, 0>{}, u0A, u1A, u2A, t0A, t1A, t2A);
    if (zc + 2 <= zhi + 1) {
      pf.store(rm, ring + slot4(zc + 2) * RS, tid, nthr);
      if (TSH) pft.store(rm, ringt + slot4(zc + 2) * RS, tid, nthr);
    }
    if (zc + 3 <= zhi + 1) {
      pf.template fetch<COH>(rm, phi1, zc + 3, nz, plane);
      if (TSH) pft.fetch(rm, thm, zc + 3, nz, plane);
    }
    __syncthreads();
    auto gather_row = [&](const int r, T& u0, T& u1, T& u2, T& t0, T& t1, T& t2) {
      const int ly = ty;
      const int y = HY ? it.y0 - 1 + ly : it.y0 + ly;  // row 0 is a halo row except in one-row blocks
      const bool icol = x >= 0 && x < nx && y >= 0 && y < ny && tx >= 1 && tx <= TILE_X && (!HY || (ly >= 1 && ly <= BY - 2));
      if (icol) {
        const bool inner = LU::has_y ? (x >= 1 && y >= 1 && zc >= 1 && x <= nx - 2 && y <= ny - 2 && zc <= nz - 2)
                                     : (x >= 1 && zc >= 1 && x <= nx - 2 && zc <= nz - 2);
        if (inner) {
#pragma unroll
          for (int i = 0; i < QU; ++i) {
            const int ex = LU::ex(i), ey = LU::ey(i), ez = LU::ez(i);
            if (ey == 0) continue;
            const T v = sHb[YU::slot(i) * PS + (ly - ey) * 32 + tx - ex];
            if (ez < 0) u0 += v;
            else if (ez > 0) u2 += v;
            else u1 += v;
          }
#pragma unroll
          for (int i = 0; i < QT; ++i) {
            const int ex = LT::ex(i), ey = LT::ey(i), ez = LT::ez(i);
            if (ey == 0) continue;
            const T v = sFb[YT::slot(i) * PS + (ly - ey) * 32 + tx - ex];
            if (ez < 0) t0 += v;
            else if (ez > 0) t2 += v;
            else t1 += v;
          }
        } else {
#pragma unroll
          for (int i = 0; i < QU; ++i) {
            const int ex = LU::ex(i), ey = LU::ey(i), ez = LU::ez(i);
            if (ey == 0) continue;
            const int sx = x - ex, sy = y - ey, sz = zc - ez;
            const bool sin = sx >= 0 && sx < nx && sy >= 0 && sy < ny;
            if (sin) {
              const T v = sHb[YU::slot(i) * PS + (ly - ey) * 32 + tx - ex];
              if (ez < 0) u0 += v;
              else if (ez > 0) u2 += v;
              else u1 += v;
            }
            if (!sin || sz < 0 || sz >= nz) u1 += sHb[YU::slot(LU::opp(i)) * PS + ly * 32 + tx];
          }
#pragma unroll
          for (int i = 0; i < QT; ++i) {
            const int ex = LT::ex(i), ey = LT::ey(i), ez = LT::ez(i);
            if (ey == 0) continue;
            const int sx = x - ex, sy = y - ey, sz = zc - ez;
            const bool sin = sx >= 0 && sx < nx && sy >= 0 && sy < ny;
            if (sin) {
              const T v = sFb[YT::slot(i) * PS + (ly - ey) * 32 + tx - ex];
              if (ez < 0) t0 += v;
              else if (ez > 0) t2 += v;
              else t1 += v;
            }
            if (!sin || sz < 0 || sz >= nz) t1 += sFb[YT::slot(LT::opp(i)) * PS + ly * 32 + tx];
          }
        }
        const int zw = zc - 1;
        // FP16/BF16: the gathered sums are in stored units; the shifts w_i U0 (w_i theta0)
        // of the populations arriving at a node add up to U0 (theta0)
        auto mU = [&](T a) { return C::shifted ? fma(a, isc_h, sh_h) : a; };
        auto mT = [&](T a) { return C::shifted ? rmul(a, isc_f) : a; };
        if (zw >= it.z0 && zw < it.z1 && zw >= 0) {
          const unsigned sw = ((unsigned)zw * ny + y) * (unsigned)nx + x;
          Unew[sw] = mU(u0);
          if (QT > 0) thnew[sw] = mT(t0);
        }
        if (zc == nz - 1 && zc >= it.z0 && zc < it.z1) {
          const unsigned sw = ((unsigned)zc * ny + y) * (unsigned)nx + x;
          Unew[sw] = mU(u1);
          if (QT > 0) thnew[sw] = mT(t1);
        }
      }
      u0 = u1;
      u1 = u2;
      u2 = 0;
      t0 = t1;
      t1 = t2;
      t2 = 0;
    };
    gather_row(0, u0A, u1A, u2A, t0A, t1A, t2A);
    buf ^= 1;
  }
}

template <int QU, int QT, typename S, int BYC>
__global__ void __launch_bounds__(32 * MAX_BLOCK_ROWS, sizeof(S) == 8 ? LBPF_UTH64_MIN_BLOCKS
                                                       : (Lat<QU>::has_y ? LBPF_UTH_MIN_BLOCKS : LBPF_UTH2D_MIN_BLOCKS)) k_uth(const SimDev* __restrict__ sims, const WorkItem* __restrict__ items,
                                                int s6) {
  uth_tile<QU, QT, S, false, BYC>(sims, items[blockIdx.x], s6);
}

// ---------------------------------------------------------------- one launch per step
// Both phases of a step in one persistent launch, so that tiles of the phase-field phase
// (bound by instruction issue) run beside tiles of the U/theta phase (bound by memory
// latency) on the same SMs.  Blocks draw tickets in order from a counter; ticket t names
// the phase-field tile or the U/theta tile of one work item.  The U/theta tile of an item
// reads phi^{n+1} over its ring (two nodes around its columns and rows, two planes around
// its z-chunk), so it waits for the done flags of the phase-field tiles that write that
// region; the host orders the tickets so that those tiles always come earlier, and a
// block draws a ticket only while it runs, so no wait depends on a tile that has not
// started.  The U/theta tiles read nothing else that the launch writes (the phase-field
// tiles write g at the other buffer parity and the new phi level; the U/theta tiles write
// h, f, U and theta at levels the phase-field tiles do not read).  The waits are bounded
// all the same: after about a second a wait gives up, sets *err (host-visible) and the tile
// goes ahead; the host then reports the step as failed.
struct StepSched {
  const int* order;    // ticket -> j >= 0: phase-field tile of item j; ~j: U/theta tile of item j
  const int* dep_off;  // the U/theta tile of item j waits for the phase-field tiles dep[dep_off[j] .. dep_off[j+1])
  const int* dep;
  unsigned* ctl;       // ctl[0]: next ticket; ctl[1 + j]: phase-field tile of item j done (zeroed before each launch)
  int* err;            // set to 1 when a wait gave up
  int ntickets;
  unsigned polls;      // bound of each wait (rounds of about 0.25 us)
};


__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One full warp waits until done[dep[k]] != 0 for every k < n, each lane polling a share
// of the flags; false when `polls` rounds passed without that.
__device__ __forceinline__ bool wait_done(const unsigned* done, const int* dep, int n, unsigned polls) {
  const int lane = threadIdx.x & 31;
  for (unsigned r = 0; r < polls; ++r) {
    bool ok = true;
    for (int k = lane; k < n; k += 32) ok = ok && ld_acquire_gpu(done + __ldg(dep + k)) != 0u;
    if (__all_sync(0xffffffffu, ok)) return true;
    __nanosleep(200);
  }
  return false;
}

template <int QP, int QU, int QT, typename S>
__global__ void __launch_bounds__(32 * MAX_BLOCK_ROWS, sizeof(S) == 8 ? LBPF_UTH64_MIN_BLOCKS
                                                       : (Lat<QU>::has_y ? LBPF_UTH_MIN_BLOCKS : LBPF_UTH2D_MIN_BLOCKS)) k_step(const SimDev* __restrict__ sims, const WorkItem* __restrict__ items,
                                                const StepSched sc, int s6) {
  __shared__ int s_ticket;
  const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
  for (;;) {
    if (lead) s_ticket = (int)atomicAdd(sc.ctl, 1u);
    __syncthreads();
    const int t = s_ticket;
    if (t >= sc.ntickets) return;  // the same for every thread of the block
    const int w = __ldg(sc.order + t);
    if (w >= 0) {
      phi_tile<QP, S, 0>(sims, items[w], s6);
      __threadfence();  // this thread's phi^{n+1} stores are visible before the flag
      __syncthreads();
      if (lead) st_release_gpu(sc.ctl + 1 + w, 1u);
    } else {
      const int j = ~w;
      if (threadIdx.y == 0) {
        const int b = __ldg(sc.dep_off + j), n = __ldg(sc.dep_off + j + 1) - b;
        if (!wait_done(sc.ctl + 1, sc.dep + b, n, sc.polls) && threadIdx.x == 0) atomicExch(sc.err, 1);
      }
      __syncthreads();
      uth_tile<QU, QT, S, true, 0>(sims, items[j], s6);
      __syncthreads();  // the next tile reuses the shared memory
    }
  }
}

}  // namespace lbpf
