// lbpf_dev.cuh -- device code of the lattice-Boltzmann phase-field step for sm_103a.
//
// One time step (Sec. 3.4, "Algorithm implementation") is two kernels:
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
// over a chunk of planes.  For every plane it recomputes the collisions on a
// one-node halo (32 x BY nodes), keeps them in shared memory and gathers the
// streamed populations of its interior columns into the zeroth moment of the
// next step, so the moment fields cost one scalar write per node and the
// distributions are read once and written once.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbpf {

// ---------------------------------------------------------------- lattices
// Table 1 (e_i) and Table 2 (w_i, A_i, B_i, e^2) of Sec. 3.4.
template <int Q>
struct Lat;

template <>
struct Lat<7> {
  static constexpr double e2 = 0.25;
  __host__ __device__ static constexpr int ex(int i) { return i == 1 ? 1 : (i == 3 ? -1 : 0); }
  __host__ __device__ static constexpr int ey(int i) { return i == 2 ? 1 : (i == 4 ? -1 : 0); }
  __host__ __device__ static constexpr int ez(int i) { return i == 5 ? 1 : (i == 6 ? -1 : 0); }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : (i == 1 ? 3 : (i == 2 ? 4 : (i == 3 ? 1 : (i == 4 ? 2 : (i == 5 ? 6 : 5)))));
  }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 0.25 : 0.125; }
  __host__ __device__ static constexpr double B(int i) { return i == 0 ? -0.75 : 0.125; }
};

template <>
struct Lat<15> {
  static constexpr double e2 = 1.0 / 3.0;
  // rows: e_0..e_6 as D3Q7, then the cube diagonals
  __host__ __device__ static constexpr int ex(int i) {
    constexpr int v[15] = {0, 1, 0, -1, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return v[i];
  }
  __host__ __device__ static constexpr int ey(int i) {
    constexpr int v[15] = {0, 0, 1, 0, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
    return v[i];
  }
  __host__ __device__ static constexpr int ez(int i) {
    constexpr int v[15] = {0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1};
    return v[i];
  }
  __host__ __device__ static constexpr int opp(int i) {
    constexpr int v[15] = {0, 3, 4, 1, 2, 6, 5, 13, 14, 11, 12, 9, 10, 7, 8};
    return v[i];
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
  __host__ __device__ static constexpr int ex(int i) {
    constexpr int v[19] = {0, 1, 0, -1, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return v[i];
  }
  __host__ __device__ static constexpr int ey(int i) {
    constexpr int v[19] = {0, 0, 1, 0, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
    return v[i];
  }
  __host__ __device__ static constexpr int ez(int i) {
    constexpr int v[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
    return v[i];
  }
  __host__ __device__ static constexpr int opp(int i) {
    constexpr int v[19] = {0, 3, 4, 1, 2, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15};
    return v[i];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr double B(int i) {
    return i == 0 ? -2.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};
// A_i = 1 for the rest population and 0 otherwise on all three lattices.

// ---------------------------------------------------------------- storage codec
// FP64/FP32: stored as is.  FP16/BF16: stored = (f - shift) * scale, decoded to
// FP32; `shift` removes the bulk value so the stored number is the small part.
template <typename S>
struct Codec;
template <>
struct Codec<double> {
  using T = double;
  static constexpr bool shifted = false;
  __device__ static __forceinline__ T dec(double s, T, T) { return s; }
  __device__ static __forceinline__ double enc(T v, T, T) { return v; }
};
template <>
struct Codec<float> {
  using T = float;
  static constexpr bool shifted = false;
  __device__ static __forceinline__ T dec(float s, T, T) { return s; }
  __device__ static __forceinline__ float enc(T v, T, T) { return v; }
};
template <>
struct Codec<__half> {
  using T = float;
  static constexpr bool shifted = true;
  __device__ static __forceinline__ T dec(__half s, T shift, T inv_scale) {
    return fmaf(__half2float(s), inv_scale, shift);
  }
  __device__ static __forceinline__ __half enc(T v, T shift, T scale) { return __float2half_rn((v - shift) * scale); }
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
};

// ---------------------------------------------------------------- descriptors
// Per-simulation constants and buffers, resident in device memory.
struct SimDev {
  int nx, ny, nz, q_theta;
  long long nsite;
  void* pop[2][3];  // [buffer][g, h, f] in the storage type, [Q][z][y][x]
  void* phi[3];     // phi levels (compute type); level s%3 is phi^n at step s
  void* U[2];       // U^n at buffer s%2
  void* th[2];      // theta^n at buffer s%2 (unused when q_theta == 0)
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
  double shift_h, shift_f;       // FP16/BF16 codec: h shifted by w_i U0, f by w_i theta0
  double scale[3], inv_scale[3]; // FP16/BF16 codec scales of g, h, f
};

struct WorkItem {
  int sim;
  int x0, y0;  // first interior column of the tile
  int z0, z1;  // planes [z0, z1) written by this block
};

constexpr int TILE_X = 30;  // interior columns per block row (block x = 32)

// ---------------------------------------------------------------- anisotropy
// a_s(n) and N = |grad phi|^2 a_s d a_s / d(grad phi) (Eq. TermesAnisotropes),
// written with n = grad phi / |grad phi| so that FP32 stays in range for small
// gradients.  kind 0: Eq. (Anisotropic-Function_As), derivatives of
// Eq. (Derivees_As); kind 1: Eq. (As_K41-K61) with its analytic derivatives.
template <typename T>
__device__ __forceinline__ T aniso_N(int kind, T e1, T e2, T gx, T gy, T gz, T G2, T& Nx, T& Ny, T& Nz) {
  const T iG = (sizeof(T) == 8) ? T(1) / sqrt(G2) : rsqrtf((float)G2);
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

__device__ __forceinline__ int ring_slot(int z) { return ((z % 3) + 3) % 3; }

// Load plane z (clamped to the domain = mirror ghost at distance 1) of a scalar
// field into a ring slot covering the block region plus one node of halo.
template <typename T>
__device__ __forceinline__ void load_ring(T* __restrict__ dst, const T* __restrict__ src, int z, int x0, int y0,
                                          int nx, int ny, int nz, int RW, int RS, int tid, int nthr) {
  const int zc = min(max(z, 0), nz - 1);
  const long long base = (long long)zc * ny * nx;
  for (int idx = tid; idx < RS; idx += nthr) {
    const int ly = idx / RW;
    const int lx = idx - ly * RW;
    const int gx = min(max(x0 - 2 + lx, 0), nx - 1);
    const int gy = min(max(y0 - 2 + ly, 0), ny - 1);
    dst[idx] = src[base + (long long)gy * nx + gx];
  }
}

// ---------------------------------------------------------------- phase field
template <int QP, typename S>
__global__ void __launch_bounds__(512) k_phi(const SimDev* __restrict__ sims, const WorkItem* __restrict__ items,
                                             int s6) {
  using C = Codec<S>;
  using T = typename C::T;
  using L = Lat<QP>;
  const WorkItem it = items[blockIdx.x];
  const SimDev& sd = sims[it.sim];
  const int nx = sd.nx, ny = sd.ny, nz = sd.nz;
  const int BY = blockDim.y;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx, nthr = 32 * BY;
  const int x = it.x0 - 1 + tx, y = it.y0 - 1 + ty;
  const bool in_xy = x >= 0 && x < nx && y >= 0 && y < ny;
  const bool icol = in_xy && tx >= 1 && tx <= TILE_X && ty >= 1 && ty <= BY - 2;
  const int par = s6 & 1;
  const long long NS = sd.nsite;
  const S* __restrict__ gin = (const S*)sd.pop[par][0];
  S* __restrict__ gout = (S*)sd.pop[par ^ 1][0];
  const T* __restrict__ phin = (const T*)sd.phi[s6 % 3];
  const T* __restrict__ phim = (const T*)sd.phi[(s6 + 2) % 3];
  T* __restrict__ phinew = (T*)sd.phi[(s6 + 1) % 3];
  const T* __restrict__ Un = (const T*)sd.U[par];
  const T* __restrict__ thn = (const T*)sd.th[par];
  const bool has_th = sd.q_theta != 0;

  const int RW = 34, RH = BY + 2, RS = RW * RH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);        // phi^n     [3][RH][RW]
  T* ringm = ring + 3 * RS;                        // phi^{n-1} [3][RH][RW] (codec shift only)
  T* sG = ring + (C::shifted ? 6 : 3) * RS;        // post-collision [QP][BY][32]
  const int PS = BY * 32;

  const T inv2dx = (T)sd.inv2dx, c_eta = (T)sd.c_eta, c_N = (T)sd.c_N, dt_tau0 = (T)sd.dt_tau0;
  const T lamM = (T)sd.lamM, lam = (T)sd.lam, e1 = (T)sd.eps1, e2 = (T)sd.eps2, g2min = (T)sd.grad2_min;
  const T theta0 = (T)sd.theta0, scale = (T)sd.scale[0], iscale = (T)sd.inv_scale[0];
  const int kind = sd.aniso;

  const int zlo = max(it.z0 - 1, 0), zhi = min(it.z1, nz - 1);
  load_ring(ring + ring_slot(zlo - 1) * RS, phin, zlo - 1, it.x0, it.y0, nx, ny, nz, RW, RS, tid, nthr);
  load_ring(ring + ring_slot(zlo) * RS, phin, zlo, it.x0, it.y0, nx, ny, nz, RW, RS, tid, nthr);
  if (C::shifted) {
    load_ring(ringm + ring_slot(zlo - 1) * RS, phim, zlo - 1, it.x0, it.y0, nx, ny, nz, RW, RS, tid, nthr);
    load_ring(ringm + ring_slot(zlo) * RS, phim, zlo, it.x0, it.y0, nx, ny, nz, RW, RS, tid, nthr);
  }
  T acc0 = 0, acc1 = 0, acc2 = 0;  // moments of planes zc-1, zc, zc+1
  const int rc = (ty + 1) * RW + (tx + 1);  // this node's ring offset

  for (int zc = zlo; zc <= zhi; ++zc) {
    load_ring(ring + ring_slot(zc + 1) * RS, phin, zc + 1, it.x0, it.y0, nx, ny, nz, RW, RS, tid, nthr);
    if (C::shifted)
      load_ring(ringm + ring_slot(zc + 1) * RS, phim, zc + 1, it.x0, it.y0, nx, ny, nz, RW, RS, tid, nthr);
    __syncthreads();
    const T* R0 = ring + ring_slot(zc) * RS;
    if (in_xy) {
      const T* Rp = ring + ring_slot(zc + 1) * RS;
      const T* Rm = ring + ring_slot(zc - 1) * RS;
      const long long site = ((long long)zc * ny + y) * nx + x;
      const T ph = R0[rc];
      // centred gradient with mirror ghosts (clamped ring)
      const T gx = (R0[rc + 1] - R0[rc - 1]) * inv2dx;
      const T gy = (R0[rc + RW] - R0[rc - RW]) * inv2dx;
      const T gz = (Rp[rc] - Rm[rc]) * inv2dx;
      const T G2 = gx * gx + gy * gy + gz * gz;
      T as = 1, Nx = 0, Ny = 0, Nz = 0;
      if (G2 >= g2min) as = aniso_N<T>(kind, e1, e2, gx, gy, gz, G2, Nx, Ny, Nz);
      const T as2 = as * as;
      const T inv_eta = T(1) / (c_eta * as2 + T(0.5));
      const T omp2 = T(1) - ph * ph;
      const T th = has_th ? thn[site] : theta0;
      const T Qdt = (ph - (lamM * Un[site] + lam * th) * omp2) * omp2 * dt_tau0;
      const bool bnd = x == 0 || y == 0 || zc == 0 || x == nx - 1 || y == ny - 1 || zc == nz - 1;
      const T a2 = bnd ? T(1) : as2;
      const T inv_a2 = T(1) / a2;
      const T oma2 = T(1) - a2;
      const bool store = icol && zc >= it.z0 && zc < it.z1;
      const T* RmP = ringm + ring_slot(zc) * RS;
#pragma unroll
      for (int i = 0; i < QP; ++i) {
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        const T wi = (T)L::w(i);
        const int sx = x - ex, sy = y - ey, sz = zc - ez;
        const bool inside = sx >= 0 && sx < nx && sy >= 0 && sy < ny && sz >= 0 && sz < nz;
        const long long src = inside ? site - ((long long)ez * ny + ey) * nx - ex : site;
        const int ii = inside ? i : L::opp(i);
        T shift_in = 0, shift_nl = 0;
        if (C::shifted) {
          const T* Rs = ringm + ring_slot(inside ? sz : zc) * RS;
          shift_in = wi * Rs[inside ? rc - ey * RW - ex : rc];
          shift_nl = wi * RmP[rc];
        }
        const T gpull = C::dec(gin[(long long)ii * NS + src], shift_in, iscale);
        const T gnl = bnd ? T(0) : C::dec(gin[(long long)i * NS + site], shift_nl, iscale);
        const T eN = (T)ex * Nx + (T)ey * Ny + (T)ez * Nz;
        const T g0 = wi * (ph - eN * c_N);
        const T gs = (gpull - oma2 * gnl - (gpull - g0) * inv_eta + wi * Qdt) * inv_a2;
        const T shift_out = C::shifted ? wi * ph : T(0);
        const auto enc = C::enc(gs, shift_out, scale);
        if (store) gout[(long long)i * NS + site] = enc;
        sG[i * PS + tid] = C::shifted ? C::dec(enc, shift_out, iscale) : gs;
      }
    }
    __syncthreads();
    if (icol) {
#pragma unroll
      for (int i = 0; i < QP; ++i) {
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        const int sx = x - ex, sy = y - ey, sz = zc - ez;
        const bool sin_xy = sx >= 0 && sx < nx && sy >= 0 && sy < ny;
        if (sin_xy) {
          const T v = sG[i * PS + tid - ey * 32 - ex];
          if (ez == 0) acc1 += v;
          else if (ez > 0) acc2 += v;
          else acc0 += v;
        }
        if (!sin_xy || sz < 0 || sz >= nz) acc1 += sG[L::opp(i) * PS + tid];
      }
      const int zw = zc - 1;
      if (zw >= it.z0 && zw < it.z1 && zw >= 0) phinew[((long long)zw * ny + y) * nx + x] = acc0;
    }
    acc0 = acc1;
    acc1 = acc2;
    acc2 = 0;
  }
  if (icol && zhi == nz - 1 && zhi >= it.z0 && zhi < it.z1) phinew[((long long)zhi * ny + y) * nx + x] = acc0;
}

// ---------------------------------------------------------------- U and theta
template <int QU, int QT, typename S>
__global__ void __launch_bounds__(512) k_uth(const SimDev* __restrict__ sims, const WorkItem* __restrict__ items,
                                             int s6) {
  using C = Codec<S>;
  using T = typename C::T;
  using LU = Lat<QU>;
  using LT = Lat<(QT > 0 ? QT : 7)>;
  const WorkItem it = items[blockIdx.x];
  const SimDev& sd = sims[it.sim];
  const int nx = sd.nx, ny = sd.ny, nz = sd.nz;
  const int BY = blockDim.y;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx, nthr = 32 * BY;
  const int x = it.x0 - 1 + tx, y = it.y0 - 1 + ty;
  const bool in_xy = x >= 0 && x < nx && y >= 0 && y < ny;
  const bool icol = in_xy && tx >= 1 && tx <= TILE_X && ty >= 1 && ty <= BY - 2;
  const int par = s6 & 1;
  const long long NS = sd.nsite;
  const S* __restrict__ hin = (const S*)sd.pop[par][1];
  S* __restrict__ hout = (S*)sd.pop[par ^ 1][1];
  const S* __restrict__ fin = (const S*)sd.pop[par][2];
  S* __restrict__ fout = (S*)sd.pop[par ^ 1][2];
  const T* __restrict__ phin = (const T*)sd.phi[s6 % 3];
  const T* __restrict__ phi1 = (const T*)sd.phi[(s6 + 1) % 3];
  const T* __restrict__ Un = (const T*)sd.U[par];
  T* __restrict__ Unew = (T*)sd.U[par ^ 1];
  const T* __restrict__ thn = (const T*)sd.th[par];
  T* __restrict__ thnew = (T*)sd.th[par ^ 1];

  const int RW = 34, RH = BY + 2, RS = RW * RH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);  // phi^{n+1} [3][RH][RW]
  T* sH = ring + 3 * RS;                     // [QU][BY][32]
  const int PS = BY * 32;
  T* sF = sH + QU * PS;                      // [QT][BY][32]

  const T inv2dx = (T)sd.inv2dx, k = (T)sd.k, inv_etaU = (T)sd.inv_etaU, c_J = (T)sd.c_J;
  const T D_dx2 = (T)sd.D_dx2, D = (T)sd.D, at_amp = (T)sd.at_amp, inv_dt = (T)sd.inv_dt, dt = (T)sd.dt;
  const T g2min = (T)sd.grad2_min, inv_etaT = (T)sd.inv_etaT;
  const T sh_h = (T)sd.shift_h, sc_h = (T)sd.scale[1], isc_h = (T)sd.inv_scale[1];
  const T sh_f = (T)sd.shift_f, sc_f = (T)sd.scale[2], isc_f = (T)sd.inv_scale[2];
  const bool at_on = sd.antitrapping != 0;
  const T opk = T(1) + k, omk = T(1) - k;

  const int zlo = max(it.z0 - 1, 0), zhi = min(it.z1, nz - 1);
  load_ring(ring + ring_slot(zlo - 1) * RS, phi1, zlo - 1, it.x0, it.y0, nx, ny, nz, RW, RS, tid, nthr);
  load_ring(ring + ring_slot(zlo) * RS, phi1, zlo, it.x0, it.y0, nx, ny, nz, RW, RS, tid, nthr);
  T u0 = 0, u1 = 0, u2 = 0, t0 = 0, t1 = 0, t2 = 0;
  const int rc = (ty + 1) * RW + (tx + 1);

  for (int zc = zlo; zc <= zhi; ++zc) {
    load_ring(ring + ring_slot(zc + 1) * RS, phi1, zc + 1, it.x0, it.y0, nx, ny, nz, RW, RS, tid, nthr);
    __syncthreads();
    if (in_xy) {
      const T* R0 = ring + ring_slot(zc) * RS;
      const T* Rp = ring + ring_slot(zc + 1) * RS;
      const T* Rm = ring + ring_slot(zc - 1) * RS;
      const long long site = ((long long)zc * ny + y) * nx + x;
      // phi^{n+1} at the node and its six neighbours (mirror ghosts)
      const T pc = R0[rc];
      const T pxp = R0[rc + 1], pxm = R0[rc - 1], pyp = R0[rc + RW], pym = R0[rc - RW], pzp = Rp[rc], pzm = Rm[rc];
      // q(phi) = (1 - phi)/2, zeta(phi) = ((1+k) - (1-k) phi)/2
      auto qf = [&](T p) { return T(0.5) * (T(1) - p); };
      auto izf = [&](T p) { return T(2) / (opk - omk * p); };
      const T qc = qf(pc), izc = izf(pc), qzc = qc * izc;
      const T iz_xp = izf(pxp), iz_xm = izf(pxm), iz_yp = izf(pyp), iz_ym = izf(pym), iz_zp = izf(pzp),
              iz_zm = izf(pzm);
      const T gpx = (pxp - pxm) * inv2dx, gpy = (pyp - pym) * inv2dx, gpz = (pzp - pzm) * inv2dx;
      const T Fx = (iz_xp - iz_xm) * inv2dx, Fy = (iz_yp - iz_ym) * inv2dx, Fz = (iz_zp - iz_zm) * inv2dx;
      const T gqzx = (qf(pxp) * iz_xp - qf(pxm) * iz_xm) * inv2dx;
      const T gqzy = (qf(pyp) * iz_yp - qf(pym) * iz_ym) * inv2dx;
      const T gqzz = (qf(pzp) * iz_zp - qf(pzm) * iz_zm) * inv2dx;
      // div(D q grad(1/zeta)) in compact face form, face q = mean of nodal q
      const T divDqF = D_dx2 * (T(0.5) * (qc + qf(pxp)) * (iz_xp - izc) - T(0.5) * (qc + qf(pxm)) * (izc - iz_xm) +
                                T(0.5) * (qc + qf(pyp)) * (iz_yp - izc) - T(0.5) * (qc + qf(pym)) * (izc - iz_ym) +
                                T(0.5) * (qc + qf(pzp)) * (iz_zp - izc) - T(0.5) * (qc + qf(pzm)) * (izc - iz_zm));
      const T U = Un[site];
      const T dphi = pc - phin[site];  // phi^{n+1} - phi^n
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
#pragma unroll
      for (int i = 0; i < QU; ++i) {
        const int ex = LU::ex(i), ey = LU::ey(i), ez = LU::ez(i);
        const T wi = (T)LU::w(i);
        const int sx = x - ex, sy = y - ey, sz = zc - ez;
        const bool inside = sx >= 0 && sx < nx && sy >= 0 && sy < ny && sz >= 0 && sz < nz;
        const long long src = inside ? site - ((long long)ez * ny + ey) * nx - ex : site;
        const int ii = inside ? i : LU::opp(i);
        const T sh = C::shifted ? wi * sh_h : T(0);
        const T hp = C::dec(hin[(long long)ii * NS + src], sh, isc_h);
        const T eJ = (T)ex * Jx + (T)ey * Jy + (T)ez * Jz;
        const T h0 = (i == 0 ? U : T(0)) + (T)LU::B(i) * (qzU + eJ * c_J);
        const T hs = hp - (hp - h0) * inv_etaU + wi * src_dt;
        const auto enc = C::enc(hs, sh, sc_h);
        if (store) hout[(long long)i * NS + site] = enc;
        sH[i * PS + tid] = C::shifted ? C::dec(enc, sh, isc_h) : hs;
      }
      if (QT > 0) {
        const T th = thn[site];
        const T qth_dt = T(0.5) * dphi;  // w_i Q_theta dt with Q_theta = dphi/dt / 2
#pragma unroll
        for (int i = 0; i < QT; ++i) {
          const int ex = LT::ex(i), ey = LT::ey(i), ez = LT::ez(i);
          const T wi = (T)LT::w(i);
          const int sx = x - ex, sy = y - ey, sz = zc - ez;
          const bool inside = sx >= 0 && sx < nx && sy >= 0 && sy < ny && sz >= 0 && sz < nz;
          const long long src = inside ? site - ((long long)ez * ny + ey) * nx - ex : site;
          const int ii = inside ? i : LT::opp(i);
          const T sh = C::shifted ? wi * sh_f : T(0);
          const T fp = C::dec(fin[(long long)ii * NS + src], sh, isc_f);
          const T fs = fp - (fp - wi * th) * inv_etaT + wi * qth_dt;
          const auto enc = C::enc(fs, sh, sc_f);
          if (store) fout[(long long)i * NS + site] = enc;
          sF[i * PS + tid] = C::shifted ? C::dec(enc, sh, isc_f) : fs;
        }
      }
    }
    __syncthreads();
    if (icol) {
#pragma unroll
      for (int i = 0; i < QU; ++i) {
        const int ex = LU::ex(i), ey = LU::ey(i), ez = LU::ez(i);
        const int sx = x - ex, sy = y - ey, sz = zc - ez;
        const bool sin_xy = sx >= 0 && sx < nx && sy >= 0 && sy < ny;
        if (sin_xy) {
          const T v = sH[i * PS + tid - ey * 32 - ex];
          if (ez == 0) u1 += v;
          else if (ez > 0) u2 += v;
          else u0 += v;
        }
        if (!sin_xy || sz < 0 || sz >= nz) u1 += sH[LU::opp(i) * PS + tid];
      }
      if (QT > 0) {
#pragma unroll
        for (int i = 0; i < QT; ++i) {
          const int ex = LT::ex(i), ey = LT::ey(i), ez = LT::ez(i);
          const int sx = x - ex, sy = y - ey, sz = zc - ez;
          const bool sin_xy = sx >= 0 && sx < nx && sy >= 0 && sy < ny;
          if (sin_xy) {
            const T v = sF[i * PS + tid - ey * 32 - ex];
            if (ez == 0) t1 += v;
            else if (ez > 0) t2 += v;
            else t0 += v;
          }
          if (!sin_xy || sz < 0 || sz >= nz) t1 += sF[LT::opp(i) * PS + tid];
        }
      }
      const int zw = zc - 1;
      if (zw >= it.z0 && zw < it.z1 && zw >= 0) {
        const long long sw = ((long long)zw * ny + y) * nx + x;
        Unew[sw] = u0;
        if (QT > 0) thnew[sw] = t0;
      }
    }
    u0 = u1; u1 = u2; u2 = 0;
    t0 = t1; t1 = t2; t2 = 0;
  }
  if (icol && zhi == nz - 1 && zhi >= it.z0 && zhi < it.z1) {
    const long long sw = ((long long)zhi * ny + y) * nx + x;
    Unew[sw] = u0;
    if (QT > 0) thnew[sw] = t0;
  }
}

}  // namespace lbpf
