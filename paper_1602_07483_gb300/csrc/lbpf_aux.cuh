// lbpf_aux.cuh -- initial condition, state import/export between the
// post-streaming convention of the C ABI and the pull layout of the step
// kernels, moment export, FP64 reductions and tip tracking.  These kernels
// take the lattice as a runtime table (they are off the per-step path).
#pragma once

#include "lbpf_dev.cuh"

namespace lbpf {

struct LatRT {
  int q;
  int e[19][3];
  int opp[19];
  double w[19], B[19];
};

template <int Q>
inline LatRT make_lat_rt_q() {
  LatRT L{};
  L.q = Q;
  for (int i = 0; i < Q; ++i) {
    L.e[i][0] = Lat<Q>::ex(i);
    L.e[i][1] = Lat<Q>::ey(i);
    L.e[i][2] = Lat<Q>::ez(i);
    L.opp[i] = Lat<Q>::opp(i);
    L.w[i] = Lat<Q>::w(i);
    L.B[i] = Lat<Q>::B(i);
  }
  return L;
}

inline LatRT make_lat_rt(int q) {
  switch (q) {
    case 5: return make_lat_rt_q<5>();
    case 7: return make_lat_rt_q<7>();
    case 9: return make_lat_rt_q<9>();
    case 15: return make_lat_rt_q<15>();
    default: return make_lat_rt_q<19>();
  }
}

__device__ __forceinline__ bool in_dom(int x, int y, int z, int nx, int ny, int nz) {
  return x >= 0 && y >= 0 && z >= 0 && x < nx && y < ny && z < nz;
}

// phi of the diffuse seeds (Sec. 4): tanh((R - r) dx / (sqrt2 W0)), max over seeds
// (tanh is increasing, so one tanh of the largest argument).
template <typename T>
__global__ void k_init_scalar(int nx, int ny, int nz, const double* __restrict__ cen, const double* __restrict__ rad,
                              int nseed, double c, T* __restrict__ out) {
  const long long n = (long long)nx * ny * nz;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % nx);
    const int y = (int)((s / nx) % ny);
    const int z = (int)(s / ((long long)nx * ny));
    double arg = 0.0;
    for (int m = 0; m < nseed; ++m) {
      const double a = x - cen[3 * m], b = y - cen[3 * m + 1], d = z - cen[3 * m + 2];
      const double v = (rad[m] - sqrt(a * a + b * b + d * d)) * c;
      if (m == 0 || v > arg) arg = v;
    }
    out[s] = (T)(nseed > 0 ? tanh(arg) : -1.0);
  }
}

// Populations of the initial condition in pull layout:
// A_i(x) = (post-streaming value at x + e_i) or, for a wall link, the value at x.
template <typename S>
__global__ void k_init_pop(SimDev sd, LatRT Lp, LatRT Lu, LatRT Lt, const typename Codec<S>::T* __restrict__ phi0,
                           double U0, double theta0) {
  using C = Codec<S>;
  using T = typename C::T;
  const int nx = sd.nx, ny = sd.ny, nz = sd.nz;
  const long long n = sd.nsite;
  S* g = (S*)sd.pop[0][0];
  S* h = (S*)sd.pop[0][1];
  S* f = (S*)sd.pop[0][2];
  T* phi = (T*)sd.phi[0];
  T* U = (T*)sd.U[0];
  T* th = (T*)sd.th[0];
  const T k = (T)sd.k;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % nx);
    const int y = (int)((s / nx) % ny);
    const int z = (int)(s / ((long long)nx * ny));
    const T px = phi0[s];
    T mphi = 0, mU = 0, mth = 0;
    for (int i = 0; i < Lp.q; ++i) {
      const int a = x + Lp.e[i][0], b = y + Lp.e[i][1], c = z + Lp.e[i][2];
      const T pn = in_dom(a, b, c, nx, ny, nz) ? phi0[((long long)c * ny + b) * nx + a] : px;
      const T wi = (T)Lp.w[i];
      g[(long long)i * n + s] = C::enc(wi * pn, wi * px, (T)sd.scale[0]);
      mphi += wi * px;
    }
    for (int i = 0; i < Lu.q; ++i) {
      const int a = x + Lu.e[i][0], b = y + Lu.e[i][1], c = z + Lu.e[i][2];
      const T pn = in_dom(a, b, c, nx, ny, nz) ? phi0[((long long)c * ny + b) * nx + a] : px;
      const T Ai = i == 0 ? T(1) : T(0);
      const T qz = T(0.5) * (T(1) - pn) / (T(0.5) * ((T(1) + k) - (T(1) - k) * pn));
      const T qzx = T(0.5) * (T(1) - px) / (T(0.5) * ((T(1) + k) - (T(1) - k) * px));
      h[(long long)i * n + s] = C::enc((Ai + (T)Lu.B[i] * qz) * (T)U0, (T)Lu.w[i] * (T)sd.shift_h, (T)sd.scale[1]);
      mU += (Ai + (T)Lu.B[i] * qzx) * (T)U0;
    }
    for (int i = 0; i < Lt.q; ++i) {
      const T wi = (T)Lt.w[i];
      f[(long long)i * n + s] = C::enc(wi * (T)theta0, wi * (T)sd.shift_f, (T)sd.scale[2]);
      mth += wi * (T)theta0;
    }
    phi[s] = mphi;
    U[s] = mU;
    if (Lt.q) th[s] = mth;
  }
}

// acc[x] += p[x]
static __global__ void k_acc(double* __restrict__ acc, const double* __restrict__ p, long long n) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x)
    acc[s] += p[s];
}

template <typename T>
__global__ void k_from_double(T* __restrict__ out, const double* __restrict__ in, long long n) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x)
    out[s] = (T)in[s];
}

template <typename T>
__global__ void k_to_double(double* __restrict__ out, const T* __restrict__ in, long long n) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x)
    out[s] = (double)in[s];
}

// Post-streaming populations (host convention) -> pull layout, for the pair
// (i, j = opp(i)).  FP16/BF16 codec shift of the value stored at x: w_i prev(x) for g and f
// (prev = phi^{n-1}, theta^{n-1}), the constant w_i U0 for h.
template <typename S>
__global__ void k_pack(SimDev sd, int field, int par, LatRT L, int i, const double* __restrict__ gi,
                       const double* __restrict__ gj, const typename Codec<S>::T* __restrict__ prev) {
  using C = Codec<S>;
  using T = typename C::T;
  const int nx = sd.nx, ny = sd.ny, nz = sd.nz;
  const long long n = sd.nsite;
  S* A = (S*)sd.pop[par][field];
  const int j = L.opp[i];
  const T wi = (T)L.w[i];
  const T cshift = field == 1 ? (T)sd.shift_h : (T)sd.shift_f;
  const T scale = (T)sd.scale[field];
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % nx);
    const int y = (int)((s / nx) % ny);
    const int z = (int)(s / ((long long)nx * ny));
    const T sh = C::shifted ? (field != 1 ? wi * prev[s] : wi * cshift) : T(0);
    {
      const int a = x + L.e[i][0], b = y + L.e[i][1], c = z + L.e[i][2];
      const double v = in_dom(a, b, c, nx, ny, nz) ? gi[((long long)c * ny + b) * nx + a] : gj[s];
      A[(long long)i * n + s] = C::enc64(v, (double)sh, (double)scale);
    }
    if (j != i) {
      const int a = x + L.e[j][0], b = y + L.e[j][1], c = z + L.e[j][2];
      const double v = in_dom(a, b, c, nx, ny, nz) ? gj[((long long)c * ny + b) * nx + a] : gi[s];
      A[(long long)j * n + s] = C::enc64(v, (double)sh, (double)scale);
    }
  }
}

// Pull layout -> post-streaming populations for the pair (i, opp(i)).
template <typename S>
__global__ void k_unpack(SimDev sd, int field, int par, LatRT L, int i, double* __restrict__ gi,
                         double* __restrict__ gj, const typename Codec<S>::T* __restrict__ prev) {
  using C = Codec<S>;
  using T = typename C::T;
  const int nx = sd.nx, ny = sd.ny, nz = sd.nz;
  const long long n = sd.nsite;
  const S* A = (const S*)sd.pop[par][field];
  const int j = L.opp[i];
  const T wi = (T)L.w[i];
  const T cshift = field == 1 ? (T)sd.shift_h : (T)sd.shift_f;
  const T isc = (T)sd.inv_scale[field];
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % nx);
    const int y = (int)((s / nx) % ny);
    const int z = (int)(s / ((long long)nx * ny));
    for (int pass = 0; pass < (j != i ? 2 : 1); ++pass) {
      const int d = pass == 0 ? i : j, o = pass == 0 ? j : i;
      const int a = x - L.e[d][0], b = y - L.e[d][1], c = z - L.e[d][2];
      const bool ins = in_dom(a, b, c, nx, ny, nz);
      const long long src = ins ? ((long long)c * ny + b) * nx + a : s;
      const T sh = C::shifted ? (field != 1 ? wi * prev[src] : wi * cshift) : T(0);
      const double v = C::dec64(A[(long long)(ins ? d : o) * n + src], (double)sh, (double)isc);
      (pass == 0 ? gi : gj)[s] = v;
    }
  }
}

// h + l += x for a float-float accumulator (h, l): an error-free sum of h and x (TwoSum,
// Knuth) whose rounding error goes into l.  The explicit _rn operations keep the compiler
// from contracting or reordering them.
__device__ __forceinline__ void ff_acc(float& h, float& l, float x) {
  const float s = __fadd_rn(h, x);
  const float bp = __fsub_rn(s, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  h = s;
  l = __fadd_rn(l, err);
}

// FP64 partial sums per block: [sum phi, sum U, sum theta, sum phi U].
template <typename T>
__global__ void k_sums(const T* __restrict__ phi, const T* __restrict__ U, const T* __restrict__ th, double theta0,
                       double k, long long n, double* __restrict__ part) {
  // sum phi, sum U, sum theta and sum phi U; the total solute follows from them (k_sums_final)
  double a = 0, b = 0, c = 0, e = 0;
  if constexpr (sizeof(T) == 8) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
      const double p = (double)phi[s], u = (double)U[s];
      a += p;
      b += u;
      if (th) c += (double)th[s];
      e = fma(p, u, e);
    }
  } else {
    // FP32 fields: each thread accumulates in float-float (about 48 significant bits; the
    // product phi U is split exactly into p u + fma(p, u, -p u)), which uses the FP32 pipes
    // instead of GB300's narrow FP64 pipe; the partials are then reduced in FP64
    float ah = 0, al = 0, bh = 0, bl = 0, ch = 0, cl = 0, eh = 0, el = 0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
      const float p = (float)phi[s], u = (float)U[s];
      ff_acc(ah, al, p);
      ff_acc(bh, bl, u);
      if (th) ff_acc(ch, cl, (float)th[s]);
      const float pr = __fmul_rn(p, u);
      ff_acc(eh, el, pr);
      el = __fadd_rn(el, fmaf(p, u, -pr));
    }
    a = (double)ah + (double)al;
    b = (double)bh + (double)bl;
    c = (double)ch + (double)cl;
    e = (double)eh + (double)el;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
    e += __shfl_down_sync(0xffffffffu, e, o);
  }
  __shared__ double red[32][4];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[wid][0] = a; red[wid][1] = b; red[wid][2] = c; red[wid][3] = e;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
    part[blockIdx.x * 4 + threadIdx.x] = t;
  }
}

// Sum the per-block partials in a fixed order (deterministic).  The total solute
// sum zeta(phi) (1 + (1-k) U), zeta = ((1+k) - (1-k) phi)/2, expands to
// ((1+k) n + (1-k^2) sum U - (1-k) sum phi - (1-k)^2 sum phi U) / 2; theta frozen at
// theta0 sums to n theta0.
static __global__ void k_sums_final(const double* __restrict__ part, int nblk, double* __restrict__ out, double k,
                                    long long n, int frozen_theta, double theta0) {
  __shared__ double t4[4];
  if (threadIdx.x < 4) {
    double t = 0;
    for (int b = 0; b < nblk; ++b) t += part[b * 4 + threadIdx.x];
    t4[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double dn = (double)n;
    out[0] = t4[0];
    out[1] = t4[1];
    out[2] = frozen_theta ? dn * theta0 : t4[2];
    out[3] = 0.5 * ((1.0 + k) * dn + (1.0 - k * k) * t4[1] - (1.0 - k) * t4[0] - (1.0 - k) * (1.0 - k) * t4[3]);
  }
}

// Tip tracking along +axis (0, 1, 2 = x, y, z of the kernel grid) from node c.  Warp r
// scans line r from c[axis] for the first crossing phi_i >= 0 > phi_{i+1}: line 0 passes
// through c; lines 1..8 are offset by j = +-1..+-4 along the first other axis b1, lines
// 9..16 along the second other axis b2.  Thread 0 then fits the parabola
// t(j) = t_tip - j^2/(2 rho) in each plane (axis, b) whose extent along b is more than one
// node and averages the planes.
template <typename T>
__global__ void k_tip(const T* __restrict__ phi, int nx, int ny, int nz, int axis, int cx, int cy, int cz,
                      double* __restrict__ out) {
  __shared__ double cross[17];
  const int r = threadIdx.y, lane = threadIdx.x;
  const int n[3] = {nx, ny, nz};
  const int b1 = axis == 0 ? 1 : 0, b2 = axis == 2 ? 1 : 2;
  int p[3] = {cx, cy, cz};
  if (r >= 1 && r <= 8) p[b1] += (r <= 4) ? r : -(r - 4);
  else if (r >= 9) p[b2] += (r <= 12) ? (r - 8) : -(r - 12);
  double res = -1.0;
  if (p[0] >= 0 && p[0] < nx && p[1] >= 0 && p[1] < ny && p[2] >= 0 && p[2] < nz) {
    const long long stride = axis == 0 ? 1 : (axis == 1 ? (long long)nx : (long long)nx * ny);
    p[axis] = 0;
    const long long line = ((long long)p[2] * ny + p[1]) * nx + p[0];
    const int len = n[axis];
    for (int base = axis == 0 ? cx : (axis == 1 ? cy : cz); base + 1 < len; base += 32) {
      const int ti = base + lane;
      bool hit = false;
      T a = 0, b = 0;
      if (ti + 1 < len) {
        a = phi[line + ti * stride];
        b = phi[line + (ti + 1) * stride];
        hit = a >= T(0) && b < T(0);
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (m) {
        const int first = __ffs(m) - 1;
        const double av = __shfl_sync(0xffffffffu, (double)a, first);
        const double bv = __shfl_sync(0xffffffffu, (double)b, first);
        res = (base + first) + av / (av - bv);
        break;
      }
    }
  }
  if (lane == 0) cross[r] = res;
  __syncthreads();
  if (r == 0 && lane == 0) {
    const double tt = cross[0];
    double sum = 0.0;
    int planes = 0;
    bool ok_all = true;
    for (int plane = 0; plane < 2; ++plane) {
      if (n[plane == 0 ? b1 : b2] == 1) continue;  // no such plane on this grid
      double num = 0, den = 0;
      bool ok = tt >= 0;
      for (int q = 0; q < 8; ++q) {
        const int j = q < 4 ? q + 1 : -(q - 3);
        const double tj = cross[1 + plane * 8 + q];
        if (tj < 0) ok = false;
        num += (double)(j * j) * (tt - tj);
        den += (double)(j * j) * (double)(j * j);
      }
      if (ok && num > 0) sum += den / (2.0 * num);
      else ok_all = false;
      ++planes;
    }
    out[0] = tt;
    out[1] = (planes > 0 && ok_all) ? sum / planes : -1.0;
  }
}

}  // namespace lbpf
