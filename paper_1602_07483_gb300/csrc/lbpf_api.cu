// lbpf_api.cu -- host runtime behind the C ABI of include/lbpf.h.
//
// Owns the device state of a simulation, validates parameters, builds the
// tile work lists of the step kernels, captures the time loop in CUDA graphs
// (six steps per graph: populations alternate with period 2 and the phi levels
// with period 3), and moves state between the host convention
// (post-streaming populations, FP64) and the device pull layout.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/lbpf.h"
#include "lbpf_aux.cuh"
#include "lbpf_table.h"

using namespace lbpf;

namespace {

constexpr int kGraphSteps = 6;
constexpr unsigned kWaitPolls = 1u << 22;  // default bound of a one-launch wait: about a second
#ifndef LBPF_ONE_LAUNCH_LAG_PCT
#define LBPF_ONE_LAUNCH_LAG_PCT 100  // lag of the one-launch schedule, % of the resident blocks
#endif

// table slots: phi and U take a moving lattice, theta may also be 0 (frozen)
int q_index(int q) {
  const int s = lattice_slot(q);
  return (s >= 0 && s < 5) ? s : -1;
}
int qt_index(int q) { return lattice_slot(q); }
double lattice_e2(int q) { return q == 7 ? 0.25 : 1.0 / 3.0; }

const KernelTable* table_for(int storage) {
  switch (storage) {
    case LBPF_F64: return &table_f64();
    case LBPF_F32: return &table_f32();
    case LBPF_F16: return &table_f16();
    case LBPF_BF16: return &table_bf16();
    default: return nullptr;
  }
}

// a_s(n) of the two anisotropy functions (Eq. Anisotropic-Function_As, Eq. As_K41-K61)
double aniso_host(int kind, double e1, double e2, double nx, double ny, double nz) {
  const double r = sqrt(nx * nx + ny * ny + nz * nz);
  nx /= r; ny /= r; nz /= r;
  const double s4 = nx * nx * nx * nx + ny * ny * ny * ny + nz * nz * nz * nz;
  if (kind == 0) return 1.0 - 3.0 * e1 + 4.0 * e1 * s4;
  const double p3 = nx * nx * ny * ny * nz * nz;
  return 1.0 + e1 * (s4 - 0.6) + e2 * (3.0 * s4 + 66.0 * p3 - 17.0 / 7.0);
}

// Smallest a_s^2 eta_phi(a_s) over interface orientations.  The non-local
// collision relaxes a uniform perturbation at the rate 1/(a_s^2 eta_phi), which
// must stay below 2.  Sampled on a fine grid of the unit sphere (a_s is smooth).
double min_effective_tau(int kind, double e1, double e2, double c_eta, double* amin_out) {
  double best = 1e300, amin = 1e300;
  const int NT = 181, NP = 360;
  for (int it = 0; it < NT; ++it) {
    const double th = M_PI * it / (NT - 1);
    for (int ip = 0; ip < NP; ++ip) {
      const double ph = 2.0 * M_PI * ip / NP;
      const double a = aniso_host(kind, e1, e2, sin(th) * cos(ph), sin(th) * sin(ph), cos(th) + 1e-300);
      const double a2 = a * a;
      best = std::min(best, a2 * (c_eta * a2 + 0.5));
      amin = std::min(amin, a);
    }
  }
  // the cube diagonal exactly
  const double a = aniso_host(kind, e1, e2, 1, 1, 1);
  best = std::min(best, a * a * (c_eta * a * a + 0.5));
  amin = std::min(amin, a);
  if (amin_out) *amin_out = amin;
  return best;
}

}  // namespace

// The one-launch schedule of a tiling (k_step): the ticket order and the dependency lists on
// the device, the ticket counter and done flags (zeroed before each launch), and the
// host-visible flag of the bounded waits.
struct OneLaunch {
  OneLaunchFn fn = nullptr;   // null: no one-launch kernel for these lattices and storage
  bool on = false;            // schedule selected (lbpf_set_schedule)
  int* d_sched = nullptr;     // order[ntickets] | dep_off[nitems + 1] | dep[...]
  unsigned* d_ctl = nullptr;  // next ticket, then one done flag per work item
  size_t ctl_bytes = 0;
  int* h_err = nullptr;       // mapped host memory, written by the device
  StepSched sc{};
  int grid = 0;               // resident blocks on the device
  size_t smem = 0;
  unsigned polls = kWaitPolls;  // bound of each wait (lbpf_set_wait_polls)
};

struct lbpf_sim {
  lbpf_grid g{};
  lbpf_grid kg{};  // grid as the kernels see it: g, or (nx, 1, ny) for the 2D lattices (paper's y on the z axis)
  lbpf_lattice lat{};
  lbpf_params p{};
  const KernelTable* kt = nullptr;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  long long nsite = 0;
  void* pop[2][3] = {};
  void* phi[3] = {};
  void* U[2] = {};
  void* th[3] = {};  // theta levels like phi (theta^{n-1} is the FP16/BF16 shift of f)
  SimDev hd{};
  SimDev* dd = nullptr;
  WorkItem* d_items = nullptr;
  int nitems = 0;
  int by = MAX_BLOCK_ROWS, zchunk = 0;
  double* d_part = nullptr;  // reduction partials + 4 results
  int npart = 0;
  double* d_small = nullptr; // tip output
  double* h_small = nullptr; // pinned
  double* d_tmp = nullptr;   // FP64 staging (3 x nsite), allocated on demand
  cudaGraphExec_t gexec = nullptr;
  bool graph_ok = false;
  int64_t steps = 0;      // steps since the state was set; fixes buffer parity and phi level
  int64_t step_base = 0;  // step count carried in from a checkpoint
  int sticky = LBPF_OK;
  double theta0 = 0.0, U0 = 0.0;
  StepLaunch fphi = nullptr, futh = nullptr;
  size_t smem_phi = 0, smem_uth = 0;
  OneLaunch ol;
  const int* batch_err = nullptr;  // wait-failure flag of the batch this handle is stepped by
};

struct lbpf_batch {
  std::vector<lbpf_sim*> sims;
  bool owns_sims = false;       // members created by lbpf_batch_create (destroyed with the batch)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev = nullptr;     // orders the batch stream against the members' own streams
  SimDev* h_desc = nullptr;     // pinned copy of the member descriptors last uploaded to dd
  SimDev* dd = nullptr;
  WorkItem* d_items = nullptr;
  int nitems = 0;
  int by = MAX_BLOCK_ROWS;
  int zchunk = 0;               // z-chunk request of the current tiling (0: each member's default)
  StepLaunch fphi = nullptr, futh = nullptr;
  size_t smem_phi = 0, smem_uth = 0;
  OneLaunch ol;
  std::vector<int> zchunks;     // z-chunk of each member under the current tiling
  cudaGraphExec_t gexec = nullptr;
  bool graph_ok = false;
};

#define CK(sim, call)                                  \
  do {                                                 \
    cudaError_t e__ = (call);                          \
    if (e__ != cudaSuccess) {                          \
      if (sim) (sim)->sticky = LBPF_ECUDA;             \
      fprintf(stderr, "lbpf: CUDA error %s at %s:%d\n", cudaGetErrorString(e__), __FILE__, __LINE__); \
      return LBPF_ECUDA;                               \
    }                                                  \
  } while (0)

namespace {


// z-chunks of about 32 planes: enough thread blocks for several waves, and the
// blocks resident at any time work on neighbouring tiles, so the one-node
// halos they re-read are found in L2 (measured best at 512^3 on GB300)
int default_zchunk(int nx, int ny, int nz, int by) {
  (void)ny;
  if (by == 1) {
    // one-row (2D) blocks are single warps: chunks of 8 to 32 rows, short enough to give
    // about 24 blocks per SM of a 152-SM GB300 when the plane is small
    const int xt = (nx + TILE_X - 1) / TILE_X;
    const int want = (152 * 24 + xt - 1) / xt;
    return std::min(std::max(nz, 1), std::min(32, std::max(8, (nz + want - 1) / want)));
  }
  if (nz <= 48) return nz;
  const int chunks = (nz + 31) / 32;
  return (nz + chunks - 1) / chunks;
}

// The dynamic shared-memory limit is an attribute of the kernel, shared by every
// simulation that launches it: raise it once to the device's opt-in maximum so
// that no handle's tiling can lower it under another handle's launches.
int raise_smem_limit(const void* fn, int device) {
  int maxsm = 0;
  if (cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return LBPF_ECUDA;
  // the dynamic limit plus the kernel's static shared memory may not exceed the opt-in maximum
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return LBPF_ECUDA;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm - (int)fa.sharedSizeBytes) !=
      cudaSuccess)
    return LBPF_ECUDA;
  return LBPF_OK;
}

// The sticky error of a handle; a bounded wait of its one-launch step (or of the batch that
// steps it) that gave up makes it LBPF_ETIMEOUT.  The flags are in mapped host memory, so
// this reads them without synchronising (a failure shows at the latest after the next
// synchronising call).
int status(lbpf_sim* s) {
  if (s->sticky == LBPF_OK && ((s->ol.h_err && *(volatile const int*)s->ol.h_err) ||
                               (s->batch_err && *(volatile const int*)s->batch_err)))
    s->sticky = LBPF_ETIMEOUT;
  return s->sticky;
}

// The bounded wait of the one-launch step on its own: one warp waits for flag[dep[0]] with at
// most `polls` rounds and writes 1 to *out if it saw the flag set, 0 if it gave up.
__global__ void k_wait_probe(const unsigned* flag, const int* dep, unsigned polls, int* out) {
  const bool ok = wait_done(flag, dep, 1, polls);
  if (threadIdx.x == 0) *out = ok ? 1 : 0;
}

void free_one_launch(OneLaunch& ol) {
  if (ol.d_sched) cudaFree(ol.d_sched);
  if (ol.d_ctl) cudaFree(ol.d_ctl);
  ol.d_sched = nullptr;
  ol.d_ctl = nullptr;
  ol.sc = StepSched{};
}

// (Re)builds the one-launch schedule of `items` on the device.  Synchronous.
int setup_one_launch(OneLaunch& ol, const std::vector<WorkItem>& items, const std::vector<TileGeom>& geo, int by,
                     size_t smem, const void* fn, int device) {
  free_one_launch(ol);
  if (!ol.h_err) {
    if (cudaHostAlloc(&ol.h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();
      ol.h_err = nullptr;
      return LBPF_ENOMEM;
    }
    *ol.h_err = 0;
  }
  int* d_err = nullptr;
  if (cudaHostGetDevicePointer((void**)&d_err, ol.h_err, 0) != cudaSuccess) return LBPF_ECUDA;
  int nb = 0, sms = 0;
  if (raise_smem_limit(fn, device) != LBPF_OK ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 32 * by, smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return LBPF_ECUDA;
  if (nb < 1) return LBPF_EINVAL;
  const int resident = nb * sms;
  // U/theta tickets trail their last phase-field tile by about one wave of resident blocks,
  // so that the tiles they wait for have normally finished when they start
  const int lag = (int)((long long)resident * LBPF_ONE_LAUNCH_LAG_PCT / 100);
  std::vector<int> order, dep_off, dep;
  if (!plan_one_launch(items, geo, by, lag, order, dep_off, dep)) return LBPF_EINVAL;
  const size_t n = items.size();
  std::vector<int> all;
  all.reserve(order.size() + dep_off.size() + dep.size());
  all.insert(all.end(), order.begin(), order.end());
  all.insert(all.end(), dep_off.begin(), dep_off.end());
  all.insert(all.end(), dep.begin(), dep.end());
  ol.ctl_bytes = (n + 1) * sizeof(unsigned);
  if (cudaMalloc(&ol.d_sched, all.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ol.d_ctl, ol.ctl_bytes) != cudaSuccess) {
    cudaGetLastError();
    free_one_launch(ol);
    return LBPF_ENOMEM;
  }
  if (cudaMemcpy(ol.d_sched, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    free_one_launch(ol);
    return LBPF_ECUDA;
  }
  ol.sc.order = ol.d_sched;
  ol.sc.dep_off = ol.d_sched + order.size();
  ol.sc.dep = ol.d_sched + order.size() + dep_off.size();
  ol.sc.ctl = ol.d_ctl;
  ol.sc.err = d_err;
  ol.sc.ntickets = (int)order.size();
  ol.sc.polls = ol.polls;
  ol.grid = std::min(resident, ol.sc.ntickets);
  ol.smem = smem;
  return LBPF_OK;
}

int set_smem_attrs(lbpf_sim* s) {
  const KernelTable& t = *s->kt;
  const int a = q_index(s->lat.q_phi), b = q_index(s->lat.q_u), c = qt_index(s->lat.q_theta);
  if (raise_smem_limit(t.phi_fn[a][0], s->device) || raise_smem_limit(t.uth_fn[b][c][0], s->device) ||
      raise_smem_limit(t.phi_fn[a][1], s->device) || raise_smem_limit(t.uth_fn[b][c][1], s->device)) {
    s->sticky = LBPF_ECUDA;
    return LBPF_ECUDA;
  }
  return LBPF_OK;
}

int apply_tiling(lbpf_sim* s, int by, int zchunk) {
  const KernelTable& t = *s->kt;
  if (lattice_is_2d(s->lat.q_phi)) by = 1;  // 2D: one-row blocks, no y halo
  s->by = by;
  const int v = block_variant(s->lat.q_phi, by);
  s->fphi = t.phi[q_index(s->lat.q_phi)][v];
  s->futh = t.uth[q_index(s->lat.q_u)][qt_index(s->lat.q_theta)][v];
  s->zchunk = zchunk > 0 ? zchunk : default_zchunk(s->kg.nx, s->kg.ny, s->kg.nz, by);
  s->smem_phi = phi_smem_bytes(t, s->lat.q_phi, by);
  s->smem_uth = uth_smem_bytes(t, s->lat.q_u, s->lat.q_theta, by);
  int maxsm = 0;
  CK(s, cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device));
  if ((int)s->smem_phi > maxsm || (int)s->smem_uth > maxsm) return LBPF_EINVAL;
  std::vector<WorkItem> items;
  build_items(0, s->kg.nx, s->kg.ny, s->kg.nz, by, s->zchunk, items);
  if (s->d_items) cudaFree(s->d_items);
  s->d_items = nullptr;
  CK(s, cudaMalloc(&s->d_items, items.size() * sizeof(WorkItem)));
  CK(s, cudaMemcpy(s->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
  s->nitems = (int)items.size();
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  s->gexec = nullptr;
  s->graph_ok = false;
  if (s->ol.on) {
    const int rc = setup_one_launch(s->ol, items, {TileGeom{s->kg.nx, s->kg.ny, s->kg.nz, s->zchunk}}, by,
                                    step_smem_bytes(t, s->lat.q_phi, s->lat.q_u, s->lat.q_theta, by),
                                    t.step_fn[q_index(s->lat.q_phi)][q_index(s->lat.q_u)][qt_index(s->lat.q_theta)],
                                    s->device);
    if (rc != LBPF_OK) return rc;
  }
  return set_smem_attrs(s);
}

// One step: the two kernels, or the one-launch kernel when `ol` is selected.
int launch_step(cudaStream_t st, StepLaunch fphi, StepLaunch futh, int nitems, int by, size_t smem_phi,
                size_t smem_uth, const SimDev* dd, const WorkItem* items, int s6, const OneLaunch* ol) {
  if (ol && ol->on) {
    if (cudaMemsetAsync(ol->d_ctl, 0, ol->ctl_bytes, st) != cudaSuccess) return LBPF_ECUDA;
    return ol->fn(dim3(ol->grid), dim3(32, by), ol->smem, st, dd, items, ol->sc, s6) == cudaSuccess ? LBPF_OK
                                                                                                 : LBPF_ECUDA;
  }
  cudaError_t e = fphi(dim3(nitems), dim3(32, by), smem_phi, st, dd, items, s6);
  if (e != cudaSuccess) return LBPF_ECUDA;
  e = futh(dim3(nitems), dim3(32, by), smem_uth, st, dd, items, s6);
  return e == cudaSuccess ? LBPF_OK : LBPF_ECUDA;
}

int capture_graph(cudaStream_t st, StepLaunch fphi, StepLaunch futh, int nitems, int by, size_t smem_phi,
                  size_t smem_uth, const SimDev* dd, const WorkItem* items, const OneLaunch* ol,
                  cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LBPF_ECUDA;
  int rc = LBPF_OK;
  for (int s6 = 0; s6 < kGraphSteps && rc == LBPF_OK; ++s6)
    rc = launch_step(st, fphi, futh, nitems, by, smem_phi, smem_uth, dd, items, s6, ol);
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (rc != LBPF_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return LBPF_ECUDA;
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  return e == cudaSuccess ? LBPF_OK : LBPF_ECUDA;
}

int ensure_tmp(lbpf_sim* s) {
  if (s->d_tmp) return LBPF_OK;
  if (cudaMalloc(&s->d_tmp, sizeof(double) * 3 * (size_t)s->nsite) != cudaSuccess) {
    cudaGetLastError();
    s->d_tmp = nullptr;
    return LBPF_ENOMEM;
  }
  return LBPF_OK;
}

int validate(const lbpf_grid* g, const lbpf_lattice* l, const lbpf_params* p) {
  if (!g || !l || !p) return LBPF_EINVAL;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return LBPF_EINVAL;
  // the step kernels address populations with 32-bit element offsets: Q * nsite < 2^32
  const long long nsite = (long long)g->nx * g->ny * g->nz;
  if (nsite * 19 >= (1LL << 32)) return LBPF_EINVAL;
  if (q_index(l->q_phi) < 0 || q_index(l->q_u) < 0 || qt_index(l->q_theta) < 0) return LBPF_EINVAL;
  // 2D lattices (D2Q5, D2Q9) run on an nz = 1 grid, all fields on 2D lattices
  const bool d2 = lattice_is_2d(l->q_phi);
  if (lattice_is_2d(l->q_u) != d2 || (l->q_theta && lattice_is_2d(l->q_theta) != d2)) return LBPF_EINVAL;
  if (d2 && g->nz != 1) return LBPF_EINVAL;
  if (!(p->W0 > 0) || !(p->tau0 > 0) || !(p->D > 0) || !(p->dx > 0) || !(p->dt > 0)) return LBPF_EINVAL;
  if (l->q_theta && !(p->kappa > 0)) return LBPF_EINVAL;
  if (!(p->k > 0) || !(p->k <= 1)) return LBPF_EINVAL;
  if (p->aniso != 0 && p->aniso != 1) return LBPF_EINVAL;
  if (!table_for(p->storage)) return LBPF_EINVAL;
  if (!isfinite(p->lambda) || !isfinite(p->Mc_inf) || !isfinite(p->eps1) || !isfinite(p->eps2)) return LBPF_EINVAL;
  if (p->grad2_min < 0) return LBPF_EINVAL;
  const double c_eta = p->W0 * p->W0 / p->tau0 * p->dt / (p->dx * p->dx) / lattice_e2(l->q_phi);
  double amin = 0;
  const double teff = min_effective_tau(p->aniso, p->eps1, p->eps2, c_eta, &amin);
  if (!(amin > 0) || !(teff > 0.5)) return LBPF_EUNSTABLE;
  return LBPF_OK;
}

void fill_dev(lbpf_sim* s) {
  const lbpf_params& p = s->p;
  SimDev& d = s->hd;
  d.nx = s->kg.nx; d.ny = s->kg.ny; d.nz = s->kg.nz;
  d.q_theta = s->lat.q_theta;
  d.nsite = s->nsite;
  for (int b = 0; b < 2; ++b)
    for (int f = 0; f < 3; ++f) d.pop[b][f] = s->pop[b][f];
  for (int l = 0; l < 3; ++l) d.phi[l] = s->phi[l];
  for (int b = 0; b < 2; ++b) d.U[b] = s->U[b];
  for (int l = 0; l < 3; ++l) d.th[l] = s->th[l];
  const double e2p = lattice_e2(s->lat.q_phi), e2u = lattice_e2(s->lat.q_u);
  const double W2t = p.W0 * p.W0 / p.tau0;
  d.inv2dx = 1.0 / (2.0 * p.dx);
  d.c_eta = W2t * p.dt / (p.dx * p.dx) / e2p;
  d.c_N = p.dt / p.dx * W2t / e2p;
  d.dt_tau0 = p.dt / p.tau0;
  d.lamM = p.lambda * p.Mc_inf;
  d.lam = p.lambda;
  d.eps1 = p.eps1; d.eps2 = p.eps2;
  d.grad2_min = p.grad2_min > 0 ? p.grad2_min : 1e-12;
  d.aniso = p.aniso;
  d.antitrapping = p.antitrapping ? 1 : 0;
  d.k = p.k;
  d.inv_etaU = 1.0 / (p.D * p.dt / (p.dx * p.dx) / e2u + 0.5);
  d.c_J = p.dt / p.dx / e2u;
  d.D_dx2 = p.D / (p.dx * p.dx);
  d.D = p.D;
  d.at_amp = p.W0 / (2.0 * sqrt(2.0));
  d.dt = p.dt;
  d.inv_dt = 1.0 / p.dt;
  d.inv_etaT = s->lat.q_theta ? 1.0 / (p.kappa * p.dt / (p.dx * p.dx) / lattice_e2(s->lat.q_theta) + 0.5) : 0.0;
  d.theta0 = s->theta0;
  d.shift_h = s->U0;
  d.shift_f = s->theta0;
  // codec scales: powers of two keeping the stored deviations well inside the FP16 range
  for (int f = 0; f < 3; ++f) {
    d.scale[f] = s->kt->shifted ? 4096.0 : 1.0;
    d.inv_scale[f] = 1.0 / d.scale[f];
  }
}

int upload_dev(lbpf_sim* s) {
  fill_dev(s);
  CK(s, cudaMemcpy(s->dd, &s->hd, sizeof(SimDev), cudaMemcpyHostToDevice));
  return LBPF_OK;
}

void free_sim(lbpf_sim* s) {
  if (!s) return;
  for (int b = 0; b < 2; ++b)
    for (int f = 0; f < 3; ++f) if (s->pop[b][f]) cudaFree(s->pop[b][f]);
  for (int l = 0; l < 3; ++l) if (s->phi[l]) cudaFree(s->phi[l]);
  for (int b = 0; b < 2; ++b)
    if (s->U[b]) cudaFree(s->U[b]);
  for (int l = 0; l < 3; ++l)
    if (s->th[l]) cudaFree(s->th[l]);
  if (s->dd) cudaFree(s->dd);
  if (s->d_items) cudaFree(s->d_items);
  if (s->d_part) cudaFree(s->d_part);
  if (s->d_small) cudaFree(s->d_small);
  if (s->h_small) cudaFreeHost(s->h_small);
  if (s->d_tmp) cudaFree(s->d_tmp);
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  free_one_launch(s->ol);
  if (s->ol.h_err) cudaFreeHost(s->ol.h_err);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

int aux_blocks_host(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)std::max<size_t>(1, std::min<size_t>(b, 152 * 32));
}

inline int s6_of(const lbpf_sim* s) { return (int)(s->steps % kGraphSteps); }
inline int par_of(const lbpf_sim* s) { return (int)(s->steps & 1); }

}  // namespace

extern "C" {

const char* lbpf_strerror(int code) {
  switch (code) {
    case LBPF_OK: return "ok";
    case LBPF_EINVAL: return "invalid argument";
    case LBPF_EUNSTABLE: return "unstable parameters: a relaxation time a_s^2 eta <= 1/2";
    case LBPF_ENOMEM: return "device allocation failed";
    case LBPF_ENAN: return "non-finite value in the fields";
    case LBPF_ECUDA: return "CUDA runtime error";
    case LBPF_ETIMEOUT: return "a bounded wait of the one-launch step gave up; the step's results are invalid";
    default: return "unknown error";
  }
}

int lbpf_create(const lbpf_grid* grid, const lbpf_lattice* lattice, const lbpf_params* params, void* cuda_stream,
                lbpf_sim** out) {
  if (!out) return LBPF_EINVAL;
  *out = nullptr;
  int rc = validate(grid, lattice, params);
  if (rc != LBPF_OK) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return LBPF_ECUDA;
  }
  lbpf_sim* s = new lbpf_sim();
  s->g = *grid;
  s->lat = *lattice;
  s->p = *params;
  s->kt = table_for(params->storage);
  s->nsite = (long long)grid->nx * grid->ny * grid->nz;
  s->kg = lattice_is_2d(lattice->q_phi) ? lbpf_grid{grid->nx, 1, grid->ny} : *grid;
  if (cudaGetDevice(&s->device) != cudaSuccess) { free_sim(s); return LBPF_ECUDA; }
  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) { free_sim(s); return LBPF_ECUDA; }
    s->own_stream = true;
  }
  const size_t N = (size_t)s->nsite;
  const int qs[3] = {lattice->q_phi, lattice->q_u, lattice->q_theta};
  bool ok = true;
  for (int b = 0; b < 2 && ok; ++b)
    for (int f = 0; f < 3 && ok; ++f)
      if (qs[f]) ok = cudaMalloc(&s->pop[b][f], (size_t)qs[f] * N * s->kt->sbytes) == cudaSuccess;
  for (int l = 0; l < 3 && ok; ++l) ok = cudaMalloc(&s->phi[l], N * s->kt->tbytes) == cudaSuccess;
  for (int b = 0; b < 2 && ok; ++b) ok = cudaMalloc(&s->U[b], N * s->kt->tbytes) == cudaSuccess;
  for (int l = 0; l < 3 && ok && lattice->q_theta; ++l) ok = cudaMalloc(&s->th[l], N * s->kt->tbytes) == cudaSuccess;
  s->npart = 1024;
  if (ok) ok = cudaMalloc(&s->d_part, sizeof(double) * (4 * s->npart + 8)) == cudaSuccess;
  if (ok) ok = cudaMalloc(&s->d_small, sizeof(double) * 8) == cudaSuccess;
  if (ok) ok = cudaMallocHost(&s->h_small, sizeof(double) * 8) == cudaSuccess;
  if (ok) ok = cudaMalloc(&s->dd, sizeof(SimDev)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_sim(s);
    return LBPF_ENOMEM;
  }
  // zero state until initialised
  for (int b = 0; b < 2; ++b)
    for (int f = 0; f < 3; ++f)
      if (s->pop[b][f]) cudaMemsetAsync(s->pop[b][f], 0, (size_t)qs[f] * N * s->kt->sbytes, s->stream);
  for (int l = 0; l < 3; ++l) cudaMemsetAsync(s->phi[l], 0, N * s->kt->tbytes, s->stream);
  for (int b = 0; b < 2; ++b) cudaMemsetAsync(s->U[b], 0, N * s->kt->tbytes, s->stream);
  for (int l = 0; l < 3; ++l)
    if (s->th[l]) cudaMemsetAsync(s->th[l], 0, N * s->kt->tbytes, s->stream);
  s->ol.fn = s->kt->step[q_index(lattice->q_phi)][q_index(lattice->q_u)][qt_index(lattice->q_theta)];
  // 32 x 8 blocks: two resident blocks per SM at 128 registers per thread
  const int by = lattice_is_2d(lattice->q_phi) ? 1 : std::min(8, std::max(4, grid->ny + 2));
  if ((rc = upload_dev(s)) != LBPF_OK || (rc = apply_tiling(s, by, 0)) != LBPF_OK) {
    free_sim(s);
    return rc;
  }
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) { free_sim(s); return LBPF_ECUDA; }
  *out = s;
  return LBPF_OK;
}

int lbpf_destroy(lbpf_sim* s) {
  if (!s) return LBPF_EINVAL;
  cudaStreamSynchronize(s->stream);
  free_sim(s);
  return LBPF_OK;
}

int64_t lbpf_steps_done(const lbpf_sim* s) { return s ? s->step_base + s->steps : -1; }

int lbpf_init_seed(lbpf_sim* s, int32_t n, const double* centres, const double* radii, double U0, double theta0) {
  if (!s || n < 1 || !centres || !radii) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  for (int m = 0; m < n; ++m)
    if (!isfinite(radii[m]) || !isfinite(centres[3 * m]) || !isfinite(centres[3 * m + 1]) ||
        !isfinite(centres[3 * m + 2]))
      return LBPF_EINVAL;
  if (!isfinite(U0) || !isfinite(theta0)) return LBPF_EINVAL;
  s->U0 = U0;
  s->theta0 = theta0;
  int rc = upload_dev(s);
  if (rc) return rc;
  double* d_seed = nullptr;
  CK(s, cudaMalloc(&d_seed, sizeof(double) * 4 * n));
  std::vector<double> cen(centres, centres + 3 * n);
  if (lattice_is_2d(s->lat.q_phi))  // kernel coordinates (x, z, y)
    for (int m = 0; m < n; ++m) std::swap(cen[3 * m + 1], cen[3 * m + 2]);
  CK(s, cudaMemcpy(d_seed, cen.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
  CK(s, cudaMemcpyAsync(d_seed + 3 * n, radii, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
  const double c = s->p.dx / (sqrt(2.0) * s->p.W0);
  // phi of the seeds into level 1 (scratch), populations at buffer 0, moments at level 0,
  // and level 2 (phi^{n-1} of the codec) = the seed profile used by the encoder.
  CK(s, s->kt->init_scalar(s->stream, s->kg.nx, s->kg.ny, s->kg.nz, d_seed, d_seed + 3 * n, n, c, s->phi[1]));
  const LatRT Lp = make_lat_rt(s->lat.q_phi), Lu = make_lat_rt(s->lat.q_u);
  LatRT Lt{};
  if (s->lat.q_theta) Lt = make_lat_rt(s->lat.q_theta);
  CK(s, s->kt->init_pop(s->stream, s->hd, Lp, Lu, Lt, s->phi[1], U0, theta0));
  CK(s, cudaMemcpyAsync(s->phi[2], s->phi[1], (size_t)s->nsite * s->kt->tbytes, cudaMemcpyDeviceToDevice, s->stream));
  // theta^{n-1} (the codec reference of f) = the initial theta
  if (s->th[0])
    CK(s, cudaMemcpyAsync(s->th[2], s->th[0], (size_t)s->nsite * s->kt->tbytes, cudaMemcpyDeviceToDevice, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  cudaFree(d_seed);
  s->steps = 0;
  s->step_base = 0;
  return LBPF_OK;
}

int lbpf_step(lbpf_sim* s, int64_t n) {
  if (!s || n < 0) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  while (n > 0) {
    if (s6_of(s) == 0 && n >= kGraphSteps) {
      if (!s->graph_ok) {
        if (s->gexec) cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
        if (capture_graph(s->stream, s->fphi, s->futh, s->nitems, s->by, s->smem_phi, s->smem_uth, s->dd,
                          s->d_items, &s->ol, &s->gexec) != LBPF_OK) {
          s->sticky = LBPF_ECUDA;
          return LBPF_ECUDA;
        }
        s->graph_ok = true;
      }
      CK(s, cudaGraphLaunch(s->gexec, s->stream));
      s->steps += kGraphSteps;
      n -= kGraphSteps;
    } else {
      if (launch_step(s->stream, s->fphi, s->futh, s->nitems, s->by, s->smem_phi, s->smem_uth, s->dd, s->d_items,
                      s6_of(s), &s->ol) != LBPF_OK) {
        s->sticky = LBPF_ECUDA;
        return LBPF_ECUDA;
      }
      s->steps += 1;
      n -= 1;
    }
  }
  return LBPF_OK;
}

int lbpf_step_timed(lbpf_sim* s, int64_t n, double ms_kernels[3]) {
  if (!s || n < 1 || !ms_kernels) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  std::vector<cudaEvent_t> ev((size_t)(2 * n + 1));
  for (auto& e : ev) CK(s, cudaEventCreate(&e));
  CK(s, cudaEventRecord(ev[0], s->stream));
  for (int64_t k = 0; k < n; ++k) {
    const int s6 = s6_of(s);
    if (s->ol.on) {
      // one launch per step: all of its time is counted as the first phase's
      if (launch_step(s->stream, s->fphi, s->futh, s->nitems, s->by, s->smem_phi, s->smem_uth, s->dd, s->d_items,
                      s6, &s->ol) != LBPF_OK) {
        s->sticky = LBPF_ECUDA;
        return LBPF_ECUDA;
      }
      CK(s, cudaEventRecord(ev[2 * k + 1], s->stream));
    } else {
      CK(s, s->fphi(dim3(s->nitems), dim3(32, s->by), s->smem_phi, s->stream, s->dd, s->d_items, s6));
      CK(s, cudaEventRecord(ev[2 * k + 1], s->stream));
      CK(s, s->futh(dim3(s->nitems), dim3(32, s->by), s->smem_uth, s->stream, s->dd, s->d_items, s6));
    }
    CK(s, cudaEventRecord(ev[2 * k + 2], s->stream));
    s->steps += 1;
  }
  CK(s, cudaEventSynchronize(ev[2 * n]));
  double tp = 0, tu = 0;
  for (int64_t k = 0; k < n; ++k) {
    float a = 0, b = 0;
    CK(s, cudaEventElapsedTime(&a, ev[2 * k], ev[2 * k + 1]));
    CK(s, cudaEventElapsedTime(&b, ev[2 * k + 1], ev[2 * k + 2]));
    tp += a;
    tu += b;
  }
  float all = 0;
  CK(s, cudaEventElapsedTime(&all, ev[0], ev[2 * n]));
  for (auto& e : ev) cudaEventDestroy(e);
  ms_kernels[0] = tp;
  ms_kernels[1] = tu;
  ms_kernels[2] = all;
  return LBPF_OK;
}

int lbpf_read_fields(lbpf_sim* s, uint32_t mask, double* phi, double* U, double* theta) {
  if (!s) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  if (((mask & LBPF_PHI) && !phi) || ((mask & LBPF_U) && !U) || ((mask & LBPF_THETA) && !theta)) return LBPF_EINVAL;
  const size_t N = (size_t)s->nsite;
  const void* src[3] = {s->phi[s6_of(s) % 3], s->U[par_of(s)], s->lat.q_theta ? s->th[s6_of(s) % 3] : nullptr};
  double* dst[3] = {(mask & LBPF_PHI) ? phi : nullptr, (mask & LBPF_U) ? U : nullptr,
                    (mask & LBPF_THETA) ? theta : nullptr};
  const bool need_tmp = s->kt->tbytes != 8;
  if (need_tmp) {
    int rc = ensure_tmp(s);
    if (rc) return rc;
  }
  for (int f = 0; f < 3; ++f) {
    if (!dst[f]) continue;
    if (!src[f]) {
      CK(s, cudaStreamSynchronize(s->stream));
      for (size_t i = 0; i < N; ++i) dst[f][i] = s->theta0;
      continue;
    }
    if (need_tmp) {
      CK(s, s->kt->to_double(s->stream, s->d_tmp, src[f], (long long)N));
      CK(s, cudaMemcpyAsync(dst[f], s->d_tmp, N * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    } else {
      CK(s, cudaMemcpyAsync(dst[f], src[f], N * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    }
    CK(s, cudaStreamSynchronize(s->stream));
  }
  return status(s);
}

int lbpf_sums(lbpf_sim* s, double out[4]) {
  if (!s || !out) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  const void* th = s->lat.q_theta ? s->th[s6_of(s) % 3] : nullptr;
  const int nblk = (int)std::min<long long>(s->npart, std::max<long long>(1, (s->nsite + 255) / 256));
  CK(s, s->kt->sums(s->stream, s->phi[s6_of(s) % 3], s->U[par_of(s)], th, s->theta0, s->p.k, s->nsite, s->d_part,
                    nblk));
  CK(s, cudaMemcpyAsync(s->h_small, s->d_part + 4 * nblk, 4 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  if (status(s)) return s->sticky;
  bool fin = true;
  for (int c = 0; c < 4; ++c) {
    out[c] = s->h_small[c];
    fin = fin && isfinite(out[c]);
  }
  return fin ? LBPF_OK : LBPF_ENAN;
}

int lbpf_tip(lbpf_sim* s, int32_t axis, const double centre_lu[3], double* x_tip, double* rho) {
  if (!s || !centre_lu || !x_tip) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  const bool d2 = lattice_is_2d(s->lat.q_phi);
  if (axis < 0 || axis > (d2 ? 1 : 2)) return LBPF_EINVAL;
  // the scan starts at the node nearest to the centre
  int c[3];
  const int n[3] = {s->g.nx, s->g.ny, s->g.nz};
  for (int a = 0; a < 3; ++a) {
    if (!isfinite(centre_lu[a])) return LBPF_EINVAL;
    const double v = floor(centre_lu[a] + 0.5);
    if (v < 0 || v >= n[a]) return LBPF_EINVAL;
    c[a] = (int)v;
  }
  // kernel coordinates: a 2D grid (nx, ny, 1) runs as (nx, 1, ny), the paper's y on the kernel's z
  const int kaxis = d2 && axis == 1 ? 2 : axis;
  CK(s, s->kt->tip(s->stream, s->phi[s6_of(s) % 3], s->kg.nx, s->kg.ny, s->kg.nz, kaxis, c[0], d2 ? c[2] : c[1],
                   d2 ? c[1] : c[2], s->d_small));
  CK(s, cudaMemcpyAsync(s->h_small, s->d_small, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  *x_tip = s->h_small[0];
  if (rho) *rho = s->h_small[1];
  return LBPF_OK;
}

namespace {
// Import post-streaming populations.  `moments` (optional, FP64, 5 x nsite):
// phi^n, phi^{n-1}, U^n, theta^n, theta^{n-1} to install instead of recomputing the
// moments from the populations, so that a checkpoint restarts bit for bit.
int import_state(lbpf_sim* s, const double* g, const double* h, const double* f, double theta0,
                 const double* moments) {
  int rc = ensure_tmp(s);
  if (rc) return rc;
  s->theta0 = theta0;
  if ((rc = upload_dev(s))) return rc;
  s->steps = 0;
  s->step_base = 0;
  const size_t N = (size_t)s->nsite;
  double* acc = s->d_tmp;
  double* b0 = s->d_tmp + N;
  double* b1 = s->d_tmp + 2 * N;
  const double* host[3] = {g, h, f};
  const int qs[3] = {s->lat.q_phi, s->lat.q_u, s->lat.q_theta};
  void* mom[3] = {s->phi[0], s->U[0], s->th[0]};
  for (int fld = 0; fld < 3; ++fld) {
    if (!qs[fld]) continue;
    const LatRT L = make_lat_rt(qs[fld]);
    if (moments) {
      const double* m = moments + (size_t)(fld == 0 ? 0 : (fld == 1 ? 2 : 3)) * N;
      CK(s, cudaMemcpyAsync(acc, m, N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    } else {
      // moments: sum over i in index order, in FP64
      CK(s, cudaMemsetAsync(acc, 0, N * sizeof(double), s->stream));
      for (int i = 0; i < qs[fld]; ++i) {
        CK(s, cudaMemcpyAsync(b0, host[fld] + (size_t)i * N, N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        k_acc<<<aux_blocks_host(N), 256, 0, s->stream>>>(acc, b0, (long long)N);
        CK(s, cudaGetLastError());
      }
    }
    CK(s, s->kt->from_double(s->stream, mom[fld], acc, (long long)N));
    void* prev = fld == 0 ? s->phi[2] : (fld == 2 ? s->th[2] : nullptr);
    if (prev) {
      // codec reference of g and f, phi^{n-1} and theta^{n-1}: the saved level, or the
      // current one for an imported state
      if (moments) {
        CK(s, cudaMemcpyAsync(acc, moments + (size_t)(fld == 0 ? 1 : 4) * N, N * sizeof(double), cudaMemcpyHostToDevice,
                              s->stream));
        CK(s, s->kt->from_double(s->stream, prev, acc, (long long)N));
      } else {
        CK(s, cudaMemcpyAsync(prev, mom[fld], N * s->kt->tbytes, cudaMemcpyDeviceToDevice, s->stream));
      }
    }
    for (int i = 0; i < qs[fld]; ++i) {
      const int j = L.opp[i];
      if (j < i) continue;
      CK(s, cudaMemcpyAsync(b0, host[fld] + (size_t)i * N, N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
      CK(s, cudaMemcpyAsync(b1, host[fld] + (size_t)j * N, N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
      CK(s, s->kt->pack(s->stream, s->hd, fld, 0, L, i, b0, b1, prev));
    }
    CK(s, cudaStreamSynchronize(s->stream));
  }
  return LBPF_OK;
}

// Export phi^n, phi^{n-1}, U^n, theta^n, theta^{n-1} as FP64 (5 x nsite).
int export_moments(lbpf_sim* s, double* out) {
  int rc = ensure_tmp(s);
  if (rc) return rc;
  const size_t N = (size_t)s->nsite;
  const bool th = s->lat.q_theta != 0;
  const void* src[5] = {s->phi[s6_of(s) % 3], s->phi[(s6_of(s) + 2) % 3], s->U[par_of(s)],
                        th ? s->th[s6_of(s) % 3] : nullptr, th ? s->th[(s6_of(s) + 2) % 3] : nullptr};
  for (int k = 0; k < 5; ++k) {
    if (!src[k]) {
      for (size_t i = 0; i < N; ++i) out[k * N + i] = s->theta0;
      continue;
    }
    CK(s, s->kt->to_double(s->stream, s->d_tmp, src[k], (long long)N));
    CK(s, cudaMemcpyAsync(out + k * N, s->d_tmp, N * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
  }
  return LBPF_OK;
}
}  // namespace

int lbpf_set_state(lbpf_sim* s, const double* g, const double* h, const double* f, double theta0) {
  if (!s || !g || !h || (s->lat.q_theta && !f)) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  return import_state(s, g, h, f, theta0, nullptr);
}

int lbpf_get_state(lbpf_sim* s, double* g, double* h, double* f) {
  if (!s) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  int rc = ensure_tmp(s);
  if (rc) return rc;
  const size_t N = (size_t)s->nsite;
  double* b0 = s->d_tmp + N;
  double* b1 = s->d_tmp + 2 * N;
  double* host[3] = {g, h, f};
  const int qs[3] = {s->lat.q_phi, s->lat.q_u, s->lat.q_theta};
  // codec references of g and f: phi^{n-1}, theta^{n-1}
  const void* prev[3] = {s->phi[(s6_of(s) + 2) % 3], nullptr, s->th[(s6_of(s) + 2) % 3]};
  for (int fld = 0; fld < 3; ++fld) {
    if (!qs[fld] || !host[fld]) continue;
    const LatRT L = make_lat_rt(qs[fld]);
    for (int i = 0; i < qs[fld]; ++i) {
      const int j = L.opp[i];
      if (j < i) continue;
      CK(s, s->kt->unpack(s->stream, s->hd, fld, par_of(s), L, i, b0, b1, prev[fld]));
      CK(s, cudaMemcpyAsync(host[fld] + (size_t)i * N, b0, N * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
      if (j != i)
        CK(s, cudaMemcpyAsync(host[fld] + (size_t)j * N, b1, N * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
      CK(s, cudaStreamSynchronize(s->stream));
    }
  }
  return LBPF_OK;
}

int lbpf_set_tiling(lbpf_sim* s, int32_t by, int32_t zchunk) {
  if (!s || by < 0 || zchunk < 0 || (by && (by < 4 || by > MAX_BLOCK_ROWS))) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  CK(s, cudaStreamSynchronize(s->stream));
  return apply_tiling(s, by ? by : s->by, zchunk ? zchunk : (by ? 0 : s->zchunk));
}

int lbpf_get_tiling(const lbpf_sim* s, int32_t* by, int32_t* zchunk) {
  if (!s) return LBPF_EINVAL;
  if (by) *by = s->by;
  if (zchunk) *zchunk = s->zchunk;
  return LBPF_OK;
}

int lbpf_set_schedule(lbpf_sim* s, int32_t schedule) {
  if (!s || (schedule != LBPF_SCHED_TWO_KERNELS && schedule != LBPF_SCHED_ONE_LAUNCH)) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  if (schedule == LBPF_SCHED_ONE_LAUNCH && !s->ol.fn) return LBPF_EINVAL;
  CK(s, cudaStreamSynchronize(s->stream));
  const bool was = s->ol.on;
  s->ol.on = schedule == LBPF_SCHED_ONE_LAUNCH;
  const int rc = apply_tiling(s, s->by, s->zchunk);
  if (rc != LBPF_OK) {
    s->ol.on = was;
    free_one_launch(s->ol);
    apply_tiling(s, s->by, s->zchunk);
  }
  if (!s->ol.on) free_one_launch(s->ol);
  return rc;
}

int lbpf_set_wait_polls(lbpf_sim* s, int32_t polls) {
  if (!s || polls < 0) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  CK(s, cudaStreamSynchronize(s->stream));
  s->ol.polls = (unsigned)polls;
  if (s->ol.d_sched) s->ol.sc.polls = s->ol.polls;
  // the step graph holds the launch parameters: capture it again at the next step
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  s->gexec = nullptr;
  s->graph_ok = false;
  return LBPF_OK;
}

int lbpf_get_schedule(const lbpf_sim* s, int32_t* schedule) {
  if (!s || !schedule) return LBPF_EINVAL;
  *schedule = s->ol.on ? LBPF_SCHED_ONE_LAUNCH : LBPF_SCHED_TWO_KERNELS;
  return LBPF_OK;
}

int lbpf_wait_probe(int32_t flag_value, int32_t polls, int32_t* seen) {
  if (!seen || polls < 1) return LBPF_EINVAL;
  unsigned* d = nullptr;  // flag, dependency index 0, result
  if (cudaMalloc(&d, 3 * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return LBPF_ENOMEM;
  }
  const unsigned h[3] = {(unsigned)flag_value, 0u, 2u};
  int out = 2;
  bool ok = cudaMemcpy(d, h, sizeof(h), cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok) {
    k_wait_probe<<<1, 32>>>(d, (const int*)(d + 1), (unsigned)polls, (int*)(d + 2));
    ok = cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
         cudaMemcpy(&out, d + 2, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
  }
  cudaFree(d);
  if (!ok || (out != 0 && out != 1)) return LBPF_ECUDA;
  *seen = out;
  return LBPF_OK;
}

}  // extern "C"

namespace {
// The device state the next step reads: populations and U at the current buffer parity and
// every phi and theta level.  A copy of these restores the handle exactly (with its step count).
void live_state(const lbpf_sim* s, std::vector<std::pair<void*, size_t>>& live) {
  const size_t N = (size_t)s->nsite;
  const int qs[3] = {s->lat.q_phi, s->lat.q_u, s->lat.q_theta};
  const int par = par_of(s);
  for (int f = 0; f < 3; ++f)
    if (qs[f]) live.push_back({s->pop[par][f], (size_t)qs[f] * N * s->kt->sbytes});
  for (int l = 0; l < 3; ++l) live.push_back({s->phi[l], N * s->kt->tbytes});
  live.push_back({s->U[par], N * s->kt->tbytes});
  for (int l = 0; l < 3; ++l)
    if (s->th[l]) live.push_back({s->th[l], N * s->kt->tbytes});
}

// Device copies of `live` enqueued on `st` (LBPF_ENOMEM, nothing held, when one does not fit).
int snapshot_state(const std::vector<std::pair<void*, size_t>>& live, cudaStream_t st, std::vector<void*>& snap) {
  snap.assign(live.size(), nullptr);
  for (size_t k = 0; k < live.size(); ++k) {
    if (cudaMalloc(&snap[k], live[k].second) != cudaSuccess) {
      cudaGetLastError();
      for (void*& p : snap) {
        if (p) cudaFree(p);
        p = nullptr;
      }
      snap.clear();
      return LBPF_ENOMEM;
    }
    if (cudaMemcpyAsync(snap[k], live[k].first, live[k].second, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return LBPF_ECUDA;
  }
  return LBPF_OK;
}

int restore_state(const std::vector<std::pair<void*, size_t>>& live, const std::vector<void*>& snap, cudaStream_t st) {
  for (size_t k = 0; k < live.size(); ++k)
    if (cudaMemcpyAsync(live[k].first, snap[k], live[k].second, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return LBPF_ECUDA;
  return LBPF_OK;
}

void free_all(std::vector<void*>& snap) {
  for (void* p : snap)
    if (p) cudaFree(p);
  snap.clear();
}
}  // namespace

extern "C" {

int lbpf_autotune(lbpf_sim* s, int32_t steps, double* best_ms) {
  if (!s || steps < 1) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  CK(s, cudaStreamSynchronize(s->stream));
  std::vector<std::pair<void*, size_t>> live;
  live_state(s, live);
  std::vector<void*> snap;
  const int src = snapshot_state(live, s->stream, snap);
  if (src != LBPF_OK) {
    free_all(snap);
    if (src == LBPF_ECUDA) s->sticky = LBPF_ECUDA;
    return src;
  }
  const int64_t steps0 = s->steps;
  const int by0 = s->by, zc0 = s->zchunk;
  cudaEvent_t e0, e1;
  CK(s, cudaEventCreate(&e0));
  CK(s, cudaEventCreate(&e1));
  double best = 1e300;
  int bbest = by0, zbest = zc0;
  const int bys[] = {4, 6, 8};
  for (int by : bys) {
    if (by > s->kg.ny + 2 && by != bys[0]) continue;
    const int zdef = default_zchunk(s->kg.nx, s->kg.ny, s->kg.nz, by);
    const int zcs[] = {zdef, std::max(8, zdef / 2), std::min(s->kg.nz, zdef * 2), s->kg.nz};
    for (int zc : zcs) {
      if (apply_tiling(s, by, zc) != LBPF_OK) { s->sticky = LBPF_OK; continue; }
      int rc = lbpf_step(s, 1);  // warm-up
      CK(s, cudaEventRecord(e0, s->stream));
      if (rc == LBPF_OK) rc = lbpf_step(s, steps);
      CK(s, cudaEventRecord(e1, s->stream));
      CK(s, cudaEventSynchronize(e1));
      float ms = 0;
      CK(s, cudaEventElapsedTime(&ms, e0, e1));
      if (rc == LBPF_OK && ms / steps < best) {
        best = ms / steps;
        bbest = by;
        zbest = zc;
      }
      // back to the snapshot and the step counter (the parity the snapshot was taken at)
      s->steps = steps0;
      if (restore_state(live, snap, s->stream) != LBPF_OK || cudaStreamSynchronize(s->stream) != cudaSuccess) {
        s->sticky = LBPF_ECUDA;
        free_all(snap);
        return LBPF_ECUDA;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  free_all(snap);
  int rc = apply_tiling(s, bbest, zbest);
  if (best_ms) *best_ms = best;
  return rc;
}

// ---------------------------------------------------------------- checkpoint

namespace {
struct CkptHeader {
  char magic[8];
  int32_t version;
  lbpf_grid grid;
  lbpf_lattice lat;
  lbpf_params params;
  int64_t steps;
  double U0, theta0;
};
}  // namespace

int lbpf_save(lbpf_sim* s, const char* path) {
  if (!s || !path) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  const size_t N = (size_t)s->nsite;
  const int qs[3] = {s->lat.q_phi, s->lat.q_u, s->lat.q_theta};
  std::vector<double> buf[3];
  for (int f = 0; f < 3; ++f) buf[f].resize((size_t)qs[f] * N);
  int rc = lbpf_get_state(s, buf[0].data(), buf[1].data(), qs[2] ? buf[2].data() : nullptr);
  if (rc) return rc;
  std::vector<double> mom(5 * N);
  if ((rc = export_moments(s, mom.data()))) return rc;
  FILE* fp = fopen(path, "wb");
  if (!fp) return LBPF_EINVAL;
  CkptHeader hdr{};
  memcpy(hdr.magic, "LBPFCKP3", 8);
  hdr.version = 3;
  hdr.grid = s->g;
  hdr.lat = s->lat;
  hdr.params = s->p;
  hdr.steps = s->step_base + s->steps;
  hdr.U0 = s->U0;
  hdr.theta0 = s->theta0;
  bool ok = fwrite(&hdr, sizeof(hdr), 1, fp) == 1;
  for (int f = 0; f < 3 && ok; ++f)
    if (qs[f]) ok = fwrite(buf[f].data(), sizeof(double), buf[f].size(), fp) == buf[f].size();
  if (ok) ok = fwrite(mom.data(), sizeof(double), mom.size(), fp) == mom.size();
  ok = (fclose(fp) == 0) && ok;
  return ok ? LBPF_OK : LBPF_EINVAL;
}

int lbpf_load(lbpf_sim* s, const char* path) {
  if (!s || !path) return LBPF_EINVAL;
  if (status(s)) return s->sticky;
  FILE* fp = fopen(path, "rb");
  if (!fp) return LBPF_EINVAL;
  CkptHeader hdr{};
  if (fread(&hdr, sizeof(hdr), 1, fp) != 1 || memcmp(hdr.magic, "LBPFCKP3", 8) != 0 ||
      memcmp(&hdr.grid, &s->g, sizeof(lbpf_grid)) != 0 || memcmp(&hdr.lat, &s->lat, sizeof(lbpf_lattice)) != 0) {
    fclose(fp);
    return LBPF_EINVAL;
  }
  const size_t N = (size_t)s->nsite;
  const int qs[3] = {s->lat.q_phi, s->lat.q_u, s->lat.q_theta};
  std::vector<double> buf[3];
  bool ok = true;
  for (int f = 0; f < 3 && ok; ++f) {
    buf[f].resize((size_t)qs[f] * N);
    if (qs[f]) ok = fread(buf[f].data(), sizeof(double), buf[f].size(), fp) == buf[f].size();
  }
  std::vector<double> mom(5 * N);
  if (ok) ok = fread(mom.data(), sizeof(double), mom.size(), fp) == mom.size();
  fclose(fp);
  if (!ok) return LBPF_EINVAL;
  s->U0 = hdr.U0;
  int rc = import_state(s, buf[0].data(), buf[1].data(), qs[2] ? buf[2].data() : nullptr, hdr.theta0, mom.data());
  if (rc) return rc;
  s->steps = 0;  // buffer phase restarts at 0
  s->step_base = hdr.steps;
  return LBPF_OK;
}

// ---------------------------------------------------------------- batch

// Work items of all member simulations for blocks of `by` rows and z-chunks of
// `zchunk` planes (0: each simulation's default), large chunks first.
static int batch_tiling(lbpf_batch* b, int by, int zchunk) {
  const KernelTable& t = *b->sims[0]->kt;
  std::vector<WorkItem> items;
  std::vector<TileGeom> geo;
  for (size_t i = 0; i < b->sims.size(); ++i) {
    const lbpf_sim* s = b->sims[i];
    const int zc = zchunk > 0 ? std::min(zchunk, s->kg.nz) : default_zchunk(s->kg.nx, s->kg.ny, s->kg.nz, by);
    build_items((int)i, s->kg.nx, s->kg.ny, s->kg.nz, by, zc, items);
    geo.push_back(TileGeom{s->kg.nx, s->kg.ny, s->kg.nz, zc});
  }
  // interleave large and small simulations: sort items by descending z-chunk work
  std::stable_sort(items.begin(), items.end(),
                   [](const WorkItem& a, const WorkItem& c) { return (a.z1 - a.z0) > (c.z1 - c.z0); });
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  if (cudaMalloc(&b->d_items, items.size() * sizeof(WorkItem)) != cudaSuccess ||
      cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return LBPF_ENOMEM;
  }
  b->nitems = (int)items.size();
  b->by = by;
  b->zchunk = zchunk;
  {
    const lbpf_lattice& l = b->sims[0]->lat;
    const int v = block_variant(l.q_phi, by);
    b->fphi = t.phi[q_index(l.q_phi)][v];
    b->futh = t.uth[q_index(l.q_u)][qt_index(l.q_theta)][v];
  }
  b->smem_phi = phi_smem_bytes(t, b->sims[0]->lat.q_phi, by);
  b->smem_uth = uth_smem_bytes(t, b->sims[0]->lat.q_u, b->sims[0]->lat.q_theta, by);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->graph_ok = false;
  if (b->ol.on) {
    const lbpf_lattice& l = b->sims[0]->lat;
    const int rc = setup_one_launch(b->ol, items, geo, by, step_smem_bytes(t, l.q_phi, l.q_u, l.q_theta, by),
                                    t.step_fn[q_index(l.q_phi)][q_index(l.q_u)][qt_index(l.q_theta)],
                                    b->sims[0]->device);
    if (rc != LBPF_OK) return rc;
    for (lbpf_sim* s : b->sims) s->batch_err = b->ol.h_err;
  }
  return LBPF_OK;
}

namespace {
// Shared set-up of both batch constructors: the members are in b->sims and b->stream is set.
int batch_init(lbpf_batch* b) {
  lbpf_sim* s0 = b->sims[0];
  for (lbpf_sim* s : b->sims) {
    if (!s) return LBPF_EINVAL;
    if (status(s)) return s->sticky;
    if (memcmp(&s->lat, &s0->lat, sizeof(lbpf_lattice)) != 0 || s->p.storage != s0->p.storage || s->device != s0->device)
      return LBPF_EINVAL;
  }
  const KernelTable& t = *s0->kt;
  const size_t n = b->sims.size();
  for (lbpf_sim* s : b->sims) cudaStreamSynchronize(s->stream);
  b->ol.fn = s0->ol.fn;
  bool ok = cudaMallocHost(&b->h_desc, n * sizeof(SimDev)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->dd, n * sizeof(SimDev)) == cudaSuccess;
  if (ok) {
    for (size_t i = 0; i < n; ++i) {
      fill_dev(b->sims[i]);
      b->h_desc[i] = b->sims[i]->hd;
    }
  }
  ok = ok && cudaMemcpy(b->dd, b->h_desc, n * sizeof(SimDev), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && batch_tiling(b, lattice_is_2d(s0->lat.q_phi) ? 1 : MAX_BLOCK_ROWS, 0) == LBPF_OK;
  const int a = q_index(s0->lat.q_phi), qb = q_index(s0->lat.q_u), qc = qt_index(s0->lat.q_theta);
  for (int v = 0; v < 2; ++v) {
    ok = ok && raise_smem_limit(t.phi_fn[a][v], s0->device) == LBPF_OK;
    ok = ok && raise_smem_limit(t.uth_fn[qb][qc][v], s0->device) == LBPF_OK;
  }
  if (!ok) {
    cudaGetLastError();
    return LBPF_ENOMEM;
  }
  return LBPF_OK;
}

// Re-upload the member descriptors when a member's state changed since the last upload
// (for instance a new U0 or theta0 from lbpf_init_seed, which the FP16 codec shifts by).
int batch_refresh(lbpf_batch* b) {
  bool changed = false;
  for (size_t i = 0; i < b->sims.size(); ++i) {
    fill_dev(b->sims[i]);
    changed = changed || memcmp(&b->sims[i]->hd, &b->h_desc[i], sizeof(SimDev)) != 0;
  }
  if (!changed) return LBPF_OK;
  // the pinned buffer may still feed an earlier upload: let the stream drain first
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LBPF_ECUDA;
  for (size_t i = 0; i < b->sims.size(); ++i) b->h_desc[i] = b->sims[i]->hd;
  if (cudaMemcpyAsync(b->dd, b->h_desc, b->sims.size() * sizeof(SimDev), cudaMemcpyHostToDevice, b->stream) !=
      cudaSuccess)
    return LBPF_ECUDA;
  return LBPF_OK;
}
}  // namespace

int lbpf_batch_from_sims(int32_t n, lbpf_sim* const* sims, void* cuda_stream, lbpf_batch** out) {
  if (!out || n < 1 || !sims) return LBPF_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!sims[i]) return LBPF_EINVAL;
  lbpf_batch* b = new lbpf_batch();
  b->sims.assign(sims, sims + n);
  b->stream = cuda_stream ? (cudaStream_t)cuda_stream : sims[0]->stream;
  const int rc = batch_init(b);
  if (rc != LBPF_OK) {
    lbpf_batch_destroy(b);
    return rc;
  }
  *out = b;
  return LBPF_OK;
}

int lbpf_batch_create(int32_t n, const lbpf_grid* grids, const lbpf_lattice* lattices, const lbpf_params* params,
                      void* cuda_stream, lbpf_batch** out) {
  if (!out || n < 1 || !grids || !lattices || !params) return LBPF_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (memcmp(&lattices[i], &lattices[0], sizeof(lbpf_lattice)) != 0 || params[i].storage != params[0].storage)
      return LBPF_EINVAL;
  lbpf_batch* b = new lbpf_batch();
  b->owns_sims = true;
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return LBPF_ECUDA;
    }
    b->own_stream = true;
  }
  int rc = LBPF_OK;
  for (int i = 0; i < n && rc == LBPF_OK; ++i) {
    lbpf_sim* s = nullptr;
    rc = lbpf_create(&grids[i], &lattices[i], &params[i], b->stream, &s);
    if (rc == LBPF_OK) b->sims.push_back(s);
  }
  if (rc == LBPF_OK) rc = batch_init(b);
  if (rc != LBPF_OK) {
    lbpf_batch_destroy(b);
    return rc;
  }
  *out = b;
  return LBPF_OK;
}

int lbpf_batch_member(const lbpf_batch* b, int32_t i, lbpf_sim** out) {
  if (!b || !out || i < 0 || i >= (int32_t)b->sims.size()) return LBPF_EINVAL;
  *out = b->sims[(size_t)i];
  return LBPF_OK;
}

int lbpf_batch_step(lbpf_batch* b, int64_t n) {
  if (!b || n < 0) return LBPF_EINVAL;
  const int64_t st0 = b->sims[0]->steps;
  for (lbpf_sim* s : b->sims) {
    if (status(s)) return s->sticky;
    if (s->steps != st0) return LBPF_EINVAL;  // batch members advance in lockstep
  }
  // work the members enqueued on their own streams comes first
  for (lbpf_sim* s : b->sims)
    if (s->stream != b->stream) {
      if (cudaEventRecord(b->ev, s->stream) != cudaSuccess || cudaStreamWaitEvent(b->stream, b->ev, 0) != cudaSuccess)
        return LBPF_ECUDA;
    }
  int rc = batch_refresh(b);
  if (rc != LBPF_OK) return rc;
  int64_t steps = st0;
  while (n > 0) {
    const int s6 = (int)(steps % kGraphSteps);
    if (s6 == 0 && n >= kGraphSteps) {
      if (!b->graph_ok) {
        if (capture_graph(b->stream, b->fphi, b->futh, b->nitems, b->by, b->smem_phi, b->smem_uth, b->dd, b->d_items,
                          &b->ol, &b->gexec) != LBPF_OK)
          return LBPF_ECUDA;
        b->graph_ok = true;
      }
      if (cudaGraphLaunch(b->gexec, b->stream) != cudaSuccess) return LBPF_ECUDA;
      steps += kGraphSteps;
      n -= kGraphSteps;
    } else {
      if (launch_step(b->stream, b->fphi, b->futh, b->nitems, b->by, b->smem_phi, b->smem_uth, b->dd, b->d_items, s6,
                      &b->ol) !=
          LBPF_OK)
        return LBPF_ECUDA;
      steps += 1;
      n -= 1;
    }
  }
  for (lbpf_sim* s : b->sims) s->steps = steps;
  // later work on a member's own stream (reads, sums, single steps) waits for the batch
  if (cudaEventRecord(b->ev, b->stream) != cudaSuccess) return LBPF_ECUDA;
  for (lbpf_sim* s : b->sims)
    if (s->stream != b->stream && cudaStreamWaitEvent(s->stream, b->ev, 0) != cudaSuccess) return LBPF_ECUDA;
  return LBPF_OK;
}

int lbpf_batch_set_tiling(lbpf_batch* b, int32_t by, int32_t zchunk) {
  if (!b || by < 0 || zchunk < 0 || (by && (by < 4 || by > MAX_BLOCK_ROWS))) return LBPF_EINVAL;
  for (lbpf_sim* s : b->sims)
    if (status(s)) return s->sticky;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LBPF_ECUDA;
  if (lattice_is_2d(b->sims[0]->lat.q_phi)) by = 1;  // 2D: one-row blocks
  return batch_tiling(b, by ? by : b->by, zchunk);
}

int lbpf_batch_set_schedule(lbpf_batch* b, int32_t schedule) {
  if (!b || (schedule != LBPF_SCHED_TWO_KERNELS && schedule != LBPF_SCHED_ONE_LAUNCH)) return LBPF_EINVAL;
  for (lbpf_sim* s : b->sims)
    if (status(s)) return s->sticky;
  if (schedule == LBPF_SCHED_ONE_LAUNCH && !b->ol.fn) return LBPF_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LBPF_ECUDA;
  const bool was = b->ol.on;
  b->ol.on = schedule == LBPF_SCHED_ONE_LAUNCH;
  const int rc = batch_tiling(b, b->by, b->zchunk);
  if (rc != LBPF_OK) {
    b->ol.on = was;
    free_one_launch(b->ol);
    batch_tiling(b, b->by, b->zchunk);
  }
  if (!b->ol.on) free_one_launch(b->ol);
  return rc;
}

int lbpf_batch_get_schedule(const lbpf_batch* b, int32_t* schedule) {
  if (!b || !schedule) return LBPF_EINVAL;
  *schedule = b->ol.on ? LBPF_SCHED_ONE_LAUNCH : LBPF_SCHED_TWO_KERNELS;
  return LBPF_OK;
}

int lbpf_batch_get_tiling(const lbpf_batch* b, int32_t* by, int32_t* zchunk) {
  if (!b) return LBPF_EINVAL;
  if (by) *by = b->by;
  if (zchunk) *zchunk = b->zchunk;
  return LBPF_OK;
}

int lbpf_batch_autotune(lbpf_batch* b, int32_t steps, double* best_ms) {
  if (!b || steps < 1) return LBPF_EINVAL;
  const int64_t st0 = b->sims[0]->steps;
  for (lbpf_sim* s : b->sims) {
    if (status(s)) return s->sticky;
    if (s->steps != st0) return LBPF_EINVAL;
  }
  for (lbpf_sim* s : b->sims)
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return LBPF_ECUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LBPF_ECUDA;
  std::vector<std::pair<void*, size_t>> live;
  for (lbpf_sim* s : b->sims) live_state(s, live);
  std::vector<void*> snap;
  int rc = snapshot_state(live, b->stream, snap);
  if (rc != LBPF_OK) {
    free_all(snap);
    return rc;
  }
  // every trial times whole graph periods: single steps up to a period boundary, one period of
  // warm-up (it also captures the trial's graph), then `steps` rounded up to whole periods
  const int64_t align = (kGraphSteps - st0 % kGraphSteps) % kGraphSteps;
  const int64_t timed = ((int64_t)steps + kGraphSteps - 1) / kGraphSteps * kGraphSteps;
  const bool is2d = lattice_is_2d(b->sims[0]->lat.q_phi);
  std::vector<std::pair<int, int>> cand;
  if (is2d) {
    for (int zc : {0, 8, 16, 32}) cand.push_back({1, zc});
  } else {
    for (int by : {4, 6, 8})
      for (int zc : {0, 12, 16, 24}) cand.push_back({by, zc});
  }
  const int by0 = b->by, zc0 = b->zchunk;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  double best = 1e300;
  int bbest = by0, zbest = zc0;
  for (size_t c = 0; c < cand.size() && ok; ++c) {
    if (batch_tiling(b, cand[c].first, cand[c].second) != LBPF_OK) continue;
    rc = lbpf_batch_step(b, align + kGraphSteps);
    ok = cudaEventRecord(e0, b->stream) == cudaSuccess;
    if (rc == LBPF_OK && ok) rc = lbpf_batch_step(b, timed);
    ok = ok && cudaEventRecord(e1, b->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0;
    ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (ok && rc == LBPF_OK && ms / timed < best) {
      best = ms / timed;
      bbest = cand[c].first;
      zbest = cand[c].second;
    }
    // every member back to the snapshot and its step count
    for (lbpf_sim* s : b->sims) s->steps = st0;
    ok = ok && restore_state(live, snap, b->stream) == LBPF_OK && cudaStreamSynchronize(b->stream) == cudaSuccess;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  free_all(snap);
  if (!ok) {
    for (lbpf_sim* s : b->sims) s->sticky = LBPF_ECUDA;
    return LBPF_ECUDA;
  }
  rc = batch_tiling(b, bbest, zbest);
  if (best_ms) *best_ms = best;
  return rc;
}

int lbpf_batch_destroy(lbpf_batch* b) {
  if (!b) return LBPF_EINVAL;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->dd) cudaFree(b->dd);
  if (b->h_desc) cudaFreeHost(b->h_desc);
  if (b->d_items) cudaFree(b->d_items);
  if (b->ev) cudaEventDestroy(b->ev);
  // borrowed members outlive the batch: they keep a failure the batch saw, not its flag
  for (lbpf_sim* s : b->sims)
    if (s && b->ol.h_err && s->batch_err == b->ol.h_err) {
      status(s);
      s->batch_err = nullptr;
    }
  free_one_launch(b->ol);
  if (b->ol.h_err) cudaFreeHost(b->ol.h_err);
  if (b->owns_sims)
    for (lbpf_sim* s : b->sims) lbpf_destroy(s);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return LBPF_OK;
}

}  // extern "C"
