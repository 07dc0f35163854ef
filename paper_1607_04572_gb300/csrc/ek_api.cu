// Host side of the C ABI declared in include/ek.h: context, device memory,
// the time-step driver and field / particle exchange.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>
#include <string>

#include "ek_internal.cuh"

using namespace ek;

namespace {
// ek_debug_fail_alloc: the n-th field allocation of ek_create from now on
// fails (0: none)
std::atomic<int> g_alloc_fault{0};
bool alloc_fault_due() {
  int n = g_alloc_fault.load();
  while (n > 0) {
    if (g_alloc_fault.compare_exchange_weak(n, n - 1)) return n == 1;
  }
  return false;
}
}  // namespace

struct ek_ctx {
  ek_params p;
  Grid g;
  Phys ph;
  cudaStream_t stream = nullptr;
  cudaStream_t aux = nullptr;        // particle work of S4/S5 runs here, beside S3
  cudaEvent_t ev_lb = nullptr;       // S2 done
  cudaEvent_t ev_part = nullptr;     // S4 + re-flag done
  cudaEvent_t ev_start = nullptr;    // step begins (the assignment may start)
  cudaEvent_t ev_join = nullptr;     // all auxiliary work of the step done
  // one captured step per parity of `cur` (the ping-pong buffers alternate)
  cudaGraphExec_t step_graph[2] = {nullptr, nullptr};
  long long graph_launches = 0;      // kernels in one captured step
  int device = 0;
  int fp32 = 0;  // storage form (EK_FP32)
  // field storage: double (FP64 form) or float / int32 species (FP32 form)
  void* f[2] = {nullptr, nullptr};
  void* rho[2] = {nullptr, nullptr};
  void* phi = nullptr;
  void* psi = nullptr;
  void* qpart = nullptr;
  void* qwall = nullptr;
  void* u = nullptr;
  void* ifield = nullptr;              // 3N reals: internal solute force on the fluid (S2)
  double* ipart = nullptr;             // 3 doubles per lattice block: its sums
  int nipart = 0;
  int nipart_cap = 0;  // rows allocated for ipart (FP32: enough for 2-plane segments)
  int nzb = 1;       // FP32 S2: z segments per tile column
  int advseg = 1;    // FP32 S3: z segments per tile column
  int overlap = 1;   // particle chain on the auxiliary stream (1) or in line (0)
  unsigned long long version = 0;  // bumped whenever captured steps go stale
  unsigned long long* fkey = nullptr;  // N: nearest-particle keys of S4
  unsigned char* vsig = nullptr;       // N: fluid bit and velocity sign codes (S2 -> S3)
  int emax = 0;                        // cells of the widest widened box
  double* tmp = nullptr;  // N doubles of staging for conversions
  size_t rsz = 8;         // bytes of a real (double / float)
  int* owner = nullptr;
  int* owner_prev = nullptr;
  unsigned char* wall = nullptr;
  void* spectrum = nullptr;
  PoissonPlan plan;
  DevParticle* dparts = nullptr;
  int P = 0;
  int Pcap = 0;
  std::vector<DevParticle> hparts;
  double* psibox = nullptr;
  int boxmax = 0;
  size_t psibox_cap = 0;  // doubles allocated for psibox
  double* fpart = nullptr;  // S4 partial sums, P * fchunks * FPART
  int fchunks = 0;
  int fcells = FORCE_CHUNK;  // widened-box cells per S4 force CTA
  double* psum = nullptr;   // (Pcap + 1) * FPART
  int2* surf = nullptr;     // surface-cell list of S5, P * boxmax entries
  int* tie_list = nullptr;  // nodes of possible nearest-surface ties (S4)
  int* tie_count = nullptr;
  int tie_cap = 1 << 16;
  float tie_thr = 0.0f;
  int* surf_count = nullptr;
  Transfer* xfer = nullptr;
  int* xfer_count = nullptr;
  int* ticket = nullptr;
  int* pticket = nullptr;   // Pcap: force (or transition) blocks done per particle
  double* tpart = nullptr;  // S5 transition momentum per CTA, 3 * tcap
  size_t tcap = 0;          // (particle, CTA) rows allocated in tpart
  int uchunks = 0;          // CTAs per particle over the union box (in use)
  ek_particle* pstage = nullptr;  // Pcap records for ek_get_particles_async
  int xfer_cap = 0;
  int* status = nullptr;
  int cur = 0;
  long long launches = 0;  // kernels enqueued by the step and stage calls so far
  bool setup_pending = true;
  bool has_qwall = false;
  bool broken = false;
  std::string err;
};

namespace {

ek_status fail(ek_ctx* c, ek_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define EK_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(ctx, EK_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

__global__ void k_set_velocity(Grid g, const int* owner, double* f, const double* u) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N || owner[n] != FLUID) return;
  double rho = 0.0;
  for (int i = 0; i < Q; ++i) rho += f[i * g.N + n];
  const double ux = u[n], uy = u[g.N + n], uz = u[2 * g.N + n];
  const double usq = ux * ux + uy * uy + uz * uz;
  for (int i = 0; i < Q; ++i) {
    const double cu = cdot(i, ux, uy, uz);
    f[i * g.N + n] = wgt(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
  }
}

__global__ void k_density(Grid g, const double* f, double* out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  double rho = 0.0;
  for (int i = 0; i < Q; ++i) rho += f[i * g.N + n];
  out[n] = rho;
}

__global__ void k_int_to_double(Grid g, const int* in, double* out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < g.N) out[n] = (double)in[n];
}

__global__ void k_u8_to_double(Grid g, const unsigned char* in, double* out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < g.N) out[n] = (double)in[n];
}

__global__ void k_double_to_u8(Grid g, const double* in, unsigned char* out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < g.N) out[n] = in[n] != 0.0 ? 1 : 0;
}

__global__ void k_psi_clamped(Grid g, const double* psi, double* out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < g.N) out[n] = fmin(psi[n], 1.0);
}

// the particle records in the exchange layout (ek_particle), for an
// asynchronous copy to the host
__global__ void k_pack_particles(const DevParticle* parts, int P, ek_particle* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const DevParticle& q = parts[i];
  ek_particle o;
  for (int d = 0; d < 3; ++d) {
    o.pos[d] = q.pos[d];
    o.vel[d] = q.vel[d];
    o.omega[d] = q.omega[d];
    o.force[d] = q.force[d];
    o.torque[d] = q.torque[d];
  }
  o.radius = q.radius;
  o.charge = q.charge;
  o.rho_p = q.mass / (4.0 / 3.0 * M_PI * q.radius * q.radius * q.radius);
  o.fixed = q.fixed;
  out[i] = o;
}

__global__ void k_count_fluid(Grid g, const int* owner, unsigned long long* count) {
  __shared__ unsigned int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < g.N && owner[n] == FLUID) atomicAdd(&s, 1u);
  __syncthreads();
  if (threadIdx.x == 0 && s) atomicAdd(count, (unsigned long long)s);
}

unsigned nblk(long long n) { return (unsigned)((n + 255) / 256); }

bool edge_ok(int n) {
  if (n < 8 || n > 1024) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

ek_status check_status(ek_ctx* ctx) {
  int st = 0;
  EK_CUDA(cudaMemcpyAsync(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  EK_CUDA(cudaStreamSynchronize(ctx->stream));
  if (st == 0) return EK_OK;
  ctx->broken = true;
  if (st & ST_OVERLAP) return fail(ctx, EK_ERR_OVERLAP, "a node lies inside two particles (or a particle and a wall)");
  if (st & ST_EXPEL) return fail(ctx, EK_ERR_EXPEL, "a newly covered node has no fluid neighbour to expel solute to");
  if (st & ST_CAPACITY) return fail(ctx, EK_ERR_STATE, "a capacity was exceeded (transition records, surface cells, or an FP32-form species value out of int32 range)");
  return fail(ctx, EK_ERR_UNSTABLE, "non-finite density, velocity or particle position");
}

PartArgs part_args(ek_ctx* ctx) {
  PartArgs a;
  a.g = ctx->g;
  a.ph = ctx->ph;
  a.parts = ctx->dparts;
  a.P = ctx->P;
  a.boxmax = ctx->boxmax;
  a.psibox = ctx->psibox;
  a.owner = ctx->owner;
  a.owner_prev = ctx->owner_prev;
  a.psi = ctx->psi;
  a.qpart = ctx->qpart;
  a.f = ctx->f[ctx->cur];
  a.rho = ctx->rho[ctx->cur];
  a.phi = ctx->phi;
  a.wall = ctx->wall;
  a.xfer = ctx->xfer;
  a.xfer_count = ctx->xfer_count;
  a.xfer_cap = ctx->xfer_cap;
  a.fpart = ctx->fpart;
  a.fchunks = ctx->fchunks;
  a.fcells = ctx->fcells;
  a.emax = ctx->emax;
  a.ifield = ctx->ifield;
  a.ipart = ctx->ipart;
  a.nipart = ctx->nipart;
  a.fkey = ctx->fkey;
  a.psum = ctx->psum;
  a.surf = ctx->surf;
  a.surf_count = ctx->surf_count;
  a.ticket = ctx->ticket;
  a.pticket = ctx->pticket;
  a.tpart = ctx->tpart;
  a.uchunks = ctx->uchunks;
  a.surf_cap = (int)std::min<size_t>(ctx->psibox_cap, (size_t)1 << 30);
  a.tie_list = ctx->tie_list;
  a.tie_count = ctx->tie_count;
  a.tie_cap = ctx->tie_cap;
  a.tie_thr = ctx->tie_thr;
  a.status = ctx->status;
  return a;
}

// constants that follow from E and the species: E . c_i per direction
void update_derived(Phys& ph) {
  for (int i = 0; i < Q; ++i) ph.ec[i] = ph.E[0] * HCX[i] + ph.E[1] * HCY[i] + ph.E[2] * HCZ[i];
}

LBArgs lb_args(ek_ctx* ctx) {
  LBArgs a;
  a.g = ctx->g;
  a.ph = ctx->ph;
  a.f_in = ctx->f[ctx->cur];
  a.f_out = ctx->f[1 - ctx->cur];
  a.rho_in = ctx->rho[ctx->cur];
  a.rho_out = ctx->rho[1 - ctx->cur];
  a.phi = ctx->phi;
  a.psi = ctx->psi;
  a.owner = ctx->owner;
  a.u = ctx->u;
  a.ifield = ctx->ifield;
  a.ipart = ctx->ipart;
  a.vsig = ctx->vsig;
  a.parts = ctx->dparts;
  a.status = ctx->status;
  a.nzb = ctx->nzb;
  a.advseg = ctx->advseg;
  return a;
}

// pull the device particle records into the host copy
void drop_graphs(ek_ctx* ctx) {
  ++ctx->version;
  for (int i = 0; i < 2; ++i) {
    if (ctx->step_graph[i]) cudaGraphExecDestroy(ctx->step_graph[i]);
    ctx->step_graph[i] = nullptr;
  }
}

ek_status download_particles(ek_ctx* ctx) {
  if (ctx->P == 0) return EK_OK;
  ctx->hparts.resize(ctx->P);
  EK_CUDA(cudaMemcpyAsync(ctx->hparts.data(), ctx->dparts, ctx->P * sizeof(DevParticle),
                          cudaMemcpyDeviceToHost, ctx->stream));
  EK_CUDA(cudaStreamSynchronize(ctx->stream));
  return EK_OK;
}

// Re-flag the whole lattice from the particle positions and refill it
// (species at bulk + counter-ions, populations at rest): runs before the first
// step after particles or walls changed.
ek_status run_setup(ek_ctx* ctx) {
  if (!ctx->setup_pending) return EK_OK;
  drop_graphs(ctx);
  double rmax = 0.0;
  for (const DevParticle& q : ctx->hparts) rmax = std::max(rmax, q.radius);
  const int edge = (int)floor(2.0 * rmax) + 4;
  const int boxmax = ctx->P ? edge * edge * edge : 0;
  const int eedge = edge + 2 * ((int)ceil(rmax) + FORCE_MARGIN);
  const int emax = ctx->P ? eedge * eedge * eedge : 0;
  {
    // window of possible nearest-surface ties (k_force_assign): twice the
    // float distance error bound 2^-21 (|d| + R + 1), |d| at most the widened
    // box's half diagonal, plus the rounding of the difference of two float
    // distances
    const double dmax = sqrt(3.0) * (rmax + ceil(rmax) + FORCE_MARGIN + 2.0) + 1.0;
    ctx->tie_thr = (float)(2.0 * ldexp(dmax + rmax + 1.0, -21) + ldexp(dmax + rmax, -22));
  }
  // cells per S4 force CTA: FORCE_CHUNK, doubled while the particles still
  // fill eight waves of 912 CTAs (152 SMs x 6) with the larger chunks
  int fcells = FORCE_CHUNK;
  while (fcells < 8 * FORCE_CHUNK &&
         (long long)ctx->P * ((emax + 2 * fcells - 1) / (2 * fcells)) >= 8LL * 152 * 6)
    fcells *= 2;
  const int fchunks = (emax + fcells - 1) / fcells;
  if (ctx->P && ((size_t)ctx->P * boxmax > ctx->psibox_cap || fchunks > ctx->fchunks)) {
    if (ctx->psibox) cudaFree(ctx->psibox);
    if (ctx->fpart) cudaFree(ctx->fpart);
    if (ctx->surf) cudaFree(ctx->surf);
    if (ctx->psum) cudaFree(ctx->psum);
    if (ctx->pticket) cudaFree(ctx->pticket);
    if (ctx->pstage) cudaFree(ctx->pstage);
    ctx->psum = nullptr;
    ctx->pticket = nullptr;
    ctx->pstage = nullptr;
    ctx->psibox = nullptr;
    ctx->fpart = nullptr;
    ctx->surf = nullptr;
    ctx->psibox_cap = 0;
    const size_t cap = (size_t)ctx->Pcap * boxmax;
    EK_CUDA(cudaMalloc(&ctx->psibox, cap * sizeof(double)));
    EK_CUDA(cudaMalloc(&ctx->fpart, (size_t)ctx->Pcap * fchunks * FPART * sizeof(double)));
    EK_CUDA(cudaMalloc(&ctx->psum, (size_t)ctx->Pcap * FPART * sizeof(double)));
    EK_CUDA(cudaMalloc(&ctx->pticket, (size_t)ctx->Pcap * sizeof(int)));
    EK_CUDA(cudaMalloc(&ctx->pstage, (size_t)ctx->Pcap * sizeof(ek_particle)));
    EK_CUDA(cudaMemsetAsync(ctx->pticket, 0, (size_t)ctx->Pcap * sizeof(int), ctx->stream));
    EK_CUDA(cudaMalloc(&ctx->surf, cap * sizeof(int2)));
    ctx->psibox_cap = cap;
    ctx->fchunks = fchunks;
  }
  const int uchunks = ctx->P ? union_chunks(boxmax) : 0;
  if (ctx->P && (size_t)ctx->Pcap * uchunks > ctx->tcap) {
    if (ctx->tpart) cudaFree(ctx->tpart);
    ctx->tpart = nullptr;
    ctx->tcap = 0;
    EK_CUDA(cudaMalloc(&ctx->tpart, (size_t)ctx->Pcap * uchunks * 3 * sizeof(double)));
    ctx->tcap = (size_t)ctx->Pcap * uchunks;
  }
  ctx->uchunks = uchunks;
  ctx->fcells = fcells;
  ctx->boxmax = boxmax;
  ctx->emax = emax;
  if (ctx->P) {
    EK_CUDA(cudaMemcpyAsync(ctx->dparts, ctx->hparts.data(), ctx->P * sizeof(DevParticle),
                            cudaMemcpyHostToDevice, ctx->stream));
  }
  PartArgs a = part_args(ctx);
  EK_CUDA(launch_reflag(a, false, ctx->stream));
  // neutralising counter-ions (reading of "bulk density": initial density on fluid nodes)
  unsigned long long* dcount = reinterpret_cast<unsigned long long*>(ctx->tmp);
  EK_CUDA(cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), ctx->stream));
  k_count_fluid<<<nblk(ctx->g.N), 256, 0, ctx->stream>>>(ctx->g, ctx->owner, dcount);
  unsigned long long nf = 0;
  EK_CUDA(cudaMemcpyAsync(&nf, dcount, sizeof(nf), cudaMemcpyDeviceToHost, ctx->stream));
  EK_CUDA(cudaStreamSynchronize(ctx->stream));
  double bulk[EK_MAX_SPECIES] = {0, 0, 0, 0};
  for (int k = 0; k < ctx->p.nspecies; ++k) bulk[k] = ctx->p.bulk[k];
  if ((ctx->p.flags & EK_NEUTRALIZE) && nf > 0) {
    double net = 0.0;
    for (const DevParticle& q : ctx->hparts) net += q.charge;
    if (ctx->has_qwall) {
      double s = 0.0;
      if (ctx->fp32) {
        std::vector<float> qw(ctx->g.N);
        EK_CUDA(cudaMemcpy(qw.data(), ctx->qwall, ctx->g.N * sizeof(float), cudaMemcpyDeviceToHost));
        for (float v : qw) s += (double)v;
      } else {
        std::vector<double> qw(ctx->g.N);
        EK_CUDA(cudaMemcpy(qw.data(), ctx->qwall, ctx->g.N * sizeof(double), cudaMemcpyDeviceToHost));
        for (double v : qw) s += v;
      }
      net += s;
    }
    double zb = 0.0;
    for (int k = 0; k < ctx->p.nspecies; ++k) zb += ctx->p.valence[k] * ctx->p.bulk[k];
    net += zb * (double)nf;
    if (net != 0.0) {
      int s = -1;
      for (int k = 0; k < ctx->p.nspecies; ++k)
        if (ctx->p.valence[k] * net < 0.0) { s = k; break; }
      if (s < 0) return fail(ctx, EK_ERR_ARG, "no species can neutralise the box");
      bulk[s] = bulk[s] - net / (ctx->p.valence[s] * (double)nf);
    }
  }
  if (ctx->fp32) {
    // one species unit is 2^-e with at least 2^20 units per initial density
    // (after neutralisation: counter-ions of a highly charged particle in a
    // dilute salt can outnumber the bulk many times), so densities up to
    // 2048 times the initial one fit int32
    for (int k = 0; k < EK_MAX_SPECIES; ++k) {
      const double ref = k < ctx->p.nspecies ? std::max(bulk[k], ctx->p.bulk[k]) : 0.0;
      const int e = ref > 0.0 ? (int)ceil(20.0 - log2(ref)) : 30;
      ctx->ph.qscale[k] = ldexp(1.0, -e);
    }
    int units[EK_MAX_SPECIES] = {0, 0, 0, 0};
    for (int k = 0; k < ctx->p.nspecies; ++k) {
      const double v = rint(bulk[k] / ctx->ph.qscale[k]);
      if (!(v >= 0.0 && v < 2147483647.0)) return fail(ctx, EK_ERR_ARG, "bulk density out of the FP32 form's range");
      units[k] = (int)v;
    }
    EK_CUDA(launch_fill32(ctx->g, ctx->ph, ctx->owner, (float*)ctx->f[ctx->cur],
                          (int*)ctx->rho[ctx->cur], units, ctx->stream));
  } else {
    EK_CUDA(launch_fill(ctx->g, ctx->ph, ctx->owner, (double*)ctx->f[ctx->cur],
                        (double*)ctx->rho[ctx->cur], bulk, ctx->stream));
  }
  ctx->setup_pending = false;
  ek_status st = check_status(ctx);
  if (st != EK_OK) return st;
  return download_particles(ctx);
}

// stage 3 (advection) is enqueued separately only by the timed driver; stage 2
// of ek_run_stage / ek_step runs S2 and S3 and swaps the buffers.
ek_status enqueue_stage(ek_ctx* ctx, int stage, cudaEvent_t mid = nullptr) {
  cudaStream_t s = ctx->stream;
  switch (stage) {
    case 1:
      if (ctx->fp32) {
        EK_CUDA(poisson_solve_f32(ctx->plan, (const int*)ctx->rho[ctx->cur],
                                  ctx->has_qwall ? (const float*)ctx->qwall : nullptr,
                                  (const float*)ctx->qpart, ctx->ph, (float*)ctx->phi,
                                  (float2*)ctx->spectrum, s));
      } else {
        EK_CUDA(poisson_solve(ctx->plan, nullptr, (const double*)ctx->rho[ctx->cur],
                              ctx->has_qwall ? (const double*)ctx->qwall : nullptr,
                              (const double*)ctx->qpart, ctx->ph, (double*)ctx->phi,
                              (double2*)ctx->spectrum, s));
      }
      ctx->launches += poisson_kernel_count(ctx->plan, ctx->fp32);
      return EK_OK;
    case 2: {
      LBArgs a = lb_args(ctx);
      EK_CUDA(ctx->fp32 ? launch_lb32(a, s) : launch_lb_fused(a, s));
      if (mid) EK_CUDA(cudaEventRecord(mid, s));
      EK_CUDA(ctx->fp32 ? launch_advection32(a, s) : launch_advection(a, s));
      ctx->launches += ctx->p.nspecies > 0 ? 2 : 1;
      ctx->cur = 1 - ctx->cur;
      return EK_OK;
    }
    case 4: {
      PartArgs a = part_args(ctx);
      EK_CUDA(launch_particle_forces(a, s));
      ctx->launches += ctx->P > 0 ? 3 : 0;
      return EK_OK;
    }
    case 5: {
      PartArgs a = part_args(ctx);
      if (ctx->P) {
        EK_CUDA(launch_reflag(a, true, s));
        ctx->launches += 7;
      }
      return EK_OK;
    }
    default:
      return fail(ctx, EK_ERR_ARG, "stage must be 1, 2, 4 or 5");
  }
}

// One full step with the particle work overlapped: after S2, S4 and the
// re-flag part of S5 (which touch neither the species nor u) run on the
// auxiliary stream while S3 runs on the context's stream; the transitions
// (which need S3's species) follow on the context's stream.
ek_status enqueue_step(ek_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  if (ctx->P && !ctx->overlap) {
    // everything in line on the context's stream (the batch tuner's other choice)
    EK_CUDA(launch_particle_forces(part_args(ctx), s, S4_ASSIGN));
    ek_status st = enqueue_stage(ctx, 1);
    if (st != EK_OK) return st;
    const LBArgs la = lb_args(ctx);
    EK_CUDA(ctx->fp32 ? launch_lb32(la, s) : launch_lb_fused(la, s));
    ctx->cur = 1 - ctx->cur;
    const PartArgs pa = part_args(ctx);
    EK_CUDA(launch_particle_forces(pa, s, S4_FORCES));
    EK_CUDA(launch_reflag(pa, true, s, 1));
    EK_CUDA(ctx->fp32 ? launch_advection32(la, s) : launch_advection(la, s));
    EK_CUDA(launch_reflag(pa, true, s, 2));
    ctx->launches += (ctx->p.nspecies > 0 ? 2 : 1) + 10;
    return EK_OK;
  }
  if (ctx->P) {
    // the nearest-surface assignment reads only the particle records, which
    // S1 and S2 do not write: it runs beside them
    EK_CUDA(cudaEventRecord(ctx->ev_start, s));
    EK_CUDA(cudaStreamWaitEvent(ctx->aux, ctx->ev_start, 0));
    EK_CUDA(launch_particle_forces(part_args(ctx), ctx->aux, S4_ASSIGN));
  }
  ek_status st = enqueue_stage(ctx, 1);
  if (st != EK_OK) return st;
  const LBArgs la = lb_args(ctx);
  EK_CUDA(ctx->fp32 ? launch_lb32(la, s) : launch_lb_fused(la, s));
  ctx->cur = 1 - ctx->cur;
  const PartArgs pa = part_args(ctx);
  if (ctx->P) {
    EK_CUDA(cudaEventRecord(ctx->ev_lb, s));
    EK_CUDA(cudaStreamWaitEvent(ctx->aux, ctx->ev_lb, 0));
    EK_CUDA(launch_particle_forces(pa, ctx->aux, S4_FORCES));
    EK_CUDA(launch_reflag(pa, true, ctx->aux, 1));
    EK_CUDA(cudaEventRecord(ctx->ev_part, ctx->aux));
    EK_CUDA(cudaEventRecord(ctx->ev_join, ctx->aux));
  }
  EK_CUDA(ctx->fp32 ? launch_advection32(la, s) : launch_advection(la, s));
  ctx->launches += ctx->p.nspecies > 0 ? 2 : 1;
  if (ctx->P) {
    EK_CUDA(cudaStreamWaitEvent(s, ctx->ev_part, 0));
    EK_CUDA(launch_reflag(pa, true, s, 2));
    EK_CUDA(cudaStreamWaitEvent(s, ctx->ev_join, 0));
    ctx->launches += 10;
  }
  return EK_OK;
}

// A full step as a CUDA graph, replayed instead of ~30 separate launches.
// Only on a caller-provided stream (the legacy default stream cannot be
// captured); the graphs are dropped whenever a kernel argument changes (set-up,
// E or body force, stream).
ek_status step_graphed(ek_ctx* ctx) {
  const int parity = ctx->cur;
  if (!ctx->step_graph[parity]) {
    const long long l0 = ctx->launches;
    cudaGraph_t graph = nullptr;
    EK_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    ek_status st = enqueue_step(ctx);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    ctx->cur = parity;  // nothing ran yet
    if (st != EK_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return fail(ctx, EK_ERR_CUDA, std::string("step capture: ") + cudaGetErrorString(e));
    // keep the priority of the auxiliary stream on its captured kernels
    e = cudaGraphInstantiate(&ctx->step_graph[parity], graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, EK_ERR_CUDA, std::string("step graph: ") + cudaGetErrorString(e));
    ctx->graph_launches = ctx->launches - l0;
    ctx->launches = l0;
  }
  EK_CUDA(cudaGraphLaunch(ctx->step_graph[parity], ctx->stream));
  ctx->cur = 1 - parity;
  ctx->launches += ctx->graph_launches;
  return EK_OK;
}

ek_status ready(ek_ctx* ctx) {
  if (!ctx) return EK_ERR_ARG;
  if (ctx->broken) return fail(ctx, EK_ERR_STATE, "context is in an error state: " + ctx->err);
  EK_CUDA(cudaSetDevice(ctx->device));
  return run_setup(ctx);
}

size_t field_size(const ek_ctx* ctx, ek_field w) {
  const size_t N = (size_t)ctx->g.N;
  switch (w) {
    case EK_FIELD_POPULATIONS: return 19 * N;
    case EK_FIELD_VELOCITY: return 3 * N;
    case EK_FIELD_E_EXT:
    case EK_FIELD_BODY_FORCE: return 3;
    default: return N;
  }
}

// Checkpoint layout: a header, then the device arrays a step reads, each as
// stored (both population buffers, the species of the current one, Psi,
// particle and wall charge, Phi, u, node owners, wall mask, the particles'
// Psi_p boxes and records).  Scratch that every step rewrites before reading
// it (spectrum, internal force, sign bytes, assignment keys, S4 partial sums,
// transfer lists) is not part of it.
constexpr unsigned long long STATE_MAGIC = 0x3130545341454b45ull;
constexpr int STATE_VERSION = 1;

struct StateHeader {
  unsigned long long magic;
  int version;
  int nx, ny, nz, nspecies, fp32, P, boxmax;
  unsigned flags;
  double E[3], g[3];
  double qscale[EK_MAX_SPECIES];
};

struct StateArray {
  void* dev;
  size_t bytes;
};

std::vector<StateArray> state_arrays(ek_ctx* ctx) {
  const size_t N = (size_t)ctx->g.N, rs = ctx->rsz, K = (size_t)ctx->p.nspecies;
  const size_t ss = ctx->fp32 ? sizeof(int) : sizeof(double);
  // both population buffers: push streaming never writes the populations of
  // boundary nodes, so the other buffer keeps values of two steps back there
  return {{ctx->f[ctx->cur], 19 * N * rs},
          {ctx->f[1 - ctx->cur], 19 * N * rs},
          {ctx->rho[ctx->cur], K * N * ss},
          {ctx->psi, N * rs},
          {ctx->qpart, N * rs},
          {ctx->qwall, N * rs},
          {ctx->phi, N * rs},
          {ctx->u, 3 * N * rs},
          {ctx->owner, N * sizeof(int)},
          {ctx->wall, N},
          {ctx->psibox, (size_t)ctx->P * (size_t)ctx->boxmax * sizeof(double)},
          {ctx->dparts, (size_t)ctx->P * sizeof(DevParticle)}};
}

StateHeader state_header(const ek_ctx* ctx) {
  StateHeader h;
  memset(&h, 0, sizeof(h));
  h.magic = STATE_MAGIC;
  h.version = STATE_VERSION;
  h.nx = ctx->g.nx;
  h.ny = ctx->g.ny;
  h.nz = ctx->g.nz;
  h.nspecies = ctx->p.nspecies;
  h.fp32 = ctx->fp32;
  h.P = ctx->P;
  h.boxmax = ctx->boxmax;
  h.flags = ctx->p.flags;
  for (int d = 0; d < 3; ++d) {
    h.E[d] = ctx->ph.E[d];
    h.g[d] = ctx->ph.g[d];
  }
  for (int k = 0; k < EK_MAX_SPECIES; ++k) h.qscale[k] = ctx->ph.qscale[k];
  return h;
}

// FFT plans of the standalone solvers, one per device and shape, kept for
// the life of the process
cudaError_t cached_plan(int nx, int ny, int nz, PoissonPlan& plan) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int>, PoissonPlan> plans;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(dev, nx, ny, nz);
  auto it = plans.find(key);
  if (it == plans.end()) {
    std::string err;
    PoissonPlan p;
    e = poisson_plan_create(p, nx, ny, nz, err);
    if (e != cudaSuccess) return e;
    it = plans.emplace(key, p).first;
  }
  plan = it->second;
  return cudaSuccess;
}

}  // namespace

extern "C" {

ek_status ek_create(const ek_params* p, ek_ctx** out) {
  if (!p || !out) return EK_ERR_ARG;
  *out = nullptr;
  if (!edge_ok(p->nx) || !edge_ok(p->ny) || !edge_ok(p->nz) || p->nx % 2) return EK_ERR_ARG;
  // node indices of the FP32 kernels are 32-bit
  if ((long long)p->nx * p->ny * p->nz >= (1LL << 31)) return EK_ERR_ARG;
  if (!(p->nu > 0.0) || !(p->rho0 > 0.0) || !(p->bjerrum >= 0.0)) return EK_ERR_ARG;
  if (p->nspecies < 0 || p->nspecies > EK_MAX_SPECIES) return EK_ERR_ARG;
  for (int k = 0; k < p->nspecies; ++k)
    if (!(p->D[k] > 0.0 && p->D[k] <= 0.39) || !(p->bulk[k] >= 0.0)) return EK_ERR_ARG;
  ek_ctx* ctx = new (std::nothrow) ek_ctx();
  if (!ctx) return EK_ERR_NOMEM;
  ctx->p = *p;
  cudaGetDevice(&ctx->device);
  Grid& g = ctx->g;
  g.nx = p->nx;
  g.ny = p->ny;
  g.nz = p->nz;
  g.N = (long long)p->nx * p->ny * p->nz;
  Phys& ph = ctx->ph;
  memset(&ph, 0, sizeof(ph));
  ph.rho0 = p->rho0;
  const double tau_e = 3.0 * p->nu + 0.5;
  double tau_o = tau_e;
  if (p->magic > 0.0) tau_o = 0.5 + p->magic / (tau_e - 0.5);
  ph.lam_e = -1.0 / tau_e;
  ph.lam_o = -1.0 / tau_o;
  ph.bjerrum = p->bjerrum;
  ph.K = p->nspecies;
  ph.pv = (p->flags & EK_PV) ? 1 : 0;
  ph.flags = p->flags;
  ctx->fp32 = (p->flags & EK_FP32) ? 1 : 0;
  ph.fp32 = ctx->fp32;
  ctx->rsz = ctx->fp32 ? sizeof(float) : sizeof(double);
  // FP32 form: one species unit is 2^-e with 2^20 units or more per bulk density
  for (int k = 0; k < EK_MAX_SPECIES; ++k) {
    int e = 30;
    if (k < p->nspecies && p->bulk[k] > 0.0) e = (int)ceil(20.0 - log2(p->bulk[k]));
    ph.qscale[k] = ldexp(1.0, -e);
  }
  const double A0 = 1.0 + 2.0 * sqrt(2.0);
  for (int k = 0; k < p->nspecies; ++k) {
    ph.z[k] = (double)p->valence[k];
    ph.D[k] = p->D[k];
    ph.dcoef[k] = p->D[k] / A0;
    ph.hinvD[k] = 0.5 / p->D[k];
    ph.hz[k] = 0.5 * (double)p->valence[k];
  }
  update_derived(ph);
  std::string perr;
  if (poisson_plan_create(ctx->plan, g.nx, g.ny, g.nz, perr) != cudaSuccess) {
    delete ctx;
    return EK_ERR_ARG;
  }
  const size_t N = (size_t)g.N;
  const int K = std::max(p->nspecies, 1);
  if (ctx->fp32 && lb32_prepare() != cudaSuccess) {
    delete ctx;
    return EK_ERR_CUDA;
  }
  bool ok = true;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (ok && alloc_fault_due()) ok = false;  // the test hook's injected failure
    if (ok && cudaMalloc(ptr, bytes) != cudaSuccess) ok = false;
  };
  const size_t rsz = ctx->rsz;  // populations, Phi, Psi, charges and u share the real size
  const size_t ssz = ctx->fp32 ? sizeof(int) : sizeof(double);
  for (int b = 0; b < 2; ++b) {
    alloc(&ctx->f[b], 19 * N * rsz);
    alloc(&ctx->rho[b], K * N * ssz);
  }
  alloc(&ctx->phi, N * rsz);
  alloc(&ctx->psi, N * rsz);
  alloc(&ctx->qpart, N * rsz);
  alloc(&ctx->qwall, N * rsz);
  alloc(&ctx->u, 3 * N * rsz);
  alloc(&ctx->ifield, 3 * N * rsz);
  {
    // lattice-block partial sums of S2: one per block of its grid
    if (ctx->fp32) ctx->nzb = lb32_segments(g, p->nspecies, (p->flags & EK_PV) != 0);
    if (ctx->fp32) ctx->advseg = adv32_segments(g, false);
    const dim3 lg = ctx->fp32 ? lattice_grid32(g, ctx->nzb) : lattice_grid(g);
    ctx->nipart = (int)(lg.x * lg.y * lg.z);
    // the FP32 segment length may be retuned down to 2 planes (ek_batch_tune)
    ctx->nipart_cap = ctx->fp32 ? (int)(lg.x * lg.y) * std::max(1, (g.nz + 1) / 2) : ctx->nipart;
    ctx->nipart_cap = std::max(ctx->nipart_cap, ctx->nipart);
  }
  alloc((void**)&ctx->ipart, (size_t)ctx->nipart_cap * 3 * sizeof(double));
  alloc((void**)&ctx->fkey, N * sizeof(unsigned long long));
  alloc((void**)&ctx->vsig, N);
  alloc((void**)&ctx->tmp, N * sizeof(double));
  alloc((void**)&ctx->owner, N * sizeof(int));
  alloc((void**)&ctx->owner_prev, N * sizeof(int));
  alloc((void**)&ctx->wall, N);
  alloc(&ctx->spectrum, poisson_spectrum_bytes(g.nx, g.ny, g.nz));
  ctx->xfer_cap = (int)std::min<long long>(19LL * g.N, 1LL << 22);
  alloc((void**)&ctx->xfer, (size_t)ctx->xfer_cap * sizeof(Transfer));
  alloc((void**)&ctx->xfer_count, sizeof(int));
  alloc((void**)&ctx->surf_count, sizeof(int));
  alloc((void**)&ctx->tie_list, (size_t)ctx->tie_cap * sizeof(int));
  alloc((void**)&ctx->tie_count, sizeof(int));
  alloc((void**)&ctx->status, sizeof(int));
  alloc((void**)&ctx->ticket, sizeof(int));
  if (!ok) {
    ek_destroy(ctx);
    return EK_ERR_NOMEM;
  }
  cudaMemset(ctx->wall, 0, N);
  cudaMemset(ctx->qwall, 0, N * rsz);
  cudaMemset(ctx->phi, 0, N * rsz);
  cudaMemset(ctx->u, 0, 3 * N * rsz);
  cudaMemset(ctx->ifield, 0, 3 * N * rsz);
  cudaMemset(ctx->fkey, 0xFF, N * sizeof(unsigned long long));
  cudaMemset(ctx->xfer_count, 0, sizeof(int));
  cudaMemset(ctx->tie_count, 0, sizeof(int));
  cudaMemset(ctx->status, 0, sizeof(int));
  cudaMemset(ctx->ticket, 0, sizeof(int));
  for (int b = 0; b < 2; ++b) {
    cudaMemset(ctx->f[b], 0, 19 * N * rsz);
    cudaMemset(ctx->rho[b], 0, K * N * ssz);
  }
  // the particle chain on the auxiliary stream is latency-bound and shares the
  // SMs with the advection: its blocks go first
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (cudaStreamCreateWithPriority(&ctx->aux, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_lb, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_part, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    ek_destroy(ctx);
    return EK_ERR_CUDA;
  }
  ek_status st = run_setup(ctx);
  if (st != EK_OK) {
    ek_destroy(ctx);
    return st;
  }
  *out = ctx;
  return EK_OK;
}

void ek_debug_fail_alloc(int n) { g_alloc_fault.store(n > 0 ? n : 0); }

ek_status ek_destroy(ek_ctx* ctx) {
  if (!ctx) return EK_ERR_ARG;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  void* ptrs[] = {ctx->f[0], ctx->f[1], ctx->rho[0], ctx->rho[1], ctx->phi, ctx->psi, ctx->qpart,
                  ctx->qwall, ctx->u, ctx->tmp, ctx->owner, ctx->owner_prev, ctx->wall,
                  ctx->spectrum, ctx->dparts, ctx->psibox, ctx->fpart, ctx->surf, ctx->xfer,
                  ctx->xfer_count, ctx->surf_count, ctx->status, ctx->ifield, ctx->ipart,
                  ctx->fkey, ctx->psum, ctx->vsig, ctx->ticket, ctx->pticket, ctx->pstage,
                  ctx->tie_list, ctx->tie_count, ctx->tpart};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  poisson_plan_destroy(ctx->plan);
  drop_graphs(ctx);
  if (ctx->aux) {
    cudaStreamSynchronize(ctx->aux);
    cudaStreamDestroy(ctx->aux);
  }
  if (ctx->ev_lb) cudaEventDestroy(ctx->ev_lb);
  if (ctx->ev_part) cudaEventDestroy(ctx->ev_part);
  if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  delete ctx;
  return EK_OK;
}

ek_status ek_add_particle(ek_ctx* ctx, const double pos[3], const double vel[3],
                          const double omega[3], double radius, double charge, double rho_p,
                          int fixed, int* out_id) {
  if (!ctx || !pos) return EK_ERR_ARG;
  if (ctx->broken) return fail(ctx, EK_ERR_STATE, "context is in an error state");
  const int nmin = std::min(ctx->g.nx, std::min(ctx->g.ny, ctx->g.nz));
  if (!(radius > 0.0) || 2.0 * radius + 6.0 > (double)nmin)
    return fail(ctx, EK_ERR_ARG, "radius must be positive with 2R + 6 <= min(nx, ny, nz)");
  if (!(rho_p > 0.0) || !isfinite(charge)) return fail(ctx, EK_ERR_ARG, "bad rho_p or charge");
  EK_CUDA(cudaSetDevice(ctx->device));
  if (!ctx->setup_pending) {
    ek_status st = download_particles(ctx);
    if (st != EK_OK) return st;
  }
  DevParticle q;
  memset(&q, 0, sizeof(q));
  const int nn[3] = {ctx->g.nx, ctx->g.ny, ctx->g.nz};
  for (int d = 0; d < 3; ++d) {
    if (!isfinite(pos[d])) return fail(ctx, EK_ERR_ARG, "non-finite position");
    double x = fmod(pos[d], (double)nn[d]);
    if (x < 0.0) x += nn[d];
    if (x >= nn[d]) x -= nn[d];
    q.pos[d] = x;
    q.vel[d] = vel ? vel[d] : 0.0;
    q.omega[d] = omega ? omega[d] : 0.0;
  }
  q.radius = radius;
  q.charge = charge;
  q.mass = rho_p * 4.0 / 3.0 * M_PI * pow(radius, 3.0);
  q.inertia = 0.4 * q.mass * pow(radius, 2.0);
  q.fixed = fixed ? 1 : 0;
  ctx->hparts.resize(ctx->P);
  ctx->hparts.push_back(q);
  if (ctx->P + 1 > ctx->Pcap) {
    const int cap = std::max(16, 2 * ctx->Pcap);
    DevParticle* nd = nullptr;
    EK_CUDA(cudaMalloc(&nd, cap * sizeof(DevParticle)));
    if (ctx->dparts) cudaFree(ctx->dparts);
    ctx->dparts = nd;
    ctx->Pcap = cap;
  }
  ctx->P += 1;
  ctx->setup_pending = true;
  if (out_id) *out_id = ctx->P - 1;
  return EK_OK;
}

ek_status ek_set_field(ek_ctx* ctx, ek_field which, int component, const double* src,
                       size_t count, int src_on_device) {
  ek_status st = ready(ctx);
  if (st != EK_OK) return st;
  if (!src) return fail(ctx, EK_ERR_ARG, "null source");
  if (count != field_size(ctx, which)) return fail(ctx, EK_ERR_ARG, "count does not match the field size");
  const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t N = (size_t)ctx->g.N;
  const Grid& g = ctx->g;
  cudaStream_t s = ctx->stream;
  const bool f32 = ctx->fp32 != 0;
  switch (which) {
    case EK_FIELD_SPECIES:
      if (component < 0 || component >= ctx->p.nspecies) return fail(ctx, EK_ERR_ARG, "bad species index");
      if (f32) {
        EK_CUDA(cudaMemcpyAsync(ctx->tmp, src, N * sizeof(double), kind, s));
        EK_CUDA(convert32(CONV_SPC_FROM_F64, g, 0, ctx->ph.qscale[component], ctx->tmp,
                          (int*)ctx->rho[ctx->cur] + component * N, ctx->status, s));
      } else {
        EK_CUDA(cudaMemcpyAsync((double*)ctx->rho[ctx->cur] + component * N, src, N * sizeof(double), kind, s));
      }
      break;
    case EK_FIELD_POPULATIONS:
      if (f32) {
        for (int i = 0; i < Q; ++i) {
          EK_CUDA(cudaMemcpyAsync(ctx->tmp, src + i * N, N * sizeof(double), kind, s));
          EK_CUDA(convert32(CONV_POP_FROM_F64, g, i, ctx->ph.rho0, ctx->tmp, ctx->f[ctx->cur], ctx->status, s));
        }
      } else {
        EK_CUDA(cudaMemcpyAsync(ctx->f[ctx->cur], src, 19 * N * sizeof(double), kind, s));
      }
      break;
    case EK_FIELD_VELOCITY:
      if (f32) {
        // stage the FP64 velocity in the idle population buffer (19 N floats >= 3 N doubles)
        double* u3 = (double*)ctx->f[1 - ctx->cur];
        EK_CUDA(cudaMemcpyAsync(u3, src, 3 * N * sizeof(double), kind, s));
        EK_CUDA(set_velocity32(g, ctx->owner, (float*)ctx->f[ctx->cur], u3, ctx->ph.rho0, s));
        for (int d = 0; d < 3; ++d)
          EK_CUDA(convert32(CONV_F64_TO_F32, g, 0, 0.0, u3 + d * N, (float*)ctx->u + d * N, ctx->status, s));
      } else {
        EK_CUDA(cudaMemcpyAsync(ctx->u, src, 3 * N * sizeof(double), kind, s));
        k_set_velocity<<<nblk(g.N), 256, 0, s>>>(g, ctx->owner, (double*)ctx->f[ctx->cur], (const double*)ctx->u);
        EK_CUDA(cudaGetLastError());
      }
      break;
    case EK_FIELD_E_EXT:
    case EK_FIELD_BODY_FORCE: {
      double v[3];
      if (src_on_device) {
        EK_CUDA(cudaMemcpyAsync(v, src, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        EK_CUDA(cudaStreamSynchronize(s));
      } else {
        memcpy(v, src, 3 * sizeof(double));  // read on the host: no wait for the stream
      }
      bool changed = false;
      for (int d = 0; d < 3; ++d) {
        if (!isfinite(v[d])) return fail(ctx, EK_ERR_ARG, "non-finite vector");
        double& dst = which == EK_FIELD_E_EXT ? ctx->ph.E[d] : ctx->ph.g[d];
        changed |= dst != v[d];
        dst = v[d];
      }
      update_derived(ctx->ph);
      // the vectors reach the kernels as launch arguments, so captured steps
      // hold the old value
      if (changed) drop_graphs(ctx);
      break;
    }
    case EK_FIELD_WALL:
      EK_CUDA(cudaMemcpyAsync(ctx->tmp, src, N * sizeof(double), kind, s));
      k_double_to_u8<<<nblk(g.N), 256, 0, s>>>(g, ctx->tmp, ctx->wall);
      EK_CUDA(cudaGetLastError());
      ctx->setup_pending = true;
      return run_setup(ctx);
    case EK_FIELD_WALL_CHARGE:
      if (f32) {
        EK_CUDA(cudaMemcpyAsync(ctx->tmp, src, N * sizeof(double), kind, s));
        EK_CUDA(convert32(CONV_F64_TO_F32, g, 0, 0.0, ctx->tmp, ctx->qwall, ctx->status, s));
      } else {
        EK_CUDA(cudaMemcpyAsync(ctx->qwall, src, N * sizeof(double), kind, s));
      }
      ctx->has_qwall = true;
      break;
    default:
      return fail(ctx, EK_ERR_ARG, "field is read-only");
  }
  EK_CUDA(cudaStreamSynchronize(s));
  return check_status(ctx);
}

ek_status ek_get_fields(ek_ctx* ctx, ek_field which, int component, double* dst, size_t count,
                        int dst_on_device) {
  if (!ctx) return EK_ERR_ARG;
  if (!ctx->broken) {
    ek_status st = ready(ctx);
    if (st != EK_OK) return st;
  }
  if (!dst) return fail(ctx, EK_ERR_ARG, "null destination");
  if (count != field_size(ctx, which)) return fail(ctx, EK_ERR_ARG, "count does not match the field size");
  const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t N = (size_t)ctx->g.N;
  const Grid& g = ctx->g;
  cudaStream_t s = ctx->stream;
  const bool f32 = ctx->fp32 != 0;
  // copy one converted N-element block (tmp) to dst + offset
  auto out_block = [&](size_t offset) -> cudaError_t {
    return cudaMemcpyAsync(dst + offset, ctx->tmp, N * sizeof(double), kind, s);
  };
  // a real field of the current form -> dst + offset
  auto out_real = [&](const void* src, size_t offset) -> cudaError_t {
    if (!f32) return cudaMemcpyAsync(dst + offset, src, N * sizeof(double), kind, s);
    cudaError_t e = convert32(CONV_F32_TO_F64, g, 0, 0.0, src, ctx->tmp, ctx->status, s);
    return e != cudaSuccess ? e : out_block(offset);
  };
  switch (which) {
    case EK_FIELD_SPECIES:
      if (component < 0 || component >= ctx->p.nspecies) return fail(ctx, EK_ERR_ARG, "bad species index");
      if (f32) {
        EK_CUDA(convert32(CONV_SPC_TO_F64, g, 0, ctx->ph.qscale[component],
                          (const int*)ctx->rho[ctx->cur] + component * N, ctx->tmp, ctx->status, s));
        EK_CUDA(out_block(0));
      } else {
        EK_CUDA(cudaMemcpyAsync(dst, (const double*)ctx->rho[ctx->cur] + component * N,
                                N * sizeof(double), kind, s));
      }
      break;
    case EK_FIELD_POPULATIONS:
      if (f32) {
        for (int i = 0; i < Q; ++i) {
          EK_CUDA(convert32(CONV_POP_TO_F64, g, i, ctx->ph.rho0, ctx->f[ctx->cur], ctx->tmp, ctx->status, s));
          EK_CUDA(out_block(i * N));
        }
      } else {
        EK_CUDA(cudaMemcpyAsync(dst, ctx->f[ctx->cur], 19 * N * sizeof(double), kind, s));
      }
      break;
    case EK_FIELD_VELOCITY:
      for (int d = 0; d < 3; ++d) EK_CUDA(out_real((const char*)ctx->u + d * N * ctx->rsz, d * N));
      break;
    case EK_FIELD_E_EXT:
    case EK_FIELD_BODY_FORCE: {
      const double* v = which == EK_FIELD_E_EXT ? ctx->ph.E : ctx->ph.g;
      EK_CUDA(cudaMemcpyAsync(dst, v, 3 * sizeof(double),
                              dst_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s));
      break;
    }
    case EK_FIELD_WALL:
      k_u8_to_double<<<nblk(g.N), 256, 0, s>>>(g, ctx->wall, ctx->tmp);
      EK_CUDA(cudaGetLastError());
      EK_CUDA(out_block(0));
      break;
    case EK_FIELD_WALL_CHARGE:
      EK_CUDA(out_real(ctx->qwall, 0));
      break;
    case EK_FIELD_DENSITY:
      if (f32) EK_CUDA(density32(g, (const float*)ctx->f[ctx->cur], ctx->ph.rho0, ctx->tmp, s));
      else k_density<<<nblk(g.N), 256, 0, s>>>(g, (const double*)ctx->f[ctx->cur], ctx->tmp);
      EK_CUDA(cudaGetLastError());
      EK_CUDA(out_block(0));
      break;
    case EK_FIELD_PHI:
      EK_CUDA(out_real(ctx->phi, 0));
      break;
    case EK_FIELD_PSI:
      if (f32) {
        EK_CUDA(out_real(ctx->psi, 0));  // clamped to 1 by S5
      } else {
        k_psi_clamped<<<nblk(g.N), 256, 0, s>>>(g, (const double*)ctx->psi, ctx->tmp);
        EK_CUDA(cudaGetLastError());
        EK_CUDA(out_block(0));
      }
      break;
    case EK_FIELD_OWNER:
      k_int_to_double<<<nblk(g.N), 256, 0, s>>>(g, ctx->owner, ctx->tmp);
      EK_CUDA(cudaGetLastError());
      EK_CUDA(out_block(0));
      break;
    case EK_FIELD_CHARGE:
      EK_CUDA(charge_density(g, ctx->ph, ctx->rho[ctx->cur], ctx->has_qwall ? ctx->qwall : nullptr,
                             ctx->qpart, ctx->tmp, s));
      EK_CUDA(out_block(0));
      break;
    default:
      return fail(ctx, EK_ERR_ARG, "unknown field");
  }
  EK_CUDA(cudaStreamSynchronize(s));
  return EK_OK;
}

ek_status ek_step_async(ek_ctx* ctx, int nsteps) {
  ek_status st = ready(ctx);
  if (st != EK_OK) return st;
  if (nsteps < 0) return fail(ctx, EK_ERR_ARG, "nsteps < 0");
  for (int t = 0; t < nsteps; ++t) {
    st = ctx->stream ? step_graphed(ctx) : enqueue_step(ctx);
    if (st != EK_OK) return st;
  }
  return EK_OK;
}

ek_status ek_step(ek_ctx* ctx, int nsteps) {
  ek_status st = ek_step_async(ctx, nsteps);
  if (st != EK_OK) return st;
  return check_status(ctx);
}

ek_status ek_step_timed(ek_ctx* ctx, int nsteps, double stage_ms[6]) {
  ek_status st = ready(ctx);
  if (st != EK_OK) return st;
  if (nsteps < 0 || !stage_ms) return fail(ctx, EK_ERR_ARG, "bad arguments");
  cudaEvent_t ev[6];
  for (int i = 0; i < 6; ++i) EK_CUDA(cudaEventCreate(&ev[i]));
  double acc[5] = {0, 0, 0, 0, 0};
  cudaEvent_t first = nullptr;
  EK_CUDA(cudaEventCreate(&first));
  EK_CUDA(cudaEventRecord(first, ctx->stream));
  for (int t = 0; t < nsteps && st == EK_OK; ++t) {
    EK_CUDA(cudaEventRecord(ev[0], ctx->stream));
    st = enqueue_stage(ctx, 1);
    if (st == EK_OK) { EK_CUDA(cudaEventRecord(ev[1], ctx->stream)); st = enqueue_stage(ctx, 2, ev[2]); }
    if (st == EK_OK) { EK_CUDA(cudaEventRecord(ev[3], ctx->stream)); st = enqueue_stage(ctx, 4); }
    if (st == EK_OK) { EK_CUDA(cudaEventRecord(ev[4], ctx->stream)); st = enqueue_stage(ctx, 5); }
    if (st != EK_OK) break;
    EK_CUDA(cudaEventRecord(ev[5], ctx->stream));
    EK_CUDA(cudaEventSynchronize(ev[5]));
    float ms;
    for (int i = 0; i < 5; ++i) {
      EK_CUDA(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
      acc[i] += ms;
    }
  }
  float total = 0.0f;
  EK_CUDA(cudaEventRecord(ev[5], ctx->stream));
  EK_CUDA(cudaEventSynchronize(ev[5]));
  EK_CUDA(cudaEventElapsedTime(&total, first, ev[5]));
  for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
  cudaEventDestroy(first);
  if (st != EK_OK) return st;
  for (int i = 0; i < 5; ++i) stage_ms[i] += acc[i];
  stage_ms[5] += total;
  return check_status(ctx);
}

long long ek_kernel_launches(const ek_ctx* ctx) { return ctx ? ctx->launches : 0; }

ek_status ek_run_stage(ek_ctx* ctx, int stage) {
  ek_status st = ready(ctx);
  if (st != EK_OK) return st;
  st = enqueue_stage(ctx, stage);
  if (st != EK_OK) return st;
  return check_status(ctx);
}

ek_status ek_get_particles(ek_ctx* ctx, ek_particle* dst, int count) {
  if (!ctx || (!dst && count > 0) || count < 0) return EK_ERR_ARG;
  if (!ctx->broken) {
    ek_status st = ready(ctx);
    if (st != EK_OK) return st;
  }
  ek_status st = download_particles(ctx);
  if (st != EK_OK) return st;
  for (int i = 0; i < std::min(count, ctx->P); ++i) {
    const DevParticle& q = ctx->hparts[i];
    ek_particle& o = dst[i];
    for (int d = 0; d < 3; ++d) {
      o.pos[d] = q.pos[d];
      o.vel[d] = q.vel[d];
      o.omega[d] = q.omega[d];
      o.force[d] = q.force[d];
      o.torque[d] = q.torque[d];
    }
    o.radius = q.radius;
    o.charge = q.charge;
    o.rho_p = q.mass / (4.0 / 3.0 * M_PI * pow(q.radius, 3.0));
    o.fixed = q.fixed;
  }
  return EK_OK;
}

ek_status ek_get_particles_async(ek_ctx* ctx, ek_particle* dst, int count) {
  if (!ctx || (!dst && count > 0) || count < 0) return EK_ERR_ARG;
  if (!ctx->broken) {
    ek_status st = ready(ctx);
    if (st != EK_OK) return st;
  }
  const int n = std::min(count, ctx->P);
  if (n == 0) return EK_OK;
  k_pack_particles<<<(n + 127) / 128, 128, 0, ctx->stream>>>(ctx->dparts, n, ctx->pstage);
  EK_CUDA(cudaGetLastError());
  EK_CUDA(cudaMemcpyAsync(dst, ctx->pstage, (size_t)n * sizeof(ek_particle), cudaMemcpyDefault,
                          ctx->stream));
  return EK_OK;
}

ek_status ek_get_state(ek_ctx* ctx, void* buf, size_t* bytes) {
  if (!ctx || !bytes) return EK_ERR_ARG;
  ek_status st = ready(ctx);
  if (st != EK_OK) return st;
  const std::vector<StateArray> arrays = state_arrays(ctx);
  size_t total = sizeof(StateHeader);
  for (const StateArray& a : arrays) total += a.bytes;
  if (!buf) {
    *bytes = total;
    return EK_OK;
  }
  if (*bytes < total) {
    *bytes = total;
    return fail(ctx, EK_ERR_ARG, "checkpoint buffer too small");
  }
  const StateHeader h = state_header(ctx);
  unsigned char* out = static_cast<unsigned char*>(buf);
  memcpy(out, &h, sizeof(h));
  size_t off = sizeof(h);
  for (const StateArray& a : arrays) {
    if (a.bytes) EK_CUDA(cudaMemcpyAsync(out + off, a.dev, a.bytes, cudaMemcpyDeviceToHost, ctx->stream));
    off += a.bytes;
  }
  EK_CUDA(cudaStreamSynchronize(ctx->stream));
  *bytes = total;
  return check_status(ctx);
}

ek_status ek_set_state(ek_ctx* ctx, const void* buf, size_t bytes) {
  if (!ctx || !buf) return EK_ERR_ARG;
  ek_status st = ready(ctx);  // a pending set-up must not overwrite the restored state later
  if (st != EK_OK) return st;
  StateHeader h;
  if (bytes < sizeof(h)) return fail(ctx, EK_ERR_ARG, "not a checkpoint (too short)");
  memcpy(&h, buf, sizeof(h));
  if (h.magic != STATE_MAGIC || h.version != STATE_VERSION)
    return fail(ctx, EK_ERR_ARG, "not a checkpoint of this library version");
  const StateHeader mine = state_header(ctx);
  bool same = h.nx == mine.nx && h.ny == mine.ny && h.nz == mine.nz && h.nspecies == mine.nspecies &&
              h.fp32 == mine.fp32 && h.P == mine.P && h.boxmax == mine.boxmax && h.flags == mine.flags;
  for (int k = 0; k < EK_MAX_SPECIES; ++k) same = same && h.qscale[k] == mine.qscale[k];
  if (!same)
    return fail(ctx, EK_ERR_STATE,
                "checkpoint of a different system (shape, species, storage form, flags, particle "
                "count or size, or species units)");
  const std::vector<StateArray> arrays = state_arrays(ctx);
  size_t total = sizeof(StateHeader);
  for (const StateArray& a : arrays) total += a.bytes;
  if (bytes < total) return fail(ctx, EK_ERR_ARG, "checkpoint truncated");
  EK_CUDA(cudaStreamSynchronize(ctx->stream));
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  size_t off = sizeof(h);
  for (const StateArray& a : arrays) {
    if (a.bytes) EK_CUDA(cudaMemcpyAsync(a.dev, in + off, a.bytes, cudaMemcpyHostToDevice, ctx->stream));
    off += a.bytes;
  }
  EK_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int d = 0; d < 3; ++d) {
    ctx->ph.E[d] = h.E[d];
    ctx->ph.g[d] = h.g[d];
  }
  if (ctx->P) {
    // the particle records are the last array
    ctx->hparts.resize(ctx->P);
    memcpy(ctx->hparts.data(), in + off - (size_t)ctx->P * sizeof(DevParticle),
           (size_t)ctx->P * sizeof(DevParticle));
  }
  drop_graphs(ctx);  // E and the body force are launch arguments of the captured steps
  return EK_OK;
}

int ek_num_particles(const ek_ctx* ctx) { return ctx ? ctx->P : 0; }

ek_status ek_set_stream(ek_ctx* ctx, void* stream) {
  if (!ctx) return EK_ERR_ARG;
  if ((cudaStream_t)stream != ctx->stream) {
    EK_CUDA(cudaStreamSynchronize(ctx->stream));
    drop_graphs(ctx);
  }
  ctx->stream = (cudaStream_t)stream;
  return EK_OK;
}

ek_status ek_sync(ek_ctx* ctx) {
  if (!ctx) return EK_ERR_ARG;
  return check_status(ctx);
}

const char* ek_last_error(const ek_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void ek_lattice_dirs(int c[57]) {
  for (int i = 0; i < Q; ++i) {
    c[3 * i] = HCX[i];
    c[3 * i + 1] = HCY[i];
    c[3 * i + 2] = HCZ[i];
  }
}

size_t ek_poisson_scratch_bytes(int nx, int ny, int nz) { return poisson_spectrum_bytes(nx, ny, nz); }

ek_status ek_poisson_solve(const double* q, double* phi, int nx, int ny, int nz, double bjerrum,
                           void* spectrum, void* stream) {
  if (!q || !phi || !spectrum || !edge_ok(nx) || !edge_ok(ny) || !edge_ok(nz) || nx % 2 ||
      !(bjerrum >= 0.0))
    return EK_ERR_ARG;
  PoissonPlan plan;
  if (cached_plan(nx, ny, nz, plan) != cudaSuccess) return EK_ERR_CUDA;
  Phys ph;
  memset(&ph, 0, sizeof(ph));
  ph.bjerrum = bjerrum;
  if (poisson_solve(plan, q, nullptr, nullptr, nullptr, ph, phi, (double2*)spectrum,
                    (cudaStream_t)stream) != cudaSuccess)
    return EK_ERR_CUDA;
  return EK_OK;
}

size_t ek_poisson_mg_scratch_bytes(int nx, int ny, int nz) {
  if (!edge_ok(nx) || !edge_ok(ny) || !edge_ok(nz) || nx % 2) return 0;
  return poisson_mg_scratch_bytes(nx, ny, nz);
}

ek_status ek_poisson_solve_mg(const double* q, double* phi, int nx, int ny, int nz, double bjerrum,
                              double tol, int max_cycles, void* scratch, void* stream, int* cycles,
                              double* residual) {
  if (!q || !phi || !scratch || !edge_ok(nx) || !edge_ok(ny) || !edge_ok(nz) || nx % 2 ||
      !(bjerrum >= 0.0) || !(tol > 0.0) || max_cycles < 1)
    return EK_ERR_ARG;
  int coarse[3];
  poisson_mg_levels(nx, ny, nz, coarse);
  PoissonPlan plan;
  if (cached_plan(coarse[0], coarse[1], coarse[2], plan) != cudaSuccess) return EK_ERR_CUDA;
  if (poisson_solve_mg(plan, q, phi, nx, ny, nz, bjerrum, tol, max_cycles, scratch,
                       (cudaStream_t)stream, cycles, residual) != cudaSuccess)
    return EK_ERR_CUDA;
  return EK_OK;
}

size_t ek_poisson_cg_scratch_bytes(int nx, int ny, int nz) {
  if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz >= (1LL << 31)) return 0;
  return poisson_cg_scratch_bytes(nx, ny, nz);
}

ek_status ek_poisson_solve_cg(const double* q, const double* eps, const unsigned char* fixed,
                              const double* phi_fixed, double* phi, int nx, int ny, int nz,
                              double bjerrum, double tol, int max_iter, void* scratch, void* stream,
                              int* iters, double* residual) {
  if (!q || !phi || !scratch || nx < 1 || ny < 1 || nz < 1 ||
      (long long)nx * ny * nz >= (1LL << 31) || !(bjerrum >= 0.0) || !(tol > 0.0) || max_iter < 1)
    return EK_ERR_ARG;
  bool bad = false;
  if (poisson_solve_cg(q, eps, fixed, phi_fixed, phi, nx, ny, nz, bjerrum, tol, max_iter, scratch,
                       (cudaStream_t)stream, iters, residual, &bad) != cudaSuccess)
    return EK_ERR_CUDA;
  return bad ? EK_ERR_ARG : EK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched ensemble: many independent systems (each an ek_ctx of its own box
// size, salt, field and particles) advanced together.  One step of all of
// them is one CUDA graph: the systems are branches of the graph (spread over
// `width` branch streams at capture), so the GPU runs their kernels side by
// side and one graph launch replaces a few dozen launches per system.
// ---------------------------------------------------------------------------
struct ek_batch {
  std::vector<ek_ctx*> sys;
  cudaStream_t stream = nullptr;  // where the step graphs are launched
  bool own_stream = false;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // keyed by the first system's ping-pong parity
  std::vector<int> cur_at[2];                      // every system's parity at capture
  std::vector<unsigned long long> version_at[2];
  std::vector<long long> dlaunch[2];               // each system's launches per replay
  int width = 16;   // branch streams used at capture
  int planes = 4;   // FP32 S2 segment length (planes per block)
  int overlap = 1;  // particle chain beside S3 in each system
  int device = 0;
  std::string err;
  // Stage launches over all systems (FP32 systems with one species count and
  // one partial-volume choice): each kernel of the step runs once for the
  // whole batch over a list of (system, block) ranges instead of once per
  // system.  Per parity key: one device block holding the argument tables and
  // the ranges, and the launches made from it.
  bool fusable = false;
  int fuse = 0;  // 1: stage launches over all systems; 0: a graph branch per system
  struct Launch {
    int variant = 0;    // FFT kernel variant
    size_t slot = 0;    // byte offset of its BatchSlot ranges in the block
    int nslot = 0, ctas = 0;
  };
  struct Fused {
    char* dev = nullptr;
    size_t o_pre = 0, o_post = 0, o_lb = 0, o_pa = 0;  // argument tables
    Launch part[PK_COUNT];
    Launch lb, adv;
    std::vector<Launch> fft[3];  // per pass, one per kernel variant
    std::vector<int> s1_alone;   // systems whose S1 runs by itself (other edges)
  } fused[2];
  cudaStream_t aux = nullptr;  // the particle chain beside S3 in the fused step
  cudaEvent_t ev_lb = nullptr, ev_part = nullptr;
  // fuse == 2: the particle kernels (but the forces) as three persistent
  // launches with grid barriers; dstatus[0] is the batch's status word, then
  // three barrier blocks of four words
  int* dstatus = nullptr;
  int chain_ctas = 0;
  long long limit_ns = 1000000000LL;  // a barrier wait gives up after this
  int leave_cta = -1;                 // failure-detection test hook
};

namespace {

ek_status bfail(ek_batch* b, ek_status st, const std::string& msg) {
  b->err = msg;
  return st;
}

void batch_drop(ek_batch* b) {
  if ((b->fused[0].dev || b->fused[1].dev) && b->stream) cudaStreamSynchronize(b->stream);
  for (int i = 0; i < 2; ++i) {
    if (b->fused[i].dev) cudaFree(b->fused[i].dev);
    b->fused[i] = ek_batch::Fused();
  }
  for (int i = 0; i < 2; ++i) {
    if (b->graph[i]) cudaGraphExecDestroy(b->graph[i]);
    b->graph[i] = nullptr;
    b->cur_at[i].clear();
    b->version_at[i].clear();
    b->dlaunch[i].clear();
  }
}

// apply the batch's segment length and overlap choice to every system
void batch_apply(ek_batch* b) {
  for (ek_ctx* c : b->sys) {
    int nzb = c->nzb;
    if (c->fp32) nzb = std::max(1, (c->g.nz + b->planes - 1) / b->planes);
    const int xt = (c->g.nx + TILE_X - 1) / TILE_X, yt = (c->g.ny + TILE_Y - 1) / TILE_Y;
    if (c->fp32 && xt * yt * nzb > c->nipart_cap) nzb = c->nipart_cap / (xt * yt);
    if (nzb != c->nzb || c->overlap != b->overlap) {
      c->nzb = nzb;
      if (c->fp32) c->nipart = xt * yt * nzb;
      c->overlap = b->overlap;
      drop_graphs(c);
    }
  }
}

ek_status batch_capture(ek_batch* b, int key) {
  const int width = std::max(1, std::min<int>(b->width, (int)b->branch.size()));
  std::vector<int> cur0(b->sys.size());
  std::vector<cudaStream_t> saved(b->sys.size());
  std::vector<long long> l0v(b->sys.size());
  for (size_t i = 0; i < b->sys.size(); ++i) {
    cur0[i] = b->sys[i]->cur;
    saved[i] = b->sys[i]->stream;
    l0v[i] = b->sys[i]->launches;
  }
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return bfail(b, EK_ERR_CUDA, "batch capture could not start");
  ek_status st = EK_OK;
  if (cudaEventRecord(b->ev_fork, b->stream) != cudaSuccess) st = EK_ERR_CUDA;
  for (int w = 0; w < width && st == EK_OK; ++w)
    if (cudaStreamWaitEvent(b->branch[w], b->ev_fork, 0) != cudaSuccess) st = EK_ERR_CUDA;
  for (size_t i = 0; i < b->sys.size() && st == EK_OK; ++i) {
    ek_ctx* c = b->sys[i];
    c->stream = b->branch[i % width];
    st = enqueue_step(c);
    c->stream = saved[i];
  }
  for (int w = 0; w < width && st == EK_OK; ++w) {
    if (cudaEventRecord(b->ev_join[w], b->branch[w]) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->ev_join[w], 0) != cudaSuccess)
      st = EK_ERR_CUDA;
  }
  const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  for (size_t i = 0; i < b->sys.size(); ++i) b->sys[i]->cur = cur0[i];  // nothing ran yet
  if (st != EK_OK || e != cudaSuccess) {
    for (size_t i = 0; i < b->sys.size(); ++i) b->sys[i]->launches = l0v[i];
    if (graph) cudaGraphDestroy(graph);
    return bfail(b, st != EK_OK ? st : EK_ERR_CUDA, "batch capture failed");
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->graph[key], graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return bfail(b, EK_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(ei));
  // the capture counted its launches on the systems: take them back and add
  // them per replay
  b->dlaunch[key].resize(b->sys.size());
  for (size_t i = 0; i < b->sys.size(); ++i) {
    b->dlaunch[key][i] = b->sys[i]->launches - l0v[i];
    b->sys[i]->launches = l0v[i];
  }
  b->cur_at[key] = cur0;
  b->version_at[key].resize(b->sys.size());
  for (size_t i = 0; i < b->sys.size(); ++i) b->version_at[key][i] = b->sys[i]->version;
  return EK_OK;
}

// The device block of the fused step for the systems' current parities: the
// particle arguments before and after S2's buffer swap, the S2/S3 entries,
// the S1 pass arguments, and per launch the ranges of the systems with work.
ek_status fused_build(ek_batch* b, int key) {
  ek_batch::Fused& F = b->fused[key];
  const size_t n = b->sys.size();
  const size_t pas = poisson_batch_args_size();
  std::vector<PartArgs> pre(n), post(n);
  std::vector<LBBatchEntry> lbt(n);
  std::vector<char> pargs(n * pas);
  for (size_t i = 0; i < n; ++i) {
    ek_ctx* c = b->sys[i];
    const int cur0 = c->cur;
    pre[i] = part_args(c);
    poisson_batch_args(&pargs[i * pas], c->plan, (const int*)c->rho[c->cur],
                       c->has_qwall ? (const float*)c->qwall : nullptr, (const float*)c->qpart, c->ph,
                       (float*)c->phi, (float2*)c->spectrum);
    lbt[i].a = lb_args(c);
    lbt[i].a.advseg = adv32_segments(c->g, true);  // one launch for all systems: wide
    lbt[i].c = make_phys32(c->ph);
    c->cur = 1 - c->cur;
    post[i] = part_args(c);
    c->cur = cur0;
  }
  const auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t off = 0;
  F.o_pre = off;
  off = up(off + n * sizeof(PartArgs));
  F.o_post = off;
  off = up(off + n * sizeof(PartArgs));
  F.o_lb = off;
  off = up(off + n * sizeof(LBBatchEntry));
  F.o_pa = off;
  off = up(off + n * pas);
  std::vector<BatchSlot> slots;  // all launches' ranges, after the tables
  const size_t o_slots = off;
  // one launch over the systems' (gx, gy) grids, in system order
  const auto make = [&](const std::vector<std::tuple<int, int, int>>& items, int variant) {
    ek_batch::Launch L;
    L.variant = variant;
    L.slot = o_slots + slots.size() * sizeof(BatchSlot);
    for (const auto& it : items) {
      const int gx = std::get<1>(it), gy = std::get<2>(it);
      if (gx <= 0 || gy <= 0) continue;
      slots.push_back(BatchSlot{L.ctas, gx, gy, std::get<0>(it)});
      L.ctas += gx * gy;
      ++L.nslot;
    }
    return L;
  };
  for (int k = 0; k < PK_COUNT; ++k) {
    std::vector<std::tuple<int, int, int>> items;
    for (size_t i = 0; i < n; ++i) {
      int gx, gy;
      particle_batch_grid(k, k <= PK_TIE ? pre[i] : post[i], gx, gy);
      items.emplace_back((int)i, gx, gy);
    }
    F.part[k] = make(items, 0);
  }
  F.s1_alone.clear();
  for (size_t i = 0; i < n; ++i)
    if (!poisson_batch_ok(b->sys[i]->plan)) F.s1_alone.push_back((int)i);
  for (int pass = 0; pass < 3; ++pass) {
    std::map<int, std::vector<std::tuple<int, int, int>>> groups;  // by kernel variant
    for (size_t i = 0; i < n; ++i) {
      if (!poisson_batch_ok(b->sys[i]->plan)) continue;
      int variant, ctas;
      poisson_batch_pass(b->sys[i]->plan, pass, &pargs[i * pas], variant, ctas);
      groups[variant].emplace_back((int)i, ctas, 1);
    }
    F.fft[pass].clear();
    for (const auto& gi : groups) F.fft[pass].push_back(make(gi.second, gi.first));
  }
  {
    std::vector<std::tuple<int, int, int>> il, ia;
    for (size_t i = 0; i < n; ++i) {
      int gx, gy;
      lb32_batch_grid(lbt[i].a, gx, gy);
      il.emplace_back((int)i, gx, gy);
      advect32_batch_grid(lbt[i].a, gx, gy);
      ia.emplace_back((int)i, gx, gy);
    }
    F.lb = make(il, 0);
    F.adv = make(ia, 0);
  }
  const size_t total = o_slots + slots.size() * sizeof(BatchSlot);
  std::vector<char> host(total, 0);
  memcpy(host.data() + F.o_pre, pre.data(), n * sizeof(PartArgs));
  memcpy(host.data() + F.o_post, post.data(), n * sizeof(PartArgs));
  memcpy(host.data() + F.o_lb, lbt.data(), n * sizeof(LBBatchEntry));
  memcpy(host.data() + F.o_pa, pargs.data(), n * pas);
  if (!slots.empty()) memcpy(host.data() + o_slots, slots.data(), slots.size() * sizeof(BatchSlot));
  if (cudaMalloc((void**)&F.dev, total) != cudaSuccess) {
    F.dev = nullptr;
    return bfail(b, EK_ERR_NOMEM, "batch tables could not be allocated");
  }
  if (cudaMemcpy(F.dev, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess)
    return bfail(b, EK_ERR_CUDA, "batch tables could not be copied");
  return EK_OK;
}

// The fused step as a graph: every kernel once for all systems, in the order
// of a single system's step (the assignment beside S1 and S2, the forces and
// the re-flag beside S3 when overlap is chosen, the transitions after both).
ek_status batch_capture_fused(ek_batch* b, int key) {
  ek_batch::Fused& F = b->fused[key];
  if (F.dev) {
    cudaStreamSynchronize(b->stream);
    cudaFree(F.dev);
    F = ek_batch::Fused();
  }
  ek_status st = fused_build(b, key);
  if (st != EK_OK) return st;
  const size_t n = b->sys.size();
  const ek_ctx* c0 = b->sys[0];
  const int K = c0->ph.K;
  const bool pv = c0->ph.pv != 0;
  char* base = F.dev;
  long long count = 0;
  std::vector<long long> alone(n, 0);
  cudaStream_t s = b->stream;
  cudaStream_t ps = b->overlap ? b->aux : s;  // where the particle chain runs
  const auto part = [&](int k, cudaStream_t on) {
    const ek_batch::Launch& L = F.part[k];
    if (L.ctas == 0) return cudaSuccess;
    ++count;
    const PartArgs* tab = (const PartArgs*)(base + (k <= PK_TIE ? F.o_pre : F.o_post));
    return launch_particle_batch(k, BatchLaunch<PartArgs>{tab, (const BatchSlot*)(base + L.slot), L.nslot, L.ctas}, on);
  };
  const auto lbl = [&](const ek_batch::Launch& L) {
    return BatchLaunch<LBBatchEntry>{(const LBBatchEntry*)(base + F.o_lb), (const BatchSlot*)(base + L.slot),
                                     L.nslot, L.ctas};
  };
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return bfail(b, EK_ERR_CUDA, "batch capture could not start");
  cudaError_t e = cudaSuccess;
  const auto ok = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  if (b->overlap) {
    ok(cudaEventRecord(b->ev_fork, s));
    ok(cudaStreamWaitEvent(b->aux, b->ev_fork, 0));
  }
  // fuse == 2: the phases between two stream-ordered points as one persistent
  // launch (its barrier block zeroed in the graph first)
  const bool chain = b->fuse == 2;
  const auto chain_launch = [&](int blk, std::initializer_list<int> kinds, cudaStream_t on) {
    ChainArgs A;
    A.tab = (const PartArgs*)(base + (*kinds.begin() <= PK_TIE ? F.o_pre : F.o_post));
    A.nph = 0;
    int most = 0;
    for (int k : kinds) {
      const ek_batch::Launch& L = F.part[k];
      if (L.ctas == 0) continue;
      A.ph[A.nph++] = ChainPhase{k, L.ctas, L.nslot, (const BatchSlot*)(base + L.slot)};
      most = std::max(most, L.ctas);
    }
    if (A.nph == 0) return cudaSuccess;
    A.bar = (unsigned*)(b->dstatus + 4 * blk);
    A.status = b->dstatus;
    A.limit_ns = b->limit_ns;
    A.leave_cta = b->leave_cta;
    cudaError_t r = cudaMemsetAsync(A.bar, 0, 4 * sizeof(unsigned), on);
    if (r != cudaSuccess) return r;
    ++count;
    return launch_particle_chain(A, std::min(most, b->chain_ctas), on);
  };
  if (chain) {
    ok(chain_launch(1, {PK_ASSIGN, PK_TIE}, ps));
  } else {
    ok(part(PK_ASSIGN, ps));
    ok(part(PK_TIE, ps));
  }
  for (int pass = 0; pass < 3; ++pass) {
    for (const ek_batch::Launch& L : F.fft[pass]) {
      ok(launch_poisson_batch(pass, L.variant, base + F.o_pa, (const BatchSlot*)(base + L.slot), L.nslot,
                              L.ctas, s));
      ++count;
    }
  }
  for (int i : F.s1_alone) {
    ek_ctx* c = b->sys[i];
    ok(poisson_solve_f32(c->plan, (const int*)c->rho[c->cur], c->has_qwall ? (const float*)c->qwall : nullptr,
                         (const float*)c->qpart, c->ph, (float*)c->phi, (float2*)c->spectrum, s));
    alone[i] += poisson_kernel_count(c->plan, true);
  }
  ok(launch_lb32_batch(lbl(F.lb), K, pv, s));
  ++count;
  if (b->overlap) {
    ok(cudaEventRecord(b->ev_lb, s));
    ok(cudaStreamWaitEvent(b->aux, b->ev_lb, 0));
  }
  if (chain) {
    ok(part(PK_FORCES, ps));
    ok(chain_launch(2, {PK_SAVE_PREV, PK_CLEAR, PK_CLAIM, PK_PSI, PK_CHARGE}, ps));
  } else {
    for (int k = PK_FORCES; k <= PK_CHARGE; ++k) ok(part(k, ps));
  }
  if (b->overlap) ok(cudaEventRecord(b->ev_part, b->aux));
  if (K > 0) {
    ok(launch_advection32_batch(lbl(F.adv), K, s));
    ++count;
  }
  if (b->overlap) ok(cudaStreamWaitEvent(s, b->ev_part, 0));
  if (chain) {
    ok(chain_launch(3, {PK_TRANS, PK_APPLY}, s));
  } else {
    ok(part(PK_TRANS, s));
    ok(part(PK_APPLY, s));
  }
  const cudaError_t ec = cudaStreamEndCapture(s, &graph);
  if (e != cudaSuccess || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return bfail(b, EK_ERR_CUDA, std::string("fused batch capture failed: ") +
                                     cudaGetErrorString(e != cudaSuccess ? e : ec));
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->graph[key], graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return bfail(b, EK_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(ei));
  // the batch's launches are counted on the first system, S1 run alone on
  // its own system
  b->dlaunch[key].assign(n, 0);
  for (size_t i = 0; i < n; ++i) b->dlaunch[key][i] = alone[i];
  b->dlaunch[key][0] += count;
  b->cur_at[key].resize(n);
  b->version_at[key].resize(n);
  for (size_t i = 0; i < n; ++i) {
    b->cur_at[key][i] = b->sys[i]->cur;
    b->version_at[key][i] = b->sys[i]->version;
  }
  return EK_OK;
}

bool batch_graph_valid(const ek_batch* b, int key) {
  if (!b->graph[key] || b->cur_at[key].size() != b->sys.size()) return false;
  for (size_t i = 0; i < b->sys.size(); ++i)
    if (b->sys[i]->cur != b->cur_at[key][i] || b->sys[i]->version != b->version_at[key][i]) return false;
  return true;
}

ek_status batch_step_once(ek_batch* b) {
  const int key = b->sys[0]->cur;
  if (!batch_graph_valid(b, key)) {
    if (b->graph[key]) {
      cudaGraphExecDestroy(b->graph[key]);
      b->graph[key] = nullptr;
    }
    ek_status st = b->fuse && b->fusable ? batch_capture_fused(b, key) : batch_capture(b, key);
    if (st != EK_OK) return st;
  }
  if (cudaGraphLaunch(b->graph[key], b->stream) != cudaSuccess)
    return bfail(b, EK_ERR_CUDA, "batch graph launch failed");
  for (size_t i = 0; i < b->sys.size(); ++i) {
    b->sys[i]->cur = 1 - b->sys[i]->cur;
    b->sys[i]->launches += b->dlaunch[key][i];
  }
  return EK_OK;
}

}  // namespace

extern "C" {

ek_status ek_batch_create(ek_ctx* const* systems, int nsys, ek_batch** out) {
  if (!systems || nsys <= 0 || !out) return EK_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < nsys; ++i) {
    if (!systems[i]) return EK_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (systems[j] == systems[i]) return EK_ERR_ARG;
  }
  ek_batch* b = new (std::nothrow) ek_batch();
  if (!b) return EK_ERR_NOMEM;
  b->sys.assign(systems, systems + nsys);
  b->device = systems[0]->device;
  for (ek_ctx* c : b->sys) {
    if (c->device != b->device) {
      delete b;
      return EK_ERR_ARG;
    }
    if (ready(c) != EK_OK || c->broken) {
      delete b;
      return EK_ERR_STATE;
    }
  }
  cudaSetDevice(b->device);
  const int nbranch = std::min(nsys, 64);
  bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  b->own_stream = true;
  b->branch.assign(nbranch, nullptr);
  b->ev_join.assign(nbranch, nullptr);
  for (int w = 0; w < nbranch && ok; ++w) {
    ok = cudaStreamCreateWithFlags(&b->branch[w], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_join[w], cudaEventDisableTiming) == cudaSuccess;
  }
  // the fused step's particle chain runs on a stream of the greatest
  // priority, as a single system's does
  int lo_pri = 0, hi_pri = 0;
  ok = ok && cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri) == cudaSuccess &&
       cudaStreamCreateWithPriority(&b->aux, cudaStreamNonBlocking, hi_pri) == cudaSuccess &&
       cudaEventCreateWithFlags(&b->ev_lb, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&b->ev_part, cudaEventDisableTiming) == cudaSuccess;
  // the systems' earlier work (set-up, fields) is on their own streams
  for (ek_ctx* c : b->sys) ok = ok && cudaStreamSynchronize(c->stream) == cudaSuccess;
  b->width = std::min(nbranch, 16);
  ok = ok && cudaMalloc((void**)&b->dstatus, 16 * sizeof(int)) == cudaSuccess &&
       cudaMemset(b->dstatus, 0, 16 * sizeof(int)) == cudaSuccess;
  b->chain_ctas = ok ? particle_chain_ctas() : 0;
  b->fusable = true;
  for (ek_ctx* c : b->sys)
    b->fusable = b->fusable && c->fp32 && c->ph.K == b->sys[0]->ph.K && c->ph.pv == b->sys[0]->ph.pv;
  b->fuse = b->fusable ? 1 : 0;
  if (!ok) {
    ek_batch_destroy(b);
    return EK_ERR_CUDA;
  }
  batch_apply(b);
  *out = b;
  return EK_OK;
}

ek_status ek_batch_destroy(ek_batch* b) {
  if (!b) return EK_ERR_ARG;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop(b);
  for (size_t w = 0; w < b->branch.size(); ++w) {
    if (b->branch[w]) cudaStreamDestroy(b->branch[w]);
    if (b->ev_join[w]) cudaEventDestroy(b->ev_join[w]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_lb) cudaEventDestroy(b->ev_lb);
  if (b->ev_part) cudaEventDestroy(b->ev_part);
  if (b->aux) cudaStreamDestroy(b->aux);
  if (b->dstatus) cudaFree(b->dstatus);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return EK_OK;
}

ek_status ek_batch_set_stream(ek_batch* b, void* stream) {
  if (!b || !stream) return EK_ERR_ARG;
  cudaSetDevice(b->device);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, EK_ERR_CUDA, "sync failed");
  if (b->own_stream) cudaStreamDestroy(b->stream);
  b->own_stream = false;
  b->stream = (cudaStream_t)stream;
  batch_drop(b);
  return EK_OK;
}

ek_status ek_batch_step_async(ek_batch* b, int nsteps) {
  if (!b || nsteps < 0) return EK_ERR_ARG;
  cudaSetDevice(b->device);
  for (ek_ctx* c : b->sys) {
    if (c->broken) return bfail(b, EK_ERR_STATE, "a system is in an error state: " + c->err);
    if (c->setup_pending) {
      // set-up runs on the system's own stream; order it before the batch
      if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, EK_ERR_CUDA, "sync failed");
      const ek_status st = ready(c);
      if (st != EK_OK) return bfail(b, st, "set-up of a system failed: " + c->err);
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bfail(b, EK_ERR_CUDA, "sync failed");
    }
  }
  for (int t = 0; t < nsteps; ++t) {
    const ek_status st = batch_step_once(b);
    if (st != EK_OK) return st;
  }
  return EK_OK;
}

ek_status ek_batch_sync(ek_batch* b) {
  if (!b) return EK_ERR_ARG;
  cudaSetDevice(b->device);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, EK_ERR_CUDA, "batch stream failed");
  int bst = 0;
  if (b->dstatus && cudaMemcpy(&bst, b->dstatus, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return bfail(b, EK_ERR_CUDA, "batch status could not be read");
  if (bst & ST_TIMEOUT) {
    // a step stopped part way: no system's state is a state of the method
    for (ek_ctx* c : b->sys) {
      c->broken = true;
      c->err = "a batch step was cut short by a grid-barrier timeout";
    }
    return bfail(b, EK_ERR_TIMEOUT, "a grid barrier of the persistent particle chain timed out");
  }
  ek_status worst = EK_OK;
  for (size_t i = 0; i < b->sys.size(); ++i) {
    const ek_status st = check_status(b->sys[i]);
    if (st != EK_OK && worst == EK_OK) {
      worst = st;
      b->err = "system " + std::to_string(i) + ": " + b->sys[i]->err;
    }
  }
  return worst;
}

ek_status ek_batch_step(ek_batch* b, int nsteps) {
  const ek_status st = ek_batch_step_async(b, nsteps);
  if (st != EK_OK) return st;
  return ek_batch_sync(b);
}

ek_status ek_batch_config(const ek_batch* b, int cfg[4]) {
  if (!b || !cfg) return EK_ERR_ARG;
  cfg[0] = b->width;
  cfg[1] = b->planes;
  cfg[2] = b->overlap;
  cfg[3] = b->fusable ? b->fuse : 0;
  return EK_OK;
}

ek_status ek_batch_wait_test(ek_batch* b, int leave_cta, double limit_ms) {
  if (!b || leave_cta < -1 || !(limit_ms > 0.0) || limit_ms > 60000.0) return EK_ERR_ARG;
  cudaSetDevice(b->device);
  b->leave_cta = leave_cta;
  b->limit_ns = (long long)(limit_ms * 1e6);
  batch_drop(b);
  return EK_OK;
}

// Autotuner: every candidate (branch width x S2 segment length x overlap of
// the particle chain) is captured and timed over `trial_steps` real steps of
// the whole batch (CUDA events on the batch stream, after one untimed step
// that uploads the graph); the fastest is kept.
ek_status ek_batch_tune(ek_batch* b, int trial_steps, double* best_ms) {
  if (!b || trial_steps <= 0) return EK_ERR_ARG;
  cudaSetDevice(b->device);
  const int nbranch = (int)b->branch.size();
  std::vector<int> widths;
  for (int w : {8, 16, 32, 64})
    if (w < nbranch) widths.push_back(w);
  widths.push_back(nbranch);
  // candidates (fuse, branch width, planes per S2 block, overlap); the fused
  // step has no branches
  std::vector<std::tuple<int, int, int, int>> cands;
  for (int pl : {2, 4, 8})
    for (int ov = 0; ov <= 1; ++ov) {
      if (b->fusable) {
        cands.emplace_back(1, b->width, pl, ov);
        if (b->chain_ctas > 0) cands.emplace_back(2, b->width, pl, ov);
      }
      for (int w : widths) cands.emplace_back(0, w, pl, ov);
    }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return bfail(b, EK_ERR_CUDA, "event creation failed");
  double best = 1e300;
  int bf = b->fuse, bw = b->width, bp = b->planes, bo = b->overlap;
  ek_status st = EK_OK;
  for (const auto& cand : cands) {
    std::tie(b->fuse, b->width, b->planes, b->overlap) = cand;
    batch_apply(b);
    batch_drop(b);
    st = ek_batch_step_async(b, 2);  // captures both parities and uploads them
    if (st != EK_OK) break;
    if (cudaEventRecord(e0, b->stream) != cudaSuccess) st = EK_ERR_CUDA;
    if (st == EK_OK) st = ek_batch_step_async(b, trial_steps);
    if (st == EK_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess ||
                        cudaEventSynchronize(e1) != cudaSuccess))
      st = EK_ERR_CUDA;
    if (st != EK_OK) break;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = (double)ms / trial_steps;
    if (per < best) {
      best = per;
      std::tie(bf, bw, bp, bo) = cand;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != EK_OK) return st;
  b->fuse = bf;
  b->width = bw;
  b->planes = bp;
  b->overlap = bo;
  batch_apply(b);
  batch_drop(b);
  if (best_ms) *best_ms = best;
  return ek_batch_sync(b);
}

ek_status ek_batch_set_config(ek_batch* b, const int cfg[4]) {
  if (!b || !cfg) return EK_ERR_ARG;
  if (cfg[0] < 1 || cfg[0] > (int)b->branch.size() || cfg[1] < 1 || cfg[1] > 64 || cfg[2] < 0 ||
      cfg[2] > 1 || cfg[3] < 0 || cfg[3] > 2)
    return bfail(b, EK_ERR_ARG, "configuration out of range");
  if (cfg[3] && !b->fusable)
    return bfail(b, EK_ERR_ARG, "the fused form needs FP32 systems with one species count and partial-volume choice");
  cudaSetDevice(b->device);
  b->width = cfg[0];
  b->planes = cfg[1];
  b->overlap = cfg[2];
  b->fuse = cfg[3];
  batch_apply(b);
  batch_drop(b);
  return EK_OK;
}

int ek_batch_size(const ek_batch* b) { return b ? (int)b->sys.size() : 0; }

const char* ek_batch_last_error(const ek_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
