// Internal declarations of the GB300 electrokinetics library: device data
// layout, the D3Q19 velocity set and the kernel launchers of each stage.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ek.h"

namespace ek {

// ---------------------------------------------------------------------------
// D3Q19 (Sec. III.A): rest, 6 faces, 12 edges; opposite pairs (i, i+1) for odd i.
// ---------------------------------------------------------------------------
constexpr int Q = 19;
// Components as compile-time functions: in unrolled loops every c_i folds
// into an add, a subtract or nothing (no table load, no multiply by +-1).
__host__ __device__ constexpr int dcx(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int dcy(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int dcz(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
// +v or -v by the sign of a (nonzero) component
__host__ __device__ __forceinline__ double csgn(int c, double v) { return c > 0 ? v : -v; }
// c_i . v with neither multiplications nor additions of zero: an edge is one
// add, a face a signed copy (after unrolling i is a constant)
__host__ __device__ __forceinline__ double cdot(int i, double x, double y, double z) {
  const int a = dcx(i), b = dcy(i), c = dcz(i);
  if (a && b) return csgn(a, x) + csgn(b, y);
  if (a && c) return csgn(a, x) + csgn(c, z);
  if (b && c) return csgn(b, y) + csgn(c, z);
  if (a) return csgn(a, x);
  if (b) return csgn(b, y);
  if (c) return csgn(c, z);
  return 0.0;
}
constexpr int HCX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
constexpr int HCY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
constexpr int HCZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
// opposite of i: i+1 for odd i, i-1 for even i > 0
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr double wgt(int i) {
  return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
}

constexpr int FLUID = -1;
constexpr int WALL = -2;

// device status word bits
enum : int {
  ST_NONFINITE = 1,
  ST_OVERLAP = 2,
  ST_EXPEL = 4,
  ST_CAPACITY = 8,
  ST_TIMEOUT = 16,  // a bounded device wait gave up (the batch's grid barrier)
};

// Particle record on the device (all FP64).
struct DevParticle {
  double pos[3], vel[3], omega[3];
  double force[3], torque[3];
  double ftrans[3];  // create/destroy momentum of the last S5, applied at the next S4
  double radius, charge, mass, inertia;
  // sum of Psi_p over the particle's box in units of 2^-13 (exact), in eight
  // partial sums (one per octant of the surface cells) that take the atomics
  unsigned long long psiunits[8];
  int nb;            // number of boundary nodes
  int fixed;
  int lo[3], hi[3];  // box [lo, hi) in unwrapped coordinates, current position
  int ulo[3], uhi[3];  // union of the previous and current boxes (transitions)
  int elo[3], ehi[3];  // box widened by ceil(R) + FORCE_MARGIN (solute force region)
  // float forms for the octree pre-test, set with the box: integer part and
  // fraction of the centre, R^2 and the pre-test margin
  int ipos[3];
  float fpos[3], fposlo[3];  // fraction of the centre as a float pair (hi + lo)
  float r2f, r2lo, psimargin;  // R^2 (the FP64 product) as a float pair
  float velf[3], omegaf[3];    // vel and omega rounded to float (FP32-form wall velocity)
};

// cells added to ceil(R) around a particle's box for the region whose solute
// force it receives
constexpr int FORCE_MARGIN = 4;

// Box geometry common to the kernels.
struct Grid {
  int nx, ny, nz;
  long long N;
};

// Physics constants passed by value to the kernels.
struct Phys {
  double rho0, lam_e, lam_o, bjerrum;
  int K;
  int pv;
  unsigned flags;
  double z[EK_MAX_SPECIES], D[EK_MAX_SPECIES];
  double dcoef[EK_MAX_SPECIES];  // D_k / A_0 (face links; edge links get 1/sqrt 2 more)
  double hinvD[EK_MAX_SPECIES];  // 1 / (2 D_k), coupling-force weight of a link flux
  double hz[EK_MAX_SPECIES];     // z_k / 2
  double E[3], g[3];
  double ec[19];                 // E . c_i per direction
  int fp32;                      // storage form: 0 FP64, 1 FP32 populations / int32 species
  double qscale[EK_MAX_SPECIES]; // FP32 form: density of one species unit (a power of 2)
};

// sign code of a velocity component for the volume-of-fluid shares
__host__ __device__ __forceinline__ unsigned sign_code(double v) { return v > 0.0 ? 1u : (v < 0.0 ? 2u : 0u); }
__host__ __device__ __forceinline__ unsigned sign_code(float v) { return v > 0.0f ? 1u : (v < 0.0f ? 2u : 0u); }

// Storage forms.  FP64: every field double.  FP32: populations stored as the
// deviation f_i - w_i rho0 in float, species as int32 multiples of qscale_k
// (exact conservation: every transfer is an integer moved from one node to
// another), Phi, Psi, u and the charge fields in float.
struct FormF64 {
  using pop_t = double;
  using spc_t = double;
  using real_t = double;
  static constexpr bool fp32 = false;
};
struct FormF32 {
  using pop_t = float;
  using spc_t = int;
  using real_t = float;
  static constexpr bool fp32 = true;
};

// Transition record: one solute transfer of S5 (target node, amount per species).
struct Transfer {
  long long node;
  double amount[EK_MAX_SPECIES];
};

// FFT plan of one axis.
struct AxisPlan {
  int n = 0;
  int nrad = 0;
  int radix[16] = {};
  double2* tw = nullptr;   // exp(-2 pi i k / n), k = 0..n-1 (device)
  double* lam = nullptr;   // 2 - 2 cos(2 pi k / n), k = 0..n-1 (device)
  float2* tw32 = nullptr;  // the same tables rounded to float (FP32 form)
  float* lam32 = nullptr;
};

struct PoissonPlan {
  int nx, ny, nz;
  AxisPlan ax, ay, az;
  bool ok = false;
};

__host__ __device__ inline int wrapi(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

// Lattice kernels run on a 3D grid of 32 x 8 thread tiles (x, y) per z plane:
// no integer division to find a node's coordinates, and a warp covers 32
// consecutive x (coalesced).
constexpr int TILE_X = 32, TILE_Y = 8;
inline dim3 lattice_grid(const Grid& g) {
  return dim3((unsigned)((g.nx + TILE_X - 1) / TILE_X), (unsigned)((g.ny + TILE_Y - 1) / TILE_Y),
              (unsigned)g.nz);
}
inline dim3 lattice_block() { return dim3(TILE_X, TILE_Y, 1); }
// the FP32 form's S2 kernel marches each (x, y) tile column through nzb
// segments of consecutive planes
inline dim3 lattice_grid32(const Grid& g, int nzb) {
  return dim3((unsigned)((g.nx + TILE_X - 1) / TILE_X), (unsigned)((g.ny + TILE_Y - 1) / TILE_Y),
              (unsigned)nzb);
}

// ---------------------------------------------------------------------------
// Launches over the systems of a batch.  One 1-D launch runs a stage for many
// systems: system s owns the CTAs [cta0, cta0 + gx * gy) and runs them as its
// own gx x gy grid (x fastest) with its own arguments, read from a device
// table.  A kernel body takes its block as a Blk, so that one body serves the
// launch for one system (the Blk from blockIdx and gridDim) and the batched
// launch (the Blk of the system's range).
// ---------------------------------------------------------------------------
struct Blk {
  int x, y;  // block coordinates in the system's grid
  int nx;    // the grid's x extent (the stride of grid-stride loops)
};
struct BatchSlot {
  int cta0, gx, gy;
  int entry;  // the system's row of the argument table
};
__device__ __forceinline__ Blk grid_blk() { return Blk{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x}; }
// the system whose range holds CTA (or work item) b (binary search over the
// ascending cta0), and the block it is in that system's grid
__device__ __forceinline__ Blk batch_blk_at(const BatchSlot* __restrict__ sl, int nsys, int b, int& sys) {
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sl[mid].cta0 <= b) lo = mid;
    else hi = mid - 1;
  }
  const BatchSlot s = sl[lo];
  sys = s.entry;
  const int l = b - s.cta0;
  return Blk{l % s.gx, l / s.gx, s.gx};
}
__device__ __forceinline__ Blk batch_blk(const BatchSlot* __restrict__ sl, int nsys, int& sys) {
  return batch_blk_at(sl, nsys, (int)blockIdx.x, sys);
}
// a batched launch: per-system argument table and ranges (device memory), the
// number of systems and the CTA total
template <class A>
struct BatchLaunch {
  const A* tab;
  const BatchSlot* slot;
  int nsys;
  int ctas;
};

// wrapped neighbour coordinates of (x, y, z)
struct Nbr {
  int xm, xp, ym, yp, zm, zp;
};
__device__ __forceinline__ Nbr make_nbr(int x, int y, int z, const Grid& g) {
  Nbr b;
  b.xm = x == 0 ? g.nx - 1 : x - 1;
  b.xp = x == g.nx - 1 ? 0 : x + 1;
  b.ym = y == 0 ? g.ny - 1 : y - 1;
  b.yp = y == g.ny - 1 ? 0 : y + 1;
  b.zm = z == 0 ? g.nz - 1 : z - 1;
  b.zp = z == g.nz - 1 ? 0 : z + 1;
  return b;
}
// coordinate + offset in {-1, 0, 1}, wrapped
__device__ __forceinline__ int nb_x(const Nbr& b, int x, int o) { return o > 0 ? b.xp : (o < 0 ? b.xm : x); }
__device__ __forceinline__ int nb_y(const Nbr& b, int y, int o) { return o > 0 ? b.yp : (o < 0 ? b.ym : y); }
__device__ __forceinline__ int nb_z(const Nbr& b, int z, int o) { return o > 0 ? b.zp : (o < 0 ? b.zm : z); }
__device__ __forceinline__ long long node_index(const Grid& g, int x, int y, int z) {
  return (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
}

// ---------------------------------------------------------------------------
// launchers (each file implements its stage)
// ---------------------------------------------------------------------------
// S1
cudaError_t poisson_plan_create(PoissonPlan& p, int nx, int ny, int nz, std::string& err);
void poisson_plan_destroy(PoissonPlan& p);
size_t poisson_spectrum_bytes(int nx, int ny, int nz);
// kernels one solve of this plan launches (the FP32 or the FP64 passes)
int poisson_kernel_count(const PoissonPlan& p, bool fp32);
// radix plan of one axis (n = 2^a 3^b); false if n has another factor
bool poisson_factor(int n, AxisPlan& P);
// charge assembly fused into the first FFT pass when rho != nullptr; else q is read.
// FP64 form: double fields, double2 spectrum.
// Multigrid solve of the same periodic problem (ek_multigrid.cu): levels down
// to a coarse grid (dims in coarse[]) that coarse_plan, an FFT plan of those
// dims, solves exactly; V-cycles until max|r| <= tol max|b|
size_t poisson_mg_scratch_bytes(int nx, int ny, int nz);
int poisson_mg_levels(int nx, int ny, int nz, int coarse[3]);
cudaError_t poisson_solve_mg(const PoissonPlan& coarse_plan, const double* q, double* phi, int nx,
                             int ny, int nz, double bjerrum, double tol, int max_cycles,
                             void* scratch, cudaStream_t s, int* cycles, double* residual);
cudaError_t poisson_solve(const PoissonPlan& p, const double* q, const double* rho,
                          const double* qwall, const double* qpart, const Phys& ph,
                          double* phi, double2* spectrum, cudaStream_t s);
// FP32 form: int32 species, float charge fields, float2 spectrum, float phi
cudaError_t poisson_solve_f32(const PoissonPlan& p, const int* rho, const float* qwall,
                              const float* qpart, const Phys& ph, float* phi, float2* spectrum,
                              cudaStream_t s);
cudaError_t charge_density(const Grid& g, const Phys& ph, const void* rho, const void* qwall,
                           const void* qpart, double* q, cudaStream_t s);
// Poisson solve with an inhomogeneous permittivity and fixed-potential nodes
// by Jacobi-preconditioned conjugate gradients (ek_krylov.cu); *bad_eps is set
// (and nothing solved) when a permittivity is not positive and finite
size_t poisson_cg_scratch_bytes(int nx, int ny, int nz);
cudaError_t poisson_solve_cg(const double* q, const double* eps, const unsigned char* fixed,
                             const double* phi_fixed, double* phi, int nx, int ny, int nz, double bjerrum,
                             double tol, int max_iter, void* scratch, cudaStream_t s, int* iters,
                             double* residual, bool* bad_eps);
// S1 of the FP32 systems of a batch whose edges are all 32, 48 or 64
// (poisson_batch_ok): pass 0 the x transform, 1 the y-z planes with the Green
// multiply, 2 the inverse x transform.  A system's entry of the argument
// table is poisson_batch_args_size() bytes written by poisson_batch_args;
// poisson_batch_pass gives the kernel variant of a pass (systems of one
// variant share a launch) and the system's CTAs in it.
bool poisson_batch_ok(const PoissonPlan& p);
size_t poisson_batch_args_size();
void poisson_batch_args(void* out, const PoissonPlan& p, const int* rho, const float* qwall,
                        const float* qpart, const Phys& ph, float* phi, float2* spectrum);
void poisson_batch_pass(const PoissonPlan& p, int pass, const void* args, int& variant, int& ctas);
cudaError_t launch_poisson_batch(int pass, int variant, const void* tab, const BatchSlot* slot, int nsys,
                                 int ctas, cudaStream_t s);

// S2 + S3
struct LBArgs {
  Grid g;
  Phys ph;
  const void* f_in;
  void* f_out;
  const void* rho_in;
  void* rho_out;
  const void* phi;
  const void* psi;
  const int* owner;
  void* u;
  void* ifield;    // real_t, 3N: solute force on the fluid minus q_ions E (fluid nodes)
  unsigned char* vsig;  // N: bit 7 fluid node; bits 0-1, 2-3, 4-5: sign code of u_x, u_y, u_z
                        // (0 zero, 1 positive, 2 negative), written by S2 for S3
  double* ipart;   // per-block sums of ifield (3 per block of the lattice grid)
  const DevParticle* parts;
  int* status;
  int nzb;         // FP32 S2: z segments per (x, y) tile column (lb32_segments)
  int advseg;      // FP32 S3: z segments per tile column (adv32_segments)
};
// Constants of the FP32 kernels, rounded once on the host.
struct Phys32 {
  float rho0, lam_e, lam_o;
  float qs[EK_MAX_SPECIES];  // density of one species unit
  float cq[EK_MAX_SPECIES];  // D_k / (A_0 qs_k): flux in units per bracket value
  float hz[EK_MAX_SPECIES];  // z_k / 2
  float ec[19];              // E . c_i
  float g[3];
  float E[3];
  float zq[EK_MAX_SPECIES];  // z_k qs_k: charge of one unit of species k
};
Phys32 make_phys32(const Phys& ph);
// one system's entry of the batched FP32 S2 / S3 launches
struct LBBatchEntry {
  LBArgs a;
  Phys32 c;
};
cudaError_t launch_lb_fused(const LBArgs& a, cudaStream_t s);
cudaError_t launch_advection(const LBArgs& a, cudaStream_t s);
// FP32-storage form
cudaError_t lb32_prepare();  // once per process, before the first launch_lb32
// z segments per tile column of the FP32 S2 grid, chosen from the occupancy
int lb32_segments(const Grid& g, int K, bool pv);
cudaError_t launch_lb32(const LBArgs& a, cudaStream_t s);
cudaError_t launch_advection32(const LBArgs& a, cudaStream_t s);
// z segments per tile column of the FP32 S3 grid: 32-plane segments on
// large boxes, 16 where the grid still fills the SMs (`wide`: the launch is
// shared with other systems, so its size does not depend on this machine: 16),
// else 8, else 4
int adv32_segments(const Grid& g, bool wide);
// the same S2 and S3 for the systems of a batch (all FP32 with the same K and
// partial-volume choice), one launch each; the per-system grids (gx, gy) that
// the ranges of L.slot must give
void lb32_batch_grid(const LBArgs& a, int& gx, int& gy);
void advect32_batch_grid(const LBArgs& a, int& gx, int& gy);
cudaError_t launch_lb32_batch(const BatchLaunch<LBBatchEntry>& L, int K, bool pv, cudaStream_t s);
cudaError_t launch_advection32_batch(const BatchLaunch<LBBatchEntry>& L, int K, cudaStream_t s);
cudaError_t launch_fill32(const Grid& g, const Phys& ph, const int* owner, float* f, int* rho,
                          const int* units, cudaStream_t s);
enum {
  CONV_POP_TO_F64 = 0,    // direction `index` of the stored deviations -> f (double)
  CONV_POP_FROM_F64 = 1,  // f (double) -> direction `index` of the deviations
  CONV_SPC_TO_F64 = 2,    // int units -> density (scale = qscale)
  CONV_SPC_FROM_F64 = 3,  // density -> int units (scale = qscale)
  CONV_F32_TO_F64 = 4,
  CONV_F64_TO_F32 = 5,
};
// N-element conversion; `scale` is rho0 for populations, qscale for species
cudaError_t convert32(int op, const Grid& g, int index, double scale, const void* in, void* out,
                      int* status, cudaStream_t s);
cudaError_t set_velocity32(const Grid& g, const int* owner, float* f, const double* u3, double rho0,
                           cudaStream_t s);
cudaError_t density32(const Grid& g, const float* f, double rho0, double* out, cudaStream_t s);

// S4 / S5 / set-up
struct PartArgs {
  Grid g;
  Phys ph;
  DevParticle* parts;
  int P;
  int boxmax;      // capacity (cells) of one particle's psibox
  double* psibox;  // P * boxmax: Psi_p over the current box
  int* owner;
  int* owner_prev;
  void* psi;        // real_t
  void* qpart;      // real_t
  void* f;          // pop_t: populations after the stream (S4 reads, S5 writes)
  void* rho;        // spc_t: species after S3 (S5 transitions)
  const void* phi;  // real_t
  const unsigned char* wall;
  Transfer* xfer;
  int* xfer_count;
  int xfer_cap;
  double* fpart;   // per (particle, chunk) partial force/torque sums of S4
  int fchunks;     // chunks per particle in fpart
  int fcells;      // widened-box cells per chunk (a multiple of FORCE_CHUNK)
  int emax;        // capacity (cells) of one particle's widened box
  const void* ifield;        // real_t, 3N (written by S2)
  const double* ipart;       // 3 per lattice block
  int nipart;                // number of lattice blocks
  unsigned long long* fkey;  // N: (surface distance, particle) of the nearest particle
  // nodes whose nearest particle the float distances cannot decide: the FP64
  // decision is taken there by a second kernel (the count is cleared by the
  // integration at the end of S4)
  int* tie_list;
  int* tie_count;
  int tie_cap;
  float tie_thr;   // float distances closer than this are a possible tie
  double* psum;              // P * FPART: per-particle sums of S4
  int2* surf;      // (particle, box cell) of the cells cut by a sphere surface
  int* surf_count;
  int surf_cap;
  int* ticket;     // particles whose S4 sums are done (reset by the last)
  int* pticket;    // P: S4 force (or S5 transition) blocks of the particle done (reset by the last)
  int uchunks;     // CTAs per particle over its union box (S5 clear and transitions)
  double* tpart;   // P * uchunks * 3: per-CTA sums of the transitions' momentum
  int* status;
};
// cells per CTA of the S4 force kernel: FORCE_T threads, each over `fcells /
// FORCE_T` rows of FORCE_T cells, fcells a multiple of FORCE_CHUNK chosen at
// set-up (larger when many particles give enough CTAs anyway, so fewer block
// sums are made); fpart holds P * fchunks * FPART doubles
constexpr int FORCE_T = 128;
constexpr int FORCE_CHUNK = 512;
// per particle: [0..5] Fh Th (momentum exchange), [6..11] Fs Ts (reaction of
// the solute force), [12] sum q and [13..15] sum q (r - r_p) of the particle's
// own charge (the field's force and torque are E and M x E times these),
// [18..20] a slice of the lattice total of the internal force (first particle
// only), [16..17] and [21..23] unused
constexpr int FPART = 24;
// S4 in two parts: the nearest-surface assignment (needs only the particle
// positions, so it may run beside S1/S2), and the forces with the
// integration (after S2), which also clear the assignment keys
constexpr int S4_ASSIGN = 1, S4_FORCES = 2, S4_ALL = 3;
cudaError_t launch_particle_forces(const PartArgs& a, cudaStream_t s, int parts = S4_ALL);
// CTAs per particle that cover its union box (previous and current box)
int union_chunks(int boxmax);
// S5; parts: 1 = re-flag, Psi and charge (no species access), 2 = transitions
// (species after S3), 3 = both
cudaError_t launch_reflag(const PartArgs& a, bool transitions, cudaStream_t s, int parts = 3);
// The kernels of S4 and of S5's transitions step, each also as one launch
// over the systems of a batch (FP32 form), in the order a step runs them:
// assignment and its FP64 tie decision (beside S1/S2); after S2 the forces
// with the integration, then the re-flag part of S5; after S3 the
// transitions and the transfers they list.
enum PartKernel {
  PK_ASSIGN, PK_TIE, PK_FORCES, PK_SAVE_PREV, PK_CLEAR, PK_CLAIM, PK_PSI, PK_CHARGE, PK_TRANS,
  PK_APPLY, PK_COUNT
};
// the grid (gx, gy) kernel k runs for one system; gx = 0: no launch (P = 0)
void particle_batch_grid(int k, const PartArgs& a, int& gx, int& gy);
cudaError_t launch_particle_batch(int k, const BatchLaunch<PartArgs>& L, cudaStream_t s);
// Several of those kernels (all but PK_FORCES) as phases of one persistent
// launch: the resident CTAs take each phase's (system, block) items in turn
// and meet at a grid barrier before the next phase.  Each wait at the barrier
// ends after limit_ns of the global timer at most: the CTA then sets
// ST_TIMEOUT in *status and the abort word, and every CTA returns.
constexpr int CHAIN_MAX = 5;
struct ChainPhase {
  int kind;  // PartKernel
  int ctas;  // items: the CTAs the batched launch would have
  int nslot;
  const BatchSlot* slot;
};
struct ChainArgs {
  const PartArgs* tab;
  ChainPhase ph[CHAIN_MAX];
  int nph;
  unsigned* bar;      // [0] arrivals, [1] generation, [2] abort; zero before the launch
  int* status;        // ST_TIMEOUT on a wait that gave up
  long long limit_ns;
  int leave_cta;      // failure-detection test: this CTA returns before the first barrier (-1: none)
};
// CTAs of the persistent launch that are resident at once (it is a
// cooperative launch of that many at most)
int particle_chain_ctas();
cudaError_t launch_particle_chain(const ChainArgs& A, int ctas, cudaStream_t s);
cudaError_t launch_fill(const Grid& g, const Phys& ph, const int* owner, double* f, double* rho,
                        const double* bulk_k, cudaStream_t s);

}  // namespace ek
