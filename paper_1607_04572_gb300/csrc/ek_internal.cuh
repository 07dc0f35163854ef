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
};

// Particle record on the device (all FP64).
struct DevParticle {
  double pos[3], vel[3], omega[3];
  double force[3], torque[3];
  double ftrans[3];  // create/destroy momentum of the last S5, applied at the next S4
  double radius, charge, mass, inertia;
  double psisum;     // sum of Psi_p over the particle's box
  int nb;            // number of boundary nodes
  int fixed;
  int lo[3], hi[3];  // box [lo, hi) in unwrapped coordinates, current position
  int ulo[3], uhi[3];  // union of the previous and current boxes (transitions)
};

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
};

// Transition record: one solute transfer of S5 (target node, amount per species).
struct Transfer {
  long long node;
  double amount[EK_MAX_SPECIES];
};

// FFT plan of one axis.
struct AxisPlan {
  int n;
  int nrad;
  int radix[16];
  double2* tw;   // exp(-2 pi i k / n), k = 0..n-1 (device)
  double* lam;   // 2 - 2 cos(2 pi k / n), k = 0..n-1 (device)
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

// ---------------------------------------------------------------------------
// launchers (each file implements its stage)
// ---------------------------------------------------------------------------
// S1
cudaError_t poisson_plan_create(PoissonPlan& p, int nx, int ny, int nz, std::string& err);
void poisson_plan_destroy(PoissonPlan& p);
size_t poisson_spectrum_bytes(int nx, int ny, int nz);
// radix plan of one axis (n = 2^a 3^b); false if n has another factor
bool poisson_factor(int n, AxisPlan& P);
// charge assembly fused into the first FFT pass when rho != nullptr; else q is read
cudaError_t poisson_solve(const PoissonPlan& p, const double* q, const double* rho,
                          const double* qwall, const double* qpart, const Phys& ph,
                          double* phi, double2* spectrum, cudaStream_t s);
cudaError_t charge_density(const Grid& g, const Phys& ph, const double* rho, const double* qwall,
                           const double* qpart, double* q, cudaStream_t s);

// S2 + S3
struct LBArgs {
  Grid g;
  Phys ph;
  const double* f_in;
  double* f_out;
  const double* rho_in;
  double* rho_out;
  const double* phi;
  const double* psi;
  const int* owner;
  double* u;
  const DevParticle* parts;
  int* status;
};
cudaError_t launch_lb_fused(const LBArgs& a, cudaStream_t s);
cudaError_t launch_advection(const LBArgs& a, cudaStream_t s);

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
  double* psi;
  double* qpart;
  const double* f;  // populations after the stream (S4 reads, S5 writes uncovered)
  double* fw;
  double* rho;      // species after S3 (S5 transitions)
  const double* phi;
  const unsigned char* wall;
  Transfer* xfer;
  int* xfer_count;
  int xfer_cap;
  double* fpart;   // per (particle, chunk) partial force/torque sums of S4
  int fchunks;     // chunks per particle in fpart
  int2* surf;      // (particle, box cell) of the cells cut by a sphere surface
  int* surf_count;
  int surf_cap;
  int* status;
};
// cells per CTA of the S4 force kernel; fpart holds P * fchunks * 12 doubles
constexpr int FORCE_CHUNK = 128;
cudaError_t launch_particle_forces(const PartArgs& a, cudaStream_t s);  // S4
cudaError_t launch_reflag(const PartArgs& a, bool transitions, cudaStream_t s);  // S5
cudaError_t launch_fill(const Grid& g, const Phys& ph, const int* owner, double* f, double* rho,
                        const double* bulk_k, cudaStream_t s);

}  // namespace ek
