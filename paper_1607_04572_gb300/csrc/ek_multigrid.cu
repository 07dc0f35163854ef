// Periodic Poisson solve of Eq. 3 by geometric multigrid: the same discrete
// problem the FFT solver of S1 solves (7-point Laplacian, periodic box,
// (6 phi - sum of the 6 neighbours) = 4 pi l_B (q - mean q), mean phi = 0),
// reached by V-cycles instead of a transform.  Levels: the box and its full
// coarsenings by 2 while every coarse edge stays even and >= 8 (coarse n_x a
// multiple of 2 for the real-to-complex transform) and the grid holds more
// than 4096 nodes; on level l the operator is 4^-l (6 phi - sum nb) (the
// same stencil on spacing 2^l).  Per V-cycle: two red-black Gauss-Seidel
// sweeps, the residual, full-weighting restriction, the coarser cycle,
// trilinear prolongation of the correction, two sweeps; the coarsest level is
// solved exactly by the FFT solver.  Red-black sweeps need even edges, which
// every level above the coarsest has.  All sums run in a fixed order.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ek_internal.cuh"

namespace ek {
namespace {

constexpr int MG_T = 256;          // threads per CTA of the grid kernels
constexpr int MG_COARSE = 4096;    // a level this small (or not coarsenable) is solved by FFT
constexpr int MG_RED_BLOCKS = 512; // partial sums of a reduction

struct Level {
  int nx, ny, nz;
  long long n;
  double c;         // 4^-l
  double* phi;      // level 0: the caller's output
  double* b;        // right-hand side
  double* r;        // residual
};

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// b = s (q - qmean), qmean = sums[1] (written by k_sum_final)
__global__ void k_mg_rhs(const double* q, double* b, long long n, double s, const double* sums) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  b[i] = s * (q[i] - sums[1]);
}

// block partial sums of x (fixed order: a grid-stride sum per thread, then a
// tree over the block)
__global__ void k_sum_partial(const double* x, long long n, double* part) {
  __shared__ double sh[MG_T];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s += x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = MG_T / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// out[0] = sum of the nblk partial sums, in order (one thread); out[1] = the
// mean over n values (one division, not one per node)
__global__ void k_sum_final(const double* part, int nblk, long long n, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < nblk; ++i) s += part[i];
  out[0] = s;
  out[1] = s / (double)n;
}

// sum of the six neighbours of node i = (x, y, z) (32-bit indices: N < 2^31)
__device__ __forceinline__ double nb_sum(const double* phi, int i, int x, int y, int z, int nx,
                                         int ny, int nz) {
  const int sy = nx, sz = nx * ny;
  return phi[i - x + wrap(x - 1, nx)] + phi[i - x + wrap(x + 1, nx)] +
         phi[i + (wrap(y - 1, ny) - y) * sy] + phi[i + (wrap(y + 1, ny) - y) * sy] +
         phi[i + (wrap(z - 1, nz) - z) * sz] + phi[i + (wrap(z + 1, nz) - z) * sz];
}

// one colour of a red-black Gauss-Seidel sweep: the nodes with
// (x + y + z) % 2 == colour take phi = (sum nb + b / c) / 6, as products
// (inv_c = 1 / c = 4^l exactly; an FP64 division costs a long sequence on the
// FP64 pipe, and the fixed point is set by the residual, which divides
// nothing); thread j takes the j-th node of the colour (n_x even: half of
// every row)
__global__ void k_mg_rbgs(double* phi, const double* b, int nx, int ny, int nz, double inv_c,
                          int colour) {
  const unsigned j = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned hx = (unsigned)nx / 2u;
  if (j >= hx * (unsigned)ny * (unsigned)nz) return;
  const unsigned row = j / hx;
  const int y = (int)(row % (unsigned)ny), z = (int)(row / (unsigned)ny);
  const int x = 2 * (int)(j - row * hx) + ((y + z + colour) & 1);
  const int i = x + nx * (int)row;
  constexpr double SIXTH = 1.0 / 6.0;
  phi[i] = (nb_sum(phi, i, x, y, z, nx, ny, nz) + b[i] * inv_c) * SIXTH;
}

// r = b - c (6 phi - sum nb)
__global__ void k_mg_resid(const double* phi, const double* b, double* r, int nx, int ny, int nz,
                           double c) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)nx * (unsigned)ny * (unsigned)nz) return;
  const unsigned row = i / (unsigned)nx;
  const int x = (int)(i - row * (unsigned)nx), y = (int)(row % (unsigned)ny), z = (int)(row / (unsigned)ny);
  r[i] = b[i] - c * (6.0 * phi[i] - nb_sum(phi, (int)i, x, y, z, nx, ny, nz));
}

// full weighting: coarse node (X, Y, Z) sits on fine node (2X, 2Y, 2Z) and
// takes the weighted mean of the 27 fine residuals around it (weights
// 1, 1/2, 1/4, 1/8 by the number of offset axes; every fine node gives a
// total weight of 1, so the mean is kept); phi_c = 0 for the cycle below
__global__ void k_mg_restrict(const double* rf, int nx, int ny, int nz, double* bc, double* phic) {
  const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)cx * (unsigned)cy * (unsigned)cz) return;
  const unsigned row = i / (unsigned)cx;
  const int X = (int)(i - row * (unsigned)cx), Y = (int)(row % (unsigned)cy), Z = (int)(row / (unsigned)cy);
  double s = 0.0;
  for (int dz = -1; dz <= 1; ++dz) {
    const int oz = wrap(2 * Z + dz, nz) * ny;
    const double wz = dz ? 0.5 : 1.0;
    for (int dy = -1; dy <= 1; ++dy) {
      const int oy = (oz + wrap(2 * Y + dy, ny)) * nx;
      const double wy = wz * (dy ? 0.5 : 1.0);
      for (int dx = -1; dx <= 1; ++dx) s += wy * (dx ? 0.5 : 1.0) * rf[oy + wrap(2 * X + dx, nx)];
    }
  }
  bc[i] = s / 8.0;
  phic[i] = 0.0;
}

// trilinear prolongation of the coarse correction, added to the fine phi
__global__ void k_mg_prolong_add(const double* phic, int nx, int ny, int nz, double* phif) {
  const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)nx * (unsigned)ny * (unsigned)nz) return;
  const unsigned row = i / (unsigned)nx;
  const int x = (int)(i - row * (unsigned)nx), y = (int)(row % (unsigned)ny), z = (int)(row / (unsigned)ny);
  // per axis: an even fine index lies on coarse node x / 2, an odd one half
  // way between (x - 1) / 2 and (x + 1) / 2 (periodic); the weight of each
  // of the (1, 2, 4 or 8) coarse nodes is 1/2 per odd axis
  const int x0 = x >> 1, x1 = (x & 1) ? wrap(x0 + 1, cx) : x0;
  const int y0 = (y >> 1) * cx, y1 = (y & 1) ? wrap((y >> 1) + 1, cy) * cx : y0;
  const int z0 = (z >> 1) * cx * cy, z1 = (z & 1) ? wrap((z >> 1) + 1, cz) * cx * cy : z0;
  // an even axis counts its one node twice and halves the sum: the same
  // value as one node at weight 1
  const double s = ((phic[z0 + y0 + x0] + phic[z0 + y0 + x1]) + (phic[z0 + y1 + x0] + phic[z0 + y1 + x1])) +
                   ((phic[z1 + y0 + x0] + phic[z1 + y0 + x1]) + (phic[z1 + y1 + x0] + phic[z1 + y1 + x1]));
  phif[i] += 0.125 * s;
}

// block maxima of |x| (a maximum does not depend on the order)
__global__ void k_absmax_partial(const double* x, long long n, double* part) {
  __shared__ double sh[MG_T];
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int w = MG_T / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_max_final(const double* part, int nblk, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double m = 0.0;
  for (int i = 0; i < nblk; ++i) m = fmax(m, part[i]);
  out[0] = m;
}

// phi -= mean phi (sums[1])
__global__ void k_sub_mean(double* phi, long long n, const double* sums) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  phi[i] -= sums[1];
}

unsigned blocks(long long n) { return (unsigned)((n + MG_T - 1) / MG_T); }

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// the levels of a box: itself, then full coarsenings while every coarse edge
// stays >= 8 and even where it must be (n_x / 2 even for the coarse FFT), as
// long as the level holds more than MG_COARSE nodes
std::vector<Level> make_levels(int nx, int ny, int nz) {
  std::vector<Level> lv;
  Level l{nx, ny, nz, (long long)nx * ny * nz, 1.0, nullptr, nullptr, nullptr};
  lv.push_back(l);
  while (l.n > MG_COARSE && l.nx % 4 == 0 && l.ny % 2 == 0 && l.nz % 2 == 0 && l.nx >= 16 &&
         l.ny >= 16 && l.nz >= 16) {
    l.nx /= 2;
    l.ny /= 2;
    l.nz /= 2;
    l.n = (long long)l.nx * l.ny * l.nz;
    l.c /= 4.0;
    lv.push_back(l);
  }
  return lv;
}

// scratch: b and r of level 0; phi, b, r of every coarser level; the
// coarsest level's spectrum; reduction slots
struct Layout {
  size_t b0, r0, coarse, spectrum, red, total;
};

Layout layout(const std::vector<Level>& lv) {
  Layout L;
  size_t off = 0;
  L.b0 = off;
  off += align256(lv[0].n * sizeof(double));
  L.r0 = off;
  off += align256(lv[0].n * sizeof(double));
  L.coarse = off;
  for (size_t k = 1; k < lv.size(); ++k) off += 3 * align256(lv[k].n * sizeof(double));
  L.spectrum = off;
  const Level& c = lv.back();
  off += align256(poisson_spectrum_bytes(c.nx, c.ny, c.nz));
  L.red = off;
  off += align256((MG_RED_BLOCKS + 4) * sizeof(double));
  L.total = off;
  return L;
}

struct Solver {
  std::vector<Level> lv;
  PoissonPlan coarse_plan;
  double2* spectrum;
  double* part;   // MG_RED_BLOCKS partial results
  double* out;    // [0] sum or maximum
  cudaStream_t s;
};

cudaError_t sum_of(const Solver& S, const double* x, long long n) {
  const int nb = (int)std::min<long long>(MG_RED_BLOCKS, (n + MG_T - 1) / MG_T);
  k_sum_partial<<<nb, MG_T, 0, S.s>>>(x, n, S.part);
  k_sum_final<<<1, 32, 0, S.s>>>(S.part, nb, n, S.out);
  return cudaGetLastError();
}

cudaError_t absmax_of(const Solver& S, const double* x, long long n, double& host) {
  const int nb = (int)std::min<long long>(MG_RED_BLOCKS, (n + MG_T - 1) / MG_T);
  k_absmax_partial<<<nb, MG_T, 0, S.s>>>(x, n, S.part);
  k_max_final<<<1, 32, 0, S.s>>>(S.part, nb, S.out);
  cudaError_t e = cudaMemcpyAsync(&host, S.out, sizeof(double), cudaMemcpyDeviceToHost, S.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S.s);
  return e;
}

cudaError_t smooth(const Solver& S, const Level& l) {
  for (int sweep = 0; sweep < 2; ++sweep)
    for (int colour = 0; colour < 2; ++colour)
      k_mg_rbgs<<<blocks(l.n / 2), MG_T, 0, S.s>>>(l.phi, l.b, l.nx, l.ny, l.nz, 1.0 / l.c, colour);
  return cudaGetLastError();
}

// one V-cycle from level k down
cudaError_t vcycle(const Solver& S, size_t k) {
  const Level& l = S.lv[k];
  if (k + 1 == S.lv.size()) {
    // exact on the coarsest level: c (6 phi - sum nb) = b is the FFT
    // solver's problem with 4 pi l_B = 1 / c
    Phys ph;
    memset(&ph, 0, sizeof(ph));
    ph.bjerrum = 1.0 / (4.0 * M_PI * l.c);
    return poisson_solve(S.coarse_plan, l.b, nullptr, nullptr, nullptr, ph, l.phi, S.spectrum, S.s);
  }
  const Level& c = S.lv[k + 1];
  cudaError_t e = smooth(S, l);
  if (e != cudaSuccess) return e;
  k_mg_resid<<<blocks(l.n), MG_T, 0, S.s>>>(l.phi, l.b, l.r, l.nx, l.ny, l.nz, l.c);
  k_mg_restrict<<<blocks(c.n), MG_T, 0, S.s>>>(l.r, l.nx, l.ny, l.nz, c.b, c.phi);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = vcycle(S, k + 1);
  if (e != cudaSuccess) return e;
  k_mg_prolong_add<<<blocks(l.n), MG_T, 0, S.s>>>(c.phi, l.nx, l.ny, l.nz, l.phi);
  return smooth(S, l);
}

}  // namespace

size_t poisson_mg_scratch_bytes(int nx, int ny, int nz) { return layout(make_levels(nx, ny, nz)).total; }

cudaError_t poisson_solve_mg(const PoissonPlan& coarse_plan, const double* q, double* phi, int nx,
                             int ny, int nz, double bjerrum, double tol, int max_cycles,
                             void* scratch, cudaStream_t s, int* cycles, double* residual) {
  Solver S;
  S.lv = make_levels(nx, ny, nz);
  const Layout L = layout(S.lv);
  unsigned char* base = static_cast<unsigned char*>(scratch);
  S.lv[0].phi = phi;
  S.lv[0].b = reinterpret_cast<double*>(base + L.b0);
  S.lv[0].r = reinterpret_cast<double*>(base + L.r0);
  size_t off = L.coarse;
  for (size_t k = 1; k < S.lv.size(); ++k) {
    const size_t sz = align256(S.lv[k].n * sizeof(double));
    S.lv[k].phi = reinterpret_cast<double*>(base + off);
    S.lv[k].b = reinterpret_cast<double*>(base + off + sz);
    S.lv[k].r = reinterpret_cast<double*>(base + off + 2 * sz);
    off += 3 * sz;
  }
  S.coarse_plan = coarse_plan;
  S.spectrum = reinterpret_cast<double2*>(base + L.spectrum);
  S.part = reinterpret_cast<double*>(base + L.red);
  S.out = S.part + MG_RED_BLOCKS;
  S.s = s;
  const Level& f = S.lv[0];
  // b = 4 pi l_B (q - mean q), read before phi (which may alias q) is written
  cudaError_t e = sum_of(S, q, f.n);
  if (e != cudaSuccess) return e;
  k_mg_rhs<<<blocks(f.n), MG_T, 0, s>>>(q, f.b, f.n, 4.0 * M_PI * bjerrum, S.out);
  e = cudaMemsetAsync(phi, 0, f.n * sizeof(double), s);
  double bmax = 0.0, rmax = 0.0;
  if (e == cudaSuccess) e = absmax_of(S, f.b, f.n, bmax);
  if (e != cudaSuccess) return e;
  int done = 0;
  while (bmax > 0.0 && done < max_cycles) {
    e = vcycle(S, 0);
    if (e != cudaSuccess) return e;
    ++done;
    k_mg_resid<<<blocks(f.n), MG_T, 0, s>>>(f.phi, f.b, f.r, f.nx, f.ny, f.nz, f.c);
    e = absmax_of(S, f.r, f.n, rmax);
    if (e != cudaSuccess) return e;
    if (rmax <= tol * bmax) break;
  }
  // the zero-mean solution (the periodic problem fixes phi up to a constant)
  e = sum_of(S, phi, f.n);
  if (e != cudaSuccess) return e;
  k_sub_mean<<<blocks(f.n), MG_T, 0, s>>>(phi, f.n, S.out);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (cycles) *cycles = done;
  if (residual) *residual = bmax > 0.0 ? rmax / bmax : 0.0;
  return e;
}

int poisson_mg_levels(int nx, int ny, int nz, int coarse[3]) {
  const std::vector<Level> lv = make_levels(nx, ny, nz);
  coarse[0] = lv.back().nx;
  coarse[1] = lv.back().ny;
  coarse[2] = lv.back().nz;
  return (int)lv.size();
}

}  // namespace ek
