// Poisson solve with an inhomogeneous permittivity and fixed-potential nodes
// by Jacobi-preconditioned conjugate gradients (FP64).
//
// The paper solves Eq. 3 (homogeneous permittivity) by FFT and leaves the
// general problem div(eps grad Phi) = -4 pi l_B q to iterative solvers such as
// SOR or Krylov subspace methods (Sec. III.C, the paragraph after Eq. 16).
// Discretisation: the 7-point operator of the periodic solve with face
// permittivities, the harmonic mean 2 eps_i eps_j / (eps_i + eps_j) of the
// face's two nodes; a free node satisfies sum_f eps_f (Phi_i - Phi_j) =
// 4 pi l_B q_i, a fixed node holds its given potential.  The operator on the
// free nodes is symmetric positive definite (semidefinite with no fixed node:
// then the charge's mean is removed and Phi is returned with mean 0, as by
// the FFT solve).
//
// Every reduction (the CG inner products) is a fixed-order sum: each thread
// of a fixed grid adds its grid-stride elements in order, the block adds its
// threads in a fixed tree, one block adds the block sums in order; so a solve
// is bit-reproducible.  The scalars alpha and beta stay on the device; the
// host reads the residual every CG_CHECK iterations.
#include <math.h>

#include <algorithm>

#include "ek_internal.cuh"

namespace ek {

namespace {

constexpr int CG_T = 256;         // threads per block
constexpr int CG_BLOCKS = 1216;   // blocks of the grid-stride kernels (8 per SM)
constexpr int CG_CHECK = 10;      // iterations between residual reads

// scalars on the device: [0] r.z, [1] p.Ap, [2] alpha, [3] beta, [4] r.r,
// [5] b.b (then sum x), [6] sum q, [7] fixed-node count, [8] permittivities
// that are not positive and finite, [9] sum of D^-1, [10] mean of r to remove
//
// Without fixed nodes the operator is singular (constants): b has mean 0, and
// so has r = b - A x in exact arithmetic, but rounding lets a constant
// component creep into r, which A cannot remove; once the rest of r has
// converged, p points along it, p.Ap vanishes and alpha blows up.  There the
// mean of r is removed every iteration (r.z and r.r are formed for the
// projected r from the partial sums of r and D^-1 r).
struct CGView {
  double* cf;       // 3N: permittivity of the +x, +y, +z face of each node
  double* dinv;     // N: 1 / diagonal on free nodes, 0 on fixed nodes
  double* r;        // N: residual
  double* p;        // N: search direction
  double* ap;       // N: A p
  double* part;     // 4 * CG_BLOCKS block sums
  double* sc;       // 12 scalars
};

size_t cg_layout(long long N, CGView* v, void* base) {
  size_t off = 0;
  auto take = [&](double** ptr, size_t count) {
    off = (off + 255) & ~(size_t)255;
    if (v) *ptr = (double*)((char*)base + off);
    off += count * sizeof(double);
  };
  double* dummy = nullptr;
  take(v ? &v->cf : &dummy, 3 * (size_t)N);
  take(v ? &v->dinv : &dummy, (size_t)N);
  take(v ? &v->r : &dummy, (size_t)N);
  take(v ? &v->p : &dummy, (size_t)N);
  take(v ? &v->ap : &dummy, (size_t)N);
  take(v ? &v->part : &dummy, 4 * CG_BLOCKS);
  take(v ? &v->sc : &dummy, 12);
  return off;
}

struct Box {
  int nx, ny, nz;
  long long N;
};

__device__ __forceinline__ double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

// the block's sum of v (every thread), in a fixed tree; valid in thread 0
__device__ __forceinline__ double block_total(double v) {
  __shared__ double ws[CG_T / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();  // ws is reused by the next call
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < CG_T / 32; ++i) t += ws[i];
  return t;
}

// the sum of part[row * CG_BLOCKS + 0 .. nb) by one block: each thread adds
// its strided entries in order, then the fixed tree; valid in thread 0
__device__ __forceinline__ double row_total(const double* part, int row, int nb) {
  double t = 0.0;
  for (int i = threadIdx.x; i < nb; i += CG_T) t += part[row * CG_BLOCKS + i];
  return block_total(t);
}

// sum of q, the number of fixed nodes and of permittivities that are not
// positive and finite (block sums)
__global__ void __launch_bounds__(CG_T) k_cg_stats(Box b, const double* q, const double* eps,
                                                   const unsigned char* fixed, double* part) {
  double sq = 0.0, nf = 0.0, ne = 0.0;
  for (long long n = blockIdx.x * (long long)CG_T + threadIdx.x; n < b.N; n += (long long)gridDim.x * CG_T) {
    sq += q[n];
    if (fixed && fixed[n]) nf += 1.0;
    if (eps && !(eps[n] > 0.0 && eps[n] < INFINITY)) ne += 1.0;
  }
  sq = block_total(sq);
  nf = block_total(nf);
  ne = block_total(ne);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sq;
    part[CG_BLOCKS + blockIdx.x] = nf;
    part[2 * CG_BLOCKS + blockIdx.x] = ne;
  }
}

// the block sums of part's rows 0, 1, 2 (CG_BLOCKS apart), each added in
// order, into sc[i0], sc[i1], sc[i2] (a negative index: that row is skipped)
__global__ void __launch_bounds__(CG_T) k_cg_total(const double* part, int nb, double* sc, int i0, int i1,
                                                   int i2) {
  const double a = row_total(part, 0, nb);
  const double c = i1 >= 0 ? row_total(part, 1, nb) : 0.0;
  const double d = i2 >= 0 ? row_total(part, 2, nb) : 0.0;
  if (threadIdx.x == 0) {
    sc[i0] = a;
    if (i1 >= 0) sc[i1] = c;
    if (i2 >= 0) sc[i2] = d;
  }
}

__device__ __forceinline__ void neighbours(const Box& b, long long n, long long (&m)[6]) {
  const int x = (int)(n % b.nx), y = (int)((n / b.nx) % b.ny), z = (int)(n / ((long long)b.nx * b.ny));
  const long long sy = b.nx, sz = (long long)b.nx * b.ny;
  m[0] = n + (x + 1 < b.nx ? 1 : 1 - b.nx);   // +x
  m[1] = n + (x > 0 ? -1 : b.nx - 1);         // -x
  m[2] = n + (y + 1 < b.ny ? sy : sy - sz);   // +y
  m[3] = n + (y > 0 ? -sy : sz - sy);         // -y
  m[4] = n + (z + 1 < b.nz ? sz : sz - b.N);  // +z
  m[5] = n + (z > 0 ? -sz : b.N - sz);        // -z
}

// faces, diagonal, right-hand side and the start x = 0 (free) / phi_fixed
// (fixed); r = b, p = z = D^-1 r; block sums of r.z and b.b
__global__ void __launch_bounds__(CG_T) k_cg_prep(Box b, CGView v, const double* q, const double* eps,
                                                  const unsigned char* fixed, const double* phi_fixed,
                                                  double* x, double scale, const double* sc, int neutral) {
  const double qmean = neutral ? sc[6] / (double)b.N : 0.0;
  double rz = 0.0, bb = 0.0, sd = 0.0;
  for (long long n = blockIdx.x * (long long)CG_T + threadIdx.x; n < b.N; n += (long long)gridDim.x * CG_T) {
    long long m[6];
    neighbours(b, n, m);
    const double en = eps ? eps[n] : 1.0;
    double f[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) f[k] = eps ? harmonic(en, eps[m[k]]) : 1.0;
    v.cf[n] = f[0];
    v.cf[b.N + n] = f[2];
    v.cf[2 * b.N + n] = f[4];
    const bool fx = fixed && fixed[n];
    if (fx) {
      const double pv = phi_fixed ? phi_fixed[n] : 0.0;
      x[n] = pv;
      v.dinv[n] = 0.0;
      v.r[n] = 0.0;
      v.p[n] = 0.0;
      continue;
    }
    double rhs = scale * (q[n] - qmean);
    double d = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      d += f[k];
      if (fixed && fixed[m[k]]) rhs += f[k] * (phi_fixed ? phi_fixed[m[k]] : 0.0);
    }
    const double di = 1.0 / d;
    x[n] = 0.0;
    v.dinv[n] = di;
    v.r[n] = rhs;
    v.p[n] = di * rhs;
    rz += di * rhs * rhs;
    bb += rhs * rhs;
    sd += di;
  }
  rz = block_total(rz);
  bb = block_total(bb);
  sd = block_total(sd);
  if (threadIdx.x == 0) {
    v.part[blockIdx.x] = rz;
    v.part[CG_BLOCKS + blockIdx.x] = bb;
    v.part[2 * CG_BLOCKS + blockIdx.x] = sd;
  }
}

// Ap on the free nodes (p is 0 on fixed nodes); block sums of p.Ap.  The
// work items are the 32 x 8 tiles of every plane (tx x ty tiles per plane);
// block b takes items b, b + gridDim.x, ...: node coordinates come from the
// item, with no division per node.
__global__ void __launch_bounds__(CG_T) k_cg_apply(Box b, CGView v, int tx, int ty) {
  const int N = (int)b.N, sy = b.nx, sz = b.nx * b.ny;
  const int items = tx * ty * b.nz;
  const double* __restrict__ cx = v.cf;
  const double* __restrict__ cy = v.cf + N;
  const double* __restrict__ cz = v.cf + 2 * (size_t)N;
  double pap = 0.0;
  for (int w = blockIdx.x; w < items; w += gridDim.x) {
    const int bx = w % tx, by = (w / tx) % ty, z = w / (tx * ty);
    const int x = bx * 32 + (threadIdx.x & 31), y = by * 8 + (threadIdx.x >> 5);
    if (x >= b.nx || y >= b.ny) continue;
    const int n = x + sy * y + sz * z;
    if (v.dinv[n] == 0.0) {
      v.ap[n] = 0.0;
      continue;
    }
    const int dxp = x + 1 < b.nx ? 1 : 1 - b.nx, dxm = x > 0 ? -1 : b.nx - 1;
    const int dyp = y + 1 < b.ny ? sy : sy - sz, dym = y > 0 ? -sy : sz - sy;
    const int dzp = z + 1 < b.nz ? sz : sz - N, dzm = z > 0 ? -sz : N - sz;
    const double pn = v.p[n];
    const double a = cx[n] * (pn - v.p[n + dxp]) + cx[n + dxm] * (pn - v.p[n + dxm]) +
                     cy[n] * (pn - v.p[n + dyp]) + cy[n + dym] * (pn - v.p[n + dym]) +
                     cz[n] * (pn - v.p[n + dzp]) + cz[n + dzm] * (pn - v.p[n + dzm]);
    v.ap[n] = a;
    pap += pn * a;
  }
  pap = block_total(pap);
  if (threadIdx.x == 0) v.part[blockIdx.x] = pap;
}

// alpha = r.z / p.Ap
__global__ void __launch_bounds__(CG_T) k_cg_alpha(CGView v, int nb) {
  const double pap = row_total(v.part, 0, nb);
  if (threadIdx.x == 0) {
    v.sc[1] = pap;
    v.sc[2] = pap > 0.0 ? v.sc[0] / pap : 0.0;
  }
}

// x += alpha p, r -= alpha Ap; block sums of the new r.z, r.r, and (for
// the projection) of r and D^-1 r
__global__ void __launch_bounds__(CG_T) k_cg_update(Box b, CGView v, double* x, int neutral) {
  const double alpha = v.sc[2];
  double rz = 0.0, rr = 0.0, s1 = 0.0, s2 = 0.0;
  for (long long n = blockIdx.x * (long long)CG_T + threadIdx.x; n < b.N; n += (long long)gridDim.x * CG_T) {
    const double di = v.dinv[n];
    if (di == 0.0) continue;
    x[n] += alpha * v.p[n];
    const double rn = v.r[n] - alpha * v.ap[n];
    v.r[n] = rn;
    rz += di * rn * rn;
    rr += rn * rn;
    s1 += rn;
    s2 += di * rn;
  }
  rz = block_total(rz);
  rr = block_total(rr);
  if (neutral) {
    s1 = block_total(s1);
    s2 = block_total(s2);
  }
  if (threadIdx.x == 0) {
    v.part[blockIdx.x] = rz;
    v.part[CG_BLOCKS + blockIdx.x] = rr;
    if (neutral) {
      v.part[2 * CG_BLOCKS + blockIdx.x] = s1;
      v.part[3 * CG_BLOCKS + blockIdx.x] = s2;
    }
  }
}

// beta = r.z(new) / r.z(old); r.r for the convergence test; with the
// projection (every node free): m = mean r, and r.z, r.r of r - m
__global__ void __launch_bounds__(CG_T) k_cg_beta(CGView v, int nb, long long N, int neutral) {
  double rz = row_total(v.part, 0, nb);
  double rr = row_total(v.part, 1, nb);
  double s1 = 0.0, s2 = 0.0;
  if (neutral) {
    s1 = row_total(v.part, 2, nb);
    s2 = row_total(v.part, 3, nb);
  }
  if (threadIdx.x == 0) {
    double m = 0.0;
    if (neutral) {
      m = s1 / (double)N;
      rz = rz - 2.0 * m * s2 + m * m * v.sc[9];
      rr = rr - m * s1;
    }
    v.sc[10] = m;
    v.sc[3] = v.sc[0] > 0.0 ? rz / v.sc[0] : 0.0;
    v.sc[0] = rz;
    v.sc[4] = rr;
  }
}

// r -= m (the projection; m = 0 with fixed nodes), p = D^-1 r + beta p on
// the free nodes
__global__ void __launch_bounds__(CG_T) k_cg_direction(Box b, CGView v) {
  const double beta = v.sc[3], m = v.sc[10];
  for (long long n = blockIdx.x * (long long)CG_T + threadIdx.x; n < b.N; n += (long long)gridDim.x * CG_T) {
    const double di = v.dinv[n];
    if (di != 0.0) {
      const double rn = v.r[n] - m;
      v.r[n] = rn;
      v.p[n] = di * rn + beta * v.p[n];
    }
  }
}

// block sums of x (for the mean of a solution without fixed nodes)
__global__ void __launch_bounds__(CG_T) k_cg_sum(Box b, const double* x, double* part) {
  double s = 0.0;
  for (long long n = blockIdx.x * (long long)CG_T + threadIdx.x; n < b.N; n += (long long)gridDim.x * CG_T)
    s += x[n];
  s = block_total(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(CG_T) k_cg_shift(Box b, double* x, const double* sc) {
  const double mean = sc[5] / (double)b.N;
  for (long long n = blockIdx.x * (long long)CG_T + threadIdx.x; n < b.N; n += (long long)gridDim.x * CG_T)
    x[n] -= mean;
}

}  // namespace

size_t poisson_cg_scratch_bytes(int nx, int ny, int nz) {
  return cg_layout((long long)nx * ny * nz, nullptr, nullptr);
}

cudaError_t poisson_solve_cg(const double* q, const double* eps, const unsigned char* fixed,
                             const double* phi_fixed, double* phi, int nx, int ny, int nz, double bjerrum,
                             double tol, int max_iter, void* scratch, cudaStream_t s, int* iters,
                             double* residual, bool* bad_eps) {
  const Box b{nx, ny, nz, (long long)nx * ny * nz};
  CGView v;
  cg_layout(b.N, &v, scratch);
  const int nb = (int)std::min<long long>(CG_BLOCKS, (b.N + CG_T - 1) / CG_T);
  const int tx = (nx + 31) / 32, ty = (ny + 7) / 8;
  const int na = (int)std::min<long long>(CG_BLOCKS, (long long)tx * ty * nz);  // operator blocks
  double h[12];
  *bad_eps = false;
  // the charge's sum, the fixed-node count and the invalid permittivities
  k_cg_stats<<<nb, CG_T, 0, s>>>(b, q, eps, fixed, v.part);
  k_cg_total<<<1, CG_T, 0, s>>>(v.part, nb, v.sc, 6, 7, 8);
  cudaError_t e = cudaMemcpyAsync(h, v.sc, 12 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (h[8] != 0.0) {
    *bad_eps = true;
    return cudaSuccess;
  }
  const int neutral = h[7] == 0.0 ? 1 : 0;  // no fixed node: remove the mean charge
  k_cg_prep<<<nb, CG_T, 0, s>>>(b, v, q, eps, fixed, phi_fixed, phi, 4.0 * M_PI * bjerrum, v.sc, neutral);
  k_cg_total<<<1, CG_T, 0, s>>>(v.part, nb, v.sc, 0, 5, 9);
  e = cudaMemcpyAsync(h, v.sc, 12 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  const double bnorm = sqrt(h[5]);
  int it = 0;
  double rel = 0.0;
  auto iterate = [&]() {
    k_cg_apply<<<na, CG_T, 0, s>>>(b, v, tx, ty);
    k_cg_alpha<<<1, CG_T, 0, s>>>(v, na);
    k_cg_update<<<nb, CG_T, 0, s>>>(b, v, phi, neutral);
    k_cg_beta<<<1, CG_T, 0, s>>>(v, nb, b.N, neutral);
    k_cg_direction<<<nb, CG_T, 0, s>>>(b, v);
  };
  // CG_CHECK iterations as one graph (a caller stream other than the legacy
  // default stream can be captured); else the launches one by one
  cudaGraphExec_t graph = nullptr;
  if (s != nullptr && bnorm > 0.0 && max_iter >= CG_CHECK) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      for (int k = 0; k < CG_CHECK; ++k) iterate();
      if (cudaStreamEndCapture(s, &g) == cudaSuccess && g) {
        if (cudaGraphInstantiate(&graph, g, 0) != cudaSuccess) graph = nullptr;
      }
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();  // a failed capture leaves the launches one by one
  }
  if (bnorm > 0.0) {
    rel = 1.0;
    while (it < max_iter && rel > tol) {
      const int batch = std::min(CG_CHECK, max_iter - it);
      if (batch == CG_CHECK && graph) {
        e = cudaGraphLaunch(graph, s);
        if (e != cudaSuccess) break;
      } else {
        for (int k = 0; k < batch; ++k) iterate();
      }
      it += batch;
      e = cudaMemcpyAsync(h, v.sc, 12 * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) break;
      rel = sqrt(h[4]) / bnorm;
      if (!(rel == rel)) break;  // not a number: reported to the caller
    }
  }
  if (graph) cudaGraphExecDestroy(graph);
  if (e != cudaSuccess) return e;
  if (neutral) {
    k_cg_sum<<<nb, CG_T, 0, s>>>(b, phi, v.part);
    k_cg_total<<<1, CG_T, 0, s>>>(v.part, nb, v.sc, 5, -1, -1);
    k_cg_shift<<<nb, CG_T, 0, s>>>(b, phi, v.sc);
  }
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (iters) *iters = it;
  if (residual) *residual = rel;
  return e;
}

}  // namespace ek
