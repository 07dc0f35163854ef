// Poisson solve with an inhomogeneous permittivity and fixed-potential nodes
// by preconditioned conjugate gradients (FP64): a multigrid V-cycle as the
// preconditioner where the box can be coarsened, else Jacobi.
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
// host reads the residual every CG_CHECK (Jacobi) or PCG_CHECK (multigrid)
// iterations.
#include <math.h>

#include <algorithm>

#include "ek_internal.cuh"

namespace ek {

namespace {

constexpr int CG_T = 256;         // threads per block
constexpr int CG_BLOCKS = 1216;   // blocks of the grid-stride kernels (8 per SM)
constexpr int CG_CHECK = 10;      // iterations between residual reads (Jacobi)
constexpr int PCG_CHECK = 2;      // with the multigrid V-cycle (an iteration costs several)

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

// ---------------------------------------------------------------------------
// Multigrid preconditioner: one V-cycle z = M r of the same operator.  Level
// l + 1 halves every edge of level l (while all are even and the coarse box
// keeps at least 2 nodes per edge); its node I covers the 8 nodes 2I + {0,1}^3.
// Coarse face permittivity: the 4 fine faces it covers, summed and halved
// (the flux through 4 faces over a distance twice as long); a coarse node is
// fixed (zero correction) when one of its nodes is.  Restriction sums the 8
// residuals, prolongation copies the coarse correction to the 8 nodes (the
// transpose of the restriction), the smoother is damped Jacobi (omega = 0.8),
// two sweeps before and after, and the coarsest level takes 40 sweeps from
// zero: every part is symmetric, so the V-cycle is a symmetric positive
// definite preconditioner for CG.
// ---------------------------------------------------------------------------
constexpr int MG_MAXLEV = 10;
constexpr double MG_OMEGA = 0.8;
constexpr int MG_COARSE_SWEEPS = 40;

struct MGLevel {
  int nx, ny, nz, n;
  double* cf;    // 3n face permittivities (+x, +y, +z)
  double* dinv;  // n: 1 / diagonal, 0 on fixed nodes
  double* x;     // n: the level's correction
  double* xt;    // n: the other Jacobi buffer
  double* b;     // n: the level's right-hand side
  double* r;     // n: residual
};

// the stencil A x at node n of level L (x is 0 on fixed nodes)
__device__ __forceinline__ double level_apply(const MGLevel& L, const double* x, int xx, int yy, int zz, int n) {
  const int sy = L.nx, sz = L.nx * L.ny;
  const int dxp = xx + 1 < L.nx ? 1 : 1 - L.nx, dxm = xx > 0 ? -1 : L.nx - 1;
  const int dyp = yy + 1 < L.ny ? sy : sy - sz, dym = yy > 0 ? -sy : sz - sy;
  const int dzp = zz + 1 < L.nz ? sz : sz - L.n, dzm = zz > 0 ? -sz : L.n - sz;
  const double* cx = L.cf;
  const double* cy = L.cf + L.n;
  const double* cz = L.cf + 2 * (size_t)L.n;
  const double xn = x[n];
  return cx[n] * (xn - x[n + dxp]) + cx[n + dxm] * (xn - x[n + dxm]) + cy[n] * (xn - x[n + dyp]) +
         cy[n + dym] * (xn - x[n + dym]) + cz[n] * (xn - x[n + dzp]) + cz[n + dzm] * (xn - x[n + dzm]);
}

// loop over the level's nodes with their coordinates: the work items are the
// 32 x 8 tiles of every plane, block b takes items b, b + gridDim.x, ... (no
// division per node)
#define MG_FOR_NODES(L)                                                                            \
  for (int w_ = blockIdx.x, tx_ = ((L).nx + 31) / 32, ty_ = ((L).ny + 7) / 8; w_ < tx_ * ty_ * (L).nz; \
       w_ += gridDim.x)                                                                            \
    if (const int xx_ = (w_ % tx_) * 32 + (int)(threadIdx.x & 31),                                 \
        yy_ = ((w_ / tx_) % ty_) * 8 + (int)(threadIdx.x >> 5), zz_ = w_ / (tx_ * ty_),            \
        n = xx_ + (L).nx * (yy_ + (L).ny * zz_);                                                   \
        xx_ < (L).nx && yy_ < (L).ny)

// one damped Jacobi sweep: out = in + omega D^-1 (b - A in); in == nullptr:
// from zero (out = omega D^-1 b)
__global__ void __launch_bounds__(CG_T) k_mg_jacobi(MGLevel L, const double* in, double* out) {
  MG_FOR_NODES(L) {
    const double di = L.dinv[n];
    if (di == 0.0) {
      out[n] = 0.0;
      continue;
    }
    if (!in) {
      out[n] = MG_OMEGA * di * L.b[n];
      continue;
    }
    out[n] = in[n] + MG_OMEGA * di * (L.b[n] - level_apply(L, in, xx_, yy_, zz_, n));
  }
}

__global__ void __launch_bounds__(CG_T) k_mg_residual(MGLevel L) {
  MG_FOR_NODES(L) {
    L.r[n] = L.dinv[n] == 0.0 ? 0.0 : L.b[n] - level_apply(L, L.x, xx_, yy_, zz_, n);
  }
}

// coarse right-hand side: the sum of the 8 fine residuals (0 at fixed nodes)
__global__ void __launch_bounds__(CG_T) k_mg_restrict(MGLevel F, MGLevel C) {
  MG_FOR_NODES(C) {
    if (C.dinv[n] == 0.0) {
      C.b[n] = 0.0;
      continue;
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int fx = 2 * xx_ + (c & 1), fy = 2 * yy_ + ((c >> 1) & 1), fz = 2 * zz_ + (c >> 2);
      s += F.r[fx + F.nx * (fy + F.ny * fz)];
    }
    C.b[n] = s;
  }
}

// fine x += the parent's coarse correction (free fine nodes)
__global__ void __launch_bounds__(CG_T) k_mg_prolong(MGLevel F, MGLevel C) {
  MG_FOR_NODES(F) {
    if (F.dinv[n] != 0.0) F.x[n] += C.x[(xx_ >> 1) + C.nx * ((yy_ >> 1) + C.ny * (zz_ >> 1))];
  }
}

// the coarse level's faces, diagonal and fixed nodes from the fine level
__global__ void __launch_bounds__(CG_T) k_mg_coarsen(MGLevel F, MGLevel C) {
  MG_FOR_NODES(C) {
    bool fixed = false;
    double fc[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int fx = 2 * xx_ + (c & 1), fy = 2 * yy_ + ((c >> 1) & 1), fz = 2 * zz_ + (c >> 2);
      const int m = fx + F.nx * (fy + F.ny * fz);
      fixed |= F.dinv[m] == 0.0;
      // the fine faces on the coarse node's + side: children with the upper
      // coordinate along that axis
      if (c & 1) fc[0] += F.cf[m];
      if ((c >> 1) & 1) fc[1] += F.cf[F.n + m];
      if (c >> 2) fc[2] += F.cf[2 * (size_t)F.n + m];
    }
    C.cf[n] = 0.5 * fc[0];
    C.cf[C.n + n] = 0.5 * fc[1];
    C.cf[2 * (size_t)C.n + n] = 0.5 * fc[2];
    C.dinv[n] = fixed ? 0.0 : 1.0;  // marks the fixed nodes; the diagonal follows
  }
}

__global__ void __launch_bounds__(CG_T) k_mg_diag(MGLevel C) {
  MG_FOR_NODES(C) {
    if (C.dinv[n] == 0.0) continue;
    const int sy = C.nx, sz = C.nx * C.ny;
    const int dxm = xx_ > 0 ? -1 : C.nx - 1, dym = yy_ > 0 ? -sy : sz - sy, dzm = zz_ > 0 ? -sz : C.n - sz;
    const double d = C.cf[n] + C.cf[n + dxm] + C.cf[C.n + n] + C.cf[C.n + n + dym] +
                     C.cf[2 * (size_t)C.n + n] + C.cf[2 * (size_t)C.n + n + dzm];
    C.dinv[n] = 1.0 / d;
  }
}
#undef MG_FOR_NODES

// the coarsest level: MG_COARSE_SWEEPS damped Jacobi sweeps from zero by one
// block (the level holds at most MG_COARSE_MAX nodes), ending in C.x
constexpr int MG_COARSE_MAX = 8192;
constexpr int MG_COARSE_T = 1024;
__global__ void __launch_bounds__(MG_COARSE_T) k_mg_coarse(MGLevel C) {
  for (int sweep = 0; sweep < MG_COARSE_SWEEPS; ++sweep) {
    const double* in = sweep == 0 ? nullptr : ((sweep & 1) ? C.xt : C.x);
    double* out = (sweep & 1) ? C.x : C.xt;
    for (int n = threadIdx.x; n < C.n; n += MG_COARSE_T) {
      const double di = C.dinv[n];
      if (di == 0.0) {
        out[n] = 0.0;
      } else if (!in) {
        out[n] = MG_OMEGA * di * C.b[n];
      } else {
        const int xx = n % C.nx, yy = (n / C.nx) % C.ny, zz = n / (C.nx * C.ny);
        out[n] = in[n] + MG_OMEGA * di * (C.b[n] - level_apply(C, in, xx, yy, zz, n));
      }
    }
    __syncthreads();
  }
}

// PCG with a general preconditioner z = M r
// x += alpha p, r -= alpha Ap; block sums of r.r and (for the projection) r
__global__ void __launch_bounds__(CG_T) k_pcg_update(Box b, CGView v, double* x) {
  const double alpha = v.sc[2];
  double rr = 0.0, s1 = 0.0;
  for (long long n = blockIdx.x * (long long)CG_T + threadIdx.x; n < b.N; n += (long long)gridDim.x * CG_T) {
    if (v.dinv[n] == 0.0) continue;
    x[n] += alpha * v.p[n];
    const double rn = v.r[n] - alpha * v.ap[n];
    v.r[n] = rn;
    rr += rn * rn;
    s1 += rn;
  }
  rr = block_total(rr);
  s1 = block_total(s1);
  if (threadIdx.x == 0) {
    v.part[CG_BLOCKS + blockIdx.x] = rr;
    v.part[2 * CG_BLOCKS + blockIdx.x] = s1;
  }
}

// r.r of the (projected) residual and the mean to remove
__global__ void __launch_bounds__(CG_T) k_pcg_mean(CGView v, int nb, long long N, int neutral) {
  const double rr = row_total(v.part, 1, nb);
  const double s1 = row_total(v.part, 2, nb);
  if (threadIdx.x == 0) {
    const double m = neutral ? s1 / (double)N : 0.0;
    v.sc[10] = m;
    v.sc[4] = neutral ? rr - m * s1 : rr;
  }
}

__global__ void __launch_bounds__(CG_T) k_pcg_project(Box b, CGView v) {
  const double m = v.sc[10];
  for (long long n = blockIdx.x * (long long)CG_T + threadIdx.x; n < b.N; n += (long long)gridDim.x * CG_T)
    if (v.dinv[n] != 0.0) v.r[n] -= m;
}

// block sums of r.z
__global__ void __launch_bounds__(CG_T) k_pcg_dot(Box b, CGView v, const double* z) {
  double t = 0.0;
  for (long long n = blockIdx.x * (long long)CG_T + threadIdx.x; n < b.N; n += (long long)gridDim.x * CG_T)
    if (v.dinv[n] != 0.0) t += v.r[n] * z[n];
  t = block_total(t);
  if (threadIdx.x == 0) v.part[blockIdx.x] = t;
}

// beta = r.z(new) / r.z(old) (first: r.z only, beta = 0)
__global__ void __launch_bounds__(CG_T) k_pcg_beta(CGView v, int nb, int first) {
  const double rz = row_total(v.part, 0, nb);
  if (threadIdx.x == 0) {
    v.sc[3] = (!first && v.sc[0] > 0.0) ? rz / v.sc[0] : 0.0;
    v.sc[0] = rz;
  }
}

// p = z + beta p on the free nodes
__global__ void __launch_bounds__(CG_T) k_pcg_direction(Box b, CGView v, const double* z) {
  const double beta = v.sc[3];
  for (long long n = blockIdx.x * (long long)CG_T + threadIdx.x; n < b.N; n += (long long)gridDim.x * CG_T)
    if (v.dinv[n] != 0.0) v.p[n] = z[n] + beta * v.p[n];
}

// the multigrid levels of a box: halving while every edge is even and the
// coarse edges stay >= 4; the coarsest must fit one block's solve
int mg_levels(int nx, int ny, int nz, int (*dims)[3]) {
  int L = 0;
  int d[3] = {nx, ny, nz};
  while (L < MG_MAXLEV) {
    dims[L][0] = d[0];
    dims[L][1] = d[1];
    dims[L][2] = d[2];
    ++L;
    if ((d[0] | d[1] | d[2]) & 1) break;
    if (d[0] / 2 < 4 || d[1] / 2 < 4 || d[2] / 2 < 4) break;
    for (int k = 0; k < 3; ++k) d[k] /= 2;
  }
  const long long coarsest = (long long)dims[L - 1][0] * dims[L - 1][1] * dims[L - 1][2];
  return (L >= 2 && coarsest <= MG_COARSE_MAX) ? L : 1;
}

}  // namespace

namespace {

// the CG arrays, then the preconditioner's: z, the fine level's Jacobi buffer
// and residual, and each coarser level's faces, diagonal, x, Jacobi buffer,
// right-hand side and residual (8 values per node)
size_t full_layout(int nx, int ny, int nz, CGView* v, void* base, MGLevel* lev, int* nlev, double** z) {
  const long long N = (long long)nx * ny * nz;
  size_t off = cg_layout(N, v, base);
  auto take = [&](size_t count) {
    off = (off + 255) & ~(size_t)255;
    double* p = base ? (double*)((char*)base + off) : nullptr;
    off += count * sizeof(double);
    return p;
  };
  int dims[MG_MAXLEV][3];
  const int L = mg_levels(nx, ny, nz, dims);
  double* zz = take((size_t)N);
  double* xt0 = take((size_t)N);
  double* r0 = take((size_t)N);
  if (lev) {
    *z = zz;
    *nlev = L;
    lev[0] = MGLevel{nx, ny, nz, (int)N, v->cf, v->dinv, zz, xt0, v->r, r0};
  }
  for (int l = 1; l < L; ++l) {
    const int n = dims[l][0] * dims[l][1] * dims[l][2];
    double* cf = take(3 * (size_t)n);
    double* di = take((size_t)n);
    double* x = take((size_t)n);
    double* xt = take((size_t)n);
    double* b = take((size_t)n);
    double* r = take((size_t)n);
    if (lev) lev[l] = MGLevel{dims[l][0], dims[l][1], dims[l][2], n, cf, di, x, xt, b, r};
  }
  return off;
}

unsigned level_blocks(const MGLevel& L) {
  const long long items = (long long)((L.nx + 31) / 32) * ((L.ny + 7) / 8) * L.nz;
  return (unsigned)std::min<long long>(CG_BLOCKS, items);
}

// z = M r: one V-cycle over the levels
void vcycle(const MGLevel* lev, int L, cudaStream_t s) {
  for (int l = 0; l < L - 1; ++l) {
    const MGLevel& A = lev[l];
    k_mg_jacobi<<<level_blocks(A), CG_T, 0, s>>>(A, nullptr, A.xt);
    k_mg_jacobi<<<level_blocks(A), CG_T, 0, s>>>(A, A.xt, A.x);
    k_mg_residual<<<level_blocks(A), CG_T, 0, s>>>(A);
    k_mg_restrict<<<level_blocks(lev[l + 1]), CG_T, 0, s>>>(A, lev[l + 1]);
  }
  k_mg_coarse<<<1, MG_COARSE_T, 0, s>>>(lev[L - 1]);
  for (int l = L - 2; l >= 0; --l) {
    const MGLevel& A = lev[l];
    k_mg_prolong<<<level_blocks(A), CG_T, 0, s>>>(A, lev[l + 1]);
    k_mg_jacobi<<<level_blocks(A), CG_T, 0, s>>>(A, A.x, A.xt);
    k_mg_jacobi<<<level_blocks(A), CG_T, 0, s>>>(A, A.xt, A.x);
  }
}

}  // namespace

size_t poisson_cg_scratch_bytes(int nx, int ny, int nz) {
  return full_layout(nx, ny, nz, nullptr, nullptr, nullptr, nullptr, nullptr);
}

cudaError_t poisson_solve_cg(const double* q, const double* eps, const unsigned char* fixed,
                             const double* phi_fixed, double* phi, int nx, int ny, int nz, double bjerrum,
                             double tol, int max_iter, void* scratch, cudaStream_t s, int* iters,
                             double* residual, bool* bad_eps) {
  const Box b{nx, ny, nz, (long long)nx * ny * nz};
  CGView v;
  MGLevel lev[MG_MAXLEV];
  int nlev = 1;
  double* z = nullptr;
  full_layout(nx, ny, nz, &v, scratch, lev, &nlev, &z);
  const bool mg = nlev >= 2;
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
    if (!mg) {
      k_cg_update<<<nb, CG_T, 0, s>>>(b, v, phi, neutral);
      k_cg_beta<<<1, CG_T, 0, s>>>(v, nb, b.N, neutral);
      k_cg_direction<<<nb, CG_T, 0, s>>>(b, v);
      return;
    }
    k_pcg_update<<<nb, CG_T, 0, s>>>(b, v, phi);
    k_pcg_mean<<<1, CG_T, 0, s>>>(v, nb, b.N, neutral);
    if (neutral) k_pcg_project<<<nb, CG_T, 0, s>>>(b, v);
    vcycle(lev, nlev, s);
    k_pcg_dot<<<nb, CG_T, 0, s>>>(b, v, z);
    k_pcg_beta<<<1, CG_T, 0, s>>>(v, nb, 0);
    k_pcg_direction<<<nb, CG_T, 0, s>>>(b, v, z);
  };
  if (mg && bnorm > 0.0) {
    // the coarse levels' operators, then p = z = M r and r.z
    for (int l = 1; l < nlev; ++l) {
      k_mg_coarsen<<<level_blocks(lev[l]), CG_T, 0, s>>>(lev[l - 1], lev[l]);
      k_mg_diag<<<level_blocks(lev[l]), CG_T, 0, s>>>(lev[l]);
    }
    vcycle(lev, nlev, s);
    k_pcg_dot<<<nb, CG_T, 0, s>>>(b, v, z);
    k_pcg_beta<<<1, CG_T, 0, s>>>(v, nb, 1);
    k_pcg_direction<<<nb, CG_T, 0, s>>>(b, v, z);
  }
  // the iterations between two residual reads as one graph (a caller stream
  // other than the legacy default stream can be captured); else the launches
  // one by one
  const int check = mg ? PCG_CHECK : CG_CHECK;
  cudaGraphExec_t graph = nullptr;
  if (s != nullptr && bnorm > 0.0 && max_iter >= check) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      for (int k = 0; k < check; ++k) iterate();
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
      const int batch = std::min(check, max_iter - it);
      if (batch == check && graph) {
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
