// S4 (particle forces and symplectic Euler integration) and S5 (re-flagging,
// octree partial volumes Psi, Psi-smeared particle charge, fluid
// create/destroy and solute expulsion/refill), FP64.
//
// All particle work is box-local: particle p touches only the cells of its
// box [lo, hi) = [floor(r - R) - 1, floor(r + R) + 2) per axis (unwrapped
// coordinates, so r_b - r never crosses the periodic seam), or of the union of
// its previous and current boxes in S5.  Grids are (particle, chunk of box
// cells).  Reductions over a particle (force, torque) run in a fixed order
// (per CTA, then over chunks), so they are deterministic; sums of Psi are
// dyadic fractions and exact in any order.
#include <math.h>

#include "ek_internal.cuh"

namespace ek {

namespace {

constexpr int PT = 256;  // threads per particle CTA

__device__ __forceinline__ int box_cells(const int lo[3], const int hi[3]) {
  return (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
}

__device__ __forceinline__ void box_coord(int c, const int lo[3], const int hi[3], int& X, int& Y,
                                          int& Z) {
  const int bx = hi[0] - lo[0], by = hi[1] - lo[1];
  X = lo[0] + c % bx;
  Y = lo[1] + (c / bx) % by;
  Z = lo[2] + c / (bx * by);
}

// periodic coordinate of a widened-box coordinate: the box lies within one
// period on either side of the lattice (2R + 6 <= edge, margin ceil(R) + 4),
// so v is in [-2n, 3n) and two conditional wraps replace a modulo
__device__ __forceinline__ int wrap_box(int v, int n) {
  v = v < 0 ? v + n : (v >= n ? v - n : v);
  return v < 0 ? v + n : (v >= n ? v - n : v);
}

__device__ __forceinline__ long long node_of(int X, int Y, int Z, const Grid& g) {
  return (long long)wrapi(X, g.nx) +
         (long long)g.nx * ((long long)wrapi(Y, g.ny) + (long long)g.ny * wrapi(Z, g.nz));
}

// squared distance, evaluated left to right without contraction so every
// inside/outside decision is reproducible bit for bit
__device__ __forceinline__ double dist2(double dx, double dy, double dz) {
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

enum { CUBE_IN = 0, CUBE_OUT = 1, CUBE_UNDECIDED = 2 };

// Cube of centre c and half-width h against the sphere (r, R^2).  Inside: all
// 8 corners strictly inside; it suffices to test the farthest corner, whose
// rounded distance bounds the rounded distance of every other corner.
// Outside: the closest point of the cube is at distance >= R.
__device__ __forceinline__ int classify(double cx, double cy, double cz, double h,
                                        const double r[3], double R2) {
  const double ax = __dsub_rn(__dsub_rn(cx, h), r[0]), bx = __dsub_rn(__dadd_rn(cx, h), r[0]);
  const double ay = __dsub_rn(__dsub_rn(cy, h), r[1]), by = __dsub_rn(__dadd_rn(cy, h), r[1]);
  const double az = __dsub_rn(__dsub_rn(cz, h), r[2]), bz = __dsub_rn(__dadd_rn(cz, h), r[2]);
  const double fx = fabs(ax) > fabs(bx) ? ax : bx;
  const double fy = fabs(ay) > fabs(by) ? ay : by;
  const double fz = fabs(az) > fabs(bz) ? az : bz;
  if (dist2(fx, fy, fz) < R2) return CUBE_IN;
  const double px = __dsub_rn(fmin(fmax(r[0], __dsub_rn(cx, h)), __dadd_rn(cx, h)), r[0]);
  const double py = __dsub_rn(fmin(fmax(r[1], __dsub_rn(cy, h)), __dadd_rn(cy, h)), r[1]);
  const double pz = __dsub_rn(fmin(fmax(r[2], __dsub_rn(cz, h)), __dadd_rn(cz, h)), r[2]);
  if (dist2(px, py, pz) >= R2) return CUBE_OUT;
  return CUBE_UNDECIDED;
}

// Single-precision pre-test of classify().  (ox, oy, oz) is the cube centre
// relative to the sphere centre in float: the centre relative to the sphere
// centre's integer part (exact: an integer plus dyadic offsets) minus the
// float fraction of the sphere centre, one rounding each (absolute error per
// component below 2 * 2^-24 (R + 2)); the float squared distances of the
// farthest corner and of the closest point are then well within
// 3.5e-6 (R + 2)^2 of the exact ones, so
// whenever they are more than `margin` = 6e-6 (R + 2)^2 away from R^2 the FP64
// decision is already known.  Returns -1 when the exact test is needed.
__device__ __forceinline__ int classify_f32(float ox, float oy, float oz, float h, float R2,
                                            float margin) {
  const float ax = fabsf(ox), ay = fabsf(oy), az = fabsf(oz);
  const float fx = ax + h, fy = ay + h, fz = az + h;
  const float dfar = fx * fx + fy * fy + fz * fz;
  if (dfar < R2 - margin) return CUBE_IN;
  const bool not_in = dfar > R2 + margin;
  const float px = fmaxf(ax - h, 0.0f), py = fmaxf(ay - h, 0.0f), pz = fmaxf(az - h, 0.0f);
  const float dnear = px * px + py * py + pz * pz;
  if (not_in) {
    if (dnear > R2 + margin) return CUBE_OUT;
    if (dnear < R2 - margin) return CUBE_UNDECIDED;
  }
  return -1;
}

// Second-tier test in float pairs (hi + lo, about 44 significant bits), for
// the sub-cubes the float pre-test cannot decide: the GPU's FP64 rate is a
// small fraction of its FP32 rate, so FP64 is left to true near-ties.  (ax,
// ay, az) is the sub-cube centre minus the centre's integer part, exact in
// float (an integer plus dyadic offsets); the centre's fraction and R^2 come as
// float pairs.  The pair arithmetic approximates the exact corner distances to
// ~1e-12 (R + 2)^2, and the FP64 test's own rounding is below 1e-13 (R + 2)^2,
// so a distance more than 1e-10 (R + 2)^2 from R^2 gives the FP64 decision.
struct f2 {
  float hi, lo;
};
__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ f2 quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  const f2 s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ f2 f2_sqr(f2 a) {
  const float p = __fmul_rn(a.hi, a.hi);
  float e = __fmaf_rn(a.hi, a.hi, -p);
  e = __fmaf_rn(__fmul_rn(2.0f, a.hi), a.lo, e);
  return quick_two_sum(p, e);
}
// |o| + h (far) or max(|o| - h, 0) (near) for o = a - (fhi + flo)
__device__ __forceinline__ void f2_axis(float a, float fhi, float flo, float h, f2& far, f2& near) {
  const f2 s = two_sum(a, -fhi);
  f2 o = quick_two_sum(s.hi, __fsub_rn(s.lo, flo));
  if (o.hi < 0.0f) o = {-o.hi, -o.lo};
  const f2 fa = two_sum(o.hi, h);
  far = quick_two_sum(fa.hi, __fadd_rn(fa.lo, o.lo));
  const f2 na = two_sum(o.hi, -h);
  near = quick_two_sum(na.hi, __fadd_rn(na.lo, o.lo));
  if (near.hi <= 0.0f) near = {0.0f, 0.0f};
}
__device__ __forceinline__ int classify_f2(float ax, float ay, float az, float h, const DevParticle& P) {
  f2 fx, fy, fz, nx, ny, nz;
  f2_axis(ax, P.fpos[0], P.fposlo[0], h, fx, nx);
  f2_axis(ay, P.fpos[1], P.fposlo[1], h, fy, ny);
  f2_axis(az, P.fpos[2], P.fposlo[2], h, fz, nz);
  const f2 mr2 = {-P.r2f, -P.r2lo};
  const float Rp = sqrtf(P.r2f) + 2.0f;
  const float tol = 1e-10f * Rp * Rp;
  const f2 df = f2_add(f2_add(f2_add(f2_sqr(fx), f2_sqr(fy)), f2_sqr(fz)), mr2);
  const float Df = __fadd_rn(df.hi, df.lo);
  if (Df < -tol) return CUBE_IN;
  if (Df <= tol) return -1;
  const f2 dn = f2_add(f2_add(f2_add(f2_sqr(nx), f2_sqr(ny)), f2_sqr(nz)), mr2);
  const float Dn = __fadd_rn(dn.hi, dn.lo);
  if (Dn > tol) return CUBE_OUT;
  if (Dn < -tol) return CUBE_UNDECIDED;
  return -1;
}

// Octree partial volume Psi_p of one cell (Sec. III.D.2): the cell is split
// into 8 sub-cells, each classified as completely inside or completely
// outside; undecided ones are split again, down to depth 4 (edge 1/16), where
// an undecided cube counts half.  Level 0 (the cell itself) is decided by
// k_claim; cells still undecided there go to k_psi_surface, which counts the
// cell's level-4 cubes that are inside or undecided, column by column (one
// warp per cell; a cube's status follows from its ancestors', so the counts
// give the tree's result exactly).  Volumes are counted in units of 1/8192
// (half a level-4 cube), so the sums are exact in any order.
constexpr int PSI_UNITS = 8192;

// sum of Psi_p over the particle's box (counts of 2^-13 units: exact)
__device__ __forceinline__ double psi_sum(const DevParticle& P) {
  unsigned long long u = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) u += P.psiunits[j];
  return (double)u / (double)PSI_UNITS;
}

// u * 2^-13 (1 <= u < 2^20) as a double, assembled from its bits: exact,
// and no FP64 instruction (the GPU's FP64 pipe is narrow and this runs once
// per surface cell)
__device__ __forceinline__ double dyadic13(unsigned u) {
  const int e = 31 - __clz(u);  // u in [2^e, 2^(e+1))
  const unsigned long long mant = ((unsigned long long)u << (52 - e)) & ((1ULL << 52) - 1ULL);
  return __longlong_as_double((long long)(((unsigned long long)(1023 + e - 13) << 52) | mant));
}
// a Psi_p entry of the box (0 or u * 2^-13, u <= 8192: a normal float with at
// most 14 significant bits) as a float, from its bits: exact
__device__ __forceinline__ float psibox_float(unsigned long long bits) {
  return bits ? __int_as_float((int)((bits >> 29) - (896ULL << 23))) : 0.0f;
}

// exact (double) centre of sub-cube `path` at level l of the cell centred
// at (X, Y, Z); path holds 3 bits per level, level 1 highest
__device__ __forceinline__ void subcube_centre_d(int path, int l, double X, double Y, double Z,
                                                 double& cx, double& cy, double& cz) {
  cx = X;
  cy = Y;
  cz = Z;
  for (int m = 1; m <= l; ++m) {
    const int bits = (path >> (3 * (l - m))) & 7;
    const double hm = ldexp(1.0, -(m + 1));
    cx += (bits & 1) ? hm : -hm;
    cy += (bits & 2) ? hm : -hm;
    cz += (bits & 4) ? hm : -hm;
  }
}

__device__ __forceinline__ float psi_margin(double R2) {
  const float Rp2 = sqrtf((float)R2) + 2.0f;
  return 6e-6f * Rp2 * Rp2;
}

// the sub-cube test in three tiers: float, float pair, FP64 (see above)
// the FP64 tier as a real call: inlined, its FP64 instructions would be
// issued (predicated off) on every pass through the caller
__device__ __noinline__ int classify_exact(int path, int l, int X, int Y, int Z, const DevParticle* P) {
  double ex, ey, ez;
  subcube_centre_d(path, l, (double)X, (double)Y, (double)Z, ex, ey, ez);
  return classify(ex, ey, ez, ldexp(1.0, -(l + 1)), P->pos, __dmul_rn(P->radius, P->radius));
}

__device__ __forceinline__ int classify_tiers(float ax, float ay, float az, int path, int l,
                                              int X, int Y, int Z, const DevParticle& P) {
  const float h = ldexpf(1.0f, -(l + 1));
  const float cx = __fsub_rn(ax, P.fpos[0]), cy = __fsub_rn(ay, P.fpos[1]), cz = __fsub_rn(az, P.fpos[2]);
  int st = classify_f32(cx, cy, cz, h, P.r2f, P.psimargin);
  if (st >= 0) return st;
  st = classify_f2(ax, ay, az, h, P);
  if (st >= 0) return st;
  return classify_exact(path, l, X, Y, Z, &P);
}

__device__ __noinline__ bool node_inside_exact(int X, int Y, int Z, const DevParticle* P) {
  const double dx = (double)X - P->pos[0], dy = (double)Y - P->pos[1], dz = (double)Z - P->pos[2];
  return dist2(dx, dy, dz) < __dmul_rn(P->radius, P->radius);
}

// node centre strictly inside the sphere: float test, FP64 within its margin
__device__ __forceinline__ bool node_inside_tiers(int X, int Y, int Z, const DevParticle& P) {
  const float dx = __fsub_rn((float)(X - P.ipos[0]), P.fpos[0]);
  const float dy = __fsub_rn((float)(Y - P.ipos[1]), P.fpos[1]);
  const float dz = __fsub_rn((float)(Z - P.ipos[2]), P.fpos[2]);
  const float d2 = dx * dx + dy * dy + dz * dz;
  if (d2 < P.r2f - P.psimargin) return true;
  if (d2 > P.r2f + P.psimargin) return false;
  return node_inside_exact(X, Y, Z, &P);
}


// typed access to the fields of the two storage forms
template <class FM>
__device__ __forceinline__ double pop_abs(const void* f, int i, long long N, long long n, double rho0) {
  const double v = (double)((const typename FM::pop_t*)f)[(long long)i * N + n];
  return FM::fp32 ? v + wgt(i) * rho0 : v;
}
template <class FM>
__device__ __forceinline__ double real_at(const void* p, long long n) {
  return (double)((const typename FM::real_t*)p)[n];
}
template <class FM>
__device__ __forceinline__ void real_set(void* p, long long n, double v) {
  ((typename FM::real_t*)p)[n] = (typename FM::real_t)v;
}
template <class FM>
__device__ __forceinline__ void real_add(void* p, long long n, double v) {
  atomicAdd((typename FM::real_t*)p + n, (typename FM::real_t)v);
}

// block-wide sum of NV doubles, fixed order; result valid in thread 0
template <int NV>
__device__ void block_sum(double (&v)[NV]) {
  __shared__ double red[PT / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double s = v[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][j] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += red[w][j];
      v[j] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// S4: forces and integration.
//   k_force_assign   every fluid node of a particle's widened box records the
//                    particle with the nearest surface (minimum image): an
//                    atomicMin on the key (quantised surface distance, index)
//   k_particle_forces  grid (particle, chunk of fcells widened-box cells):
//                    momentum exchange (Eq. 11), the solute force on the
//                    particle (reaction of the internal solute force on the
//                    fluid of its nodes) and the field on its own charge
//                    The last block of a particle sums its rows; the last
//                    particle takes the remainder of the solute force on
//                    nodes no particle claims, split evenly, and integrates
//                    (symplectic Euler)
// All sums run in a fixed order, so the result is deterministic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double min_image(double d, int n) {
  if (d > 0.5 * (double)n) return d - (double)n;
  if (d < -0.5 * (double)n) return d + (double)n;
  return d;
}

// cell c of the widened box: node index and minimum-image offset from the
// centre.  Returns true for the first copy of a node (a widened box can be
// wider than the lattice), so per-node sums count every node once.
__device__ __forceinline__ bool ext_cell(const DevParticle& P, int c, const Grid& g, int& X, int& Y,
                                        int& Z, long long& n, double& dx, double& dy, double& dz,
                                        int* wrapped = nullptr) {
  box_coord(c, P.elo, P.ehi, X, Y, Z);
  const bool first = X - P.elo[0] < g.nx && Y - P.elo[1] < g.ny && Z - P.elo[2] < g.nz;
  const int x = wrapi(X, g.nx), y = wrapi(Y, g.ny), z = wrapi(Z, g.nz);
  if (wrapped) {
    wrapped[0] = x;
    wrapped[1] = y;
    wrapped[2] = z;
  }
  n = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
  dx = min_image(__dsub_rn((double)x, P.pos[0]), g.nx);
  dy = min_image(__dsub_rn((double)y, P.pos[1]), g.ny);
  dz = min_image(__dsub_rn((double)z, P.pos[2]), g.nz);
  return first;
}

// FP64 surface distance of node (x, y, z) (wrapped coordinates) from particle
// P: minimum-image offset, squares summed left to right, correctly rounded
// square root, minus R; every operation rounded to nearest, no contraction.
__device__ __forceinline__ double surface_distance64(const DevParticle& P, int x, int y, int z,
                                                     const Grid& g) {
  const double dx = min_image(__dsub_rn((double)x, P.pos[0]), g.nx);
  const double dy = min_image(__dsub_rn((double)y, P.pos[1]), g.ny);
  const double dz = min_image(__dsub_rn((double)z, P.pos[2]), g.nz);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return __dsub_rn(__dsqrt_rn(d2), P.radius);
}

__device__ __forceinline__ float key_distance(unsigned long long key) {
  unsigned bits = (unsigned)(key >> 20);
  bits = (bits & 0x80000000u) ? (bits & 0x7FFFFFFFu) : ~bits;
  return __uint_as_float(bits);
}

// The nearest particle of a node is the one with the smallest FP64 surface
// distance (surface_distance64), equal distances to the lower index.  The key
// holds a float estimate of it: the offset from the centre's integer part and
// float fraction, wrapped in float, squares summed, sqrt, minus R.  Its error
// against the FP64 distance is below 2^-24 (5.5 |d| + 2 R + 4.4) <=
// 2^-21 (|d| + R + 1) (offset 2^-23 (|d| + 1.25) per axis, the square sum,
// the root, R rounded to float, the difference), so when the float and the
// FP64 orders disagree the two distances lie within 2 such bounds of each
// other, and of the final minimum.  Whichever of the two writes its key second
// then finds the other's (or a smaller, still within the window) in the value
// atomicMin returns and lists the node; k_tie_resolve decides the listed nodes
// in FP64.
__device__ __forceinline__ void force_assign_body(const PartArgs& a, const Blk bk) {
  const int p = bk.x;
  const DevParticle& P = a.parts[p];
  const int c = bk.y * blockDim.x + threadIdx.x;
  if (c >= box_cells(P.elo, P.ehi)) return;
  int X, Y, Z;
  box_coord(c, P.elo, P.ehi, X, Y, Z);  // a repeated node gets the same key
  const int x = wrap_box(X, a.g.nx), y = wrap_box(Y, a.g.ny), z = wrap_box(Z, a.g.nz);
  const long long n = (long long)x + (long long)a.g.nx * ((long long)y + (long long)a.g.ny * z);
  auto off = [](int v, int ip, float fr, int nn) {
    const float hn = 0.5f * (float)nn;
    float d = __fsub_rn((float)(v - ip), fr);
    if (d > hn) d = __fsub_rn(d, (float)nn);
    else if (d < -hn) d = __fadd_rn(d, (float)nn);
    return d;
  };
  const float fx = off(x, P.ipos[0], P.fpos[0], a.g.nx);
  const float fy = off(y, P.ipos[1], P.fpos[1], a.g.ny);
  const float fz = off(z, P.ipos[2], P.fpos[2], a.g.nz);
  const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)), __fmul_rn(fz, fz));
  const float dsurf = __fsub_rn(__fsqrt_rn(d2), (float)P.radius);
  unsigned bits = __float_as_uint(dsurf);
  bits = (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
  const unsigned long long key = ((unsigned long long)bits << 20) | (unsigned long long)p;
  const unsigned long long old = atomicMin(a.fkey + n, key);
  if (old != ~0ULL && (int)(old & 0xFFFFFull) != p) {
    const float dold = key_distance(old);
    if (dsurf - dold <= a.tie_thr && dold - dsurf <= a.tie_thr) {
      const int slot = atomicAdd(a.tie_count, 1);
      if (slot < a.tie_cap) a.tie_list[slot] = (int)n;
      else atomicOr(a.status, ST_CAPACITY);
    }
  }
}

__global__ void k_force_assign(PartArgs a) { force_assign_body(a, grid_blk()); }

// FP64 decision on the listed nodes: one warp per entry, its lanes over the
// particles whose widened box holds the node; the smallest (distance, index)
// wins and its index replaces the key's.  A node listed twice gets the same
// answer twice.
__device__ __forceinline__ void tie_resolve_body(const PartArgs& a, const Blk bk) {
  const int lane = threadIdx.x & 31;
  const int warp = (bk.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (bk.nx * blockDim.x) >> 5;
  const int count = min(*a.tie_count, a.tie_cap);
  const Grid g = a.g;
  for (int e = warp; e < count; e += nwarps) {
    const long long n = a.tie_list[e];
    const int x = (int)(n % g.nx), y = (int)((n / g.nx) % g.ny), z = (int)(n / ((long long)g.nx * g.ny));
    double best = INFINITY;
    int who = 0x7FFFFFFF;
    for (int q = lane; q < a.P; q += 32) {
      const DevParticle& P = a.parts[q];
      const int ex = P.ehi[0] - P.elo[0], ey = P.ehi[1] - P.elo[1], ez = P.ehi[2] - P.elo[2];
      const bool in = (ex >= g.nx || wrapi(x - P.elo[0], g.nx) < ex) &&
                      (ey >= g.ny || wrapi(y - P.elo[1], g.ny) < ey) &&
                      (ez >= g.nz || wrapi(z - P.elo[2], g.nz) < ez);
      if (!in) continue;
      const double s = surface_distance64(P, x, y, z, g);
      if (s < best) {  // q rises with the loop: an equal distance keeps the lower index
        best = s;
        who = q;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double sb = __shfl_xor_sync(0xFFFFFFFFu, best, o);
      const int wb = __shfl_xor_sync(0xFFFFFFFFu, who, o);
      if (sb < best || (sb == best && wb < who)) {
        best = sb;
        who = wb;
      }
    }
    if (lane == 0 && who != 0x7FFFFFFF) a.fkey[n] = (a.fkey[n] & ~0xFFFFFull) | (unsigned long long)who;
  }
}

__global__ void k_tie_resolve(PartArgs a) { tie_resolve_body(a, grid_blk()); }

// Sum of FORCE_T values per component, fixed order: the block's values are
// transposed through shared memory and each of 4 threads per component adds a
// strided quarter, then one thread adds the quarters.  Components of a group
// no thread touched are skipped (they stay 0).  Result in out[j] for
// threadIdx.x == j < NV.  Few FP64 instructions: a warp-shuffle tree would
// spend 5 * NV double adds per thread.
template <int NC>
__device__ void column_sums(const double* tab, int nrow, int stride, int col0, double* out);
__device__ void integrate_all(const PartArgs& a);

template <int NV, class Get>
__device__ void block_sum_t(Get v, const bool (&group_on)[NV / 6], double* out) {
  __shared__ double tr[NV][FORCE_T + 1];
  __shared__ double quarter[NV][4];
  const int t = threadIdx.x;
#pragma unroll
  for (int j = 0; j < NV; ++j)
    if (group_on[j / 6]) tr[j][t] = v(j);
  __syncthreads();
  if (t < 4 * NV) {
    const int j = t >> 2, w = t & 3;
    double s = 0.0;
    if (group_on[j / 6])
      for (int i = w; i < FORCE_T; i += 4) s += tr[j][i];
    quarter[j][w] = s;
  }
  __syncthreads();
  if (t < NV) out[t] = ((quarter[t][0] + quarter[t][1]) + quarter[t][2]) + quarter[t][3];
}

// Per fluid node x next to particle p, with d0 = x - r_p and
// w = V + Omega x d0: the boundary velocity of a link c_i (at x + c_i or its
// midpoint) has c_i . v_b = c_i . w, since c_i . (Omega x c_i) = 0, and the
// link torque (x + c_i - r_p) x F_i sums to d0 x sum_i F_i, since
// c_i x c_i = 0.  So the per-link work is one dot product and one add.
// The field on the particle's own charge is kept as sum q and sum q (r - r_p)
// (force E sum q, torque (sum q (r - r_p)) x E).
// Block (p, b) takes the rows b, b + nb, b + 2 nb, ... of FORCE_T cells of the
// widened box (nb blocks for this particle), so the cells next to the sphere
// are spread over all blocks.
template <class FM>
__device__ __forceinline__ void particle_forces_body(const PartArgs& a, const Blk bk) {
  const int p = bk.x;
  const DevParticle& P = a.parts[p];
  const Grid g = a.g;
  const long long N = g.N;
  const int ncell = box_cells(P.elo, P.ehi);
  const int nb = (ncell + a.fcells - 1) / a.fcells;
  if ((int)bk.y >= nb) return;  // whole CTA beyond this particle's widened box
  const bool pv = a.ph.pv != 0;
  // the charge per unit weight (FP64 form: every thread; FP32 form: one
  // thread of the block, in float to the others, as the GPU's FP64 pipe is
  // narrow)
  auto charge_norm = [&]() {
    if (pv)
      return (a.ph.flags & EK_CHARGE_NORM_VP)
                 ? P.charge / (4.0 / 3.0 * M_PI * P.radius * P.radius * P.radius)
                 : (psi_sum(P) > 0.0 ? P.charge / psi_sum(P) : 0.0);
    return P.nb > 0 ? P.charge / (double)P.nb : 0.0;
  };
  double qnorm = 0.0;
  float qnormf = 0.0f;
  bool qnz = false;  // qnorm != 0
  if (FM::fp32) {
    __shared__ float s_qn;
    __shared__ int s_qnz;
    if (threadIdx.x == 0) {
      const double q = charge_norm();
      s_qn = (float)q;
      s_qnz = q != 0.0;
    }
    __syncthreads();
    qnormf = s_qn;
    qnz = s_qnz != 0;
  } else {
    qnorm = charge_norm();
  }
  const double rho0 = a.ph.rho0;
  // the particle's velocities, rho0 and centre in float (FP32 form; the
  // particle record keeps float copies of the velocities and the centre's
  // integer part and fraction)
  const float vxf = P.velf[0], vyf = P.velf[1], vzf = P.velf[2];
  const float qxf = P.omegaf[0], qyf = P.omegaf[1], qzf = P.omegaf[2];
  const float rho0f = (float)rho0;
  double acc[FPART];
#pragma unroll
  for (int j = 0; j < FPART; ++j) acc[j] = 0.0;
  // FP32 form: the reaction sums run in float per thread (the ifield is float;
  // the GPU's FP64 rate is a small fraction of its FP32 rate), with offsets
  // from the centre split into an integer part and the centre's fraction
  float racc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  // FP32 form: momentum exchange [0..5] and own charge [6..9] in float
  float macc[10] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  const int cxi = P.ipos[0], cyi = P.ipos[1], czi = P.ipos[2];  // floor(pos)
  const float frx = P.fpos[0], fry = P.fpos[1], frz = P.fpos[2];  // pos - floor(pos), rounded
  bool touched[4] = {false, false, false, false};
  const int rows = a.fcells / FORCE_T;
  // FP32 form: a thread's cells are rows of FORCE_T apart in the widened
  // box's x-fastest order, nb rows per step, so their box-local coordinates
  // advance by a fixed step with carries (no division per cell); wrap_box
  // gives the node
  const int ebx = P.ehi[0] - P.elo[0], eby = P.ehi[1] - P.elo[1];
  const int rstep = nb * FORCE_T;
  const int sX = rstep % ebx, sY = (rstep / ebx) % eby, sZ = rstep / (ebx * eby);
  int lX = 0, lY = 0, lZ = 0;  // box-local coordinates of the next cell
  // cell c of the widened box (FP32 form: the cell at lX, lY, lZ):
  // coordinates, node, first copy of the node
  auto locate = [&](int c, int& X, int& Y, int& Z, long long& n, int (&w3)[3], double& mx, double& my,
                    double& mz) {
    if (FM::fp32) {
      X = P.elo[0] + lX;
      Y = P.elo[1] + lY;
      Z = P.elo[2] + lZ;
      w3[0] = wrap_box(X, g.nx);
      w3[1] = wrap_box(Y, g.ny);
      w3[2] = wrap_box(Z, g.nz);
      n = (long long)(w3[0] + g.nx * (w3[1] + g.ny * w3[2]));
      return lX < g.nx && lY < g.ny && lZ < g.nz;
    }
    return ext_cell(P, c, g, X, Y, Z, n, mx, my, mz, w3);
  };
  // the next row's cell is located and its owner and key loaded while this
  // one is processed (the loads of consecutive rows overlap)
  int nX, nY, nZ, nw3[3];
  long long nn = 0;
  double nmx = 0.0, nmy = 0.0, nmz = 0.0;
  bool nfirst = false;
  int nown = FLUID;
  unsigned long long nkey = ~0ULL;
  // FP32 form: the internal force of the next cell too (most cells of a
  // widened box are the particle's own), so no load waits on the key
  float nif[3] = {0.0f, 0.0f, 0.0f};
  const float* const ifl = (const float*)a.ifield;
  auto fetch = [&]() {
    nown = a.owner[nn];
    nkey = a.fkey[nn];
    if (FM::fp32) {
      nif[0] = ifl[nn];
      nif[1] = ifl[N + nn];
      nif[2] = ifl[2 * N + nn];
    }
  };
  int cnext = (int)bk.y * FORCE_T + threadIdx.x;
  bool nvalid = cnext < ncell;
  if (FM::fp32) {
    lX = cnext % ebx;
    lY = (cnext / ebx) % eby;
    lZ = cnext / (ebx * eby);
  }
  if (nvalid) {
    nfirst = locate(cnext, nX, nY, nZ, nn, nw3, nmx, nmy, nmz);
    fetch();
  }
  // Links into the sphere start at fluid nodes within R + sqrt(2) of the
  // centre (a covered node lies within R); the test below takes R + 1.5.  The
  // box offsets X - r_p it measures are the minimum-image ones for every
  // linked node once each edge is at least 2 R + 4 (a box cell lies within
  // R + 2 of the centre along each axis); smaller lattices test every cell.
  const int nmin = min(g.nx, min(g.ny, g.nz));
  bool gate;
  double rlink = 0.0;
  float rlink2f = 0.0f;
  if (FM::fp32) {
    // float suffices: the bounds leave margins of 0.5 and 0.086 lattice units
    const float Rf = sqrtf(P.r2f);
    gate = 2.0f * Rf + 4.0f <= (float)nmin;
    rlink2f = (Rf + 1.5f) * (Rf + 1.5f);
  } else {
    gate = 2.0 * P.radius + 4.0 <= (double)nmin;
    rlink = P.radius + 1.5;
  }
  for (int k = 0; k < rows; ++k) {
    if (!nvalid) break;
    const int X = nX, Y = nY, Z = nZ;
    const long long n = nn;
    const double mx = nmx, my = nmy, mz = nmz;
    const int w3[3] = {nw3[0], nw3[1], nw3[2]};
    const bool first = nfirst;
    const int own = nown;
    const unsigned long long key = nkey;
    const float ifx = nif[0], ify = nif[1], ifz = nif[2];
    cnext = ((int)bk.y + (k + 1) * nb) * FORCE_T + threadIdx.x;
    nvalid = k + 1 < rows && cnext < ncell;
    if (FM::fp32) {
      lX += sX;
      lY += sY;
      lZ += sZ;
      if (lX >= ebx) {
        lX -= ebx;
        ++lY;
      }
      if (lY >= eby) {
        lY -= eby;
        ++lZ;
      }
    }
    if (nvalid) {
      nfirst = locate(cnext, nX, nY, nZ, nn, nw3, nmx, nmy, nmz);
      fetch();
    }
    const bool in_box = X >= P.lo[0] && X < P.hi[0] && Y >= P.lo[1] && Y < P.hi[1] &&
                        Z >= P.lo[2] && Z < P.hi[2];
    bool near = own == FLUID && in_box;
    if (near && gate) {
      if (FM::fp32) {
        const float ex = __fsub_rn((float)(X - P.ipos[0]), P.fpos[0]);
        const float ey = __fsub_rn((float)(Y - P.ipos[1]), P.fpos[1]);
        const float ez = __fsub_rn((float)(Z - P.ipos[2]), P.fpos[2]);
        near = ex * ex + ey * ey + ez * ez < rlink2f;
      } else {
        const double ex = (double)X - P.pos[0], ey = (double)Y - P.pos[1], ez = (double)Z - P.pos[2];
        near = ex * ex + ey * ey + ez * ez < rlink * rlink;
      }
    }
    if (near) {
      // momentum exchange on every link from this fluid node into the particle
      // (Eq. 11): the links first (all 18 owner loads in flight together), the
      // FP64 arithmetic only at nodes next to the surface
      const Nbr b = make_nbr(w3[0], w3[1], w3[2], g);
      unsigned links = 0;
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const long long m = node_index(g, nb_x(b, w3[0], dcx(i)), nb_y(b, w3[1], dcy(i)),
                                       nb_z(b, w3[2], dcz(i)));
        if (a.owner[m] == p) links |= 1u << i;
      }
      if (links && FM::fp32) {
        // FP32 form, in float: the populations are stored as deviations
        // g = f - w rho0, so f*_i + f_ibar = 2 g_ibar + 2 w rho0 + 6 w rho0 c.w;
        // the deviation terms are small, and the rest-density term is summed
        // as an exact integer count of 36 w_i c_i
        const float d0x = __fsub_rn((float)(X - P.ipos[0]), P.fpos[0]);
        const float d0y = __fsub_rn((float)(Y - P.ipos[1]), P.fpos[1]);
        const float d0z = __fsub_rn((float)(Z - P.ipos[2]), P.fpos[2]);
        const float wx = vxf + (qyf * d0z - qzf * d0y);
        const float wy = vyf + (qzf * d0x - qxf * d0z);
        const float wz = vzf + (qxf * d0y - qyf * d0x);
        const float r0 = rho0f;
        float fx = 0.0f, fy = 0.0f, fz = 0.0f;
        int kx = 0, ky = 0, kz = 0;  // sum of 36 w_i c_i over the links
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          if (!(links & (1u << i))) continue;
          const float gdev = ((const float*)a.f)[(long long)opp(i) * N + n];
          float cw = 0.0f;
          if (dcx(i)) cw = dcx(i) > 0 ? cw + wx : cw - wx;
          if (dcy(i)) cw = dcy(i) > 0 ? cw + wy : cw - wy;
          if (dcz(i)) cw = dcz(i) > 0 ? cw + wz : cw - wz;
          const float mom = 2.0f * gdev + 6.0f * (float)wgt(i) * r0 * cw;
          const int k36 = i < 7 ? 2 : 1;
          if (dcx(i)) { fx = dcx(i) > 0 ? fx + mom : fx - mom; kx += dcx(i) * k36; }
          if (dcy(i)) { fy = dcy(i) > 0 ? fy + mom : fy - mom; ky += dcy(i) * k36; }
          if (dcz(i)) { fz = dcz(i) > 0 ? fz + mom : fz - mom; kz += dcz(i) * k36; }
        }
        const float cst = 2.0f * r0 / 36.0f;
        fx += cst * (float)kx;
        fy += cst * (float)ky;
        fz += cst * (float)kz;
        touched[0] = true;
        macc[0] += fx;
        macc[1] += fy;
        macc[2] += fz;
        macc[3] += d0y * fz - d0z * fy;
        macc[4] += d0z * fx - d0x * fz;
        macc[5] += d0x * fy - d0y * fx;
      } else if (links) {
        const double d0x = (double)X - P.pos[0], d0y = (double)Y - P.pos[1], d0z = (double)Z - P.pos[2];
        const double wx = P.vel[0] + (P.omega[1] * d0z - P.omega[2] * d0y);
        const double wy = P.vel[1] + (P.omega[2] * d0x - P.omega[0] * d0z);
        const double wz = P.vel[2] + (P.omega[0] * d0y - P.omega[1] * d0x);
        double fx = 0.0, fy = 0.0, fz = 0.0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          if (!(links & (1u << i))) continue;
          const double refl = pop_abs<FM>(a.f, opp(i), N, n, rho0);
          const double fs = refl + 6.0 * wgt(i) * rho0 * cdot(i, wx, wy, wz);  // the population that hit the wall
          const double mom = fs + refl;
          if (dcx(i)) fx = dcx(i) > 0 ? fx + mom : fx - mom;
          if (dcy(i)) fy = dcy(i) > 0 ? fy + mom : fy - mom;
          if (dcz(i)) fz = dcz(i) > 0 ? fz + mom : fz - mom;
        }
        touched[0] = true;
        acc[0] += fx;
        acc[1] += fy;
        acc[2] += fz;
        acc[3] += d0y * fz - d0z * fy;
        acc[4] += d0z * fx - d0x * fz;
        acc[5] += d0x * fy - d0y * fx;
      }
    }
    // reaction of the internal solute force on the fluid nodes this particle claims
    // the key of a node is cleared by the particle it names, right after
    // reading it: any other particle reading it meanwhile finds either that
    // key or an empty one, and neither names it
    bool mine = false;
    if (first && (int)(key & 0xFFFFFull) == p) {
      a.fkey[n] = ~0ULL;
      mine = true;
    }
    if (mine && own == FLUID) {
      touched[1] = true;
      if (FM::fp32) {
        const float ix = ifx, iy = ify, iz = ifz;
        // minimum-image offset of the wrapped node from the centre
        const float hx = 0.5f * (float)g.nx, hy = 0.5f * (float)g.ny, hz = 0.5f * (float)g.nz;
        float ox = (float)(w3[0] - cxi) - frx, oy = (float)(w3[1] - cyi) - fry, oz = (float)(w3[2] - czi) - frz;
        ox = ox > hx ? ox - (float)g.nx : (ox < -hx ? ox + (float)g.nx : ox);
        oy = oy > hy ? oy - (float)g.ny : (oy < -hy ? oy + (float)g.ny : oy);
        oz = oz > hz ? oz - (float)g.nz : (oz < -hz ? oz + (float)g.nz : oz);
        racc[0] -= ix;
        racc[1] -= iy;
        racc[2] -= iz;
        racc[3] -= oy * iz - oz * iy;
        racc[4] -= oz * ix - ox * iz;
        racc[5] -= ox * iy - oy * ix;
      } else {
        const double ix = real_at<FM>(a.ifield, n);
        const double iy = real_at<FM>(a.ifield, N + n);
        const double iz = real_at<FM>(a.ifield, 2 * N + n);
        acc[6] -= ix;
        acc[7] -= iy;
        acc[8] -= iz;
        acc[9] -= my * iz - mz * iy;
        acc[10] -= mz * ix - mx * iz;
        acc[11] -= mx * iy - my * ix;
      }
    }
    // the particle's own charge in this cell
    if (in_box) {
      double qq = 0.0;
      float psf = 0.0f;
      bool has_q = false;
      if (pv) {
        const int bx = P.hi[0] - P.lo[0], by = P.hi[1] - P.lo[1];
        const int cb = (X - P.lo[0]) + bx * ((Y - P.lo[1]) + by * (Z - P.lo[2]));
        const double ps = a.psibox[(long long)p * a.boxmax + cb];
        if (FM::fp32) {
          // the weight itself is applied in float below
          psf = psibox_float((unsigned long long)__double_as_longlong(ps));
          has_q = psf != 0.0f;
        } else {
          qq = qnorm * ps;
          has_q = qq != 0.0;
        }
      } else if (own == p) {
        qq = qnorm;
        psf = 1.0f;
        has_q = FM::fp32 ? qnz : qq != 0.0;
      }
      if (has_q) {
        touched[2] = true;
        if (FM::fp32) {
          const float qf = qnormf * psf;
          macc[6] += qf;
          macc[7] += qf * __fsub_rn((float)(X - P.ipos[0]), P.fpos[0]);
          macc[8] += qf * __fsub_rn((float)(Y - P.ipos[1]), P.fpos[1]);
          macc[9] += qf * __fsub_rn((float)(Z - P.ipos[2]), P.fpos[2]);
        } else {
          acc[12] += qq;
          acc[13] += qq * ((double)X - P.pos[0]);
          acc[14] += qq * ((double)Y - P.pos[1]);
          acc[15] += qq * ((double)Z - P.pos[2]);
        }
      }
    }
  }
  float facc[FPART];
  if (FM::fp32) {
#pragma unroll
    for (int j = 0; j < FPART; ++j) facc[j] = 0.0f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      facc[j] = macc[j];
      facc[6 + j] = racc[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) facc[12 + j] = macc[6 + j];
  }
  // a slice of the lattice-block sums of the internal force (S2), carried by
  // the first particle's blocks, so that the lattice total is ready when the
  // per-particle rows are summed
  if (p == 0) {
    const int per = (a.nipart + nb - 1) / nb;
    const int r0 = (int)bk.y * per, r1 = min(r0 + per, a.nipart);
    double lat = 0.0;  // component threadIdx.x % 3 (the stride 126 keeps it)
    for (int q = threadIdx.x; q < 3 * (r1 - r0) && threadIdx.x < 126; q += 126) {
      lat += __ldcg(a.ipart + 3LL * r0 + q);
      touched[3] = true;
    }
    const int j = threadIdx.x % 3;
    if (j == 0) acc[18] = lat;
    else if (j == 1) acc[19] = lat;
    else acc[20] = lat;
  }
  bool on[4];
  on[0] = __syncthreads_or(touched[0]);
  on[1] = __syncthreads_or(touched[1]);
  on[2] = __syncthreads_or(touched[2]);
  on[3] = __syncthreads_or(touched[3]);
  double* out = a.fpart + ((long long)p * a.fchunks + bk.y) * FPART;
  if (FM::fp32) {
    // each thread's float sums over its own few cells, widened to FP64 (the
    // lattice slice is FP64 already); everything above them in FP64
    block_sum_t<FPART>([&](int j) { return (j >= 18 && j < 21) ? acc[j] : (double)facc[j]; }, on, out);
  } else {
    block_sum_t<FPART>([&](int j) { return acc[j]; }, on, out);
  }
  // the particle's last block sums its rows; the last particle integrates
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(a.pticket + p, 1) == nb - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  column_sums<FPART>(a.fpart + (long long)p * a.fchunks * FPART, nb, FPART, 0,
                     a.psum + (long long)p * FPART);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    a.pticket[p] = 0;
    last = atomicAdd(a.ticket, 1) == a.P - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  integrate_all(a);
  if (threadIdx.x == 0) {
    *a.ticket = 0;
    *a.tie_count = 0;  // the next step's assignment lists its ties afresh
  }
}

template <class FM>
__global__ void __launch_bounds__(FORCE_T, FM::fp32 ? 5 : 4) k_particle_forces(PartArgs a) {
  particle_forces_body<FM>(a, grid_blk());
}

// New box of a particle at `pos`: the cells within R (+1 below, +2 above),
// the union with the previous box (moved into the periodic image of the new
// one, as the position wraps when the particle crosses the boundary), and the
// box widened by ceil(R) + FORCE_MARGIN for the solute-force assignment.
// Axis d alone (the integration runs one thread per axis).
__device__ void box_update_axis(DevParticle& P, int d, double pos, int nn, bool setup) {
  const int lo = (int)floor(pos - P.radius) - 1;
  const int hi = (int)floor(pos + P.radius) + 2;
  int olo = P.lo[d], ohi = P.hi[d];
  // shift = rint((lo - olo) / nn) nn, in integers (ties to even): the
  // quotient of two integers with nn <= 1024 lies at least 1 / 2048 from any
  // half-integer it is not, so rounding it first would change nothing
  const int k = lo - olo;
  int q = k >= 0 ? k / nn : -((nn - 1 - k) / nn);  // floor(k / nn)
  const int r = k - q * nn;                         // in [0, nn)
  if (2 * r > nn || (2 * r == nn && (q & 1))) ++q;
  const int shift = q * nn;
  olo += shift;
  ohi += shift;
  P.ulo[d] = setup ? lo : min(lo, olo);
  P.uhi[d] = setup ? hi : max(hi, ohi);
  P.lo[d] = lo;
  P.hi[d] = hi;
  const int m = (int)ceil(P.radius) + FORCE_MARGIN;
  P.elo[d] = lo - m;
  P.ehi[d] = hi + m;
  P.ipos[d] = (int)floor(pos);
  const double frac = pos - (double)P.ipos[d];  // exact
  P.fpos[d] = (float)frac;
  P.fposlo[d] = (float)(frac - (double)P.fpos[d]);
}

// the radius in the forms the inside tests use
__device__ void radius_forms(DevParticle& P) {
  const double R2 = __dmul_rn(P.radius, P.radius);
  P.r2f = (float)R2;
  P.r2lo = (float)(R2 - (double)P.r2f);
  P.psimargin = psi_margin(R2);
}

__device__ void box_update_one(DevParticle& P, const double pos[3], const int nn[3], bool setup) {
  for (int d = 0; d < 3; ++d) {
    box_update_axis(P, d, pos[d], nn[d], setup);
    P.velf[d] = (float)P.vel[d];
    P.omegaf[d] = (float)P.omega[d];
  }
  radius_forms(P);
}

// Column sums of a row-major table (nrow rows of `stride` doubles; columns
// col0 .. col0 + NC - 1) by a block of FORCE_T threads, fixed order: thread
// t < G * NC takes column t % NC of rows t / NC, t / NC + G, ... (eight loads
// in flight at a time), then thread j < NC adds the partials of the groups
// that hold rows (min(G, nrow); the others would add zeros) in order.
// Result in out[j] (shared or global) for threadIdx.x == j.
template <int NC>
__device__ void column_sums(const double* tab, int nrow, int stride, int col0, double* out) {
  constexpr int G = FORCE_T / NC;
  __shared__ double part[G * NC];
  const int t = threadIdx.x;
  if (t < G * NC) {
    const int j = t % NC;
    double s = 0.0;
    int r = t / NC;
    for (; r + 7 * G < nrow; r += 8 * G) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcg(tab + (long long)(r + u * G) * stride + col0 + j);
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; r < nrow; r += G) s += __ldcg(tab + (long long)r * stride + col0 + j);
    part[t] = s;
  }
  __syncthreads();
  if (t < NC) {
    const int gu = min(G, nrow);
    double s = 0.0;
    for (int r = 0; r < gu; ++r) s += part[r * NC + t];
    out[t] = s;
  }
  __syncthreads();
}

// Run by the block that finishes S4 last: the remainder of the solute force
// on nodes no particle claims (lattice total of the internal force minus the
// claimed sums) is split evenly; every particle then moves by symplectic
// Euler (Sec. III.B), and its boxes follow the new position (start of S5).
// Up to FORCE_T / 4 particles take four lanes each, lane d < 3 doing axis d,
// so that the FP64 divisions of the three axes (by the mass, the moment of
// inertia, the box edge) run side by side instead of one after another in
// one thread; more particles take one thread each (all three axes).
__device__ void integrate_all(const PartArgs& a) {
  __shared__ double claimed[3], total[3], rem[3];
  __shared__ unsigned char fin[3 * FORCE_T];
  column_sums<3>(a.psum, a.P, FPART, 18, total);
  column_sums<3>(a.psum, a.P, FPART, 6, claimed);
  if (threadIdx.x < 3)
    rem[threadIdx.x] = (total[threadIdx.x] + claimed[threadIdx.x]) / (double)a.P;  // claimed holds -sum i
  __syncthreads();
  const bool quad = a.P <= FORCE_T / 4;
  const int per_pass = quad ? FORCE_T / 4 : FORCE_T;
  const int pl = quad ? (int)threadIdx.x >> 2 : (int)threadIdx.x;
  const int d0 = quad ? (int)(threadIdx.x & 3) : 0, dstep = quad ? 3 : 1;
  const double* E = a.ph.E;
  for (int base = 0; base < a.P; base += per_pass) {
    const int p = base + pl;
    const bool on = p < a.P;
    double posd[3] = {0.0, 0.0, 0.0};
    if (on) {
      DevParticle* Pp = a.parts + p;
      const double* acc = a.psum + (long long)p * FPART;
      for (int d = d0; d < 3; d += dstep) {
        const int d1 = d == 2 ? 0 : d + 1, d2 = d == 0 ? 2 : d - 1;  // (d, d1, d2) cyclic
        const int nn = d == 0 ? a.g.nx : (d == 1 ? a.g.ny : a.g.nz);
        // field on the own charge: E sum q, (sum q (r - r_p)) x E
        const double Tq = __ldcg(acc + 13 + d1) * E[d2] - __ldcg(acc + 13 + d2) * E[d1];
        const double F = __ldcg(acc + d) + __ldcg(acc + 6 + d) + __ldcg(acc + 12) * E[d] - rem[d] +
                         Pp->ftrans[d];
        const double T = __ldcg(acc + 3 + d) + __ldcg(acc + 9 + d) + Tq;
        double pos = Pp->pos[d], vel = Pp->vel[d], omega = Pp->omega[d];
        if (!Pp->fixed) {
          vel = vel + F / Pp->mass;
          omega = omega + T / Pp->inertia;
          pos = pos + vel;
          // into [0, n): one period at any sane speed; a step longer than a
          // period is wrapped all the same, so that every box stays within one
          // period of the lattice (the cell kernels rely on it)
          if (pos >= (double)nn || pos < 0.0) {
            pos -= floor(pos / (double)nn) * (double)nn;
            if (pos < 0.0) pos += (double)nn;  // the quotient rounded up
            if (pos >= (double)nn) pos -= (double)nn;
          }
          if (!isfinite(pos)) atomicOr(a.status, ST_NONFINITE);
        }
        Pp->force[d] = F;
        Pp->torque[d] = T;
        Pp->ftrans[d] = 0.0;
        Pp->pos[d] = pos;
        Pp->vel[d] = vel;
        Pp->omega[d] = omega;
        Pp->velf[d] = (float)vel;
        Pp->omegaf[d] = (float)omega;
        // S5 starts here: the boxes follow the new position
        fin[3 * pl + d] = isfinite(pos) ? 1 : 0;
        if (d == 0) posd[0] = pos;
        else if (d == 1) posd[1] = pos;
        else posd[2] = pos;
      }
    }
    __syncthreads();
    if (on && d0 < 3 && fin[3 * pl] && fin[3 * pl + 1] && fin[3 * pl + 2]) {
      DevParticle& P = a.parts[p];
      for (int d = d0; d < 3; d += dstep)
        box_update_axis(P, d, d == 0 ? posd[0] : (d == 1 ? posd[1] : posd[2]),
                        d == 0 ? a.g.nx : (d == 1 ? a.g.ny : a.g.nz), false);
      if (d0 == 0) radius_forms(P);
    }
    __syncthreads();
  }
}

// set-up only (in a step the box follows the position in integrate_all)
__global__ void k_box_update(PartArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  DevParticle& P = a.parts[p];
  const int nn[3] = {a.g.nx, a.g.ny, a.g.nz};
  const double pos[3] = {P.pos[0], P.pos[1], P.pos[2]};
  box_update_one(P, pos, nn, true);
  for (int j = 0; j < 8; ++j) P.psiunits[j] = 0;
  P.nb = 0;
}

__device__ __forceinline__ void save_prev_body(const PartArgs& a, const Blk bk) {
  DevParticle& P = a.parts[bk.x];
  if (bk.y == 0 && threadIdx.x == 0) {  // k_claim and k_psi_surface sum these afresh
    for (int j = 0; j < 8; ++j) P.psiunits[j] = 0;
    P.nb = 0;
    // the transfer list of the last step's transitions has been applied;
    // this step's transitions append to an empty one (a kernel of the chain
    // instead of a memset node after the transfers)
    if (bk.x == 0) *a.xfer_count = 0;
  }
  const int c = bk.y * blockDim.x + threadIdx.x;
  if (c >= box_cells(P.ulo, P.uhi)) return;
  int X, Y, Z;
  box_coord(c, P.ulo, P.uhi, X, Y, Z);
  const long long n = node_of(X, Y, Z, a.g);
  a.owner_prev[n] = a.owner[n];
}

__global__ void k_save_prev(PartArgs a) { save_prev_body(a, grid_blk()); }

template <class FM>
__device__ __forceinline__ void clear_body(const PartArgs& a, const Blk bk) {
  const DevParticle& P = a.parts[bk.x];
  // the surface-cell list of the last step has been read; k_claim refills it
  if (bk.x == 0 && bk.y == 0 && threadIdx.x == 0) *a.surf_count = 0;
  const int c = bk.y * blockDim.x + threadIdx.x;
  if (c >= box_cells(P.ulo, P.uhi)) return;
  int X, Y, Z;
  box_coord(c, P.ulo, P.uhi, X, Y, Z);
  const long long n = node_of(X, Y, Z, a.g);
  if (a.owner[n] >= 0) a.owner[n] = FLUID;
  real_set<FM>(a.psi, n, 0.0);
  real_set<FM>(a.qpart, n, 0.0);
}

template <class FM>
__global__ void k_clear(PartArgs a) { clear_body<FM>(a, grid_blk()); }

template <class FM>
__global__ void k_reset_all(PartArgs a) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.g.N) return;
  a.owner[n] = (a.wall && a.wall[n]) ? WALL : FLUID;
  real_set<FM>(a.psi, n, 0.0);
  real_set<FM>(a.qpart, n, 0.0);
}

// boundary nodes (cell centre strictly inside) and the level-0 octree test of
// every cell of the current box; cells cut by the surface are queued for
// k_psi_surface
template <class FM>
__device__ __forceinline__ void claim_body(const PartArgs& a, const Blk bk) {
  const int p = bk.x;
  DevParticle& P = a.parts[p];
  const int c = bk.y * blockDim.x + threadIdx.x;
  const int ncell = box_cells(P.lo, P.hi);
  double ps = 0.0;
  int inside = 0;
  if (c < ncell) {
    int X, Y, Z;
    box_coord(c, P.lo, P.hi, X, Y, Z);
    const long long n = node_of(X, Y, Z, a.g);
    const double R2 = __dmul_rn(P.radius, P.radius);
    if (node_inside_tiers(X, Y, Z, P)) {
      inside = 1;
      const int old = atomicCAS(a.owner + n, FLUID, p);
      if (old != FLUID) atomicOr(a.status, ST_OVERLAP);
    }
    const int s0 = classify_tiers((float)(X - P.ipos[0]), (float)(Y - P.ipos[1]),
                                  (float)(Z - P.ipos[2]), 0, 0, X, Y, Z, P);
    if (s0 == CUBE_IN) {
      ps = 1.0;
      real_add<FM>(a.psi, n, 1.0);
    } else if (s0 == CUBE_UNDECIDED) {
      const int slot = atomicAdd(a.surf_count, 1);
      if (slot < a.surf_cap) a.surf[slot] = make_int2(p, c);
      else atomicOr(a.status, ST_CAPACITY);
    }
    a.psibox[(long long)p * a.boxmax + c] = ps;
  }
  // level 0 decides whole cells: Psi_p is 0 or 1 here, so both sums are counts
  const int nin = __syncthreads_count(ps != 0.0);
  const int nbd = __syncthreads_count(inside);
  if (threadIdx.x == 0) {
    if (nin) atomicAdd(&P.psiunits[0], (unsigned long long)nin * PSI_UNITS);
    if (nbd) atomicAdd(&P.nb, nbd);
  }
}

template <class FM>
__global__ void __launch_bounds__(PT) k_claim(PartArgs a) { claim_body<FM>(a, grid_blk()); }

// Psi_p of a surface cell (level 0 undecided) from the finest level alone.
// In FP64 the octree's decisions are inherited: a cube decided inside at some
// level has every level-4 sub-cube inside too, since a sub-cube's farthest
// corner is no farther from the centre, axis by axis, than its parent's, and
// rounding to nearest is monotone, so the rounded squared distance is no
// larger; likewise a cube decided outside has every sub-cube outside (its
// closest point is no closer).  Hence Psi_p = (2 N_in + N_und) / 8192 over the
// 4096 level-4 cubes, N_in of them with the farthest corner strictly inside,
// N_und the rest of those with the closest point nearer than R; that is
// (N_in + N_near) / 8192 with N_near = N_in + N_und, bit for bit the
// hierarchical result.
//
// One warp per cell, the 256 columns of 16 level-4 cubes along the axis u in
// which the cell lies farthest from the centre spread over the lanes.  When the
// centre lies beyond the cell's extent along u the distance of a column's
// planes grows from the near end, so the planes whose far corner is inside
// form a prefix (T planes: T - 1 inside cubes) and so do the cubes whose near
// face is nearer than R (T_N cubes).  T and T_N are estimated from a float
// square root, then settled by testing the planes at the boundary, each in
// float, with the exact FP64 test of the octree where the float distance lies
// within the margin of R^2 (see classify_f32).  A centre within the cell's u
// extent (cells of spheres below R = 2) takes every plane's test.
constexpr int PSI_CTA = 256;  // threads per CTA of k_psi_surface

struct PsiCell {
  const DevParticle* P;
  int X[3];     // the cell (unwrapped coordinates)
  float fb[3];  // X - integer part of the centre (exact in float)
  float R2f, margin;
  double R2;
  int u, v, w;  // column axis and the two across it
};

// offset of plane m (0..16) of the cell along axis a from the centre, the FP64
// value of the octree's test: the plane's exact coordinate minus the centre,
// rounded (the float estimate in the kernel is one rounding of the exact float
// difference of the plane and the centre's float fraction)
__device__ __forceinline__ double plane_off_d(const PsiCell& c, int a, int m) {
  return __dsub_rn((double)c.X[a] + (0.0625 * (double)m - 0.5), c.P->pos[a]);
}
// far (largest magnitude) or near (0 when the centre lies within) offset of
// slab j (planes j, j + 1) along axis a
__device__ __forceinline__ float slab_f(float a0, float a1, bool far) {
  if (far) return fmaxf(fabsf(a0), fabsf(a1));
  return (a0 <= 0.0f && a1 >= 0.0f) ? 0.0f : fminf(fabsf(a0), fabsf(a1));
}
__device__ __forceinline__ double slab_d(double a0, double a1, bool far) {
  if (far) return fmax(fabs(a0), fabs(a1));
  return (a0 <= 0.0 && a1 >= 0.0) ? 0.0 : fmin(fabs(a0), fabs(a1));
}

// the FP64 test of the octree for the point whose u offset is the plane mu
// (or, with mu1 >= 0, the near face of the slab mu..mu1) and whose v and w
// offsets are the far or near ones of slabs j and l: squared distance summed
// x, y, z left to right, against R^2.  A real call: inlined, its FP64
// instructions would be issued (predicated off) on every float test.
__device__ __noinline__ bool psi_exact(const PsiCell* c, int mu, int mu1, int j, int l, bool far) {
  double o[3];
  const double a0 = plane_off_d(*c, c->u, mu);
  o[c->u] = mu1 >= 0 ? slab_d(a0, plane_off_d(*c, c->u, mu1), far) : fabs(a0);
  o[c->v] = slab_d(plane_off_d(*c, c->v, j), plane_off_d(*c, c->v, j + 1), far);
  o[c->w] = slab_d(plane_off_d(*c, c->w, l), plane_off_d(*c, c->w, l + 1), far);
  return dist2(o[0], o[1], o[2]) < c->R2;
}

// float test with the FP64 one where the float squared distance is within the
// margin of R^2
__device__ __forceinline__ bool psi_test(const PsiCell& c, float gu, float gvw2, int mu, int mu1,
                                         int j, int l, bool far) {
  const float d = gu * gu + gvw2;
  if (d < c.R2f - c.margin) return true;
  if (d > c.R2f + c.margin) return false;
  return psi_exact(&c, mu, mu1, j, l, far);
}

// count of the planes t >= 0 (offset e0 + t/16 from the near end, at most
// tmax) with (e0 + t/16)^2 + S < R^2: ceil(v), v = 16 (sqrt(R^2 - S) - e0),
// decided (sure) when v lies farther than its error bound from an integer;
// a column beyond R^2 by more than twice the margin has none (every float
// test of its planes exceeds R^2 plus the margin: its sum is at least S);
// within twice the margin of R^2 it is left to the plane tests
__device__ __forceinline__ int psi_count(float S, float R2f, float margin, float e0, int tmax, bool& sure) {
  const float A = R2f - S;
  const float ra = rsqrtf(A);
  const float sa = A * ra;  // the root within a few ulp
  const float v = (sa - e0) * 16.0f;
  // |A - exact| < margin: the root off by < margin / sqrt(A) (ra within 1%);
  // the approximate root, e0 and v off by less than 2^-21 (sqrt(A) + e0 + 1)
  // together
  const float err = 32.0f * (1.01f * margin * ra + 4.8e-7f * (sa + e0 + 1.0f));
  const bool out = A < -2.0f * margin;
  sure = out || (A > 2.0f * margin && fabsf(v - rintf(v)) > err);
  return out ? 0 : min(max((int)ceilf(v), 0), tmax);
}

// the same count where psi_count is not sure: from the estimate, the planes
// at the boundary are tested (float, with the FP64 test of the octree within
// the margin of R^2) until the first plane outside
__device__ __noinline__ int psi_settle(const PsiCell* c, float S, float e0, int tmax, int near, int step,
                                       float bu, float fu, int j, int l, bool far) {
  const float A = c->R2f - S;
  int T;
  if (A <= 2.0f * c->margin) {
    T = A > 0.0f ? min(max((int)ceilf((sqrtf(A) - e0) * 16.0f), 0), tmax) : 0;
  } else {
    const float ra = rsqrtf(A);
    T = min(max((int)ceilf((A * ra - e0) * 16.0f), 0), tmax);
  }
  auto off = [](float b, float f, int m) { return __fsub_rn(b + (0.0625f * (float)m - 0.5f), f); };
  auto pin = [&](int t) {
    const int m = near + step * t;
    return psi_test(*c, fabsf(off(bu, fu, m)), S, m, -1, j, l, far);
  };
  while (T > 0 && !pin(T - 1)) --T;
  while (T < tmax && pin(T)) ++T;
  return T;
}

template <class FM>
__device__ __forceinline__ void psi_surface_body(const PartArgs& a, const Blk bk) {
  // per warp: the squared far and near offsets of the 16 slabs along w
  __shared__ float wslab[PSI_CTA / 32][2][16];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int warp = (bk.x * PSI_CTA + threadIdx.x) >> 5;
  const int nwarps = (bk.nx * PSI_CTA) >> 5;
  const int count = min(*a.surf_count, a.surf_cap);
  for (int e = warp; e < count; e += nwarps) {
    const int2 pc = a.surf[e];
    const DevParticle& P = a.parts[pc.x];
    int X[3];
    box_coord(pc.y, P.lo, P.hi, X[0], X[1], X[2]);
    float fb[3];
    for (int d = 0; d < 3; ++d) fb[d] = (float)(X[d] - P.ipos[d]);
    const float R2f = P.r2f, margin = P.psimargin;
    // the column axis: the largest distance of the cell centre from the centre
    float best = -1.0f;
    int u = 0;
    for (int d = 0; d < 3; ++d) {
      const float o = fabsf(__fsub_rn(fb[d], P.fpos[d]));
      if (o > best) {
        best = o;
        u = d;
      }
    }
    const int v = u == 0 ? 1 : 0;
    const int w = u == 2 ? 1 : 2;
    // near end of the columns: the plane nearest the centre, when the centre
    // lies beyond the cell along u.  Exact without FP64: the centre is
    // ipos + frac with frac = fpos + fposlo (the residual's sign exact), so
    // pos <= X - 1/2 iff m = X - ipos >= 2, or m = 1 and frac <= 1/2, and
    // pos >= X + 1/2 iff m <= -1, or m = 0 and frac >= 1/2
    const int mu_ = X[u] - P.ipos[u];
    const float fh = P.fpos[u], fl = P.fposlo[u];
    const bool le_half = fh < 0.5f || (fh == 0.5f && fl <= 0.0f);
    const bool ge_half = fh > 0.5f || (fh == 0.5f && fl >= 0.0f);
    const int near = (mu_ >= 2 || (mu_ == 1 && le_half)) ? 0
                     : ((mu_ <= -1 || (mu_ == 0 && ge_half)) ? 16 : -1);
    const int step = near == 0 ? 1 : -1;
    // per-axis constants of the float offsets (registers, not indexed)
    const float bu = fb[u], bv = fb[v], bw = fb[w];
    const float fu = P.fpos[u], fv_ = P.fpos[v], fw_ = P.fpos[w];
    auto off = [](float b, float f, int m) { return __fsub_rn(b + (0.0625f * (float)m - 0.5f), f); };
    // the squared far and near offsets across the columns are separable: a
    // lane's columns share one v slab (j = lane mod 16) and take their w slabs
    // (l) from the warp's table
    const int jl = lane & 15;
    float FV2, NV2;
    {
      const float v0 = off(bv, fv_, jl), v1 = off(bv, fv_, jl + 1);
      const float w0 = off(bw, fw_, jl), w1 = off(bw, fw_, jl + 1);
      const float fv = slab_f(v0, v1, true), nv = slab_f(v0, v1, false);
      const float fw = slab_f(w0, w1, true), nw = slab_f(w0, w1, false);
      FV2 = fv * fv;
      NV2 = nv * nv;
      if (lane < 16) {
        wslab[wib][0][jl] = fw * fw;
        wslab[wib][1][jl] = nw * nw;
      }
    }
    __syncwarp();
    // the cell in the form the plane tests take (built where they run)
    auto cell = [&]() {
      PsiCell c;
      c.P = &P;
      for (int d = 0; d < 3; ++d) {
        c.X[d] = X[d];
        c.fb[d] = fb[d];
      }
      c.R2f = R2f;
      c.margin = margin;
      c.R2 = __dmul_rn(P.radius, P.radius);
      c.u = u;
      c.v = v;
      c.w = w;
      return c;
    };
    int units = 0;
    const float e0 = near >= 0 ? fabsf(off(bu, fu, near)) : 0.0f;
    if (near >= 0) {
      // T: planes t = 0..16 from the near end whose far corner is inside
      // (T - 1 inside cubes); TN: cubes t = 0..15 whose near face is nearer
      // than R.  Counts the float estimate cannot decide are marked and
      // settled after the loop.
      unsigned unsure = 0u;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int l = (lane >> 4) + 2 * q;
        const float far2 = FV2 + wslab[wib][0][l];
        const float near2 = NV2 + wslab[wib][1][l];
        bool s1, s2;
        const int T = psi_count(far2, R2f, margin, e0, 17, s1);
        const int TN = psi_count(near2, R2f, margin, e0, 16, s2);
        units += (s1 ? max(T - 1, 0) : 0) + (s2 ? TN : 0);
        unsure |= (s1 ? 0u : 1u << (2 * q)) | (s2 ? 0u : 2u << (2 * q));
      }
      if (unsure) {
        const PsiCell c = cell();
        do {
          const int b = __ffs(unsure) - 1;
          unsure &= unsure - 1u;
          const int q = b >> 1, l = (lane >> 4) + 2 * q;
          if (b & 1) {
            const float near2 = NV2 + wslab[wib][1][l];
            units += psi_settle(&c, near2, e0, 16, near, step, bu, fu, jl, l, false);
          } else {
            const float far2 = FV2 + wslab[wib][0][l];
            units += max(psi_settle(&c, far2, e0, 17, near, step, bu, fu, jl, l, true) - 1, 0);
          }
        } while (unsure);
      }
    } else {
      // the centre within the cell's extent along u: every cube
      const PsiCell c = cell();
#pragma unroll 1
      for (int q = 0; q < 8; ++q) {
        const int j = jl, l = (lane >> 4) + 2 * q;
        const float far2 = FV2 + wslab[wib][0][l];
        const float near2 = NV2 + wslab[wib][1][l];
        bool prev = psi_test(c, fabsf(off(bu, fu, 0)), far2, 0, -1, j, l, true);
        for (int k = 0; k < 16; ++k) {
          const float a0 = off(bu, fu, k), a1 = off(bu, fu, k + 1);
          const bool in1 = psi_test(c, fabsf(a1), far2, k + 1, -1, j, l, true);
          if (prev && in1) units += 1;
          prev = in1;
          if (psi_test(c, slab_f(a0, a1, false), near2, k, k + 1, j, l, false)) units += 1;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) units += __shfl_xor_sync(0xffffffffu, units, o);
    if (lane == 0 && units > 0) {
      // dyadic with 13 fraction bits: every sum below is exact, in any order
      const long long n = node_of(X[0], X[1], X[2], a.g);
      a.psibox[(long long)pc.x * a.boxmax + pc.y] = dyadic13((unsigned)units);
      if (FM::fp32) atomicAdd((float*)a.psi + n, (float)units * (1.0f / (float)PSI_UNITS));
      else atomicAdd((double*)a.psi + n, dyadic13((unsigned)units));
      // integer counts, spread over eight addresses (the total of one
      // particle would otherwise serialise the atomics of all its cells)
      atomicAdd(&a.parts[pc.x].psiunits[pc.y & 7], (unsigned long long)units);
    }
    __syncwarp();  // the table is rewritten for the warp's next cell
  }
}

template <class FM>
__global__ void __launch_bounds__(PSI_CTA) k_psi_surface(PartArgs a) {
  psi_surface_body<FM>(a, grid_blk());
}

// Psi-smeared particle charge (Eq. 21), or spread over the boundary nodes
template <class FM>
__device__ __forceinline__ void charge_scatter_body(const PartArgs& a, const Blk bk) {
  const int p = bk.x;
  const DevParticle& P = a.parts[p];
  const int c = bk.y * blockDim.x + threadIdx.x;
  if (c >= box_cells(P.lo, P.hi)) return;
  int X, Y, Z;
  box_coord(c, P.lo, P.hi, X, Y, Z);
  const long long n = node_of(X, Y, Z, a.g);
  // all Psi_p have been added (k_claim): clamp the sum to 1 once, so readers
  // of psi need no min (idempotent where boxes overlap)
  if (real_at<FM>(a.psi, n) > 1.0) real_set<FM>(a.psi, n, 1.0);
  double q = 0.0;
  if (a.ph.pv) {
    const double ps = a.psibox[(long long)p * a.boxmax + c];
    if (ps == 0.0) return;
    if (a.ph.flags & EK_CHARGE_NORM_VP)
      q = P.charge * ps / (4.0 / 3.0 * M_PI * P.radius * P.radius * P.radius);
    else
      q = P.charge * ps / psi_sum(P);
  } else {
    if (a.owner[n] != p || P.nb == 0) return;
    q = P.charge / (double)P.nb;
  }
  real_add<FM>(a.qpart, n, q);
}

template <class FM>
__global__ void k_charge_scatter(PartArgs a) { charge_scatter_body<FM>(a, grid_blk()); }

__device__ __forceinline__ bool steady_fluid(const PartArgs& a, long long m) {
  return a.owner_prev[m] == FLUID && a.owner[m] == FLUID;
}

// Newly covered / uncovered nodes of particle p (Sec. III.B, III.D.1).  Solute
// transfers are computed from the values before the transitions and recorded;
// k_apply_transfers adds them afterwards.  FP32 form: species are integers and
// every split is an integer split (the remainder of an expulsion goes one
// unit each to the first receivers in direction order), so the totals stay
// exact.
template <class FM>
__device__ __forceinline__ void transitions_body(const PartArgs& a, const Blk bk) {
  using pop_t = typename FM::pop_t;
  using spc_t = typename FM::spc_t;
  constexpr unsigned FULL = 0xffffffffu;
  const int p = bk.x;
  DevParticle& P = a.parts[p];
  const int c = bk.y * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const Grid g = a.g;
  const long long N = g.N;
  const double rho0 = a.ph.rho0;
  const int K = a.ph.K;
  pop_t* f = (pop_t*)a.f;
  const spc_t* rho = (const spc_t*)a.rho;
  int X = 0, Y = 0, Z = 0;
  bool covered = false, uncovered = false;
  if (c < box_cells(P.ulo, P.uhi)) {
    box_coord(c, P.ulo, P.uhi, X, Y, Z);
    const long long n = node_of(X, Y, Z, g);
    const int old = a.owner_prev[n], nw = a.owner[n];
    covered = old == FLUID && nw == p;
    uncovered = old == p && nw == FLUID;
  }
  // momentum the particle receives from this thread's node: that of the
  // destroyed fluid, or minus that of the created fluid
  double mom[3] = {0.0, 0.0, 0.0};
  // The warp takes its transition nodes one after another, all 32 lanes on
  // each: lane k (1 <= k < Q) looks at the neighbour in direction k, lane
  // i < Q at population i, so the loads of a node are issued together.  Sums
  // over lanes go through a fixed shuffle tree.
  auto warp_sum = [&](double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
  };
  unsigned todo = __ballot_sync(FULL, covered || uncovered);
  while (todo) {
    const int src = __ffs(todo) - 1;
    todo &= todo - 1;
    const int Xs = __shfl_sync(FULL, X, src), Ys = __shfl_sync(FULL, Y, src), Zs = __shfl_sync(FULL, Z, src);
    const bool cov = __shfl_sync(FULL, covered ? 1 : 0, src) != 0;
    const long long ns = node_of(Xs, Ys, Zs, g);
    // the neighbours that are fluid before and after the re-flag
    long long mk = ns;
    bool sf = false;
    if (lane >= 1 && lane < Q) {
      mk = node_of(Xs + dcx(lane), Ys + dcy(lane), Zs + dcz(lane), g);
      sf = steady_fluid(a, mk);
    }
    const unsigned fm = __ballot_sync(FULL, sf);
    const int nf = __popc(fm);
    const int rank = __popc(fm & ((1u << lane) - 1u));  // place in the list, direction order
    double mx = 0.0, my = 0.0, mz = 0.0;
    if (cov) {
      // destroyed fluid: its momentum goes to the particle
      if (lane < Q) {
        const double fi = pop_abs<FM>(f, lane, N, ns, rho0);
        if (dcx(lane)) mx = csgn(dcx(lane), fi);
        if (dcy(lane)) my = csgn(dcy(lane), fi);
        if (dcz(lane)) mz = csgn(dcz(lane), fi);
        f[(long long)lane * N + ns] = FM::fp32 ? (pop_t)(-wgt(lane) * rho0) : (pop_t)0;
      }
    } else {
      // created fluid: f^eq(mean neighbour density, v_b), momentum taken from
      // the particle
      double d = 0.0;
      if (sf) {
#pragma unroll
        for (int i = 0; i < Q; ++i) d += pop_abs<FM>(f, i, N, mk, rho0);
      }
      const double sum = warp_sum(d);
      const double rbar = nf > 0 ? sum / (double)nf : rho0;
      // v_b at this node, unwrapped into the particle's current box
      const double Xu = (double)(P.lo[0] + wrapi(wrapi(Xs, g.nx) - P.lo[0], g.nx));
      const double Yu = (double)(P.lo[1] + wrapi(wrapi(Ys, g.ny) - P.lo[1], g.ny));
      const double Zu = (double)(P.lo[2] + wrapi(wrapi(Zs, g.nz) - P.lo[2], g.nz));
      const double dx = Xu - P.pos[0], dy = Yu - P.pos[1], dz = Zu - P.pos[2];
      const double vx = P.vel[0] + (P.omega[1] * dz - P.omega[2] * dy);
      const double vy = P.vel[1] + (P.omega[2] * dx - P.omega[0] * dz);
      const double vz = P.vel[2] + (P.omega[0] * dy - P.omega[1] * dx);
      const double usq = vx * vx + vy * vy + vz * vz;
      if (lane < Q) {
        const double cu = dcx(lane) * vx + dcy(lane) * vy + dcz(lane) * vz;
        const double shape = 3.0 * cu + 4.5 * cu * cu - 1.5 * usq;
        const double fi = wgt(lane) * rbar * (1.0 + shape);
        // FP32 form stores the deviation from w_i rho0, formed without cancellation
        f[(long long)lane * N + ns] =
            FM::fp32 ? (pop_t)(wgt(lane) * ((rbar - rho0) + rbar * shape)) : (pop_t)fi;
        if (dcx(lane)) mx = -csgn(dcx(lane), fi);
        if (dcy(lane)) my = -csgn(dcy(lane), fi);
        if (dcz(lane)) mz = -csgn(dcz(lane), fi);
      }
    }
    mx = warp_sum(mx);
    my = warp_sum(my);
    mz = warp_sum(mz);
    if (lane == src) {
      mom[0] = mx;
      mom[1] = my;
      mom[2] = mz;
    }
    // solute: expelled to the neighbours (covered) or refilled from them,
    // Eqs. 17-18 (uncovered); records applied after every transition is known
    if (cov) {
      if (nf == 0) {
        if (lane == 0) atomicOr(a.status, ST_EXPEL);
        continue;
      }
      if (K == 0) continue;
      int slot = 0;
      if (lane == 0) slot = atomicAdd(a.xfer_count, 1 + nf);
      slot = __shfl_sync(FULL, slot, 0);
      if (slot + 1 + nf > a.xfer_cap) {
        if (lane == 0) atomicOr(a.status, ST_CAPACITY);
        continue;
      }
      if (lane == 0) {
        Transfer self;
        self.node = ns;
        for (int k = 0; k < EK_MAX_SPECIES; ++k) self.amount[k] = k < K ? -(double)rho[k * N + ns] : 0.0;
        a.xfer[slot] = self;
      }
      if (sf) {
        Transfer tr;
        tr.node = mk;
        for (int k = 0; k < EK_MAX_SPECIES; ++k) {
          if (k >= K) {
            tr.amount[k] = 0.0;
          } else if (FM::fp32) {
            const int r = (int)rho[k * N + ns];
            const int share = r / nf, rem = r - share * nf;  // rem has the sign of r
            const int extra = (rank < (rem < 0 ? -rem : rem)) ? (rem < 0 ? -1 : 1) : 0;
            tr.amount[k] = (double)(share + extra);
          } else {
            tr.amount[k] = (double)rho[k * N + ns] / (double)nf;
          }
        }
        a.xfer[slot + 1 + rank] = tr;
      }
    } else {
      if ((a.ph.flags & EK_VACATE_ZERO) || nf == 0 || K == 0) continue;
      // refill, Eqs. 17-18: each neighbour gives rho/(N_f + 1)
      int slot = 0;
      if (lane == 0) slot = atomicAdd(a.xfer_count, 2 * nf);
      slot = __shfl_sync(FULL, slot, 0);
      if (slot + 2 * nf > a.xfer_cap) {
        if (lane == 0) atomicOr(a.status, ST_CAPACITY);
        continue;
      }
      if (sf) {
        Transfer give, take;
        give.node = mk;
        take.node = ns;
        for (int k = 0; k < EK_MAX_SPECIES; ++k) {
          double sh = 0.0;
          if (k < K) {
            if (FM::fp32) sh = (double)((int)rho[k * N + mk] / (nf + 1));
            else sh = (double)rho[k * N + mk] / (double)(nf + 1);
          }
          give.amount[k] = -sh;
          take.amount[k] = sh;
        }
        a.xfer[slot + 2 * rank] = give;
        a.xfer[slot + 2 * rank + 1] = take;
      }
    }
  }
  // the particle's transition momentum, summed in a fixed order: the CTA's
  // nodes in a fixed tree, then the CTAs' sums in chunk order by the
  // particle's last CTA, added to the momentum the next integration applies
  {
    __shared__ double tr[3][PT];
    __shared__ double quarter[3][4];
    __shared__ bool last;
    const int t = threadIdx.x;
    if (__syncthreads_or(covered || uncovered)) {
      tr[0][t] = mom[0];
      tr[1][t] = mom[1];
      tr[2][t] = mom[2];
      __syncthreads();
      if (t < 12) {
        const int d = t >> 2, w = t & 3;
        double sq = 0.0;
        for (int i = w; i < PT; i += 4) sq += tr[d][i];
        quarter[d][w] = sq;
      }
      __syncthreads();
      if (t < 3) {
        a.tpart[((long long)p * a.uchunks + bk.y) * 3 + t] =
            ((quarter[t][0] + quarter[t][1]) + quarter[t][2]) + quarter[t][3];
        __threadfence();
      }
    } else if (t < 3) {
      a.tpart[((long long)p * a.uchunks + bk.y) * 3 + t] = 0.0;  // no transition in this CTA
      __threadfence();
    }
    __syncthreads();
    if (t == 0) last = atomicAdd(a.pticket + p, 1) == a.uchunks - 1;
    __syncthreads();
    if (last) {
      __threadfence();
      if (t < 3) {
        double sum = 0.0;
        for (int j = 0; j < a.uchunks; ++j) sum += __ldcg(a.tpart + ((long long)p * a.uchunks + j) * 3 + t);
        P.ftrans[t] += sum;
      }
      if (t == 0) a.pticket[p] = 0;
    }
  }
}

template <class FM>
__global__ void __launch_bounds__(PT) k_transitions(PartArgs a) { transitions_body<FM>(a, grid_blk()); }

template <class FM>
__device__ __forceinline__ void apply_transfers_body(const PartArgs& a, const Blk bk) {
  using spc_t = typename FM::spc_t;
  spc_t* rho = (spc_t*)a.rho;
  const int count = min(*a.xfer_count, a.xfer_cap);
  for (int r = bk.x * blockDim.x + threadIdx.x; r < count; r += bk.nx * blockDim.x) {
    const Transfer t = a.xfer[r];
    for (int k = 0; k < a.ph.K; ++k) {
      if (FM::fp32) atomicAdd((int*)rho + k * a.g.N + t.node, (int)t.amount[k]);
      else atomicAdd((double*)rho + k * a.g.N + t.node, t.amount[k]);
    }
  }
}

template <class FM>
__global__ void k_apply_transfers(PartArgs a) { apply_transfers_body<FM>(a, grid_blk()); }

template <class FM>
cudaError_t particle_forces_t(const PartArgs& a, cudaStream_t s, int parts) {
  const unsigned echunks = (unsigned)((a.emax + PT - 1) / PT);
  if (parts & S4_ASSIGN) {
    k_force_assign<<<dim3(a.P, echunks), PT, 0, s>>>(a);
    k_tie_resolve<<<8, 256, 0, s>>>(a);
  }
  if (parts & S4_FORCES) k_particle_forces<FM><<<dim3(a.P, a.fchunks), FORCE_T, 0, s>>>(a);
  return cudaGetLastError();
}

// parts: 1 = everything up to the charge scatter (reads no species), 2 = the
// transitions (read and write the species after S3); 3 = both
template <class FM>
cudaError_t reflag_t(const PartArgs& a, bool transitions, cudaStream_t s, int parts = 3) {
  const Grid& g = a.g;
  const unsigned uchunks = (unsigned)union_chunks(a.boxmax);
  if (!(parts & 1)) {
    if (a.P == 0 || !transitions) return cudaSuccess;
    // (k_save_prev of this step emptied the transfer list)
    k_transitions<FM><<<dim3(a.P, uchunks), PT, 0, s>>>(a);
    k_apply_transfers<FM><<<152, 256, 0, s>>>(a);
    return cudaGetLastError();
  }
  if (!transitions) {
    k_reset_all<FM><<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(a);
  }
  if (a.P == 0) return cudaGetLastError();
  if (!transitions) k_box_update<<<(a.P + 127) / 128, 128, 0, s>>>(a);
  // union boxes are at most one cell wider than a box per axis
  const unsigned bchunks = (unsigned)((a.boxmax + PT - 1) / PT);
  if (transitions) {
    k_save_prev<<<dim3(a.P, uchunks), PT, 0, s>>>(a);
    k_clear<FM><<<dim3(a.P, uchunks), PT, 0, s>>>(a);
  }
  if (!transitions) cudaMemsetAsync(a.surf_count, 0, sizeof(int), s);  // else k_clear resets it
  k_claim<FM><<<dim3(a.P, bchunks), PT, 0, s>>>(a);
  k_psi_surface<FM><<<8 * 152, PSI_CTA, 0, s>>>(a);
  k_charge_scatter<FM><<<dim3(a.P, bchunks), PT, 0, s>>>(a);
  if (transitions && (parts & 2)) {
    k_transitions<FM><<<dim3(a.P, uchunks), PT, 0, s>>>(a);
    k_apply_transfers<FM><<<152, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// The same kernels as one launch over the systems of a batch (FP32 form):
// each CTA finds its system's arguments and its block in that system's grid.
#define EK_PART_BATCH(NAME, BODY, BOUNDS)                                                    \
  __global__ void BOUNDS NAME(const PartArgs* __restrict__ tab, const BatchSlot* __restrict__ sl, \
                              int nsys) {                                                    \
    int sys;                                                                                 \
    const Blk bk = batch_blk(sl, nsys, sys);                                                 \
    BODY(tab[sys], bk);                                                                      \
  }
EK_PART_BATCH(k_force_assign_batch, force_assign_body, __launch_bounds__(PT))
EK_PART_BATCH(k_tie_resolve_batch, tie_resolve_body, __launch_bounds__(256))
EK_PART_BATCH(k_particle_forces_batch, particle_forces_body<FormF32>, __launch_bounds__(FORCE_T, 4))
EK_PART_BATCH(k_save_prev_batch, save_prev_body, __launch_bounds__(PT))
EK_PART_BATCH(k_clear_batch, clear_body<FormF32>, __launch_bounds__(PT))
EK_PART_BATCH(k_claim_batch, claim_body<FormF32>, __launch_bounds__(PT))
EK_PART_BATCH(k_psi_surface_batch, psi_surface_body<FormF32>, __launch_bounds__(PSI_CTA))
EK_PART_BATCH(k_charge_scatter_batch, charge_scatter_body<FormF32>, __launch_bounds__(PT))
EK_PART_BATCH(k_transitions_batch, transitions_body<FormF32>, __launch_bounds__(PT))
EK_PART_BATCH(k_apply_transfers_batch, apply_transfers_body<FormF32>, __launch_bounds__(256))
#undef EK_PART_BATCH

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier of the persistent chain (all CTAs resident).  Thread 0 reads
// the generation, arrives, and the last arrival resets the count and
// advances the generation; the others wait for that, for the abort word, or
// until limit_ns has passed (then they set the timeout status and the abort
// word).  Returns false when the kernel must end.
__device__ bool chain_barrier(const ChainArgs& A) {
  __shared__ int go;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* bar = A.bar;
    int ok = bar[2] == 0u;
    if (ok) {
      const unsigned gen = bar[1];
      __threadfence();
      if (atomicAdd(A.bar, 1u) == gridDim.x - 1) {
        atomicExch(A.bar, 0u);
        __threadfence();
        atomicAdd(A.bar + 1, 1u);
      } else {
        const long long t0 = global_ns();
        while (bar[1] == gen) {
          if (bar[2] != 0u) {
            ok = 0;
            break;
          }
          if (global_ns() - t0 > A.limit_ns) {
            atomicOr(A.status, ST_TIMEOUT);
            atomicExch(A.bar + 2, 1u);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    go = ok;
  }
  __syncthreads();
  return go != 0;
}

// The phases of the chain: a CTA takes items blockIdx.x, + gridDim.x, ... of
// each phase (each item one block of a system's grid, CTA-uniform, so the
// bodies' own barriers are met by the whole CTA).
__global__ void __launch_bounds__(256) k_particle_chain(ChainArgs A) {
  if ((int)blockIdx.x == A.leave_cta) return;
  for (int q = 0; q < A.nph; ++q) {
    if (q > 0 && !chain_barrier(A)) return;
    const ChainPhase& P = A.ph[q];
    for (int w = (int)blockIdx.x; w < P.ctas; w += (int)gridDim.x) {
      int sys;
      const Blk bk = batch_blk_at(P.slot, P.nslot, w, sys);
      const PartArgs& a = A.tab[sys];
      switch (P.kind) {
        case PK_ASSIGN: force_assign_body(a, bk); break;
        case PK_TIE: tie_resolve_body(a, bk); break;
        case PK_SAVE_PREV: save_prev_body(a, bk); break;
        case PK_CLEAR: clear_body<FormF32>(a, bk); break;
        case PK_CLAIM: claim_body<FormF32>(a, bk); break;
        case PK_PSI: psi_surface_body<FormF32>(a, bk); break;
        case PK_CHARGE: charge_scatter_body<FormF32>(a, bk); break;
        case PK_TRANS: transitions_body<FormF32>(a, bk); break;
        case PK_APPLY: apply_transfers_body<FormF32>(a, bk); break;
        default: break;
      }
    }
  }
}

}  // namespace

int particle_chain_ctas() {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_particle_chain, 256, 0) != cudaSuccess)
    return 0;
  return sms * per;
}

cudaError_t launch_particle_chain(const ChainArgs& A, int ctas, cudaStream_t s) {
  if (ctas <= 0 || A.nph <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_particle_chain, A);
}

// union boxes are at most one cell wider per axis than a box of boxmax cells
int union_chunks(int boxmax) {
  const int edge = (int)round(cbrt((double)boxmax)) + 1;
  return (edge * edge * edge + PT - 1) / PT;
}

void particle_batch_grid(int k, const PartArgs& a, int& gx, int& gy) {
  gx = a.P;
  gy = 1;
  if (a.P == 0) return;
  const int uchunks = union_chunks(a.boxmax);
  const int bchunks = (a.boxmax + PT - 1) / PT;
  switch (k) {
    case PK_ASSIGN: gy = (a.emax + PT - 1) / PT; break;
    case PK_FORCES: gy = a.fchunks; break;
    case PK_SAVE_PREV:
    case PK_CLEAR:
    case PK_TRANS: gy = uchunks; break;
    case PK_CLAIM:
    case PK_CHARGE: gy = bchunks; break;
    // grid-stride kernels: their lists are short for a few particles (a CTA
    // per system), Psi's surface cells some hundreds per particle (eight
    // warps per CTA, eight CTAs per particle)
    case PK_TIE:
    case PK_APPLY: gx = 1; break;
    case PK_PSI: gx = std::min(8 * 152, 8 * a.P); break;
    default: gx = 0;
  }
}

cudaError_t launch_particle_batch(int k, const BatchLaunch<PartArgs>& L, cudaStream_t s) {
  if (L.ctas == 0) return cudaSuccess;
  const unsigned n = (unsigned)L.ctas;
  switch (k) {
    case PK_ASSIGN: k_force_assign_batch<<<n, PT, 0, s>>>(L.tab, L.slot, L.nsys); break;
    case PK_TIE: k_tie_resolve_batch<<<n, 256, 0, s>>>(L.tab, L.slot, L.nsys); break;
    case PK_FORCES: k_particle_forces_batch<<<n, FORCE_T, 0, s>>>(L.tab, L.slot, L.nsys); break;
    case PK_SAVE_PREV: k_save_prev_batch<<<n, PT, 0, s>>>(L.tab, L.slot, L.nsys); break;
    case PK_CLEAR: k_clear_batch<<<n, PT, 0, s>>>(L.tab, L.slot, L.nsys); break;
    case PK_CLAIM: k_claim_batch<<<n, PT, 0, s>>>(L.tab, L.slot, L.nsys); break;
    case PK_PSI: k_psi_surface_batch<<<n, PSI_CTA, 0, s>>>(L.tab, L.slot, L.nsys); break;
    case PK_CHARGE: k_charge_scatter_batch<<<n, PT, 0, s>>>(L.tab, L.slot, L.nsys); break;
    case PK_TRANS: k_transitions_batch<<<n, PT, 0, s>>>(L.tab, L.slot, L.nsys); break;
    case PK_APPLY: k_apply_transfers_batch<<<n, 256, 0, s>>>(L.tab, L.slot, L.nsys); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_particle_forces(const PartArgs& a, cudaStream_t s, int parts) {
  if (a.P == 0) return cudaSuccess;
  return a.ph.fp32 ? particle_forces_t<FormF32>(a, s, parts) : particle_forces_t<FormF64>(a, s, parts);
}

cudaError_t launch_reflag(const PartArgs& a, bool transitions, cudaStream_t s, int parts) {
  return a.ph.fp32 ? reflag_t<FormF32>(a, transitions, s, parts)
                   : reflag_t<FormF64>(a, transitions, s, parts);
}

}  // namespace ek
