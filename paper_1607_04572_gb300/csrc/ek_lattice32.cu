// S2 and S3 of the FP32-storage form: populations stored as the deviation
// g_i = f_i - w_i rho0 in float, species as int32 multiples of qscale_k,
// Phi / Psi / u in float, arithmetic in float.
//
// Exact conservation with 4-byte species: every link flux is quantised to an
// integer number of units and computed with bitwise the same operations from
// both of its end nodes (symmetric operands, no contraction), so the two ends
// see exactly opposite integers and the lattice total never changes; the
// volume-of-fluid shares are likewise computed identically by the source
// (outflow) and the destination (inflow) thread.
//
// Partial-volume flux without divisions: with A = rho_x (1 - Psi_y) and
// B = rho_y (1 - Psi_x), Eq. 20 becomes
//   J = D/(A_0 |c|) [(A - B) + z/2 (A + B)(Phi_x - Phi_y + E.c)],
// which is antisymmetric by construction.
#include <math.h>

#include <algorithm>

#include "ek_internal.cuh"

namespace ek {

namespace {

__device__ __forceinline__ float csgnf(int c, float v) { return c > 0 ? v : -v; }
__device__ __forceinline__ float cdotf(int i, float x, float y, float z) {
  const int a = dcx(i), b = dcy(i), c = dcz(i);
  if (a && b) return csgnf(a, x) + csgnf(b, y);
  if (a && c) return csgnf(a, x) + csgnf(c, z);
  if (b && c) return csgnf(b, y) + csgnf(c, z);
  if (a) return csgnf(a, x);
  if (b) return csgnf(b, y);
  if (c) return csgnf(c, z);
  return 0.0f;
}

}  // namespace

Phys32 make_phys32(const Phys& ph) {
  Phys32 p;
  p.rho0 = (float)ph.rho0;
  p.lam_e = (float)ph.lam_e;
  p.lam_o = (float)ph.lam_o;
  for (int k = 0; k < EK_MAX_SPECIES; ++k) {
    p.qs[k] = (float)ph.qscale[k];
    p.cq[k] = ph.qscale[k] > 0.0 ? (float)(ph.dcoef[k] / ph.qscale[k]) : 0.0f;
    p.hz[k] = (float)ph.hz[k];
  }
  for (int i = 0; i < 19; ++i) p.ec[i] = (float)ph.ec[i];
  for (int d = 0; d < 3; ++d) {
    p.g[d] = (float)ph.g[d];
    p.E[d] = (float)ph.E[d];
  }
  for (int k = 0; k < EK_MAX_SPECIES; ++k) p.zq[k] = (float)(ph.z[k] * ph.qscale[k]);
  return p;
}

namespace {

// The neighbourhood of a node as its three x coordinates, row offsets and
// plane offsets (periodic, 32-bit: N < 2^31): a neighbour's index is one
// three-operand add.
struct Off3 {
  int X0, X1, X2, Y0, Y1, Y2, Z0, Z1, Z2;
};
__device__ __forceinline__ Off3 make_off3(const Nbr& b, int x, int y, int z, int nx, int ny) {
  const int nxy = nx * ny;
  return {b.xm, x, b.xp, nx * b.ym, nx * y, nx * b.yp, nxy * b.zm, nxy * z, nxy * b.zp};
}
__device__ __forceinline__ int nbr32(int d, const Off3& o) {
  return (dcx(d) > 0 ? o.X2 : (dcx(d) < 0 ? o.X0 : o.X1)) +
         (dcy(d) > 0 ? o.Y2 : (dcy(d) < 0 ? o.Y0 : o.Y1)) +
         (dcz(d) > 0 ? o.Z2 : (dcz(d) < 0 ? o.Z0 : o.Z1));
}

// block total of the per-thread sums: warps in float (32 threads, each over
// its segment's nodes), the warp sums in FP64; the GPU's FP64 rate is a small
// fraction of its FP32 rate, so the per-node accumulation stays in float
__device__ __forceinline__ void block_sum3(float (&v)[3], double* ipart, long long blk) {
  __shared__ double red[TILE_X * TILE_Y / 32][3];
  const int t = threadIdx.x + TILE_X * threadIdx.y;
  const int lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) {
    float s = v[cc];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][cc] = (double)s;
  }
  __syncthreads();
  if (t == 0) {
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      double s = 0.0;
      for (int w = 0; w < TILE_X * TILE_Y / 32; ++w) s += red[w][cc];
      ipart[3 * blk + cc] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// 2.5D-tiled S2 (FP32 form) with asynchronous staging.  A 32 x 8 thread block
// owns a (32 x 8) column of consecutive planes (the grid's z dimension splits
// each column into nzb segments of about 8 planes).  The stencil fields of the planes
// z - 1, z, z + 1 -- species (raw int units), Psi, Phi and the node class --
// sit in a 4-slot shared-memory ring with a one-node halo, and the
// populations of plane z in one of two shared buffers.  While plane z is
// computed, cp.async copies plane z + 2's stencil fields and plane z + 1's
// populations in, so the global-memory latency of the loads overlaps the
// arithmetic instead of stalling it; every value is read from global memory
// once per block.
// ---------------------------------------------------------------------------
constexpr int HX = TILE_X + 2, HY = TILE_Y + 2;  // tile with halo
constexpr int HP = HX * HY;                    // nodes of one halo plane
constexpr int TN = TILE_X * TILE_Y;            // nodes of one tile plane
constexpr int RING = 4;

template <int K>
struct LBRing {
  int own[RING][HP];
  float phi[RING][HP];
  float psi[RING][HP];                // Psi as copied; 1 - Psi once landed
  int rho[K > 0 ? K : 1][RING][HP];   // int units as copied; rho qscale (float bits) once landed
  float pop[2][Q][TN];
};

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// all groups but the newest `n` are complete (for this thread's copies)
template <int n>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(n) : "memory");
}

// periodic coordinate of a tile-halo position v in [-1, n + 33).  One wrap
// is exact for every position a node of the box reads (at most n); the
// positions past it, which exist only for edges below the tile width and are
// never read, are clamped into the box so that their loads stay in bounds.
__device__ __forceinline__ int halo_wrap(int v, int n) {
  v = v < 0 ? v + n : (v >= n ? v - n : v);
  return min(v, n - 1);
}

// in-plane offsets (x + nx y) of the thread's halo-tile nodes e = tid and
// tid + TN (-1: none); the same in every plane
__device__ __forceinline__ void halo_offsets(int (&hoff)[2], int x0, int y0, const LBArgs& a) {
  const int tid = threadIdx.x + TILE_X * threadIdx.y;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int e = tid + q * TN;
    const int ey = e / HX, ex = e - ey * HX;
    hoff[q] = e < HP ? halo_wrap(x0 - 1 + ex, a.g.nx) + a.g.nx * halo_wrap(y0 - 1 + ey, a.g.ny) : -1;
  }
}

// stencil fields of plane zz (periodic) into ring slot `slot`
template <int K, bool PV>
__device__ __forceinline__ void stage_plane(LBRing<K>& t, int slot, int zz, const int (&hoff)[2],
                                            const LBArgs& a) {
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const size_t N = (size_t)a.g.N;
  const int z = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
  const int tid = threadIdx.x + TILE_X * threadIdx.y;
  const size_t pz = (size_t)nx * ny * z;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (hoff[q] < 0) continue;
    const int e = tid + q * TN;
    const size_t m = (size_t)hoff[q] + pz;
    cp_async4(&t.own[slot][e], a.owner + m);
    cp_async4(&t.phi[slot][e], (const float*)a.phi + m);
    if (PV) cp_async4(&t.psi[slot][e], (const float*)a.psi + m);
#pragma unroll
    for (int k = 0; k < K; ++k) cp_async4(&t.rho[k][slot][e], (const int*)a.rho_in + k * N + m);
  }
}

// populations of plane z (z < nz) into buffer `buf`: 16-byte copies of four
// consecutive nodes when rows are 16-byte aligned (nx % 4 == 0), else 4 bytes
template <int K>
__device__ __forceinline__ void stage_pops(LBRing<K>& t, int buf, int z, int x0, int y0,
                                           const LBArgs& a) {
  const int nx = a.g.nx, ny = a.g.ny;
  const size_t N = (size_t)a.g.N;
  const float* f = (const float*)a.f_in;
  const int tid = threadIdx.x + TILE_X * threadIdx.y;
  const size_t zoff = (size_t)nx * ny * z;
  if ((nx & 3) == 0) {
    // chunk tid + 256 j: population (tid >> 6) + 4 j, row (tid >> 3) % 8, four
    // nodes at 4 (tid % 8): the row and nodes are the thread's own in every
    // chunk, so only the population advances
    const int r = (tid >> 3) & 7, q = (tid & 7) * 4, i0 = tid >> 6;
    const int y = y0 + r, x = x0 + q;
    if (y < ny && x < nx) {
      const float* src = f + i0 * N + zoff + (size_t)y * nx + x;
      float* dst = &t.pop[buf][i0][r * TILE_X + q];
#pragma unroll
      for (int j = 0; j < (Q + 3) / 4; ++j)
        if (i0 + 4 * j < Q) cp_async16(dst + j * 4 * TN, src + (size_t)(4 * j) * N);
    }
  } else {
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x < nx && y < ny) {
      const size_t n = zoff + (size_t)y * nx + x;
#pragma unroll
      for (int i = 0; i < Q; ++i) cp_async4(&t.pop[buf][i][tid], f + i * N + n);
    }
  }
}

template <int K>
constexpr size_t lb32_smem() { return sizeof(LBRing<K>); }

// One node of plane z.  SIMPLE: the block's stencil planes hold fluid nodes
// only and Psi = 0 (no particle or wall near), so every link is a fluid link,
// the partial-volume factors are 1 and nothing bounces back; the arithmetic is
// the same as in the general path with those values.
template <int K, bool PV, bool SIMPLE>
__device__ __forceinline__ void lb32_node(const LBRing<K>& t, const LBArgs& a, const Phys32& c,
                                          int x, int y, int z, int tid, int ex, int ey,
                                          float (&iv)[3]) {
  float* __restrict__ g_out = (float*)a.f_out;
  const int* __restrict__ n_in = (const int*)a.rho_in;
  int* __restrict__ n_out = (int*)a.rho_out;
  float* __restrict__ u = (float*)a.u;
  float* __restrict__ ifield = (float*)a.ifield;
  const size_t N = (size_t)a.g.N;
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const int sl[3] = {(z + 3) & 3, z & 3, (z + 1) & 3};  // planes z - 1, z, z + 1
  const int e0 = ex + HX * ey;
  const int n = x + nx * (y + ny * z);
  const Nbr b = make_nbr(x, y, z, a.g);
  const Off3 nb = make_off3(b, x, y, z, nx, ny);
  if (!SIMPLE && t.own[sl[1]][e0] != FLUID) {
    a.vsig[n] = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) (n_out + k * N)[n] = (n_in + k * N)[n];
    u[n] = 0.0f;
    (u + N)[n] = 0.0f;
    (u + 2 * N)[n] = 0.0f;
    ifield[n] = 0.0f;
    (ifield + N)[n] = 0.0f;
    (ifield + 2 * N)[n] = 0.0f;
  } else {
    unsigned fluid = SIMPLE ? 0xFFFFFFFEu : 0u;
    if (!SIMPLE) {
#pragma unroll
      for (int d = 1; d < Q; ++d)
        if (t.own[sl[1 + dcz(d)]][e0 + dcx(d) + HX * dcy(d)] == FLUID) fluid |= 1u << d;
    }
    // ---- S2a: quantised link fluxes (symmetric operands) and coupling force ----
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
    int S[K > 0 ? K : 1];
    float r0[K > 0 ? K : 1];
    const float om0 = PV ? t.psi[sl[1]][e0] : 1.0f;
    const float phi0 = t.phi[sl[1]][e0];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      S[k] = 0;
      r0[k] = __int_as_float(t.rho[k][sl[1]][e0]);
    }
#pragma unroll
    for (int d = 1; d < Q; ++d) {
      if (K == 0 || !(fluid & (1u << d))) continue;
      const int sd = sl[1 + dcz(d)], ed = e0 + dcx(d) + HX * dcy(d);
      const float omj = PV ? t.psi[sd][ed] : 1.0f;
      const float dphi = __fadd_rn(__fsub_rn(phi0, t.phi[sd][ed]), c.ec[d]);
      float tsum = 0.0f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float rb = __int_as_float(t.rho[k][sd][ed]);
        const float A = PV ? __fmul_rn(r0[k], omj) : r0[k];
        const float B = PV ? __fmul_rn(rb, om0) : rb;
        float br = fmaf(__fadd_rn(A, B), __fmul_rn(c.hz[k], dphi), __fsub_rn(A, B));
        if (d >= 7) br = __fmul_rn(br, 0.70710678f);
        S[k] += __float2int_rn(__fmul_rn(br, c.cq[k]));
        tsum += br;
      }
      if (dcx(d)) gx += csgnf(dcx(d), tsum);
      if (dcy(d)) gy += csgnf(dcy(d), tsum);
      if (dcz(d)) gz += csgnf(dcz(d), tsum);
    }
    float qion = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int nk = (n_in + k * N)[n];
      (n_out + k * N)[n] = nk - S[k];
      qion = fmaf(c.zq[k], (float)nk, qion);
    }
    constexpr float HALF_INV_A0 = 0.13060193748187072f;
    {
      const float ix = gx * HALF_INV_A0 - qion * c.E[0];
      const float iy = gy * HALF_INV_A0 - qion * c.E[1];
      const float iz = gz * HALF_INV_A0 - qion * c.E[2];
      ifield[n] = ix;
      (ifield + N)[n] = iy;
      (ifield + 2 * N)[n] = iz;
      iv[0] += ix;
      iv[1] += iy;
      iv[2] += iz;
    }
    // ---- S2b: TRT collision on the deviations (pair form) ----
    float g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = t.pop[z & 1][i][tid];
    float drho = g[0], jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const float pd = g[i] - g[i + 1];
      drho += g[i] + g[i + 1];
      if (dcx(i)) jx += csgnf(dcx(i), pd);
      if (dcy(i)) jy += csgnf(dcy(i), pd);
      if (dcz(i)) jz += csgnf(dcz(i), pd);
    }
    const float rho = c.rho0 + drho;
    const float Fx = fmaf(gx, HALF_INV_A0, c.g[0]);
    const float Fy = fmaf(gy, HALF_INV_A0, c.g[1]);
    const float Fz = fmaf(gz, HALF_INV_A0, c.g[2]);
    const float irho = 1.0f / rho;
    const float ux = (jx + 0.5f * Fx) * irho;
    const float uy = (jy + 0.5f * Fy) * irho;
    const float uz = (jz + 0.5f * Fz) * irho;
    const float usq = ux * ux + uy * uy + uz * uz;
    const float uF = ux * Fx + uy * Fy + uz * Fz;
    const float le = c.lam_e, lo = c.lam_o;
    const float gg = 2.0f + le;
    const float qx = fmaf(-lo, jx, Fx), qy = fmaf(-lo, jy, Fy), qz = fmaf(-lo, jz, Fz);
    const float base = fmaf(-1.5f * gg, uF, -le * fmaf(-1.5f * rho, usq, drho));
    const float hle = 0.5f * le, hlo = 0.5f * lo;
    const float k45 = -4.5f * le * rho;
    if (!isfinite(rho) || !isfinite(usq)) atomicOr(a.status, ST_NONFINITE);
    u[n] = ux;
    (u + N)[n] = uy;
    (u + 2 * N)[n] = uz;
    a.vsig[n] = (unsigned char)(0x80u | sign_code(ux) | (sign_code(uy) << 2) | (sign_code(uz) << 4));
    // ---- collide each pair and push-stream it (velocity bounce-back, Eq. 12) ----
    g_out[n] = fmaf(1.0f + le, g[0], (float)wgt(0) * base);
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const float w = (float)wgt(i);
      const float cu = cdotf(i, ux, uy, uz);
      const float cf = cdotf(i, Fx, Fy, Fz);
      const float cqv = cdotf(i, qx, qy, qz);
      const float Ep = w * fmaf(cu, fmaf(4.5f * gg, cf, k45 * cu), base);
      const float Em = 3.0f * w * cqv;
      const float X = fmaf(hle, g[i] + g[i + 1], Ep);
      const float Y = fmaf(hlo, g[i] - g[i + 1], Em);
      const float gsd[2] = {g[i] + (X + Y), g[i + 1] + (X - Y)};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int d = i + h;
        if (fluid & (1u << d)) {
          (g_out + d * N)[nbr32(d, nb)] = gsd[h];
        } else {
          float cvb = 0.0f;
          const int om = t.own[sl[1 + dcz(d)]][e0 + dcx(d) + HX * dcy(d)];
          if (om >= 0) {
            const DevParticle& P = a.parts[om];
            const int xb = dcx(d) > 0 ? b.xp : (dcx(d) < 0 ? b.xm : x);
            const int yb = dcy(d) > 0 ? b.yp : (dcy(d) < 0 ? b.ym : y);
            const int zb = dcz(d) > 0 ? b.zp : (dcz(d) < 0 ? b.zm : z);
            // wall velocity at the boundary node in float (it enters the
            // float population): the offset from the centre as integer part
            // minus the centre's fraction, the velocities as float copies
            const float dx = __fsub_rn((float)(P.lo[0] + wrapi(xb - P.lo[0], nx) - P.ipos[0]), P.fpos[0]);
            const float dy = __fsub_rn((float)(P.lo[1] + wrapi(yb - P.lo[1], ny) - P.ipos[1]), P.fpos[1]);
            const float dz = __fsub_rn((float)(P.lo[2] + wrapi(zb - P.lo[2], nz) - P.ipos[2]), P.fpos[2]);
            const float vx = P.velf[0] + (P.omegaf[1] * dz - P.omegaf[2] * dy);
            const float vy = P.velf[1] + (P.omegaf[2] * dx - P.omegaf[0] * dz);
            const float vz = P.velf[2] + (P.omegaf[0] * dy - P.omegaf[1] * dx);
            cvb = cdotf(d, vx, vy, vz);
          }
          (g_out + opp(d) * N)[n] = gsd[h] - 6.0f * (float)wgt(d) * c.rho0 * cvb;
        }
      }
    }
  }
}

// One block of the S2 grid: tile (bx, by), z segment bz; blk is the block's
// row of the per-block sums.
template <int K, bool PV>
__device__ __forceinline__ void lb32_block(const LBArgs& a, const Phys32& c, int bx, int by, int bz,
                                           long long blk) {
  extern __shared__ __align__(16) unsigned char lb_smem[];
  LBRing<K>& t = *reinterpret_cast<LBRing<K>*>(lb_smem);
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const int x0 = bx * TILE_X, y0 = by * TILE_Y;
  const int z0 = (int)((long long)bz * nz / a.nzb);
  const int zend = (int)((long long)(bz + 1) * nz / a.nzb);
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  const int tid = threadIdx.x + TILE_X * threadIdx.y;
  const bool in_xy = x < nx && y < ny;
  const int ex = threadIdx.x + 1, ey = threadIdx.y + 1;
  float iv[3] = {0.0f, 0.0f, 0.0f};
  int hoff[2];
  halo_offsets(hoff, x0, y0, a);
  // ring slot of plane zz: zz mod 4 (zz >= -1)
  stage_plane<K, PV>(t, (z0 + 3) & 3, z0 - 1, hoff, a);
  stage_plane<K, PV>(t, z0 & 3, z0, hoff, a);
  stage_plane<K, PV>(t, (z0 + 1) & 3, z0 + 1, hoff, a);
  stage_pops<K>(t, z0 & 1, z0, x0, y0, a);
  cp_async_commit();
  // A landed halo plane: does it hold a non-fluid node or Psi > 0?  And its
  // species and Psi are converted once, in place, to the operands of the link
  // fluxes (rho qscale and 1 - Psi, the same operations each of the 19 uses
  // would repeat).  Each thread handles the elements it copied itself
  // (complete after its own wait); the barrier that follows publishes them.
  auto plane_flag = [&](int slot) -> int {
    bool f = false;
    for (int e = tid; e < HP; e += TN) {
      f |= t.own[slot][e] != FLUID || (PV && t.psi[slot][e] != 0.0f);
      if (PV) t.psi[slot][e] = __fsub_rn(1.0f, t.psi[slot][e]);
#pragma unroll
      for (int k = 0; k < K; ++k)
        t.rho[k][slot][e] = __float_as_int(__fmul_rn((float)t.rho[k][slot][e], c.qs[k]));
    }
    return f ? 1 : 0;
  };
  int fm1 = 0, f0 = 0;  // flags of planes z - 1 and z
  for (int z = z0; z < zend; ++z) {
    // plane z + 2 and the populations of z + 1 (empty group at the end)
    if (z + 1 < zend) {
      stage_plane<K, PV>(t, (z + 2) & 3, z + 2, hoff, a);
      stage_pops<K>(t, (z + 1) & 1, z + 1, x0, y0, a);
    }
    cp_async_commit();
    cp_async_wait<1>();
    if (z == z0) {
      fm1 = __syncthreads_or(plane_flag((z0 + 3) & 3));
      f0 = __syncthreads_or(plane_flag(z0 & 3));
    }
    const int fp1 = __syncthreads_or(plane_flag((z + 1) & 3));  // also publishes all copies
    if (in_xy) {
      if (!(fm1 | f0 | fp1)) lb32_node<K, false, true>(t, a, c, x, y, z, tid, ex, ey, iv);
      else lb32_node<K, PV, false>(t, a, c, x, y, z, tid, ex, ey, iv);
    }
    fm1 = f0;
    f0 = fp1;
    __syncthreads();  // the next copies overwrite the slots of plane z - 1 and populations z
  }
  cp_async_wait<0>();
  block_sum3(iv, a.ipart, blk);
}

template <int K, bool PV>
__global__ void __launch_bounds__(256, 2) k_lb32_tiled(LBArgs a, Phys32 c) {
  lb32_block<K, PV>(a, c, blockIdx.x, blockIdx.y, blockIdx.z,
                    blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z));
}

// S2 of a batch's systems in one launch: system s runs its xt x (yt nzb) grid
// (tiles x fastest, then y, then the z segment), the block sums in the same
// rows as its own launch would
template <int K, bool PV>
__global__ void __launch_bounds__(256, 2) k_lb32_batch(const LBBatchEntry* __restrict__ tab,
                                                       const BatchSlot* __restrict__ slot, int nsys) {
  int sys;
  const Blk b = batch_blk(slot, nsys, sys);
  const LBBatchEntry& e = tab[sys];
  const int yt = (e.a.g.ny + TILE_Y - 1) / TILE_Y;
  lb32_block<K, PV>(e.a, e.c, b.x, b.y % yt, b.y / yt, b.x + (long long)b.nx * b.y);
}

// sign code (bits 0-1 of c >> shift) as -1, 0, +1
__device__ __forceinline__ int sign_of(unsigned c, int shift) {
  const unsigned v = (c >> shift) & 3u;
  return v == 1u ? 1 : (v == 2u ? -1 : 0);
}

// ---------------------------------------------------------------------------
// S3 (FP32 form), tiled push.  A 32 x 8 block marches through a segment of
// planes of its (x, y) tile column.  The cell of a fluid node displaced by its
// velocity v (Eq. 15's volume-of-fluid advection) overlaps the node itself
// and the offsets {0, sign(v_a)}^3 \ 0; the share landing at offset o is
// rho_k prod_a (o_a ? |v_a| : 1 - |v_a|), quantised to integer units.  Every
// node of the tile and its one-node halo adds the shares it sends into
// shared-memory accumulators of the receiving positions (integer atomics:
// the sums do not depend on the order), and every node of the tile takes
// from its own accumulator the shares it sends to fluid nodes (a share aimed
// at a boundary node stays where it is).  A plane is complete once the
// planes on both sides have pushed; its nodes then add their accumulator to
// S2's result.  A share is computed by the same operations in every block
// that holds its source, so a source's loss and its destination's gain are
// the same integers and the species totals do not change.
// ---------------------------------------------------------------------------
constexpr int AW = HX + 2, AH = HY + 2;  // accumulator plane: the halo tile with a margin of one
constexpr int AP = AW * AH;
constexpr int HALO = HP - TN;            // halo nodes of a tile plane

template <int K>
struct AdvRing {
  int acc[4][K > 0 ? K : 1][AP];  // shares received minus shares sent, plane p in slot p & 3
  unsigned char sg[4][HP];        // sign bytes of S2 (bit 7 fluid, sign codes of u), slot p & 3
};

template <int K>
constexpr size_t adv32_smem() { return sizeof(AdvRing<K>); }

// the sources of a thread: 0 its own node of the tile, 1 the halo node with
// the thread's index (threads below HALO): the top row, the bottom row, then
// the left and the right column of the halo.  Halo-tile index e (stride HX),
// accumulator index (stride AW, one further in from the margin) and the
// in-plane offset of the node in the box (-1: none).
struct AdvPos {
  int e[2], pos[2], hoff[2];
};
__device__ __forceinline__ AdvPos adv_positions(int x0, int y0, const LBArgs& a) {
  const int tid = threadIdx.x + TILE_X * threadIdx.y;
  int ex[2] = {(int)threadIdx.x + 1, 0}, ey[2] = {(int)threadIdx.y + 1, 0};
  if (tid < HX) {
    ex[1] = tid;
  } else if (tid < 2 * HX) {
    ex[1] = tid - HX;
    ey[1] = HY - 1;
  } else if (tid < 2 * HX + TILE_Y) {
    ey[1] = tid - 2 * HX + 1;
  } else {
    ex[1] = HX - 1;
    ey[1] = tid - 2 * HX - TILE_Y + 1;
  }
  AdvPos p;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    p.e[q] = ex[q] + HX * ey[q];
    p.pos[q] = ex[q] + 1 + AW * (ey[q] + 1);
    p.hoff[q] = q == 0 || tid < HALO
                    ? halo_wrap(x0 - 1 + ex[q], a.g.nx) + a.g.nx * halo_wrap(y0 - 1 + ey[q], a.g.ny)
                    : -1;
  }
  return p;
}

// the sign bytes, velocities and species of a thread's sources in one plane,
// loaded one plane ahead of use
template <int K>
struct AdvSrc {
  unsigned sgn[2];
  float v[2][3];
  int r[2][K > 0 ? K : 1];
};

__device__ __forceinline__ int wrap_plane(int zz, int nz) {
  return zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
}

template <int K>
__device__ __forceinline__ void adv_load(AdvSrc<K>& R, const AdvPos& P, int zz, const LBArgs& a) {
  const int N = (int)a.g.N;
  const int pz = a.g.nx * a.g.ny * wrap_plane(zz, a.g.nz);
  const float* __restrict__ ux = (const float*)a.u;
  const float* __restrict__ uy = ux + N;
  const float* __restrict__ uz = uy + N;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    R.sgn[q] = 0u;
    if (P.hoff[q] >= 0) {
      const int m = P.hoff[q] + pz;
      R.sgn[q] = a.vsig[m];
      R.v[q][0] = ux[m];
      R.v[q][1] = uy[m];
      R.v[q][2] = uz[m];
#pragma unroll
      for (int k = 0; k < K; ++k) R.r[q][k] = ((const int*)a.rho_in + (size_t)k * N)[m];
    }
  }
}

__device__ __forceinline__ void adv_sign(unsigned (&s)[2], const AdvPos& P, int zz, const LBArgs& a) {
  const int pz = a.g.nx * a.g.ny * wrap_plane(zz, a.g.nz);
#pragma unroll
  for (int q = 0; q < 2; ++q) s[q] = P.hoff[q] >= 0 ? a.vsig[P.hoff[q] + pz] : 0u;
}

template <int K>
__device__ __forceinline__ void adv_sign_put(AdvRing<K>& t, int zz, const AdvPos& P, const unsigned (&s)[2]) {
#pragma unroll
  for (int q = 0; q < 2; ++q)
    if (P.hoff[q] >= 0) t.sg[zz & 3][P.e[q]] = (unsigned char)s[q];
}

// source q of plane p: its shares added at the receiving positions; a node of
// the tile (OWN) also takes from its own accumulator the shares it sends to
// fluid nodes.  The share of offset o is the same product, in the same order,
// wherever it is computed: (w_x w_y) w_z with w_a = |v_a| or 1 - |v_a|.
template <int K, bool OWN>
__device__ __forceinline__ void adv_push(AdvRing<K>& t, int p, const AdvPos& P, const AdvSrc<K>& R, int q) {
  const unsigned s = R.sgn[q];
  if (!(s & 0x80u)) return;  // not a fluid node: sends nothing
  const int sx = sign_of(s, 0), sy = sign_of(s, 2), sz = sign_of(s, 4);
  const float ax = fabsf(R.v[q][0]), ay = fabsf(R.v[q][1]), az = fabsf(R.v[q][2]);
  const float bx = __fsub_rn(1.0f, ax), by = __fsub_rn(1.0f, ay), bz = __fsub_rn(1.0f, az);
  const float wxy[4] = {__fmul_rn(bx, by), __fmul_rn(ax, by), __fmul_rn(bx, ay), __fmul_rn(ax, ay)};
  float rf[K > 0 ? K : 1];
#pragma unroll
  for (int k = 0; k < K; ++k) rf[k] = (float)R.r[q][k];
  // a share whose offset has a component where v has none is zero: it adds
  // nothing wherever it lands
  int* const a0 = &t.acc[p & 3][0][P.pos[q]];
  int* const a1 = &t.acc[(p + sz) & 3][0][P.pos[q]];
  const unsigned char* const f0 = &t.sg[p & 3][P.e[q]];
  const unsigned char* const f1 = &t.sg[(p + sz) & 3][P.e[q]];
  const int dy = sy * AW, fy = sy * HX;
  int net[K > 0 ? K : 1];
#pragma unroll
  for (int k = 0; k < K; ++k) net[k] = 0;
#pragma unroll
  for (int o = 1; o < 8; ++o) {
    const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
    const float frac = __fmul_rn(wxy[o & 3], oz ? az : bz);
    int* const dst = (oz ? a1 : a0) + (ox ? sx : 0) + (oy ? dy : 0);
    bool fl = false;
    if (OWN) fl = ((oz ? f1 : f0)[(ox ? sx : 0) + (oy ? fy : 0)] & 0x80u) != 0u;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int v = __float2int_rn(__fmul_rn(rf[k], frac));
      atomicAdd(dst + k * AP, v);
      if (OWN && fl) net[k] += v;
    }
  }
  if (OWN) {
#pragma unroll
    for (int k = 0; k < K; ++k) atomicAdd(a0 + k * AP, -net[k]);
  }
}

template <int K>
__device__ __forceinline__ void adv_zero(AdvRing<K>& t, int slot) {
  int4* z = reinterpret_cast<int4*>(&t.acc[slot][0][0]);
  const int tid = threadIdx.x + TILE_X * threadIdx.y;
  for (int i = tid; i < K * AP / 4; i += TN) z[i] = make_int4(0, 0, 0, 0);
}

template <int K>
__device__ __forceinline__ void advect32_block(const LBArgs& a, int bx, int by, int bz, int nseg) {
  extern __shared__ __align__(16) unsigned char adv_smem[];
  AdvRing<K>& t = *reinterpret_cast<AdvRing<K>*>(adv_smem);
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const int N = (int)a.g.N;
  const int x0 = bx * TILE_X, y0 = by * TILE_Y;
  const int z0 = (int)((long long)bz * nz / nseg);
  const int zend = (int)((long long)(bz + 1) * nz / nseg);
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  const int tid = threadIdx.x + TILE_X * threadIdx.y;
  const bool in_xy = x < nx && y < ny;
  const bool halo = tid < HALO;
  int* nout[K > 0 ? K : 1];
#pragma unroll
  for (int k = 0; k < K; ++k) nout[k] = (int*)a.rho_out + (size_t)k * N;
  const AdvPos P = adv_positions(x0, y0, a);
  AdvSrc<K> R;
  unsigned sgn[2];
  // Plane z is complete when planes z - 1, z and z + 1 have pushed; a push of
  // plane p needs the sign bytes of planes p - 1 .. p + 1 (the fluid test of
  // the receiving nodes).  Before the loop: all slots zero, the sign bytes of
  // planes z0 - 1 .. z0 + 1, pushes of planes z0 - 1 (only its shares into
  // plane z0 count) and z0.
  for (int s = 0; s < 4; ++s) adv_zero<K>(t, s);
  for (int i = tid; i < 4 * HP; i += TN) (&t.sg[0][0])[i] = 0;
  __syncthreads();
  for (int zz = z0 - 1; zz <= z0 + 1; ++zz) {
    adv_sign(sgn, P, zz, a);
    adv_sign_put<K>(t, zz, P, sgn);
  }
  adv_load<K>(R, P, z0 - 1, a);
  __syncthreads();
  adv_push<K, true>(t, z0 - 1, P, R, 0);
  if (halo) adv_push<K, false>(t, z0 - 1, P, R, 1);
  adv_load<K>(R, P, z0, a);
  __syncthreads();
  adv_zero<K>(t, (z0 - 2) & 3);  // the slot of plane z0 + 2: planes z0 - 2's shares
  adv_push<K, true>(t, z0, P, R, 0);
  if (halo) adv_push<K, false>(t, z0, P, R, 1);
  adv_load<K>(R, P, z0 + 1, a);
  adv_sign(sgn, P, z0 + 2, a);
  const int c = (threadIdx.y + 1) * HX + threadIdx.x + 1;        // the node's halo-tile index
  const int pc = threadIdx.x + 2 + AW * (threadIdx.y + 2);       // and accumulator index
  for (int z = z0; z < zend; ++z) {
    const int n = x + nx * (y + ny * z);
    int s2[K > 0 ? K : 1];
    if (in_xy) {
#pragma unroll
      for (int k = 0; k < K; ++k) s2[k] = nout[k][n];  // S2's result, issued early
    }
    adv_sign_put<K>(t, z + 2, P, sgn);
    __syncthreads();  // the sign bytes of plane z + 2; slot z + 2 zero
    adv_push<K, true>(t, z + 1, P, R, 0);
    if (halo) adv_push<K, false>(t, z + 1, P, R, 1);
    if (z + 1 < zend) {
      adv_load<K>(R, P, z + 2, a);
      adv_sign(sgn, P, z + 3, a);
    }
    __syncthreads();  // plane z complete
    if (in_xy && (t.sg[z & 3][c] & 0x80u)) {
#pragma unroll
      for (int k = 0; k < K; ++k) nout[k][n] = s2[k] + t.acc[z & 3][k][pc];
    }
    adv_zero<K>(t, (z - 1) & 3);  // the slot of plane z + 3
  }
}

template <int K>
__global__ void __launch_bounds__(256) k_advect32(LBArgs a, Phys32 c) {
  (void)c;
  advect32_block<K>(a, blockIdx.x, blockIdx.y, blockIdx.z, a.advseg);
}

// S3 of a batch's systems in one launch (system s: its xt x (yt nseg) grid)
template <int K>
__global__ void __launch_bounds__(256) k_advect32_batch(const LBBatchEntry* __restrict__ tab,
                                                        const BatchSlot* __restrict__ slot, int nsys) {
  int sys;
  const Blk b = batch_blk(slot, nsys, sys);
  const LBArgs& a = tab[sys].a;
  const int yt = (a.g.ny + TILE_Y - 1) / TILE_Y;
  advect32_block<K>(a, b.x, b.y % yt, b.y / yt, a.advseg);
}

__global__ void k_fill32(Grid g, const int* owner, float* f, int* rho, int K, float rho0, int n0,
                         int n1, int n2, int n3) {
  const long long N = g.N;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const bool fl = owner[n] == FLUID;
  const int nk[4] = {n0, n1, n2, n3};
  for (int k = 0; k < K; ++k) rho[k * N + n] = fl ? nk[k] : 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i * N + n] = fl ? 0.0f : -(float)wgt(i) * rho0;
}

// field conversions between the FP64 exchange format and the FP32 storage
__global__ void k_pop_to_f64(long long N, int i, float rho0, const float* g, double* out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N) out[n] = (double)g[i * N + n] + wgt(i) * (double)rho0;
}
__global__ void k_pop_from_f64(long long N, int i, float rho0, const double* in, float* g) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N) g[i * N + n] = (float)(in[n] - wgt(i) * (double)rho0);
}
__global__ void k_spc_to_f64(long long N, double q, const int* in, double* out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N) out[n] = (double)in[n] * q;
}
__global__ void k_spc_from_f64(long long N, double q, const double* in, int* out, int* status) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double v = rint(in[n] / q);
  if (!(fabs(v) < 2147483647.0)) {
    atomicOr(status, ST_CAPACITY);
    out[n] = 0;
    return;
  }
  out[n] = (int)v;
}
__global__ void k_f32_to_f64(long long N, const float* in, double* out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N) out[n] = (double)in[n];
}
__global__ void k_f64_to_f32(long long N, const double* in, float* out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N) out[n] = (float)in[n];
}
// f = f^eq(current rho, u) on fluid nodes, u given in FP64 (3 components)
__global__ void k_set_velocity32(Grid g, const int* owner, float* f, const double* u3, float rho0) {
  const long long N = g.N;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N || owner[n] != FLUID) return;
  double drho = 0.0;
  for (int i = 0; i < Q; ++i) drho += (double)f[i * N + n];
  const double rho = (double)rho0 + drho;
  const double ux = u3[n], uy = u3[N + n], uz = u3[2 * N + n];
  const double usq = ux * ux + uy * uy + uz * uz;
  for (int i = 0; i < Q; ++i) {
    const double cu = cdot(i, ux, uy, uz);
    f[i * N + n] = (float)(wgt(i) * (drho + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq)));
  }
}
__global__ void k_density32(Grid g, const float* f, float rho0, double* out) {
  const long long N = g.N;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double s = (double)rho0;
  for (int i = 0; i < Q; ++i) s += (double)f[i * N + n];
  out[n] = s;
}

unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

// shared memory above the 48 KB default, set once per kernel before any launch
// (in particular before a step is captured into a graph)
cudaError_t lb32_prepare() {
  cudaError_t e = cudaSuccess;
#define EK_ATTR(KK)                                                                          \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(k_lb32_tiled<KK, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)lb32_smem<KK>());                                          \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(k_lb32_tiled<KK, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)lb32_smem<KK>());                                          \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(k_lb32_batch<KK, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)lb32_smem<KK>());                                          \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(k_lb32_batch<KK, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)lb32_smem<KK>());
  EK_ATTR(0)
  EK_ATTR(1)
  EK_ATTR(2)
  EK_ATTR(3)
  EK_ATTR(4)
#undef EK_ATTR
#define EK_ADV_ATTR(KK)                                                                   \
  if (e == cudaSuccess)                                                                    \
    e = cudaFuncSetAttribute(k_advect32<KK>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                             (int)adv32_smem<KK>());                                       \
  if (e == cudaSuccess)                                                                    \
    e = cudaFuncSetAttribute(k_advect32_batch<KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)adv32_smem<KK>());
  EK_ADV_ATTR(1)
  EK_ADV_ATTR(2)
  EK_ADV_ATTR(3)
  EK_ADV_ATTR(4)
#undef EK_ADV_ATTR
  return e;
}

// Segments per tile column: about 4 planes each, with two blocks of 256
// threads per SM (up to 128 registers, no spills).  Measured on GB300 at 128^3
// (ms per launch): 4-plane segments 0.123, 3 planes 0.127, 2 planes 0.136,
// 1 plane 0.173; with three blocks per SM (80 registers, spills) 8-plane
// segments 0.185 and 16-plane 0.200.  Short segments let the block scheduler
// balance the SMs; one-plane segments pay three halo planes per plane.
int lb32_segments(const Grid& g, int K, bool pv) {
  (void)K;
  (void)pv;
  return std::max(1, (g.nz + 3) / 4);
}

cudaError_t launch_lb32(const LBArgs& a, cudaStream_t s) {
  const Phys32 c = make_phys32(a.ph);
  const bool pv = a.ph.pv != 0;
  switch (a.ph.K) {
#define EK_CASE(KK)                                                                        \
  case KK:                                                                                 \
    if (pv) k_lb32_tiled<KK, true><<<lattice_grid32(a.g, a.nzb), lattice_block(), lb32_smem<KK>(), s>>>(a, c); \
    else k_lb32_tiled<KK, false><<<lattice_grid32(a.g, a.nzb), lattice_block(), lb32_smem<KK>(), s>>>(a, c);   \
    break;
    EK_CASE(0)
    EK_CASE(1)
    EK_CASE(2)
    EK_CASE(3)
    EK_CASE(4)
#undef EK_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_advection32(const LBArgs& a, cudaStream_t s) {
  const Phys32 c = make_phys32(a.ph);
  switch (a.ph.K) {
    case 0: return cudaSuccess;
    case 1: k_advect32<1><<<lattice_grid32(a.g, a.advseg), lattice_block(), adv32_smem<1>(), s>>>(a, c); break;
    case 2: k_advect32<2><<<lattice_grid32(a.g, a.advseg), lattice_block(), adv32_smem<2>(), s>>>(a, c); break;
    case 3: k_advect32<3><<<lattice_grid32(a.g, a.advseg), lattice_block(), adv32_smem<3>(), s>>>(a, c); break;
    case 4: k_advect32<4><<<lattice_grid32(a.g, a.advseg), lattice_block(), adv32_smem<4>(), s>>>(a, c); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

void lb32_batch_grid(const LBArgs& a, int& gx, int& gy) {
  const dim3 g = lattice_grid32(a.g, a.nzb);
  gx = (int)g.x;
  gy = (int)(g.y * g.z);
}

// Planes per S3 segment.  Every segment pushes the plane on each side of it
// as well, so long segments waste less; short ones give the block scheduler
// enough blocks to balance the SMs (five blocks of 256 threads fit on one).
// Measured on GB300 (ms per launch): 128^3 4/8/16/32 planes 0.041, 0.038,
// 0.037, 0.053; 256^3 (K = 3) 0.341, 0.287, 0.262, 0.265; 512^3 1.99, 1.64,
// 1.48, 1.40.  A batch launch (wide) holds many systems: 16 planes.
int adv32_segments(const Grid& g, bool wide) {
  const long long cols = (long long)((g.nx + TILE_X - 1) / TILE_X) * ((g.ny + TILE_Y - 1) / TILE_Y);
  auto blocks = [&](int p) { return cols * ((g.nz + p - 1) / p); };
  int planes = 4;
  if (!wide && blocks(32) >= 8192) planes = 32;
  else if (wide || blocks(16) >= 3 * 152) planes = 16;
  else if (blocks(8) >= 3 * 152) planes = 8;
  return std::max(1, (g.nz + planes - 1) / planes);
}

void advect32_batch_grid(const LBArgs& a, int& gx, int& gy) {
  const dim3 g = lattice_grid32(a.g, a.advseg);
  gx = (int)g.x;
  gy = (int)(g.y * g.z);
}

cudaError_t launch_lb32_batch(const BatchLaunch<LBBatchEntry>& L, int K, bool pv, cudaStream_t s) {
  if (L.ctas == 0) return cudaSuccess;
  switch (K) {
#define EK_CASE(KK)                                                                            \
  case KK:                                                                                     \
    if (pv) k_lb32_batch<KK, true><<<L.ctas, lattice_block(), lb32_smem<KK>(), s>>>(L.tab, L.slot, L.nsys); \
    else k_lb32_batch<KK, false><<<L.ctas, lattice_block(), lb32_smem<KK>(), s>>>(L.tab, L.slot, L.nsys);   \
    break;
    EK_CASE(0)
    EK_CASE(1)
    EK_CASE(2)
    EK_CASE(3)
    EK_CASE(4)
#undef EK_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_advection32_batch(const BatchLaunch<LBBatchEntry>& L, int K, cudaStream_t s) {
  if (L.ctas == 0) return cudaSuccess;
  switch (K) {
    case 0: return cudaSuccess;
    case 1: k_advect32_batch<1><<<L.ctas, lattice_block(), adv32_smem<1>(), s>>>(L.tab, L.slot, L.nsys); break;
    case 2: k_advect32_batch<2><<<L.ctas, lattice_block(), adv32_smem<2>(), s>>>(L.tab, L.slot, L.nsys); break;
    case 3: k_advect32_batch<3><<<L.ctas, lattice_block(), adv32_smem<3>(), s>>>(L.tab, L.slot, L.nsys); break;
    case 4: k_advect32_batch<4><<<L.ctas, lattice_block(), adv32_smem<4>(), s>>>(L.tab, L.slot, L.nsys); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fill32(const Grid& g, const Phys& ph, const int* owner, float* f, int* rho,
                          const int* units, cudaStream_t s) {
  k_fill32<<<blocks_for(g.N, 256), 256, 0, s>>>(g, owner, f, rho, ph.K, (float)ph.rho0, units[0],
                                                   units[1], units[2], units[3]);
  return cudaGetLastError();
}

cudaError_t convert32(int op, const Grid& g, int index, double scale, const void* in, void* out,
                      int* status, cudaStream_t s) {
  const long long N = g.N;
  const unsigned nb = blocks_for(N, 256);
  switch (op) {
    case CONV_POP_TO_F64: k_pop_to_f64<<<nb, 256, 0, s>>>(N, index, (float)scale, (const float*)in, (double*)out); break;
    case CONV_POP_FROM_F64: k_pop_from_f64<<<nb, 256, 0, s>>>(N, index, (float)scale, (const double*)in, (float*)out); break;
    case CONV_SPC_TO_F64: k_spc_to_f64<<<nb, 256, 0, s>>>(N, scale, (const int*)in, (double*)out); break;
    case CONV_SPC_FROM_F64: k_spc_from_f64<<<nb, 256, 0, s>>>(N, scale, (const double*)in, (int*)out, status); break;
    case CONV_F32_TO_F64: k_f32_to_f64<<<nb, 256, 0, s>>>(N, (const float*)in, (double*)out); break;
    case CONV_F64_TO_F32: k_f64_to_f32<<<nb, 256, 0, s>>>(N, (const double*)in, (float*)out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t set_velocity32(const Grid& g, const int* owner, float* f, const double* u3, double rho0,
                           cudaStream_t s) {
  k_set_velocity32<<<blocks_for(g.N, 256), 256, 0, s>>>(g, owner, f, u3, (float)rho0);
  return cudaGetLastError();
}

cudaError_t density32(const Grid& g, const float* f, double rho0, double* out, cudaStream_t s) {
  k_density32<<<blocks_for(g.N, 256), 256, 0, s>>>(g, f, (float)rho0, out);
  return cudaGetLastError();
}

}  // namespace ek
