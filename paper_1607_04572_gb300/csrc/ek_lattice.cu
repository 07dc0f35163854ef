// S2 (Capuani link fluxes + coupling force fused with the TRT/BGK collision,
// Guo force term and push streaming with velocity bounce-back) and S3 (species
// update: flux divergence + volume-of-fluid advection), FP64 form.
//
// One thread per lattice node, node index x + nx*(y + ny*z).  Populations and
// species are structure-of-arrays (direction- / species-major), so every load
// and store of a warp touches consecutive x: coalesced 8-byte accesses.  The
// neighbour loads of the flux stencil are served by L1/L2 (each value is read
// by up to 19 threads of neighbouring warps).
#include <math.h>

#include "ek_internal.cuh"

namespace ek {

namespace {

__device__ __forceinline__ long long nbr_index(int d, int x, int y, int z, const Nbr& b,
                                               int nx, int ny) {
  const int X = dcx(d) > 0 ? b.xp : (dcx(d) < 0 ? b.xm : x);
  const int Y = dcy(d) > 0 ? b.yp : (dcy(d) < 0 ? b.ym : y);
  const int Z = dcz(d) > 0 ? b.zp : (dcz(d) < 0 ? b.zm : z);
  return (long long)X + (long long)nx * ((long long)Y + (long long)ny * Z);
}

// Boundary velocity v_b = v + omega x (r_b - r) of particle p at wrapped node
// (xb, yb, zb) (Eq. 10).  The node is unwrapped into the particle's box
// [lo, lo + n) so that r_b - r is never taken across the periodic seam.
__device__ __forceinline__ void boundary_velocity(const DevParticle& P, int xb, int yb, int zb,
                                                  const Grid& g, double vb[3]) {
  const double X = (double)(P.lo[0] + wrapi(xb - P.lo[0], g.nx));
  const double Y = (double)(P.lo[1] + wrapi(yb - P.lo[1], g.ny));
  const double Z = (double)(P.lo[2] + wrapi(zb - P.lo[2], g.nz));
  const double dx = X - P.pos[0], dy = Y - P.pos[1], dz = Z - P.pos[2];
  vb[0] = P.vel[0] + (P.omega[1] * dz - P.omega[2] * dy);
  vb[1] = P.vel[1] + (P.omega[2] * dx - P.omega[0] * dz);
  vb[2] = P.vel[2] + (P.omega[0] * dy - P.omega[1] * dx);
}

// One fluid node of S2.  iv receives the node's internal solute force on the
// fluid, i = f_ext - q_ions E (zero off the fluid), also stored in ifield.
template <int K, bool PV>
__device__ __forceinline__ void lb_node(const LBArgs& a, int x, int y, int z, double (&iv)[3]) {
  const double* f_in = (const double*)a.f_in;
  double* f_out = (double*)a.f_out;
  const double* rho_in = (const double*)a.rho_in;
  double* rho_out = (double*)a.rho_out;
  const double* phi = (const double*)a.phi;
  const double* psi = (const double*)a.psi;
  double* u = (double*)a.u;
  const long long N = a.g.N;
  const int nx = a.g.nx, ny = a.g.ny;
  const long long n = node_index(a.g, x, y, z);
  double* ifield = (double*)a.ifield;
  if (a.owner[n] != FLUID) {
    // boundary node: no fluid, no solute transport
    a.vsig[n] = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) rho_out[k * N + n] = rho_in[k * N + n];
    u[n] = 0.0;
    u[N + n] = 0.0;
    u[2 * N + n] = 0.0;
    ifield[n] = 0.0;
    ifield[N + n] = 0.0;
    ifield[2 * N + n] = 0.0;
    return;
  }
  const Nbr b = make_nbr(x, y, z, a.g);

  // ---- S2a: diffusive + migrative link fluxes (Eq. 20; Eq. 13 without PV) ----
  // Link flux J_k = (D_k / A_0) * s_l * [(a - b) + z_k/2 (a + b) dphi],
  // s_l = (1 - Psi)(1 - Psi') / |c_l|.  Accumulated per species as
  // S_k = sum_l s_l [..] (the divergence is D_k/A_0 S_k) and, over species,
  // G = sum_l c_l sum_k s_l [..]; the coupling force (Eq. 16 with the 1/2 of a
  // link seen from both ends) is sum_k J_k c / (2 D_k) = G / (2 A_0).
  double gx = 0.0, gy = 0.0, gz = 0.0;
  double S[K > 0 ? K : 1];
  double r0[K > 0 ? K : 1];
  double om0 = 1.0;
  if (PV) om0 = 1.0 - psi[n];  // psi is clamped to [0, 1] by S5
#pragma unroll
  for (int k = 0; k < K; ++k) {
    S[k] = 0.0;
    r0[k] = rho_in[k * N + n];
  }
  if (PV && om0 != 1.0) {
    const double inv = 1.0 / om0;
#pragma unroll
    for (int k = 0; k < K; ++k) r0[k] *= inv;
  }
  if (K > 0) {
    const double phi0 = phi[n];
    const double s_face = om0, s_edge = om0 * 0.70710678118654752;
#pragma unroll
    for (int d = 1; d < Q; ++d) {
      const long long m = nbr_index(d, x, y, z, b, nx, ny);
      if (a.owner[m] != FLUID) continue;  // no flux into or out of boundary nodes
      double omj = 1.0;
      if (PV) omj = 1.0 - psi[m];
      const double sl = (d < 7 ? s_face : s_edge) * omj;
      const double dphi = (phi0 - phi[m]) + a.ph.ec[d];
      double tsum = 0.0;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        double rb = rho_in[k * N + m];
        if (PV && omj != 1.0) rb = rb / omj;
        const double br = fma(r0[k] + rb, a.ph.hz[k] * dphi, r0[k] - rb);
        const double T = br * sl;
        S[k] += T;
        tsum += T;
      }
      if (dcx(d)) gx += csgn(dcx(d), tsum);
      if (dcy(d)) gy += csgn(dcy(d), tsum);
      if (dcz(d)) gz += csgn(dcz(d), tsum);
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) rho_out[k * N + n] = rho_in[k * N + n] - a.ph.dcoef[k] * S[k];
  constexpr double HALF_INV_A0 = 0.13060193748187072;  // 1 / (2 (1 + 2 sqrt 2))

  // ---- S2b: collision (Eqs. 8-9), TRT in pair form ----
  // With s = f_i + f_ibar, d = f_i - f_ibar and the equilibrium/force parts
  //   Ep = Delta+_i - lambda_e f^eq+_i,  Em = Delta-_i - lambda_o f^eq-_i,
  // f*_i    = f_i    + lambda_e s/2 + lambda_o d/2 + Ep + Em,
  // f*_ibar = f_ibar + lambda_e s/2 - lambda_o d/2 + Ep - Em.
  double f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = f_in[i * N + n];
  double ps[Q], pd[Q];
  double rho = f[0], jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    ps[i] = f[i] + f[i + 1];
    pd[i] = f[i] - f[i + 1];
    rho += ps[i];
    if (dcx(i)) jx += csgn(dcx(i), pd[i]);
    if (dcy(i)) jy += csgn(dcy(i), pd[i]);
    if (dcz(i)) jz += csgn(dcz(i), pd[i]);
  }
  {
    // internal solute force: coupling force minus the field's push on the local ion charge
    double qion = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) qion += a.ph.z[k] * rho_in[k * N + n];
    iv[0] = gx * HALF_INV_A0 - qion * a.ph.E[0];
    iv[1] = gy * HALF_INV_A0 - qion * a.ph.E[1];
    iv[2] = gz * HALF_INV_A0 - qion * a.ph.E[2];
    ifield[n] = iv[0];
    ifield[N + n] = iv[1];
    ifield[2 * N + n] = iv[2];
  }
  const double Fx = gx * HALF_INV_A0 + a.ph.g[0];
  const double Fy = gy * HALF_INV_A0 + a.ph.g[1];
  const double Fz = gz * HALF_INV_A0 + a.ph.g[2];
  const double irho = 1.0 / rho;
  const double ux = (jx + 0.5 * Fx) * irho;
  const double uy = (jy + 0.5 * Fy) * irho;
  const double uz = (jz + 0.5 * Fz) * irho;
  const double usq = ux * ux + uy * uy + uz * uz;
  const double uF = ux * Fx + uy * Fy + uz * Fz;
  const double le = a.ph.lam_e, lo = a.ph.lam_o;
  const double gg = 2.0 + le;  // 2 (1 + lambda_e / 2)
  // odd part: Em = 3 w c.(F - lambda_o j)
  const double qx = fma(-lo, jx, Fx), qy = fma(-lo, jy, Fy), qz = fma(-lo, jz, Fz);
  // even part per weight class: Ep = cu (4.5 w gg cf - 4.5 w rho lambda_e cu)
  //                                  + w (-1.5 gg uF - lambda_e rho (1 - 1.5 usq))
  const double base = fma(-1.5 * gg, uF, -le * rho * fma(-1.5, usq, 1.0));
  const double hle = 0.5 * le, hlo = 0.5 * lo;
  double fs[Q];
  fs[0] = fma(1.0 + le, f[0], wgt(0) * base);
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const double w = wgt(i);
    const double cu = cdot(i, ux, uy, uz);
    const double cf = cdot(i, Fx, Fy, Fz);
    const double cq = cdot(i, qx, qy, qz);
    const double Ep = w * fma(cu, fma(4.5 * gg, cf, -4.5 * le * rho * cu), base);
    const double Em = 3.0 * w * cq;
    const double X = fma(hle, ps[i], Ep);
    const double Y = fma(hlo, pd[i], Em);
    fs[i] = f[i] + (X + Y);
    fs[i + 1] = f[i + 1] + (X - Y);
  }
  if (!isfinite(rho) || !isfinite(usq)) atomicOr(a.status, ST_NONFINITE);
  u[n] = ux;
  u[N + n] = uy;
  u[2 * N + n] = uz;
  a.vsig[n] = (unsigned char)(0x80u | sign_code(ux) | (sign_code(uy) << 2) | (sign_code(uz) << 4));

  // ---- push stream with velocity bounce-back (Eq. 12) ----
  f_out[n] = fs[0];
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const long long m = nbr_index(i, x, y, z, b, nx, ny);
    const int om = a.owner[m];
    if (om == FLUID) {
      f_out[i * N + m] = fs[i];
    } else {
      double cvb = 0.0;
      if (om >= 0) {
        const int xb = dcx(i) > 0 ? b.xp : (dcx(i) < 0 ? b.xm : x);
        const int yb = dcy(i) > 0 ? b.yp : (dcy(i) < 0 ? b.ym : y);
        const int zb = dcz(i) > 0 ? b.zp : (dcz(i) < 0 ? b.zm : z);
        double vb[3];
        boundary_velocity(a.parts[om], xb, yb, zb, a.g, vb);
        cvb = cdot(i, vb[0], vb[1], vb[2]);
      }
      f_out[opp(i) * N + n] = fs[i] - 6.0 * wgt(i) * a.ph.rho0 * cvb;
    }
  }
}

// Sum of three doubles over a block of the lattice grid, fixed order; thread
// 0 writes it to ipart[3 * block].
__device__ __forceinline__ void block_sum3(double (&v)[3], double* ipart) {
  __shared__ double red[TILE_X * TILE_Y / 32][3];
  const int t = threadIdx.x + TILE_X * threadIdx.y;
  const int lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double s = v[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][c] = s;
  }
  __syncthreads();
  if (t == 0) {
    const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int w = 0; w < TILE_X * TILE_Y / 32; ++w) s += red[w][c];
      ipart[3 * blk + c] = s;
    }
  }
}

template <int K, bool PV>
__global__ void __launch_bounds__(256, 2) k_lb_fused(LBArgs a) {
  const int x = blockIdx.x * TILE_X + threadIdx.x;
  const int y = blockIdx.y * TILE_Y + threadIdx.y;
  const int z = blockIdx.z;
  double iv[3] = {0.0, 0.0, 0.0};
  if (x < a.g.nx && y < a.g.ny) lb_node<K, PV>(a, x, y, z, iv);
  block_sum3(iv, a.ipart);
}

// sign (-1, 0, +1) and magnitude of a double from its bits: integer work
// only, so the advection's tests cost no FP64 instructions (-0 counts as 0)
__device__ __forceinline__ int sgn_bits(double v) {
  const long long b = __double_as_longlong(v);
  if ((b << 1) == 0) return 0;
  return b < 0 ? -1 : 1;
}
__device__ __forceinline__ double abs_bits(double v) {
  return __longlong_as_double(__double_as_longlong(v) & 0x7fffffffffffffffLL);
}

// S3: rho' = (rho - div J) + volume-of-fluid advection.  rho_out holds
// rho - div J (written by S2) and is updated in place; rho_in is the species
// field at the start of the step (the advected one).  The cell displaced by
// u overlaps the neighbours at offsets s with s_a in {0, sign(u_a)}; the share
// of offset s is prod_a w_a, w_a = 1 - |u_a| (s_a = 0) or |u_a|.
template <int K>
__global__ void __launch_bounds__(256) k_advect(LBArgs a) {
  const double* rho_in = (const double*)a.rho_in;
  double* rho_out = (double*)a.rho_out;
  const double* u = (const double*)a.u;
  const long long N = a.g.N;
  const int x = blockIdx.x * TILE_X + threadIdx.x;
  const int y = blockIdx.y * TILE_Y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= a.g.nx || y >= a.g.ny) return;
  const long long n = node_index(a.g, x, y, z);
  if (!(a.vsig[n] & 0x80u)) return;  // fluid bit of S2 (the flags may change meanwhile)
  const Nbr b = make_nbr(x, y, z, a.g);
  double acc[K];
  double rs[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    acc[k] = rho_out[k * N + n];
    rs[k] = rho_in[k * N + n];
  }
  // outflow of this cell
  const double ux = u[n], uy = u[N + n], uz = u[2 * N + n];
  const int sx = sgn_bits(ux), sy = sgn_bits(uy), sz = sgn_bits(uz);
  const double ax = abs_bits(ux), ay = abs_bits(uy), az = abs_bits(uz);
  const double bx = 1.0 - ax, by = 1.0 - ay, bz = 1.0 - az;
  for (int oz = 0; oz <= (sz != 0); ++oz) {
    for (int oy = 0; oy <= (sy != 0); ++oy) {
      for (int ox = 0; ox <= (sx != 0); ++ox) {
        if (!ox && !oy && !oz) continue;
        const long long m = node_index(a.g, nb_x(b, x, ox ? sx : 0), nb_y(b, y, oy ? sy : 0),
                                       nb_z(b, z, oz ? sz : 0));
        if (!(a.vsig[m] & 0x80u)) continue;  // share aimed at a boundary stays here
        const double frac = (ox ? ax : bx) * (oy ? ay : by) * (oz ? az : bz);
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] -= rs[k] * frac;
      }
    }
  }
  // inflow from the 26 neighbours y = x - s: only those whose velocity points
  // here along every nonzero component of s contribute
  for (int qz = -1; qz <= 1; ++qz) {
    for (int qy = -1; qy <= 1; ++qy) {
      for (int qx = -1; qx <= 1; ++qx) {
        if (!qx && !qy && !qz) continue;
        const long long m = node_index(a.g, nb_x(b, x, -qx), nb_y(b, y, -qy), nb_z(b, z, -qz));
        // the source must be fluid and move towards this node along every nonzero q
        const unsigned mask = 0x80u | (qx ? 3u : 0u) | (qy ? 12u : 0u) | (qz ? 48u : 0u);
        const unsigned want = 0x80u | (qx > 0 ? 1u : (qx < 0 ? 2u : 0u)) |
                              (qy > 0 ? 4u : (qy < 0 ? 8u : 0u)) | (qz > 0 ? 16u : (qz < 0 ? 32u : 0u));
        if ((a.vsig[m] & mask) != want) continue;
        const double vx = u[m], vy = u[N + m], vz = u[2 * N + m];
        if ((qx && sgn_bits(vx) != qx) || (qy && sgn_bits(vy) != qy) || (qz && sgn_bits(vz) != qz))
          continue;
        const double wx = qx ? abs_bits(vx) : 1.0 - abs_bits(vx);
        const double wy = qy ? abs_bits(vy) : 1.0 - abs_bits(vy);
        const double wz = qz ? abs_bits(vz) : 1.0 - abs_bits(vz);
        const double frac = wx * wy * wz;
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] += rho_in[k * N + m] * frac;
      }
    }
  }
  bool bad = false;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    rho_out[k * N + n] = acc[k];
    bad |= !isfinite(acc[k]);
  }
  if (bad) atomicOr(a.status, ST_NONFINITE);
}

__global__ void k_fill(Grid g, const int* owner, double* f, double* rho, int K, double rho0,
                       double b0, double b1, double b2, double b3) {
  const long long N = g.N;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const bool fl = owner[n] == FLUID;
  const double bk[4] = {b0, b1, b2, b3};
  for (int k = 0; k < K; ++k) rho[k * N + n] = fl ? bk[k] : 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i * N + n] = fl ? wgt(i) * rho0 : 0.0;
}

unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_lb_fused(const LBArgs& a, cudaStream_t s) {
  const bool pv = a.ph.pv != 0;
  switch (a.ph.K) {
#define EK_CASE(KK)                                                   \
  case KK:                                                            \
    if (pv) k_lb_fused<KK, true><<<lattice_grid(a.g), lattice_block(), 0, s>>>(a);               \
    else k_lb_fused<KK, false><<<lattice_grid(a.g), lattice_block(), 0, s>>>(a);                 \
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

cudaError_t launch_advection(const LBArgs& a, cudaStream_t s) {
  switch (a.ph.K) {
    case 0: return cudaSuccess;
    case 1: k_advect<1><<<lattice_grid(a.g), lattice_block(), 0, s>>>(a); break;
    case 2: k_advect<2><<<lattice_grid(a.g), lattice_block(), 0, s>>>(a); break;
    case 3: k_advect<3><<<lattice_grid(a.g), lattice_block(), 0, s>>>(a); break;
    case 4: k_advect<4><<<lattice_grid(a.g), lattice_block(), 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fill(const Grid& g, const Phys& ph, const int* owner, double* f, double* rho,
                        const double* bulk_k, cudaStream_t s) {
  k_fill<<<blocks_for(g.N, 256), 256, 0, s>>>(g, owner, f, rho, ph.K, ph.rho0, bulk_k[0],
                                                 bulk_k[1], bulk_k[2], bulk_k[3]);
  return cudaGetLastError();
}

}  // namespace ek
