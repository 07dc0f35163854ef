// S1: charge assembly and the periodic Poisson solve of Eq. 3 by hand-written
// batched FFT kernels (FP64).
//
//   lap_7 Phi = -4 pi l_B q,    Phi^(k) = 4 pi l_B q^(k) / lambda(k),
//   lambda(k) = sum_a (2 - 2 cos(2 pi k_a / n_a)),  Phi^(0) = 0,
//
// i.e. the exact inverse of the 7-point Laplacian on the periodic lattice (the
// k = 0 mode is a uniform neutralising background).
//
// Passes (each a kernel, lines staged in shared memory):
//   X  real-to-complex along x, two real rows packed as one complex row, with
//      the charge assembly q = sum_k z_k rho_k + rho_wall + q_particles fused
//      into the load; writes the half spectrum S[z][y][kx], kx <= nx/2
//   Y  complex FFT along y, tiles of consecutive kx (coalesced rows)
//   Z  complex FFT along z, Green multiply, inverse FFT along z (fused)
//   Y  inverse
//   X  complex-to-real along x, two rows per complex FFT; writes Phi
// Each line FFT is a mixed-radix (4, 2, 3) Stockham autosort transform
// (Govindaraju et al., SC 2008 formulation), ping-ponging between two shared
// memory buffers, so no bit reversal pass is needed.
#include <math.h>
#include <cstdint>
#include <cstring>

#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <algorithm>

#include <cooperative_groups.h>

#include "ek_internal.cuh"

namespace ek {

namespace cg = cooperative_groups;

namespace {

constexpr int LINE_ELEMS = 1024;  // complex elements staged per CTA and buffer (16 KB)
constexpr int FFT_THREADS = 256;

// real type -> complex type
template <typename R> struct CT;
template <> struct CT<double> { using type = double2; };
template <> struct CT<float> { using type = float2; };

__device__ __forceinline__ double2 mkc(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 mkc(float x, float y) { return make_float2(x, y); }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cmulconj(C a, C b) {  // a * conj(b)
  return mkc(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// multiply by -i (forward) or +i (inverse)
template <typename C> __device__ __forceinline__ C rot(C a, bool inverse) {
  return inverse ? mkc(-a.y, a.x) : mkc(a.y, -a.x);
}
// twiddle exp(-2 pi i k / n) and Laplacian eigenvalue of an axis, per precision
__device__ __forceinline__ double2 twiddle(const AxisPlan& P, int k, double) { return P.tw[k]; }
__device__ __forceinline__ float2 twiddle(const AxisPlan& P, int k, float) { return P.tw32[k]; }
__device__ __forceinline__ double lambda_of(const AxisPlan& P, int k, double) { return P.lam[k]; }
__device__ __forceinline__ float lambda_of(const AxisPlan& P, int k, float) { return P.lam32[k]; }

// Stockham FFT of `nl` lines of length n stored line-major in `a`; `b` is the
// second buffer.  Returns the buffer holding the result.  All threads of the
// CTA must call it.
template <typename C>
__device__ C* fft_lines(C* a, C* b, int nl, const AxisPlan& P, bool inverse) {
  using R = decltype(C().x);
  const int n = P.n;
  int Ns = 1;
  for (int s = 0; s < P.nrad; ++s) {
    const int RAD = P.radix[s];
    const int nb = n / RAD;
    const int twstep = n / (Ns * RAD);
    for (int t = threadIdx.x; t < nl * nb; t += blockDim.x) {
      const int line = t / nb;
      const int j = t - line * nb;
      const C* in = a + line * n;
      C* out = b + line * n;
      const int k = j % Ns;
      C v[4];
      for (int r = 0; r < RAD; ++r) {
        C e = in[j + r * nb];
        if (r > 0 && k > 0) {
          const C w = twiddle(P, (k * r * twstep) % n, R(0));
          e = inverse ? cmulconj(e, w) : cmul(e, w);
        }
        v[r] = e;
      }
      C o[4];
      if (RAD == 2) {
        o[0] = cadd(v[0], v[1]);
        o[1] = csub(v[0], v[1]);
      } else if (RAD == 4) {
        const C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        const C s13 = cadd(v[1], v[3]), d13 = rot(csub(v[1], v[3]), inverse);
        o[0] = cadd(s02, s13);
        o[2] = csub(s02, s13);
        o[1] = cadd(d02, d13);
        o[3] = csub(d02, d13);
      } else {  // radix 3
        const R c = R(0.86602540378443865);  // sin(2 pi / 3)
        const C s = cadd(v[1], v[2]);
        const C d = csub(v[1], v[2]);
        const C tt = mkc(v[0].x - R(0.5) * s.x, v[0].y - R(0.5) * s.y);
        const C rd = rot(mkc(c * d.x, c * d.y), inverse);
        o[0] = cadd(v[0], s);
        o[1] = cadd(tt, rd);
        o[2] = csub(tt, rd);
      }
      const int base = (j / Ns) * Ns * RAD + k;
      for (int r = 0; r < RAD; ++r) out[base + r * Ns] = o[r];
    }
    __syncthreads();
    C* tmp = a;
    a = b;
    b = tmp;
    Ns *= RAD;
  }
  return a;
}

template <typename R>
struct PassArgs {
  using C = typename CT<R>::type;
  int nx, ny, nz, nxh;
  AxisPlan ax, ay, az;
  const R* q;          // charge (used when rho == nullptr)
  const void* rho;     // species, K*N: R, or int units of qscale (charge assembled on the fly)
  bool int_species;
  const R* qwall;
  const R* qpart;
  int K;
  R z[EK_MAX_SPECIES];  // z_k, times qscale_k for int species
  C* S;                // half spectrum (nx/2+1)*ny*nz
  R* phi;
  R green_scale;       // 4 pi l_B / N
};

template <typename R>
__device__ __forceinline__ R charge_at(const PassArgs<R>& a, long long i, long long N) {
  if (a.rho == nullptr) return a.q[i];
  R q = R(0);
  if (a.int_species) {
#pragma unroll
    for (int k = 0; k < EK_MAX_SPECIES; ++k)
      if (k < a.K) q += a.z[k] * (R)((const int*)a.rho)[k * N + i];
  } else {
#pragma unroll
    for (int k = 0; k < EK_MAX_SPECIES; ++k)
      if (k < a.K) q += a.z[k] * ((const R*)a.rho)[k * N + i];
  }
  if (a.qwall) q += a.qwall[i];
  if (a.qpart) q += a.qpart[i];
  return q;
}

// the charge of four consecutive nodes i..i+3 (i % 4 == 0, every array 16-byte
// aligned): the operations of charge_at, lane by lane, on 16-byte loads
__device__ __forceinline__ float4 charge_at4(const PassArgs<float>& a, long long i, long long N) {
  if (a.rho == nullptr) return *reinterpret_cast<const float4*>(a.q + i);
  float4 q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (a.int_species) {
#pragma unroll
    for (int k = 0; k < EK_MAX_SPECIES; ++k)
      if (k < a.K) {
        const int4 v = *reinterpret_cast<const int4*>((const int*)a.rho + k * N + i);
        q.x += a.z[k] * (float)v.x;
        q.y += a.z[k] * (float)v.y;
        q.z += a.z[k] * (float)v.z;
        q.w += a.z[k] * (float)v.w;
      }
  } else {
#pragma unroll
    for (int k = 0; k < EK_MAX_SPECIES; ++k)
      if (k < a.K) {
        const float4 v = *reinterpret_cast<const float4*>((const float*)a.rho + k * N + i);
        q.x += a.z[k] * v.x;
        q.y += a.z[k] * v.y;
        q.z += a.z[k] * v.z;
        q.w += a.z[k] * v.w;
      }
  }
  if (a.qwall) {
    const float4 v = *reinterpret_cast<const float4*>(a.qwall + i);
    q.x += v.x;
    q.y += v.y;
    q.z += v.z;
    q.w += v.w;
  }
  if (a.qpart) {
    const float4 v = *reinterpret_cast<const float4*>(a.qpart + i);
    q.x += v.x;
    q.y += v.y;
    q.z += v.z;
    q.w += v.w;
  }
  return q;
}

// X pass, forward: rows r0 = 2p, r1 = 2p + 1 packed as a + i b.
template <typename R>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_x_fwd(PassArgs<R> a, int pairs_per_cta) {
  using C = typename CT<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  const int n = a.nx;
  const int nrows = a.ny * a.nz;
  const long long N = (long long)a.nx * a.ny * a.nz;
  const int p0 = blockIdx.x * pairs_per_cta;
  C* b0 = smem;
  C* b1 = smem + pairs_per_cta * n;
  for (int t = threadIdx.x; t < pairs_per_cta * n; t += blockDim.x) {
    const int l = t / n, x = t - l * n;
    const int r0 = 2 * (p0 + l), r1 = r0 + 1;
    R re = R(0), im = R(0);
    if (r0 < nrows) re = charge_at(a, (long long)r0 * n + x, N);
    if (r1 < nrows) im = charge_at(a, (long long)r1 * n + x, N);
    b0[t] = mkc(re, im);
  }
  __syncthreads();
  C* res = fft_lines(b0, b1, pairs_per_cta, a.ax, false);
  const int nxh = a.nxh;
  for (int t = threadIdx.x; t < pairs_per_cta * nxh; t += blockDim.x) {
    const int l = t / nxh, k = t - l * nxh;
    const int r0 = 2 * (p0 + l), r1 = r0 + 1;
    if (r0 >= nrows) continue;
    const C Zk = res[l * n + k];
    const C Zm = res[l * n + (k == 0 ? 0 : n - k)];
    // A_k = (Z_k + conj Z_{n-k}) / 2,  B_k = (Z_k - conj Z_{n-k}) / (2 i)
    const C A = mkc(R(0.5) * (Zk.x + Zm.x), R(0.5) * (Zk.y - Zm.y));
    const C B = mkc(R(0.5) * (Zk.y + Zm.y), R(-0.5) * (Zk.x - Zm.x));
    a.S[(long long)r0 * nxh + k] = A;
    if (r1 < nrows) a.S[(long long)r1 * nxh + k] = B;
  }
}

// Y or Z pass on tiles of `tx` consecutive kx.  axis 1: lines along y for
// each z; axis 2: lines along z for each y, with the Green multiply and the
// inverse transform fused.
template <typename R>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_yz(PassArgs<R> a, int axis, int tx, bool inverse) {
  using C = typename CT<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  const int nxh = a.nxh;
  const int ntile = (nxh + tx - 1) / tx;
  const int tile = blockIdx.x % ntile;
  const int other = blockIdx.x / ntile;  // z (axis 1) or y (axis 2)
  const int kx0 = tile * tx;
  const AxisPlan& P = axis == 1 ? a.ay : a.az;
  const int n = P.n;
  const long long stride = axis == 1 ? (long long)nxh : (long long)nxh * a.ny;
  const long long base = axis == 1 ? (long long)other * a.ny * nxh : (long long)other * nxh;
  C* b0 = smem;
  C* b1 = smem + tx * n;
  // element t = j * tx + c : line c (kx0 + c), position j
  for (int t = threadIdx.x; t < tx * n; t += blockDim.x) {
    const int j = t / tx, c = t - j * tx;
    C v = mkc(R(0), R(0));
    if (kx0 + c < nxh) v = a.S[base + j * stride + kx0 + c];
    b0[c * n + j] = v;
  }
  __syncthreads();
  C* res;
  if (axis == 1) {
    res = fft_lines(b0, b1, tx, P, inverse);
  } else {
    res = fft_lines(b0, b1, tx, P, false);
    C* other_buf = res == b0 ? b1 : b0;
    // Green function of the 7-point Laplacian; here `other` is ky
    const R ly = lambda_of(a.ay, other, R(0));
    for (int t = threadIdx.x; t < tx * n; t += blockDim.x) {
      const int c = t / n, j = t - c * n;
      const int kx = kx0 + c;
      R g = R(0);
      if (kx < nxh) {
        const R lam = lambda_of(a.ax, kx, R(0)) + ly + lambda_of(a.az, j, R(0));
        g = (kx == 0 && other == 0 && j == 0) ? R(0) : a.green_scale / lam;
      }
      const C v = res[t];
      res[t] = mkc(v.x * g, v.y * g);
    }
    __syncthreads();
    res = fft_lines(res, other_buf, tx, P, true);
  }
  for (int t = threadIdx.x; t < tx * n; t += blockDim.x) {
    const int j = t / tx, c = t - j * tx;
    if (kx0 + c < nxh) a.S[base + j * stride + kx0 + c] = res[c * n + j];
  }
}

// X pass, inverse (complex-to-real), two rows per complex transform.
template <typename R>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_x_inv(PassArgs<R> a, int pairs_per_cta) {
  using C = typename CT<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  const int n = a.nx;
  const int nxh = a.nxh;
  const int nrows = a.ny * a.nz;
  const int p0 = blockIdx.x * pairs_per_cta;
  C* b0 = smem;
  C* b1 = smem + pairs_per_cta * n;
  for (int t = threadIdx.x; t < pairs_per_cta * n; t += blockDim.x) {
    const int l = t / n, k = t - l * n;
    const int r0 = 2 * (p0 + l), r1 = r0 + 1;
    C A = mkc(R(0), R(0)), B = mkc(R(0), R(0));
    const bool upper = k > n / 2;
    const int kk = upper ? n - k : k;
    if (r0 < nrows) A = a.S[(long long)r0 * nxh + kk];
    if (r1 < nrows) B = a.S[(long long)r1 * nxh + kk];
    if (upper) {
      A.y = -A.y;
      B.y = -B.y;
    }
    // Z = A + i B
    b0[t] = mkc(A.x - B.y, A.y + B.x);
  }
  __syncthreads();
  C* res = fft_lines(b0, b1, pairs_per_cta, a.ax, true);
  for (int t = threadIdx.x; t < pairs_per_cta * n; t += blockDim.x) {
    const int l = t / n, x = t - l * n;
    const int r0 = 2 * (p0 + l), r1 = r0 + 1;
    if (r0 < nrows) a.phi[(long long)r0 * n + x] = res[t].x;
    if (r1 < nrows) a.phi[(long long)r1 * n + x] = res[t].y;
  }
}

// ---------------------------------------------------------------------------
// Fast path of the FP32 form for edges 2^k and 3 2^k from 24 to 512: the same
// five passes, with each line transform specialised at compile time.  A stage
// of radix R (16, 8, 4 or 3) loads R elements into registers, applies the stage
// twiddles from a shared-memory table, does the length-R DFT in registers
// (even/odd splits down to radix 4, constant twiddles) and stores in
// Stockham order; a length-128 line takes two stages (16 x 8).  Shared-memory
// rows are padded by one element every 16, which keeps the strided stores of
// the first stage free of bank conflicts.
// ---------------------------------------------------------------------------
constexpr int FAST_T = 256;           // threads per CTA of the y / z passes
constexpr int FAST_ELEMS = 2048;      // complex elements per CTA and buffer (before padding)
// the x passes gather the charge (or scatter Phi) straight from the lattice:
// more, smaller CTAs keep more loads in flight
constexpr int FAST_XT = 256;
constexpr int FAST_XELEMS = 1024;
constexpr int FAST_IT = 128;      // inverse x pass
constexpr int FAST_IELEMS = 2048;
__host__ __device__ constexpr int fpad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int fast_radix(int n, int s) {
  // radices of the stages: 32 = 8 4, 64 = 8 8, 128 = 16 8, 256 = 16 16, 512 = 8 8 8,
  // 24 = 8 3, 48 = 16 3, 96 = 8 4 3, 192 = 16 4 3, 384 = 16 8 3
  return n == 32 ? (s == 0 ? 8 : s == 1 ? 4 : 0)
       : n == 64 ? (s < 2 ? 8 : 0)
       : n == 128 ? (s == 0 ? 16 : s == 1 ? 8 : 0)
       : n == 256 ? (s < 2 ? 16 : 0)
       : n == 512 ? (s < 3 ? 8 : 0)
       : n == 24 ? (s == 0 ? 8 : s == 1 ? 3 : 0)
       : n == 48 ? (s == 0 ? 16 : s == 1 ? 3 : 0)
       : n == 96 ? (s == 0 ? 8 : s == 1 ? 4 : s == 2 ? 3 : 0)
       : n == 192 ? (s == 0 ? 16 : s == 1 ? 4 : s == 2 ? 3 : 0)
       : n == 384 ? (s == 0 ? 16 : s == 1 ? 8 : s == 2 ? 3 : 0)
       : 0;
}
inline bool fast_edge(int n) {
  return n == 24 || n == 32 || n == 48 || n == 64 || n == 96 || n == 128 || n == 192 || n == 256 ||
         n == 384 || n == 512;
}

// multiply by exp(-+2 pi i k / R) (forward: minus), k < R / 2, R = 8, 16 or 32
template <int R, bool INV>
__device__ __forceinline__ float2 wconst(int k, float2 z) {
  // cos and sin of 2 pi m / 32, m = 0..15
  constexpr float C32[16] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f,
                             0.83146961230254523708f, 0.70710678118654752440f,
                             0.55557023301960222474f, 0.38268343236508977173f,
                             0.19509032201612826785f, 0.0f, -0.19509032201612826785f,
                             -0.38268343236508977173f, -0.55557023301960222474f,
                             -0.70710678118654752440f, -0.83146961230254523708f,
                             -0.92387953251128675613f, -0.98078528040323044913f};
  constexpr float S32[16] = {0.0f, 0.19509032201612826785f, 0.38268343236508977173f,
                             0.55557023301960222474f, 0.70710678118654752440f,
                             0.83146961230254523708f, 0.92387953251128675613f,
                             0.98078528040323044913f, 1.0f, 0.98078528040323044913f,
                             0.92387953251128675613f, 0.83146961230254523708f,
                             0.70710678118654752440f, 0.55557023301960222474f,
                             0.38268343236508977173f, 0.19509032201612826785f};
  const int m = k * (32 / R);
  if (m == 0) return z;
  if (m == 8) return INV ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
  const float c = C32[m], sn = INV ? S32[m] : -S32[m];
  return make_float2(z.x * c - z.y * sn, z.x * sn + z.y * c);
}

template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
  if constexpr (R == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 3) {
    // X1,2 = v0 - (v1 + v2)/2 -+ i (sqrt 3 / 2)(v1 - v2) (forward; inverse conjugate)
    const float2 sm = cadd(v[1], v[2]), df = csub(v[1], v[2]);
    const float2 t = make_float2(v[0].x - 0.5f * sm.x, v[0].y - 0.5f * sm.y);
    const float c = 0.86602540378443865f;
    const float2 r = rot(make_float2(c * df.x, c * df.y), INV);
    v[0] = cadd(v[0], sm);
    v[1] = cadd(t, r);
    v[2] = csub(t, r);
  } else if constexpr (R == 4) {
    const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const float2 s13 = cadd(v[1], v[3]), d13 = rot(csub(v[1], v[3]), INV);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  } else {
    float2 e[R / 2], o[R / 2];
#pragma unroll
    for (int r = 0; r < R / 2; ++r) {
      e[r] = v[2 * r];
      o[r] = v[2 * r + 1];
    }
    dft_reg<R / 2, INV>(e);
    dft_reg<R / 2, INV>(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      const float2 t = wconst<R, INV>(k, o[k]);
      v[k] = cadd(e[k], t);
      v[k + R / 2] = csub(e[k], t);
    }
  }
}

// one Stockham stage of radix R after stages of total radix NS, on nl lines
// of length N (padded rows of LS elements)
template <int N, int NS, int R, bool INV>
__device__ __forceinline__ void fast_stage(const float2* in, float2* out, int nl, const float2* tw) {
  constexpr int M = N / R;
  constexpr int LS = fpad(N);
  for (int t = threadIdx.x; t < nl * M; t += blockDim.x) {
    const int line = t / M, j = t % M;
    const float2* src = in + line * LS;
    float2* dst = out + line * LS;
    const int k = j % NS;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[fpad(j + r * M)];
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = tw[r * k * (N / (NS * R))];
        v[r] = INV ? cmulconj(v[r], w) : cmul(v[r], w);
      }
    }
    dft_reg<R, INV>(v);
    const int base = (j / NS) * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[fpad(base + r * NS)] = v[r];
  }
  __syncthreads();
}

// transform nl lines held in a (b is scratch); returns the buffer with the result
template <int N, bool INV>
__device__ float2* fast_fft(float2* a, float2* b, int nl, const float2* tw) {
  constexpr int R0 = fast_radix(N, 0), R1 = fast_radix(N, 1), R2 = fast_radix(N, 2);
  fast_stage<N, 1, R0, INV>(a, b, nl, tw);
  if constexpr (R1 == 0) {
    return b;
  } else {
    fast_stage<N, R0, R1, INV>(b, a, nl, tw);
    if constexpr (R2 == 0) {
      return a;
    } else {
      fast_stage<N, R0 * R1, R2, INV>(a, b, nl, tw);
      return b;
    }
  }
}

template <int N>
__device__ __forceinline__ void load_twiddles(float2* tw, const AxisPlan& P) {
  for (int k = threadIdx.x; k < N; k += blockDim.x) tw[k] = P.tw32[k];
}

// X pass, forward, rows r0 = 2p, r1 = 2p + 1 packed as a + i b (as k_fft_x_fwd).
// KMAJOR: the half spectrum is stored kx-major, S[kx][z][y], so that each
// (y, z) plane is contiguous for k_fast_yzplane2; else S[z][y][kx].
template <int NX, bool KMAJOR, bool VEC>
__device__ __forceinline__ void fast_x_fwd_body(const PassArgs<float>& a, int bx) {
  constexpr int PPC = FAST_XELEMS / NX > 0 ? FAST_XELEMS / NX : 1;  // row pairs per CTA
  constexpr int LS = fpad(NX);
  __shared__ __align__(16) float2 buf[2][PPC * LS];
  __shared__ float2 tw[NX];
  load_twiddles<NX>(tw, a.ax);
  const int nrows = a.ny * a.nz;
  const long long N = (long long)NX * a.ny * a.nz;
  const int p0 = bx * PPC;
  // every load of the thread is issued before the first shared-memory store:
  // the stores go through no pointer the loads could alias, so the latencies
  // overlap instead of adding up
  if constexpr (VEC) {
    // four consecutive x of one row pair per item
    static_assert(NX % 4 == 0, "16-byte items");
    constexpr int NV = PPC * NX / 4, PER = (NV + FAST_XT - 1) / FAST_XT;
    float4 re[PER], im[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int t = threadIdx.x + q * FAST_XT;
      const int l = t / (NX / 4), x = 4 * (t - l * (NX / 4));
      const int r0 = 2 * (p0 + l), r1 = r0 + 1;
      re[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      im[q] = re[q];
      if (t < NV && r0 < nrows) re[q] = charge_at4(a, (long long)r0 * NX + x, N);
      if (t < NV && r1 < nrows) im[q] = charge_at4(a, (long long)r1 * NX + x, N);
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int t = threadIdx.x + q * FAST_XT;
      if (t < NV) {
        const int l = t / (NX / 4), x = 4 * (t - l * (NX / 4));
        float2* d = &buf[0][l * LS + fpad(x)];  // x .. x + 3 lie in one padding group of 16
        d[0] = make_float2(re[q].x, im[q].x);
        d[1] = make_float2(re[q].y, im[q].y);
        d[2] = make_float2(re[q].z, im[q].z);
        d[3] = make_float2(re[q].w, im[q].w);
      }
    }
  } else {
    constexpr int PER = (PPC * NX + FAST_XT - 1) / FAST_XT;
    float re[PER], im[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int t = threadIdx.x + q * FAST_XT;
      const int l = t / NX, x = t % NX;
      const int r0 = 2 * (p0 + l), r1 = r0 + 1;
      re[q] = 0.0f;
      im[q] = 0.0f;
      if (t < PPC * NX && r0 < nrows) re[q] = charge_at(a, (long long)r0 * NX + x, N);
      if (t < PPC * NX && r1 < nrows) im[q] = charge_at(a, (long long)r1 * NX + x, N);
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int t = threadIdx.x + q * FAST_XT;
      if (t < PPC * NX) buf[0][(t / NX) * LS + fpad(t % NX)] = make_float2(re[q], im[q]);
    }
  }
  __syncthreads();
  const float2* res = fast_fft<NX, false>(buf[0], buf[1], PPC, tw);
  constexpr int NXH = NX / 2 + 1;
  for (int t = threadIdx.x; t < PPC * NXH; t += FAST_XT) {
    // kx-major: consecutive threads take consecutive rows of one kx
    const int l = KMAJOR ? t % PPC : t / NXH, k = KMAJOR ? t / PPC : t % NXH;
    const int r0 = 2 * (p0 + l), r1 = r0 + 1;
    if (r0 >= nrows) continue;
    const float2 Zk = res[l * LS + fpad(k)];
    const float2 Zm = res[l * LS + fpad(k == 0 ? 0 : NX - k)];
    const float2 A = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
    const float2 B = make_float2(0.5f * (Zk.y + Zm.y), -0.5f * (Zk.x - Zm.x));
    if (KMAJOR) {
      a.S[(long long)k * nrows + r0] = A;
      if (r1 < nrows) a.S[(long long)k * nrows + r1] = B;
    } else {
      a.S[(long long)r0 * NXH + k] = A;
      if (r1 < nrows) a.S[(long long)r1 * NXH + k] = B;
    }
  }
}

template <int NX, bool KMAJOR, bool VEC>
__global__ void __launch_bounds__(FAST_XT) k_fast_x_fwd(PassArgs<float> a) {
  fast_x_fwd_body<NX, KMAJOR, VEC>(a, blockIdx.x);
}

// Y (AXIS 1, forward or inverse) or Z (AXIS 2: forward, Green multiply,
// inverse) pass on tiles of tx consecutive kx (as k_fft_yz)
template <int NL, int AXIS, bool INV>
__global__ void __launch_bounds__(FAST_T) k_fast_yz(PassArgs<float> a, int tx) {
  constexpr int LS = fpad(NL);
  __shared__ __align__(16) float2 buf[2][(FAST_ELEMS / NL) * LS];
  __shared__ float2 tw[NL];
  const AxisPlan& P = AXIS == 1 ? a.ay : a.az;
  load_twiddles<NL>(tw, P);
  const int nxh = a.nxh;
  const int ntile = (nxh + tx - 1) / tx;
  const int tile = blockIdx.x % ntile;
  const int other = blockIdx.x / ntile;  // z (axis 1) or ky (axis 2)
  const int kx0 = tile * tx;
  const int nc = min(tx, nxh - kx0);
  const long long stride = AXIS == 1 ? (long long)nxh : (long long)nxh * a.ny;
  const long long base = AXIS == 1 ? (long long)other * a.ny * nxh : (long long)other * nxh;
  {
    // all of the thread's loads before its first shared-memory store
    constexpr int TXMAX = FAST_ELEMS / NL < 16 ? FAST_ELEMS / NL : 16;  // nc <= TXMAX
    constexpr int PER = (TXMAX * NL + FAST_T - 1) / FAST_T;
    float2 v[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int t = threadIdx.x + q * FAST_T;
      const int j = t / nc, c = t - j * nc;
      if (t < nc * NL) v[q] = a.S[base + j * stride + kx0 + c];
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int t = threadIdx.x + q * FAST_T;
      const int j = t / nc, c = t - j * nc;
      if (t < nc * NL) buf[0][c * LS + fpad(j)] = v[q];
    }
  }
  __syncthreads();
  float2* res;
  if constexpr (AXIS == 1) {
    res = fast_fft<NL, INV>(buf[0], buf[1], nc, tw);
  } else {
    res = fast_fft<NL, false>(buf[0], buf[1], nc, tw);
    const float ly = lambda_of(a.ay, other, 0.0f);
    for (int t = threadIdx.x; t < nc * NL; t += FAST_T) {
      const int c = t / NL, j = t % NL;
      const int kx = kx0 + c;
      const float lam = lambda_of(a.ax, kx, 0.0f) + ly + lambda_of(a.az, j, 0.0f);
      const float g = (kx == 0 && other == 0 && j == 0) ? 0.0f : a.green_scale / lam;
      float2& v = res[c * LS + fpad(j)];
      v = make_float2(v.x * g, v.y * g);
    }
    __syncthreads();
    res = fast_fft<NL, true>(res, res == buf[0] ? buf[1] : buf[0], nc, tw);
  }
  for (int t = threadIdx.x; t < nc * NL; t += FAST_T) {
    const int j = t / nc, c = t - j * nc;
    a.S[base + j * stride + kx0 + c] = res[c * LS + fpad(j)];
  }
}

// Y (AXIS 1, forward or inverse) or Z (AXIS 2: forward, Green multiply,
// inverse) pass for lines of NL = 16 N2 points (256, 512) as four-step
// transforms on tiles of TX = 256 / N2 consecutive kx: x[N2 n1 + n2] ->
// X[k1 + 16 k2].  Thread (c, n2) holds the 16 points n1 of its line in
// registers, transforms them, multiplies by the twiddle exp(-+2 pi i n2 k1 / NL)
// and writes them to shared memory; after one barrier thread (c, k1) reads the
// N2 points n2 and transforms them.  The Z pass keeps the result in
// registers for the Green multiply and runs the inverse the same way back.
// The shared layout c + TX (n2 + N2 k1) makes both the writes and the reads
// of a warp contiguous.
template <int NL, int AXIS, bool INV>
__global__ void __launch_bounds__(256) k_line4(PassArgs<float> a) {
  constexpr int N1 = 16, N2 = NL / 16, TX = 256 / N2;
  __shared__ __align__(16) float2 T[TX * NL];
  __shared__ float2 tw[NL];
  const AxisPlan& P = AXIS == 1 ? a.ay : a.az;
  load_twiddles<NL>(tw, P);
  const int nxh = a.nxh;
  const int ntile = (nxh + TX - 1) / TX;
  const int tile = blockIdx.x % ntile;
  const int other = blockIdx.x / ntile;  // z (axis 1) or ky (axis 2)
  const int kx0 = tile * TX;
  const long long stride = AXIS == 1 ? (long long)nxh : (long long)nxh * a.ny;
  const long long base = (AXIS == 1 ? (long long)other * a.ny * nxh : (long long)other * nxh) + kx0;
  const int t = threadIdx.x;
  const int c = t % TX;
  const bool col = kx0 + c < nxh;
  constexpr bool FINV = AXIS == 1 && INV;  // direction of the first transform
  {
    // thread (c, n2): the 16 points x[N2 n1 + n2]
    const int n2 = t / TX;
    float2 v[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1)
      v[n1] = col ? a.S[base + (long long)(N2 * n1 + n2) * stride + c] : make_float2(0.0f, 0.0f);
    __syncthreads();  // the twiddles
    dft_reg<N1, FINV>(v);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const float2 w = tw[n2 * k1];
      T[c + TX * (n2 + N2 * k1)] = FINV ? cmulconj(v[k1], w) : cmul(v[k1], w);
    }
  }
  __syncthreads();
  if (t < TX * N1) {
    // thread (c, k1): the N2 points n2, giving X[k1 + 16 k2]
    const int k1 = t / TX;
    float2 z[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) z[n2] = T[c + TX * (n2 + N2 * k1)];
    dft_reg<N2, FINV>(z);
    if constexpr (AXIS == 1) {
      if (col) {
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) a.S[base + (long long)(k1 + N1 * k2) * stride + c] = z[k2];
      }
      return;
    } else {
      const int kx = kx0 + c;
      const float lxy = lambda_of(a.ax, col ? kx : 0, 0.0f) + lambda_of(a.ay, other, 0.0f);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int j = k1 + N1 * k2;
        const float lam = lxy + lambda_of(a.az, j, 0.0f);
        const float g = (kx == 0 && other == 0 && j == 0) ? 0.0f : a.green_scale / lam;
        z[k2] = make_float2(z[k2].x * g, z[k2].y * g);
      }
      // back: the N2 points k2 of this k1, then the twiddle
      dft_reg<N2, true>(z);
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) T[c + TX * (n2 + N2 * k1)] = cmulconj(z[n2], tw[n2 * k1]);
    }
  }
  if constexpr (AXIS == 2) {
    __syncthreads();
    const int n2 = t / TX;
    float2 v[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = T[c + TX * (n2 + N2 * k1)];
    dft_reg<N1, true>(v);
    if (col) {
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) a.S[base + (long long)(N2 * n1 + n2) * stride + c] = v[n1];
    }
  }
}

template <int NL, int AXIS, bool INV>
void launch_line4(PassArgs<float>& a, cudaStream_t s) {
  constexpr int TX = 256 / (NL / 16);
  const int ntile = (a.nxh + TX - 1) / TX;
  const int nother = AXIS == 1 ? a.nz : a.ny;
  k_line4<NL, AXIS, INV><<<(unsigned)(ntile * nother), 256, 0, s>>>(a);
}

// X pass, inverse (complex-to-real), two rows per complex transform (as k_fft_x_inv).
// Each stored coefficient kk <= NX / 2 is loaded once and gives the inputs k = kk
// and, conjugated, k = NX - kk; the thread's loads are all issued before its
// first shared-memory store.
template <int NX, bool KMAJOR>
__device__ __forceinline__ void fast_x_inv_body(const PassArgs<float>& a, int bx) {
  constexpr int PPC = FAST_IELEMS / NX > 0 ? FAST_IELEMS / NX : 1;
  constexpr int LS = fpad(NX);
  constexpr int NXH = NX / 2 + 1;
  constexpr int PER = (PPC * NXH + FAST_IT - 1) / FAST_IT;
  __shared__ __align__(16) float2 buf[2][PPC * LS];
  __shared__ float2 tw[NX];
  load_twiddles<NX>(tw, a.ax);
  const int nrows = a.ny * a.nz;
  const int p0 = bx * PPC;
  float2 A[PER], B[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int t = threadIdx.x + q * FAST_IT;
    const int l = KMAJOR ? t % PPC : t / NXH, kk = KMAJOR ? t / PPC : t % NXH;
    const int r0 = 2 * (p0 + l), r1 = r0 + 1;
    A[q] = make_float2(0.0f, 0.0f);
    B[q] = A[q];
    if (t < PPC * NXH) {
      if (KMAJOR) {
        if (r0 < nrows) A[q] = a.S[(long long)kk * nrows + r0];
        if (r1 < nrows) B[q] = a.S[(long long)kk * nrows + r1];
      } else {
        if (r0 < nrows) A[q] = a.S[(long long)r0 * NXH + kk];
        if (r1 < nrows) B[q] = a.S[(long long)r1 * NXH + kk];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int t = threadIdx.x + q * FAST_IT;
    if (t < PPC * NXH) {
      const int l = KMAJOR ? t % PPC : t / NXH, kk = KMAJOR ? t / PPC : t % NXH;
      buf[0][l * LS + fpad(kk)] = make_float2(A[q].x - B[q].y, A[q].y + B[q].x);
      if (kk > 0 && kk < NX - NXH + 1) {  // 0 < kk < NX / 2: the upper half, conjugated
        const float2 Ac = make_float2(A[q].x, -A[q].y), Bc = make_float2(B[q].x, -B[q].y);
        buf[0][l * LS + fpad(NX - kk)] = make_float2(Ac.x - Bc.y, Ac.y + Bc.x);
      }
    }
  }
  __syncthreads();
  const float2* res = fast_fft<NX, true>(buf[0], buf[1], PPC, tw);
  for (int t = threadIdx.x; t < PPC * NX; t += FAST_IT) {
    const int l = t / NX, x = t % NX;
    const int r0 = 2 * (p0 + l), r1 = r0 + 1;
    const float2 v = res[l * LS + fpad(x)];
    if (r0 < nrows) a.phi[(long long)r0 * NX + x] = v.x;
    if (r1 < nrows) a.phi[(long long)r1 * NX + x] = v.y;
  }
}

template <int NX, bool KMAJOR>
__global__ void __launch_bounds__(FAST_IT) k_fast_x_inv(PassArgs<float> a) {
  fast_x_inv_body<NX, KMAJOR>(a, blockIdx.x);
}

template <int NX>
void launch_fast_x(PassArgs<float>& a, bool inverse, bool kmajor, cudaStream_t s) {
  const int npairs = (a.ny * a.nz + 1) / 2;
  if (inverse) {
    constexpr int ppc = FAST_IELEMS / NX > 0 ? FAST_IELEMS / NX : 1;
    const unsigned g = (unsigned)((npairs + ppc - 1) / ppc);
    if (kmajor) k_fast_x_inv<NX, true><<<g, FAST_IT, 0, s>>>(a);
    else k_fast_x_inv<NX, false><<<g, FAST_IT, 0, s>>>(a);
  } else {
    constexpr int ppc = FAST_XELEMS / NX > 0 ? FAST_XELEMS / NX : 1;
    const unsigned g = (unsigned)((npairs + ppc - 1) / ppc);
    // 16-byte loads when every charge array is 16-byte aligned (N % 4 == 0: NX % 4 == 0)
    const auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    const bool vec = al(a.q) && al(a.rho) && al(a.qwall) && al(a.qpart);
    if (vec) {
      if (kmajor) k_fast_x_fwd<NX, true, true><<<g, FAST_XT, 0, s>>>(a);
      else k_fast_x_fwd<NX, false, true><<<g, FAST_XT, 0, s>>>(a);
    } else {
      if (kmajor) k_fast_x_fwd<NX, true, false><<<g, FAST_XT, 0, s>>>(a);
      else k_fast_x_fwd<NX, false, false><<<g, FAST_XT, 0, s>>>(a);
    }
  }
}

template <int NL, int AXIS, bool INV>
void launch_fast_yz_n(PassArgs<float>& a, cudaStream_t s) {
  // tiles of at most FAST_ELEMS / NL (<= 16) columns, balanced over nxh
  const int txmax = std::min(16, FAST_ELEMS / NL);
  const int ntile = (a.nxh + txmax - 1) / txmax;
  const int tx = (a.nxh + ntile - 1) / ntile;
  const int nother = AXIS == 1 ? a.nz : a.ny;
  k_fast_yz<NL, AXIS, INV><<<(unsigned)(ntile * nother), FAST_T, 0, s>>>(a, tx);
}

template <int AXIS, bool INV>
void launch_fast_yz(PassArgs<float>& a, int n, cudaStream_t s) {
  switch (n) {
    case 24: launch_fast_yz_n<24, AXIS, INV>(a, s); break;
    case 32: launch_fast_yz_n<32, AXIS, INV>(a, s); break;
    case 48: launch_fast_yz_n<48, AXIS, INV>(a, s); break;
    case 64: launch_fast_yz_n<64, AXIS, INV>(a, s); break;
    case 96: launch_fast_yz_n<96, AXIS, INV>(a, s); break;
    case 128: launch_fast_yz_n<128, AXIS, INV>(a, s); break;
    case 192: launch_fast_yz_n<192, AXIS, INV>(a, s); break;
    case 256: launch_line4<256, AXIS, INV>(a, s); break;
    case 384: launch_fast_yz_n<384, AXIS, INV>(a, s); break;
    default: launch_line4<512, AXIS, INV>(a, s); break;
  }
}

void launch_fast_x_any(PassArgs<float>& a, bool inverse, bool kmajor, cudaStream_t s) {
  switch (a.nx) {
    case 24: launch_fast_x<24>(a, inverse, kmajor, s); break;
    case 32: launch_fast_x<32>(a, inverse, kmajor, s); break;
    case 48: launch_fast_x<48>(a, inverse, kmajor, s); break;
    case 64: launch_fast_x<64>(a, inverse, kmajor, s); break;
    case 96: launch_fast_x<96>(a, inverse, kmajor, s); break;
    case 128: launch_fast_x<128>(a, inverse, kmajor, s); break;
    case 192: launch_fast_x<192>(a, inverse, kmajor, s); break;
    case 256: launch_fast_x<256>(a, inverse, kmajor, s); break;
    case 384: launch_fast_x<384>(a, inverse, kmajor, s); break;
    default: launch_fast_x<512>(a, inverse, kmajor, s); break;
  }
}

// ---------------------------------------------------------------------------
// The y and z passes of one kx plane in one kernel: when a (y, z) plane of the
// kx-major half spectrum fits in the shared memory of two CTAs (edges
// 32..128), a cluster of two loads it (contiguous), transforms along y and z,
// multiplies by the Green function, transforms back and stores it: three
// kernels and four round trips through L2 become one.  Each stage runs in
// place: every thread reads its sub-transforms' elements into registers, the
// block synchronises, then every thread writes its results.
// ---------------------------------------------------------------------------

// E contiguous elements of the spectrum (rows of NY) to and from the padded
// shared-memory layout, in batches of up to 8 per thread whose global loads
// (or shared-memory loads) are all issued before the first store
template <int E, int NY, int LS, int T>
__device__ __forceinline__ void plane_load(const float2* __restrict__ src, float2* pl) {
  constexpr int PER = (E + T - 1) / T, B = PER < 8 ? PER : 8;
#pragma unroll
  for (int q0 = 0; q0 < PER; q0 += B) {
    float2 v[B];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int e = threadIdx.x + (q0 + q) * T;
      if (q0 + q < PER && e < E) v[q] = src[e];
    }
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int e = threadIdx.x + (q0 + q) * T;
      if (q0 + q < PER && e < E) pl[(e / NY) * LS + fpad(e % NY)] = v[q];
    }
  }
}
template <int E, int NY, int LS, int T>
__device__ __forceinline__ void plane_store(const float2* pl, float2* __restrict__ dst) {
  constexpr int PER = (E + T - 1) / T, B = PER < 8 ? PER : 8;
#pragma unroll
  for (int q0 = 0; q0 < PER; q0 += B) {
    float2 v[B];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int e = threadIdx.x + (q0 + q) * T;
      if (q0 + q < PER && e < E) v[q] = pl[(e / NY) * LS + fpad(e % NY)];
    }
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int e = threadIdx.x + (q0 + q) * T;
      if (q0 + q < PER && e < E) dst[e] = v[q];
    }
  }
}

// one in-place Stockham stage of radix R over the lines of the plane.  Along
// y (ALONG_Y): NLINES = NZ lines of length N = NY, element (line, i) at
// line * LSY + fpad(i); along z: NY lines of length NZ, element (line, i) at
// i * LSY + fpad(line), consecutive threads on consecutive lines.
template <int N, int NLINES, int NS, int R, bool INV, bool ALONG_Y, int LSY, int T>
__device__ __forceinline__ void plane_stage(float2* pl, const float2* tw) {
  constexpr int M = N / R;
  constexpr int ITEMS = NLINES * M;
  constexpr int PER = (ITEMS + T - 1) / T;
  float2 v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int t = threadIdx.x + q * T;
    if (t < ITEMS) {
      const int line = ALONG_Y ? t / M : t % NLINES, j = ALONG_Y ? t % M : t / NLINES;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = j + r * M;
        v[q][r] = ALONG_Y ? pl[line * LSY + fpad(i)] : pl[i * LSY + fpad(line)];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int t = threadIdx.x + q * T;
    if (t < ITEMS) {
      const int line = ALONG_Y ? t / M : t % NLINES, j = ALONG_Y ? t % M : t / NLINES;
      const int k = j % NS;
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const float2 w = tw[r * k * (N / (NS * R))];
          v[q][r] = INV ? cmulconj(v[q][r], w) : cmul(v[q][r], w);
        }
      }
      dft_reg<R, INV>(v[q]);
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = base + r * NS;
        if (ALONG_Y) pl[line * LSY + fpad(i)] = v[q][r];
        else pl[i * LSY + fpad(line)] = v[q][r];
      }
    }
  }
  __syncthreads();
}

template <int N, int NLINES, bool INV, bool ALONG_Y, int LSY, int T>
__device__ __forceinline__ void plane_fft(float2* pl, const float2* tw) {
  constexpr int R0 = fast_radix(N, 0), R1 = fast_radix(N, 1), R2 = fast_radix(N, 2);
  plane_stage<N, NLINES, 1, R0, INV, ALONG_Y, LSY, T>(pl, tw);
  if constexpr (R1 != 0) plane_stage<N, NLINES, R0, R1, INV, ALONG_Y, LSY, T>(pl, tw);
  if constexpr (R2 != 0) plane_stage<N, NLINES, R0 * R1, R2, INV, ALONG_Y, LSY, T>(pl, tw);
}

// Two CTAs per plane use twice the SMs of one (nx / 2 + 1 CTAs would leave
// most SMs idle at edges <= 128).  CTA r loads z lines [r NZ/2, (r+1) NZ/2) and transforms them along y into
// `pa` ([z][y]); each CTA then writes every element to the CTA that owns its
// y half (distributed shared memory), into `pb` ([z][y - r NY/2], all z), so
// that CTA r transforms y lines [r NY/2, (r+1) NY/2) along z, multiplies by the
// Green function and transforms back; a second exchange returns the z halves
// for the inverse y transform.  Every line goes through the same stages as
// in a one-CTA transform of the plane.  A cluster barrier separates
// each exchange from the reads that follow it; no CTA touches the peer's
// shared memory after the last one, so either may exit first.
constexpr int PLANE2_T = 512;

template <int NY, int NZ>
__device__ __forceinline__ void fast_yzplane2_body(const PassArgs<float>& a, int bx) {
  constexpr int HZ = NZ / 2, HY = NY / 2;
  constexpr int LSA = fpad(NY), LSB = fpad(HY);
  extern __shared__ __align__(16) unsigned char plane_smem[];
  float2* pa = reinterpret_cast<float2*>(plane_smem);  // [z - r HZ][y], HZ rows
  float2* pb = pa + HZ * LSA;                          // [z][y - r HY], NZ rows
  float2* twy = pb + NZ * LSB;
  float2* twz = twy + NY;
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  cl.barrier_arrive();  // the peer has started before its shared memory is written
  const int kx = bx >> 1;
  for (int k = threadIdx.x; k < NY; k += PLANE2_T) twy[k] = a.ay.tw32[k];
  for (int k = threadIdx.x; k < NZ; k += PLANE2_T) twz[k] = a.az.tw32[k];
  const float2* src = a.S + (long long)kx * NY * NZ + (long long)r * HZ * NY;
  plane_load<HZ * NY, NY, LSA, PLANE2_T>(src, pa);
  __syncthreads();
  plane_fft<NY, HZ, false, true, LSA, PLANE2_T>(pa, twy);
  float2* const pb0 = cl.map_shared_rank(pb, 0);
  float2* const pb1 = cl.map_shared_rank(pb, 1);
  cl.barrier_wait();
#pragma unroll 4
  for (int e = threadIdx.x; e < HZ * NY; e += PLANE2_T) {
    const int zl = e / NY, y = e % NY, o = y / HY;
    (o ? pb1 : pb0)[(r * HZ + zl) * LSB + fpad(y - o * HY)] = pa[zl * LSA + fpad(y)];
  }
  cl.sync();
  plane_fft<NZ, HY, false, false, LSB, PLANE2_T>(pb, twz);
  const float lx = lambda_of(a.ax, kx, 0.0f);
  for (int e = threadIdx.x; e < NZ * HY; e += PLANE2_T) {
    const int z = e / HY, yl = e % HY, y = r * HY + yl;
    const float lam = lx + lambda_of(a.ay, y, 0.0f) + lambda_of(a.az, z, 0.0f);
    const float g = (kx == 0 && y == 0 && z == 0) ? 0.0f : a.green_scale / lam;
    float2& v = pb[z * LSB + fpad(yl)];
    v = make_float2(v.x * g, v.y * g);
  }
  __syncthreads();
  plane_fft<NZ, HY, true, false, LSB, PLANE2_T>(pb, twz);
  float2* const pa0 = cl.map_shared_rank(pa, 0);
  float2* const pa1 = cl.map_shared_rank(pa, 1);
#pragma unroll 4
  for (int e = threadIdx.x; e < NZ * HY; e += PLANE2_T) {
    const int z = e / HY, yl = e % HY, o = z / HZ;
    (o ? pa1 : pa0)[(z - o * HZ) * LSA + fpad(r * HY + yl)] = pb[z * LSB + fpad(yl)];
  }
  cl.sync();
  plane_fft<NY, HZ, true, true, LSA, PLANE2_T>(pa, twy);
  plane_store<HZ * NY, NY, LSA, PLANE2_T>(pa, a.S + (long long)kx * NY * NZ + (long long)r * HZ * NY);
}

template <int NY, int NZ>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PLANE2_T, 1)
    k_fast_yzplane2(PassArgs<float> a) {
  fast_yzplane2_body<NY, NZ>(a, blockIdx.x);
}

template <int NY, int NZ>
constexpr size_t plane2_smem_bytes() {
  return ((size_t)(NZ / 2) * fpad(NY) + (size_t)NZ * fpad(NY / 2) + NY + NZ) * sizeof(float2);
}

// the plane kernels that exist: NY, NZ in {32, 48, 64, 128}
inline bool plane_edge(int n) { return n == 32 || n == 48 || n == 64 || n == 128; }

template <int NY, int NZ>
cudaError_t launch_plane_nn(PassArgs<float>& a, cudaStream_t s) {
  k_fast_yzplane2<NY, NZ><<<2 * (unsigned)a.nxh, PLANE2_T, plane2_smem_bytes<NY, NZ>(), s>>>(a);
  return cudaGetLastError();
}

template <int NY>
cudaError_t launch_plane_n(PassArgs<float>& a, cudaStream_t s) {
  switch (a.nz) {
    case 32: return launch_plane_nn<NY, 32>(a, s);
    case 48: return launch_plane_nn<NY, 48>(a, s);
    case 64: return launch_plane_nn<NY, 64>(a, s);
    default: return launch_plane_nn<NY, 128>(a, s);
  }
}

cudaError_t launch_plane(PassArgs<float>& a, cudaStream_t s) {
  switch (a.ny) {
    case 32: return launch_plane_n<32>(a, s);
    case 48: return launch_plane_n<48>(a, s);
    case 64: return launch_plane_n<64>(a, s);
    default: return launch_plane_n<128>(a, s);
  }
}

template <int NY, int NZ>
cudaError_t plane_attr_nn() {
  return cudaFuncSetAttribute(k_fast_yzplane2<NY, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)plane2_smem_bytes<NY, NZ>());
}
template <int NY>
cudaError_t plane_attr_n() {
  cudaError_t e = plane_attr_nn<NY, 32>();
  if (e == cudaSuccess) e = plane_attr_nn<NY, 48>();
  if (e == cudaSuccess) e = plane_attr_nn<NY, 64>();
  if (e == cudaSuccess) e = plane_attr_nn<NY, 128>();
  return e;
}

template <class FM>
__global__ void k_charge(Grid g, Phys ph, const void* rho, const void* qwall, const void* qpart,
                         double* q) {
  using spc_t = typename FM::spc_t;
  using real_t = typename FM::real_t;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  double s = 0.0;
  for (int k = 0; k < ph.K; ++k) {
    const double r = (double)((const spc_t*)rho)[k * g.N + n];
    s += ph.z[k] * (FM::fp32 ? r * ph.qscale[k] : r);
  }
  if (qwall) s += (double)((const real_t*)qwall)[n];
  if (qpart) s += (double)((const real_t*)qpart)[n];
  q[n] = s;
}

bool factor(int n, AxisPlan& P) {
  P.n = n;
  P.nrad = 0;
  int m = n;
  while (m % 4 == 0) { P.radix[P.nrad++] = 4; m /= 4; }
  while (m % 2 == 0) { P.radix[P.nrad++] = 2; m /= 2; }
  while (m % 3 == 0) { P.radix[P.nrad++] = 3; m /= 3; }
  return m == 1 && P.nrad <= 16;
}

cudaError_t axis_create(AxisPlan& P, int n) {
  std::vector<double2> tw(n);
  std::vector<double> lam(n);
  std::vector<float2> tw32(n);
  std::vector<float> lam32(n);
  for (int k = 0; k < n; ++k) {
    const double ang = 2.0 * M_PI * (double)k / (double)n;
    tw[k] = make_double2(cos(ang), -sin(ang));
    lam[k] = 2.0 - 2.0 * cos(ang);
    tw32[k] = make_float2((float)tw[k].x, (float)tw[k].y);
    lam32[k] = (float)lam[k];
  }
  cudaError_t e = cudaMalloc(&P.tw, n * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&P.lam, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&P.tw32, n * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&P.lam32, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(P.tw, tw.data(), n * sizeof(double2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(P.lam, lam.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(P.tw32, tw32.data(), n * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(P.lam32, lam32.data(), n * sizeof(float), cudaMemcpyHostToDevice);
  return e;
}


// ---------------------------------------------------------------------------
// S1 of the FP32 systems of a batch.  A system whose edges are all 32, 48 or
// 64 runs its three passes (x forward, the y-z planes, x inverse) in launches
// shared with the other systems of the same kernel variant; the bodies are
// those of the single-system kernels, so the results are the same.
// ---------------------------------------------------------------------------
template <int NX, bool VEC>
__global__ void __launch_bounds__(FAST_XT) k_fast_x_fwd_batch(const PassArgs<float>* __restrict__ tab,
                                                              const BatchSlot* __restrict__ sl, int nsys) {
  int sys;
  const Blk bk = batch_blk(sl, nsys, sys);
  fast_x_fwd_body<NX, true, VEC>(tab[sys], bk.x);
}

template <int NX>
__global__ void __launch_bounds__(FAST_IT) k_fast_x_inv_batch(const PassArgs<float>* __restrict__ tab,
                                                              const BatchSlot* __restrict__ sl, int nsys) {
  int sys;
  const Blk bk = batch_blk(sl, nsys, sys);
  fast_x_inv_body<NX, true>(tab[sys], bk.x);
}

// every system's range is 2 nxh CTAs and starts at an even CTA, so a cluster
// (two consecutive CTAs) lies in one system and its rank is the block's parity
template <int NY, int NZ>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PLANE2_T, 1)
    k_fast_yzplane2_batch(const PassArgs<float>* __restrict__ tab, const BatchSlot* __restrict__ sl,
                          int nsys) {
  int sys;
  const Blk bk = batch_blk(sl, nsys, sys);
  fast_yzplane2_body<NY, NZ>(tab[sys], bk.x);
}

inline bool batch_edge(int n) { return n == 32 || n == 48 || n == 64; }

template <int NX>
int fast_x_ctas(int ny, int nz, bool inverse) {
  const int npairs = (ny * nz + 1) / 2;
  constexpr int pf = FAST_XELEMS / NX > 0 ? FAST_XELEMS / NX : 1;
  constexpr int pi = FAST_IELEMS / NX > 0 ? FAST_IELEMS / NX : 1;
  const int ppc = inverse ? pi : pf;
  return (npairs + ppc - 1) / ppc;
}

template <int NY, int NZ>
cudaError_t plane_batch_launch(const PassArgs<float>* tab, const BatchSlot* sl, int nsys, int ctas,
                               cudaStream_t s) {
  k_fast_yzplane2_batch<NY, NZ><<<(unsigned)ctas, PLANE2_T, plane2_smem_bytes<NY, NZ>(), s>>>(tab, sl, nsys);
  return cudaGetLastError();
}

template <int NY, int NZ>
cudaError_t plane_batch_attr_nn() {
  return cudaFuncSetAttribute(k_fast_yzplane2_batch<NY, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)plane2_smem_bytes<NY, NZ>());
}
template <int NY>
cudaError_t plane_batch_attr_n() {
  cudaError_t e = plane_batch_attr_nn<NY, 32>();
  if (e == cudaSuccess) e = plane_batch_attr_nn<NY, 48>();
  if (e == cudaSuccess) e = plane_batch_attr_nn<NY, 64>();
  return e;
}
}  // namespace

bool poisson_factor(int n, AxisPlan& P) { return factor(n, P); }

size_t poisson_spectrum_bytes(int nx, int ny, int nz) {
  return (size_t)(nx / 2 + 1) * (size_t)ny * (size_t)nz * sizeof(double2);
}

cudaError_t poisson_plan_create(PoissonPlan& p, int nx, int ny, int nz, std::string& err) {
  p = PoissonPlan();
  // the y-z plane kernels keep a whole plane in shared memory (up to 141 KB);
  // set once per plan, before any launch or stream capture
  {
    cudaError_t e = plane_attr_n<32>();
    if (e == cudaSuccess) e = plane_attr_n<48>();
    if (e == cudaSuccess) e = plane_attr_n<64>();
    if (e == cudaSuccess) e = plane_attr_n<128>();
    if (e == cudaSuccess) e = plane_batch_attr_n<32>();
    if (e == cudaSuccess) e = plane_batch_attr_n<48>();
    if (e == cudaSuccess) e = plane_batch_attr_n<64>();
    if (e != cudaSuccess) {
      err = "shared-memory size of the plane FFT kernels could not be set";
      return e;
    }
  }
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  if (nx % 2 != 0 || nx > LINE_ELEMS || ny > LINE_ELEMS || nz > LINE_ELEMS || nx < 2 ||
      !factor(nx, p.ax) || !factor(ny, p.ay) || !factor(nz, p.az)) {
    err = "box edges must be 2^a 3^b (nx even), at most 1024";
    return cudaErrorInvalidValue;
  }
  cudaError_t e = axis_create(p.ax, nx);
  if (e == cudaSuccess) e = axis_create(p.ay, ny);
  if (e == cudaSuccess) e = axis_create(p.az, nz);
  if (e != cudaSuccess) {
    poisson_plan_destroy(p);
    err = "allocating FFT tables failed";
    return e;
  }
  p.ok = true;
  return cudaSuccess;
}

void poisson_plan_destroy(PoissonPlan& p) {
  for (AxisPlan* a : {&p.ax, &p.ay, &p.az}) {
    if (a->tw) cudaFree(a->tw);
    if (a->lam) cudaFree(a->lam);
    if (a->tw32) cudaFree(a->tw32);
    if (a->lam32) cudaFree(a->lam32);
    a->tw = nullptr;
    a->lam = nullptr;
    a->tw32 = nullptr;
    a->lam32 = nullptr;
  }
  p.ok = false;
}

namespace {

template <typename R>
cudaError_t run_passes(const PoissonPlan& p, PassArgs<R>& a, double bjerrum, cudaStream_t s) {
  using C = typename CT<R>::type;
  a.nx = p.nx;
  a.ny = p.ny;
  a.nz = p.nz;
  a.nxh = p.nx / 2 + 1;
  a.ax = p.ax;
  a.ay = p.ay;
  a.az = p.az;
  const double N = (double)p.nx * p.ny * p.nz;
  a.green_scale = (R)(4.0 * M_PI * bjerrum / N);
  if constexpr (std::is_same<R, float>::value) {
    if (fast_edge(p.nx) && fast_edge(p.ny) && fast_edge(p.nz)) {
      if (plane_edge(p.ny) && plane_edge(p.nz)) {
        launch_fast_x_any(a, false, true, s);
        launch_plane(a, s);
        launch_fast_x_any(a, true, true, s);
        return cudaGetLastError();
      }
      launch_fast_x_any(a, false, false, s);
      launch_fast_yz<1, false>(a, p.ny, s);
      launch_fast_yz<2, false>(a, p.nz, s);
      launch_fast_yz<1, true>(a, p.ny, s);
      launch_fast_x_any(a, true, false, s);
      return cudaGetLastError();
    }
  }
  const int nrows = p.ny * p.nz;
  const int npairs = (nrows + 1) / 2;
  const int ppc = LINE_ELEMS / p.nx > 0 ? LINE_ELEMS / p.nx : 1;
  const unsigned gx = (unsigned)((npairs + ppc - 1) / ppc);
  const size_t smx = 2 * (size_t)ppc * p.nx * sizeof(C);
  k_fft_x_fwd<R><<<gx, FFT_THREADS, smx, s>>>(a, ppc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int txy = LINE_ELEMS / p.ny > 16 ? 16 : (LINE_ELEMS / p.ny > 0 ? LINE_ELEMS / p.ny : 1);
  const int txz = LINE_ELEMS / p.nz > 16 ? 16 : (LINE_ELEMS / p.nz > 0 ? LINE_ELEMS / p.nz : 1);
  const unsigned gy = (unsigned)(((a.nxh + txy - 1) / txy) * p.nz);
  const unsigned gz = (unsigned)(((a.nxh + txz - 1) / txz) * p.ny);
  const size_t smy = 2 * (size_t)txy * p.ny * sizeof(C);
  const size_t smz = 2 * (size_t)txz * p.nz * sizeof(C);
  k_fft_yz<R><<<gy, FFT_THREADS, smy, s>>>(a, 1, txy, false);
  k_fft_yz<R><<<gz, FFT_THREADS, smz, s>>>(a, 2, txz, false);
  k_fft_yz<R><<<gy, FFT_THREADS, smy, s>>>(a, 1, txy, true);
  k_fft_x_inv<R><<<gx, FFT_THREADS, smx, s>>>(a, ppc);
  return cudaGetLastError();
}

}  // namespace

int poisson_kernel_count(const PoissonPlan& p, bool fp32) {
  if (fp32 && fast_edge(p.nx) && fast_edge(p.ny) && fast_edge(p.nz) && plane_edge(p.ny) &&
      plane_edge(p.nz))
    return 3;  // x, the y-z plane kernel, inverse x
  return 5;    // x, y, z (with the Green multiply and the inverse z), inverse y, inverse x
}

cudaError_t poisson_solve(const PoissonPlan& p, const double* q, const double* rho,
                          const double* qwall, const double* qpart, const Phys& ph,
                          double* phi, double2* spectrum, cudaStream_t s) {
  PassArgs<double> a;
  a.q = q;
  a.rho = rho;
  a.int_species = false;
  a.qwall = qwall;
  a.qpart = qpart;
  a.K = ph.K;
  for (int k = 0; k < EK_MAX_SPECIES; ++k) a.z[k] = ph.z[k];
  a.S = spectrum;
  a.phi = phi;
  return run_passes<double>(p, a, ph.bjerrum, s);
}

cudaError_t poisson_solve_f32(const PoissonPlan& p, const int* rho, const float* qwall,
                              const float* qpart, const Phys& ph, float* phi, float2* spectrum,
                              cudaStream_t s) {
  PassArgs<float> a;
  a.q = nullptr;
  a.rho = rho;
  a.int_species = true;
  a.qwall = qwall;
  a.qpart = qpart;
  a.K = ph.K;
  for (int k = 0; k < EK_MAX_SPECIES; ++k) a.z[k] = (float)(ph.z[k] * ph.qscale[k]);
  a.S = spectrum;
  a.phi = phi;
  return run_passes<float>(p, a, ph.bjerrum, s);
}

bool poisson_batch_ok(const PoissonPlan& p) {
  return batch_edge(p.nx) && batch_edge(p.ny) && batch_edge(p.nz);
}

size_t poisson_batch_args_size() { return sizeof(PassArgs<float>); }

void poisson_batch_args(void* out, const PoissonPlan& p, const int* rho, const float* qwall,
                        const float* qpart, const Phys& ph, float* phi, float2* spectrum) {
  PassArgs<float> a;
  a.nx = p.nx;
  a.ny = p.ny;
  a.nz = p.nz;
  a.nxh = p.nx / 2 + 1;
  a.ax = p.ax;
  a.ay = p.ay;
  a.az = p.az;
  a.q = nullptr;
  a.rho = rho;
  a.int_species = true;
  a.qwall = qwall;
  a.qpart = qpart;
  a.K = ph.K;
  for (int k = 0; k < EK_MAX_SPECIES; ++k) a.z[k] = (float)(ph.z[k] * ph.qscale[k]);
  a.S = spectrum;
  a.phi = phi;
  const double N = (double)p.nx * p.ny * p.nz;
  a.green_scale = (float)(4.0 * M_PI * ph.bjerrum / N);
  memcpy(out, &a, sizeof(a));
}

void poisson_batch_pass(const PoissonPlan& p, int pass, const void* args, int& variant, int& ctas) {
  const PassArgs<float>& a = *(const PassArgs<float>*)args;
  variant = -1;
  ctas = 0;
  if (!poisson_batch_ok(p)) return;
  if (pass == 1) {
    variant = p.ny * 256 + p.nz;
    ctas = 2 * (p.nx / 2 + 1);
    return;
  }
  const bool inverse = pass == 2;
  ctas = p.nx == 32 ? fast_x_ctas<32>(p.ny, p.nz, inverse)
                    : (p.nx == 48 ? fast_x_ctas<48>(p.ny, p.nz, inverse) : fast_x_ctas<64>(p.ny, p.nz, inverse));
  const auto al = [](const void* q) { return ((uintptr_t)q & 15) == 0; };
  const bool vec = al(a.q) && al(a.rho) && al(a.qwall) && al(a.qpart);
  variant = inverse ? p.nx : 2 * p.nx + (vec ? 1 : 0);
}

cudaError_t launch_poisson_batch(int pass, int variant, const void* tab, const BatchSlot* slot, int nsys,
                                 int ctas, cudaStream_t s) {
  if (ctas == 0) return cudaSuccess;
  const PassArgs<float>* t = (const PassArgs<float>*)tab;
  const unsigned n = (unsigned)ctas;
  if (pass == 0) {
    switch (variant) {
      case 64: k_fast_x_fwd_batch<32, false><<<n, FAST_XT, 0, s>>>(t, slot, nsys); break;
      case 65: k_fast_x_fwd_batch<32, true><<<n, FAST_XT, 0, s>>>(t, slot, nsys); break;
      case 96: k_fast_x_fwd_batch<48, false><<<n, FAST_XT, 0, s>>>(t, slot, nsys); break;
      case 97: k_fast_x_fwd_batch<48, true><<<n, FAST_XT, 0, s>>>(t, slot, nsys); break;
      case 128: k_fast_x_fwd_batch<64, false><<<n, FAST_XT, 0, s>>>(t, slot, nsys); break;
      case 129: k_fast_x_fwd_batch<64, true><<<n, FAST_XT, 0, s>>>(t, slot, nsys); break;
      default: return cudaErrorInvalidValue;
    }
  } else if (pass == 2) {
    switch (variant) {
      case 32: k_fast_x_inv_batch<32><<<n, FAST_IT, 0, s>>>(t, slot, nsys); break;
      case 48: k_fast_x_inv_batch<48><<<n, FAST_IT, 0, s>>>(t, slot, nsys); break;
      case 64: k_fast_x_inv_batch<64><<<n, FAST_IT, 0, s>>>(t, slot, nsys); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (variant) {
#define EK_PLANE(NY, NZ) \
  case NY * 256 + NZ: return plane_batch_launch<NY, NZ>(t, slot, nsys, ctas, s);
      EK_PLANE(32, 32) EK_PLANE(32, 48) EK_PLANE(32, 64)
      EK_PLANE(48, 32) EK_PLANE(48, 48) EK_PLANE(48, 64)
      EK_PLANE(64, 32) EK_PLANE(64, 48) EK_PLANE(64, 64)
#undef EK_PLANE
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

cudaError_t charge_density(const Grid& g, const Phys& ph, const void* rho, const void* qwall,
                           const void* qpart, double* q, cudaStream_t s) {
  if (ph.fp32) k_charge<FormF32><<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(g, ph, rho, qwall, qpart, q);
  else k_charge<FormF64><<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(g, ph, rho, qwall, qpart, q);
  return cudaGetLastError();
}

}  // namespace ek
