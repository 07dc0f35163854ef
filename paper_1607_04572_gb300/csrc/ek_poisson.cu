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

#include <map>
#include <mutex>
#include <tuple>

#include "ek_internal.cuh"

namespace ek {

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
    for (int k = 0; k < a.K; ++k) q += a.z[k] * (R)((const int*)a.rho)[k * N + i];
  } else {
    for (int k = 0; k < a.K; ++k) q += a.z[k] * ((const R*)a.rho)[k * N + i];
  }
  if (a.qwall) q += a.qwall[i];
  if (a.qpart) q += a.qpart[i];
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

}  // namespace

bool poisson_factor(int n, AxisPlan& P) { return factor(n, P); }

size_t poisson_spectrum_bytes(int nx, int ny, int nz) {
  return (size_t)(nx / 2 + 1) * (size_t)ny * (size_t)nz * sizeof(double2);
}

cudaError_t poisson_plan_create(PoissonPlan& p, int nx, int ny, int nz, std::string& err) {
  p = PoissonPlan();
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

cudaError_t charge_density(const Grid& g, const Phys& ph, const void* rho, const void* qwall,
                           const void* qpart, double* q, cudaStream_t s) {
  if (ph.fp32) k_charge<FormF32><<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(g, ph, rho, qwall, qpart, q);
  else k_charge<FormF64><<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(g, ph, rho, qwall, qpart, q);
  return cudaGetLastError();
}

}  // namespace ek
