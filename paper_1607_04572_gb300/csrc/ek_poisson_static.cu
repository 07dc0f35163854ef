// Poisson solve that allocates nothing: the same FFT kernels as
// ek_poisson_solve, with the spectrum scratch and the twiddle / eigenvalue
// tables in file-scope device arrays of fixed size instead of memory from
// cudaMalloc.  See ek_poisson_solve_static in include/ek.h.
#include <math.h>
#include <string.h>

#include <mutex>

#include "ek_internal.cuh"

using namespace ek;

namespace {

constexpr size_t STATIC_SPECTRUM = (size_t)1 << 19;  // complex doubles: 8 MiB
constexpr int STATIC_EDGE = 1024;                    // longest supported box edge
constexpr int MAX_DEVICES = 64;

// Device-side storage, present on every GPU that loads the library until the
// process exits.  In host code these names are host-side stand-ins, not device
// addresses: only the pointers from cudaGetSymbolAddress may reach a kernel.
static __device__ __align__(256) double2 g_spectrum[STATIC_SPECTRUM];
static __device__ __align__(256) double2 g_twiddle[3 * STATIC_EDGE];
static __device__ __align__(256) double g_lambda[3 * STATIC_EDGE];

struct DeviceTables {
  bool ready = false;           // symbol addresses resolved on this device
  double2* spectrum = nullptr;  // device address of g_spectrum
  double2* twiddle = nullptr;   // device address of g_twiddle
  double* lambda = nullptr;     // device address of g_lambda
  int nx = 0, ny = 0, nz = 0;   // box whose tables are loaded
  PoissonPlan plan;
};

std::mutex g_mutex;
DeviceTables g_tables[MAX_DEVICES];
// host staging of one table refill (fixed size: no allocation)
double2 h_twiddle[3 * STATIC_EDGE];
double h_lambda[3 * STATIC_EDGE];

bool edge_supported(int n) {
  if (n < 8 || n > STATIC_EDGE) return false;
  int m = n;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

}  // namespace

extern "C" ek_status ek_poisson_solve_static(const double* q, double* phi, int nx, int ny, int nz,
                                             double bjerrum, void* stream) {
  if (!q || !phi || !edge_supported(nx) || !edge_supported(ny) || !edge_supported(nz) ||
      nx % 2 != 0 || !(bjerrum >= 0.0))
    return EK_ERR_ARG;
  if ((size_t)(nx / 2 + 1) * (size_t)ny * (size_t)nz > STATIC_SPECTRUM) return EK_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EK_ERR_CUDA;
  if (dev < 0 || dev >= MAX_DEVICES) return EK_ERR_ARG;
  PoissonPlan plan;
  double2* spectrum = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceTables& t = g_tables[dev];
    if (!t.ready) {
      // once per device, with that device current
      if (cudaGetSymbolAddress((void**)&t.spectrum, g_spectrum) != cudaSuccess) return EK_ERR_CUDA;
      if (cudaGetSymbolAddress((void**)&t.twiddle, g_twiddle) != cudaSuccess) return EK_ERR_CUDA;
      if (cudaGetSymbolAddress((void**)&t.lambda, g_lambda) != cudaSuccess) return EK_ERR_CUDA;
      t.ready = true;
    }
    if (t.nx != nx || t.ny != ny || t.nz != nz) {
      PoissonPlan p;
      const int n3[3] = {nx, ny, nz};
      AxisPlan* ax3[3] = {&p.ax, &p.ay, &p.az};
      for (int a = 0; a < 3; ++a) {
        if (!poisson_factor(n3[a], *ax3[a])) return EK_ERR_ARG;
        for (int k = 0; k < n3[a]; ++k) {
          const double ang = 2.0 * M_PI * (double)k / (double)n3[a];
          h_twiddle[a * STATIC_EDGE + k] = make_double2(cos(ang), -sin(ang));
          h_lambda[a * STATIC_EDGE + k] = 2.0 - 2.0 * cos(ang);
        }
        ax3[a]->tw = t.twiddle + a * STATIC_EDGE;
        ax3[a]->lam = t.lambda + a * STATIC_EDGE;
      }
      // The refill is queued on the caller's stream: an earlier solve still
      // queued there reads the old tables before they are overwritten, and
      // the solve below reads the new ones.  A copy from pageable memory
      // returns once its source has been staged, so the host buffers may be
      // refilled by the next call.
      cudaStream_t s = (cudaStream_t)stream;
      if (cudaMemcpyAsync(t.twiddle, h_twiddle, sizeof(h_twiddle), cudaMemcpyHostToDevice, s) !=
              cudaSuccess ||
          cudaMemcpyAsync(t.lambda, h_lambda, sizeof(h_lambda), cudaMemcpyHostToDevice, s) !=
              cudaSuccess) {
        t.nx = t.ny = t.nz = 0;
        return EK_ERR_CUDA;
      }
      p.nx = nx;
      p.ny = ny;
      p.nz = nz;
      p.ok = true;
      t.plan = p;
      t.nx = nx;
      t.ny = ny;
      t.nz = nz;
    }
    plan = t.plan;
    spectrum = t.spectrum;
  }
  Phys ph;
  memset(&ph, 0, sizeof(ph));
  ph.bjerrum = bjerrum;
  if (poisson_solve(plan, q, nullptr, nullptr, nullptr, ph, phi, spectrum, (cudaStream_t)stream) !=
      cudaSuccess)
    return EK_ERR_CUDA;
  return EK_OK;
}
