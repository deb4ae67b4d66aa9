// Allocation-free variant of one weighted additive Schwarz correction,
// u += sum_s R_s^T W A_ss^{-1} R_s r.
//
// The regular path (sem_smooth) keeps the element-blocked correction buffer E
// in device memory that sem_create allocates.  This variant needs no handle and
// never allocates: E lives in a file-scope static device array of fixed size,
// which every GPU that loads the library holds until the process exits.  Its
// device address is looked up once per device with cudaGetSymbolAddress, on
// the first call made while that device is current, and kept for the life of
// the process.  cudaDeviceReset destroys the array with the context, so the
// kept address is stale afterwards: a process that resets a device must not
// call this entry point on that device again.
#include <mutex>
#include <string>

#include "kernels.h"
#include "sem_schwarz.h"

namespace sem {
void set_last_error(const std::string& msg);  // defined with sem_last_error in sem_api.cu
}

namespace {

// 2 Mi doubles = 16 MiB: enough for n_x n_y m^2 <= 2^21, e.g. 64 x 64
// elements at p = 16 with n_o = 2 (m = 21).
constexpr size_t kScratchDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_sweep_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

int noalloc_fail(int code, const std::string& m) {
  sem::set_last_error(m);
  return code;
}

bool dir_ok(const sem_sweep_tables* t) {
  if (!t || !t->tab || !t->S || !t->lam || !t->w) return false;
  if (t->p < 2 || t->p > 32 || (t->p & (t->p - 1))) return false;
  if (t->n < 2 || t->n_o < 0 || t->n_o > t->p - 1) return false;
  return true;
}

}  // namespace

extern "C" int sem_schwarz_correction_noalloc(const sem_sweep_tables* tx, const sem_sweep_tables* ty,
                                              const double* r, double* u, void* stream) {
  if (!dir_ok(tx) || !dir_ok(ty) || !r || !u)
    return noalloc_fail(SEM_BAD_ARG, "sem_schwarz_correction_noalloc: invalid tables or vectors");
  if (tx->p != ty->p || tx->n_o != ty->n_o || (tx->periodic != 0) != (ty->periodic != 0))
    return noalloc_fail(SEM_BAD_ARG, "sem_schwarz_correction_noalloc: x and y tables disagree on p, n_o or periodicity");
  const int p = tx->p, no = tx->n_o, m = p + 1 + 2 * no;
  const bool per = tx->periodic != 0;
  if (per && (m > tx->n * p || m > ty->n * p))
    return noalloc_fail(SEM_BAD_ARG, "sem_schwarz_correction_noalloc: subdomain window larger than the periodic mesh");
  const size_t need = (size_t)tx->n * ty->n * m * m;
  if (need > kScratchDoubles)
    return noalloc_fail(SEM_BAD_ARG, "sem_schwarz_correction_noalloc: needs " + std::to_string(need) +
                                         " doubles of scratch (n_x n_y m^2); the static limit is " +
                                         std::to_string(kScratchDoubles));
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return noalloc_fail(SEM_CUDA_ERROR, "sem_schwarz_correction_noalloc: no usable current CUDA device");
  }
  // The FP64 local solve keeps four m x m and four m-long arrays of one
  // subdomain in shared memory; a window too large for the device's per-block
  // limit is a bad argument, rejected before anything is launched.
  int smem_optin = 0;
  if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(SEM_CUDA_ERROR, "sem_schwarz_correction_noalloc: cannot query the shared-memory limit");
  }
  const size_t smem_need = sizeof(double) * (4 * (size_t)m * m + 4 * (size_t)m);
  if (smem_need > (size_t)smem_optin)
    return noalloc_fail(SEM_BAD_ARG, "sem_schwarz_correction_noalloc: window m = " + std::to_string(m) + " needs " +
                                         std::to_string(smem_need) + " bytes of shared memory per block; the device allows " +
                                         std::to_string(smem_optin));
  double* E = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_sweep_scratch);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(SEM_CUDA_ERROR, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      g_scratch_ptr[dev] = static_cast<double*>(ptr);
    }
    E = g_scratch_ptr[dev];
  }
  auto view = [&](const sem_sweep_tables* t) {
    sem::DirView<double> v{};
    v.p = p;
    v.n = t->n;
    v.N = per ? t->n * p : t->n * p + 1;
    v.periodic = per ? 1 : 0;
    v.n_o = no;
    v.m = m;
    v.Le = nullptr;  // the correction uses no operator tables
    v.Mg = nullptr;
    v.tab = t->tab;
    v.S = t->S;
    v.lam = t->lam;
    v.w = t->w;
    return v;
  };
  const sem::DirView<double> dx = view(tx), dy = view(ty);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The sweep writes every entry of E that the scatter reads (each CTA fills
  // its whole m x m block), so the scratch needs no clearing between calls.
  cudaError_t e = sem::launch_sweep<double, double>(dx, dy, r, E, 0, nullptr, s);
  if (e == cudaSuccess) e = sem::launch_scatter<double, double>(dx, dy, E, u, true, s);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear it, so that no later launch reports this failure as its own
    return noalloc_fail(SEM_CUDA_ERROR, std::string("launch: ") + cudaGetErrorString(e));
  }
  return SEM_OK;
}
