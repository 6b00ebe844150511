// Allocation-free variant of the energy + Riemannian gradient call.
//
// moto_energy_grad needs a moto_ctx, and creating one allocates device
// scratch.  Some callers cannot allocate: a host framework that owns all
// device memory and hands a library only the buffers of each call, or a caller
// that must not risk the device-wide synchronisation that cudaMalloc and
// cudaFree may imply.  moto_energy_grad_noalloc serves them: the only scratch
// it needs (the per-block partial sums of the deterministic energy reduction,
// an arrival counter and a status word) lives in the file-scope device array
// below, which every GPU that loads this library keeps until the process
// exits.  The caller passes the spins and the output buffers, as for
// moto_energy_grad.
#include <mutex>

#include "internal.h"

namespace {

// Partial sums for up to kMaxBlocks blocks of the energy stencil (two doubles
// each), then the arrival counter and the status word.
constexpr long long kMaxBlocks = 32768;
constexpr size_t kScratchDoubles = 2 * (size_t)kMaxBlocks + 32;
static __device__ __align__(256) double moto_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch[kMaxDevices] = {nullptr};

// Device address of the array on the current device, looked up once per
// device with that device current (the symbol's host-side name is only a
// stand-in and must never be handed to a kernel).
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MOTO_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, moto_noalloc_scratch) != cudaSuccess || !p) return MOTO_ERR_CUDA;
    g_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_scratch[dev];
  return MOTO_OK;
}

}  // namespace

extern "C" int moto_energy_grad_noalloc(const moto_model* model, int dtype, const void* m_dev, void* g_dev,
                                        void* s_dev, double* out_dev, void* stream) {
  if (!model || !m_dev) return MOTO_ERR_ARG;
  if (model->L1 < 5 || model->L2 < 5 || model->n_shells < 1 || model->n_shells > 3) return MOTO_ERR_ARG;
  if (dtype != MOTO_F32 && dtype != MOTO_F64) return MOTO_ERR_ARG;
  // sizes checked in 64-bit before anything is formed in int: the site count
  // has moto_create's cap, and the tile count must fit the fixed array
  if ((long long)model->L1 * model->L2 > (1LL << 30)) return MOTO_ERR_ARG;
  if (moto::stencil_blocks(model->L1, model->L2) > kMaxBlocks) return MOTO_ERR_ARG;
  moto::ModelDev md;
  md.L1 = model->L1;
  md.L2 = model->L2;
  md.N = model->L1 * model->L2;
  md.n_shells = model->n_shells;
  for (int i = 0; i < 3; ++i) md.J[i] = i < model->n_shells ? model->J[i] : 0.0;
  md.D = model->D;
  md.K = model->K;
  md.muB = model->muB;
  // an error left pending by the caller's own work is not this call's: refuse
  // to launch rather than report it (and clear it) as ours
  if (cudaPeekAtLastError() != cudaSuccess) return MOTO_ERR_CUDA;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  double* part = scratch;
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + 2 * (size_t)kMaxBlocks);
  int* status = reinterpret_cast<int*>(scratch + 2 * (size_t)kMaxBlocks + 1);
  cudaStream_t st = (cudaStream_t)stream;
  // the counter and the status word must start at zero; the partial sums are
  // overwritten by every launch
  if (cudaMemsetAsync(counter, 0, 2 * sizeof(double), st) != cudaSuccess) return MOTO_ERR_CUDA;
  if (dtype == MOTO_F32)
    moto::launch_energy_grad<float>(md, (const float*)m_dev, (float*)g_dev, (float*)s_dev, part, counter, out_dev,
                                    status, false, st);
  else
    moto::launch_energy_grad<double>(md, (const double*)m_dev, (double*)g_dev, (double*)s_dev, part, counter,
                                     out_dev, status, false, st);
  if (cudaGetLastError() != cudaSuccess) return MOTO_ERR_CUDA;
  return MOTO_OK;
}
