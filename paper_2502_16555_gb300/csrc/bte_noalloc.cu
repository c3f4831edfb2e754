// bte_init_maxwellian_static: the initial-state fill for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another runtime's memory pool that owns
// every device allocation, or a host program that hands this library device buffers it obtained
// elsewhere. Such a caller can build a handle with BTE_FLAG_HOST_ONLY (the host-side operators only,
// no device memory, no CUDA call) and still fill its own state buffer through this entry point.
//
// The only device scratch this needs (the nr B-spline coefficients of the unit Maxwellian, which
// bte_init_maxwellian keeps in a buffer of the handle) lives in the file-scope array below, sized for
// at most kMaxCoef coefficients. Every GPU that loads libbte holds it (32 KB) until the process exits.
// bte_create already limits nr to 880, so the kMaxCoef check guards the array should that limit
// ever be raised.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "bte_internal.h"
#include "bte_kernels.h"

namespace {

constexpr int kMaxCoef = 4096;     // largest nr this entry point accepts
constexpr int kMaxDevices = 128;

static __device__ __align__(256) double g_maxwellian_coef[kMaxCoef];

std::mutex g_mu;
double* g_coef_addr[kMaxDevices] = {};  // device address of g_maxwellian_coef, per device

}  // namespace

extern "C" bte_status bte_init_maxwellian_static(const bte_handle* h, double* F_dev, const double* ne_dev,
                                                 double Te_eV) {
  if (!h) return BTE_EINVAL;
  const bte::HostOps& o = *bte::handle_ops(h);
  if (!F_dev || !ne_dev || !(Te_eV > 0)) return bte::handle_fail(h, BTE_EINVAL, "bad arguments");
  if (o.nr > kMaxCoef)
    return bte::handle_fail(h, BTE_EINVAL,
                            "nr = " + std::to_string(o.nr) + " exceeds the " + std::to_string(kMaxCoef) +
                                "-coefficient static scratch of bte_init_maxwellian_static");
  // the coefficient copy below reads a host vector that is freed when this call returns, so it
  // must not be recorded into a graph: refuse while the handle's stream is capturing
  cudaStream_t st = bte::handle_stream(h);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess)
    return bte::handle_fail(h, BTE_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  if (cs != cudaStreamCaptureStatusNone)
    return bte::handle_fail(h, BTE_ESTATE,
                            "bte_init_maxwellian_static must not be called while the handle's stream is capturing");
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bte::handle_fail(h, BTE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return bte::handle_fail(h, BTE_EINVAL, "device ordinal out of range");
  double* scratch = nullptr;
  {
    // first call on this device: look up the array's device address with the device current
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_coef_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_maxwellian_coef);
      if (e != cudaSuccess)
        return bte::handle_fail(h, BTE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_coef_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_coef_addr[dev];
  }
  const std::vector<double> c = bte::maxwellian_coeffs(o, Te_eV);
  // the host vector is pageable, so this copy has taken the data before it returns
  e = cudaMemcpyAsync(scratch, c.data(), sizeof(double) * c.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return bte::handle_fail(h, BTE_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
  bte::launch_fill_maxwellian(F_dev, ne_dev, scratch, o.nx, o.nt, o.nr, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return bte::handle_fail(h, BTE_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return BTE_OK;
}
