// Batched stepping of independent discharges with uneven grids and pressures (declared in
// include/bte.h, bte_batch_*). Every instance is an ordinary handle; the batch records one CUDA
// graph whose branches are the instances' step sequences (they run concurrently on the GPU),
// framed by one kernel that writes every instance's field E_i(t + dt/2) from a device-side clock
// and one that advances the clocks, so n steps are n launches of the same graph with no host work
// in between. The semi-implicit step of each instance is that of eqs. "bte_semi_implicit"
// (arXiv 2502.16555); batching changes only how the launches reach the GPU.
//
// Autotuner: for every distinct instance shape (nx, nr, ntheta, nl, precision) it times one
// short run of each algorithm variant on a scratch Maxwellian state and keeps the fastest for all
// instances of that shape: the tensor-core (TF32x3) or CUDA-core trailing update; on the tensor
// cores the update's tile shape: panels in pairs (K = 256) on 256 x 256 tiles of CTA pairs or on
// 128 x 128 tiles of single CTAs, or one panel at a time (K = 128, 128 x 128 tiles); and the panel
// kernel's column-block width (16 columns x 4 rows per thread, or 8 x 8).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "bte_internal.h"

struct bte_batch {
  std::vector<bte_handle*> hs;
  cudaStream_t user = nullptr;  // the caller's stream (may be the legacy default stream)
  cudaStream_t st = nullptr;    // the batch's own stream: captures and launches the graph
  cudaEvent_t ready = nullptr;
  std::vector<cudaStream_t> branch;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  // device: clocks and field parameters [5][count] (t, dt, V0, freq, L), E pointers, nx
  double* dpar = nullptr;
  double** dE = nullptr;
  int* dnx = nullptr;
  std::vector<double*> E;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<double*> F_captured;
  unsigned long long launches_per_step = 0;
  std::vector<unsigned long long> inst_launches;  // per instance and step
  std::vector<bte::Variant> variant;
  std::string err;
};

namespace {

std::string g_batch_create_error;

bte_status bfail(bte_batch* b, bte_status s, const std::string& m) {
  if (b) b->err = m;
  else g_batch_create_error = m;
  return s;
}

#define BB_CUDA(b, call)                                                                        \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return bfail((b), BTE_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

constexpr double kTwoPi = 6.283185307179586476925286766559;

// E_i[x] = V0_i / L_i sin(2 pi f_i (t_i + dt_i / 2)) for every instance i (one CTA each).
__global__ void batch_field_kernel(const double* __restrict__ par, int count, double* const* __restrict__ E,
                                   const int* __restrict__ nx) {
  const int i = blockIdx.x;
  const double t = par[i], dt = par[count + i], V0 = par[2 * count + i], f = par[3 * count + i],
               L = par[4 * count + i];
  const double e = V0 / L * sin(kTwoPi * f * (t + 0.5 * dt));
  for (int x = threadIdx.x; x < nx[i]; x += blockDim.x) E[i][x] = e;
}

__global__ void batch_advance_kernel(double* par, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) par[i] += par[count + i];
}

void release_graph(bte_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->F_captured.clear();
}

bte_status capture(bte_batch* b, double* const* F) {
  release_graph(b);
  const int count = static_cast<int>(b->hs.size());
  std::vector<unsigned long long> before(count);
  for (int i = 0; i < count; ++i) before[i] = bte::handle_launches(b->hs[i]);
  // relaxed: a launcher's first use may set a kernel attribute or encode a tensor map
  BB_CUDA(b, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeRelaxed));
  bte_status s = BTE_OK;
  batch_field_kernel<<<count, 128, 0, b->st>>>(b->dpar, count, b->dE, b->dnx);
  cudaError_t ce = cudaEventRecord(b->fork, b->st);
  for (int i = 0; i < count && s == BTE_OK && ce == cudaSuccess; ++i) {
    ce = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
    if (ce != cudaSuccess) break;
    s = bte::handle_enqueue_step(b->hs[i], F[i], b->E[i], 0.0, 0.0, 0.0, b->branch[i]);
    if (s != BTE_OK) break;
    ce = cudaEventRecord(b->join[i], b->branch[i]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->st, b->join[i], 0);
  }
  batch_advance_kernel<<<1, 64, 0, b->st>>>(b->dpar, count);
  cudaGraph_t g = nullptr;
  cudaError_t ee = cudaStreamEndCapture(b->st, &g);
  if (s != BTE_OK) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, s, "capturing an instance's step failed");
  }
  if (ce != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, BTE_ECUDA, std::string("stream capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ee));
  }
  b->graph = g;
  BB_CUDA(b, cudaGraphInstantiate(&b->exec, b->graph, 0));
  b->launches_per_step = 2;
  b->inst_launches.assign(count, 0);
  for (int i = 0; i < count; ++i) {
    const unsigned long long n = bte::handle_launches(b->hs[i]) - before[i];
    b->launches_per_step += n;
    b->inst_launches[i] = n;
    bte::handle_add_launches(b->hs[i], 0ull - n);  // captured, not launched: counted per replay
  }
  b->F_captured.assign(F, F + count);
  return BTE_OK;
}

// Device time of `steps` steps of handle h on F (scratch) with the uniform sinusoidal field.
bte_status time_variant(bte_batch* b, bte_handle* h, double* F, int steps, float& ms) {
  cudaEvent_t e0, e1;
  BB_CUDA(b, cudaEventCreate(&e0));
  BB_CUDA(b, cudaEventCreate(&e1));
  const bte::HostOps& o = *bte::handle_ops(h);
  bte_status s = bte::handle_reset_status(h, b->st);
  if (s == BTE_OK) s = bte::handle_enqueue_step(h, F, nullptr, 0.0, 100.0, 13.56e6, b->st);  // warm-up
  cudaEventRecord(e0, b->st);
  for (int k = 0; k < steps && s == BTE_OK; ++k)
    s = bte::handle_enqueue_step(h, F, nullptr, (k + 1) * o.dt, 100.0, 13.56e6, b->st);
  cudaEventRecord(e1, b->st);
  cudaError_t ce = cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != BTE_OK) return s;
  if (ce != cudaSuccess) return bfail(b, BTE_ECUDA, cudaGetErrorString(ce));
  return BTE_OK;
}

bte_status autotune(bte_batch* b) {
  using Key = std::tuple<int, int, int, int, int>;
  std::map<Key, bte::Variant> best;
  for (size_t i = 0; i < b->hs.size(); ++i) {
    bte_handle* h = b->hs[i];
    const bte::HostOps& o = *bte::handle_ops(h);
    bte_info info;
    bte_get_info(h, &info);
    const Key key{o.nx, o.nr, o.nt, o.nl, info.precision};
    auto it = best.find(key);
    if (it == best.end()) {
      // scratch state: a 2 eV Maxwellian of density 1e15 m^-3 at every point
      const size_t D = static_cast<size_t>(o.nx) * o.nv;
      double *F = nullptr, *ne = nullptr;
      BB_CUDA(b, cudaMalloc(&F, D * sizeof(double)));
      BB_CUDA(b, cudaMalloc(&ne, o.nx * sizeof(double)));
      std::vector<double> one(o.nx, 1e15);
      cudaMemcpy(ne, one.data(), o.nx * sizeof(double), cudaMemcpyHostToDevice);
      bte_status s = bte_init_maxwellian(h, F, ne, 2.0);
      std::vector<bte::Variant> cands;
      for (int w : {0, info.precision == BTE_MIXED ? 8 : 4}) {
        if (bte::handle_has_tc(h)) {
          cands.push_back({true, w, true, 2});
          cands.push_back({true, w, true, 1});
          cands.push_back({true, w, false, 1});
        }
        cands.push_back({false, w, true, 2});
      }
      float tbest = 1e30f;
      bte::Variant win = bte::handle_get_variant(h);
      for (auto& c : cands) {
        if (s != BTE_OK) break;
        bte::handle_set_variant(h, c);
        float ms = 0.f;
        s = time_variant(b, h, F, 2, ms);
        if (s == BTE_OK && ms < tbest) tbest = ms, win = c;
      }
      cudaFree(F);
      cudaFree(ne);
      if (s != BTE_OK) return bfail(b, s, "autotuning: a trial step failed");
      it = best.emplace(key, win).first;
    }
    bte::handle_set_variant(h, it->second);
    b->variant[i] = it->second;
  }
  return BTE_OK;
}

}  // namespace

extern "C" {

bte_status bte_batch_create(int count, bte_handle* const* handles, void* stream, unsigned flags, bte_batch** out) {
  if (!out) return bfail(nullptr, BTE_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || count > 4096 || !handles) return bfail(nullptr, BTE_EINVAL, "count must be in [1, 4096]");
  for (int i = 0; i < count; ++i) {
    if (!handles[i]) return bfail(nullptr, BTE_EINVAL, "a handle is NULL");
    if (bte::handle_device_status(handles[i]) != BTE_OK)
      return bfail(nullptr, BTE_ESTATE, "every handle needs device buffers and cross sections");
    if (bte::handle_profiling(handles[i])) return bfail(nullptr, BTE_ESTATE, "a handle is recording a profile");
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return bfail(nullptr, BTE_EINVAL, "a handle appears twice");
  }
  bte_batch* b = new bte_batch();
  b->hs.assign(handles, handles + count);
  b->user = static_cast<cudaStream_t>(stream);
  b->variant.resize(count);
  auto bad = [&](bte_status s) {
    g_batch_create_error = b->err;
    bte_batch_destroy(b);
    return s;
  };
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming) != cudaSuccess)
    return bad(bfail(b, BTE_ECUDA, "creating the batch stream"));
  b->branch.resize(count);
  b->join.resize(count);
  for (int i = 0; i < count; ++i) {
    if (cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess)
      return bad(bfail(b, BTE_ECUDA, "creating branch streams"));
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    return bad(bfail(b, BTE_ECUDA, "creating events"));
  std::vector<double> par(5 * static_cast<size_t>(count));
  std::vector<int> nx(count);
  b->E.resize(count);
  for (int i = 0; i < count; ++i) {
    const bte::HostOps& o = *bte::handle_ops(b->hs[i]);
    par[count + i] = o.dt;
    par[4 * count + i] = o.L;
    nx[i] = o.nx;
    if (cudaMalloc(&b->E[i], sizeof(double) * o.nx) != cudaSuccess) return bad(bfail(b, BTE_ENOMEM, "cudaMalloc"));
  }
  if (cudaMalloc(&b->dpar, sizeof(double) * par.size()) != cudaSuccess ||
      cudaMalloc(&b->dE, sizeof(double*) * count) != cudaSuccess ||
      cudaMalloc(&b->dnx, sizeof(int) * count) != cudaSuccess)
    return bad(bfail(b, BTE_ENOMEM, "cudaMalloc"));
  if (cudaMemcpy(b->dpar, par.data(), sizeof(double) * par.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->dE, b->E.data(), sizeof(double*) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->dnx, nx.data(), sizeof(int) * count, cudaMemcpyHostToDevice) != cudaSuccess)
    return bad(bfail(b, BTE_ECUDA, "uploading batch parameters"));
  for (int i = 0; i < count; ++i) b->variant[i] = bte::handle_get_variant(b->hs[i]);
  if (flags & BTE_BATCH_AUTOTUNE) {
    bte_status s = autotune(b);
    if (s != BTE_OK) return bad(s);
  }
  *out = b;
  return BTE_OK;
}

bte_status bte_batch_run(bte_batch* b, double* const* F_dev, int n_steps, const double* t0_s, const double* V0,
                         const double* freq_Hz, bte_status* status_out) {
  if (!b) return bfail(nullptr, BTE_EINVAL, "batch is NULL");
  const int count = static_cast<int>(b->hs.size());
  if (!F_dev || !t0_s || !V0 || !freq_Hz || n_steps < 0) return bfail(b, BTE_EINVAL, "bad arguments");
  for (int i = 0; i < count; ++i) {
    if (!F_dev[i]) return bfail(b, BTE_EINVAL, "a state pointer is NULL");
    if (!std::isfinite(t0_s[i]) || !std::isfinite(V0[i]) || !std::isfinite(freq_Hz[i]))
      return bfail(b, BTE_EINVAL, "non-finite time or field parameter");
    if (bte::handle_profiling(b->hs[i])) return bfail(b, BTE_ESTATE, "a handle is recording a profile");
  }
  if (!b->exec || !std::equal(b->F_captured.begin(), b->F_captured.end(), F_dev)) {
    bte_status s = capture(b, F_dev);
    if (s != BTE_OK) return s;
  }
  // the batch's stream starts after the work the caller has enqueued on its own stream
  BB_CUDA(b, cudaEventRecord(b->ready, b->user));
  BB_CUDA(b, cudaStreamWaitEvent(b->st, b->ready, 0));
  std::vector<double> tv(t0_s, t0_s + count), v0(V0, V0 + count), fq(freq_Hz, freq_Hz + count);
  BB_CUDA(b, cudaMemcpyAsync(b->dpar, tv.data(), sizeof(double) * count, cudaMemcpyHostToDevice, b->st));
  BB_CUDA(b, cudaMemcpyAsync(b->dpar + 2 * count, v0.data(), sizeof(double) * count, cudaMemcpyHostToDevice, b->st));
  BB_CUDA(b, cudaMemcpyAsync(b->dpar + 3 * count, fq.data(), sizeof(double) * count, cudaMemcpyHostToDevice, b->st));
  for (int i = 0; i < count; ++i) {
    bte_status s = bte::handle_reset_status(b->hs[i], b->st);
    if (s != BTE_OK) return s;
  }
  for (int k = 0; k < n_steps; ++k) BB_CUDA(b, cudaGraphLaunch(b->exec, b->st));
  BB_CUDA(b, cudaStreamSynchronize(b->st));  // also keeps tv, v0, fq alive until copied
  for (int i = 0; i < count; ++i) bte::handle_add_launches(b->hs[i], b->inst_launches[i] * n_steps);
  bte_status first = BTE_OK;
  for (int i = 0; i < count; ++i) {
    const bte_status s = bte::handle_read_status(b->hs[i]);
    if (status_out) status_out[i] = s;
    if (s != BTE_OK && first == BTE_OK) first = s, b->err = std::string("instance ") + std::to_string(i) + ": " + bte_last_error(b->hs[i]);
  }
  return first;
}

bte_status bte_batch_get_info(const bte_batch* b, int i, int* tensor_cores, int* panel_w, int* tc_pair,
                              int* tc_cg, unsigned long long* launches_per_step) {
  if (!b) return bfail(nullptr, BTE_EINVAL, "batch is NULL");
  if (i < 0 || i >= static_cast<int>(b->hs.size())) return bfail(const_cast<bte_batch*>(b), BTE_EINVAL, "index out of range");
  if (tensor_cores) *tensor_cores = b->variant[i].tc ? 1 : 0;
  if (panel_w) *panel_w = b->variant[i].panel_w;
  if (tc_pair) *tc_pair = b->variant[i].pair ? 1 : 0;
  if (tc_cg) *tc_cg = b->variant[i].cg;
  if (launches_per_step) *launches_per_step = b->launches_per_step;
  return BTE_OK;
}

bte_status bte_batch_destroy(bte_batch* b) {
  if (!b) return BTE_OK;
  if (b->st) cudaStreamSynchronize(b->st);
  release_graph(b);
  if (b->st) cudaStreamDestroy(b->st);
  if (b->ready) cudaEventDestroy(b->ready);
  for (auto s : b->branch)
    if (s) cudaStreamDestroy(s);
  for (auto e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto p : b->E) cudaFree(p);
  cudaFree(b->dpar);
  cudaFree(b->dE);
  cudaFree(b->dnx);
  delete b;
  return BTE_OK;
}

const char* bte_batch_last_error(const bte_batch* b) {
  return b ? b->err.c_str() : g_batch_create_error.c_str();
}

}  // extern "C"
