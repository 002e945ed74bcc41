// pf_solve_potential_noalloc: the Jacobi-PCG Poisson solve for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: real-time loops that must not stall on
// the allocator (cudaMalloc and cudaFree can synchronize the device), and
// processes whose device memory is reserved up front by another allocator
// (a fixed pool, or a framework that owns every byte).  This entry point takes
// the inputs and the output from the caller and keeps every intermediate
// vector (r, p, q, face masks, reduction partials, solver scalars) in one
// file-scope __device__ array of PF_NOALLOC_SCRATCH_BYTES.  Every GPU that
// loads the library holds that array until the process exits.
//
// The call blocks (it polls the solver's convergence flag and reads its
// scalars back), so it must not be made while its stream, or the legacy
// stream, is being captured into a CUDA graph: it checks and refuses.
//
// The array's name is only a host-side stand-in in host code, so every call
// looks up the device address with cudaGetSymbolAddress (with the caller's
// device current) and passes it to the kernels.  Calls share the array:
// concurrent or overlapping calls race.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "pf.h"
#include "pf_internal.h"

namespace {

constexpr size_t kScratchBytes = PF_NOALLOC_SCRATCH_BYTES;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

pf_status fail(pf_status st, const char* msg) {
  pf::set_global_error(msg);
  return st;
}

// Is p device (or managed) memory that device dev can address as its own?
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

struct Layout {
  size_t r, p0, p1, q, tlo, thi, vlo, vhi, part, S, total;
};

Layout layout(const pf_params* p) {
  const size_t w = p->precision == PF_FP32 ? 4 : 8;
  const size_t n = (size_t)p->nx * p->ny * p->nz, nxy = (size_t)p->nx * p->ny;
  const size_t max_tiles = (size_t)((p->nx + pf::MTX - 1) / pf::MTX) * ((p->ny + pf::MTY - 1) / pf::MTY) * p->nz;
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off += up256(b);
    return o;
  };
  L.r = take(n * w);
  L.p0 = take(n * w);
  L.p1 = take(n * w);
  L.q = take(n * w);
  L.tlo = take(nxy);
  L.thi = take(nxy);
  L.vlo = take(nxy * w);
  L.vhi = take(nxy * w);
  L.part = take(sizeof(double) * std::max<size_t>((size_t)pf::MAX_GRID * pf::MAX_NV, pf::MAX_NV * max_tiles));
  L.S = take(sizeof(pf::Scalars));
  L.total = off;
  return L;
}

#define NA_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) {                           \
      pf::set_global_error(#call, cudaGetErrorString(e_)); \
      return PF_ERR_CUDA;                              \
    }                                                  \
  } while (0)

// Host array -> device face data of type T, through a fixed stack buffer
// (a copy from pageable memory returns once the buffer has been staged).
template <typename T>
pf_status upload_volts(T* dst, const double* src, size_t n, cudaStream_t st) {
  T buf[1024];
  for (size_t i = 0; i < n; i += 1024) {
    const size_t m = std::min<size_t>(1024, n - i);
    for (size_t k = 0; k < m; ++k) buf[k] = src ? (T)src[i + k] : (T)0;
    NA_CUDA(cudaMemcpyAsync(dst + i, buf, m * sizeof(T), cudaMemcpyHostToDevice, st));
  }
  return PF_OK;
}

template <typename T>
pf_status solve(const pf_params* prm, cudaStream_t st, char* base, const Layout& Ly, const T* P, T* phi,
                const int8_t* tlo, const double* vlo, const int8_t* thi, const double* vhi, int singular,
                pf_step_info* info) {
  int dev = 0, nsm = 0;
  NA_CUDA(cudaGetDevice(&dev));
  NA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  pf::Geo g;
  pf::LaunchCfg L;
  pf::setup_launch(prm, nsm, st, g, L);
  pf::Dev<T> d{};
  d.phi = phi;
  d.r = (T*)(base + Ly.r);
  d.p0 = (T*)(base + Ly.p0);
  d.p1 = (T*)(base + Ly.p1);
  d.q = (T*)(base + Ly.q);
  d.bc.tlo = (const int8_t*)(base + Ly.tlo);
  d.bc.thi = (const int8_t*)(base + Ly.thi);
  d.bc.vlo = (const T*)(base + Ly.vlo);
  d.bc.vhi = (const T*)(base + Ly.vhi);
  d.part = (double*)(base + Ly.part);
  d.S = (pf::Scalars*)(base + Ly.S);

  // The array keeps the previous call's contents: masks and the solver state
  // are written afresh, the scalar block (tile and reduction counters) zeroed.
  const size_t nxy = (size_t)g.nxy;
  if (tlo) NA_CUDA(cudaMemcpyAsync(base + Ly.tlo, tlo, nxy, cudaMemcpyHostToDevice, st));
  else NA_CUDA(cudaMemsetAsync(base + Ly.tlo, 0, nxy, st));
  if (thi) NA_CUDA(cudaMemcpyAsync(base + Ly.thi, thi, nxy, cudaMemcpyHostToDevice, st));
  else NA_CUDA(cudaMemsetAsync(base + Ly.thi, 0, nxy, st));
  pf_status s = upload_volts<T>((T*)(base + Ly.vlo), vlo, nxy, st);
  if (s != PF_OK) return s;
  s = upload_volts<T>((T*)(base + Ly.vhi), vhi, nxy, st);
  if (s != PF_OK) return s;
  pf::Scalars init;
  std::memset(&init, 0, sizeof(init));
  init.rtol = prm->poisson_rtol;
  init.maxit = prm->poisson_maxit;
  init.done = 1;
  NA_CUDA(cudaMemcpyAsync(d.S, &init, sizeof(init), cudaMemcpyHostToDevice, st));

  int64_t launches = singular ? 3 : 2;     // rhs (+ mean) and the final update (+ mean removal)
  auto launched = [&](const char* what) -> pf_status {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return PF_OK;
    char msg[256];
    std::snprintf(msg, sizeof(msg), "%s launch (march grid %d, vx %d, tz %d, flat grid %d): %s", what,
                  L.march.grid, L.march.vx, L.march.tz, L.flat_grid, cudaGetErrorString(e));
    return fail(PF_ERR_CUDA, msg);
  };
  if (singular) pf::launch_rhs_mean<T>(L, g, d, P);
  pf::launch_rhs<T>(L, g, d, P, 0, 0);
  if (launched("rhs") != PF_OK) return PF_ERR_CUDA;
  pf::Scalars host;
  int issued = 0, batch = std::min(16, prm->poisson_maxit);
  for (;;) {
    for (int i = 0; i < batch; ++i) {
      pf::launch_cg_p<T>(L, g, d, 0);
      if (launched("cg_p") != PF_OK) return PF_ERR_CUDA;
      pf::launch_cg_r<T>(L, g, d, 0, 0, 0);
      if (launched("cg_r") != PF_OK) return PF_ERR_CUDA;
    }
    issued += batch;
    launches += 2 * batch;
    NA_CUDA(cudaMemcpyAsync(&host, d.S, sizeof(host), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    if (host.done) break;
    if (issued >= prm->poisson_maxit) return fail(PF_ERR_STATE, "internal: the solver did not stop at maxit");
    batch = std::min(std::min(2 * batch, 512), prm->poisson_maxit - issued);
  }
  pf::launch_cg_finish<T>(L, g, d, singular);
  if (launched("cg_finish") != PF_OK) return PF_ERR_CUDA;
  if (singular) pf::launch_sub_mean<T>(L, g, d);
  if (launched("sub_mean") != PF_OK) return PF_ERR_CUDA;
  NA_CUDA(cudaMemcpyAsync(&host, d.S, sizeof(host), cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaStreamSynchronize(st));
  pf_status result = PF_OK;
  if (host.nonfinite) result = fail(PF_ERR_NONFINITE, "non-finite value in the Poisson solver scalars");
  else if (host.nonconv) result = fail(PF_ERR_NOCONV, "the Poisson solve hit poisson_maxit");
  if (info) {
    info->steps_done = 0;
    info->last_iters = host.last_iters;
    info->total_iters = host.total_iters;
    info->last_relres = host.last_rel;
    info->nonconverged = host.nonconv;
    info->status = result;
    info->kernel_launches = launches + (singular ? 1 : 0);
    info->graph_steps = 0;
    info->max_iters = host.max_iters;
    info->solves = host.solves;
  }
  return result;
}

}  // namespace

extern "C" {

pf_status pf_solve_potential_noalloc(const pf_params* params, void* cuda_stream, const void* P, void* phi,
                                     const int8_t* type_lo, const double* volt_lo, const int8_t* type_hi,
                                     const double* volt_hi, pf_step_info* info) {
  if (!params) return fail(PF_ERR_ARG, "params is NULL");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // The solve synchronizes the stream and copies from host buffers: neither
  // is legal while the stream (or the legacy stream) is being captured, so
  // this is checked before any other CUDA call.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t ce = cudaStreamIsCapturing(st, &cap);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    pf::set_global_error("the allocation-free solve cannot run during stream capture (it blocks)",
                         cudaGetErrorString(ce));
    return PF_ERR_STATE;
  }
  if (cap != cudaStreamCaptureStatusNone)
    return fail(PF_ERR_STATE, "the allocation-free solve cannot run while its stream is being captured (it blocks)");
  if (params->solver != PF_PCG_JACOBI || params->has_eps)
    return fail(PF_ERR_ARG, "the allocation-free solve supports solver PF_PCG_JACOBI with has_eps = 0");
  if (pf_workspace_bytes(params) == 0) return fail(PF_ERR_ARG, "invalid parameters");
  if (!P || !phi) return fail(PF_ERR_ARG, "P and phi must be non-NULL device pointers");
  if (((uintptr_t)P % 16) || ((uintptr_t)phi % 16)) return fail(PF_ERR_ARG, "P and phi must be 16-byte aligned");
  const Layout Ly = layout(params);
  if (Ly.total > kScratchBytes) {
    char msg[256];
    std::snprintf(msg, sizeof(msg),
                  "grid needs %zu bytes of scratch; the allocation-free solve holds at most %zu bytes "
                  "(about %zu cells in FP64, %zu in FP32)",
                  Ly.total, kScratchBytes, kScratchBytes / 40, kScratchBytes / 20);
    return fail(PF_ERR_ARG, msg);
  }
  const size_t nxy = (size_t)params->nx * params->ny;
  int singular = 1;
  if (!params->periodic_z) {
    for (size_t i = 0; i < nxy; ++i) {
      const int a = type_lo ? type_lo[i] : 0, b = type_hi ? type_hi[i] : 0;
      if ((a != PF_NEUMANN && a != PF_DIRICHLET) || (b != PF_NEUMANN && b != PF_DIRICHLET))
        return fail(PF_ERR_ARG, "face types must be PF_NEUMANN or PF_DIRICHLET");
      if (a == PF_DIRICHLET || b == PF_DIRICHLET) singular = 0;
    }
  }
  int dev = 0;
  NA_CUDA(cudaGetDevice(&dev));
  if (!on_device(P, dev) || !on_device(phi, dev))
    return fail(PF_ERR_ARG, "P and phi must be device (or managed) memory of the current device");
  // Device address of the array in this device's context, looked up on every
  // call (cheap, allocates nothing, and stays right across cudaDeviceReset).
  void* ptr = nullptr;
  NA_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
  char* base = (char*)ptr;
  if (params->precision == PF_FP32)
    return solve<float>(params, st, base, Ly, (const float*)P, (float*)phi, type_lo, volt_lo, type_hi, volt_hi,
                        singular, info);
  return solve<double>(params, st, base, Ly, (const double*)P, (double*)phi, type_lo, volt_lo, type_hi, volt_hi,
                       singular, info);
}

}  // extern "C"
