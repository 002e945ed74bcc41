// C ABI of the TDGL + Poisson library (declared in include/pf.h).
//
// Host-side driver: argument checks, workspace layout, boundary masks, and
// the time loop.  Per step: r0 = b(P_n) - A phi (warm start, Section
// Numerical Performance), Jacobi-PCG iterations until the on-device
// convergence flag is set, the deferred last x update, then the
// forward-Euler TDGL update into the second polarization buffer (Section
// Time Integration).  The host never sees alpha/beta; it only polls the flag
// once per batch of iterations to stop issuing more.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pf.h"
#include "pf_internal.h"

using pf::Geo;
using pf::Scalars;

namespace {

// Message of the last failure without a context (pf_create, the
// allocation-free solve): a fixed buffer, so recording it never allocates.
thread_local char g_create_error[512];

constexpr size_t ALIGN = 256;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

// One multigrid level on the host: dimensions, coarsening factors to the
// next level and workspace offsets (level 0 uses r, z, zt and the fine masks).
struct MgLevelHost {
  int nx, ny, nz;
  int fx, fy, fz;
  double ax, ay, az;
  size_t f, e, et, tlo, thi;
  size_t eps = 0, invd = 0;       // coarse levels with a permittivity field: eps and 1/diag
  pf::MarchCfg mc;
  long long n() const { return (long long)nx * ny * nz; }
  long long nxy() const { return (long long)nx * ny; }
};

// Level dimensions: halve every even dimension until none can be halved.
std::vector<MgLevelHost> mg_levels(const pf_params* p) {
  std::vector<MgLevelHost> L;
  MgLevelHost l{};
  l.nx = p->nx;
  l.ny = p->ny;
  l.nz = p->nz;
  const double ih2 = 1.0 / (p->dx * p->dx);
  l.ax = l.ay = l.az = ih2;
  for (;;) {
    l.fx = (l.nx % 2 == 0 && l.nx > 1) ? 2 : 1;
    l.fy = (l.ny % 2 == 0 && l.ny > 1) ? 2 : 1;
    l.fz = (l.nz % 2 == 0 && l.nz > 1) ? 2 : 1;
    const bool last = (l.fx == 1 && l.fy == 1 && l.fz == 1) || (int)L.size() + 1 == pf::MG_MAX_LEVELS;
    if (last) l.fx = l.fy = l.fz = 1;
    L.push_back(l);
    if (last) break;
    MgLevelHost c{};
    c.nx = l.nx / l.fx;
    c.ny = l.ny / l.fy;
    c.nz = l.nz / l.fz;
    c.ax = l.ax / (l.fx * l.fx);
    c.ay = l.ay / (l.fy * l.fy);
    c.az = l.az / (l.fz * l.fz);
    l = c;
  }
  return L;
}

struct Layout {
  size_t P_alt, plo, r, p0, p1, q, invd, hist[3], clo, cx, tlo, thi, vlo, vhi, ctr, xctr, part, S, diag, loop, z, zt,
      total;
  bool adj = false;               // psi and vzero exist (PF_FLAG_ADJOINT)
  size_t psi = 0, vzero = 0;      // adjoint potential; zero face voltages
  std::vector<MgLevelHost> mg;
};

bool params_valid(const pf_params* p, std::string* why) {
  auto fail = [&](const char* m) {
    if (why) *why = m;
    return false;
  };
  if (!p) return fail("params is NULL");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail("nx, ny, nz must be >= 1");
  if ((double)p->nx * p->ny * p->nz > 4.0e10) return fail("grid too large");
  if (!(p->dx > 0.0) || !std::isfinite(p->dx)) return fail("dx must be finite and > 0");
  if (p->precision != PF_FP64 && p->precision != PF_FP32) return fail("precision must be PF_FP64 or PF_FP32");
  if (p->solver != PF_PCG_JACOBI && p->solver != PF_PCG_MG) return fail("solver must be PF_PCG_JACOBI or PF_PCG_MG");
  if (!(p->poisson_rtol > 0.0) || !std::isfinite(p->poisson_rtol)) return fail("poisson_rtol must be > 0");
  if (p->poisson_maxit < 1) return fail("poisson_maxit must be >= 1");
  if (p->periodic_z != 0 && p->periodic_z != 1) return fail("periodic_z must be 0 or 1");
  if (p->has_eps != 0 && p->has_eps != 1) return fail("has_eps must be 0 or 1");
  if (p->solver == PF_PCG_MG) {
    std::vector<MgLevelHost> L = mg_levels(p);
    if (L.size() < 2) return fail("multigrid needs at least one even grid dimension");
    if (L.back().n() > pf::MG_MAX_COARSE)
      return fail("multigrid: the coarsest level has more than 1024 cells (make nx, ny, nz powers of two "
                  "times small factors)");
  }
  for (double v : {p->a1, p->a11, p->a12, p->g, p->L, p->dt})
    if (!std::isfinite(v)) return fail("coefficients must be finite");
  if (p->flags & ~(PF_FLAG_NO_GRAPHS | PF_FLAG_ADJOINT | PF_FLAG_WARM_LAST | PF_FLAG_PLAIN_FP32))
    return fail("unknown bits in flags");
  if (p->integrator != PF_EULER && p->integrator != PF_HEUN) return fail("integrator must be PF_EULER or PF_HEUN");
  if (p->poisson_every < 0) return fail("poisson_every must be >= 0");
  if (p->n_air < 0 || p->n_air >= p->nz) return fail("n_air must be in 0 .. nz - 1");
  if (p->n_air > 0 && p->periodic_z) return fail("air layers need non-periodic z (periodic_z = 0)");
  if (p->extrap_order < 0 || p->extrap_order > 3) return fail("extrap_order must be in 0 .. 3");
  for (int i = 0; i < 2; ++i)
    if (p->reserved[i] != 0) return fail("reserved fields must be zero");
  return true;
}

// Does pf_step start its solves from an extrapolation of the last ones?  (Forward
// Euler: its solves are equally spaced in time, every step or every k-th.)
bool extrapolates(const pf_params* p) {
  return !(p->flags & PF_FLAG_WARM_LAST) && p->integrator == PF_EULER;
}

// FP32 time series keep the potential compensated (see k_cg_finish_comp) unless the
// problem is singular (all-periodic: its mean removal acts on phi alone).
bool comp_buffers(const pf_params* p) { return extrapolates(p) && p->precision == PF_FP32; }

// Is the FP32 polarization state kept compensated (P plus an FP32 remainder,
// see k_tdgl)?  FP32 forward Euler, unless PF_FLAG_PLAIN_FP32 asks for the
// plain state or the context serves the adjoint (whose recomputed segments
// restart from stored states and must repeat the forward pass bit for bit).
bool comp_state(const pf_params* p) {
  return p->precision == PF_FP32 && p->integrator == PF_EULER &&
         !(p->flags & (PF_FLAG_PLAIN_FP32 | PF_FLAG_ADJOINT));
}

Layout layout_of(const pf_params* p) {
  const size_t w = p->precision == PF_FP32 ? 4 : 8;
  const size_t n = (size_t)p->nx * p->ny * p->nz, nxy = (size_t)p->nx * p->ny;
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align_up(bytes);
    return o;
  };
  L.P_alt = take(3 * n * w);
  L.plo = take(comp_state(p) ? 3 * n * 2 : 0);          // bf16
  L.r = take(n * w);
  L.p0 = take(n * w);
  L.p1 = take(n * w);
  L.q = take(n * w);
  L.invd = take(p->has_eps ? n * w : 0);
  for (size_t& h : L.hist) h = take(extrapolates(p) ? n * w : 0);   // ring of past potentials (or differences)
  L.clo = take(comp_buffers(p) ? n * w : 0);    // remainder of the compensated potential
  L.cx = take(comp_buffers(p) ? n * w : 0);     // the solve's correction to it

  L.tlo = take(nxy);
  L.thi = take(nxy);
  L.vlo = take(nxy * w);
  L.vhi = take(nxy * w);
  L.ctr = take(sizeof(long long));   // step counter of the thermal noise (zeroed by pf_bind)
  L.xctr = take(2 * sizeof(long long));   // solves in the extrapolation history, and its block ticket
  // reduction partials: per block (flat kernels) or per tile (plane-march
  // kernels; at most one tile per column group of MTX x MTY and plane)
  const size_t max_tiles = (size_t)((p->nx + pf::MTX - 1) / pf::MTX) * ((p->ny + pf::MTY - 1) / pf::MTY) * p->nz;
  L.part = take(sizeof(double) * std::max<size_t>((size_t)pf::MAX_GRID * pf::MAX_NV, pf::MAX_NV * max_tiles));
  L.S = take(sizeof(Scalars));
  L.diag = take(8 * sizeof(double));
  L.loop = take(2 * sizeof(long long));   // bodies left in a persistent step loop
  if (p->flags & PF_FLAG_ADJOINT) {
    L.adj = true;
    L.psi = take(n * w);
    L.vzero = take(nxy * w);
  }
  L.z = L.zt = 0;
  if (p->solver == PF_PCG_MG) {
    L.mg = mg_levels(p);
    L.z = take(n * w);
    L.zt = take(n * w);
    for (size_t k = 0; k < L.mg.size(); ++k) {
      MgLevelHost& l = L.mg[k];
      if (k == 0) {
        l.f = L.r;
        l.e = L.z;
        l.et = L.zt;
        l.tlo = L.tlo;
        l.thi = L.thi;
      } else {
        l.f = take((size_t)l.n() * w);
        l.e = take((size_t)l.n() * w);
        l.et = take((size_t)l.n() * w);
        l.tlo = take((size_t)l.nxy());
        l.thi = take((size_t)l.nxy());
        if (p->has_eps) {
          l.eps = take((size_t)l.n() * w);
          l.invd = take((size_t)l.n() * w);
        }
      }
    }
  }
  L.total = off;
  return L;
}

}  // namespace

namespace pf {
void set_global_error(const char* what, const char* detail) {
  if (detail) std::snprintf(g_create_error, sizeof(g_create_error), "%s: %s", what, detail);
  else std::snprintf(g_create_error, sizeof(g_create_error), "%s", what);
}
}  // namespace pf

struct pf_ctx {
  pf_params prm;
  cudaStream_t stream = nullptr;
  int device = 0;
  int nsm = 0;
  Geo geo{};
  pf::LaunchCfg L{};
  Layout lay{};
  bool bound = false;
  void* P_user = nullptr;
  void* phi = nullptr;
  const void* eps = nullptr;
  char* ws = nullptr;
  int cur = 0;                    // 0: state in P_user, 1: in the workspace copy
  int singular = 1;               // no Dirichlet face anywhere (or periodic z)
  bool invd_dirty = true;
  int est_iters = 8;              // iterations issued before the first poll
  int est_iters_adj = 8;          // the same for the adjoint solves
  std::vector<int8_t> tlo_h, thi_h;
  Scalars* S_tmpl = nullptr;      // pinned host: template written at each call
  Scalars* S_host = nullptr;      // pinned host: mirror read back
  std::string err;
  int64_t launches = 0;           // kernels launched by the current call
  // Whole-step CUDA graphs, one per (polarization buffer parity, with or
  // without the potential solve); each Krylov loop is a conditional while
  // node driven from the device.  Captured on first use.
  cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaGraphExec_t gloop = nullptr;   // persistent loop: two steps per body, many steps per launch
  bool loop_broken = false;          // the loop graph cannot be built here: one launch per step
  int graph_key = -1;             // singular flag the graphs were captured for
  bool graphs_broken = false;     // capture not possible: host-driven loop
  int64_t graph_steps = 0;        // steps of the current call run as graphs
  int64_t graph_fixed = 0;        // kernels of those steps outside the Krylov loops
  int64_t graph_solves = 0;       // Poisson solves of those steps
  int64_t nstep = 0;              // steps since pf_bind (schedules poisson_every)
  uint64_t gen = 0;               // bumped by every change that invalidates captured graphs
  double noise_sigma = 0.0;       // thermal random force (pf_set_noise)
  unsigned long long noise_seed = 0;
  int tile_bps = 0;               // blocks per SM requested by pf_set_tiling (0: as many as fit)
  int mg_whole = 0;               // 1: no multigrid sweep is split into interior and face launches
  cudaStream_t cap_stream = nullptr;
  bool async_open = false;        // pf_step_async work enqueued since the last pf_step_wait
  int64_t async_steps = 0;        // steps of that work

  // Profiling: events recorded between consecutive launches; each record
  // says which kernel family ran in the interval and what it moved.
  struct Rec {
    int fam;
    double bytes;
    int kind;                     // 0 always runs; 1 CG launch of iteration iter_no (1-based);
                                  // 2 V-cycle number iter_no (0-based) of its solve
    int iter_no;
    int first_bytes_alt;          // 1: cg_p, first iteration moves bytes_first
    double bytes_first;
  };
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  std::vector<Rec> recs;
  bool have_base = false;
  std::vector<pf_kernel_stat> stats;

  pf_status fail(pf_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    err = buf;
    return st;
  }
  pf_status cuda_fail(cudaError_t e, const char* where) {
    return fail(PF_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
  }
};

#define PF_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return ctx->cuda_fail(e_, #call); \
  } while (0)

namespace {

enum Fam {
  F_RHS_MEAN, F_RHS, F_CG_P, F_CG_R, F_FINISH, F_SUB_MEAN, F_TDGL, F_INVDIAG, F_TDGL_ADJ, F_DIAG, F_EXTRAP,
  F_MG_PRE, F_MG_RR, F_MG_COARSE, F_MG_POST1, F_MG_POST2, F_MG_PRR, F_MG_PP, F_COUNT
};
const char* const FAM_NAMES[F_COUNT] = {"rhs_mean", "rhs",      "cg_p",     "cg_r",     "cg_finish",
                                        "sub_mean", "tdgl",     "invdiag",  "tdgl_adj", "diag",     "extrap",
                                        "mg_pre",   "mg_rr",    "mg_bottom", "mg_post1", "mg_post2", "mg_prr",
                                        "mg_pp"};
constexpr int MG_KINDS = F_COUNT - F_MG_PRE;

// Multigrid families are kept per level: family id F_COUNT + level * MG_KINDS + kind.
int mg_fam(int kind, size_t level) { return F_COUNT + (int)level * MG_KINDS + (kind - F_MG_PRE); }

void prof_reset(pf_ctx* ctx) {
  const int total = F_COUNT + MG_KINDS * pf::MG_MAX_LEVELS;
  ctx->stats.assign(total, pf_kernel_stat{});
  for (int f = 0; f < total; ++f) {
    if (f < F_COUNT)
      std::snprintf(ctx->stats[f].name, sizeof(ctx->stats[f].name), "%s", FAM_NAMES[f]);
    else
      std::snprintf(ctx->stats[f].name, sizeof(ctx->stats[f].name), "%s.L%d",
                    FAM_NAMES[F_MG_PRE + (f - F_COUNT) % MG_KINDS], (f - F_COUNT) / MG_KINDS);
  }
  ctx->recs.clear();
  ctx->have_base = false;
}

cudaError_t prof_event(pf_ctx* ctx, size_t i) {
  while (ctx->ev.size() <= i) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    ctx->ev.push_back(e);
  }
  return cudaEventRecord(ctx->ev[i], ctx->stream);
}

// Call before a launch: records the interval's opening event once.
void before_launch(pf_ctx* ctx) {
  if (ctx->prof && !ctx->have_base) {
    prof_event(ctx, 0);
    ctx->have_base = true;
  }
}

// Call after a launch: counts it and closes its timing interval.
void after_launch(pf_ctx* ctx, int fam, double bytes, int kind = 0, int iter_no = 0, double bytes_first = -1.0) {
  ctx->launches += 1;
  if (!ctx->prof) return;
  pf_ctx::Rec r{fam, bytes, kind, iter_no, bytes_first >= 0.0 ? 1 : 0, bytes_first};
  ctx->recs.push_back(r);
  prof_event(ctx, ctx->recs.size());
}

// After a host wait on the stream: turn the recorded intervals into stats.
// CG launches numbered beyond the solve's executed iteration count returned
// at entry and are booked as idle.
void prof_harvest(pf_ctx* ctx, int executed_iters, int done) {
  if (!ctx->prof || !ctx->have_base) return;
  for (size_t i = 0; i < ctx->recs.size(); ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]);
    const pf_ctx::Rec& r = ctx->recs[i];
    pf_kernel_stat& st = ctx->stats[r.fam];
    const bool idle = (r.kind == 1 && r.iter_no > executed_iters) ||
                      (r.kind == 2 && (r.iter_no > executed_iters || (r.iter_no == executed_iters && done)));
    if (idle) {
      st.idle_launches += 1;
      continue;
    }
    st.launches += 1;
    st.total_ms += ms;
    st.bytes += (r.first_bytes_alt && r.iter_no == 1) ? r.bytes_first : r.bytes;
  }
  ctx->recs.clear();
  ctx->have_base = false;
}

template <typename T>
pf::Dev<T> dev_view(pf_ctx* ctx) {
  pf::Dev<T> d{};
  char* ws = ctx->ws;
  const Layout& L = ctx->lay;
  d.phi = (T*)ctx->phi;
  d.eps = ctx->prm.has_eps ? (const T*)ctx->eps : nullptr;
  d.invd = ctx->prm.has_eps ? (T*)(ws + L.invd) : nullptr;
  d.r = (T*)(ws + L.r);
  d.p0 = (T*)(ws + L.p0);
  d.p1 = (T*)(ws + L.p1);
  d.q = (T*)(ws + L.q);
  d.z = L.z ? (T*)(ws + L.z) : nullptr;
  d.bc.tlo = (const int8_t*)(ws + L.tlo);
  d.bc.thi = (const int8_t*)(ws + L.thi);
  d.bc.vlo = (const T*)(ws + L.vlo);
  d.bc.vhi = (const T*)(ws + L.vhi);
  d.part = (double*)(ws + L.part);
  d.S = (Scalars*)(ws + L.S);
  d.plo = comp_state(&ctx->prm) ? (unsigned short*)(ws + L.plo) : nullptr;
  return d;
}

// Thermal-noise arguments of a TDGL launch; advance: the step's last update.
pf::Noise noise_of(pf_ctx* ctx, int advance) {
  pf::Noise nz{};
  nz.amp = ctx->noise_sigma * std::sqrt(ctx->prm.dt);
  nz.seed = ctx->noise_seed;
  nz.step = (long long*)(ctx->ws + ctx->lay.ctr);
  nz.advance = advance;
  return nz;
}

template <typename T>
pf::MgView<T> mg_view(pf_ctx* ctx, size_t k) {
  const MgLevelHost& l = ctx->lay.mg[k];
  pf::MgView<T> v{};
  v.g.nx = l.nx;
  v.g.ny = l.ny;
  v.g.nz = l.nz;
  v.g.periodic_z = ctx->prm.periodic_z;
  v.g.zair = l.nz;
  v.g.nxy = l.nxy();
  v.g.n = l.n();
  v.ax = (T)l.ax;
  v.ay = (T)l.ay;
  v.az = (T)l.az;
  v.fx = l.fx;
  v.fy = l.fy;
  v.fz = l.fz;
  v.tlo = (const int8_t*)(ctx->ws + l.tlo);
  v.thi = (const int8_t*)(ctx->ws + l.thi);
  v.f = (T*)(ctx->ws + l.f);
  v.e = (T*)(ctx->ws + l.e);
  v.et = (T*)(ctx->ws + l.et);
  v.eps = nullptr;
  v.invd = nullptr;
  if (ctx->prm.has_eps) {
    v.eps = k == 0 ? (const T*)ctx->eps : (const T*)(ctx->ws + l.eps);
    v.invd = (const T*)(ctx->ws + (k == 0 ? ctx->lay.invd : l.invd));
  }
  v.mc = l.mc;
  v.split = !ctx->mg_whole && pf::mg_split_level(l.n(), l.nz, ctx->prm.periodic_z, ctx->prm.has_eps) ? 1 : 0;
  return v;
}

// 1/diag(A) of the fine operator when a permittivity field is bound and, for
// the multigrid preconditioner, every coarse level's permittivity and 1/diag
// (after a bind or an electrode change).
template <typename T>
void refresh_invd(pf_ctx* ctx, const pf::LaunchCfg& L, bool count) {
  if (!ctx->prm.has_eps || !ctx->invd_dirty) return;
  const double N = (double)ctx->geo.n, w = sizeof(T);
  if (count) before_launch(ctx);
  pf::launch_invdiag<T>(L, ctx->geo, dev_view<T>(ctx));
  if (count) after_launch(ctx, F_INVDIAG, 2 * N * w);
  else ctx->launches += 1;
  for (size_t k = 1; k < ctx->lay.mg.size(); ++k) {
    const MgLevelHost& l = ctx->lay.mg[k];
    pf::launch_mg_eps_level<T>(L, mg_view<T>(ctx, k - 1), mg_view<T>(ctx, k), (T*)(ctx->ws + l.eps),
                               (T*)(ctx->ws + l.invd));
    ctx->launches += 2;
  }
  ctx->invd_dirty = false;
}

// First level of the one-block V-cycle tail: the first level after the
// finest with at most MG_TAIL_CELLS cells, or the coarsest level (no tail)
// when that leaves fewer than two levels for the tail.
size_t mg_tail_start(const Layout& lay, size_t word) {
  const size_t nl = lay.mg.size();
  size_t k0 = nl - 1;
  for (size_t k = 1; k < nl; ++k)
    if (lay.mg[k].n() <= pf::MG_TAIL_CELLS) {
      k0 = k;
      break;
    }
  // the tail's level arrays must fit in shared memory
  for (; k0 + 1 < nl; ++k0) {
    size_t cells = 0;
    for (size_t k = k0; k < nl; ++k) cells += (size_t)lay.mg[k].n();
    if (3 * cells * word <= (size_t)pf::MG_TAIL_SMEM && nl - k0 <= (size_t)pf::MG_TAIL_LEVELS) break;
  }
  return k0;
}

// One V-cycle z = M^-1 r (number j of its solve, for the profiler): one
// kernel per phase down to level k0, the rest of the cycle in one block.
template <typename T>
void vcycle(pf_ctx* ctx, int j) {
  const size_t nl = ctx->lay.mg.size();
  const size_t k0 = mg_tail_start(ctx->lay, sizeof(T));
  const double w = sizeof(T);
  pf::Scalars* S = (pf::Scalars*)(ctx->ws + ctx->lay.S);
  double* part = (double*)(ctx->ws + ctx->lay.part);
  const double e = ctx->prm.has_eps ? 1.0 : 0.0;   // eps read with the field, 1/diag with f
  // Fused post-sweeps on the finest level keep the pre-smoothed correction out
  // of z (in z_tmp) and put e' in q, which is dead between the residual update
  // and the next search direction.
  const bool fused_post = k0 > 0 && pf::mg_fused_post<T>(mg_view<T>(ctx, 0));
  auto view = [&](size_t k) {
    pf::MgView<T> v = mg_view<T>(ctx, k);
    if (k == 0 && fused_post) v.e = v.et;
    return v;
  };
  for (size_t k = 0; k < k0; ++k) {
    const pf::MgView<T> lv = view(k), cv = view(k + 1);
    const double N = (double)lv.g.n;
    before_launch(ctx);
    const double rest = 1.0 / (lv.fx * lv.fy * lv.fz);
    const double Nf = 2.0 * pf::MG_SPLIT_B * (double)lv.g.nxy;   // cells of the face slabs of a split level
    // fused interior (f read once, e and the coarse rhs written) between the face slabs' own launches
    const int nf = pf::launch_mg_prr<T>(ctx->L, lv, cv, S, [&](int part_no) {
      if (part_no == 0) after_launch(ctx, mg_fam(F_MG_PRE, k), 2 * Nf * w, 2, j);
      else if (part_no == 1) after_launch(ctx, mg_fam(F_MG_PRR, k), (2 + rest) * (N - Nf) * w, 2, j);
      else after_launch(ctx, mg_fam(F_MG_RR, k), (2 + rest) * Nf * w, 2, j);
    });
    if (nf > 0) continue;
    int nk = pf::launch_mg_pre<T>(ctx->L, lv, S);
    after_launch(ctx, mg_fam(F_MG_PRE, k), (2 + 2 * e) * N * w, 2, j);
    ctx->launches += nk - 1;
    nk = pf::launch_mg_rr<T>(ctx->L, lv, cv, S);
    after_launch(ctx, mg_fam(F_MG_RR, k), (2 + e + rest) * N * w, 2, j);
    ctx->launches += nk - 1;
  }
  if (k0 + 1 < nl) {
    pf::MgTail<T> t{};
    t.nl = (int)(nl - k0);
    int off = 0;
    for (size_t k = k0; k < nl; ++k) {
      t.lv[k - k0] = mg_view<T>(ctx, k);
      t.off[k - k0] = off;
      off += 3 * (int)t.lv[k - k0].g.n;
    }
    t.smem_elems = off;
    const double cells = (double)t.lv[0].g.n;
    before_launch(ctx);
    pf::launch_mg_tail<T>(ctx->L, t, ctx->singular, S);
    after_launch(ctx, mg_fam(F_MG_COARSE, k0), 2.0 * cells * w, 2, j);
  } else {
    const pf::MgView<T> cv = mg_view<T>(ctx, nl - 1);
    before_launch(ctx);
    pf::launch_mg_coarse<T>(ctx->L, cv, ctx->singular, S);
    after_launch(ctx, mg_fam(F_MG_COARSE, nl - 1), 2.0 * (double)cv.g.n * w, 2, j);
  }
  for (size_t k = k0; k-- > 0;) {
    const pf::MgView<T> lv = view(k), cv = view(k + 1);
    const double N = (double)lv.g.n;
    before_launch(ctx);
    if (k == 0 && fused_post) {
      T* const z = mg_view<T>(ctx, 0).e;
      const double Nf = 2.0 * pf::MG_SPLIT_B * (double)lv.g.nxy, rest = 1.0 / (lv.fx * lv.fy * lv.fz);
      // face slabs' first sweep, fused interior (e, e_c and f read, the result written), face slabs' second sweep
      pf::launch_mg_pp<T>(ctx->L, lv, cv, (T*)(ctx->ws + ctx->lay.q), z, part, S, [&](int part_no) {
        if (part_no == 0) after_launch(ctx, mg_fam(F_MG_POST1, k), (3 + rest) * Nf * w, 2, j);
        else if (part_no == 1) after_launch(ctx, mg_fam(F_MG_PP, k), (3 + rest) * (N - Nf) * w, 2, j);
        else after_launch(ctx, mg_fam(F_MG_POST2, k), 3 * Nf * w, 2, j);
      });
      continue;
    }
    int nk = pf::launch_mg_post1<T>(ctx->L, lv, cv, S);
    after_launch(ctx, mg_fam(F_MG_POST1, k), (3 + 2 * e + 1.0 / (lv.fx * lv.fy * lv.fz)) * N * w, 2, j);
    ctx->launches += nk - 1;
    nk = pf::launch_mg_post2<T>(ctx->L, lv, k == 0, part, S);
    after_launch(ctx, mg_fam(F_MG_POST2, k), (3 + 2 * e) * N * w, 2, j);
    ctx->launches += nk - 1;
  }
}

void recompute_singular(pf_ctx* ctx) {
  if (ctx->prm.periodic_z) {
    ctx->singular = 1;
    return;
  }
  bool any = false;
  for (int8_t t : ctx->tlo_h) any |= (t == PF_DIRICHLET);
  for (int8_t t : ctx->thi_h) any |= (t == PF_DIRICHLET);
  ctx->singular = any ? 0 : 1;
}

// Reset the per-call solver state on the device.
pf_status reset_scalars(pf_ctx* ctx) {
  ctx->launches = 0;
  ctx->graph_steps = 0;
  ctx->graph_fixed = 0;
  ctx->graph_solves = 0;
  Scalars& s = *ctx->S_tmpl;
  std::memset(&s, 0, sizeof(Scalars));
  s.rtol = ctx->prm.poisson_rtol;
  s.maxit = ctx->prm.poisson_maxit;
  s.done = 1;
  PF_CUDA(cudaMemcpyAsync(ctx->lay.S + ctx->ws, &s, sizeof(Scalars), cudaMemcpyHostToDevice, ctx->stream));
  return PF_OK;
}

pf_status read_scalars(pf_ctx* ctx) {
  PF_CUDA(cudaMemcpyAsync(ctx->S_host, ctx->lay.S + ctx->ws, sizeof(Scalars), cudaMemcpyDeviceToHost,
                          ctx->stream));
  PF_CUDA(cudaStreamSynchronize(ctx->stream));
  return PF_OK;
}

// 1 + the highest order of the extrapolated start.  extrap_order, or
// automatically: a start inherits the previous solves' residuals (each up to
// the tolerance) times the sum of the weights' magnitudes (3, 7, 15 for orders
// 1, 2, 3) and the truncation error of the order.  So the cubic pays at tight
// tolerances, the quadratic at looser ones (above 5e-7), and the linear while
// the thermal noise roughens the potential series.
int extrap_kcap(const pf_ctx* ctx) {
  const int o = ctx->prm.extrap_order;
  if (o > 0) return 1 + o;
  if (ctx->noise_sigma > 0.0) return 2;
  return ctx->prm.poisson_rtol > 5e-7 ? 3 : 4;
}

// Is this context's next step solve compensated (see comp_buffers)?
bool compensated(const pf_ctx* ctx) { return comp_buffers(&ctx->prm) && !ctx->singular; }

// The step solve's view of a compensated potential: the Krylov iterate is the
// correction, the start is the pair phi + lo.
template <typename T>
void comp_view(pf_ctx* ctx, pf::Dev<T>& d) {
  char* ws = ctx->ws;
  d.cp.hi = (T*)ctx->phi;
  d.cp.lo = (T*)(ws + ctx->lay.clo);
  for (int i = 0; i < 3; ++i) d.cp.ring[i] = (T*)(ws + ctx->lay.hist[i]);
  d.cp.nsolve = (long long*)(ws + ctx->lay.xctr);
  d.cp.kcap = extrap_kcap(ctx);
  d.phi = (T*)(ws + ctx->lay.cx);
}

// Does a graph-captured step solve run its second iteration outside the
// Krylov loop too, with the form that reads no correction (compensated
// multigrid solves with eps = 1)?
bool peel_second(const pf_ctx* ctx) {
  return compensated(ctx) && ctx->prm.solver == PF_PCG_MG && !ctx->prm.has_eps;
}

// Does a step solve start with k_extrap?  (Compensated series form their
// start at the end of the solve before.)
bool plain_extrap(const pf_ctx* ctx) { return extrapolates(&ctx->prm) && !compensated(ctx); }

// Extrapolated initial guess of the next step solve, in the bound phi buffer.
template <typename T>
void launch_extrap_of(pf_ctx* ctx, const pf::LaunchCfg& L) {
  long long* xc = (long long*)(ctx->ws + ctx->lay.xctr);
  T* const ring[3] = {(T*)(ctx->ws + ctx->lay.hist[0]), (T*)(ctx->ws + ctx->lay.hist[1]),
                      (T*)(ctx->ws + ctx->lay.hist[2])};
  pf::launch_extrap<T>(L, ctx->geo.n, (T*)ctx->phi, ring, xc, (unsigned*)(xc + 1), extrap_kcap(ctx));
}

// Forget the extrapolation history (the next step solve starts from phi; a
// compensated one from phi + 0 with increment 0 and correction 0).
pf_status reset_history(pf_ctx* ctx) {
  if (!extrapolates(&ctx->prm)) return PF_OK;
  PF_CUDA(cudaMemsetAsync(ctx->ws + ctx->lay.xctr, 0, sizeof(long long), ctx->stream));
  if (comp_buffers(&ctx->prm)) {
    const size_t bytes = (size_t)ctx->geo.n * sizeof(float);
    PF_CUDA(cudaMemsetAsync(ctx->ws + ctx->lay.clo, 0, bytes, ctx->stream));
    PF_CUDA(cudaMemsetAsync(ctx->ws + ctx->lay.cx, 0, bytes, ctx->stream));
    PF_CUDA(cudaMemsetAsync(ctx->ws + ctx->lay.hist[0], 0, bytes, ctx->stream));
  }
  return PF_OK;
}

// The adjoint solve's view: the unknown is psi and every electrode is at 0 V.
template <typename T>
void adjoint_view(pf_ctx* ctx, pf::Dev<T>& d) {
  d.phi = (T*)(ctx->ws + ctx->lay.psi);
  d.bc.vlo = (const T*)(ctx->ws + ctx->lay.vzero);
  d.bc.vhi = d.bc.vlo;
}

// One Poisson solve for the polarization P (device pointer of the current
// state): r0, PCG iterations until the device flag says done, final update.
// adj: solve for the adjoint potential instead (P is then the cotangent).
template <typename T>
pf_status solve(pf_ctx* ctx, const T* P, bool adj = false, bool step_solve = false) {
  pf::Dev<T> d = dev_view<T>(ctx);
  if (adj) adjoint_view<T>(ctx, d);
  const bool comp = step_solve && !adj && compensated(ctx);
  if (comp) comp_view<T>(ctx, d);
  int& est_iters = adj ? ctx->est_iters_adj : ctx->est_iters;
  const Geo& g = ctx->geo;
  const double N = (double)g.n, w = sizeof(T), e = ctx->prm.has_eps ? 1.0 : 0.0;
  refresh_invd<T>(ctx, ctx->L, true);
  if (step_solve && plain_extrap(ctx)) {
    before_launch(ctx);
    launch_extrap_of<T>(ctx, ctx->L);
    after_launch(ctx, F_EXTRAP, 6 * N * w);   // steady state: 4 reads, 2 writes
  }
  if (ctx->singular) {
    before_launch(ctx);
    pf::launch_rhs_mean<T>(ctx->L, g, d, P);
    after_launch(ctx, F_RHS_MEAN, (3 + e) * N * w);
  }
  before_launch(ctx);
  pf::launch_rhs<T>(ctx->L, g, d, P, 0, 0);
  after_launch(ctx, F_RHS, (5 + 2 * e + (comp ? 1 : 0)) * N * w);
  const int mg = ctx->prm.solver == PF_PCG_MG;
  if (mg) vcycle<T>(ctx, 0);
  PF_CUDA(cudaGetLastError());
  // Every issued iteration either runs or returns at entry once the device
  // flag is set, and the device sets it by iteration maxit at the latest.
  const int maxit = ctx->prm.poisson_maxit;
  int issued = 0;
  int batch = std::max(1, std::min(est_iters, maxit));
  for (;;) {
    for (int i = 0; i < batch; ++i) {
      const int it = issued + i + 1;
      before_launch(ctx);
      pf::launch_cg_p<T>(ctx->L, g, d, mg, it == 1, comp && mg && e == 0.0 && it == 2);
      // the multigrid first iteration stages z alone (p = z), except with eps
      // the second iteration of a compensated multigrid solve reads no x (still 0)
      const double cgp = (comp && mg && e == 0.0 && it == 2 ? 5 : 6 + 2 * e) * N * w;
      after_launch(ctx, F_CG_P, cgp, 1, it, (mg && e == 0.0) ? 3 * N * w : (6 + 2 * e) * N * w);
      pf::launch_cg_r<T>(ctx->L, g, d, mg, 0, 0);
      after_launch(ctx, F_CG_R, (3 + e) * N * w, 1, it);
      if (mg) vcycle<T>(ctx, it);
    }
    issued += batch;
    PF_CUDA(cudaGetLastError());
    pf_status st = read_scalars(ctx);
    if (st != PF_OK) return st;
    prof_harvest(ctx, ctx->S_host->iter, ctx->S_host->done);
    if (ctx->S_host->done) break;
    if (issued >= maxit)
      return ctx->fail(PF_ERR_STATE, "internal: solver did not stop after %d iterations", issued);
    batch = std::min(std::max(2, est_iters / 8), maxit - issued);
  }
  const Scalars& s = *ctx->S_host;
  if (!s.zero_x) est_iters = std::max(1, s.iter);
  before_launch(ctx);
  pf::launch_cg_finish<T>(ctx->L, g, d, ctx->singular);
  // compensated: read hi, s, three slots (+ p when an update is owed, + x once
  // written), write hi, s, two slots
  after_launch(ctx, F_FINISH,
               (comp ? 9.0 + (s.pending ? 1.0 : 0.0) + (s.xzero ? 0.0 : 1.0)
                     : s.zero_x ? 1.0 : (s.pending ? 3.0 : 1.0)) * N * w);
  if (ctx->singular) {
    pf::launch_sub_mean<T>(ctx->L, g, d);
    after_launch(ctx, F_SUB_MEAN, 2 * N * w);
  }
  PF_CUDA(cudaGetLastError());
  return PF_OK;
}

void drop_graphs(pf_ctx* ctx) {
  for (cudaGraphExec_t& e : ctx->gexec) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
  if (ctx->gloop) cudaGraphExecDestroy(ctx->gloop);
  ctx->gloop = nullptr;
  ctx->graph_key = -1;
}

// Does step ctx->nstep solve the potential (poisson_every, Section Numerical
// Performance)?
bool refresh_step(const pf_ctx* ctx) {
  const int k = ctx->prm.poisson_every;
  return k <= 1 || ctx->nstep % k == 0;
}

// Kernels of one step outside the Krylov loops, and per Krylov iteration.
// Kernels of one V-cycle: four per level above the tail (two for a split
// level's pre and post1, and for its post2 below the finest), plus the tail or
// the coarse solve.
int64_t vcycle_kernels(const pf_ctx* ctx) {
  const size_t k0 = mg_tail_start(ctx->lay, ctx->prm.precision == PF_FP32 ? 4 : 8);
  int64_t n = 1;
  for (size_t k = 0; k < k0; ++k) {
    const MgLevelHost& l = ctx->lay.mg[k];
    const bool split = !ctx->mg_whole && pf::mg_split_level(l.n(), l.nz, ctx->prm.periodic_z, ctx->prm.has_eps);
    n += 4 + (split ? (k == 0 ? 2 : 3) : 0);
  }
  return n;
}

void step_kernel_counts(const pf_ctx* ctx, int refresh, int64_t* fixed, int64_t* per_iter) {
  const int64_t vc = ctx->prm.solver == PF_PCG_MG ? vcycle_kernels(ctx) : 0;
  const bool heun = ctx->prm.integrator == PF_HEUN;
  const int64_t per_solve = (ctx->singular ? 2 : 0) + 2 + vc + (plain_extrap(ctx) ? 1 : 0);
  *per_iter = 2 + vc;
  // graph-captured multigrid solves run their first iteration (compensated
  // ones their first two) outside the loop
  const int64_t peeled = vc ? *per_iter * (peel_second(ctx) ? 2 : 1) : 0;
  *fixed = (refresh ? (heun ? 2 : 1) * (per_solve + peeled) : 0) + (heun ? 2 : 1);
}

// Append one whole time step of film ctx, reading P from buffer cur, to
// graph after the nodes deps (empty: a root); on return deps holds the
// step's last node.  With refresh = 1 the potential is solved:
//   solve(P)   [b mean] r0 = b - A phi (+ first V-cycle); while { CG
//              iteration (+ V-cycle) } with the condition set by the kernels;
//              last x update [mean removal]
//   Euler      solve(P_n); TDGL update into buffer cur ^ 1
//   Heun       solve(P_n); predictor into buffer cur ^ 1; solve(P^p);
//              corrector back into buffer cur
// Launches are captured on stream st (capture mode thread-local).
template <typename T>
cudaError_t append_step(pf_ctx* ctx, cudaGraph_t graph, std::vector<cudaGraphNode_t>& deps, int cur, int refresh,
                        cudaStream_t st) {
  const pf::LaunchCfg saved = ctx->L;
  const int64_t saved_launches = ctx->launches;
  ctx->L.stream = st;
  pf::Dev<T> d = dev_view<T>(ctx);
  const Geo& g = ctx->geo;
  T* Pbuf[2] = {(T*)ctx->P_user, (T*)(ctx->ws + ctx->lay.P_alt)};
  const double coef[5] = {ctx->prm.a1, ctx->prm.a11, ctx->prm.a12, ctx->prm.g, ctx->prm.dt * ctx->prm.L};
  const int mg = ctx->prm.solver == PF_PCG_MG;
  const bool heun = ctx->prm.integrator == PF_HEUN;
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaError_t e = cudaSuccess;
  // Capture the launches of body after deps; deps becomes the capture's frontier.
  auto segment = [&](auto&& body) {
    if (e != cudaSuccess) return;
    e = cudaStreamBeginCaptureToGraph(st, graph, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), mode);
    if (e != cudaSuccess) return;
    body();
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* fr = nullptr;
    size_t nfr = 0;
    e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &fr, nullptr, &nfr);
    if (e == cudaSuccess) deps.assign(fr, fr + nfr);
    cudaGraph_t g_out = graph;
    const cudaError_t e2 = cudaStreamEndCapture(st, &g_out);
    if (e == cudaSuccess) e = e2;
  };
  // One Poisson solve for the state P with its own loop condition.
  pf::Dev<T> ds = d;
  if (compensated(ctx)) comp_view<T>(ctx, ds);
  auto solve_nodes = [&](const T* P) {
    const pf::Dev<T>& d = ds;
    cudaGraphConditionalHandle h = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    segment([&] {
      if (plain_extrap(ctx)) launch_extrap_of<T>(ctx, ctx->L);
      if (ctx->singular) pf::launch_rhs_mean<T>(ctx->L, g, d, P);
      pf::launch_rhs<T>(ctx->L, g, d, P, h, 1);
      if (mg) {                  // the first iteration (p = z) runs outside the loop
        vcycle<T>(ctx, 0);
        pf::launch_cg_p<T>(ctx->L, g, d, mg, 1);
        pf::launch_cg_r<T>(ctx->L, g, d, mg, h, 1);
        vcycle<T>(ctx, 1);
        if (peel_second(ctx)) {  // and so does the second (x still 0, not read)
          pf::launch_cg_p<T>(ctx->L, g, d, mg, 0, 1);
          pf::launch_cg_r<T>(ctx->L, g, d, mg, h, 1);
          vcycle<T>(ctx, 2);
        }
      }
    });
    if (e != cudaSuccess) return;
    cudaGraphNode_t cnode = nullptr;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&cnode, graph, deps.data(), nullptr, deps.size(), &cp);
    if (e != cudaSuccess) return;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, mode);
    if (e != cudaSuccess) return;
    pf::launch_cg_p<T>(ctx->L, g, d, mg);
    pf::launch_cg_r<T>(ctx->L, g, d, mg, h, 1);
    if (mg) vcycle<T>(ctx, 1);
    e = cudaStreamEndCapture(st, &body);
    deps.assign(1, cnode);
    segment([&] {
      pf::launch_cg_finish<T>(ctx->L, g, d, ctx->singular);
      if (ctx->singular) pf::launch_sub_mean<T>(ctx->L, g, d);
    });
  };
  T* Pn = Pbuf[cur];
  T* Pq = Pbuf[cur ^ 1];
  if (refresh) solve_nodes(Pn);
  if (heun) {
    segment([&] { pf::launch_tdgl<T>(ctx->L, g, d, Pn, Pq, coef, 0, noise_of(ctx, 0)); });
    if (refresh) solve_nodes(Pq);
    segment([&] { pf::launch_tdgl<T>(ctx->L, g, d, Pq, Pn, coef, 1, noise_of(ctx, 1)); });
  } else {
    segment([&] { pf::launch_tdgl<T>(ctx->L, g, d, Pn, Pq, coef, 0, noise_of(ctx, 1)); });
  }
  ctx->L = saved;
  ctx->launches = saved_launches;
  return e;
}

// Capture one whole time step of this film as its own executable graph.
template <typename T>
pf_status capture_step(pf_ctx* ctx, int cur, int refresh, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaGraphNode_t> deps;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  if (e == cudaSuccess) e = append_step<T>(ctx, graph, deps, cur, refresh, ctx->cap_stream);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ctx->fail(PF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  }
  *out = exec;
  return PF_OK;
}

// One graph running pairs of forward-Euler steps in a device-driven while
// loop: a conditional node whose body is the step from buffer 0, the step
// from buffer 1 and k_loop_next, which counts the bodies down (every step
// solves the potential: poisson_every <= 1).  A multi-step call then costs
// one graph launch however many steps it takes.
template <typename T>
pf_status capture_loop(pf_ctx* ctx, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  cudaGraphConditionalHandle h = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    std::vector<cudaGraphNode_t> deps;
    e = append_step<T>(ctx, body, deps, 0, 1, ctx->cap_stream);
    if (e == cudaSuccess) e = append_step<T>(ctx, body, deps, 1, 1, ctx->cap_stream);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(ctx->cap_stream, body, deps.data(), nullptr, deps.size(),
                                        cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      pf::launch_loop_next((long long*)(ctx->ws + ctx->lay.loop), h, ctx->cap_stream);
      cudaGraph_t g2 = body;
      e = cudaStreamEndCapture(ctx->cap_stream, &g2);
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ctx->fail(PF_ERR_CUDA, "step loop graph: %s", cudaGetErrorString(e));
  }
  *out = exec;
  return PF_OK;
}

// Graph-launched steps: no host round trip inside a step.  Returns false
// (nothing launched) when graphs cannot be used here.
template <typename T>
bool run_steps_graph(pf_ctx* ctx, int nsteps, pf_status* st) {
  *st = PF_OK;
  if (ctx->prof || ctx->graphs_broken || nsteps == 0 || (ctx->prm.flags & PF_FLAG_NO_GRAPHS)) return false;
  if (ctx->graph_key != ctx->singular) {
    drop_graphs(ctx);
    if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      ctx->graphs_broken = true;
      return false;
    }
    // the graph of the first step is captured here, so that a failing
    // capture falls back to host-driven steps before anything is launched
    const int slot = ctx->cur * 2 + (refresh_step(ctx) ? 1 : 0);
    if (capture_step<T>(ctx, ctx->cur, slot & 1, &ctx->gexec[slot]) != PF_OK) {
      drop_graphs(ctx);
      ctx->graphs_broken = true;
      ctx->err.clear();
      return false;
    }
    ctx->graph_key = ctx->singular;
  }
  refresh_invd<T>(ctx, ctx->L, false);
  const bool heun = ctx->prm.integrator == PF_HEUN;
  // many forward-Euler steps that all solve: pairs of them in one persistent launch
  if (!heun && ctx->prm.poisson_every <= 1 && ctx->cur == 0 && nsteps >= 4 && !ctx->loop_broken) {
    if (!ctx->gloop && capture_loop<T>(ctx, &ctx->gloop) != PF_OK) {
      ctx->loop_broken = true;           // one launch per step from here on
      ctx->err.clear();
    }
    if (ctx->gloop) {
      const long long pairs = nsteps / 2;
      pf::launch_loop_set((long long*)(ctx->ws + ctx->lay.loop), pairs, ctx->stream);
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaGraphLaunch(ctx->gloop, ctx->stream);
      if (e != cudaSuccess) {
        *st = ctx->cuda_fail(e, "persistent step loop");
        return true;
      }
      int64_t fixed = 0, per_iter = 0;
      step_kernel_counts(ctx, 1, &fixed, &per_iter);
      ctx->graph_fixed += 2 * pairs * fixed + pairs;   // and the counter kernel of every body
      ctx->launches += 1;                              // the count setter
      ctx->graph_solves += 2 * pairs;
      ctx->graph_steps += 2 * pairs;
      ctx->nstep += 2 * pairs;
      nsteps -= (int)(2 * pairs);
    }
  }
  for (int s = 0; s < nsteps; ++s) {
    const int refresh = refresh_step(ctx) ? 1 : 0;
    const int slot = ctx->cur * 2 + refresh;
    if (!ctx->gexec[slot]) {
      const pf_status cs = capture_step<T>(ctx, ctx->cur, refresh, &ctx->gexec[slot]);
      if (cs != PF_OK) {
        *st = cs;
        return true;
      }
    }
    const cudaError_t e = cudaGraphLaunch(ctx->gexec[slot], ctx->stream);
    if (e != cudaSuccess) {
      *st = ctx->cuda_fail(e, "cudaGraphLaunch");
      return true;
    }
    int64_t fixed = 0, per_iter = 0;
    step_kernel_counts(ctx, refresh, &fixed, &per_iter);
    ctx->graph_fixed += fixed;
    ctx->graph_solves += refresh ? (heun ? 2 : 1) : 0;
    ctx->graph_steps += 1;
    if (!heun) ctx->cur ^= 1;
    ctx->nstep += 1;
  }
  return true;
}

// Copy the state back into the bound P buffer when the last step left it in
// the workspace copy.
template <typename T>
pf_status consolidate(pf_ctx* ctx) {
  if (ctx->cur == 1) {
    PF_CUDA(cudaMemcpyAsync(ctx->P_user, ctx->ws + ctx->lay.P_alt, sizeof(T) * 3 * (size_t)ctx->geo.n,
                            cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->cur = 0;
  }
  return PF_OK;
}

// Run nsteps steps; with keep_parity the state may stay in the workspace copy
// (ctx->cur = 1) for the caller to read or consolidate.
template <typename T>
pf_status run_steps(pf_ctx* ctx, int nsteps, bool keep_parity = false) {
  pf::Dev<T> d = dev_view<T>(ctx);
  const Geo& g = ctx->geo;
  T* Pbuf[2] = {(T*)ctx->P_user, (T*)(ctx->ws + ctx->lay.P_alt)};
  const double coef[5] = {ctx->prm.a1, ctx->prm.a11, ctx->prm.a12, ctx->prm.g, ctx->prm.dt * ctx->prm.L};
  const bool heun = ctx->prm.integrator == PF_HEUN;
  // compensated state: 3 bf16 remainders read and written, 6 half-words = 3 words
  const double tdgl_bytes = (comp_state(&ctx->prm) ? 10.0 : 7.0) * (double)g.n * sizeof(T);
  pf_status gst;
  if (run_steps_graph<T>(ctx, nsteps, &gst)) {
    if (gst != PF_OK) return gst;
    nsteps = 0;
  }
  for (int s = 0; s < nsteps; ++s) {
    const bool refresh = refresh_step(ctx);
    T* P = Pbuf[ctx->cur];
    T* Q = Pbuf[ctx->cur ^ 1];
    if (refresh) {
      pf_status st = solve<T>(ctx, P, false, true);
      if (st != PF_OK) return st;
    }
    before_launch(ctx);
    pf::launch_tdgl<T>(ctx->L, g, d, P, Q, coef, 0, noise_of(ctx, heun ? 0 : 1));
    after_launch(ctx, F_TDGL, tdgl_bytes);
    PF_CUDA(cudaGetLastError());
    if (heun) {
      if (refresh) {
        pf_status st = solve<T>(ctx, Q, false, true);
        if (st != PF_OK) return st;
      }
      before_launch(ctx);
      pf::launch_tdgl<T>(ctx->L, g, d, Q, P, coef, 1, noise_of(ctx, 1));
      after_launch(ctx, F_TDGL, tdgl_bytes + 3.0 * (double)g.n * sizeof(T));
      PF_CUDA(cudaGetLastError());
    } else {
      ctx->cur ^= 1;
    }
    ctx->nstep += 1;
  }
  if (keep_parity) return PF_OK;
  return consolidate<T>(ctx);
}

// Copy the host face masks to the device: the fine level and, for the
// multigrid hierarchy, every coarse level (a coarse face cell is an electrode
// where any of its fine children is).  Waits for the copies.
pf_status upload_masks(pf_ctx* ctx) {
  const Layout& L = ctx->lay;
  PF_CUDA(cudaMemcpyAsync(ctx->ws + L.tlo, ctx->tlo_h.data(), ctx->tlo_h.size(), cudaMemcpyHostToDevice,
                          ctx->stream));
  PF_CUDA(cudaMemcpyAsync(ctx->ws + L.thi, ctx->thi_h.data(), ctx->thi_h.size(), cudaMemcpyHostToDevice,
                          ctx->stream));
  // masks[2k], masks[2k+1]: z_lo / z_hi masks of level k (kept alive until the copies finish)
  std::vector<std::vector<int8_t>> masks;
  masks.reserve(2 * L.mg.size() + 2);
  masks.push_back(ctx->tlo_h);
  masks.push_back(ctx->thi_h);
  for (size_t k = 0; k + 1 < L.mg.size(); ++k) {
    const MgLevelHost &f = L.mg[k], &c = L.mg[k + 1];
    std::vector<int8_t> clo((size_t)c.nxy(), 0), chi((size_t)c.nxy(), 0);
    const std::vector<int8_t>&flo = masks[2 * k], &fhi = masks[2 * k + 1];
    for (int y = 0; y < f.ny; ++y)
      for (int x = 0; x < f.nx; ++x) {
        const size_t fi = (size_t)y * f.nx + x, ci = (size_t)(y / f.fy) * c.nx + x / f.fx;
        clo[ci] = std::max(clo[ci], flo[fi]);
        chi[ci] = std::max(chi[ci], fhi[fi]);
      }
    masks.push_back(std::move(clo));
    masks.push_back(std::move(chi));
    PF_CUDA(cudaMemcpyAsync(ctx->ws + c.tlo, masks[2 * k + 2].data(), (size_t)c.nxy(), cudaMemcpyHostToDevice,
                            ctx->stream));
    PF_CUDA(cudaMemcpyAsync(ctx->ws + c.thi, masks[2 * k + 3].data(), (size_t)c.nxy(), cudaMemcpyHostToDevice,
                            ctx->stream));
  }
  PF_CUDA(cudaStreamSynchronize(ctx->stream));
  return PF_OK;
}

pf_status finish_info(pf_ctx* ctx, int nsteps, pf_step_info* info) {
  pf_status st = read_scalars(ctx);
  if (st != PF_OK) return st;
  prof_harvest(ctx, 0, 1);
  const Scalars& s = *ctx->S_host;
  pf_status result = PF_OK;
  if (s.nonfinite) result = ctx->fail(PF_ERR_NONFINITE, "non-finite value in the Poisson solver scalars");
  else if (s.nonconv) result = ctx->fail(PF_ERR_NOCONV, "%d Poisson solve(s) hit poisson_maxit", s.nonconv);
  if (info) {
    info->steps_done = nsteps;
    info->last_iters = s.last_iters;
    info->total_iters = s.total_iters;
    info->last_relres = s.last_rel;
    info->nonconverged = s.nonconv;
    info->status = result;
    int64_t fixed = 0, per_iter = 0;
    step_kernel_counts(ctx, 1, &fixed, &per_iter);
    // graph-launched steps: kernels = fixed part + one loop body per iteration
    // (multigrid: per iteration after the first, which is in the fixed part)
    // loop bodies: the iterations past the peeled ones, sum of max(0, iters - peeled)
    const int64_t mg = ctx->prm.solver == PF_PCG_MG;
    const int64_t bodies = !mg ? s.total_iters
                           : peel_second(ctx)
                               ? s.total_iters - 2 * ctx->graph_solves + s.zero_solves + s.short_solves
                               : s.total_iters + s.zero_solves - ctx->graph_solves;
    info->kernel_launches = ctx->launches + (ctx->graph_steps ? ctx->graph_fixed + bodies * per_iter : 0);
    info->graph_steps = ctx->graph_steps;
    info->max_iters = s.max_iters;
    info->solves = s.solves;
  }
  return result;
}

pf_status check_ready(pf_ctx* ctx) {
  if (!ctx) return PF_ERR_ARG;
  if (!ctx->bound) return ctx->fail(PF_ERR_STATE, "no buffers bound (call pf_bind first)");
  return PF_OK;
}

// Bound, and no pf_step_async work waiting for its pf_step_wait.
pf_status idle_ready(pf_ctx* ctx) {
  const pf_status st = check_ready(ctx);
  if (st != PF_OK) return st;
  if (ctx->async_open) return ctx->fail(PF_ERR_STATE, "pf_step_async work is pending (call pf_step_wait first)");
  return PF_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

size_t pf_workspace_bytes(const pf_params* params) {
  if (!params_valid(params, nullptr)) return 0;
  return layout_of(params).total;
}

pf_status pf_create(const pf_params* params, void* cuda_stream, pf_ctx** out) {
  std::string why;
  if (!out) {
    pf::set_global_error("out is NULL");
    return PF_ERR_ARG;
  }
  *out = nullptr;
  if (!params_valid(params, &why)) {
    pf::set_global_error(why.c_str());
    return PF_ERR_ARG;
  }
  pf_ctx* ctx = new pf_ctx();
  ctx->prm = *params;
  ctx->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->S_tmpl, 2 * sizeof(Scalars));
  if (e != cudaSuccess) {
    pf::set_global_error("CUDA", cudaGetErrorString(e));
    delete ctx;
    return PF_ERR_CUDA;
  }
  ctx->S_host = ctx->S_tmpl + 1;
  Geo& g = ctx->geo;
  pf::setup_launch(params, ctx->nsm, ctx->stream, g, ctx->L);
  ctx->lay = layout_of(params);
  if (!ctx->lay.mg.empty()) {
    const int rmg = ctx->nsm * (params->precision == PF_FP32 ? pf::mg_blocks_per_sm<float>()
                                                             : pf::mg_blocks_per_sm<double>());
    for (MgLevelHost& l : ctx->lay.mg)
      l.mc = pf::march_cfg(l.nx, l.ny, l.nz, rmg, l.fz == 2, params->precision == PF_FP32 ? 4 : 8);
  }
  ctx->tlo_h.assign((size_t)g.nxy, 0);
  ctx->thi_h.assign((size_t)g.nxy, 0);
  recompute_singular(ctx);
  prof_reset(ctx);
  *out = ctx;
  return PF_OK;
}

pf_status pf_bind(pf_ctx* ctx, void* P, void* phi, const void* eps, void* workspace, size_t workspace_bytes) {
  if (!ctx) return PF_ERR_ARG;
  if (ctx->async_open) return ctx->fail(PF_ERR_STATE, "pf_step_async work is pending (call pf_step_wait first)");
  ctx->bound = false;
  if (!P || !phi || !workspace) return ctx->fail(PF_ERR_ARG, "P, phi and workspace must be non-NULL");
  if (ctx->prm.has_eps && !eps) return ctx->fail(PF_ERR_ARG, "has_eps = 1 but eps is NULL");
  if (workspace_bytes < ctx->lay.total)
    return ctx->fail(PF_ERR_ARG, "workspace too small: %zu < %zu bytes", workspace_bytes, ctx->lay.total);
  if (((uintptr_t)workspace % ALIGN) != 0) return ctx->fail(PF_ERR_ARG, "workspace must be 256-byte aligned");
  if (((uintptr_t)P % 16) || ((uintptr_t)phi % 16) || (eps && ctx->prm.has_eps && ((uintptr_t)eps % 16)))
    return ctx->fail(PF_ERR_ARG, "P, phi and eps must be 16-byte aligned");
  if (!is_device_ptr(P) || !is_device_ptr(phi) || !is_device_ptr(workspace) ||
      (ctx->prm.has_eps && !is_device_ptr(eps)))
    return ctx->fail(PF_ERR_ARG, "P, phi, eps and workspace must be device pointers");
  drop_graphs(ctx);
  ctx->gen += 1;
  ctx->P_user = P;
  ctx->phi = phi;
  ctx->eps = ctx->prm.has_eps ? eps : nullptr;
  ctx->ws = (char*)workspace;
  ctx->cur = 0;
  ctx->nstep = 0;
  ctx->invd_dirty = true;
  const Layout& L = ctx->lay;
  PF_CUDA(cudaMemsetAsync(ctx->ws + L.tlo, 0, L.part - L.tlo, ctx->stream));
  std::fill(ctx->tlo_h.begin(), ctx->tlo_h.end(), 0);
  std::fill(ctx->thi_h.begin(), ctx->thi_h.end(), 0);
  recompute_singular(ctx);
  PF_CUDA(cudaMemsetAsync(ctx->ws + L.S, 0, sizeof(Scalars), ctx->stream));
  if (comp_state(&ctx->prm))
    PF_CUDA(cudaMemsetAsync(ctx->ws + L.plo, 0, 3 * (size_t)ctx->geo.n * sizeof(unsigned short), ctx->stream));
  if (L.adj) {
    const size_t w = ctx->prm.precision == PF_FP32 ? 4 : 8;
    PF_CUDA(cudaMemsetAsync(ctx->ws + L.psi, 0, (size_t)ctx->geo.n * w, ctx->stream));
    PF_CUDA(cudaMemsetAsync(ctx->ws + L.vzero, 0, (size_t)ctx->geo.nxy * w, ctx->stream));
  }
  pf_status ms = upload_masks(ctx);
  if (ms != PF_OK) return ms;
  ctx->bound = true;
  return PF_OK;
}

pf_status pf_set_bc(pf_ctx* ctx, int32_t face, const int8_t* type_xy, const double* volts_xy) {
  pf_status st = idle_ready(ctx);
  if (st != PF_OK) return st;
  if (face != PF_ZLO && face != PF_ZHI) return ctx->fail(PF_ERR_ARG, "face must be PF_ZLO or PF_ZHI");
  if (!type_xy) return ctx->fail(PF_ERR_ARG, "type_xy is NULL");
  const size_t nxy = (size_t)ctx->geo.nxy;
  for (size_t i = 0; i < nxy; ++i)
    if (type_xy[i] != PF_NEUMANN && type_xy[i] != PF_DIRICHLET)
      return ctx->fail(PF_ERR_ARG, "type_xy[%zu] = %d is neither PF_NEUMANN nor PF_DIRICHLET", i, (int)type_xy[i]);
  if (volts_xy)
    for (size_t i = 0; i < nxy; ++i)
      if (!std::isfinite(volts_xy[i])) return ctx->fail(PF_ERR_ARG, "volts_xy[%zu] is not finite", i);
  const Layout& L = ctx->lay;
  char* vdst = ctx->ws + (face == PF_ZLO ? L.vlo : L.vhi);
  if (ctx->prm.precision == PF_FP32) {
    std::vector<float> v(nxy, 0.f);
    if (volts_xy)
      for (size_t i = 0; i < nxy; ++i) v[i] = (float)volts_xy[i];
    PF_CUDA(cudaMemcpyAsync(vdst, v.data(), nxy * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    PF_CUDA(cudaStreamSynchronize(ctx->stream));
  } else {
    std::vector<double> v(nxy, 0.0);
    if (volts_xy) std::memcpy(v.data(), volts_xy, nxy * sizeof(double));
    PF_CUDA(cudaMemcpyAsync(vdst, v.data(), nxy * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    PF_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  std::vector<int8_t>& h = face == PF_ZLO ? ctx->tlo_h : ctx->thi_h;
  const bool types_changed = std::memcmp(h.data(), type_xy, nxy) != 0;
  std::memcpy(h.data(), type_xy, nxy);
  recompute_singular(ctx);
  ctx->invd_dirty = true;
  ctx->gen += 1;
  if (types_changed) {           // a new electrode layout: the old potentials are no guide
    st = reset_history(ctx);
    if (st != PF_OK) return st;
  }
  return upload_masks(ctx);
}

pf_status pf_step_async(pf_ctx* ctx, int32_t nsteps) {
  pf_status st = check_ready(ctx);
  if (st != PF_OK) return st;
  if (nsteps < 0) return ctx->fail(PF_ERR_ARG, "nsteps must be >= 0");
  if (!ctx->async_open) {
    st = reset_scalars(ctx);
    if (st != PF_OK) return st;
    ctx->async_open = true;
    ctx->async_steps = 0;
  }
  st = ctx->prm.precision == PF_FP32 ? run_steps<float>(ctx, nsteps) : run_steps<double>(ctx, nsteps);
  if (st != PF_OK) {
    ctx->async_open = false;
    ctx->async_steps = 0;
    return st;
  }
  ctx->async_steps += nsteps;
  return PF_OK;
}

pf_status pf_step_wait(pf_ctx* ctx, pf_step_info* info) {
  pf_status st = check_ready(ctx);
  if (st != PF_OK) return st;
  if (!ctx->async_open) {          // nothing pending: an empty report
    st = reset_scalars(ctx);
    if (st != PF_OK) return st;
  }
  const int64_t n = ctx->async_steps;
  ctx->async_open = false;
  ctx->async_steps = 0;
  return finish_info(ctx, (int)n, info);
}

pf_status pf_step(pf_ctx* ctx, int32_t nsteps, pf_step_info* info) {
  const pf_status st = pf_step_async(ctx, nsteps);
  if (st != PF_OK) return st;
  return pf_step_wait(ctx, info);
}

pf_status pf_step_host(pf_ctx* ctx, void* P_host, void* phi_host, int32_t nsteps, pf_step_info* info) {
  pf_status st = idle_ready(ctx);
  if (st != PF_OK) return st;
  if (!P_host || !phi_host) return ctx->fail(PF_ERR_ARG, "P_host and phi_host must be non-NULL");
  if (nsteps < 0) return ctx->fail(PF_ERR_ARG, "nsteps must be >= 0");
  const size_t w = ctx->prm.precision == PF_FP32 ? 4 : 8;
  const size_t n = (size_t)ctx->geo.n;
  st = reset_scalars(ctx);
  if (st != PF_OK) return st;
  // The state goes to and comes from whichever polarization buffer the step
  // reads and writes, so no device-side copy is needed between steps.
  auto pbuf = [&]() -> void* { return ctx->cur ? (void*)(ctx->ws + ctx->lay.P_alt) : ctx->P_user; };
  for (int s = 0; s < nsteps; ++s) {
    PF_CUDA(cudaMemcpyAsync(pbuf(), P_host, 3 * n * w, cudaMemcpyHostToDevice, ctx->stream));
    PF_CUDA(cudaMemcpyAsync(ctx->phi, phi_host, n * w, cudaMemcpyHostToDevice, ctx->stream));
    st = ctx->prm.precision == PF_FP32 ? run_steps<float>(ctx, 1, true) : run_steps<double>(ctx, 1, true);
    if (st != PF_OK) return st;
    PF_CUDA(cudaMemcpyAsync(P_host, pbuf(), 3 * n * w, cudaMemcpyDeviceToHost, ctx->stream));
    PF_CUDA(cudaMemcpyAsync(phi_host, ctx->phi, n * w, cudaMemcpyDeviceToHost, ctx->stream));
  }
  st = ctx->prm.precision == PF_FP32 ? consolidate<float>(ctx) : consolidate<double>(ctx);
  if (st != PF_OK) return st;
  return finish_info(ctx, nsteps, info);
}

pf_status pf_true_residual(pf_ctx* ctx, const void* P, double* out) {
  pf_status st = idle_ready(ctx);
  if (st != PF_OK) return st;
  if (!out) return ctx->fail(PF_ERR_ARG, "out is NULL");
  const size_t w = ctx->prm.precision == PF_FP32 ? 4 : 8;
  if (P && (((uintptr_t)P % w) != 0 || !is_device_ptr(P)))
    return ctx->fail(PF_ERR_ARG, "P must be NULL or an aligned device pointer");
  const void* Pp = P ? P : ctx->P_user;
  double* dres = (double*)(ctx->ws + ctx->lay.diag);
  if (ctx->prm.precision == PF_FP32) {
    pf::Dev<float> d = dev_view<float>(ctx);
    if (compensated(ctx)) {             // the compensated potential: bound phi + remainder
      pf::Dev<float> dc = d;
      comp_view<float>(ctx, dc);
      d.cp = dc.cp;
    }
    pf::launch_true_residual<float>(ctx->L, ctx->geo, d, (const float*)Pp, ctx->singular, dres);
  } else {
    pf::launch_true_residual<double>(ctx->L, ctx->geo, dev_view<double>(ctx), (const double*)Pp, ctx->singular,
                                     dres);
  }
  PF_CUDA(cudaGetLastError());
  double h[3];
  PF_CUDA(cudaMemcpyAsync(h, dres, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PF_CUDA(cudaStreamSynchronize(ctx->stream));
  out[0] = std::sqrt(h[0]);
  out[1] = std::sqrt(h[1]);
  out[2] = std::sqrt(h[2]);
  return PF_OK;
}

pf_status pf_solve_potential(pf_ctx* ctx, pf_step_info* info) {
  pf_status st = idle_ready(ctx);
  if (st != PF_OK) return st;
  if (ctx->cur != 0) return ctx->fail(PF_ERR_STATE, "internal: state not in the bound P buffer");
  st = reset_scalars(ctx);
  if (st != PF_OK) return st;
  st = ctx->prm.precision == PF_FP32 ? solve<float>(ctx, (const float*)ctx->P_user)
                                     : solve<double>(ctx, (const double*)ctx->P_user);
  if (st != PF_OK) return st;
  st = reset_history(ctx);
  if (st != PF_OK) return st;
  return finish_info(ctx, 0, info);
}

pf_status pf_adjoint_step(pf_ctx* ctx, const void* lam_in, void* lam_out, double* grad_params,
                          double* grad_volts, pf_step_info* info) {
  pf_status st = idle_ready(ctx);
  if (st != PF_OK) return st;
  if (!ctx->lay.adj) return ctx->fail(PF_ERR_STATE, "the context was created without PF_FLAG_ADJOINT");
  if (ctx->prm.integrator != PF_EULER || ctx->prm.poisson_every > 1 || ctx->noise_sigma != 0.0 || ctx->prm.n_air > 0)
    return ctx->fail(PF_ERR_NOTIMPL, "the adjoint step exists for forward Euler with a solve every step, no thermal "
                                     "noise and no air layers only");
  if (!lam_in || !lam_out || !grad_params) return ctx->fail(PF_ERR_ARG, "lam_in, lam_out and grad_params must be non-NULL");
  if (((uintptr_t)lam_in % 16) || ((uintptr_t)lam_out % 16))
    return ctx->fail(PF_ERR_ARG, "lam_in and lam_out must be 16-byte aligned");
  if (((uintptr_t)grad_params % 8) || ((uintptr_t)grad_volts % 8))
    return ctx->fail(PF_ERR_ARG, "grad_params and grad_volts must be 8-byte aligned");
  if (!is_device_ptr(lam_in) || !is_device_ptr(lam_out) || !is_device_ptr(grad_params) ||
      (grad_volts && !is_device_ptr(grad_volts)))
    return ctx->fail(PF_ERR_ARG, "lam_in, lam_out, grad_params and grad_volts must be device pointers");
  const size_t w = ctx->prm.precision == PF_FP32 ? 4 : 8;
  const size_t n = (size_t)ctx->geo.n;
  auto overlap = [](const void* a, size_t na, const void* b, size_t nb) {
    const char *pa = (const char*)a, *pb = (const char*)b;
    return pa < pb + nb && pb < pa + na;
  };
  if (overlap(lam_out, 3 * n * w, lam_in, 3 * n * w) || overlap(lam_out, 3 * n * w, ctx->P_user, 3 * n * w) ||
      overlap(lam_out, 3 * n * w, ctx->phi, n * w) || overlap(lam_out, 3 * n * w, ctx->ws, ctx->lay.total))
    return ctx->fail(PF_ERR_ARG, "lam_out overlaps lam_in or a bound buffer");
  if (ctx->cur != 0) return ctx->fail(PF_ERR_STATE, "internal: state not in the bound P buffer");
  st = reset_scalars(ctx);
  if (st != PF_OK) return st;
  const double coef[5] = {ctx->prm.a1, ctx->prm.a11, ctx->prm.a12, ctx->prm.g, ctx->prm.dt * ctx->prm.L};
  double* gv_lo = grad_volts;
  double* gv_hi = grad_volts ? grad_volts + ctx->geo.nxy : nullptr;
  if (ctx->prm.precision == PF_FP32) {
    st = solve<float>(ctx, (const float*)lam_in, true);
    if (st != PF_OK) return st;
    pf::Dev<float> d = dev_view<float>(ctx);
    before_launch(ctx);
    pf::launch_tdgl_adj<float>(ctx->L, ctx->geo, d, (const float*)lam_in, (float*)lam_out,
                               (const float*)(ctx->ws + ctx->lay.psi), (const float*)ctx->P_user, coef,
                               grad_params, gv_lo, gv_hi);
  } else {
    st = solve<double>(ctx, (const double*)lam_in, true);
    if (st != PF_OK) return st;
    pf::Dev<double> d = dev_view<double>(ctx);
    before_launch(ctx);
    pf::launch_tdgl_adj<double>(ctx->L, ctx->geo, d, (const double*)lam_in, (double*)lam_out,
                                (const double*)(ctx->ws + ctx->lay.psi), (const double*)ctx->P_user, coef,
                                grad_params, gv_lo, gv_hi);
  }
  after_launch(ctx, F_TDGL_ADJ, 10.0 * (double)n * w);
  PF_CUDA(cudaGetLastError());
  return finish_info(ctx, 0, info);
}

pf_status pf_diagnostics(pf_ctx* ctx, double threshold, double* out) {
  pf_status st = idle_ready(ctx);
  if (st != PF_OK) return st;
  if (!out) return ctx->fail(PF_ERR_ARG, "out is NULL");
  if (!std::isfinite(threshold)) return ctx->fail(PF_ERR_ARG, "threshold must be finite");
  if (ctx->cur != 0) return ctx->fail(PF_ERR_STATE, "internal: state not in the bound P buffer");
  const double coef[4] = {ctx->prm.a1, ctx->prm.a11, ctx->prm.a12, threshold};
  double* dsum = (double*)(ctx->ws + ctx->lay.diag);
  ctx->launches = 0;
  before_launch(ctx);
  if (ctx->prm.precision == PF_FP32)
    pf::launch_diag<float>(ctx->L, ctx->geo, dev_view<float>(ctx), (const float*)ctx->P_user, coef, dsum);
  else
    pf::launch_diag<double>(ctx->L, ctx->geo, dev_view<double>(ctx), (const double*)ctx->P_user, coef, dsum);
  after_launch(ctx, F_DIAG, 4.0 * (double)ctx->geo.n * (ctx->prm.precision == PF_FP32 ? 4 : 8));
  PF_CUDA(cudaGetLastError());
  double h[8];
  PF_CUDA(cudaMemcpyAsync(h, dsum, 7 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PF_CUDA(cudaStreamSynchronize(ctx->stream));
  prof_harvest(ctx, 0, 1);
  const double n = (double)ctx->geo.n;
  out[0] = h[0] / n;
  out[1] = h[1] / n;
  out[2] = h[2] / n;
  out[3] = h[3] / n;
  out[4] = h[4];
  out[5] = 0.5 * ctx->prm.g * h[5] * ctx->geo.ih2;
  out[6] = -0.5 * h[6];
  return PF_OK;
}

pf_status pf_profile_enable(pf_ctx* ctx, int32_t enable) {
  if (!ctx) return PF_ERR_ARG;
  if (ctx->async_open) return ctx->fail(PF_ERR_STATE, "pf_step_async work is pending (call pf_step_wait first)");
  if (enable != 0 && enable != 1) return ctx->fail(PF_ERR_ARG, "enable must be 0 or 1");
  ctx->prof = enable == 1;
  prof_reset(ctx);
  return PF_OK;
}

int32_t pf_profile_read(const pf_ctx* ctx, pf_kernel_stat* out, int32_t max) {
  if (!ctx) return -1;
  const int32_t n = (int32_t)ctx->stats.size();
  for (int32_t i = 0; i < n && i < max && out; ++i) out[i] = ctx->stats[i];
  return n;
}


pf_status pf_set_noise(pf_ctx* ctx, double sigma, uint64_t seed) {
  if (!ctx) return PF_ERR_ARG;
  if (ctx->async_open) return ctx->fail(PF_ERR_STATE, "pf_step_async work is pending (call pf_step_wait first)");
  if (!std::isfinite(sigma) || sigma < 0.0) return ctx->fail(PF_ERR_ARG, "sigma must be finite and >= 0");
  drop_graphs(ctx);
  ctx->noise_sigma = sigma;
  ctx->noise_seed = (unsigned long long)seed;
  ctx->gen += 1;
  return PF_OK;
}

pf_status pf_get_tiling(const pf_ctx* ctx, pf_tiling* out) {
  if (!ctx) return PF_ERR_ARG;
  if (!out) return const_cast<pf_ctx*>(ctx)->fail(PF_ERR_ARG, "out is NULL");
  out->vx = ctx->L.march.vx;
  out->tz = ctx->L.march.tz;
  out->blocks_per_sm = ctx->tile_bps;
  out->mg_whole = ctx->mg_whole;
  return PF_OK;
}

pf_status pf_set_tiling(pf_ctx* ctx, const pf_tiling* t) {
  if (!ctx) return PF_ERR_ARG;
  if (ctx->async_open) return ctx->fail(PF_ERR_STATE, "pf_step_async work is pending (call pf_step_wait first)");
  if (!t) return ctx->fail(PF_ERR_ARG, "tiling is NULL");
  const int fp32 = ctx->prm.precision == PF_FP32;
  const int vmax = fp32 ? 4 : 2;
  if (t->vx != 1 && t->vx != vmax) return ctx->fail(PF_ERR_ARG, "vx must be 1 or %d", vmax);
  if (t->vx > 1 && ctx->prm.nx % t->vx != 0) return ctx->fail(PF_ERR_ARG, "nx is not a multiple of vx = %d", t->vx);
  if (t->tz < 1 || t->tz > 64) return ctx->fail(PF_ERR_ARG, "tz must be in 1 .. 64");
  if (t->blocks_per_sm < 0 || t->blocks_per_sm > 64) return ctx->fail(PF_ERR_ARG, "blocks_per_sm must be in 0 .. 64");
  if (t->mg_whole != 0 && t->mg_whole != 1) return ctx->fail(PF_ERR_ARG, "mg_whole must be 0 or 1");
  const Geo& g = ctx->geo;
  const int occ = pf::march_blocks_per_sm(fp32, ctx->prm.has_eps);
  const int bps = t->blocks_per_sm > 0 ? std::min(t->blocks_per_sm, occ) : occ;
  pf::MarchCfg m{};
  m.vx = t->vx;
  m.tiles_x = (g.nx + pf::MTX * m.vx - 1) / (pf::MTX * m.vx);
  m.tiles_y = (g.ny + pf::MTY - 1) / pf::MTY;
  m.tz = std::min(t->tz, g.nz);
  m.ntiles = (long long)m.tiles_x * m.tiles_y * ((g.nz + m.tz - 1) / m.tz);
  m.grid = (int)std::min<long long>(m.ntiles, std::min<long long>(pf::MAX_GRID, (long long)bps * ctx->nsm));
  m.bps = t->blocks_per_sm;
  drop_graphs(ctx);
  ctx->L.march = m;
  ctx->tile_bps = t->blocks_per_sm;
  ctx->mg_whole = t->mg_whole;
  ctx->gen += 1;
  return PF_OK;
}

pf_status pf_destroy(pf_ctx* ctx) {
  if (!ctx) return PF_OK;
  drop_graphs(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  if (ctx->S_tmpl) cudaFreeHost(ctx->S_tmpl);
  delete ctx;
  return PF_OK;
}

const char* pf_last_error(const pf_ctx* ctx) {
  if (!ctx) return g_create_error;
  return ctx->err.c_str();
}

}  // extern "C"

// ------------------------------------------------------------------ batch

struct pf_batch {
  std::vector<pf_ctx*> films;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  char* ws = nullptr;
  size_t off_state = 0, off_table = 0, off_part = 0, off_hist = 0, off_loop = 0;
  int64_t max_records = 0;
  int record_every = 1;
  long long max_nxy = 0;
  std::vector<pf::BatchFilm> table;
  cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaGraphExec_t gloop = nullptr;   // persistent loop: two batch steps per body
  bool loop_broken = false;
  std::vector<uint64_t> gen;         // film generations the graphs were captured for
  std::vector<pf_step_info> infos;
  std::string err;

  pf_status fail(pf_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    err = buf;
    return st;
  }
};

namespace {

thread_local char g_batch_error[512];

struct BatchLayout {
  size_t state, table, part, hist, loop, total;
};

BatchLayout batch_layout(int nfilms, int64_t max_records) {
  BatchLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align_up(bytes);
    return o;
  };
  L.state = take(sizeof(pf::BatchState));
  L.table = take(sizeof(pf::BatchFilm) * (size_t)nfilms);
  L.part = take(sizeof(double) * 3 * pf::BATCH_REC_BLOCKS * (size_t)nfilms);
  L.hist = take(sizeof(double) * 4 * (size_t)nfilms * (size_t)max_records);
  L.loop = take(2 * sizeof(long long));   // bodies left in a persistent batch loop
  L.total = off;
  return L;
}

void batch_drop_graphs(pf_batch* b) {
  for (cudaGraphExec_t& e : b->gexec) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
  if (b->gloop) cudaGraphExecDestroy(b->gloop);
  b->gloop = nullptr;
}

pf_status batch_upload_table(pf_batch* b) {
  if (cudaMemcpyAsync(b->ws + b->off_table, b->table.data(), sizeof(pf::BatchFilm) * b->table.size(),
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    return b->fail(PF_ERR_CUDA, "batch table upload: %s", cudaGetErrorString(e));
  }
  return PF_OK;
}

// One batch step as a graph: the ramp kernel, every film's step as an
// independent branch after it, the loop record after all of them.
// Append one batch step (ramp, every film's step from buffer cur, loop record)
// to graph after the nodes deps; on return deps holds the record node.
cudaError_t batch_append(pf_batch* b, cudaGraph_t graph, std::vector<cudaGraphNode_t>& deps, int cur, int refresh) {
  cudaError_t e = cudaSuccess;
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  const pf::BatchFilm* table = (const pf::BatchFilm*)(b->ws + b->off_table);
  pf::BatchState* bs = (pf::BatchState*)(b->ws + b->off_state);
  const int nf = (int)b->films.size();
  auto segment = [&](std::vector<cudaGraphNode_t>& dp, auto&& body) {
    if (e != cudaSuccess) return;
    e = cudaStreamBeginCaptureToGraph(b->cap, graph, dp.empty() ? nullptr : dp.data(), nullptr, dp.size(), mode);
    if (e != cudaSuccess) return;
    body();
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* fr = nullptr;
    size_t nfr = 0;
    e = cudaStreamGetCaptureInfo(b->cap, &cs, nullptr, nullptr, &fr, nullptr, &nfr);
    if (e == cudaSuccess) dp.assign(fr, fr + nfr);
    cudaGraph_t g_out = graph;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g_out);
    if (e == cudaSuccess) e = e2;
  };
  std::vector<cudaGraphNode_t> ramp = deps;
  segment(ramp, [&] { pf::launch_batch_ramp(table, nf, b->max_nxy, bs, b->cap); });
  std::vector<cudaGraphNode_t> joined;
  for (pf_ctx* c : b->films) {
    if (e != cudaSuccess) break;
    std::vector<cudaGraphNode_t> dp = ramp;
    e = c->prm.precision == PF_FP32 ? append_step<float>(c, graph, dp, cur, refresh, b->cap)
                                    : append_step<double>(c, graph, dp, cur, refresh, b->cap);
    joined.insert(joined.end(), dp.begin(), dp.end());
  }
  const int buf = b->films[0]->prm.integrator == PF_HEUN ? cur : cur ^ 1;
  double* part = (double*)(b->ws + b->off_part);
  double* hist = (double*)(b->ws + b->off_hist);
  segment(joined, [&] { pf::launch_batch_record(table, nf, buf, bs, part, hist, b->cap); });
  deps = joined;
  return e;
}

pf_status batch_capture(pf_batch* b, int cur, int refresh, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  std::vector<cudaGraphNode_t> deps;
  if (e == cudaSuccess) e = batch_append(b, graph, deps, cur, refresh);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return b->fail(PF_ERR_CUDA, "batch graph capture: %s", cudaGetErrorString(e));
  }
  *out = exec;
  return PF_OK;
}

// The persistent form: pairs of batch steps (buffer 0, then buffer 1) in a
// device-driven while loop counted down by k_loop_next, so that a whole
// pf_batch_step call is one graph launch.
pf_status batch_capture_loop(pf_batch* b, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  cudaGraphConditionalHandle h = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    std::vector<cudaGraphNode_t> deps;
    e = batch_append(b, body, deps, 0, 1);
    if (e == cudaSuccess) e = batch_append(b, body, deps, 1, 1);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(b->cap, body, deps.data(), nullptr, deps.size(),
                                        cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      pf::launch_loop_next((long long*)(b->ws + b->off_loop), h, b->cap);
      cudaGraph_t g2 = body;
      e = cudaStreamEndCapture(b->cap, &g2);
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return b->fail(PF_ERR_CUDA, "batch step loop graph: %s", cudaGetErrorString(e));
  }
  *out = exec;
  return PF_OK;
}

}  // namespace

extern "C" {

size_t pf_batch_workspace_bytes(int32_t nfilms, int64_t max_records) {
  if (nfilms < 1 || max_records < 0) return 0;
  return batch_layout(nfilms, max_records).total;
}

pf_status pf_batch_create(pf_ctx* const* films, int32_t nfilms, void* workspace, size_t workspace_bytes,
                          int64_t max_records, int32_t record_every, pf_batch** out) {
  auto gfail = [&](pf_status st, const char* m) {
    std::snprintf(g_batch_error, sizeof(g_batch_error), "%s", m);
    return st;
  };
  if (!out) return gfail(PF_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!films || nfilms < 1) return gfail(PF_ERR_ARG, "need at least one film");
  if (max_records < 0 || record_every < 1) return gfail(PF_ERR_ARG, "max_records must be >= 0, record_every >= 1");
  const BatchLayout L = batch_layout(nfilms, max_records);
  if (!workspace || workspace_bytes < L.total) return gfail(PF_ERR_ARG, "workspace missing or too small");
  if (((uintptr_t)workspace % ALIGN) != 0) return gfail(PF_ERR_ARG, "workspace must be 256-byte aligned");
  if (!is_device_ptr(workspace)) return gfail(PF_ERR_ARG, "workspace must be a device pointer");
  for (int i = 0; i < nfilms; ++i) {
    pf_ctx* c = films[i];
    if (!c || !c->bound) return gfail(PF_ERR_ARG, "every film must be a bound context");
    if (c->async_open) return gfail(PF_ERR_STATE, "a film has pf_step_async work pending (call pf_step_wait first)");
    for (int j = 0; j < i; ++j)
      if (films[j] == c) return gfail(PF_ERR_ARG, "a film appears twice");
    const pf_ctx* f0 = films[0];
    if (c->stream != f0->stream) return gfail(PF_ERR_ARG, "all films must use the same CUDA stream");
    if (c->prm.integrator != f0->prm.integrator || std::max(1, c->prm.poisson_every) != std::max(1, f0->prm.poisson_every))
      return gfail(PF_ERR_ARG, "all films must use the same integrator and poisson_every");
    if (c->nstep != f0->nstep || c->cur != 0) return gfail(PF_ERR_STATE, "all films must be at the same step");
  }
  pf_batch* b = new pf_batch();
  b->films.assign(films, films + nfilms);
  b->stream = films[0]->stream;
  b->ws = (char*)workspace;
  b->off_state = L.state;
  b->off_table = L.table;
  b->off_part = L.part;
  b->off_hist = L.hist;
  b->off_loop = L.loop;
  b->max_records = max_records;
  b->record_every = record_every;
  b->gen.assign(nfilms, 0);
  b->infos.assign(nfilms, pf_step_info{});
  b->table.resize(nfilms);
  for (int i = 0; i < nfilms; ++i) {
    pf_ctx* c = films[i];
    pf::BatchFilm& f = b->table[i];
    f = pf::BatchFilm{};
    f.P[0] = c->P_user;
    f.P[1] = c->ws + c->lay.P_alt;
    f.volt = nullptr;
    f.n = c->geo.n;
    f.nxy = c->geo.nxy;
    f.amp = 0.0;
    f.period = 1.0;
    f.fp32 = c->prm.precision == PF_FP32;
    b->max_nxy = std::max(b->max_nxy, (long long)c->geo.nxy);
  }
  pf::BatchState st{};
  st.record_every = record_every;
  st.max_records = max_records;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->ws + b->off_state, &st, sizeof(st), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    std::snprintf(g_batch_error, sizeof(g_batch_error), "CUDA: %s", cudaGetErrorString(e));
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return PF_ERR_CUDA;
  }
  if (batch_upload_table(b) != PF_OK) {
    std::snprintf(g_batch_error, sizeof(g_batch_error), "%s", b->err.c_str());
    cudaStreamDestroy(b->cap);
    delete b;
    return PF_ERR_CUDA;
  }
  *out = b;
  return PF_OK;
}

pf_status pf_batch_set_ramp(pf_batch* b, int32_t film, int32_t face, double amplitude, double period) {
  if (!b) return PF_ERR_ARG;
  if (film < 0 || film >= (int)b->films.size()) return b->fail(PF_ERR_ARG, "film index out of range");
  if (face != PF_ZLO && face != PF_ZHI) return b->fail(PF_ERR_ARG, "face must be PF_ZLO or PF_ZHI");
  if (!std::isfinite(amplitude) || !std::isfinite(period) || period < 0.0)
    return b->fail(PF_ERR_ARG, "amplitude must be finite and period >= 0");
  pf_ctx* c = b->films[film];
  pf::BatchFilm& f = b->table[film];
  if (period == 0.0) {
    f.volt = nullptr;
  } else {
    f.volt = c->ws + (face == PF_ZLO ? c->lay.vlo : c->lay.vhi);
    f.amp = amplitude;
    f.period = period;
  }
  return batch_upload_table(b);
}

pf_status pf_batch_step(pf_batch* b, int32_t nsteps, pf_step_info* info) {
  if (!b) return PF_ERR_ARG;
  if (nsteps < 0) return b->fail(PF_ERR_ARG, "nsteps must be >= 0");
  const int nf = (int)b->films.size();
  pf_ctx* f0 = b->films[0];
  for (pf_ctx* c : b->films) {
    if (!c->bound) return b->fail(PF_ERR_STATE, "a film is no longer bound");
    if (c->async_open) return b->fail(PF_ERR_STATE, "a film has pf_step_async work pending");
    if (c->nstep != f0->nstep || c->cur != 0) return b->fail(PF_ERR_STATE, "films are no longer at the same step");
  }
  bool stale = false;
  for (int i = 0; i < nf; ++i) stale |= b->gen[i] != b->films[i]->gen;
  if (stale) {
    batch_drop_graphs(b);
    for (int i = 0; i < nf; ++i) b->gen[i] = b->films[i]->gen;
  }
  for (pf_ctx* c : b->films) {
    pf_status st = reset_scalars(c);
    if (st != PF_OK) return b->fail(st, "film: %s", c->err.c_str());
    if (c->prm.precision == PF_FP32) refresh_invd<float>(c, c->L, false);
    else refresh_invd<double>(c, c->L, false);
  }
  const bool heun = f0->prm.integrator == PF_HEUN;
  auto book = [&](int refresh, long long steps) {    // host bookkeeping of graph-run steps
    for (pf_ctx* c : b->films) {
      int64_t fixed = 0, per_iter = 0;
      step_kernel_counts(c, refresh, &fixed, &per_iter);
      c->graph_fixed += steps * fixed;
      c->graph_solves += refresh ? steps * (heun ? 2 : 1) : 0;
      c->graph_steps += steps;
      if (!heun && (steps & 1)) c->cur ^= 1;
      c->nstep += steps;
    }
  };
  long long loop_launches = 0;
  // many forward-Euler steps that all solve: pairs of batch steps in one persistent launch
  if (!heun && f0->prm.poisson_every <= 1 && f0->cur == 0 && nsteps >= 4 && !b->loop_broken) {
    if (!b->gloop && batch_capture_loop(b, &b->gloop) != PF_OK) {
      b->loop_broken = true;             // one launch per batch step from here on
      b->err.clear();
    }
    if (b->gloop) {
      const long long pairs = nsteps / 2;
      pf::launch_loop_set((long long*)(b->ws + b->off_loop), pairs, b->stream);
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaGraphLaunch(b->gloop, b->stream);
      if (e != cudaSuccess) return b->fail(PF_ERR_CUDA, "persistent batch loop: %s", cudaGetErrorString(e));
      book(1, 2 * pairs);
      loop_launches = 1 + pairs;                     // the count setter and every body's counter
      nsteps -= (int)(2 * pairs);
    }
  }
  const int total_steps = nsteps + (int)(2 * (loop_launches > 0 ? loop_launches - 1 : 0));
  for (int s = 0; s < nsteps; ++s) {
    const int refresh = refresh_step(f0) ? 1 : 0;
    const int cur = f0->cur;
    const int slot = cur * 2 + refresh;
    if (!b->gexec[slot]) {
      pf_status st = batch_capture(b, cur, refresh, &b->gexec[slot]);
      if (st != PF_OK) return st;
    }
    const cudaError_t e = cudaGraphLaunch(b->gexec[slot], b->stream);
    if (e != cudaSuccess) return b->fail(PF_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    book(refresh, 1);
  }
  nsteps = total_steps;
  pf_status worst = PF_OK;
  pf_step_info sum{};
  sum.steps_done = nsteps;
  for (int i = 0; i < nf; ++i) {
    pf_ctx* c = b->films[i];
    if (c->cur == 1) {
      const size_t w = c->prm.precision == PF_FP32 ? 4 : 8;
      if (cudaMemcpyAsync(c->P_user, c->ws + c->lay.P_alt, 3 * (size_t)c->geo.n * w, cudaMemcpyDeviceToDevice,
                          c->stream) != cudaSuccess)
        return b->fail(PF_ERR_CUDA, "copy back: %s", cudaGetErrorString(cudaGetLastError()));
      c->cur = 0;
    }
    pf_step_info& fi = b->infos[i];
    fi = pf_step_info{};
    const pf_status st = finish_info(c, nsteps, &fi);
    if (st == PF_ERR_CUDA || st == PF_ERR_STATE) return b->fail(st, "film %d: %s", i, c->err.c_str());
    if (st == PF_ERR_NONFINITE || (st == PF_ERR_NOCONV && worst == PF_OK)) worst = st;
    sum.last_iters = std::max(sum.last_iters, fi.last_iters);
    sum.total_iters += fi.total_iters;
    sum.max_iters = std::max(sum.max_iters, fi.max_iters);
    sum.solves += fi.solves;
    sum.last_relres = std::max(sum.last_relres, fi.last_relres);
    sum.nonconverged += fi.nonconverged;
    sum.kernel_launches += fi.kernel_launches;
    sum.graph_steps = nsteps;
  }
  sum.kernel_launches += 2LL * nsteps + loop_launches;   // the ramp and record kernels (and loop counters)
  sum.status = worst;
  if (info) *info = sum;
  if (worst != PF_OK) b->fail(worst, "%s", worst == PF_ERR_NONFINITE ? "a film went non-finite" : "a Poisson solve hit poisson_maxit");
  return worst;
}

pf_status pf_batch_film_info(const pf_batch* b, int32_t film, pf_step_info* info) {
  if (!b || !info || film < 0 || film >= (int)b->films.size()) return PF_ERR_ARG;
  *info = b->infos[film];
  return PF_OK;
}

pf_status pf_batch_read_loops(pf_batch* b, double* out, int64_t max_out, int64_t* nrecords) {
  if (!b) return PF_ERR_ARG;
  if (!nrecords || max_out < 0 || (max_out > 0 && !out)) return b->fail(PF_ERR_ARG, "bad output arguments");
  pf::BatchState st{};
  cudaError_t e = cudaMemcpyAsync(&st, b->ws + b->off_state, sizeof(st), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return b->fail(PF_ERR_CUDA, "read loops: %s", cudaGetErrorString(e));
  const int64_t stored = std::min<int64_t>(st.records, b->max_records);
  const int64_t n = std::min<int64_t>(stored, max_out);
  const size_t bytes = sizeof(double) * 4 * b->films.size() * (size_t)n;
  if (bytes) {
    e = cudaMemcpyAsync(out, b->ws + b->off_hist, bytes, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b->fail(PF_ERR_CUDA, "read loops: %s", cudaGetErrorString(e));
  }
  *nrecords = stored;
  return PF_OK;
}

pf_status pf_batch_destroy(pf_batch* b) {
  if (!b) return PF_OK;
  batch_drop_graphs(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return PF_OK;
}

const char* pf_batch_last_error(const pf_batch* b) {
  if (!b) return g_batch_error;
  return b->err.c_str();
}

}  // extern "C"
