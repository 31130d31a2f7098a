// C ABI of the GB300 DG2 / multiwavelet-MRA flood solver (include/mwdg.h):
// context, device memory, host orchestration of the kernels in
// mwdg_kernels.cuh.  Method: Sharifian & Kesserwani, arXiv 2107.02750.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "mwdg_internal.h"

using namespace mwdg;

namespace {

constexpr int KNOT_CAP = 4096;

const char *kclass_name(int c) {
  static const char *names[KC_COUNT] = {"mra_encode", "mra_flags",  "mra_decode", "compact",
                                        "dt_reduce",  "control",    "friction",   "limit",
                                        "view_encode", "dg2_update_stage1", "dg2_update_stage2"};
  return (c >= 0 && c < KC_COUNT) ? names[c] : "?";
}

}  // namespace

struct mwdg_ctx {
  mwdg_params p{};
  cudaStream_t st = nullptr;
  Geo g{};
  Ptrs<double> pd{};
  Ptrs<float> pf{};
  std::vector<void *> allocs;
  Ctl *ctl = nullptr;
  double *d_vert = nullptr;
  double *d_knot_t = nullptr, *d_knot_Q = nullptr;
  double *d_fields = nullptr;    // 3 finest rasters for read-back
  int32_t *d_active = nullptr;   // level, i, j for read-back
  double *d_coef = nullptr;      // coefficients for read-back
  int32_t *d_gauge_ij = nullptr; // gauge cells and their values for read-back
  double *d_gauge_out = nullptr;
  int gauge_cap = 0;
  int grid_leaves = 0;
  int part_cap = 0;          // entries of the volume's per-block partial sums
  bool shape_set = false;    // the caller chose grid_leaves
  bool dem = false, initial = false, stepped = false, failed = false, encoded = false;
  bool vmax_fresh = false;   // max |v0| on the device is that of the current leaves
  // one captured step (CUDA graph), replayed while the parameters it bakes in
  // are unchanged; not used on the legacy default stream or while profiling
  bool use_graph = true;
  cudaGraphExec_t graph = nullptr;
  // the adaptation's fork (a second stream and two events, made with an
  // adaptive context)
  Fork fk{nullptr, nullptr, nullptr};
  int graph_launches = 0;
  int64_t generation = 0;   // bumped whenever the captured step becomes stale
  int static_eta = 0;   // static run with a free-surface initial state
  int64_t launches = 0;
  std::string err;
  // per-kernel timing
  bool prof = false;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, cudaEvent_t>> marks;
  double kms[KC_COUNT] = {};
  int64_t kcount[KC_COUNT] = {};
};

namespace {

mwdg_status fail(mwdg_ctx *c, mwdg_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) {
    c->err = buf;
    if (s == MWDG_ERR_CUDA || s == MWDG_ERR_NONFINITE) c->failed = true;
  }
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(c, MWDG_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                  __FILE__, __LINE__);                                                    \
  } while (0)

#define CHECK_LAUNCH()                                                                    \
  do {                                                                                    \
    cudaError_t e_ = cudaGetLastError();                                                  \
    if (e_ != cudaSuccess)                                                                \
      return fail(c, MWDG_ERR_CUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_),  \
                  __FILE__, __LINE__);                                                    \
  } while (0)

#define LIVE(c)                                                                           \
  do {                                                                                    \
    if (!(c)) return MWDG_ERR_ARG;                                                        \
    if ((c)->failed) return MWDG_ERR_STATE;                                               \
  } while (0)

bool all_finite(const double *a, size_t n) {
  for (size_t k = 0; k < n; k++)
    if (!std::isfinite(a[k])) return false;
  return true;
}

template <typename T>
mwdg_status alloc(mwdg_ctx *c, T **p, size_t n) {
  void *q = nullptr;
  CK(cudaMalloc(&q, n * sizeof(T)));
  c->allocs.push_back(q);
  *p = (T *)q;
  return MWDG_OK;
}

void mark_cb(void *arg, int cls) {
  mwdg_ctx *c = (mwdg_ctx *)arg;
  if (!c->prof) return;
  cudaEvent_t ev;
  if (!c->pool.empty()) {
    ev = c->pool.back();
    c->pool.pop_back();
  } else if (cudaEventCreate(&ev) != cudaSuccess) {
    return;
  }
  cudaEventRecord(ev, c->st);
  c->marks.emplace_back(cls, ev);
}

// attribute the time between consecutive marks to the earlier mark's class
mwdg_status flush_marks(mwdg_ctx *c) {
  if (c->marks.empty()) return MWDG_OK;
  CK(cudaStreamSynchronize(c->st));
  for (size_t q = 0; q + 1 < c->marks.size(); q++) {
    int cls = c->marks[q].first;
    if (cls < 0) continue;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->marks[q].second, c->marks[q + 1].second));
    c->kms[cls] += ms;
    c->kcount[cls] += 1;
  }
  for (size_t q = 0; q + 1 < c->marks.size(); q++) c->pool.push_back(c->marks[q].second);
  auto last = c->marks.back();
  c->marks.clear();
  c->marks.push_back(last);
  return MWDG_OK;
}

template <typename T> Ptrs<T> &ptrs(mwdg_ctx *c);
template <> Ptrs<double> &ptrs<double>(mwdg_ctx *c) { return c->pd; }
template <> Ptrs<float> &ptrs<float>(mwdg_ctx *c) { return c->pf; }

template <typename T>
mwdg_status allocate_state(mwdg_ctx *c) {
  Ptrs<T> &p = ptrs<T>(c);
  const size_t P = (size_t)c->g.P;
  mwdg_status s;
  if ((s = alloc(c, &p.U, 9 * P)) || (s = alloc(c, &p.Ui, 9 * P)) || (s = alloc(c, &p.Wn, 9 * P)) ||
      (s = alloc(c, &p.Wi, 9 * P)) || (s = alloc(c, &p.FZ, 12 * P)) || (s = alloc(c, &p.Z, 3 * P)) ||
      (s = alloc(c, &p.NM, P)) || (s = alloc(c, &p.DZ, P)) ||
      (s = alloc(c, &p.kind, P)) || (s = alloc(c, &p.kind_new, P)) || (s = alloc(c, &p.flag, P)) ||
      (s = alloc(c, &p.flag2, P)) || (s = alloc(c, &p.leaves, P)) || (s = alloc(c, &p.nbr, 4 * P)) ||
      (s = alloc(c, &p.nleaf, 1)))
    return s;
  const size_t nb = (P + 2048 - 1) / 2048 + 1;
  if ((s = alloc(c, &p.blk, nb)) || (s = alloc(c, &p.part, (size_t)c->grid_leaves))) return s;
  c->part_cap = c->grid_leaves;
  CK(cudaMemsetAsync(p.U, 0, 9 * P * sizeof(T), c->st));
  CK(cudaMemsetAsync(p.Ui, 0, 9 * P * sizeof(T), c->st));
  CK(cudaMemsetAsync(p.Wn, 0, 9 * P * sizeof(T), c->st));
  CK(cudaMemsetAsync(p.Wi, 0, 9 * P * sizeof(T), c->st));
  CK(cudaMemsetAsync(p.FZ, 0, 12 * P * sizeof(T), c->st));
  CK(cudaMemsetAsync(p.Z, 0, 3 * P * sizeof(T), c->st));
  CK(cudaMemsetAsync(p.NM, 0, P * sizeof(T), c->st));
  CK(cudaMemsetAsync(p.DZ, 0, P * sizeof(double), c->st));
  CK(cudaMemsetAsync(p.flag, 0, P, c->st));
  CK(cudaMemsetAsync(p.flag2, 0, P, c->st));
  p.ctl = c->ctl;
  p.knot_t = c->d_knot_t;
  p.knot_Q = c->d_knot_Q;
  return MWDG_OK;
}

// run a launcher on the context's precision
template <typename F>
int dispatch(mwdg_ctx *c, F &&f) {
  if (c->g.prec == MWDG_F64) return f(c->pd, (double *)nullptr);
  return f(c->pf, (float *)nullptr);
}

Ctl fresh_ctl() {
  Ctl h{};
  h.t = 0.0;
  h.dt = 0.0;
  h.t_end = 1e300;
  h.dtmin = 0x7ff0000000000000ULL;
  return h;
}

mwdg_status read_ctl(mwdg_ctx *c, Ctl *h) {
  CK(cudaMemcpyAsync(h, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (h->nonfinite) return fail(c, MWDG_ERR_NONFINITE, "non-finite value in the solution");
  return MWDG_OK;
}

// queue the regridding of a static run from the topography details: flags,
// closure, 2:1 grading to a fixed point, kinds, encode of the finest state
mwdg_status build_static_grid(mwdg_ctx *c, int is_eta_encoded) {
  const Geo &g = c->g;
  c->launches += dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    return Launch<T>::static_flags(g, p, c->st) + Launch<T>::closure(g, p.flag, c->st);
  });
  for (int it = 0; it < 4 * (g.L + 2); it++) {
    int zero = 0, changed = 0;
    CK(cudaMemcpyAsync(&c->ctl->changed, &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
    c->launches += dispatch(c, [&](auto &p, auto *) {
      using T = std::remove_pointer_t<decltype(p.U)>;
      return Launch<T>::grading_sweep(g, p, c->st);
    });
    CHECK_LAUNCH();
    CK(cudaMemcpyAsync(&changed, &c->ctl->changed, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (!changed) break;
  }
  c->launches += dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    int n = Launch<T>::kinds(g, p, p.flag, c->st) + Launch<T>::encode_dense_U(g, p, c->st);
    if (is_eta_encoded) n += Launch<T>::eta_rule_leaves(g, p, c->st);
    return n + Launch<T>::compact(g, p, c->st);
  });
  CHECK_LAUNCH();
  return MWDG_OK;
}

void drop_graph(mwdg_ctx *c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  c->generation++;
}

// the kernels of one step: [adaptive: encode, flags, decode, compaction],
// time step, both RK2 stages (the last block closes the step)
int launch_step(mwdg_ctx *c, int with_maxabs) {
  const Geo &g = c->g;
  return dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    int n = 0;
    const int adaptive = (g.mode == MWDG_ADAPTIVE);
    if (adaptive) n += Launch<T>::adapt(g, p, 0, with_maxabs, c->st, mark_cb, c, 1, c->fk.join ? &c->fk : nullptr);
    n += Launch<T>::step(g, p, c->grid_leaves, c->st, mark_cb, c, adaptive);
    return n;
  });
}

mwdg_status queue_step(mwdg_ctx *c) {
  const bool adaptive = c->g.mode == MWDG_ADAPTIVE;
  const bool graphable = c->use_graph && !c->prof && c->st != nullptr && (c->vmax_fresh || !adaptive);
  if (graphable) {
    if (!c->graph) {
      cudaGraph_t gr = nullptr;
      CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
      c->graph_launches = launch_step(c, 0);
      cudaError_t e1 = cudaStreamEndCapture(c->st, &gr);
      if (e1 != cudaSuccess || !gr)
        return fail(c, MWDG_ERR_CUDA, "step capture: %s", cudaGetErrorString(e1));
      cudaError_t e2 = cudaGraphInstantiate(&c->graph, gr, 0);
      cudaGraphDestroy(gr);
      if (e2 != cudaSuccess) return fail(c, MWDG_ERR_CUDA, "step graph: %s", cudaGetErrorString(e2));
    }
    CK(cudaGraphLaunch(c->graph, c->st));
    c->launches += c->graph_launches;
  } else {
    c->launches += launch_step(c, adaptive && !c->vmax_fresh);
    CHECK_LAUNCH();
  }
  c->stepped = true;
  c->encoded = false;
  c->vmax_fresh = true;
  return MWDG_OK;
}

__global__ void k_reset_reductions(Ctl *c) {
  c->dtmin = 0x7ff0000000000000ULL;
  c->vmax[0] = c->vmax[1] = c->vmax[2] = 0ULL;
}

// the reductions a step starts from, over the current leaves
mwdg_status prime(mwdg_ctx *c) {
  k_reset_reductions<<<1, 1, 0, c->st>>>(c->ctl);
  c->launches += 1 + dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    return Launch<T>::prime(c->g, p, c->grid_leaves, c->st);
  });
  CHECK_LAUNCH();
  c->vmax_fresh = true;
  return MWDG_OK;
}

template <typename T>
__global__ void k_fill_nm(T *nm, long long off, long long n, const double *src, double val) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  nm[off + k] = (T)(src ? src[k] : val);
}

__global__ void k_set_tend(Ctl *c, double t_end) { c->t_end = t_end; }
__global__ void k_set_dt_fixed(Ctl *c, double dt) { c->dt_fixed = dt; }

__global__ void k_check_finite(const double *a, long long n, int *flag) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    if (!isfinite(a[k])) *flag = 1;
}

// A raster of rows x cols doubles with a row stride of ld elements (0: cols)
// from the caller's memory (host, or device when on_device) into the
// contiguous device buffer dst; a raster with a non-finite value is refused
// (a device raster is checked on the device, which synchronises).
mwdg_status stage_raster(mwdg_ctx *c, const double *src, size_t rows, size_t cols, int64_t ld, bool on_device,
                         double *dst, const char *what) {
  if (ld == 0) ld = (int64_t)cols;
  if (ld < (int64_t)cols) return fail(c, MWDG_ERR_ARG, "%s: row stride %lld is below the row length %zu", what,
                                      (long long)ld, cols);
  const size_t pitch = (size_t)ld * sizeof(double), width = cols * sizeof(double);
  if (!on_device) {
    for (size_t r = 0; r < rows; r++)
      if (!all_finite(src + r * (size_t)ld, cols)) return fail(c, MWDG_ERR_NONFINITE, "non-finite %s value", what);
    CK(cudaMemcpy2DAsync(dst, width, src, pitch, width, rows, cudaMemcpyHostToDevice, c->st));
    return MWDG_OK;
  }
  CK(cudaMemcpy2DAsync(dst, width, src, pitch, width, rows, cudaMemcpyDeviceToDevice, c->st));
  int flag = 0;
  CK(cudaMemcpyAsync(&c->ctl->bad_input, &flag, sizeof flag, cudaMemcpyHostToDevice, c->st));
  const long long n = (long long)(rows * cols);
  k_check_finite<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, c->st>>>(dst, n, &c->ctl->bad_input);
  c->launches++;
  CHECK_LAUNCH();
  CK(cudaMemcpyAsync(&flag, &c->ctl->bad_input, sizeof flag, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (flag) return fail(c, MWDG_ERR_NONFINITE, "non-finite %s value", what);
  return MWDG_OK;
}

}  // namespace

extern "C" {

const char *mwdg_status_string(mwdg_status s) {
  switch (s) {
    case MWDG_OK: return "ok";
    case MWDG_ERR_ARG: return "invalid argument";
    case MWDG_ERR_DIMS: return "invalid dimensions";
    case MWDG_ERR_CUDA: return "CUDA error";
    case MWDG_ERR_NONFINITE: return "non-finite value";
    case MWDG_ERR_TIMEOUT: return "device wait timed out";
    case MWDG_ERR_STATE: return "invalid state";
    case MWDG_ERR_CAPACITY: return "capacity exceeded";
  }
  return "unknown status";
}

mwdg_status mwdg_params_default(mwdg_params *p) {
  if (!p) return MWDG_ERR_ARG;
  memset(p, 0, sizeof *p);
  p->M = p->N = 1;
  p->L = 0;
  p->mode = MWDG_UNIFORM;
  p->precision = MWDG_F64;
  p->limiter = 1;
  for (int e = 0; e < 4; e++) p->bc[e] = MWDG_WALL;
  p->dx = 1.0;
  p->eps = 1e-3;
  p->cfl = 0.33;
  p->g = 9.80665;
  p->h_dry = 1e-3;
  p->dt_max = 1.0;
  return MWDG_OK;
}

mwdg_status mwdg_create(const mwdg_params *p, mwdg_ctx **out) {
  if (!p || !out) return MWDG_ERR_ARG;
  *out = nullptr;
  if (p->L < 0 || p->L > MWDG_LMAX || p->M < 1 || p->N < 1 || !(p->dx > 0.0)) return MWDG_ERR_DIMS;
  if ((int64_t)p->M << p->L > (1 << 20) || (int64_t)p->N << p->L > (1 << 20)) return MWDG_ERR_DIMS;
  if (p->mode < MWDG_UNIFORM || p->mode > MWDG_ADAPTIVE || p->precision < MWDG_F64 ||
      p->precision > MWDG_F32 || !(p->cfl > 0.0) || !(p->g > 0.0) || !(p->h_dry >= 0.0) ||
      !(p->dt_max > 0.0) || !std::isfinite(p->eps) || p->eps < 0.0 ||
      (p->iface_rule != MWDG_IFACE_PAPER && p->iface_rule != MWDG_IFACE_REFLUX) ||
      (p->iface_rule == MWDG_IFACE_REFLUX && p->mode == MWDG_ADAPTIVE) ||
      (p->scheme != MWDG_DG2 && p->scheme != MWDG_FV1 && p->scheme != MWDG_ACC) ||
      (p->scheme == MWDG_ACC && p->mode == MWDG_ADAPTIVE))
    return MWDG_ERR_ARG;
  mwdg_ctx *c = new mwdg_ctx();
  c->p = *p;
  if (const char *e = getenv("MWDG_NO_GRAPH")) c->use_graph = !(e[0] == '1');
  c->st = (cudaStream_t)p->cuda_stream;
  Geo &g = c->g;
  g.mode = p->mode;
  g.prec = p->precision;
  g.limiter = p->limiter;
  g.iface = p->iface_rule;
  g.scheme = p->scheme;
  if (p->mode == MWDG_UNIFORM) {  // a uniform grid is the single level of an L = 0 hierarchy
    g.L = 0;
    g.M = p->M << p->L;
    g.N = p->N << p->L;
  } else {
    g.L = p->L;
    g.M = p->M;
    g.N = p->N;
  }
  g.off[0] = 0;
  for (int l = 0; l <= g.L; l++) {
    g.nxl[l] = g.M << l;
    g.nyl[l] = g.N << l;
    g.dxl[l] = p->dx * (double)(1LL << (g.L - l));
    g.off[l + 1] = g.off[l] + (long long)g.nxl[l] * g.nyl[l];
  }
  g.P = g.off[g.L + 1];
  g.g = p->g;
  g.hd = p->h_dry;
  g.cfl = p->cfl;
  g.dt_max = p->dt_max;
  g.eps = p->eps;
  g.area = (double)g.nxl[g.L] * g.dxl[g.L] * (double)g.nyl[g.L] * g.dxl[g.L];
  sync_single(g);
  for (int e = 0; e < 4; e++) g.bc[e] = p->bc[e];
  g.inflow_edge = -1;
  g.inflow_c0 = 0;
  g.inflow_c1 = -1;
  g.nknots = 0;
  g.rain_rate = 0.0;
  g.rain_t_end = 0.0;
  g.coarse_nodes = 256;
  if (const char *e = getenv("MWDG_COARSE_NODES")) g.coarse_nodes = atoll(e);
  c->grid_leaves = (int)std::min<long long>((g.P + 255) / 256, 152 * 8);
  mwdg_status s;
  if ((s = alloc(c, &c->ctl, 1)) || (s = alloc(c, &c->d_knot_t, KNOT_CAP)) ||
      (s = alloc(c, &c->d_knot_Q, KNOT_CAP)) ||
      (s = alloc(c, &c->d_vert, (size_t)(g.nxl[g.L] + 1) * (g.nyl[g.L] + 1)))) {
    mwdg_destroy(c);
    return s;
  }
  s = (g.prec == MWDG_F64) ? allocate_state<double>(c) : allocate_state<float>(c);
  if (s) {
    mwdg_destroy(c);
    return s;
  }
  if (g.mode == MWDG_ADAPTIVE) {  // the adaptation's fork
    if (cudaStreamCreateWithFlags(&c->fk.aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fk.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fk.join, cudaEventDisableTiming) != cudaSuccess) {
      mwdg_destroy(c);
      return MWDG_ERR_CUDA;
    }
  }
  Ctl h = fresh_ctl();
  if (cudaMemcpyAsync(c->ctl, &h, sizeof h, cudaMemcpyHostToDevice, c->st) != cudaSuccess) {
    mwdg_destroy(c);
    return MWDG_ERR_CUDA;
  }
  c->launches += dispatch(c, [&](auto &pp, auto *) {
    using T = std::remove_pointer_t<decltype(pp.U)>;
    int n = (g.L == 0) ? Launch<T>::kinds(g, pp, pp.flag, c->st) : Launch<T>::all_finest(g, pp, c->st);
    return n + Launch<T>::compact(g, pp, c->st);
  });
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->st) != cudaSuccess) {
    mwdg_destroy(c);
    return MWDG_ERR_CUDA;
  }
  *out = c;
  return MWDG_OK;
}

void mwdg_destroy(mwdg_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  drop_graph(c);
  if (c->fk.aux) {
    cudaStreamSynchronize(c->fk.aux);
    cudaStreamDestroy(c->fk.aux);
  }
  if (c->fk.fork) cudaEventDestroy(c->fk.fork);
  if (c->fk.join) cudaEventDestroy(c->fk.join);
  for (void *q : c->allocs) cudaFree(q);
  for (auto &m : c->marks) cudaEventDestroy(m.second);
  for (auto ev : c->pool) cudaEventDestroy(ev);
  delete c;
}

static mwdg_status load_dem(mwdg_ctx *c, const double *z_vert, int64_t ld, bool on_device) {
  LIVE(c);
  if (!z_vert) return fail(c, MWDG_ERR_ARG, "z_vert is NULL");
  const Geo &g = c->g;
  mwdg_status st = stage_raster(c, z_vert, (size_t)g.nyl[g.L] + 1, (size_t)g.nxl[g.L] + 1, ld, on_device,
                                c->d_vert, "DEM");
  if (st) return st;
  unsigned long long zero = 0;
  CK(cudaMemcpyAsync(&c->ctl->vmax[0], &zero, sizeof zero, cudaMemcpyHostToDevice, c->st));
  c->launches += dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    const long long P = g.P, o = g.off[g.L];
    return Launch<T>::project(g, p, c->d_vert, p.Z + o, p.Z + P + o, p.Z + 2 * P + o, c->st) +
           Launch<T>::load_dem_pyramid(g, p, c->st);
  });
  CHECK_LAUNCH();
  CK(cudaMemcpyAsync(&c->ctl->vmax[0], &zero, sizeof zero, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->dem = true;
  c->initial = false;
  return MWDG_OK;
}

mwdg_status mwdg_load_dem(mwdg_ctx *c, const double *z_vert, int64_t ld) { return load_dem(c, z_vert, ld, false); }
mwdg_status mwdg_load_dem_dev(mwdg_ctx *c, const double *z_vert, int64_t ld) { return load_dem(c, z_vert, ld, true); }

static mwdg_status load_roughness(mwdg_ctx *c, const double *n_cell, int64_t ld, bool on_device) {
  LIVE(c);
  if (!n_cell) return fail(c, MWDG_ERR_ARG, "n_cell is NULL");
  const Geo &g = c->g;
  const size_t n = (size_t)g.nxl[g.L] * g.nyl[g.L];
  mwdg_status st = stage_raster(c, n_cell, (size_t)g.nyl[g.L], (size_t)g.nxl[g.L], ld, on_device, c->d_vert,
                                "roughness");
  if (st) return st;
  c->launches += dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    k_fill_nm<T><<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>(p.NM, g.off[g.L], (long long)n, c->d_vert, 0.0);
    return 1 + Launch<T>::roughness_pyramid(g, p, c->st);
  });
  CHECK_LAUNCH();
  CK(cudaStreamSynchronize(c->st));
  return MWDG_OK;
}

mwdg_status mwdg_load_roughness(mwdg_ctx *c, const double *n_cell, int64_t ld) {
  return load_roughness(c, n_cell, ld, false);
}
mwdg_status mwdg_load_roughness_dev(mwdg_ctx *c, const double *n_cell, int64_t ld) {
  return load_roughness(c, n_cell, ld, true);
}

mwdg_status mwdg_set_roughness_scalar(mwdg_ctx *c, double nval) {
  LIVE(c);
  if (!std::isfinite(nval) || nval < 0.0) return fail(c, MWDG_ERR_ARG, "invalid roughness");
  const Geo &g = c->g;
  c->launches += dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    k_fill_nm<T><<<(unsigned)((g.P + 255) / 256), 256, 0, c->st>>>(p.NM, 0, g.P, nullptr, nval);
    return 1;
  });
  CHECK_LAUNCH();
  return MWDG_OK;
}

static mwdg_status load_initial(mwdg_ctx *c, const double *h_vert, const double *qx_vert, const double *qy_vert,
                                int64_t ld, int32_t is_eta, bool on_device) {
  LIVE(c);
  if (!h_vert || !qx_vert || !qy_vert) return fail(c, MWDG_ERR_ARG, "NULL initial raster");
  if (!c->dem) return fail(c, MWDG_ERR_STATE, "mwdg_load_dem must come first");
  const Geo &g = c->g;
  const size_t nvx = (size_t)g.nxl[g.L] + 1, nvy = (size_t)g.nyl[g.L] + 1;
  const double *src[3] = {h_vert, qx_vert, qy_vert};
  if (!on_device)  // every raster checked before any of them is used
    for (int v = 0; v < 3; v++)
      for (size_t r = 0; r < nvy; r++)
        if (!all_finite(src[v] + r * (size_t)(ld ? ld : (int64_t)nvx), nvx))
          return fail(c, MWDG_ERR_NONFINITE, "non-finite initial value");
  for (int v = 0; v < 3; v++) {
    mwdg_status st = stage_raster(c, src[v], nvy, nvx, ld, on_device, c->d_vert, "initial");
    if (st) return st;
    c->launches += dispatch(c, [&](auto &p, auto *) {
      using T = std::remove_pointer_t<decltype(p.U)>;
      const long long P = g.P, o = g.off[g.L];
      T *b = p.U + 3 * v * P;
      int n = Launch<T>::project(g, p, c->d_vert, b + o, b + P + o, b + 2 * P + o, c->st);
      if (v == 0 && is_eta && g.mode == MWDG_STATIC) {
        // keep the projected free surface for the per-leaf wet/dry split
        for (int m = 0; m < 3; m++)
          cudaMemcpyAsync(p.Wn + m * P + o, b + m * P + o, (size_t)(P - o) * sizeof(T),
                          cudaMemcpyDeviceToDevice, c->st);
      }
      return n;
    });
    CHECK_LAUNCH();
  }
  c->launches += dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    // ACC: face discharges (held in the second stage view) start at zero
    if (g.scheme == MWDG_ACC) cudaMemsetAsync(p.Wi, 0, 4 * (size_t)g.P * sizeof(T), c->st);
    return Launch<T>::initial_finest(g, p, is_eta ? 1 : 0, c->st);
  });
  CHECK_LAUNCH();
  mwdg_status s = MWDG_OK;
  if (g.mode == MWDG_STATIC) {
    c->static_eta = (is_eta && g.L > 0) ? 1 : 0;
    s = build_static_grid(c, c->static_eta);
  } else {
    c->launches += dispatch(c, [&](auto &p, auto *) {
      using T = std::remove_pointer_t<decltype(p.U)>;
      int n = (g.L == 0) ? Launch<T>::kinds(g, p, p.flag, c->st) : Launch<T>::all_finest(g, p, c->st);
      return n + Launch<T>::compact(g, p, c->st);
    });
    CHECK_LAUNCH();
  }
  if (s) return s;
  Ctl h = fresh_ctl();
  CK(cudaMemcpyAsync(c->ctl, &h, sizeof h, cudaMemcpyHostToDevice, c->st));
  if ((s = prime(c))) return s;
  CK(cudaStreamSynchronize(c->st));
  if (g.mode == MWDG_STATIC && !c->shape_set) {
    // a static grid's leaves are fixed: about one leaf per thread of the
    // leaf kernels (152 to 4864 blocks), unless the caller chose a shape
    int nl = 0;
    CK(cudaMemcpy(&nl, g.prec == MWDG_F64 ? c->pd.nleaf : c->pf.nleaf, sizeof nl, cudaMemcpyDeviceToHost));
    c->grid_leaves = (int)std::min<long long>(std::max<long long>((nl + 255) / 256, 152), 152 * 32);
    drop_graph(c);
  }
  c->initial = true;
  c->stepped = false;
  c->encoded = false;
  return MWDG_OK;
}

mwdg_status mwdg_load_initial(mwdg_ctx *c, const double *h_vert, const double *qx_vert, const double *qy_vert,
                              int32_t is_eta) {
  return load_initial(c, h_vert, qx_vert, qy_vert, 0, is_eta, false);
}
mwdg_status mwdg_load_initial_dev(mwdg_ctx *c, const double *h_vert, const double *qx_vert, const double *qy_vert,
                                  int64_t ld, int32_t is_eta) {
  return load_initial(c, h_vert, qx_vert, qy_vert, ld, is_eta, true);
}

mwdg_status mwdg_set_inflow(mwdg_ctx *c, int32_t edge, int32_t c0, int32_t c1, const double *t,
                            const double *Q, int32_t nknots) {
  LIVE(c);
  Geo &g = c->g;
  if (nknots == 0) {
    g.inflow_edge = -1;
    g.nknots = 0;
    drop_graph(c);
    return MWDG_OK;
  }
  if (edge < 0 || edge > 3 || nknots < 1 || nknots > KNOT_CAP || !t || !Q)
    return fail(c, MWDG_ERR_ARG, "invalid inflow arguments");
  const int len = (edge < 2) ? g.nyl[g.L] : g.nxl[g.L];
  if (c0 < 0 || c1 < c0 || c1 >= len) return fail(c, MWDG_ERR_DIMS, "inflow cells outside the edge");
  if (!all_finite(t, nknots) || !all_finite(Q, nknots)) return fail(c, MWDG_ERR_NONFINITE, "non-finite hydrograph");
  for (int k = 1; k < nknots; k++)
    if (!(t[k] > t[k - 1])) return fail(c, MWDG_ERR_ARG, "hydrograph times must increase");
  CK(cudaMemcpyAsync(c->d_knot_t, t, nknots * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->d_knot_Q, Q, nknots * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  g.inflow_edge = edge;
  g.inflow_c0 = c0;
  g.inflow_c1 = c1;
  g.nknots = nknots;
  drop_graph(c);
  return MWDG_OK;
}

mwdg_status mwdg_set_rain(mwdg_ctx *c, double rate, double t_stop) {
  LIVE(c);
  if (!std::isfinite(rate) || rate < 0.0 || std::isnan(t_stop)) return fail(c, MWDG_ERR_ARG, "invalid rain");
  c->g.rain_rate = rate;
  c->g.rain_t_end = t_stop;
  drop_graph(c);
  return MWDG_OK;
}

mwdg_status mwdg_mra_encode(mwdg_ctx *c) {
  LIVE(c);
  if (c->g.mode != MWDG_ADAPTIVE) return fail(c, MWDG_ERR_STATE, "encode needs adaptive mode");
  if (!c->initial) return fail(c, MWDG_ERR_STATE, "no initial state");
  const Geo &g = c->g;
  c->launches += dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    return Launch<T>::adapt(g, p, 1, c->vmax_fresh ? 0 : 1, c->st, mark_cb, c);
  });
  CHECK_LAUNCH();
  c->encoded = true;
  c->vmax_fresh = true;
  return MWDG_OK;
}

mwdg_status mwdg_mra_adapt(mwdg_ctx *c, double eps, int64_t *n_active) {
  LIVE(c);
  if (!std::isfinite(eps) || eps < 0.0) return fail(c, MWDG_ERR_ARG, "invalid epsilon");
  if (!c->initial) return fail(c, MWDG_ERR_STATE, "no initial state");
  Geo &g = c->g;
  if (g.mode == MWDG_UNIFORM) return fail(c, MWDG_ERR_STATE, "uniform grids do not adapt");
  g.eps = eps;
  sync_single(g);
  drop_graph(c);
  if (g.mode == MWDG_STATIC) {
    if (c->stepped) return fail(c, MWDG_ERR_STATE, "a static grid is fixed once stepping started");
    mwdg_status s = build_static_grid(c, c->static_eta);
    if (s) return s;
    if ((s = prime(c))) return s;
  } else {
    // full encode with this epsilon, then threshold, regularise, decode
    const int with_max = c->vmax_fresh ? 0 : 1;
    c->launches += dispatch(c, [&](auto &p, auto *) {
      using T = std::remove_pointer_t<decltype(p.U)>;
      return Launch<T>::adapt(g, p, 0, with_max, c->st, mark_cb, c);
    });
    CHECK_LAUNCH();
    c->encoded = false;
    mwdg_status s = prime(c);  // max |v0| and dt over the new leaves
    if (s) return s;
  }
  if (n_active) {
    int n = 0;
    CK(cudaMemcpyAsync(&n, (g.prec == MWDG_F64) ? c->pd.nleaf : c->pf.nleaf, sizeof(int),
                       cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    *n_active = n;
  }
  return MWDG_OK;
}

mwdg_status mwdg_dg2_step(mwdg_ctx *c, double *dt_out) {
  LIVE(c);
  if (!c->initial) return fail(c, MWDG_ERR_STATE, "no initial state");
  mwdg_status s = queue_step(c);
  if (s) return s;
  if (dt_out) {
    Ctl h;
    if ((s = read_ctl(c, &h))) return s;
    *dt_out = h.dt;
  }
  return MWDG_OK;
}

mwdg_status mwdg_dg2_step_dt(mwdg_ctx *c, double dt) {
  LIVE(c);
  if (!c->initial) return fail(c, MWDG_ERR_STATE, "no initial state");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, MWDG_ERR_ARG, "dt must be positive and finite");
  k_set_dt_fixed<<<1, 1, 0, c->st>>>(c->ctl, dt);
  c->launches++;
  mwdg_status s = queue_step(c);
  // the prescribed step is withdrawn on every path
  k_set_dt_fixed<<<1, 1, 0, c->st>>>(c->ctl, 0.0);
  c->launches++;
  if (s) return s;
  CHECK_LAUNCH();
  return MWDG_OK;
}

mwdg_status mwdg_run_steps(mwdg_ctx *c, int64_t nsteps) {
  LIVE(c);
  if (!c->initial) return fail(c, MWDG_ERR_STATE, "no initial state");
  if (nsteps < 0) return fail(c, MWDG_ERR_ARG, "negative step count");
  for (int64_t k = 0; k < nsteps; k++) {
    mwdg_status s = queue_step(c);
    if (s) return s;
  }
  return MWDG_OK;
}

mwdg_status mwdg_run_to_time(mwdg_ctx *c, double t_end, int64_t *steps_out) {
  LIVE(c);
  if (!c->initial) return fail(c, MWDG_ERR_STATE, "no initial state");
  if (std::isnan(t_end)) return fail(c, MWDG_ERR_ARG, "t_end is NaN");
  Ctl h;
  mwdg_status s;
  if ((s = read_ctl(c, &h))) return s;
  const long long start = h.steps;
  k_set_tend<<<1, 1, 0, c->st>>>(c->ctl, t_end);
  c->launches++;
  int batch = 8;
  while (s == MWDG_OK && h.t < t_end) {
    const long long before = h.steps;
    for (int k = 0; k < batch && s == MWDG_OK; k++) s = queue_step(c);
    if (s == MWDG_OK) s = read_ctl(c, &h);
    if (s != MWDG_OK || h.steps == before) break;  // a failure, or dt reached zero
    // queue about as many steps as the last step length says are left
    double left = (h.dt > 0.0) ? (t_end - h.t) / h.dt : 1.0;
    batch = (int)std::max(1.0, std::min(256.0, std::ceil(left * 1.05) + 1.0));
  }
  // the end time is withdrawn on every path, so that later steps are not
  // clamped to it
  k_set_tend<<<1, 1, 0, c->st>>>(c->ctl, 1e300);
  c->launches++;
  if (s) return s;
  CHECK_LAUNCH();
  if (steps_out) *steps_out = h.steps - start;
  return MWDG_OK;
}

// the three finest rasters into the context's contiguous read-back buffer
static mwdg_status fields_to_buffer(mwdg_ctx *c) {
  const Geo &g = c->g;
  const size_t n = (size_t)g.nxl[g.L] * g.nyl[g.L];
  if (!c->d_fields) {
    mwdg_status s = alloc(c, &c->d_fields, 3 * n);
    if (s) return s;
  }
  double *b = c->d_fields;
  c->launches += dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    return Launch<T>::fields(g, p, b, b + n, b + 2 * n, c->st);
  });
  CHECK_LAUNCH();
  return MWDG_OK;
}

// from the read-back buffer to the caller's rasters (row stride ld; 0: nx)
static mwdg_status fields_out(mwdg_ctx *c, double *h, double *u, double *v, int64_t ld, cudaMemcpyKind kind) {
  const Geo &g = c->g;
  const size_t nx = (size_t)g.nxl[g.L], ny = (size_t)g.nyl[g.L], n = nx * ny;
  double *dst[3] = {h, u, v};
  for (int q = 0; q < 3; q++)
    if (dst[q])
      CK(cudaMemcpy2DAsync(dst[q], (size_t)ld * sizeof(double), c->d_fields + q * n, nx * sizeof(double),
                           nx * sizeof(double), ny, kind, c->st));
  return MWDG_OK;
}

mwdg_status mwdg_read_fields_dev(mwdg_ctx *c, double *h, double *u, double *v, int64_t ld) {
  LIVE(c);
  const Geo &g = c->g;
  const int64_t nx = g.nxl[g.L];
  if (ld != 0 && ld < nx) return fail(c, MWDG_ERR_ARG, "row stride %lld is below the row length %lld",
                                      (long long)ld, (long long)nx);
  if (ld == 0 || ld == nx) {  // straight into the caller's rasters
    c->launches += dispatch(c, [&](auto &p, auto *) {
      using T = std::remove_pointer_t<decltype(p.U)>;
      return Launch<T>::fields(g, p, h, u, v, c->st);
    });
    CHECK_LAUNCH();
    return MWDG_OK;
  }
  mwdg_status s = fields_to_buffer(c);
  if (s) return s;
  return fields_out(c, h, u, v, ld, cudaMemcpyDeviceToDevice);
}

mwdg_status mwdg_read_fields(mwdg_ctx *c, double *h, double *u, double *v, int64_t ld) {
  LIVE(c);
  const Geo &g = c->g;
  const int64_t nx = g.nxl[g.L];
  if (ld == 0) ld = nx;
  if (ld < nx) return fail(c, MWDG_ERR_ARG, "row stride %lld is below the row length %lld", (long long)ld,
                           (long long)nx);
  mwdg_status s = fields_to_buffer(c);
  if (s) return s;
  if ((s = fields_out(c, h, u, v, ld, cudaMemcpyDeviceToHost))) return s;
  CK(cudaStreamSynchronize(c->st));
  return MWDG_OK;
}

mwdg_status mwdg_read_gauges(mwdg_ctx *c, const int32_t *ij, int32_t n, double *h, double *u, double *v) {
  LIVE(c);
  if (n < 0 || (n > 0 && !ij)) return fail(c, MWDG_ERR_ARG, "invalid gauge list");
  const Geo &g = c->g;
  for (int32_t q = 0; q < n; q++)
    if (ij[2 * q] < 0 || ij[2 * q] >= g.nxl[g.L] || ij[2 * q + 1] < 0 || ij[2 * q + 1] >= g.nyl[g.L])
      return fail(c, MWDG_ERR_ARG, "gauge %d (%d, %d) outside the grid", q, ij[2 * q], ij[2 * q + 1]);
  if (n == 0) return MWDG_OK;
  if (n > c->gauge_cap) {
    int cap = 256;
    while (cap < n) cap *= 2;
    mwdg_status s;
    if ((s = alloc(c, &c->d_gauge_ij, 2 * (size_t)cap)) || (s = alloc(c, &c->d_gauge_out, 3 * (size_t)cap))) return s;
    c->gauge_cap = cap;
  }
  CK(cudaMemcpyAsync(c->d_gauge_ij, ij, 2 * (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, c->st));
  c->launches += dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    return Launch<T>::gauges(g, p, c->d_gauge_ij, n, c->d_gauge_out, c->st);
  });
  CHECK_LAUNCH();
  double *dst[3] = {h, u, v};
  for (int q = 0; q < 3; q++)
    if (dst[q])
      CK(cudaMemcpyAsync(dst[q], c->d_gauge_out + (size_t)q * n, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost,
                         c->st));
  CK(cudaStreamSynchronize(c->st));
  return MWDG_OK;
}

mwdg_status mwdg_read_active(mwdg_ctx *c, int32_t *level, int32_t *i, int32_t *j, double *coeffs,
                             int64_t cap, int64_t *n) {
  LIVE(c);
  if (!n) return fail(c, MWDG_ERR_ARG, "n is NULL");
  const Geo &g = c->g;
  int cnt = 0;
  CK(cudaMemcpyAsync(&cnt, (g.prec == MWDG_F64) ? c->pd.nleaf : c->pf.nleaf, sizeof(int),
                     cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  *n = cnt;
  if (!level && !i && !j && !coeffs) return MWDG_OK;
  if (cap < cnt) return fail(c, MWDG_ERR_CAPACITY, "capacity %lld < %d leaves", (long long)cap, cnt);
  if (!c->d_active) {
    mwdg_status s;
    if ((s = alloc(c, &c->d_active, 3 * (size_t)g.P)) || (s = alloc(c, &c->d_coef, 9 * (size_t)g.P))) return s;
  }
  const size_t P = (size_t)g.P;
  c->launches += dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    return Launch<T>::read_active(g, p, c->d_active, c->d_active + P, c->d_active + 2 * P, c->d_coef, c->st);
  });
  CHECK_LAUNCH();
  if (cnt > 0) {
    if (level) CK(cudaMemcpyAsync(level, c->d_active, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
    if (i) CK(cudaMemcpyAsync(i, c->d_active + P, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
    if (j) CK(cudaMemcpyAsync(j, c->d_active + 2 * P, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
    if (coeffs) CK(cudaMemcpyAsync(coeffs, c->d_coef, 9 * (size_t)cnt * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  }
  CK(cudaStreamSynchronize(c->st));
  if (g.mode == MWDG_UNIFORM && level)
    for (int q = 0; q < cnt; q++) level[q] = c->p.L;  // reported on the finest level of the parameters
  return MWDG_OK;
}

mwdg_status mwdg_get_time(mwdg_ctx *c, double *t, int64_t *steps) {
  LIVE(c);
  Ctl h;
  mwdg_status s = read_ctl(c, &h);
  if (s) return s;
  if (t) *t = h.t;
  if (steps) *steps = h.steps;
  return MWDG_OK;
}

mwdg_status mwdg_get_counters(mwdg_ctx *c, int64_t *steps, int64_t *updates) {
  LIVE(c);
  Ctl h;
  mwdg_status s = read_ctl(c, &h);
  if (s) return s;
  if (steps) *steps = h.steps;
  if (updates) *updates = h.updates;
  return MWDG_OK;
}

mwdg_status mwdg_get_volume(mwdg_ctx *c, double *V, double *V_in, double *V_out, double *V_rain,
                            double *V_clip, int64_t *n_clip) {
  LIVE(c);
  const Geo &g = c->g;
  c->launches += dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    // as many blocks as the partial sums hold (the kernel strides over the
    // leaves, so any count covers them; the launch shape may have grown)
    return Launch<T>::volume(g, p, std::min(c->grid_leaves, c->part_cap), c->st);
  });
  CHECK_LAUNCH();
  Ctl h;
  mwdg_status s = read_ctl(c, &h);
  if (s) return s;
  if (V) *V = h.volume;
  if (V_in) *V_in = h.v_in;
  if (V_out) *V_out = h.v_out;
  if (V_rain) *V_rain = h.v_rain;
  if (V_clip) *V_clip = h.v_clip;
  if (n_clip) *n_clip = (int64_t)h.n_clip;
  return MWDG_OK;
}

namespace {
struct StateHeader {
  char magic[8];
  int32_t version, prec, L, M, N, mode;
  int64_t P;
  Ctl ctl;
};
constexpr char kMagic[8] = {'M', 'W', 'D', 'G', 'S', 'T', '0', '1'};

size_t state_bytes(const mwdg_ctx *c) {
  const size_t P = (size_t)c->g.P, ts = (c->g.prec == MWDG_F64) ? 8 : 4;
  const size_t acc = (c->g.scheme == MWDG_ACC) ? 4 * P * ts : 0;  // ACC face discharges
  return sizeof(StateHeader) + P + 9 * P * ts + 3 * P * ts + P * ts + P * 8 + acc;
}
}  // namespace

mwdg_status mwdg_state_bytes(mwdg_ctx *c, int64_t *bytes) {
  LIVE(c);
  if (!bytes) return fail(c, MWDG_ERR_ARG, "bytes is NULL");
  *bytes = (int64_t)state_bytes(c);
  return MWDG_OK;
}

mwdg_status mwdg_save_state(mwdg_ctx *c, void *buf, int64_t cap) {
  LIVE(c);
  if (!buf) return fail(c, MWDG_ERR_ARG, "buffer is NULL");
  if (cap < (int64_t)state_bytes(c)) return fail(c, MWDG_ERR_CAPACITY, "state buffer too small");
  const Geo &g = c->g;
  StateHeader h{};
  memcpy(h.magic, kMagic, 8);
  h.version = 1;
  h.prec = g.prec;
  h.L = g.L;
  h.M = g.M;
  h.N = g.N;
  h.mode = g.mode;
  h.P = g.P;
  mwdg_status s = read_ctl(c, &h.ctl);
  if (s) return s;
  char *b = (char *)buf;
  memcpy(b, &h, sizeof h);
  b += sizeof h;
  const size_t P = (size_t)g.P, ts = (g.prec == MWDG_F64) ? 8 : 4;
  const void *kind = (g.prec == MWDG_F64) ? (void *)c->pd.kind : (void *)c->pf.kind;
  const void *U = (g.prec == MWDG_F64) ? (void *)c->pd.U : (void *)c->pf.U;
  const void *Z = (g.prec == MWDG_F64) ? (void *)c->pd.Z : (void *)c->pf.Z;
  const void *NM = (g.prec == MWDG_F64) ? (void *)c->pd.NM : (void *)c->pf.NM;
  const void *DZ = (g.prec == MWDG_F64) ? (void *)c->pd.DZ : (void *)c->pf.DZ;
  CK(cudaMemcpyAsync(b, kind, P, cudaMemcpyDeviceToHost, c->st));
  b += P;
  CK(cudaMemcpyAsync(b, U, 9 * P * ts, cudaMemcpyDeviceToHost, c->st));
  b += 9 * P * ts;
  CK(cudaMemcpyAsync(b, Z, 3 * P * ts, cudaMemcpyDeviceToHost, c->st));
  b += 3 * P * ts;
  CK(cudaMemcpyAsync(b, NM, P * ts, cudaMemcpyDeviceToHost, c->st));
  b += P * ts;
  CK(cudaMemcpyAsync(b, DZ, P * 8, cudaMemcpyDeviceToHost, c->st));
  b += P * 8;
  if (g.scheme == MWDG_ACC) {
    const void *Wi = (g.prec == MWDG_F64) ? (void *)c->pd.Wi : (void *)c->pf.Wi;
    CK(cudaMemcpyAsync(b, Wi, 4 * P * ts, cudaMemcpyDeviceToHost, c->st));
  }
  CK(cudaStreamSynchronize(c->st));
  return MWDG_OK;
}

mwdg_status mwdg_load_state(mwdg_ctx *c, const void *buf, int64_t size) {
  LIVE(c);
  if (!buf || size < (int64_t)sizeof(StateHeader)) return fail(c, MWDG_ERR_ARG, "not a state buffer");
  const Geo &g = c->g;
  StateHeader h;
  memcpy(&h, buf, sizeof h);
  if (memcmp(h.magic, kMagic, 8) != 0 || h.version != 1) return fail(c, MWDG_ERR_ARG, "not a state buffer");
  if (h.prec != g.prec || h.L != g.L || h.M != g.M || h.N != g.N || h.P != g.P || h.mode != g.mode)
    return fail(c, MWDG_ERR_DIMS, "state belongs to another grid or precision");
  if (size < (int64_t)state_bytes(c)) return fail(c, MWDG_ERR_ARG, "state buffer truncated");
  const char *b = (const char *)buf + sizeof h;
  const size_t P = (size_t)g.P, ts = (g.prec == MWDG_F64) ? 8 : 4;
  void *kind = (g.prec == MWDG_F64) ? (void *)c->pd.kind : (void *)c->pf.kind;
  void *U = (g.prec == MWDG_F64) ? (void *)c->pd.U : (void *)c->pf.U;
  void *Z = (g.prec == MWDG_F64) ? (void *)c->pd.Z : (void *)c->pf.Z;
  void *NM = (g.prec == MWDG_F64) ? (void *)c->pd.NM : (void *)c->pf.NM;
  void *DZ = (g.prec == MWDG_F64) ? (void *)c->pd.DZ : (void *)c->pf.DZ;
  CK(cudaMemcpyAsync(kind, b, P, cudaMemcpyHostToDevice, c->st));
  b += P;
  CK(cudaMemcpyAsync(U, b, 9 * P * ts, cudaMemcpyHostToDevice, c->st));
  b += 9 * P * ts;
  CK(cudaMemcpyAsync(Z, b, 3 * P * ts, cudaMemcpyHostToDevice, c->st));
  b += 3 * P * ts;
  CK(cudaMemcpyAsync(NM, b, P * ts, cudaMemcpyHostToDevice, c->st));
  b += P * ts;
  CK(cudaMemcpyAsync(DZ, b, P * 8, cudaMemcpyHostToDevice, c->st));
  b += P * 8;
  if (g.scheme == MWDG_ACC) {
    void *Wi = (g.prec == MWDG_F64) ? (void *)c->pd.Wi : (void *)c->pf.Wi;
    CK(cudaMemcpyAsync(Wi, b, 4 * P * ts, cudaMemcpyHostToDevice, c->st));
  }
  Ctl ctl = h.ctl;
  ctl.t_end = 1e300;
  ctl.blocks_done = 0u;
  CK(cudaMemcpyAsync(c->ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, c->st));
  c->launches += dispatch(c, [&](auto &p, auto *) {
    using T = std::remove_pointer_t<decltype(p.U)>;
    return Launch<T>::compact(g, p, c->st);
  });
  CHECK_LAUNCH();
  mwdg_status sp = prime(c);
  if (sp) return sp;
  CK(cudaStreamSynchronize(c->st));
  c->dem = c->initial = true;
  c->stepped = true;
  c->encoded = false;
  return MWDG_OK;
}

mwdg_status mwdg_profile(mwdg_ctx *c, int32_t enable) {
  LIVE(c);
  mwdg_status s = flush_marks(c);
  if (s) return s;
  for (auto &m : c->marks) c->pool.push_back(m.second);
  c->marks.clear();
  if (enable) {
    for (int k = 0; k < KC_COUNT; k++) {
      c->kms[k] = 0.0;
      c->kcount[k] = 0;
    }
  }
  c->prof = enable != 0;
  drop_graph(c);
  return MWDG_OK;
}

mwdg_status mwdg_kernel_times(mwdg_ctx *c, const char **names, double *ms, int64_t *launches, int32_t cap,
                              int32_t *n) {
  LIVE(c);
  mwdg_status s = flush_marks(c);
  if (s) return s;
  for (int k = 0; k < KC_COUNT && k < cap; k++) {
    if (names) names[k] = kclass_name(k);
    if (ms) ms[k] = c->kms[k];
    if (launches) launches[k] = c->kcount[k];
  }
  if (n) *n = KC_COUNT;
  return MWDG_OK;
}

mwdg_status mwdg_launch_count(mwdg_ctx *c, int64_t *n) {
  if (!c || !n) return MWDG_ERR_ARG;
  *n = c->launches;
  return MWDG_OK;
}

const char *mwdg_last_error(const mwdg_ctx *c) { return c ? c->err.c_str() : "no context"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Launch shape and ensembles
// ---------------------------------------------------------------------------
mwdg_status mwdg_set_launch_shape(mwdg_ctx *c, int32_t grid_leaves, int64_t coarse_nodes) {
  LIVE(c);
  if (grid_leaves > 65535) return fail(c, MWDG_ERR_ARG, "grid_leaves above 65535");
  if (grid_leaves > 0) {
    c->grid_leaves = grid_leaves;
    c->shape_set = true;
  }
  if (coarse_nodes > 0) c->g.coarse_nodes = coarse_nodes;
  drop_graph(c);
  return MWDG_OK;
}

mwdg_status mwdg_get_launch_shape(mwdg_ctx *c, int32_t *grid_leaves, int64_t *coarse_nodes) {
  LIVE(c);
  if (grid_leaves) *grid_leaves = c->grid_leaves;
  if (coarse_nodes) *coarse_nodes = c->g.coarse_nodes;
  return MWDG_OK;
}

struct mwdg_ensemble {
  std::vector<mwdg_ctx *> m;
  cudaStream_t st = nullptr;          // the caller's stream: ensemble work is ordered on it
  std::vector<cudaStream_t> br;       // one branch stream per member (used while capturing)
  std::vector<cudaEvent_t> ev;        // per member: ordering and join events
  cudaEvent_t fork = nullptr, done = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<int64_t> gen;           // member generations the graph was built from
  std::vector<int> nk;                // kernels per member in one ensemble step
  bool own_st = false;                // st created here (no caller stream)
  // batched launches: members of the adaptive DG2 pipeline with the same
  // precision step together, one launch per kernel over all their blocks
  int batch = 0;                                // members per batched group (0: none)
  std::vector<std::vector<int>> groups;         // members of each batched group
  std::vector<std::vector<BatchLaunch>> plans;  // its launches and member tables
  std::string err;
};

namespace {

mwdg_status efail(mwdg_ensemble *e, mwdg_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (e) e->err = buf;
  return s;
}

#define ECK(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return efail(e, MWDG_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                   __FILE__, __LINE__);                                                   \
  } while (0)

void ens_drop_graph(mwdg_ensemble *e) {
  if (e->graph) cudaGraphExecDestroy(e->graph);
  e->graph = nullptr;
}

// the batched groups' member tables (after the work that reads them)
void ens_free_plans(mwdg_ensemble *e) {
  if (!e->plans.empty() && e->st) cudaStreamSynchronize(e->st);
  for (auto &pl : e->plans)
    for (BatchLaunch &b : pl)
      if (b.tab) cudaFree(b.tab);
  e->plans.clear();
  e->groups.clear();
}

bool batchable(const mwdg_ctx *c) {
  return c->g.mode == MWDG_ADAPTIVE && c->g.scheme == MWDG_DG2 && c->g.L >= 1;
}

// groups of up to BMAX batchable members of one precision (two or more)
// and their launch plans
mwdg_status ens_plan(mwdg_ensemble *e) {
  ens_free_plans(e);
  if (e->batch < 2) return MWDG_OK;
  for (int prec : {MWDG_F32, MWDG_F64}) {
    std::vector<int> cand;
    for (size_t k = 0; k < e->m.size(); k++)
      if (batchable(e->m[k]) && e->m[k]->g.prec == prec) cand.push_back((int)k);
    for (size_t a = 0; a < cand.size(); a += (size_t)e->batch) {
      const size_t b = std::min(cand.size(), a + (size_t)e->batch);
      if (b - a >= 2) e->groups.emplace_back(cand.begin() + a, cand.begin() + b);
    }
  }
  for (const std::vector<int> &grp : e->groups) {
    e->plans.emplace_back();
    std::vector<const Geo *> gs;
    std::vector<int> gl;
    for (int k : grp) {
      gs.push_back(&e->m[k]->g);
      gl.push_back(e->m[k]->grid_leaves);
    }
    bool ok;
    if (e->m[grp[0]]->g.prec == MWDG_F64) {
      std::vector<const Ptrs<double> *> ps;
      for (int k : grp) ps.push_back(&e->m[k]->pd);
      ok = Launch<double>::batch_plan((int)grp.size(), gs.data(), ps.data(), gl.data(), e->plans.back());
    } else {
      std::vector<const Ptrs<float> *> ps;
      for (int k : grp) ps.push_back(&e->m[k]->pf);
      ok = Launch<float>::batch_plan((int)grp.size(), gs.data(), ps.data(), gl.data(), e->plans.back());
    }
    if (!ok) {
      cudaGetLastError();
      ens_free_plans(e);
      return efail(e, MWDG_ERR_CUDA, "ensemble: batched launch tables could not be allocated");
    }
  }
  return MWDG_OK;
}

// members ready to step (reductions of their current leaves), and ensemble
// work ordered after each member's earlier work
mwdg_status ens_begin(mwdg_ensemble *e) {
  for (size_t k = 0; k < e->m.size(); k++) {
    mwdg_ctx *c = e->m[k];
    if (!c || c->failed) return efail(e, MWDG_ERR_STATE, "member %zu is in an error state", k);
    if (!c->initial) return efail(e, MWDG_ERR_STATE, "member %zu has no initial state", k);
    if (c->prof) return efail(e, MWDG_ERR_STATE, "member %zu has per-kernel timing on", k);
    if (c->g.mode == MWDG_ADAPTIVE && !c->vmax_fresh) {
      mwdg_status s = prime(c);
      if (s) return efail(e, s, "member %zu: %s", k, c->err.c_str());
    }
    ECK(cudaEventRecord(e->ev[k], c->st));
    ECK(cudaStreamWaitEvent(e->st, e->ev[k], 0));
  }
  return MWDG_OK;
}

// members' later work ordered after the ensemble work; step bookkeeping
mwdg_status ens_end(mwdg_ensemble *e, int64_t graph_launches) {
  ECK(cudaEventRecord(e->done, e->st));
  for (mwdg_ctx *c : e->m) {
    ECK(cudaStreamWaitEvent(c->st, e->done, 0));
    if (graph_launches > 0) {
      c->stepped = true;
      c->encoded = false;
      c->vmax_fresh = true;
    }
  }
  return MWDG_OK;
}

// one ensemble step as a graph: fork, every member's step on its own branch
// stream, join
mwdg_status ens_graph(mwdg_ensemble *e) {
  bool stale = !e->graph;
  for (size_t k = 0; k < e->m.size() && !stale; k++) stale = e->gen[k] != e->m[k]->generation;
  if (!stale) return MWDG_OK;
  ens_drop_graph(e);
  mwdg_status ps = ens_plan(e);
  if (ps != MWDG_OK) return ps;
  std::vector<char> grouped(e->m.size(), 0);
  for (const std::vector<int> &grp : e->groups)
    for (int k : grp) grouped[k] = 1;
  cudaGraph_t gr = nullptr;
  ECK(cudaStreamBeginCapture(e->st, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaEventRecord(e->fork, e->st);
  // each batched group on the branch of its first member
  for (size_t q = 0; q < e->groups.size() && err == cudaSuccess; q++) {
    const int k0 = e->groups[q][0];
    err = cudaStreamWaitEvent(e->br[k0], e->fork, 0);
    if (err != cudaSuccess) break;
    const int nl = e->m[k0]->g.prec == MWDG_F64 ? Launch<double>::batch_step(e->plans[q], e->br[k0])
                                                : Launch<float>::batch_step(e->plans[q], e->br[k0]);
    for (int k : e->groups[q]) e->nk[k] = 0;
    e->nk[k0] = nl;
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(e->ev[k0], e->br[k0]);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(e->st, e->ev[k0], 0);
  }
  for (size_t k = 0; k < e->m.size() && err == cudaSuccess; k++) {
    if (grouped[k]) continue;
    mwdg_ctx *c = e->m[k];
    err = cudaStreamWaitEvent(e->br[k], e->fork, 0);
    if (err != cudaSuccess) break;
    cudaStream_t own = c->st;
    c->st = e->br[k];
    e->nk[k] = launch_step(c, 0);
    c->st = own;
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(e->ev[k], e->br[k]);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(e->st, e->ev[k], 0);
  }
  cudaError_t e1 = cudaStreamEndCapture(e->st, &gr);
  if (err != cudaSuccess || e1 != cudaSuccess || !gr) {
    if (gr) cudaGraphDestroy(gr);
    return efail(e, MWDG_ERR_CUDA, "ensemble capture: %s",
                 cudaGetErrorString(err != cudaSuccess ? err : e1));
  }
  cudaError_t e2 = cudaGraphInstantiate(&e->graph, gr, 0);
  cudaGraphDestroy(gr);
  if (e2 != cudaSuccess) return efail(e, MWDG_ERR_CUDA, "ensemble graph: %s", cudaGetErrorString(e2));
  for (size_t k = 0; k < e->m.size(); k++) e->gen[k] = e->m[k]->generation;
  return MWDG_OK;
}

mwdg_status ens_launch(mwdg_ensemble *e, int64_t n) {
  for (int64_t q = 0; q < n; q++) ECK(cudaGraphLaunch(e->graph, e->st));
  for (size_t k = 0; k < e->m.size(); k++) e->m[k]->launches += (int64_t)e->nk[k] * n;
  return MWDG_OK;
}

}  // namespace

mwdg_status mwdg_ensemble_create(mwdg_ctx *const *members, int32_t n, void *cuda_stream, mwdg_ensemble **out) {
  if (!members || !out || n < 1) return MWDG_ERR_ARG;
  *out = nullptr;
  for (int32_t a = 0; a < n; a++) {
    if (!members[a]) return MWDG_ERR_ARG;
    if (members[a]->failed || !members[a]->initial) return MWDG_ERR_STATE;
    for (int32_t b = 0; b < a; b++)
      if (members[a] == members[b]) return MWDG_ERR_ARG;
  }
  mwdg_ensemble *e = new mwdg_ensemble();
  e->m.assign(members, members + n);
  e->st = (cudaStream_t)cuda_stream;
  e->gen.assign(n, -1);
  e->nk.assign(n, 0);
  bool ok = true;
  if (!e->st) {  // a capturable stream of its own
    ok = cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking) == cudaSuccess;
    e->own_st = ok;
  }
  ok = ok && cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&e->done, cudaEventDisableTiming) == cudaSuccess;
  for (int32_t k = 0; k < n && ok; k++) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    if (s) e->br.push_back(s);
    if (ev) e->ev.push_back(ev);
  }
  if (!ok) {
    mwdg_ensemble_destroy(e);
    return MWDG_ERR_CUDA;
  }
  *out = e;
  return MWDG_OK;
}

void mwdg_ensemble_destroy(mwdg_ensemble *e) {
  if (!e) return;
  if (e->st) cudaStreamSynchronize(e->st);
  ens_drop_graph(e);
  ens_free_plans(e);
  for (cudaStream_t s : e->br) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (cudaEvent_t ev : e->ev) cudaEventDestroy(ev);
  if (e->fork) cudaEventDestroy(e->fork);
  if (e->done) cudaEventDestroy(e->done);
  if (e->own_st && e->st) cudaStreamDestroy(e->st);
  delete e;
}

mwdg_status mwdg_ensemble_step(mwdg_ensemble *e, int64_t n) {
  if (!e) return MWDG_ERR_ARG;
  if (n < 0) return efail(e, MWDG_ERR_ARG, "negative step count");
  mwdg_status s;
  if ((s = ens_begin(e)) || (s = ens_graph(e)) || (s = ens_launch(e, n))) return s;
  return ens_end(e, n);
}

mwdg_status mwdg_ensemble_run_to_time(mwdg_ensemble *e, double t_end, int64_t *graph_launches_out) {
  if (!e) return MWDG_ERR_ARG;
  if (std::isnan(t_end)) return efail(e, MWDG_ERR_ARG, "t_end is NaN");
  mwdg_status s;
  if ((s = ens_begin(e)) || (s = ens_graph(e))) return s;
  const size_t nm = e->m.size();
  for (mwdg_ctx *c : e->m) k_set_tend<<<1, 1, 0, e->st>>>(c->ctl, t_end);
  ECK(cudaGetLastError());
  std::vector<Ctl> h(nm);
  auto read_all = [&]() -> mwdg_status {
    for (size_t k = 0; k < nm; k++)
      ECK(cudaMemcpyAsync(&h[k], e->m[k]->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, e->st));
    ECK(cudaStreamSynchronize(e->st));
    for (size_t k = 0; k < nm; k++)
      if (h[k].nonfinite) {
        e->m[k]->failed = true;
        e->m[k]->err = "non-finite value in the solution";
        return efail(e, MWDG_ERR_NONFINITE, "member %zu: non-finite value in the solution", k);
      }
    return MWDG_OK;
  };
  if ((s = read_all())) return s;
  int64_t launched = 0;
  int batch = 8;
  for (;;) {
    bool open = false;
    long long before = 0;
    for (size_t k = 0; k < nm; k++) {
      open = open || h[k].t < t_end;
      before += h[k].steps;
    }
    if (!open) break;
    if ((s = ens_launch(e, batch))) return s;
    launched += batch;
    if ((s = read_all())) return s;
    long long after = 0;
    double left = 1.0;
    for (size_t k = 0; k < nm; k++) {
      after += h[k].steps;
      if (h[k].t < t_end && h[k].dt > 0.0) left = std::max(left, (t_end - h[k].t) / h[k].dt);
    }
    if (after == before) break;  // every open member's dt reached zero
    batch = (int)std::max(1.0, std::min(256.0, std::ceil(left * 1.05) + 1.0));
  }
  for (mwdg_ctx *c : e->m) k_set_tend<<<1, 1, 0, e->st>>>(c->ctl, 1e300);
  ECK(cudaGetLastError());
  if (graph_launches_out) *graph_launches_out = launched;
  return ens_end(e, launched);
}

mwdg_status mwdg_ensemble_tune(mwdg_ensemble *e, int32_t steps, int64_t *chosen) {
  if (!e) return MWDG_ERR_ARG;
  if (steps < 1) return efail(e, MWDG_ERR_ARG, "steps must be positive");
  static const int grids[] = {152, 304, 608, 1216};
  static const long long coarse[] = {64, 256, 1024};
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  ECK(cudaEventCreate(&t0));
  ECK(cudaEventCreate(&t1));
  mwdg_status s = MWDG_OK;
  for (size_t k = 0; k < e->m.size() && s == MWDG_OK; k++) {
    mwdg_ctx *c = e->m[k];
    std::vector<char> saved(state_bytes(c));
    if ((s = mwdg_save_state(c, saved.data(), (int64_t)saved.size()))) break;
    const int grid0 = c->grid_leaves;
    const long long coarse0 = c->g.coarse_nodes;
    const int grid_max = (int)std::max<long long>(1, std::min<long long>((c->g.P + 255) / 256, 152 * 8));
    float best = 1e30f;
    int bg = grid0;
    long long bc = coarse0;
    for (int gi : grids) {
      const int gsz = std::min(gi, grid_max);
      for (long long cn : coarse) {
        if ((s = mwdg_set_launch_shape(c, gsz, cn))) break;
        if ((s = queue_step(c))) break;  // warm-up (captures the step)
        cudaEventRecord(t0, c->st);
        for (int q = 0; q < steps && s == MWDG_OK; q++) s = queue_step(c);
        cudaEventRecord(t1, c->st);
        if (s || cudaEventSynchronize(t1) != cudaSuccess) {
          if (!s) s = MWDG_ERR_CUDA;
          break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (ms < best) {
          best = ms;
          bg = gsz;
          bc = cn;
        }
        if ((s = mwdg_load_state(c, saved.data(), (int64_t)saved.size()))) break;
      }
      if (s) break;
    }
    if (s) {
      efail(e, s, "tuning member %zu: %s", k, c->err.c_str());
      break;
    }
    if ((s = mwdg_set_launch_shape(c, bg, bc))) break;
    if (chosen) {
      chosen[2 * k] = bg;
      chosen[2 * k + 1] = bc;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  ens_drop_graph(e);
  return s;
}

mwdg_status mwdg_ensemble_set_batched(mwdg_ensemble *e, int32_t group) {
  if (!e) return MWDG_ERR_ARG;
  if (group < 0 || group > BMAX) return efail(e, MWDG_ERR_ARG, "group size outside 0..%d", BMAX);
  if (group == 1) group = 0;
  if (e->batch != group) {
    e->batch = group;
    if (e->st) cudaStreamSynchronize(e->st);
    ens_drop_graph(e);
    ens_free_plans(e);
    std::fill(e->gen.begin(), e->gen.end(), -1);
  }
  return MWDG_OK;
}

const char *mwdg_ensemble_last_error(const mwdg_ensemble *e) { return e ? e->err.c_str() : "null ensemble"; }
