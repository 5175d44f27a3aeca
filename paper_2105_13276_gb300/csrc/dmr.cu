// dmr.cu -- host side of the C ABI declared in include/dmr.h: configuration,
// workspace layout, stream-ordered orchestration of the kernels in
// dmr_kernels.cuh, per-period CUDA graphs and the growth decision.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include "dmr.h"
#include "dmr_kernels.cuh"
#include "dmr_adjoint.cuh"
#include "dmr_period.cuh"

namespace {

// CODATA 2018 (SI)
constexpr double C0 = 299792458.0;
constexpr double MU0 = 1.25663706212e-6;
constexpr double EPS0 = 8.8541878128e-12;
constexpr double QE = 1.602176634e-19;
constexpr double ME = 9.1093837015e-31;
constexpr double PI = 3.14159265358979323846;

thread_local std::string g_err;

constexpr int kTrialLaunches = 20;   // launches per autotuner trial graph

// Mean duration (ms) of one of n back-to-back launches made by `launch`,
// captured in a CUDA graph on st and replayed (best of three timed replays
// after one untimed): the periods run as graphs too, and direct launches of
// small kernels would measure the host's launch rate instead.
template <class F>
cudaError_t graph_time(cudaStream_t st, F&& launch, int n, float* ms_out) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  for (int w = 0; w < n; ++w) launch();
  e = cudaStreamEndCapture(st, &g);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) return e;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess && rep > 0 && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best) best = ms;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaGraphExecDestroy(ge);
  *ms_out = best / (float)n;
  return e;
}

std::string fmt(const char* f, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, f);
  vsnprintf(buf, sizeof buf, f, ap);
  va_end(ap);
  return buf;
}

inline size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Physical set-up derived from a dmr_config (Sec. II.A readings).
struct Derived {
  double omega, lam, k, nu_m, dxc, dxf, dtc, dtf, De, Da, r_ei, nu_scale, nu_a, n_crit, n_th,
      g_th, T;
  int64_t cap;
  int m_ex, m_ey;   // threshold-line jumps (growth = 2)
  int nu_model;     // 0 air fit, 1 Townsend form
  double town_A, town_B;
  int boundary;     // 0 Mur, 1 CPML
  int pml;          // CPML thickness (coarse cells)
  int margin;       // the fine rectangle stays this many coarse cells inside
  int coupling;     // 0 fine E means and density back to the coarse mesh, 1 density only
};

int derive(const dmr_config* c, Derived* d, std::string* err) {
  if (!c) { *err = "null config"; return DMR_EINVAL; }
  if (c->nx < 4 || c->ny < 4) { *err = "nx and ny must be >= 4"; return DMR_EINVAL; }
  if (c->r < 1 || c->r > 16) { *err = "r must be in [1, 16]"; return DMR_EINVAL; }
  if (c->n_lambda < 1 || c->steps_per_period < 1) { *err = "n_lambda and steps_per_period must be >= 1"; return DMR_EINVAL; }
  if (c->precision != 0 && c->precision != 1) { *err = "precision must be 0 (fp64) or 1 (fp32)"; return DMR_EINVAL; }
  if (!(c->freq > 0) || !(c->p_torr > 0) || !std::isfinite(c->E0)) { *err = "freq and p_torr must be > 0, E0 finite"; return DMR_EINVAL; }
  if (c->buffer_cells < 0) { *err = "buffer_cells must be >= 0"; return DMR_EINVAL; }
  if (c->growth < 0 || c->growth > 2) { *err = "growth must be 0, 1 or 2"; return DMR_EINVAL; }
  d->m_ex = c->m_ex >= 0 ? c->m_ex : 2 * c->buffer_cells;
  d->m_ey = c->m_ey >= 0 ? c->m_ey : c->buffer_cells;
  if (c->nu_model != 0 && c->nu_model != 1) { *err = "nu_model must be 0 or 1"; return DMR_EINVAL; }
  d->nu_model = c->nu_model;
  d->town_A = c->town_A > 0 ? c->town_A : 1500.0;     // 15 /(cm Torr)
  d->town_B = c->town_B > 0 ? c->town_B : 36500.0;    // 365 V/(cm Torr)
  if (c->boundary != 0 && c->boundary != 1) { *err = "boundary must be 0 (Mur) or 1 (CPML)"; return DMR_EINVAL; }
  d->boundary = c->boundary;
  if (c->coupling != 0 && c->coupling != 1) { *err = "coupling must be 0 (two-way) or 1 (density only)"; return DMR_EINVAL; }
  d->coupling = c->coupling;
  d->pml = c->pml_cells > 0 ? c->pml_cells : 8;
  d->margin = c->boundary == 1 ? d->pml + 2 : 0;
  if (c->boundary == 1 && (2 * d->pml + 2 > c->nx || 2 * d->pml + 2 > c->ny)) {
    *err = "the CPML layers leave no interior";
    return DMR_EINVAL;
  }
  d->omega = 2.0 * PI * c->freq;
  d->lam = C0 / c->freq;
  d->k = d->omega / C0;
  d->nu_m = 5.3e9 * c->p_torr;                       // Sec. II.A
  d->dxc = d->lam / (double)c->n_lambda;
  d->dxf = d->lam / ((double)c->r * (double)c->n_lambda);
  d->dtc = 1.0 / (c->freq * (double)c->steps_per_period);
  d->dtf = 1.0 / (c->freq * (double)((int64_t)c->r * c->steps_per_period));
  d->De = c->De >= 0 ? c->De : 0.1 * 760.0 / c->p_torr;
  d->Da = c->Da >= 0 ? c->Da : d->De / 100.0;
  const double beta = c->beta_rec >= 0 ? c->beta_rec : 1.0;
  const double Te = c->Te > 0 ? c->Te : 300.0;
  d->r_ei = beta * 1e-13 * std::sqrt(300.0 / Te);   // Sec. II.A, m^3/s
  d->nu_scale = c->nu_scale >= 0 ? c->nu_scale : 1.0;
  d->nu_a = c->nu_a;
  d->n_crit = ME * EPS0 * d->omega * d->omega / (QE * QE);
  d->n_th = c->n_th >= 0 ? c->n_th : 1e-3 * d->n_crit;
  d->g_th = c->g_th > 0 ? c->g_th : d->n_th / (4.0 * d->dxc);
  d->T = 1.0 / c->freq;
  const int64_t full = (int64_t)c->r * c->nx * (int64_t)c->r * c->ny;
  d->cap = c->patch_cap_cells > 0 ? std::min<int64_t>(c->patch_cap_cells, full) : full;
  // stability guard
  const double courant = (double)c->n_lambda / (double)c->steps_per_period;
  if (courant > 1.0 / std::sqrt(2.0)) {
    *err = fmt("Courant number %.4f > 1/sqrt(2)", courant);
    return DMR_EUNSTABLE;
  }
  const double dmax = std::max(d->De, d->Da);
  if (dmax * d->T / (d->dxf * d->dxf) > 0.25) {
    *err = fmt("diffusion number %.4f > 1/4", dmax * d->T / (d->dxf * d->dxf));
    return DMR_EUNSTABLE;
  }
  return DMR_OK;
}

constexpr int BX = dmr::TX, BY = dmr::TY;

struct Layout {
  size_t es = 8;       // bytes per field element
  int pc = 0;          // coarse pitch (elements)
  size_t cplane = 0;   // coarse elements per array
  size_t fplane = 0;   // fine elements per array (capacity)
  int nblk_c = 0, nblk_f = 0;
  size_t off_c[14] = {}, off_cS2 = 0;     // Ex Ey Hz vx vy n ntmp D nu, then Ex' Ey' Hz' vx' vy'
  size_t off_f[2][11] = {}, off_fS2[2] = {};  // Ex Ey Hz vx vy n, then Ex' Ey' Hz' vx' vy'
  size_t off_ftmp[3] = {};                // ntmp D nu
  size_t off_cErms = 0, off_fErms[2] = {};  // E_rms of the last completed period (nodes)
  size_t off_tab[4] = {};                 // ckx_c skx_c ckx_f skx_f
  size_t off_ph[4] = {};                  // sin/cos of the phase per step: coarse, fine
  size_t off_mask = 0, off_part[4] = {}, off_ctl = 0, off_view = 0;
  size_t off_psi[8] = {};                 // CPML psi, parity 0 then 1: Hz (x, y), Ex (y), Ey (x)
  size_t off_pmlc[8] = {};                // CPML b, c: x cells, y cells, x nodes, y nodes
  size_t off_sched = 0, off_ptab = 0;     // persistent period: counters + unit flags, argument tables
  int nsched = 0;                         // words at off_sched (cleared by every period end)
  size_t total = 0;
};

// persistent period words: the fine sub-step counts (one 128-byte line each),
// then one near-rectangle count per step of a period, then the coarse unit flags
constexpr int kSchedCnt = dmr::kCntStride * (dmr::kMaxR + 1);

int64_t fine_pitch(int64_t nfx) { return (int64_t)up((size_t)nfx + 1, 64); }

int make_layout(const dmr_config* c, const Derived& d, Layout* L, std::string* err) {
  L->es = c->precision == 1 ? 4 : 8;
  const int64_t nx = c->nx, ny = c->ny, r = c->r;
  L->pc = (int)up((size_t)nx + 1, 64);
  L->cplane = (size_t)(ny + 1) * L->pc;
  if (r > 1) {
    // any rectangle with nfx*nfy <= cap fits (nfy+1) * roundup(nfx+1, 64) elements
    const int64_t bound = d.cap + r * nx + 64 * (r * ny + 1) + 64;
    const int64_t full = (r * ny + 1) * fine_pitch(r * nx);
    L->fplane = (size_t)std::min(bound, full);
  }
  if ((int64_t)L->cplane >= (1ll << 31) || (int64_t)L->fplane >= (1ll << 31)) {
    *err = "mesh too large for 32-bit element indices";
    return DMR_EINVAL;
  }
  L->nblk_c = (int)(((nx + 1 + BX - 1) / BX) * ((ny + 1 + BY - 1) / BY));
  L->nblk_f = r > 1 ? (int)(((r * nx + 1 + BX - 1) / BX) * ((r * ny + 1 + BY - 1) / BY)) : 0;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = up(o + bytes, 256); return at; };
  for (int q = 0; q < 14; ++q) L->off_c[q] = take(L->cplane * L->es);
  L->off_cS2 = take(L->cplane * 8);
  L->off_cErms = take(L->cplane * L->es);
  if (r > 1) {
    for (int s = 0; s < 2; ++s) {
      for (int q = 0; q < 11; ++q) L->off_f[s][q] = take(L->fplane * L->es);
      L->off_fS2[s] = take(L->fplane * 8);
      L->off_fErms[s] = take(L->fplane * L->es);
    }
    for (int q = 0; q < 3; ++q) L->off_ftmp[q] = take(L->fplane * L->es);
  }
  L->off_tab[0] = take((size_t)(nx + 1) * L->es);
  L->off_tab[1] = take((size_t)(nx + 1) * L->es);
  L->off_tab[2] = take((size_t)(r * nx + 1) * L->es);
  L->off_tab[3] = take((size_t)(r * nx + 1) * L->es);
  L->off_ph[0] = take((size_t)c->steps_per_period * L->es);
  L->off_ph[1] = take((size_t)c->steps_per_period * L->es);
  L->off_ph[2] = take((size_t)r * c->steps_per_period * L->es);
  L->off_ph[3] = take((size_t)r * c->steps_per_period * L->es);
  L->off_mask = take((size_t)(nx + 1) * (ny + 1));
  L->off_part[0] = take((size_t)L->nblk_c * 8);
  L->off_part[1] = take((size_t)std::max(L->nblk_f, 1) * 8);
  L->off_part[2] = take((size_t)L->nblk_c * 8);
  L->off_part[3] = take((size_t)std::max(L->nblk_f, 1) * 8);
  L->off_ctl = take(sizeof(dmr::Ctl));
  L->off_view = take(std::max(L->cplane, L->fplane) * 8);
  if (d.boundary == 1) {
    for (int q = 0; q < 8; ++q) L->off_psi[q] = take(L->cplane * L->es);
    const size_t len[8] = {(size_t)nx, (size_t)nx, (size_t)ny, (size_t)ny,
                           (size_t)nx + 1, (size_t)nx + 1, (size_t)ny + 1, (size_t)ny + 1};
    for (int q = 0; q < 8; ++q) L->off_pmlc[q] = take(len[q] * L->es);
  }
  {
    // persistent period: kSchedCnt count words, one count per step, then one
    // flag per coarse unit (at most one unit per EM_WARPS node rows of a strip)
    const int64_t gx = (nx + 1 + dmr::STRIP_W - 1) / dmr::STRIP_W;
    const int64_t uy = (ny + 1 + dmr::EM_WARPS - 1) / dmr::EM_WARPS;
    L->nsched = (int)(kSchedCnt + c->steps_per_period + gx * uy);
    L->off_sched = take((size_t)L->nsched * 4);
    const size_t ea = L->es == 4 ? sizeof(dmr::EmArgs<float>) : sizeof(dmr::EmArgs<double>);
    L->off_ptab = take(2 * (dmr::kMaxR + 1) * ea);
  }
  L->total = o;
  return DMR_OK;
}

// --------------------------------------------------------------------------
struct Base {
  dmr_config cfg{};
  Derived d{};
  Layout L{};
  char* ws = nullptr;
  cudaStream_t st = nullptr;
  std::string err;
  int64_t m = 0;            // coarse steps done (time level of coarse E)
  int num_sms = 152;
  int64_t launches = 0;
  bool capturing = false;
  int64_t graph_nodes = 0;
  bool graphs = false;
  // the EM steps of a whole period in one persistent launch (k_period)
  bool persist = false;
  int prow_c = 0, prow_f = 0;          // node rows per warp of its coarse / fine units (0: chosen)
  long long sched_limit = 1ll << 22;   // polls of one of its waits before it gives up
  int sched_stall = 0;                 // test: one unit waits for a count nothing reaches
  bool dead = false;                   // such a wait gave up: the run's fields are lost
  bool in_batch = false;               // a run of a batch (its launches go through segment tables)
  cudaGraphExec_t gexec = nullptr;
  int g_cpar = 0, g_fpar = 0, g_rvalid = 0;   // state the graph was captured in
  std::vector<int32_t> replay;
  size_t replay_pos = 0;
  bool has_fine = false;
  int rect[4] = {-1, -1, -1, -1};
  // timing: event pairs around launches; direct launches use a pool that is
  // recycled every period, a captured graph owns its events until dropped
  bool timing = false;
  std::vector<cudaEvent_t> evd, evg;
  size_t evd_used = 0;
  struct Pend { int cls; int a, b; double units; };
  std::vector<Pend> pend, gpend;
  double kt_ms[8] = {};
  int64_t kt_n[8] = {};
  double kt_units[8] = {};

  virtual ~Base() {
    if (gexec) cudaGraphExecDestroy(gexec);
    for (auto e : evd) cudaEventDestroy(e);
    for (auto e : evg) cudaEventDestroy(e);
  }
  int fail(int code, const std::string& msg) { err = msg; return code; }
  int ck(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return DMR_OK;
    return fail(DMR_ECUDA, fmt("%s: %s", what, cudaGetErrorString(e)));
  }
  void drop_graph() {
    if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
    gpend.clear();
    for (auto e : evg) cudaEventDestroy(e);
    evg.clear();
  }
  int ev_get() {
    if (capturing) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      evg.push_back(e);
      return (int)evg.size() - 1;
    }
    if (evd_used >= evd.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      evd.push_back(e);
    }
    return (int)evd_used++;
  }
  cudaEvent_t ev_at(int idx, bool graph) const { return graph ? evg[idx] : evd[idx]; }
  // inside a stream capture a plain record only orders work; the external
  // flag turns it into an event-record node that fires on every replay
  void record(cudaEvent_t e) {
    if (capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
  }
  unsigned timing_mask = 0xffffffffu;
  // units: algorithmic bytes the timed launch must move (0: not a bandwidth kernel)
  int tbeg(int cls, double units) {
    if (!timing || !((timing_mask >> cls) & 1u)) return -1;
    int a = ev_get();
    if (a < 0) return -1;
    record(ev_at(a, capturing));
    auto& v = capturing ? gpend : pend;
    v.push_back({cls, a, -1, units});
    return (int)v.size() - 1;
  }
  void tend(int h) {
    if (h < 0) return;
    auto& v = capturing ? gpend : pend;
    int b = ev_get();
    if (b < 0) { v[h].cls = -1; return; }
    record(ev_at(b, capturing));
    v[h].b = b;
  }
  void harvest(const std::vector<Pend>& v, bool graph) {
    for (const auto& p : v) {
      if (p.cls < 0 || p.b < 0) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev_at(p.a, graph), ev_at(p.b, graph)) == cudaSuccess) {
        kt_ms[p.cls] += ms;
        kt_n[p.cls] += 1;
        kt_units[p.cls] += p.units;
      }
    }
  }
  void harvest_period(bool graph_ran) {
    if (!timing) return;
    harvest(pend, false);
    pend.clear();
    evd_used = 0;
    if (graph_ran) harvest(gpend, true);
  }
  void counted(int k) {
    if (capturing) graph_nodes += k; else launches += k;
  }

  virtual int init() = 0;
  virtual int seed(double n0, double x0, double y0, double sx, double sy, int add) = 0;
  virtual int set_patch(const int32_t* r4) = 0;
  virtual int advance(int64_t n) = 0;
  virtual int shape(int field, int level, int32_t* s, int32_t* eb) const = 0;
  virtual int read(int field, int level, void* dst, size_t bytes, int dev) = 0;
  virtual int write(int field, int level, const void* src, size_t bytes, int dev) = 0;
  virtual int stats(double* out) = 0;
  virtual int autotune(int32_t* wps, double* trial_ms) = 0;
  virtual void set_shape(int wps) = 0;
  virtual void set_cols(int cols) = 0;
  virtual void get_shape(int32_t* out) const = 0;
  virtual int adj_record(int64_t n, int64_t K, void* ckpt, size_t bytes) = 0;
  virtual size_t adj_ckpt_bytes(int64_t n, int64_t K) const = 0;
  virtual size_t adj_bytes() const = 0;
  virtual int adj_backward(const void* dLdn, void* ws, size_t bytes, void* ckpt, size_t cbytes,
                           double* dE0, double* dnu, void* dseed) = 0;
  virtual int time_launch(int form, int reps, double* ms, double* bytes) = 0;
  virtual size_t state_bytes() const = 0;
  virtual int save_state(void* dst, size_t bytes) = 0;
  virtual int load_state(const void* src, size_t bytes) = 0;
};

// Header of a saved run state (dmr_save_state): the host-side step counter,
// buffer parities and rectangle, position-independent, followed in the
// caller's buffer by an image of the whole workspace.
struct StateHdr {
  char magic[8];
  uint32_t version, es;
  uint64_t total;
  int64_t m;
  int32_t cpar, fpar, cur, has_fine, rvalid;
  int32_t rect[4];
  int64_t replay_pos;   // periods of a replayed refinement log consumed
  dmr_config cfg;
};
constexpr size_t kStateHdrBytes = 512;
static_assert(sizeof(StateHdr) <= kStateHdrBytes, "state header too large");
constexpr char kStateMagic[8] = {'D', 'M', 'R', 'S', 'T', 'A', 'T', 'E'};

// Configurations describe the same run (field by field: padding bytes of the
// struct are not compared).
bool same_config(const dmr_config& a, const dmr_config& b) {
  return a.nx == b.nx && a.ny == b.ny && a.r == b.r && a.n_lambda == b.n_lambda &&
         a.steps_per_period == b.steps_per_period && a.precision == b.precision &&
         a.buffer_cells == b.buffer_cells && a.growth == b.growth &&
         a.patch_cap_cells == b.patch_cap_cells && a.freq == b.freq && a.E0 == b.E0 &&
         a.p_torr == b.p_torr && a.De == b.De && a.Da == b.Da && a.beta_rec == b.beta_rec &&
         a.Te == b.Te && a.nu_scale == b.nu_scale && a.nu_a == b.nu_a && a.n_th == b.n_th &&
         a.g_th == b.g_th && a.m_ex == b.m_ex && a.m_ey == b.m_ey && a.nu_model == b.nu_model &&
         a.town_A == b.town_A && a.town_B == b.town_B && a.boundary == b.boundary &&
         a.pml_cells == b.pml_cells && a.coupling == b.coupling;
}

template <class T>
struct Engine final : Base {
  // C and F[cur] always point at the current (level n) E/H buffers; the
  // other buffer of each pair receives the next level (double buffering).
  dmr::Mesh<T> C{};
  T* cE[2][5] = {};          // [parity][Ex, Ey, Hz, vx, vy]
  int cpar = 0;
  T *c_ntmp = nullptr, *c_D = nullptr, *c_nu = nullptr;
  dmr::Mesh<T> F[2]{};
  T* fptr[2][6] = {};        // [set][Ex, Ey, Hz, vx, vy, n] (parity 0)
  T* fE1[2][5] = {};         // [set][Ex', Ey', Hz', vx', vy'] (parity 1)
  double* fS2[2] = {};
  T* cErms = nullptr;
  T* fErms[2] = {};          // [set]
  int cur = 0, fpar = 0;
  // the fine arrays hold the result of sub-steps for the current rectangle, so
  // the coarse E under it is their mean (false at start and after growth)
  bool rvalid = false;
  T *f_ntmp = nullptr, *f_D = nullptr, *f_nu = nullptr;
  T *ckx_c = nullptr, *skx_c = nullptr, *ckx_f = nullptr, *skx_f = nullptr;
  T* ph[4] = {};             // sin, cos of w t per step of a period: coarse, fine
  uint8_t* mask = nullptr;
  T* psi[2][4] = {};         // CPML psi by parity: Hz (x, y), Ex (y), Ey (x)
  T* pmlc[8] = {};           // CPML b, c: x cells, y cells, x nodes, y nodes
  double* part[4] = {};
  dmr::Ctl* ctl = nullptr;
  double* view = nullptr;
  int nblk_f_cur = 0;

  template <class P>
  P* at(size_t off) { return reinterpret_cast<P*>(ws + off); }

  // ---- persistent period -------------------------------------------------
  std::vector<dmr::EmArgs<T>> ptab_h;   // launch arguments [parity][phase] of the prepared period
  dmr::PerSched psched{};
  int pgrid = 0;
  size_t psmem = 0;

  bool persist_on() const { return persist && cfg.r <= dmr::kMaxR; }

  // node rows per warp as em_rows constrains them: a multiple of rr (the
  // strips of the last fine sub-step align with the coarse cells), or one
  // row when rr divides the warps of a block
  static int rows_for(int rows, int rr) {
    rows = std::max(1, std::min(rows, 64));
    if (rr > 1) {
      if (rows == 1 && dmr::EM_WARPS % rr == 0) return 1;
      rows = (rows + rr - 1) / rr * rr;
      return std::min(rows, 64 - 64 % rr);
    }
    return rows;
  }
  static void set_rows(dmr::EmArgs<T>* A, int rows, int rr) {
    A->rows = rows_for(rows, rr);
    const int sy = (A->m.ny + 1 + A->rows - 1) / A->rows;
    A->nblk = A->gx * ((sy + dmr::EM_WARPS - 1) / dmr::EM_WARPS);
  }

  // Arguments, unit counts and grid of the persistent period starting at
  // coarse level m0 (a period boundary); the tables go to the workspace on
  // the stream.  Rows per warp: as set, else one row for the fine units and
  // the fewest coarse rows that leave one unit of a step per resident block.
  int prep_period(int64_t m0) {
    const int NT = cfg.steps_per_period, r = cfg.r;
    const bool fine = has_fine;
    const int nph = fine ? r + 1 : 1;
    const bool pml = d.boundary == 1;
    psmem = 2 * (size_t)nph * sizeof(dmr::EmArgs<T>);
    int bpsm = 0;
    cudaError_t e = pml ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, dmr::k_period<T, true>,
                                                                       32 * dmr::EM_WARPS, psmem)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, dmr::k_period<T, false>,
                                                                       32 * dmr::EM_WARPS, psmem);
    if (e != cudaSuccess) return ck(e, "persistent period occupancy");
    if (bpsm < 1) return fail(DMR_ECUDA, "the persistent period kernel does not fit on an SM");
    const long long G = (long long)bpsm * num_sms;
    ptab_h.assign(2 * (size_t)nph, dmr::EmArgs<T>{});
    for (int par = 0; par < 2; ++par) {
      const int cp = cpar ^ par;
      const int f0 = (fpar + par * r) & 1;   // fine parity at the start of coarse step m0 + par
      dmr::EmArgs<T> Ac, Af;
      em_args_for(1, m0 + par, cp, f0, rvalid, &Ac, fine ? &Af : nullptr);
      ptab_h[par * nph] = Ac;
      if (fine) {
        ptab_h[par * nph + 1] = Af;
        for (int k = 2; k <= r; ++k) {
          em_args_for(k, m0 + par, cp, (f0 + k - 1) & 1, rvalid, nullptr, &Af);
          ptab_h[par * nph + k] = Af;
        }
      }
    }
    auto units = [&](int rc, int rf) {
      dmr::EmArgs<T> a = ptab_h[0];
      set_rows(&a, rc, 1);
      long long n = a.nblk;
      for (int k = 1; k < nph; ++k) {
        a = ptab_h[k];
        set_rows(&a, rf, k == r ? r : 1);
        n += a.nblk + a.ncfb;
      }
      return n;
    };
    static const int cand[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
    int rc = prow_c, rf = prow_f > 0 ? prow_f : 1;
    if (rc <= 0) {
      rc = 64;
      for (int t : cand)
        if (units(t, rf) <= G) { rc = t; break; }
      if (units(rc, rf) > G && prow_f <= 0) {
        rc = rf = 64;
        for (int t : cand)
          if (units(t, t) <= G) { rc = rf = t; break; }
      }
    }
    for (int par = 0; par < 2; ++par) {
      set_rows(&ptab_h[par * nph], rc, 1);
      for (int k = 1; k < nph; ++k) set_rows(&ptab_h[par * nph + k], rf, k == r ? r : 1);
    }
    if (fine && d.coupling == 0) {
      // the coarse step leaves the edges the last fine sub-step restricts (a8)
      for (int par = 0; par < 2; ++par) {
        dmr::RestrW<T>& Wc = ptab_h[par * nph].W;
        Wc = ptab_h[par * nph + r].W;
        Wc.on = 0;
        Wc.skip = 1;
      }
    }
    dmr::PerSched S{};
    unsigned* sw = at<unsigned>(L.off_sched);
    S.cnt = sw;
    S.rnq = sw + kSchedCnt;
    S.flag = sw + kSchedCnt + NT;
    S.ctl = ctl;
    S.m0 = m0;
    S.limit = sched_limit;
    S.NT = NT;
    S.r = fine ? r : 1;
    const dmr::EmArgs<T>& Ac = ptab_h[0];
    S.nC = Ac.nblk;
    S.gxC = Ac.gx;
    S.nyC = Ac.nblk / Ac.gx;
    S.rowsC = Ac.rows;
    S.swC = Ac.sw;
    if (S.nC + kSchedCnt + NT > L.nsched) return fail(DMR_ECAPACITY, "persistent period: too many coarse units");
    long long nU = S.nC, nFt = 0;
    for (int k = 1; k < nph; ++k) {
      S.nF[k] = ptab_h[k].nblk + ptab_h[k].ncfb;
      nFt += S.nF[k];
    }
    nU += nFt;
    S.nFt = (int)nFt;
    if (nU > (1ll << 30)) return fail(DMR_ECAPACITY, "persistent period: too many units");
    S.nU = (int)nU;
    constexpr int kMargin = 3;   // coarse cells around the rectangle read or written by the fine steps
    S.rn[0] = rect[0] - kMargin; S.rn[1] = rect[1] - kMargin;
    S.rn[2] = rect[2] + kMargin; S.rn[3] = rect[3] + kMargin;
    S.nRN = 0;
    if (fine)
      for (int u = 0; u < S.nC; ++u) {
        const int bx = u % S.gxC, by = u / S.gxC;
        const int i0 = bx * S.swC - 1, i1 = bx * S.swC + S.swC;
        const int j0 = by * dmr::EM_WARPS * S.rowsC - 1, j1 = (by + 1) * dmr::EM_WARPS * S.rowsC;
        if (i1 >= S.rn[0] && i0 <= S.rn[2] && j1 >= S.rn[1] && j0 <= S.rn[3]) ++S.nRN;
      }
    S.stall = sched_stall;
    psched = S;
    pgrid = (int)std::min<long long>(nU, G);
    return ck(cudaMemcpyAsync(at<char>(L.off_ptab), ptab_h.data(), psmem, cudaMemcpyHostToDevice, st),
              "upload persistent period arguments");
  }

  // the prepared persistent period: one cooperative launch (every block resident)
  int go_period() {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)pgrid);
    lc.blockDim = dim3(32 * dmr::EM_WARPS);
    lc.dynamicSmemBytes = psmem;
    lc.stream = st;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeCooperative;
    la[0].val.cooperative = 1;
    lc.attrs = la;
    lc.numAttrs = 1;
    const dmr::EmArgs<T>* tab = at<dmr::EmArgs<T>>(L.off_ptab);
    // algorithmic bytes of the period's EM steps, as the per-step launches count them
    const int NT = cfg.steps_per_period, r = cfg.r;
    const double cn = (double)(C.nx + 1) * (C.ny + 1);
    double units = em_bytes(cn, true) * (NT - 1) + em_bytes(cn, false);
    if (has_fine) {
      const double fn = (double)(F[cur].nx + 1) * (F[cur].ny + 1);
      units += em_bytes(fn, true) * ((double)r * NT - 1) + em_bytes(fn, false) +
               (double)NT * 2.0 * (double)L.es * (rect[2] - rect[0] + 1) * (rect[3] - rect[1] + 1);
    }
    int h = tbeg(5, units);
    cudaError_t e = d.boundary == 1 ? cudaLaunchKernelEx(&lc, dmr::k_period<T, true>, tab, psched)
                                    : cudaLaunchKernelEx(&lc, dmr::k_period<T, false>, tab, psched);
    tend(h);
    counted(1);
    return ck(e, "persistent period launch");
  }

  // host state after a persistent period (the parities N_T coarse steps and
  // r N_T fine sub-steps leave)
  void after_period() {
    const int NT = cfg.steps_per_period;
    if (NT & 1) flip_coarse();
    if (has_fine && (((int64_t)cfg.r * NT) & 1)) flip_fine();
    if (has_fine) rvalid = true;
  }

  int init() override {
    for (int q = 0; q < 5; ++q) { cE[0][q] = at<T>(L.off_c[q]); cE[1][q] = at<T>(L.off_c[9 + q]); }
    C.Ex = cE[0][0]; C.Ey = cE[0][1]; C.Hz = cE[0][2]; C.vx = cE[0][3]; C.vy = cE[0][4];
    C.n = at<T>(L.off_c[5]);
    c_ntmp = at<T>(L.off_c[6]); c_D = at<T>(L.off_c[7]); c_nu = at<T>(L.off_c[8]);
    C.S2 = at<double>(L.off_cS2);
    C.nx = cfg.nx; C.ny = cfg.ny; C.p = L.pc;
    cErms = at<T>(L.off_cErms);
    if (cfg.r > 1) {
      for (int s = 0; s < 2; ++s) {
        for (int q = 0; q < 6; ++q) fptr[s][q] = at<T>(L.off_f[s][q]);
        for (int q = 0; q < 5; ++q) fE1[s][q] = at<T>(L.off_f[s][6 + q]);
        fS2[s] = at<double>(L.off_fS2[s]);
        fErms[s] = at<T>(L.off_fErms[s]);
      }
      f_ntmp = at<T>(L.off_ftmp[0]); f_D = at<T>(L.off_ftmp[1]); f_nu = at<T>(L.off_ftmp[2]);
    }
    ckx_c = at<T>(L.off_tab[0]); skx_c = at<T>(L.off_tab[1]);
    ckx_f = at<T>(L.off_tab[2]); skx_f = at<T>(L.off_tab[3]);
    for (int q = 0; q < 4; ++q) ph[q] = at<T>(L.off_ph[q]);
    mask = at<uint8_t>(L.off_mask);
    if (d.boundary == 1) {
      for (int q = 0; q < 4; ++q) { psi[0][q] = at<T>(L.off_psi[q]); psi[1][q] = at<T>(L.off_psi[4 + q]); }
      for (int q = 0; q < 8; ++q) pmlc[q] = at<T>(L.off_pmlc[q]);
    }
    for (int q = 0; q < 4; ++q) part[q] = at<double>(L.off_part[q]);
    ctl = at<dmr::Ctl>(L.off_ctl);
    view = at<double>(L.off_view);
    int s = ck(cudaMemsetAsync(ws, 0, L.total, st), "cudaMemsetAsync(workspace)");
    if (s) return s;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      int v = 0;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) num_sms = v;
    }
    // incident-wave column tables: cos(k x), sin(k x) at the node columns
    std::vector<T> tc(cfg.nx + 1), ts(cfg.nx + 1);
    for (int g = 0; g <= cfg.nx; ++g) {
      double x = (double)g * d.dxc;
      tc[g] = (T)std::cos(d.k * x);
      ts[g] = (T)std::sin(d.k * x);
    }
    if ((s = ck(cudaMemcpyAsync(ckx_c, tc.data(), tc.size() * sizeof(T), cudaMemcpyHostToDevice, st), "upload tables"))) return s;
    if ((s = ck(cudaMemcpyAsync(skx_c, ts.data(), ts.size() * sizeof(T), cudaMemcpyHostToDevice, st), "upload tables"))) return s;
    const int nf = cfg.r * cfg.nx;
    std::vector<T> fc(nf + 1), fs(nf + 1);
    for (int g = 0; g <= nf; ++g) {
      double x = (double)g * d.dxf;
      fc[g] = (T)std::cos(d.k * x);
      fs[g] = (T)std::sin(d.k * x);
    }
    if ((s = ck(cudaMemcpyAsync(ckx_f, fc.data(), fc.size() * sizeof(T), cudaMemcpyHostToDevice, st), "upload tables"))) return s;
    if ((s = ck(cudaMemcpyAsync(skx_f, fs.data(), fs.size() * sizeof(T), cudaMemcpyHostToDevice, st), "upload tables"))) return s;
    // phase tables: the sin / cos that make_step evaluates for each step of a period
    for (int rr = 1; rr <= (cfg.r > 1 ? 2 : 1); ++rr) {
      const int mr = rr == 1 ? 1 : cfg.r;
      const int64_t N = (int64_t)mr * cfg.steps_per_period;
      std::vector<T> ps(N), pcv(N);
      for (int64_t q = 0; q < N; ++q) {
        const double phase = 2.0 * PI * (double)q / (double)N;
        ps[q] = (T)std::sin(phase);
        pcv[q] = (T)std::cos(phase);
      }
      T* dsn = ph[rr == 1 ? 0 : 2];
      T* dcs = ph[rr == 1 ? 1 : 3];
      if ((s = ck(cudaMemcpyAsync(dsn, ps.data(), N * sizeof(T), cudaMemcpyHostToDevice, st), "upload phases"))) return s;
      if ((s = ck(cudaMemcpyAsync(dcs, pcv.data(), N * sizeof(T), cudaMemcpyHostToDevice, st), "upload phases"))) return s;
    }
    if (d.boundary == 1) {
      // CPML coefficients (the oracle's formula): sigma = smax (depth/L)^3,
      // b = exp(-sigma dt / eps0), c = b - 1
      const double smax = 0.8 * 4.0 / (std::sqrt(MU0 / EPS0) * d.dxc);
      const int Lc = d.pml;
      // n entries at positions q + shift (cell centres 0.5, nodes 0) of a
      // mesh extent cells long
      auto coef = [&](int n, double shift, int extent, T* bd, T* cd) -> int {
        std::vector<T> bv(n), cv(n);
        for (int q = 0; q < n; ++q) {
          const double pos = q + shift;
          const double dep = std::max(std::max(Lc - pos, pos - (extent - Lc)), 0.0) / Lc;
          const double bb = std::exp(-smax * dep * dep * dep * d.dtc / EPS0);
          bv[q] = (T)bb;
          cv[q] = (T)(bb - 1.0);
        }
        int e = ck(cudaMemcpyAsync(bd, bv.data(), n * sizeof(T), cudaMemcpyHostToDevice, st), "upload CPML");
        if (!e) e = ck(cudaMemcpyAsync(cd, cv.data(), n * sizeof(T), cudaMemcpyHostToDevice, st), "upload CPML");
        if (!e) e = ck(cudaStreamSynchronize(st), "CPML sync");
        return e;
      };
      if ((s = coef(cfg.nx, 0.5, cfg.nx, pmlc[0], pmlc[1]))) return s;
      if ((s = coef(cfg.ny, 0.5, cfg.ny, pmlc[2], pmlc[3]))) return s;
      if ((s = coef(cfg.nx + 1, 0.0, cfg.nx, pmlc[4], pmlc[5]))) return s;
      if ((s = coef(cfg.ny + 1, 0.0, cfg.ny, pmlc[6], pmlc[7]))) return s;
    }
    return ck(cudaStreamSynchronize(st), "init sync");
  }

  static dim3 nodes_grid(int nx, int ny) { return dim3((nx + 1 + BX - 1) / BX, (ny + 1 + BY - 1) / BY); }

  // node rows per warp of the strip EM kernel: enough warps to fill the GPU
  // (about 48 per SM); small meshes get 1-2 rows per warp so a launch costs
  // about one memory latency, large ones up to 64 (the warm-up row is 1/rows)
  int warps_per_sm = 48;     // strip-height policy (the batch autotuner may change it)
  int warps_per_sm_fine = 48;   // the same for the fine sub-steps after the first (own launches)
  int lanecols = 1;             // node columns per lane of the EM strips (2: em_strips2, FP32)
  // rows per warp of an EM launch over an nx x ny mesh with sw-column strips;
  // a multiple of rr, or 1 (the last fine sub-step sums Ey over the r rows of
  // a coarse row)
  int em_rows(int nx, int ny, int sw, int rr, int wps, bool cross_ok = true) const {
    const long long sx = (nx + 1 + sw - 1) / sw;
    const long long target = (long long)num_sms * wps;
    long long rows = (sx * (ny + 1) + target - 1) / target;
    rows = std::min<long long>(64, std::max<long long>(1, rows));
    // one row per warp stays one row when r divides the warps of a block
    // (the block's warps then sum Ey in groups of r, em_strips); not in a
    // batch, whose blocks each stage their segment's arguments first, so
    // halving the rows there doubles that work
    if (rr > 1 && rows == 1 && dmr::EM_WARPS % rr == 0 && !in_batch && cross_ok) return 1;
    rows = (rows + rr - 1) / rr * rr;
    return (int)std::min<long long>(rows, 64 - 64 % rr);
  }


  T* fineE(int set, int par, int q) const { return par ? fE1[set][q] : fptr[set][q]; }

  void flip_coarse() {
    cpar ^= 1;
    C.Ex = cE[cpar][0]; C.Ey = cE[cpar][1]; C.Hz = cE[cpar][2]; C.vx = cE[cpar][3]; C.vy = cE[cpar][4];
  }
  void flip_fine() {
    fpar ^= 1;
    F[cur].Ex = fineE(cur, fpar, 0); F[cur].Ey = fineE(cur, fpar, 1); F[cur].Hz = fineE(cur, fpar, 2);
    F[cur].vx = fineE(cur, fpar, 3); F[cur].vy = fineE(cur, fpar, 4);
  }

  dmr::Mesh<T> fine_view(int set, const int* rc) const {
    dmr::Mesh<T> f;
    f.Ex = fptr[set][0]; f.Ey = fptr[set][1]; f.Hz = fptr[set][2];
    f.vx = fptr[set][3]; f.vy = fptr[set][4]; f.n = fptr[set][5]; f.S2 = fS2[set];
    f.nx = cfg.r * (rc[2] - rc[0]);
    f.ny = cfg.r * (rc[3] - rc[1]);
    f.p = (int)fine_pitch(f.nx);
    return f;
  }

  bool side_on_edge(int sd) const {
    switch (sd) {
      case dmr::SIDE_LEFT: return rect[0] == 0;
      case dmr::SIDE_RIGHT: return rect[2] == cfg.nx;
      case dmr::SIDE_BOTTOM: return rect[1] == 0;
      default: return rect[3] == cfg.ny;
    }
  }

  dmr::Step<T> make_step(int rr, int64_t level, bool accum) const {
    const double dx = d.lam / ((double)rr * (double)cfg.n_lambda);
    const double dt = 1.0 / (cfg.freq * (double)((int64_t)rr * cfg.steps_per_period));
    const double h = 0.5 * d.nu_m * dt;
    dmr::Step<T> s;
    s.ch = (T)(dt / (MU0 * dx));
    s.ce = (T)(dt / (EPS0 * dx));
    s.cj = (T)(dt * QE / (2.0 * EPS0));
    s.va = (T)((1.0 - h) / (1.0 + h));
    s.vb = (T)((QE * dt / ME) / (1.0 + h));
    s.mur = (T)((C0 * dt - dx) / (C0 * dt + dx));
    const int64_t N = (int64_t)rr * cfg.steps_per_period;
    const double phase = 2.0 * PI * (double)(level % N) / (double)N;
    s.E0 = (T)cfg.E0;
    s.sphi = (T)std::sin(phase);
    s.cphi = (T)std::cos(phase);
    if (rr == 1) { s.ckx = ckx_c; s.skx = skx_c; }
    else { s.ckx = ckx_f + (size_t)rr * rect[0]; s.skx = skx_f + (size_t)rr * rect[0]; }
    s.accum = accum ? 1 : 0;
    return s;
  }

  dmr::Dens make_dens(int rr) const {
    dmr::Dens q;
    q.N = (double)((int64_t)rr * cfg.steps_per_period);
    const double w = d.omega / d.nu_m;
    q.g = 1.0 + w * w;
    q.hp = 100.0 * cfg.p_torr;
    q.A = d.nu_model == 1 ? d.nu_scale * d.town_A * cfg.p_torr : d.nu_scale * 5.14e11 * cfg.p_torr;
    q.model = d.nu_model;
    q.tBp = d.town_B * cfg.p_torr;
    q.mu_e = QE / (ME * d.nu_m);
    q.nu_m = d.nu_m; q.nu_a = d.nu_a; q.De = d.De; q.Da = d.Da;
    q.wp2c = QE * QE / (ME * EPS0);
    q.heat = QE * QE / (ME * d.nu_m);
    q.T = d.T;
    const double dx = rr == 1 ? d.dxc : d.dxf;
    q.dx2 = dx * dx;
    q.r_ei = d.r_ei;
    q.invN = 1.0 / q.N;
    q.invg = 1.0 / q.g;
    q.inv_hp = 1.0 / q.hp;
    return q;
  }

  int launched(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DMR_ECUDA, fmt("launch %s: %s", what, cudaGetErrorString(e)));
    return DMR_OK;
  }

  // rows / columns of the fine->coarse E transfer (a8)
  void restr_bounds(int* jlo, int* jhi, int* ilo, int* ihi) const {
    *jlo = side_on_edge(dmr::SIDE_BOTTOM) ? rect[1] : rect[1] + 1;
    *jhi = side_on_edge(dmr::SIDE_TOP) ? rect[3] : rect[3] - 1;
    *ilo = side_on_edge(dmr::SIDE_LEFT) ? rect[0] : rect[0] + 1;
    *ihi = side_on_edge(dmr::SIDE_RIGHT) ? rect[2] : rect[2] - 1;
  }

  // algorithmic bytes of one fused EM launch over `pts` grid points: Ex, Ey,
  // Hz, vx, vy read and written, n read, S2 (fp64) read and written if summed
  double em_bytes(double pts, bool accum) const {
    return pts * (11.0 * (double)L.es + (accum ? 16.0 : 0.0));
  }

  // An EM launch that directly follows another EM launch on the stream may
  // start (as a programmatic dependent launch) while that one finishes: its
  // kernel waits for it before touching memory (pdl_enter).  Not used after
  // any other stream operation, nor while per-kernel events are recorded.
  template <class... P, class... A>
  void launch_em_kernel(void (*kern)(P...), int nb, bool pdl, A&&... args) const {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(nb);
    lc.blockDim = dim3(32 * dmr::EM_WARPS);
    lc.dynamicSmemBytes = 0;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = pdl ? at : nullptr;
    lc.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&lc, kern, std::forward<A>(args)...);
  }
  // coarse EM launches compile the CPML terms in only for CPML runs
  void go_em(int nb, const dmr::EmArgs<T>& A, bool pdl = false) const {
    if constexpr (sizeof(T) == 4) {
      if (A.lw == 2) {
        if (A.W.on && A.W.r == 2) launch_em_kernel(dmr::k_em_w2<true, 2>, nb, pdl, A);
        else if (A.W.on) launch_em_kernel(dmr::k_em_w2<true, 4>, nb, pdl, A);
        else launch_em_kernel(dmr::k_em_w2<false, 0>, nb, pdl, A);
        return;
      }
    }
    if (A.pml.on) launch_em_kernel(dmr::k_em<T, true>, nb, pdl, A);
    else if (A.W.on && A.W.r == 2) launch_em_kernel(dmr::k_em<T, false, true, 2>, nb, pdl, A);
    else if (A.W.on && A.W.r == 4) launch_em_kernel(dmr::k_em<T, false, true, 4>, nb, pdl, A);
    else if (A.W.on) launch_em_kernel(dmr::k_em<T, false, true>, nb, pdl, A);
    else launch_em_kernel(dmr::k_em<T, false>, nb, pdl, A);
  }
  void go_em2(int nb, const dmr::EmArgs<T>& A0, const dmr::EmArgs<T>& A1, bool pdl = false) const {
    if (A0.pml.on) launch_em_kernel(dmr::k_em2<T, true>, nb, pdl, A0, A1);
    else launch_em_kernel(dmr::k_em2<T, false>, nb, pdl, A0, A1);
  }

  // rr: strips of a multiple of rr columns and rows per warp a multiple of rr
  // (the last fine sub-step of a coarse step, which writes the a8 means); 1
  // otherwise
  dmr::EmArgs<T> em_args(const dmr::Mesh<T>& src, T* const* dst, const dmr::Step<T>& c,
                         const dmr::Bnd<T>& b, int rr = 1, int wps = 0, bool w2_ok = false) const {
    dmr::EmArgs<T> A;
    A.m = src;
    A.dEx = dst[0]; A.dEy = dst[1]; A.dHz = dst[2]; A.dvx = dst[3]; A.dvy = dst[4];
    A.c = c; A.b = b;
    A.pml = dmr::Pml<T>{};
    A.W = dmr::RestrW<T>{};
    // two node columns per lane where the run asks for them: the fine
    // sub-steps with launches of their own (w2_ok) in FP32 runs without CPML,
    // not in a batch or a persistent period; the last one at r = 2 or 4 only,
    // with rows per warp a multiple of r
    const bool w2 = w2_ok && lanecols == 2 && sizeof(T) == 4 && !in_batch && !persist_on() &&
                    d.boundary != 1 && (rr == 1 || rr == 2 || rr == 4);
    A.lw = w2 ? 2 : 1;
    A.sw = w2 ? dmr::STRIP_W2 - dmr::STRIP_W2 % rr : dmr::STRIP_W - dmr::STRIP_W % rr;
    A.rows = em_rows(src.nx, src.ny, A.sw, rr, wps > 0 ? wps : warps_per_sm, !w2);
    A.gx = (src.nx + 1 + A.sw - 1) / A.sw;
    const int sy = (src.ny + 1 + A.rows - 1) / A.rows;
    A.nblk = A.gx * ((sy + dmr::EM_WARPS - 1) / dmr::EM_WARPS);
    A.ncfb = 0;   // blocks per coarse-fine side (em_cfb)
    for (int q = 0; q < 4; ++q)
      if (b.mode[q] == dmr::BC_CFB) {
        const int len = (q == dmr::SIDE_BOTTOM || q == dmr::SIDE_TOP) ? src.nx : src.ny;
        A.ncfb += (len + 32 * dmr::EM_WARPS - 1) / (32 * dmr::EM_WARPS);
      }
    return A;
  }

  // Arguments of the EM launches of coarse step mlev: the coarse step (Ac,
  // phase k = 1 only) and fine sub-step k (Af), for coarse buffer parity cp,
  // fine parity fp at the start of sub-step k, restriction state rv.
  void em_args_for(int k, int64_t mlev, int cp, int fp, bool rv, dmr::EmArgs<T>* Ac,
                   dmr::EmArgs<T>* Af) const {
    const int NT = cfg.steps_per_period, r = cfg.r;
    dmr::Step<T> sc = make_step(1, mlev, (mlev % NT) != 0);
    dmr::Mesh<T> src = C;
    src.Ex = cE[cp][0]; src.Ey = cE[cp][1]; src.Hz = cE[cp][2]; src.vx = cE[cp][3]; src.vy = cE[cp][4];
    T* const* cdst = cE[cp ^ 1];
    // the coarse arrays already hold the fine->coarse mean under the rectangle
    // (written by the last fine sub-step of the previous coarse step, a8), so
    // the coarse step reads plain arrays
    (void)rv;
    const dmr::Mesh<T> fsrc = fine_at(fp);
    if (Ac) {
      dmr::Bnd<T> bc{};
      for (int q = 0; q < 4; ++q) bc.mode[q] = d.boundary == 1 ? dmr::BC_PEC : dmr::BC_MUR;
      bc.r = 1;
      *Ac = em_args(src, cdst, sc, bc);
      Ac->kind = 0; Ac->N = NT; Ac->r = 1; Ac->ps = ph[0]; Ac->pc = ph[1];
      if (d.boundary == 1) {
        dmr::Pml<T>& P = Ac->pml;
        P.on = 1;
        P.L = d.pml;
        P.hx = psi[cp][0]; P.hy = psi[cp][1]; P.exy = psi[cp][2]; P.eyx = psi[cp][3];
        P.dhx = psi[cp ^ 1][0]; P.dhy = psi[cp ^ 1][1]; P.dexy = psi[cp ^ 1][2]; P.deyx = psi[cp ^ 1][3];
        P.bxh = pmlc[0]; P.cxh = pmlc[1]; P.byh = pmlc[2]; P.cyh = pmlc[3];
        P.bxn = pmlc[4]; P.cxn = pmlc[5]; P.byn = pmlc[6]; P.cyn = pmlc[7];
      }
    }
    if (!Af || !has_fine) return;
    dmr::Bnd<T> bf{};
    bf.r = r;
    for (int q = 0; q < 4; ++q) {
      if (side_on_edge(q)) { bf.mode[q] = dmr::BC_MUR; continue; }
      bf.mode[q] = dmr::BC_CFB;
      if (q == dmr::SIDE_BOTTOM || q == dmr::SIDE_TOP) {
        bf.at[q] = q == dmr::SIDE_BOTTOM ? rect[1] : rect[3];
        const size_t off = (size_t)bf.at[q] * C.p;
        bf.old_line[q] = src.Ex + off;
        bf.new_line[q] = cdst[0] + off;
        bf.stride[q] = 1;
        bf.len[q] = cfg.nx;
        bf.start[q] = rect[0];
      } else {
        bf.at[q] = q == dmr::SIDE_LEFT ? rect[0] : rect[2];
        const size_t off = (size_t)bf.at[q];
        bf.old_line[q] = src.Ey + off;
        bf.new_line[q] = cdst[1] + off;
        bf.stride[q] = C.p;
        bf.len[q] = cfg.ny;
        bf.start[q] = rect[1];
      }
    }
    bf.cm = src;
    bf.cc = sc;
    bf.cps = ph[0]; bf.cpc = ph[1]; bf.cN = NT;
    const int64_t mf = (int64_t)r * mlev + (k - 1);
    dmr::Step<T> sf = make_step(r, mf, (mf % ((int64_t)r * NT)) != 0);
    bf.frac = (T)((double)k / (double)r);
    bf.recompute = k == 1 ? 1 : 0;
    T* fdst[5] = {fineE(cur, fp ^ 1, 0), fineE(cur, fp ^ 1, 1), fineE(cur, fp ^ 1, 2),
                  fineE(cur, fp ^ 1, 3), fineE(cur, fp ^ 1, 4)};
    // the last sub-step's strips align with the coarse cells (a8 column groups and row sums)
    // sub-steps after the first run alone, with their own strip height
    *Af = em_args(fsrc, fdst, sf, bf, k == r ? r : 1, k > 1 ? warps_per_sm_fine : warps_per_sm, k > 1);
    Af->kind = 1; Af->N = r * NT; Af->r = r; Af->ps = ph[2]; Af->pc = ph[3];
    if (k == r && d.coupling == 0) {
      // a8: the last sub-step writes the mean of r collinear fine edges into
      // the coarse E^{n+1} (the coarse step's output buffer)
      dmr::RestrW<T>& W = Af->W;
      W.on = 1;
      W.cEx = cdst[0]; W.cEy = cdst[1]; W.cp = C.p;
      W.I0 = rect[0]; W.J0 = rect[1]; W.I1 = rect[2]; W.J1 = rect[3]; W.r = r;
      restr_bounds(&W.jlo, &W.jhi, &W.ilo, &W.ihi);
      W.rinv = (T)(1.0 / (double)r);
    }
  }

  // fine mesh view with E/H/v of parity fp
  dmr::Mesh<T> fine_at(int fp) const {
    dmr::Mesh<T> f = F[cur];
    f.Ex = fineE(cur, fp, 0); f.Ey = fineE(cur, fp, 1); f.Hz = fineE(cur, fp, 2);
    f.vx = fineE(cur, fp, 3); f.vy = fineE(cur, fp, 4);
    return f;
  }

  // true right after an EM launch on the stream (nothing else in between)
  bool last_em = false;
  // FP32 only: measured on the 512^2 run, programmatic launches take the
  // FP32 period from 0.598 to 0.585 ms but the FP64 one from 2.49 to 3.35 ms
  bool pdl_next() const { return last_em && !timing && sizeof(T) == 4; }

  // one coarse step from level mlev.  The coarse step (reading the coarse E,
  // which under the rectangle holds the fine mean the previous step's last
  // sub-step wrote) and the first fine sub-step (which evaluates the coarse
  // E^{n+1} on its boundary lines itself) are independent and share one
  // launch; fine sub-steps 2..r follow, the last writing the new fine mean
  // into the coarse E^{n+1}.
  int launch_coarse_step(int64_t mlev) {
    const int NT = cfg.steps_per_period, r = cfg.r;
    const bool acc_c = (mlev % NT) != 0;
    dmr::EmArgs<T> Ac, Af;
    em_args_for(1, mlev, cpar, fpar, rvalid, &Ac, has_fine ? &Af : nullptr);
    const double cbytes = em_bytes((double)(C.nx + 1) * (C.ny + 1), acc_c);
    if (!has_fine) {
      int h = tbeg(0, cbytes);
      go_em(Ac.nblk + Ac.ncfb, Ac, pdl_next());
      tend(h);
      last_em = true;
      counted(1);
      flip_coarse();
      return launched("coarse EM");
    }
    const int cp0 = cpar;
    const double fn = (double)(F[cur].nx + 1) * (F[cur].ny + 1);
    for (int k = 1; k <= r; ++k) {
      const int64_t mf = (int64_t)r * mlev + (k - 1);
      const bool acc_f = (mf % ((int64_t)r * NT)) != 0;
      if (k > 1) em_args_for(k, mlev, cp0, fpar, rvalid, nullptr, &Af);
      if (k == 1) {
        int h = tbeg(0, cbytes + em_bytes(fn, acc_f));
        go_em2(Ac.nblk + Ac.ncfb + Af.nblk + Af.ncfb, Ac, Af, pdl_next());
        tend(h);
        flip_coarse();
      } else {
        // the last sub-step also writes the coarse E means under the rectangle (a8)
        const double wb = k == r ? 2.0 * (double)L.es * (rect[2] - rect[0] + 1) * (rect[3] - rect[1] + 1) : 0.0;
        int h = tbeg(1, em_bytes(fn, acc_f) + wb);
        go_em(Af.nblk + Af.ncfb, Af, pdl_next());
        tend(h);
      }
      last_em = true;
      counted(1);
      flip_fine();
    }
    rvalid = true;
    return launched("EM step");
  }

  // continuity step, totals and flags at the end of a period (coarse level
  // mlev): three launches over the coarse mesh's and the fine rectangle's
  // node tiles (rates, new density, commit with flags and FP64 totals)
  int launch_period_end(int64_t mlev) {
    const int r = cfg.r;
    last_em = false;
    int h = tbeg(3, 0.0);
    dmr::PeArgs<T> A{};
    const dim3 gc = nodes_grid(C.nx, C.ny);
    A.C.m = C;
    A.C.c = make_step(1, mlev, true);
    A.C.d = make_dens(1);
    A.C.w = dmr::Wts{cfg.nx, cfg.ny, has_fine ? 1 : 0, rect[0], rect[1], rect[2], rect[3]};
    A.C.D = c_D; A.C.nu = c_nu; A.C.ntmp = c_ntmp; A.C.erms = cErms;
    A.C.partP = part[0]; A.C.partN = part[2];
    A.C.gx = (int)gc.x; A.C.nb = (int)(gc.x * gc.y);
    A.F.nb = 0;
    A.F.partP = part[1]; A.F.partN = part[3];
    A.r = r;
    A.rect = make_int4(rect[0], rect[1], rect[2], rect[3]);
    A.ctl = ctl;
    A.mask = mask;
    A.dxc2 = d.dxc * d.dxc;
    A.dxf2 = d.dxf * d.dxf;
    A.period = d.T;
    A.sched = at<unsigned>(L.off_sched);
    A.nsched = L.nsched;
    if (has_fine) {
      const dmr::Mesh<T>& f = F[cur];
      const dim3 gf = nodes_grid(f.nx, f.ny);
      A.F.m = f;
      A.F.c = make_step(r, (int64_t)r * mlev, true);
      A.F.d = make_dens(r);
      A.F.w = dmr::Wts{f.nx, f.ny, 0, 0, 0, 0, 0};
      A.F.D = f_D; A.F.nu = f_nu; A.F.ntmp = f_ntmp; A.F.erms = fErms[cur];
      A.F.gx = (int)gf.x; A.F.nb = (int)(gf.x * gf.y);
      dmr::Dir<T>& dir = A.dir;
      dir.r = r;
      for (int q = 0; q < 4; ++q) {
        if (side_on_edge(q)) continue;
        dir.on[q] = 1;
        if (q == dmr::SIDE_BOTTOM || q == dmr::SIDE_TOP) {
          dir.at[q] = q == dmr::SIDE_BOTTOM ? rect[1] : rect[3];
          dir.len[q] = cfg.nx + 1;
          dir.start[q] = rect[0];
        } else {
          dir.at[q] = q == dmr::SIDE_LEFT ? rect[0] : rect[2];
          dir.len[q] = cfg.ny + 1;
          dir.start[q] = rect[1];
        }
      }
      A.n_th = (T)d.n_th;
      A.gs = (T)(1.0 / (2.0 * d.dxc * d.g_th));
    }
    const int nb = A.C.nb + A.F.nb;
    const dim3 blk(BX, BY);
    dmr::k_pe_rates<T><<<nb, blk, 0, st>>>(A);
    dmr::k_pe_density<T><<<nb, blk, 0, st>>>(A);
    dmr::k_pe_commit<T><<<nb, blk, 0, st>>>(A);
    tend(h);
    counted(3);
    return launched("period end");
  }

  // host side of the period end: read the control block, stability guard,
  // growth policy (or replay), expansion
  // pinned host copy of the control block (a copy into pageable memory is
  // staged through a driver buffer); host memory, allocated at first use
  dmr::Ctl* hctl = nullptr;
  ~Engine() override {
    if (hctl) cudaFreeHost(hctl);
  }
  int period_end_host(bool graph_ran = false) {
    if (!hctl)
      if (int s = ck(cudaHostAlloc(reinterpret_cast<void**>(&hctl), sizeof(dmr::Ctl), cudaHostAllocDefault),
                     "pinned control block")) { hctl = nullptr; return s; }
    if (int s = ck(cudaMemcpyAsync(hctl, ctl, sizeof(dmr::Ctl), cudaMemcpyDeviceToHost, st), "read control block")) return s;
    if (int s = ck(cudaStreamSynchronize(st), "period sync")) return s;
    const dmr::Ctl hc = *hctl;
    harvest_period(graph_ran);
    return period_decide(hc);
  }

  // stability guard and growth decision from a period's control block
  int period_decide(const dmr::Ctl& hc) {
    if (hc.err & dmr::kSchedErr) {
      dead = true;
      return fail(DMR_ETIMEOUT, "a bounded wait of the persistent period launch gave up; the period's "
                                "fields are lost (dmr_load_state restores a saved state)");
    }
    if (hc.err) return fail(DMR_EUNSTABLE, "NaN in the density or totals at a period end");
    const double wp_lim = (2.0 / (has_fine ? d.dtf : d.dtc));
    const double n_lim = wp_lim * wp_lim * ME * EPS0 / (QE * QE);
    if (hc.st[4] >= n_lim)
      return fail(DMR_EUNSTABLE, fmt("density %.3e reaches w_p dt >= 2", hc.st[4]));
    if (!has_fine) return DMR_OK;
    int nr[4] = {rect[0], rect[1], rect[2], rect[3]};
    if (!replay.empty()) {
      if (replay_pos * 4 + 3 < replay.size()) {
        for (int q = 0; q < 4; ++q) nr[q] = replay[replay_pos * 4 + q];
        ++replay_pos;
      }
    } else if (cfg.growth == 2) {
      // threshold lines (Sec. III.D): a hit side jumps out by m_ex / m_ey
      const int k = d.margin;   // CPML: the rectangle stays out of the layer
      if (hc.side & 1) nr[0] = std::max(rect[0] - d.m_ex, k);
      if (hc.side & 2) nr[1] = std::max(rect[1] - d.m_ey, k);
      if (hc.side & 4) nr[2] = std::min(rect[2] + d.m_ex, cfg.nx - k);
      if (hc.side & 8) nr[3] = std::min(rect[3] + d.m_ey, cfg.ny - k);
    } else if (cfg.growth == 1 && hc.nflag > 0) {
      const int b = cfg.buffer_cells;
      const int k = d.margin;
      const int c4[4] = {std::max(hc.bbox[0] - b, k), std::max(hc.bbox[1] - b, k),
                         std::min(hc.bbox[2] + b, cfg.nx - k), std::min(hc.bbox[3] + b, cfg.ny - k)};
      nr[0] = std::min(rect[0], c4[0]);
      nr[1] = std::min(rect[1], c4[1]);
      nr[2] = std::max(rect[2], c4[2]);
      nr[3] = std::max(rect[3], c4[3]);
    }
    if (nr[0] == rect[0] && nr[1] == rect[1] && nr[2] == rect[2] && nr[3] == rect[3]) return DMR_OK;
    return expand(nr);
  }

  int check_rect(const int* nr) {
    const int k = d.margin;
    if (!(k <= nr[0] && nr[0] < nr[2] && nr[2] <= cfg.nx - k && k <= nr[1] && nr[1] < nr[3] &&
          nr[3] <= cfg.ny - k))
      return fail(DMR_EINVAL, fmt("bad rectangle (%d,%d,%d,%d)%s", nr[0], nr[1], nr[2], nr[3],
                                  k ? " (it must stay out of the CPML layer)" : ""));
    if (has_fine && !(nr[0] <= rect[0] && nr[1] <= rect[1] && nr[2] >= rect[2] && nr[3] >= rect[3]))
      return fail(DMR_EINVAL, "the rectangle can only grow");
    const int64_t cells = (int64_t)cfg.r * (nr[2] - nr[0]) * (int64_t)cfg.r * (nr[3] - nr[1]);
    if (cells > d.cap)
      return fail(DMR_ECAPACITY, fmt("rectangle of %lld fine cells exceeds the capacity %lld",
                                     (long long)cells, (long long)d.cap));
    return DMR_OK;
  }

  int expand(const int* nr) {
    if (int s = check_rect(nr)) return s;
    const int nxt = has_fine ? 1 - cur : cur;
    dmr::Mesh<T> nf = fine_view(nxt, nr);
    if ((size_t)(nf.ny + 1) * nf.p > L.fplane) return fail(DMR_ECAPACITY, "fine arrays exceed the workspace");
    dmr::Mesh<T> of = has_fine ? F[cur] : nf;
    const int oI0 = has_fine ? rect[0] : nr[0], oJ0 = has_fine ? rect[1] : nr[1];
    int h = tbeg(4, 0.0);
    dmr::k_expand<T><<<nodes_grid(nf.nx, nf.ny), dim3(BX, BY), 0, st>>>(
        nf, of, C, nr[0], nr[1], oI0, oJ0, has_fine ? 1 : 0, cfg.r, fErms[nxt], fErms[cur], cErms);
    tend(h);
    counted(1);
    if (int s = launched("expand")) return s;
    cur = nxt;
    F[cur] = nf;
    fpar = 0;
    rvalid = false;
    for (int q = 0; q < 4; ++q) rect[q] = nr[q];
    has_fine = true;
    drop_graph();
    return DMR_OK;
  }

  int seed(double n0, double x0, double y0, double sx, double sy, int add) override {
    if (!(sx > 0) || !(sy > 0)) return fail(DMR_EINVAL, "seed widths must be > 0");
    const dim3 blk(BX, BY);
    dmr::k_seed<T><<<nodes_grid(C.nx, C.ny), blk, 0, st>>>(C, 0, 0, d.dxc, n0, x0, y0, sx, sy, add);
    counted(1);
    if (has_fine) {
      dmr::Mesh<T> f = F[cur];
      dmr::k_seed<T><<<nodes_grid(f.nx, f.ny), blk, 0, st>>>(f, cfg.r * rect[0], cfg.r * rect[1],
                                                             d.dxf, n0, x0, y0, sx, sy, add);
      inject();
      counted(1);
    }
    return launched("seed");
  }

  void inject() {
    const dim3 g((rect[2] - rect[0] + 1 + BX - 1) / BX, (rect[3] - rect[1] + 1 + BY - 1) / BY);
    dmr::k_inject<T><<<g, dim3(BX, BY), 0, st>>>(C, F[cur], rect[0], rect[1], rect[2], rect[3], cfg.r);
    counted(1);
  }

  int set_patch(const int32_t* r4) override {
    if (cfg.r == 1) return fail(DMR_ESTATE, "r = 1: a uniform mesh has no fine rectangle");
    if (m % cfg.steps_per_period != 0) return fail(DMR_ESTATE, "the rectangle changes only at a period boundary");
    int nr[4] = {r4[0], r4[1], r4[2], r4[3]};
    if (has_fine && nr[0] == rect[0] && nr[1] == rect[1] && nr[2] == rect[2] && nr[3] == rect[3]) return DMR_OK;
    return expand(nr);
  }

  int advance(int64_t n) override {
    if (n < 0) return fail(DMR_EINVAL, "negative step count");
    if (dead) return fail(DMR_ESTATE, "the run's fields were lost when a bounded wait gave up; load a saved state");
    const int NT = cfg.steps_per_period;
    last_em = false;   // other work may have been queued on the stream since
    while (n > 0) {
      if (graphs && m % NT == 0 && n >= NT) {
        // a graph holds the buffer parities it was captured with
        if (gexec && (g_cpar != cpar || g_fpar != fpar || g_rvalid != (int)rvalid)) drop_graph();
        if (!gexec) {
          if (int s = capture()) return s;
        }
        if (int s = ck(cudaGraphLaunch(gexec, st), "cudaGraphLaunch")) return s;
        last_em = false;
        launches += graph_nodes;
        m += NT;
        n -= NT;
        if (NT & 1) flip_coarse();
        if (has_fine && (((int64_t)cfg.r * NT) & 1)) flip_fine();
        if (has_fine) rvalid = true;
        if (int s = period_end_host(true)) return s;
        continue;
      }
      if (persist_on() && m % NT == 0 && n >= NT) {
        // one persistent launch for the period's EM steps, then the period end
        drop_graph();   // the argument tables of a captured period would change
        if (int s = prep_period(m)) return s;
        if (int s = go_period()) return s;
        last_em = false;
        m += NT;
        n -= NT;
        after_period();
        if (int s = launch_period_end(m)) return s;
        if (int s = period_end_host()) return s;
        continue;
      }
      if (int s = launch_coarse_step(m)) return s;
      ++m;
      --n;
      if (m % NT == 0) {
        if (int s = launch_period_end(m)) return s;
        if (int s = period_end_host()) return s;
      }
    }
    return DMR_OK;
  }

  int capture() {
    drop_graph();
    const int NT = cfg.steps_per_period;
    cudaGraph_t g = nullptr;
    const bool per = persist_on();
    if (per) {
      // the argument tables go to the workspace before the capture; the graph
      // launches read them on every replay
      if (int s = prep_period(m)) return s;
    }
    if (int s = ck(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture")) return s;
    capturing = true;
    graph_nodes = 0;
    // capturing advances the host-side buffer parities; put them back after
    const int c0 = cpar, f0 = fpar;
    const bool rv0 = rvalid;
    int s = DMR_OK;
    last_em = false;   // the graph's first launch follows the previous replay's copy
    if (per) {
      s = go_period();
      if (!s) after_period();
    } else {
      for (int q = 0; q < NT && !s; ++q) s = launch_coarse_step(m + q);
    }
    if (!s) s = launch_period_end(m + NT);
    capturing = false;
    if (cpar != c0) flip_coarse();
    if (has_fine && fpar != f0) flip_fine();
    rvalid = rv0;
    g_cpar = c0;
    g_fpar = f0;
    g_rvalid = (int)rv0;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (s) { if (g) cudaGraphDestroy(g); gpend.clear(); return s; }
    if (e != cudaSuccess) { gpend.clear(); return ck(e, "end capture"); }
    e = cudaGraphInstantiate(&gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { gexec = nullptr; gpend.clear(); return ck(e, "graph instantiate"); }
    return DMR_OK;
  }

  int dims(int field, int level, int* rows, int* cols, int* es) const {
    int nx, ny;
    if (level == 0) { nx = C.nx; ny = C.ny; }
    else if (level == 1 && has_fine) { nx = F[cur].nx; ny = F[cur].ny; }
    else return DMR_ESTATE;
    *es = (int)L.es;
    switch (field) {
      case DMR_FIELD_EX: case DMR_FIELD_VX: *rows = ny + 1; *cols = nx; break;
      case DMR_FIELD_EY: case DMR_FIELD_VY: *rows = ny; *cols = nx + 1; break;
      case DMR_FIELD_HZ: *rows = ny; *cols = nx; break;
      case DMR_FIELD_NE: case DMR_FIELD_ERMS: *rows = ny + 1; *cols = nx + 1; break;
      case DMR_FIELD_S2: *rows = ny + 1; *cols = nx + 1; *es = 8; break;
      case DMR_FIELD_MASK:
        if (level != 0 || cfg.r == 1) return DMR_ESTATE;
        *rows = ny + 1; *cols = nx + 1; *es = 1; break;
      default: return DMR_EINVAL;
    }
    return DMR_OK;
  }

  int shape(int field, int level, int32_t* s, int32_t* eb) const override {
    int rows, cols, es;
    int st_ = dims(field, level, &rows, &cols, &es);
    if (st_) return st_;
    s[0] = rows; s[1] = cols;
    if (eb) *eb = es;
    return DMR_OK;
  }

  void* field_ptr(int field, int level) {
    const dmr::Mesh<T>& mm = level == 0 ? C : F[cur];
    switch (field) {
      case DMR_FIELD_EX: return mm.Ex;
      case DMR_FIELD_EY: return mm.Ey;
      case DMR_FIELD_HZ: return mm.Hz;
      case DMR_FIELD_VX: return mm.vx;
      case DMR_FIELD_VY: return mm.vy;
      case DMR_FIELD_NE: return mm.n;
      case DMR_FIELD_S2: return mm.S2;
      case DMR_FIELD_ERMS: return level == 0 ? cErms : fErms[cur];
      default: return mask;
    }
  }

  int read(int field, int level, void* dst, size_t bytes, int dev) override {
    int rows, cols, es;
    if (int s = dims(field, level, &rows, &cols, &es)) return fail(s, "no such field / level");
    if (bytes < (size_t)rows * cols * es) return fail(DMR_ECAPACITY, "destination too small");
    const int p = field == DMR_FIELD_MASK ? cols : (level == 0 ? C.p : F[cur].p);
    const void* src = field_ptr(field, level);
    if (field == DMR_FIELD_S2 && m % cfg.steps_per_period != 0) {
      // S2 holds the levels before the current one; add the current level so
      // the result is the running sum through the present E level
      const int rr = level == 0 ? 1 : cfg.r;
      const int64_t lev = level == 0 ? m : (int64_t)cfg.r * m;
      dmr::Step<T> s = make_step(rr, lev, true);
      const dmr::Mesh<T>& mm = level == 0 ? C : F[cur];
      dmr::k_s2_view<T><<<nodes_grid(mm.nx, mm.ny), dim3(BX, BY), 0, st>>>(mm, s, view);
      counted(1);
      if (int e = launched("S2 view")) return e;
      src = view;
    }
    if (field == DMR_FIELD_ERMS && m % cfg.steps_per_period != 0) {
      // within a period: the RMS over the samples taken so far (the stored
      // array holds the last completed period's E_rms)
      const int rr = level == 0 ? 1 : cfg.r;
      const int64_t lev = level == 0 ? m : (int64_t)cfg.r * m;
      const int64_t q = lev % ((int64_t)rr * cfg.steps_per_period);
      dmr::Step<T> s = make_step(rr, lev, true);
      const dmr::Mesh<T>& mm = level == 0 ? C : F[cur];
      dmr::k_erms_view<T><<<nodes_grid(mm.nx, mm.ny), dim3(BX, BY), 0, st>>>(
          mm, s, (double)q, reinterpret_cast<T*>(view));
      counted(1);
      if (int e = launched("E_rms view")) return e;
      src = view;
    }
    const size_t wb = (size_t)cols * es;
    cudaError_t e = cudaMemcpy2DAsync(dst, wb, src, (size_t)p * es, wb, rows,
                                      dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    if (int s = ck(e, "cudaMemcpy2DAsync(read)")) return s;
    if (!dev) return ck(cudaStreamSynchronize(st), "read sync");
    return DMR_OK;
  }

  int write(int field, int level, const void* src, size_t bytes, int dev) override {
    if (field == DMR_FIELD_MASK || field == DMR_FIELD_ERMS)
      return fail(DMR_EINVAL, "the mask and E_rms are derived quantities, not writable");
    int rows, cols, es;
    if (int s = dims(field, level, &rows, &cols, &es)) return fail(s, "no such field / level");
    if (bytes < (size_t)rows * cols * es) return fail(DMR_ECAPACITY, "source too small");
    const int p = level == 0 ? C.p : F[cur].p;
    const size_t wb = (size_t)cols * es;
    cudaError_t e = cudaMemcpy2DAsync(field_ptr(field, level), (size_t)p * es, src, wb, wb, rows,
                                      dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (int s = ck(e, "cudaMemcpy2DAsync(write)")) return s;
    if (field == DMR_FIELD_NE && level == 1) inject();
    if (!dev) return ck(cudaStreamSynchronize(st), "write sync");
    return launched("write");
  }

  // ======================================================================
  // Adjoint (reverse mode) with the refinement schedule held fixed.
  // adj_record: advance n steps from a period boundary, keeping a full copy of
  // the workspace every K steps and the rectangle after every period.
  // adj_backward: for each segment in reverse order, restore its checkpoint,
  // recompute the segment with every step's E^l and v^{l+1/2} (and each
  // period's density, S2 and last-level E) written to a tape, then sweep the
  // tape backwards with the adjoint kernels of dmr_adjoint.cuh.
  // ======================================================================
  struct HostState {
    int64_t m;
    int cpar, fpar, cur;
    int rect[4];
    bool has_fine, rvalid;
    dmr::Mesh<T> C, F0, F1;
  };
  struct Rec {
    bool valid = false;
    int64_t m0 = 0, n = 0, K = 0;
    char* ckpt = nullptr;
    std::vector<HostState> ck;
    std::vector<int32_t> log;      // rectangle after each recorded period
  } rec;

  HostState save_host() const {
    HostState h;
    h.m = m; h.cpar = cpar; h.fpar = fpar; h.cur = cur;
    for (int q = 0; q < 4; ++q) h.rect[q] = rect[q];
    h.has_fine = has_fine; h.rvalid = rvalid;
    h.C = C; h.F0 = F[0]; h.F1 = F[1];
    return h;
  }
  void load_host(const HostState& h) {
    m = h.m; cpar = h.cpar; fpar = h.fpar; cur = h.cur;
    for (int q = 0; q < 4; ++q) rect[q] = h.rect[q];
    has_fine = h.has_fine; rvalid = h.rvalid;
    C = h.C; F[0] = h.F0; F[1] = h.F1;
  }
  size_t wbytes() const { return up(L.total, 256); }

  size_t adj_ckpt_bytes(int64_t n, int64_t K) const override {
    if (K <= 0 || n <= 0) return 0;
    return (size_t)((n + K - 1) / K) * wbytes();
  }

  int adj_record(int64_t n, int64_t K, void* ckpt, size_t bytes) override {
    const int NT = cfg.steps_per_period;
    if (d.boundary != 0) return fail(DMR_EINVAL, "the adjoint needs the Mur boundary (boundary = 0)");
    if (n <= 0 || K <= 0 || n % NT || K % NT)
      return fail(DMR_EINVAL, "steps and checkpoint interval must be positive multiples of steps_per_period");
    if (m % NT) return fail(DMR_ESTATE, "recording starts at a period boundary");
    if (!ckpt || bytes < adj_ckpt_bytes(n, K)) return fail(DMR_ECAPACITY, "checkpoint buffer too small");
    rec = Rec();
    rec.m0 = m; rec.n = n; rec.K = K; rec.ckpt = (char*)ckpt;
    const std::vector<int32_t> user_replay = replay;
    const size_t user_pos = replay_pos;
    for (int64_t done = 0; done < n;) {
      rec.ck.push_back(save_host());
      if (int s = ck(cudaMemcpyAsync(rec.ckpt + (rec.ck.size() - 1) * wbytes(), ws, L.total,
                                     cudaMemcpyDeviceToDevice, st), "checkpoint")) return s;
      const int64_t seg = std::min<int64_t>(K, n - done);
      for (int64_t q = 0; q < seg; q += NT) {
        if (int s = advance(NT)) return s;
        for (int k = 0; k < 4; ++k) rec.log.push_back(has_fine ? rect[k] : -1);
      }
      done += seg;
    }
    replay = user_replay;
    replay_pos = user_pos;
    rec.valid = true;
    return ck(cudaStreamSynchronize(st), "record sync");
  }

  // fine dims (cells, pitch) of a rectangle
  void fdims(const int* rc, int* nx, int* ny, int* p) const {
    *nx = cfg.r * (rc[2] - rc[0]);
    *ny = cfg.r * (rc[3] - rc[1]);
    *p = (int)fine_pitch(*nx);
  }
  size_t fplane_b(const int* rc) const {
    int nx, ny, p;
    fdims(rc, &nx, &ny, &p);
    return (size_t)(ny + 1) * p * L.es;
  }
  size_t cplane_b() const { return L.cplane * L.es; }

  // tape bytes of one recorded segment starting at period index p0
  size_t seg_tape_bytes(int64_t p0, int64_t periods) const {
    const int NT = cfg.steps_per_period, r = cfg.r;
    size_t b = 0;
    for (int64_t p = p0; p < p0 + periods; ++p) {
      int rc[4];
      const HostState& h0 = rec.ck[0];
      for (int k = 0; k < 4; ++k) rc[k] = p == 0 ? h0.rect[k] : rec.log[(size_t)(p - 1) * 4 + k];
      const bool fine = cfg.r > 1 && rc[0] >= 0;
      const size_t fb = fine ? fplane_b(rc) : 0;
      b += (size_t)NT * (4 * up(cplane_b(), 256) + (fine ? (size_t)4 * r * up(fb, 256) : 0));
      b += 3 * up(cplane_b(), 256) + up(L.cplane * 8, 256);
      if (fine) b += 3 * up(fb, 256) + up(fb / L.es * 8, 256);
    }
    return b;
  }

  size_t adj_fixed_bytes() const {
    const size_t mx = std::max(L.cplane, L.fplane);
    size_t b = 11 * up(cplane_b(), 256);                          // coarse adjoints
    if (cfg.r > 1) b += 2 * 11 * up(L.fplane * L.es, 256);        // fine adjoints, two layouts
    b += 6 * up(mx * L.es, 256);                                  // continuity-step scratch
    b += 256;                                                     // FP64 sums
    b += 4 * side_line_bytes();                                   // Eq. 5b^T E^n shares
    return b;
  }
  size_t side_line_bytes() const {
    return up((size_t)(std::max(cfg.nx, cfg.ny) + 2) * L.es, 256);
  }

  size_t adj_bytes() const override {
    if (!rec.valid) return 0;
    const int64_t ppseg = rec.K / cfg.steps_per_period;
    const int64_t periods = rec.n / cfg.steps_per_period;
    size_t mx = 0;
    for (int64_t p0 = 0; p0 < periods; p0 += ppseg)
      mx = std::max(mx, seg_tape_bytes(p0, std::min(ppseg, periods - p0)));
    return adj_fixed_bytes() + 2 * mx;   // two segment tapes (recompute and sweep overlap)
  }

  struct StepRec {
    int64_t m;
    int rect[4];
    bool fine, rvalid;
    const T *cEx, *cEy, *cvx, *cvy;
    std::vector<const T*> fEx, fEy, fvx, fvy;   // per sub-step k (index k - 1)
  };
  struct PerRec {
    int64_t L;
    int rect_b[4], rect_a[4], cur_b, cur_a;
    bool fine, expanded, rvalid;
    const T *cEx, *cEy, *nc, *fEx, *fEy, *nf;
    const double *S2c, *S2f;
  };

  // tape allocator
  char* tape = nullptr;
  size_t tape_used = 0, tape_cap = 0;
  // tape slots never go past the caller's buffer: an overflowing request is
  // counted (and reported after the segment) but gets no slot
  bool tape_over = false;
  char* tape_slot(size_t bytes) {
    if (tape_used + up(bytes, 256) > tape_cap) { tape_over = true; return nullptr; }
    char* d = tape + tape_used;
    tape_used += up(bytes, 256);
    return d;
  }
  // Tape copies are queued and issued together by flush_tape() (one gather
  // launch instead of a copy call each).  The recording issues the flush
  // before any launch that overwrites a queued source.
  dmr::TapeJobs tjobs{};
  size_t tjob_max16 = 0;
  const T* tape_copy(const void* src, size_t bytes) {
    T* d = reinterpret_cast<T*>(tape_slot(bytes));
    if (!d) return d;
    if (bytes % 16 != 0 || ((uintptr_t)src % 16) != 0) {
      cudaMemcpyAsync(d, src, bytes, cudaMemcpyDeviceToDevice, st);
      return d;
    }
    if (tjobs.n == dmr::kTapeJobs) flush_tape();
    tjobs.src[tjobs.n] = reinterpret_cast<const int4*>(src);
    tjobs.dst[tjobs.n] = reinterpret_cast<int4*>(d);
    tjobs.n16[tjobs.n] = (long long)(bytes / 16);
    tjob_max16 = std::max(tjob_max16, bytes / 16);
    ++tjobs.n;
    return d;
  }
  void flush_tape() {
    if (tjobs.n == 0) return;
    const int gx = (int)std::min<size_t>(256, (tjob_max16 + 255) / 256);
    dmr::ka_tape_gather<<<dim3(std::max(gx, 1), tjobs.n), 256, 0, st>>>(tjobs);
    tjobs.n = 0;
    tjob_max16 = 0;
  }
  double* tape_alloc_d(size_t bytes) { return reinterpret_cast<double*>(tape_slot(bytes)); }

  dmr::Step<T> make_step_at(int rr, int64_t level, bool accum, int i0) const {
    const int save = rect[0];
    Engine<T>* self = const_cast<Engine<T>*>(this);
    self->rect[0] = i0;
    dmr::Step<T> s_ = make_step(rr, level, accum);
    self->rect[0] = save;
    return s_;
  }

  // one coarse step with its tape records: the launches of launch_coarse_step
  // (the coarse step with the first fine sub-step, then sub-steps 2..r) with
  // the tape copies queued after each and flushed before any launch that
  // overwrites their sources (double buffering keeps the inputs of a launch
  // until the launch after it).  At r = 2 one flush per coarse step, before
  // its first launch, covers all of them: the step's own inputs are queued
  // ahead of it, and what the step leaves (v outputs, sub-step 2's inputs)
  // stays intact until the next step's first launch.
  int record_step(StepRec* R) {
    const int r = cfg.r;
    R->m = m;
    for (int k = 0; k < 4; ++k) R->rect[k] = rect[k];
    R->fine = has_fine;
    R->rvalid = rvalid;
    const int cp0 = cpar;
    const bool one_flush = has_fine && r == 2;
    const size_t fb = has_fine ? fplane_b(rect) : 0;
    if (one_flush) {
      R->cEx = tape_copy(C.Ex, cplane_b());          // E^n
      R->cEy = tape_copy(C.Ey, cplane_b());
      R->fEx.push_back(tape_copy(F[cur].Ex, fb));    // sub-step 1's input
      R->fEy.push_back(tape_copy(F[cur].Ey, fb));
      flush_tape();
    }
    dmr::EmArgs<T> Ac, Af;
    em_args_for(1, m, cpar, fpar, rvalid, &Ac, has_fine ? &Af : nullptr);
    if (has_fine) go_em2(Ac.nblk + Ac.ncfb + Af.nblk + Af.ncfb, Ac, Af);
    else go_em(Ac.nblk + Ac.ncfb, Ac);
    counted(1);
    if (!one_flush) {
      R->cEx = tape_copy(C.Ex, cplane_b());        // E^n (this step's input parity)
      R->cEy = tape_copy(C.Ey, cplane_b());
    }
    flip_coarse();
    R->cvx = tape_copy(C.vx, cplane_b());        // v^{n+1/2}
    R->cvy = tape_copy(C.vy, cplane_b());
    if (has_fine) {
      for (int k = 1; k <= r; ++k) {
        if (k > 1) {
          em_args_for(k, m, cp0, fpar, rvalid, nullptr, &Af);
          go_em(Af.nblk + Af.ncfb, Af);
          counted(1);
        }
        if (!(one_flush && k == 1)) {
          R->fEx.push_back(tape_copy(F[cur].Ex, fb));   // the sub-step's input
          R->fEy.push_back(tape_copy(F[cur].Ey, fb));
        }
        flip_fine();
        R->fvx.push_back(tape_copy(F[cur].vx, fb));   // its v output
        R->fvy.push_back(tape_copy(F[cur].vy, fb));
        if (!one_flush) flush_tape();
      }
      rvalid = true;
    } else {
      flush_tape();
    }
    ++m;
    return launched("recorded EM step");
  }

  int record_period(PerRec* P) {
    P->L = m;
    for (int k = 0; k < 4; ++k) P->rect_b[k] = rect[k];
    P->cur_b = cur;
    P->fine = has_fine;
    P->rvalid = rvalid;
    P->cEx = tape_copy(C.Ex, cplane_b());
    P->cEy = tape_copy(C.Ey, cplane_b());
    P->nc = tape_copy(C.n, cplane_b());
    double* s2c = tape_alloc_d(L.cplane * 8);
    if (s2c)
      dmr::k_s2_view<T><<<nodes_grid(C.nx, C.ny), dim3(BX, BY), 0, st>>>(C, make_step(1, m, true), s2c);
    P->S2c = s2c;
    if (has_fine) {
      const size_t fb = fplane_b(rect);
      P->fEx = tape_copy(F[cur].Ex, fb);
      P->fEy = tape_copy(F[cur].Ey, fb);
      P->nf = tape_copy(F[cur].n, fb);
      double* s2f = tape_alloc_d(fb / L.es * 8);
      if (s2f)
        dmr::k_s2_view<T><<<nodes_grid(F[cur].nx, F[cur].ny), dim3(BX, BY), 0, st>>>(
            F[cur], make_step(cfg.r, (int64_t)cfg.r * m, true), s2f);
      P->S2f = s2f;
    }
    flush_tape();   // before the period end rewrites n
    if (int s = launch_period_end(m)) return s;
    if (int s = period_end_host()) return s;
    P->expanded = has_fine && (rect[0] != P->rect_b[0] || rect[1] != P->rect_b[1] ||
                               rect[2] != P->rect_b[2] || rect[3] != P->rect_b[3]);
    for (int k = 0; k < 4; ++k) P->rect_a[k] = rect[k];
    P->cur_a = cur;
    return DMR_OK;
  }

  // adjoint arrays of one mesh
  struct AdjArr {
    T* E[2][2];      // [buffer][x, y]
    T *H, *H2;       // adjoint of the present H level; the other buffer of the pair
    T *vx, *vy, *n, *ntmp, *S2;
  };

  dmr::Modes modes_of(const int* rc) const {
    dmr::Modes md;
    md.m[dmr::SIDE_LEFT] = rc[0] == 0 ? dmr::BC_MUR : dmr::BC_CFB;
    md.m[dmr::SIDE_RIGHT] = rc[2] == cfg.nx ? dmr::BC_MUR : dmr::BC_CFB;
    md.m[dmr::SIDE_BOTTOM] = rc[1] == 0 ? dmr::BC_MUR : dmr::BC_CFB;
    md.m[dmr::SIDE_TOP] = rc[3] == cfg.ny ? dmr::BC_MUR : dmr::BC_CFB;
    return md;
  }

  dmr::AdjM<T> adjm(const AdjArr& a, int in, int nx, int ny, int p) const {
    dmr::AdjM<T> A;
    A.aEx_in = a.E[in][0]; A.aEy_in = a.E[in][1];
    A.aEx_out = a.E[in ^ 1][0]; A.aEy_out = a.E[in ^ 1][1];
    A.aHz = a.H; A.aHz_out = a.H2; A.avx = a.vx; A.avy = a.vy; A.an = a.n; A.aS2 = a.S2;
    A.nx = nx; A.ny = ny; A.p = p;
    return A;
  }

  void restrict_t(const AdjArr& ca, int cin, const AdjArr& fa, int fin, const int* rc) {
    const int r = cfg.r;
    int jlo = side_at(rc, dmr::SIDE_BOTTOM) ? rc[1] : rc[1] + 1;
    int jhi = side_at(rc, dmr::SIDE_TOP) ? rc[3] : rc[3] - 1;
    int ilo = side_at(rc, dmr::SIDE_LEFT) ? rc[0] : rc[0] + 1;
    int ihi = side_at(rc, dmr::SIDE_RIGHT) ? rc[2] : rc[2] - 1;
    int fnx, fny, fp;
    fdims(rc, &fnx, &fny, &fp);
    const dim3 g((rc[2] - rc[0] + 1 + BX - 1) / BX, (rc[3] - rc[1] + 1 + BY - 1) / BY);
    dmr::ka_restrict<T><<<g, dim3(BX, BY), 0, st>>>(ca.E[cin][0], ca.E[cin][1], C.p, fa.E[fin][0],
                                                    fa.E[fin][1], fp, rc[0], rc[1], rc[2], rc[3], r,
                                                    jlo, jhi, ilo, ihi);
  }
  bool side_at(const int* rc, int sd) const {
    switch (sd) {
      case dmr::SIDE_LEFT: return rc[0] == 0;
      case dmr::SIDE_RIGHT: return rc[2] == cfg.nx;
      case dmr::SIDE_BOTTOM: return rc[1] == 0;
      default: return rc[3] == cfg.ny;
    }
  }

  int adj_backward(const void* dLdn, void* wsa, size_t bytes, void* ckpt, size_t cbytes,
                   double* dE0, double* dnu, void* dseed) override {
    if (!rec.valid) return fail(DMR_ESTATE, "dmr_adjoint_record has not run");
    if ((char*)ckpt != rec.ckpt || cbytes < adj_ckpt_bytes(rec.n, rec.K))
      return fail(DMR_EINVAL, "pass the checkpoint buffer given to dmr_adjoint_record");
    if (!wsa || bytes < adj_bytes()) return fail(DMR_ECAPACITY, "adjoint workspace too small");
    const int NT = cfg.steps_per_period, r = cfg.r;
    const bool dmr_ = cfg.r > 1;
    char* w = (char*)wsa;
    size_t o = 0;
    auto take = [&](size_t b) { char* q = w + o; o += up(b, 256); return q; };
    AdjArr ca, fa[2];
    {
      T* pl[11];
      for (int k = 0; k < 11; ++k) pl[k] = (T*)take(cplane_b());
      ca.E[0][0] = pl[0]; ca.E[0][1] = pl[1]; ca.E[1][0] = pl[2]; ca.E[1][1] = pl[3];
      ca.H = pl[4]; ca.vx = pl[5]; ca.vy = pl[6]; ca.n = pl[7]; ca.ntmp = pl[8]; ca.S2 = pl[9];
      ca.H2 = pl[10];
    }
    for (int sset = 0; sset < 2 && dmr_; ++sset) {
      T* pl[11];
      for (int k = 0; k < 11; ++k) pl[k] = (T*)take(L.fplane * L.es);
      fa[sset].E[0][0] = pl[0]; fa[sset].E[0][1] = pl[1]; fa[sset].E[1][0] = pl[2]; fa[sset].E[1][1] = pl[3];
      fa[sset].H = pl[4]; fa[sset].vx = pl[5]; fa[sset].vy = pl[6]; fa[sset].n = pl[7];
      fa[sset].ntmp = pl[8]; fa[sset].S2 = pl[9]; fa[sset].H2 = pl[10];
    }
    const size_t mx = std::max(L.cplane, L.fplane);
    T* sc[6];
    for (int k = 0; k < 6; ++k) sc[k] = (T*)take(mx * L.es);
    double* sums = (double*)take(256);
    T* side_lines[4];
    for (int k = 0; k < 4; ++k) side_lines[k] = (T*)take(side_line_bytes());
    adj_side = side_lines;
    // two segment tapes: the recompute of segment sg - 1 (on a stream of its
    // own) runs while the reverse sweep of segment sg (on the run's stream)
    // reads the other tape
    const size_t tseg = ((bytes - o) / 2) & ~(size_t)255;
    char* tapes[2] = {w + o, w + o + tseg};
    if (int s_ = ck(cudaMemsetAsync(w, 0, o, st), "zero adjoints")) return s_;
    // dL/dn at the end (dense coarse map) -> pitched adjoint of the coarse density
    if (int s_ = ck(cudaMemcpy2DAsync(ca.n, (size_t)C.p * L.es, dLdn, (size_t)(C.nx + 1) * L.es,
                                      (size_t)(C.nx + 1) * L.es, C.ny + 1, cudaMemcpyDeviceToDevice, st),
                    "load dL/dn")) return s_;
    const bool graphs0 = graphs;
    graphs = false;
    drop_graph();
    const std::vector<int32_t> user_replay = replay;
    const size_t user_pos = replay_pos;
    int cin = 0, fin = 0;       // which adjoint E buffer holds the "in" level
    int fset = -1;              // fine adjoint layout in use (= forward set index)
    const int64_t ppseg = rec.K / NT;
    const int nseg = (int)rec.ck.size();
    const dmr::Dens dc = make_dens(1), df = make_dens(r);
    const double A1 = (d.nu_model == 1 ? d.town_A : 5.14e11) * cfg.p_torr;   // d nu_i / d s_nu, per unit
    const cudaStream_t sr = st;
    cudaStream_t sq = nullptr;
    cudaEvent_t ev_rec[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr}, ev_go = nullptr;
    int st_ = ck(cudaStreamCreateWithFlags(&sq, cudaStreamNonBlocking), "recompute stream");
    for (int k = 0; k < 2 && !st_; ++k) {
      st_ = ck(cudaEventCreateWithFlags(&ev_rec[k], cudaEventDisableTiming), "event");
      if (!st_) st_ = ck(cudaEventCreateWithFlags(&ev_rev[k], cudaEventDisableTiming), "event");
    }
    if (!st_) st_ = ck(cudaEventCreateWithFlags(&ev_go, cudaEventDisableTiming), "event");
    // the recompute stream starts after everything queued on the run's stream
    if (!st_) st_ = ck(cudaEventRecord(ev_go, sr), "event record");
    if (!st_) st_ = ck(cudaStreamWaitEvent(sq, ev_go, 0), "stream wait");
    std::vector<StepRec> steps[2];
    std::vector<PerRec> pers[2];
    // restore segment sg's start and recompute it onto tape sg & 1, on sq
    auto recompute = [&](int sg) -> int {
      const int b = sg & 1;
      st = sq;
      tape = tapes[b];
      tape_cap = tseg;
      tape_used = 0;
      tape_over = false;
      int s_ = ck(cudaMemcpyAsync(ws, rec.ckpt + (size_t)sg * wbytes(), L.total, cudaMemcpyDeviceToDevice, st),
                  "restore checkpoint");
      if (!s_) {
        load_host(rec.ck[sg]);
        const int64_t p0 = (int64_t)sg * ppseg;
        const int64_t periods = std::min<int64_t>(ppseg, rec.n / NT - p0);
        replay.assign(rec.log.begin() + p0 * 4, rec.log.begin() + (p0 + periods) * 4);
        replay_pos = 0;
        steps[b].clear();
        pers[b].clear();
        for (int64_t pp = 0; pp < periods && !s_; ++pp) {
          for (int q = 0; q < NT && !s_; ++q) {
            steps[b].emplace_back();
            s_ = record_step(&steps[b].back());
          }
          if (s_) break;
          pers[b].emplace_back();
          s_ = record_period(&pers[b].back());
        }
      }
      if (!s_ && tape_over) s_ = fail(DMR_ECAPACITY, "adjoint tape overflow");
      if (!s_) s_ = ck(cudaEventRecord(ev_rec[b], sq), "event record");
      st = sr;
      return s_;
    };
    if (!st_) st_ = recompute(nseg - 1);
    if (!st_) fset = cur;
    for (int sg = nseg - 1; sg >= 0 && !st_; --sg) {
      const int b = sg & 1;
      if ((st_ = ck(cudaStreamWaitEvent(sr, ev_rec[b], 0), "stream wait"))) break;
      // ---- reverse sweep over the segment
      for (int64_t idx = (int64_t)steps[b].size() - 1; idx >= 0 && !st_; --idx) {
        const StepRec& R = steps[b][idx];
        const PerRec& P = pers[b][idx / NT];
        if ((idx + 1) % NT == 0) {
          // period end at level P.L (forward order: restriction, S2 sample,
          // continuity steps, commit, growth)
          if (P.expanded) {
            dmr::ExpT<T> e;
            int nnx, nny, np_, onx, ony, op;
            fdims(P.rect_a, &nnx, &nny, &np_);
            fdims(P.rect_b, &onx, &ony, &op);
            const AdjArr& nA = fa[P.cur_a];
            const AdjArr& oA = fa[P.cur_b];
            e.nEx = nA.E[fin][0]; e.nEy = nA.E[fin][1]; e.nHz = nA.H; e.nvx = nA.vx; e.nvy = nA.vy; e.nn = nA.n;
            e.oEx = oA.E[fin][0]; e.oEy = oA.E[fin][1]; e.oHz = oA.H; e.ovx = oA.vx; e.ovy = oA.vy; e.on = oA.n;
            e.cEx = ca.E[cin][0]; e.cEy = ca.E[cin][1]; e.cHz = ca.H; e.cvx = ca.vx; e.cvy = ca.vy; e.cn = ca.n;
            e.nnx = nnx; e.nny = nny; e.np = np_; e.onx = onx; e.ony = ony; e.op = op;
            e.cnx = C.nx; e.cny = C.ny; e.cp = C.p;
            e.I0 = P.rect_a[0]; e.J0 = P.rect_a[1]; e.oI0 = P.rect_b[0]; e.oJ0 = P.rect_b[1]; e.r = r;
            dmr::ka_expand<T><<<nodes_grid(nnx, nny), dim3(BX, BY), 0, st>>>(e);
            fset = P.cur_b;
          }
          st_ = adj_period(P, ca, fa, cin, fin, fset, sc, sums, dc, df, A1);
          if (st_) break;
        }
        // ---- coarse step R.m: fine sub-steps r..1, then the coarse step
        st_ = adj_step(R, P, ca, fa, cin, fin, fset, sums);
      }
      if (st_) break;
      if ((st_ = ck(cudaEventRecord(ev_rev[b], sr), "event record"))) break;
      if (sg > 0) {
        // the next segment's tape is free once the sweep that read it is done
        // (no wait before the first use: an event never recorded has completed)
        if ((st_ = ck(cudaStreamWaitEvent(sq, ev_rev[(sg - 1) & 1], 0), "stream wait"))) break;
        st_ = recompute(sg - 1);
      }
    }
    st = sr;
    if (sq) {
      cudaStreamSynchronize(sq);
      cudaStreamDestroy(sq);
    }
    for (int k = 0; k < 2; ++k) {
      if (ev_rec[k]) cudaEventDestroy(ev_rec[k]);
      if (ev_rev[k]) cudaEventDestroy(ev_rev[k]);
    }
    if (ev_go) cudaEventDestroy(ev_go);
    // seed map gradient: initial fine density (+ the coarse nodes it was copied to)
    if (!st_) {
      const HostState& h0 = rec.ck[0];
      if (dmr_ && h0.has_fine) {
        int fnx, fny, fp;
        fdims(h0.rect, &fnx, &fny, &fp);
        const int* rc = h0.rect;
        const dim3 gi((rc[2] - rc[0] + 1 + BX - 1) / BX, (rc[3] - rc[1] + 1 + BY - 1) / BY);
        dmr::ka_inject<T><<<gi, dim3(BX, BY), 0, st>>>(ca.n, C.p, fa[fset < 0 ? h0.cur : fset].n, fp,
                                                       rc[0], rc[1], rc[2], rc[3], r);
        if (dseed)
          st_ = ck(cudaMemcpy2DAsync(dseed, (size_t)(fnx + 1) * L.es, fa[fset < 0 ? h0.cur : fset].n,
                                     (size_t)fp * L.es, (size_t)(fnx + 1) * L.es, fny + 1,
                                     cudaMemcpyDeviceToDevice, st), "write seed gradient");
      } else if (dseed) {
        st_ = ck(cudaMemcpy2DAsync(dseed, (size_t)(C.nx + 1) * L.es, ca.n, (size_t)C.p * L.es,
                                   (size_t)(C.nx + 1) * L.es, C.ny + 1, cudaMemcpyDeviceToDevice, st),
                 "write seed gradient");
      }
    }
    double hs[2] = {0.0, 0.0};
    if (!st_) st_ = ck(cudaMemcpyAsync(hs, sums, sizeof hs, cudaMemcpyDeviceToHost, st), "read sums");
    if (!st_) st_ = ck(cudaStreamSynchronize(st), "backward sync");
    if (dE0) *dE0 = hs[0];
    if (dnu) *dnu = hs[1];
    replay = user_replay;
    replay_pos = user_pos;
    graphs = graphs0;
    tape = nullptr;
    return st_ ? st_ : launched("adjoint");
  }

  // reverse of the period end at level P.L (after any growth^T): commit^T,
  // Dirichlet^T, fine and coarse continuity^T, S2 sample^T, restriction^T
  int adj_period(const PerRec& P, AdjArr& ca, AdjArr* fa, int cin, int fin, int fset, T** sc,
                 double* sums, const dmr::Dens& dc, const dmr::Dens& df, double A1) {
    const int r = cfg.r;
    const dim3 blk(BX, BY);
    if (P.fine) {
      int fnx, fny, fp;
      fdims(P.rect_b, &fnx, &fny, &fp);
      AdjArr& A = fa[fset];
      const int* rc = P.rect_b;
      const dim3 gi((rc[2] - rc[0] + 1 + BX - 1) / BX, (rc[3] - rc[1] + 1 + BY - 1) / BY);
      dmr::ka_inject<T><<<gi, blk, 0, st>>>(ca.n, C.p, A.n, fp, rc[0], rc[1], rc[2], rc[3], r);
      dmr::Dir<T> dir{};
      dir.r = r;
      for (int q = 0; q < 4; ++q) {
        if (side_at(rc, q)) continue;
        dir.on[q] = 1;
        if (q == dmr::SIDE_BOTTOM || q == dmr::SIDE_TOP) {
          dir.line[q] = ca.n + (size_t)(q == dmr::SIDE_BOTTOM ? rc[1] : rc[3]) * C.p;
          dir.stride[q] = 1; dir.len[q] = cfg.nx + 1; dir.start[q] = rc[0];
        } else {
          dir.line[q] = ca.n + (q == dmr::SIDE_LEFT ? rc[0] : rc[2]);
          dir.stride[q] = C.p; dir.len[q] = cfg.ny + 1; dir.start[q] = rc[1];
        }
      }
      const dim3 gf = nodes_grid(fnx, fny);
      dmr::ka_dir<T><<<gf, blk, 0, st>>>(A.n, fnx, fny, fp, dir);
      // the fine density adjoint kernels read the S2 sum as T: convert in place
      dmr::ka_rates_d<T><<<gf, blk, 0, st>>>(P.nf, P.S2f, df, A1, fnx, fny, fp, sc[0], sc[1], sc[2],
                                             sc[3], sc[4], sc[5]);
      dmr::ka_density<T><<<gf, blk, 0, st>>>(P.nf, sc[0], sc[1], sc[2], sc[3], sc[4], sc[5], A.n,
                                             A.ntmp, A.S2, df, dir, fnx, fny, fp, sums + 1);
      std::swap(A.n, A.ntmp);
    }
    {
      const dim3 gc = nodes_grid(C.nx, C.ny);
      dmr::Dir<T> none{};
      dmr::ka_rates_d<T><<<gc, blk, 0, st>>>(P.nc, P.S2c, dc, A1, C.nx, C.ny, C.p, sc[0], sc[1],
                                             sc[2], sc[3], sc[4], sc[5]);
      dmr::ka_density<T><<<gc, blk, 0, st>>>(P.nc, sc[0], sc[1], sc[2], sc[3], sc[4], sc[5], ca.n,
                                             ca.ntmp, ca.S2, dc, none, C.nx, C.ny, C.p, sums + 1);
      std::swap(ca.n, ca.ntmp);
      dmr::Step<T> s_ = make_step(1, P.L, true);
      dmr::ka_s2<T><<<gc, blk, 0, st>>>(ca.E[cin][0], ca.E[cin][1], P.cEx, P.cEy, ca.S2, s_, C.nx,
                                        C.ny, C.p, sums);
    }
    if (P.fine) {
      int fnx, fny, fp;
      fdims(P.rect_b, &fnx, &fny, &fp);
      AdjArr& A = fa[fset];
      dmr::Step<T> s_ = make_step_at(r, (int64_t)r * P.L, true, P.rect_b[0]);
      dmr::ka_s2<T><<<nodes_grid(fnx, fny), blk, 0, st>>>(A.E[fin][0], A.E[fin][1], P.fEx, P.fEy, A.S2,
                                                          s_, fnx, fny, fp, sums);
      if (P.rvalid && d.coupling == 0) restrict_t(ca, cin, A, fin, P.rect_b);
    }
    return launched("adjoint period end");
  }

  // reverse of coarse step R.m: fine sub-steps r..1, then the coarse step,
  // then the transfer^T of the restricted coarse edges to the fine mesh
  // the four Eq. 5b^T line buffers of the present backward sweep
  T** adj_side = nullptr;

  // one reversed-step launch: part P0 (and its mesh's side samples), then P1.
  // Programmatic dependent launches were measured slower here: the early
  // blocks hold SM slots that the segment recompute on the other stream needs.
  void go_ka_eh(const dmr::NodePart<T>& P0, int nb0, const dmr::CfbT<T>& cb, int ncfb, const dmr::NodePart<T>& P1,
                int nb1, double* sums) const {
    dmr::ka_eh<T><<<nb0 + ncfb + nb1, dim3(BX, BY), 0, st>>>(P0, P1, cb, nb0, ncfb, sums);
  }

  // Reverse of coarse step R.m in r + 1 launches of ka_eh: per fine sub-step
  // (r..1) H^T and E^T with the Eq. 5b^T scatter; then the coarse nodes
  // within 2 nodes of the rectangle, which add the Eq. 5b^T shares of the
  // coarse E^n and transpose the fine->coarse transfer (a8) of the step
  // before.  The other coarse nodes neither read what the fine sub-steps of
  // this step write nor write what they read, so they run inside the launches
  // of fine sub-steps r and 1 (half of their block rows each).  Every adjoint
  // E edge and H cell is stored by one launch (E and H adjoints are
  // double-buffered), so no buffer is cleared between steps.
  int adj_step(const StepRec& R, const PerRec& P, AdjArr& ca, AdjArr* fa, int& cin, int& fin,
               int fset, double* sums) {
    const int NT = cfg.steps_per_period, r = cfg.r;
    const dim3 gc = nodes_grid(C.nx, C.ny);
    dmr::NodePart<T> Pc{};   // the coarse step's node blocks, all of them
    Pc.a = adjm(ca, cin, C.nx, C.ny, C.p);
    Pc.f.Ex = R.cEx; Pc.f.Ey = R.cEy; Pc.f.vx = R.cvx; Pc.f.vy = R.cvy; Pc.f.n = P.nc;
    Pc.c = make_step(1, R.m, (R.m % NT) != 0);
    for (int q = 0; q < 4; ++q) Pc.md.m[q] = dmr::BC_MUR;
    Pc.nbx = (int)gc.x;
    Pc.nby = (int)gc.y;
    Pc.sx0 = Pc.sy0 = 1;     // nothing skipped
    Pc.sx1 = Pc.sy1 = 0;
    const dmr::CfbT<T> cnone{};
    const dmr::NodePart<T> empty{};
    if (!R.fine) {
      go_ka_eh(Pc, Pc.nbx * Pc.nby, cnone, 0, empty, 0, sums);
      std::swap(ca.H, ca.H2);
      cin ^= 1;
      return launched("adjoint step");
    }
    int fnx, fny, fp;
    fdims(R.rect, &fnx, &fny, &fp);
    AdjArr& A = fa[fset];
    const dmr::Modes md = modes_of(R.rect);
    dmr::CfbT<T> cb{};
    dmr::CoarseT<T> ct{};
    for (int q = 0; q < 4; ++q) {
      cb.mode[q] = md.m[q];
      if (q == dmr::SIDE_BOTTOM || q == dmr::SIDE_TOP) {
        cb.start[q] = R.rect[0]; cb.len[q] = cfg.nx; cb.at[q] = q == dmr::SIDE_BOTTOM ? R.rect[1] : R.rect[3];
      } else {
        cb.start[q] = R.rect[1]; cb.len[q] = cfg.ny; cb.at[q] = q == dmr::SIDE_LEFT ? R.rect[0] : R.rect[2];
      }
    }
    cb.r = r;
    cb.cp = C.p;
    cb.new_x = ca.E[cin][0]; cb.new_y = ca.E[cin][1];
    for (int q = 0; q < 4; ++q) {
      cb.old_line[q] = adj_side[q];
      ct.side_on[q] = md.m[q] == dmr::BC_CFB;
      ct.side_at[q] = cb.at[q];
      ct.side[q] = adj_side[q];
    }
    int ncfb = 0;
    for (int q = 0; q < 4; ++q)
      if (md.m[q] == dmr::BC_CFB) ncfb += (q == dmr::SIDE_BOTTOM || q == dmr::SIDE_TOP) ? fnx : fny;
    const int nbc = (ncfb + BX * BY - 1) / (BX * BY);
    // coarse blocks within 2 nodes of the rectangle (after the fine
    // sub-steps) and the two halves of the rest (beside sub-steps r and 1)
    dmr::NodePart<T> Pn = Pc, Pfar[2] = {Pc, Pc};
    const int sx0 = std::max(R.rect[0] - 2, 0) / BX, sx1 = std::min(R.rect[2] + 2, C.nx) / BX;
    const int sy0 = std::max(R.rect[1] - 2, 0) / BY, sy1 = std::min(R.rect[3] + 2, C.ny) / BY;
    Pn.bx0 = sx0; Pn.nbx = sx1 - sx0 + 1;
    Pn.by0 = sy0; Pn.nby = sy1 - sy0 + 1;
    const int half = (int)gc.y / 2;
    Pfar[0].nby = half;
    Pfar[1].by0 = half;
    Pfar[1].nby = (int)gc.y - half;
    for (int h = 0; h < 2; ++h) {
      Pfar[h].sx0 = sx0; Pfar[h].sx1 = sx1;
      Pfar[h].sy0 = sy0; Pfar[h].sy1 = sy1;
    }
    const dim3 gf = nodes_grid(fnx, fny);
    for (int k = r; k >= 1; --k) {
      const int64_t mf = (int64_t)r * R.m + (k - 1);
      dmr::NodePart<T> Pf{};
      Pf.a = adjm(A, fin, fnx, fny, fp);
      Pf.f.Ex = R.fEx[k - 1]; Pf.f.Ey = R.fEy[k - 1]; Pf.f.vx = R.fvx[k - 1]; Pf.f.vy = R.fvy[k - 1];
      Pf.f.n = P.nf;
      Pf.c = make_step_at(r, mf, (mf % ((int64_t)r * NT)) != 0, R.rect[0]);
      Pf.md = md;
      Pf.nbx = (int)gf.x;
      Pf.nby = (int)gf.y;
      Pf.sx0 = Pf.sy0 = 1;
      Pf.sx1 = Pf.sy1 = 0;
      cb.frac = (T)((double)k / (double)r);
      const int side = k == r ? 0 : (k == 1 ? 1 : -1);
      const dmr::NodePart<T>& P1 = side >= 0 ? Pfar[side] : empty;
      const int nb1 = side >= 0 ? P1.nbx * P1.nby : 0;
      go_ka_eh(Pf, Pf.nbx * Pf.nby, cb, nbc, P1, nb1, sums);
      std::swap(A.H, A.H2);
      fin ^= 1;
    }
    if (R.rvalid && d.coupling == 0) {
      // a8^T of the previous step's transfer, into the fine E^n adjoint
      ct.restr = 1;
      ct.I0 = R.rect[0]; ct.J0 = R.rect[1]; ct.I1 = R.rect[2]; ct.J1 = R.rect[3]; ct.r = r;
      ct.jlo = side_at(R.rect, dmr::SIDE_BOTTOM) ? R.rect[1] : R.rect[1] + 1;
      ct.jhi = side_at(R.rect, dmr::SIDE_TOP) ? R.rect[3] : R.rect[3] - 1;
      ct.ilo = side_at(R.rect, dmr::SIDE_LEFT) ? R.rect[0] : R.rect[0] + 1;
      ct.ihi = side_at(R.rect, dmr::SIDE_RIGHT) ? R.rect[2] : R.rect[2] - 1;
      ct.fEx = A.E[fin][0]; ct.fEy = A.E[fin][1]; ct.fp = fp;
    }
    Pn.ct = ct;
    go_ka_eh(Pn, Pn.nbx * Pn.nby, cnone, 0, empty, 0, sums);
    std::swap(ca.H, ca.H2);
    cin ^= 1;
    return launched("adjoint step");
  }

  // Autotuner of the strip height for this run: times the first EM launch of
  // the present step for five warps-per-SM targets.  At a period boundary
  // that launch adds no E^2 sample and only writes the next-level buffers, so
  // repeating it leaves the run unchanged.
  void set_shape(int wps) override {
    warps_per_sm = wps;
    warps_per_sm_fine = wps;
    drop_graph();
  }
  void set_cols(int cols) override {
    lanecols = cols;
    drop_graph();
  }
  void get_shape(int32_t* out) const override {
    out[0] = warps_per_sm;
    out[1] = warps_per_sm_fine;
    out[2] = lanecols;
  }

  int autotune(int32_t* wps_out, double* trial_ms) override {
    if (m % cfg.steps_per_period != 0) return fail(DMR_ESTATE, "autotune at a period boundary");
    const int cand[5] = {8, 16, 32, 48, 96};
    // node columns per lane of the later fine sub-steps tried: 1, and 2
    // where the run can use them; two must be more than 1 % faster
    const int ncols = (sizeof(T) == 4 && d.boundary != 1 && !in_batch && !persist_on()) ? 2 : 1;
    double best = 1e30;
    int best_w = warps_per_sm;
    for (int c = 0; c < 5; ++c) {
      warps_per_sm = cand[c];
      // the steady form of the launch (coarse step reading the fine E under
      // the rectangle), also right after the start or a growth; its output
      // buffers are rewritten in full by the next real step
      dmr::EmArgs<T> Ac, Af;
      em_args_for(1, m, cpar, fpar, has_fine, &Ac, has_fine ? &Af : nullptr);
      auto launch = [&]() {
        if (has_fine)
          go_em2(Ac.nblk + Ac.ncfb + Af.nblk + Af.ncfb, Ac, Af);
        else
          go_em(Ac.nblk + Ac.ncfb, Ac);
      };
      float ms = 0.f;
      if (int s_ = ck(graph_time(st, launch, kTrialLaunches, &ms), "autotune trial")) return s_;
      launches += 4 * kTrialLaunches;
      if (trial_ms) trial_ms[c] = ms;
      if (ms < best) { best = ms; best_w = cand[c]; }
    }
    warps_per_sm = best_w;
    if (has_fine && cfg.r >= 2) {
      // The coarse step's launches as they run: the merged launch, then fine
      // sub-steps 2..r (each reading the present fine state, writing
      // next-level buffers and adding its E^2 sample; the last one writing
      // the fine->coarse means), ten coarse steps per graph, programmatic
      // dependent launches in FP32 as in the periods, for each combination of
      // the two strip heights (and node columns per lane of sub-steps 2..r).
      // Timing one launch kind alone left near-ties that cost up to 25 % in
      // the real sequence.  The samples go into S2, so S2 is kept in the
      // idle fine set (rewritten at the next growth) and put back.
      const size_t s2b = (size_t)(F[cur].ny + 1) * (size_t)F[cur].p * sizeof(double);
      if (int s_ = ck(cudaMemcpyAsync(fS2[cur ^ 1], fS2[cur], s2b, cudaMemcpyDeviceToDevice, st),
                      "autotune: keep S2")) return s_;
      const int pc[4] = {16, 32, 48, 96};
      double best_p = 1e30;
      int bc = best_w, bf = warps_per_sm_fine, blc = lanecols;
      const bool pdl = sizeof(T) == 4;
      for (int lc = 1; lc <= ncols; ++lc)
      for (int a_ = 0; a_ < 4; ++a_)
        for (int f_ = 0; f_ < 4; ++f_) {
          lanecols = lc;
          warps_per_sm = pc[a_];
          warps_per_sm_fine = pc[f_];
          dmr::EmArgs<T> Ac, A1;
          std::vector<dmr::EmArgs<T>> Ak(cfg.r + 1);
          em_args_for(1, m, cpar, fpar, true, &Ac, &A1);
          for (int k = 2; k <= cfg.r; ++k) em_args_for(k, m, cpar, fpar, true, nullptr, &Ak[k]);
          auto launch = [&]() {
            for (int q = 0; q < kTrialLaunches / 2; ++q) {
              go_em2(Ac.nblk + Ac.ncfb + A1.nblk + A1.ncfb, Ac, A1, pdl && q > 0);
              for (int k = 2; k <= cfg.r; ++k) go_em(Ak[k].nblk + Ak[k].ncfb, Ak[k], pdl);
            }
          };
          float ms = 0.f;
          if (int s_ = ck(graph_time(st, launch, 1, &ms), "autotune trial (coarse step)")) return s_;
          launches += 4 * (int64_t)(kTrialLaunches / 2) * cfg.r;
          // ties (within 1 %) go to the shorter strips, and to one column per
          // lane
          if (ms < best_p * 0.99 ||
              (ms <= best_p * 1.01 && lc == blc && (pc[a_] > bc || (pc[a_] == bc && pc[f_] > bf)))) {
            if (ms < best_p) best_p = ms;
            bc = pc[a_];
            bf = pc[f_];
            blc = lc;
          }
        }
      warps_per_sm = bc;
      warps_per_sm_fine = bf;
      lanecols = blc;
      best_w = bc;
      if (int s_ = ck(cudaMemcpyAsync(fS2[cur], fS2[cur ^ 1], s2b, cudaMemcpyDeviceToDevice, st),
                      "autotune: restore S2")) return s_;
    }
    drop_graph();
    if (wps_out) *wps_out = best_w;
    return launched("autotune");
  }

  // Measured duration of one EM launch form of the present step, as CUDA-graph
  // replays of reps back-to-back copies on the run's stream (at a period
  // boundary; the run is left unchanged): form 0 the first launch of a coarse
  // step at a period boundary (coarse step + first fine sub-step, no E^2
  // sample), 1 the same launch in the form of the other steps of a period
  // (with the E^2 samples; the sums are kept aside and put back), 2 the last
  // fine sub-step alone (with its E^2 sample and the fine->coarse transfer).
  // *bytes: the launch's algorithmic bytes.
  int time_launch(int form, int reps, double* ms_out, double* bytes_out) override {
    if (m % cfg.steps_per_period != 0) return fail(DMR_ESTATE, "launch timing at a period boundary");
    if (form < 0 || form > 2 || reps < 1 || reps > 1000) return fail(DMR_EINVAL, "form must be 0, 1 or 2 and reps in [1, 1000]");
    if (form == 2 && !has_fine) return fail(DMR_ESTATE, "form 2 needs a fine rectangle");
    const double cn = (double)(C.nx + 1) * (C.ny + 1);
    const double fn = has_fine ? (double)(F[cur].nx + 1) * (F[cur].ny + 1) : 0.0;
    const size_t cs2 = L.cplane * sizeof(double);
    const size_t fs2 = has_fine ? (size_t)(F[cur].ny + 1) * (size_t)F[cur].p * sizeof(double) : 0;
    // the E^2 sums a mid-period form adds to: coarse into the read-out
    // buffer, fine into the idle fine set (rewritten at the next growth)
    if (form >= 1) {
      if (int s_ = ck(cudaMemcpyAsync(view, C.S2, cs2, cudaMemcpyDeviceToDevice, st), "keep S2")) return s_;
      if (has_fine)
        if (int s_ = ck(cudaMemcpyAsync(fS2[cur ^ 1], fS2[cur], fs2, cudaMemcpyDeviceToDevice, st), "keep S2")) return s_;
    }
    dmr::EmArgs<T> Ac, Af;
    double bytes = 0.0;
    std::function<void()> launch;
    if (form <= 1) {
      // form 1: the launch of coarse step m + 1 of the period (both meshes
      // add their E^2 samples), on the present buffers
      em_args_for(1, m + form, cpar, fpar, has_fine, &Ac, has_fine ? &Af : nullptr);
      bytes = em_bytes(cn, form == 1) + (has_fine ? em_bytes(fn, form == 1) : 0.0);
      launch = [&]() {
        if (has_fine) go_em2(Ac.nblk + Ac.ncfb + Af.nblk + Af.ncfb, Ac, Af);
        else go_em(Ac.nblk + Ac.ncfb, Ac);
      };
    } else {
      em_args_for(cfg.r, m, cpar, fpar, true, nullptr, &Af);
      bytes = em_bytes(fn, true) + 2.0 * (double)L.es * (rect[2] - rect[0] + 1) * (rect[3] - rect[1] + 1);
      launch = [&]() { go_em(Af.nblk + Af.ncfb, Af); };
    }
    float ms = 0.f;
    int s_ = ck(graph_time(st, launch, reps, &ms), "launch timing");
    launches += 4 * reps;
    if (form >= 1) {
      int s2 = ck(cudaMemcpyAsync(C.S2, view, cs2, cudaMemcpyDeviceToDevice, st), "restore S2");
      if (!s2 && has_fine) s2 = ck(cudaMemcpyAsync(fS2[cur], fS2[cur ^ 1], fs2, cudaMemcpyDeviceToDevice, st), "restore S2");
      if (!s_) s_ = s2;
    }
    if (!s_) s_ = ck(cudaStreamSynchronize(st), "launch timing sync");
    drop_graph();
    if (s_) return s_;
    if (ms_out) *ms_out = ms;
    if (bytes_out) *bytes_out = bytes;
    return launched("launch timing");
  }

  // ---- checkpoint / resume of the whole run state (caller-owned buffer)
  size_t state_bytes() const override { return kStateHdrBytes + up(L.total, 256); }

  int save_state(void* dst, size_t bytes) override {
    if (in_batch) return fail(DMR_ESTATE, "runs of a batch are not saved one by one");
    if (!dst || ((uintptr_t)dst & 255u)) return fail(DMR_EINVAL, "state buffer must be a 256-byte aligned device pointer");
    if (bytes < state_bytes()) return fail(DMR_ECAPACITY, fmt("state buffer too small: %zu < %zu bytes", bytes, state_bytes()));
    StateHdr h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kStateMagic, sizeof h.magic);
    h.version = 1;
    h.es = (uint32_t)L.es;
    h.total = L.total;
    h.m = m;
    h.cpar = cpar; h.fpar = fpar; h.cur = cur;
    h.has_fine = has_fine ? 1 : 0;
    h.rvalid = rvalid ? 1 : 0;
    for (int q = 0; q < 4; ++q) h.rect[q] = rect[q];
    h.replay_pos = (int64_t)replay_pos;
    h.cfg = cfg;
    char* d = static_cast<char*>(dst);
    last_em = false;
    if (int s_ = ck(cudaMemcpyAsync(d + kStateHdrBytes, ws, L.total, cudaMemcpyDeviceToDevice, st), "save state"))
      return s_;
    if (int s_ = ck(cudaMemcpyAsync(d, &h, sizeof h, cudaMemcpyHostToDevice, st), "save state header"))
      return s_;
    return ck(cudaStreamSynchronize(st), "save state sync");
  }

  int load_state(const void* src, size_t bytes) override {
    if (in_batch) return fail(DMR_ESTATE, "runs of a batch are not loaded one by one");
    if (!src || ((uintptr_t)src & 255u)) return fail(DMR_EINVAL, "state buffer must be a 256-byte aligned device pointer");
    if (bytes < kStateHdrBytes) return fail(DMR_ECAPACITY, "state buffer too small");
    StateHdr h;
    const char* sp = static_cast<const char*>(src);
    if (int s_ = ck(cudaMemcpyAsync(&h, sp, sizeof h, cudaMemcpyDeviceToHost, st), "load state header")) return s_;
    if (int s_ = ck(cudaStreamSynchronize(st), "load state sync")) return s_;
    if (memcmp(h.magic, kStateMagic, sizeof h.magic) != 0 || h.version != 1)
      return fail(DMR_EINVAL, "not a saved DMR state");
    if (h.es != L.es || h.total != L.total || !same_config(h.cfg, cfg))
      return fail(DMR_EINVAL, "the state was saved by a run of another configuration");
    if (bytes < state_bytes()) return fail(DMR_ECAPACITY, "state buffer too small");
    if (h.m < 0 || (h.cpar | h.fpar | h.cur) & ~1 || (cfg.r == 1 && h.has_fine))
      return fail(DMR_EINVAL, "corrupt state header");
    if (int s_ = ck(cudaMemcpyAsync(ws, sp + kStateHdrBytes, L.total, cudaMemcpyDeviceToDevice, st), "load state"))
      return s_;
    drop_graph();
    last_em = false;
    dead = false;
    rec = Rec();
    m = h.m;
    cpar = h.cpar;
    C.Ex = cE[cpar][0]; C.Ey = cE[cpar][1]; C.Hz = cE[cpar][2]; C.vx = cE[cpar][3]; C.vy = cE[cpar][4];
    has_fine = h.has_fine != 0;
    rvalid = h.rvalid != 0;
    cur = h.cur;
    for (int q = 0; q < 4; ++q) rect[q] = h.rect[q];
    if (has_fine) {
      F[cur] = fine_view(cur, rect);
      fpar = 0;
      if (h.fpar) flip_fine();
    } else {
      fpar = 0;
    }
    // a replayed refinement log continues where it stood when the state was
    // saved (the log itself is this run's own setting)
    replay_pos = std::min<size_t>((size_t)std::max<int64_t>(h.replay_pos, 0), replay.size() / 4);
    return DMR_OK;
  }

  int stats(double* out) override {
    dmr::Ctl hc;
    if (int s = ck(cudaMemcpyAsync(&hc, ctl, sizeof hc, cudaMemcpyDeviceToHost, st), "stats")) return s;
    if (int s = ck(cudaStreamSynchronize(st), "stats sync")) return s;
    const double fine_cells = has_fine ? (double)F[cur].nx * (double)F[cur].ny : 0.0;
    out[DMR_STAT_T] = (double)m * d.dtc;
    out[DMR_STAT_R] = has_fine ? fine_cells / ((double)cfg.r * cfg.r * (double)cfg.nx * cfg.ny) : 0.0;
    out[DMR_STAT_FINE_CELLS] = fine_cells;
    out[DMR_STAT_NE] = hc.st[0];
    out[DMR_STAT_PABS] = hc.st[1];
    out[DMR_STAT_WABS] = hc.st[2];
    out[DMR_STAT_PERIODS] = hc.st[3];
    out[DMR_STAT_COARSE_STEPS] = (double)m;
    out[DMR_STAT_NMAX] = hc.st[4];
    out[DMR_STAT_FLAGS] = (double)hc.nflag;
    return DMR_OK;
  }
};

// --------------------------------------------------------------------------
// Batched runs: independent DMR runs (sizes, E0, pressure, seeds may differ;
// precision, r and N_T shared) advanced together.  Per coarse step one launch
// covers every run's coarse step and first fine sub-step (segment tables in
// device memory; the level-dependent values are looked up in the kernel), one
// launch per later fine sub-step; each run's period-end kernels are parallel
// branches of the same per-period CUDA graph; one gather kernel collects the
// runs' control blocks for a single read-back.
__global__ void k_gather_ctl(const dmr::Ctl* const* src, dmr::Ctl* dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = *src[i];
}

struct BatchBase {
  std::string err;
  int64_t launches = 0;
  int tuned_wps = 0;
  double tune_ms[8] = {};
  virtual ~BatchBase() {}
  virtual int advance(int64_t n) = 0;
  virtual int set_graphs(bool on) = 0;
  virtual int autotune() = 0;
  virtual int nruns() const = 0;
  virtual Base* run(int k) = 0;
  int fail(int code, const std::string& msg) { err = msg; return code; }
};

// bytes of the batch's own tables (segment arguments, offsets, control blocks)
size_t batch_table_bytes(int n, int r, int es) {
  const size_t args = es == 4 ? sizeof(dmr::EmArgs<float>) : sizeof(dmr::EmArgs<double>);
  const size_t nseg = (size_t)4 * 2 * n + (size_t)2 * (r > 1 ? r - 1 : 0) * n;
  const size_t ntab = 4 + 2 * (size_t)(r > 1 ? r - 1 : 0);
  return up(nseg * args, 256) + up((nseg + ntab) * sizeof(int), 256) +
         up((size_t)n * sizeof(void*), 256) + up((size_t)n * sizeof(dmr::Ctl), 256);
}

template <class T>
struct Batch final : BatchBase {
  std::vector<Engine<T>*> runs;
  cudaStream_t st = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  char* tdev = nullptr;       // table area (device)
  size_t tbytes = 0;
  dmr::Ctl** ctl_ptrs = nullptr;
  dmr::Ctl* ctl_all = nullptr;
  int NT = 0, r = 1;
  int64_t m = 0;
  bool graphs = true;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_nodes = 0;
  struct Tab { const dmr::EmArgs<T>* args; const int* off; int nseg; int nblk; };
  Tab t1[2][2] = {};          // phase 1: [first step after a table build][coarse parity]
  std::vector<Tab> tk[2];     // phase k = 2..r: [coarse parity][k - 2]
  std::vector<int> shape;     // segment block counts the graph was captured with
  bool first_pending = true;

  ~Batch() override {
    if (gexec) cudaGraphExecDestroy(gexec);
    for (auto s_ : side) cudaStreamDestroy(s_);
    for (auto e : join) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    for (auto e : runs) delete e;
  }
  int nruns() const override { return (int)runs.size(); }
  Base* run(int k) override { return runs[k]; }
  int ck(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return DMR_OK;
    return fail(DMR_ECUDA, fmt("%s: %s", what, cudaGetErrorString(e)));
  }
  int run_fail(int k, int code) { return fail(code, fmt("run %d: %s", k, runs[k]->err.c_str())); }

  int init() {
    side.resize(runs.size());
    join.resize(runs.size());
    for (size_t q = 0; q < runs.size(); ++q) {
      if (int s = ck(cudaStreamCreateWithFlags(&side[q], cudaStreamNonBlocking), "stream")) return s;
      if (int s = ck(cudaEventCreateWithFlags(&join[q], cudaEventDisableTiming), "event")) return s;
    }
    if (int s = ck(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "event")) return s;
    std::vector<dmr::Ctl*> ptrs(runs.size());
    for (size_t q = 0; q < runs.size(); ++q) ptrs[q] = runs[q]->ctl;
    if (int s = ck(cudaMemcpyAsync(ctl_ptrs, ptrs.data(), ptrs.size() * sizeof(void*),
                                   cudaMemcpyHostToDevice, st), "upload control pointers")) return s;
    return ck(cudaStreamSynchronize(st), "batch init sync");
  }

  // (re)build and upload the segment tables from the runs' present state
  int build_tables() {
    std::vector<dmr::EmArgs<T>> segs;
    std::vector<int> offs;
    std::vector<std::pair<size_t, size_t>> marks;   // (first segment, first offset) per table
    auto add_table = [&](std::vector<dmr::EmArgs<T>>& v) {
      marks.push_back({segs.size(), offs.size()});
      int acc = 0;
      for (auto& a : v) { offs.push_back(acc); acc += a.nblk + a.ncfb; segs.push_back(a); }
      offs.push_back(acc);
    };
    for (int first = 0; first < 2; ++first)
      for (int cp = 0; cp < 2; ++cp) {
        // all first fine sub-steps, then all coarse steps: the fine side
        // blocks carry the longest dependent chain and are dispatched first
        std::vector<dmr::EmArgs<T>> v, vc;
        for (auto* e : runs) {
          dmr::EmArgs<T> Ac, Af;
          const bool rv = first ? e->rvalid : e->has_fine;
          e->em_args_for(1, m, cp, 0, rv, &Ac, e->has_fine ? &Af : nullptr);
          vc.push_back(Ac);
          if (e->has_fine) v.push_back(Af);
        }
        v.insert(v.end(), vc.begin(), vc.end());
        add_table(v);
      }
    for (int cp = 0; cp < 2; ++cp)
      for (int k = 2; k <= r; ++k) {
        std::vector<dmr::EmArgs<T>> v;
        for (auto* e : runs) {
          if (!e->has_fine) continue;
          dmr::EmArgs<T> Af;
          e->em_args_for(k, m, cp, (k - 1) & 1, true, nullptr, &Af);
          v.push_back(Af);
        }
        add_table(v);
      }
    const size_t abytes = up(segs.size() * sizeof(dmr::EmArgs<T>), 256);
    const size_t obytes = offs.size() * sizeof(int);
    if (abytes + obytes > tbytes) return fail(DMR_ECAPACITY, "batch tables exceed their area");
    std::vector<char> stage(abytes + obytes, 0);
    memcpy(stage.data(), segs.data(), segs.size() * sizeof(dmr::EmArgs<T>));
    memcpy(stage.data() + abytes, offs.data(), obytes);
    if (int s = ck(cudaMemcpyAsync(tdev, stage.data(), stage.size(), cudaMemcpyHostToDevice, st),
                   "upload batch tables")) return s;
    if (int s = ck(cudaStreamSynchronize(st), "table sync")) return s;
    const auto* A = reinterpret_cast<const dmr::EmArgs<T>*>(tdev);
    const int* O = reinterpret_cast<const int*>(tdev + abytes);
    std::vector<int> new_shape;
    auto tab = [&](size_t t) {
      Tab x;
      const size_t s0 = marks[t].first, o0 = marks[t].second;
      const size_t s1 = t + 1 < marks.size() ? marks[t + 1].first : segs.size();
      x.args = A + s0;
      x.off = O + o0;
      x.nseg = (int)(s1 - s0);
      x.nblk = offs[o0 + x.nseg];
      new_shape.push_back(x.nblk);
      return x;
    };
    size_t t = 0;
    for (int first = 0; first < 2; ++first)
      for (int cp = 0; cp < 2; ++cp) t1[first][cp] = tab(t++);
    for (int cp = 0; cp < 2; ++cp) {
      tk[cp].clear();
      for (int k = 2; k <= r; ++k) tk[cp].push_back(tab(t++));
    }
    if (new_shape != shape) {
      shape = new_shape;
      if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
    }
    // the first-step tables differ from the steady ones while a run's fine
    // mesh has not stepped since it was (re)built
    first_pending = false;
    for (auto* e : runs) first_pending |= e->has_fine && !e->rvalid;
    return DMR_OK;
  }

  int launch_em(const Tab& t, int64_t level, int k) {
    if (t.nseg == 0 || t.nblk == 0) return 0;
    if (k > 1 && k == r)   // the last fine sub-step writes the fine->coarse E mean
      dmr::k_em_batch<T, true><<<t.nblk, 32 * dmr::EM_WARPS, 0, st>>>(t.args, t.off, t.nseg, (long long)level, k);
    else
      dmr::k_em_batch<T><<<t.nblk, 32 * dmr::EM_WARPS, 0, st>>>(t.args, t.off, t.nseg, (long long)level, k);
    return 1;
  }

  // EM launches of coarse step q of the period starting at level m0
  int launch_step(int64_t m0, int q, bool first) {
    const int cp = (int)((m0 + q) & 1);
    int n = launch_em(t1[first ? 1 : 0][cp], m0 + q, 1);
    for (int k = 2; k <= r; ++k) n += launch_em(tk[cp][k - 2], m0 + q, k);
    return n;
  }

  int check_state() {
    for (size_t q = 0; q < runs.size(); ++q) {
      auto* e = runs[q];
      if (e->m != m || e->cpar != (int)(m & 1) || (e->has_fine && e->fpar != 0))
        return fail(DMR_ESTATE, fmt("run %d was advanced outside the batch", (int)q));
    }
    return DMR_OK;
  }

  // host state of every run after one coarse step done by the batch
  void after_step() {
    for (auto* e : runs) {
      e->flip_coarse();
      if (e->has_fine) {
        for (int k = 0; k < r; ++k) e->flip_fine();
        e->rvalid = true;
      }
      ++e->m;
    }
    ++m;
  }

  int period_end_direct() {
    for (auto* e : runs)
      if (int s = e->launch_period_end(m)) return fail(s, e->err);
    k_gather_ctl<<<(int)((runs.size() + 127) / 128), 128, 0, st>>>(ctl_ptrs, ctl_all, (int)runs.size());
    launches += 1;
    return decide();
  }

  // read all control blocks once, then each run's stability guard and growth
  int decide() {
    std::vector<dmr::Ctl> hc(runs.size());
    if (int s = ck(cudaMemcpyAsync(hc.data(), ctl_all, hc.size() * sizeof(dmr::Ctl),
                                   cudaMemcpyDeviceToHost, st), "read control blocks")) return s;
    if (int s = ck(cudaStreamSynchronize(st), "period sync")) return s;
    bool changed = false;
    for (size_t q = 0; q < runs.size(); ++q) {
      auto* e = runs[q];
      int old[4] = {e->rect[0], e->rect[1], e->rect[2], e->rect[3]};
      if (int s = e->period_decide(hc[q])) return run_fail((int)q, s);
      for (int k = 0; k < 4; ++k) changed |= old[k] != e->rect[k];
    }
    // a grown rectangle changes the period-end launches captured in the graph
    if (changed && gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
    if (changed || first_pending) return build_tables();
    return DMR_OK;
  }

  int capture() {
    if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
    cudaGraph_t g = nullptr;
    if (int s = ck(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture")) return s;
    int s = DMR_OK;
    graph_nodes = 0;
    for (int q = 0; q < NT; ++q) graph_nodes += launch_step(m, q, q == 0 && first_pending);
    // period ends: one parallel branch per run
    cudaEventRecord(fork, st);
    std::vector<bool> rv(runs.size());
    for (size_t q = 0; q < runs.size() && !s; ++q) {
      auto* e = runs[q];
      cudaStreamWaitEvent(side[q], fork, 0);
      e->st = side[q];
      e->capturing = true;
      e->graph_nodes = 0;
      rv[q] = e->rvalid;
      if (e->has_fine) e->rvalid = true;     // the fine mesh will have stepped by then
      s = e->launch_period_end(m + NT);
      graph_nodes += e->graph_nodes;
      e->capturing = false;
      e->rvalid = rv[q];
      e->st = st;
      cudaEventRecord(join[q], side[q]);
      cudaStreamWaitEvent(st, join[q], 0);
    }
    k_gather_ctl<<<(int)((runs.size() + 127) / 128), 128, 0, st>>>(ctl_ptrs, ctl_all, (int)runs.size());
    graph_nodes += 1;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (s) { if (g) cudaGraphDestroy(g); return fail(s, "period-end capture failed"); }
    if (e != cudaSuccess) return ck(e, "end capture");
    e = cudaGraphInstantiate(&gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { gexec = nullptr; return ck(e, "graph instantiate"); }
    gexec_first = first_pending;
    return DMR_OK;
  }
  bool gexec_first = false;

  int advance(int64_t n) override {
    if (n < 0) return fail(DMR_EINVAL, "negative step count");
    if (int s = check_state()) return s;
    if (shape.empty())
      if (int s = build_tables()) return s;
    while (n > 0) {
      const int q0 = (int)(m % NT);
      if (graphs && q0 == 0 && n >= NT) {
        if (gexec && first_pending && !gexec_first) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
        if (!gexec)
          if (int s = capture()) return s;
        if (int s = ck(cudaGraphLaunch(gexec, st), "cudaGraphLaunch")) return s;
        launches += graph_nodes;
        for (int q = 0; q < NT; ++q) after_step();
        n -= NT;
        if (int s = decide()) return s;
        continue;
      }
      launches += launch_step(m - q0, q0, q0 == 0 && first_pending);
      if (int s = ck(cudaGetLastError(), "batched EM launch")) return s;
      after_step();
      --n;
      if (m % NT == 0) {
        if (int s = period_end_direct()) return s;
      }
    }
    return DMR_OK;
  }

  int set_graphs(bool on) override {
    graphs = on;
    if (!on && gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
    return DMR_OK;
  }

  // Autotuner: the strip height (rows per warp) follows a warps-per-SM target;
  // each candidate is timed on the phase-1 launch of the current step.  At a
  // period boundary that launch adds no E^2 sample and writes only the
  // next-level buffers, so repeating it leaves the run unchanged.
  int autotune() override {
    if (int s = check_state()) return s;
    if (m % NT != 0) return fail(DMR_ESTATE, "autotune at a period boundary");
    const int cand[5] = {1, 2, 4, 8, 16};   // batches favour long strips (fewer blocks to stage)
    double best = 1e30;
    int best_w = 48;
    for (int c = 0; c < 5; ++c) {
      for (auto* e : runs) e->warps_per_sm = e->warps_per_sm_fine = cand[c];
      if (int s = build_tables()) return s;
      const Tab& t = t1[0][m & 1];   // steady tables (see Engine::autotune)
      float ms = 0.f;
      if (int s = ck(graph_time(st, [&]() { launch_em(t, m, 1); }, 5, &ms), "autotune trial")) return s;
      tune_ms[c] = ms;
      launches += 4 * 5;
      if (tune_ms[c] < best) { best = tune_ms[c]; best_w = cand[c]; }
    }
    for (auto* e : runs) e->warps_per_sm = e->warps_per_sm_fine = best_w;
    tuned_wps = best_w;
    return build_tables();
  }
};

}  // namespace

struct dmr_ctx {
  Base* e;
  bool borrowed = false;   // a run of a batch: owned by the batch
};

struct dmr_batch {
  BatchBase* b;
  std::vector<dmr_ctx> ctxs;
};

namespace {
int batch_check(const dmr_config* cfgs, int n, std::vector<Derived>* ds, std::vector<Layout>* ls,
                size_t* total, std::string* err) {
  if (!cfgs || n < 1) { *err = "need at least one configuration"; return DMR_EINVAL; }
  ds->resize(n);
  ls->resize(n);
  size_t tot = 0;
  for (int q = 0; q < n; ++q) {
    std::string e;
    if (int s = derive(&cfgs[q], &(*ds)[q], &e)) { *err = fmt("run %d: %s", q, e.c_str()); return s; }
    if (int s = make_layout(&cfgs[q], (*ds)[q], &(*ls)[q], &e)) { *err = fmt("run %d: %s", q, e.c_str()); return s; }
    if (cfgs[q].precision != cfgs[0].precision || cfgs[q].r != cfgs[0].r ||
        cfgs[q].steps_per_period != cfgs[0].steps_per_period) {
      *err = "runs of a batch share precision, r and steps_per_period";
      return DMR_EINVAL;
    }
    if ((*ds)[q].boundary != 0) { *err = fmt("run %d: batched runs need the Mur boundary", q); return DMR_EINVAL; }
    tot += up((*ls)[q].total, 256);
  }
  if (cfgs[0].steps_per_period % 2 != 0 || (cfgs[0].r > 1 && cfgs[0].r % 2 != 0)) {
    *err = "a batch needs an even steps_per_period and r = 1 or even";
    return DMR_EINVAL;
  }
  *total = batch_table_bytes(n, cfgs[0].r, cfgs[0].precision == 1 ? 4 : 8) + tot;
  return DMR_OK;
}

template <class T>
int batch_make(const dmr_config* cfgs, int n, const std::vector<Derived>& ds,
               const std::vector<Layout>& ls, char* ws, cudaStream_t st, BatchBase** out,
               std::string* err) {
  auto* b = new (std::nothrow) Batch<T>();
  if (!b) { *err = "out of host memory"; return DMR_EINVAL; }
  b->st = st;
  b->NT = cfgs[0].steps_per_period;
  b->r = cfgs[0].r;
  const size_t es = cfgs[0].precision == 1 ? 4 : 8;
  const size_t tb = batch_table_bytes(n, b->r, (int)es);
  // table area: segment arguments and offsets, then control pointers and blocks
  const size_t ctl_bytes = up((size_t)n * sizeof(dmr::Ctl), 256);
  const size_t ptr_bytes = up((size_t)n * sizeof(void*), 256);
  b->tdev = ws;
  b->tbytes = tb - ctl_bytes - ptr_bytes;
  b->ctl_ptrs = reinterpret_cast<dmr::Ctl**>(ws + b->tbytes);
  b->ctl_all = reinterpret_cast<dmr::Ctl*>(ws + b->tbytes + ptr_bytes);
  size_t o = tb;
  for (int q = 0; q < n; ++q) {
    auto* e = new (std::nothrow) Engine<T>();
    if (!e) { delete b; *err = "out of host memory"; return DMR_EINVAL; }
    e->cfg = cfgs[q];
    e->d = ds[q];
    e->L = ls[q];
    e->ws = ws + o;
    e->st = st;
    e->in_batch = true;
    o += up(ls[q].total, 256);
    b->runs.push_back(e);
    if (int s = e->init()) { *err = fmt("run %d: %s", q, e->err.c_str()); delete b; return s; }
  }
  if (int s = b->init()) { *err = b->err; delete b; return s; }
  *out = b;
  return DMR_OK;
}
}  // namespace

extern "C" {

size_t dmr_workspace_bytes(const dmr_config* cfg) {
  Derived d;
  Layout L;
  std::string err;
  if (derive(cfg, &d, &err) || make_layout(cfg, d, &L, &err)) {
    g_err = err;
    return 0;
  }
  return L.total;
}

int dmr_create(const dmr_config* cfg, void* ws, size_t bytes, void* stream, dmr_ctx** out) {
  if (!out) { g_err = "null output pointer"; return DMR_EINVAL; }
  *out = nullptr;
  Derived d;
  Layout L;
  std::string err;
  if (int s = derive(cfg, &d, &err)) { g_err = err; return s; }
  if (int s = make_layout(cfg, d, &L, &err)) { g_err = err; return s; }
  if (!ws || ((uintptr_t)ws & 255u)) { g_err = "workspace must be a 256-byte aligned device pointer"; return DMR_EINVAL; }
  if (bytes < L.total) { g_err = fmt("workspace too small: %zu < %zu bytes", bytes, L.total); return DMR_ECAPACITY; }
  Base* e = cfg->precision == 1 ? (Base*)new (std::nothrow) Engine<float>()
                                : (Base*)new (std::nothrow) Engine<double>();
  if (!e) { g_err = "out of host memory"; return DMR_EINVAL; }
  e->cfg = *cfg;
  e->d = d;
  e->L = L;
  e->ws = (char*)ws;
  e->st = (cudaStream_t)stream;
  if (int s = e->init()) { g_err = e->err; delete e; return s; }
  dmr_ctx* c = new (std::nothrow) dmr_ctx{e};
  if (!c) { delete e; g_err = "out of host memory"; return DMR_EINVAL; }
  *out = c;
  return DMR_OK;
}

void dmr_destroy(dmr_ctx* ctx) {
  if (!ctx || ctx->borrowed) return;
  delete ctx->e;
  delete ctx;
}

const char* dmr_last_error(const dmr_ctx* ctx) {
  if (!ctx) return g_err.c_str();
  return ctx->e->err.c_str();
}

#define CTX_OR_FAIL(c)               \
  if (!(c)) {                        \
    g_err = "null context";          \
    return DMR_EINVAL;               \
  }

int dmr_seed_gaussian(dmr_ctx* ctx, double n0, double x0, double y0, double sx, double sy, int add) {
  CTX_OR_FAIL(ctx);
  return ctx->e->seed(n0, x0, y0, sx, sy, add);
}

int dmr_set_patch(dmr_ctx* ctx, const int32_t rect[4]) {
  CTX_OR_FAIL(ctx);
  if (!rect) return ctx->e->fail(DMR_EINVAL, "null rectangle");
  return ctx->e->set_patch(rect);
}

int dmr_get_patch(const dmr_ctx* ctx, int32_t rect[4]) {
  CTX_OR_FAIL(ctx);
  if (!rect) return ctx->e->fail(DMR_EINVAL, "null output pointer");
  for (int q = 0; q < 4; ++q) rect[q] = ctx->e->has_fine ? ctx->e->rect[q] : -1;
  return DMR_OK;
}

int dmr_advance(dmr_ctx* ctx, int64_t n) {
  CTX_OR_FAIL(ctx);
  return ctx->e->advance(n);
}

int dmr_replay_log(dmr_ctx* ctx, const int32_t* rects, int64_t n_periods) {
  CTX_OR_FAIL(ctx);
  if (n_periods < 0 || (n_periods > 0 && !rects)) return ctx->e->fail(DMR_EINVAL, "bad replay log");
  ctx->e->replay.assign(rects, rects + 4 * n_periods);
  ctx->e->replay_pos = 0;
  return DMR_OK;
}

int dmr_field_shape(const dmr_ctx* ctx, int field, int level, int32_t shape[2], int32_t* eb) {
  CTX_OR_FAIL(ctx);
  if (!shape) return ctx->e->fail(DMR_EINVAL, "null output pointer");
  return ctx->e->shape(field, level, shape, eb);
}

int dmr_read(const dmr_ctx* ctx, int field, int level, void* dst, size_t bytes, int dev) {
  CTX_OR_FAIL(ctx);
  if (!dst) return ctx->e->fail(DMR_EINVAL, "null destination");
  return ctx->e->read(field, level, dst, bytes, dev);
}

int dmr_write(dmr_ctx* ctx, int field, int level, const void* src, size_t bytes, int dev) {
  CTX_OR_FAIL(ctx);
  if (!src) return ctx->e->fail(DMR_EINVAL, "null source");
  return ctx->e->write(field, level, src, bytes, dev);
}

int dmr_stats(const dmr_ctx* ctx, double out[DMR_NSTATS]) {
  CTX_OR_FAIL(ctx);
  if (!out) return ctx->e->fail(DMR_EINVAL, "null output pointer");
  return ctx->e->stats(out);
}

int dmr_set_graphs(dmr_ctx* ctx, int enable) {
  CTX_OR_FAIL(ctx);
  ctx->e->graphs = enable != 0;
  if (!enable) ctx->e->drop_graph();
  return DMR_OK;
}

int dmr_set_persistent(dmr_ctx* ctx, int enable, int32_t rows_coarse, int32_t rows_fine) {
  CTX_OR_FAIL(ctx);
  if (rows_coarse < 0 || rows_coarse > 64 || rows_fine < 0 || rows_fine > 64)
    return ctx->e->fail(DMR_EINVAL, "rows per warp outside [0, 64]");
  if (ctx->e->in_batch) return ctx->e->fail(DMR_ESTATE, "runs of a batch step in the batch's launches");
  ctx->e->persist = enable != 0;
  ctx->e->prow_c = rows_coarse;
  ctx->e->prow_f = rows_fine;
  ctx->e->drop_graph();
  return DMR_OK;
}

int dmr_test_stall(dmr_ctx* ctx, int stall, int64_t polls) {
  CTX_OR_FAIL(ctx);
  if (polls < 1) return ctx->e->fail(DMR_EINVAL, "polls must be >= 1");
  ctx->e->sched_stall = stall != 0;
  ctx->e->sched_limit = polls;
  ctx->e->drop_graph();
  return DMR_OK;
}

int dmr_set_launch_shape(dmr_ctx* ctx, int32_t warps_per_sm) {
  CTX_OR_FAIL(ctx);
  if (warps_per_sm < 1 || warps_per_sm > 1024) return ctx->e->fail(DMR_EINVAL, "warps_per_sm outside [1, 1024]");
  ctx->e->set_shape(warps_per_sm);
  return DMR_OK;
}

int dmr_set_strip_columns(dmr_ctx* ctx, int32_t columns_per_lane) {
  CTX_OR_FAIL(ctx);
  if (columns_per_lane < 1 || columns_per_lane > 2) return ctx->e->fail(DMR_EINVAL, "columns_per_lane must be 1 or 2");
  if (ctx->e->in_batch) return ctx->e->fail(DMR_ESTATE, "runs of a batch step in the batch's launches");
  ctx->e->set_cols(columns_per_lane);
  return DMR_OK;
}

int dmr_get_launch_shape(const dmr_ctx* ctx, int32_t shape[3]) {
  CTX_OR_FAIL(ctx);
  if (!shape) return ctx->e->fail(DMR_EINVAL, "null output pointer");
  ctx->e->get_shape(shape);
  return DMR_OK;
}

int dmr_set_timing(dmr_ctx* ctx, int enable) {
  CTX_OR_FAIL(ctx);
  ctx->e->timing = enable != 0;
  ctx->e->timing_mask = (unsigned)enable;
  ctx->e->drop_graph();
  ctx->e->pend.clear();
  ctx->e->evd_used = 0;
  for (int q = 0; q < 8; ++q) { ctx->e->kt_ms[q] = 0; ctx->e->kt_n[q] = 0; ctx->e->kt_units[q] = 0; }
  return DMR_OK;
}

int dmr_kernel_time(const dmr_ctx* ctx, int kclass, double* ms, int64_t* n, double* units) {
  CTX_OR_FAIL(ctx);
  if (kclass < 0 || kclass >= 8) return DMR_EINVAL;
  if (ms) *ms = ctx->e->kt_ms[kclass];
  if (n) *n = ctx->e->kt_n[kclass];
  if (units) *units = ctx->e->kt_units[kclass];
  return DMR_OK;
}

const char* dmr_kernel_class_name(int kclass) {
  static const char* names[] = {"em_step", "fine_em", "restrict", "period_end", "expand", "em_period"};
  if (kclass < 0 || kclass >= 6) return nullptr;
  return names[kclass];
}

int dmr_launch_count(const dmr_ctx* ctx, int64_t* n) {
  CTX_OR_FAIL(ctx);
  if (!n) return ctx->e->fail(DMR_EINVAL, "null output pointer");
  *n = ctx->e->launches;
  return DMR_OK;
}

int dmr_sync(const dmr_ctx* ctx) {
  CTX_OR_FAIL(ctx);
  return ctx->e->ck(cudaStreamSynchronize(ctx->e->st), "sync");
}

size_t dmr_batch_workspace_bytes(const dmr_config* cfgs, int32_t n) {
  std::vector<Derived> ds;
  std::vector<Layout> ls;
  size_t total = 0;
  std::string err;
  if (batch_check(cfgs, n, &ds, &ls, &total, &err)) { g_err = err; return 0; }
  return total;
}

int dmr_batch_create(const dmr_config* cfgs, int32_t n, void* ws, size_t bytes, void* stream,
                     dmr_batch** out) {
  if (!out) { g_err = "null output pointer"; return DMR_EINVAL; }
  *out = nullptr;
  std::vector<Derived> ds;
  std::vector<Layout> ls;
  size_t total = 0;
  std::string err;
  if (int s = batch_check(cfgs, n, &ds, &ls, &total, &err)) { g_err = err; return s; }
  if (!ws || ((uintptr_t)ws & 255u)) { g_err = "workspace must be a 256-byte aligned device pointer"; return DMR_EINVAL; }
  if (bytes < total) { g_err = fmt("workspace too small: %zu < %zu bytes", bytes, total); return DMR_ECAPACITY; }
  if (!stream) { g_err = "a batch needs a non-default stream (it is captured in CUDA graphs)"; return DMR_EINVAL; }
  BatchBase* b = nullptr;
  const int s = cfgs[0].precision == 1
                    ? batch_make<float>(cfgs, n, ds, ls, (char*)ws, (cudaStream_t)stream, &b, &err)
                    : batch_make<double>(cfgs, n, ds, ls, (char*)ws, (cudaStream_t)stream, &b, &err);
  if (s) { g_err = err; return s; }
  dmr_batch* h = new (std::nothrow) dmr_batch{b, {}};
  if (!h) { delete b; g_err = "out of host memory"; return DMR_EINVAL; }
  h->ctxs.resize(n);
  for (int q = 0; q < n; ++q) { h->ctxs[q].e = b->run(q); h->ctxs[q].borrowed = true; }
  *out = h;
  return DMR_OK;
}

void dmr_batch_destroy(dmr_batch* b) {
  if (!b) return;
  delete b->b;
  delete b;
}

dmr_ctx* dmr_batch_run(dmr_batch* b, int32_t k) {
  if (!b || k < 0 || k >= b->b->nruns()) return nullptr;
  return &b->ctxs[k];
}

int dmr_batch_advance(dmr_batch* b, int64_t n) {
  if (!b) { g_err = "null batch"; return DMR_EINVAL; }
  return b->b->advance(n);
}

int dmr_batch_set_graphs(dmr_batch* b, int enable) {
  if (!b) { g_err = "null batch"; return DMR_EINVAL; }
  return b->b->set_graphs(enable != 0);
}

int dmr_batch_autotune(dmr_batch* b, int32_t* warps_per_sm, double trial_ms[5]) {
  if (!b) { g_err = "null batch"; return DMR_EINVAL; }
  const int s = b->b->autotune();
  if (warps_per_sm) *warps_per_sm = b->b->tuned_wps;
  if (trial_ms)
    for (int q = 0; q < 5; ++q) trial_ms[q] = b->b->tune_ms[q];
  return s;
}

int dmr_batch_launch_count(const dmr_batch* b, int64_t* n) {
  if (!b || !n) { g_err = "null argument"; return DMR_EINVAL; }
  *n = b->b->launches;
  for (int q = 0; q < b->b->nruns(); ++q) *n += b->b->run(q)->launches;
  return DMR_OK;
}

const char* dmr_batch_last_error(const dmr_batch* b) {
  if (!b) return g_err.c_str();
  return b->b->err.c_str();
}

size_t dmr_adjoint_checkpoint_bytes(const dmr_ctx* ctx, int64_t n_steps, int64_t K) {
  if (!ctx) return 0;
  return ctx->e->adj_ckpt_bytes(n_steps, K);
}

int dmr_adjoint_record(dmr_ctx* ctx, int64_t n_steps, int64_t K, void* ckpt, size_t bytes) {
  CTX_OR_FAIL(ctx);
  return ctx->e->adj_record(n_steps, K, ckpt, bytes);
}

size_t dmr_adjoint_workspace_bytes(const dmr_ctx* ctx) {
  if (!ctx) return 0;
  return ctx->e->adj_bytes();
}

int dmr_adjoint_backward(dmr_ctx* ctx, const void* dL_dn, void* ws, size_t bytes, void* ckpt,
                         size_t ckpt_bytes, double* dL_dE0, double* dL_dnu_scale, void* dL_dseed) {
  CTX_OR_FAIL(ctx);
  if (!dL_dn) return ctx->e->fail(DMR_EINVAL, "null dL/dn");
  return ctx->e->adj_backward(dL_dn, ws, bytes, ckpt, ckpt_bytes, dL_dE0, dL_dnu_scale, dL_dseed);
}

int dmr_autotune(dmr_ctx* ctx, int32_t* warps_per_sm, double trial_ms[5]) {
  CTX_OR_FAIL(ctx);
  return ctx->e->autotune(warps_per_sm, trial_ms);
}

int dmr_time_launch(dmr_ctx* ctx, int form, int reps, double* ms_per_launch, double* algorithmic_bytes) {
  CTX_OR_FAIL(ctx);
  return ctx->e->time_launch(form, reps, ms_per_launch, algorithmic_bytes);
}

size_t dmr_state_bytes(const dmr_ctx* ctx) {
  if (!ctx) return 0;
  return ctx->e->state_bytes();
}

int dmr_save_state(dmr_ctx* ctx, void* dev_dst, size_t bytes) {
  CTX_OR_FAIL(ctx);
  return ctx->e->save_state(dev_dst, bytes);
}

int dmr_load_state(dmr_ctx* ctx, const void* dev_src, size_t bytes) {
  CTX_OR_FAIL(ctx);
  return ctx->e->load_state(dev_src, bytes);
}

}  // extern "C"
