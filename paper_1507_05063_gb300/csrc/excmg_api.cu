// C ABI of libexcmg (include/excmg.h): argument checks, workspace layout, and the host
// side of Algorithm 1 -- the level loop, the CG loop with its convergence reads, the
// MIXED iterative refinement, the batched phases and the adjoint.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "excmg_internal.cuh"

namespace excmg {

Grid3 make_grid(int nx, int ny, int nz, double Lx, double Ly, double Lz) {
  Grid3 g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.sy = nx + 1;
  g.sz = (long long)(nx + 1) * (ny + 1);
  g.hx = Lx / nx;
  g.hy = Ly / ny;
  g.hz = Lz / nz;
  return g;
}

Grid3 padded_f32(const Grid3& g) {
  Grid3 p = g;
  p.sy = (g.nx + 1 + 3) & ~3LL;
  p.sz = p.sy * (g.ny + 1);
  return p;
}

Coef make_coef(const Grid3& g) {
  const double a = 1.0 / (g.hx * g.hx), b = 1.0 / (g.hy * g.hy), c = 1.0 / (g.hz * g.hz);
  Coef A;
  A.c0 = 8.0 * (a + b + c);
  A.fx = -(4.0 * a - b - c);
  A.fy = -(4.0 * b - a - c);
  A.fz = -(4.0 * c - a - b);
  A.exy = -0.5 * (a + b);
  A.exz = -0.5 * (a + c);
  A.eyz = -0.5 * (b + c);
  return A;
}

Tiling make_tiling(const Grid3& g, int tz) {
  if (tz < 1) tz = 1;
  Tiling t;
  t.tz = tz;
  t.ntx = (g.nx + 1 + kTX - 1) / kTX;
  t.nty = (g.ny + 1 + kTY - 1) / kTY;
  t.ntz = (g.nz + 1 + tz - 1) / tz;
  return t;
}

// Slab depth of the residual kernel: among 1..64 the one minimising (rounds of the tiles
// that hold interior nodes over the residual grid) x (planes per tile, halo included).
// Tiles of boundary nodes only cost nothing (k_residual writes zeros there), and every
// block of a round waits for the slowest, so a deep slab that leaves blocks idle loses
// to a thin one that fills every block.
int choose_res_tz(const Grid3& g, int grid_blocks, int requested, int rows) {
  if (requested > 0) return requested;
  int best = 16;
  double best_cost = 1e300;
  const int cands[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32, 48, 64};
  for (int tz : cands) {
    const long long tiles = (long long)((g.nx + kTX - 1) / kTX) *
                            ((g.ny + kTY * rows - 1) / (kTY * rows)) * ((g.nz + tz - 1) / tz);
    const long long rounds = (tiles + grid_blocks - 1) / grid_blocks;
    const double cost = (double)rounds * (std::min(tz, g.nz + 1) + 2);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = tz;
    }
  }
  return best;
}

Tiling make_res_tiling(const Grid3& g, int tz, int rows) {
  Tiling t = make_tiling(g, tz);
  t.nty = (g.ny + 1 + kTY * rows - 1) / (kTY * rows);
  return t;
}

int res_rows_model(const Grid3& g) { return g.nodes() >= kResWideMinNodes ? kResRowsWide : 1; }


// Slab depth: among 1..64 the one minimising (waves of tiles) x (planes staged per tile),
// a model of the stencil kernel's time when every block runs at the same rate.  Large
// grids get deep slabs (little halo re-staging); small, latency-bound grids get thin
// slabs and so more tiles in flight.
int choose_tz(const Grid3& g, int grid_blocks, int requested) {
  if (requested > 0) return requested;
  int best = 16;
  double best_cost = 1e300;
  const int cands[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
  for (int tz : cands) {
    const Tiling t = make_tiling(g, tz);
    const long long tiles = t.count();
    const long long waves = (tiles + grid_blocks - 1) / grid_blocks;
    const int depth = std::min(tz, g.nz + 1);
    const double cost = (double)waves * (depth + 2);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = tz;
    }
  }
  return best;
}

}  // namespace excmg

using namespace excmg;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Level {
  int nx, ny, nz;
  long long nodes() const { return (long long)(nx + 1) * (ny + 1) * (nz + 1); }
};

// Validated level list of a grid, coarsest first; empty if invalid.
std::vector<Level> levels_of(const excmg_grid* gr) {
  std::vector<Level> out;
  if (!gr) return out;
  if (!(gr->Lx > 0) || !(gr->Ly > 0) || !(gr->Lz > 0)) return out;
  if (gr->Nx0 < 2 || gr->Ny0 < 2 || gr->Nz0 < 2) return out;
  if (gr->Nx0 % 2 || gr->Ny0 % 2 || gr->Nz0 % 2) return out;
  if (gr->Nx % gr->Nx0 || gr->Ny % gr->Ny0 || gr->Nz % gr->Nz0) return out;
  const int rx = gr->Nx / gr->Nx0, ry = gr->Ny / gr->Ny0, rz = gr->Nz / gr->Nz0;
  if (rx != ry || rx != rz || rx < 4 || (rx & (rx - 1))) return out;
  int lv = 0;
  while ((1 << lv) < rx) ++lv;
  if (lv + 1 > EXCMG_MAX_LEVELS) return out;
  if ((long long)(gr->Nx + 1) * (gr->Ny + 1) * (gr->Nz + 1) > (1LL << 40)) return out;
  for (int l = 0; l <= lv; ++l) out.push_back({gr->Nx0 << l, gr->Ny0 << l, gr->Nz0 << l});
  return out;
}

// The single grid Nx x Ny x Nz (coarsest-grid fields ignored); empty if invalid.
std::vector<Level> single_level(const excmg_grid* gr) {
  std::vector<Level> out;
  if (!gr) return out;
  if (!(gr->Lx > 0) || !(gr->Ly > 0) || !(gr->Lz > 0)) return out;
  if (gr->Nx < 2 || gr->Ny < 2 || gr->Nz < 2) return out;
  if ((long long)(gr->Nx + 1) * (gr->Ny + 1) * (gr->Nz + 1) > (1LL << 40)) return out;
  out.push_back({gr->Nx, gr->Ny, gr->Nz});
  return out;
}

bool options_ok(const excmg_options* o) {
  if (!o) return false;
  if (o->precision != EXCMG_FP64 && o->precision != EXCMG_MIXED) return false;
  if (!(o->eps >= 0) || !(o->eps_coarse >= 0) || o->max_iter < 0) return false;
  if (o->precision == EXCMG_MIXED && (!(o->inner_tol > 0) || !(o->inner_tol < 1) || o->max_refine < 1))
    return false;
  if (o->fixed_iters && o->precision != EXCMG_FP64) return false;
  if (o->tile_z < 0 || o->tile_z > 256 || o->chunk < 0 || o->mixed_min_nodes < 0) return false;
  if (o->dsolve != EXCMG_DSOLVE_DIRECT && o->dsolve != EXCMG_DSOLVE_CG) return false;
  if (!(o->eps_ratio >= 0) || !std::isfinite(o->eps_ratio)) return false;
  if (o->prolong != EXCMG_PROLONG_QUARTIC && o->prolong != EXCMG_PROLONG_QUADRATIC &&
      o->prolong != EXCMG_PROLONG_LINEAR)
    return false;
  if (o->history && (o->history_len < 1 || o->precision != EXCMG_FP64)) return false;
  if (o->rhs_norm != EXCMG_RHS_NORM_LIFT && o->rhs_norm != EXCMG_RHS_NORM_FORCING) return false;
  if (!(o->wait_timeout_ms >= 0) || !std::isfinite(o->wait_timeout_ms) || o->wait_timeout_ms > 3.6e6)
    return false;
  if (o->test_phantom_blocks < 0 || o->test_phantom_blocks > 64) return false;
  if (o->autotune < -1 || o->autotune > 1) return false;
  if (o->res_rows != 0 && o->res_rows != 1 && o->res_rows != kResRowsWide) return false;
  return true;
}

}  // namespace

bool excmg::options_valid(const excmg_options* o) { return options_ok(o); }

namespace {

// ---- launch-shape tuning (options.autotune) ----
// A process-wide cache of measured launch shapes per level grid, engine class (float64
// CG or the float32 tensor-copy engine of MIXED inner solves) and device: the residual's
// slab depth and the slab depth of the CG engine that runs the level.  Filled by the
// tuning pass of excmg_solve (autotune = 1), read by every solve (autotune >= 0).
struct TuneKey {
  int nx, ny, nz, f32, dev;
  bool operator<(const TuneKey& o) const {
    if (nx != o.nx) return nx < o.nx;
    if (ny != o.ny) return ny < o.ny;
    if (nz != o.nz) return nz < o.nz;
    if (f32 != o.f32) return f32 < o.f32;
    return dev < o.dev;
  }
};
std::map<TuneKey, excmg_tuning> g_tune;
std::mutex g_tune_mu;

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

bool tune_lookup(const Grid3& g, bool f32, excmg_tuning* out) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(TuneKey{g.nx, g.ny, g.nz, f32 ? 1 : 0, current_device()});
  if (it == g_tune.end()) return false;
  if (out) *out = it->second;
  return true;
}

void tune_store(const Grid3& g, bool f32, const excmg_tuning& t) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[TuneKey{g.nx, g.ny, g.nz, f32 ? 1 : 0, current_device()}] = t;
}

// Per-problem workspace layout.
struct ProbLayout {
  size_t coarse_off[EXCMG_MAX_LEVELS];  // u of levels 0 .. L-2 (float64)
  size_t r, pa, pb, q;                  // float64 CG vectors (finest size)
  size_t r32, pa32, pb32, q32, e32;     // float32 CG vectors (MIXED)
  size_t rhs64;                         // MIXED: 2 RHS(f) of the level being refined
  size_t s0, s1;                        // resident CG: s by step parity (its grids' size)
  size_t bytes;
};

long long mixed_min(const excmg_options* o) {
  return o->mixed_min_nodes > 0 ? o->mixed_min_nodes : kMixedMinNodes;
}

ProbLayout prob_layout(const std::vector<Level>& lv, bool mixed, bool need_fp64_vectors,
                       long long minn = kMixedMinNodes) {
  ProbLayout L;
  memset(&L, 0, sizeof(L));
  size_t off = 0;
  for (size_t l = 0; l + 1 < lv.size(); ++l) {
    L.coarse_off[l] = off;
    off = align_up(off + sizeof(double) * lv[l].nodes());
  }
  const long long nf = lv.back().nodes();
  // float32 vectors use the padded row pitch (padded_f32): nodes of the finest level
  const long long nf32 = (long long)((lv.back().nx + 1 + 3) & ~3) * (lv.back().ny + 1) * (lv.back().nz + 1);
  // float64 CG vectors: every level (FP64), or the levels MIXED solves in float64
  long long n64 = 0;
  for (size_t k = 0; k < lv.size(); ++k)  // (levels 0 and 1: DSOLVE works in float64)
    if (!mixed || need_fp64_vectors || lv[k].nodes() < minn || k < 2) n64 = std::max(n64, lv[k].nodes());
  if (n64 > 0) {
    L.r = off;
    off = align_up(off + sizeof(double) * n64);
    L.pa = off;
    off = align_up(off + sizeof(double) * n64);
    L.pb = off;
    off = align_up(off + sizeof(double) * n64);
    L.q = off;
    off = align_up(off + sizeof(double) * n64);
    // two more float64 vectors for the levels small enough for the resident CG
    long long nres = 0;
    for (const Level& l : lv)
      if (l.nodes() <= kResidentMaxNodes && (!mixed || need_fp64_vectors || l.nodes() < minn))
        nres = std::max(nres, l.nodes());
    if (nres > 0) {
      L.s0 = off;
      off = align_up(off + sizeof(double) * nres);
      L.s1 = off;
      off = align_up(off + sizeof(double) * nres);
    }
  }
  if (mixed) {
    const size_t v32 = sizeof(float) * nf32;
    L.r32 = off;
    off = align_up(off + v32);
    L.pa32 = off;
    off = align_up(off + v32);
    L.pb32 = off;
    off = align_up(off + v32);
    L.q32 = off;
    off = align_up(off + v32);
    L.e32 = off;
    off = align_up(off + v32);
    L.rhs64 = off;
    off = align_up(off + sizeof(double) * nf);
  }
  L.bytes = off;
  return L;
}

// Common header of every workspace: states, counters, partials, descriptor tables.
struct Header {
  size_t st, counters, bar, partials, cgd, cgf, resd, prold, tmaps;
  size_t bytes;
};

// States: one per (problem, level): slot = problem * EXCMG_MAX_LEVELS + level.
int state_slots(int nprob) { return std::max(nprob, 1) * (int)EXCMG_MAX_LEVELS; }
int slot_of(int problem, int level) { return problem * (int)EXCMG_MAX_LEVELS + level; }

Header header_layout(int nprob) {
  Header H;
  size_t off = 0;
  H.st = off;
  off = align_up(off + sizeof(CGState) * state_slots(nprob));
  H.counters = off;
  off = align_up(off + sizeof(unsigned) * state_slots(nprob));
  H.bar = off;  // per problem: barrier arrival count + time-out flag; then the team-slot counter
  off = align_up(off + (2 * sizeof(unsigned)) * std::max(nprob, 1) + sizeof(unsigned));
  H.partials = off;
  off = align_up(off + sizeof(double) * 2 * (size_t)nprob * kMaxGrid);
  H.cgd = off;
  off = align_up(off + sizeof(CGDesc<double>) * nprob);
  H.cgf = off;
  off = align_up(off + sizeof(CGDesc<float>) * nprob);
  H.resd = off;
  off = align_up(off + sizeof(ResDesc) * nprob);
  H.prold = off;
  off = align_up(off + sizeof(ProlongDesc) * nprob);
  H.tmaps = off;
  off = align_up(off + sizeof(TmapSet) * nprob);
  H.bytes = off;
  return H;
}

#define CK(call)                              \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return EXCMG_ERR_CUDA; \
  } while (0)

// One problem's static data for a solve.
struct Prob {
  bool cascade = true;   // levels of Algorithm 1 (0 and 1: DSOLVE); false: one CG grid
  std::vector<Level> lv;
  excmg_grid gr;
  const double* f;
  const double* g;
  double* u;             // finest output
  char* base;            // its workspace region
  ProbLayout L;
  double* level_u(int l) {
    return (l + 1 == (int)lv.size()) ? u : reinterpret_cast<double*>(base + L.coarse_off[l]);
  }
  Grid3 grid(int l) const {
    return make_grid(lv[l].nx, lv[l].ny, lv[l].nz, gr.Lx, gr.Ly, gr.Lz);
  }
  View fview(int l) const {
    const int s = lv.back().nx / lv[l].nx;
    const Grid3 fg = grid((int)lv.size() - 1);
    return View{f, s, s * fg.sy, s * fg.sz};
  }
  View gview(int l) const {
    const int s = lv.back().nx / lv[l].nx;
    const Grid3 fg = grid((int)lv.size() - 1);
    return View{g, s, s * fg.sy, s * fg.sz};
  }
};

// Event timing of kernel launches (options.profile): one record per launch.
struct Prof {
  struct Rec {
    int kind;
    size_t e0, e1;   // indices into pool
    double nodes;
    bool real;
    int iter_slot;   // >= 0: nodes are per CG step, times the steps of that state slot
    int level;       // level of the solve the launch worked on (-1: not known)
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> recs;
  ~Prof() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
  size_t event() {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) e = nullptr;
    pool.push_back(e);
    return pool.size() - 1;
  }
  // Sum the records into stats after the stream has been synchronised.
  void report(excmg_stats* st, const std::vector<CGState>& states) const {
    if (!st) return;
    for (const Rec& r : recs) {
      if (!r.real || !pool[r.e0] || !pool[r.e1]) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pool[r.e0], pool[r.e1]) != cudaSuccess) continue;
      double nodes = r.nodes;
      if (r.iter_slot >= 0) {
        const int steps = r.iter_slot < (int)states.size() ? states[r.iter_slot].iter : 0;
        if (steps <= 0) continue;
        nodes *= steps;
      }
      st->prof_ms[r.kind] += ms;
      st->prof_launches[r.kind] += 1;
      st->prof_nodes[r.kind] += nodes;
      if (r.level >= 0 && r.level < EXCMG_MAX_LEVELS) st->ms_level[r.level] += ms;
      st->ms_total += ms;
    }
  }
};

struct Ctx {
  char* ws;
  Header H;
  cudaStream_t s;
  double* hist = nullptr;         // device r.r history of the finest level (options.history)
  int level = -1;                 // level being solved (profiling of single solves)
  long long* launches = nullptr;  // kernels launched by this call
  Prof* prof = nullptr;           // set when the call is profiled
  bool persistent_ok = false;     // single-problem CG may use the cooperative kernel
  bool defer = false;             // the caller reads the CG states after the whole call
  unsigned long long wait_ns = 20000000000ull;  // bound of every device-side wait
  int phantom = 0;                // test only: never-launched members per cooperative team
  // Bracket one launch: record an event before `fn` and after it.
  template <typename F>
  cudaError_t timed(int kind, double nodes, F fn) const {
    if (launches) *launches += 1;
    if (!prof) return fn();
    const size_t a = prof->event(), b = prof->event();
    if (prof->pool[a]) cudaEventRecord(prof->pool[a], s);
    cudaError_t e = fn();
    if (prof->pool[b]) cudaEventRecord(prof->pool[b], s);
    prof->recs.push_back({kind, a, b, nodes, true, -1, level});
    return e;
  }
  CGState* st() const { return reinterpret_cast<CGState*>(ws + H.st); }
  unsigned* counters() const { return reinterpret_cast<unsigned*>(ws + H.counters); }
  unsigned* bar() const { return reinterpret_cast<unsigned*>(ws + H.bar); }
  int* bar_err() const { return reinterpret_cast<int*>(ws + H.bar + sizeof(unsigned)); }
  double* partials() const { return reinterpret_cast<double*>(ws + H.partials); }
  CGDesc<double>* cgd() const { return reinterpret_cast<CGDesc<double>*>(ws + H.cgd); }
  CGDesc<float>* cgf() const { return reinterpret_cast<CGDesc<float>*>(ws + H.cgf); }
  ResDesc* resd() const { return reinterpret_cast<ResDesc*>(ws + H.resd); }
  ProlongDesc* prold() const { return reinterpret_cast<ProlongDesc*>(ws + H.prold); }
  TmapSet* tmaps() const { return reinterpret_cast<TmapSet*>(ws + H.tmaps); }
  // the wait bound and test option of `o`
  void set_waits(const excmg_options* o) {
    if (o->wait_timeout_ms > 0) wait_ns = (unsigned long long)(o->wait_timeout_ms * 1e6);
    phantom = o->test_phantom_blocks;
  }
};

// options.history: the device copy at the end of the workspace
size_t hist_bytes(const excmg_options* o) {
  return o->history ? align_up(sizeof(double) * (size_t)o->history_len) : 0;
}

// The finest level's r.r history -> options.history as ||r_k|| / ||b||, k <= iters.
excmg_status copy_history(const Ctx& c, const excmg_options* o, const CGState& S) {
  if (!o->history || !c.hist) return EXCMG_OK;
  const int n = std::min(S.iter + 1, o->history_len);
  if (n <= 0) return EXCMG_OK;
  std::vector<double> h(n);
  CK(cudaMemcpy(h.data(), c.hist, sizeof(double) * n, cudaMemcpyDeviceToHost));
  for (int k = 0; k < n; ++k) o->history[k] = S.bb > 0 ? sqrt(h[k] / S.bb) : 0.0;
  return EXCMG_OK;
}

// The CG states come back through a small page-locked, device-mapped host buffer that a
// one-block kernel fills (one per host thread, grown on demand, kept for the thread's
// life).  A copy-engine transfer would queue behind the caller's own device-to-host
// copies on other streams: a concurrent 2.2 GB download of the previous solution held
// every state read of a MIXED solve until it finished (+11 ms per 1024x512x512 solve).
struct StateMirror {
  CGState* host = nullptr;
  CGState* dev = nullptr;
  int cap = 0;
  ~StateMirror() {
    if (host) cudaFreeHost(host);
  }
};
thread_local StateMirror g_mirror;

excmg_status read_states(const Ctx& c, int nprob, std::vector<CGState>& hs) {
  hs.resize(nprob);
  if (g_mirror.cap < nprob) {
    if (g_mirror.host) cudaFreeHost(g_mirror.host);
    g_mirror = StateMirror();
    const int cap = std::max(nprob, 64);
    void* h = nullptr;
    void* d = nullptr;
    if (cudaHostAlloc(&h, sizeof(CGState) * cap, cudaHostAllocMapped | cudaHostAllocPortable) == cudaSuccess &&
        cudaHostGetDevicePointer(&d, h, 0) == cudaSuccess) {
      g_mirror.host = static_cast<CGState*>(h);
      g_mirror.dev = static_cast<CGState*>(d);
      g_mirror.cap = cap;
    } else {
      if (h) cudaFreeHost(h);
      cudaGetLastError();
    }
  }
  if (g_mirror.cap >= nprob) {
    if (c.launches) *c.launches += 1;
    CK(launch_export_states(c.st(), g_mirror.dev, nprob, c.s));
    CK(cudaStreamSynchronize(c.s));
    memcpy(hs.data(), g_mirror.host, sizeof(CGState) * nprob);
  } else {  // no mapped buffer: a plain copy
    CK(cudaMemcpyAsync(hs.data(), c.st(), sizeof(CGState) * nprob, cudaMemcpyDeviceToHost, c.s));
    CK(cudaStreamSynchronize(c.s));
  }
  return EXCMG_OK;
}

// Runs CG steps over the problems described by `descs` (device copy, `n` entries) until
// every one of them is done.  Returns the number of convergence reads.
template <typename T>
excmg_status cg_loop(const Ctx& c, int n, CGDesc<T>* ddesc, long long tiles, int grid,
                     const std::vector<int>& slots, int nslots, int chunk0,
                     std::vector<CGState>& hs, double nodes, std::vector<CGDesc<T>>& hd) {
  // Every problem runs all its CG steps inside one launch when the device supports it:
  // small grids (all of this phase's problems up to kClusterMaxNodes nodes) each in one
  // thread-block cluster with the vectors in shared memory; larger ones in a cooperative
  // launch where problem p gets a team of blocks and iterates on its own.
  const int coop = persistent_cg_blocks<T>();
  // a single float64 grid that fits the resident CG (vectors in shared memory)
  // (the smallest grids stay on the cluster kernel below: its exchange through
  // distributed shared memory beats the global round trips of the resident one there)
  if (n == 1 && sizeof(T) == 8 && c.persistent_ok && hd[0].s0 && hd[0].s1 &&
      hd[0].g.nodes() > kResidentMinNodes && hd[0].g.nodes() <= kResidentMaxNodes) {
    ResidentDesc D;
    memset(&D, 0, sizeof(D));
    size_t smem = 0;
    if (resident_box(hd[0].g, D, smem)) {
      D.g = hd[0].g;
      D.A = hd[0].A;
      D.slot = hd[0].slot;
      D.x = reinterpret_cast<double*>(hd[0].x);
      D.r = reinterpret_cast<double*>(hd[0].r);
      D.r1 = reinterpret_cast<double*>(hd[0].pa);
      D.w0 = reinterpret_cast<double*>(hd[0].pb);
      D.w1 = reinterpret_cast<double*>(hd[0].q);
      D.s0 = reinterpret_cast<double*>(hd[0].s0);
      D.s1 = reinterpret_cast<double*>(hd[0].s1);
      D.hist = hd[0].hist;
      D.hist_len = hd[0].hist_len;
      double2* pairs = reinterpret_cast<double2*>(c.partials());  // 2 G pairs
      CK(cudaMemsetAsync(c.bar(), 0, 2 * sizeof(unsigned), c.s));  // counter, time-out flag
      if (c.launches) *c.launches += 1;
      if (c.prof) {
        const size_t a = c.prof->event(), b = c.prof->event();
        if (c.prof->pool[a]) cudaEventRecord(c.prof->pool[a], c.s);
        CK(launch_cg_resident(D, smem, c.st(), pairs, c.bar(), c.bar_err(), c.s));
        if (c.prof->pool[b]) cudaEventRecord(c.prof->pool[b], c.s);
        c.prof->recs.push_back({EXCMG_K_CG_RESIDENT_F64, a, b, nodes, true, slots[0], c.level});
      } else {
        CK(launch_cg_resident(D, smem, c.st(), pairs, c.bar(), c.bar_err(), c.s));
      }
      if (c.defer) return EXCMG_OK;
      excmg_status e = read_states(c, nslots, hs);
      if (e == EXCMG_OK && c.prof) {
        // states are read now: count the steps before a later residual resets them
        Prof::Rec& rec = c.prof->recs.back();
        rec.nodes *= hs[slots[0]].iter;
        rec.iter_slot = -1;
        rec.real = hs[slots[0]].iter > 0;
      }
      return e;
    }
  }
  // MIXED inner solves (float32): the tensor-copy engine when every problem has its
  // maps; it also applies the right-hand side's scale inside its first step.  Every
  // other engine gets the scale from k_scale_rhs first.
  // The small grids of the phase run in one cluster each when all of them fit one.
  int csize = 0;
  size_t csmem = 0;
  long long cmax = 0;
  if (coop >= n && coop > 0 && c.persistent_ok) {
    for (int p = 0; p < n; ++p) {
      const int cp = hd[p].g.nodes() <= kClusterMaxNodes ? cluster_cg_size<T>(hd[p].g) : 0;
      if (cp == 0) {
        csize = 0;
        break;
      }
      csize = std::max(csize, cp);
    }
    for (int p = 0; p < n && csize > 0; ++p) {
      csmem = std::max(csmem, cluster_cg_smem(hd[p].g, csize, sizeof(T)));
      cmax = std::max(cmax, hd[p].g.nodes());
    }
  }
  const bool small = csize > 0;
  bool tma = false;
  int coop_used = coop;
  if constexpr (sizeof(T) == 4) {
    bool all = c.persistent_ok && coop >= n && coop > 0 && !small;
    for (int p = 0; p < n && all; ++p) all = hd[p].tm != nullptr;
    const int ct = all ? persistent_cg_blocks_tma() : -1;
    tma = all && ct >= n;
    if (tma) coop_used = ct;
    bool pending = false;
    for (int p = 0; p < n; ++p) {
      pending = pending || hd[p].fold_scale;
      if (!tma) hd[p].fold_scale = 0;
    }
    if (pending && !tma) {
      CK(cudaMemcpyAsync(ddesc, hd.data(), sizeof(CGDesc<T>) * n, cudaMemcpyHostToDevice, c.s));
      CK(c.timed(EXCMG_K_CORRECT, nodes, [&] { return launch_scale_rhs(n, ddesc, tiles, grid, c.st(), c.s); }));
    }
  }
  if (coop >= n && coop > 0 && c.persistent_ok) {
    int grid_total = 0;
    if (!small) {
      // team sizes: a lone problem takes every co-resident block it can use; in a batch
      // each problem takes about one block per two tiles, and teams are formed in order
      // of decreasing size (slots are taken in order by the blocks of one launch)
      std::vector<int> g(n), order(n);
      long long slots = 0;
      for (int p = 0; p < n; ++p) {
        const long long tp = hd[p].t.count();
        const long long want = (n == 1) ? tp : (tp + 1) / 2;
        g[p] = (int)std::max(1LL, std::min<long long>(want, coop_used));
        order[p] = p;
        slots += g[p];
      }
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return g[a] > g[b]; });
      int begin = 0;
      for (int p : order) {
        hd[p].blk_begin = begin;
        // test only: members that are never launched, so the team's barriers cannot
        // complete and its waits run out (options.test_phantom_blocks)
        hd[p].blk_count = g[p] + c.phantom;
        begin += g[p] + c.phantom;
      }
      grid_total = (int)std::min<long long>(slots, coop_used);
      CK(cudaMemcpyAsync(ddesc, hd.data(), sizeof(CGDesc<T>) * n, cudaMemcpyHostToDevice, c.s));
      CK(cudaMemsetAsync(c.bar(), 0, (2 * sizeof(unsigned)) * n + sizeof(unsigned), c.s));
    }
    auto launch = [&]() -> cudaError_t {
      if (small) return launch_cg_cluster<T>(n, ddesc, csize, csmem, cmax, c.st(), c.s);
      return launch_cg_persistent<T>(n, ddesc, grid_total, c.st(), c.partials(), c.bar(), c.wait_ns, tma, c.s);
    };
    const int kind = small ? (sizeof(T) == 8 ? EXCMG_K_CG_CLUSTER_F64 : EXCMG_K_CG_CLUSTER_F32)
                           : (sizeof(T) == 8 ? EXCMG_K_CG_F64 : EXCMG_K_CG_F32);
    if (c.launches) *c.launches += 1;
    if (c.prof && n == 1) {
      const size_t a = c.prof->event(), b = c.prof->event();
      if (c.prof->pool[a]) cudaEventRecord(c.prof->pool[a], c.s);
      CK(launch());
      if (c.prof->pool[b]) cudaEventRecord(c.prof->pool[b], c.s);
      c.prof->recs.push_back({kind, a, b, nodes, true, slots[0], c.level});
    } else {
      CK(launch());
    }
    if (c.defer) return EXCMG_OK;
    excmg_status e = read_states(c, nslots, hs);
    if (e == EXCMG_OK && c.prof && n == 1) {
      // states are read now: count the steps before a later residual resets them
      Prof::Rec& rec = c.prof->recs.back();
      rec.nodes *= hs[slots[0]].iter;
      rec.iter_slot = -1;
      rec.real = hs[slots[0]].iter > 0;
    }
    return e;
  }
  int chunk = chunk0 > 0 ? chunk0 : 4;
  Prof* prof = (c.prof && n == 1) ? c.prof : nullptr;
  const int kspmv = sizeof(T) == 8 ? EXCMG_K_SPMV_F64 : EXCMG_K_SPMV_F32;
  const int kupd = sizeof(T) == 8 ? EXCMG_K_UPDATE_F64 : EXCMG_K_UPDATE_F32;
  const size_t rec0 = prof ? prof->recs.size() : 0;
  int launched = 0;
  for (;;) {
    for (int m = 0; m < chunk; ++m) {
      if (prof) {
        const size_t e0 = prof->event(), e1 = prof->event(), e2 = prof->event();
        CK(launch_cg_step<T>(n, ddesc, tiles, grid, c.st(), c.partials(), c.counters(), c.s,
                             prof->pool[e0], prof->pool[e1], prof->pool[e2]));
        prof->recs.push_back({kspmv, e0, e1, nodes, true, -1, c.level});
        prof->recs.push_back({kupd, e1, e2, nodes, true, -1, c.level});
      } else {
        CK(launch_cg_step<T>(n, ddesc, tiles, grid, c.st(), c.partials(), c.counters(), c.s));
      }
      ++launched;
      if (c.launches) *c.launches += 2;
    }
    excmg_status e = read_states(c, nslots, hs);
    if (e != EXCMG_OK) return e;
    bool all = true;
    for (int sl : slots) all = all && hs[sl].done;
    if (all) break;
    if (chunk0 <= 0) chunk = std::min(chunk * 2, 64);
  }
  if (prof) {
    // steps issued after convergence returned at once: not counted
    const int real = std::min(hs[slots[0]].iter, launched);
    for (size_t k = rec0 + 2 * (size_t)real; k < prof->recs.size(); ++k) prof->recs[k].real = false;
  }
  return EXCMG_OK;
}

int tiles_grid(long long tiles) { return persistent_grid(tiles); }

// One linear system A x = b of a solve phase: its residual descriptor (b from f and the
// Dirichlet data in x's boundary, or from `src`), its float64 CG descriptor and its
// float32 correction descriptor (MIXED).
struct Item {
  ResDesc res;
  CGDesc<double> d64;
  CGDesc<float> d32;
  double* rhs_cache;    // MIXED: 2 RHS(f) kept between refinement residuals (NULL: none)
  double eps;           // stop at ||r|| <= eps ||b||
  long long nodes;
  // results
  int iters, refs, status;
  double relres;
};

ResDesc make_res(const Grid3& g, int tile_z, int slot, const double* x, View f,
                 const double* src, int rows) {
  ResDesc r;
  memset(&r, 0, sizeof(r));
  r.g = g;
  r.A = make_coef(g);
  r.rows = rows;
  r.t = make_res_tiling(g, choose_res_tz(g, residual_grid(1LL << 40, rows), tile_z, rows), rows);
  r.slot = slot;
  r.u = x;
  r.f = f;
  r.src = src;
  r.want_b = 1;
  r.osy = g.sy;
  r.osz = g.sz;
  return r;
}

// FP64: residual, then CG<double> until ||r|| <= eps ||b|| (fixed counts when
// `fixed` is given).  MIXED: iterative refinement -- float64 residual r, float32 CG on
// A e = r from e = 0 to inner_tol, x += e -- until ||r|| <= eps ||b||.
excmg_status solve_items_impl(const Ctx& c, std::vector<Item>& items, const excmg_options* o,
                              int nslots, const int* fixed, bool mixed);

// MIXED mode splits the systems: grids below kMixedMinNodes run the float64 CG,
// larger ones the float32-inner refinement.
excmg_status solve_items(const Ctx& c, std::vector<Item>& items, const excmg_options* o,
                         int nslots, const int* fixed) {
  if (o->precision != EXCMG_MIXED) return solve_items_impl(c, items, o, nslots, fixed, false);
  const long long minn = mixed_min(o);
  std::vector<Item> small, large;
  std::vector<int> where;
  for (auto& it : items) {
    const bool fp64 = it.nodes < minn || it.d64.direct;  // DSOLVE levels stay float64
    where.push_back(fp64 ? 0 : 1);
    (fp64 ? small : large).push_back(it);
  }
  Ctx cs = c;
  cs.defer = false;  // MIXED calls read their states per level
  excmg_status e = solve_items_impl(cs, small, o, nslots, nullptr, false);
  if (e != EXCMG_OK) return e;
  e = solve_items_impl(cs, large, o, nslots, nullptr, true);
  if (e != EXCMG_OK) return e;
  size_t a = 0, b = 0;
  for (size_t k = 0; k < items.size(); ++k) items[k] = where[k] ? large[b++] : small[a++];
  return EXCMG_OK;
}

excmg_status solve_items_impl(const Ctx& c, std::vector<Item>& items, const excmg_options* o,
                              int nslots, const int* fixed, bool mixed) {
  const int n = (int)items.size();
  std::vector<CGState> hs;
  std::vector<ResDesc> hr;
  long long tiles = 0, rtiles = 0;  // CG tiles, residual tiles
  // one residual launch serves every problem: they share its rows per thread (one
  // row unless all of them take more)
  int rows = kResRowsWide;
  for (auto& it : items) rows = std::min(rows, it.res.rows);
  for (int a = 0; a < n; ++a) {
    Item& it = items[a];
    it.iters = it.refs = 0;
    it.status = EXCMG_OK;
    it.relres = 0.0;
    if (it.res.rows != rows) {
      it.res.t = make_res_tiling(it.res.g, it.res.t.tz, rows);
      it.res.rows = rows;
    }
    ResDesc r = it.res;
    r.tile_begin = rtiles;
    if (!it.d64.direct) rtiles += r.t.count();  // DSOLVE levels form their own b
    it.d64.tile_begin = tiles;
    it.d32.tile_begin = tiles;
    tiles += it.d64.t.count();
    if (mixed) {
      r.r = it.d32.r;
      r.osy = it.d32.g.sy;  // the padded float32 layout
      r.osz = it.d32.g.sz;
      // the inner solve stops at inner_tol x its starting residual, or as soon as its
      // residual is below half the outer target (more float32 steps would be wasted:
      // EXCMG's initial guess is often within a few orders of the tolerance)
      r.tol_b2 = 0.25 * it.eps * it.eps;
      r.tol_r2 = o->inner_tol * o->inner_tol;
      r.fixed = 0;
      r.max_iter = o->max_iter;
    } else {
      r.r = it.d64.r;
      r.tol_b2 = it.eps * it.eps;
      r.tol_r2 = 0.0;
      r.fixed = fixed ? 1 : 0;
      r.max_iter = fixed ? fixed[a] : o->max_iter;
    }
    it.res = r;
    if (!it.d64.direct) hr.push_back(r);
  }
  if (n == 0) return EXCMG_OK;
  double nodes_sum = 0.0;
  for (auto& it : items) nodes_sum += (double)it.nodes;
  if (!mixed) {
    std::vector<CGDesc<double>> hd;
    std::vector<int> slots;
    for (auto& it : items) {
      hd.push_back(it.d64);
      slots.push_back(it.d64.slot);
    }
    const int grid = tiles_grid(tiles);
    const int nres = (int)hr.size();
    double res_nodes = 0.0;
    for (auto& it : items)
      if (!it.d64.direct) res_nodes += (double)it.nodes;
    CK(cudaMemcpyAsync(c.cgd(), hd.data(), sizeof(CGDesc<double>) * n, cudaMemcpyHostToDevice, c.s));
    if (nres > 0) {
      CK(cudaMemcpyAsync(c.resd(), hr.data(), sizeof(ResDesc) * nres, cudaMemcpyHostToDevice, c.s));
      CK(c.timed(EXCMG_K_RESIDUAL, res_nodes, [&] {
        return launch_residual(false, nres, c.resd(), rtiles, residual_grid(rtiles, rows), c.st(),
                               c.partials(), c.counters(), c.s, rows);
      }));
    }
    // DSOLVE levels: one direct solve each (their states are done with 0 steps, so the
    // CG engines skip them)
    int ndirect = 0;
    size_t dsm = 0;
    double dnodes = 0.0;
    for (auto& it : items)
      if (it.d64.direct) {
        ++ndirect;
        dsm = std::max(dsm, dsolve_smem(it.d64.g));
        dnodes += (double)it.nodes;
      }
    if (ndirect > 0)
      CK(c.timed(EXCMG_K_DSOLVE, dnodes, [&] { return launch_dsolve(n, c.cgd(), dsm, c.st(), c.s); }));
    excmg_status e = EXCMG_OK;
    if (ndirect < n) {
      e = cg_loop<double>(c, n, c.cgd(), tiles, grid, slots, nslots, o->chunk, hs, nodes_sum, hd);
    } else if (!c.defer) {
      e = read_states(c, nslots, hs);
    }
    if (e != EXCMG_OK) return e;
    if (c.defer) return EXCMG_OK;  // the caller reads every state at the end
    for (auto& it : items) {
      const CGState& S = hs[it.d64.slot];
      it.iters = S.iter;
      it.relres = S.bb > 0 ? sqrt(S.rr / S.bb) : 0.0;
      it.status = S.status;
    }
    return EXCMG_OK;
  }
  for (auto& it : items) {
    CK(cudaMemsetAsync(it.d32.x, 0, sizeof(float) * it.d32.g.nodes(), c.s));
    if (c.launches) *c.launches += 1;
    CK(launch_zero_far_faces(it.d32, c.s));
  }
  std::vector<int> cur(n);
  for (int a = 0; a < n; ++a) cur[a] = a;
  for (int pass = 0;; ++pass) {
    std::vector<ResDesc> rr;
    long long rt = 0;
    for (int a : cur) {
      ResDesc r = items[a].res;
      r.tile_begin = rt;
      rt += r.t.count();
      if (items[a].rhs_cache && !r.src) {
        if (pass == 0) {
          r.rhs_out = items[a].rhs_cache;  // keep 2 RHS(f) for the later passes
        } else {
          r.rhs2 = items[a].rhs_cache;     // r = LHS(u) - RHS(f) without recomputing RHS
          r.want_b = 0;                    // ||b|| is already in the state
        }
      }
      rr.push_back(r);
    }
    const int nr = (int)rr.size();
    double rnodes = 0.0;
    for (int a : cur) rnodes += (double)items[a].nodes;
    CK(cudaMemcpyAsync(c.resd(), rr.data(), sizeof(ResDesc) * nr, cudaMemcpyHostToDevice, c.s));
    CK(c.timed(EXCMG_K_RESIDUAL, rnodes, [&] {
      return launch_residual(true, nr, c.resd(), rt, residual_grid(rt, rows), c.st(), c.partials(),
                             c.counters(), c.s, rows);
    }));
    excmg_status e = read_states(c, nslots, hs);
    if (e != EXCMG_OK) return e;
    std::vector<int> next;
    for (int a : cur) {
      Item& it = items[a];
      const CGState& S = hs[it.d32.slot];
      it.relres = S.bb > 0 ? sqrt(S.rr / S.bb) : 0.0;
      if (S.status != EXCMG_OK) {
        it.status = S.status;
      } else if (!(S.rr <= it.eps * it.eps * S.bb)) {
        if (it.refs >= o->max_refine)
          it.status = EXCMG_ERR_NOT_CONVERGED;
        else
          next.push_back(a);
      }
    }
    if (next.empty()) return EXCMG_OK;
    std::vector<CGDesc<float>> fd;
    std::vector<int> fslots;
    long long ft = 0;
    for (int a : next) {
      CGDesc<float> d = items[a].d32;
      d.tile_begin = ft;
      ft += d.t.count();
      // scale r to unit root-mean-square over the interior unknowns
      const double rr = hs[d.slot].rr;
      const double nint = (double)(d.g.nx - 1) * (d.g.ny - 1) * (d.g.nz - 1);
      d.scale = (rr > 0.0 && nint > 0.0) ? 1.0 / sqrt(rr / nint) : 1.0;
      if (!isfinite(d.scale) || d.scale <= 0.0) d.scale = 1.0;
      d.fold_scale = 1;  // applied by the CG engine (cg_loop)
      fd.push_back(d);
      fslots.push_back(d.slot);
    }
    const int nf = (int)fd.size();
    const int fgrid = tiles_grid(ft);
    double fnodes = 0.0;
    for (int a : next) fnodes += (double)items[a].nodes;
    // tensor maps of r, p_a, p_b for the float32 engine that stages planes by tensor copies
    std::vector<TmapSet> maps(nf);
    bool maps_ok = true;
    for (int k = 0; k < nf && maps_ok; ++k)
      maps_ok = encode_plane_map(&maps[k].r, fd[k].r, fd[k].g) &&
                encode_plane_map(&maps[k].pa, fd[k].pa, fd[k].g) &&
                encode_plane_map(&maps[k].pb, fd[k].pb, fd[k].g);
    if (maps_ok) {
      CK(cudaMemcpyAsync(c.tmaps(), maps.data(), sizeof(TmapSet) * nf, cudaMemcpyHostToDevice, c.s));
      for (int k = 0; k < nf; ++k) fd[k].tm = c.tmaps() + k;
    }
    CK(cudaMemcpyAsync(c.cgf(), fd.data(), sizeof(CGDesc<float>) * nf, cudaMemcpyHostToDevice, c.s));
    e = cg_loop<float>(c, nf, c.cgf(), ft, fgrid, fslots, nslots, o->chunk, hs, fnodes, fd);
    if (e != EXCMG_OK) return e;
    std::vector<int> go;
    for (int a : next) {
      const CGState& S = hs[items[a].d32.slot];
      items[a].iters += S.iter;
      items[a].refs += 1;
      // an inner solve that hits max_iter is not fatal: refinement continues; a device
      // wait that ran out or a non-finite reduction ends this system's refinement
      if (S.status == EXCMG_ERR_TIMEOUT || S.status == EXCMG_ERR_NONFINITE)
        items[a].status = S.status;
      else
        go.push_back(a);
    }
    CK(c.timed(EXCMG_K_CORRECT, fnodes, [&] { return launch_add_correction(nf, c.cgf(), ft, fgrid, c.s); }));
    if (go.empty()) return EXCMG_OK;
    cur = go;
  }
}

// The engine class of a level grid g under options o: true when its CG runs in float32
// (MIXED inner solves; the DSOLVE levels 0 and 1 of a cascade are float64).
bool level_f32(const Grid3& g, bool dsolve_level, const excmg_options* o) {
  return o->precision == EXCMG_MIXED && g.nodes() >= mixed_min(o) && !dsolve_level;
}

// Launch shapes of a level: the caller's tile_z, else the tuned ones (options.autotune
// >= 0 and a cache entry), else the models.
struct Shapes {
  int res_tz, cg_tz, tma_tz, res_rows;
};
Shapes level_shapes(const Grid3& g, bool dsolve_level, const excmg_options* o) {
  Shapes sh;
  const int tz = choose_tz(g, persistent_grid(1LL << 40), o->tile_z);
  sh.cg_tz = tz;
  sh.tma_tz = o->tile_z > 0 ? tz : tma_slab_depth(tz);
  sh.res_rows = o->res_rows > 0 ? o->res_rows : res_rows_model(g);
  sh.res_tz = choose_res_tz(g, residual_grid(1LL << 40, sh.res_rows), o->tile_z, sh.res_rows);
  excmg_tuning t;
  if (o->tile_z == 0 && o->autotune >= 0 && tune_lookup(g, level_f32(g, dsolve_level, o), &t)) {
    // an entry's cg_tz is 0 where the single solve's engine for the grid is not tiled
    // (resident or cluster): the model's depth stays for the tiled engines of a batch
    if (t.res_tz > 0 && (o->res_rows == 0 || o->res_rows == t.res_rows)) {
      sh.res_tz = t.res_tz;
      if (t.res_rows > 0) sh.res_rows = t.res_rows;
    }
    if (t.cg_tz > 0) {
      if (level_f32(g, dsolve_level, o))
        sh.tma_tz = t.cg_tz;
      else
        sh.cg_tz = t.cg_tz;
    }
  }
  return sh;
}

Item make_item(Prob& p, int l, int slot, const excmg_options* o) {
  const Grid3 g = p.grid(l);
  const Shapes sh = level_shapes(g, p.cascade && l < 2, o);
  const int tz = sh.cg_tz;
  const Tiling t = make_tiling(g, tz);
  Item it;
  memset(&it, 0, sizeof(it));
  const double ratio = o->eps_ratio > 0 ? o->eps_ratio : 1.0;
  it.eps = (l < 2) ? o->eps_coarse : o->eps * std::pow(ratio, (double)((int)p.lv.size() - 1 - l));
  it.nodes = g.nodes();
  it.res = make_res(g, sh.res_tz, slot, p.level_u(l), p.fview(l), nullptr, sh.res_rows);
  it.res.forcing = o->rhs_norm == EXCMG_RHS_NORM_FORCING;
  CGDesc<double>& d = it.d64;
  d.g = g;
  d.A = it.res.A;
  d.t = t;
  d.slot = slot;
  d.x = p.level_u(l);
  d.r = reinterpret_cast<double*>(p.base + p.L.r);
  d.pa = reinterpret_cast<double*>(p.base + p.L.pa);
  d.pb = reinterpret_cast<double*>(p.base + p.L.pb);
  d.q = reinterpret_cast<double*>(p.base + p.L.q);
  d.direct = 0;  // set by the cascade for its DSOLVE levels
  d.forcing = it.res.forcing;
  const bool res = p.L.s1 > 0 && g.nodes() <= kResidentMaxNodes;
  d.s0 = res ? reinterpret_cast<double*>(p.base + p.L.s0) : nullptr;
  d.s1 = res ? reinterpret_cast<double*>(p.base + p.L.s1) : nullptr;
  d.aux = nullptr;
  CGDesc<float>& f = it.d32;
  f.g = padded_f32(g);  // float32 vectors: padded rows
  f.A = it.res.A;
  f.t = t;
  // the tensor-copy engine: slabs of whole tensor copies (unless the caller fixed tile_z)
  f.tt = make_tma_tiling(g, sh.tma_tz);
  f.slot = slot;
  f.x = reinterpret_cast<float*>(p.base + p.L.e32);
  f.r = reinterpret_cast<float*>(p.base + p.L.r32);
  f.pa = reinterpret_cast<float*>(p.base + p.L.pa32);
  f.pb = reinterpret_cast<float*>(p.base + p.L.pb32);
  f.q = reinterpret_cast<float*>(p.base + p.L.q32);
  f.s0 = f.s1 = nullptr;
  f.direct = 0;
  f.aux = p.level_u(l);
  f.aux_sy = g.sy;
  f.aux_sz = g.sz;
  f.scale = 1.0;
  f.fold_scale = 0;
  f.tm = nullptr;
  it.rhs_cache = p.L.rhs64 ? reinterpret_cast<double*>(p.base + p.L.rhs64) : nullptr;
  return it;
}

// The tuning pass of options.autotune = 1 (single solves): for every level from 2 up
// without a cache entry, time the residual at candidate slab depths and, where the
// level's CG engine is tiled (the persistent float64 engine above kResidentMaxNodes
// nodes, or the float32 tensor-copy engine), three CG steps at candidate slab depths;
// each candidate runs on the level's own solution array (overwritten by the solve
// afterwards: boundary = g, interior = 0 at every start) with CUDA events around every
// launch.  The fastest of each, and the model's choice with its time, go to the cache.
excmg_status tune_levels(Prob& p, const excmg_options* o, const Ctx& c0) {
  for (int l = 2; l < (int)p.lv.size(); ++l) {
    const Grid3 g = p.grid(l);
    const bool f32 = level_f32(g, false, o);
    if (tune_lookup(g, f32, nullptr)) continue;
    excmg_options om = *o;
    om.autotune = -1;
    om.profile = 1;
    om.history = nullptr;
    om.fixed_iters = nullptr;
    om.max_iter = 3;
    om.eps = 1e-300;
    om.max_refine = 1;
    om.inner_tol = 1e-30;
    const Shapes model = level_shapes(g, false, &om);
    const bool cg_tiled = f32 || g.nodes() > kResidentMaxNodes;
    // one run: residual + three CG steps at slab depth tz for both, the residual with
    // `rows` rows per thread; returns the mean residual launch and the mean CG step (ms)
    auto run = [&](int tz, int rows, double& res_ms, double& step_ms) -> excmg_status {
      excmg_options ot = om;
      ot.tile_z = tz;
      ot.res_rows = rows;
      Ctx c = c0;
      c.defer = false;
      c.hist = nullptr;
      long long launches = 0;
      c.launches = &launches;
      Prof prof;
      c.prof = &prof;
      c.level = l;
      CK(launch_boundary_init(g, p.gview(l), p.level_u(l), c.s));
      std::vector<Item> items{make_item(p, l, slot_of(0, l), &ot)};
      const int fixed = 3;
      excmg_status e = solve_items(c, items, &ot, state_slots(1), f32 ? nullptr : &fixed);
      if (e != EXCMG_OK) return e;
      CK(cudaStreamSynchronize(c.s));
      std::vector<CGState> hs;
      e = read_states(c, state_slots(1), hs);
      if (e != EXCMG_OK) return e;
      excmg_stats st;
      memset(&st, 0, sizeof(st));
      prof.report(&st, hs);
      res_ms = st.prof_launches[EXCMG_K_RESIDUAL] ? st.prof_ms[EXCMG_K_RESIDUAL] / st.prof_launches[EXCMG_K_RESIDUAL] : 0.0;
      const int k = f32 ? EXCMG_K_CG_F32 : EXCMG_K_CG_F64;
      const double steps = items[0].iters > 0 ? items[0].iters : 1;
      step_ms = st.prof_launches[k] ? st.prof_ms[k] / steps : 0.0;
      return EXCMG_OK;
    };
    excmg_tuning t;
    memset(&t, 0, sizeof(t));
    t.N[0] = g.nx;
    t.N[1] = g.ny;
    t.N[2] = g.nz;
    t.f32 = f32 ? 1 : 0;
    t.res_tz = t.res_tz_model = model.res_tz;
    t.res_rows = t.res_rows_model = model.res_rows;
    t.cg_tz = t.cg_tz_model = cg_tiled ? (f32 ? model.tma_tz : model.cg_tz) : 0;
    double best_res = 1e300, best_cg = 1e300;
    std::vector<int> cands = {2, 4, 6, 8, 10, 12, 16, 20, 24, 32, 48};
    for (int& c : cands)
      if (f32 && cg_tiled) c = tma_slab_depth(c);  // CG candidates for the tensor-copy engine
    cands.push_back(model.res_tz);
    cands.push_back(f32 ? model.tma_tz : model.cg_tz);
    std::sort(cands.begin(), cands.end());
    cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
    // the CG engine's depths are timed in the one-row runs; the residual's over both
    // row counts
    const int row_cands[] = {1, kResRowsWide};
    for (int rows : row_cands)
      for (int tz : cands) {
        if (tz < 1 || tz > g.nz + 1) continue;
        double rm = 0.0, sm = 0.0;
        excmg_status e = run(tz, rows, rm, sm);
        if (e != EXCMG_OK) return e;
        if (rm > 0 && rm < best_res) {
          best_res = rm;
          t.res_tz = tz;
          t.res_rows = rows;
        }
        if (tz == model.res_tz && rows == model.res_rows) t.res_ms_model = rm;
        if (rows == 1 && cg_tiled && sm > 0) {
          if (sm < best_cg) {
            best_cg = sm;
            t.cg_tz = tz;
          }
          if (tz == t.cg_tz_model) t.cg_ms_model = sm;
        }
      }
    t.res_ms = best_res < 1e300 ? best_res : 0.0;
    t.cg_ms = best_cg < 1e300 ? best_cg : 0.0;
    if (t.res_ms_model == 0.0) t.res_ms_model = t.res_ms;
    tune_store(g, f32, t);
  }
  return EXCMG_OK;
}

// The level loop of Algorithm 1 for one or more problems (a single solve is nprob = 1).
// Problems are aligned on their finest level: in phase s, problem i works on level
// s - (maxL - L_i).
excmg_status run_excmg(std::vector<Prob>& P, const excmg_options* o, double* u_tilde,
                       excmg_stats* stats, const Ctx& c0) {
  const int np = (int)P.size();
  long long launches = 0;
  Ctx c = c0;
  c.launches = &launches;
  Prof prof;
  if (o->profile && np == 1) c.prof = &prof;
  // one CG state per (problem, level); an FP64 solve reads them all once, at the end
  long long max_count = o->max_iter;
  if (o->fixed_iters)
    for (size_t l = 0; l < P[0].lv.size(); ++l) max_count = std::max<long long>(max_count, o->fixed_iters[l]);
  c.persistent_ok = (long long)kMaxGrid * (2 * max_count + 4) < (1LL << 32);
  c.set_waits(o);
  c.defer = o->precision == EXCMG_FP64;
  struct Report {
    excmg_stats* st;
    long long* n;
    ~Report() {
      if (st) st[0].launches = *n;
    }
  } report{stats, &launches};
  int maxL = 0;
  for (auto& p : P) maxL = std::max(maxL, (int)p.lv.size());
  CK(cudaMemsetAsync(c.counters(), 0, sizeof(unsigned) * np, c.s));
  if (o->autotune == 1 && np == 1 && !o->fixed_iters) {
    const excmg_status e = tune_levels(P[0], o, c);
    if (e != EXCMG_OK) return e;
  }
  excmg_status result = EXCMG_OK;
  if (stats) {
    for (int i = 0; i < np; ++i) {
      memset(&stats[i], 0, sizeof(excmg_stats));
      stats[i].levels = (int)P[i].lv.size();
      for (int l = 0; l < stats[i].levels; ++l) {
        stats[i].N[l][0] = P[i].lv[l].nx;
        stats[i].N[l][1] = P[i].lv[l].ny;
        stats[i].N[l][2] = P[i].lv[l].nz;
      }
    }
  }
  std::vector<ProlongDesc> hp(np);
  // Levels 0 and 1 are independent (each DSOLVE starts from the Dirichlet data alone): when
  // both take the direct solve, a problem's level 1 joins the phase of its level 0, and
  // one k_dsolve launch serves both.
  auto direct_level = [&](const Prob& p, int l) {
    return l < 2 && l < (int)p.lv.size() && o->dsolve == EXCMG_DSOLVE_DIRECT && dsolve_fits(p.grid(l));
  };
  std::vector<char> level1_early(np, 0);
  for (int phase = 0; phase < maxL; ++phase) {
    if (np == 1) c.level = phase;
    std::vector<int> act, lev;
    for (int i = 0; i < np; ++i) {
      const int l = phase - (maxL - (int)P[i].lv.size());
      if (l < 0 || (l == 1 && level1_early[i])) continue;
      act.push_back(i);
      lev.push_back(l);
      if (l == 0 && direct_level(P[i], 0) && direct_level(P[i], 1)) {
        act.push_back(i);
        lev.push_back(1);
        level1_early[i] = 1;
      }
    }
    if (act.empty()) continue;
    const int na = (int)act.size();
    // 1. initial guess: zero inside (levels 0, 1) or w_h = EXP_finite(u_2h, u_4h)
    int npro = 0;
    long long pblocks = 0;
    double pnodes = 0.0;
    for (int a = 0; a < na; ++a) {
      Prob& p = P[act[a]];
      const int l = lev[a];
      const Grid3 g = p.grid(l);
      if (l < 2) {
        // DSOLVE by the direct solve writes the boundary itself (and forms b)
        if (!direct_level(p, l))
          CK(c.timed(EXCMG_K_INIT, (double)g.nodes(), [&] { return launch_boundary_init(g, p.gview(l), p.level_u(l), c.s); }));
      } else {
        ProlongDesc d;
        d.g = g;
        d.u2h = p.level_u(l - 1);
        d.u4h = p.level_u(l - 2);
        d.gb = p.gview(l);
        d.w = p.level_u(l);
        d.nbx = (g.nx + 31) / 32;
        d.nby = g.ny / 8;
        d.nbz = g.nz / 8;
        d.block_begin = pblocks;
        pblocks += (long long)d.nbx * d.nby * d.nbz;
        pnodes += (double)g.nodes();
        hp[npro++] = d;
      }
    }
    if (npro > 0) {
      CK(cudaMemcpyAsync(c.prold(), hp.data(), sizeof(ProlongDesc) * npro, cudaMemcpyHostToDevice, c.s));
      if (o->prolong == EXCMG_PROLONG_QUARTIC) {
        CK(c.timed(EXCMG_K_EXP_FINITE, pnodes, [&] { return launch_exp_finite(npro, c.prold(), pblocks, c.s); }));
      } else {
        const int points = o->prolong == EXCMG_PROLONG_QUADRATIC ? 3 : 2;
        CK(c.timed(EXCMG_K_PROLONG_CMP, pnodes,
                   [&] { return launch_prolong_cmp(points, npro, c.prold(), pblocks, c.s); }));
      }
    }
    // 2. CG (FP64) or refinement (MIXED) on every active problem's level
    std::vector<Item> items;
    std::vector<int> fixed;
    for (int a = 0; a < na; ++a) {
      items.push_back(make_item(P[act[a]], lev[a], slot_of(act[a], lev[a]), o));
      // DSOLVE (levels 0 and 1 of the cascade): the direct solve when the grid fits
      CGDesc<double>& d = items.back().d64;
      d.direct = (lev[a] < 2 && o->dsolve == EXCMG_DSOLVE_DIRECT && dsolve_fits(d.g)) ? 1 : 0;
      if (d.direct) {
        d.f = P[act[a]].fview(lev[a]);
        d.gb = P[act[a]].gview(lev[a]);
      }
      if (o->fixed_iters) fixed.push_back(o->fixed_iters[lev[a]]);
      if (c.hist && act[a] == 0 && lev[a] == (int)P[0].lv.size() - 1) {  // options.history
        Item& it = items.back();
        it.res.hist = it.d64.hist = c.hist;
        it.res.hist_len = it.d64.hist_len = o->history_len;
      }
    }
    excmg_status e = solve_items(c, items, o, state_slots(np), o->fixed_iters ? fixed.data() : nullptr);
    if (e != EXCMG_OK) return e;
    if (c.defer) continue;
    for (int a = 0; a < na; ++a) {
      const Item& it = items[a];
      if (stats) {
        stats[act[a]].iters[lev[a]] = it.iters;
        stats[act[a]].refinements[lev[a]] = it.refs;
        stats[act[a]].relres[lev[a]] = it.relres;
      }
      if (it.status != EXCMG_OK && result == EXCMG_OK) result = (excmg_status)it.status;
    }
    if (result == EXCMG_ERR_NONFINITE) return result;
  }
  if (u_tilde && np == 1) {
    Prob& p = P[0];
    const int l = (int)p.lv.size() - 1;
    CK(c.timed(EXCMG_K_EXP_TRUE, (double)p.grid(l).nodes(), [&] {
      return launch_exp_true(p.grid(l), p.level_u(l), p.level_u(l - 1), u_tilde, c.s);
    }));
  }
  CK(cudaStreamSynchronize(c.s));
  CK(cudaGetLastError());
  std::vector<CGState> hs;
  if (c.defer || c.prof) {
    excmg_status e = read_states(c, state_slots(np), hs);
    if (e != EXCMG_OK) return e;
  }
  if (c.defer) {
    for (int i = 0; i < np; ++i)
      for (int l = 0; l < (int)P[i].lv.size(); ++l) {
        const CGState& S = hs[slot_of(i, l)];
        if (stats) {
          stats[i].iters[l] = S.iter;
          stats[i].relres[l] = S.bb > 0 ? sqrt(S.rr / S.bb) : 0.0;
        }
        if (S.status != EXCMG_OK && (result == EXCMG_OK || S.status == EXCMG_ERR_NONFINITE))
          result = (excmg_status)S.status;
      }
  }
  if (c.prof) prof.report(stats, hs);
  if (c.defer && c.hist) {
    const excmg_status e = copy_history(c, o, hs[slot_of(0, (int)P[0].lv.size() - 1)]);
    if (e != EXCMG_OK) return e;
  }
  return result;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }


// Memory the current device's kernels may read: device or managed memory, or
// page-locked host memory mapped at the same address (read over the host link).
bool device_readable(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

bool device_memory(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

void excmg_default_options(excmg_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = EXCMG_FP64;
  o->eps = 1e-9;
  o->eps_coarse = 1e-12;
  o->max_iter = 100000;
  o->inner_tol = 1e-4;
  o->max_refine = 50;
  o->fixed_iters = nullptr;
  o->tile_z = 0;
  o->chunk = 0;
  o->mixed_min_nodes = 0;
  o->profile = 0;
  o->dsolve = EXCMG_DSOLVE_DIRECT;
  o->eps_ratio = 1.0;
  o->prolong = EXCMG_PROLONG_QUARTIC;
  o->rhs_norm = EXCMG_RHS_NORM_LIFT;
  o->wait_timeout_ms = 0.0;
  o->test_phantom_blocks = 0;
  o->autotune = 0;
  o->res_rows = 0;
}

int excmg_tuning_entries(excmg_tuning* out, int max) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  int n = 0;
  for (const auto& kv : g_tune) {
    if (out && n < max) out[n] = kv.second;
    ++n;
  }
  return n;
}

void excmg_tuning_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
}

const char* excmg_status_string(excmg_status s) {
  switch (s) {
    case EXCMG_OK: return "EXCMG_OK";
    case EXCMG_ERR_INVALID_ARG: return "EXCMG_ERR_INVALID_ARG";
    case EXCMG_ERR_NOT_CONVERGED: return "EXCMG_ERR_NOT_CONVERGED";
    case EXCMG_ERR_CUDA: return "EXCMG_ERR_CUDA";
    case EXCMG_ERR_NONFINITE: return "EXCMG_ERR_NONFINITE";
    case EXCMG_ERR_TIMEOUT: return "EXCMG_ERR_TIMEOUT";
    case EXCMG_ERR_WORKSPACE: return "EXCMG_ERR_WORKSPACE";
  }
  return "EXCMG_UNKNOWN_STATUS";
}

int excmg_num_levels(const excmg_grid* grid) {
  const auto lv = levels_of(grid);
  return lv.empty() ? -1 : (int)lv.size();
}

size_t excmg_workspace_size(const excmg_grid* grid, const excmg_options* opt) {
  const auto lv = levels_of(grid);
  if (lv.empty() || !options_ok(opt)) return 0;
  return header_layout(1).bytes + prob_layout(lv, opt->precision == EXCMG_MIXED, false, mixed_min(opt)).bytes +
         hist_bytes(opt);
}

size_t excmg_workspace_size_batched(int nprob, const excmg_grid* grids, const excmg_options* opt) {
  if (nprob < 1 || nprob > kMaxProb || !grids || !options_ok(opt) || opt->fixed_iters || opt->history)
    return 0;
  size_t total = header_layout(nprob).bytes;
  for (int i = 0; i < nprob; ++i) {
    const auto lv = levels_of(&grids[i]);
    if (lv.empty()) return 0;
    total += prob_layout(lv, opt->precision == EXCMG_MIXED, false, mixed_min(opt)).bytes;
  }
  return total;
}

excmg_status excmg_solve(const excmg_grid* grid, const double* f, const double* g,
                         const excmg_options* opt, double* u, double* u_tilde, void* ws,
                         size_t ws_bytes, excmg_stats* stats, void* stream) {
  const auto lv = levels_of(grid);
  if (lv.empty() || !options_ok(opt) || !f || !g || !u) return EXCMG_ERR_INVALID_ARG;
  if (!aligned(f, 8) || !aligned(g, 8) || !aligned(u, 8) || (u_tilde && !aligned(u_tilde, 8)))
    return EXCMG_ERR_INVALID_ARG;
  if (u == f || u == g || (u_tilde && (u_tilde == u || u_tilde == f || u_tilde == g)))
    return EXCMG_ERR_INVALID_ARG;
  if (opt->fixed_iters)
    for (size_t l = 0; l < lv.size(); ++l)
      if (opt->fixed_iters[l] < 0) return EXCMG_ERR_INVALID_ARG;
  const size_t need = excmg_workspace_size(grid, opt);
  if (!ws || ws_bytes < need || !aligned(ws, kAlign)) return EXCMG_ERR_WORKSPACE;
  // where the arrays live (a driver query, after the plain argument checks)
  if (!device_readable(f) || !device_readable(g) || !device_memory(u) ||
      (u_tilde && !device_memory(u_tilde)))
    return EXCMG_ERR_INVALID_ARG;
  Ctx c;
  c.ws = static_cast<char*>(ws);
  c.H = header_layout(1);
  c.s = static_cast<cudaStream_t>(stream);
  std::vector<Prob> P(1);
  P[0].lv = lv;
  P[0].gr = *grid;
  P[0].f = f;
  P[0].g = g;
  P[0].u = u;
  P[0].base = c.ws + c.H.bytes;
  P[0].L = prob_layout(lv, opt->precision == EXCMG_MIXED, false, mixed_min(opt));
  if (opt->history) c.hist = reinterpret_cast<double*>(P[0].base + P[0].L.bytes);
  return run_excmg(P, opt, u_tilde, stats, c);
}

excmg_status excmg_solve_batched(int nprob, const excmg_grid* grids, const double* const* f,
                                 const double* const* g, const excmg_options* opt,
                                 double* const* u, void* ws, size_t ws_bytes,
                                 excmg_stats* stats, void* stream) {
  if (nprob < 1 || nprob > kMaxProb || !grids || !f || !g || !u || !options_ok(opt) ||
      opt->fixed_iters)
    return EXCMG_ERR_INVALID_ARG;
  const size_t need = excmg_workspace_size_batched(nprob, grids, opt);
  if (need == 0) return EXCMG_ERR_INVALID_ARG;
  if (!ws || ws_bytes < need || !aligned(ws, kAlign)) return EXCMG_ERR_WORKSPACE;
  Ctx c;
  c.ws = static_cast<char*>(ws);
  c.H = header_layout(nprob);
  c.s = static_cast<cudaStream_t>(stream);
  std::vector<Prob> P(nprob);
  char* base = c.ws + c.H.bytes;
  for (int i = 0; i < nprob; ++i) {
    P[i].lv = levels_of(&grids[i]);
    if (!f[i] || !g[i] || !u[i] || !aligned(f[i], 8) || !aligned(g[i], 8) || !aligned(u[i], 8))
      return EXCMG_ERR_INVALID_ARG;
    P[i].gr = grids[i];
    P[i].f = f[i];
    P[i].g = g[i];
    P[i].u = u[i];
    P[i].base = base;
    P[i].L = prob_layout(P[i].lv, opt->precision == EXCMG_MIXED, false, mixed_min(opt));
    base += P[i].L.bytes;
  }
  // Problems whose finest grid has kBatchSoloNodes nodes or more run one after another,
  // each on the whole GPU with a single solve's engines (the shared-memory CG up to 2^20
  // nodes, every SM above); the others share the launches of one batch, where their CG
  // runs as a team of blocks per problem.  Each problem keeps its own workspace region;
  // the runs share the header's states in stream order.
  std::vector<int> solo, team;
  for (int i = 0; i < nprob; ++i) {
    const Level& fl = P[i].lv.back();
    const long long nodes = (long long)(fl.nx + 1) * (fl.ny + 1) * (fl.nz + 1);
    (nodes >= kBatchSoloNodes ? solo : team).push_back(i);
  }
  if (solo.empty()) return run_excmg(P, opt, nullptr, stats, c);
  excmg_status result = EXCMG_OK;
  long long launches = 0;
  auto run_part = [&](const std::vector<int>& idx) -> excmg_status {
    std::vector<Prob> part;
    for (int i : idx) part.push_back(P[i]);
    std::vector<excmg_stats> st(idx.size());
    const excmg_status e = run_excmg(part, opt, nullptr, stats ? st.data() : nullptr, c);
    if (stats) {
      launches += st[0].launches;
      for (size_t k = 0; k < idx.size(); ++k) {
        stats[idx[k]] = st[k];
        stats[idx[k]].launches = 0;
      }
    }
    return e;
  };
  for (int i : solo) {
    const excmg_status e = run_part({i});
    if (e != EXCMG_OK && e != EXCMG_ERR_NOT_CONVERGED) return e;
    if (e != EXCMG_OK) result = e;
  }
  if (!team.empty()) {
    const excmg_status e = run_part(team);
    if (e != EXCMG_OK && e != EXCMG_ERR_NOT_CONVERGED) return e;
    if (e != EXCMG_OK) result = e;
  }
  if (stats) stats[0].launches = launches;
  return result;
}

excmg_status excmg_exp_finite(const excmg_grid* grid, const double* u2h, const double* u4h,
                              const double* g, double* w, void* stream) {
  if (!grid || !u2h || !u4h || !w) return EXCMG_ERR_INVALID_ARG;
  if (grid->Nx % 8 || grid->Ny % 8 || grid->Nz % 8 || grid->Nx < 8 || grid->Ny < 8 || grid->Nz < 8)
    return EXCMG_ERR_INVALID_ARG;
  if (!(grid->Lx > 0) || !(grid->Ly > 0) || !(grid->Lz > 0)) return EXCMG_ERR_INVALID_ARG;
  const Grid3 gg = make_grid(grid->Nx, grid->Ny, grid->Nz, grid->Lx, grid->Ly, grid->Lz);
  ProlongDesc d;
  d.g = gg;
  d.u2h = u2h;
  d.u4h = u4h;
  d.gb = View{g, 1, gg.sy, gg.sz};  // p == NULL: keep the interpolated boundary
  d.w = w;
  d.nbx = (gg.nx + 31) / 32;
  d.nby = gg.ny / 8;
  d.nbz = gg.nz / 8;
  d.block_begin = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(launch_exp_finite_one(d, s));
  CK(cudaStreamSynchronize(s));
  return EXCMG_OK;
}

excmg_status excmg_exp_true(const excmg_grid* grid, const double* uh, const double* u2h,
                            double* ut, void* stream) {
  if (!grid || !uh || !u2h || !ut) return EXCMG_ERR_INVALID_ARG;
  if (grid->Nx % 2 || grid->Ny % 2 || grid->Nz % 2 || grid->Nx < 2 || grid->Ny < 2 || grid->Nz < 2)
    return EXCMG_ERR_INVALID_ARG;
  if (!(grid->Lx > 0) || !(grid->Ly > 0) || !(grid->Lz > 0)) return EXCMG_ERR_INVALID_ARG;
  const Grid3 gg = make_grid(grid->Nx, grid->Ny, grid->Nz, grid->Lx, grid->Ly, grid->Lz);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(launch_exp_true(gg, uh, u2h, ut, s));
  CK(cudaStreamSynchronize(s));
  return EXCMG_OK;
}

excmg_status excmg_grad(const excmg_grid* grid, const double* u, double* ux, double* uy,
                        double* uz, void* stream) {
  if (!grid || !u || !ux || !uy || !uz) return EXCMG_ERR_INVALID_ARG;
  if (grid->Nx < 4 || grid->Ny < 4 || grid->Nz < 4) return EXCMG_ERR_INVALID_ARG;
  if (!(grid->Lx > 0) || !(grid->Ly > 0) || !(grid->Lz > 0)) return EXCMG_ERR_INVALID_ARG;
  if (ux == u || uy == u || uz == u || ux == uy || ux == uz || uy == uz) return EXCMG_ERR_INVALID_ARG;
  const Grid3 gg = make_grid(grid->Nx, grid->Ny, grid->Nz, grid->Lx, grid->Ly, grid->Lz);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(launch_grad(gg, u, ux, uy, uz, s));
  CK(cudaStreamSynchronize(s));
  return EXCMG_OK;
}

size_t excmg_workspace_size_level(const excmg_grid* grid, const excmg_options* opt) {
  const auto lv = single_level(grid);
  if (lv.empty() || !options_ok(opt)) return 0;
  return header_layout(1).bytes + prob_layout(lv, opt->precision == EXCMG_MIXED, false, mixed_min(opt)).bytes +
         hist_bytes(opt);
}

excmg_status excmg_cg(const excmg_grid* grid, const double* f, const excmg_options* opt,
                      double* u, void* ws, size_t ws_bytes, excmg_stats* stats, void* stream) {
  const auto lv = single_level(grid);
  if (lv.empty() || !options_ok(opt) || !f || !u || u == f) return EXCMG_ERR_INVALID_ARG;
  if (opt->fixed_iters && opt->fixed_iters[0] < 0) return EXCMG_ERR_INVALID_ARG;
  const size_t need = excmg_workspace_size_level(grid, opt);
  if (!ws || ws_bytes < need || !aligned(ws, kAlign)) return EXCMG_ERR_WORKSPACE;
  Ctx c;
  c.ws = static_cast<char*>(ws);
  c.H = header_layout(1);
  c.s = static_cast<cudaStream_t>(stream);
  Prob p;
  p.cascade = false;
  p.lv = lv;
  p.gr = *grid;
  p.f = f;
  p.g = u;
  p.u = u;
  p.base = c.ws + c.H.bytes;
  p.L = prob_layout(lv, opt->precision == EXCMG_MIXED, false, mixed_min(opt));
  const int l = (int)lv.size() - 1;
  std::vector<Item> items{make_item(p, l, 0, opt)};
  items[0].eps = opt->eps;
  if (opt->history) {
    c.hist = reinterpret_cast<double*>(p.base + p.L.bytes);
    items[0].res.hist = items[0].d64.hist = c.hist;
    items[0].res.hist_len = items[0].d64.hist_len = opt->history_len;
  }
  long long launches = 0;
  Prof prof;
  c.launches = &launches;
  c.level = 0;
  if (opt->profile) c.prof = &prof;
  const long long max_count = opt->fixed_iters ? std::max(opt->max_iter, opt->fixed_iters[0]) : opt->max_iter;
  c.persistent_ok = (long long)kMaxGrid * (2 * max_count + 4) < (1LL << 32);
  c.set_waits(opt);
  CK(cudaMemsetAsync(c.counters(), 0, sizeof(unsigned), c.s));
  excmg_status e = solve_items(c, items, opt, 1, opt->fixed_iters);
  if (e != EXCMG_OK) return e;
  CK(cudaStreamSynchronize(c.s));
  std::vector<CGState> hs;
  e = read_states(c, 1, hs);
  if (e != EXCMG_OK) return e;
  e = copy_history(c, opt, hs[0]);
  if (e != EXCMG_OK) return e;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->launches = launches;
    prof.report(stats, hs);
    stats->levels = 1;
    stats->N[0][0] = lv[l].nx;
    stats->N[0][1] = lv[l].ny;
    stats->N[0][2] = lv[l].nz;
    stats->iters[0] = items[0].iters;
    stats->refinements[0] = items[0].refs;
    stats->relres[0] = items[0].relres;
  }
  return (excmg_status)items[0].status;
}

excmg_status excmg_residual(const excmg_grid* grid, const double* f, const double* u, double* r,
                            double* rnorm, double* bnorm, void* ws, size_t ws_bytes,
                            void* stream) {
  const auto lv = single_level(grid);
  if (lv.empty() || !f || !u || !r || r == u || r == f) return EXCMG_ERR_INVALID_ARG;
  excmg_options o;
  excmg_default_options(&o);
  const size_t need = excmg_workspace_size_level(grid, &o);
  if (!ws || ws_bytes < need || !aligned(ws, kAlign)) return EXCMG_ERR_WORKSPACE;
  Ctx c;
  c.ws = static_cast<char*>(ws);
  c.H = header_layout(1);
  c.s = static_cast<cudaStream_t>(stream);
  const Grid3 g = make_grid(grid->Nx, grid->Ny, grid->Nz, grid->Lx, grid->Ly, grid->Lz);
  const int rows = res_rows_model(g);
  ResDesc d = make_res(g, 0, 0, u, View{f, 1, g.sy, g.sz}, nullptr, rows);
  d.r = r;
  CK(cudaMemsetAsync(c.counters(), 0, sizeof(unsigned), c.s));
  CK(cudaMemcpyAsync(c.resd(), &d, sizeof(d), cudaMemcpyHostToDevice, c.s));
  CK(launch_residual(false, 1, c.resd(), d.t.count(), residual_grid(d.t.count(), rows), c.st(),
                     c.partials(), c.counters(), c.s, rows));
  std::vector<CGState> hs;
  excmg_status e = read_states(c, 1, hs);
  if (e != EXCMG_OK) return e;
  if (rnorm) *rnorm = sqrt(hs[0].rr);
  if (bnorm) *bnorm = sqrt(hs[0].bb);
  return EXCMG_OK;
}

size_t excmg_workspace_size_adjoint(const excmg_grid* grid, const excmg_options* opt) {
  if (!grid || !options_ok(opt) || opt->fixed_iters) return 0;
  if (grid->Nx < 2 || grid->Ny < 2 || grid->Nz < 2) return 0;
  if (!(grid->Lx > 0) || !(grid->Ly > 0) || !(grid->Lz > 0)) return 0;
  const long long nf = (long long)(grid->Nx + 1) * (grid->Ny + 1) * (grid->Nz + 1);
  std::vector<Level> lv{{grid->Nx, grid->Ny, grid->Nz}};
  // lambda (float64) + the CG vectors of one level
  return header_layout(1).bytes + align_up(sizeof(double) * nf) +
         prob_layout(lv, opt->precision == EXCMG_MIXED, false, mixed_min(opt)).bytes;
}

excmg_status excmg_adjoint(const excmg_grid* grid, const double* dLdu, const excmg_options* opt,
                           double* dLdf, double* dLdg, void* ws, size_t ws_bytes,
                           excmg_stats* stats, void* stream) {
  if (!grid || !dLdu || !dLdf || !dLdg || !options_ok(opt) || opt->fixed_iters)
    return EXCMG_ERR_INVALID_ARG;
  if (dLdf == dLdg || dLdf == dLdu || dLdg == dLdu) return EXCMG_ERR_INVALID_ARG;
  const size_t need = excmg_workspace_size_adjoint(grid, opt);
  if (need == 0) return EXCMG_ERR_INVALID_ARG;
  if (!ws || ws_bytes < need || !aligned(ws, kAlign)) return EXCMG_ERR_WORKSPACE;
  Ctx c;
  c.ws = static_cast<char*>(ws);
  c.H = header_layout(1);
  c.s = static_cast<cudaStream_t>(stream);
  const Grid3 g = make_grid(grid->Nx, grid->Ny, grid->Nz, grid->Lx, grid->Ly, grid->Lz);
  const long long nf = g.nodes();
  // lambda lives in front of the level vectors; it starts at zero (zero boundary too)
  double* lam = reinterpret_cast<double*>(c.ws + c.H.bytes);
  Prob p;
  p.cascade = false;
  p.lv = std::vector<Level>{{grid->Nx, grid->Ny, grid->Nz}};
  p.gr = *grid;
  p.f = nullptr;
  p.g = nullptr;
  p.u = lam;
  p.base = c.ws + c.H.bytes + align_up(sizeof(double) * nf);
  p.L = prob_layout(p.lv, opt->precision == EXCMG_MIXED, false, mixed_min(opt));
  c.persistent_ok = (long long)kMaxGrid * (2LL * opt->max_iter + 4) < (1LL << 32);
  c.set_waits(opt);
  CK(cudaMemsetAsync(c.counters(), 0, sizeof(unsigned), c.s));
  CK(cudaMemsetAsync(lam, 0, sizeof(double) * nf, c.s));
  Item it = make_item(p, 0, 0, opt);
  it.eps = opt->eps;
  // b = s = (dL/du) on interior nodes: r = LHS(lambda) + s = s - A lambda
  it.res.f = View{nullptr, 0, 0, 0};
  it.res.src = dLdu;
  std::vector<Item> items{it};
  excmg_status e = solve_items(c, items, opt, 1, nullptr);
  if (e != EXCMG_OK) return e;
  CK(launch_adjoint_finish(g, it.res.A, lam, dLdu, dLdf, dLdg, c.s));
  CK(cudaStreamSynchronize(c.s));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->levels = 1;
    stats->N[0][0] = g.nx;
    stats->N[0][1] = g.ny;
    stats->N[0][2] = g.nz;
    stats->iters[0] = items[0].iters;
    stats->refinements[0] = items[0].refs;
    stats->relres[0] = items[0].relres;
  }
  return (excmg_status)items[0].status;
}

}  // extern "C"
