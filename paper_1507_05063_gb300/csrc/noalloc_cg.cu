// excmg_cg_noalloc: the one-grid float64 CG of excmg_cg with its scratch memory built
// into the library, for callers that cannot allocate device memory themselves.
//
// Who needs it: code that must not call cudaMalloc after start-up -- a host application
// or framework that owns every byte of device memory through its own pool, a loop that
// cannot afford cudaMalloc's implicit device synchronisation, or a language binding with
// no way to reach a CUDA allocator.  Such a caller passes only its inputs and outputs.
//
// The scratch is one file-scope device array of EXCMG_NOALLOC_SCRATCH_BYTES (16 MiB).
// Every GPU that loads the library holds it until the process exits.  It is shared by
// every call: a call clears what must start at zero (the reduction counters) and
// overwrites the rest, so results never depend on a previous call, but two calls whose
// work overlaps on the GPU (different streams, or different host threads) race on it.
//
// In host code the array's name is only a host-side stand-in; the device address is
// looked up with cudaGetSymbolAddress the first time the entry point runs on a device
// (with that device current) and cached per device.
#include <math.h>
#include <string.h>

#include <mutex>

#include "excmg_internal.cuh"

// The built-in scratch: file scope, one copy on every device that loads the library.
static __device__ __align__(256) unsigned char g_noalloc_scratch[EXCMG_NOALLOC_SCRATCH_BYTES];

namespace {

using namespace excmg;

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

constexpr size_t kA = 256;
size_t up(size_t v) { return (v + kA - 1) / kA * kA; }

// Scratch layout: state | counter | partials (one value per block) | the two
// descriptors | r, p_a, p_b, q (float64, one node array each).
struct Layout {
  size_t st, counters, partials, resd, cgd, r, pa, pb, q, bytes;
};

Layout layout(long long nodes) {
  Layout L;
  size_t o = 0;
  L.st = o;
  o = up(o + sizeof(CGState));
  L.counters = o;
  o = up(o + sizeof(unsigned));
  L.partials = o;
  o = up(o + 2 * sizeof(double) * kMaxGrid);
  L.resd = o;
  o = up(o + sizeof(ResDesc));
  L.cgd = o;
  o = up(o + sizeof(CGDesc<double>));
  L.r = o;
  o = up(o + sizeof(double) * nodes);
  L.pa = o;
  o = up(o + sizeof(double) * nodes);
  L.pb = o;
  o = up(o + sizeof(double) * nodes);
  L.q = o;
  o = up(o + sizeof(double) * nodes);
  L.bytes = o;
  return L;
}

// Device address of the built-in scratch for the current device (set up once).
excmg_status scratch_address(char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EXCMG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return EXCMG_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<char*>(g_noalloc_ptr[dev]);
  return EXCMG_OK;
}

#define CKN(call)                                   \
  do {                                              \
    if ((call) != cudaSuccess) return EXCMG_ERR_CUDA; \
  } while (0)

}  // namespace

extern "C" excmg_status excmg_cg_noalloc(const excmg_grid* grid, const double* f,
                                         const excmg_options* opt, double* u,
                                         excmg_stats* stats, void* stream) {
  if (!grid || !f || !u || !opt || u == f) return EXCMG_ERR_INVALID_ARG;
  if (!(grid->Lx > 0) || !(grid->Ly > 0) || !(grid->Lz > 0)) return EXCMG_ERR_INVALID_ARG;
  if (grid->Nx < 2 || grid->Ny < 2 || grid->Nz < 2) return EXCMG_ERR_INVALID_ARG;
  if (!options_valid(opt) || opt->precision != EXCMG_FP64) return EXCMG_ERR_INVALID_ARG;
  // the residual history and the per-launch timing need host-side buffers and events
  // this entry point does not keep: refused rather than silently left unfilled
  if (opt->history || opt->profile) return EXCMG_ERR_INVALID_ARG;
  if (opt->fixed_iters && opt->fixed_iters[0] < 0) return EXCMG_ERR_INVALID_ARG;
  const long long nodes = (long long)(grid->Nx + 1) * (grid->Ny + 1) * (grid->Nz + 1);
  if (nodes > (1LL << 40)) return EXCMG_ERR_INVALID_ARG;
  const Layout L = layout(nodes);
  if (L.bytes > (size_t)EXCMG_NOALLOC_SCRATCH_BYTES) return EXCMG_ERR_WORKSPACE;  // grid too large

  char* base = nullptr;
  const excmg_status se = scratch_address(&base);
  if (se != EXCMG_OK) return se;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CGState* st = reinterpret_cast<CGState*>(base + L.st);
  unsigned* counters = reinterpret_cast<unsigned*>(base + L.counters);
  double* partials = reinterpret_cast<double*>(base + L.partials);

  const Grid3 g = make_grid(grid->Nx, grid->Ny, grid->Nz, grid->Lx, grid->Ly, grid->Lz);
  const Tiling t = make_tiling(g, choose_tz(g, persistent_grid(1LL << 40), opt->tile_z));
  const int nblk = persistent_grid(t.count());
  ResDesc rd;
  memset(&rd, 0, sizeof(rd));
  rd.g = g;
  rd.A = make_coef(g);
  rd.rows = 1;
  rd.t = make_res_tiling(g, choose_res_tz(g, residual_grid(1LL << 40, 1), opt->tile_z, 1), 1);
  rd.slot = 0;
  rd.u = u;
  rd.f = View{f, 1, g.sy, g.sz};
  rd.src = nullptr;
  rd.r = base + L.r;
  rd.want_b = 1;
  rd.forcing = opt->rhs_norm == EXCMG_RHS_NORM_FORCING;
  rd.fixed = opt->fixed_iters ? 1 : 0;
  rd.max_iter = opt->fixed_iters ? opt->fixed_iters[0] : opt->max_iter;
  rd.tol_b2 = opt->eps * opt->eps;
  rd.tol_r2 = 0.0;
  CGDesc<double> cd;
  memset(&cd, 0, sizeof(cd));
  cd.g = g;
  cd.A = rd.A;
  cd.t = t;
  cd.slot = 0;
  cd.x = u;
  cd.r = reinterpret_cast<double*>(base + L.r);
  cd.pa = reinterpret_cast<double*>(base + L.pa);
  cd.pb = reinterpret_cast<double*>(base + L.pb);
  cd.q = reinterpret_cast<double*>(base + L.q);
  cd.aux = nullptr;

  // the reduction counter must start at zero; everything else is written before use
  CKN(cudaMemsetAsync(counters, 0, sizeof(unsigned), s));
  CKN(cudaMemcpyAsync(base + L.resd, &rd, sizeof(rd), cudaMemcpyHostToDevice, s));
  CKN(cudaMemcpyAsync(base + L.cgd, &cd, sizeof(cd), cudaMemcpyHostToDevice, s));
  const ResDesc* drd = reinterpret_cast<const ResDesc*>(base + L.resd);
  const CGDesc<double>* dcd = reinterpret_cast<const CGDesc<double>*>(base + L.cgd);
  CKN(launch_residual(false, 1, drd, rd.t.count(), residual_grid(rd.t.count(), 1), st, partials,
                      counters, s, 1));
  long long launches = 1;
  CGState hs;
  int chunk = opt->chunk > 0 ? opt->chunk : 4;
  for (;;) {
    for (int m = 0; m < chunk; ++m) {
      CKN(launch_cg_step<double>(1, dcd, t.count(), nblk, st, partials, counters, s));
      launches += 2;
    }
    CKN(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    CKN(cudaStreamSynchronize(s));
    if (hs.done) break;
    if (opt->chunk <= 0) chunk = chunk * 2 < 64 ? chunk * 2 : 64;
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->levels = 1;
    stats->N[0][0] = g.nx;
    stats->N[0][1] = g.ny;
    stats->N[0][2] = g.nz;
    stats->iters[0] = hs.iter;
    stats->relres[0] = hs.bb > 0 ? sqrt(hs.rr / hs.bb) : 0.0;
    stats->launches = launches;
  }
  return (excmg_status)hs.status;
}
