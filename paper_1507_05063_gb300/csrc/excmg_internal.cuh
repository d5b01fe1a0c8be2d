// Internal declarations shared by the CUDA translation units of libexcmg.
//
// Data layout: every level's node array is dense float64 (or float32 for the inner
// correction solve of MIXED mode), x fastest, node (i,j,k) at i + sy*j + sz*k with
// sy = nx+1, sz = (nx+1)(ny+1).  Arrays used by CG (x, r, p, q) hold zeros on boundary
// nodes except x, whose boundary holds the Dirichlet data g: the stencil applied to p
// with zero boundary is exactly A p on the interior unknowns (Section 2, eq. FD).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "excmg.h"

namespace excmg {

constexpr int kMaxProb = 128;    // problems per batched launch
constexpr int kThreads = 256;    // threads of every tiled kernel
constexpr int kTX = 32;          // x-width of a stencil tile (one warp)
constexpr int kTY = 8;           // y-rows of a stencil tile
// y-rows per thread of the residual kernel: 1 or kResRowsWide, per launch (ResDesc.rows).
// Four rows share their W + E sums (7% faster on 1024x512x512) but run 16 warps per SM
// instead of 24 (17% slower on 512x256x128); the tuning cache decides per level grid,
// else grids of at least EXCMG_RES_WIDE_MIN_NODES nodes take four.
constexpr int kResRowsWide = 4;
#ifndef EXCMG_RES_WIDE_MIN_NODES
#define EXCMG_RES_WIDE_MIN_NODES (1LL << 26)
#endif
constexpr long long kResWideMinNodes = EXCMG_RES_WIDE_MIN_NODES;
constexpr int kMaxGrid = 4096;   // cap on persistent grid size (partials per problem)
#ifndef EXCMG_CLUSTER_MAX_NODES
#define EXCMG_CLUSTER_MAX_NODES 20000
#endif
#ifndef EXCMG_RESIDENT_MIN_NODES
#define EXCMG_RESIDENT_MIN_NODES 2000
#endif
// grids up to kClusterMaxNodes nodes can run all their CG steps in one thread-block
// cluster; a single float64 grid of more than kResidentMinNodes nodes takes the resident
// engine instead (measured faster from about 5,000 nodes: 8.2 vs 8.7 us per step)
constexpr long long kClusterMaxNodes = EXCMG_CLUSTER_MAX_NODES;
constexpr long long kResidentMinNodes = EXCMG_RESIDENT_MIN_NODES;
// MIXED mode solves grids below this many nodes in float64 by default: there CG is
// latency-bound, float32 saves nothing and refinement would add host round trips.
constexpr long long kMixedMinNodes = 1LL << 21;

struct Grid3 {
  int nx, ny, nz;      // cells per direction
  long long sy, sz;    // node strides
  double hx, hy, hz;   // meshsizes
  __host__ __device__ long long nodes() const { return sz * (long long)(nz + 1); }
};

Grid3 make_grid(int nx, int ny, int nz, double Lx, double Ly, double Lz);
// The same grid with the row pitch of the float32 CG vectors: rows padded to a multiple
// of 4 floats (16 bytes), so that every row and plane starts 16-byte aligned, as the
// tensor copies (cp.async.bulk.tensor) and 16-byte vector accesses need.
Grid3 padded_f32(const Grid3& g);


// The option checks every entry point applies (excmg_api.cu).
bool options_valid(const excmg_options* o);

// Weights of A = -(printed left-hand side of eq. compact).  a = 1/hx^2 ...
// centre 8(a+b+c); x-faces -(4a-b-c); y-faces -(4b-a-c); z-faces -(4c-a-b);
// xy-edges -(a+b)/2; xz-edges -(a+c)/2; yz-edges -(b+c)/2.
struct Coef {
  double c0, fx, fy, fz, exy, exz, eyz;
};
Coef make_coef(const Grid3& g);

// A finest-grid node array seen at the nodes of a coarser level (injection).
struct View {
  const double* p;
  long long sx, sy, sz;
  __device__ __forceinline__ double at(long long i, long long j, long long k) const {
    return p[i * sx + j * sy + k * sz];
  }
};

// CG scalars of one problem, resident in device memory (workspace).
struct CGState {
  double rr;      // r.r of the current residual
  double pq;      // p.Ap of the current step
  double alpha, beta;
  double tol2;    // stop when rr <= tol2
  double bb;      // ||b||^2 of the level
  double rr0;     // rr when the loop started
  int iter, max_iter;
  int done;       // 1: no further CG work for this problem
  int first;      // 1: next step sets p = r
  int status;     // excmg_status
  int fixed;      // 1: max_iter is an exact count, reaching it is not an error
};

// Tiling of one problem's node box for the stencil and vector kernels: tiles of
// kTX x kTY columns and tz planes.
struct Tiling {
  int ntx, nty, ntz, tz;
  __host__ __device__ long long count() const { return (long long)ntx * nty * ntz; }
};
Tiling make_tiling(const Grid3& g, int tz);
// The residual kernel's tiling: kTY * rows rows per tile, the same x-width, slab depth tz
// (choose_res_tz: the residual's own model of its launch).
Tiling make_res_tiling(const Grid3& g, int tz, int rows);
int choose_res_tz(const Grid3& g, int grid_blocks, int requested, int rows);
// The model's rows per thread of the residual kernel for grid g (1 or kResRowsWide).
int res_rows_model(const Grid3& g);
int choose_tz(const Grid3& g, int grid_blocks, int requested);

// Tensor maps of one float32 CG problem (cp.async.bulk.tensor): r and the two p buffers,
// each a 3D map of the padded array (x extent nx + 1, so the padding reads as zero) with
// a box of a tile's columns and their halo over several planes ((kTX + 8) x (rows of a
// tile + 2) x planes per copy: cg_kernels.cu).
struct alignas(64) TmapSet {
  CUtensorMap r, pa, pb;
};

// One problem of a CG phase.
template <typename T>
struct CGDesc {
  Grid3 g;
  Coef A;
  Tiling t;
  Tiling tt;              // float32 tensor-copy engine: its own tiles (make_tma_tiling)
  long long tile_begin;   // first global tile index of this problem
  int slot;               // index of this problem's CGState
  T* x;
  T* r;
  T* pa;                  // p buffers: even steps read pa and write pb, odd steps swap
  T* pb;
  T* q;
  T* s0;                  // resident CG (float64 grids up to kResidentMaxNodes): s by
  T* s1;                  //   step parity (NULL elsewhere)
  double* aux;            // MIXED inner solve: the float64 level solution u += x / scale
  long long aux_sy, aux_sz;  // node strides of aux (unpadded float64 layout)
  double scale;           // MIXED inner solve: it solves A x = scale * r (r scaled to O(1)
                          // so float32 products neither underflow nor overflow)
  int fold_scale;         // 1: r is still unscaled; the first CG step applies `scale`
  const TmapSet* tm;      // float32 persistent CG: tensor maps of r, pa, pb (device)
  int blk_begin;          // persistent CG: this problem's blocks are [blk_begin,
  int blk_count;          //   blk_begin + blk_count) of the cooperative grid
  int direct;             // 1: the level is solved by DSOLVE (k_dsolve), not by CG
  View f;                 // DSOLVE: f and the Dirichlet data at this level's nodes
  View gb;
  double* hist;           // NULL, or r.r after each CG step k = 1 .. hist_len - 1 (device)
  int hist_len;
  int forcing;            // DSOLVE: ||f_h|| of the state is the forcing norm (rhs_norm)
};

// One problem of a residual phase: r = LHS(u) - RHS(f) (= b - A u_I) in float64,
// written as TR; rr and (optionally) bb reduced; then the CG state is initialised.
struct ResDesc {
  Grid3 g;
  Coef A;
  Tiling t;
  long long tile_begin;
  int slot;             // index of this problem's CGState
  const double* u;      // level solution, boundary = g
  View f;               // f at this level's nodes (unused when src is set)
  const double* src;    // NULL, or b given directly on interior nodes: r = LHS(u) + src
                        // (the adjoint's A lambda = s with lambda's boundary zero)
  const double* rhs2;   // NULL, or 2 RHS(f) on interior nodes as an earlier pass kept it
                        // in rhs_out (MIXED refinement steps after the first)
  double* rhs_out;      // NULL, or receives 2 RHS(f) on interior nodes (f path only)
  void* r;              // TR* output
  long long osy, osz;   // node strides of r (the padded layout when TR is float; the
                        // padding columns nx + 1 .. osy - 1 are written as zeros)
  double tol_b2;        // tol2 = max(tol_b2 * bb, tol_r2 * rr)
  double tol_r2;
  int want_b;           // compute bb (else keep the state's bb)
  int forcing;          // bb = ||RHS(f)||^2 over the interior (the FORCING reading of
                        // ||f_h||), or ||b||^2 with the lift where that is zero; else
                        // bb = ||b||^2 (LIFT)
  int max_iter;
  int fixed;            // exact iteration count
  double* hist;         // NULL, or receives r.r of the start in hist[0] (device)
  int hist_len;
  int rows;             // y-rows per thread of the tiling t (1 or kResRowsWide); the same
                        // for every problem of one launch
};

// Launch helpers (defined in cg_kernels.cu).  `descs` point to DEVICE copies.
// One CG step = the stencil launch then the update launch.  When e0/e1/e2 are not
// null, events are recorded before, between and after the two launches.
template <typename T>
cudaError_t launch_cg_step(int nprob, const CGDesc<T>* descs, long long total_tiles, int grid,
                           CGState* st, double* partials, unsigned* counters,
                           cudaStream_t s, cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr,
                           cudaEvent_t e2 = nullptr);
cudaError_t launch_residual(bool out_float, int nprob, const ResDesc* descs,
                            long long total_tiles, int grid, CGState* st, double* partials,
                            unsigned* counters, cudaStream_t s, int rows);
// Copies n CG states into a device-mapped page-locked host buffer (dst: its device
// address), by one block: the states reach the host without a copy-engine transfer.
cudaError_t launch_export_states(const CGState* src, CGState* dst, int n, cudaStream_t s);
// Zeros p_a, p_b and q of one float32 problem on its far boundary faces (x = nx and the
// padding columns, y = ny, z = nz), which the tensor-copy engine reads but never writes.
cudaError_t launch_zero_far_faces(const CGDesc<float>& d, cudaStream_t s);
cudaError_t launch_add_correction(int nprob, const CGDesc<float>* inner, long long total_tiles,
                                  int grid, cudaStream_t s);
// MIXED: r *= scale on every problem's float32 residual, and the CG state's r.r and
// tolerance by scale^2 (before the inner solve).
cudaError_t launch_scale_rhs(int nprob, const CGDesc<float>* inner, long long total_tiles,
                             int grid, CGState* st, cudaStream_t s);
int persistent_grid(long long total_tiles);
// Blocks of a residual launch: all co-resident blocks of k_residual, at most one per tile.
int residual_grid(long long total_tiles, int rows);

// All CG steps of every problem of `descs` in one cooperative launch.  Problem p owns
// the blocks [blk_begin, blk_begin + blk_count) and iterates independently of the
// others; its reductions cross a barrier over its own blocks only (bounded waits;
// EXCMG_ERR_TIMEOUT in its state if a wait runs out).  `bar` holds two zeroed words per
// problem (arrival count, time-out flag); `partials` 2 x kMaxGrid doubles per problem.
// persistent_cg_blocks() is the largest co-resident grid, or -1 if the device has no
// cooperative launch.
template <typename T>
int persistent_cg_blocks();
// All CG steps of each problem in one thread-block cluster of `csize` CTAs (grid =
// nprob clusters), x, r, p, q in the cluster's shared memory (cluster_cg.cu).
// cluster_cg_size: the cluster size for grid g (1..16), or 0 if g does not fit or the
// device cannot launch it; cluster_cg_smem: dynamic shared memory per CTA for g at csize.
template <typename T>
int cluster_cg_size(const Grid3& g);
size_t cluster_cg_smem(const Grid3& g, int csize, size_t elem);
template <typename T>
cudaError_t launch_cg_cluster(int nprob, const CGDesc<T>* descs, int csize, size_t smem,
                              long long max_nodes, CGState* st, cudaStream_t s);
// wait_ns bounds every device-side wait of the launch (grid barriers, tensor-copy
// completions); tma selects the float32 engine whose stencil planes stream through
// tensor copies (every problem's desc.tm set).
template <typename T>
cudaError_t launch_cg_persistent(int nprob, const CGDesc<T>* descs, int grid, CGState* st,
                                 double* partials, unsigned* bar, unsigned long long wait_ns,
                                 bool tma, cudaStream_t s);
// Co-resident blocks of the float32 tensor-copy engine.
int persistent_cg_blocks_tma();
// Slab depth for the float32 tensor-copy engine: tz moved to the nearest depth whose
// tz + 2 planes (the slab and its two halo planes) are whole copies.
int tma_slab_depth(int tz);
// The tensor-copy engine's tiling of g: tiles of kTX columns x (its rows per thread x
// kTY) rows x tz planes.
Tiling make_tma_tiling(const Grid3& g, int tz);
// Encodes the tensor map of one padded float32 node array of grid g32 (padded_f32);
// false if the driver entry point is missing or the encoding fails.
bool encode_plane_map(CUtensorMap* m, float* base, const Grid3& g32);

// All CG steps of ONE float64 grid of up to kResidentMaxNodes nodes in a cooperative
// grid whose blocks keep the level's vectors in shared memory (resident_cg.cu).
#ifndef EXCMG_RESIDENT_MAX_NODES
#define EXCMG_RESIDENT_MAX_NODES (1 << 20)
#endif
constexpr long long kResidentMaxNodes = EXCMG_RESIDENT_MAX_NODES;
// excmg_solve_batched: problems with a finest grid of at least this many nodes run as
// single solves, one after another; smaller ones share the batch's launches.
#ifndef EXCMG_BATCH_SOLO_NODES
#define EXCMG_BATCH_SOLO_NODES (1LL << 18)
#endif
constexpr long long kBatchSoloNodes = EXCMG_BATCH_SOLO_NODES;
struct ResidentDesc {
  Grid3 g;
  Coef A;
  int slot;               // CGState of the problem
  int bx, by, bz;         // interior nodes per box
  int nbx, nby, nbz;      // boxes per direction (grid = their product)
  double* x;              // level solution (boundary = g)
  double* r;              // residual r_0 in, last r out; also the even-step copy of r
  double* r1;             // odd-step copy of r
  double* w0;             // w = A r, even / odd steps
  double* w1;
  double* s0;             // s, even / odd steps
  double* s1;
  double* hist;           // NULL, or r.r after each CG step k = 1 .. hist_len - 1 (device)
  int hist_len;
};
// Chooses the boxes for grid g; false if the grid does not fit or the device has no
// cooperative launch.  smem: dynamic shared memory per block.
bool resident_box(const Grid3& g, ResidentDesc& D, size_t& smem);
// pairs: 2 G double2 (G = nbx nby nbz); counter, err: zeroed.
cudaError_t launch_cg_resident(const ResidentDesc& D, size_t smem, CGState* st, double2* pairs,
                               unsigned* counter, int* err, cudaStream_t s);

// DSOLVE by the discrete sine transform (dsolve_kernels.cu): one block per descriptor
// with `direct` set (others return at once); x's interior = A^{-1} r, r = the residual
// of the result, the CG state done with 0 steps.  dsolve_fits: the grid's interior fits
// one block's shared memory; dsolve_smem: the bytes it needs.
bool dsolve_fits(const Grid3& g);
size_t dsolve_smem(const Grid3& g);
cudaError_t launch_dsolve(int nprob, const CGDesc<double>* descs, size_t smem, CGState* st,
                          cudaStream_t s);

// Transfer kernels (transfer_kernels.cu).
struct ProlongDesc {
  Grid3 g;              // fine grid (h)
  const double* u2h;    // grid with g.n/2 cells
  const double* u4h;    // grid with g.n/4 cells
  View gb;              // Dirichlet data at fine nodes, or p == nullptr
  double* w;            // fine node array
  long long block_begin;
  int nbx, nby, nbz;    // blocks of 32x8x8 fine cells
};
cudaError_t launch_exp_finite(int nprob, const ProlongDesc* descs, long long total_blocks,
                              cudaStream_t s);
cudaError_t launch_exp_finite_one(const ProlongDesc& desc, cudaStream_t s);
// The comparison prolongations: points = 3 (extrapolation, then tri-quadratic) or 2
// (trilinear interpolation of u_2h); same descriptors and brick grid as EXP_finite.
cudaError_t launch_prolong_cmp(int points, int nprob, const ProlongDesc* descs,
                               long long total_blocks, cudaStream_t s);
cudaError_t launch_exp_true(const Grid3& g, const double* uh, const double* u2h, double* ut,
                            cudaStream_t s);
cudaError_t launch_boundary_init(const Grid3& g, View gb, double* u, cudaStream_t s);
cudaError_t launch_adjoint_finish(const Grid3& g, const Coef& A, const double* lam,
                                  const double* dLdu, double* dLdf, double* dLdg,
                                  cudaStream_t s);

// Gradient kernels (grad_kernels.cu).
cudaError_t launch_grad(const Grid3& g, const double* u, double* ux, double* uy, double* uz,
                        cudaStream_t s);

}  // namespace excmg
