// Matrix-free stencil CG for the 19-point compact scheme (Section 2, eq. compact) and
// the CG loop of Algorithm 1 (one step per pass of its WHILE loop).
//
// One CG step is two launches, both persistent over z-slab tiles of kTX x kTY columns:
//   k_dir_spmv_dot : p_new = r + beta p_old (p = r on the first step), q = A p_new,
//                    partial sums of p.q; the last block forms alpha = r.r / p.q.
//   k_update_dot   : x += alpha p, r -= alpha q, partial sums of r.r; the last block
//                    forms beta, counts the step and applies the stopping test
//                    ||r|| <= eps ||b|| (or the iteration cap).
// The stencil marches in z through one shared-memory plane (with its x/y halo) at a
// time: for each plane it forms per column
//   C_k = c0 P + fx (P_{i-1}+P_{i+1}) + fy (P_{j-1}+P_{j+1}) + exy (4 xy-edge values)
//   T_k = fz P + exz (P_{i-1}+P_{i+1}) + eyz (P_{j-1}+P_{j+1})
// and (A p)_k = C_k + T_{k-1} + T_{k+1}: the z-face and z-edge terms of plane k are the
// "T" terms of its neighbour planes, so each plane is staged once and the 19-point sum
// costs 14 floating-point operations per node.
// Reductions are deterministic: fixed tile order per block, a fixed-order tree per
// block, and a fixed-order sum of the per-block partials by the last block to arrive.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "excmg_internal.cuh"

namespace excmg {

namespace {

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; the result is valid in thread 0.  Every thread must call.
// float64 instructions are scarce on this GPU (2 per clock per SM, 64-clock latency), so
// only warp 0 adds: every thread parks its value in shared memory, then each lane of
// warp 0 sums blockDim/32 of them in a fixed order and the warp reduces by shuffles.
// The order is fixed, so the result is deterministic.
__device__ double block_sum(double v) {
  __shared__ double s_v[kThreads];
  const int lane = threadIdx.x & 31;
  __syncthreads();
  s_v[threadIdx.x] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    // kThreads / 32 values per lane as a pairwise tree (a short dependence chain)
    double w[kThreads / 32];
#pragma unroll
    for (int u = 0; u < kThreads / 32; ++u) w[u] = s_v[lane + 32 * u];
#pragma unroll
    for (int d = 1; d < kThreads / 32; d *= 2)
#pragma unroll
      for (int u = 0; u + d < kThreads / 32; u += 2 * d) w[u] += w[u + d];
    t = warp_sum(w[0]);
  }
  return t;
}

// Warp-0 sum of src[0 .. n) from global memory (through L2) in a fixed order: each lane
// takes the values lane, lane + 32, ... in chunks of kSumChunk loads in flight, sums a
// chunk as a pairwise tree, then the lanes reduce by shuffles.  Valid in lane 0.
constexpr int kSumChunk = 8;
__device__ __forceinline__ double warp0_sum_global(const double* src, int n) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  for (int i0 = 0; i0 < n; i0 += 32 * kSumChunk) {
    double w[kSumChunk];
#pragma unroll
    for (int u = 0; u < kSumChunk; ++u) {
      const int i = i0 + lane + 32 * u;
      w[u] = i < n ? __ldcg(src + i) : 0.0;
    }
#pragma unroll
    for (int d = 1; d < kSumChunk; d *= 2)
#pragma unroll
      for (int u = 0; u + d < kSumChunk; u += 2 * d) w[u] += w[u + d];
    acc += w[0];
  }
  return warp_sum(acc);
}

template <typename D>
__device__ __forceinline__ int find_problem(const D* descs, int nprob, long long t, int p) {
  while (p + 1 < nprob && t >= descs[p + 1].tile_begin) ++p;
  return p;
}

struct TileXYZ {
  int x0, y0, z0, z1;
};

__device__ __forceinline__ TileXYZ tile_coords(const Grid3& g, const Tiling& tl, long long lt) {
  TileXYZ c;
  const int bx = (int)(lt % tl.ntx);
  const long long r = lt / tl.ntx;
  const int by = (int)(r % tl.nty);
  const int bz = (int)(r / tl.nty);
  c.x0 = bx * kTX;
  c.y0 = by * kTY;
  c.z0 = bz * tl.tz;
  c.z1 = min(c.z0 + tl.tz, g.nz + 1);
  return c;
}

// Publish this block's per-problem partial sums (NV values per problem) and let the
// last block to arrive for problem p reduce the gridDim.x partials of p in index order
// and call fin(p, sums).  The slot of problem p's state is descs[p].slot.
template <int NV, typename Fin>
__device__ void publish_and_finish(int nprob, const int* s_active, const double* s_part,
                                   double* partials, unsigned* counters, const Fin& fin) {
  __shared__ int s_last[kMaxProb];
  const int G = gridDim.x;
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
    s_last[p] = 0;
    if (s_active[p]) {
#pragma unroll
      for (int v = 0; v < NV; ++v)
        partials[((long long)p * NV + v) * G + blockIdx.x] = s_part[p * NV + v];
      __threadfence();
      const unsigned t = atomicAdd(&counters[p], 1u);
      s_last[p] = (t == (unsigned)G - 1u);
    }
  }
  __syncthreads();
  for (int p = 0; p < nprob; ++p) {
    if (!s_last[p]) continue;  // shared value: uniform across the block
    __threadfence();
    double sums[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v)
      sums[v] = threadIdx.x < 32 ? warp0_sum_global(partials + ((long long)p * NV + v) * G, G) : 0.0;
    if (threadIdx.x == 0) {
      fin(p, sums);
      counters[p] = 0u;
    }
    __syncthreads();
  }
}

template <typename T>
struct FinAlpha {
  const CGDesc<T>* descs;
  CGState* st;
  __device__ void operator()(int p, const double* s) const {
    CGState& S = st[descs[p].slot];
    const double pq = s[0];
    S.pq = pq;
    if (pq == 0.0 && S.rr == 0.0) {  // exact solution reached in fixed-count mode
      S.alpha = 0.0;
      S.done = 1;
    } else if (!(pq > 0.0) || !isfinite(pq)) {
      S.alpha = 0.0;
      S.status = EXCMG_ERR_NONFINITE;
      S.done = 1;
    } else {
      S.alpha = S.rr / pq;
    }
  }
};

template <typename T>
struct FinBeta {
  const CGDesc<T>* descs;
  CGState* st;
  __device__ void operator()(int p, const double* s) const {
    CGState& S = st[descs[p].slot];
    const double rr = s[0];
    S.beta = (S.rr > 0.0) ? rr / S.rr : 0.0;
    S.rr = rr;
    S.iter += 1;
    S.first = 0;
    const CGDesc<T>& d = descs[p];
    if (d.hist && S.iter < d.hist_len) d.hist[S.iter] = rr;
    if (!isfinite(rr)) {
      S.status = EXCMG_ERR_NONFINITE;
      S.done = 1;
    } else if (rr <= S.tol2) {
      S.done = 1;
    } else if (S.iter >= S.max_iter) {
      S.done = 1;
      S.status = S.fixed ? EXCMG_OK : EXCMG_ERR_NOT_CONVERGED;
    }
  }
};

struct FinRes {
  const ResDesc* descs;
  CGState* st;
  __device__ void operator()(int p, const double* s) const {
    const ResDesc& d = descs[p];
    CGState& S = st[d.slot];
    const double rr = s[0];
    // s[1] = ||b||^2 (lift included), s[2] = ||RHS(f)||^2: the two readings of ||f_h||
    const double bb = !d.want_b ? S.bb : (d.forcing && s[2] > 0.0) ? s[2] : s[1];
    S.rr = rr;
    S.rr0 = rr;
    S.bb = bb;
    S.alpha = 0.0;
    S.beta = 0.0;
    S.pq = 0.0;
    S.iter = 0;
    S.first = 1;
    S.max_iter = d.max_iter;
    S.fixed = d.fixed;
    S.status = EXCMG_OK;
    S.tol2 = d.fixed ? -1.0 : fmax(d.tol_b2 * bb, d.tol_r2 * rr);
    if (d.hist && d.hist_len > 0) d.hist[0] = rr;
    S.done = d.fixed ? (d.max_iter <= 0) : (rr <= S.tol2 || d.max_iter <= 0);
    // no step allowed and the start does not pass the test: the level is unconverged
    if (!d.fixed && d.max_iter <= 0 && !(rr <= S.tol2)) S.status = EXCMG_ERR_NOT_CONVERGED;
    if (!isfinite(rr) || !isfinite(bb)) {
      S.status = EXCMG_ERR_NONFINITE;
      S.done = 1;
    }
  }
};

// Loads of CG vectors bypass L1 (ld.global.cg): in the persistent kernel other blocks
// rewrite them between grid barriers, and L1 is not coherent across SMs.
__device__ __forceinline__ double ldv(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldv(const float* p) { return __ldcg(p); }

// One stencil tile: p_new = r + beta p_old (p = r when first), q = A p_new on the tile's
// nodes, returns this thread's share of p.q.  `sp` is the block's staging buffer and
// `buf` its current half (advanced per plane).  All threads of the block must call.
// The (kTX+2) x (kTY+2) halo plane is staged by the block's threads, at most two
// elements each; the loads of plane k+1 are issued into registers before the barrier
// and arithmetic of plane k, so global-memory latency overlaps the stencil work.
constexpr int kStage = (kTX + 2) * (kTY + 2);
static_assert(kStage <= 2 * kThreads, "a staged plane must need at most two loads per thread");

template <typename T>
struct PlaneLoad {
  T r0, p0, r1, p1;
};

template <typename T>
__device__ __forceinline__ void load_plane(PlaneLoad<T>& L, const Grid3& g, const TileXYZ& c, int kk,
                                           bool first, const T* __restrict__ r,
                                           const T* __restrict__ pold) {
  L.r0 = L.p0 = L.r1 = L.p1 = T(0);
  if (kk < 0 || kk > g.nz) return;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int idx = threadIdx.x + h * kThreads;
    if (idx >= kStage) break;
    const int ly = idx / (kTX + 2), lx = idx - ly * (kTX + 2);
    const int gi = c.x0 - 1 + lx, gj = c.y0 - 1 + ly;
    if (gi >= 0 && gi <= g.nx && gj >= 0 && gj <= g.ny) {
      const long long o = gi + gj * g.sy + (long long)kk * g.sz;
      const T rv = ldv(r + o);
      const T pv = first ? T(0) : ldv(pold + o);
      if (h == 0) {
        L.r0 = rv;
        L.p0 = pv;
      } else {
        L.r1 = rv;
        L.p1 = pv;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void store_plane(const PlaneLoad<T>& L, T beta,
                                            T (*plane)[kTX + 2]) {
  T* flat = &plane[0][0];
  flat[threadIdx.x] = fmaT(beta, L.p0, L.r0);
  if (threadIdx.x + kThreads < kStage) flat[threadIdx.x + kThreads] = fmaT(beta, L.p1, L.r1);
}

template <typename T>
__device__ __forceinline__ T spmv_tile(const CGDesc<T>& d, long long lt, bool first, T beta,
                                       const T* __restrict__ pold, T* __restrict__ pnew,
                                       T (*sp)[kTY + 2][kTX + 2], int& buf) {
  const Grid3 g = d.g;
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  const T* __restrict__ r = d.r;
  T* __restrict__ q = d.q;
  const TileXYZ c = tile_coords(g, d.t, lt);
  const int i = c.x0 + tx, j = c.y0 + ty;
  // own nodes include the padding columns nx + 1 .. sy - 1 of a padded float32 array,
  // which get p = q = 0 (the flat update then leaves them zero)
  const bool own = (i < g.sy) && (j <= g.ny);
  const bool inxy = (i > 0) && (i < g.nx) && (j > 0) && (j < g.ny);
  const T c0 = (T)d.A.c0, fx = (T)d.A.fx, fy = (T)d.A.fy, fz = (T)d.A.fz;
  const T exy = (T)d.A.exy, exz = (T)d.A.exz, eyz = (T)d.A.eyz;
  const T bta = first ? T(0) : beta;
  T Pm1 = T(0), Cm1 = T(0), Tm1 = T(0), Tm2 = T(0), tacc = T(0);
  // float32 keeps two planes in flight (it is bound by load latency), float64 one (it is
  // bound by the FP64 pipe and short of registers)
  constexpr bool kDeep = sizeof(T) == 4;
  PlaneLoad<T> nxt, nxt2;
  load_plane(nxt, g, c, c.z0 - 1, first, r, pold);
  if (kDeep) load_plane(nxt2, g, c, c.z0, first, r, pold);
  for (int kk = c.z0 - 1; kk <= c.z1; ++kk) {
    store_plane(nxt, bta, sp[buf]);
    if (kDeep) {
      nxt = nxt2;
      if (kk + 1 < c.z1) load_plane(nxt2, g, c, kk + 2, first, r, pold);
    } else if (kk < c.z1) {
      load_plane(nxt, g, c, kk + 1, first, r, pold);
    }
    __syncthreads();
    const T P = sp[buf][ty + 1][tx + 1];
    const T SX = sp[buf][ty + 1][tx] + sp[buf][ty + 1][tx + 2];
    const T SY = sp[buf][ty][tx + 1] + sp[buf][ty + 2][tx + 1];
    const T EXY = (sp[buf][ty][tx] + sp[buf][ty][tx + 2]) + (sp[buf][ty + 2][tx] + sp[buf][ty + 2][tx + 2]);
    const T Ck = fmaT(c0, P, fmaT(fx, SX, fmaT(fy, SY, exy * EXY)));
    const T Tk = fmaT(fz, P, fmaT(exz, SX, eyz * SY));
    const int kc = kk - 1;
    if (kc >= c.z0 && own) {
      const long long o = i + j * g.sy + (long long)kc * g.sz;
      const bool interior = inxy && kc > 0 && kc < g.nz;
      const T qv = interior ? (Cm1 + Tm2) + Tk : T(0);
      pnew[o] = Pm1;
      q[o] = qv;
      tacc = fmaT(Pm1, qv, tacc);
    }
    Tm2 = Tm1;
    Tm1 = Tk;
    Cm1 = Ck;
    Pm1 = P;
    buf ^= 1;
  }
  return tacc;
}

// One update tile: x += alpha p, r -= alpha q on the tile's nodes; returns this thread's
// share of r.r.
template <typename T>
__device__ __forceinline__ T update_tile(const CGDesc<T>& d, long long lt, T alpha,
                                         const T* __restrict__ pn, T sigma = T(1)) {
  const Grid3 g = d.g;
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  const T* __restrict__ q = d.q;
  T* __restrict__ x = d.x;
  T* __restrict__ r = d.r;
  const TileXYZ c = tile_coords(g, d.t, lt);
  const int i = c.x0 + tx, j = c.y0 + ty;
  T tacc = T(0);
  if (i <= g.nx && j <= g.ny) {
    long long o = i + j * g.sy + (long long)c.z0 * g.sz;
#pragma unroll 4
    for (int k = c.z0; k < c.z1; ++k, o += g.sz) {
      const T xv = fmaT(alpha, ldv(pn + o), ldv(x + o));
      const T rv = fmaT(-alpha, ldv(q + o), sigma * ldv(r + o));
      x[o] = xv;
      r[o] = rv;
      tacc = fmaT(rv, rv, tacc);
    }
  }
  return tacc;
}

// The update x += alpha p, r -= alpha q over a flat range of a problem's node array
// (it is elementwise: any partition works once p and q are complete), with 16-byte
// vector accesses when all four arrays allow them.  Block bl of G takes the chunks
// bl, bl + G, ... of kChunk elements.  Returns this thread's share of r.r.
constexpr int kChunk = 4 * kThreads * 2;  // elements per chunk: 2 vector steps per thread

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec<double> {
  using type = double2;
  static constexpr int n = 2;
};

__device__ __forceinline__ float4 ldv4(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldv4(const double2* p) { return __ldcg(p); }

// kRev: the blocks walk the chunks from the end of the array back to its start.  The
// stencil phase before it walks its tiles forward, so the chunks this phase takes first
// are the ones the stencil phase wrote last, still in L2 (and the chunks it takes last
// are the first the next stencil phase reads).
template <typename T, bool kRev = false>
__device__ __forceinline__ double update_flat(const CGDesc<T>& d, int bl, int G, T alpha,
                                              const T* __restrict__ pn, T sigma = T(1)) {
  const long long n = d.g.nodes();
  T* __restrict__ x = d.x;
  T* __restrict__ r = d.r;
  const T* __restrict__ q = d.q;
  double acc = 0.0;
  constexpr int V = Vec<T>::n;
  using VT = typename Vec<T>::type;
  // 16-byte vectors when the four arrays sit equally far from a 16-byte boundary: the
  // `lead` elements before it are done one by one (block 0), the rest in vectors
  const uintptr_t ax = reinterpret_cast<uintptr_t>(x);
  const bool vec = (((ax ^ reinterpret_cast<uintptr_t>(r)) | (ax ^ reinterpret_cast<uintptr_t>(q)) |
                     (ax ^ reinterpret_cast<uintptr_t>(pn))) & 15) == 0 && (ax % sizeof(T)) == 0;
  const long long lead = vec ? (long long)(((16 - (ax & 15)) & 15) / sizeof(T)) : 0;
  if (bl == 0 && threadIdx.x < lead && threadIdx.x < n) {
    const long long o = threadIdx.x;
    const T xv = fmaT(alpha, ldv(pn + o), ldv(x + o));
    const T rv = fmaT(-alpha, ldv(q + o), sigma * ldv(r + o));
    x[o] = xv;
    r[o] = rv;
    acc += (double)(rv * rv);
  }
  const long long nch = n > lead ? (n - lead + kChunk - 1) / kChunk : 0;
  for (long long m = bl; m < nch; m += G) {
    const long long c0 = lead + (kRev ? nch - 1 - m : m) * kChunk;
    const long long c1 = c0 + kChunk < n ? c0 + kChunk : n;
    T tacc = T(0);
    if (vec && c1 - c0 == kChunk) {
#pragma unroll
      for (int k = 0; k < kChunk / (V * kThreads); ++k) {
        const long long o = c0 + ((long long)k * kThreads + threadIdx.x) * V;
        const VT pv = ldv4(reinterpret_cast<const VT*>(pn + o));
        const VT qv = ldv4(reinterpret_cast<const VT*>(q + o));
        VT xv = ldv4(reinterpret_cast<const VT*>(x + o));
        VT rv = ldv4(reinterpret_cast<const VT*>(r + o));
        const T* pe = reinterpret_cast<const T*>(&pv);
        const T* qe = reinterpret_cast<const T*>(&qv);
        T* xe = reinterpret_cast<T*>(&xv);
        T* re = reinterpret_cast<T*>(&rv);
#pragma unroll
        for (int e = 0; e < V; ++e) {
          xe[e] = fmaT(alpha, pe[e], xe[e]);
          re[e] = fmaT(-alpha, qe[e], sigma * re[e]);
          tacc = fmaT(re[e], re[e], tacc);
        }
        *reinterpret_cast<VT*>(x + o) = xv;
        *reinterpret_cast<VT*>(r + o) = rv;
      }
    } else {
      for (long long o = c0 + threadIdx.x; o < c1; o += kThreads) {
        const T xv = fmaT(alpha, ldv(pn + o), ldv(x + o));
        const T rv = fmaT(-alpha, ldv(q + o), sigma * ldv(r + o));
        x[o] = xv;
        r[o] = rv;
        tacc = fmaT(rv, rv, tacc);
      }
    }
    acc += (double)tacc;
  }
  return acc;
}

// ---------------------------------------------------------------------------------
// Tensor-copy staging of the float32 stencil (the MIXED inner solves).  A block's
// stencil planes -- r and p_old of (kTX + 8) x (kTileY + 2) nodes, the tile's columns with
// a one-node halo in y and a 16-byte aligned halo of four in x -- stream through a ring
// of kStages shared-memory stages: thread 0 issues the two cp.async.bulk.tensor copies
// of a plane kStages planes ahead, and a "full" mbarrier per stage counts their bytes.
// No register holds a load and no block barrier separates the planes: every thread forms
// the p_new = sigma r + beta p_old values of its (rows + 2) x 3 neighbourhood straight
// from the stage, each warp releases the stage through an "empty" mbarrier when it is done with
// it, and thread 0 refills a stage once all warps have released it -- so warps drift
// apart by up to kStages planes and hide each other's latencies.  Out-of-range boxes
// (x < 0, y < 0, planes -1 and nz + 1, the padding columns) read as zeros.
// ---------------------------------------------------------------------------------
// Two rows per thread (tiles of 32 x 16 columns) in boxes of four planes: 9% faster per
// step than one row in boxes of six on 512x256x128, the same on 1024x512x512.
#ifndef EXCMG_TMA_ROWS
#define EXCMG_TMA_ROWS 2
#endif
#ifndef EXCMG_TMA_STAGES
#define EXCMG_TMA_STAGES 3
#endif
#ifndef EXCMG_TMA_PLANES
#define EXCMG_TMA_PLANES 4
#endif
constexpr int kRT = EXCMG_TMA_ROWS;        // y-rows per thread (consecutive)
constexpr int kTileY = kTY * kRT;          // y-rows of a tile of this engine
constexpr int kBoxX = kTX + 8;
constexpr int kBoxY = kTileY + 2;
constexpr int kStages = EXCMG_TMA_STAGES;
constexpr int kZs = EXCMG_TMA_PLANES;  // planes per copy (the box's z extent)
constexpr unsigned kBoxBytes = kBoxX * kBoxY * kZs * sizeof(float);
// a box's shared-memory slot, rounded up to 128 bytes so that every copy destination is
// 128-byte aligned
constexpr int kBoxSlot = ((kBoxBytes + 127) / 128) * 128 / sizeof(float);
constexpr int kWarps = kThreads / 32;

struct TmaRing {
  float stage[kStages][2][kBoxSlot];      // r and p_old of kZs planes per stage (kZs x kBoxY x kBoxX)
  unsigned long long full[kStages];       // the stage's copies have landed
  unsigned long long empty[kStages];      // every warp is done reading the stage
  int abort;                              // a wait ran out: the block leaves the step
};
static_assert(kBoxSlot * sizeof(float) % 128 == 0, "stage slots must keep 128-byte alignment");

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, P;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the barrier's phase `parity` to complete; false after wait_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity,
                                          unsigned long long wait_ns) {
  if (mbar_test(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_test(b, parity)) return true;
    if (global_ns() - t0 > wait_ns) return false;
  }
}

// One box of kZs planes (x, y, z .. z + kZs - 1) of a padded float32 array into shared
// memory; its bytes complete the transaction count of barrier b.  x is a multiple of 4.
__device__ __forceinline__ void tma_planes(float* dst, const CUtensorMap* m, unsigned long long* b,
                                           int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(m), "r"(x), "r"(y), "r"(z), "r"(smem_u32(b))
      : "memory");
}

// Parity bits of the ring's barriers, carried by every thread across the steps of a
// launch (full: the next phase each stage's copies complete; empty: thread 0's record of
// the stages' releases).
struct RingPhases {
  unsigned full = 0, empty = 0;
};

// Origin of tile lt of the tensor-copy engine's tiling (tiles of kTX x kTileY columns).
// The tiles cover nodes 0 .. n - 1 per direction: the far boundary faces (index n, and
// the padding columns) are never written by the engine; p and q hold zeros there from
// k_zero_far_faces, and the stencil reads them as halo.
__device__ __forceinline__ TileXYZ tma_tile_coords(const Grid3& g, const Tiling& tl, long long lt) {
  TileXYZ c;
  const int bx = (int)(lt % tl.ntx);
  const long long r = lt / tl.ntx;
  const int by = (int)(r % tl.nty);
  const int bz = (int)(r / tl.nty);
  c.x0 = bx * kTX;
  c.y0 = by * kTileY;
  c.z0 = bz * tl.tz;
  c.z1 = min(c.z0 + tl.tz, g.nz);
  return c;
}

// The K1 body over the tiles bl, bl + G, ... (desc.tt: tiles of kTX x kTileY columns) of
// one float32 problem with tensor-copy staging: p_new = sigma r + beta p_old (sigma = the
// folded RHS scale on the first step, else 1; p_old not read on the first step),
// q = A p_new, and this thread's share of p.q.  Each thread applies the stencil to kRT
// consecutive rows of one column, so the rows share the p_new values they have in
// common.  A tile's planes z0 - 1 .. z1 arrive kZs at a time (the last box of a tile
// may reach past z1; those planes are not used).  A wait that runs out sets ring.abort;
// every thread leaves its loop when it sees it, and the flag is read again after the
// block barrier that follows the call.
__device__ double spmv_tiles_tma(const CGDesc<float>& d, int bl, int G, bool first, float beta,
                                 float sigma, const CUtensorMap* mr, const CUtensorMap* mp,
                                 float* __restrict__ pnew, TmaRing& R, RingPhases& ph,
                                 unsigned long long wait_ns) {
  const Grid3 g = d.g;
  const Tiling tl = d.tt;
  const long long T = tl.count();
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX, lane = threadIdx.x & 31;
  float* __restrict__ q = d.q;
  const float c0 = (float)d.A.c0, fx = (float)d.A.fx, fy = (float)d.A.fy, fz = (float)d.A.fz;
  const float exy = (float)d.A.exy, exz = (float)d.A.exz, eyz = (float)d.A.eyz;
  const unsigned tx_bytes = first ? kBoxBytes : 2 * kBoxBytes;
  volatile int* abort = &R.abort;
  // producer cursor (thread 0): tile, its origin and the first plane of the next copy;
  // the tile's coordinates are formed once per tile
  long long lt = bl;
  TileXYZ lc{0, 0, 0, 0};
  int lkk = 0;
  if (lt < T) {
    lc = tma_tile_coords(g, tl, lt);
    lkk = lc.z0 - 1;
  }
  int issued = 0, consumed = 0;  // boxes copied / applied in this call (thread 0's counts)
  auto issue = [&](int slot) {
    ++issued;
    mbar_arrive_tx(&R.full[slot], tx_bytes);
    tma_planes(&R.stage[slot][0][0], mr, &R.full[slot], lc.x0 - 4, lc.y0 - 1, lkk);
    if (!first) tma_planes(&R.stage[slot][1][0], mp, &R.full[slot], lc.x0 - 4, lc.y0 - 1, lkk);
    lkk += kZs;
    if (lkk > lc.z1) {
      lt += G;
      if (lt < T) {
        lc = tma_tile_coords(g, tl, lt);
        lkk = lc.z0 - 1;
      }
    }
  };
  if (threadIdx.x == 0)
    for (int st = 0; st < kStages && lt < T; ++st) issue(st);
  int slot = 0;
  double acc = 0.0;
  bool stop = false;
  // this thread's neighbourhood in a plane of a stage: rows ty kRT .. ty kRT + kRT + 1,
  // columns tx + 3 .. tx + 5 (stage column c holds x = x0 - 4 + c, row r y = y0 - 1 + r)
  const int base = ty * kRT * kBoxX + tx + 3;
  for (long long t = bl; t < T && !stop; t += G) {
    const TileXYZ c = tma_tile_coords(g, tl, t);
    const int i = c.x0 + tx, j0 = c.y0 + ty * kRT;
    // own nodes include the padding columns nx + 1 .. sy - 1, which get p = q = 0
    const bool colx = (i > 0) && (i < g.nx), ownx = i < g.sy;
    float Pm1[kRT], Cm1[kRT], Tm1[kRT], Tm2[kRT];
#pragma unroll
    for (int r = 0; r < kRT; ++r) Pm1[r] = Cm1[r] = Tm1[r] = Tm2[r] = 0.f;
    float tacc = 0.f;
    for (int k0 = c.z0 - 1; k0 <= c.z1; k0 += kZs) {
      if (!mbar_wait(&R.full[slot], (ph.full >> slot) & 1u, wait_ns)) *abort = 1;
      ph.full ^= 1u << slot;
      if (*abort) {
        stop = true;
        break;
      }
      const int np = min(kZs, c.z1 + 1 - k0);  // planes of this box that the tile uses
#pragma unroll 1
      for (int pz = 0; pz < np; ++pz) {
        const float* rs = &R.stage[slot][0][pz * kBoxY * kBoxX + base];
        const float* ps = &R.stage[slot][1][pz * kBoxY * kBoxX + base];
        float v[kRT + 2][3];
#pragma unroll
        for (int a = 0; a < kRT + 2; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b)
            v[a][b] = first ? sigma * rs[a * kBoxX + b] : fmaf(beta, ps[a * kBoxX + b], rs[a * kBoxX + b]);
        const int kc = k0 + pz - 1;
        const bool emit = kc >= c.z0 && ownx;
        const bool zin = kc > 0 && kc < g.nz;
#pragma unroll
        for (int r = 0; r < kRT; ++r) {
          const float P = v[r + 1][1];
          const float SX = v[r + 1][0] + v[r + 1][2];
          const float SY = v[r][1] + v[r + 2][1];
          const float EXY = (v[r][0] + v[r][2]) + (v[r + 2][0] + v[r + 2][2]);
          const float Ck = fmaf(c0, P, fmaf(fx, SX, fmaf(fy, SY, exy * EXY)));
          const float Tk = fmaf(fz, P, fmaf(exz, SX, eyz * SY));
          const int j = j0 + r;
          if (emit && j <= g.ny) {
            const long long o = i + j * g.sy + (long long)kc * g.sz;
            const bool interior = colx && j > 0 && j < g.ny && zin;
            const float qv = interior ? (Cm1[r] + Tm2[r]) + Tk : 0.f;
            pnew[o] = Pm1[r];
            q[o] = qv;
            tacc = fmaf(Pm1[r], qv, tacc);
          }
          Tm2[r] = Tm1[r];
          Tm1[r] = Tk;
          Cm1[r] = Ck;
          Pm1[r] = P;
        }
      }
      // the stage is read: this warp releases it
      __syncwarp();
      if (lane == 0) mbar_arrive(&R.empty[slot]);
      if (threadIdx.x == 0) {
        ++consumed;
        // refill this stage with the box kStages ahead once every warp has released it
        if (lt < T) {
          if (!mbar_wait(&R.empty[slot], (ph.empty >> slot) & 1u, wait_ns)) *abort = 1;
          ph.empty ^= 1u << slot;
          if (!*abort) issue(slot);
        }
      }
      slot = slot + 1 == kStages ? 0 : slot + 1;
    }
    acc += (double)tacc;
  }
  if (threadIdx.x == 0) {
    // the releases of the last boxes' stages (no refill waited for them), then, after a
    // wait that ran out, the copies still in flight: nothing lands in shared memory or
    // is left half-counted once the block moves on
    const int tail = issued < kStages ? issued : kStages;
    int s0 = (consumed - tail) % kStages;
    if (s0 < 0) s0 += kStages;
    for (int n = 0; n < tail && !stop; ++n) {
      const int st = (s0 + n) % kStages;
      if (!mbar_wait(&R.empty[st], (ph.empty >> st) & 1u, wait_ns)) *abort = 1;
      ph.empty ^= 1u << st;
    }
    if (stop || *abort) {
      for (int n = consumed; n < issued; ++n) {
        mbar_wait(&R.full[slot], (ph.full >> slot) & 1u, wait_ns);
        ph.full ^= 1u << slot;
        slot = slot + 1 == kStages ? 0 : slot + 1;
      }
    }
  }
  return acc;
}

// ---------------------------------------------------------------------------------
// K1: p_new = r + beta p_old, q = A p_new, sum p.q
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_dir_spmv_dot(int nprob, const CGDesc<T>* __restrict__ descs, long long total_tiles,
                   CGState* st, double* partials, unsigned* counters) {
  __shared__ T sp[2][kTY + 2][kTX + 2];
  __shared__ int s_active[kMaxProb];
  __shared__ double s_part[kMaxProb];
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
    s_active[p] = !st[descs[p].slot].done;
    s_part[p] = 0.0;
  }
  __syncthreads();
  int buf = 0, cur = -1, p = 0;
  double acc = 0.0;
  for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    p = find_problem(descs, nprob, t, p);
    if (p != cur) {
      if (cur >= 0) {
        const double s = block_sum(acc);
        if (threadIdx.x == 0) s_part[cur] += s;
      }
      acc = 0.0;
      cur = p;
    }
    if (!s_active[p]) continue;
    const CGDesc<T>& d = descs[p];
    const CGState& S = st[d.slot];
    const int it = S.iter;
    acc += (double)spmv_tile<T>(d, t - d.tile_begin, S.first != 0, (T)S.beta,
                                (it & 1) ? d.pb : d.pa, (it & 1) ? d.pa : d.pb, sp, buf);
  }
  if (cur >= 0) {
    const double s = block_sum(acc);
    if (threadIdx.x == 0) s_part[cur] += s;
  }
  __syncthreads();
  publish_and_finish<1>(nprob, s_active, s_part, partials, counters, FinAlpha<T>{descs, st});
}

// ---------------------------------------------------------------------------------
// K2: x += alpha p, r -= alpha q, sum r.r, stopping test
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_update_dot(int nprob, const CGDesc<T>* __restrict__ descs, long long total_tiles,
                 CGState* st, double* partials, unsigned* counters) {
  __shared__ int s_active[kMaxProb];
  __shared__ double s_part[kMaxProb];
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
    s_active[p] = !st[descs[p].slot].done;
    s_part[p] = 0.0;
  }
  __syncthreads();
  int cur = -1, p = 0;
  double acc = 0.0;
  for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    p = find_problem(descs, nprob, t, p);
    if (p != cur) {
      if (cur >= 0) {
        const double s = block_sum(acc);
        if (threadIdx.x == 0) s_part[cur] += s;
      }
      acc = 0.0;
      cur = p;
    }
    if (!s_active[p]) continue;
    const CGDesc<T>& d = descs[p];
    const CGState& S = st[d.slot];
    const int it = S.iter;
    acc += (double)update_tile<T>(d, t - d.tile_begin, (T)S.alpha, (it & 1) ? d.pa : d.pb);
  }
  if (cur >= 0) {
    const double s = block_sum(acc);
    if (threadIdx.x == 0) s_part[cur] += s;
  }
  __syncthreads();
  publish_and_finish<1>(nprob, s_active, s_part, partials, counters, FinBeta<T>{descs, st});
}

// ---------------------------------------------------------------------------------
// Persistent CG: every CG step of one problem in one cooperative launch.  Each step
// runs the K1 body over the block's tiles, a grid-wide reduction of p.q, the K2 body,
// and a grid-wide reduction of r.r.  A reduction is: each block writes its partial,
// one grid barrier, then every block sums all partials in index order -- so every
// block derives bit-identical alpha, beta and the same stopping decision, and no
// second barrier or broadcast is needed.  Barrier waits are bounded: on time-out the
// kernel records EXCMG_ERR_TIMEOUT and returns.
// ---------------------------------------------------------------------------------
// Every wait of a cooperative CG launch gives up after wait_ns nanoseconds of the
// global timer (default 20 s: a team's first barrier may wait for members still
// finishing another problem of a batch).

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Every block arrives once; returns false in every block that saw a time-out (its own
// wait ran out after wait_ns, or another block's did: the shared error flag).
__device__ bool grid_barrier(unsigned* bar, unsigned target, int* err, unsigned long long wait_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    // release: this block's writes (ordered before it by the block barrier) become
    // visible before the arrival; the acquire loads below see every other block's
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    int ok = 1;
    unsigned spins = 0;
    unsigned long long t0 = 0;
    while (ld_acquire(bar) < target) {
      if (*(volatile int*)err) {
        ok = 0;
        break;
      }
      if (++spins == 4096) t0 = global_ns();
      if (spins > 4096) {  // tight polling first, then back off and watch the clock
        if (global_ns() - t0 > wait_ns) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    if (!ok) atomicExch(err, 1);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Sum of n partials in a fixed order, identical in every block (warp 0 only: the adds
// are float64).  Result in thread 0.
__device__ double sum_partials_all(const double* part, int n) {
  return threadIdx.x < 32 ? warp0_sum_global(part, n) : 0.0;
}

#ifndef EXCMG_PERSIST_MIN_BLOCKS
#define EXCMG_PERSIST_MIN_BLOCKS 3
#endif

// The CG loop of one problem, run by the G = d.blk_count blocks of its team (this block
// is member bl).  kTma: the float32 engine whose K1 body stages its planes by tensor
// copies (ring R); returns true if the ring was abandoned after a wait ran out.
template <typename T, bool kTma>
__device__ bool cg_team(const CGDesc<T>& d, int p, int bl, CGState* st, double* partials,
                        unsigned* bars, T (*sp)[kTY + 2][kTX + 2], double& s_scalar, int& buf,
                        TmaRing* R, RingPhases& phases, unsigned long long wait_ns) {
  const int G = d.blk_count;
  CGState* S = st + d.slot;
  if (S->done) return false;  // same value in every block of this team
  const long long total_tiles = d.t.count();
  double* partA = partials + (long long)p * 2 * kMaxGrid;
  double* partB = partA + G;
  unsigned* bar = bars + 2 * p;
  int* err = reinterpret_cast<int*>(bars + 2 * p + 1);
  double rr = S->rr, beta = S->beta, tol2 = S->tol2, pq = 0.0, alpha = 0.0;
  int iter = S->iter;
  const int max_iter = S->max_iter, fixed = S->fixed;
  bool first = S->first != 0;
  // MIXED: the right-hand side is scaled inside the first step (r <- scale r), so the
  // state's r.r and tolerance scale by scale^2 here
  const bool fold = first && d.fold_scale;
  if (fold) {
    rr *= d.scale * d.scale;
    tol2 *= d.scale * d.scale;
  }
  int status = EXCMG_OK;
  bool broken = false;
  unsigned nbar = 0;
  // a team of one block needs no grid barrier, only the block's own
  auto sync_all = [&]() -> bool {
    if (G == 1) {
      __syncthreads();
      return true;
    }
    return grid_barrier(bar, ++nbar * (unsigned)G, err, wait_ns);
  };
  for (;;) {
    const T sigma = (first && fold) ? (T)d.scale : T(1);
    // K1 body
    const T* pold = (iter & 1) ? d.pb : d.pa;
    T* pnew = (iter & 1) ? d.pa : d.pb;
    double acc = 0.0;
    if constexpr (kTma) {
      const CUtensorMap* mp = (iter & 1) ? &d.tm->pb : &d.tm->pa;
      acc = spmv_tiles_tma(d, bl, G, first, (float)beta, sigma, &d.tm->r, mp, pnew, *R, phases, wait_ns);
      __syncthreads();
      if (R->abort) {  // uniform: read after the block barrier
        broken = true;
        status = EXCMG_ERR_TIMEOUT;
        if (threadIdx.x == 0) atomicExch(err, 1);
        break;
      }
    } else {
      for (long long t = bl; t < total_tiles; t += G)
        acc += (double)spmv_tile<T>(d, t, first, (T)beta, pold, pnew, sp, buf);
    }
    double bs = block_sum(acc);
    if (threadIdx.x == 0) partA[bl] = bs;
    if (!sync_all()) {
      status = EXCMG_ERR_TIMEOUT;
      break;
    }
    bs = sum_partials_all(partA, G);
    if (threadIdx.x == 0) s_scalar = bs;
    __syncthreads();
    pq = s_scalar;
    if (pq == 0.0 && rr == 0.0) break;  // exact solution (fixed-count mode)
    if (!(pq > 0.0) || !isfinite(pq)) {
      status = EXCMG_ERR_NONFINITE;
      break;
    }
    alpha = rr / pq;
    // K2 body.  Elementwise: large grids take a flat, vectorised partition of the node
    // array; grids too small to give every block a full chunk keep the tile partition
    // (every block busy, one short column each -- lower latency)
    acc = 0.0;
    if (d.g.nodes() >= (long long)G * kChunk) {
      acc = update_flat<T, kTma>(d, bl, G, (T)alpha, pnew, sigma);
    } else {
      for (long long t = bl; t < total_tiles; t += G)
        acc += (double)update_tile<T>(d, t, (T)alpha, pnew, sigma);
    }
    bs = block_sum(acc);
    if (threadIdx.x == 0) partB[bl] = bs;
    if (kTma) {
      // the next step's tensor copies (async proxy) read r and p written here and by the
      // other blocks (generic proxy): order them after the grid barrier's acquire
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    if (!sync_all()) {
      status = EXCMG_ERR_TIMEOUT;
      break;
    }
    if (kTma) asm volatile("fence.proxy.async.global;" ::: "memory");
    bs = sum_partials_all(partB, G);
    if (threadIdx.x == 0) s_scalar = bs;
    __syncthreads();
    const double rrn = s_scalar;
    beta = (rr > 0.0) ? rrn / rr : 0.0;
    rr = rrn;
    iter += 1;
    first = false;
    if (bl == 0 && threadIdx.x == 0 && d.hist && iter < d.hist_len) d.hist[iter] = rr;
    if (!isfinite(rr)) {
      status = EXCMG_ERR_NONFINITE;
      break;
    }
    if (rr <= tol2) break;
    if (iter >= max_iter) {
      if (!fixed) status = EXCMG_ERR_NOT_CONVERGED;
      break;
    }
  }
  if (bl == 0 && threadIdx.x == 0) {
    S->rr = rr;
    S->pq = pq;
    S->alpha = alpha;
    S->beta = beta;
    S->iter = iter;
    S->first = first ? 1 : 0;
    S->status = status;
    S->done = 1;
  }
  return broken;
}

// Blocks form one team per problem: each block takes the next slot from an atomic
// counter; slots [blk_begin, blk_begin + blk_count) of problem p are its team.  Slots
// are handed out in order, so at most one team is ever partly formed and every earlier
// team finishes and frees its blocks: a team whose members arrive late only waits.
// A block whose team is done takes the next slot; a block past the last slot exits.
// kTma (float32 only): K1 stages its stencil planes by tensor copies.
#ifndef EXCMG_PERSIST_TMA_MIN_BLOCKS
#define EXCMG_PERSIST_TMA_MIN_BLOCKS 2
#endif
template <typename T, bool kTma>
__global__ void __launch_bounds__(kThreads, kTma ? EXCMG_PERSIST_TMA_MIN_BLOCKS : EXCMG_PERSIST_MIN_BLOCKS)
    k_cg_persistent(int nprob, const CGDesc<T>* __restrict__ descs, CGState* st,
                    double* partials, unsigned* bars, unsigned long long wait_ns) {
  __shared__ double s_scalar;
  __shared__ int s_slot;
  T(*sp)[kTY + 2][kTX + 2] = nullptr;
  TmaRing* R = nullptr;
  if constexpr (kTma) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];  // sizeof(TmaRing) bytes
    TmaRing& ring = *reinterpret_cast<TmaRing*>(dyn_smem);
    R = &ring;
    if (threadIdx.x == 0) {
      for (int k = 0; k < kStages; ++k) {
        mbar_init(&ring.full[k], 1);
        mbar_init(&ring.empty[k], kWarps);
      }
      ring.abort = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      // the tensor maps were copied to global memory before the launch
      for (int q = 0; q < nprob; ++q) {
        const TmapSet* m = descs[q].tm;
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&m->r) : "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&m->pa) : "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&m->pb) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&m->r) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&m->pa) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&m->pb) : "memory");
      }
    }
  } else {
    __shared__ T stage[2][kTY + 2][kTX + 2];
    sp = stage;
  }
  unsigned* slot_counter = bars + 2 * nprob;
  int total_slots = 0;
  for (int q = 0; q < nprob; ++q) total_slots = max(total_slots, descs[q].blk_begin + descs[q].blk_count);
  int buf = 0;
  RingPhases phases;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_slot = (int)atomicAdd(slot_counter, 1u);
    __syncthreads();
    const int slot = s_slot;
    if (slot >= total_slots) return;
    int p = 0;
    while (p < nprob && !(slot >= descs[p].blk_begin && slot < descs[p].blk_begin + descs[p].blk_count)) ++p;
    if (p >= nprob) return;  // unreachable: every slot below total_slots has a team
    if (cg_team<T, kTma>(descs[p], p, slot - descs[p].blk_begin, st, partials, bars, sp, s_scalar,
                         buf, R, phases, wait_ns))
      return;  // the copy ring was abandoned: this block takes no further work
  }
}



// ---------------------------------------------------------------------------------
// K3: r = LHS(u) - RHS(f) = b - A u_I (float64), sums r.r and b.b, CG state init
// ---------------------------------------------------------------------------------
#ifndef EXCMG_RES_MINB
#define EXCMG_RES_MINB 3  // one row per thread: 24 warps per SM, measured faster than 16
#endif
#ifndef EXCMG_RES_MINB_WIDE
// four rows per thread share the W + E sums of their neighbourhood (2 row sums per node
// instead of 3) and need 128 registers: 16 warps per SM (at 80 registers they spill)
#define EXCMG_RES_MINB_WIDE 2
#endif

// A residual tile: kTX columns along x (one warp) x kTY * R rows along y (each thread
// takes R adjacent rows) x tz planes, covering nodes 0 .. n per direction.
// (Tiles of the interior nodes 1 .. n, with the index-0 boundary nodes written by their
// neighbours, hold no padding for power-of-two grids but measured 40% slower.)
template <int R>
__device__ __forceinline__ TileXYZ res_tile_coords(const Grid3& g, const Tiling& tl, long long lt) {
  TileXYZ c;
  const int bx = (int)(lt % tl.ntx);
  const long long r = lt / tl.ntx;
  const int by = (int)(r % tl.nty);
  const int bz = (int)(r / tl.nty);
  c.x0 = bx * kTX;
  c.y0 = by * kTY * R;
  c.z0 = bz * tl.tz;
  c.z1 = min(c.z0 + tl.tz, g.nz + 1);
  return c;
}

// The Dirichlet lift of node (i, j, k) next to an x or y boundary face: the part of its
// 19-point sum over boundary nodes, grouped as the sum itself is (in-plane part of
// plane k, plus the out-of-plane parts of planes k - 1 and k + 1, which are whole
// boundary planes when k - 1 = 0 or k + 1 = nz).  Direct loads: about 3% of the nodes.
__device__ double perim_lift(const double* __restrict__ u, const Grid3& g, const Coef& A, int i,
                             int j, int k) {
  const bool bxm = (i - 1 == 0), bxp = (i + 1 == g.nx), bym = (j - 1 == 0), byp = (j + 1 == g.ny);
  auto at = [&](int x, int y, int z) { return __ldg(u + x + (long long)y * g.sy + (long long)z * g.sz); };
  // out-of-plane part of plane kk: whole plane if it is a boundary plane, else its
  // boundary columns
  auto lt = [&](int kk) -> double {
    if (kk == 0 || kk == g.nz) {
      const double SX = at(i - 1, j, kk) + at(i + 1, j, kk), SY = at(i, j - 1, kk) + at(i, j + 1, kk);
      return fma(A.fz, at(i, j, kk), fma(A.exz, SX, A.eyz * SY));
    }
    const double mSX = (bxm ? at(i - 1, j, kk) : 0.0) + (bxp ? at(i + 1, j, kk) : 0.0);
    const double mSY = (bym ? at(i, j - 1, kk) : 0.0) + (byp ? at(i, j + 1, kk) : 0.0);
    return fma(A.exz, mSX, A.eyz * mSY);
  };
  const double mSX = (bxm ? at(i - 1, j, k) : 0.0) + (bxp ? at(i + 1, j, k) : 0.0);
  const double mSY = (bym ? at(i, j - 1, k) : 0.0) + (byp ? at(i, j + 1, k) : 0.0);
  const double mEXY = ((bxm || bym) ? at(i - 1, j - 1, k) : 0.0) + ((bxp || bym) ? at(i + 1, j - 1, k) : 0.0) +
                      ((bxm || byp) ? at(i - 1, j + 1, k) : 0.0) + ((bxp || byp) ? at(i + 1, j + 1, k) : 0.0);
  const double LC = fma(A.fx, mSX, fma(A.fy, mSY, A.exy * mEXY));
  return (LC + lt(k - 1)) + lt(k + 1);
}

// Twice the right-hand side of eq. (compact) at interior node (i, j, k): 6 f_c + the 6
// face values of f (the face values are re-read through L1 by the neighbouring threads),
// or the value an earlier pass kept, or -2 b when b is given directly.  o is the node's
// offset.
__device__ __forceinline__ double res_rhs2(const ResDesc& d, int i, int j, int k, long long o) {
  if (d.rhs2 != nullptr) return d.rhs2[o];
  if (d.src != nullptr) return -2.0 * d.src[o];
  const View& F = d.f;
  return fma(6.0, F.at(i, j, k), ((F.at(i - 1, j, k) + F.at(i + 1, j, k)) +
                                  (F.at(i, j - 1, k) + F.at(i, j + 1, k)) +
                                  (F.at(i, j, k - 1) + F.at(i, j, k + 1))));
}

// The residual's block sums of one problem (r.r, ||b||^2 with the lift, ||RHS(f)||^2)
// added to its three partials in shared memory.  Called at problem switches only; kept
// out of line so that it adds no registers to the plane loop.
__device__ __noinline__ void residual_flush(double acc_r, double acc_b, double acc_b4, double* part) {
  const double s1 = block_sum(acc_r);
  const double s2 = block_sum(fma(0.25, acc_b4, acc_b));
  const double s3 = block_sum(0.25 * acc_b4);
  if (threadIdx.x == 0) {
    part[0] += s1;
    part[1] += s2;
    part[2] += s3;
  }
}

// Each thread marches its R rows of one x-column through the tile's planes.  Per
// plane it loads the (R + 2) x 3 neighbourhood (through the read-only cache:
// neighbouring threads share the lines; no staging, no block barrier) and forms, per row,
// the in-plane part C = c0 P + fx S_x + fy S_y + exy E_xy and the out-of-plane part
// T = fz P + exz S_x + eyz S_y of the 19-point sum, with S_x = W + E computed once per
// loaded row and shared by the rows above and below (E_xy of row j = S_x(j-1) + S_x(j+1),
// the same grouping as (SW + SE) + (NW + NE)); the sum at plane k is C_k + T_{k-1} +
// T_{k+1}.  The first and last plane of a tile contribute T only.  b (for ||b||) is
// -RHS away from the boundary; next to a z-boundary plane its lift is that plane's T;
// next to a y boundary face it is formed by perim_lift (the whole warp is such a row).
// Next to an x boundary face only one lane of the warp is such a node: those nodes are
// left out of the plane loop and formed after it, one lane per plane, so a warp issues
// the lift once for up to 32 planes instead of once per plane for one lane.
template <typename TR, int R>
__global__ void __launch_bounds__(kThreads, R > 1 ? EXCMG_RES_MINB_WIDE : EXCMG_RES_MINB)
    k_residual(int nprob, const ResDesc* __restrict__ descs, long long total_tiles,
               CGState* st, double* partials, unsigned* counters) {
  static_assert(kTX == 32, "one warp per x-run of a residual tile row");
  __shared__ int s_active[kMaxProb];
  __shared__ double s_part[3 * kMaxProb];
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
    s_active[p] = 1;
    s_part[3 * p] = 0.0;
    s_part[3 * p + 1] = 0.0;
    s_part[3 * p + 2] = 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  int cur = -1, p = 0;
  // acc_b4 sums (2 RHS)^2 over every interior node: ||RHS(f)||^2 = acc_b4 / 4 is the
  // forcing reading of ||f_h||.  b = -RHS - lift, and the lift is nonzero only next to
  // the boundary, so ||b||^2 = acc_b4 / 4 + acc_b with acc_b summing b^2 - RHS^2 =
  // lift (lift + 2 RHS) over those nodes (the lift reading).
  double acc_r = 0.0, acc_b = 0.0, acc_b4 = 0.0;
  auto flush = [&](int q) { residual_flush(acc_r, acc_b, acc_b4, s_part + 3 * q); };
  for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    p = find_problem(descs, nprob, t, p);
    if (p != cur) {
      if (cur >= 0) flush(cur);
      acc_r = acc_b = acc_b4 = 0.0;
      cur = p;
    }
    const ResDesc& d = descs[p];
    const Grid3 g = d.g;
    const double* __restrict__ u = d.u;
    TR* __restrict__ rout = reinterpret_cast<TR*>(d.r);
    // output strides: the padded float32 layout, or the grid's own for float64
    const long long osy = sizeof(TR) == 4 ? d.osy : g.sy, osz = sizeof(TR) == 4 ? d.osz : g.sz;
    const TileXYZ c = res_tile_coords<R>(g, d.t, t - d.tile_begin);
    const int i = c.x0 + tx, jb = c.y0 + R * ty;  // rows jb .. jb + R - 1
    if (c.x0 >= g.nx || c.y0 >= g.ny || c.z0 >= g.nz) {
      // a tile of boundary nodes only (the last column, row or plane of the grid and the
      // padding beyond it): r = 0, no arithmetic
      for (int kc = c.z0; kc < c.z1; ++kc)
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const int j = jb + q;
          if (i < osy && j <= g.ny) rout[i + j * osy + (long long)kc * osz] = (TR)0.0;
        }
      continue;
    }
    const bool colx = (i > 0) && (i < g.nx);
    const bool want_b = d.want_b != 0;
    const Coef A = d.A;
    double Cm1[R], Tm1[R], Tm2[R];
#pragma unroll
    for (int q = 0; q < R; ++q) Cm1[q] = Tm1[q] = Tm2[q] = 0.0;
    for (int kk = c.z0 - 1; kk <= c.z1; ++kk) {
      const bool need_c = (kk >= c.z0) && (kk < c.z1);  // C of the tile's own planes only
      // the neighbourhood: rows jb - 1 .. jb + R (index y = row - jb + 1), columns i - 1,
      // i, i + 1; zero outside the grid
      double Pv[R + 2], SXv[R + 2];
      const bool kin = kk >= 0 && kk <= g.nz;
      const double* pl = u + (long long)kk * g.sz;
#pragma unroll
      for (int y = 0; y < R + 2; ++y) {
        const int gj = jb - 1 + y;
        const bool rin = kin && gj >= 0 && gj <= g.ny;
        const double* row = pl + (long long)gj * g.sy;
        const double W = (rin && i - 1 >= 0 && i - 1 <= g.nx) ? __ldg(row + i - 1) : 0.0;
        const double E = (rin && i + 1 <= g.nx) ? __ldg(row + i + 1) : 0.0;
        Pv[y] = (rin && i <= g.nx) ? __ldg(row + i) : 0.0;
        SXv[y] = W + E;
      }
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int y = q + 1, j = jb + q;
        const double SX = SXv[y], SY = Pv[y - 1] + Pv[y + 1], P = Pv[y];
        double Ck = 0.0;
        if (need_c) Ck = fma(A.c0, P, fma(A.fx, SX, fma(A.fy, SY, A.exy * (SXv[y - 1] + SXv[y + 1]))));
        const double Tk = fma(A.fz, P, fma(A.exz, SX, A.eyz * SY));
        const int kc = kk - 1;
        if (kc >= c.z0 && i <= g.nx && j <= g.ny) {
          const long long o = i + j * g.sy + (long long)kc * g.sz;
          double rv = 0.0;
          if (colx && j > 0 && j < g.ny && kc > 0 && kc < g.nz) {
            // twice the right-hand side (kept as it is for the later passes); the factor
            // 1/2 is applied inside the fused multiply-add below, exactly
            const double rhs2 = res_rhs2(d, i, j, kc, o);
            if (d.rhs_out) d.rhs_out[o] = rhs2;
            // LHS(u) - RHS = -(A-stencil of u over all 19 nodes) - RHS
            rv = fma(-0.5, rhs2, -((Cm1[q] + Tm2[q]) + Tk));
            acc_r = fma(rv, rv, acc_r);
            if (want_b) {
              acc_b4 = fma(rhs2, rhs2, acc_b4);
              const bool yface = (j == 1 || j == g.ny - 1), xface = (i == 1 || i == g.nx - 1);
              if ((yface || !xface) && (yface || kc < 2 || kc > g.nz - 2)) {
                const double lift = yface ? perim_lift(u, g, A, i, j, kc)
                                          : (kc == 1 ? Tm2[q] : 0.0) + (kc == g.nz - 1 ? Tk : 0.0);
                acc_b = fma(lift, lift + rhs2, acc_b);
              }  // next to an x face only: after the plane loop; elsewhere b = -RHS
            }
          }
          rout[i + j * osy + (long long)kc * osz] = (TR)rv;
        } else if (sizeof(TR) == 4 && kc >= c.z0 && i > g.nx && i < osy && j <= g.ny) {
          rout[i + j * osy + (long long)kc * osz] = (TR)0.0;  // padding column
        }
        Tm2[q] = Tm1[q];
        Tm1[q] = Tk;
        Cm1[q] = Ck;
      }
    }
    if (want_b) {
      // b of the tile's nodes next to an x face and no y face (columns 1 and nx - 1, rows
      // 2 .. ny - 2): the warp of such a row takes them one lane per plane.  A warp is one
      // x-run of 32 columns (kTX = 32), so its columns are c.x0 .. c.x0 + 31 in every row.
      const int lane = threadIdx.x & 31;
      const int k_lo = max(c.z0, 1), k_hi = min(c.z1, g.nz);  // interior planes of the tile
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int j = jb + q;
        if (j < 2 || j > g.ny - 2) continue;
        for (int side = 0; side < 2; ++side) {
          const int xi = side == 0 ? 1 : g.nx - 1;
          if (side == 1 && xi == 1) break;  // nx = 2: a single interior column
          if (xi < c.x0 || xi >= c.x0 + kTX) continue;
          for (int k0 = k_lo; k0 < k_hi; k0 += 32) {
            const int kc = k0 + lane;
            if (kc < k_hi) {
              const long long o = xi + j * g.sy + (long long)kc * g.sz;
              const double lift = perim_lift(u, g, A, xi, j, kc);
              acc_b = fma(lift, lift + res_rhs2(d, xi, j, kc, o), acc_b);
            }
          }
        }
      }
    }
  }
  if (cur >= 0) flush(cur);
  __syncthreads();
  publish_and_finish<3>(nprob, s_active, s_part, partials, counters, FinRes{descs, st});
}

// MIXED refinement: u += e / scale (the float32 correction of the scaled system), then
// e = 0 for the next inner solve.  e has the padded float32 layout, u the unpadded
// float64 one, whose nodes are one contiguous run: the threads stride through u's flat
// index m (eight elements in flight each, consecutive lanes on consecutive nodes), and
// e's index is m plus the padding of the rows before it, m / (nx + 1) found by a
// multiply-high with the rounded-up reciprocal 2^64 / (nx + 1) (exact for m < 2^32 and
// far beyond).  No row is split into a short last pass.
__global__ void __launch_bounds__(kThreads)
    k_add_correction(int nprob, const CGDesc<float>* __restrict__ descs) {
  constexpr int kU = 8;
  const unsigned long long tid = (unsigned long long)blockIdx.x * kThreads + threadIdx.x;
  const unsigned long long nth = (unsigned long long)gridDim.x * kThreads;
  for (int p = 0; p < nprob; ++p) {
    const CGDesc<float>& d = descs[p];
    const Grid3 g = d.g;
    const unsigned long long n1 = (unsigned long long)g.nx + 1;
    const unsigned long long rows = (unsigned long long)(g.ny + 1) * (g.nz + 1);
    const double inv = 1.0 / d.scale;
    float* __restrict__ e = d.x;
    double* __restrict__ u = d.aux;
    if (d.aux_sy == (long long)n1 && d.aux_sz == (long long)(n1 * (g.ny + 1))) {
      const unsigned long long n = n1 * rows;
      const unsigned long long M = ~0ULL / n1 + 1;  // ceil(2^64 / n1); 2^64 / n1 if a power of 2
      const unsigned long long pad = (unsigned long long)g.sy - n1;
      for (unsigned long long m0 = tid; m0 < n; m0 += kU * nth) {
        float ev[kU];
        double uv[kU];
        unsigned long long oe[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
          const unsigned long long m = m0 + k * nth;
          oe[k] = m + __umul64hi(m, M) * pad;
          ev[k] = m < n ? __ldcs(e + oe[k]) : 0.f;
          uv[k] = m < n ? __ldcs(u + m) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < kU; ++k) {
          const unsigned long long m = m0 + k * nth;
          if (m < n) {
            __stcs(u + m, fma((double)ev[k], inv, uv[k]));
            __stcs(e + oe[k], 0.f);
          }
        }
      }
    } else {
      // u with other strides: a warp per row (j, k), lanes along x
      const int lane = threadIdx.x & 31;
      for (unsigned long long row = tid >> 5; row < rows; row += nth >> 5) {
        const long long j = (long long)(row % (g.ny + 1)), k = (long long)(row / (g.ny + 1));
        float* er = e + j * g.sy + k * g.sz;
        double* ur = u + j * d.aux_sy + k * d.aux_sz;
        for (int i = lane; i <= g.nx; i += 32) {
          ur[i] = fma((double)er[i], inv, ur[i]);
          er[i] = 0.f;
        }
      }
    }
  }
}

// MIXED: r *= scale (in float64, then rounded); one thread per problem rescales r.r and
// the inner tolerance of that problem's CG state.
__global__ void __launch_bounds__(kThreads)
    k_scale_rhs(int nprob, const CGDesc<float>* __restrict__ descs, long long total_tiles,
                CGState* st) {
  if (blockIdx.x == 0)
    for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
      CGState& S = st[descs[p].slot];
      const double s2 = descs[p].scale * descs[p].scale;
      S.rr *= s2;
      S.tol2 *= s2;
    }
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  int p = 0;
  for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    p = find_problem(descs, nprob, t, p);
    const CGDesc<float>& d = descs[p];
    const Grid3 g = d.g;
    const TileXYZ c = tile_coords(g, d.t, t - d.tile_begin);
    const int i = c.x0 + tx, j = c.y0 + ty;
    if (i > g.nx || j > g.ny) continue;
    long long o = i + j * g.sy + (long long)c.z0 * g.sz;
    for (int k = c.z0; k < c.z1; ++k, o += g.sz) d.r[o] = (float)((double)d.r[o] * d.scale);
  }
}

int g_max_grid = 0;
int g_coop_grid[2] = {0, 0};  // co-resident blocks of k_cg_persistent<double>, <float>
int g_coop_grid_tma = 0;      // the same for the float32 tensor-copy engine

}  // namespace

// Dynamic shared memory of a k_cg_persistent launch (the tensor-copy ring).
template <bool kTma>
size_t persistent_smem() {
  return kTma ? sizeof(TmaRing) : 0;
}

template <typename T, bool kTma>
int coop_blocks(int& cached) {
  if (cached == 0) {
    int dev = 0, sms = 0, occ = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (kTma)
      cudaFuncSetAttribute(k_cg_persistent<T, kTma>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)persistent_smem<kTma>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg_persistent<T, kTma>, kThreads,
                                                  persistent_smem<kTma>());
    cached = (coop && sms > 0 && occ > 0) ? std::min(sms * occ, kMaxGrid) : -1;
  }
  return cached;
}

template <typename T>
int persistent_cg_blocks() {
  return coop_blocks<T, false>(g_coop_grid[sizeof(T) == 8 ? 0 : 1]);
}
template int persistent_cg_blocks<double>();
template int persistent_cg_blocks<float>();

int persistent_cg_blocks_tma() { return coop_blocks<float, true>(g_coop_grid_tma); }

template <typename T>
cudaError_t launch_cg_persistent(int nprob, const CGDesc<T>* descs, int grid, CGState* st,
                                 double* partials, unsigned* bar, unsigned long long wait_ns,
                                 bool tma, cudaStream_t s) {
  void* args[] = {(void*)&nprob, (void*)&descs, (void*)&st, (void*)&partials, (void*)&bar,
                  (void*)&wait_ns};
  const void* fn = (const void*)k_cg_persistent<T, false>;
  size_t smem = 0;
  if constexpr (sizeof(T) == 4) {
    if (tma) {
      fn = (const void*)k_cg_persistent<float, true>;
      smem = persistent_smem<true>();
    }
  }
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), args, smem, s);
}
template cudaError_t launch_cg_persistent<double>(int, const CGDesc<double>*, int, CGState*, double*,
                                                  unsigned*, unsigned long long, bool, cudaStream_t);
template cudaError_t launch_cg_persistent<float>(int, const CGDesc<float>*, int, CGState*, double*,
                                                 unsigned*, unsigned long long, bool, cudaStream_t);

// cuTensorMapEncodeTiled, looked up once through the runtime (no link against libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

Tiling make_tma_tiling(const Grid3& g, int tz) {
  if (tz < 1) tz = 1;
  Tiling t;
  t.tz = tz;
  // nodes 0 .. n - 1 per direction (see tma_tile_coords): whole tiles on power-of-two
  // grids
  t.ntx = (g.nx + kTX - 1) / kTX;
  t.nty = (g.ny + kTileY - 1) / kTileY;
  t.ntz = (g.nz + tz - 1) / tz;
  return t;
}

int tma_slab_depth(int tz) {
  // the slab depth nearest tz whose tz + 2 planes are whole copies of kZs planes
  if (tz + 2 <= kZs) return kZs - 2 > 0 ? kZs - 2 : tz;
  const int lo = ((tz + 2) / kZs) * kZs - 2, hi = lo + kZs;
  return (tz - lo <= hi - tz) ? lo : hi;
}

bool encode_plane_map(CUtensorMap* m, float* base, const Grid3& g32) {
  static EncodeTiledFn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (g32.sy & 3)) return false;
  // x extent nx + 1: the padding columns are outside the map and read as zeros
  const cuuint64_t dims[3] = {(cuuint64_t)g32.nx + 1, (cuuint64_t)g32.ny + 1, (cuuint64_t)g32.nz + 1};
  const cuuint64_t strides[2] = {(cuuint64_t)g32.sy * sizeof(float), (cuuint64_t)g32.sz * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)kBoxX, (cuuint32_t)kBoxY, (cuuint32_t)kZs};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int persistent_grid(long long total_tiles) {
  if (g_max_grid == 0) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dir_spmv_dot<double>, kThreads, 0);
    if (sms <= 0) sms = 1;
    if (occ <= 0) occ = 1;
    g_max_grid = sms * occ;
    if (g_max_grid > kMaxGrid) g_max_grid = kMaxGrid;
  }
  long long g = total_tiles < g_max_grid ? total_tiles : g_max_grid;
  return g < 1 ? 1 : (int)g;
}

static int g_res_grid[2] = {0, 0};

int residual_grid(long long total_tiles, int rows) {
  const int w = rows > 1 ? 1 : 0;
  if (g_res_grid[w] == 0) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (w)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_residual<double, kResRowsWide>, kThreads, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_residual<double, 1>, kThreads, 0);
    if (sms <= 0) sms = 1;
    if (occ <= 0) occ = 1;
    g_res_grid[w] = sms * occ;
    // the residual publishes 3 partials per block into room for 2 x kMaxGrid
    if (g_res_grid[w] > 2 * kMaxGrid / 3) g_res_grid[w] = 2 * kMaxGrid / 3;
  }
  long long g = total_tiles < g_res_grid[w] ? total_tiles : g_res_grid[w];
  return g < 1 ? 1 : (int)g;
}

template <typename T>
cudaError_t launch_cg_step(int nprob, const CGDesc<T>* descs, long long total_tiles, int grid,
                           CGState* st, double* partials, unsigned* counters, cudaStream_t s,
                           cudaEvent_t e0, cudaEvent_t e1, cudaEvent_t e2) {
  if (e0) cudaEventRecord(e0, s);
  k_dir_spmv_dot<T><<<grid, kThreads, 0, s>>>(nprob, descs, total_tiles, st, partials, counters);
  if (e1) cudaEventRecord(e1, s);
  k_update_dot<T><<<grid, kThreads, 0, s>>>(nprob, descs, total_tiles, st, partials, counters);
  if (e2) cudaEventRecord(e2, s);
  return cudaGetLastError();
}
template cudaError_t launch_cg_step<double>(int, const CGDesc<double>*, long long, int, CGState*,
                                            double*, unsigned*, cudaStream_t, cudaEvent_t,
                                            cudaEvent_t, cudaEvent_t);
template cudaError_t launch_cg_step<float>(int, const CGDesc<float>*, long long, int, CGState*,
                                           double*, unsigned*, cudaStream_t, cudaEvent_t,
                                           cudaEvent_t, cudaEvent_t);

cudaError_t launch_residual(bool out_float, int nprob, const ResDesc* descs, long long total_tiles,
                            int grid, CGState* st, double* partials, unsigned* counters,
                            cudaStream_t s, int rows) {
  if (rows != 1 && rows != kResRowsWide) return cudaErrorInvalidValue;
  if (out_float && rows > 1)
    k_residual<float, kResRowsWide><<<grid, kThreads, 0, s>>>(nprob, descs, total_tiles, st, partials, counters);
  else if (out_float)
    k_residual<float, 1><<<grid, kThreads, 0, s>>>(nprob, descs, total_tiles, st, partials, counters);
  else if (rows > 1)
    k_residual<double, kResRowsWide><<<grid, kThreads, 0, s>>>(nprob, descs, total_tiles, st, partials, counters);
  else
    k_residual<double, 1><<<grid, kThreads, 0, s>>>(nprob, descs, total_tiles, st, partials, counters);
  return cudaGetLastError();
}

// Zeros of p_a, p_b and q on the far boundary faces of a padded float32 grid: the
// columns nx .. sy - 1 of every row, the row ny and the plane nz.  The tensor-copy CG
// engine never writes these nodes (its tiles end at n - 1) and reads them as halo.
__global__ void k_zero_far_faces(Grid3 g, float* a, float* b, float* c) {
  const long long rows = (long long)(g.ny + 1) * (g.nz + 1);
  const int cx = g.sy - g.nx;  // columns nx .. sy - 1
  const long long n1 = rows * cx, n2 = (long long)g.sy * (g.nz + 1), n3 = (long long)g.sy * (g.ny + 1);
  const long long n = n1 + n2 + n3;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    long long o;
    if (t < n1) {
      const long long row = t / cx;
      o = (long long)(g.nx + (int)(t % cx)) + (row % (g.ny + 1)) * g.sy + (row / (g.ny + 1)) * g.sz;
    } else if (t < n1 + n2) {
      const long long u = t - n1;
      o = (u % g.sy) + (long long)g.ny * g.sy + (u / g.sy) * g.sz;
    } else {
      const long long u = t - n1 - n2;
      o = (u % g.sy) + (u / g.sy) * g.sy + (long long)g.nz * g.sz;
    }
    a[o] = 0.f;
    b[o] = 0.f;
    c[o] = 0.f;
  }
}

__global__ void k_export_states(const unsigned* __restrict__ src, unsigned* dst, int words) {
  for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
}

cudaError_t launch_export_states(const CGState* src, CGState* dst, int n, cudaStream_t s) {
  static_assert(sizeof(CGState) % sizeof(unsigned) == 0, "CGState is copied in 32-bit words");
  const int words = (int)(sizeof(CGState) / sizeof(unsigned)) * n;
  k_export_states<<<1, kThreads, 0, s>>>(reinterpret_cast<const unsigned*>(src),
                                         reinterpret_cast<unsigned*>(dst), words);
  return cudaGetLastError();
}

cudaError_t launch_zero_far_faces(const CGDesc<float>& d, cudaStream_t s) {
  const long long n = (long long)(d.g.ny + 1) * (d.g.nz + 1) * (d.g.sy - d.g.nx) +
                      (long long)d.g.sy * (d.g.nz + d.g.ny + 2);
  const long long blocks = std::min<long long>((n + kThreads - 1) / kThreads, 4096);
  k_zero_far_faces<<<(int)std::max<long long>(blocks, 1), kThreads, 0, s>>>(d.g, d.pa, d.pb, d.q);
  return cudaGetLastError();
}

cudaError_t launch_add_correction(int nprob, const CGDesc<float>* inner, long long total_tiles,
                                  int grid, cudaStream_t s) {
  (void)total_tiles;
  (void)grid;
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_add_correction, kThreads, 0);
    blocks = std::max(1, sms) * std::max(1, occ);
  }
  k_add_correction<<<blocks, kThreads, 0, s>>>(nprob, inner);
  return cudaGetLastError();
}

cudaError_t launch_scale_rhs(int nprob, const CGDesc<float>* inner, long long total_tiles,
                             int grid, CGState* st, cudaStream_t s) {
  k_scale_rhs<<<grid, kThreads, 0, s>>>(nprob, inner, total_tiles, st);
  return cudaGetLastError();
}

}  // namespace excmg
