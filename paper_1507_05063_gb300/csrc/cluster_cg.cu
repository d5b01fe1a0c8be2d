// Small-grid CG on one thread-block cluster per problem.
//
// On the coarse grids of the cascade (a few hundred to a few thousand nodes) a CG step is
// bound by latency: every global reduction is a data dependence of the next phase, and on
// GB300 each float64 add of a reduction tree or divide waits on the narrow FP64 pipe.
// Here a cluster of C CTAs (C = 1..16, one SM each) keeps the whole grid in shared memory
// for all steps of the level, and each step takes ONE reduction:
//
//   * the recurrence is the single-reduction form of CG of Chronopoulos and Gear (1989):
//     with w = A r and s = A p carried by recurrence,
//        p = r + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,
//        w = A r,  gamma = r.r,  delta = w.r   (one reduction for both),
//        beta' = gamma' / gamma,  alpha' = gamma' / (delta' - beta' gamma' / alpha);
//     in exact arithmetic its x and r are those of the standard recurrence (the smoother
//     of Algorithm 1), so the loop stops on the same recursive residual r.r <= tol2 after
//     the same step; only the rounding differs;
//   * the node array 0..n-1 (x fastest) is cut into C contiguous ranges of m nodes; CTA c
//     holds x, p, two copies of w and s (by step parity) of its range, and two copies of
//     r extended by a halo of H = sy + sz nodes on each side (the largest offset of the
//     19-point stencil).  The halo of the new r is recomputed locally from the owners'
//     previous r, w, s read through distributed shared memory (DSMEM), with the same
//     fused operations as the owner, so it is bit-identical and no barrier is needed
//     between the update and the stencil;
//   * the reduction: values parked in shared memory, CTA sums in warp 0, stored into slots
//     of every CTA of the cluster (DSMEM), a cluster barrier, then every CTA adds the C
//     slots in the same order -- all CTAs hold bit-identical alpha, beta and stop
//     decisions, so they take the same number of barriers.
// Scalars are formed by warp 0 (alpha and beta as one two-lane divide): on GB300 a warp
// instruction on the FP64 pipe costs the same for one lane as for 32.
#include <cuda_runtime.h>

#include <algorithm>

#include "excmg_internal.cuh"

namespace excmg {
namespace {

constexpr int kClMax = 16;

__device__ __forceinline__ double fmaC(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaC(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Cluster-wide barrier; release/acquire orders shared-memory (and DSMEM) accesses of all
// CTAs of the cluster around it.
__device__ __forceinline__ void cl_sync() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of the same shared-memory object in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned cl_map(const void* local, unsigned rank) {
  const unsigned la = (unsigned)__cvta_generic_to_shared(local);
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
  return ra;
}

// Generic address of the same shared-memory object in CTA `rank`: plain loads through
// it are ordinary memory operations the compiler may batch and overlap.
template <typename P>
__device__ __forceinline__ const P* cl_peer(const P* local, unsigned rank) {
  unsigned long long ra;
  asm("mapa.u64 %0, %1, %2;" : "=l"(ra) : "l"(reinterpret_cast<unsigned long long>(local)), "r"(rank));
  return reinterpret_cast<const P*>(ra);
}
__device__ __forceinline__ void st_cl(double* local, unsigned rank, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(cl_map(local, rank)), "d"(v) : "memory");
}

__device__ __forceinline__ double xor_sum(double v, int from) {
  for (int o = from; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums of (a, b) over every thread of the cluster, returned in every lane of warp 0
// (bit-identical in every CTA); other warps get 0.  Contains one cluster barrier.  Both
// sums share each float64 warp instruction: lanes 0-15 carry a, lanes 16-31 carry b (on
// GB300 a float64 warp instruction costs the narrow FP64 pipe the same for one sum or
// two, and a step waits on this chain).
template <int NW>
__device__ double2 cluster_sum2(double a, double b, double* s_park, double* slots,
                                unsigned me, int csize) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, h = lane & 15;
  // the CTA's sums: values parked in shared memory, added by warp 0 (2 NW per lane as a
  // pairwise tree, then a butterfly over 16 lanes)
  s_park[threadIdx.x] = a;
  s_park[32 * NW + threadIdx.x] = b;
  __syncthreads();
  if (warp == 0) {
    const double* src = s_park + (lane < 16 ? 0 : 32 * NW);
    double v[2 * NW];
#pragma unroll
    for (int u = 0; u < 2 * NW; ++u) v[u] = src[h + 16 * u];
#pragma unroll
    for (int w = 1; w < 2 * NW; w *= 2)
#pragma unroll
      for (int u = 0; u + w < 2 * NW; u += 2 * w) v[u] += v[u + w];
    const double r = xor_sum(v[0], 8);
    // every lane holds both CTA sums (lane c stores into CTA c, and the cluster may have
    // more CTAs than this CTA has warps -- a CTA given a wrong partial would take other
    // decisions than its peers)
    const double ta = __shfl_sync(0xffffffffu, r, 0), tb = __shfl_sync(0xffffffffu, r, 16);
    if (lane < csize) {
      st_cl(slots + me, (unsigned)lane, ta);
      st_cl(slots + kClMax + me, (unsigned)lane, tb);
    }
  }
  if (csize > 1) {
    cl_sync();
  } else {
    __syncthreads();  // a cluster of one CTA: the block barrier orders its shared memory
  }
  double2 t = make_double2(0.0, 0.0);
  if (warp == 0) {
    // the C slots of a in lanes 0-15, of b in lanes 16-31; a butterfly over the smallest
    // power of two >= csize lanes of each half: fixed order (csize is the same in every
    // CTA), so identical in every CTA
    double v = h < csize ? slots[(lane < 16 ? 0 : kClMax) + h] : 0.0;
    int from = 1;
    while (from < csize) from <<= 1;
    v = xor_sum(v, from >> 1);
    t.x = __shfl_sync(0xffffffffu, v, 0);
    t.y = __shfl_sync(0xffffffffu, v, 16);
  }
  return t;
}

// 19-point A-stencil at flat offset 0 of P (interior node).
template <typename T>
__device__ __forceinline__ T stencil19(const T* P, int sy, int sz, T c0, T fx, T fy, T fz, T exy,
                                       T exz, T eyz) {
  const T SX = P[-1] + P[1], SY = P[-sy] + P[sy], SZ = P[-sz] + P[sz];
  const T EXY = (P[-1 - sy] + P[1 - sy]) + (P[-1 + sy] + P[1 + sy]);
  const T EXZ = (P[-1 - sz] + P[1 - sz]) + (P[-1 + sz] + P[1 + sz]);
  const T EYZ = (P[-sy - sz] + P[sy - sz]) + (P[-sy + sz] + P[sy + sz]);
  return fmaC(c0, P[0], fmaC(fx, SX, fmaC(fy, SY, fmaC(fz, SZ, fmaC(exy, EXY, fmaC(exz, EXZ, eyz * EYZ))))));
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT)
    k_cg_cluster(const CGDesc<T>* __restrict__ descs, CGState* st, int csize) {
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) unsigned char s_raw[];
  __shared__ double s_park[2 * NT];
  // two slot sets, alternating per reduction: a peer's stores for the next reduction can
  // only start after the barrier that follows this CTA's reads of the current one
  __shared__ double s_slots[2][2 * kClMax];
  __shared__ double s_alpha, s_beta;
  __shared__ int s_stop;
  const unsigned me = cl_rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const CGDesc<T>& d = descs[blockIdx.x / csize];
  CGState* S = st + d.slot;
  // identical in every CTA: nothing writes the state before the cluster barriers below
  if (S->done) return;
  const Grid3 g = d.g;
  const int n = (int)g.nodes();
  const int sy = (int)g.sy, sz = (int)g.sz;
  const int m = (n + csize - 1) / csize;
  const int H = sy + sz;
  const int lo = (int)me * m;
  const int cnt = max(0, min(n - lo, m));
  const int ext = m + 2 * H;
  T* xs = reinterpret_cast<T*>(s_raw);
  T* ps = xs + m;
  T* W0 = ps + m;
  T* W1 = W0 + m;
  T* S0 = W1 + m;
  T* S1 = S0 + m;
  T* R0 = S1 + m;  // extended: own range at [H, H + m)
  T* R1 = R0 + ext;
  const T c0 = (T)d.A.c0, fx = (T)d.A.fx, fy = (T)d.A.fy, fz = (T)d.A.fz;
  const T exy = (T)d.A.exy, exz = (T)d.A.exz, eyz = (T)d.A.eyz;
  auto interior = [&](int o) {
    const int i = o % sy, j = (o / sy) % (g.ny + 1), k = o / sz;
    return i > 0 && i < g.nx && j > 0 && j < g.ny && k > 0 && k < g.nz;
  };
  // r_0 on the own range and its halo (from the level's r in global memory); x, p = 0,
  // s_{-1} = 0
  for (int e = (int)threadIdx.x - H; e < m + H; e += NT) {
    const int o = lo + e;
    R0[H + e] = (o >= 0 && o < n) ? d.r[o] : T(0);
  }
  for (int e = threadIdx.x; e < m; e += NT) {
    xs[e] = e < cnt ? d.x[lo + e] : T(0);
    ps[e] = T(0);
    S1[e] = T(0);
  }
  __syncthreads();
  // w_0 = A r_0, delta_0 = w_0.r_0
  double acc_d = 0.0;
  for (int e = threadIdx.x; e < cnt; e += NT) {
    const int o = lo + e;
    T wv = T(0);
    if (interior(o)) {
      wv = stencil19(R0 + H + e, sy, sz, c0, fx, fy, fz, exy, exz, eyz);
      acc_d = fma((double)wv, (double)R0[H + e], acc_d);
    }
    W0[e] = wv;
  }
  // every CTA of the cluster must have started before any distributed-shared-memory
  // access (the reductions store into the peers' slots)
  if (csize > 1) cl_sync();
  // scalars: warp 0 keeps identical copies in all lanes (and in every CTA)
  double gam = S->rr, alpha = 0.0, beta = 0.0, delta = 0.0;
  const double tol2 = S->tol2;
  int iter = S->iter;
  const int max_iter = S->max_iter, fixed = S->fixed;
  int status = EXCMG_OK;
  {
    const double2 red = cluster_sum2<NW>(0.0, acc_d, s_park, s_slots[0], me, csize);
    if (warp == 0) {
      delta = red.y;
      int stop = 0;
      if (delta == 0.0 && gam == 0.0) {
        stop = 1;  // exact solution (fixed-count mode)
      } else if (!(delta > 0.0) || !isfinite(delta)) {
        status = EXCMG_ERR_NONFINITE;
        stop = 1;
      } else {
        alpha = gam / delta;
      }
      if (lane == 0) {
        s_stop = stop;
        s_alpha = alpha;
        s_beta = 0.0;
      }
    }
    __syncthreads();
  }
  int par = 0;  // r_i in R[par], w_i in W[par], s_{i-1} in S[par ^ 1]; slot set par ^ 1
  bool stop = s_stop != 0;
  while (!stop) {
    const T aT = (T)s_alpha, bT = (T)s_beta;
    const T* Rc = par ? R1 : R0;
    T* Rn = par ? R0 : R1;
    const T* Wc = par ? W1 : W0;
    T* Wn = par ? W0 : W1;
    const T* Sp = par ? S0 : S1;  // s_{i-1}
    T* Sc = par ? S1 : S0;        // s_i
    // 1a. own range: p, s, x, r
    for (int e = threadIdx.x; e < m; e += NT) {
      T rn = T(0);
      if (e < cnt) {
        const T r = Rc[H + e];
        const T pv = fmaC(bT, ps[e], r);
        const T sv = fmaC(bT, Sp[e], Wc[e]);
        ps[e] = pv;
        Sc[e] = sv;
        xs[e] = fmaC(aT, pv, xs[e]);
        rn = fmaC(-aT, sv, r);
      }
      Rn[H + e] = rn;
    }
    // 1b. halo (H nodes on each side): the new r from the owners' r, w, s with the same
    // fused operations as the owner (bit-identical); the peer loads of kHB nodes are
    // issued together
    constexpr int kHB = 4;
    for (int h0 = threadIdx.x; h0 < 2 * H; h0 += kHB * NT) {
      T rv[kHB], wv[kHB], sv[kHB];
#pragma unroll
      for (int u = 0; u < kHB; ++u) {
        const int h = h0 + u * NT;
        const int e = h < H ? h - H : m + (h - H);
        const int o = lo + e;
        rv[u] = wv[u] = sv[u] = T(0);
        if (h < 2 * H && o >= 0 && o < n) {
          const unsigned owner = (unsigned)(o / m);
          const int le = o - (int)owner * m;
          rv[u] = *cl_peer(Rc + H + le, owner);
          wv[u] = *cl_peer(Wc + le, owner);
          sv[u] = *cl_peer(Sp + le, owner);
        }
      }
#pragma unroll
      for (int u = 0; u < kHB; ++u) {
        const int h = h0 + u * NT;
        if (h < 2 * H) {
          const int e = h < H ? h - H : m + (h - H);
          Rn[H + e] = fmaC(-aT, fmaC(bT, sv[u], wv[u]), rv[u]);
        }
      }
    }
    __syncthreads();
    // 2. w = A r, gamma = r.r, delta = w.r on the own range
    double acc_g = 0.0;
    acc_d = 0.0;
    for (int e = threadIdx.x; e < cnt; e += NT) {
      const int o = lo + e;
      const T rv = Rn[H + e];
      T wv = T(0);
      if (interior(o)) wv = stencil19(Rn + H + e, sy, sz, c0, fx, fy, fz, exy, exz, eyz);
      Wn[e] = wv;
      acc_g = fma((double)rv, (double)rv, acc_g);
      acc_d = fma((double)wv, (double)rv, acc_d);
    }
    const double2 red = cluster_sum2<NW>(acc_g, acc_d, s_park, s_slots[par ^ 1], me, csize);
    if (warp == 0) {
      const double gn = red.x, dn = red.y;
      iter += 1;
      if (me == 0 && lane == 0 && d.hist && iter < d.hist_len) d.hist[iter] = gn;
      int st_ = 0;
      if (!isfinite(gn) || !isfinite(dn)) {
        status = EXCMG_ERR_NONFINITE;
        st_ = 1;
      } else if (gn <= tol2 || gn == 0.0) {
        st_ = 1;  // converged (or exact solution in fixed-count mode)
      } else if (iter >= max_iter) {
        if (!fixed) status = EXCMG_ERR_NOT_CONVERGED;
        st_ = 1;
      } else {
        // beta' = gn / gam;  alpha' = gn / (dn - beta' gn / alpha) = gn k / (dn k - gn^2)
        // with k = gam alpha: both divides in one instruction (lanes 0 and 1)
        const double k = gam * alpha;
        const double den = fma(dn, k, -gn * gn);
        if (!(den > 0.0)) {
          status = EXCMG_ERR_NONFINITE;
          st_ = 1;
        } else {
          const double q = (lane == 0 ? gn * k : gn) / (lane == 0 ? den : gam);
          alpha = __shfl_sync(0xffffffffu, q, 0);
          beta = __shfl_sync(0xffffffffu, q, 1);
        }
      }
      gam = gn;
      delta = dn;
      if (lane == 0) {
        s_stop = st_;
        s_alpha = alpha;
        s_beta = beta;
      }
    }
    __syncthreads();
    stop = s_stop != 0;
    par ^= 1;
  }
  // x_{i+1} and r_{i+1} (r in R[par] after the flip)
  const T* Rf = par ? R1 : R0;
  for (int e = threadIdx.x; e < cnt; e += NT) {
    d.x[lo + e] = xs[e];
    d.r[lo + e] = Rf[H + e];
  }
  if (me == 0 && threadIdx.x == 0) {
    S->rr = gam;
    S->pq = delta;
    S->alpha = alpha;
    S->beta = beta;
    S->iter = iter;
    S->first = 0;
    S->status = status;
    S->done = 1;
  }
  cl_sync();  // no CTA leaves while a peer could still address its shared memory
}

constexpr size_t kClStaticSmem = 10 * 1024;  // static shared memory of k_cg_cluster (<= 512 threads), rounded up

int g_cl_max_smem = 0;           // largest dynamic shared memory per CTA (opt-in)
int g_cl_ok[2][5] = {};          // [T][log2 C]: 0 unknown, 1 launchable, -1 not

template <typename T, int NT>
bool cluster_attrs() {
  if (cudaFuncSetAttribute(k_cg_cluster<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           g_cl_max_smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_cg_cluster<T, NT>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                           1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

template <typename T>
int cluster_ok(int lc) {
  int& ok = g_cl_ok[sizeof(T) == 8 ? 0 : 1][lc];
  if (ok != 0) return ok;
  ok = -1;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  g_cl_max_smem = optin - (int)kClStaticSmem;
  if (g_cl_max_smem <= 0) return ok;
  if (!cluster_attrs<T, 128>() || !cluster_attrs<T, 256>() || !cluster_attrs<T, 512>()) return ok;
  // the largest CTA with the largest shared memory: every smaller launch fits too
  const int C = 1 << lc;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = (size_t)g_cl_max_smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, k_cg_cluster<T, 512>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return ok;
  }
  ok = ncl > 0 ? 1 : -1;
  return ok;
}

}  // namespace

size_t cluster_cg_smem(const Grid3& g, int csize, size_t elem) {
  const long long n = g.nodes();
  const long long m = (n + csize - 1) / csize;
  const long long H = g.sy + g.sz;
  return (size_t)(8 * m + 4 * H) * elem;
}

#ifndef EXCMG_CLUSTER_NODES_PER_CTA
#define EXCMG_CLUSTER_NODES_PER_CTA 160
#endif

template <typename T>
int cluster_cg_size(const Grid3& g) {
  const long long n = g.nodes();
  int lc = 0;
  while (lc < 4 && (n + (1LL << lc) - 1) / (1LL << lc) > EXCMG_CLUSTER_NODES_PER_CTA) ++lc;
  // the smallest size from there whose shared memory fits and that the device can launch
  for (; lc <= 4; ++lc) {
    if (cluster_ok<T>(lc) != 1) continue;
    if (cluster_cg_smem(g, 1 << lc, sizeof(T)) <= (size_t)g_cl_max_smem) return 1 << lc;
  }
  return 0;
}
template int cluster_cg_size<double>(const Grid3&);
template int cluster_cg_size<float>(const Grid3&);

template <typename T>
cudaError_t launch_cg_cluster(int nprob, const CGDesc<T>* descs, int csize, size_t smem,
                              long long max_nodes, CGState* st, cudaStream_t s) {
  // threads per CTA from the nodes per CTA: small ranges keep the reduction tree short
  const long long m = (max_nodes + csize - 1) / csize;
  const int nt = m <= 160 ? 128 : (m <= 640 ? 256 : 512);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nprob * csize));
  cfg.blockDim = dim3((unsigned)nt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (nt == 128) return cudaLaunchKernelEx(&cfg, k_cg_cluster<T, 128>, descs, st, csize);
  if (nt == 256) return cudaLaunchKernelEx(&cfg, k_cg_cluster<T, 256>, descs, st, csize);
  return cudaLaunchKernelEx(&cfg, k_cg_cluster<T, 512>, descs, st, csize);
}
template cudaError_t launch_cg_cluster<double>(int, const CGDesc<double>*, int, size_t, long long,
                                               CGState*, cudaStream_t);
template cudaError_t launch_cg_cluster<float>(int, const CGDesc<float>*, int, size_t, long long,
                                              CGState*, cudaStream_t);

}  // namespace excmg
