// Level CG with the level's vectors resident in shared memory, for one grid of up to a
// few hundred thousand nodes (the middle levels of the cascade, where a CG step is bound
// by latency, not by the FP64 pipe or HBM).
//
// A cooperative grid of G blocks; block b owns a box of BX x BY x BZ interior nodes and
// keeps in shared memory, for all steps of the level, x, p, s, w of its box and r of its
// box plus a one-node halo.  The recurrence is the single-reduction form of CG of
// Chronopoulos and Gear (1989), as in the cluster kernel:
//
//    p = r + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,
//    w = A r,  gamma = r.r,  delta = w.r   (one grid reduction for both),
//    beta' = gamma' / gamma,  alpha' = gamma' / (delta' - beta' gamma' / alpha);
//
// in exact arithmetic x and r are those of the standard recurrence (the smoother of
// Algorithm 1), and the loop stops on the same recursive residual r.r <= tol2.
//
// Halo exchange through global memory (L2): every step each block publishes the new r, s
// and w of its box into node arrays of the level (two copies by step parity), and the
// next step recomputes the new r on its halo from its neighbours' published r, w, s with
// the same fused operations as the owner (bit-identical).  So one step needs one grid-wide
// synchronisation, the reduction's: per-block partials, one arrival counter (release /
// acquire, bounded wait: EXCMG_ERR_TIMEOUT), then every block adds the G partials in
// index order, so all blocks hold bit-identical scalars and take the same decisions.
#include <cuda_runtime.h>

#include <algorithm>

#include "excmg_internal.cuh"

namespace excmg {
namespace {

constexpr int kRsThreads = 256;
constexpr unsigned long long kRsSpinLimit = 1ull << 25;
constexpr int kRsHB = 6;  // halo nodes per thread whose loads are issued ahead
constexpr int kRsPB = 8;  // block partials per lane in flight

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ double rs_xor_sum(double v, int from) {
  for (int o = from; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sums of (a, b) over the first nw warps (the warps that own nodes; the others
// hold zeros), valid in every lane of warp 0.  Those threads park their values in shared
// memory; warp 0 adds them with a and b packed into the two half-warps (lanes 0-15 the
// a-values, lanes 16-31 the b-values: 2 nw values per lane as a pairwise tree, then a
// butterfly over 16 lanes), so each level of the dependence chain is one float64 warp
// instruction for both sums.  On GB300 every float64 warp instruction costs the narrow
// FP64 pipe the same whether it carries one sum or two.  nw is the same in every block.
__device__ double2 rs_block_sum2(double a, double b, double* s_park, int nw) {
  if (threadIdx.x < 32 * nw) {
    s_park[threadIdx.x] = a;
    s_park[kRsThreads + threadIdx.x] = b;
  }
  __syncthreads();
  double2 t = make_double2(0.0, 0.0);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x, h = lane & 15;
    const double* src = s_park + (lane < 16 ? 0 : kRsThreads);
    const int nv = 2 * nw;  // values per lane
    double v[kRsThreads / 16];
#pragma unroll
    for (int u = 0; u < kRsThreads / 16; ++u) v[u] = u < nv ? src[h + 16 * u] : 0.0;
#pragma unroll
    for (int w = 1; w < kRsThreads / 16; w *= 2)
#pragma unroll
      for (int u = 0; u + w < kRsThreads / 16; u += 2 * w)
        if (u + w < nv) v[u] += v[u + w];
    const double r = rs_xor_sum(v[0], 8);
    t = make_double2(__shfl_sync(0xffffffffu, r, 0), __shfl_sync(0xffffffffu, r, 16));
  }
  return t;
}

// Reduction number `seq` (1, 2, ...): thread 0 stores this block's partials as pair b of
// the set seq & 1 (two sets: a block can be one reduction ahead of another's reads, never
// two), arrives on the counter with release semantics -- which also publishes every
// global store the block's threads made before the block barrier that precedes this
// call -- and waits (bounded) until all G blocks have arrived.  Returns, in every
// thread, false if the wait ran out or another block reported a time-out.
__device__ bool rs_arrive_wait(double2 part, double2* pairs, unsigned* counter, int G, unsigned seq,
                               int* err, int* s_ok) {
  if (threadIdx.x == 0) {
    __stcg(&pairs[(size_t)(seq & 1) * G + blockIdx.x], part);
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(counter) : "memory");
    const unsigned target = seq * (unsigned)G;
    int ok = 1;
    unsigned long long spins = 0;
    while (ld_acquire_u32(counter) < target) {
      if (++spins > kRsSpinLimit || *(volatile int*)err) {
        ok = 0;
        break;
      }
      if (spins > 4096) __nanosleep(64);
    }
    if (!ok) atomicExch(err, 1);
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Warp 0, after the wait: the sums of the G pairs of set seq & 1, in a fixed order,
// identical in every lane and every block.  As in rs_block_sum2 the two sums share the
// warp: lanes 0-15 take the first members of pairs h, h + 16, ... (h = lane mod 16),
// lanes 16-31 the second members (kRsPB loads in flight, a tree within the lane), then a
// butterfly over 16 lanes.
__device__ double2 rs_read_pairs(const double2* pairs, int G, unsigned seq) {
  const double* set = reinterpret_cast<const double*>(pairs + (size_t)(seq & 1) * G);
  const int lane = threadIdx.x & 31, h = lane & 15, m = lane >> 4;
  double acc = 0.0;
  for (int i0 = 0; i0 < G; i0 += 16 * kRsPB) {
    const int nv = min(kRsPB, (G - i0 + 15) / 16);  // values per lane in this chunk
    double v[kRsPB];
#pragma unroll
    for (int u = 0; u < kRsPB; ++u) {
      const int i = i0 + h + 16 * u;
      v[u] = i < G ? __ldcg(set + 2 * i + m) : 0.0;
    }
#pragma unroll
    for (int w = 1; w < kRsPB; w *= 2)
#pragma unroll
      for (int u = 0; u + w < kRsPB; u += 2 * w)
        if (u + w < nv) v[u] += v[u + w];
    acc += v[0];
  }
  const double r = rs_xor_sum(acc, 8);
  return make_double2(__shfl_sync(0xffffffffu, r, 0), __shfl_sync(0xffffffffu, r, 16));
}

// 19-point A-stencil at offset 0 of P with strides (1, ey, ez).  `shallow`: the seven
// weighted terms as a tree (two more float64 instructions, three fewer levels of
// dependence) -- for boxes of at most one node per thread, where a step waits on the
// chain rather than on the FP64 pipe's throughput.
__device__ __forceinline__ double rs_stencil(const double* P, int ey, int ez, const Coef& A,
                                             bool shallow) {
  const double SX = P[-1] + P[1], SY = P[-ey] + P[ey], SZ = P[-ez] + P[ez];
  const double EXY = (P[-1 - ey] + P[1 - ey]) + (P[-1 + ey] + P[1 + ey]);
  const double EXZ = (P[-1 - ez] + P[1 - ez]) + (P[-1 + ez] + P[1 + ez]);
  const double EYZ = (P[-ey - ez] + P[ey - ez]) + (P[-ey + ez] + P[ey + ez]);
  if (shallow) {
    const double t1 = fma(A.c0, P[0], A.fx * SX), t2 = fma(A.fy, SY, A.fz * SZ);
    const double t3 = fma(A.exy, EXY, A.exz * EXZ);
    return (t1 + t2) + fma(A.eyz, EYZ, t3);
  }
  return fma(A.c0, P[0], fma(A.fx, SX, fma(A.fy, SY, fma(A.fz, SZ, fma(A.exy, EXY, fma(A.exz, EXZ, A.eyz * EYZ))))));
}

__global__ void __launch_bounds__(kRsThreads)
    k_cg_resident(const ResidentDesc D, CGState* st, double2* pairs, unsigned* counter, int* err) {
  extern __shared__ __align__(16) double s_vec[];
  __shared__ double s_park[2 * kRsThreads];
  __shared__ int s_ok;
  __shared__ double s_alpha, s_beta;
  __shared__ int s_stop;
  CGState* S = st + D.slot;
  if (S->done) return;  // identical in every block: the state is written after the last wait
  const Grid3 g = D.g;
  const int G = gridDim.x;
  const int BX = D.bx, BY = D.by, BZ = D.bz;
  const int EX = BX + 2, EY = BY + 2, EZ = BZ + 2;
  const int B = BX * BY * BZ, ext = EX * EY * EZ;
  const int nw_own = min(kRsThreads, B + 31) / 32;  // warps that own nodes
  const bool shallow = B <= kRsThreads;               // at most one node per thread
  const int b = blockIdx.x;
  const int ibx = b % D.nbx, iby = (b / D.nbx) % D.nby, ibz = b / (D.nbx * D.nby);
  // global node of box-local (0, 0, 0); the halo starts one node before
  const int i0 = 1 + ibx * BX, j0 = 1 + iby * BY, k0 = 1 + ibz * BZ;
  double* R = s_vec;  // ext: (lx+1) + EX (ly+1) + EX EY (lz+1)
  double* X = R + ext;
  double* P = X + B;
  double* Sv = P + B;
  double* W = Sv + B;
  const Coef A = D.A;
  // own node q of the box: its index in R and in the level's node array; valid = the
  // node exists (boxes at the far faces of the grid may be partial)
  struct Own {
    int e;
    bool valid;
    long long o;
  };
  auto own_node = [&](int q) -> Own {
    const int lx = q % BX, ly = (q / BX) % BY, lz = q / (BX * BY);
    const int gi = i0 + lx, gj = j0 + ly, gk = k0 + lz;
    Own w;
    w.e = (lx + 1) + EX * ((ly + 1) + EY * (lz + 1));
    w.o = gi + gj * g.sy + (long long)gk * g.sz;
    w.valid = gi < g.nx && gj < g.ny && gk < g.nz;
    return w;
  };
  // boxes of at most one node per thread: this thread's node, computed once (the index
  // arithmetic divides by the box extents) instead of in every step
  const Own mine = own_node(threadIdx.x < B ? threadIdx.x : 0);
  auto node_of = [&](int q) -> Own { return shallow ? mine : own_node(q); };
  // shell position h (0 .. ext - B - 1): the 2 z-faces, then the 2 y-faces, then the 2
  // x-faces of the extended box
  const int zf = EX * EY, yf = EX * BZ, xf = BY * BZ;
  const int nshell = 2 * (zf + yf + xf);
  auto shell_node = [&](int h, int& e, int& gi, int& gj, int& gk) {
    int ex, ey, ez;
    if (h < 2 * zf) {
      ez = h < zf ? 0 : EZ - 1;
      const int r = h % zf;
      ex = r % EX;
      ey = r / EX;
    } else if (h < 2 * (zf + yf)) {
      const int h2 = h - 2 * zf;
      ey = h2 < yf ? 0 : EY - 1;
      const int r = h2 % yf;
      ex = r % EX;
      ez = 1 + r / EX;
    } else {
      const int h3 = h - 2 * (zf + yf);
      ex = h3 < xf ? 0 : EX - 1;
      const int r = h3 % xf;
      ey = 1 + r % BY;
      ez = 1 + r / BY;
    }
    e = ex + EX * (ey + EY * ez);
    gi = i0 - 1 + ex;
    gj = j0 - 1 + ey;
    gk = k0 - 1 + ez;
  };
  auto interior = [&](int gi, int gj, int gk) {
    return gi > 0 && gi < g.nx && gj > 0 && gj < g.ny && gk > 0 && gk < g.nz;
  };
  // ---- start: r_0 on the box and its halo, x; p = s = 0; w_0 = A r_0; publish w_0, s = 0
  for (int e = threadIdx.x; e < ext; e += kRsThreads) R[e] = 0.0;
  __syncthreads();
  for (int q = threadIdx.x; q < B; q += kRsThreads) {
    const Own w = own_node(q);
    R[w.e] = w.valid ? D.r[w.o] : 0.0;
    X[q] = w.valid ? D.x[w.o] : 0.0;
    P[q] = 0.0;
    Sv[q] = 0.0;
  }
  for (int h = threadIdx.x; h < nshell; h += kRsThreads) {
    int e, gi, gj, gk;
    shell_node(h, e, gi, gj, gk);
    R[e] = interior(gi, gj, gk) ? D.r[gi + gj * g.sy + (long long)gk * g.sz] : 0.0;
  }
  __syncthreads();
  double acc_d = 0.0;
  for (int q = threadIdx.x; q < B; q += kRsThreads) {
    const Own n = own_node(q);
    double w = 0.0;
    if (n.valid) {
      w = rs_stencil(R + n.e, EX, EX * EY, A, shallow);
      acc_d = fma(w, R[n.e], acc_d);
      D.w0[n.o] = w;
      D.s0[n.o] = 0.0;
    }
    W[q] = w;
  }
  // CG scalars: warp 0 keeps identical copies in all its lanes (and in every block)
  double gam = S->rr, alpha = 0.0, beta = 0.0, delta = 0.0;
  const double tol2 = S->tol2;
  int iter = S->iter;
  const int max_iter = S->max_iter, fixed = S->fixed;
  int status = EXCMG_OK;
  const int lane = threadIdx.x & 31;
  // the published r, w, s of up to kRsHB halo nodes per thread, loaded right after each
  // reduction's wait, so that the load latency overlaps the reading of the partials and
  // the scalar arithmetic (zero on the boundary)
  double hr[kRsHB], hw[kRsHB], hs[kRsHB];
  int he[kRsHB];
  // this thread's shell nodes (index in R, offset in the level's arrays or -1 outside the
  // interior), computed once: after each wait the loads issue at once
  int ho[kRsHB];
#pragma unroll
  for (int u = 0; u < kRsHB; ++u) {
    const int h = threadIdx.x + u * kRsThreads;
    he[u] = -1;
    ho[u] = -1;
    if (h < nshell) {
      int gi, gj, gk;
      shell_node(h, he[u], gi, gj, gk);
      if (interior(gi, gj, gk)) ho[u] = gi + gj * g.sy + gk * g.sz;
    }
  }
  auto load_halo = [&](int par) {
    const double* Rg = par ? D.r1 : D.r;
    const double* Wg = par ? D.w1 : D.w0;
    const double* Sg = par ? D.s1 : D.s0;
#pragma unroll
    for (int u = 0; u < kRsHB; ++u) {
      hr[u] = hw[u] = hs[u] = 0.0;
      if (ho[u] >= 0) {
        hr[u] = __ldcg(Rg + ho[u]);
        hw[u] = __ldcg(Wg + ho[u]);
        hs[u] = __ldcg(Sg + ho[u]);
      }
    }
  };
  unsigned seq = 1;
  {
    const double2 part = rs_block_sum2(0.0, acc_d, s_park, nw_own);
    const bool ok = rs_arrive_wait(part, pairs, counter, G, seq, err, &s_ok);
    if (ok) load_halo(0);
    if (threadIdx.x < 32) {
      int stop = 0;
      if (!ok) {
        status = EXCMG_ERR_TIMEOUT;
        stop = 1;
      } else {
        delta = rs_read_pairs(pairs, G, seq).y;
        if (delta == 0.0 && gam == 0.0) {
          stop = 1;  // exact solution (fixed-count mode)
        } else if (!(delta > 0.0) || !isfinite(delta)) {
          status = EXCMG_ERR_NONFINITE;
          stop = 1;
        } else {
          alpha = gam / delta;
        }
      }
      if (lane == 0) {
        s_stop = stop;
        s_alpha = alpha;
        s_beta = 0.0;
      }
    }
    ++seq;
    __syncthreads();
  }
  int par = 0;  // step i reads the published r_i, w_i, s_{i-1} of parity par
  while (!s_stop) {
    const double a = s_alpha, bt = s_beta;
    const double* Rg = par ? D.r1 : D.r;
    const double* Wg = par ? D.w1 : D.w0;
    const double* Sg = par ? D.s1 : D.s0;
    double* Rn = par ? D.r : D.r1;
    double* Wn = par ? D.w0 : D.w1;
    double* Sn = par ? D.s0 : D.s1;
    // 1. own nodes: p, s, x, r; publish r and s
    for (int q = threadIdx.x; q < B; q += kRsThreads) {
      const Own n = node_of(q);
      if (!n.valid) continue;
      const int e = n.e;
      const long long o = n.o;
      const double r = R[e];
      const double pv = fma(bt, P[q], r);
      const double sv = fma(bt, Sv[q], W[q]);
      P[q] = pv;
      Sv[q] = sv;
      X[q] = fma(a, pv, X[q]);
      const double rn = fma(-a, sv, r);
      R[e] = rn;
      __stcg(Rn + o, rn);
      __stcg(Sn + o, sv);
    }
    // 2. the halo's new r, with the owner's fused operations; shells larger than kRsHB
    // per thread finish with plain loads
#pragma unroll
    for (int u = 0; u < kRsHB; ++u)
      if (he[u] >= 0) R[he[u]] = fma(-a, fma(bt, hs[u], hw[u]), hr[u]);
    for (int h = threadIdx.x + kRsHB * kRsThreads; h < nshell; h += kRsThreads) {
      int e, gi, gj, gk;
      shell_node(h, e, gi, gj, gk);
      double rn = 0.0;
      if (interior(gi, gj, gk)) {
        const long long o = gi + gj * g.sy + (long long)gk * g.sz;
        rn = fma(-a, fma(bt, __ldcg(Sg + o), __ldcg(Wg + o)), __ldcg(Rg + o));
      }
      R[e] = rn;
    }
    __syncthreads();
    // 3. w = A r, gamma, delta; publish w
    double acc_g = 0.0;
    acc_d = 0.0;
    for (int q = threadIdx.x; q < B; q += kRsThreads) {
      const Own n = node_of(q);
      double w = 0.0;
      if (n.valid) {
        const double r = R[n.e];
        w = rs_stencil(R + n.e, EX, EX * EY, A, shallow);
        acc_g = fma(r, r, acc_g);
        acc_d = fma(w, r, acc_d);
        __stcg(Wn + n.o, w);
      }
      W[q] = w;
    }
    // 4. the grid reduction (it also orders every block's publications before the next
    // step's halo loads); the next halo's loads; scalars
    const double2 part = rs_block_sum2(acc_g, acc_d, s_park, nw_own);
    const bool ok = rs_arrive_wait(part, pairs, counter, G, seq, err, &s_ok);
    par ^= 1;
    if (ok) load_halo(par);
    if (threadIdx.x < 32) {
      int stop = 0;
      if (!ok) {
        status = EXCMG_ERR_TIMEOUT;
        stop = 1;
      } else {
        const double2 red = rs_read_pairs(pairs, G, seq);
        const double gn = red.x, dn = red.y;
        iter += 1;
        if (b == 0 && lane == 0 && D.hist && iter < D.hist_len) D.hist[iter] = gn;
        if (!isfinite(gn) || !isfinite(dn)) {
          status = EXCMG_ERR_NONFINITE;
          stop = 1;
        } else if (gn <= tol2 || gn == 0.0) {
          stop = 1;  // converged (or exact solution in fixed-count mode)
        } else if (iter >= max_iter) {
          if (!fixed) status = EXCMG_ERR_NOT_CONVERGED;
          stop = 1;
        } else {
          // alpha' = gn / (dn - beta' gn / alpha) = gn k / (dn k - gn^2), k = gam alpha;
          // beta' = gn / gam: both divides in one instruction (lanes 0 and 1)
          const double k = gam * alpha;
          const double den = fma(dn, k, -gn * gn);
          if (!(den > 0.0)) {
            status = EXCMG_ERR_NONFINITE;
            stop = 1;
          } else {
            const double q = (lane == 0 ? gn * k : gn) / (lane == 0 ? den : gam);
            alpha = __shfl_sync(0xffffffffu, q, 0);
            beta = __shfl_sync(0xffffffffu, q, 1);
          }
        }
        gam = gn;
        delta = dn;
      }
      if (lane == 0) {
        s_stop = stop;
        s_alpha = alpha;
        s_beta = beta;
      }
    }
    ++seq;
    __syncthreads();
  }
  // x and the last r of the box
  for (int q = threadIdx.x; q < B; q += kRsThreads) {
    const Own n = own_node(q);
    if (!n.valid) continue;
    D.x[n.o] = X[q];
    D.r[n.o] = R[n.e];
  }
  if (b == 0 && threadIdx.x == 0) {
    S->rr = gam;
    S->pq = delta;
    S->alpha = alpha;
    S->beta = beta;
    S->iter = iter;
    S->first = 0;
    S->status = status;
    S->done = 1;
  }
}

int g_rs_blocks_per_sm = 0;  // at the largest shared memory a box may take
int g_rs_sms = 0;
size_t g_rs_max_smem = 0;

}  // namespace

size_t resident_smem(int bx, int by, int bz) {
  const size_t ext = (size_t)(bx + 2) * (by + 2) * (bz + 2);
  return sizeof(double) * (ext + 4 * (size_t)bx * by * bz);
}

#ifndef EXCMG_RESIDENT_MAX_SMEM
#define EXCMG_RESIDENT_MAX_SMEM (96 * 1024)
#endif

bool resident_box(const Grid3& g, ResidentDesc& D, size_t& smem) {
  if (g_rs_sms == 0) {
    int dev = 0, coop = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&g_rs_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    g_rs_max_smem = std::min<size_t>(EXCMG_RESIDENT_MAX_SMEM, (size_t)std::max(0, optin - 2048));
    if (!coop || g_rs_sms <= 0 ||
        cudaFuncSetAttribute(k_cg_resident, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)g_rs_max_smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_rs_blocks_per_sm, k_cg_resident, kRsThreads,
                                                      g_rs_max_smem) != cudaSuccess) {
      cudaGetLastError();
      g_rs_blocks_per_sm = 0;
    }
    if (g_rs_sms <= 0) g_rs_sms = 1;
  }
  if (g_rs_blocks_per_sm <= 0) return false;
  const int ni = g.nx - 1, nj = g.ny - 1, nk = g.nz - 1;
  if (ni < 1 || nj < 1 || nk < 1) return false;
  const long long max_blocks = std::min<long long>((long long)g_rs_sms * g_rs_blocks_per_sm, kMaxGrid);
  // per-step model in SM clocks: the busiest SM's float64 work (~12.5 clocks per node,
  // 2 DFMA per clock, plus ~400 per block for its reduction), the halo loads of a box
  // (3 per shell node), and the grid reduction's share per block (arrival, partials)
  double best = 1e300;
  bool found = false;
  const int bxs[] = {32, 16, 8};
  const int bys[] = {1, 2, 4, 8, 16, 32};
  const int bzs[] = {1, 2, 4, 8, 16, 32};
  for (int bx : bxs)
    for (int by : bys)
      for (int bz : bzs) {
        const long long nb = (long long)((ni + bx - 1) / bx) * ((nj + by - 1) / by) * ((nk + bz - 1) / bz);
        if (nb > max_blocks) continue;
        const size_t sm = resident_smem(bx, by, bz);
        if (sm > g_rs_max_smem) continue;
        const double B = (double)bx * by * bz;
        const double shell = (double)(bx + 2) * (by + 2) * (bz + 2) - B;
        const double per_sm = (double)((nb + g_rs_sms - 1) / g_rs_sms);
        const double cost = per_sm * (B * 12.5 + 400.0) + shell * 6.0 + (double)nb * 12.0;
        if (cost < best) {
          best = cost;
          found = true;
          D.bx = bx;
          D.by = by;
          D.bz = bz;
          D.nbx = (ni + bx - 1) / bx;
          D.nby = (nj + by - 1) / by;
          D.nbz = (nk + bz - 1) / bz;
          smem = sm;
        }
      }
  return found;
}

cudaError_t launch_cg_resident(const ResidentDesc& D, size_t smem, CGState* st, double2* pairs,
                               unsigned* counter, int* err, cudaStream_t s) {
  const int grid = D.nbx * D.nby * D.nbz;
  ResidentDesc d = D;
  void* args[] = {(void*)&d, (void*)&st, (void*)&pairs, (void*)&counter, (void*)&err};
  return cudaLaunchCooperativeKernel((const void*)k_cg_resident, dim3(grid), dim3(kRsThreads), args,
                                     smem, s);
}

}  // namespace excmg
