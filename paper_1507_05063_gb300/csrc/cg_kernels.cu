// Matrix-free stencil CG for the 19-point compact scheme (Section 2, eq. compact) and
// the CG loop of Algorithm 1 (lines 7-9).
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
__device__ double block_sum(double v) {
  __shared__ double s_w[kThreads / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_w[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (lane < kThreads / 32) ? s_w[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
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
    for (int v = 0; v < NV; ++v) {
      double acc = 0.0;
      const volatile double* src = partials + ((long long)p * NV + v) * G;
      for (int i = threadIdx.x; i < G; i += blockDim.x) acc += src[i];
      sums[v] = block_sum(acc);
    }
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
    const double bb = d.want_b ? s[1] : S.bb;
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
    S.done = d.fixed ? (d.max_iter <= 0) : (rr <= S.tol2 || d.max_iter <= 0);
    if (!isfinite(rr) || !isfinite(bb)) {
      S.status = EXCMG_ERR_NONFINITE;
      S.done = 1;
    }
  }
};

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
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
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
    const Grid3 g = d.g;
    const CGState& S = st[d.slot];
    const bool first = S.first != 0;
    const T beta = (T)S.beta;
    const int it = S.iter;
    const T* __restrict__ r = d.r;
    const T* __restrict__ pold = (it & 1) ? d.pb : d.pa;
    T* __restrict__ pnew = (it & 1) ? d.pa : d.pb;
    T* __restrict__ q = d.q;
    const TileXYZ c = tile_coords(g, d.t, t - d.tile_begin);
    const int i = c.x0 + tx, j = c.y0 + ty;
    const bool own = (i <= g.nx) && (j <= g.ny);
    const bool inxy = (i > 0) && (i < g.nx) && (j > 0) && (j < g.ny);
    const T c0 = (T)d.A.c0, fx = (T)d.A.fx, fy = (T)d.A.fy, fz = (T)d.A.fz;
    const T exy = (T)d.A.exy, exz = (T)d.A.exz, eyz = (T)d.A.eyz;
    T Pm1 = T(0), Cm1 = T(0), Tm1 = T(0), Tm2 = T(0), tacc = T(0);
    for (int kk = c.z0 - 1; kk <= c.z1; ++kk) {
      const bool plane_in = (kk >= 0) && (kk <= g.nz);
      for (int idx = threadIdx.x; idx < (kTX + 2) * (kTY + 2); idx += kThreads) {
        const int ly = idx / (kTX + 2), lx = idx - ly * (kTX + 2);
        const int gi = c.x0 - 1 + lx, gj = c.y0 - 1 + ly;
        T v = T(0);
        if (plane_in && gi >= 0 && gi <= g.nx && gj >= 0 && gj <= g.ny) {
          const long long o = gi + gj * g.sy + (long long)kk * g.sz;
          v = first ? r[o] : fmaT(beta, pold[o], r[o]);
        }
        sp[buf][ly][lx] = v;
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
    acc += (double)tacc;
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
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
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
    const Grid3 g = d.g;
    const CGState& S = st[d.slot];
    const T alpha = (T)S.alpha;
    const int it = S.iter;
    const T* __restrict__ pn = (it & 1) ? d.pa : d.pb;
    const T* __restrict__ q = d.q;
    T* __restrict__ x = d.x;
    T* __restrict__ r = d.r;
    const TileXYZ c = tile_coords(g, d.t, t - d.tile_begin);
    const int i = c.x0 + tx, j = c.y0 + ty;
    T tacc = T(0);
    if (i <= g.nx && j <= g.ny) {
      long long o = i + j * g.sy + (long long)c.z0 * g.sz;
#pragma unroll 4
      for (int k = c.z0; k < c.z1; ++k, o += g.sz) {
        const T xv = fmaT(alpha, pn[o], x[o]);
        const T rv = fmaT(-alpha, q[o], r[o]);
        x[o] = xv;
        r[o] = rv;
        tacc = fmaT(rv, rv, tacc);
      }
    }
    acc += (double)tacc;
  }
  if (cur >= 0) {
    const double s = block_sum(acc);
    if (threadIdx.x == 0) s_part[cur] += s;
  }
  __syncthreads();
  publish_and_finish<1>(nprob, s_active, s_part, partials, counters, FinBeta<T>{descs, st});
}

// ---------------------------------------------------------------------------------
// K3: r = LHS(u) - RHS(f) = b - A u_I (float64), sums r.r and b.b, CG state init
// ---------------------------------------------------------------------------------
template <typename TR>
__global__ void __launch_bounds__(kThreads)
    k_residual(int nprob, const ResDesc* __restrict__ descs, long long total_tiles,
               CGState* st, double* partials, unsigned* counters) {
  __shared__ double su[2][kTY + 2][kTX + 2];
  __shared__ double sb[2][kTY + 2][kTX + 2];
  __shared__ int s_active[kMaxProb];
  __shared__ double s_part[2 * kMaxProb];
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
    s_active[p] = 1;
    s_part[2 * p] = 0.0;
    s_part[2 * p + 1] = 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  int buf = 0, cur = -1, p = 0;
  double acc_r = 0.0, acc_b = 0.0;
  for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    p = find_problem(descs, nprob, t, p);
    if (p != cur) {
      if (cur >= 0) {
        const double s1 = block_sum(acc_r);
        const double s2 = block_sum(acc_b);
        if (threadIdx.x == 0) {
          s_part[2 * cur] += s1;
          s_part[2 * cur + 1] += s2;
        }
      }
      acc_r = acc_b = 0.0;
      cur = p;
    }
    const ResDesc& d = descs[p];
    const Grid3 g = d.g;
    const double* __restrict__ u = d.u;
    TR* __restrict__ rout = reinterpret_cast<TR*>(d.r);
    const TileXYZ c = tile_coords(g, d.t, t - d.tile_begin);
    const int i = c.x0 + tx, j = c.y0 + ty;
    const bool own = (i <= g.nx) && (j <= g.ny);
    const bool inxy = (i > 0) && (i < g.nx) && (j > 0) && (j < g.ny);
    const Coef A = d.A;
    // C/T terms of the stencil of u (all 19 nodes) and of its boundary part (the lift)
    double Cm1 = 0, Tm1 = 0, Tm2 = 0, LCm1 = 0, LTm1 = 0, LTm2 = 0;
    for (int kk = c.z0 - 1; kk <= c.z1; ++kk) {
      const bool plane_in = (kk >= 0) && (kk <= g.nz);
      const bool plane_bnd = (kk == 0) || (kk == g.nz);
      for (int idx = threadIdx.x; idx < (kTX + 2) * (kTY + 2); idx += kThreads) {
        const int ly = idx / (kTX + 2), lx = idx - ly * (kTX + 2);
        const int gi = c.x0 - 1 + lx, gj = c.y0 - 1 + ly;
        double v = 0.0, vb = 0.0;
        if (plane_in && gi >= 0 && gi <= g.nx && gj >= 0 && gj <= g.ny) {
          v = u[gi + gj * g.sy + (long long)kk * g.sz];
          const bool bnd = plane_bnd || gi == 0 || gi == g.nx || gj == 0 || gj == g.ny;
          vb = bnd ? v : 0.0;
        }
        su[buf][ly][lx] = v;
        sb[buf][ly][lx] = vb;
      }
      __syncthreads();
      double Ck, Tk, LCk, LTk;
      {
        const double P = su[buf][ty + 1][tx + 1];
        const double SX = su[buf][ty + 1][tx] + su[buf][ty + 1][tx + 2];
        const double SY = su[buf][ty][tx + 1] + su[buf][ty + 2][tx + 1];
        const double EXY = (su[buf][ty][tx] + su[buf][ty][tx + 2]) + (su[buf][ty + 2][tx] + su[buf][ty + 2][tx + 2]);
        Ck = fma(A.c0, P, fma(A.fx, SX, fma(A.fy, SY, A.exy * EXY)));
        Tk = fma(A.fz, P, fma(A.exz, SX, A.eyz * SY));
      }
      {
        const double P = sb[buf][ty + 1][tx + 1];
        const double SX = sb[buf][ty + 1][tx] + sb[buf][ty + 1][tx + 2];
        const double SY = sb[buf][ty][tx + 1] + sb[buf][ty + 2][tx + 1];
        const double EXY = (sb[buf][ty][tx] + sb[buf][ty][tx + 2]) + (sb[buf][ty + 2][tx] + sb[buf][ty + 2][tx + 2]);
        LCk = fma(A.c0, P, fma(A.fx, SX, fma(A.fy, SY, A.exy * EXY)));
        LTk = fma(A.fz, P, fma(A.exz, SX, A.eyz * SY));
      }
      const int kc = kk - 1;
      if (kc >= c.z0 && own) {
        const long long o = i + j * g.sy + (long long)kc * g.sz;
        const bool interior = inxy && kc > 0 && kc < g.nz;
        double rv = 0.0;
        if (interior) {
          const View& F = d.f;
          const double rhs =
              d.src ? -d.src[o]
                    : 0.5 * (6.0 * F.at(i, j, kc) + ((F.at(i - 1, j, kc) + F.at(i + 1, j, kc)) +
                                                     (F.at(i, j - 1, kc) + F.at(i, j + 1, kc)) +
                                                     (F.at(i, j, kc - 1) + F.at(i, j, kc + 1))));
          // LHS(u) = -(A-stencil of u over all 19 nodes); b = LHS(boundary part) - RHS
          rv = -((Cm1 + Tm2) + Tk) - rhs;
          const double bv = -((LCm1 + LTm2) + LTk) - rhs;
          acc_r = fma(rv, rv, acc_r);
          acc_b = fma(bv, bv, acc_b);
        }
        rout[o] = (TR)rv;
      }
      Tm2 = Tm1;
      Tm1 = Tk;
      Cm1 = Ck;
      LTm2 = LTm1;
      LTm1 = LTk;
      LCm1 = LCk;
      buf ^= 1;
    }
  }
  if (cur >= 0) {
    const double s1 = block_sum(acc_r);
    const double s2 = block_sum(acc_b);
    if (threadIdx.x == 0) {
      s_part[2 * cur] += s1;
      s_part[2 * cur + 1] += s2;
    }
  }
  __syncthreads();
  publish_and_finish<2>(nprob, s_active, s_part, partials, counters, FinRes{descs, st});
}

// MIXED refinement: u += e (float32 correction), then e = 0 for the next inner solve.
__global__ void __launch_bounds__(kThreads)
    k_add_correction(int nprob, const CGDesc<float>* __restrict__ descs, long long total_tiles) {
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
    for (int k = c.z0; k < c.z1; ++k, o += g.sz) {
      d.aux[o] += (double)d.x[o];
      d.x[o] = 0.0f;
    }
  }
}

int g_max_grid = 0;

}  // namespace

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
                            cudaStream_t s) {
  if (out_float)
    k_residual<float><<<grid, kThreads, 0, s>>>(nprob, descs, total_tiles, st, partials, counters);
  else
    k_residual<double><<<grid, kThreads, 0, s>>>(nprob, descs, total_tiles, st, partials, counters);
  return cudaGetLastError();
}

cudaError_t launch_add_correction(int nprob, const CGDesc<float>* inner, long long total_tiles,
                                  int grid, cudaStream_t s) {
  k_add_correction<<<grid, kThreads, 0, s>>>(nprob, inner, total_tiles);
  return cudaGetLastError();
}

}  // namespace excmg
