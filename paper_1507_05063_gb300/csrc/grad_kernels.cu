// Gradient of the FD solution (Section 5, text of Example 1):
//  * boundary nodes of a line: the one-sided fourth-order five-point formulas
//      D_0 = (-25/12 u_0 + 4 u_1 - 3 u_2 + 4/3 u_3 - 1/4 u_4) / h, and its mirror at N;
//  * interior nodes: the compact (Collatz) system
//      (1/6) D_{i-1} + (4/6) D_i + (1/6) D_{i+1} = (u_{i+1} - u_{i-1}) / (2h),
//    solved by the Thomas algorithm on every grid line of the direction.
// The elimination factors of the constant tridiagonal matrix (c'_t = c / m_t,
// 1 / m_t with m_t = b - a c'_{t-1}) are the same for every line; they converge
// geometrically (ratio (2 - sqrt 3)^2 ~ 0.072 per step) so a 64-entry table holds them
// to the last bit and the last entry serves for t >= 64.  The forward sweep's values are
// kept in the output array and overwritten by the back substitution: no scratch memory.
// y- and z-lines: one thread per line, neighbouring threads on neighbouring x, so each
// step is a coalesced row access.  x-lines: one warp per 32 lines, staging 32-node
// chunks of the lines through shared memory so that global accesses stay coalesced.
#include <math.h>

#include "excmg_internal.cuh"

namespace excmg {

namespace {

constexpr int kTab = 64;
constexpr int kAhead = 8;  // line steps whose loads are in flight together (strided lines)

// The factors of the forward sweep written as dp_t = (u_{i+1} - u_{i-1}) A_t + B_t dp_{t-1}
// (A_t = (1/(2h)) / m_t, B_t = -(1/6) / m_t; the first step's dp_{t-1} is D_0, the
// last one's carries + D_N: the boundary derivatives moved to the right-hand side), and
// c'_t of the back substitution.
__device__ void thomas_table(double* cp, double* A, double* B, int n, double i2h) {
  // a = c = 1/6, b = 4/6
  const double a = 1.0 / 6.0, c = 1.0 / 6.0, b = 4.0 / 6.0;
  double prev = 0.0;
  const int m = n < kTab ? n : kTab;
  for (int t = 0; t < m; ++t) {
    const double piv = (t == 0) ? b : b - a * prev;
    const double im = 1.0 / piv;
    A[t] = i2h * im;
    B[t] = -a * im;
    cp[t] = c / piv;
    prev = cp[t];
  }
}

__device__ __forceinline__ double d_left(double u0, double u1, double u2, double u3, double u4, double ih) {
  return (-25.0 / 12.0 * u0 + 4.0 * u1 - 3.0 * u2 + 4.0 / 3.0 * u3 - 0.25 * u4) * ih;
}
__device__ __forceinline__ double d_right(double uN, double u1, double u2, double u3, double u4, double ih) {
  return (25.0 / 12.0 * uN - 4.0 * u1 + 3.0 * u2 - 4.0 / 3.0 * u3 + 0.25 * u4) * ih;
}

// Lines along a strided direction: node t of line L is base(L) + t * step.  Lines are
// indexed by (a, b) with a fastest: base = a * sa + b * sb.  A thread runs two lines,
// L and L + half (half = ceil(lines / 2)): two independent recurrences interleaved, so
// the dependent FP64 operations of one overlap the other's (each step of the forward
// sweep is a product and an FMA on the previous step's value); neighbouring threads
// still take neighbouring a, so every step stays a coalesced row access.
__global__ void __launch_bounds__(kThreads)
    k_grad_strided(const double* __restrict__ u, double* __restrict__ out, int N, double h,
                   long long step, int na, int nb, long long sa, long long sb) {
  __shared__ double cp[kTab], A[kTab], B[kTab];
  const double ih = 1.0 / h, i2h = 0.5 / h;
  if (threadIdx.x == 0) thomas_table(cp, A, B, N - 1, i2h);
  __syncthreads();
  const long long nl = (long long)na * nb, half = (nl + 1) / 2;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < half;
       L += (long long)gridDim.x * blockDim.x) {
    const bool two = L + half < nl;
    const long long L1 = two ? L + half : L;  // the second line (a copy of the first if none)
    const double* __restrict__ U0 = u + (L % na) * sa + (L / na) * sb;
    const double* __restrict__ U1 = u + (L1 % na) * sa + (L1 / na) * sb;
    double* __restrict__ D0p = out + (L % na) * sa + (L / na) * sb;
    double* __restrict__ D1p = out + (L1 % na) * sa + (L1 / na) * sb;
    const double a0 = d_left(U0[0], U0[step], U0[2 * step], U0[3 * step], U0[4 * step], ih);
    const double a1 = d_left(U1[0], U1[step], U1[2 * step], U1[3 * step], U1[4 * step], ih);
    const double n0 = d_right(U0[N * step], U0[(N - 1) * step], U0[(N - 2) * step], U0[(N - 3) * step],
                              U0[(N - 4) * step], ih);
    const double n1 = d_right(U1[N * step], U1[(N - 1) * step], U1[(N - 2) * step], U1[(N - 3) * step],
                              U1[(N - 4) * step], ih);
    D0p[0] = a0;
    D0p[N * step] = n0;
    if (two) {
      D1p[0] = a1;
      D1p[N * step] = n1;
    }
    // forward sweep over unknowns t = 0..N-2 (node i = t + 1), kAhead steps at a time:
    // the steps' loads are issued before their arithmetic, so each line has kAhead loads
    // in flight instead of one (the recurrence only waits on the first)
    double um0 = U0[0], uc0 = U0[step], dp0 = a0;
    double um1 = U1[0], uc1 = U1[step], dp1 = a1;
    auto fstep = [&](int i, double up0, double up1) {
      const int t = i - 1 < kTab ? i - 1 : kTab - 1;
      if (i == N - 1) {
        dp0 += n0;
        dp1 += n1;
      }
      dp0 = fma(B[t], dp0, (up0 - um0) * A[t]);
      dp1 = fma(B[t], dp1, (up1 - um1) * A[t]);
      D0p[(long long)i * step] = dp0;
      if (two) D1p[(long long)i * step] = dp1;
      um0 = uc0;
      uc0 = up0;
      um1 = uc1;
      uc1 = up1;
    };
    int i = 1;
    for (; i + kAhead - 1 <= N - 1; i += kAhead) {
      double q0[kAhead], q1[kAhead];
#pragma unroll
      for (int k = 0; k < kAhead; ++k) {
        const long long o = (long long)(i + 1 + k) * step;
        q0[k] = U0[o];
        q1[k] = U1[o];
      }
#pragma unroll
      for (int k = 0; k < kAhead; ++k) fstep(i + k, q0[k], q1[k]);
    }
    for (; i <= N - 1; ++i) {
      const long long o = (long long)(i + 1) * step;
      fstep(i, U0[o], U1[o]);
    }
    // back substitution, likewise kAhead nodes' loads at a time
    double x0 = dp0, x1 = dp1;
    auto bstep = [&](int i, double d0, double d1) {
      const int t = i - 1 < kTab ? i - 1 : kTab - 1;
      const long long o = (long long)i * step;
      x0 = d0 - cp[t] * x0;
      D0p[o] = x0;
      if (two) {
        x1 = d1 - cp[t] * x1;
        D1p[o] = x1;
      }
    };
    i = N - 2;
    for (; i - kAhead + 1 >= 1; i -= kAhead) {
      double r0[kAhead], r1[kAhead];
#pragma unroll
      for (int k = 0; k < kAhead; ++k) {
        const long long o = (long long)(i - k) * step;
        r0[k] = D0p[o];
        r1[k] = two ? D1p[o] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < kAhead; ++k) bstep(i - k, r0[k], r1[k]);
    }
    for (; i >= 1; --i) {
      const long long o = (long long)i * step;
      bstep(i, D0p[o], two ? D1p[o] : 0.0);
    }
  }
}

// Copies w <= 34 consecutive nodes x0 .. x0 + w - 1 of the 32 lines L0 .. L0 + 31 (those
// below nlines) into tile[line][0 .. w - 1], lanes along x (coalesced).  Eight lines'
// loads are issued before their stores, so sixteen loads per lane are in flight at once
// (a loop that stored each line before loading the next waited for every load in turn).
// src may be written by this kernel (the forward sweep's values in `out`), so the loads
// take the coherent path.
__device__ __forceinline__ void stage_rows(double (*tile)[35], const double* src, long long L0,
                                           long long nlines, long long stride, int x0, int w,
                                           int lane) {
  for (int l0 = 0; l0 < 32; l0 += 8) {
    double v[8][2];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const long long Ll = L0 + l0 + k;
      const double* row = src + (Ll < nlines ? Ll : L0) * stride + x0;
      v[k][0] = (Ll < nlines && lane < w) ? row[lane] : 0.0;
      v[k][1] = (Ll < nlines && lane + 32 < w) ? row[lane + 32] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      tile[l0 + k][lane] = v[k][0];
      if (lane < 3) tile[l0 + k][32 + lane] = v[k][1];
    }
  }
}

// The reverse of stage_rows for w <= 32 nodes: tile[line][0 .. w - 1] to nodes
// x0 .. x0 + w - 1 of the lines below nlines.
__device__ __forceinline__ void unstage_rows(double (*tile)[35], double* dst, long long L0,
                                             long long nlines, long long stride, int x0, int w,
                                             int lane) {
#pragma unroll 8
  for (int l = 0; l < 32; ++l) {
    const long long Ll = L0 + l;
    if (Ll < nlines && lane < w) dst[Ll * stride + x0 + lane] = tile[l][lane];
  }
}

// x-lines: one warp handles 32 consecutive lines (line = j + (ny+1) k), chunks of 32
// x-nodes staged through shared memory.
__global__ void __launch_bounds__(32)
    k_grad_x(const double* __restrict__ u, double* __restrict__ out, int N, double h,
             long long nlines) {
  __shared__ double cp[kTab], A[kTab], B[kTab];
  __shared__ double tile[32][35];  // [line][x0-1 .. x0+32]
  const double ih = 1.0 / h, i2h = 0.5 / h;
  if (threadIdx.x == 0) thomas_table(cp, A, B, N - 1, i2h);
  __syncwarp();
  const int lane = threadIdx.x;
  const long long stride = N + 1;
  for (long long L0 = (long long)blockIdx.x * 32; L0 < nlines; L0 += (long long)gridDim.x * 32) {
    const long long L = L0 + lane;
    const bool mine = L < nlines;
    double D0 = 0.0, DN = 0.0;
    if (mine) {
      const double* U = u + L * stride;
      D0 = d_left(U[0], U[1], U[2], U[3], U[4], ih);
      DN = d_right(U[N], U[N - 1], U[N - 2], U[N - 3], U[N - 4], ih);
      out[L * stride] = D0;
      out[L * stride + N] = DN;
    }
    // forward sweep, chunk by chunk: unknown nodes i = 1..N-1
    double dp = D0;
    for (int x0 = 1; x0 <= N - 1; x0 += 32) {
      const int cnt = min(32, N - x0);  // nodes x0 .. x0+cnt-1
      __syncwarp();
      stage_rows(tile, u, L0, nlines, stride, x0 - 1, cnt + 2, lane);
      __syncwarp();
      if (mine) {
        for (int c = 0; c < cnt; ++c) {
          const int i = x0 + c;
          const int t = i - 1 < kTab ? i - 1 : kTab - 1;
          if (i == N - 1) dp += DN;
          dp = fma(B[t], dp, (tile[lane][c + 2] - tile[lane][c]) * A[t]);
          tile[lane][c] = dp;
        }
      }
      __syncwarp();
      unstage_rows(tile, out, L0, nlines, stride, x0, cnt, lane);
    }
    // back substitution, chunks from the end
    double xv = 0.0;
    bool last = true;
    for (int x1 = N - 1; x1 >= 1; x1 -= 32) {
      const int cnt = min(32, x1);  // nodes x1-cnt+1 .. x1
      const int xs = x1 - cnt + 1;
      __syncwarp();
      stage_rows(tile, out, L0, nlines, stride, xs, cnt, lane);
      __syncwarp();
      if (mine) {
        for (int c = cnt - 1; c >= 0; --c) {
          const int i = xs + c;
          if (last) {
            xv = tile[lane][c];  // x_{N-1} = dp_{N-1}
            last = false;
          } else {
            const int t = i - 1 < kTab ? i - 1 : kTab - 1;
            xv = tile[lane][c] - cp[t] * xv;
          }
          tile[lane][c] = xv;
        }
      }
      last = false;
      __syncwarp();
      unstage_rows(tile, out, L0, nlines, stride, xs, cnt, lane);
    }
  }
}

int grid_for(long long items, int per_block) {
  long long b = (items + per_block - 1) / per_block;
  if (b > 152 * 32) b = 152 * 32;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_grad(const Grid3& g, const double* u, double* ux, double* uy, double* uz,
                        cudaStream_t s) {
  const long long nlx = (long long)(g.ny + 1) * (g.nz + 1);
  k_grad_x<<<grid_for(nlx, 32), 32, 0, s>>>(u, ux, g.nx, g.hx, nlx);
  // y-lines: a = i (fastest), b = k; two lines per thread
  k_grad_strided<<<grid_for(((long long)(g.nx + 1) * (g.nz + 1) + 1) / 2, kThreads), kThreads, 0, s>>>(
      u, uy, g.ny, g.hy, g.sy, g.nx + 1, g.nz + 1, 1, g.sz);
  // z-lines: a = i + sy*j flattened (fastest), b unused
  k_grad_strided<<<grid_for((g.sz + 1) / 2, kThreads), kThreads, 0, s>>>(u, uz, g.nz, g.hz, g.sz,
                                                                        (int)g.sz, 1, 1, 0);
  return cudaGetLastError();
}

}  // namespace excmg
