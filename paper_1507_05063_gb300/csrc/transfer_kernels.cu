// Level-to-level transfers of Algorithm 1 (Section 3.3):
//   EXP_finite(u_2h, u_4h) -> w_h   (line 6; eqs. jiedian, zhongdian, inter)
//   EXP_true(u_h, u_2h)    -> u~_h  (line 10; eqs. t1, chenlin)
// and the adjoint's transposed right-hand-side / lift operators.
//
// EXP_finite works on bricks of 32 x 8 x 8 fine cells (four interpolation cells along x,
// each cell = 2x2x2 elements of grid 4h = 8 fine cells per direction).  Per brick:
//  1. stage the 17x5x5 nodes of grid 2h and the 9x3x3 nodes of grid 4h in shared memory;
//  2. w at every node of grid 2h: u_2h + (1/16) * (mean of d = u_2h - u_4h over the
//     grid-4h corners of the edge / face / element it is the centre of; d itself at a
//     grid-4h node).  This is eq. (jiedian) at corners ((17u1 - u0)/16 = u1 + d/16),
//     eq. (zhongdian) at edge midpoints (u1 + (d_a + d_b)/32), and the arithmetic means
//     of eq. (zhongdian) over the two face diagonals / four space diagonals;
//  3. tri-quartic interpolation (eq. inter) as three one-dimensional quartic passes
//     (x, then y, then z) with the Lagrange weights at the quarter points: the tensor
//     product l_i(xi) l_j(eta) l_k(zeta) applied by sum factorisation, ~6 FMA per node
//     instead of the 125 of the 604x125 matrix form.
#include <math.h>

#include "excmg_internal.cuh"

namespace excmg {

namespace {

// 128 * l_m(t) for the five nodes t = 0..4 of a cell and t = 1/2, 3/2, 5/2, 7/2
// (Lagrange basis of Section 3.3; exact in binary floating point after / 128).
__constant__ double c_wq[4][5] = {
    {35.0 / 128, 140.0 / 128, -70.0 / 128, 28.0 / 128, -5.0 / 128},
    {-5.0 / 128, 60.0 / 128, 90.0 / 128, -20.0 / 128, 3.0 / 128},
    {3.0 / 128, -20.0 / 128, 90.0 / 128, 60.0 / 128, -5.0 / 128},
    {-5.0 / 128, 28.0 / 128, -70.0 / 128, 140.0 / 128, 35.0 / 128},
};

constexpr int BX1 = 17, BY1 = 5, BZ1 = 5;  // grid-2h nodes of a brick
constexpr int BX0 = 9, BY0 = 3, BZ0 = 3;   // grid-4h nodes of a brick
constexpr int BXF = 33, BYF = 9, BZF = 9;  // fine nodes of a brick

struct BrickSmem {
  double u1[BZ1][BY1][BX1];
  double d[BZ0][BY0][BX0];
  double w[BZ1][BY1][BX1];
  double x[BZ1][BY1][BXF];
  double y[BZ1][BYF][BXF];
};

// One brick (local index lb) of EXP_finite for descriptor d.
__device__ void exp_finite_brick(const ProlongDesc& d, long long lb, BrickSmem& S) {
  auto& s_u1 = S.u1;
  auto& s_d = S.d;
  auto& s_w = S.w;
  auto& s_x = S.x;
  auto& s_y = S.y;
  {
    const Grid3 g = d.g;
    const int bx = (int)(lb % d.nbx);
    const int by = (int)((lb / d.nbx) % d.nby);
    const int bz = (int)(lb / ((long long)d.nbx * d.nby));
    const int n1x = g.nx / 2, n1y = g.ny / 2, n1z = g.nz / 2;
    const int n0x = g.nx / 4, n0y = g.ny / 4, n0z = g.nz / 4;
    const long long s1y = n1x + 1, s1z = (long long)(n1x + 1) * (n1y + 1);
    const long long s0y = n0x + 1, s0z = (long long)(n0x + 1) * (n0y + 1);
    __syncthreads();  // shared buffers of the previous brick are free
    // 1. stage grid-2h and grid-4h values
    for (int idx = threadIdx.x; idx < BZ1 * BY1 * BX1; idx += kThreads) {
      const int ix = idx % BX1, jy = (idx / BX1) % BY1, kz = idx / (BX1 * BY1);
      const int I = 16 * bx + ix, J = 4 * by + jy, K = 4 * bz + kz;
      s_u1[kz][jy][ix] = (I <= n1x && J <= n1y && K <= n1z) ? d.u2h[I + J * s1y + K * s1z] : 0.0;
    }
    for (int idx = threadIdx.x; idx < BZ0 * BY0 * BX0; idx += kThreads) {
      const int ix = idx % BX0, jy = (idx / BX0) % BY0, kz = idx / (BX0 * BY0);
      const int I = 8 * bx + ix, J = 2 * by + jy, K = 2 * bz + kz;
      s_d[kz][jy][ix] = (I <= n0x && J <= n0y && K <= n0z) ? d.u4h[I + J * s0y + K * s0z] : 0.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < BZ0 * BY0 * BX0; idx += kThreads) {
      const int ix = idx % BX0, jy = (idx / BX0) % BY0, kz = idx / (BX0 * BY0);
      s_d[kz][jy][ix] = s_u1[2 * kz][2 * jy][2 * ix] - s_d[kz][jy][ix];
    }
    __syncthreads();
    // 2. extrapolated values at the grid-2h nodes
    for (int idx = threadIdx.x; idx < BZ1 * BY1 * BX1; idx += kThreads) {
      const int ix = idx % BX1, jy = (idx / BX1) % BY1, kz = idx / (BX1 * BY1);
      const int ox = ix & 1, oy = jy & 1, oz = kz & 1;
      const int cx = ix >> 1, cy = jy >> 1, cz = kz >> 1;
      double sum = 0.0;
      for (int a = 0; a <= oz; ++a)
        for (int bb = 0; bb <= oy; ++bb)
          for (int c = 0; c <= ox; ++c) sum += s_d[cz + a][cy + bb][cx + c];
      // (1/16) * mean over 2^(ox+oy+oz) corners: a power-of-two scale, exact as a product
      const double scale = 0.0625 / (double)(1 << (ox + oy + oz));
      s_w[kz][jy][ix] = fma(sum, scale, s_u1[kz][jy][ix]);
    }
    __syncthreads();
    // 3a. quartic along x
    for (int idx = threadIdx.x; idx < BZ1 * BY1 * BXF; idx += kThreads) {
      const int lx = idx % BXF, jy = (idx / BXF) % BY1, kz = idx / (BXF * BY1);
      double v;
      if ((lx & 1) == 0) {
        v = s_w[kz][jy][lx >> 1];
      } else {
        const int I = (lx - 1) >> 1, base = (I >> 2) << 2, t = I & 3;
        v = 0.0;
#pragma unroll
        for (int m = 0; m < 5; ++m) v = fma(c_wq[t][m], s_w[kz][jy][base + m], v);
      }
      s_x[kz][jy][lx] = v;
    }
    __syncthreads();
    // 3b. quartic along y
    for (int idx = threadIdx.x; idx < BZ1 * BYF * BXF; idx += kThreads) {
      const int lx = idx % BXF, ly = (idx / BXF) % BYF, kz = idx / (BXF * BYF);
      double v;
      if ((ly & 1) == 0) {
        v = s_x[kz][ly >> 1][lx];
      } else {
        const int t = (ly - 1) >> 1;
        v = 0.0;
#pragma unroll
        for (int m = 0; m < 5; ++m) v = fma(c_wq[t][m], s_x[kz][m][lx], v);
      }
      s_y[kz][ly][lx] = v;
    }
    __syncthreads();
    // 3c. quartic along z, boundary data, store
    for (int idx = threadIdx.x; idx < BZF * BYF * BXF; idx += kThreads) {
      const int lx = idx % BXF, ly = (idx / BXF) % BYF, lz = idx / (BXF * BYF);
      const int gx = 32 * bx + lx, gy = 8 * by + ly, gz = 8 * bz + lz;
      if (gx > g.nx || gy > g.ny || gz > g.nz) continue;
      if ((lx == BXF - 1 && gx != g.nx) || (ly == BYF - 1 && gy != g.ny) ||
          (lz == BZF - 1 && gz != g.nz))
        continue;  // owned by the next brick
      double v;
      const bool bnd = gx == 0 || gx == g.nx || gy == 0 || gy == g.ny || gz == 0 || gz == g.nz;
      if (bnd && d.gb.p != nullptr) {
        v = d.gb.at(gx, gy, gz);
      } else if ((lz & 1) == 0) {
        v = s_y[lz >> 1][ly][lx];
      } else {
        const int t = (lz - 1) >> 1;
        v = 0.0;
#pragma unroll
        for (int m = 0; m < 5; ++m) v = fma(c_wq[t][m], s_y[m][ly][lx], v);
      }
      d.w[gx + gy * g.sy + (long long)gz * g.sz] = v;
    }
  }
}

__global__ void __launch_bounds__(kThreads)
    k_exp_finite(int nprob, const ProlongDesc* __restrict__ descs, long long total_blocks) {
  __shared__ BrickSmem S;
  int p = 0;
  for (long long b = blockIdx.x; b < total_blocks; b += gridDim.x) {
    while (p + 1 < nprob && b >= descs[p + 1].block_begin) ++p;
    exp_finite_brick(descs[p], b - descs[p].block_begin, S);
  }
}

__global__ void __launch_bounds__(kThreads) k_exp_finite_one(ProlongDesc d, long long total_blocks) {
  __shared__ BrickSmem S;
  for (long long b = blockIdx.x; b < total_blocks; b += gridDim.x) exp_finite_brick(d, b, S);
}

// EXP_true: u~ = u_h + (1/15) (mean of d = u_h - u_2h over the grid-2h corners of the
// edge / face / element the node is the centre of; d itself at grid-2h nodes).
__global__ void __launch_bounds__(kThreads)
    k_exp_true(Grid3 g, const double* __restrict__ uh, const double* __restrict__ u2h,
               double* __restrict__ ut) {
  const long long n = g.nodes();
  const int n1x = g.nx / 2, n1y = g.ny / 2;
  const long long s1y = n1x + 1, s1z = (long long)(n1x + 1) * (n1y + 1);
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % g.sy);
    const int j = (int)((o / g.sy) % (g.ny + 1));
    const int k = (int)(o / g.sz);
    const int ox = i & 1, oy = j & 1, oz = k & 1;
    const int cx = i >> 1, cy = j >> 1, cz = k >> 1;
    double sum = 0.0;
    for (int a = 0; a <= oz; ++a)
      for (int b = 0; b <= oy; ++b)
        for (int c = 0; c <= ox; ++c) {
          const int I = cx + c, J = cy + b, K = cz + a;
          sum += uh[2 * I + 2 * J * g.sy + 2LL * K * g.sz] - u2h[I + J * s1y + K * s1z];
        }
    // (1/15) * mean over the corners; the reciprocals are compile-time constants
    const double inv = (ox + oy + oz == 0) ? 1.0 / 15.0
                     : (ox + oy + oz == 1) ? 1.0 / 30.0
                     : (ox + oy + oz == 2) ? 1.0 / 60.0 : 1.0 / 120.0;
    ut[o] = fma(sum, inv, uh[o]);
  }
}

// Levels 0 and 1 start CG from zero: u = g on the boundary, 0 inside.
__global__ void __launch_bounds__(kThreads) k_boundary_init(Grid3 g, View gb, double* __restrict__ u) {
  const long long n = g.nodes();
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % g.sy);
    const int j = (int)((o / g.sy) % (g.ny + 1));
    const int k = (int)(o / g.sz);
    const bool bnd = i == 0 || i == g.nx || j == 0 || j == g.ny || k == 0 || k == g.nz;
    u[o] = bnd ? gb.at(i, j, k) : 0.0;
  }
}

// Adjoint outputs from lambda (zero on boundary nodes):
//   dL/df = -R^T lambda = -(3 lambda_m + (1/2) sum of lambda at the 6 face neighbours)
//   dL/dg = LHS^T lambda + dL/du on boundary nodes, 0 inside (LHS weights = -A weights).
__global__ void __launch_bounds__(kThreads)
    k_adjoint_finish(Grid3 g, Coef A, const double* __restrict__ lam,
                     const double* __restrict__ dLdu, double* __restrict__ dLdf,
                     double* __restrict__ dLdg) {
  const long long n = g.nodes();
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % g.sy);
    const int j = (int)((o / g.sy) % (g.ny + 1));
    const int k = (int)(o / g.sz);
    auto L = [&](int di, int dj, int dk) -> double {
      const int a = i + di, b = j + dj, c = k + dk;
      if (a < 0 || a > g.nx || b < 0 || b > g.ny || c < 0 || c > g.nz) return 0.0;
      return lam[a + b * g.sy + (long long)c * g.sz];
    };
    const double faces = (L(1, 0, 0) + L(-1, 0, 0)) + (L(0, 1, 0) + L(0, -1, 0)) + (L(0, 0, 1) + L(0, 0, -1));
    dLdf[o] = -(3.0 * lam[o] + 0.5 * faces);
    const bool bnd = i == 0 || i == g.nx || j == 0 || j == g.ny || k == 0 || k == g.nz;
    if (!bnd) {
      dLdg[o] = 0.0;
      continue;
    }
    const double sx = L(1, 0, 0) + L(-1, 0, 0), sy = L(0, 1, 0) + L(0, -1, 0), sz = L(0, 0, 1) + L(0, 0, -1);
    const double exy = (L(1, 1, 0) + L(-1, 1, 0)) + (L(1, -1, 0) + L(-1, -1, 0));
    const double exz = (L(1, 0, 1) + L(-1, 0, 1)) + (L(1, 0, -1) + L(-1, 0, -1));
    const double eyz = (L(0, 1, 1) + L(0, -1, 1)) + (L(0, 1, -1) + L(0, -1, -1));
    const double Al = A.c0 * lam[o] + A.fx * sx + A.fy * sy + A.fz * sz + A.exy * exy + A.exz * exz + A.eyz * eyz;
    dLdg[o] = -Al + dLdu[o];
  }
}

int flat_grid(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 152 * 16) b = 152 * 16;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_exp_finite(int nprob, const ProlongDesc* descs, long long total_blocks,
                              cudaStream_t s) {
  long long grid = total_blocks < 152 * 8 ? total_blocks : 152 * 8;
  if (grid < 1) grid = 1;
  k_exp_finite<<<(int)grid, kThreads, 0, s>>>(nprob, descs, total_blocks);
  return cudaGetLastError();
}

cudaError_t launch_exp_finite_one(const ProlongDesc& d, cudaStream_t s) {
  const long long total = (long long)d.nbx * d.nby * d.nbz;
  long long grid = total < 152 * 8 ? total : 152 * 8;
  if (grid < 1) grid = 1;
  k_exp_finite_one<<<(int)grid, kThreads, 0, s>>>(d, total);
  return cudaGetLastError();
}

cudaError_t launch_exp_true(const Grid3& g, const double* uh, const double* u2h, double* ut,
                            cudaStream_t s) {
  k_exp_true<<<flat_grid(g.nodes()), kThreads, 0, s>>>(g, uh, u2h, ut);
  return cudaGetLastError();
}

cudaError_t launch_boundary_init(const Grid3& g, View gb, double* u, cudaStream_t s) {
  k_boundary_init<<<flat_grid(g.nodes()), kThreads, 0, s>>>(g, gb, u);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_finish(const Grid3& g, const Coef& A, const double* lam,
                                  const double* dLdu, double* dLdf, double* dLdg,
                                  cudaStream_t s) {
  k_adjoint_finish<<<flat_grid(g.nodes()), kThreads, 0, s>>>(g, A, lam, dLdu, dLdf, dLdg);
  return cudaGetLastError();
}

}  // namespace excmg
