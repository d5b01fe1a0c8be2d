// Level-to-level transfers of Algorithm 1 (Section 3.3):
//   EXP_finite(u_2h, u_4h) -> w_h   (the initial guess; eqs. jiedian, zhongdian, inter)
//   EXP_true(u_h, u_2h)    -> u~_h  (the optional last step; eqs. t1, chenlin)
// and the adjoint's transposed right-hand-side / lift operators.
//
// EXP_finite works on bricks of 32 x 8 x 8 fine cells (four interpolation cells along x,
// each cell = 2x2x2 elements of grid 4h = 8 fine cells per direction).  Per brick:
//  1. w at every node of grid 2h: u_2h + (1/16) * (mean of d = u_2h - u_4h over the
//     grid-4h corners of the edge / face / element it is the centre of; d itself at a
//     grid-4h node).  This is eq. (jiedian) at corners ((17u1 - u0)/16 = u1 + d/16),
//     eq. (zhongdian) at edge midpoints (u1 + (d_a + d_b)/32), and the arithmetic means
//     of eq. (zhongdian) over the two face diagonals / four space diagonals.  The corner
//     sums are formed separably (x, then y, then z: one add per odd coordinate) and the
//     power-of-two factor 1/(16 * 2^(number of odd coordinates)) is applied in one FMA;
//  2. tri-quartic interpolation (eq. inter) as three one-dimensional quartic passes
//     (x, then y, then z) with the Lagrange weights at the half-integer points of a cell:
//     the tensor product l_i(xi) l_j(eta) l_k(zeta) applied by sum factorisation, ~6 FMA
//     per node instead of the 125 of the 604x125 matrix form.
// Every pass splits its outputs by parity (copies at even positions, arithmetic at odd
// ones) so that the float64 work of a warp runs with all lanes active: on GB300 a warp
// instruction on the narrow FP64 pipe costs the same whether 16 or 32 lanes need it.
//
// The same brick code, instantiated with fewer interpolation points, gives the two
// comparison prolongations of the library's prolong option: the extrapolated grid-2h
// values interpolated tri-quadratically over cells of 2x2x2 grid-2h elements (the
// interpolation of the earlier EXCMG for linear elements, which the first remark of
// Section 3.3 contrasts with the tri-quartic one), and plain trilinear interpolation of
// u_2h with no extrapolation (the cascadic multigrid prolongation of Section 3).
#include <math.h>

#include <algorithm>

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

// 8 * l_m(t) of the quadratic basis on the nodes 0, 1, 2 at t = 1/2, 3/2, and the linear
// interpolation at the midpoint of two nodes (both exact in binary floating point).
__constant__ double c_wquad[2][3] = {{3.0 / 8, 6.0 / 8, -1.0 / 8}, {-1.0 / 8, 6.0 / 8, 3.0 / 8}};
__constant__ double c_wlin[1][2] = {{0.5, 0.5}};

constexpr int BX1 = 17, BY1 = 5, BZ1 = 5;  // grid-2h nodes of a brick
constexpr int BX0 = 9, BY0 = 3, BZ0 = 3;   // grid-4h nodes of a brick
constexpr int BXF = 33, BYF = 9, BZF = 9;  // fine nodes of a brick

struct BrickSmem {
  double wq[4][5];            // c_wq, indexed per lane
  double u1[BZ1][BY1][BX1];   // grid-2h values
  double tx[BZ0][BY0][BX1];   // corner sums of d along x (grid-4h rows, grid-2h columns)
  double ty[BZ0][BY1][BX1];   // ... then along y
  double w[BZ1][BY1][BX1];    // extrapolated values at the grid-2h nodes
  double x[BZ1][BY1][BXF];    // after the quartic pass along x
  double y[BZ1][BYF][BXF];    // after the quartic pass along y
};

// One brick (local index lb) of the prolongation for descriptor d.  P interpolation
// points per direction over cells of P - 1 grid-2h elements: 5 is EXP_finite (eq. inter);
// 3 the tri-quadratic comparison; 2 the trilinear one, which also skips the
// extrapolation (w = u_2h at the grid-2h nodes).  The brick (16 x 4 x 4 grid-2h
// elements) holds whole cells for each P.
template <int P>
__device__ void exp_finite_brick(const ProlongDesc& d, long long lb, BrickSmem& S) {
  constexpr int C = P - 1;  // grid-2h elements per cell and direction
  const Grid3 g = d.g;
  const int bx = (int)(lb % d.nbx);
  const int by = (int)((lb / d.nbx) % d.nby);
  const int bz = (int)(lb / ((long long)d.nbx * d.nby));
  const int n1x = g.nx / 2, n1y = g.ny / 2, n1z = g.nz / 2;
  const int n0x = g.nx / 4, n0y = g.ny / 4, n0z = g.nz / 4;
  const long long s1y = n1x + 1, s1z = (long long)(n1x + 1) * (n1y + 1);
  const long long s0y = n0x + 1, s0z = (long long)(n0x + 1) * (n0y + 1);
  // d = u_2h - u_4h at grid-4h node (I, J, K) of the level (0 outside the grid)
  auto dval = [&](int I, int J, int K) -> double {
    if (I > n0x || J > n0y || K > n0z) return 0.0;
    return d.u2h[2 * I + 2 * J * s1y + 2 * K * s1z] - d.u4h[I + J * s0y + K * s0z];
  };
  __syncthreads();  // shared buffers of the previous brick are free
  // 1a. stage grid-2h values; corner sums of d along x (even columns: d, odd: d_a + d_b)
  if (P == 2) {  // no extrapolation: w = u_2h
    for (int idx = threadIdx.x; idx < BZ1 * BY1 * BX1; idx += kThreads) {
      const int ix = idx % BX1, jy = (idx / BX1) % BY1, kz = idx / (BX1 * BY1);
      const int I = 16 * bx + ix, J = 4 * by + jy, K = 4 * bz + kz;
      S.w[kz][jy][ix] = (I <= n1x && J <= n1y && K <= n1z) ? d.u2h[I + J * s1y + K * s1z] : 0.0;
    }
  } else {
  for (int idx = threadIdx.x; idx < BZ1 * BY1 * BX1; idx += kThreads) {
    const int ix = idx % BX1, jy = (idx / BX1) % BY1, kz = idx / (BX1 * BY1);
    const int I = 16 * bx + ix, J = 4 * by + jy, K = 4 * bz + kz;
    S.u1[kz][jy][ix] = (I <= n1x && J <= n1y && K <= n1z) ? d.u2h[I + J * s1y + K * s1z] : 0.0;
  }
  for (int idx = threadIdx.x; idx < BZ0 * BY0 * BX0; idx += kThreads) {
    const int i0 = idx % BX0, j0 = (idx / BX0) % BY0, k0 = idx / (BX0 * BY0);
    S.tx[k0][j0][2 * i0] = dval(8 * bx + i0, 2 * by + j0, 2 * bz + k0);
  }
  for (int idx = threadIdx.x; idx < BZ0 * BY0 * (BX0 - 1); idx += kThreads) {
    const int i0 = idx % (BX0 - 1), j0 = (idx / (BX0 - 1)) % BY0, k0 = idx / ((BX0 - 1) * BY0);
    const int I = 8 * bx + i0, J = 2 * by + j0, K = 2 * bz + k0;
    S.tx[k0][j0][2 * i0 + 1] = dval(I, J, K) + dval(I + 1, J, K);
  }
  __syncthreads();
  // 1b. along y
  for (int idx = threadIdx.x; idx < BZ0 * BY0 * BX1; idx += kThreads) {
    const int ix = idx % BX1, j0 = (idx / BX1) % BY0, k0 = idx / (BX1 * BY0);
    S.ty[k0][2 * j0][ix] = S.tx[k0][j0][ix];
  }
  for (int idx = threadIdx.x; idx < BZ0 * (BY0 - 1) * BX1; idx += kThreads) {
    const int ix = idx % BX1, j0 = (idx / BX1) % (BY0 - 1), k0 = idx / (BX1 * (BY0 - 1));
    S.ty[k0][2 * j0 + 1][ix] = S.tx[k0][j0][ix] + S.tx[k0][j0 + 1][ix];
  }
  __syncthreads();
  // 1c. along z, and w = u_2h + sum / (16 * 2^(odd coordinates)) (a power of two: exact)
  for (int idx = threadIdx.x; idx < BZ0 * BY1 * BX1; idx += kThreads) {
    const int ix = idx % BX1, jy = (idx / BX1) % BY1, k0 = idx / (BX1 * BY1);
    const double scale = 0.0625 / (double)(1 << ((ix & 1) + (jy & 1)));
    S.w[2 * k0][jy][ix] = fma(S.ty[k0][jy][ix], scale, S.u1[2 * k0][jy][ix]);
  }
  for (int idx = threadIdx.x; idx < (BZ0 - 1) * BY1 * BX1; idx += kThreads) {
    const int ix = idx % BX1, jy = (idx / BX1) % BY1, k0 = idx / (BX1 * BY1);
    const double scale = 0.03125 / (double)(1 << ((ix & 1) + (jy & 1)));
    S.w[2 * k0 + 1][jy][ix] = fma(S.ty[k0][jy][ix] + S.ty[k0 + 1][jy][ix], scale, S.u1[2 * k0 + 1][jy][ix]);
  }
  }  // P != 2
  __syncthreads();
  // 2a. interpolation along x: even fine columns are grid-2h columns
  for (int idx = threadIdx.x; idx < BZ1 * BY1 * BX1; idx += kThreads) {
    const int ix = idx % BX1, jy = (idx / BX1) % BY1, kz = idx / (BX1 * BY1);
    S.x[kz][jy][2 * ix] = S.w[kz][jy][ix];
  }
  for (int idx = threadIdx.x; idx < BZ1 * BY1 * (BX1 - 1); idx += kThreads) {
    const int I = idx % (BX1 - 1), jy = (idx / (BX1 - 1)) % BY1, kz = idx / ((BX1 - 1) * BY1);
    const int t = I % C, base = I - t;
    double v = 0.0;
#pragma unroll
    for (int m = 0; m < P; ++m) v = fma(S.wq[t][m], S.w[kz][jy][base + m], v);
    S.x[kz][jy][2 * I + 1] = v;
  }
  __syncthreads();
  // 2b. along y (odd fine row 2q + 1 lies in the cell starting at grid-2h row q - q % C)
  for (int idx = threadIdx.x; idx < BZ1 * BY1 * BXF; idx += kThreads) {
    const int lx = idx % BXF, jy = (idx / BXF) % BY1, kz = idx / (BXF * BY1);
    S.y[kz][2 * jy][lx] = S.x[kz][jy][lx];
  }
  for (int idx = threadIdx.x; idx < BZ1 * (BY1 - 1) * BXF; idx += kThreads) {
    const int lx = idx % BXF, q = (idx / BXF) % (BY1 - 1), kz = idx / (BXF * (BY1 - 1));
    const int t = q % C, base = q - t;
    double v = 0.0;
#pragma unroll
    for (int m = 0; m < P; ++m) v = fma(S.wq[t][m], S.x[kz][base + m][lx], v);
    S.y[kz][2 * q + 1][lx] = v;
  }
  __syncthreads();
  // 2c. along z, boundary data, store.  Main part: the 32 x 8 x 8 nodes whose
  // brick-local coordinates are all below the brick's far faces -- one fine plane per
  // pass of the block, one row of 32 nodes per warp (uniform parity, coalesced stores).
  const bool has_g = d.gb.p != nullptr;
  auto value = [&](int lx, int ly, int lz, int gx, int gy, int gz) -> double {
    const bool bnd = gx == 0 || gx == g.nx || gy == 0 || gy == g.ny || gz == 0 || gz == g.nz;
    if (bnd && has_g) return d.gb.at(gx, gy, gz);
    if ((lz & 1) == 0) return S.y[lz >> 1][ly][lx];
    const int q = (lz - 1) >> 1, t = q % C, base = q - t;
    double v = 0.0;
#pragma unroll
    for (int m = 0; m < P; ++m) v = fma(S.wq[t][m], S.y[base + m][ly][lx], v);
    return v;
  };
  for (int idx = threadIdx.x; idx < 32 * 8 * 8; idx += kThreads) {
    const int lx = idx & 31, ly = (idx >> 5) & 7, lz = idx >> 8;
    const int gx = 32 * bx + lx, gy = 8 * by + ly, gz = 8 * bz + lz;
    if (gx > g.nx || gy > g.ny || gz > g.nz) continue;
    d.w[gx + gy * g.sy + (long long)gz * g.sz] = value(lx, ly, lz, gx, gy, gz);
  }
  // far faces of the brick that lie on the far faces of the grid (no next brick owns them)
  const bool xe = 32 * bx + 32 == g.nx, ye = 8 * by + 8 == g.ny, ze = 8 * bz + 8 == g.nz;
  if (xe || ye || ze) {
    for (int idx = threadIdx.x; idx < BZF * BYF * BXF; idx += kThreads) {
      const int lx = idx % BXF, ly = (idx / BXF) % BYF, lz = idx / (BXF * BYF);
      const bool far = (lx == 32) || (ly == 8) || (lz == 8);
      if (!far || (lx == 32 && !xe) || (ly == 8 && !ye) || (lz == 8 && !ze)) continue;
      const int gx = 32 * bx + lx, gy = 8 * by + ly, gz = 8 * bz + lz;
      if (gx > g.nx || gy > g.ny || gz > g.nz) continue;
      d.w[gx + gy * g.sy + (long long)gz * g.sz] = value(lx, ly, lz, gx, gy, gz);
    }
  }
}

// Weights of the P-point interpolation at the C = P - 1 half-integer points of a cell.
template <int P>
__device__ __forceinline__ void load_weights(BrickSmem& S) {
  constexpr int C = P - 1;
  if (threadIdx.x < C * P) {
    const int t = threadIdx.x / P, m = threadIdx.x % P;
    S.wq[t][m] = P == 5 ? c_wq[t][m] : (P == 3 ? c_wquad[t][m] : c_wlin[t][m]);
  }
}

template <int P>
__device__ __forceinline__ void prolong_bricks(int nprob, const ProlongDesc* __restrict__ descs,
                                               long long total_blocks, BrickSmem& S) {
  load_weights<P>(S);
  int p = 0;
  for (long long b = blockIdx.x; b < total_blocks; b += gridDim.x) {
    while (p + 1 < nprob && b >= descs[p + 1].block_begin) ++p;
    exp_finite_brick<P>(descs[p], b - descs[p].block_begin, S);
  }
}

__global__ void __launch_bounds__(kThreads)
    k_exp_finite(int nprob, const ProlongDesc* __restrict__ descs, long long total_blocks) {
  __shared__ BrickSmem S;
  prolong_bricks<5>(nprob, descs, total_blocks, S);
}

// The comparison prolongations (P = 3: extrapolation + tri-quadratic; P = 2: trilinear).
template <int P>
__global__ void __launch_bounds__(kThreads)
    k_prolong_cmp(int nprob, const ProlongDesc* __restrict__ descs, long long total_blocks) {
  __shared__ BrickSmem S;
  prolong_bricks<P>(nprob, descs, total_blocks, S);
}

__global__ void __launch_bounds__(kThreads) k_exp_finite_one(ProlongDesc d, long long total_blocks) {
  __shared__ BrickSmem S;
  load_weights<5>(S);
  for (long long b = blockIdx.x; b < total_blocks; b += gridDim.x) exp_finite_brick<5>(d, b, S);
}

// EXP_true: u~ = u_h + (1/15) (mean of d = u_h - u_2h over the grid-2h corners of the
// edge / face / element the node is the centre of; d itself at grid-2h nodes).
// EXP_true tiles: 64 x 8 x 2 fine nodes per block, whose grid-2h corners are the
// 33 x 5 x 2 coarse nodes from (x0/2, y0/2, z0/2).
constexpr int kEtX = 64, kEtY = 8, kEtZ = 2;
constexpr int kEcX = kEtX / 2 + 1, kEcY = kEtY / 2 + 1, kEcZ = kEtZ / 2 + 1;

__global__ void __launch_bounds__(kThreads)
    k_exp_true(Grid3 g, const double* __restrict__ uh, const double* __restrict__ u2h,
               double* __restrict__ ut, int ntx, int nty) {
  // EXP_true (eqs. t1, chenlin): u~ = u_h + (1/15) x (mean of d over the grid-2h corners
  // of the node's edge, face or cell), d = u_h - u_2h at grid-2h nodes (a grid-2h node is
  // its own corner).  The block forms d at the coarse corners of its tile once, in
  // shared memory.  A node sums d over its corner rows (J, J + oy) x (K, K + oz) -- oy
  // and oz are the same in every lane of a warp (a warp owns fixed rows and planes of
  // the tile), so these branches do not diverge and only existing corners cost FP64
  // instructions (GB300 issues few) -- at the two corner columns I and I + ox; for even
  // i both columns are I, and the sum of the two counts it twice, so the mean over the
  // distinct corners is (e_I + e_{I+ox}) / (2 nrows) in every lane.
  __shared__ double D[kEcZ][kEcY][kEcX];
  const int bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, bz = blockIdx.x / (ntx * nty);
  const int x0 = bx * kEtX, y0 = by * kEtY, z0 = bz * kEtZ;
  const int I0 = x0 / 2, J0 = y0 / 2, K0 = z0 / 2;
  const int n1x = g.nx / 2, n1y = g.ny / 2, n1z = g.nz / 2;
  const long long s1y = n1x + 1, s1z = (long long)(n1x + 1) * (n1y + 1);
  for (int e = threadIdx.x; e < kEcX * kEcY * kEcZ; e += kThreads) {
    const int a = e % kEcX, b = (e / kEcX) % kEcY, c = e / (kEcX * kEcY);
    const int I = I0 + a, J = J0 + b, K = K0 + c;
    double dv = 0.0;
    if (I <= n1x && J <= n1y && K <= n1z)
      dv = uh[2LL * I + 2LL * J * g.sy + 2LL * K * g.sz] - u2h[I + J * s1y + K * s1z];
    D[c][b][a] = dv;
  }
  __syncthreads();
  const int tx = threadIdx.x % kEtX, tq = threadIdx.x / kEtX;  // tq = 0 .. 3
  const int i = x0 + tx;
  if (i > g.nx) return;  // no barrier below
  const int ox = i & 1, ia = (i >> 1) - I0;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int jl = tq + 4 * (m & 1), kl = m >> 1;
    const int j = y0 + jl, k = z0 + kl;
    if (j > g.ny || k > g.nz) continue;
    const int oy = j & 1, oz = k & 1, ja = (j >> 1) - J0, ka = (k >> 1) - K0;
    double e0 = D[ka][ja][ia], e1 = D[ka][ja][ia + ox];
    if (oy) {  // uniform in the warp
      e0 += D[ka][ja + 1][ia];
      e1 += D[ka][ja + 1][ia + ox];
    }
    if (oz) {
      double f0 = D[ka + 1][ja][ia], f1 = D[ka + 1][ja][ia + ox];
      if (oy) {
        f0 += D[ka + 1][ja + 1][ia];
        f1 += D[ka + 1][ja + 1][ia + ox];
      }
      e0 += f0;
      e1 += f1;
    }
    // (1/15) x 1 / (2 x the number of corner rows): compile-time constants
    const int nrows = (1 + oy) * (1 + oz);
    const double w = nrows == 1 ? 1.0 / 30.0 : (nrows == 2 ? 1.0 / 60.0 : 1.0 / 120.0);
    const long long o = i + (long long)j * g.sy + (long long)k * g.sz;
    ut[o] = fma(e0 + e1, w, uh[o]);
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

// Blocks of a grid-stride elementwise launch over n items: at most 16 per SM of the
// current device.
int flat_grid(long long n) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  long long b = (n + kThreads - 1) / kThreads;
  if (b > (long long)sms * 16) b = (long long)sms * 16;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

// Co-resident blocks of an EXP_finite kernel on the whole device (one full wave).
static int brick_wave(const void* kernel, int& cache) {
  if (cache == 0) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, 0);
    cache = std::max(1, sms) * std::max(1, occ);
  }
  return cache;
}
static int g_wave_many = 0, g_wave_one = 0;

cudaError_t launch_exp_finite(int nprob, const ProlongDesc* descs, long long total_blocks,
                              cudaStream_t s) {
  const long long wave = brick_wave((const void*)k_exp_finite, g_wave_many);
  const long long grid = std::max(1LL, std::min(total_blocks, wave));
  k_exp_finite<<<(int)grid, kThreads, 0, s>>>(nprob, descs, total_blocks);
  return cudaGetLastError();
}

static int g_wave_quad = 0, g_wave_lin = 0;

cudaError_t launch_prolong_cmp(int points, int nprob, const ProlongDesc* descs,
                               long long total_blocks, cudaStream_t s) {
  if (points != 3 && points != 2) return cudaErrorInvalidValue;
  const void* k = points == 3 ? (const void*)k_prolong_cmp<3> : (const void*)k_prolong_cmp<2>;
  const long long wave = brick_wave(k, points == 3 ? g_wave_quad : g_wave_lin);
  const long long grid = std::max(1LL, std::min(total_blocks, wave));
  if (points == 3) {
    k_prolong_cmp<3><<<(int)grid, kThreads, 0, s>>>(nprob, descs, total_blocks);
  } else {
    k_prolong_cmp<2><<<(int)grid, kThreads, 0, s>>>(nprob, descs, total_blocks);
  }
  return cudaGetLastError();
}

cudaError_t launch_exp_finite_one(const ProlongDesc& d, cudaStream_t s) {
  const long long total = (long long)d.nbx * d.nby * d.nbz;
  const long long wave = brick_wave((const void*)k_exp_finite_one, g_wave_one);
  const long long grid = std::max(1LL, std::min(total, wave));
  k_exp_finite_one<<<(int)grid, kThreads, 0, s>>>(d, total);
  return cudaGetLastError();
}

cudaError_t launch_exp_true(const Grid3& g, const double* uh, const double* u2h, double* ut,
                            cudaStream_t s) {
  const int ntx = (g.nx + 1 + kEtX - 1) / kEtX, nty = (g.ny + 1 + kEtY - 1) / kEtY;
  const long long ntz = (g.nz + 1 + kEtZ - 1) / kEtZ;
  const long long blocks = (long long)ntx * nty * ntz;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_exp_true<<<(unsigned)blocks, kThreads, 0, s>>>(g, uh, u2h, ut, ntx, nty);
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
