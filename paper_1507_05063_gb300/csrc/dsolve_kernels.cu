// DSOLVE of Algorithm 1 (the direct solves on the two coarsest grids) by the discrete
// sine transform.
//
// On a box with Dirichlet boundary the interior operator of the 19-point scheme is a sum
// of tensor products of the 1D neighbour-sum operator T (T v_i = v_{i-1} + v_{i+1}, zero
// outside): A = c0 I + fx Tx + fy Ty + fz Tz + exy Tx Ty + exz Tx Tz + eyz Ty Tz.  The sine
// vectors s_k(i) = sin(pi i k / n), i, k = 1 .. n-1, are eigenvectors of T with
// eigenvalues mu_k = 2 cos(pi k / n), so with the sine matrix S (S^2 = (n/2) I per
// direction)
//     A^{-1} b = (2/nx)(2/ny)(2/nz) S Lambda^{-1} S b,
//     Lambda(kx,ky,kz) = c0 + fx mu_x + fy mu_y + fz mu_z + exy mu_x mu_y + exz mu_x mu_z
//                        + eyz mu_y mu_z.
// One block per problem forms b from f and the Dirichlet data (the residual of the start
// with g on the boundary and zero inside: -RHS(f) minus the lift), writes g into the
// level's boundary nodes, transforms b along x, y and z (dense sine matrices in shared
// memory, built from a table of the 2 n_d distinct values sin(pi m / n_d): (mx + my + mz)
// FMA per unknown per direction of the transform), divides, transforms back, writes u's
// interior, and checks the result: r = b - A u on the interior, r.r and b.b into the
// problem's CG state (0 steps, done).  Everything but u's nodes and the state stays in
// shared memory, so one launch can solve levels 0 and 1 side by side.  The cascade launches no boundary initialisation
// and no residual for these levels.
#include <cuda_runtime.h>

#include <algorithm>

#include "excmg_internal.cuh"

namespace excmg {
namespace {

constexpr int kDsThreads = 256;

__device__ __forceinline__ double ds_block_sum(double v, double* s_park) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_park[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < kDsThreads / 32 ? s_park[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// out[... k ...] = sum_i S[k][i] in[... i ...] along one axis of an (mx, my, mz) array
// (x fastest).  S is m x m, row k = mode k + 1, column i = node i + 1.
__device__ void ds_axis(const double* in, double* out, const double* S, int mx, int my, int mz,
                        int axis) {
  const int n = mx * my * mz;
  const int m = axis == 0 ? mx : (axis == 1 ? my : mz);
  const int stride = axis == 0 ? 1 : (axis == 1 ? mx : mx * my);
  for (int t = threadIdx.x; t < n; t += kDsThreads) {
    const int ix = t % mx, iy = (t / mx) % my, iz = t / (mx * my);
    const int k = axis == 0 ? ix : (axis == 1 ? iy : iz);
    const double* src = in + (t - k * stride);  // the line's first element
    const double* row = S + k * m;
    double acc = 0.0;
    for (int i = 0; i < m; ++i) acc = fma(row[i], src[i * stride], acc);
    out[t] = acc;
  }
}

__global__ void __launch_bounds__(kDsThreads)
    k_dsolve(const CGDesc<double>* __restrict__ descs, CGState* st) {
  extern __shared__ __align__(16) double s_ds[];
  __shared__ double s_park[kDsThreads / 32];
  const CGDesc<double>& d = descs[blockIdx.x];
  if (!d.direct) return;
  CGState* S = st + d.slot;
  const Grid3 g = d.g;
  const int mx = g.nx - 1, my = g.ny - 1, mz = g.nz - 1;
  const int n = mx * my * mz;
  double* V = s_ds;          // n
  double* W = V + n;         // n
  double* Bv = W + n;        // n: b (kept for the check; the workspace vectors are shared
                             // by the levels this launch solves together)
  double* Sx = Bv + n;       // mx * mx
  double* Sy = Sx + mx * mx; // my * my
  double* Sz = Sy + my * my; // mz * mz
  double* C = Sz + mz * mz;  // mx + my + mz: 2 cos(pi k / n_d), the eigenvalues of T
  double* T = C + mx + my + mz;  // 2 (nx + ny + nz): sin(pi m / n_d), m = 0 .. 2 n_d - 1
  double* Tx = T;
  double* Ty = Tx + 2 * g.nx;
  double* Tz = Ty + 2 * g.ny;
  for (int t = threadIdx.x; t < 2 * g.nx; t += kDsThreads) Tx[t] = sinpi((double)t / g.nx);
  for (int t = threadIdx.x; t < 2 * g.ny; t += kDsThreads) Ty[t] = sinpi((double)t / g.ny);
  for (int t = threadIdx.x; t < 2 * g.nz; t += kDsThreads) Tz[t] = sinpi((double)t / g.nz);
  for (int t = threadIdx.x; t < mx + my + mz; t += kDsThreads) {
    const int ax = t < mx ? 0 : (t < mx + my ? 1 : 2);
    const int k = t - (ax == 0 ? 0 : (ax == 1 ? mx : mx + my)) + 1;
    C[t] = 2.0 * cospi((double)k / (ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz)));
  }
  // g on the level's boundary nodes
  const long long nodes = g.nodes();
  for (long long o = threadIdx.x; o < nodes; o += kDsThreads) {
    const int i = (int)(o % g.sy), j = (int)((o / g.sy) % (g.ny + 1)), k = (int)(o / g.sz);
    if (i == 0 || i == g.nx || j == 0 || j == g.ny || k == 0 || k == g.nz) d.x[o] = d.gb.at(i, j, k);
  }
  __syncthreads();
  // sine matrices: sin(pi i k / n_d) = table[(i k) mod 2 n_d]
  auto fill = [&](double* M, const double* tab, int m, int nd) {
    for (int t = threadIdx.x; t < m * m; t += kDsThreads) {
      const int k = t / m + 1, i = t % m + 1;
      M[t] = tab[(i * k) % (2 * nd)];
    }
  };
  fill(Sx, Tx, mx, g.nx);
  fill(Sy, Ty, my, g.ny);
  fill(Sz, Tz, mz, g.nz);
  // b on the interior: -(A-stencil of the start: g on the boundary, 0 inside) - RHS(f)
  const Coef A = d.A;
  auto ub = [&](int i, int j, int k) -> double {
    return (i == 0 || i == g.nx || j == 0 || j == g.ny || k == 0 || k == g.nz) ? d.gb.at(i, j, k) : 0.0;
  };
  double acc_b = 0.0, acc_f4 = 0.0;  // ||b||^2 and ||2 RHS(f)||^2: the readings of ||f_h||
  for (int t = threadIdx.x; t < n; t += kDsThreads) {
    const int i = t % mx + 1, j = (t / mx) % my + 1, k = t / (mx * my) + 1;
    const View& F = d.f;
    const double rhs2 = fma(6.0, F.at(i, j, k), ((F.at(i - 1, j, k) + F.at(i + 1, j, k)) +
                                                 (F.at(i, j - 1, k) + F.at(i, j + 1, k)) +
                                                 (F.at(i, j, k - 1) + F.at(i, j, k + 1))));
    const double SX = ub(i - 1, j, k) + ub(i + 1, j, k), SY = ub(i, j - 1, k) + ub(i, j + 1, k);
    const double SZ = ub(i, j, k - 1) + ub(i, j, k + 1);
    const double EXY = (ub(i - 1, j - 1, k) + ub(i + 1, j - 1, k)) + (ub(i - 1, j + 1, k) + ub(i + 1, j + 1, k));
    const double EXZ = (ub(i - 1, j, k - 1) + ub(i + 1, j, k - 1)) + (ub(i - 1, j, k + 1) + ub(i + 1, j, k + 1));
    const double EYZ = (ub(i, j - 1, k - 1) + ub(i, j + 1, k - 1)) + (ub(i, j - 1, k + 1) + ub(i, j + 1, k + 1));
    const double lift = fma(A.fx, SX, fma(A.fy, SY, fma(A.fz, SZ, fma(A.exy, EXY, fma(A.exz, EXZ, A.eyz * EYZ)))));
    const double b = fma(-0.5, rhs2, -lift);
    V[t] = b;
    Bv[t] = b;
    acc_b = fma(b, b, acc_b);
    acc_f4 = fma(rhs2, rhs2, acc_f4);
  }
  const double bb_lift = ds_block_sum(acc_b, s_park);
  __syncthreads();
  const double bb_force = 0.25 * ds_block_sum(acc_f4, s_park);
  const double bb = (d.forcing && bb_force > 0.0) ? bb_force : bb_lift;
  __syncthreads();
  ds_axis(V, W, Sx, mx, my, mz, 0);
  __syncthreads();
  ds_axis(W, V, Sy, mx, my, mz, 1);
  __syncthreads();
  ds_axis(V, W, Sz, mx, my, mz, 2);
  __syncthreads();
  const double* Cx = C;
  const double* Cy = C + mx;
  const double* Cz = C + mx + my;
  const double scale = 8.0 / ((double)g.nx * g.ny * g.nz);
  for (int t = threadIdx.x; t < n; t += kDsThreads) {
    const int ix = t % mx, iy = (t / mx) % my, iz = t / (mx * my);
    const double ux = Cx[ix], uy = Cy[iy], uz = Cz[iz];
    const double lam = A.c0 + A.fx * ux + A.fy * uy + A.fz * uz + A.exy * ux * uy + A.exz * ux * uz +
                       A.eyz * uy * uz;
    W[t] = W[t] * (scale / lam);
  }
  __syncthreads();
  ds_axis(W, V, Sx, mx, my, mz, 0);
  __syncthreads();
  ds_axis(V, W, Sy, mx, my, mz, 1);
  __syncthreads();
  ds_axis(W, V, Sz, mx, my, mz, 2);
  __syncthreads();
  // u's interior, and the check r = b - A u (u = 0 on the boundary of the interior
  // array: the lift is in b)
  double acc = 0.0;
  const int sy = mx, sz = mx * my;
  for (int t = threadIdx.x; t < n; t += kDsThreads) {
    const int ix = t % mx, iy = (t / mx) % my, iz = t / (mx * my);
    auto at = [&](int dx, int dy, int dz) -> double {
      const int x = ix + dx, y = iy + dy, z = iz + dz;
      if (x < 0 || x >= mx || y < 0 || y >= my || z < 0 || z >= mz) return 0.0;
      return V[t + dx + dy * sy + dz * sz];
    };
    const double SX = at(-1, 0, 0) + at(1, 0, 0), SY = at(0, -1, 0) + at(0, 1, 0);
    const double SZ = at(0, 0, -1) + at(0, 0, 1);
    const double EXY = (at(-1, -1, 0) + at(1, -1, 0)) + (at(-1, 1, 0) + at(1, 1, 0));
    const double EXZ = (at(-1, 0, -1) + at(1, 0, -1)) + (at(-1, 0, 1) + at(1, 0, 1));
    const double EYZ = (at(0, -1, -1) + at(0, 1, -1)) + (at(0, -1, 1) + at(0, 1, 1));
    const double Au = fma(A.c0, V[t], fma(A.fx, SX, fma(A.fy, SY, fma(A.fz, SZ,
                      fma(A.exy, EXY, fma(A.exz, EXZ, A.eyz * EYZ))))));
    const long long o = (ix + 1) + (iy + 1) * g.sy + (long long)(iz + 1) * g.sz;
    const double r = Bv[t] - Au;
    d.x[o] = V[t];
    acc = fma(r, r, acc);
  }
  const double rr = ds_block_sum(acc, s_park);
  if (threadIdx.x == 0) {
    S->rr = rr;
    S->rr0 = rr;
    S->bb = bb;
    S->alpha = S->beta = S->pq = 0.0;
    S->tol2 = 0.0;
    S->iter = 0;
    S->max_iter = 0;
    S->fixed = 0;
    S->first = 0;
    S->done = 1;
    S->status = isfinite(rr) && isfinite(bb) ? EXCMG_OK : EXCMG_ERR_NONFINITE;
  }
}

}  // namespace

size_t dsolve_smem(const Grid3& g) {
  const size_t mx = g.nx - 1, my = g.ny - 1, mz = g.nz - 1;
  return sizeof(double) *
         (3 * mx * my * mz + mx * mx + my * my + mz * mz + (mx + my + mz) + 2 * (g.nx + g.ny + g.nz));
}

static int g_ds_max_smem = 0;

bool dsolve_fits(const Grid3& g) {
  if (g_ds_max_smem == 0) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    g_ds_max_smem = std::max(1, optin - 1024);
    if (cudaFuncSetAttribute(k_dsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, g_ds_max_smem) !=
        cudaSuccess) {
      cudaGetLastError();
      g_ds_max_smem = -1;
    }
  }
  return g_ds_max_smem > 0 && g.nx >= 2 && g.ny >= 2 && g.nz >= 2 &&
         dsolve_smem(g) <= (size_t)g_ds_max_smem;
}

cudaError_t launch_dsolve(int nprob, const CGDesc<double>* descs, size_t smem, CGState* st,
                          cudaStream_t s) {
  k_dsolve<<<nprob, kDsThreads, smem, s>>>(descs, st);
  return cudaGetLastError();
}

}  // namespace excmg
