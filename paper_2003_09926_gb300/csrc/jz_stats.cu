// jz_stats.cu -- time statistics of the axial velocity, as the paper's
// validation reports them (Section 6: the time-averaged axial velocity <U>,
// the rms of its fluctuation u_rms, radial profiles at fixed distances from
// the inlet averaged in the azimuthal direction, and the potential core, the
// region where <U> is at least 95% of the jet's inlet velocity).
//
// Each sample adds u = (rho u) / rho and u^2 of every grid node to FP64
// running sums held in the caller's device buffer (dense [k][j][i], one
// thread per node, in sample order, so the sums are those of a sequential
// loop over samples, each u^2 rounded before it is added).  Means and rms
// are formed on the host from the sums.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "jz_internal.h"

namespace jz {

namespace {

template <typename ST>
__global__ void k_stats_sample(Layout L, const ST* __restrict__ Q, double* __restrict__ su, double* __restrict__ su2) {
  const long long N = (long long)L.n[0] * L.n[1] * L.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % L.n[0]);
    const int j = (int)((t / L.n[0]) % L.n[1]);
    const int k = (int)(t / ((long long)L.n[0] * L.n[1]));
    const long long n = L.at(i, j, k);
    const double u = (double)Q[L.npad + n] / (double)Q[n];
    su[t] += u;
    su2[t] = __dadd_rn(su2[t], __dmul_rn(u, u));  // u^2 rounded before the sum (no fused multiply-add)
  }
}

// coordinates (y, z) of the nodes of plane i, dense [k][j]
__global__ void k_stats_plane_yz(Layout L, Coords C, int i, double* __restrict__ yz) {
  const int m = L.n[1] * L.n[2];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
    const int j = t % L.n[1], k = t / L.n[1];
    yz[2 * t] = C.x(1, i, j, k);
    yz[2 * t + 1] = C.x(2, i, j, k);
  }
}

// axial coordinate of the nodes (i, jc, kc), one per plane
__global__ void k_stats_axis_x(Layout L, Coords C, int jc, int kc, double* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n[0]; i += gridDim.x * blockDim.x) x[i] = C.x(0, i, jc, kc);
}

int grid_blocks_s(long long work) {
  long long b = (work + 255) / 256;
  const long long cap = 32LL * device_sm_count();
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

cudaError_t launch_stats_sample(const GridDev& g, double* su, double* su2, cudaStream_t s) {
  const long long N = (long long)g.L.n[0] * g.L.n[1] * g.L.n[2];
  if (g.prec == JZ_P64)
    k_stats_sample<double><<<grid_blocks_s(N), 256, 0, s>>>(g.L, (const double*)g.Q0, su, su2);
  else
    k_stats_sample<float><<<grid_blocks_s(N), 256, 0, s>>>(g.L, (const float*)g.Q0, su, su2);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_stats_plane_yz(const GridDev& g, int i, double* yz, cudaStream_t s) {
  k_stats_plane_yz<<<grid_blocks_s((long long)g.L.n[1] * g.L.n[2]), 256, 0, s>>>(g.L, g.C, i, yz);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_stats_axis_x(const GridDev& g, int jc, int kc, double* x, cudaStream_t s) {
  k_stats_axis_x<<<grid_blocks_s(g.L.n[0]), 256, 0, s>>>(g.L, g.C, jc, kc, x);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace jz
