// jz_common.cuh -- layout, flow constants and small device helpers shared by
// the CUDA translation units of the library (not part of the public ABI).
//
// HBM layout of one grid (all arrays inside the caller's buffer):
//   field[var][k][j][i], i fastest, two ghost layers on every face (the
//   paper's two-layer ghost fringe, Section 4.3).  Node (i, j, k) with
//   i, j, k in [-2, n+1] sits at element (i+2) + (j+2)*pitch + (k+2)*plane.
//   The row pitch is a multiple of 32 elements, so every row (starting at
//   ghost index -2) begins on a 128-byte boundary for FP32 and a 256-byte
//   boundary for FP64, and a tile row of ti+4 elements starting at a tile
//   origin that is a multiple of 4 is 16-byte aligned.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/jz.h"

namespace jz {

constexpr int NG = 2;  // ghost layers

struct Layout {
  int n[3];          // nodes per direction
  int pitch;         // elements per i-row (multiple of 32)
  long long plane;   // elements per k-plane
  long long npad;    // elements per field
  int lo[3], hi[3];  // range of nodes updated by the Runge-Kutta stages
  int per[3];        // periodic flags
  int pn[3];         // distinct nodes of a periodic direction (n; n - 1 azimuthally on a cylinder)
  int bc[6];         // boundary kind per face
  int cyl;           // cylindrical grid: centreline at j = 0, azimuth k
  __host__ __device__ __forceinline__ long long at(int i, int j, int k) const {
    return (long long)(i + NG) + (long long)(j + NG) * pitch + (long long)(k + NG) * plane;
  }
  // the grid node whose value a padded index holds: wrap with the period,
  // else clamp onto the first / last node
  __host__ __device__ __forceinline__ int map1(int d, int idx) const {
    if (per[d]) {
      const int r = idx % pn[d];
      return r < 0 ? r + pn[d] : r;
    }
    return idx < 0 ? 0 : (idx > n[d] - 1 ? n[d] - 1 : idx);
  }
  // ... and across the centreline of a cylindrical grid: (i, -j, k + P/2)
  __host__ __device__ __forceinline__ void map_node(int& i, int& j, int& k) const {
    if (cyl && j < 0) {
      j = -j;
      k += pn[2] / 2;
    }
    i = map1(0, i);
    j = map1(1, j);
    k = map1(2, k);
  }
};

// Flow constants, in double; kernels narrow them to their arithmetic type.
struct FlowC {
  double gamma, gm1, cp;  // ratio of specific heats, gamma-1, Cp = 1/(gamma-1)
  double mu_inf, s1;      // Sutherland law
  double pr, prt, cs;     // Prandtl numbers, Smagorinsky constant
  double k2, k4, sigma;   // dissipation constants
  double mach, r0, theta, noise;
  int ic;
  int sgs;      // JZ_SGS_SMAGORINSKY or JZ_SGS_VREMAN
  int viscous;  // mu_inf > 0 or cs > 0
  // the viscous rate factor max(4/3, gamma/Pr), and FP32 roundings of the
  // constants the FP32 boundary fill and reductions use per node (formed on
  // the host: GB300's FP64 pipe is narrow, and a conversion or division on
  // it per node dominated the FP32 fill)
  double vfac;
  float gamma_f, gm1_f, pe_f, vfac_f;  // gamma, gamma - 1, 1/gamma, vfac
};

// a flow constant in the arithmetic type T: the FP64 value, or its FP32
// rounding formed on the host
template <typename T>
__device__ __forceinline__ T flow_const(double d, float f) {
  if constexpr (sizeof(T) == 4)
    return f;
  else
    return (T)d;
}

// 1-D coordinate tables (FP64), indexed by node index + NG:
//   box: x_d(i,j,k) = base[d][i_d] + amp * h[d][i_d] * sn[d][0][i] * sn[d][1][j] * sn[d][2][k]
//   cylinder: x = base[0][i], (y, z) = base[1][j] (cth[k], sth[k]), base[1] the radius
struct Coords {
  const double* base[3];
  const double* h[3];
  const double* sn[3][3];
  const double* cth;  // cos / sin of the azimuth (cylinder)
  const double* sth;
  double amp;
  int cyl;
  __device__ __forceinline__ double x(int d, int i, int j, int k) const {
    if (cyl) return d == 0 ? base[0][i + NG] : base[1][j + NG] * (d == 1 ? cth[k + NG] : sth[k + NG]);
    int id = d == 0 ? i : (d == 1 ? j : k);
    double b = base[d][id + NG];
    if (amp == 0.0) return b;
    double prod = 1.0;
    prod *= sn[d][0][i + NG];
    prod *= sn[d][1][j + NG];
    prod *= sn[d][2][k + NG];
    return b + amp * h[d][id + NG] * prod;
  }
};

// Device-resident scalars of one grid.
struct Scalars {
  double dt;          // current time step
  double time;        // simulated time
  long long step;     // completed steps
  double cfl;         // CFL number of the current step (0 = fixed dt)
  double dt_fixed;    // fixed time step when cfl == 0
  double rate;        // this grid's largest stable-step rate (blocks of one grid: combined over the blocks)
  unsigned int count; // last-block counter of the time-step reduction
  unsigned int dcount;// last-block counter of the diagnostics reduction
  int err;            // sticky device error flag
  int errinfo[7];     // first failure: barrier, parity, plane, tile x, tile y, chunk, stage input
  double diag[16];    // diagnostics result
  jz_diag out;        // the same in the public layout (copied out by jz_diagnostics_async)
};

constexpr int RED_BLOCKS = 1216;  // capacity of the reduction partials (grids are clamped to it)
constexpr int RED_THREADS = 256;
constexpr int DIAG_WORDS = 11;    // per-block diagnostics partial

// Face kinds.  BC_EXCHANGE marks a face of a block of a larger grid that lies
// inside that grid: its ghost layers are copies of the neighbouring block's
// nodes (halo exchange), and its first / last node is updated like any
// interior node.
// BC_AXIS is the centreline face (j = 0) of a cylindrical grid.
enum { BC_PERIODIC = 0, BC_INFLOW = 1, BC_FARFIELD = 2, BC_EXCHANGE = 3, BC_AXIS = 4 };

// SplitMix64 (Steele, Lea & Flood 2014): first output of a generator whose
// state is x, written from the published definition.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double unit53(uint64_t r) {
  return (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

template <typename T> __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

// Per-node diagnostic quantities of a conserved state q, in the state's
// arithmetic type T: pressure and the squared Mach number (the maximum over
// nodes is taken on the square; its root is taken once at the end).
template <typename T>
__host__ __device__ __forceinline__ void diag_node(const T q[5], T gm1, T gamma, T& p, T& m2) {
  const T ri = T(1) / q[0];
  const T k = (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) * ri;  // rho |u|^2
  p = gm1 * (q[4] - T(0.5) * k);
  m2 = k / (gamma * p);  // |u|^2 / c^2 with c^2 = gamma p / rho
}

// Running sum of one conserved variable: plain FP64 for FP64 states; for
// FP32 states an FP32 sum with the rounding error of every addition carried
// in a second FP32 word (Knuth's TwoSum), folded to FP64 at the end.
template <typename T> struct RunSum;
template <> struct RunSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct RunSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x, bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// launch accounting (defined in jz_api.cu)
void count_launches(uint64_t n);

}  // namespace jz
