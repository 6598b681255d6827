// jz_grid.cu -- grid generation (coordinates, metric terms), initial state,
// boundary conditions with ghost fill, and host<->device state conversion.
//
// Paper: arXiv 2003.09926, Section 3 (generalised curvilinear transformation,
// Eq. 2 energy, boundary conditions: supersonic inflow and Riemann far field),
// Section 4.2 (Jacobian and metric terms computed once after the mesh is
// read; boundary update at the start of every Runge-Kutta stage) and
// Section 4.3 (two-layer ghost fringe).
#include <algorithm>
#include <climits>
#include <vector>
#include <cmath>

#include "jz_fastmath.cuh"
#include "jz_internal.h"

namespace jz {

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// 1-D coordinate tables
// ---------------------------------------------------------------------------

// tanh clustering about s = +-r_c/H: G(s) = s - (c/H)[tanh((Hs - r_c)/w) + tanh((Hs + r_c)/w)]
__device__ double stretch_g(const TabParams& p, double H, double s) {
  return s - (p.stretch_c / H) * (tanh((H * s - p.cluster_r) / p.stretch_w) + tanh((H * s + p.cluster_r) / p.stretch_w));
}

// coordinate at global index idx along direction d; on a cylindrical grid
// direction 1 is the radius r in [0, hi[1]] (the odd clustering function on
// s = j / (nj - 1), so r(-j) = -r(j)) and direction 2 the azimuth
// 2 pi (k mod P) / P
__device__ double base_coord(const TabParams& p, int d, double idx) {
  int n = p.gn[d];
  double lo = p.lo[d], hi = p.hi[d];
  if (p.cyl && d == 1) {
    const double s = idx / (n - 1);
    return p.stretch_c == 0.0 ? hi * s : hi * stretch_g(p, hi, s) / stretch_g(p, hi, 1.0);
  }
  if (p.cyl && d == 2) {
    const int P = p.pn[2], kk = (int)idx;
    return 2.0 * kPi * (double)(((kk % P) + P) % P) / P;
  }
  if (p.per[d]) return lo + (hi - lo) * idx / n;
  if (d == 0 || p.stretch_c == 0.0) return lo + (hi - lo) * idx / (n - 1);
  double H = 0.5 * (hi - lo), C = 0.5 * (hi + lo);
  double s = -1.0 + 2.0 * idx / (n - 1);
  return C + H * stretch_g(p, H, s) / stretch_g(p, H, 1.0);
}

// tables layout: for d: base[d] (n_d+4), h[d] (n_d+4); then for d, e: sn[d][e] (n_e+4);
// then cos and sin of the azimuth (n_2+4 each)
__global__ void k_tables(TabParams p, double* tab) {
  long long off = 0;
  long long base_off[3], h_off[3], sn_off[3][3];
  for (int d = 0; d < 3; ++d) { base_off[d] = off; off += p.n[d] + 2 * NG; h_off[d] = off; off += p.n[d] + 2 * NG; }
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < 3; ++e) { sn_off[d][e] = off; off += p.n[e] + 2 * NG; }
  const long long c_off = off, s_off = off + p.n[2] + 2 * NG;
  off += 2LL * (p.n[2] + 2 * NG);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < off; t += (long long)gridDim.x * blockDim.x) {
    if (t >= c_off) {  // azimuth tables (used by cylindrical grids)
      const bool c = t < s_off;
      const int idx = (int)(t - (c ? c_off : s_off)) - NG + p.off[2];
      const double th = p.cyl ? base_coord(p, 2, idx) : 0.0;
      tab[t] = c ? cos(th) : sin(th);
      continue;
    }
    // find which table t belongs to
    for (int d = 0; d < 3; ++d) {
      long long len = p.n[d] + 2 * NG;
      if (t >= base_off[d] && t < base_off[d] + len) {
        int idx = (int)(t - base_off[d]) - NG + p.off[d];
        tab[t] = base_coord(p, d, idx);
      }
      if (t >= h_off[d] && t < h_off[d] + len) {
        int idx = (int)(t - h_off[d]) - NG + p.off[d];
        tab[t] = 0.5 * (base_coord(p, d, idx + 1.0) - base_coord(p, d, idx - 1.0));
      }
      for (int e = 0; e < 3; ++e) {
        long long le = p.n[e] + 2 * NG;
        if (t >= sn_off[d][e] && t < sn_off[d][e] + le) {
          int idx = (int)(t - sn_off[d][e]) - NG + p.off[e];
          int P = p.per[e] ? p.gn[e] : p.gn[e] - 1;
          tab[t] = sin(2.0 * kPi * p.m[3 * d + e] * idx / P + p.th[3 * d + e]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// metric terms (conservative form) and Jacobian, FP64 arithmetic
// ---------------------------------------------------------------------------

// Over the local box [a, b]: the grid nodes, plus the first ghost layer
// behind a face of a block that lies inside the larger grid (the stage
// kernel reads the metrics of its one-node halo there).
template <typename MT>
__global__ void k_metrics(Layout L, Coords C, MT* __restrict__ M, int a0, int a1, int a2, int b0, int b1, int b2) {
  const long long E0 = b0 - a0 + 1, E1 = b1 - a1 + 1, N = E0 * E1 * (b2 - a2 + 1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    int i = a0 + (int)(t % E0);
    int j = a1 + (int)((t / E0) % E1);
    int k = a2 + (int)(t / (E0 * E1));
    const int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    auto X = [&](int m, int di, int dj, int dk) { return C.x(m, i + di, j + dj, k + dk); };
    // D_b x_p at the node shifted by o: half the difference across direction b
    auto D = [&](int p, int b, int oi, int oj, int ok) {
      return 0.5 * (X(p, oi + e[b][0], oj + e[b][1], ok + e[b][2]) - X(p, oi - e[b][0], oj - e[b][1], ok - e[b][2]));
    };
    long long n = L.at(i, j, k);
    for (int kd = 0; kd < 3; ++kd) {
      int b = (kd + 1) % 3, c = (kd + 2) % 3;
      for (int md = 0; md < 3; ++md) {
        int p = (md + 1) % 3, q = (md + 2) % 3;
        // d_c( D_b x_p * x_q ) - d_b( D_c x_p * x_q )
        double t1 = 0.5 * (D(p, b, e[c][0], e[c][1], e[c][2]) * X(q, e[c][0], e[c][1], e[c][2]) -
                           D(p, b, -e[c][0], -e[c][1], -e[c][2]) * X(q, -e[c][0], -e[c][1], -e[c][2]));
        double t2 = 0.5 * (D(p, c, e[b][0], e[b][1], e[b][2]) * X(q, e[b][0], e[b][1], e[b][2]) -
                           D(p, c, -e[b][0], -e[b][1], -e[b][2]) * X(q, -e[b][0], -e[b][1], -e[b][2]));
        M[(long long)(3 * kd + md) * L.npad + n] = (MT)(t1 - t2);
      }
    }
    // the centreline of a cylindrical grid has zero volume in this form:
    // it takes J of the adjacent radial node
    const int oj = (C.cyl && j == 0) ? 1 : 0;
    double A[3][3];  // A[m][k] = d x_m / d xi_k
    for (int md = 0; md < 3; ++md)
      for (int kd = 0; kd < 3; ++kd) A[md][kd] = D(md, kd, 0, oj, 0);
    double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                 A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    M[9LL * L.npad + n] = (MT)(1.0 / det);
  }
}

// ---------------------------------------------------------------------------
// shell enumeration (padded nodes outside a box [a, b])
// ---------------------------------------------------------------------------

__device__ __forceinline__ int outside_index(int q, int a, int b) {
  int nlow = a + NG;  // indices -NG .. a-1
  return q < nlow ? q - NG : b + 1 + (q - nlow);
}

__device__ __forceinline__ void shell_node(const Shell& s, long long t, int& i, int& j, int& k) {
  long long E0 = s.E[0], E1 = s.E[1];
  if (t < s.cz) {
    int q = (int)(t / (E0 * E1));
    long long r = t - (long long)q * E0 * E1;
    k = outside_index(q, s.a[2], s.b[2]);
    j = (int)(r / E0) - NG;
    i = (int)(r % E0) - NG;
    return;
  }
  t -= s.cz;
  if (t < s.cy) {
    long long nyo = E1 - (s.b[1] - s.a[1] + 1);
    k = s.a[2] + (int)(t / (nyo * E0));
    long long r = t % (nyo * E0);
    j = outside_index((int)(r / E0), s.a[1], s.b[1]);
    i = (int)(r % E0) - NG;
    return;
  }
  t -= s.cy;
  long long nxo = E0 - (s.b[0] - s.a[0] + 1);
  long long nyi = s.b[1] - s.a[1] + 1;
  k = s.a[2] + (int)(t / (nyi * nxo));
  long long r = t % (nyi * nxo);
  j = s.a[1] + (int)(r / nxo);
  i = outside_index((int)(r % nxo), s.a[0], s.b[0]);
}

template <typename T>
__global__ void k_fill_ghosts(Layout L, Shell s, T* __restrict__ F, int ncomp) {
  long long tot = s.total();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    shell_node(s, t, i, j, k);
    int mi = i, mj = j, mk = k;
    L.map_node(mi, mj, mk);
    long long g = L.at(i, j, k), src = L.at(mi, mj, mk);
    for (int c = 0; c < ncomp; ++c) F[(long long)c * L.npad + g] = F[(long long)c * L.npad + src];
  }
}

// ---------------------------------------------------------------------------
// gas model helpers (Eq. 2, equation of state)
// ---------------------------------------------------------------------------

// Elementary operations of the boundary formulas: IEEE, or (FAST, FP32
// states of the P32 and P32_M64 modes) the hardware approximations of the
// stage kernels.  The P32_S64 mode keeps IEEE operations: its boundary
// values enter the FP64 state of the neighbouring nodes every stage, and an
// approximation's bias of an ulp there measurably raised its long-run error.
template <typename T, bool FAST>
struct BcMath {
  static __device__ __forceinline__ T rcp(T x) { return T(1) / x; }
  static __device__ __forceinline__ T div(T a, T b) { return a / b; }
  static __device__ __forceinline__ T sqrt_(T x) { return sqrt(x); }
  static __device__ __forceinline__ T powp(T x, T e) { return pow(x, e); }
};
template <>
struct BcMath<float, true> : stg::Fn<float> {};

template <typename T, bool FAST = false>
__device__ __forceinline__ void to_conserved(T gm1, T rho, T u, T v, T w, T p, T q[5]) {
  q[0] = rho;
  q[1] = rho * u;
  q[2] = rho * v;
  q[3] = rho * w;
  q[4] = BcMath<T, FAST>::div(p, gm1) + T(0.5) * rho * (u * u + v * v + w * w);
}

__device__ __forceinline__ double jet_profile(const FlowC& F, double r) {
  return 0.5 * F.mach * (1.0 - tanh((r - F.r0) / (2.0 * F.theta)));
}

// Riemann-invariant far field against air at rest (rho 1, u 0, p 1/gamma):
// R+ = u_n + 2c/(g-1) from the interior, R- = -2/(g-1) from outside; entropy
// and tangential velocity from the upwind side; supersonic normal speed
// copies the upwind state.
template <typename T, bool FAST>
__device__ void riemann_farfield(const FlowC& F, const T qi[5], const T n[3], T qb[5]) {
  using M = BcMath<T, FAST>;
  const T g = flow_const<T>(F.gamma, F.gamma_f), gm1 = flow_const<T>(F.gm1, F.gm1_f);
  T rho_i = qi[0];
  T ri = M::rcp(rho_i);
  T u[3] = {qi[1] * ri, qi[2] * ri, qi[3] * ri};
  T p_i = gm1 * (qi[4] - T(0.5) * rho_i * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  T c_i = M::sqrt_(g * p_i * ri);
  T un_i = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  if (un_i >= c_i) {
    for (int v = 0; v < 5; ++v) qb[v] = qi[v];
    return;
  }
  const T p_e = M::rcp(g);
  if (un_i <= -c_i) {
    to_conserved<T, FAST>(gm1, T(1), T(0), T(0), T(0), p_e, qb);
    return;
  }
  T Rp = un_i + M::div(T(2) * c_i, gm1);
  T Rm = M::div(-T(2), gm1);  // exterior u_n = 0, c = 1
  T un = T(0.5) * (Rp + Rm);
  T c = T(0.25) * gm1 * (Rp - Rm);
  T s, ut[3];
  if (un > T(0)) {
    s = M::div(p_i, M::powp(rho_i, g));
    for (int d = 0; d < 3; ++d) ut[d] = u[d] - un_i * n[d];
  } else {
    s = p_e;  // p_e / rho_e^g with rho_e = 1
    for (int d = 0; d < 3; ++d) ut[d] = T(0);
  }
  T rho = M::powp(M::div(c * c, g * s), M::rcp(gm1));
  T p = M::div(rho * c * c, g);
  to_conserved<T, FAST>(gm1, rho, ut[0] + un * n[0], ut[1] + un * n[1], ut[2] + un * n[2], p, qb);
}

// Six boxes covering the padded nodes that lie inside an outer box [ol, oh]
// but outside an inner box [il, ih] (z slabs over the whole outer plane, y
// slabs over the inner k range, x slabs over the inner j, k range).
struct Slabs {
  int a[6][3], e[6][3];  // box origin and extent per slab
};

Slabs make_slabs(const int ol[3], const int oh[3], const int il[3], const int ih[3]) {
  Slabs s;
  const int E0 = oh[0] - ol[0] + 1, E1 = oh[1] - ol[1] + 1;
  const int in1 = ih[1] - il[1] + 1, in2 = ih[2] - il[2] + 1;
  auto box = [&](int q, int a0, int e0, int a1, int e1, int a2, int e2) {
    s.a[q][0] = a0; s.e[q][0] = e0; s.a[q][1] = a1; s.e[q][1] = e1; s.a[q][2] = a2; s.e[q][2] = e2;
  };
  box(0, ol[0], E0, ol[1], E1, ol[2], il[2] - ol[2]);
  box(1, ol[0], E0, ol[1], E1, ih[2] + 1, oh[2] - ih[2]);
  box(2, ol[0], E0, ol[1], il[1] - ol[1], il[2], in2);
  box(3, ol[0], E0, ih[1] + 1, oh[1] - ih[1], il[2], in2);
  box(4, ol[0], il[0] - ol[0], il[1], in1, il[2], in2);
  box(5, ih[0] + 1, oh[0] - ih[0], il[1], in1, il[2], in2);
  return s;
}

__device__ __forceinline__ bool slab_node(const Slabs& sl, int q, int t, int& i, int& j, int& k) {
  const int e0 = sl.e[q][0], e1 = sl.e[q][1];
  if (t >= e0 * e1 * sl.e[q][2]) return false;
  i = sl.a[q][0] + t % e0;
  j = sl.a[q][1] + (t / e0) % e1;
  k = sl.a[q][2] + t / (e0 * e1);
  return true;
}

// Boundary fill in one pass over the padded nodes of the slabs (bc_slabs:
// outside the updated box, one or two ghost layers deep), nodes [t_begin,
// t_end) of slab q with stride t_step: each takes the value of the grid
// node its index maps to (wrap, clamp for the ghost layers behind a face,
// or across the centreline of a cylindrical grid): a
// copy when that node is updated by the stages, its boundary-condition value
// (computed here from the interior node it reads, or, on the centreline,
// from the azimuthal means computed before this pass) when it is a boundary
// node.  Only updated nodes are read, so the pass is race-free in one
// launch, and every node gets the value of a boundary pass followed by a
// ghost copy.
template <typename ST, typename MT, bool FAST>
__device__ __forceinline__ void fill_slab(const Layout& L, const Slabs& sl, int q, int t_begin, int t_step, int t_end,
                                          const double* inflow,
                                          const double* axis, const FlowC& F, ST* __restrict__ Q,
                                          const MT* __restrict__ M) {
  // one node per thread (four per thread with their loads issued together
  // measured slower: fewer resident threads)
  constexpr int U = 1;
  const int tot = min(t_end, sl.e[q][0] * sl.e[q][1] * sl.e[q][2]);
  const int bw = t_step;
  for (int tb = t_begin; tb < tot; tb += t_step * U) {
    long long dst[U], src[U], nb[U];
    int kind[U], face[U], inf[U];  // kind: 0 copy, 1 inflow, 2 far field, 3 centreline, -1 none
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int i, j, k;
      kind[u] = -1;
      face[u] = 0;
      inf[u] = 0;
      src[u] = nb[u] = dst[u] = 0;
      if (!slab_node(sl, q, tb + u * bw, i, j, k)) continue;
      // ghosts behind a face inside a larger grid are the halo exchange's
      if ((i < 0 && L.bc[0] == BC_EXCHANGE) || (i >= L.n[0] && L.bc[1] == BC_EXCHANGE) ||
          (j < 0 && L.bc[2] == BC_EXCHANGE) || (j >= L.n[1] && L.bc[3] == BC_EXCHANGE) ||
          (k < 0 && L.bc[4] == BC_EXCHANGE) || (k >= L.n[2] && L.bc[5] == BC_EXCHANGE))
        continue;
      dst[u] = L.at(i, j, k);
      int mi = i, mj = j, mk = k;
      L.map_node(mi, mj, mk);
      if (mi >= L.lo[0] && mi <= L.hi[0] && mj >= L.lo[1] && mj <= L.hi[1] && mk >= L.lo[2] && mk <= L.hi[2]) {
        kind[u] = 0;
        src[u] = L.at(mi, mj, mk);
        continue;
      }
      // boundary node (mi, mj, mk): the face latest in the order y-, y+, z-,
      // z+, x+, x- decides
      const int idx[3] = {mi, mj, mk};
      const int order[6] = {2, 3, 4, 5, 1, 0};
      int f = -1;
#pragma unroll
      for (int o = 0; o < 6; ++o) {
        const int ff = order[o], d = ff / 2;
        if (L.bc[ff] == BC_PERIODIC || L.bc[ff] == BC_EXCHANGE) continue;
        if (idx[d] == ((ff % 2 == 0) ? 0 : L.n[d] - 1)) f = ff;
      }
      face[u] = f;
      if (f < 0) continue;  // not reached: a node outside the updated box lies on some face
      if (L.bc[f] == BC_INFLOW) {  // x- face only: profile tabulated per (j, k)
        kind[u] = 1;
        inf[u] = mk * L.n[1] + mj;
        continue;
      }
      if (L.bc[f] == BC_AXIS) {  // azimuthal mean of the adjacent radial line
        kind[u] = 3;
        inf[u] = mi;
        continue;
      }
      kind[u] = 2;  // far field: nearest updated node, normal at the boundary node
      int ci[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) ci[d] = idx[d] < L.lo[d] ? L.lo[d] : (idx[d] > L.hi[d] ? L.hi[d] : idx[d]);
      src[u] = L.at(ci[0], ci[1], ci[2]);
      // on the centreline the face metric vanishes: normal of the adjacent radial node
      nb[u] = L.at(mi, (L.cyl && mj == 0) ? 1 : mj, mk);
    }
    ST qv[U][5], mv[U][3];
    double uin[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      uin[u] = 0.0;
      if (kind[u] == 0 || kind[u] == 2) {
#pragma unroll
        for (int v = 0; v < 5; ++v) qv[u][v] = Q[(long long)v * L.npad + src[u]];
      }
      if (kind[u] == 2) {
        const int d = face[u] / 2;
#pragma unroll
        for (int c = 0; c < 3; ++c) mv[u][c] = (ST)M[(long long)(3 * d + c) * L.npad + nb[u]];
      }
      if (kind[u] == 1) uin[u] = inflow[inf[u]];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (kind[u] < 0) continue;
      ST v[5];
      if (kind[u] == 0) {
#pragma unroll
        for (int c = 0; c < 5; ++c) v[c] = qv[u][c];
      } else if (kind[u] == 1) {
        to_conserved<ST, FAST>(flow_const<ST>(F.gm1, F.gm1_f), ST(1), (ST)uin[u], ST(0), ST(0),
                               flow_const<ST>(1.0 / F.gamma, F.pe_f), v);
      } else if (kind[u] == 3) {
#pragma unroll
        for (int c = 0; c < 5; ++c) v[c] = (ST)axis[c * L.n[0] + inf[u]];
      } else {
        const ST a = mv[u][0], b = mv[u][1], cc = mv[u][2];
        const ST sgn = (face[u] % 2 == 0) ? ST(-1) : ST(1);
        const ST inv = BcMath<ST, FAST>::div(sgn, BcMath<ST, FAST>::sqrt_(a * a + b * b + cc * cc));
        const ST n[3] = {a * inv, b * inv, cc * inv};
        riemann_farfield<ST, FAST>(F, qv[u], n, v);
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) Q[(long long)c * L.npad + dst[u]] = v[c];
    }
  }
}

template <typename ST, typename MT, bool FAST>
__global__ void k_bc_fill(const __grid_constant__ Layout L, const __grid_constant__ Slabs sl,
                          const double* __restrict__ inflow, const double* __restrict__ axis,
                          const __grid_constant__ FlowC F, ST* __restrict__ Q, const MT* __restrict__ M) {
  fill_slab<ST, MT, FAST>(L, sl, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, INT_MAX, inflow,
                    axis, F, Q, M);
}

// Centreline of a cylindrical grid (the paper's singularity treatment,
// Section 3 and Section 4.3): for every axial index i and variable v, the
// mean of Q_v over the P distinct azimuthal nodes of the radial line j = 1,
// summed in azimuthal order in FP64 -- the sequential order the paper keeps
// so that a partitioned run reproduces the serial one bit for bit.
// A block takes 32 consecutive i of one variable (blockIdx.y); lane = i.
// This is the general form, used for FP64 states: the loads are issued in
// parallel, the azimuth going through shared memory in chunks of 24 KB (96
// FP64 values per i), seven warps loading the next chunk (one coalesced row
// of 32 i per load) while warp 0 adds the current one value by value in
// azimuthal order.  FP32 states take axis_mean_f32 below.
constexpr int AX_WARPS = 8;
constexpr int AX_BYTES = 24576;  // one chunk buffer; two are used

// rows first + r, r = wr, wr + NW, ... < m, of the 32 i-columns into dst[r]:
// all loads of a warp issued before the first store
template <typename ST, int NW, int CH>
__device__ __forceinline__ void ax_load(ST (*dst)[32], const ST* q, long long plane, int first, int m, int wr,
                                        bool live, int lane) {
  constexpr int U = (CH + NW - 1) / NW;
  ST x[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int r = wr + u * NW;
    x[u] = (live && r < m) ? q[(long long)(first + r) * plane] : ST(0);
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int r = wr + u * NW;
    if (r < m) dst[r][lane] = x[u];
  }
}

template <typename ST>
__device__ __forceinline__ void axis_mean(const Layout& L, const ST* __restrict__ Q, double* __restrict__ axis) {
  constexpr int CH = AX_BYTES / (32 * (int)sizeof(ST));
  __shared__ ST buf[2][CH][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int v = blockIdx.y, P = L.pn[2], nch = (P + CH - 1) / CH;
  for (int bx = blockIdx.x; bx * 32 < L.n[0]; bx += gridDim.x) {  // block-uniform trip count
    const int i = bx * 32 + lane;
    const bool live = i < L.n[0];
    const ST* q = Q + (long long)v * L.npad + L.at(live ? i : 0, 1, 0);
    ax_load<ST, AX_WARPS, CH>(buf[0], q, L.plane, 0, min(CH, P), w, live, lane);  // chunk 0: every warp
    __syncthreads();
    double s = 0.0;
    for (int c = 0; c < nch; ++c) {
      const int base = c * CH, m = min(CH, P - base);
      if (w == 0) {
        const ST* b = &buf[c & 1][0][lane];
        for (int r = 0; r < m; ++r) s += (double)b[r * 32];
      } else if (c + 1 < nch) {
        ax_load<ST, AX_WARPS - 1, CH>(buf[(c + 1) & 1], q, L.plane, base + CH, min(CH, P - base - CH), w - 1, live,
                                      lane);
      }
      __syncthreads();
    }
    if (w == 0 && live) axis[v * L.n[0] + i] = s / P;
  }
}

// FP32 state.  Every partial sum of the sequential order is a multiple of
// 2^e, e the exponent of the unit in the last place of the smallest nonzero
// value, and at most sum |x| in magnitude; when that bound is below 2^(e+53)
// no partial sum rounds in FP64, so the sequential result is the exact sum,
// formed here as an integer sum of x / 2^e in any order (all warps, one pass
// for the exponent and the bound, one for the sum).  Otherwise, and for
// non-finite values, warp 0 runs the sequential chain.  On GB300 a warp-wide
// FP64 add or conversion occupies the FP64 pipe for many cycles, so the
// chain of P of them took about 30 us per launch on its own.
__device__ __forceinline__ void axis_mean_f32(const Layout& L, const float* __restrict__ Q, double* __restrict__ axis) {
  __shared__ int s_emin[AX_WARPS][32];
  __shared__ float s_abs[AX_WARPS][32];
  __shared__ long long s_acc[AX_WARPS][32];
  __shared__ int s_exact[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int v = blockIdx.y, P = L.pn[2];
  for (int bx = blockIdx.x; bx * 32 < L.n[0]; bx += gridDim.x) {  // block-uniform trip count
    const int i = bx * 32 + lane;
    const bool live = i < L.n[0];
    const float* q = Q + (long long)v * L.npad + L.at(live ? i : 0, 1, 0);
    int emin = INT_MAX;  // exponent of the smallest unit in the last place (nonzero values)
    float sabs = 0.f;    // sum of magnitudes; +inf marks a non-finite value
    if (live) {
#pragma unroll 12
      for (int k = w; k < P; k += AX_WARPS) {
        const unsigned b = __float_as_uint(q[(long long)k * L.plane]);
        const int E = (int)((b >> 23) & 0xffu);
        if (E == 255) sabs = INFINITY;
        if ((b & 0x7fffffffu) != 0u) emin = min(emin, E == 0 ? -149 : E - 150);
        sabs += __uint_as_float(b & 0x7fffffffu);
      }
    }
    s_emin[w][lane] = emin;
    s_abs[w][lane] = sabs;
    __syncthreads();
    if (w == 0) {
      int em = INT_MAX;
      float sa = 0.f;
      for (int r = 0; r < AX_WARPS; ++r) {
        em = min(em, s_emin[r][lane]);
        sa += s_abs[r][lane];
      }
      // the FP32 sum of P magnitudes is within a factor 1 + 2 P 2^-24 of the true sum
      const bool exact = em == INT_MAX ||
                         (isfinite(sa) && (double)sa * (1.0 + 2.0 * P * 0x1p-24) < ldexp(1.0, em + 53));
      s_exact[lane] = exact;
      s_emin[0][lane] = em;
    }
    __syncthreads();
    const int em = s_emin[0][lane];
    const bool exact = s_exact[lane] != 0;
    long long acc = 0;
    if (live && exact && em != INT_MAX) {
#pragma unroll 12
      for (int k = w; k < P; k += AX_WARPS) {
        const unsigned b = __float_as_uint(q[(long long)k * L.plane]);
        const int E = (int)((b >> 23) & 0xffu);
        const long long m = (long long)((b & 0x7fffffu) | (E ? 0x800000u : 0u));
        const long long t = m << ((E == 0 ? -149 : E - 150) - em);  // < 2^53 by the bound
        acc += (b >> 31) ? -t : t;
      }
    }
    s_acc[w][lane] = acc;
    __syncthreads();
    if (w == 0 && live) {
      double s = 0.0;
      if (exact) {
        long long t = 0;
        for (int r = 0; r < AX_WARPS; ++r) t += s_acc[r][lane];
        s = em == INT_MAX ? 0.0 : ldexp((double)t, em);
      } else {
        for (int k = 0; k < P; ++k) s += (double)q[(long long)k * L.plane];
      }
      axis[v * L.n[0] + i] = s / P;
    }
    __syncthreads();  // the shared arrays are reused by the next 32 columns
  }
}

template <typename ST>
__device__ __forceinline__ void axis_mean_any(const Layout& L, const ST* __restrict__ Q, double* __restrict__ axis) {
  if constexpr (sizeof(ST) == 4)
    axis_mean_f32(L, Q, axis);
  else
    axis_mean<ST>(L, Q, axis);
}

template <typename ST>
__global__ void __launch_bounds__(32 * AX_WARPS) k_axis_mean(const __grid_constant__ Layout L, const ST* __restrict__ Q,
                                                             double* __restrict__ axis) {
  axis_mean_any<ST>(L, Q, axis);
}

// batched versions: grid blockIdx.z of the table, state copy `which`
struct BcCtx {
  Layout L;
  Slabs fill;
  const double* inflow;
  double* axis;
  FlowC F;
  void* Q[3];
  const void* M;
};

// one work item per block: (grid, slab, first node, end node) of the slab's
// enumeration, at most BC_ITEM_NODES nodes, so that the blocks follow the
// slab sizes of uneven grids
template <typename ST, typename MT, bool FAST>
__global__ void k_bc_fill_batch(const BcCtx* __restrict__ ctx, const int4* __restrict__ items, int which) {
  const int4 w = items[blockIdx.x];
  const BcCtx& X = ctx[w.x];
  fill_slab<ST, MT, FAST>(X.L, X.fill, w.y, w.z + threadIdx.x, blockDim.x, w.w, X.inflow, X.axis, X.F, (ST*)X.Q[which],
                    (const MT*)X.M);
}

template <typename ST>
__global__ void __launch_bounds__(32 * AX_WARPS) k_axis_mean_batch(const BcCtx* __restrict__ ctx, int which) {
  const BcCtx& X = ctx[blockIdx.z];
  if (X.L.cyl) axis_mean_any<ST>(X.L, (const ST*)X.Q[which], X.axis);
}

// Halo exchange between blocks of one grid (the paper's ghost exchange,
// Section 4.2, between blocks on one device): each entry copies the two node
// layers of block src next to a shared face into the two ghost layers of
// block dst behind it, over the padded extents of the other two directions.
// One launch per direction, in the order i, j, k, so that edge and corner
// ghosts take values already exchanged in the earlier directions.
template <typename ST>
__global__ void k_exchange(const XEntry* __restrict__ xs, int which) {
  const XEntry& X = xs[blockIdx.y];
  const int d = X.d, e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
  const long long per_var = 2LL * X.ea * X.eb;
  const long long tot = 5 * per_var;
  ST* dq = (ST*)X.dq[which];
  const ST* sq = (const ST*)X.sq[which];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(t / per_var);
    long long r = t - v * per_var;
    const int a = (int)(r % X.ea) - NG;  // fastest: direction e1
    r /= X.ea;
    const int b = (int)(r % X.eb) - NG;
    const int l = (int)(r / X.eb);
    int di[3], si[3];
    di[d] = X.dfirst + l;
    si[d] = X.sfirst + l;
    di[e1] = si[e1] = a;
    di[e2] = si[e2] = b;
    const long long dofs = (di[0] + NG) + (di[1] + NG) * X.dpitch + (di[2] + NG) * X.dplane;
    const long long sofs = (si[0] + NG) + (si[1] + NG) * X.spitch + (si[2] + NG) * X.splane;
    dq[v * X.dnpad + dofs] = sq[v * X.snpad + sofs];
  }
}

// Face halo of a block for a neighbour on another rank: the two node layers
// [first, first + 1] along direction d over the padded extents of the other
// two directions, as a dense buffer [v][l][b][a] (a fastest: direction e1,
// then e2, in i, j, k order).  pack copies state -> buffer, unpack buffer ->
// state.
template <typename ST, bool PACK>
__global__ void k_halo(Layout L, ST* __restrict__ Q, ST* __restrict__ buf, int d, int first) {
  const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
  const int ea = L.n[e1] + 2 * NG, eb = L.n[e2] + 2 * NG;
  const long long per_var = 2LL * ea * eb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 5 * per_var;
       t += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(t / per_var);
    long long r = t - v * per_var;
    const int a = (int)(r % ea) - NG;
    r /= ea;
    const int b = (int)(r % eb) - NG;
    const int l = (int)(r / eb);
    int idx[3];
    idx[d] = first + l;
    idx[e1] = a;
    idx[e2] = b;
    const long long o = v * L.npad + L.at(idx[0], idx[1], idx[2]);
    if (PACK)
      buf[t] = Q[o];
    else
      Q[o] = buf[t];
  }
}

// axial inflow velocity of the jet profile at the x- face nodes (FP64, once per state_init)
__global__ void k_inflow(Layout L, Coords C, FlowC F, double* __restrict__ inflow) {
  const int n = L.n[1] * L.n[2];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int j = t % L.n[1], k = t / L.n[1];
    const double y = C.x(1, 0, j, k), z = C.x(2, 0, j, k);
    inflow[t] = jet_profile(F, sqrt(y * y + z * z));
  }
}

// ---------------------------------------------------------------------------
// initial state (jet column plus seeded noise, or air at rest)
// ---------------------------------------------------------------------------

// The noise of a node is keyed to its global linear index (goff: global index
// of local node 0, gn: global node counts), so a block of a larger grid gets
// the values of the same nodes of the whole grid.
template <typename ST>
__global__ void k_init(Layout L, Coords C, FlowC F, uint64_t seed, ST* __restrict__ Q, double* __restrict__ Q0d,
                       int go0, int go1, int go2, int gn0, int gn1) {
  long long N = (long long)L.n[0] * L.n[1] * L.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % L.n[0]);
    int j = (int)((t / L.n[0]) % L.n[1]);
    int k = (int)(t / ((long long)L.n[0] * L.n[1]));
    double u[3] = {0.0, 0.0, 0.0};
    if (F.ic == JZ_IC_JET) {
      double y = C.x(1, i, j, k), z = C.x(2, i, j, k);
      u[0] = jet_profile(F, sqrt(y * y + z * z));
      const uint64_t lin = (uint64_t)(i + go0) + (uint64_t)gn0 * ((uint64_t)(j + go1) + (uint64_t)gn1 * (uint64_t)(k + go2));
      for (int m = 0; m < 3; ++m) {
        double xi = unit53(splitmix64(seed ^ (3ULL * lin + (uint64_t)m)));
        u[m] += F.noise * F.mach * (2.0 * xi - 1.0);
      }
    }
    double q[5];
    to_conserved<double>(F.gm1, 1.0, u[0], u[1], u[2], 1.0 / F.gamma, q);
    long long n = L.at(i, j, k);
    for (int v = 0; v < 5; ++v) Q[(long long)v * L.npad + n] = (ST)q[v];
    if (Q0d)
      for (int v = 0; v < 5; ++v) Q0d[(long long)v * L.npad + n] = q[v];
  }
}

// the state Q (rounded to ST) and, for a JZ_P32_S64 grid, its FP64 copy Q0d
template <typename ST>
__global__ void k_unpack(Layout L, const double* __restrict__ dense, ST* __restrict__ Q, double* __restrict__ Q0d) {
  long long N = (long long)L.n[0] * L.n[1] * L.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 5 * N; t += (long long)gridDim.x * blockDim.x) {
    int v = (int)(t / N);
    long long r = t - v * N;
    int i = (int)(r % L.n[0]);
    int j = (int)((r / L.n[0]) % L.n[1]);
    int k = (int)(r / ((long long)L.n[0] * L.n[1]));
    const long long e = (long long)v * L.npad + L.at(i, j, k);
    Q[e] = (ST)dense[t];
    if (Q0d) Q0d[e] = dense[t];
  }
}

// Q0d (FP64 state of a JZ_P32_S64 grid, else null) supplies the updated
// nodes (and the superposed azimuthal plane of a cylinder, a copy of plane 0);
// boundary nodes come from the state Q.
template <typename ST>
__global__ void k_pack(Layout L, const ST* __restrict__ Q, const double* __restrict__ Q0d, double* __restrict__ dense) {
  long long N = (long long)L.n[0] * L.n[1] * L.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 5 * N; t += (long long)gridDim.x * blockDim.x) {
    int v = (int)(t / N);
    long long r = t - v * N;
    int i = (int)(r % L.n[0]);
    int j = (int)((r / L.n[0]) % L.n[1]);
    int k = (int)(r / ((long long)L.n[0] * L.n[1]));
    int mi = i, mj = j, mk = k;
    L.map_node(mi, mj, mk);
    if (Q0d && mi >= L.lo[0] && mi <= L.hi[0] && mj >= L.lo[1] && mj <= L.hi[1] && mk >= L.lo[2] && mk <= L.hi[2])
      dense[t] = Q0d[(long long)v * L.npad + L.at(mi, mj, mk)];
    else
      dense[t] = (double)Q[(long long)v * L.npad + L.at(i, j, k)];
  }
}

// one metric field f (S^k_m at 3k+m, J at 9) of the grid's own nodes, widened
template <typename MT>
__global__ void k_pack_metric(Layout L, const MT* __restrict__ M, int f, double* __restrict__ dense) {
  const long long N = (long long)L.n[0] * L.n[1] * L.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % L.n[0]);
    const int j = (int)((t / L.n[0]) % L.n[1]);
    const int k = (int)(t / ((long long)L.n[0] * L.n[1]));
    dense[t] = (double)M[(long long)f * L.npad + L.at(i, j, k)];
  }
}

int grid_blocks(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  const long long cap = 32LL * device_sm_count();
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace

Shell make_shell(const Layout& L, const int a[3], const int b[3]) {
  Shell s;
  for (int d = 0; d < 3; ++d) { s.a[d] = a[d]; s.b[d] = b[d]; s.E[d] = L.n[d] + 2 * NG; }
  long long E0 = s.E[0], E1 = s.E[1], E2 = s.E[2];
  long long in0 = b[0] - a[0] + 1, in1 = b[1] - a[1] + 1, in2 = b[2] - a[2] + 1;
  s.cz = (E2 - in2) * E1 * E0;
  s.cy = in2 * (E1 - in1) * E0;
  s.cx = in2 * in1 * (E0 - in0);
  return s;
}

cudaError_t launch_tables(const TabParams& p, double* tables, cudaStream_t s) {
  long long len = 0;
  for (int d = 0; d < 3; ++d) len += 2LL * (p.n[d] + 2 * NG) + 3LL * (p.n[d] + 2 * NG);
  len += 2LL * (p.n[2] + 2 * NG);
  k_tables<<<grid_blocks(len, 256), 256, 0, s>>>(p, tables);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_metrics(const GridDev& g, cudaStream_t s) {
  // grid nodes, extended by one ghost layer behind faces inside a larger grid
  int a[3], b[3];
  for (int d = 0; d < 3; ++d) {
    a[d] = g.L.bc[2 * d] == BC_EXCHANGE ? -1 : 0;
    b[d] = g.L.bc[2 * d + 1] == BC_EXCHANGE ? g.L.n[d] : g.L.n[d] - 1;
  }
  const long long N = (long long)(b[0] - a[0] + 1) * (b[1] - a[1] + 1) * (b[2] - a[2] + 1);
  Shell sh = make_shell(g.L, a, b);  // the remaining ghost nodes copy the node their index maps to
  if (g.prec == JZ_P32 || g.prec == JZ_P32_S64) {
    k_metrics<float><<<grid_blocks(N, 128), 128, 0, s>>>(g.L, g.C, (float*)g.M, a[0], a[1], a[2], b[0], b[1], b[2]);
    k_fill_ghosts<float><<<grid_blocks(sh.total(), 256), 256, 0, s>>>(g.L, sh, (float*)g.M, 10);
  } else {
    k_metrics<double><<<grid_blocks(N, 128), 128, 0, s>>>(g.L, g.C, (double*)g.M, a[0], a[1], a[2], b[0], b[1], b[2]);
    k_fill_ghosts<double><<<grid_blocks(sh.total(), 256), 256, 0, s>>>(g.L, sh, (double*)g.M, 10);
  }
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_init(const GridDev& g, uint64_t seed, cudaStream_t s) {
  long long N = (long long)g.L.n[0] * g.L.n[1] * g.L.n[2];
  k_inflow<<<grid_blocks((long long)g.L.n[1] * g.L.n[2], 256), 256, 0, s>>>(g.L, g.C, g.F, g.inflow);
  count_launches(1);
  if (g.prec == JZ_P64)
    k_init<double><<<grid_blocks(N, 256), 256, 0, s>>>(g.L, g.C, g.F, seed, (double*)g.Q0, nullptr, g.goff[0],
                                                       g.goff[1], g.goff[2], g.gn[0], g.gn[1]);
  else
    k_init<float><<<grid_blocks(N, 256), 256, 0, s>>>(g.L, g.C, g.F, seed, (float*)g.Q0, g.Q0d, g.goff[0],
                                                      g.goff[1], g.goff[2], g.gn[0], g.gn[1]);
  count_launches(1);
  return cudaGetLastError();
}

// the padded nodes outside the updated box [lo, hi]
// The padded nodes a boundary pass sets.  Behind a physical face (inflow,
// far field, centreline) the stages read one ghost layer only: the first
// updated node is one in from the boundary node, so its five-point stencil
// reaches one node past it, and the second layer enters nothing but the
// residual of the boundary node, which is not updated.  The per-stage pass
// (full = false) therefore sets the boundary nodes and the first ghost
// layer there; periodic directions and exchange faces keep both layers.  The
// pass after a state is set (full = true) covers both layers everywhere.
Slabs bc_slabs(const Layout& L, bool full) {
  int pad_lo[3], pad_hi[3];
  for (int a = 0; a < 3; ++a) {
    const bool keep_lo = full || L.bc[2 * a] == BC_PERIODIC || L.bc[2 * a] == BC_EXCHANGE;
    const bool keep_hi = full || L.bc[2 * a + 1] == BC_PERIODIC || L.bc[2 * a + 1] == BC_EXCHANGE;
    pad_lo[a] = keep_lo ? -NG : -1;
    pad_hi[a] = keep_hi ? L.n[a] + 1 : L.n[a];
  }
  return make_slabs(pad_lo, pad_hi, L.lo, L.hi);
}

// blocks per slab: at most 128 (six slabs then hold about one resident wave
// of the fill's 256-thread blocks, which stride over their slab; on the
// 256x192x192 grid 0.031 ms per fill against 0.036 ms with up to 1024)
int slab_blocks(const Slabs& sl) {
  long long big = 1;
  for (int q = 0; q < 6; ++q) {
    long long c = (long long)sl.e[q][0] * sl.e[q][1] * sl.e[q][2];
    big = c > big ? c : big;
  }
  int b = grid_blocks(big, 256);
  return b < 128 ? b : 128;
}

cudaError_t launch_bc(const GridDev& g, void* Q, cudaStream_t s, bool full) {
  const Slabs sl = bc_slabs(g.L, full);
  const dim3 b(slab_blocks(sl), 6);
  if (g.L.cyl) {
    const dim3 ab((g.L.n[0] + 31) / 32, 5);
    if (g.prec == JZ_P64)
      k_axis_mean<double><<<ab, 32 * AX_WARPS, 0, s>>>(g.L, (const double*)Q, g.axis);
    else
      k_axis_mean<float><<<ab, 32 * AX_WARPS, 0, s>>>(g.L, (const float*)Q, g.axis);
    count_launches(1);
  }
  switch (g.prec) {
    case JZ_P64:
      k_bc_fill<double, double, false><<<b, 256, 0, s>>>(g.L, sl, g.inflow, g.axis, g.F, (double*)Q,
                                                         (const double*)g.M);
      break;
    case JZ_P32_M64:
      k_bc_fill<float, double, true><<<b, 256, 0, s>>>(g.L, sl, g.inflow, g.axis, g.F, (float*)Q, (const double*)g.M);
      break;
    case JZ_P32_S64:
      k_bc_fill<float, float, false><<<b, 256, 0, s>>>(g.L, sl, g.inflow, g.axis, g.F, (float*)Q, (const float*)g.M);
      break;
    default:
      k_bc_fill<float, float, true><<<b, 256, 0, s>>>(g.L, sl, g.inflow, g.axis, g.F, (float*)Q, (const float*)g.M);
      break;
  }
  count_launches(1);
  return cudaGetLastError();
}

size_t bc_ctx_bytes() { return sizeof(BcCtx); }

// fills the host-side table entry
void bc_ctx_fill(void* dst, const GridDev& g) {
  BcCtx& X = *(BcCtx*)dst;
  X.L = g.L;
  X.fill = bc_slabs(g.L, false);
  X.inflow = g.inflow;
  X.axis = g.axis;
  X.F = g.F;
  X.Q[0] = g.Q0;
  X.Q[1] = g.QA;
  X.Q[2] = g.QB;
  X.M = g.M;
}

void bc_fill_items(const GridDev& g, int grid, std::vector<int4>& out) {
  const Slabs sl = bc_slabs(g.L, false);
  for (int q = 0; q < 6; ++q) {
    const int tot = sl.e[q][0] * sl.e[q][1] * sl.e[q][2];
    for (int t = 0; t < tot; t += BC_ITEM_NODES) out.push_back(make_int4(grid, q, t, std::min(tot, t + BC_ITEM_NODES)));
  }
}

cudaError_t launch_bc_batch(int prec, const void* ctx, int n, const int4* items, int nitems, int which, bool cyl,
                            cudaStream_t s) {
  const BcCtx* X = (const BcCtx*)ctx;
  if (cyl) {  // some grid of the batch is cylindrical: centreline means first
    const dim3 ab(8, 5, n);
    if (prec == JZ_P64)
      k_axis_mean_batch<double><<<ab, 32 * AX_WARPS, 0, s>>>(X, which);
    else
      k_axis_mean_batch<float><<<ab, 32 * AX_WARPS, 0, s>>>(X, which);
    count_launches(1);
  }
  switch (prec) {
    case JZ_P64: k_bc_fill_batch<double, double, false><<<nitems, 256, 0, s>>>(X, items, which); break;
    case JZ_P32_M64: k_bc_fill_batch<float, double, true><<<nitems, 256, 0, s>>>(X, items, which); break;
    case JZ_P32_S64: k_bc_fill_batch<float, float, false><<<nitems, 256, 0, s>>>(X, items, which); break;
    default: k_bc_fill_batch<float, float, true><<<nitems, 256, 0, s>>>(X, items, which); break;
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const GridDev& g, const double* dense, cudaStream_t s) {
  long long N = 5LL * g.L.n[0] * g.L.n[1] * g.L.n[2];
  if (g.prec == JZ_P64)
    k_unpack<double><<<grid_blocks(N, 256), 256, 0, s>>>(g.L, dense, (double*)g.Q0, nullptr);
  else
    k_unpack<float><<<grid_blocks(N, 256), 256, 0, s>>>(g.L, dense, (float*)g.Q0, g.Q0d);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pack_metric(const GridDev& g, int f, double* dense, cudaStream_t s) {
  const long long N = (long long)g.L.n[0] * g.L.n[1] * g.L.n[2];
  if (g.prec == JZ_P64 || g.prec == JZ_P32_M64)
    k_pack_metric<double><<<grid_blocks(N, 256), 256, 0, s>>>(g.L, (const double*)g.M, f, dense);
  else
    k_pack_metric<float><<<grid_blocks(N, 256), 256, 0, s>>>(g.L, (const float*)g.M, f, dense);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pack(const GridDev& g, double* dense, cudaStream_t s) {
  long long N = 5LL * g.L.n[0] * g.L.n[1] * g.L.n[2];
  if (g.prec == JZ_P64)
    k_pack<double><<<grid_blocks(N, 256), 256, 0, s>>>(g.L, (const double*)g.Q0, nullptr, dense);
  else
    k_pack<float><<<grid_blocks(N, 256), 256, 0, s>>>(g.L, (const float*)g.Q0, g.Q0d, dense);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_halo(const GridDev& g, void* Q, void* buf, int d, int first, bool pack, cudaStream_t s) {
  const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
  const long long N = 10LL * (g.L.n[e1] + 2 * NG) * (g.L.n[e2] + 2 * NG);
  const int blocks = grid_blocks(N, 256);
  if (g.prec == JZ_P64) {
    if (pack) k_halo<double, true><<<blocks, 256, 0, s>>>(g.L, (double*)Q, (double*)buf, d, first);
    else k_halo<double, false><<<blocks, 256, 0, s>>>(g.L, (double*)Q, (double*)buf, d, first);
  } else {
    if (pack) k_halo<float, true><<<blocks, 256, 0, s>>>(g.L, (float*)Q, (float*)buf, d, first);
    else k_halo<float, false><<<blocks, 256, 0, s>>>(g.L, (float*)Q, (float*)buf, d, first);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_exchange(int prec, const void* entries, int begin, int count, int blocks, int which,
                            cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const XEntry* X = (const XEntry*)entries + begin;
  const dim3 grid(blocks, count);
  if (prec == JZ_P64)
    k_exchange<double><<<grid, 256, 0, s>>>(X, which);
  else
    k_exchange<float><<<grid, 256, 0, s>>>(X, which);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace jz
