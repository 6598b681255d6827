// jz_stage.cu -- the fused Runge-Kutta stage kernel: residual evaluation and
// stage update in one pass over HBM.
//
// Paper: arXiv 2003.09926, Section 3 and Section 4.2 (Fig. jazzy): per
// Runge-Kutta sub-step, the inviscid flux (centred, 2nd order, in general
// curvilinear coordinates), the anisotropic scalar artificial dissipation
// (Turkel & Vatsa, pressure sensor, five-point stencil, Section 4.3) and the
// viscous flux (Stokes stress, Fourier heat flux, Sutherland viscosity,
// Eqs. q_mod, sutherland, tau_mod) plus a Smagorinsky (or Vreman) eddy viscosity, then the
// update Q^(l) = Q^(0) - alpha_l dt J R(Q^(l-1)) of the 5-stage scheme.
//
// Residual in face form.  With G^k = E^k - F^k the contravariant inviscid
// minus viscous flux at a node and d^k the dissipative face flux,
//   R_n = sum_k [ (G^k_{n+1} - G^k_{n-1})/2 - (d^k_{n+1/2} - d^k_{n-1/2}) ]
//       = sum_k [ h^k_{n+1/2} - h^k_{n-1/2} ],   h_{n+1/2} = (G_n + G_{n+1})/2 - d_{n+1/2},
// algebraically identical, telescoping exactly (discrete conservation by
// construction); each face flux is formed once.
//
// GPU organisation (2.5-D streaming, one CTA per SM):
//  - a CTA owns a TI x TJ tile of (i, j) columns (tile origins at multiples of
//    TI, TJ) and marches in k over a chunk of kc planes;
//  - TMA (cp.async.bulk.tensor) stages the raw conserved variables of one
//    plane over the tile plus a two-node halo (the paper's two-layer ghost
//    fringe) into shared memory two planes ahead (double buffer), and the ten
//    metric fields of one plane one plane ahead; completion is tracked by
//    mbarriers whose waits are bounded;
//  - each staged plane is converted once into a 4-plane ring of node records
//    (rho, u, v, w, e, p, T);
//  - the CTA has one thread per node of the plus-shaped node set of a plane
//    (tile nodes plus the one-node i and j halo): every thread forms one
//    node's flux G^k, radius lambda~^k and sensor nu^k per plane (tile
//    threads for all three directions, halo threads for their own
//    direction), so the expensive node work is balanced across warps;
//  - i and j face fluxes go through shared memory, the k face flux of a
//    column stays in its thread's registers;
//  - the residual of plane t is completed and Q^(l) written with J and
//    Q^(0) held in registers;
//  - every configuration is compiled for the Smagorinsky flow model of the
//    workloads with constant flags and once with the flags read at run time.
#include <cmath>
#include <cstdint>

#include "jz_stage_common.cuh"

namespace jz {

using namespace stg;

namespace {

// ---------------------------------------------------------------------------
// kernel configuration and shared-memory layout
// ---------------------------------------------------------------------------

template <typename R, typename MT, int TI_, int TJ_>
struct Cfg {
  static constexpr int TI = TI_, TJ = TJ_;
  static constexpr int NTILE = TI * TJ;
  static constexpr int NJH = 2 * TI;                 // j-halo nodes (rows -1 and TJ)
  static constexpr int NIH = 2 * TJ;                 // i-halo nodes (columns -1 and TI)
  static constexpr int NT = NTILE + NJH + NIH;       // threads per CTA
  static constexpr int RW = TI + 4, RH = TJ + 4, PL = RW * RH;  // staged plane: tile + 2-node halo
  static constexpr size_t al(size_t x) { return (x + 127) / 128 * 128; }
  static constexpr size_t RAW_B = al(sizeof(R) * 5 * PL);
  static constexpr size_t MET_B = al(sizeof(MT) * 10 * PL);
  static constexpr size_t RING_B = al(sizeof(R) * 4 * NV * PL);
  static constexpr size_t GI_B = al(sizeof(R) * 5 * TJ * (TI + 2));
  static constexpr size_t GJ_B = al(sizeof(R) * 5 * (TJ + 2) * TI);
  static constexpr size_t LI_B = al(sizeof(R) * 2 * TJ * (TI + 2));
  static constexpr size_t LJ_B = al(sizeof(R) * 2 * (TJ + 2) * TI);
  static constexpr size_t HI_B = al(sizeof(R) * 5 * TJ * (TI + 1));
  static constexpr size_t HJ_B = al(sizeof(R) * 5 * (TJ + 1) * TI);
  static constexpr size_t O_RAW0 = 0;
  static constexpr size_t O_RAW1 = O_RAW0 + RAW_B;
  static constexpr size_t O_MET = O_RAW1 + RAW_B;
  static constexpr size_t O_RING = O_MET + MET_B;
  static constexpr size_t O_GI = O_RING + RING_B;
  static constexpr size_t O_GJ = O_GI + GI_B;
  static constexpr size_t O_LI = O_GJ + GJ_B;
  static constexpr size_t O_LJ = O_LI + LI_B;
  static constexpr size_t O_HI = O_LJ + LJ_B;
  static constexpr size_t O_HJ = O_HI + HI_B;
  static constexpr size_t O_BAR = O_HJ + HJ_B;
  static constexpr size_t BYTES = O_BAR + 128;
  // CTAs per SM that fit (227 KB per SM, ~1 KB reserved per CTA)
  static constexpr int MINB = 2 * (BYTES + 1024 + 128) <= 232448 ? 2 : 1;
  static constexpr uint32_t RAW_TX = sizeof(R) * 5 * PL;
  static constexpr uint32_t MET_TX = sizeof(MT) * 10 * PL;
};

}  // namespace

namespace {

template <typename R, int RW, int PL>
__device__ __forceinline__ R ring_at(const R* ring, int slot, int var, int y, int x) {
  return ring[(slot * NV + var) * PL + y * RW + x];
}

// Node quantities of node (x, y) of the centre plane (ring slot sC; the
// planes below / above in sM / sP): G^k = E^k - F^k, lambda~^k and nu^k.
// DIR = 0: all three directions; DIR = 1 / 2: direction i / j only.
template <typename R, typename MT, int RW, int PL, int DIR, int MD>
__device__ __forceinline__ void node_flux(const R* __restrict__ ring, const MT* __restrict__ met, int sM, int sC, int sP,
                                          int x, int y, const KConst<R>& c, R G[3][5], R lt[3], R nu[3], R& Jn) {
  const int lx = x + 2, ly = y + 2, o = ly * RW + lx;
  R S[9];
#pragma unroll
  for (int f = 0; f < 9; ++f) S[f] = (R)met[f * PL + o];
  Jn = (R)met[9 * PL + o];
  auto at = [&](int slot, int var, int dy, int dx) { return ring[(slot * NV + var) * PL + o + dy * RW + dx]; };
  const R rho = at(sC, V_RHO, 0, 0);
  const R u = at(sC, V_U, 0, 0), v = at(sC, V_V, 0, 0), w = at(sC, V_W, 0, 0);
  const R e = at(sC, V_E, 0, 0), p = at(sC, V_P, 0, 0), T = at(sC, V_T, 0, 0);
  constexpr int K0 = DIR == 0 ? 0 : DIR - 1;
  constexpr int K1 = DIR == 0 ? 3 : DIR;

  R Fv[3][4];  // viscous flux vectors F_m (m = x, y, z), components 1..4
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q) Fv[m][q] = R(0);
  if (ModelFlags<MD>::viscous(c)) {
    const int var[4] = {V_U, V_V, V_W, V_T};
    R g[4][3];  // Cartesian gradients of u, v, w, T: J/2 sum_k S^k_m (phi_+ - phi_-)
    const R hJ = R(0.5) * Jn;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const R d0 = at(sC, var[q], 0, 1) - at(sC, var[q], 0, -1);
      const R d1 = at(sC, var[q], 1, 0) - at(sC, var[q], -1, 0);
      const R d2 = at(sP, var[q], 0, 0) - at(sM, var[q], 0, 0);
#pragma unroll
      for (int m = 0; m < 3; ++m) g[q][m] = hJ * (S[m] * d0 + S[3 + m] * d1 + S[6 + m] * d2);
    }
    const R mu = Fn<R>::div(c.mu_inf * T * Fn<R>::sqrt_(T) * c.s1p1, T + c.s1);  // Sutherland
    R mu_t = R(0);
    // Smagorinsky or Vreman, Delta = J^(-1/3); an unfused product, so that
    // mu + mu_t rounds alike in the constant-flag and runtime-flag builds
    if (ModelFlags<MD>::sgs(c)) mu_t = Fn<R>::mul_rn(rho, eddy_nu<R, ModelFlags<MD>::eddy>(c, g, Jn));
    const R mue = mu + mu_t;
    const R kap = c.cp * (mu * c.inv_pr + mu_t * c.inv_prt);
    const R div3 = (g[0][0] + g[1][1] + g[2][2]) * R(2.0 / 3.0);
    const R t01 = mue * (g[0][1] + g[1][0]), t02 = mue * (g[0][2] + g[2][0]), t12 = mue * (g[1][2] + g[2][1]);
    Fv[0][0] = mue * (R(2) * g[0][0] - div3); Fv[0][1] = t01; Fv[0][2] = t02;
    Fv[1][0] = t01; Fv[1][1] = mue * (R(2) * g[1][1] - div3); Fv[1][2] = t12;
    Fv[2][0] = t02; Fv[2][1] = t12; Fv[2][2] = mue * (R(2) * g[2][2] - div3);
#pragma unroll
    for (int m = 0; m < 3; ++m) Fv[m][3] = u * Fv[m][0] + v * Fv[m][1] + w * Fv[m][2] + kap * g[3][m];
  }

  R lam[3], U[3];
  const R cson = Fn<R>::sqrt_(T);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    U[k] = S[3 * k] * u + S[3 * k + 1] * v + S[3 * k + 2] * w;
    const R sn = Fn<R>::sqrt_(S[3 * k] * S[3 * k] + S[3 * k + 1] * S[3 * k + 1] + S[3 * k + 2] * S[3 * k + 2]);
    lam[k] = fabs(U[k]) + cson * sn;
  }
  R sq[3] = {R(0), R(0), R(0)};
  if (ModelFlags<MD>::sig_half(c)) {
#pragma unroll
    for (int k = 0; k < 3; ++k) sq[k] = Fn<R>::sqrt_(lam[k]);
  }
  const R m1 = rho * u, m2 = rho * v, m3 = rho * w;
#pragma unroll
  for (int k = K0; k < K1; ++k) {
    const R Sx = S[3 * k], Sy = S[3 * k + 1], Sz = S[3 * k + 2];
    R Fk[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) Fk[q] = Sx * Fv[0][q] + Sy * Fv[1][q] + Sz * Fv[2][q];
    // E^k = [rho U, rho u U + S_x p, rho v U + S_y p, rho w U + S_z p, (e + p) U]
    G[k][0] = rho * U[k];
    G[k][1] = m1 * U[k] + Sx * p - Fk[0];
    G[k][2] = m2 * U[k] + Sy * p - Fk[1];
    G[k][3] = m3 * U[k] + Sz * p - Fk[2];
    G[k][4] = (e + p) * U[k] - Fk[3];
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    if (ModelFlags<MD>::sig_half(c))  // lambda (1 + (la/l)^1/2 + (lb/l)^1/2) = lambda + sqrt(lambda) (sqrt(la) + sqrt(lb))
      lt[k] = lam[k] + sq[k] * (sq[a] + sq[b]);
    else
      lt[k] = lam[k] > R(0) ? lam[k] * (R(1) + Fn<R>::powp(Fn<R>::div(lam[a], lam[k]), c.sigma) +
                                        Fn<R>::powp(Fn<R>::div(lam[b], lam[k]), c.sigma))
                            : R(0);  // zero face metric (a centreline): the limit for sigma < 1
    R pm, pp;
    if (k == 0) { pm = at(sC, V_P, 0, -1); pp = at(sC, V_P, 0, 1); }
    else if (k == 1) { pm = at(sC, V_P, -1, 0); pp = at(sC, V_P, 1, 0); }
    else { pm = at(sM, V_P, 0, 0); pp = at(sP, V_P, 0, 0); }
    nu[k] = Fn<R>::div(fabs(pp - R(2) * p + pm), pp + R(2) * p + pm);
  }
}

// face flux h = (G_a + G_b)/2 - lam [eps2 (q_b - q_a) - eps4 (q_{b+1} - 3 q_b + 3 q_a - q_{a-1})]
template <typename R>
__device__ __forceinline__ R face_h(R Ga, R Gb, R qam, R qa, R qb, R qbp, R lam, R e2, R e4) {
  return R(0.5) * (Ga + Gb) - lam * (e2 * (qb - qa) - e4 * (qbp - R(3) * qb + R(3) * qa - qam));
}

template <typename R>
__device__ __forceinline__ void face_coeffs(const KConst<R>& c, R lta, R ltb, R nua, R nub, R& lam, R& e2, R& e4) {
  lam = R(0.5) * (lta + ltb);
  e2 = c.k2 * rmax(nua, nub);
  e4 = rmax(R(0), c.k4 - e2);
}

// The five face fluxes between four consecutive nodes n-1, n, n+1, n+2 of a
// ring line (offsets o0..o3 in one ring slot or slots s0..s3).
template <typename R, int PL>
__device__ __forceinline__ void face5(const R* ring, const int so[4], const int oo[4], const R Ga[5], const R Gb[5],
                                      R lam, R e2, R e4, R h[5]) {
  R rho[4], q[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) rho[n] = ring[(so[n] * NV + V_RHO) * PL + oo[n]];
  h[0] = face_h<R>(Ga[0], Gb[0], rho[0], rho[1], rho[2], rho[3], lam, e2, e4);
#pragma unroll
  for (int c = 1; c < 4; ++c) {
#pragma unroll
    for (int n = 0; n < 4; ++n) q[n] = rho[n] * ring[(so[n] * NV + c) * PL + oo[n]];  // rho u_c
    h[c] = face_h<R>(Ga[c], Gb[c], q[0], q[1], q[2], q[3], lam, e2, e4);
  }
#pragma unroll
  for (int n = 0; n < 4; ++n) q[n] = ring[(so[n] * NV + V_E) * PL + oo[n]];
  h[4] = face_h<R>(Ga[4], Gb[4], q[0], q[1], q[2], q[3], lam, e2, e4);
}

// One work item: the tile (bx, by) and k-chunk bz of grid X for stage st.
// ph[] counts completed phases of the three mbarriers (identical in every
// thread); issued[] / waited[] are kept by thread 0 for the timeout path.
// S64: the state between time steps is FP64 (X.Q0d, interior nodes): the
// update adds the FP32 increment to it in FP64, stages 1-4 round their
// output to FP32 (it feeds only the FP32 flux evaluation), and stage 5 writes
// both the FP64 state and its FP32 copy (the next step's flux input).
template <typename R, typename MT, int TI, int TJ, bool S64, int MD>
__device__ __forceinline__ void stage_item(const StageCtx<R, MT>& X, const StageSel& st, int bx, int by, int bz,
                                           unsigned char* smem, uint32_t ph[3], int issued[3], int waited[3],
                                           bool& failed) {
  using C = Cfg<R, MT, TI, TJ>;
  constexpr int RW = C::RW, PL = C::PL, NTILE = C::NTILE;
  R* raw[2] = {reinterpret_cast<R*>(smem + C::O_RAW0), reinterpret_cast<R*>(smem + C::O_RAW1)};
  MT* met = reinterpret_cast<MT*>(smem + C::O_MET);
  R* ring = reinterpret_cast<R*>(smem + C::O_RING);
  R* Gi = reinterpret_cast<R*>(smem + C::O_GI);
  R* Gj = reinterpret_cast<R*>(smem + C::O_GJ);
  R* Li = reinterpret_cast<R*>(smem + C::O_LI);
  R* Lj = reinterpret_cast<R*>(smem + C::O_LJ);
  R* Hi = reinterpret_cast<R*>(smem + C::O_HI);
  R* Hj = reinterpret_cast<R*>(smem + C::O_HJ);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::O_BAR);  // [0],[1]: raw buffers, [2]: metrics

  const Layout& L = X.L;
  const KConst<R> c = X.k;
  const int tid = threadIdx.x;
  const int i0 = bx * TI, j0 = by * TJ;  // tile origin (node indices)
  const int t0 = L.lo[2] + bz * X.kc;
  const int t1 = min(t0 + X.kc, L.hi[2] + 1);
  const int pbase = t0 - 2;  // first staged plane
  const uint32_t xtx = st.stall ? kStallBytes : 0u;
  const long long wlim = st.stall ? kStallLimit : kWaitLimit;

  // node-pass role of this thread: tile node, j-halo node or i-halo node
  int nx, ny, role;
  if (tid < NTILE) { role = 0; nx = tid % TI; ny = tid / TI; }
  else if (tid < NTILE + C::NJH) { role = 2; const int h = tid - NTILE; nx = h % TI; ny = (h / TI) ? TJ : -1; }
  else { role = 1; const int h = tid - NTILE - C::NJH; ny = h % TJ; nx = (h / TJ) ? TI : -1; }
  const int gi = i0 + nx, gj = j0 + ny;
  const bool own = role == 0 && gi >= L.lo[0] && gi <= L.hi[0] && gj >= L.lo[1] && gj <= L.hi[1];

  // staged plane p goes to raw buffer (p - pbase) & 1; every barrier has at
  // most one load in flight, so the parity to wait for is its count of
  // completed phases ph[b] (kept identically by all threads) mod 2
  auto issue_raw = [&](int p) {
    if (tid == 0) {
      const int b = (p - pbase) & 1;
      ++issued[b];
      fence_async_shared();
      mbar_expect_tx(&bar[b], C::RAW_TX + xtx);
      tma_load_4d(raw[b], &X.tmQ[st.qin], &bar[b], i0, j0, p + NG, 0);
    }
  };
  auto issue_met = [&](int p) {
    if (tid == 0) {
      ++issued[2];
      fence_async_shared();
      mbar_expect_tx(&bar[2], C::MET_TX + xtx);
      tma_load_4d(met, &X.tmM, &bar[2], i0, j0, p + NG, 0);
    }
  };
  // on a bounded-wait timeout, the first failing CTA records where it gave up
  auto record = [&](int b, int parity, int p) {
    if (atomicCAS(X.err, 0, 1) == 0) {
      int* info = X.err + 1;
      info[0] = b; info[1] = parity; info[2] = p; info[3] = bx; info[4] = by; info[5] = bz; info[6] = st.qin;
    }
  };
  auto wait_bar = [&](int b) {
    const bool ok = mbar_wait_bounded(&bar[b], ph[b] & 1, wlim);
    if (!ok && tid == 0) record(b, ph[b] & 1, -100);
    ++ph[b];
    if (ok && tid == 0) ++waited[b];
    return __syncthreads_or(!ok) == 0;
  };
  // convert staged plane p into ring slot p & 3
  auto convert = [&](int p) {
    const R* rq = raw[(p - pbase) & 1];
    R* dst = ring + ((p + 8) & 3) * NV * PL;
    for (int e = tid; e < PL; e += C::NT) {
      const R q0 = rq[e], q1 = rq[PL + e], q2 = rq[2 * PL + e], q3 = rq[3 * PL + e], q4 = rq[4 * PL + e];
      const R ri = Fn<R>::rcp(q0);
      const R u = q1 * ri, v = q2 * ri, w = q3 * ri;
      const R pr = c.gm1 * (q4 - R(0.5) * q0 * (u * u + v * v + w * w));
      dst[V_RHO * PL + e] = q0;
      dst[V_U * PL + e] = u;
      dst[V_V * PL + e] = v;
      dst[V_W * PL + e] = w;
      dst[V_E * PL + e] = q4;
      dst[V_P * PL + e] = pr;
      dst[V_T * PL + e] = c.gamma * pr * ri;
    }
  };
  // wait for staged plane p (and, when with_met, the metrics of plane
  // met_plane) with one barrier, convert plane p, then stage plane p + 2
  auto fetch_plane = [&](int p, bool with_met, int met_plane) {
    const int b = (p - pbase) & 1;
    bool ok = mbar_wait_bounded(&bar[b], ph[b] & 1, wlim);
    if (!ok && tid == 0) record(b, ph[b] & 1, p);
    ++ph[b];
    if (ok && tid == 0) ++waited[b];
    if (with_met) {
      const bool okm = ok && mbar_wait_bounded(&bar[2], ph[2] & 1, wlim);
      if (ok && !okm && tid == 0) record(2, ph[2] & 1, met_plane);
      ++ph[2];
      if (okm && tid == 0) ++waited[2];
      ok = okm;
    }
    if (__syncthreads_or(!ok)) return false;
    convert(p);
    __syncthreads();  // raw buffer b consumed, ring slot of p written
    if (p + 2 <= t1 + 1) issue_raw(p + 2);
    return true;
  };

  // node pass for plane kk: stores i/j node data to shared memory, returns
  // the k-direction data (tile threads) in registers
  auto node_pass = [&](int kk, R G3[5], R& lt3, R& nu3, R& Jn) {
    const int sM = (kk + 7) & 3, sC = (kk + 8) & 3, sP = (kk + 9) & 3;
    R G[3][5], lt[3], nu[3];
    if (role == 0) {
      node_flux<R, MT, RW, PL, 0, MD>(ring, met, sM, sC, sP, nx, ny, c, G, lt, nu, Jn);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Gi[(v * TJ + ny) * (TI + 2) + nx + 1] = G[0][v];
        Gj[(v * (TJ + 2) + ny + 1) * TI + nx] = G[1][v];
        G3[v] = G[2][v];
      }
      Li[(0 * TJ + ny) * (TI + 2) + nx + 1] = lt[0];
      Li[(1 * TJ + ny) * (TI + 2) + nx + 1] = nu[0];
      Lj[(0 * (TJ + 2) + ny + 1) * TI + nx] = lt[1];
      Lj[(1 * (TJ + 2) + ny + 1) * TI + nx] = nu[1];
      lt3 = lt[2];
      nu3 = nu[2];
    } else if (role == 1) {
      R Jh;
      node_flux<R, MT, RW, PL, 1, MD>(ring, met, sM, sC, sP, nx, ny, c, G, lt, nu, Jh);
      const int col = nx + 1;
#pragma unroll
      for (int v = 0; v < 5; ++v) Gi[(v * TJ + ny) * (TI + 2) + col] = G[0][v];
      Li[(0 * TJ + ny) * (TI + 2) + col] = lt[0];
      Li[(1 * TJ + ny) * (TI + 2) + col] = nu[0];
    } else {
      R Jh;
      node_flux<R, MT, RW, PL, 2, MD>(ring, met, sM, sC, sP, nx, ny, c, G, lt, nu, Jh);
      const int row = ny + 1;
#pragma unroll
      for (int v = 0; v < 5; ++v) Gj[(v * (TJ + 2) + row) * TI + nx] = G[1][v];
      Lj[(0 * (TJ + 2) + row) * TI + nx] = lt[1];
      Lj[(1 * (TJ + 2) + row) * TI + nx] = nu[1];
    }
  };

  // i/j face fluxes of plane kk, then the i/j residual part of tile nodes
  auto face_pass = [&](int kk, R Rij[5]) {
    const int s = (kk + 8) & 3;
    auto iface = [&](int x, int y) {  // face between x-1 and x in row y
      R lam, e2, e4, Ga[5], Gb[5], h[5];
      face_coeffs<R>(c, Li[(0 * TJ + y) * (TI + 2) + x], Li[(0 * TJ + y) * (TI + 2) + x + 1],
                     Li[(1 * TJ + y) * (TI + 2) + x], Li[(1 * TJ + y) * (TI + 2) + x + 1], lam, e2, e4);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Ga[v] = Gi[(v * TJ + y) * (TI + 2) + x];
        Gb[v] = Gi[(v * TJ + y) * (TI + 2) + x + 1];
      }
      const int base = (y + 2) * RW + x;  // ring column of node x-2
      const int so[4] = {s, s, s, s}, oo[4] = {base, base + 1, base + 2, base + 3};
      face5<R, PL>(ring, so, oo, Ga, Gb, lam, e2, e4, h);
#pragma unroll
      for (int v = 0; v < 5; ++v) Hi[(v * TJ + y) * (TI + 1) + x] = h[v];
    };
    auto jface = [&](int x, int y) {  // face between y-1 and y in column x
      R lam, e2, e4, Ga[5], Gb[5], h[5];
      face_coeffs<R>(c, Lj[(0 * (TJ + 2) + y) * TI + x], Lj[(0 * (TJ + 2) + y + 1) * TI + x],
                     Lj[(1 * (TJ + 2) + y) * TI + x], Lj[(1 * (TJ + 2) + y + 1) * TI + x], lam, e2, e4);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Ga[v] = Gj[(v * (TJ + 2) + y) * TI + x];
        Gb[v] = Gj[(v * (TJ + 2) + y + 1) * TI + x];
      }
      const int base = y * RW + x + 2;  // ring row of node y-2
      const int so[4] = {s, s, s, s}, oo[4] = {base, base + RW, base + 2 * RW, base + 3 * RW};
      face5<R, PL>(ring, so, oo, Ga, Gb, lam, e2, e4, h);
#pragma unroll
      for (int v = 0; v < 5; ++v) Hj[(v * (TJ + 1) + y) * TI + x] = h[v];
    };
    if (role == 0) {
      iface(nx, ny);
      jface(nx, ny);
    } else {
      const int h = tid - NTILE;  // the last i-face of each row and j-face of each column
      if (h < TJ) iface(TI, h);
      else if (h < TJ + TI) jface(h - TJ, TJ);
    }
    __syncthreads();
    if (role == 0) {
#pragma unroll
      for (int v = 0; v < 5; ++v)
        Rij[v] = (Hi[(v * TJ + ny) * (TI + 1) + nx + 1] - Hi[(v * TJ + ny) * (TI + 1) + nx]) +
                 (Hj[(v * (TJ + 1) + ny + 1) * TI + nx] - Hj[(v * (TJ + 1) + ny) * TI + nx]);
    }
  };

  // k face flux between planes ka and ka+1 of this thread's column
  auto kface = [&](int ka, const R Ga[5], const R Gb[5], R lta, R ltb, R nua, R nub, R h[5]) {
    R lam, e2, e4;
    face_coeffs<R>(c, lta, ltb, nua, nub, lam, e2, e4);
    const int o = (ny + 2) * RW + nx + 2;
    const int so[4] = {(ka + 7) & 3, (ka + 8) & 3, (ka + 9) & 3, (ka + 10) & 3}, oo[4] = {o, o, o, o};
    face5<R, PL>(ring, so, oo, Ga, Gb, lam, e2, e4, h);
  };

  const R adt = (R)(st.alpha * X.sc->dt);
  const long long npad = L.npad;
  R* const Qo = X.Q[st.qout];

  // ---- prologue: stage planes t0-2 .. t0+1 and the metrics of t0-1
  issue_raw(t0 - 2);
  issue_raw(t0 - 1);
  issue_met(t0 - 1);
  R G3m[5], lt3m = 0, nu3m = 0, Jm = 0;
  R G3c[5], lt3c = 0, nu3c = 0, Jc = 0;
  R Rc[5], hprev[5];
  if (!fetch_plane(t0 - 2, false, 0) || !fetch_plane(t0 - 1, false, 0) || !fetch_plane(t0, false, 0) ||
      !fetch_plane(t0 + 1, true, t0 - 1)) {
    failed = true;
  } else {
    node_pass(t0 - 1, G3m, lt3m, nu3m, Jm);
    __syncthreads();  // metrics buffer and node buffers consumed
    issue_met(t0);
    if (!wait_bar(2)) {
      failed = true;
    } else {
      node_pass(t0, G3c, lt3c, nu3c, Jc);
      __syncthreads();
      issue_met(t0 + 1);
      face_pass(t0, Rc);
      if (role == 0) kface(t0 - 1, G3m, G3c, lt3m, lt3c, nu3m, nu3c, hprev);
    }
  }

  // ---- march in k
  for (int t = t0; t < t1 && !failed; ++t) {
    R q0[5];
    double q0d[5];
    long long n = 0;
    if (own) {
      n = L.at(gi, gj, t);
      if constexpr (S64) {
#pragma unroll
        for (int v = 0; v < 5; ++v) q0d[v] = X.Q0d[v * npad + n];
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) q0[v] = X.Q[0][v * npad + n];
      }
    }
    // the barrier inside fetch_plane also orders the previous iteration's
    // reads of ring slot t-2 and of the face buffers before they are rewritten
    if (!fetch_plane(t + 2, true, t + 1)) { failed = true; break; }
    R G3n[5], lt3n = 0, nu3n = 0, Jn = 0;
    node_pass(t + 1, G3n, lt3n, nu3n, Jn);
    __syncthreads();
    if (t + 2 <= t1) issue_met(t + 2);
    R Rn[5];
    face_pass(t + 1, Rn);
    if (role == 0) {
      R hk[5];
      kface(t, G3c, G3n, lt3c, lt3n, nu3c, nu3n, hk);
      if (own) {
        if constexpr (S64) {
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            const double qn = q0d[v] - (double)(adt * Jc * (Rc[v] + (hk[v] - hprev[v])));
            Qo[v * npad + n] = (R)qn;
            if (st.qout == 0) X.Q0d[v * npad + n] = qn;
          }
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) Qo[v * npad + n] = q0[v] - adt * Jc * (Rc[v] + (hk[v] - hprev[v]));
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        G3c[v] = G3n[v];
        Rc[v] = Rn[v];
        hprev[v] = hk[v];
      }
      lt3c = lt3n;
      nu3c = nu3n;
      Jc = Jn;
    }
  }

}

// One grid: one CTA per (tile, k-chunk).  MD: the flow model (constant
// flags, or read at run time).
template <typename R, typename MT, int TI, int TJ, bool S64, int MD>
__global__ void __launch_bounds__(Cfg<R, MT, TI, TJ>::NT, Cfg<R, MT, TI, TJ>::MINB)
    k_stage(const __grid_constant__ StageCtx<R, MT> X, const StageSel st) {
  using C = Cfg<R, MT, TI, TJ>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::O_BAR);
  init_barriers(bar);
  uint32_t ph[3] = {0, 0, 0};
  int issued[3] = {0, 0, 0}, waited[3] = {0, 0, 0};
  bool failed = false;
  stage_item<R, MT, TI, TJ, S64, MD>(X, st, blockIdx.x, blockIdx.y, blockIdx.z, smem, ph, issued, waited, failed);
  if (failed) drain_after_timeout(bar, X.err, issued, waited, st.stall ? kStallBytes : 0u);
}

// Many grids: persistent CTAs (one per SM) take work items (grid, tile,
// k-chunk) from a device queue, largest first.
// MD: the flow model every grid of the batch shares (kModelSmagorinsky), or
// kMixedModels: each work item in the build of its own grid's model, as
// when the grid is stepped alone.
constexpr int kMixedModels = -1;
template <typename R, typename MT, int TI, int TJ, bool S64, int MD>
__global__ void __launch_bounds__(Cfg<R, MT, TI, TJ>::NT, Cfg<R, MT, TI, TJ>::MINB)
    k_stage_batch(const StageCtx<R, MT>* __restrict__ ctx, const int4* __restrict__ items, int nitems,
                  unsigned int* queue, const StageSel st) {
  using C = Cfg<R, MT, TI, TJ>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::O_BAR);
  __shared__ int next;
  init_barriers(bar);
  uint32_t ph[3] = {0, 0, 0};
  int issued[3] = {0, 0, 0}, waited[3] = {0, 0, 0};
  bool failed = false;
  int gsel = 0;
  for (;;) {
    if (threadIdx.x == 0) next = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int it = next;
    __syncthreads();
    if (it >= nitems) break;
    const int4 w = items[it];
    gsel = w.x;
    if (MD == kModelSmagorinsky || (MD == kMixedModels && flow_model(ctx[w.x].k) == kModelSmagorinsky))
      stage_item<R, MT, TI, TJ, S64, kModelSmagorinsky>(ctx[w.x], st, w.y, w.z, w.w, smem, ph, issued, waited, failed);
    else
      stage_item<R, MT, TI, TJ, S64, kModelRuntime>(ctx[w.x], st, w.y, w.z, w.w, smem, ph, issued, waited, failed);
    if (failed) break;
  }
  if (failed) drain_after_timeout(bar, ctx[gsel].err, issued, waited, st.stall ? kStallBytes : 0u);
}

// tile shapes per precision (one CTA per SM)
// (a 32 x 8 FP32 tile with two CTAs per SM measured slower: the larger halo
// share outweighs the overlap of the two CTAs' barriers)
constexpr int TI32 = 32, TJ32 = 16;  // P32: 608 threads, 191 KB: one CTA per SM
constexpr int TIM = 32, TJM = 16;    // P32_M64: 608 threads, 220 KB (FP64 metric staging): one CTA per SM
constexpr int TI64 = 16, TJ64 = 16;  // FP64: 320 threads, 207 KB

// The scalar kernels are built for two flow models: the configurations'
// (Smagorinsky, sigma = 1/2) with constant flags, and every other with the
// flags read at run time.  The two builds may fuse a multiplication into an
// addition differently, so a batch of grids that do not all take the
// Smagorinsky build runs every grid in the build of its own model (both are
// inlined into that kernel): a grid's state is bitwise the one it reaches
// alone.
template <typename R, typename MT, int TI, int TJ, bool S64 = false>
cudaError_t configure_one() {
  const int bytes = (int)Cfg<R, MT, TI, TJ>::BYTES;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_stage<R, MT, TI, TJ, S64, kModelRuntime>, a, bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_stage<R, MT, TI, TJ, S64, kModelSmagorinsky>, a, bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_stage_batch<R, MT, TI, TJ, S64, kModelSmagorinsky>, a, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_stage_batch<R, MT, TI, TJ, S64, kMixedModels>, a, bytes);
}


template <typename R, typename MT>
void fill_ctx(StageCtx<R, MT>& X, const GridDev& g) {
  X.tmQ[0] = g.tmQ[0];
  X.tmQ[1] = g.tmQ[1];
  X.tmQ[2] = g.tmQ[2];
  X.tmM = g.tmM;
  X.tmMv = g.tmMv;
  X.tmQ0u = g.tmQ0u;
  X.L = g.L;
  X.Q[0] = (R*)g.Q0;
  X.Q[1] = (R*)g.QA;
  X.Q[2] = (R*)g.QB;
  X.Q0d = (double*)g.Q0d;
  X.sc = g.sc;
  X.err = &g.sc->err;
  X.F = g.F;
  X.k = make_kconst<R>(g.F);
  X.kc = g.kc;
}

template <typename R, typename MT, int TI, int TJ, bool S64 = false>
cudaError_t launch_one(const GridDev& g, int stage, int qsel, int qout, cudaStream_t s) {
  using Cf = Cfg<R, MT, TI, TJ>;
  StageCtx<R, MT> X;
  fill_ctx(X, g);
  const StageSel st{kRkAlpha[stage], qsel, qout, g.stall_test};
  const int nz = g.L.hi[2] - g.L.lo[2] + 1;
  dim3 grid((g.L.hi[0] + TI) / TI, (g.L.hi[1] + TJ) / TJ, (nz + g.kc - 1) / g.kc);
  if (flow_model(X.k) == kModelSmagorinsky)
    k_stage<R, MT, TI, TJ, S64, kModelSmagorinsky><<<grid, Cf::NT, Cf::BYTES, s>>>(X, st);
  else
    k_stage<R, MT, TI, TJ, S64, kModelRuntime><<<grid, Cf::NT, Cf::BYTES, s>>>(X, st);
  count_launches(1);
  return cudaGetLastError();
}

template <typename R, typename MT, int TI, int TJ, bool S64 = false>
cudaError_t launch_batch(const void* ctx, const int4* items, int nitems, unsigned int* queue, int stage, int qsel,
                         int qout, int model, cudaStream_t s) {
  using Cf = Cfg<R, MT, TI, TJ>;
  const StageSel st{kRkAlpha[stage], qsel, qout, 0};
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  const int slots = device_sm_count() * Cf::MINB;
  const int ctas = nitems < slots ? nitems : slots;
  const auto* X = (const StageCtx<R, MT>*)ctx;
  if (model == kModelSmagorinsky)
    k_stage_batch<R, MT, TI, TJ, S64, kModelSmagorinsky><<<ctas, Cf::NT, Cf::BYTES, s>>>(X, items, nitems, queue, st);
  else
    k_stage_batch<R, MT, TI, TJ, S64, kMixedModels><<<ctas, Cf::NT, Cf::BYTES, s>>>(X, items, nitems, queue, st);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

int stage_ctas_per_sm(int prec) {
  switch (prec) {
    case JZ_P64: return Cfg<double, double, TI64, TJ64>::MINB;
    case JZ_P32_M64: return Cfg<float, double, TIM, TJM>::MINB;
    default: return Cfg<float, float, TI32, TJ32>::MINB;
  }
}

int grid_ctas_per_sm(const GridDev& g) {
  if (g.prec == JZ_P32 && g.variant == 2) return vr_ctas_per_sm(g.vti, g.vtj);
  return stage_ctas_per_sm(g.prec);
}

StageTiling stage_tiling(int prec) {
  if (prec == JZ_P64) return {TI64, TJ64};
  if (prec == JZ_P32_M64) return {TIM, TJM};
  return {TI32, TJ32};
}

cudaError_t stage_configure() {
  cudaError_t e;
  if ((e = configure_one<double, double, TI64, TJ64>()) != cudaSuccess) return e;
  if ((e = configure_one<float, double, TIM, TJM>()) != cudaSuccess) return e;
  if ((e = configure_one<float, float, TI32, TJ32>()) != cudaSuccess) return e;
  if ((e = configure_one<float, float, TI32, TJ32, true>()) != cudaSuccess) return e;
  if ((e = stage_v_configure_32x16()) != cudaSuccess) return e;
  if ((e = stage_v_configure_16x32()) != cudaSuccess) return e;
  if ((e = stage_v_configure_16x16()) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_stage(const GridDev& g, int stage, int qsel, int qout, cudaStream_t s) {
  switch (g.prec) {
    case JZ_P64: return launch_one<double, double, TI64, TJ64>(g, stage, qsel, qout, s);
    case JZ_P32_M64: return launch_one<float, double, TIM, TJM>(g, stage, qsel, qout, s);
    case JZ_P32_S64: return launch_one<float, float, TI32, TJ32, true>(g, stage, qsel, qout, s);
    default:
      if (g.variant == 2) {
        StageCtx<float, float> X;
        fill_ctx(X, g);
        const StageSel st{kRkAlpha[stage], qsel, qout, g.stall_test};
        if (g.vti == 16 && g.vtj == 32) return launch_stage_v_16x32(X, st, s);
        if (g.vti == 16 && g.vtj == 16) return launch_stage_v_16x16(X, st, s);
        return launch_stage_v_32x16(X, st, s);
      }
      return launch_one<float, float, TI32, TJ32>(g, stage, qsel, qout, s);
  }
}

size_t stage_ctx_bytes(int prec) {
  switch (prec) {
    case JZ_P64: return sizeof(StageCtx<double, double>);
    case JZ_P32_M64: return sizeof(StageCtx<float, double>);
    default: return sizeof(StageCtx<float, float>);
  }
}

void stage_ctx_fill(void* dst, const GridDev& g) {
  switch (g.prec) {
    case JZ_P64: fill_ctx(*(StageCtx<double, double>*)dst, g); break;
    case JZ_P32_M64: fill_ctx(*(StageCtx<float, double>*)dst, g); break;
    default: fill_ctx(*(StageCtx<float, float>*)dst, g); break;
  }
}

int stage_model(const GridDev& g) { return flow_model(make_kconst<float>(g.F)); }

cudaError_t launch_stage_batch(int prec, int variant, StageTiling tile, const void* ctx, const int4* items,
                               int nitems, unsigned int* queue, int stage, int qsel, int qout, int model,
                               cudaStream_t s) {
  if (prec == JZ_P32 && variant == 2) {
    const StageSel st{kRkAlpha[stage], qsel, qout, 0};
    if (tile.ti == 16 && tile.tj == 32) return launch_stage_v_batch_16x32(ctx, items, nitems, queue, st, model, s);
    if (tile.ti == 16 && tile.tj == 16) return launch_stage_v_batch_16x16(ctx, items, nitems, queue, st, model, s);
    return launch_stage_v_batch_32x16(ctx, items, nitems, queue, st, model, s);
  }
  switch (prec) {
    case JZ_P64: return launch_batch<double, double, TI64, TJ64>(ctx, items, nitems, queue, stage, qsel, qout, model, s);
    case JZ_P32_M64:
      return launch_batch<float, double, TIM, TJM>(ctx, items, nitems, queue, stage, qsel, qout, model, s);
    case JZ_P32_S64:
      return launch_batch<float, float, TI32, TJ32, true>(ctx, items, nitems, queue, stage, qsel, qout, model, s);
    default: return launch_batch<float, float, TI32, TJ32>(ctx, items, nitems, queue, stage, qsel, qout, model, s);
  }
}

}  // namespace jz
