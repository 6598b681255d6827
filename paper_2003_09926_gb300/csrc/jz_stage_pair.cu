// jz_stage_pair.cu -- the fused Runge-Kutta stage kernel for FP32 state and
// FP32 metrics, with paired nodes and packed FP32x2 arithmetic.
//
// Same method and same per-plane pipeline as the scalar kernel in
// jz_stage.cu (arXiv 2003.09926, Section 3 and Section 4.2: inviscid flux,
// Turkel-Vatsa dissipation, viscous flux with Smagorinsky SGS, 5-stage
// update; residual in face form), organised for Blackwell's packed FP32x2
// instructions (FFMA2 / FMUL2 / FADD2):
//  - a tile thread owns two nodes of the same column eight rows apart,
//    (x, y) and (x, y + 8), of a 32 x 16 tile, and computes both at once in
//    float2 arithmetic;
//  - the shared-memory ring, node-flux and face arrays hold node pairs in
//    that row pairing (a "pair row" yp holds rows yp and yp + 8), so a pair's
//    neighbours are one 64-bit load away;
//  - 304 threads: 256 tile pairs, 16 i-halo pairs (columns -1 and 32), 32
//    j-halo threads (each the two nodes of rows -1 and 16 of a column, read
//    with two 32-bit loads);
//  - TMA staging of raw state planes and metric planes, bounded mbarrier
//    waits, k-chunking and work items exactly as in the scalar kernel.
#include <cmath>
#include <cstdint>

#include "jz_stage_common.cuh"

namespace jz {

using namespace stg;

namespace {

// ---------------------------------------------------------------------------
// geometry and shared-memory layout
// ---------------------------------------------------------------------------

constexpr size_t al128(size_t x) { return (x + 127) / 128 * 128; }

struct PG {
  static constexpr int TI = 32, TJ = 16, D = 8;           // tile, pair offset
  static constexpr int RW = TI + 4, RH = TJ + 4, PL = RW * RH;  // staged plane (natural rows)
  static constexpr int PR = D + 4, PPL = PR * RW;         // pair rows -2 .. D+1
  static constexpr int NTP = TI * D;                      // tile pair threads
  static constexpr int NIH = 2 * D;                       // i-halo pair threads
  static constexpr int NJH = TI;                          // j-halo threads
  static constexpr int NT = NTP + NIH + NJH;              // 304
  static constexpr size_t RAW_B = al128(4 * 5 * PL);
  static constexpr size_t MET_B = al128(4 * 10 * PL);
  static constexpr size_t RING_B = al128(8 * 4 * NV * PPL);
  static constexpr size_t GI_B = al128(8 * 5 * D * (TI + 2));      // i node fluxes, columns -1..TI
  static constexpr size_t LI_B = al128(8 * 2 * D * (TI + 2));
  static constexpr size_t GJ_B = al128(8 * 5 * (D + 2) * TI);      // j node fluxes, pair rows -1..D
  static constexpr size_t LJ_B = al128(8 * 2 * (D + 2) * TI);
  static constexpr size_t HI_B = al128(8 * 5 * D * (TI + 1));      // i faces x - 1/2, x = 0..TI
  static constexpr size_t HJ_B = al128(8 * 5 * (D + 1) * TI);      // j pair faces yf = 0..D
  static constexpr size_t O_RAW0 = 0, O_RAW1 = O_RAW0 + RAW_B, O_MET = O_RAW1 + RAW_B, O_RING = O_MET + MET_B;
  static constexpr size_t O_GI = O_RING + RING_B, O_LI = O_GI + GI_B, O_GJ = O_LI + LI_B, O_LJ = O_GJ + GJ_B;
  static constexpr size_t O_HI = O_LJ + LJ_B, O_HJ = O_HI + HI_B, O_BAR = O_HJ + HJ_B;
  static constexpr size_t BYTES = O_BAR + 128;
  static constexpr uint32_t RAW_TX = 4 * 5 * PL, MET_TX = 4 * 10 * PL;
};

// node-flux input accessor: value of (slot, var) at offset (dy, dx) from the
// pair's node(s).  Tile and i-halo pairs read one float2 of the pair ring;
// j-halo threads combine row -1 (x of pair row -1) and row TJ (y of pair row D).
struct PairAcc {
  const f2* ring;
  int o;  // pair-ring offset of the node pair within a plane
  __device__ __forceinline__ f2 operator()(int slot, int var, int dy, int dx) const {
    return ring[(slot * NV + var) * PG::PPL + o + dy * PG::RW + dx];
  }
};
struct SplitAcc {
  const float* ring;  // the pair ring viewed as floats
  int ox, oy;         // pair-ring offsets of the row -1 and row TJ nodes
  __device__ __forceinline__ f2 operator()(int slot, int var, int dy, int dx) const {
    const int b = (slot * NV + var) * PG::PPL + dy * PG::RW + dx;
    return f2(ring[2 * (b + ox)], ring[2 * (b + oy) + 1]);
  }
};

// G^k = E^k - F^k, lambda~^k, nu^k of a node pair (DIR 0: all directions,
// 1 / 2: i / j only).  Same formulas as the scalar node_flux.
template <int DIR, typename Acc>
__device__ __forceinline__ void node_flux_pair(const Acc at, int sM, int sC, int sP, const f2 S[9], f2 Jn,
                                               const KConst<float>& c, f2 G[3][5], f2 lt[3], f2 nu[3]) {
  const f2 rho = at(sC, V_RHO, 0, 0);
  const f2 u = at(sC, V_U, 0, 0), v = at(sC, V_V, 0, 0), w = at(sC, V_W, 0, 0);
  const f2 e = at(sC, V_E, 0, 0), p = at(sC, V_P, 0, 0), T = at(sC, V_T, 0, 0);
  constexpr int K0 = DIR == 0 ? 0 : DIR - 1;
  constexpr int K1 = DIR == 0 ? 3 : DIR;
  f2 Fv[3][4];
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q) Fv[m][q] = f2(0.f);
  if (c.viscous) {
    const int var[4] = {V_U, V_V, V_W, V_T};
    f2 g[4][3];
    const f2 hJ = f2(0.5f) * Jn;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const f2 d0 = at(sC, var[q], 0, 1) - at(sC, var[q], 0, -1);
      const f2 d1 = at(sC, var[q], 1, 0) - at(sC, var[q], -1, 0);
      const f2 d2 = at(sP, var[q], 0, 0) - at(sM, var[q], 0, 0);
#pragma unroll
      for (int m = 0; m < 3; ++m) g[q][m] = hJ * fma2(S[m], d0, fma2(S[3 + m], d1, S[6 + m] * d2));
    }
    const f2 mu = c.mu_inf * T * sqrt2(T) * f2(c.s1p1) * rcp2(T + f2(c.s1));
    f2 mu_t = f2(0.f);
    if (c.sgs) {
      const f2 s12 = f2(0.5f) * (g[0][1] + g[1][0]), s13 = f2(0.5f) * (g[0][2] + g[2][0]);
      const f2 s23 = f2(0.5f) * (g[1][2] + g[2][1]);
      f2 ss = fma2(g[0][0], g[0][0], fma2(g[1][1], g[1][1], g[2][2] * g[2][2]));
      ss = fma2(f2(2.f), fma2(s12, s12, fma2(s13, s13, s23 * s23)), ss);
      mu_t = rho * f2(c.cs2) * sqrt2(f2(2.f) * ss) * jm23_2(Jn);
    }
    const f2 mue = mu + mu_t;
    const f2 kap = f2(c.cp) * fma2(mu, f2(c.inv_pr), mu_t * f2(c.inv_prt));
    const f2 div3 = (g[0][0] + g[1][1] + g[2][2]) * f2(2.0f / 3.0f);
    const f2 t01 = mue * (g[0][1] + g[1][0]), t02 = mue * (g[0][2] + g[2][0]), t12 = mue * (g[1][2] + g[2][1]);
    Fv[0][0] = mue * fma2(f2(2.f), g[0][0], f2(0.f) - div3); Fv[0][1] = t01; Fv[0][2] = t02;
    Fv[1][0] = t01; Fv[1][1] = mue * fma2(f2(2.f), g[1][1], f2(0.f) - div3); Fv[1][2] = t12;
    Fv[2][0] = t02; Fv[2][1] = t12; Fv[2][2] = mue * fma2(f2(2.f), g[2][2], f2(0.f) - div3);
#pragma unroll
    for (int m = 0; m < 3; ++m) Fv[m][3] = fma2(u, Fv[m][0], fma2(v, Fv[m][1], fma2(w, Fv[m][2], kap * g[3][m])));
  }
  f2 lam[3], U[3];
  const f2 cson = sqrt2(T);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    U[k] = fma2(S[3 * k], u, fma2(S[3 * k + 1], v, S[3 * k + 2] * w));
    const f2 sn = sqrt2(fma2(S[3 * k], S[3 * k], fma2(S[3 * k + 1], S[3 * k + 1], S[3 * k + 2] * S[3 * k + 2])));
    lam[k] = fma2(cson, sn, abs2(U[k]));
  }
  f2 sq[3] = {f2(0.f), f2(0.f), f2(0.f)};
  if (c.sig_half) {
#pragma unroll
    for (int k = 0; k < 3; ++k) sq[k] = sqrt2(lam[k]);
  }
  const f2 m1 = rho * u, m2 = rho * v, m3 = rho * w, ep = e + p;
#pragma unroll
  for (int k = K0; k < K1; ++k) {
    const f2 Sx = S[3 * k], Sy = S[3 * k + 1], Sz = S[3 * k + 2];
    f2 Fk[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) Fk[q] = fma2(Sx, Fv[0][q], fma2(Sy, Fv[1][q], Sz * Fv[2][q]));
    G[k][0] = rho * U[k];
    G[k][1] = fma2(m1, U[k], fma2(Sx, p, f2(0.f) - Fk[0]));
    G[k][2] = fma2(m2, U[k], fma2(Sy, p, f2(0.f) - Fk[1]));
    G[k][3] = fma2(m3, U[k], fma2(Sz, p, f2(0.f) - Fk[2]));
    G[k][4] = fma2(ep, U[k], f2(0.f) - Fk[3]);
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    if (c.sig_half)
      lt[k] = fma2(sq[k], sq[a] + sq[b], lam[k]);
    else
      lt[k] = lam[k] * (f2(1.f) + pow2(lam[a] * rcp2(lam[k]), c.sigma) + pow2(lam[b] * rcp2(lam[k]), c.sigma));
    f2 pm, pp;
    if (k == 0) { pm = at(sC, V_P, 0, -1); pp = at(sC, V_P, 0, 1); }
    else if (k == 1) { pm = at(sC, V_P, -1, 0); pp = at(sC, V_P, 1, 0); }
    else { pm = at(sM, V_P, 0, 0); pp = at(sP, V_P, 0, 0); }
    nu[k] = abs2(fma2(f2(-2.f), p, pp + pm)) * rcp2(fma2(f2(2.f), p, pp + pm));
  }
}

// face flux h = (Ga + Gb)/2 - lam [eps2 (qb - qa) - eps4 (qbp - 3 qb + 3 qa - qam)]
__device__ __forceinline__ f2 face_h2(f2 Ga, f2 Gb, f2 qam, f2 qa, f2 qb, f2 qbp, f2 lam, f2 e2, f2 e4) {
  const f2 d1 = qb - qa;
  const f2 d3 = fma2(f2(3.f), qa - qb, qbp - qam);
  return fma2(f2(0.5f), Ga + Gb, f2(0.f) - lam * (e2 * d1 - e4 * d3));
}

__device__ __forceinline__ void face_coeffs2(const KConst<float>& c, f2 lta, f2 ltb, f2 nua, f2 nub, f2& lam, f2& e2,
                                             f2& e4) {
  lam = f2(0.5f) * (lta + ltb);
  e2 = f2(c.k2) * max2(nua, nub);
  e4 = max2(f2(0.f), f2(c.k4) - e2);
}

// the five face fluxes of a pair line from four pair-ring offsets
__device__ __forceinline__ void face5_pair(const f2* ring, const int so[4], const int oo[4], const f2 Ga[5],
                                           const f2 Gb[5], f2 lam, f2 e2, f2 e4, f2 h[5]) {
  f2 rho[4], q[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) rho[n] = ring[(so[n] * NV + V_RHO) * PG::PPL + oo[n]];
  h[0] = face_h2(Ga[0], Gb[0], rho[0], rho[1], rho[2], rho[3], lam, e2, e4);
#pragma unroll
  for (int cc = 1; cc < 4; ++cc) {
#pragma unroll
    for (int n = 0; n < 4; ++n) q[n] = rho[n] * ring[(so[n] * NV + cc) * PG::PPL + oo[n]];
    h[cc] = face_h2(Ga[cc], Gb[cc], q[0], q[1], q[2], q[3], lam, e2, e4);
  }
#pragma unroll
  for (int n = 0; n < 4; ++n) q[n] = ring[(so[n] * NV + V_E) * PG::PPL + oo[n]];
  h[4] = face_h2(Ga[4], Gb[4], q[0], q[1], q[2], q[3], lam, e2, e4);
}

// One work item (tile bx, by; k-chunk bz) of the paired kernel.
__device__ __forceinline__ void pair_item(const StageCtx<float, float>& X, const StageSel& st, int bx, int by, int bz,
                                          unsigned char* smem, uint32_t ph[3], int issued[3], int waited[3],
                                          bool& failed) {
  constexpr int TI = PG::TI, TJ = PG::TJ, D = PG::D, RW = PG::RW, PL = PG::PL, PPL = PG::PPL;
  float* raw[2] = {reinterpret_cast<float*>(smem + PG::O_RAW0), reinterpret_cast<float*>(smem + PG::O_RAW1)};
  const float* met = reinterpret_cast<const float*>(smem + PG::O_MET);
  float* metw = reinterpret_cast<float*>(smem + PG::O_MET);
  f2* ring = reinterpret_cast<f2*>(smem + PG::O_RING);
  f2* Gi = reinterpret_cast<f2*>(smem + PG::O_GI);
  f2* Li = reinterpret_cast<f2*>(smem + PG::O_LI);
  f2* Gj = reinterpret_cast<f2*>(smem + PG::O_GJ);
  f2* Lj = reinterpret_cast<f2*>(smem + PG::O_LJ);
  f2* Hi = reinterpret_cast<f2*>(smem + PG::O_HI);
  f2* Hj = reinterpret_cast<f2*>(smem + PG::O_HJ);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + PG::O_BAR);

  const Layout& L = X.L;
  const KConst<float> c = X.k;
  const int tid = threadIdx.x;
  const int i0 = bx * TI, j0 = by * TJ;
  const int t0 = L.lo[2] + bz * X.kc;
  const int t1 = min(t0 + X.kc, L.hi[2] + 1);
  const int pbase = t0 - 2;

  // roles: 0 tile pair (x, yp) -> rows yp, yp + D; 1 i-halo pair; 2 j-halo (rows -1 and TJ)
  int role, px, py;
  if (tid < PG::NTP) { role = 0; px = tid % TI; py = tid / TI; }
  else if (tid < PG::NTP + PG::NIH) { role = 1; const int h = tid - PG::NTP; px = (h / D) ? TI : -1; py = h % D; }
  else { role = 2; px = tid - PG::NTP - PG::NIH; py = -1; }
  const int gi = i0 + px;
  const int gja = j0 + py, gjb = j0 + py + D;
  const bool in_i = role == 0 && gi >= L.lo[0] && gi <= L.hi[0];
  const bool own_a = in_i && gja >= L.lo[1] && gja <= L.hi[1];
  const bool own_b = in_i && gjb >= L.lo[1] && gjb <= L.hi[1];

  auto record = [&](int b, int parity, int p) {
    if (atomicCAS(X.err, 0, 1) == 0) {
      int* info = X.err + 1;
      info[0] = b; info[1] = parity; info[2] = p; info[3] = bx; info[4] = by; info[5] = bz; info[6] = st.qin;
    }
  };
  auto issue_raw = [&](int p) {
    if (tid == 0) {
      const int b = (p - pbase) & 1;
      ++issued[b];
      fence_async_shared();
      mbar_expect_tx(&bar[b], PG::RAW_TX);
      tma_load_4d(raw[b], &X.tmQ[st.qin], &bar[b], i0, j0, p + NG, 0);
    }
  };
  auto issue_met = [&](int p) {
    if (tid == 0) {
      ++issued[2];
      fence_async_shared();
      mbar_expect_tx(&bar[2], PG::MET_TX);
      tma_load_4d(metw, &X.tmM, &bar[2], i0, j0, p + NG, 0);
    }
  };
  auto wait_bar = [&](int b) {
    const bool ok = mbar_wait_bounded(&bar[b], ph[b] & 1);
    if (!ok && tid == 0) record(b, ph[b] & 1, -100);
    ++ph[b];
    if (ok && tid == 0) ++waited[b];
    return __syncthreads_or(!ok) == 0;
  };
  // staged plane p (natural rows) -> pair ring slot p & 3
  auto convert = [&](int p) {
    const float* rq = raw[(p - pbase) & 1];
    f2* dst = ring + ((p + 8) & 3) * NV * PPL;
    for (int e = tid; e < PPL; e += PG::NT) {
      const int ya = e / RW, xi = e - ya * RW;  // pair row index (0..PR-1), column
      const int na = ya * RW + xi, nb = (ya + D) * RW + xi;
      const f2 q0(rq[na], rq[nb]), q1(rq[PL + na], rq[PL + nb]), q2(rq[2 * PL + na], rq[2 * PL + nb]);
      const f2 q3(rq[3 * PL + na], rq[3 * PL + nb]), q4(rq[4 * PL + na], rq[4 * PL + nb]);
      const f2 ri = rcp2(q0);
      const f2 u = q1 * ri, v = q2 * ri, w = q3 * ri;
      const f2 pr = f2(c.gm1) * (q4 - f2(0.5f) * q0 * fma2(u, u, fma2(v, v, w * w)));
      dst[V_RHO * PPL + e] = q0;
      dst[V_U * PPL + e] = u;
      dst[V_V * PPL + e] = v;
      dst[V_W * PPL + e] = w;
      dst[V_E * PPL + e] = q4;
      dst[V_P * PPL + e] = pr;
      dst[V_T * PPL + e] = f2(c.gamma) * pr * ri;
    }
  };
  auto fetch_plane = [&](int p, bool with_met, int met_plane) {
    const int b = (p - pbase) & 1;
    bool ok = mbar_wait_bounded(&bar[b], ph[b] & 1);
    if (!ok && tid == 0) record(b, ph[b] & 1, p);
    ++ph[b];
    if (ok && tid == 0) ++waited[b];
    if (with_met) {
      const bool okm = ok && mbar_wait_bounded(&bar[2], ph[2] & 1);
      if (ok && !okm && tid == 0) record(2, ph[2] & 1, met_plane);
      ++ph[2];
      if (okm && tid == 0) ++waited[2];
      ok = okm;
    }
    if (__syncthreads_or(!ok)) return false;
    convert(p);
    __syncthreads();
    if (p + 2 <= t1 + 1) issue_raw(p + 2);
    return true;
  };

  // metric pair of rows ya, yb (natural staged rows, offsets from row -2) at column x
  auto load_S = [&](int ya, int yb, int x, f2 S[9], f2& Jn) {
    const int oa = (ya + 2) * RW + x + 2, ob = (yb + 2) * RW + x + 2;
#pragma unroll
    for (int f = 0; f < 9; ++f) S[f] = f2(met[f * PL + oa], met[f * PL + ob]);
    Jn = f2(met[9 * PL + oa], met[9 * PL + ob]);
  };

  auto node_pass = [&](int kk, f2 G3[5], f2& lt3, f2& nu3, f2& Jn) {
    const int sM = (kk + 7) & 3, sC = (kk + 8) & 3, sP = (kk + 9) & 3;
    if (role == 0) {
      f2 G[3][5], lt[3], nu[3], S[9];
      load_S(py, py + D, px, S, Jn);
      const PairAcc at{ring, (py + 2) * RW + px + 2};
      node_flux_pair<0>(at, sM, sC, sP, S, Jn, c, G, lt, nu);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Gi[(v * D + py) * (TI + 2) + px + 1] = G[0][v];
        Gj[(v * (D + 2) + py + 1) * TI + px] = G[1][v];
        G3[v] = G[2][v];
      }
      Li[(0 * D + py) * (TI + 2) + px + 1] = lt[0];
      Li[(1 * D + py) * (TI + 2) + px + 1] = nu[0];
      Lj[(0 * (D + 2) + py + 1) * TI + px] = lt[1];
      Lj[(1 * (D + 2) + py + 1) * TI + px] = nu[1];
      // rows D-1 and D also appear in pair rows -1 (as y) and D (as x)
      float* Gjf = reinterpret_cast<float*>(Gj);
      float* Ljf = reinterpret_cast<float*>(Lj);
      if (py == D - 1) {
#pragma unroll
        for (int v = 0; v < 5; ++v) Gjf[2 * ((v * (D + 2) + 0) * TI + px) + 1] = G[1][v].v.x;
        Ljf[2 * ((0 * (D + 2) + 0) * TI + px) + 1] = lt[1].v.x;
        Ljf[2 * ((1 * (D + 2) + 0) * TI + px) + 1] = nu[1].v.x;
      }
      if (py == 0) {
#pragma unroll
        for (int v = 0; v < 5; ++v) Gjf[2 * ((v * (D + 2) + D + 1) * TI + px)] = G[1][v].v.y;
        Ljf[2 * ((0 * (D + 2) + D + 1) * TI + px)] = lt[1].v.y;
        Ljf[2 * ((1 * (D + 2) + D + 1) * TI + px)] = nu[1].v.y;
      }
      lt3 = lt[2];
      nu3 = nu[2];
    } else if (role == 1) {
      f2 G[3][5], lt[3], nu[3], S[9], Jh;
      load_S(py, py + D, px, S, Jh);
      const PairAcc at{ring, (py + 2) * RW + px + 2};
      node_flux_pair<1>(at, sM, sC, sP, S, Jh, c, G, lt, nu);
      const int col = px + 1;
#pragma unroll
      for (int v = 0; v < 5; ++v) Gi[(v * D + py) * (TI + 2) + col] = G[0][v];
      Li[(0 * D + py) * (TI + 2) + col] = lt[0];
      Li[(1 * D + py) * (TI + 2) + col] = nu[0];
    } else {
      // rows -1 (pair row -1, x half) and TJ (pair row D, y half)
      f2 G[3][5], lt[3], nu[3], S[9], Jh;
      load_S(-1, TJ, px, S, Jh);
      const SplitAcc at{reinterpret_cast<const float*>(ring), (-1 + 2) * RW + px + 2, (D + 2) * RW + px + 2};
      node_flux_pair<2>(at, sM, sC, sP, S, Jh, c, G, lt, nu);
      float* Gjf = reinterpret_cast<float*>(Gj);
      float* Ljf = reinterpret_cast<float*>(Lj);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Gjf[2 * ((v * (D + 2) + 0) * TI + px)] = G[1][v].v.x;
        Gjf[2 * ((v * (D + 2) + D + 1) * TI + px) + 1] = G[1][v].v.y;
      }
      Ljf[2 * ((0 * (D + 2) + 0) * TI + px)] = lt[1].v.x;
      Ljf[2 * ((1 * (D + 2) + 0) * TI + px)] = nu[1].v.x;
      Ljf[2 * ((0 * (D + 2) + D + 1) * TI + px) + 1] = lt[1].v.y;
      Ljf[2 * ((1 * (D + 2) + D + 1) * TI + px) + 1] = nu[1].v.y;
    }
  };

  auto face_pass = [&](int kk, f2 Rij[5]) {
    const int s = (kk + 8) & 3;
    auto iface = [&](int x, int yp) {  // faces x - 1/2 of pair row yp
      f2 lam, e2, e4, Ga[5], Gb[5], h[5];
      face_coeffs2(c, Li[(0 * D + yp) * (TI + 2) + x], Li[(0 * D + yp) * (TI + 2) + x + 1],
                   Li[(1 * D + yp) * (TI + 2) + x], Li[(1 * D + yp) * (TI + 2) + x + 1], lam, e2, e4);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Ga[v] = Gi[(v * D + yp) * (TI + 2) + x];
        Gb[v] = Gi[(v * D + yp) * (TI + 2) + x + 1];
      }
      const int base = (yp + 2) * RW + x;  // pair-ring column of node x - 2
      const int so[4] = {s, s, s, s}, oo[4] = {base, base + 1, base + 2, base + 3};
      face5_pair(ring, so, oo, Ga, Gb, lam, e2, e4, h);
#pragma unroll
      for (int v = 0; v < 5; ++v) Hi[(v * D + yp) * (TI + 1) + x] = h[v];
    };
    auto jface = [&](int x, int yf) {  // faces (yf-1 | yf) and (yf+D-1 | yf+D) of column x
      f2 lam, e2, e4, Ga[5], Gb[5], h[5];
      face_coeffs2(c, Lj[(0 * (D + 2) + yf) * TI + x], Lj[(0 * (D + 2) + yf + 1) * TI + x],
                   Lj[(1 * (D + 2) + yf) * TI + x], Lj[(1 * (D + 2) + yf + 1) * TI + x], lam, e2, e4);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Ga[v] = Gj[(v * (D + 2) + yf) * TI + x];
        Gb[v] = Gj[(v * (D + 2) + yf + 1) * TI + x];
      }
      const int base = yf * RW + x + 2;  // pair row yf - 2
      const int so[4] = {s, s, s, s}, oo[4] = {base, base + RW, base + 2 * RW, base + 3 * RW};
      face5_pair(ring, so, oo, Ga, Gb, lam, e2, e4, h);
#pragma unroll
      for (int v = 0; v < 5; ++v) Hj[(v * (D + 1) + yf) * TI + x] = h[v];
    };
    if (role == 0) {
      iface(px, py);
      jface(px, py);
    } else {
      const int h = tid - PG::NTP;  // the last i-face of each pair row, the last j pair-face of each column
      if (h < D) iface(TI, h);
      else if (h < D + TI) jface(h - D, D);
    }
    __syncthreads();
    if (role == 0) {
#pragma unroll
      for (int v = 0; v < 5; ++v)
        Rij[v] = (Hi[(v * D + py) * (TI + 1) + px + 1] - Hi[(v * D + py) * (TI + 1) + px]) +
                 (Hj[(v * (D + 1) + py + 1) * TI + px] - Hj[(v * (D + 1) + py) * TI + px]);
    }
  };

  auto kface = [&](int ka, const f2 Ga[5], const f2 Gb[5], f2 lta, f2 ltb, f2 nua, f2 nub, f2 h[5]) {
    f2 lam, e2, e4;
    face_coeffs2(c, lta, ltb, nua, nub, lam, e2, e4);
    const int o = (py + 2) * RW + px + 2;
    const int so[4] = {(ka + 7) & 3, (ka + 8) & 3, (ka + 9) & 3, (ka + 10) & 3}, oo[4] = {o, o, o, o};
    face5_pair(ring, so, oo, Ga, Gb, lam, e2, e4, h);
  };

  const float adt = (float)(st.alpha * X.sc->dt);
  const long long npad = L.npad;
  float* const Qo = X.Q[st.qout];

  issue_raw(t0 - 2);
  issue_raw(t0 - 1);
  issue_met(t0 - 1);
  f2 G3m[5], lt3m = f2(0.f), nu3m = f2(0.f), Jm = f2(0.f);
  f2 G3c[5], lt3c = f2(0.f), nu3c = f2(0.f), Jc = f2(0.f);
  f2 Rc[5], hprev[5];
  if (!fetch_plane(t0 - 2, false, 0) || !fetch_plane(t0 - 1, false, 0) || !fetch_plane(t0, false, 0) ||
      !fetch_plane(t0 + 1, true, t0 - 1)) {
    failed = true;
  } else {
    node_pass(t0 - 1, G3m, lt3m, nu3m, Jm);
    __syncthreads();
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

  for (int t = t0; t < t1 && !failed; ++t) {
    float q0a[5], q0b[5];
    long long na = 0, nb = 0;
    if (own_a) {
      na = L.at(gi, gja, t);
#pragma unroll
      for (int v = 0; v < 5; ++v) q0a[v] = X.Q[0][v * npad + na];
    }
    if (own_b) {
      nb = L.at(gi, gjb, t);
#pragma unroll
      for (int v = 0; v < 5; ++v) q0b[v] = X.Q[0][v * npad + nb];
    }
    if (!fetch_plane(t + 2, true, t + 1)) { failed = true; break; }
    f2 G3n[5], lt3n = f2(0.f), nu3n = f2(0.f), Jn = f2(0.f);
    node_pass(t + 1, G3n, lt3n, nu3n, Jn);
    __syncthreads();
    if (t + 2 <= t1) issue_met(t + 2);
    f2 Rn[5];
    face_pass(t + 1, Rn);
    if (role == 0) {
      f2 hk[5];
      kface(t, G3c, G3n, lt3c, lt3n, nu3c, nu3n, hk);
      const f2 aJ = f2(adt) * Jc;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const f2 r = aJ * (Rc[v] + (hk[v] - hprev[v]));
        if (own_a) Qo[v * npad + na] = q0a[v] - r.v.x;
        if (own_b) Qo[v * npad + nb] = q0b[v] - r.v.y;
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

__global__ void __launch_bounds__(PG::NT, 1)
    k_stage_pair(const __grid_constant__ StageCtx<float, float> X, const StageSel st) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + PG::O_BAR);
  init_barriers(bar);
  uint32_t ph[3] = {0, 0, 0};
  int issued[3] = {0, 0, 0}, waited[3] = {0, 0, 0};
  bool failed = false;
  pair_item(X, st, blockIdx.x, blockIdx.y, blockIdx.z, smem, ph, issued, waited, failed);
  if (failed) drain_after_timeout(bar, X.err, issued, waited);
}

__global__ void __launch_bounds__(PG::NT, 1)
    k_stage_pair_batch(const StageCtx<float, float>* __restrict__ ctx, const int4* __restrict__ items, int nitems,
                       unsigned int* queue, const StageSel st) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + PG::O_BAR);
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
    pair_item(ctx[w.x], st, w.y, w.z, w.w, smem, ph, issued, waited, failed);
    if (failed) break;
  }
  if (failed) drain_after_timeout(bar, ctx[gsel].err, issued, waited);
}

}  // namespace

cudaError_t stage_pair_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_stage_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PG::BYTES);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_stage_pair_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PG::BYTES);
}

cudaError_t launch_stage_pair(const StageCtx<float, float>& X, const StageSel& st, cudaStream_t s) {
  const Layout& L = X.L;
  const int nz = L.hi[2] - L.lo[2] + 1;
  dim3 grid((L.hi[0] + PG::TI) / PG::TI, (L.hi[1] + PG::TJ) / PG::TJ, (nz + X.kc - 1) / X.kc);
  k_stage_pair<<<grid, PG::NT, PG::BYTES, s>>>(X, st);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_stage_pair_batch(const void* ctx, const int4* items, int nitems, unsigned int* queue,
                                    const StageSel& st, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  const int ctas = nitems < 152 ? nitems : 152;
  k_stage_pair_batch<<<ctas, PG::NT, PG::BYTES, s>>>((const StageCtx<float, float>*)ctx, items, nitems, queue, st);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace jz
